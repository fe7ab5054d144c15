"""Slab decomposition of one scene across ranks (one rank per GPU) -- a prototype.

The substep shards by spatial slabs along the tank's long axis x: rank r owns the particles
whose x lies in [e_r, e_{r+1}).  Before a substep each rank receives from its two
neighbours their owned particles within `halo` of its own slab (the ghosts); the per-rank
substep then computes the owned particles' densities and forces from owned + ghost
particles, and integrates only the owned ones; after it each body's coupling wrench, summed
by every rank over the body particles it owns, is summed over ranks (an allreduce of 6
doubles per body).  With a halo of twice the support radius the ghosts' own densities are
complete where the owned particles need them (every ghost within R of the slab has all of
its neighbours among owned + ghosts), so one exchange of positions and velocities per
substep replaces a second exchange of ghost densities before the force pass.  Particles
change owner when they cross a slab edge: after the substep every rank keeps the particles
now in its slab and hands the others to their new owner (the same neighbour exchange).

This module holds the decomposition and the data movement only; the exchanges go through
torch.distributed (gloo on CPU, NCCL between GPUs; no multicast, no library kernel on peer
memory).  The per-rank substep is the caller's.  Free rigid bodies would need each rank to
integrate the body from the allreduced wrench before the next substep; soft bodies whose
springs cross a slab edge are not handled.
"""
from __future__ import annotations

import numpy as np


class Slabs:
    """Equal slabs of [x_lo, x_hi) along x for `world` ranks; the outer slabs extend to
    infinity (particles outside the tank still have an owner)."""

    def __init__(self, x_lo: float, x_hi: float, world: int, halo: float):
        if world < 1 or not (x_hi > x_lo) or not (halo > 0.0):
            raise ValueError("bad slab decomposition")
        self.world = world
        self.halo = float(halo)
        self.edges = np.linspace(x_lo, x_hi, world + 1)
        self.edges[0], self.edges[-1] = -np.inf, np.inf

    def owner(self, x: np.ndarray) -> np.ndarray:
        """Owning rank of each particle (positions (n, 3))."""
        return np.searchsorted(self.edges[1:-1], np.asarray(x)[:, 0], side="right").astype(np.int64)

    def ghost_masks(self, x: np.ndarray, rank: int):
        """Of the particles rank owns, those within `halo` of the left and of the right
        neighbour's slab (the ghosts it sends them); (left, right) boolean masks, all False
        where the neighbour does not exist."""
        x0 = np.asarray(x)[:, 0]
        left = (x0 < self.edges[rank] + self.halo) if rank > 0 else np.zeros(x0.shape, bool)
        right = (x0 >= self.edges[rank + 1] - self.halo) if rank < self.world - 1 else np.zeros(x0.shape, bool)
        return left, right


def _swap(rows, rank: int, peer: int):
    """Send `rows` (a float64 tensor (n, k)) to `peer` and receive its rows (blocking; the
    lower rank sends first so the pair cannot deadlock)."""
    import torch
    import torch.distributed as dist
    k = rows.shape[1]
    n_out = torch.tensor([rows.shape[0]], dtype=torch.int64)
    n_in = torch.zeros(1, dtype=torch.int64)
    if rank < peer:
        dist.send(n_out, peer)
        dist.recv(n_in, peer)
    else:
        dist.recv(n_in, peer)
        dist.send(n_out, peer)
    got = torch.zeros((int(n_in.item()), k), dtype=torch.float64)
    if rank < peer:
        if rows.shape[0]:
            dist.send(rows.contiguous(), peer)
        if got.shape[0]:
            dist.recv(got, peer)
    else:
        if got.shape[0]:
            dist.recv(got, peer)
        if rows.shape[0]:
            dist.send(rows.contiguous(), peer)
    return got


def neighbour_exchange(rows: np.ndarray, to_left: np.ndarray, to_right: np.ndarray, rank: int,
                       world: int) -> np.ndarray:
    """Rows (float64 (n, k)) selected by the masks go to the left / right neighbour; returns
    the rows received from both neighbours (left's first)."""
    import torch
    parts = []
    rows_t = torch.from_numpy(np.ascontiguousarray(rows, np.float64))
    # pair (r, r+1) exchanges first for even r, then for odd r: no rank waits on a cycle
    for phase in (0, 1):
        for peer, mask in ((rank - 1, to_left), (rank + 1, to_right)):
            if peer < 0 or peer >= world or (min(rank, peer) % 2) != phase:
                continue
            got = _swap(rows_t[torch.from_numpy(np.asarray(mask))], rank, peer)
            parts.append((peer, got.numpy()))
    parts.sort(key=lambda p: p[0])
    k = rows.shape[1]
    return np.concatenate([p[1] for p in parts]) if parts else np.zeros((0, k))


def pack(x: np.ndarray, v: np.ndarray, ids: np.ndarray) -> np.ndarray:
    """(x, v, id) rows as float64 (FP32 values and int32 ids are exact in FP64)."""
    return np.concatenate([np.asarray(x, np.float64), np.asarray(v, np.float64),
                           np.asarray(ids, np.float64)[:, None]], 1)


def unpack(rows: np.ndarray):
    return (rows[:, 0:3].astype(np.float32), rows[:, 3:6].astype(np.float32),
            rows[:, 6].astype(np.int64))


def allreduce_wrench(w: np.ndarray) -> np.ndarray:
    """Sum of the per-rank wrenches (bodies x 6, FP64) over all ranks."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(np.ascontiguousarray(w, np.float64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.numpy()


def migrate(ids: np.ndarray, x: np.ndarray, v: np.ndarray, slabs: "Slabs", rank: int, world: int):
    """Owner hand-over after a substep: of this rank's particles (global ids, FP32 positions
    and velocities after the substep), those whose position now lies in a neighbour's slab
    go to that neighbour (one exchange); returns this rank's particles: the ones that stayed,
    then the arrivals, and the number of arrivals."""
    own = slabs.owner(x)
    if np.any(np.abs(own - rank) > 1):
        raise ValueError("a particle crossed more than one slab in one substep")
    stay = own == rank
    gx, gv, gid = unpack(neighbour_exchange(pack(x, v, ids), own == rank - 1, own == rank + 1, rank, world))
    return (np.concatenate([np.asarray(ids)[stay], gid]), np.concatenate([np.asarray(x, np.float32)[stay], gx]),
            np.concatenate([np.asarray(v, np.float32)[stay], gv]), int(gid.size))


def particle_positions(scene, step: int = 0) -> np.ndarray:
    """Positions (id order) used to assign owners: fluid and static / soft particles as
    given, rigid particles placed from the body's pose at substep `step` (the grab path's
    row for a grabbed body, clamped to its last; FP64, then FP32; the substep itself
    places them again)."""
    xs = [np.asarray(scene.fluid_x, np.float32)]
    for bi, b in enumerate(scene.bodies):
        if b.kind == 2:                               # rigid
            row = None
            if bi == scene.grab_body and scene.trajectory is not None:
                row = scene.trajectory[min(step, scene.trajectory.shape[0] - 1), :7]
            pose = (row if row is not None else b.pose).astype(np.float64)
            w, x, y, z = pose[3:7] / np.linalg.norm(pose[3:7])
            R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                          [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                          [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
            xs.append((np.asarray(b.xyz, np.float64) @ R.T + pose[:3]).astype(np.float32))
        else:
            xs.append(np.asarray(b.xyz, np.float32))
    return np.concatenate(xs)


def particle_velocities(scene) -> np.ndarray:
    v = np.zeros((scene.n_total, 3), np.float32)
    v[:scene.n_fluid] = scene.fluid_v
    return v


def sub_scene(scene, ids: np.ndarray, x: np.ndarray, v: np.ndarray):
    """The scene restricted to the particles `ids` (global ids; x, v their rows): fluid
    particles as fluid, each body's particles as that body (rigid: their body-frame
    offsets with the body's pose); returns (scene, sub_ids) with sub_ids[k] the global id
    of the sub-scene's particle k."""
    from . import scenes as _sc
    nf = scene.n_fluid
    fl = ids < nf
    bodies, first, grab = [], nf, -1
    for bi, b in enumerate(scene.bodies):
        if b.springs is not None and len(b.springs):
            raise NotImplementedError("soft-body springs across slabs are not handled")
        sel = (ids >= first) & (ids < first + b.n)
        local = ids[sel] - first
        first += b.n
        if not sel.any():
            continue
        order = np.argsort(local)
        nb = _sc.Body(b.kind, np.asarray(b.xyz, np.float32)[local[order]], b.spacing, mass=b.mass,
                      inertia=b.inertia, pose=b.pose, vel=b.vel, grab_local=b.grab_local)
        if bi == scene.grab_body:
            grab = len(bodies)
        bodies.append((nb, ids[sel][order]))
    fo = np.argsort(ids[fl])
    sub = _sc.Scene("slab", scene.params, np.ascontiguousarray(x[fl][fo]), np.ascontiguousarray(v[fl][fo]),
                    scene.fluid_spacing, [b for b, _ in bodies], grab_body=grab, trajectory=scene.trajectory,
                    n_substeps=scene.n_substeps)
    sub_ids = np.concatenate([ids[fl][fo]] + [g for _, g in bodies]).astype(np.int64)
    return sub, sub_ids


def owned_and_ghosts(scene, slabs: "Slabs", rank: int, world: int):
    """This rank's owned particles and the ghosts its neighbours send it (one exchange):
    (owned ids, x, v), (ghost ids, x, v)."""
    x_all, v_all = particle_positions(scene), particle_velocities(scene)
    own = slabs.owner(x_all) == rank
    ids = np.nonzero(own)[0]
    x, v = x_all[own], v_all[own]
    left, right = slabs.ghost_masks(x, rank)
    gx, gv, gid = unpack(neighbour_exchange(pack(x, v, ids), left, right, rank, world))
    return (ids, x, v), (gid, gx, gv)
