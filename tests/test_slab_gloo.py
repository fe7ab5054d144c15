"""Slab decomposition across ranks (two gloo ranks on CPU, no GPU): each rank owns the
particles of its x-slab, receives the ghosts within twice the support radius from its
neighbour through torch.distributed, computes one substep of its owned particles from owned
+ ghosts, and the grabbed body's wrench is the allreduce of the ranks' partial sums.  The
per-rank substep here is the FP64 oracle, so the test checks the decomposition and its data
movement: keys bit-equal, densities, accelerations and the wrench equal to one undivided
oracle substep of the whole scene (to FP64 summation order)."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2511_15908_gb300 import scenes, slab


def _scene():
    return scenes.with_velocity_noise(scenes.held_cube_tank(seed=3, n=(14, 10, 12), cube_cells=6),
                                      seed=3, sigma=0.3)


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(1)
    sc = _scene()
    R = 2.0 * float(np.float32(sc.params["h"]))
    tank_x = 14 * sc.fluid_spacing
    sl = slab.Slabs(0.0, tank_x, world, halo=2.0 * R)
    (ids, x, v), (gid, gx, gv) = slab.owned_and_ghosts(sc, sl, rank, world)
    own = np.zeros(sc.n_total, bool)
    own[ids] = True
    sub, sub_ids = slab.sub_scene(sc, np.concatenate([ids, gid]), np.concatenate([x, gx]), np.concatenate([v, gv]))
    res = oracle.System(sub, mode=1).substep()
    gids = sub_ids[res["id"]]                     # global id of each sorted slot
    mine = np.isin(gids, ids)
    # the wrench: this rank's owned body particles, pair force m a, torque about the grab point
    first = sc.n_fluid + sum(b.n for b in sc.bodies[:sc.grab_body])
    body = sc.bodies[sc.grab_body]
    in_body = mine & (gids >= first) & (gids < first + body.n)
    sysm = oracle.System(sub, mode=1)
    m_sorted = np.abs(sysm.m[res["src"]].astype(np.float64))
    f = m_sorted[in_body, None] * res["acc"][in_body]
    xg = sc.trajectory[0, :3].astype(np.float64)            # grab point: the centre (local 0)
    tau = np.cross(res["x_new"][in_body] - xg, f)
    w = np.zeros((1, 6))
    w[0, :3], w[0, 3:] = f.sum(0), tau.sum(0)
    w_all = slab.allreduce_wrench(w)
    out[rank] = dict(ids=gids[mine], key=res["key"][mine], rho=res["rho"][mine], acc=res["acc"][mine],
                     wrench=w_all[0], n_own=int(own.sum()), n_ghost=int(gid.size))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_equal_one_undivided_substep():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 31000 + os.getpid() % 2000
        ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    sc = _scene()
    ref = oracle.System(sc, mode=1).substep()
    rid = ref["id"]
    by_id = lambda k: dict(zip(rid, ref[k]))            # noqa: E731
    key, rho = by_id("key"), by_id("rho")
    acc = dict(zip(rid, ref["acc"]))
    seen = np.concatenate([res[r]["ids"] for r in range(2)])
    assert np.array_equal(np.sort(seen), np.arange(sc.n_total))     # every particle owned once
    for r in range(2):
        d = res[r]
        assert d["n_ghost"] > 0 and d["n_own"] > 0
        np.testing.assert_array_equal(d["key"], [key[i] for i in d["ids"]])
        rr = np.array([rho[i] for i in d["ids"]])
        assert np.max(np.abs(d["rho"] - rr) / rr) <= 1e-12
        aa = np.array([acc[i] for i in d["ids"]])
        scale = np.maximum(np.linalg.norm(aa, axis=1), 0.981)
        assert np.max(np.linalg.norm(d["acc"] - aa, axis=1) / scale) <= 1e-10
    wref = ref["wrench"][sc.grab_body]
    for r in range(2):
        np.testing.assert_allclose(res[r]["wrench"][:3], wref[:3], rtol=1e-9, atol=1e-12 * np.abs(wref[:3]).max())
        np.testing.assert_allclose(res[r]["wrench"][3:], wref[3:], rtol=1e-7,
                                   atol=1e-9 * np.abs(wref[3:]).max() + 1e-14)


def _rank_multi(rank, world, port, n_sub, out):
    """n_sub substeps with the oracle as the per-rank substep: ghosts exchanged before each,
    the owned fluid particles that left the slab handed over after each; the held cube's
    and the walls' particles are owned by position."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    oracle.set_threads(1)
    sc = _scene()
    s = sc.fluid_spacing
    R = 2.0 * float(np.float32(sc.params["h"]))
    # the middle edge on a column of particles (7.5 s), so that some cross it
    sl = slab.Slabs(0.0, 15 * s, world, halo=2.0 * R)
    nf = sc.n_fluid
    x0 = slab.particle_positions(sc)
    own = sl.owner(x0[:nf]) == rank
    ids_f = np.nonzero(own)[0]
    x_f, v_f = x0[:nf][own], slab.particle_velocities(sc)[:nf][own]
    first = nf + sum(b.n for b in sc.bodies[:sc.grab_body])
    nbody = sc.bodies[sc.grab_body].n
    wrenches, arrivals = [], 0
    for k in range(n_sub):
        xb = slab.particle_positions(sc, step=k)[nf:]
        ob = sl.owner(xb) == rank
        ids = np.concatenate([ids_f, nf + np.nonzero(ob)[0]])
        x = np.concatenate([x_f, xb[ob]])
        v = np.concatenate([v_f, np.zeros((int(ob.sum()), 3), np.float32)])
        left, right = sl.ghost_masks(x, rank)
        gx, gv, gid = slab.unpack(slab.neighbour_exchange(slab.pack(x, v, ids), left, right, rank, world))
        sub, sub_ids = slab.sub_scene(sc, np.concatenate([ids, gid]), np.concatenate([x, gx]),
                                      np.concatenate([v, gv]))
        sysm = oracle.System(sub, mode=1)
        sysm.step_index = k
        m_slot = np.abs(sysm.m.astype(np.float64))
        res = sysm.substep()
        gids = sub_ids[res["id"]]
        mine_f = np.isin(gids, ids_f)
        # the wrench: pair forces on this rank's particles of the held cube
        in_body = np.isin(gids, ids) & (gids >= first) & (gids < first + nbody)
        f = m_slot[res["src"]][in_body, None] * res["acc"][in_body]
        xg = sc.trajectory[min(k, sc.trajectory.shape[0] - 1), :3].astype(np.float64)
        w = np.zeros((1, 6))
        w[0, :3], w[0, 3:] = f.sum(0), np.cross(res["x_new"][in_body] - xg, f).sum(0)
        wrenches.append(slab.allreduce_wrench(w)[0])
        ids_f, x_f, v_f, n_in = slab.migrate(gids[mine_f], res["x_new"][mine_f].astype(np.float32),
                                             res["v_new"][mine_f].astype(np.float32), sl, rank, world)
        arrivals += n_in
    out[rank] = dict(ids=ids_f, x=x_f, v=v_f, wrench=np.array(wrenches), arrivals=arrivals)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_follow_one_undivided_run_with_handover():
    """Five substeps on two slabs, particles handed over between them, against five
    undivided oracle substeps: every fluid particle owned once at the end, its FP32
    position and velocity equal to the undivided run's (both FP64 substeps rounded to the
    FP32 state; they differ only in summation order), the allreduced wrench of every
    substep equal to the undivided one."""
    n_sub = 5
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 33000 + os.getpid() % 2000
        ps = [ctx.Process(target=_rank_multi, args=(r, 2, port, n_sub, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(600)
            assert p.exitcode == 0
        res = dict(out)
    sc = _scene()
    sysr = oracle.System(sc, mode=1)
    wref = []
    for _ in range(n_sub):
        r = sysr.substep()
        wref.append(r["wrench"][sc.grab_body])
    x_ref = np.empty((sc.n_total, 3), np.float32)
    v_ref = np.empty((sc.n_total, 3), np.float32)
    x_ref[sysr.id] = sysr.x
    v_ref[sysr.id] = sysr.v
    ids = np.concatenate([res[r]["ids"] for r in range(2)])
    assert np.array_equal(np.sort(ids), np.arange(sc.n_fluid))
    assert res[0]["arrivals"] + res[1]["arrivals"] > 0, "no particle changed slab"
    for r in range(2):
        d = res[r]
        dx = np.abs(d["x"].astype(np.float64) - x_ref[d["ids"]])
        dv = np.abs(d["v"].astype(np.float64) - v_ref[d["ids"]])
        assert dx.max() <= 1e-7, dx.max()
        assert dv.max() <= 1e-6 * max(1.0, float(np.abs(v_ref).max())), dv.max()
        wr = np.array(wref)
        np.testing.assert_allclose(d["wrench"][:, :3], wr[:, :3], rtol=1e-9, atol=1e-12 * np.abs(wr[:, :3]).max())
        np.testing.assert_allclose(d["wrench"][:, 3:], wr[:, 3:], rtol=1e-7, atol=1e-9 * np.abs(wr[:, 3:]).max() + 1e-14)


def test_slab_owner_and_ghost_masks():
    sl = slab.Slabs(0.0, 1.0, 4, halo=0.1)
    x = np.array([[-5.0, 0, 0], [0.1, 0, 0], [0.25, 0, 0], [0.3, 0, 0], [0.99, 0, 0], [7.0, 0, 0]])
    np.testing.assert_array_equal(sl.owner(x), [0, 0, 1, 1, 3, 3])
    left, right = sl.ghost_masks(x, 1)
    np.testing.assert_array_equal(left, x[:, 0] < 0.35)
    np.testing.assert_array_equal(right, x[:, 0] >= 0.4)
    left0, _ = sl.ghost_masks(x, 0)
    assert not left0.any()
    _, right3 = sl.ghost_masks(x, 3)
    assert not right3.any()


def test_migrate_refuses_a_particle_that_crossed_two_slabs():
    # the check runs before any message is exchanged
    sl = slab.Slabs(0.0, 3.0, 3, halo=0.1)
    ids = np.array([5, 6])
    x = np.array([[0.5, 0, 0], [2.5, 0, 0]], np.float32)      # the second is in rank 2's slab
    with pytest.raises(ValueError):
        slab.migrate(ids, x, np.zeros_like(x), sl, 0, 3)


def test_particle_positions_follow_the_grab_path():
    sc = _scene()
    first = sc.n_fluid + sum(b.n for b in sc.bodies[:sc.grab_body])
    n = sc.bodies[sc.grab_body].n
    traj = np.repeat(sc.trajectory[:1], 3, axis=0).copy()
    traj[2, 0] += 0.05                                       # the body moves 5 cm along x
    sc.trajectory = traj
    p0 = slab.particle_positions(sc, step=0)[first:first + n]
    p2 = slab.particle_positions(sc, step=2)[first:first + n]
    p9 = slab.particle_positions(sc, step=9)[first:first + n]  # past the path's end: its last row
    np.testing.assert_allclose(p2 - p0, np.tile([0.05, 0, 0], (n, 1)), atol=1e-6)
    np.testing.assert_array_equal(p9, p2)
