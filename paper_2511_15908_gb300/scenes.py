"""Seeded synthetic scenes for the SPH coupling substep.

This module only lays out inputs: fluid lattices with jitter, static wall shells,
lattice-sampled rigid and soft bodies, and the grabbed body's prescribed path.  It
holds none of the method's arithmetic (no kernel, density, force, hashing or
integration), so both the CUDA path and the CPU oracle can consume its arrays.

Scene recipes (all lengths in metres, z is up, gravity -9.81 along z):

* ``dam_break``      16^3 fluid block at spacing 0.02 in the corner of a 0.5 m box
                     with a two-layer static wall shell (open top) and one free
                     0.1 m rigid cube of density 500 sampled at half spacing.
* ``stirring_tank``  125 x 125 x 16 fluid at spacing 0.008 in a 1 x 1 x 0.5 m tank,
                     a 0.02 x 0.2 x 0.3 m paddle sampled at 0.004, grabbed and driven
                     on a horizontal circle (radius 0.2 m, 1 Hz, seeded phase).
* ``coupled``        1,000,000 fluid at spacing 0.01 in a 2 x 1 x 0.6 m tank, a solid
                     sphere probe (r 0.0964 m at 0.005, about 30k particles) on a
                     seeded random-walk grab path, and a 24^3 soft cube at 0.01.
* ``batched``        64 stirring scenes with fluid counts log-uniform in [8k, 256k].

Smoothing length h equals the fluid spacing, so the kernel support 2h is twice the
spacing; the pressure constant is k = c^2 with c = 0.4 h / dt (an acoustic CFL of 0.4);
kinematic viscosity 1e-3 m^2/s.  The grid cell edge is h enlarged by 0.1 % (half the
support radius): the neighbour search clips each row of cells to the support sphere, and
cells near h leave the fewest candidates to test (any cell >= h is valid).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

KIND_STATIC = 1
KIND_RIGID = 2
KIND_SOFT = 3

FLAG_CLAMP_PRESSURE = 1 << 0   # negative pressures are clamped to zero
FLAG_RECORD = 1 << 1           # keep per-particle acceleration and neighbour counts
FLAG_TAIT = 1 << 3             # Tait equation of state instead of the linear one
FLAG_VOLUME_BOUNDARY = 1 << 4  # boundary particles weighted by volume (psi) instead of mass


@dataclass
class Body:
    kind: int
    xyz: np.ndarray                 # static: world positions; rigid: body-frame offsets
                                    # about the centre of mass; soft: world positions
    spacing: float                  # sampling spacing (SPH mass = rho0 * spacing^3)
    mass: float = 0.0               # inertial mass of a rigid body
    inertia: np.ndarray = field(default_factory=lambda: np.zeros((3, 3), np.float32))
    pose: np.ndarray = field(default_factory=lambda: np.array([0, 0, 0, 1, 0, 0, 0], np.float32))
    vel: np.ndarray = field(default_factory=lambda: np.zeros(6, np.float32))
    springs: Optional[np.ndarray] = None   # (ns, 2) local index pairs (soft)
    young: float = 0.0
    poisson: float = 0.0
    grab_local: np.ndarray = field(default_factory=lambda: np.zeros(3, np.float32))
    anchors: Optional[np.ndarray] = None   # soft: local indices of pinned particles

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


@dataclass
class Scene:
    name: str
    params: dict
    fluid_x: np.ndarray             # (nf, 3) float32
    fluid_v: np.ndarray             # (nf, 3) float32
    fluid_spacing: float
    bodies: List[Body]
    grab_body: int = -1             # index into bodies, -1 = nothing grabbed
    trajectory: Optional[np.ndarray] = None   # (T, 13) float32 x,q(wxyz),v,w per substep
    n_substeps: int = 100

    @property
    def n_fluid(self) -> int:
        return int(self.fluid_x.shape[0])

    @property
    def n_total(self) -> int:
        return self.n_fluid + sum(b.n for b in self.bodies)


def make_params(spacing, dt, lo, hi, *, rho0=1000.0, nu=1e-3, flags=FLAG_CLAMP_PRESSURE,
                cfl=0.4, smooth_window=20, cell_over_h=1.001):
    h = float(spacing)
    c = cfl * h / dt
    return dict(h=h, rho0=float(rho0), k=float(c * c), nu=float(nu),
                g=(0.0, 0.0, -9.81), dt=float(dt),
                lo=tuple(float(a) for a in lo), hi=tuple(float(a) for a in hi),
                cell=float(np.float32(cell_over_h * h)), flags=int(flags),
                visc_eps=0.01, spring_zeta=0.1, smooth_window=int(smooth_window))


def _lattice(n, spacing, origin):
    """Cell-centred lattice points origin + (i + 0.5) * spacing, i < n per axis, x fastest."""
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([i, j, k], axis=-1).reshape(-1, 3).astype(np.float64)
    return (pts + 0.5) * spacing + np.asarray(origin, np.float64)


def _jitter(rng, pts, spacing, frac=0.01):
    return pts + rng.uniform(-frac * spacing, frac * spacing, size=pts.shape)


def wall_shell(box_lo, box_hi, spacing, layers=2):
    """Static walls: `layers` lattice layers outside the box on the sides and bottom (open top)."""
    box_lo = np.asarray(box_lo, np.float64)
    box_hi = np.asarray(box_hi, np.float64)
    n = np.rint((box_hi - box_lo) / spacing).astype(int)
    ii = np.arange(-layers, n[0] + layers)
    jj = np.arange(-layers, n[1] + layers)
    kk = np.arange(-layers, n[2])
    K, J, I = np.meshgrid(kk, jj, ii, indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    outside = (I < 0) | (I >= n[0]) | (J < 0) | (J >= n[1]) | (K < 0)
    pts = np.stack([I[outside], J[outside], K[outside]], -1).astype(np.float64)
    return ((pts + 0.5) * spacing + box_lo).astype(np.float32)


def solid_box(size, spacing):
    """Body-frame lattice of a solid box centred on the origin."""
    n = np.maximum(np.rint(np.asarray(size) / spacing).astype(int), 1)
    return (_lattice(n, spacing, -0.5 * n * spacing)).astype(np.float32), n


def solid_sphere(radius, spacing):
    m = int(np.ceil(radius / spacing)) + 1
    pts = _lattice((2 * m, 2 * m, 2 * m), spacing, (-m * spacing,) * 3)
    keep = np.sum(pts * pts, axis=1) <= radius * radius
    return pts[keep].astype(np.float32)


def lattice_springs(n):
    """18-neighbour lattice springs (6 axis + 12 face diagonals) of an n[0] x n[1] x n[2] block."""
    nx, ny, nz = n
    idx = np.arange(nx * ny * nz).reshape(nz, ny, nx)
    offs = [(1, 0, 0), (0, 1, 0), (0, 0, 1),
            (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]
    pairs = []
    for dx, dy, dz in offs:
        z0, z1 = max(0, -dz), nz - max(0, dz)
        y0, y1 = max(0, -dy), ny - max(0, dy)
        x0, x1 = max(0, -dx), nx - max(0, dx)
        a = idx[z0:z1, y0:y1, x0:x1]
        b = idx[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
        pairs.append(np.stack([a.ravel(), b.ravel()], -1))
    return np.concatenate(pairs).astype(np.int32)


def _box_inertia(mass, size):
    a, b, c = size
    return (mass / 12.0) * np.diag([b * b + c * c, a * a + c * c, a * a + b * b]).astype(np.float32)


def _settle_columns(pts, spacing, top, g_over_k):
    """Move lattice layers down so that the layer spacing at depth d below the surface is
    spacing / (1 + g d / k): the density a linear equation of state p = k (rho - rho0) needs
    to carry the fluid's weight, p = rho0 g d.  Mass per unit height of the uncompressed
    column is rho0, of the settled one rho0 (1 + g d / k), so an uncompressed depth zeta
    maps to d with zeta = d + g d^2 / (2 k); the floor stays where it is."""
    def depth(zeta):
        return (np.sqrt(1.0 + 2.0 * g_over_k * zeta) - 1.0) / g_over_k
    out = pts.copy()
    z0 = out[:, 2].min() - 0.5 * spacing
    zeta = np.maximum(top - out[:, 2], 0.0)
    out[:, 2] = z0 + depth(top - z0) - depth(zeta)
    return out


def _fill_fluid(rng, cols, spacing, origin, count, carve, g_over_k=None):
    """Fill columns bottom-up with a lattice, skip points that `carve` rejects, keep `count`.
    With g_over_k (= |g| / k) the lattice starts settled under its own weight (see
    _settle_columns) instead of at uniform rest density, which would first collapse."""
    nx, ny = cols
    nz = int(np.ceil(count / (nx * ny))) + 8
    pts = _lattice((nx, ny, nz), spacing, origin)
    if g_over_k is not None:
        # the surface of the uncompressed fill of `count` points, then settle and carve
        kept = pts[~carve(pts)] if carve is not None else pts
        top = kept[:count, 2].max() + 0.5 * spacing
        pts = _settle_columns(pts, spacing, top, g_over_k)
    if carve is not None:
        pts = pts[~carve(pts)]
    if pts.shape[0] < count:
        raise ValueError("fluid lattice too small for the requested count")
    pts = pts[:count]
    return _jitter(rng, pts, spacing).astype(np.float32)


def circle_trajectory(rng, n_sub, dt, centre, radius=0.2, freq=1.0, z=0.0):
    phase = rng.uniform(0.0, 2.0 * np.pi)
    t = np.arange(n_sub) * dt
    ang = 2.0 * np.pi * freq * t + phase
    traj = np.zeros((n_sub, 13), np.float64)
    traj[:, 0] = centre[0] + radius * np.cos(ang)
    traj[:, 1] = centre[1] + radius * np.sin(ang)
    traj[:, 2] = z
    traj[:, 3] = 1.0
    w = 2.0 * np.pi * freq
    traj[:, 7] = -radius * w * np.sin(ang)
    traj[:, 8] = radius * w * np.cos(ang)
    return traj.astype(np.float32)


def random_walk_trajectory(rng, n_sub, dt, start, lo, hi, sigma=0.05, vmax=0.5):
    """Velocity random walk v += N(0, sigma^2) per substep, |v| <= vmax, reflected at lo/hi."""
    traj = np.zeros((n_sub, 13), np.float64)
    x = np.asarray(start, np.float64).copy()
    v = np.zeros(3)
    for s in range(n_sub):
        traj[s, 0:3] = x
        traj[s, 3] = 1.0
        traj[s, 7:10] = v
        v = v + rng.normal(0.0, sigma, 3)
        sp = np.linalg.norm(v)
        if sp > vmax:
            v *= vmax / sp
        x = x + v * dt
        for a in range(3):
            if x[a] < lo[a]:
                x[a] = 2 * lo[a] - x[a]
                v[a] = -v[a]
            if x[a] > hi[a]:
                x[a] = 2 * hi[a] - x[a]
                v[a] = -v[a]
    return traj.astype(np.float32)


def episode_trajectory(n_episodes, per_episode, dt, start, lo, hi, seed0=0, sigma=0.02, vmax=0.4):
    """A grab path of n_episodes seeded random-walk episodes of per_episode substeps (seeds
    seed0, seed0 + 1, ...), each starting at rest where the previous one ended."""
    parts, x = [], np.asarray(start, np.float64)
    for e in range(n_episodes):
        seg = random_walk_trajectory(np.random.default_rng(seed0 + e), per_episode, dt, x, lo, hi,
                                     sigma=sigma, vmax=vmax)
        parts.append(seg)
        x = seg[-1, 0:3].astype(np.float64)
    return np.concatenate(parts)


def dam_break(seed=0, n_side=16, n_substeps=100, grab=False, cube_pos=(0.4, 0.25, 0.12)):
    """3D dam break: n_side^3 fluid at 0.02 m, 0.5 m static box, one free 0.1 m cube (density 500)."""
    rng = np.random.default_rng(seed)
    s = 0.02
    box = 0.5
    dt = 1e-3
    fluid = _jitter(rng, _lattice((n_side,) * 3, s, (0.0, 0.0, 0.0)), s).astype(np.float32)
    walls = Body(KIND_STATIC, wall_shell((0, 0, 0), (box, box, box), s), s)
    cube_local, _ = solid_box((0.1, 0.1, 0.1), s / 2)
    cube_mass = 500.0 * 0.1 ** 3
    cube = Body(KIND_RIGID, cube_local, s / 2, mass=cube_mass,
                inertia=_box_inertia(cube_mass, (0.1, 0.1, 0.1)),
                pose=np.array([*cube_pos, 1, 0, 0, 0], np.float32))
    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s), (box + 3 * s, box + 3 * s, 1.5 * box))
    sc = Scene("dam_break", params, fluid, np.zeros_like(fluid), s, [walls, cube],
               n_substeps=n_substeps)
    if grab:
        sc.grab_body = 1
        sc.trajectory = random_walk_trajectory(rng, n_substeps, dt, cube_pos,
                                               (0.08, 0.08, 0.08), (0.42, 0.42, 0.35),
                                               sigma=0.02, vmax=0.4)
    return sc


def stirring_tank(seed=0, n_fluid=250_000, cols=(125, 125), tank=(1.0, 1.0, 0.5),
                  n_substeps=2000, spacing=0.008, paddle=(0.02, 0.2, 0.3)):
    """Stirring tank: fluid at 0.008 m, grabbed paddle on a 0.2 m / 1 Hz circle."""
    rng = np.random.default_rng(seed)
    s = spacing
    dt = 5e-4
    tx, ty, tz = tank
    centre = np.array([tx / 2, ty / 2])
    p_local, _ = solid_box(paddle, s / 2)
    pz = 0.02 + paddle[2] / 2
    radius = min(0.2, 0.5 * min(tx, ty) - paddle[1])
    traj = circle_trajectory(rng, n_substeps, dt, centre, radius=radius, z=pz)
    p0 = traj[0, :3].astype(np.float64)
    half = np.asarray(paddle) / 2 + 0.5 * s

    def carve(pts):
        return np.all(np.abs(pts - p0) <= half, axis=1)

    fluid = _fill_fluid(rng, cols, s, (0.0, 0.0, 0.0), n_fluid, carve)
    walls = Body(KIND_STATIC, wall_shell((0, 0, 0), tank, s), s)
    pmass = 500.0 * float(np.prod(paddle))
    pad = Body(KIND_RIGID, p_local, s / 2, mass=pmass, inertia=_box_inertia(pmass, paddle),
               pose=traj[0, :7].copy(), vel=traj[0, 7:].copy())
    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s), (tx + 3 * s, ty + 3 * s, 1.2 * tz))
    return Scene("stirring_tank", params, fluid, np.zeros_like(fluid), s, [walls, pad],
                 grab_body=1, trajectory=traj, n_substeps=n_substeps)


def coupled(seed=0, n_fluid=1_000_000, cols=(200, 100), tank=(2.0, 1.0, 0.6), n_substeps=1000,
            spacing=0.01, probe_r=0.0964, soft_n=24, young=5e4, poisson=0.45, settled=True,
            wall_layers=2):
    """Coupled scene: fluid at 0.01 m, random-walk sphere probe, free soft cube.  The fluid
    starts settled under its own weight (layers closer near the floor); started at uniform
    rest density, the 0.5 m column first collapses and the pressure overshoot pushes corner
    particles through the two wall layers within ~250 substeps."""
    rng = np.random.default_rng(seed)
    s = spacing
    dt = 5e-4
    tx, ty, tz = tank
    depth = n_fluid / (cols[0] * cols[1]) * s
    probe_c = np.array([0.3 * tx, 0.5 * ty, 0.5 * depth])
    probe_local = solid_sphere(probe_r, s / 2)
    soft_local, soft_dims = solid_box((soft_n * s,) * 3, s)
    soft_c = np.array([0.7 * tx, 0.5 * ty, depth - 0.5 * soft_n * s + 0.25 * soft_n * s])
    soft_xyz = (soft_local.astype(np.float64) + soft_c).astype(np.float32)
    soft_half = 0.5 * soft_n * s + 0.5 * s

    def carve(pts):
        in_probe = np.sum((pts - probe_c) ** 2, axis=1) <= (probe_r + 0.5 * s) ** 2
        in_soft = np.all(np.abs(pts - soft_c) <= soft_half, axis=1)
        return in_probe | in_soft

    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s), (tx + 3 * s, ty + 3 * s, 1.4 * tz))
    g_over_k = 9.81 / params["k"] if settled else None
    fluid = _fill_fluid(rng, cols, s, (0.0, 0.0, 0.0), n_fluid, carve, g_over_k)
    walls = Body(KIND_STATIC, wall_shell((0, 0, 0), tank, s, layers=wall_layers), s)
    pmass = 1000.0 * probe_local.shape[0] * (s / 2) ** 3
    inertia = np.eye(3, dtype=np.float32) * np.float32(0.4 * pmass * probe_r ** 2)
    m = probe_r + 0.02
    traj = random_walk_trajectory(rng, n_substeps, dt, probe_c, (m, m, m),
                                  (tx - m, ty - m, tz - m))
    probe = Body(KIND_RIGID, probe_local, s / 2, mass=pmass, inertia=inertia,
                 pose=traj[0, :7].copy(), vel=traj[0, 7:].copy())
    soft = Body(KIND_SOFT, soft_xyz, s, springs=lattice_springs(soft_dims), young=young,
                poisson=poisson)
    return Scene("coupled", params, fluid, np.zeros_like(fluid), s, [walls, probe, soft],
                 grab_body=1, trajectory=traj, n_substeps=n_substeps)


def batched_counts(seed=0, n_scenes=64, lo=8_000, hi=256_000):
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n_scenes)).astype(np.int64)


def batched(seed=0, n_scenes=64, n_substeps=200, lo=8_000, hi=256_000, compact=False,
            cell_over_h=1.001):
    """Independent stirring scenes with log-uniform fluid counts (depth 16 layers at 0.008 m).
    compact: small tanks for small counts (side from 12 columns, 0.2 m walls, a 0.15 m
    paddle) instead of at least 40 columns and 0.5 m walls, so that walls do not dwarf the
    fluid of a scene of a few thousand particles.  cell_over_h: the grid's cell edge."""
    counts = batched_counts(seed, n_scenes, lo, hi)
    scenes = []
    for i, c in enumerate(counts):
        side = int(np.ceil(np.sqrt(c / 16.0)))
        side = max(side, 12 if compact else 40)
        tank = (side * 0.008, side * 0.008, 0.2 if compact else 0.5)
        paddle = (0.02, min(0.2, 0.25 * side * 0.008), 0.15 if compact else 0.3)
        sc = stirring_tank(seed=1000 + i, n_fluid=int(c), cols=(side, side), tank=tank,
                           n_substeps=n_substeps, paddle=paddle)
        sc.params["cell"] = float(np.float32(cell_over_h * sc.params["h"]))
        scenes.append(sc)
    return scenes


def tiny(seed=0, n=(4, 4, 4), spacing=0.02, dt=1e-3, with_bodies=True):
    """A few hundred particles: fluid block, small wall patch, one rigid and one soft body."""
    rng = np.random.default_rng(seed)
    s = spacing
    fluid = _jitter(rng, _lattice(n, s, (0.0, 0.0, 0.0)), s).astype(np.float32)
    v = rng.uniform(-0.1, 0.1, fluid.shape).astype(np.float32)
    bodies = []
    if with_bodies:
        floor = _lattice((n[0] + 2, n[1] + 2, 1), s, (-s, -s, -1.2 * s)).astype(np.float32)
        bodies.append(Body(KIND_STATIC, floor, s))
        loc, _ = solid_box((2 * s, 2 * s, 2 * s), s / 2)
        bodies.append(Body(KIND_RIGID, loc, s / 2, mass=0.004,
                           inertia=_box_inertia(0.004, (2 * s,) * 3),
                           pose=np.array([n[0] * s + 0.6 * s, 0.5 * n[1] * s, 1.1 * s,
                                          0.9659258, 0.0, 0.258819, 0.0], np.float32),
                           vel=np.array([-0.05, 0.02, 0.0, 0.3, -0.2, 0.5], np.float32)))
        sl, sd = solid_box((2 * s, 2 * s, 2 * s), s)
        sxyz = (sl.astype(np.float64) + np.array([0.5 * n[0] * s, n[1] * s + 0.9 * s,
                                                   0.8 * s])).astype(np.float32)
        sxyz = _jitter(rng, sxyz, s, 0.05).astype(np.float32)
        bodies.append(Body(KIND_SOFT, sxyz, s, springs=lattice_springs(sd), young=5e3,
                           poisson=0.45))
    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s),
                         ((n[0] + 4) * s, (n[1] + 4) * s, (n[2] + 4) * s))
    return Scene("tiny", params, fluid, v, s, bodies, grab_body=-1, n_substeps=10)


def cloth_springs(nx, ny):
    """Springs of an nx x ny sheet (local index j * nx + i): structural (to the next
    particle along x and along y), shear (both diagonals of each square) and bending
    (to the particle two steps away along x and along y)."""
    idx = np.arange(nx * ny).reshape(ny, nx)
    pairs = [np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], 1),
             np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], 1),
             np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()], 1),
             np.stack([idx[:-1, 1:].ravel(), idx[1:, :-1].ravel()], 1),
             np.stack([idx[:, :-2].ravel(), idx[:, 2:].ravel()], 1),
             np.stack([idx[:-2, :].ravel(), idx[2:, :].ravel()], 1)]
    return np.concatenate(pairs).astype(np.int32)


def cloth_plane(nx, ny, spacing, origin, young=5e4, anchors="corners"):
    """A horizontal soft cloth of nx x ny particles at `spacing` from `origin` (x, y, z),
    with anchor particles at its four corners, along its two x-edges or none."""
    i, j = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    xyz = np.stack([origin[0] + i.ravel() * spacing, origin[1] + j.ravel() * spacing,
                    np.full(nx * ny, float(origin[2]))], 1).astype(np.float32)
    if anchors == "corners":
        anc = np.array([0, nx - 1, (ny - 1) * nx, ny * nx - 1], np.int32)
    elif anchors == "edges":
        anc = np.concatenate([np.arange(nx), (ny - 1) * nx + np.arange(nx)]).astype(np.int32)
    else:
        anc = None
    return Body(KIND_SOFT, xyz, spacing, springs=cloth_springs(nx, ny), young=young,
                poisson=0.3, anchors=anc)


def cloth_bath(seed=0, n=(12, 12, 6), cloth=(16, 16), spacing=0.02, dt=5e-4, anchors="corners"):
    """A fluid block with a cloth plane stretched just above it (anchored), a floor below."""
    rng = np.random.default_rng(seed)
    s = spacing
    fluid = _jitter(rng, _lattice(n, s, (0.0, 0.0, 0.0)), s).astype(np.float32)
    floor = _lattice((n[0] + 4, n[1] + 4, 1), s, (-2 * s, -2 * s, -1.2 * s)).astype(np.float32)
    off = ((n[0] - cloth[0]) * s / 2, (n[1] - cloth[1]) * s / 2, (n[2] + 0.6) * s)
    sheet = cloth_plane(cloth[0], cloth[1], s, off, anchors=anchors)
    bodies = [Body(KIND_STATIC, floor, s), sheet]
    params = make_params(s, dt, (-4 * s, -4 * s, -3 * s),
                         ((n[0] + 4) * s, (n[1] + 4) * s, (n[2] + 6) * s))
    return Scene("cloth_bath", params, fluid, np.zeros_like(fluid), s, bodies, grab_body=-1,
                 n_substeps=10)


def column(seed=0, n=(6, 6, 20), spacing=0.02, dt=1e-3):
    """Hydrostatic column: fluid in a closed-bottom shaft of static walls."""
    rng = np.random.default_rng(seed)
    s = spacing
    fluid = _jitter(rng, _lattice(n, s, (0.0, 0.0, 0.0)), s).astype(np.float32)
    box_hi = (n[0] * s, n[1] * s, (n[2] + 4) * s)
    walls = Body(KIND_STATIC, wall_shell((0, 0, 0), box_hi, s), s)
    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s),
                         (box_hi[0] + 3 * s, box_hi[1] + 3 * s, box_hi[2] + 3 * s))
    return Scene("column", params, fluid, np.zeros_like(fluid), s, [walls], n_substeps=2000)


def held_cube_tank(seed=0, n=(14, 14, 18), cube_cells=6, spacing=0.02, dt=1e-3, nu=5e-3):
    """A tank of fluid at rest with a cube held still at mid-depth (a grabbed body whose path
    is one fixed pose).  The cube fills `cube_cells`^3 lattice cells carved out of the
    fluid, sampled at half the fluid spacing; its faces lie on lattice cell faces."""
    rng = np.random.default_rng(seed)
    s = spacing
    c = int(cube_cells)
    lo_c = np.array([(n[0] - c) // 2, (n[1] - c) // 2, (n[2] - c) // 2])
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    ijk = np.stack([i, j, k], -1).reshape(-1, 3)
    inside = np.all((ijk >= lo_c) & (ijk < lo_c + c), axis=1)
    fluid = _jitter(rng, (ijk[~inside] + 0.5) * s, s).astype(np.float32)
    box_hi = (n[0] * s, n[1] * s, (n[2] + 4) * s)
    walls = Body(KIND_STATIC, wall_shell((0, 0, 0), box_hi, s), s)
    a = c * s
    cube_local, _ = solid_box((a, a, a), s / 2)
    centre = (lo_c + 0.5 * c) * s
    pose = np.array([*centre, 1, 0, 0, 0], np.float32)
    cube = Body(KIND_RIGID, cube_local, s / 2, mass=500.0 * a ** 3,
                inertia=_box_inertia(500.0 * a ** 3, (a, a, a)), pose=pose)
    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s),
                         (box_hi[0] + 3 * s, box_hi[1] + 3 * s, box_hi[2] + 3 * s), nu=nu)
    traj = np.zeros((1, 13), np.float32)
    traj[0, :7] = pose
    return Scene("held_cube_tank", params, fluid, np.zeros_like(fluid), s, [walls, cube],
                 grab_body=1, trajectory=traj, n_substeps=2000)


def three_balls_tank(seed=0, ratios=(0.1, 0.3, 1.0), n=(24, 12, 10), radius=0.05, spacing=0.02,
                     dt=1e-3, nu=5e-3):
    """Free balls of the given densities relative to the fluid's (Sec. 4 demo: 0.1, 0.3, 1.0)
    placed half-submerged in a tank of fluid at rest, along x at the fluid surface; the
    fluid cells within a ball are carved out.  Balls are sampled at half the spacing."""
    rng = np.random.default_rng(seed)
    s = spacing
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    cells = (np.stack([i, j, k], -1).reshape(-1, 3) + 0.5) * s
    surface = n[2] * s
    centres = [np.array([(m + 0.5) * n[0] * s / len(ratios), 0.5 * n[1] * s, surface])
               for m in range(len(ratios))]
    keep = np.ones(len(cells), bool)
    for c in centres:
        keep &= np.linalg.norm(cells - c, axis=1) > radius
    fluid = _jitter(rng, cells[keep], s).astype(np.float32)
    box_hi = (n[0] * s, n[1] * s, (n[2] + 8) * s)
    bodies = [Body(KIND_STATIC, wall_shell((0, 0, 0), box_hi, s), s)]
    ball = solid_sphere(radius, s / 2)
    vol = 4.0 / 3.0 * np.pi * radius ** 3
    for r, c in zip(ratios, centres):
        mass = r * 1000.0 * vol
        bodies.append(Body(KIND_RIGID, ball, s / 2, mass=mass,
                           inertia=(0.4 * mass * radius ** 2 * np.eye(3)).astype(np.float32),
                           pose=np.array([*c, 1, 0, 0, 0], np.float32)))
    params = make_params(s, dt, (-3 * s, -3 * s, -3 * s),
                         (box_hi[0] + 3 * s, box_hi[1] + 3 * s, box_hi[2] + 3 * s), nu=nu)
    return Scene("three_balls_tank", params, fluid, np.zeros_like(fluid), s, bodies,
                 n_substeps=3000)


def released_cube_tank(seed=0, sigma=0.2, **kw):
    """The held-cube tank with the cube let go (density 500: it rises) and seeded random
    fluid and cube velocities: undriven two-way coupling in a closed tank."""
    sc = held_cube_tank(seed=seed, **kw)
    sc.name = "released_cube_tank"
    sc.grab_body = -1
    sc.trajectory = None
    return with_velocity_noise(sc, seed=seed, sigma=sigma)


def with_velocity_noise(scene: Scene, seed: int = 0, sigma: float = 0.2) -> Scene:
    """Seeded Gaussian fluid velocities and rigid-body velocities (exercises viscosity
    and the kinematic boundary velocities from the very first substep)."""
    rng = np.random.default_rng(seed)
    scene.fluid_v = rng.normal(0.0, sigma, scene.fluid_x.shape).astype(np.float32)
    for b in scene.bodies:
        if b.kind == KIND_RIGID:
            b.vel = rng.normal(0.0, sigma, 6).astype(np.float32)
            b.vel[3:] *= 5.0
    if scene.trajectory is not None:
        scene.trajectory = scene.trajectory.copy()
        scene.trajectory[:, 10:13] = rng.normal(0.0, sigma, 3).astype(np.float32)
    return scene


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial surrogate parameters in the layout W1[128][269] b1 W2[128][128] b2
    W3[128][128] b3 W4[6][128] b4: weights uniform in +-1/sqrt(fan_in), biases zero."""
    rng = np.random.default_rng(seed)
    sizes = [(128, 269), (128,), (128, 128), (128,), (128, 128), (128,), (6, 128), (6,)]
    out = []
    for s in sizes:
        out.append(rng.uniform(-1, 1, s) / np.sqrt(s[1]) if len(s) == 2 else np.zeros(s))
    return np.concatenate([a.ravel() for a in out]).astype(np.float32)


def mlp_identity_norm() -> np.ndarray:
    """Standardisation vectors xmean[269] xstd[269] ymean[6] ystd[6] that leave data as is."""
    return np.concatenate([np.zeros(269), np.ones(269), np.zeros(6), np.ones(6)]).astype(np.float32)
