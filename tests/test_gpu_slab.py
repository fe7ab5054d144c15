"""The slab decomposition with the library as the per-rank substep: two gloo ranks (two
processes on one GPU; their kernels never wait on each other -- the exchanges are host
messages between substeps) each run the substep of their owned particles plus the ghosts
received from the other rank, and the grabbed body's wrench is the allreduce of the ranks'
partial sums.  Against one undivided run of the whole scene on the same GPU: keys and
neighbour counts bit-equal, densities within 1e-5, every acceleration within the parity
bar, the wrench within 1e-4."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2511_15908_gb300 import scenes, slab

pytestmark = pytest.mark.gpu
G = 9.81


def _scene():
    return scenes.with_velocity_noise(scenes.held_cube_tank(seed=5, n=(18, 10, 12), cube_cells=6),
                                      seed=5, sigma=0.3)


def _mass_by_id(sc):
    import oracle
    m = [np.full(sc.n_fluid, oracle.particle_mass(sc.params["rho0"], sc.fluid_spacing), np.float64)]
    for b in sc.bodies:
        m.append(np.full(b.n, oracle.particle_mass(sc.params["rho0"], b.spacing), np.float64))
    return np.concatenate(m)


def _run(sc, sph):
    """One substep with the record flag: keys and neighbour counts, density, acceleration (id
    order of `sc`)."""
    sim = sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_RECORD)
    sim.step(1)
    keys, ids, _ = sim.sort()
    key = np.empty(sc.n_total, np.uint32)
    key[ids] = keys
    st = sim.state(record=True)
    w = sim.body_wrench(sc.grab_body) if sc.grab_body >= 0 else None
    sim.close()
    return key, st["nnbr"], st["rho"], st["acc"].astype(np.float64), w


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2511_15908_gb300 import sph
    sph.load()
    sc = _scene()
    R = 2.0 * float(np.float32(sc.params["h"]))
    sl = slab.Slabs(0.0, 18 * sc.fluid_spacing, world, halo=2.0 * R)
    (ids, x, v), (gid, gx, gv) = slab.owned_and_ghosts(sc, sl, rank, world)
    sub, sub_ids = slab.sub_scene(sc, np.concatenate([ids, gid]), np.concatenate([x, gx]), np.concatenate([v, gv]))
    key, nnbr, rho, acc, _ = _run(sub, sph)
    mine = np.isin(sub_ids, ids)
    g = sub_ids[mine]
    # the grabbed body's wrench over this rank's owned body particles: pair force m a and
    # its torque about the grab point (the body's centre), FP64
    first = sc.n_fluid + sum(b.n for b in sc.bodies[:sc.grab_body])
    body = sc.bodies[sc.grab_body]
    sel = mine & (sub_ids >= first) & (sub_ids < first + body.n)
    m = _mass_by_id(sc)[sub_ids[sel]]
    f = m[:, None] * acc[sel]
    xg = sc.trajectory[0, :3].astype(np.float64)
    xb = slab.particle_positions(sc)[sub_ids[sel]].astype(np.float64)
    w = np.zeros((1, 6))
    w[0, :3], w[0, 3:] = f.sum(0), np.cross(xb - xg, f).sum(0)
    w_all = slab.allreduce_wrench(w)
    out[rank] = dict(ids=g, key=key[mine], nnbr=nnbr[mine], rho=rho[mine], acc=acc[mine],
                     wrench=w_all[0], n_ghost=int(gid.size))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_equal_one_undivided_gpu_substep():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15908_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = 33000 + os.getpid() % 2000
        ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    from paper_2511_15908_gb300 import sph
    sph.load()
    sc = _scene()
    key, nnbr, rho, acc, wref = _run(sc, sph)
    seen = np.concatenate([res[r]["ids"] for r in range(2)])
    assert np.array_equal(np.sort(seen), np.arange(sc.n_total))
    for r in range(2):
        d = res[r]
        i = d["ids"]
        assert d["n_ghost"] > 0
        np.testing.assert_array_equal(d["key"], key[i])
        np.testing.assert_array_equal(d["nnbr"], nnbr[i])
        assert np.max(np.abs(d["rho"].astype(np.float64) - rho[i]) / rho[i]) <= 1e-5
        scale = np.maximum(np.linalg.norm(acc[i], axis=1), 0.1 * G)
        assert np.max(np.linalg.norm(d["acc"] - acc[i], axis=1) / scale) <= 1e-4
        F, T = d["wrench"][:3], d["wrench"][3:]
        assert np.linalg.norm(F - wref[:3]) <= 1e-4 * np.linalg.norm(wref[:3])
        assert np.linalg.norm(T - wref[3:]) <= 1e-4 * np.linalg.norm(wref[3:])
