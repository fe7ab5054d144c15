"""The benchmark's multi-rank arithmetic on CPU: two gloo ranks (no GPU).

Each rank times its own replica; the job's time is the slowest rank's and the job's
throughput counts every rank's particles over that time.
"""
import importlib.util
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    local = [3.0, 5.0][rank]                 # this rank's seconds
    t = b.max_over_ranks(local, device="cpu")
    out[rank] = (t, b.job_rate(1000.0, world, t), b._dist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29000 + os.getpid() % 2000
        ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        t, rate, d = res[r]
        assert t == 5.0
        assert rate == pytest.approx(2 * 1000.0 / 5.0)
        assert d == (2, r, r)


def test_single_process_passes_through():
    b = _bench()
    assert b.max_over_ranks(2.5, device="cpu") == 2.5
    assert b.job_rate(10.0, 1, 2.0) == 5.0


def test_cancellation_ratios_rebuild_the_oracle_wrench():
    # the per-particle pair forces and the grab point R(q) l_g + t the ratios use must give
    # back the oracle's own wrench; a ratio is at least 1 (triangle inequality)
    from paper_2511_15908_gb300 import scenes
    bench = _bench()
    sc = scenes.with_velocity_noise(scenes.dam_break(seed=3, grab=True, cube_pos=(0.2, 0.2, 0.15)),
                                    seed=3, sigma=0.3)
    # a grab point off the centre of mass: the torque is taken about it
    sc.bodies[sc.grab_body].grab_local = np.array([0.02, -0.01, 0.03], np.float32)
    _, out, m = bench._oracle_substep_time(sc)
    k = bench._cancellation(sc, out, m, sc.grab_body)
    w = out["wrench"][sc.grab_body]
    np.testing.assert_allclose(k["force_from_pairs"], w[:3], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(k["torque_from_pairs"], w[3:], rtol=1e-6, atol=1e-9 * np.abs(w[3:]).max())
    assert k["kappa_force"] >= 1.0 and k["kappa_torque"] >= 1.0
