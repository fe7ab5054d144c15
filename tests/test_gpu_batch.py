"""Batched form: many scenes of uneven size in one persistent launch per substep."""
import numpy as np
import pytest

from paper_2511_15908_gb300 import scenes

from test_gpu_parity import check_one_substep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15908_gb300 import build, sph as _sph
    build.build()
    _sph.load()
    return _sph


def _scene_set():
    """Uneven scenes: stirring tanks of log-spread sizes, a dam break and a soft-body tank."""
    out = []
    for i, n in enumerate([8_000, 21_000, 55_000, 9_500]):
        side = max(40, int(np.ceil(np.sqrt(n / 16.0))))
        out.append(scenes.with_velocity_noise(
            scenes.stirring_tank(seed=100 + i, n_fluid=n, cols=(side, side),
                                 tank=(side * 0.008, side * 0.008, 0.5), n_substeps=64,
                                 paddle=(0.02, min(0.2, 0.25 * side * 0.008), 0.3)),
            seed=i, sigma=0.1))
    out.append(scenes.dam_break(seed=7, n_substeps=64))
    out.append(scenes.coupled(seed=3, n_fluid=30_000, cols=(50, 30), tank=(0.5, 0.3, 0.4),
                              n_substeps=64, probe_r=0.03, soft_n=6))
    return out


def _snapshot(sim):
    st = sim.state()
    bodies = [sim.body(b) for b in range(len(sim.scene.bodies))]
    return st["x"], st["v"], st["rho"], bodies, sim.diag()


@pytest.mark.parametrize("bps", [None, -1])
def test_batched_substeps_bit_identical_to_single_scene(sph, bps):
    # None: the structure the batch starts with (the persistent kernel); -1: scene graph
    scs = _scene_set()
    solo = [sph.Simulation(sc) for sc in scs]
    for s in solo:
        s.step(3)
        s.step(4)
    bsims = [sph.Simulation(sc) for sc in scs]
    batch = sph.Batch(bsims)
    if bps is not None:
        batch.configure(bps, 1)
    batch.step(3)
    batch.step(4)
    batch.sync()
    for a, b in zip(solo, bsims):
        xa, va, ra, ba, _ = _snapshot(a)
        xb, vb, rb, bb, _ = _snapshot(b)
        assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ra, rb)
        for p, q in zip(ba, bb):
            assert np.array_equal(p, q)
        if a.scene.grab_body >= 0:
            assert np.array_equal(a.grab_wrench(), b.grab_wrench())
            assert np.array_equal(a.wrench_log(7), b.wrench_log(7))
    batch.close()


def test_batched_volume_boundaries_bit_identical_and_mixed(sph):
    # the boundary-volume phase runs only for scenes that set the flag; a batch mixing
    # both kinds must step each scene exactly as it steps alone, in both launch structures
    scs = _scene_set()[3:6]
    for i in (0, 2):
        scs[i].params = dict(scs[i].params, flags=scs[i].params["flags"] | scenes.FLAG_VOLUME_BOUNDARY)
    solo = [sph.Simulation(sc) for sc in scs]
    for s in solo:
        s.step(4)
    for bps in (-1, 0, 1):
        bsims = [sph.Simulation(sc) for sc in scs]
        batch = sph.Batch(bsims)
        batch.configure(bps, 1)
        batch.step(4)
        batch.sync()
        for a, b in zip(solo, bsims):
            xa, va, ra, ba, _ = _snapshot(a)
            xb, vb, rb, bb, _ = _snapshot(b)
            assert np.array_equal(xa, xb) and np.array_equal(va, vb) and np.array_equal(ra, rb)
        batch.close()


def test_batched_one_substep_matches_oracle(sph):
    # the parity checks of the plain path, with the substep run by the batched launch
    scs = _scene_set()[3:6]

    class BatchedSim(sph.Simulation):
        def step(self, n=1):
            b = sph.Batch([self])
            b.step(n)
            b.sync()
            b.close()

    for sc in scs:
        orig = sph.Simulation
        try:
            sph.Simulation = BatchedSim
            check_one_substep(sph, sc, mode=1)
        finally:
            sph.Simulation = orig


def test_autotuner_picks_a_valid_geometry_and_keeps_results(sph):
    scs = _scene_set()[:3]
    bsims = [sph.Simulation(sc) for sc in scs]
    batch = sph.Batch(bsims)
    max_bps = batch.info()["blocks_per_sm"]
    bps, chunk = batch.tune(substeps_per_trial=1)
    assert -1 <= bps <= max_bps and chunk in (1, 2, 4)
    batch.step(2)
    batch.sync()
    for sc, b in zip(scs, bsims):
        a = sph.Simulation(sc)
        # warm-up + 1 timed substep per tuner candidate: scene graph, per phase, and
        # 3 fetch sizes for each persistent geometry
        for _ in range(max_bps * 3 + 2):
            a.step(2)
        a.step(2)
        assert np.array_equal(a.state()["x"], b.state()["x"])
    batch.close()


def test_per_phase_launches_equal_persistent(sph):
    scs = _scene_set()[:4]
    out = []
    for bps in (0, 1):
        sims = [sph.Simulation(sc) for sc in scs]
        batch = sph.Batch(sims)
        batch.configure(bps, 2)
        batch.step(5)
        batch.sync()
        out.append([s.state()["x"] for s in sims])
        batch.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_grid_barrier_gives_up_and_reports_timeout(sph):
    sc = scenes.dam_break(seed=1)
    sim = sph.Simulation(sc)
    batch = sph.Batch([sim])
    batch.test_barrier(missing_blocks=1, spin_limit=2048)
    with pytest.raises(sph.SphError) as e:
        batch.sync()
    assert e.value.status == sph.ERR_TIMEOUT
    # the barrier was reset: the batch still steps correctly afterwards
    batch.step(2)
    batch.sync()
    ref = sph.Simulation(sc)
    ref.step(2)
    assert np.array_equal(ref.state()["x"], sim.state()["x"])
    batch.close()
