"""The low-latency passes (SPH_FLAG_LOW_LATENCY: the density pass with 32 or 16 threads per
particle, the force pass with 8):

- one substep against the oracle with the same bars as the default pass (keys, order,
  cell_start and neighbour counts bit-exact, densities within 1e-5, every acceleration within
  1e-4 max(|a|, 0.1 g), wrenches within 1e-4), on scenes with every body kind, a grabbed
  half-spacing cube, cell edges from h to 2h, a neighbour list too short for most
  particles, the Tait equation of state and anchored, cut cloth;
- against the default passes: the same neighbour counts and sorted order, densities apart by
  at most one rounding of the FP32 excess rho - rho0 and one of rho (the float-pair sums are
  added in another order), trajectories that stay together over 20 substeps;
- where the flag has no effect: volume boundaries (bit-identical to the unflagged scene) and
  inside a batch (every structure equals unflagged single-scene stepping bit for bit).
"""
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


def _flagged(sph, sc):
    sc.params = dict(sc.params, flags=sc.params["flags"] | sph.FLAG_LOW_LATENCY)
    return sc


def test_tiny_scene_all_body_kinds(sph):
    check_one_substep(sph, _flagged(sph, scenes.tiny(seed=0, n=(6, 6, 6))), mode=0)


def test_dam_break_grabbed_half_spacing_cube(sph):
    sc = scenes.with_velocity_noise(scenes.dam_break(seed=3, grab=True, cube_pos=(0.4, 0.4, 0.2)),
                                    seed=9, sigma=0.3)
    check_one_substep(sph, _flagged(sph, sc), mode=0)


def test_coupled_reduced_with_soft_body(sph):
    sc = scenes.with_velocity_noise(
        scenes.coupled(seed=0, n_fluid=60_000, cols=(60, 40), tank=(0.6, 0.4, 0.4), n_substeps=10,
                       probe_r=0.04, soft_n=8), seed=4, sigma=0.2)
    check_one_substep(sph, _flagged(sph, sc), mode=1)


@pytest.mark.parametrize("cell_over_h", [1.0, 2.002])
def test_cell_edges_from_h_to_2h(sph, cell_over_h):
    sc = scenes.dam_break(seed=3, grab=True, cube_pos=(0.4, 0.4, 0.2))
    sc.params = dict(sc.params, cell=float(np.float32(cell_over_h * sc.params["h"])))
    check_one_substep(sph, _flagged(sph, sc), mode=0)


def test_short_neighbour_list_takes_the_rescan(sph):
    # 6 list slots: the force pass searches again for almost every particle, in the order
    # the group wrote the list in
    sc = scenes.dam_break(seed=5, grab=True, cube_pos=(0.3, 0.3, 0.15))
    check_one_substep(sph, _flagged(sph, sc), mode=0, max_neighbours=6)


def test_same_neighbours_as_the_default_pass(sph):
    # one substep from the same state: same order and counts, densities within the final
    # roundings; 20 substeps: trajectories that stay together
    scs = [scenes.with_velocity_noise(
               scenes.batched(seed=4, n_scenes=1, lo=100, hi=400, compact=True, n_substeps=40)[0],
               seed=1, sigma=0.2),
           scenes.with_velocity_noise(scenes.dam_break(seed=0, n_substeps=40), seed=2, sigma=0.3)]
    for sc in scs:
        sims = [sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_RECORD | extra)
                for extra in (0, sph.FLAG_LOW_LATENCY)]
        for sim in sims:
            sim.step(1)
        a, b = (sim.state(record=True) for sim in sims)
        for u, w in zip(sims[0].sort(), sims[1].sort()):
            np.testing.assert_array_equal(u, w)
        np.testing.assert_array_equal(a["nnbr"], b["nnbr"])
        # rho = rho0 + (rho - rho0): the two sums, both exact to ~1e-13, can round the FP32
        # excess differently, and then rho0 + excess (one unit of each at most)
        rho0 = np.float32(sc.params["rho0"])
        d = np.abs(a["rho"].astype(np.float64) - b["rho"])
        tol = np.spacing(np.abs(a["rho"] - rho0)) + np.spacing(np.abs(a["rho"]))
        assert np.all(d <= tol), float((d / tol).max())
        print(f"[{sc.name}] densities apart: {np.mean(d > 0):.2%}")
        for sim in sims:
            sim.step(19)
        a, b = (sim.state() for sim in sims)
        assert np.abs(a["x"] - b["x"]).max() <= 1e-3 * sc.fluid_spacing
        for sim in sims:
            sim.close()


def test_no_effect_with_volume_boundaries(sph):
    sc = scenes.dam_break(seed=3, grab=True, cube_pos=(0.4, 0.4, 0.2))
    sc.params = dict(sc.params, flags=sc.params["flags"] | scenes.FLAG_VOLUME_BOUNDARY)
    out = []
    for extra in (0, sph.FLAG_LOW_LATENCY):
        sim = sph.Simulation(sc, flags=sc.params["flags"] | extra)
        sim.step(10)
        st = sim.state()
        out.append((st["x"], st["v"], st["rho"], sim.body(1), sim.grab_wrench(smoothed=False)))
        sim.close()
    for u, w in zip(*out):
        assert np.array_equal(u, w)


@pytest.mark.parametrize("bps", [-1, 0])
def test_batch_runs_one_thread_per_particle(sph, bps):
    # flagged scenes in a batch (-1: their own kernels as graph branches; 0: one kernel per
    # phase) step exactly like the unflagged scenes stepped alone
    scs = scenes.batched(seed=4, n_scenes=3, lo=100, hi=400, compact=True, n_substeps=20) \
        + [scenes.dam_break(seed=7, n_substeps=20)]
    solo = [sph.Simulation(sc) for sc in scs]
    for s in solo:
        s.step(6)
    flagged = [sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_LOW_LATENCY) for sc in scs]
    batch = sph.Batch(flagged)
    batch.configure(bps, 1)
    batch.step(6)
    batch.sync()
    for a, b in zip(solo, flagged):
        sa, sb = a.state(), b.state()
        assert np.array_equal(sa["x"], sb["x"]) and np.array_equal(sa["v"], sb["v"])
        assert np.array_equal(sa["rho"], sb["rho"])
    batch.close()
    for s in solo + flagged:
        s.close()


def test_tait_eos_dam_break(sph):
    # the Tait equation of state in the group density pass
    sc = scenes.with_velocity_noise(scenes.dam_break(seed=3, grab=True, cube_pos=(0.4, 0.4, 0.2)),
                                    seed=10, sigma=0.3)
    sc.params = dict(sc.params, flags=sc.params["flags"] | scenes.FLAG_TAIT)
    check_one_substep(sph, _flagged(sph, sc), mode=0)


@pytest.mark.parametrize("anchors", ["corners", "edges"])
def test_cloth_bath_with_anchors(sph, anchors):
    # springs, anchors and the cloth's soft particles go through the shared tail of the
    # force passes; one substep against the oracle
    sc = scenes.with_velocity_noise(scenes.cloth_bath(seed=1, anchors=anchors), seed=21, sigma=0.2)
    check_one_substep(sph, _flagged(sph, sc), mode=0)


def test_cut_cloth_then_substep_matches_oracle(sph):
    import oracle
    from test_gpu_parity import _by_id, G, ACC_TOL
    rng = np.random.default_rng(200)
    sc = scenes.with_velocity_noise(scenes.cloth_bath(seed=0), seed=40, sigma=0.2)
    sheet = sc.bodies[1]
    lo, hi = sheet.xyz.min(0), sheet.xyz.max(0)
    for _ in range(50):                          # a blade with no ambiguous spring
        c = lo + rng.uniform(0.2, 0.8, 3) * (hi - lo)
        blade = (c + rng.normal(0, 0.08, (3, 3))).astype(np.float32)
        sysm = oracle.System(sc, mode=0)
        n_orc, per_body = sysm.cut_springs(blade)
        if n_orc > 3 and not any(near.any() for _, near in per_body):
            break
    else:
        pytest.fail("no unambiguous blade found")
    sim = sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_RECORD | sph.FLAG_LOW_LATENCY)
    assert sim.cut_springs(blade) == n_orc
    sim.step(1)
    st = sim.state(record=True)
    ref = sysm.substep()
    n = sc.n_total
    acc_ref = _by_id(ref, "acc", n)
    scale = np.maximum(np.linalg.norm(acc_ref, axis=1), 0.1 * G)
    dif = np.linalg.norm(st["acc"].astype(np.float64) - acc_ref, axis=1)
    assert np.all(dif <= ACC_TOL * scale), (dif / scale).max()
    sim.close()
