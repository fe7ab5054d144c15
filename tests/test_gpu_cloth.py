"""GPU parity of the cloth plane with anchors and of the incision (Sec. 4), against the
FP64 oracle.  The incision's decisions are FP32 on the GPU and FP64 in the oracle; the
blades used here are checked by the oracle to have no spring within 1e-5 (in the test's
parameters) of a decision bound, so the cut sets must be equal -- and since a spring cut
on one side only would change the next substep's accelerations by its full force, the
parity of that substep checks which springs were cut, not only how many.
"""
import numpy as np
import pytest

import oracle
from paper_2511_15908_gb300 import scenes
from test_gpu_parity import check_one_substep, _by_id, G, ACC_TOL

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


def test_cloth_bath_one_substep(sph):
    sc = scenes.with_velocity_noise(scenes.cloth_bath(seed=0), seed=20, sigma=0.2)
    check_one_substep(sph, sc, mode=0)


def test_cloth_edges_anchored_one_substep(sph):
    sc = scenes.cloth_bath(seed=1, anchors="edges")
    check_one_substep(sph, sc, mode=1)


def test_anchors_do_not_move(sph):
    sc = scenes.cloth_bath(seed=2)
    sim = sph.Simulation(sc)
    x0 = sim.state()["x"].copy()
    sim.step(200)
    x = sim.state()["x"]
    first = sc.n_fluid + sc.bodies[0].n
    anc = first + sc.bodies[1].anchors
    assert np.array_equal(x[anc], x0[anc])
    sim.close()


def test_column_blade_cuts_5ny_minus_2(sph):
    sc = scenes.cloth_bath(seed=3, cloth=(16, 12), anchors="none")
    sim = sph.Simulation(sc)
    sheet = sc.bodies[1]
    xc = float(sheet.xyz[5, 0]) + 0.5 * sc.fluid_spacing
    blade = [[xc, -1.0, -1.0], [xc, 3.0, -1.0], [xc, -1.0, 3.0]]
    assert sim.cut_springs(blade) == 5 * 12 - 2
    assert sim.cut_springs(blade) == 0
    sim.close()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_blade_cut_then_substep_matches_oracle(sph, seed):
    rng = np.random.default_rng(100 + seed)
    sc = scenes.with_velocity_noise(scenes.cloth_bath(seed=seed), seed=30 + seed, sigma=0.2)
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
    sim = sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_RECORD)
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
