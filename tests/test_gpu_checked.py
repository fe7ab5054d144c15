"""The bounds-checked build (-DSPH_CHECKED) on the GPU.  Every index the kernels take from
data (cell keys, sorted slots, particle ids, neighbour-list entries, spring partners) is
checked against its buffer; a failed check would latch SPH_ERR_BOUNDS.  Each case runs the
same scene through both libraries: the checked one must report nothing and, since the
checks only redirect accesses that never happen, give bit-identical results.  This stands
in for a memory sanitizer, which this project cannot run.
"""
import numpy as np
import pytest

from paper_2511_15908_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_15908_gb300 import build, sph as _sph
    build.build()
    build.build(checked=True)
    _sph.load()
    _sph.load(_sph.CHECKED_LIB_PATH)
    return _sph


def _run(sph, make, lib, steps, flags_or=0, max_neighbours=0, cut=None):
    sc = make()
    sim = sph.Simulation(sc, flags=sc.params["flags"] | flags_or, lib=lib,
                         max_neighbours=max_neighbours)
    for i, n in enumerate(steps):
        if cut is not None and i == 1:
            sim.cut_springs(cut(sc))
        sim.step(n)
        sim.sync()
    st = sim.state(record=bool(flags_or & sph.FLAG_RECORD))
    out = [st["x"], st["v"], st["rho"]] + [sim.body(b) for b in range(len(sc.bodies))]
    if sc.grab_body >= 0:
        out.append(sim.grab_wrench())
    sim.close()
    return out


def _blade(sc):
    xc = float(sc.bodies[-1].xyz[5, 0]) + 0.5 * sc.fluid_spacing
    return [[xc, -1.0, -1.0], [xc, 3.0, -1.0], [xc, -1.0, 3.0]]


CASES = {
    "tiny_all_kinds": (lambda: scenes.with_velocity_noise(scenes.tiny(seed=1, n=(8, 8, 8)), seed=1),
                       (1, 9), 0, 0, None),
    "grabbed_record": (lambda: scenes.dam_break(seed=3, grab=True), (1, 20), 2, 0, None),
    "list_overflow_rescan": (lambda: scenes.with_velocity_noise(scenes.dam_break(seed=4), seed=4),
                             (1, 6), 0, 8, None),
    "cloth_cut": (lambda: scenes.cloth_bath(seed=5, anchors="corners"), (3, 10), 0, 0, _blade),
    "tait": (lambda: scenes.dam_break(seed=6, grab=True), (1, 10), 8, 0, None),
    "volume_boundary": (lambda: scenes.coupled(seed=7, n_fluid=40_000, cols=(50, 40),
                                               tank=(0.5, 0.4, 0.4), n_substeps=20, probe_r=0.04,
                                               soft_n=6), (1, 12), 16, 0, None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_checked_build_reports_nothing_and_matches(sph, name):
    make, steps, flags_or, max_nb, cut = CASES[name]
    plain = _run(sph, make, sph.LIB_PATH, steps, flags_or, max_nb, cut)
    checked = _run(sph, make, sph.CHECKED_LIB_PATH, steps, flags_or, max_nb, cut)
    for i, (a, b) in enumerate(zip(plain, checked)):
        assert np.array_equal(a, b), f"{name}: item {i} differs between the builds"


def test_checked_batch_reports_nothing_and_matches(sph):
    outs = []
    for lib in (sph.LIB_PATH, sph.CHECKED_LIB_PATH):
        sims = [sph.Simulation(scenes.with_velocity_noise(scenes.dam_break(seed=s), seed=s), lib=lib)
                for s in (8, 9, 10)]
        bt = sph.Batch(sims)
        bt.configure(-1)
        bt.step(8)
        bt.sync()
        outs.append([sm.state()["x"] for sm in sims])
        bt.close()
        for sm in sims:
            sm.sync()
            sm.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
