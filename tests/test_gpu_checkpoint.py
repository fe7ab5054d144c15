"""Checkpoint and resume through the C ABI: a handle created from the same scene that loads a
checkpoint continues bit-identically to the run that was never interrupted (positions,
velocities, body table, raw and smoothed grab wrench, wrench log), and a checkpoint of
another scene, or bytes that are not a checkpoint, are refused.
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
    _sph.load()
    return _sph


def _grabbed():
    return scenes.with_velocity_noise(
        scenes.dam_break(seed=6, grab=True, n_substeps=200, cube_pos=(0.3, 0.3, 0.15)),
        seed=6, sigma=0.3)


def _cloth():
    return scenes.cloth_bath(seed=2, anchors="corners")


def _snapshot(sim, sc, grabbed):
    st = sim.state()
    out = [st["x"], st["v"]] + [sim.body(b) for b in range(len(sc.bodies))]
    if grabbed:
        out += [sim.grab_wrench(smoothed=False), sim.grab_wrench(smoothed=True), sim.wrench_log(9)]
    return out


@pytest.mark.parametrize("make,grabbed,cut", [(_grabbed, True, False), (_cloth, False, True)])
def test_resume_is_bit_identical(sph, make, grabbed, cut, tmp_path):
    sc = make()
    xc = float(sc.bodies[-1].xyz[5, 0]) + 0.5 * sc.fluid_spacing
    blade = [[xc, -1.0, -1.0], [xc, 3.0, -1.0], [xc, -1.0, 3.0]]
    a = sph.Simulation(sc)
    a.step(7)
    if cut:
        assert a.cut_springs(blade) > 0
    a.step(6)
    ck = a.checkpoint()
    a.step(5)
    a.step(4)
    want = _snapshot(a, sc, grabbed)
    info_a = a.info()
    a.close()

    for via_file in (False, True):
        b = sph.Simulation(make())
        if via_file:
            p = str(tmp_path / "ck.npz")
            np.savez(p, checkpoint=ck)
            b.load_checkpoint(p)
        else:
            b.restore(ck)
        b.step(5)
        b.step(4)
        got = _snapshot(b, sc, grabbed)
        assert b.info()[4] == info_a[4]              # substeps advanced
        b.close()
        for i, (u, w) in enumerate(zip(got, want)):
            assert np.array_equal(u, w), f"item {i} differs after resume"


def test_checkpoint_taken_after_resume_equals_the_original(sph):
    sc = _grabbed()
    a = sph.Simulation(sc)
    a.step(9)
    ck = a.checkpoint()
    b = sph.Simulation(_grabbed())
    b.restore(ck)
    assert np.array_equal(b.checkpoint(), ck)
    a.close()
    b.close()


def test_foreign_or_damaged_checkpoints_are_refused(sph):
    a = sph.Simulation(_grabbed())
    a.step(3)
    ck = a.checkpoint()
    other = sph.Simulation(_cloth())
    with pytest.raises(sph.SphError) as e:
        other.restore(ck)
    assert e.value.status == sph.ERR_ARG
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(sph.SphError) as e:
        a.restore(bad)
    assert e.value.status == sph.ERR_ARG
    with pytest.raises(sph.SphError) as e:
        a.restore(ck[:-1])
    assert e.value.status == sph.ERR_ARG
    # a refused load leaves the handle as it was
    a.step(2)
    a.sync()
    assert np.all(np.isfinite(a.state()["x"]))
    a.close()
    other.close()


def test_haptic_cycle_equals_the_three_calls(sph):
    sc = _grabbed()
    b = sc.grab_body
    outs = []
    for fused in (False, True):
        sim = sph.Simulation(sc)
        sim.step(3)
        ws = []
        for i in range(6):
            row = sc.trajectory[10 + i]
            if fused:
                ws.append(sim.haptic_cycle(sim.body_ids[b], row[:7], row[7:], 2, smoothed=bool(i % 2)).copy())
            else:
                sim.set_grab_pose(sim.body_ids[b], row[:7], row[7:])
                sim.step(2)
                ws.append(sim.grab_wrench(smoothed=bool(i % 2)))
        st = sim.state()
        outs.append((np.array(ws), st["x"], st["v"], sim.body(b)))
        sim.close()
    for u, w in zip(*outs):
        assert np.array_equal(u, w)


@pytest.mark.parametrize("low_latency", [False, True])
def test_one_substep_haptic_cycle_equals_the_three_calls(sph, low_latency):
    # the haptic tick's form, one substep and the raw wrench, with both density and force
    # passes: the wrenches, the state and the cycle log (read through the smoothed wrench)
    # are the three calls' bit for bit
    sc = _grabbed()
    b = sc.grab_body
    flags = sc.params["flags"] | (sph.FLAG_LOW_LATENCY if low_latency else 0)
    outs = []
    for fused in (False, True):
        sim = sph.Simulation(sc, flags=flags)
        sim.step(3)
        ws = []
        for i in range(8):
            row = sc.trajectory[10 + i]
            if fused:
                ws.append(sim.haptic_cycle(sim.body_ids[b], row[:7], row[7:], 1).copy())
            else:
                sim.set_grab_pose(sim.body_ids[b], row[:7], row[7:])
                sim.step(1)
                ws.append(sim.grab_wrench(smoothed=False))
        st = sim.state()
        outs.append((np.array(ws), sim.grab_wrench(smoothed=True), st["x"], st["v"], sim.body(b),
                     sim.info()[4]))
        sim.close()
    for u, w in zip(*outs):
        assert np.array_equal(u, w)


def test_readme_example_runs(sph):
    # the usage example of the README, verbatim apart from the assertions
    sc = scenes.dam_break(seed=0, grab=True)
    sim = sph.Simulation(sc)
    b = sim.body_ids[sc.grab_body]
    for row in sc.trajectory[:60]:
        wrench = sim.haptic_cycle(b, row[:7], row[7:], n_substeps=1)
    assert wrench.shape == (6,) and np.all(np.isfinite(wrench))
    ck = sim.checkpoint()
    sim.close()
    sim2 = sph.Simulation(sc)
    sim2.restore(ck)
    assert sim2.info()[4] == 60
    sim2.close()
    fast = sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_LOW_LATENCY)
    fast.step(10)
    assert np.all(np.isfinite(fast.state()["x"]))
    fast.close()


def test_released_body_is_a_free_body(sph):
    # release (body id -1) leaves the body free with its last pose and velocity: stepping
    # on equals, bit for bit, a scene that had the free body from the start
    grabbed = scenes.with_velocity_noise(
        scenes.dam_break(seed=8, grab=True, cube_pos=(0.2, 0.2, 0.15)), seed=8, sigma=0.3)
    row = grabbed.trajectory[0]
    free = scenes.with_velocity_noise(
        scenes.dam_break(seed=8, grab=True, cube_pos=(0.2, 0.2, 0.15)), seed=8, sigma=0.3)
    b = free.grab_body
    free.bodies[b].pose = row[:7].copy()
    free.bodies[b].vel = row[7:].copy()
    free.grab_body, free.trajectory = -1, None
    a = sph.Simulation(grabbed)
    a.set_grab_pose(-1, None)
    c = sph.Simulation(free)
    outs = []
    for sim in (a, c):
        sim.step(25)
        st = sim.state()
        outs.append((st["x"], st["v"], sim.body(b), sim.body_wrench(b)))
        sim.close()
    for u, w in zip(*outs):
        assert np.array_equal(u, w)
    assert not np.array_equal(outs[0][2][7:10], row[7:10])     # it moved under gravity


def test_set_state_overwrites_fluid_and_soft_particles(sph):
    # two scenes with the same bodies and body states but different fluid states
    s2 = scenes.with_velocity_noise(scenes.tiny(seed=1, n=(8, 8, 8)), seed=12, sigma=0.3)
    s1 = scenes.with_velocity_noise(scenes.tiny(seed=1, n=(8, 8, 8)), seed=12, sigma=0.3)
    rng = np.random.default_rng(13)
    s1.fluid_v = rng.normal(0.0, 0.3, s1.fluid_v.shape).astype(np.float32)
    s1.fluid_x = (s1.fluid_x + rng.uniform(-1e-3, 1e-3, s1.fluid_x.shape)).astype(np.float32)
    st2 = sph.Simulation(s2).state()                # id order, fluid and bodies
    ref = sph.Simulation(s2)
    ref.step(1)
    want = ref.state()
    # before the first substep: the handle becomes the other scene, bit for bit
    a = sph.Simulation(s1)
    a.set_state(st2["x"], st2["v"])
    a.step(1)
    got = a.state()
    assert np.array_equal(got["x"], want["x"]) and np.array_equal(got["v"], want["v"])
    # after substeps of its own (its free rigid body has moved): the next substep agrees
    # with a fresh handle holding the same fluid state and the body where it now is (the
    # slot order it sorts from, and with it the order of each sum, differs)
    b = sph.Simulation(s1)
    b.step(5)
    s3 = scenes.with_velocity_noise(scenes.tiny(seed=1, n=(8, 8, 8)), seed=12, sigma=0.3)
    for i, body in enumerate(s3.bodies):
        if body.kind == scenes.KIND_RIGID:
            row = b.body(i)
            body.pose, body.vel = row[:7].copy(), row[7:13].copy()
    b.set_state(st2["x"], st2["v"])
    b.step(1)
    c = sph.Simulation(s3)
    c.step(1)
    got, want3 = b.state(), c.state()
    nf = s2.n_fluid
    assert np.abs(got["x"][:nf] - want3["x"][:nf]).max() < 1e-6
    vscale = max(1.0, np.abs(want3["v"][:nf]).max())
    assert np.abs(got["v"][:nf] - want3["v"][:nf]).max() < 1e-3 * vscale
    for sim in (ref, a, b, c):
        sim.close()


def test_new_grab_path_mid_run_starts_at_its_first_row(sph):
    sc = scenes.dam_break(seed=6, grab=True, n_substeps=200, cube_pos=(0.3, 0.3, 0.15))
    b = sc.grab_body
    sim = sph.Simulation(sc)
    sim.step(10)
    rng = np.random.default_rng(4)
    path = scenes.random_walk_trajectory(rng, 30, float(sc.params["dt"]), (0.25, 0.25, 0.2),
                                         (0.08, 0.08, 0.08), (0.42, 0.42, 0.35), sigma=0.05, vmax=0.5)
    sim.set_grab_path(path)
    for k in range(1, 8):
        sim.step(1)
        np.testing.assert_array_equal(sim.body(b)[:7], path[k - 1, :7])
    sim.step(25)                                 # past the path's end: it holds the last row
    np.testing.assert_array_equal(sim.body(b)[:7], path[-1, :7])
    sim.close()
