"""The learned wrench surrogate: the BF16 tcgen05 MLP (forward, backward, Adam) and its descriptor,
against the FP64 oracle with BF16 rounding at the same points."""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
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


def _data(B, seed=0):
    rng = np.random.default_rng(seed)
    params = scenes.mlp_init_params(seed)
    o = 128 * 269
    params[o:o + 128] = rng.normal(0, 0.1, 128).astype(np.float32)
    norm = np.concatenate([rng.normal(0, 1, 269), rng.uniform(0.5, 2, 269), rng.normal(0, 1, 6),
                           rng.uniform(0.5, 2, 6)]).astype(np.float32)
    X = (norm[:269] + norm[269:538] * rng.normal(0, 1, (B, 269))).astype(np.float32)
    T = (norm[538:544] + norm[544:550] * rng.normal(0, 1, (B, 6))).astype(np.float32)
    return params, norm, X, T


def test_forward_matches_oracle(sph):
    import torch
    params, norm, X, _ = _data(300)          # 3 row tiles, ragged tail
    m = sph.Surrogate(max_batch=512)
    m.set_params(params, norm)
    y = m.forward(torch.tensor(X, device="cuda"))
    m.sync()
    ref = omlp.forward(params, norm, X, bf=True)
    got = y.cpu().numpy().astype(np.float64)
    # element by element, per output: both sides round to BF16 at the same points, so they
    # differ where an FP32 tensor-core sum and the FP64 sum round an activation to
    # neighbouring BF16 numbers (one unit: 2^-8 relative)
    rms = np.sqrt(np.mean(ref * ref, axis=0))
    ratio = np.abs(got - ref) / (2.0 ** -6 * np.abs(ref) + 2.0 ** -8 * rms)
    print(f"max |dy| / (2^-6 |y| + 2^-8 rms) = {ratio.max():.3f}")
    assert ratio.max() <= 1.0, ratio.max()
    m.close()


@pytest.mark.parametrize("B", [272, 130, 1100])
def test_gradients_match_oracle(sph, B):
    """272: three row tiles, five K chunks of the batch contraction in five K slices; 130: a
    ragged row tile and a two-row K chunk (the batch capacity is not a multiple of 8 either,
    so the column-major copies have padded rows); 1100: 18 K chunks over 8 K slices of 3
    chunks, the last two slices empty (written as zeros)."""
    import torch
    params, norm, X, T = _data(B, seed=1)
    m = sph.Surrogate(max_batch=B + 3)
    m.set_params(params, norm)
    g, loss = m.gradients(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"))
    lref, gref = omlp.grad(params, norm, X, T, bf=True)
    assert loss == pytest.approx(lref, rel=1e-4)
    bounds = [0, 128 * 269, 128 * 270, 128 * 270 + 16384, 128 * 271 + 16384, 128 * 271 + 32768,
              128 * 272 + 32768, 128 * 272 + 32768 + 768, omlp.param_count()]
    for a, b in zip(bounds[:-1], bounds[1:]):
        ga, gb = g[a:b].astype(np.float64), gref[a:b]
        # element by element: both sides round to BF16 at the same points, so they differ
        # only where an FP32 tensor-core sum and the FP64 sum round an activation or a
        # back-propagated value to neighbouring BF16 numbers (one unit: 2^-8 relative)
        rms = np.sqrt(np.mean(gb * gb))
        ratio = np.abs(ga - gb) / (2.0 ** -6 * np.abs(gb) + 2.0 ** -8 * rms)
        print(f"block [{a}, {b}): max |dg| / (2^-6 |g| + 2^-8 rms) = {ratio.max():.3f}")
        assert ratio.max() <= 1.0, (a, b, ratio.max())
    m.close()


def test_adam_training_fits_a_teacher(sph):
    import torch
    rng = np.random.default_rng(5)
    B = 1024
    teacher = scenes.mlp_init_params(11)
    norm = scenes.mlp_identity_norm()
    X = rng.normal(0, 1, (B, 269)).astype(np.float32)
    T = omlp.forward(teacher, norm, X, bf=False).astype(np.float32)
    m = sph.Surrogate(max_batch=B)
    m.set_params(scenes.mlp_init_params(3), norm)
    x, t = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    first = m.train_step(x, t, 1e-3, want_loss=True)
    for _ in range(300):
        m.train_step(x, t, 1e-3)
    last = m.train_step(x, t, 1e-3, want_loss=True)
    assert last < 0.1 * first, (first, last)
    m.close()


def test_descriptor_matches_oracle(sph):
    import torch
    sc = scenes.with_velocity_noise(
        scenes.stirring_tank(seed=2, n_fluid=30_000, cols=(50, 50), tank=(0.4, 0.4, 0.3), n_substeps=10,
                             paddle=(0.02, 0.1, 0.2)), seed=9, sigma=0.2)
    sim = sph.Simulation(sc)
    sim.step(1)
    d = sim.descriptor()
    ref_sub = oracle.System(sc, mode=1).substep()
    n = sc.n_total
    rho = np.empty(n)
    rho[ref_sub["id"]] = ref_sub["rho"]
    nf = sc.n_fluid
    m = np.full(nf, np.float32(1000) * np.float32(np.float32(np.float32(0.008) * np.float32(0.008)) * np.float32(0.008)),
                np.float64)
    row = sc.trajectory[0]
    ref = omlp.descriptor(sc.fluid_x, sc.fluid_v.astype(np.float64), rho[:nf], m, np.ones(nf, np.int32),
                          row[:3].astype(np.float64), row, np.float32(sc.params["h"]))
    np.testing.assert_array_equal(d[:13], row)
    cells = d[13:].reshape(64, 4)
    rc = ref[13:].reshape(64, 4)
    assert np.array_equal(cells[:, 0] > 0, rc[:, 0] > 0)
    assert (rc[:, 0] > 0).sum() >= 8
    np.testing.assert_allclose(cells[:, 0], rc[:, 0], rtol=2e-6, atol=0)
    np.testing.assert_allclose(cells[:, 1:], rc[:, 1:], rtol=1e-5, atol=1e-6)
    sim.close()


def _rot(q):
    w, x, y, z = (float(v) for v in q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_haptic_tick_matches_oracle_network(sph):
    # sph_surrogate_tick: scale-free inputs from the tick's pose and the anchor's descriptor,
    # the network, and the anchor's exact wrench plus the prediction, all on the device;
    # checked against the inputs restated here in FP64 from the documented formulas, the
    # oracle's network (BF16 at the same rounding points) and the anchor's wrench
    import torch
    sc = scenes.with_velocity_noise(
        scenes.stirring_tank(seed=3, n_fluid=30_000, cols=(50, 50), tank=(0.4, 0.4, 0.3), n_substeps=40,
                             paddle=(0.02, 0.1, 0.2)), seed=3, sigma=0.2)
    sim = sph.Simulation(sc)
    sim.step(5)
    params, norm, _, _ = _data(1, seed=4)
    m = sph.Surrogate(max_batch=64)
    m.set_params(params, norm)
    m.anchor(sim)
    anchor = sim.descriptor()                  # the same descriptor the anchor recorded
    w_a = sim.grab_wrench()
    h = float(np.float32(sc.params["h"]))
    c = float(np.sqrt(np.float32(sc.params["k"]), dtype=np.float32))
    rho0 = float(np.float32(sc.params["rho0"]))
    fs = rho0 * c * c * h * h
    R = _rot(anchor[3:7])
    for j, row in enumerate(sc.trajectory[6:12]):
        tau = float(np.float32((j + 1) * 5e-4))
        got = m.tick(row, tau)
        a = anchor.astype(np.float64)
        t = row.astype(np.float64)
        x = np.empty(269)
        x[0:3] = R.T @ (t[0:3] - a[0:3]) / h
        x[3] = tau * c / h
        x[4:7] = R.T @ (t[7:10] - a[7:10]) / c
        x[7:10] = R.T @ t[7:10] / c
        x[10:13] = R.T @ t[10:13] * h / c
        cells = a[13:].reshape(64, 4)
        x[13::4] = cells[:, 0] / rho0 - 1.0
        v = (R.T @ cells[:, 1:].T).T / c
        x[14::4], x[15::4], x[16::4] = v[:, 0], v[:, 1], v[:, 2]
        y = omlp.forward(params, norm, x[None, :].astype(np.float32), bf=True)[0]
        want = np.concatenate([w_a[:3] + R @ y[:3] * fs, w_a[3:] + R @ y[3:] * fs * h])
        dif = np.abs(got - want)
        scale = np.concatenate([np.full(3, np.abs(R @ y[:3] * fs).max()), np.full(3, np.abs(R @ y[3:] * fs * h).max())])
        assert np.all(dif <= 2e-3 * scale + 1e-9 * np.abs(w_a)), (j, got, want)
    with pytest.raises(sph.SphError):
        m2 = sph.Surrogate(max_batch=8)
        try:
            m2.tick(sc.trajectory[0], 0.0)           # no anchor yet
        finally:
            m2.close()
    sim.close()
    m.close()


def test_surrogate_beats_the_update_cycle_hold_at_1khz(sph):
    """What the trained network gains over the method without it: at 1 kHz haptic ticks on
    substeps after the training ones, run live through the library's tick (anchor at every
    ~60 Hz update cycle), the surrogate (exact wrench of the last update cycle + learned
    correction) against holding that exact wrench, and against the paper's rolling average
    over 20 update cycles."""
    from paper_2511_15908_gb300 import surrogate
    n_train, n_cycles = 15000, 150
    sc = scenes.stirring_tank(seed=4, n_fluid=40_000, cols=(50, 50), tank=(0.4, 0.4, 0.3),
                              n_substeps=n_train + 40 * n_cycles, paddle=(0.02, 0.1, 0.2))
    sim = sph.Simulation(sc)
    desc, wr = surrogate.log_run(sim, n_train)
    dt = float(np.float32(sc.params["dt"]))
    cycle, tick = 33, 2                     # dt 5e-4 s: 16.5 ms update cycle, 1 ms tick
    model = sph.Surrogate(max_batch=2048)
    model.set_scene(sc.params)
    x, y = surrogate.pairs(model, desc, wr, cycle, dt)
    losses = surrogate.fit(model, x, y, steps=2000, batch=1024, lr=1e-3)
    assert losses[-1][1] < losses[0][1]
    ev = surrogate.haptic_loop(sim, model, sc.trajectory, n_cycles, cycle, tick, dt)
    print("haptic errors:", ev)
    assert ev["surrogate"]["force"] < ev["hold"]["force"]
    assert ev["surrogate"]["force"] < ev["rolling"]["force"]
    assert ev["surrogate"]["torque"] < ev["hold"]["torque"]
    assert ev["surrogate"]["force"] <= 0.05          # the form's 5 % target
    assert ev["surrogate"]["torque"] <= 0.05
    lat = surrogate.inference_latency_us(sim, model, sc.trajectory)
    print("tick latency:", lat)
    assert lat["host_us"] < 1000.0
    sim.close()
    model.close()
