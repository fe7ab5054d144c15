"""Training data, training and haptic-rate evaluation of the learned wrench surrogate.

The haptic device needs a force every millisecond, while the engine's update cycle -- the
rate at which the paper's method hands the device a new (rolling-averaged) coupling force
(Sec. 3.3) -- is about 60 Hz.  The surrogate fills the gap: at every 1 kHz tick it predicts
the grabbed body's wrench as the exact wrench of the last update cycle plus a learned
correction.  The correction is the network's output for 269 inputs: 13 kinematic values
relative to the last cycle -- the grab point's displacement since the cycle (3), the time
since the cycle started (1), the change of linear velocity since the cycle (3), the current
linear and angular velocity (6) -- and the pooled fluid grid of the cycle (256).  The exact FP64 coupling
reduction of the substep is therefore both the anchor (fallback) and the reference.

Everything numerical runs in the library's kernels (descriptor, MLP forward/backward/Adam,
the substep itself); this module only schedules calls, selects rows and moves arrays.
"""
from __future__ import annotations

import numpy as np

from . import scenes, sph

N_IN, N_OUT = 269, 6


def log_run(sim: "sph.Simulation", n_substeps: int, chunk: int = 2048):
    """Advance `sim` n_substeps substeps; return the per-substep descriptor (n, 269) and
    the exact grab wrench of the same substep (n, 6)."""
    import torch
    desc = torch.empty((n_substeps, N_IN), dtype=torch.float32, device=sim.device)
    wr = []
    done = 0
    while done < n_substeps:
        k = min(chunk, n_substeps - done)
        for i in range(k):
            sim.step(1)
            sim.descriptor_into(desc[done + i])
        try:
            wr.append(sim.wrench_log(k))
        except sph.SphError as e:
            # particles that splash out of the grid are reported once and clamped; the
            # coupling wrench is still exact for the particles in the domain
            if e.status != sph.ERR_DOMAIN:
                raise
            wr.append(sim.wrench_log(k))
        done += k
    try:
        sim.sync()
    except sph.SphError as e:
        if e.status != sph.ERR_DOMAIN:
            raise
    return desc.cpu().numpy(), np.concatenate(wr)


def cycle_start(n: int, cycle: int) -> np.ndarray:
    return (np.arange(n) // cycle) * cycle


def lagged_inputs(desc: np.ndarray, cycle: int, dt: float) -> np.ndarray:
    """Input of substep t relative to the first substep c of its update cycle (the last SPH
    state the haptic loop has seen): displacement x_t - x_c, time (t - c) dt, velocity change
    v_t - v_c, current v_t and w_t, and the fluid grid of substep c."""
    n = desc.shape[0]
    c = cycle_start(n, cycle)
    x = np.empty_like(desc)
    x[:, 0:3] = desc[:, 0:3] - desc[c, 0:3]
    x[:, 3] = (np.arange(n) - c) * dt
    x[:, 4:7] = desc[:, 7:10] - desc[c, 7:10]
    x[:, 7:13] = desc[:, 7:13]
    x[:, 13:] = desc[c, 13:]
    return x


def residual_targets(wrench: np.ndarray, cycle: int) -> np.ndarray:
    """Target of substep t: its exact wrench minus the exact wrench of substep c."""
    return wrench - wrench[cycle_start(wrench.shape[0], cycle)]


def standardisation(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """xmean[269] xstd[269] ymean[6] ystd[6] (constant features keep std 1)."""
    xm, xs = x.mean(0), x.std(0)
    ym, ys = y.mean(0), y.std(0)
    xs = np.where(xs > 1e-6 * max(1.0, float(np.abs(xm).max())), xs, 1.0)
    ys = np.where(ys > 1e-12, ys, 1.0)
    return np.concatenate([xm, xs, ym, ys]).astype(np.float32)


def fit(model: "sph.Surrogate", x: np.ndarray, y: np.ndarray, steps: int = 3000, batch: int = 1024,
        lr: float = 1e-3, seed: int = 0, init_seed: int = 0):
    """Train from seeded initial weights with Adam on random minibatches (device gathers)."""
    import torch
    model.set_params(scenes.mlp_init_params(init_seed), standardisation(x, y))
    xd = torch.tensor(np.ascontiguousarray(x, np.float32), device=model.device)
    yd = torch.tensor(np.ascontiguousarray(y, np.float32), device=model.device)
    g = torch.Generator(device=model.device)
    g.manual_seed(seed)
    losses = []
    n = xd.shape[0]
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=model.device, generator=g)
        lr_s = lr * (0.1 ** (s / max(1, steps)))          # exponential decay to lr / 10
        want = (s % 100 == 0) or s == steps - 1
        loss = model.train_step(xd[idx], yd[idx], lr_s, want_loss=want)
        if want:
            losses.append((s, loss))
    model.sync()
    return losses


def predict(model: "sph.Surrogate", x: np.ndarray) -> np.ndarray:
    import torch
    out = []
    xd = torch.tensor(np.ascontiguousarray(x, np.float32), device=model.device)
    for a in range(0, xd.shape[0], model.max_batch):
        out.append(model.forward(xd[a:a + model.max_batch]).cpu().numpy())
    return np.concatenate(out).astype(np.float64)


def haptic_errors(desc: np.ndarray, wrench: np.ndarray, model: "sph.Surrogate", cycle: int,
                  tick: int, dt: float, window: int = 20):
    """Relative RMS errors at haptic ticks (every `tick` substeps) against the exact wrench:
    hold (last update cycle's wrench), rolling mean of the last `window` cycle wrenches
    (the paper's smoothing) and the surrogate."""
    n = desc.shape[0]
    t = np.arange(0, n, tick)
    c = (t // cycle) * cycle
    exact = wrench[t]
    hold = wrench[c]
    cyc_w = wrench[::cycle]
    k = t // cycle
    roll = np.stack([cyc_w[max(0, i - window + 1):i + 1].mean(0) for i in k])
    pred = hold + predict(model, lagged_inputs(desc, cycle, dt)[t])

    def rel(p, part):
        sl = slice(0, 3) if part == "force" else slice(3, 6)
        return float(np.sqrt(np.mean(np.sum((p[:, sl] - exact[:, sl]) ** 2, 1)))
                     / max(np.sqrt(np.mean(np.sum(exact[:, sl] ** 2, 1))), 1e-30))

    out = {}
    for name, p in (("hold", hold), ("rolling", roll), ("surrogate", pred)):
        out[name] = {"force": rel(p, "force"), "torque": rel(p, "torque")}
    out["gain_vs_hold"] = out["hold"]["force"] / max(out["surrogate"]["force"], 1e-30)
    out["ticks"] = int(t.size)
    return out


def inference_latency_us(sim: "sph.Simulation", model: "sph.Surrogate", reps: int = 200) -> float:
    """Device time of one haptic tick: descriptor + batch-1 forward (CUDA events)."""
    import torch
    d = torch.empty((1, N_IN), dtype=torch.float32, device=sim.device)
    y = torch.empty((1, N_OUT), dtype=torch.float32, device=sim.device)
    s = model.stream
    sim.sync()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):
        for _ in range(5):
            sim.descriptor_into(d[0])
            torch.cuda.current_stream().wait_stream(sim.stream)
            model.forward(d, y)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(reps):
        ev0.record(sim.stream)
        sim.descriptor_into(d[0])
        s.wait_stream(sim.stream)
        model.forward(d, y)
        ev1.record(s)
        ev1.synchronize()
        total += ev0.elapsed_time(ev1)
    return 1e3 * total / reps
