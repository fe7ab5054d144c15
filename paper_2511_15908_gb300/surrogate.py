"""Training data, training and haptic-rate evaluation of the learned wrench surrogate.

The haptic device needs a force every millisecond, while the engine's update cycle -- the
rate at which the paper's method hands the device a new (rolling-averaged) coupling force
(Sec. 3.3) -- is about 60 Hz.  The surrogate fills the gap: at every 1 kHz tick it predicts
the grabbed body's wrench as the exact wrench of the last update cycle (the anchor) plus a
learned correction.  The network reads 269 scale-free inputs that the library builds on
the device from the tick's grab pose and velocity and the anchor's descriptor (pose,
velocity and the pooled fluid grid around the grab point): see sph_surrogate_tick.  The
exact FP64 coupling reduction of the substep is both the anchor (fallback) and the
reference.

Everything numerical runs in the library's kernels (descriptor, features, targets, MLP
forward/backward/Adam, the tick, the substep itself); this module only schedules calls,
selects rows and moves arrays.
"""
from __future__ import annotations

import time

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
        wr.append(_wrench_log(sim, k))
        done += k
    try:
        sim.sync()
    except sph.SphError as e:
        if e.status != sph.ERR_DOMAIN:
            raise
    return desc.cpu().numpy(), np.concatenate(wr)


def _wrench_log(sim: "sph.Simulation", n: int) -> np.ndarray:
    """The last n substeps' exact grab wrenches; a latched out-of-domain report (particles
    that splashed out of the grid are clamped into border cells; the coupling wrench is
    still exact for the particles in the domain) is read once and the log read again."""
    try:
        return sim.wrench_log(n)
    except sph.SphError as e:
        if e.status != sph.ERR_DOMAIN:
            raise
        return sim.wrench_log(n)


def cycle_start(n: int, cycle: int, first: int = 0) -> np.ndarray:
    """Anchor substep of every substep: the first substep of its update cycle."""
    t = np.arange(n)
    return first + ((t - first) // cycle) * cycle


def pairs(model: "sph.Surrogate", desc: np.ndarray, wrench: np.ndarray, cycle: int, dt: float,
          rows=None):
    """Network inputs and targets (CUDA tensors) of the logged substeps `rows` (default: all),
    each against the first substep of its update cycle, built by the library
    (sph_surrogate_features / sph_surrogate_targets)."""
    import torch
    n = desc.shape[0]
    t = np.arange(n) if rows is None else np.asarray(rows)
    c = cycle_start(n, cycle)[t]
    dev = model.device
    ticks = torch.tensor(np.ascontiguousarray(desc[t, :13]), device=dev)
    anchors = torch.tensor(np.ascontiguousarray(desc[c]), device=dev)
    tau = torch.tensor(((t - c) * dt).astype(np.float32), device=dev)
    x = model.features(ticks, anchors, tau)
    y = model.targets(torch.tensor(np.ascontiguousarray(wrench[t]), device=dev),
                      torch.tensor(np.ascontiguousarray(wrench[c]), device=dev), anchors)
    return x, y


def standardisation(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """xmean[269] xstd[269] ymean[6] ystd[6] (constant features keep std 1)."""
    xm, xs = x.mean(0), x.std(0)
    ym, ys = y.mean(0), y.std(0)
    xs = np.where(xs > 1e-6 * max(1.0, float(np.abs(xm).max())), xs, 1.0)
    ys = np.where(ys > 1e-12, ys, 1.0)
    return np.concatenate([xm, xs, ym, ys]).astype(np.float32)


def fit(model: "sph.Surrogate", x, y, steps: int = 3000, batch: int = 1024, lr: float = 1e-3,
        seed: int = 0, init_seed: int = 0, val_frac: float = 0.0, eval_every: int = 250):
    """Train from seeded initial weights with Adam on random minibatches (device gathers);
    x, y: CUDA tensors (n, 269) and (n, 6), rows in time order.  With val_frac > 0 the last
    val_frac of the rows are held out for validation: their MSE (standardised outputs) is
    taken every eval_every steps and the weights of the best evaluation are kept (early
    stopping).  Returns [(step, training loss)], and with validation also the
    [(step, validation loss)] list."""
    import torch
    n_all = x.shape[0]
    n = n_all - int(round(val_frac * n_all)) if val_frac > 0 else n_all
    norm = standardisation(x[:n].cpu().numpy().astype(np.float64), y[:n].cpu().numpy().astype(np.float64))
    model.set_params(scenes.mlp_init_params(init_seed), norm)
    ym = torch.tensor(norm[2 * N_IN:2 * N_IN + N_OUT], device=model.device)
    ys = torch.tensor(norm[2 * N_IN + N_OUT:], device=model.device)

    def val_loss():
        tot = 0.0
        for a in range(n, n_all, model.max_batch):
            yp = model.forward(x[a:min(n_all, a + model.max_batch)])
            d = (yp - y[a:min(n_all, a + model.max_batch)]) / ys
            tot += float((d * d).sum())
        return tot / ((n_all - n) * N_OUT)

    g = torch.Generator(device=model.device)
    g.manual_seed(seed)
    losses, vals = [], []
    best = (np.inf, None)
    for s in range(steps):
        idx = torch.randint(0, n, (min(batch, n),), device=model.device, generator=g)
        lr_s = lr * (0.1 ** (s / max(1, steps)))          # exponential decay to lr / 10
        want = (s % 100 == 0) or s == steps - 1
        loss = model.train_step(x[idx], y[idx], lr_s, want_loss=want)
        if want:
            losses.append((s, loss))
        if n < n_all and ((s + 1) % eval_every == 0 or s == steps - 1):
            v = val_loss()
            vals.append((s + 1, v))
            if v < best[0]:
                best = (v, model.get_params())
    model.sync()
    if best[1] is not None:
        model.set_params(best[1])                          # keeps the standardisation
        return losses, vals
    return losses


def train_step_ms(model: "sph.Surrogate", x, y, batch: int = 1024, steps: int = 200, seed: int = 0) -> float:
    """Device time of one training step (forward, backward, Adam) on minibatches of the pairs
    x, y: CUDA events on the model's stream around `steps` steps after 20 untimed ones.  The
    steps update the model (callers time a model they are done with, or one they refit)."""
    import torch
    g = torch.Generator(device=model.device)
    g.manual_seed(seed)
    n = x.shape[0]
    idx = [torch.randint(0, n, (min(batch, n),), device=model.device, generator=g) for _ in range(8)]
    xs = [x[i].contiguous() for i in idx]
    ys = [y[i].contiguous() for i in idx]
    for k in range(20):
        model.train_step(xs[k % 8], ys[k % 8], 1e-5)
    model.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(model.stream)
    for k in range(steps):
        model.train_step(xs[k % 8], ys[k % 8], 1e-5)
    e1.record(model.stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _rel(p, exact, part):
    sl = slice(0, 3) if part == "force" else slice(3, 6)
    return float(np.sqrt(np.mean(np.sum((p[:, sl] - exact[:, sl]) ** 2, 1)))
                 / max(np.sqrt(np.mean(np.sum(exact[:, sl] ** 2, 1))), 1e-30))


def haptic_loop(sim: "sph.Simulation", model: "sph.Surrogate", path: np.ndarray, n_cycles: int,
                cycle: int, tick: int, dt: float, window: int = 20):
    """The haptic loop run live: at the start of every update cycle the last substep becomes
    the anchor (sph_surrogate_anchor); the cycle's substeps run; the 1 kHz ticks of the
    cycle (every `tick` substeps) each call sph_surrogate_tick with the grab path's pose and
    velocity at that substep.  Relative RMS errors against the exact wrench of the tick's
    substep: the surrogate, holding the anchor's wrench, and the rolling mean of the last
    `window` anchor wrenches (the paper's smoothing).  Also the host time of a tick call."""
    exact, hold, roll, pred = [], [], [], []
    anchors = []
    t_tick, n_tick = 0.0, 0
    base = int(sim.info()[4])                 # substeps already run; the path continues here
    for k in range(n_cycles):
        sim.step(1)
        model.anchor(sim)
        sim.step(cycle - 1)
        w = _wrench_log(sim, cycle)           # exact wrench of the cycle's substeps
        anchors.append(w[0])
        a0 = w[0]
        r = np.mean(anchors[-window:], axis=0)
        for j in range(0, cycle, tick):
            row = path[min(base + k * cycle + j, path.shape[0] - 1)]
            t0 = time.perf_counter()
            p = model.tick(row, j * dt)
            t_tick += time.perf_counter() - t0
            n_tick += 1
            exact.append(w[j])
            hold.append(a0)
            roll.append(r)
            pred.append(p)
    exact, hold, roll, pred = (np.asarray(a) for a in (exact, hold, roll, pred))
    out = {}
    for name, p in (("hold", hold), ("rolling", roll), ("surrogate", pred)):
        out[name] = {"force": _rel(p, exact, "force"), "torque": _rel(p, exact, "torque")}
    out["gain_vs_hold"] = out["hold"]["force"] / max(out["surrogate"]["force"], 1e-30)
    out["ticks"] = int(n_tick)
    out["tick_host_us"] = 1e6 * t_tick / max(n_tick, 1)
    return out


def offline_errors(model: "sph.Surrogate", desc: np.ndarray, wrench: np.ndarray, cycle: int, tick: int,
                   dt: float, window: int = 20):
    """The same errors from logged substeps (network inputs and outputs through the library's
    batched feature and forward calls; the prediction is taken back to the world frame and
    the wrench units here, in FP64)."""
    import torch
    n = desc.shape[0]
    t = np.arange(0, n, tick)
    c = cycle_start(n, cycle)[t]
    x, _ = pairs(model, desc, wrench, cycle, dt, rows=t)
    y = []
    for a in range(0, x.shape[0], model.max_batch):
        y.append(model.forward(x[a:a + model.max_batch]).cpu().numpy())
    y = np.concatenate(y).astype(np.float64)
    sc = model.scales()
    fs = sc["rho0"] * sc["c"] ** 2 * sc["h"] ** 2
    q = desc[c, 3:7].astype(np.float64)
    w_, x_, y_, z_ = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    R = np.stack([np.stack([1 - 2 * (y_ * y_ + z_ * z_), 2 * (x_ * y_ - w_ * z_), 2 * (x_ * z_ + w_ * y_)], -1),
                  np.stack([2 * (x_ * y_ + w_ * z_), 1 - 2 * (x_ * x_ + z_ * z_), 2 * (y_ * z_ - w_ * x_)], -1),
                  np.stack([2 * (x_ * z_ - w_ * y_), 2 * (y_ * z_ + w_ * x_), 1 - 2 * (x_ * x_ + y_ * y_)], -1)], 1)
    dF = np.einsum("nij,nj->ni", R, y[:, :3]) * fs
    dT = np.einsum("nij,nj->ni", R, y[:, 3:]) * fs * sc["h"]
    exact = wrench[t]
    hold = wrench[c]
    pred = hold + np.concatenate([dF, dT], 1)
    cyc_w = wrench[::cycle]
    roll = np.stack([cyc_w[max(0, i - window + 1):i + 1].mean(0) for i in t // cycle])
    out = {}
    for name, p in (("hold", hold), ("rolling", roll), ("surrogate", pred)):
        out[name] = {"force": _rel(p, exact, "force"), "torque": _rel(p, exact, "torque")}
    out["gain_vs_hold"] = out["hold"]["force"] / max(out["surrogate"]["force"], 1e-30)
    out["ticks"] = int(t.size)
    return out


def jitter_floor(wrench: np.ndarray, half: int = 2):
    """Relative RMS of the part of the exact wrench that changes faster than a centred
    moving average over 2 half + 1 substeps: wrench content no input that varies smoothly
    in time (pose, velocity, a lagged fluid grid) can predict.  Force and torque."""
    k = 2 * half + 1
    ker = np.ones(k) / k
    sm = np.stack([np.convolve(wrench[:, a], ker, mode="same") for a in range(6)], 1)
    sl = slice(half, wrench.shape[0] - half)
    return {"force": _rel(sm[sl], wrench[sl], "force"), "torque": _rel(sm[sl], wrench[sl], "torque")}


def inference_latency_us(sim: "sph.Simulation", model: "sph.Surrogate", path: np.ndarray,
                         reps: int = 200) -> dict:
    """Latency of the haptic tick: the device time of anchor + tick kernels (CUDA events on
    the model's stream around one sph_surrogate_tick, anchor excluded) and the host time of
    the whole call (pose in, wrench out)."""
    import torch
    sim.step(1)
    model.anchor(sim)
    row = path[0]
    for _ in range(5):
        model.tick(row, 1e-3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dev, host = 0.0, 0.0
    for _ in range(reps):
        ev0.record(model.stream)
        t0 = time.perf_counter()
        model.tick(row, 1e-3)
        host += time.perf_counter() - t0
        ev1.record(model.stream)
        ev1.synchronize()
        dev += ev0.elapsed_time(ev1)
    return {"device_us": 1e3 * dev / reps, "host_us": 1e6 * host / reps}
