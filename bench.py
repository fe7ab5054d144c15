"""Benchmark of the SPH coupling substep on GB300 (one JSON line on stdout).

Workload (N=1): the coupled scene -- 1,000,000 fluid particles at 0.01 m in a 2 x 1 x 0.6 m
tank, two-layer static walls, a 30k-particle sphere probe on a seeded random-walk grab
path and a 24^3 soft cube (1,161,538 particles in total), dt 5e-4 s.  One step = one
substep (hash, scan, stable reorder, springs, density, forces + integrate, FP64 wrench
reduction + rigid update), replayed from the captured CUDA graph.  The state starts in
HBM; a 256 MB buffer is written between timed steps so every step starts with a cold
L2 (the working set, ~100-190 MB, is of L2 size).  `value` = fluid particle-steps per
second over all ranks.

With --gpus N (torchrun) every rank runs its own independent replica (the substep of
one scene does not shard); value = sum of particles over ranks x steps / max time.
--impl reference times the FP64 CPU oracle on this host's cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 1M particles (fluid particles x substeps / s)"
UNIT = "particle-steps/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "traffic.json")
KERNEL_SRC = [os.path.join(ROOT, "paper_2511_15908_gb300", "csrc", f)
              for f in ("sph_device.cuh", "sph_kernels.cu", "sph_internal.cuh")]

# Algorithmic cost model (documented in the design notes):
BYTES_PER_PARTICLE_STEP = 168          # HBM bytes of one substep per particle
FORCE_BYTES_PER_PARTICLE = 72          # force pass: read x, v, (rho, P); write x, v
DENSITY_BYTES_PER_PARTICLE = 20        # density pass: read x (16), write rho (4)
FORCE_FLOPS_PER_PAIR = 50              # the method's flops per pair (pressure + viscosity)
DENSITY_FLOPS_PER_PAIR = 15            # the method's flops per pair (r, W, m W, sum)
FP32_LANES_PER_SM, SMS = 128, 152
SPIN_UP_SUBSTEPS = 300                 # untimed: the probe stirs the settled tank first


def _peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SRC:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel):
    """DRAM bytes per launch from a committed ncu capture, if the kernel is unchanged."""
    try:
        with open(TRAFFIC_PATH) as f:
            t = json.load(f)
    except OSError:
        return None
    e = t.get(kernel)
    if not e or e.get("source_sha") != _kernel_hash():
        return None
    return e.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"sph_bench_clocks_{os.getpid()}_rank{index}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait(timeout=10)
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device: str = "cuda") -> float:
    """The largest of each rank's x (the job's time is its slowest rank's); x itself when
    no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return world * units_per_rank / seconds


def _workload(name, fluid=None):
    from paper_2511_15908_gb300 import scenes
    if name == "coupled" and fluid:
        # the same tank depth, spacing, probe and soft cube on a shorter tank (profiling
        # captures on a reduced scene)
        cols_x = max(40, int(round(fluid / (100 * 50))))
        return scenes.coupled(seed=0, n_fluid=int(fluid), cols=(cols_x, 100),
                              tank=(0.01 * cols_x, 1.0, 0.6), n_substeps=4096)
    if name == "coupled":
        return scenes.coupled(seed=0, n_substeps=4096)      # settled fill (see scenes.coupled)
    if name == "stirring":
        return scenes.stirring_tank(seed=0, n_substeps=4096)
    if name == "dam_break":
        return scenes.dam_break(seed=0, n_substeps=4096, grab=True)   # the cube on a grab path
    raise ValueError(name)


def _oracle_substep_time(sc, max_seconds=60.0):
    """Time one FP64 grid-oracle substep of `sc` on all host cores; returns (s, result, the
    signed particle masses in the result's sorted order)."""
    import oracle
    sysm = oracle.System(sc, mode=1)
    t0 = time.perf_counter()
    out = sysm.substep()
    return time.perf_counter() - t0, out, sysm.m.astype(np.float64)


def _cancellation(sc, out, m_sorted, g):
    """Cancellation ratios of the grabbed body's wrench in one oracle substep:
    kappa_F = sum_i |f_i| / |sum_i f_i| and kappa_tau = sum_i |r_i x f_i| / |sum_i r_i x f_i|
    over its particles (f_i = m_i a_i, the pair force; r_i from the grab point).  An FP32
    error of the pair forces reaches the summed wrench amplified by kappa."""
    first = sc.n_fluid + sum(b.n for b in sc.bodies[:g])
    ids = out["id"]
    sel = (ids >= first) & (ids < first + sc.bodies[g].n)
    f = np.abs(m_sorted[sel])[:, None] * out["acc"][sel]
    t, q = out["body_new"][g][:3], out["body_new"][g][3:7]
    w, x, y, z = q / np.linalg.norm(q)
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                  [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                  [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
    xg = R @ np.asarray(sc.bodies[g].grab_local, np.float64) + t
    tau = np.cross(out["x_new"][sel] - xg, f)
    F, T = f.sum(axis=0), tau.sum(axis=0)
    return {"kappa_force": float(np.linalg.norm(f, axis=1).sum() / max(np.linalg.norm(F), 1e-300)),
            "kappa_torque": float(np.linalg.norm(tau, axis=1).sum() / max(np.linalg.norm(T), 1e-300)),
            "force_from_pairs": F.tolist(), "torque_from_pairs": T.tolist()}


def _oracle_modes():
    """A table of CPU-baseline timings: the oracle (as it stands) in brute-force mode on the
    dam break and in grid mode on the dam break, the stirring tank and the coupled scene, on
    all host cores and on one; ms per substep (each a bounded number of substeps)."""
    import oracle
    from paper_2511_15908_gb300 import scenes
    cases = [("brute", "dam_break", 0, lambda: scenes.dam_break(seed=0), 1),
             ("grid", "dam_break", 1, lambda: scenes.dam_break(seed=0), 3),
             ("grid", "stirring", 1, lambda: scenes.stirring_tank(seed=0, n_substeps=8), 1),
             ("grid", "coupled", 1, lambda: scenes.coupled(seed=0, n_substeps=8), 1)]
    out = {}
    for kind, name, mode, make, reps in cases:
        sc = make()
        for threads in (0, 1):
            oracle.set_threads(threads)
            sysm = oracle.System(sc, mode=mode)
            t0 = time.perf_counter()
            for _ in range(reps):
                sysm.substep()
            ms = 1e3 * (time.perf_counter() - t0) / reps
            out[f"{kind}_{name}_{'all_cores' if threads == 0 else '1_core'}_ms"] = ms
    oracle.set_threads(0)
    return out


def _workload_name(name, sc):
    return (f"{name} scene: {sc.n_fluid} fluid + {sc.n_total - sc.n_fluid} boundary/soft "
            f"particles, dt {sc.params['dt']}")


def _reference_config(args, full):
    """The same workload line as the CUDA arm's."""
    return {"workload": _workload_name(args.workload, full), "particles_all": full.n_total,
            "particles_fluid": full.n_fluid, "parallelism": "host cores (oracle)",
            "sample": "the full scene's first substeps from its settled fill (the CUDA arm "
                      "times the stirred state after a 300-substep spin-up)"}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on this host's cores."""
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    sc = _workload(args.workload, args.fluid)
    sysm = oracle.System(sc, mode=1)
    for _ in range(args.warmup):
        sysm.substep()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sysm.substep()
    dt = time.perf_counter() - t0
    value = sc.n_fluid * args.steps / dt
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _reference_config(args, sc),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} substeps (after {args.warmup} untimed) of the "
                                       f"full scene ({sc.n_total} particles), FP64 uniform-grid "
                                       "oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _batch_run(scs, args, tune=True):
    """Batch of `scs` (autotuned launch structure unless tune is False), warmed up; returns
    (sims, batch, choice, substeps advanced)."""
    from paper_2511_15908_gb300 import sph
    sims = [sph.Simulation(sc) for sc in scs]
    batch = sph.Batch(sims)
    choice = batch.tune(substeps_per_trial=2) if tune else None
    for _ in range(args.warmup):
        batch.step(1)
    batch.sync()
    return sims, batch, choice, int(sims[0].info()[4])


def batched_set(name, make, args, cells=(1.001, 2.002)):
    """One set of independent scenes: the project's autotuner picks the grid cell edge (over
    `cells`, in h; each candidate's scenes built and tuned) and, for it, the launch structure
    (persistent cooperative kernel at 1..max resident blocks per SM x 1/2/4 tiles per fetch,
    one kernel per phase, or every scene's kernels as graph branches; sph_batch_tune).  The
    batch then runs args.steps substeps back to back between device events, against the same
    scenes stepped one by one (graph replay per scene, one stream each) from the same state."""
    import torch
    from paper_2511_15908_gb300 import sph
    k = max(args.steps, 10)
    trials = {}
    best = None
    for cell in cells:
        scs = make(cell)
        sims, batch, choice, _ = _batch_run(scs, args)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(batch.stream)
        batch.step(5)
        e1.record(batch.stream)
        batch.sync()
        ms = e0.elapsed_time(e1) / 5
        trials[f"{cell}h"] = {"ms_per_step": ms, "blocks_per_sm": choice[0], "tiles_per_fetch": choice[1]}
        for x in sims:
            x.close()
        batch.close()
        if best is None or ms < best[1]:
            best = (cell, ms, choice)
    cell, _, choice = best
    scs = make(cell)
    sims, batch, _, _ = _batch_run(scs, args, tune=False)
    batch.configure(*choice)
    for _ in range(3):
        batch.step(1)
    batch.sync()
    advanced = int(sims[0].info()[4])
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(batch.stream)
    for _ in range(k):
        batch.step(1)
    ev1.record(batch.stream)
    batch.sync()
    t_b = ev0.elapsed_time(ev1) / 1e3
    nf = sum(sc.n_fluid for sc in scs)
    na = sum(sc.n_total for sc in scs)
    solo = [sph.Simulation(sc) for sc in scs]
    for s_ in solo:
        s_.step(advanced)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(solo[0].stream)
    for s_ in solo[1:]:
        s_.stream.wait_event(e0)
    for _ in range(k):
        for s_ in solo:
            s_.step(1)
    for s_ in solo[1:]:
        done = torch.cuda.Event()
        done.record(s_.stream)
        solo[0].stream.wait_event(done)
    e1.record(solo[0].stream)
    e1.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    # batched and one-by-one stepping of the same scenes give identical wrenches
    werr = 0.0
    for a, b in zip(sims[:4], solo[:4]):
        wa, wb = a.grab_wrench(), b.grab_wrench()
        werr = max(werr, float(np.linalg.norm(wa - wb) / max(np.linalg.norm(wa), 1e-30)))
    info = batch.info()
    bps = info["blocks_per_sm"]
    out = {"workload": f"{name}: {len(scs)} stirring scenes, {nf} fluid / {na} particles",
           "scenes": len(scs), "value": nf * k / t_b, "unit": UNIT, "ms_per_step": 1e3 * t_b / k,
           "all_particle_steps_per_s": na * k / t_b,
           "one_by_one_ms_per_step": 1e3 * t_seq / k,
           "speedup_vs_one_by_one": (t_seq / k) / (t_b / k),
           "autotuned": {"cell_over_h": cell, "blocks_per_sm": bps, "tiles_per_fetch": info["tiles_per_fetch"],
                         "sms": info["sms"], "candidates": trials},
           "grab_wrench_rel_diff_vs_one_by_one": werr,
           "gpu_launches_per_step": (9 if bps == 0 else 8 * len(scs) if bps < 0 else 1),
           "launch_structure": ("one kernel per phase over all scenes" if bps == 0
                                else "every scene's own kernels as branches of one graph" if bps < 0
                                else "one persistent cooperative kernel"),
           "timing": f"{k} substeps back to back between device events, both sides from the same state"}
    for x in sims + solo:
        x.close()
    batch.close()
    return out


def batched_form(args, flush_l2_factory):
    """Batched scenes: (a) the configuration named for the form -- 64 stirring scenes of
    log-uniform fluid counts 8k-256k (8 M particles, compute-bound); (b) 256 compact stirring
    scenes of 2k-8k fluid (2.7 M particles, 6.5k-17k per scene); (c) a launch-bound set --
    512 compact scenes of 500-2k fluid (2.8 M particles, mostly tank walls)."""
    from paper_2511_15908_gb300 import scenes
    n_sub = args.steps + args.warmup + 200
    return {"stirring_64_8k_256k": batched_set(
                "64 scenes, fluid log-uniform 8k-256k (seed 0)",
                lambda cell: scenes.batched(seed=0, n_substeps=n_sub, cell_over_h=cell), args),
            "stirring_256_compact_2k_8k": batched_set(
                "256 compact scenes, fluid log-uniform 2k-8k (seed 1)",
                lambda cell: scenes.batched(seed=1, n_scenes=256, lo=2000, hi=8000, compact=True,
                                            n_substeps=n_sub, cell_over_h=cell), args),
            "stirring_512_compact_500_2k": batched_set(
                "512 compact scenes, fluid log-uniform 500-2k (seed 2)",
                lambda cell: scenes.batched(seed=2, n_scenes=512, lo=500, hi=2000, compact=True,
                                            n_substeps=n_sub, cell_over_h=cell), args)}


def variant_form(args, sc, flush_l2_factory, flag, what):
    """A variant of the method (a flag) on the same workload: ms per substep and the density
    and force passes, timed like the plain path."""
    import torch
    from paper_2511_15908_gb300 import sph
    sim = sph.Simulation(sc, flags=sc.params["flags"] | flag)
    sim.set_profiling(True)
    flush = flush_l2_factory(sim.stream)
    domain = [0]
    for _ in range(max(3, args.warmup)):
        flush()
        sim.step(1)
    _reported(sim.sync, domain, sph)
    n = max(5, args.steps)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    kt = np.zeros((n, len(sph.KERNELS)))
    for i in range(n):
        flush()
        ev0[i].record(sim.stream)
        sim.step(1)
        ev1[i].record(sim.stream)
        kt[i] = _reported(sim.kernel_times, domain, sph)
    _reported(sim.sync, domain, sph)
    ms = float(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)]))
    km = kt.mean(axis=0)
    sim.close()
    return {"ms_per_substep": ms, "value": sc.n_fluid / (ms / 1e3), "unit": UNIT,
            "density_ms": float(km[sph.KERNELS.index("density")]),
            "force_ms": float(km[sph.KERNELS.index("force")]), "out_of_domain_reports": domain[0],
            "what": what}


def isosurface_form(args, sc):
    """Alg. 2's isosurface kernels on the same workload after 20 substeps: the corner density
    field (hash of the current state + field pass) and marching cubes, cube = h,
    isovalue rho0 / 2, device time with CUDA events on the simulation's stream."""
    import torch
    from paper_2511_15908_gb300 import sph
    sim = sph.Simulation(sc)
    domain = [0]
    sim.step(20)
    _reported(sim.sync, domain, sph)
    cube = float(np.float32(sc.params["h"]))
    iso = float(np.float32(0.5 * sc.params["rho0"]))
    dims, origin = sph.iso_grid(sc.params, cube)
    s = sim.stream
    field_ms, mc_ms, n_tris = [], [], 0
    for rep in range(6):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(s)
        f = sim.iso_field(cube)
        e1.record(s)
        tris = sph.iso_polygonize(f, dims, origin, cube, iso, max_tris=4 << 20, stream=s)
        e2.record(s)
        e2.synchronize()
        if rep > 0:
            field_ms.append(e0.elapsed_time(e1))
            mc_ms.append(e1.elapsed_time(e2))
        n_tris = int(tris.shape[0])
    sim.close()
    return {"field_ms": float(np.median(field_ms)), "polygonize_ms": float(np.median(mc_ms)),
            "triangles": n_tris, "corners": int(np.prod(dims)), "cube": cube, "isovalue": iso,
            "what": "sph_iso_field (hash of the current state + fluid density at every corner) "
                    "and sph_iso_polygonize (count, scan, write) after 20 substeps"}


def cloth_form(args, flush_l2_factory):
    """The cloth plane with anchors and incision (Sec. 4): a 100 x 100 soft sheet anchored at
    its corners over a 100 x 100 x 40 fluid block, timed per substep like the plain path,
    before and after a full-width incision; the incision call (sort of the current state +
    the segment-triangle test over every spring) is timed on the simulation's stream."""
    import torch
    from paper_2511_15908_gb300 import scenes, sph
    sc = scenes.cloth_bath(seed=0, n=(100, 100, 40), cloth=(100, 100), anchors="corners")
    sim = sph.Simulation(sc)
    sim.set_profiling(True)
    flush = flush_l2_factory(sim.stream)
    domain = [0]
    # a fixed, short run: the block has a floor but no walls, and spreads out of the grid
    # domain after a few hundred substeps
    n = 20

    def timed():
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
        kt = np.zeros((n, len(sph.KERNELS)))
        for i in range(n):
            flush()
            ev0[i].record(sim.stream)
            sim.step(1)
            ev1[i].record(sim.stream)
            kt[i] = _reported(sim.kernel_times, domain, sph)
        _reported(sim.sync, domain, sph)
        km = kt.mean(axis=0)
        return (float(np.mean([a.elapsed_time(b) for a, b in zip(ev0, ev1)])),
                float(km[sph.KERNELS.index("density")]), float(km[sph.KERNELS.index("force")]))

    for _ in range(3):
        flush()
        sim.step(1)
    _reported(sim.sync, domain, sph)
    before = timed()
    sheet = sc.bodies[1]
    xc = float(sheet.xyz[50, 0]) + 0.5 * sc.fluid_spacing
    blade = [[xc, -10.0, -10.0], [xc, 30.0, -10.0], [xc, -10.0, 30.0]]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(sim.stream)
    n_cut = _reported(lambda: sim.cut_springs(blade), domain, sph)
    e1.record(sim.stream)
    e1.synchronize()
    cut_ms = e0.elapsed_time(e1)
    after = timed()
    n_springs = int(sheet.springs.shape[0])
    sim.close()
    return {"ms_per_substep": before[0], "value": sc.n_fluid / (before[0] / 1e3), "unit": UNIT,
            "density_ms": before[1], "force_ms": before[2],
            "after_cut": {"ms_per_substep": after[0], "density_ms": after[1], "force_ms": after[2]},
            "cut_ms": cut_ms, "springs": n_springs, "springs_cut": n_cut,
            "fluid": sc.n_fluid, "cloth_particles": sheet.n, "out_of_domain_reports": domain[0],
            "what": "cloth bath: 100 x 100 sheet (corner anchors, structural/shear/bending "
                    "springs) over 400k fluid particles, dt 5e-4, 3 warm-up and 20 timed "
                    "substeps before and 20 after the incision; incision = one "
                    "sph_cut_springs call with a full-width blade between two columns"}


def size_sweep_form(args, flush_l2_factory, sc_main):
    """Substep time against particle count (the paper relates particle count to frame rate):
    the dam break (4,096 fluid), the stirring tank (250k fluid) and the coupled scene (1M
    fluid), each 10 warm-up and 50 timed substeps with an L2 flush before each, CUDA events
    on the simulation's stream; the two small scenes also with the low-latency density pass
    (SPH_FLAG_LOW_LATENCY), and a compact stirring scene (369 fluid, 4,821 particles)."""
    import torch
    from paper_2511_15908_gb300 import scenes, sph
    out = {}
    compact = scenes.batched(seed=4, n_scenes=1, lo=100, hi=400, compact=True, n_substeps=64)[0]
    ll = sph.FLAG_LOW_LATENCY
    for name, sc, extra in (("dam_break_4k", scenes.dam_break(seed=0), 0),
                            ("dam_break_4k_low_latency", scenes.dam_break(seed=0), ll),
                            ("compact_stirring_369", compact, 0),
                            ("compact_stirring_369_low_latency", compact, ll),
                            ("stirring_250k", scenes.stirring_tank(seed=0, n_substeps=64), 0),
                            ("coupled_1M", sc_main, 0)):
        sim = sph.Simulation(sc, flags=sc.params["flags"] | extra)
        flush = flush_l2_factory(sim.stream)
        domain = [0]
        for _ in range(10):
            flush()
            sim.step(1)
        _reported(sim.sync, domain, sph)
        n = 50
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for e0, e1 in ev:
            flush()
            e0.record(sim.stream)
            sim.step(1)
            e1.record(sim.stream)
        _reported(sim.sync, domain, sph)
        ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
        out[name] = {"particles_all": int(sc.n_total), "particles_fluid": int(sc.n_fluid),
                     "ms_per_substep": ms, "substeps_per_s": 1e3 / ms,
                     "fluid_particle_steps_per_s": sc.n_fluid / (ms / 1e3)}
        sim.close()
    return out


def surrogate_form(args):
    """The learned wrench surrogate: the BF16 tcgen05 MLP at 1 kHz haptic ticks, trained on the
    GPU from logged (descriptor, wrench) pairs.  (a) The stirring tank (250k fluid): trained on
    its first substeps, then evaluated LIVE through the library's tick (sph_surrogate_anchor at
    every ~60 Hz update cycle, sph_surrogate_tick every 1 ms with the grab path's pose).
    (b) The dam-break pairs of the cube grab (2000 seeded episodes of 100 substeps = 200k
    pairs): held-out episodes, and transfer of that network to the stirring tank (inputs and
    outputs are scale-free).  Errors are relative RMS against the exact FP64 coupling
    reduction at every tick; beside them the wrench's substep-scale jitter, the part no
    smooth input can predict."""
    import torch
    from paper_2511_15908_gb300 import scenes, sph, surrogate
    out = {}
    n, n_train = args.sur_substeps, int(0.75 * args.sur_substeps)
    sc = scenes.stirring_tank(seed=0, n_substeps=n + 8192)
    dt = float(np.float32(sc.params["dt"]))
    cycle, tick = 33, 2                          # dt 5e-4 s: 16.5 ms update cycle, 1 ms tick
    sim = sph.Simulation(sc)
    t0 = time.perf_counter()
    desc, wr = surrogate.log_run(sim, n_train)
    t_log = time.perf_counter() - t0
    model = sph.Surrogate(max_batch=2048)
    model.set_scene(sc.params)
    x, y = surrogate.pairs(model, desc, wr, cycle, dt)
    t0 = time.perf_counter()
    steps = 20000
    losses, vals = surrogate.fit(model, x, y, steps=steps, batch=1024, lr=1e-3, val_frac=0.1)
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t0
    n_cycles = (n - n_train) // cycle
    ev = surrogate.haptic_loop(sim, model, sc.trajectory, n_cycles, cycle, tick, dt)
    lat = surrogate.inference_latency_us(sim, model, sc.trajectory)
    t_step = surrogate.train_step_ms(model, x, y, batch=1024)     # after the evaluation
    out["stirring_logged"] = {"train_pairs": n_train, "eval_ticks": ev["ticks"], "errors": ev,
                              "evaluated": "live: sph_surrogate_anchor per update cycle, "
                                           "sph_surrogate_tick per 1 kHz tick (held-out substeps "
                                           "after the training ones)",
                              "train_steps": steps, "train_s": t_fit, "log_s": t_log,
                              "train_step_ms_batch1024": t_step,
                              "first_last_loss": [losses[0][1], losses[-1][1]],
                              "early_stopping": {"validation": "last 10 % of the training pairs",
                                                 "best_step_and_loss": list(min(vals, key=lambda v: v[1]))},
                              "jitter_floor": surrogate.jitter_floor(wr)}
    out["tick_latency_us"] = lat
    per_ep = 100
    nd = args.sur_dam_episodes * per_ep
    nd_train = (3 * args.sur_dam_episodes // 4) * per_ep
    sd = scenes.dam_break(seed=1, grab=True, n_substeps=per_ep, cube_pos=(0.4, 0.4, 0.2))
    sd.trajectory = scenes.episode_trajectory(args.sur_dam_episodes, per_ep, float(sd.params["dt"]),
                                              (0.4, 0.4, 0.2), (0.08, 0.08, 0.08), (0.42, 0.42, 0.35),
                                              seed0=1000)
    sim_d = sph.Simulation(sd, max_path=nd + 16)
    d_d, w_d = surrogate.log_run(sim_d, nd)
    dtd = float(np.float32(sd.params["dt"]))
    cyc_d = 17                                   # dt 1e-3 s: ~60 Hz update cycle, 1 kHz tick
    model_d = sph.Surrogate(max_batch=2048)
    model_d.set_scene(sd.params)
    xd_, yd_ = surrogate.pairs(model_d, d_d, w_d, cyc_d, dtd, rows=np.arange(nd_train))
    surrogate.fit(model_d, xd_, yd_, steps=20000, batch=1024, lr=1e-3, val_frac=0.1)
    ev_in = surrogate.offline_errors(model_d, d_d[nd_train:], w_d[nd_train:], cyc_d, 1, dtd)
    # the stirring tank's held-out substeps in its own scales (first logged after training)
    model_d.set_scene(sc.params)
    d_s, w_s = surrogate.log_run(sim, 2048)
    ev_tr = surrogate.offline_errors(model_d, d_s, w_s, cycle, tick, dt)
    out["dam_break_trained"] = {"train_pairs": nd_train, "episodes": args.sur_dam_episodes,
                                "substeps_per_episode": per_ep, "held_out_dam_break_1khz": ev_in,
                                "transfer_to_stirring_1khz": ev_tr,
                                "jitter_floor": surrogate.jitter_floor(w_d)}
    out["target_rel_err"] = 0.05
    for m_ in (model, model_d):
        m_.close()
    sim.close()
    sim_d.close()
    return out


def _reported(fn, counter, sph):
    """Call fn(); a latched out-of-domain report (particles that splashed over the tank
    walls are clamped into border cells) is counted and the read repeated -- the status
    clears once reported and the data is unchanged."""
    try:
        return fn()
    except sph.SphError as e:
        if e.status != sph.ERR_DOMAIN:
            raise
        counter[0] += 1
        return fn()


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_2511_15908_gb300 import build, sph
    build.build()
    sc = _workload(args.workload, args.fluid)
    if args.low_latency:
        sc.params = dict(sc.params, flags=sc.params["flags"] | sph.FLAG_LOW_LATENCY)
    peaks, peak_kind = _peaks()

    # first substep with the record flag: accelerations for the parity figure against the
    # oracle (compared at the end, after the GPU timing); then the same scene on through
    # the spin-up (the record flag does not change the dynamics) for the neighbour
    # statistics of the stirred state, which give the algorithmic flop count
    rec = sph.Simulation(sc, flags=sc.params["flags"] | sph.FLAG_RECORD)
    rec.step(1)
    acc_first = rec.state(record=True)["acc"]
    rec.step(SPIN_UP_SUBSTEPS)
    rec_domain = [0]
    _reported(rec.sync, rec_domain, sph)
    nn = rec.state(record=True)["nnbr"]
    pairs = float(np.sum(nn, dtype=np.int64) + sc.n_total)   # density includes self
    mean_nbrs = float(np.mean(nn))
    rec.close()
    del rec

    sim = sph.Simulation(sc)
    sim.set_profiling(True)
    n_all = sc.n_total
    # first substep: grab-wrench error against the FP64 oracle
    sim.step(1)
    w_gpu = sim.grab_wrench()

    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = sim.stream

    def flush_l2():
        with torch.cuda.stream(stream):
            flush.fill_(1)

    domain = [0]
    # the stirred regime: the probe walks through the settled tank for SPIN_UP_SUBSTEPS
    # untimed substeps before the warm-up and the timed steps
    sim.step(SPIN_UP_SUBSTEPS)
    _reported(sim.sync, domain, sph)
    # the timed region records events around the density pass only (each event node in the
    # graph costs the substep a few microseconds); the per-kernel split comes from a separate
    # pass after it
    sim.set_profiling(2)
    for _ in range(args.warmup):
        flush_l2()
        sim.step(1)
    _reported(sim.sync, domain, sph)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ktimes = np.zeros((args.steps, len(sph.KERNELS)))
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush_l2()
            ev0[i].record(stream)
            sim.step(1)
            ev1[i].record(stream)
            ktimes[i] = _reported(sim.kernel_times, domain, sph)   # synchronises the stream
        torch.cuda.synchronize()
    _reported(sim.sync, domain, sph)
    step_ms = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])
    total_s = max_over_ranks(float(step_ms.sum()) / 1e3)
    if world > 1:
        torch.distributed.barrier()
    value = job_rate(sc.n_fluid * args.steps, world, total_s)
    ms_per_step = 1e3 * total_s / args.steps
    density_live_ms = float(ktimes[:, sph.KERNELS.index("density")].mean())

    # per-kernel split: the same substeps with events around every kernel, untimed
    sim.set_profiling(1)
    ktimes_all = np.zeros((max(5, args.steps), len(sph.KERNELS)))
    for i in range(ktimes_all.shape[0]):
        flush_l2()
        sim.step(1)
        ktimes_all[i] = _reported(sim.kernel_times, domain, sph)
    kmean = ktimes_all.mean(axis=0)
    shares = {k: float(v) for k, v in zip(sph.KERNELS, kmean / kmean.sum())}
    dom = int(np.argmax(kmean))
    dom_name = sph.KERNELS[dom]
    clock_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    alu_nominal = SMS * FP32_LANES_PER_SM * 2 * clock_mhz * 1e6 / 1e12      # TFLOP/s
    alu_peak = sph.measure_fp32_fma(local)                                  # measured here
    # the dominant kernel's duration in the timed region itself (its events are recorded there)
    t_dom = (density_live_ms if dom_name == "density" else kmean[dom]) / 1e3
    if dom_name == "force":
        flops = FORCE_FLOPS_PER_PAIR * (pairs - n_all)
    elif dom_name == "density":
        flops = DENSITY_FLOPS_PER_PAIR * pairs
    else:
        flops = None
    if flops is not None:
        achieved = flops / t_dom / 1e12
        roofline = {"bound": "alu", "kernel": dom_name, "achieved": achieved, "peak": alu_peak,
                    "unit": "TFLOP/s", "frac": achieved / alu_peak,
                    "traffic": None if args.low_latency else _traffic(dom_name),
                    "flops_per_pair": (DENSITY_FLOPS_PER_PAIR if dom_name == "density"
                                       else FORCE_FLOPS_PER_PAIR),
                    "pairs_per_launch": pairs if dom_name == "density" else pairs - n_all,
                    "mean_neighbours": mean_nbrs,
                    "peak_source": "measured: FP32 FMA probe kernel (sph_measure_fp32_fma, "
                                   "full occupancy, best of 5, CUDA events)",
                    "peak_nominal": alu_nominal}
    else:
        bytes_ = FORCE_BYTES_PER_PARTICLE * n_all
        achieved = bytes_ / t_dom / 1e9
        roofline = {"bound": "hbm", "kernel": dom_name, "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                    "traffic": None if args.low_latency else _traffic(dom_name)}
    force_hbm = FORCE_BYTES_PER_PARTICLE * n_all / (kmean[6] / 1e3) / 1e9
    density_hbm = DENSITY_BYTES_PER_PARTICLE * n_all / (density_live_ms / 1e3) / 1e9
    step_hbm = BYTES_PER_PARTICLE_STEP * n_all / (ms_per_step / 1e3) / 1e9

    # end to end through the public API: host pose in, one substep, host wrench out, as a
    # user's haptic loop runs it (the per-kernel profiling events off: the plain graph of
    # one substep and the update cycle's end)
    sim.set_profiling(False)
    sim.step(1)                               # untimed: captures that graph
    _reported(sim.sync, domain, sph)
    path = sc.trajectory
    e2e_s = 0.0
    pose_h = torch.empty(13, dtype=torch.float32).pin_memory().numpy()
    wrench_h = np.zeros(6, np.float64)
    grab_id = sim.body_ids[sc.grab_body]
    done = int(sim.info()[4])                 # substeps so far: the path continues from here
    for i in range(args.steps):
        flush_l2()
        torch.cuda.synchronize()
        row = path[min(done + i, path.shape[0] - 1)]
        t0 = time.perf_counter()
        pose_h[:] = row
        try:
            sim.haptic_cycle(grab_id, pose_h[:7], pose_h[7:], 1, out=wrench_h)
        except sph.SphError as e:         # particles over the walls: counted, state valid
            if e.status != sph.ERR_DOMAIN:
                raise
            domain[0] += 1
        e2e_s += time.perf_counter() - t0
    if (domain[0] or rec_domain[0]) and args.workload == "coupled" and not args.fluid:
        # a particle left the grid domain: the workload is not the one this line describes
        # (the other workloads splash by design -- the dam break's jet -- and report the count)
        raise RuntimeError(f"{domain[0] + rec_domain[0]} out-of-domain reports during the run")
    e2e_s = max_over_ranks(e2e_s)
    e2e_value = job_rate(sc.n_fluid * args.steps, world, e2e_s)
    sim.close()

    # CPU baseline (rank 0, N = 1), after every GPU timing so that the host's OpenMP
    # threads run alone: the oracle as it stands, one substep, host cores; its wrench is
    # also the FP64 reference of the first substep's grab wrench.
    cpu = None
    wrench_err = None
    acc_parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t_cpu, out, m_sorted = _oracle_substep_time(sc)
        ref_wrench = out["wrench"][sc.grab_body]
        cpu = {"value": sc.n_fluid / t_cpu, "unit": UNIT, "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": f"1 substep of the full coupled scene ({sc.n_total} particles), "
                         f"FP64 uniform-grid oracle, {t_cpu:.2f} s"}
        cpu["modes"] = _oracle_modes()
        fe = np.linalg.norm(w_gpu[:3] - ref_wrench[:3]) / max(np.linalg.norm(ref_wrench[:3]), 1e-30)
        te = np.linalg.norm(w_gpu[3:] - ref_wrench[3:]) / max(np.linalg.norm(ref_wrench[3:]), 1e-30)
        kap = _cancellation(sc, out, m_sorted, sc.grab_body)
        wrench_err = {"force_rel": float(fe), "torque_rel": float(te),
                      "kappa_force": kap["kappa_force"], "kappa_torque": kap["kappa_torque"]}
        # every particle's acceleration of the first substep against the oracle's
        acc_ref = np.empty_like(out["acc"])
        acc_ref[out["id"]] = out["acc"]
        rel = (np.linalg.norm(acc_first.astype(np.float64) - acc_ref, axis=1)
               / np.maximum(np.linalg.norm(acc_ref, axis=1), 0.1 * 9.81))
        acc_parity = {"bar": "|da| <= 1e-4 max(|a|, 0.1 g), every particle",
                      "particles": int(rel.size), "frac_within": float(np.mean(rel <= 1e-4)),
                      "max_rel": float(rel.max()), "what": "first substep, record flag, all "
                      "particle kinds, against the FP64 grid oracle"}

    forms = {}
    if not args.no_forms:
        def factory(st):
            def f():
                with torch.cuda.stream(st):
                    flush.fill_(1)
            return f
        forms["batched"] = batched_form(args, factory)
        forms["surrogate"] = surrogate_form(args)
        from paper_2511_15908_gb300 import sph as _sph
        forms["tait_eos"] = variant_form(
            args, sc, factory, _sph.FLAG_TAIT,
            "same workload with SPH_FLAG_TAIT (p = B((rho/rho0)^7 - 1), B = k rho0 / 7)")
        forms["volume_boundary"] = variant_form(
            args, sc, factory, _sph.FLAG_VOLUME_BOUNDARY,
            "same workload with SPH_FLAG_VOLUME_BOUNDARY (boundary weights psi = rho0 / "
            "sum_boundary W; the density interval includes the psi pass)")
        forms["isosurface"] = isosurface_form(args, sc)
        forms["cloth"] = cloth_form(args, factory)
        forms["size_sweep"] = size_sweep_form(args, factory, sc)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 (f64 wrench/momentum reductions)", "data": "synthetic",
                "config": {"workload": _workload_name(args.workload, sc), "particles_all": n_all,
                           "particles_fluid": sc.n_fluid, "l2": "flushed between steps",
                           "parallelism": f"replicas x{world}",
                           "all_particle_steps_per_s": value * n_all / sc.n_fluid,
                           "regime": f"stirred: timed after {SPIN_UP_SUBSTEPS + 1 + args.warmup} "
                                     "untimed substeps of the probe's random walk from the "
                                     "settled fill",
                           "out_of_domain_reports": domain[0],
                           "density_pass": ("low latency: 32 or 16 threads per particle"
                                            if args.low_latency else "one thread per particle")},
                # per timed substep: hash, single-pass scan, scatter, rank + gather, density,
                # force, wrench, cycle end
                "gpu_launches": 8 * args.steps,
                "kernel_ms": {k: float(v) for k, v in zip(sph.KERNELS, kmean)},
                "kernel_share": shares,
                "kernel_ms_source": "a pass of the same substeps after the timed region, events "
                                    "around every kernel (the timed region records the density "
                                    "pass's alone)",
                "density_ms_timed_region": density_live_ms,
                "roofline": roofline,
                "hbm_step": {"bytes_per_particle": BYTES_PER_PARTICLE_STEP,
                             "achieved_gbs": step_hbm, "peak_gbs": peaks["hbm_gbs"],
                             "frac": step_hbm / peaks["hbm_gbs"]},
                "force_hbm_frac": force_hbm / peaks["hbm_gbs"],
                "density_hbm": {"bytes_per_particle": DENSITY_BYTES_PER_PARTICLE,
                                "achieved_gbs": density_hbm, "frac": density_hbm / peaks["hbm_gbs"]},
                "grab_wrench_err_vs_oracle": wrench_err,
                "acc_parity": acc_parity,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 64,
                        "d2h_bytes_per_step": 60,
                        "what": "sph_haptic_cycle: host pose and velocity in (as kernel "
                                "arguments), one substep, host wrench out (synchronising); "
                                "per-kernel profiling off, as in a user's haptic loop"},
                "clocks": clk.summary(),
                "cpu_baseline": cpu,
                "forms": forms}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="coupled", choices=["coupled", "stirring", "dam_break"])
    ap.add_argument("--fluid", type=int, default=0,
                    help="coupled scene on a shorter tank with this many fluid particles (profiling)")
    ap.add_argument("--low-latency", action="store_true",
                    help="run the workload with SPH_FLAG_LOW_LATENCY (small scenes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / surrogate forms")
    ap.add_argument("--sur-substeps", type=int, default=32000)
    ap.add_argument("--sur-dam-episodes", type=int, default=2000)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
