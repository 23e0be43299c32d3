"""Throughput of the DISCOS wall-bounded hot path on GB300.

Workload (one GPU, the default): a 256 x 128 x 256 channel with a conducting
(Dirichlet) bottom wall and a dielectric (Neumann) top wall, 400,000 +-1
ions, l_B = 0.96, E_x = 0.02, the full wet step (cell list, charge
spreading, Poisson, field interpolation, P3M near field with images, LJ and
wall forces, force spreading with RFD thermal forcing, stochastic stress,
staggered Stokes, two velocity interpolations, midpoint update with the
near-wall dry tensor), single-precision bulk with double wall-normal solves.
One step = one pass of that path over all ions.  `--workload
wet_channel_128x64x128` selects the 128 x 64 x 128 Neumann channel with
20,000 ions instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME]

Under torchrun each rank runs an independent replica (the path does not
shard; replicas only) and rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ion-timesteps/s"
WORKLOADS = {
    "iceo_channel_256x128x256": "iceo_channel_256x128x256: 256x128x256 cells, conducting bottom and dielectric "
                                "top wall, 400000 ions, full wet step, FP32+FP64 islands",
    "wet_channel_128x64x128": "wet_channel_128x64x128: 128x64x128 cells, Neumann walls, 20000 ions, "
                              "full wet step, FP32+FP64 islands",
}
DEFAULT_WORKLOAD = "iceo_channel_256x128x256"


def whole_job_rate(units_local, t_ms_local, dist=None, device="cpu"):
    """Units processed by all ranks per second of the slowest rank (each rank
    runs its own replica: weak scaling, no collective on the data path).
    Returns (rate, max time over ranks in ms)."""
    if dist is None:
        return units_local / (t_ms_local * 1e-3), t_ms_local
    import torch
    t = torch.tensor([float(t_ms_local)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / (float(t.item()) * 1e-3), float(t.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def clocks_sampler():
    """Start nvidia-smi sampling of clocks and throttle reasons; returns a stop fn."""
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    path = os.path.join("/tmp", f"discos_clocks_{os.getpid()}.csv")
    try:
        f = open(path, "w")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "50"],
                             stdout=f, stderr=subprocess.DEVNULL)
    except Exception:
        return lambda dev: None

    def stop(dev):
        p.terminate()
        try:
            p.wait(timeout=5)
        except Exception:
            p.kill()
        f.close()
        with open(path) as lines:
            return parse_clocks(lines, dev)
    return stop


def parse_clocks(lines, dev):
    """Summary of nvidia-smi samples (the query of clocks_sampler, csv without
    header or units) for GPU `dev`: median SM clock under load, the maximum
    SM clock, and every throttle reason seen active; None without samples."""
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [s.strip() for s in line.split(",")]
        if len(parts) < 9 or parts[0] != str(dev):
            continue
        try:
            sm.append(float(parts[1]))
            mx = float(parts[2])
        except ValueError:
            continue
        for n, v in zip(names, parts[5:9]):
            if v.lower() == "active":
                reasons.add(n)
    if not sm:
        return None
    sm.sort()
    return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# Conjugate-gradient iterations the oracle's Poisson solve (rtol 1e-13,
# oracle/poisson.py) takes on the 256 x 128 x 256 channel's charge density of
# this workload (1233 when run to convergence once: 409 s with per-iteration
# residual checks, about 240 s without).  The baseline below times 40 of them
# at full size and scales to this count rather than spending minutes per run.
ORACLE_CG_ITERATIONS = {"iceo_channel_256x128x256": 1233}


def cpu_baseline(workload=DEFAULT_WORKLOAD, small_seconds=12.0):
    """Time the FP64 oracle (as it stands) on a bounded sample, single-threaded.

    256 x 128 x 256 channel: the full-size electrostatic stage of one step --
    charge spreading of all 400,000 ions (timed), the CG Poisson solve (40
    iterations timed, scaled to the iteration count of a full solve), the
    field interpolation to all ions (timed) and the brute-force near field
    with images (400 target ions timed, scaled to all ions).  The oracle's
    Stokes solve (sparse LU of the 25M-unknown MAC system) is not run at this
    size, so the figure is an upper bound of the oracle's rate for the full
    wet step.  Other workloads: whole oracle wet steps of a 32 x 16 x 16
    channel with 300 ions."""
    if workload == "iceo_channel_256x128x256":
        code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, os.path.join({ROOT!r}, 'tests'))
import numpy as np
import scipy.sparse.linalg as spla
from paper_2204_14167_gb300 import presets, synth
from helpers import oracle_params
from oracle import gridops, poisson, particles
cfg, rec = presets.iceo_channel_256x128x256()
pos, q, sp = synth.ions(cfg.dims, rec['n_pos'], rec['n_neg'], rec['seed'], rec['ymargin'], rec['min_sep'])
p = oracle_params(cfg)
N = pos.shape[1]
t0 = time.perf_counter(); rho = gridops.spread_charge(p['kernel_es'], pos, q, cfg.dims, cfg.bc); t_spread = time.perf_counter() - t0
A = poisson.assemble(cfg.dims, cfg.bc)
b = poisson.rhs(rho, cfg.bc, cfg.phi_b, poisson.wall_slopes(cfg.bc, cfg.surf_charge, cfg.lB), cfg.lB).ravel()
t0 = time.perf_counter(); phi, info = spla.cg(A, b, rtol=1e-13, atol=0.0, maxiter=40); t_cg = time.perf_counter() - t0
phi = phi.reshape(rho.shape)
slopes = poisson.wall_slopes(cfg.bc, cfg.surf_charge, cfg.lB)
t0 = time.perf_counter(); gridops.efield_at_ions(p['kernel_es'], pos, phi, cfg.bc, cfg.phi_b, slopes); t_interp = time.perf_counter() - t0
tg = np.arange(0, N, N // 400)
t0 = time.perf_counter(); particles.near_field(pos, q, sp, p, p['fp_table'], targets=tg); t_near = time.perf_counter() - t0
print(json.dumps(dict(N=N, t_spread=t_spread, t_cg40=t_cg, t_interp=t_interp, t_near=t_near, n_near=len(tg))))
"""
    else:
        code = f"""
import os, sys, time, json
sys.path.insert(0, {ROOT!r}); sys.path.insert(0, os.path.join({ROOT!r}, 'tests'))
import numpy as np
from paper_2204_14167_gb300 import presets, synth
from helpers import oracle_params
from oracle import integrate
cfg, rec = presets.wet_channel_small()
pos, q, sp = synth.ions(cfg.dims, rec['n_pos'], rec['n_neg'], rec['seed'], rec['ymargin'], rec['min_sep'])
p = oracle_params(cfg)
integrate.wet_step(p, pos, q, sp, 0)
t0 = time.perf_counter(); n = 0
while time.perf_counter() - t0 < {small_seconds}:
    pos, F, c, _ = integrate.wet_step(p, pos, q, sp, n + 1); n += 1
dt = time.perf_counter() - t0
print(json.dumps(dict(steps=n, seconds=dt, ions=int(pos.shape[1]))))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1200)
    if r.returncode != 0:
        return {"value": None, "unit": METRIC, "cores": 1, "kind": "oracle", "error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    if workload == "iceo_channel_256x128x256":
        iters = ORACLE_CG_ITERATIONS[workload]
        t_step = d["t_spread"] + d["t_cg40"] / 40.0 * iters + d["t_interp"] + d["t_near"] * d["N"] / d["n_near"]
        sample = (f"full-size electrostatic stage of one oracle step on the 256x128x256 channel, "
                  f"{d['N']} ions: spread {d['t_spread']:.1f} s, CG 40 iterations {d['t_cg40']:.1f} s "
                  f"scaled to {iters}, interpolation {d['t_interp']:.1f} s, near field {d['n_near']} ions "
                  f"{d['t_near']:.1f} s scaled to all; Stokes stage not run (upper bound); single thread")
        return {"value": d["N"] / t_step, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample,
                "seconds_per_step": t_step}
    return {"value": d["ions"] * d["steps"] / d["seconds"], "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{d['steps']} FP64 oracle wet steps of a 32x16x16 channel with {d['ions']} ions "
                      f"({d['seconds']:.1f} s, single thread)"}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    # one bounded sample (the full-size sample already takes about 30 s; the
    # step count does not change what it measures)
    b = cpu_baseline(args.workload, small_seconds=max(2.0, 20.0 / max(args.steps, 1)))
    v = b.get("value")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": b["seconds_per_step"] * 1e3 if b.get("seconds_per_step") else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "reference_sample": b.get("sample")},
            "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": b.get("sample")},
            "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    cfg, rec = getattr(presets, args.workload)(dg.MIXED)
    cfg.seed = cfg.seed + rank
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"] + rank, rec["ymargin"], rec["min_sep"])
    N = pos.shape[1]
    h = dg.Discos(cfg)
    x = torch.tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    shape = h.tune_transforms()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")   # > L2 (129 MB)
    stream = torch.cuda.current_stream()
    step = 0
    for _ in range(args.warmup):
        h.step(x, qd, step0=step, nsteps=1)
        step += 1
    torch.cuda.synchronize()

    # dominant kernel family (by per-step time), then the timed region with a
    # live event probe on that family
    # clock samples from here to the end of the timed region (the probe
    # pre-pass keeps the GPU under the same load while nvidia-smi starts)
    stop_clocks = clocks_sampler()
    breakdown, step = kernel_breakdown(dg, h, x, qd, step)
    dominant = max(breakdown, key=breakdown.get)
    dg.probe(h, dominant)

    # device-timed region: K steps, L2 flushed between steps (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n_launch0 = dg.launch_count()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts[k].record(stream)
        h.step(x, qd, step0=step, nsteps=1)
        ends[k].record(stream)
        step += 1
    torch.cuda.synchronize()
    n_launches = dg.launch_count() - n_launch0
    if dist:
        dist.barrier()
    clocks = stop_clocks(dev)
    t_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    probe_ms, probe_n = dg.probe_read(h)
    dg.probe(h, None)
    value, t_ms = whole_job_rate(N * args.steps, t_ms, dist, "cuda")
    ms_per_step = t_ms / args.steps

    # end to end through the public API with host buffers: pinned H2D of the
    # step's positions and charges, the step, D2H of the new positions; the
    # same L2 policy as the device-timed loop (flushed between steps, outside
    # the events)
    xh = torch.tensor(pos, dtype=torch.float32).pin_memory()
    qh = torch.tensor(q, dtype=torch.float32).pin_memory()
    out_h = torch.empty_like(xh).pin_memory()
    starts2 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends2 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.fill_(float(k))
        starts2[k].record(stream)
        x.copy_(xh, non_blocking=True)
        qd.copy_(qh, non_blocking=True)
        h.step(x, qd, step0=step, nsteps=1)
        out_h.copy_(x, non_blocking=True)
        ends2[k].record(stream)
        step += 1
    torch.cuda.synchronize()
    e2e_ms = sum(s.elapsed_time(e) for s, e in zip(starts2, ends2))
    e2e = {"value": whole_job_rate(N * args.steps, e2e_ms, dist, "cuda")[0], "unit": METRIC,
           "h2d_bytes_per_step": int(xh.numel() * 4 + qh.numel() * 4),
           "d2h_bytes_per_step": int(out_h.numel() * 4)}

    peaks = _peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    nbytes = algorithmic_bytes(dominant, cfg, N)
    avg_s = probe_ms * 1e-3 / max(probe_n, 1)
    achieved = nbytes / avg_s / 1e9 if nbytes else None
    rl = {"roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                       "frac": achieved / peak if achieved else None, "traffic": MEASURED_TRAFFIC[args.workload].get(dominant),
                       "algorithmic_bytes_per_launch": nbytes, "avg_launch_us": avg_s * 1e6,
                       "launches_timed": probe_n, "peak_source": "measured" if peaks else "fallback"},
          "stages_ms": {k: round(v, 5) for k, v in breakdown.items()}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOADS[args.workload], "ions": N, "grid": [cfg.Nx, cfg.Ny, cfg.Nz],
                           "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas{ws}",
                           "transform_shape": {"fx_pairs": shape[0], "fx_threads": shape[1], "fz_tile": shape[2]}},
                "clocks": clocks, "e2e": e2e, "roofline": rl.get("roofline"), "stages_ms": rl.get("stages_ms"),
                "gpu_launches": int(n_launches), "device_fault": h.fault(sync=True)}
        if not args.no_forms and ws == 1:
            line["production_forms"] = production_forms()
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def production_forms(steps=20):
    """The production forms beside the headline, each on its own workload:
    the 128 x 64 x 128 channel in both precisions (and the force difference
    between them); the 256 x 128 x 256 channel on the plain FP64 path and in
    mixed precision with residual refinement of every Poisson and Stokes
    solve, with their force and one-step displacement differences against
    FP64; the same channel in the paper's ICEO geometry (both walls dielectric,
    a metal strip in the bottom wall); batched replicas against the plain
    single-channel path stepping the same replicas one by one; and the
    differentiable energy (forward + hand-written backward)."""
    import torch

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}

    def guarded(name, fn):
        try:
            fn()
        except Exception as exc:       # an auxiliary measurement never hides the headline line
            out[name] = {"error": f"{type(exc).__name__}: {exc}"}
        torch.cuda.synchronize()
        torch.cuda.empty_cache()

    guarded("wet_channel_128x64x128", lambda: _wet128(out, timed, steps))
    guarded("iceo_channel_256x128x256", lambda: _iceo(out, timed))
    guarded("iceo_strip_256x128x256", lambda: _strip(out, timed))
    guarded("batched_replicas_512x32^3", lambda: _batched(out, timed))
    guarded("energy_forward_backward_64^3_fp64", lambda: _energy(out, timed))
    return out


def _stepper(h, x, q, counter):
    def f():
        h.step(x, q, step0=counter[0], nsteps=1)
        counter[0] += 1
    return f


def _wet128(out, timed, steps):
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth
    cfg, rec = presets.wet_channel_128x64x128(dg.FP64)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    N = pos.shape[1]
    h64 = dg.Discos(cfg)
    x64 = torch.tensor(pos, dtype=torch.float64, device="cuda")
    q64 = torch.tensor(q, dtype=torch.float64, device="cuda")
    cfgm, _ = presets.wet_channel_128x64x128(dg.MIXED)
    hm = dg.Discos(cfgm)
    hm.tune_transforms()
    xm, qm = x64.float().contiguous(), q64.float()
    err = float(torch.linalg.norm(hm.forces(xm, qm).double() - h64.forces(x64, q64)) /
                torch.linalg.norm(h64.forces(x64, q64)))
    c = [0]
    _stepper(hm, xm, qm, c)()
    msm = timed(_stepper(hm, xm, qm, c), steps)
    _stepper(h64, x64, q64, c)()
    ms64 = timed(_stepper(h64, x64, q64, c), max(steps // 2, 3))
    out["wet_channel_128x64x128"] = {"ions": N, "mixed_ion_steps_per_s": N / (msm * 1e-3), "mixed_ms_per_step": msm,
                                     "fp64_ion_steps_per_s": N / (ms64 * 1e-3), "fp64_ms_per_step": ms64,
                                     "mixed_vs_fp64_force_rel_l2": err,
                                     "device_fault": [hm.fault(sync=True), h64.fault(sync=True)]}


def _iceo(out, timed):
    import numpy as np
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth
    # the 256 x 128 x 256 channel with 400k ions: FP64 against mixed precision
    # with one sweep of residual refinement of every Poisson and Stokes solve
    c5, r5 = presets.iceo_channel_256x128x256(dg.FP64)
    p5, q5, _ = synth.ions(c5.dims, r5["n_pos"], r5["n_neg"], r5["seed"], r5["ymargin"], r5["min_sep"])
    N5 = p5.shape[1]
    h5d = dg.Discos(c5)
    c5r, _ = presets.iceo_channel_256x128x256(dg.MIXED)
    c5r.max_refine = 1
    h5r = dg.Discos(c5r)
    h5r.tune_transforms()
    c5m, _ = presets.iceo_channel_256x128x256(dg.MIXED)
    h5m = dg.Discos(c5m)
    x5m = torch.tensor(p5, dtype=torch.float32, device="cuda").contiguous()
    q5m = torch.tensor(q5, dtype=torch.float32, device="cuda")
    x5d, q5d = x5m.double().contiguous(), q5m.double()
    F5d = h5d.forces(x5d, q5d)
    nF = torch.linalg.norm(F5d)
    err_m = float(torch.linalg.norm(h5m.forces(x5m, q5m).double() - F5d) / nF)
    err_r = float(torch.linalg.norm(h5r.forces(x5m, q5m).double() - F5d) / nF)
    # one step from the same state: displacement difference against FP64
    xa, xb = x5m.clone(), x5d.clone()
    h5r.step(xa, q5m, step0=3, nsteps=1)
    h5d.step(xb, q5d, step0=3, nsteps=1)
    torch.cuda.synchronize()
    stokes_hist = h5r.refine_history_stokes()
    poisson_hist = h5r.refine_history()

    def disp(a, b0):
        d = a.double() - b0.double()
        for ax, L in ((0, c5.Nx), (2, c5.Nz)):
            d[ax] -= L * torch.round(d[ax] / L)
        return d
    dref = disp(xb, x5d)
    derr = float(torch.linalg.norm(disp(xa, x5d) - dref) / torch.linalg.norm(dref))
    c = [10]
    _stepper(h5r, x5m, q5m, c)()
    msr = timed(_stepper(h5r, x5m, q5m, c), 10)
    _stepper(h5d, x5d, q5d, c)()
    msd = timed(_stepper(h5d, x5d, q5d, c), 3)
    out["iceo_channel_256x128x256"] = {
        "ions": N5, "fp64_ion_steps_per_s": N5 / (msd * 1e-3), "fp64_ms_per_step": msd,
        "mixed_refined_ion_steps_per_s": N5 / (msr * 1e-3), "mixed_refined_ms_per_step": msr,
        "mixed_vs_fp64_force_rel_l2": err_m, "mixed_refined_vs_fp64_force_rel_l2": err_r,
        "mixed_refined_vs_fp64_step_rel_l2": derr,
        "poisson_residual_history": poisson_hist, "stokes_residual_history": stokes_hist,
        "device_fault": [h5r.fault(sync=True), h5d.fault(sync=True)]}


def _strip(out, timed):
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth
    cfg, rec = presets.iceo_strip_256x128x256(dg.MIXED)
    pos, q, _ = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    h = dg.Discos(cfg)
    h.tune_transforms()
    x = torch.tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    c = [0]
    _stepper(h, x, qd, c)()
    ms = timed(_stepper(h, x, qd, c), 10)
    N = pos.shape[1]
    out["iceo_strip_256x128x256"] = {"ions": N, "mixed_ion_steps_per_s": N / (ms * 1e-3), "mixed_ms_per_step": ms,
                                     "strip_columns": [cfg.strip_x[0], cfg.strip_x[1]],
                                     "device_fault": h.fault(sync=True)}


def _batched(out, timed):
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets
    # batched replicas: 512 channels of 32^3, 64..512 ions each
    cfgb, recb = presets.batched_channels_32()
    posb, qb, spb, off = presets.batched_ions(cfgb, recb)
    hb = dg.Discos(cfgb)
    xb = torch.tensor(posb, dtype=torch.float32, device="cuda").contiguous()
    qbd = torch.tensor(qb, dtype=torch.float32, device="cuda")
    R = len(off) - 1
    hist = torch.zeros((R, 1, cfgb.Ny), dtype=torch.int32, device="cuda")
    sums = torch.zeros((R, 4), dtype=torch.float64, device="cuda")
    b = hb.make_batch(xb, qbd, off, hist=hist, sums=sums)
    spl, _ = hb.tune_batched(b, trial_steps=32)
    K = 64
    bst = [0]

    def bstep():
        hb.step_batched(b, step0=bst[0], nsteps=K)
        bst[0] += K
    bstep()
    msb = timed(bstep, 2) / K
    # the same replicas through the single-channel path, one replica at a time
    nrep = 8
    xs = [xb[:, off[r]:off[r + 1]].contiguous() for r in range(nrep)]
    qs = [qbd[off[r]:off[r + 1]].contiguous() for r in range(nrep)]

    def plain_reps():
        for r in range(nrep):
            hb.step(xs[r], qs[r], step0=0, nsteps=1)
    plain_reps()
    msp = timed(plain_reps, 5)
    ions_sub = off[nrep]
    out["batched_replicas_512x32^3"] = {
        "ion_steps_per_s": off[-1] / (msb * 1e-3), "ms_per_step": msb, "ions": off[-1], "replicas": R,
        "steps_per_launch": spl, "graph": True,
        "plain_single_channel_ion_steps_per_s": ions_sub / (msp * 1e-3), "device_fault": hb.fault(sync=True)}



def _energy(out, timed):
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth
    from paper_2204_14167_gb300.autograd import energy as denergy
    # differentiable energy on 64^3 with 4096 ions
    cfge, rece = presets.energy_channel_64(dg.FP64)
    pose, qe, _ = synth.ions(cfge.dims, rece["n_pos"], rece["n_neg"], rece["seed"], rece["ymargin"], rece["min_sep"])
    he = dg.Discos(cfge)
    xe = torch.tensor(pose, dtype=torch.float64, device="cuda").requires_grad_(True)
    qe_ = torch.tensor(qe, dtype=torch.float64, device="cuda").requires_grad_(True)
    pb = torch.tensor(cfge.phi_b, dtype=torch.float64, requires_grad=True)

    def fb():
        U = denergy(he, xe, qe_, pb)
        U.backward()
    fb()
    mse = timed(fb, 10)
    out["energy_forward_backward_64^3_fp64"] = {"ms_per_call": mse, "ions": int(pose.shape[1])}


def run_profile(args):
    """The bench workload's steps alone: a short, fixed launch sequence for ncu."""
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets, synth
    cfg, rec = getattr(presets, args.workload)(dg.MIXED)
    pos, q, sp = synth.ions(cfg.dims, rec["n_pos"], rec["n_neg"], rec["seed"], rec["ymargin"], rec["min_sep"])
    h = dg.Discos(cfg)
    if args.transform_shape:
        h.set_transform_shape(*[int(v) for v in args.transform_shape.split(",")])
    else:
        h.tune_transforms()
    x = torch.tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    n0 = dg.launch_count()
    h.step(x, qd, step0=0, nsteps=args.warmup)
    torch.cuda.synchronize()
    n1 = dg.launch_count()
    h.step(x, qd, step0=args.warmup, nsteps=args.steps)
    torch.cuda.synchronize()
    print(f"profile: {n1 - n0} warm-up launches, {dg.launch_count() - n1} measured launches")


def run_profile_batched(args):
    """Batched replicas alone for ncu: 152 replicas of 32^3 (one per SM), one
    launch per step, no graph."""
    import torch
    import paper_2204_14167_gb300 as dg
    from paper_2204_14167_gb300 import presets
    cfg, rec = presets.batched_channels_32(R=152)
    pos, q, sp, off = presets.batched_ions(cfg, rec)
    h = dg.Discos(cfg)
    x = torch.tensor(pos, dtype=torch.float32, device="cuda").contiguous()
    qd = torch.tensor(q, dtype=torch.float32, device="cuda")
    b = h.make_batch(x, qd, off)
    h.set_batched_shape(1)
    for k in range(args.warmup + args.steps):
        h.step_batched(b, step0=k, nsteps=1)
    torch.cuda.synchronize()
    print(f"profile-batched: {off[-1]} ions in {len(off) - 1} replicas, {args.warmup + args.steps} launches, "
          f"fault word {h.fault(sync=True)}")


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


# DRAM bytes (read + write) per launch from ncu captures of the current kernels
# on the 256 x 128 x 256 channel (the per-kernel summary of that channel under
# profiles/), averaged over a step's launches of the family; a family whose
# kernel changed after its capture has no entry (reported as null), and the
# 128 x 64 x 128 channel has none
MEASURED_TRAFFIC = {"wet_channel_128x64x128": {},
                    "iceo_channel_256x128x256": {"fft_z": 100.7e6, "fft_x": 98.3e6, "stokes_y": 451.6e6,
                                                 "spread_force": 156.3e6, "interp_v": 111.5e6,
                                                 "interp_e": 45.0e6, "spread_charge": 40.0e6, "near_field": 8.5e6}}


def algorithmic_bytes(family, cfg, N):
    """Bytes one launch of a kernel family must move at minimum (float32 bulk
    data, float64 factor tables of the low modes ignored), for the workload's
    sizes.  G = Nx Ny Nz cells, M = (Nx/2+1) Nz transverse modes."""
    Nx, Ny, Nz = cfg.Nx, cfg.Ny, cfg.Nz
    G = Nx * Ny * Nz
    Gf = Nx * Nz * (3 * Ny + 1)
    M = (Nx // 2 + 1) * Nz
    w = 4 if cfg.kernel_hy == 0 else 6
    we = 4 if cfg.kernel_es == 0 else 6
    if family == "stokes_y":      # spectra in and out, 4 single-precision factor rows per mode row
        return M * (2 * (3 * Ny + 1) * 8 + 4 * Ny * 4 + 20)
    if family == "poisson_y":
        return M * (2 * Ny * 8 + Ny * 4)
    if family == "fft_z":         # per launch, averaged over the Poisson (1 field) and Stokes (3 fields) launches
        return (Nz * Ny * M // Nz * 8 * 2 + Nz * (3 * Ny + 1) * M // Nz * 8 * 2) // 2
    if family == "fft_x":
        return (G * 4 + G // Nx * (Nx // 2 + 1) * 8 + Gf * 4 + Gf // Nx * (Nx // 2 + 1) * 8) // 2
    if family == "noise":
        return Gf * 4
    # gathers and scatters: each grid value read (or read and written) once,
    # plus the per-ion data; a stencil point shared by several ions is
    # counted once (the rest is L2 reuse, not DRAM traffic)
    if family == "interp_v":      # velocity grid in; position, index in; velocity out
        return Gf * 4 + N * (12 + 4 + 12)
    if family == "interp_e":      # potential in; position, charge, near-field force, index in; force out
        return G * 4 + N * (12 + 4 + 12 + 4 + 12)
    if family == "spread_force":  # accumulates into the noise-initialised forcing: read and write it
        return 2 * Gf * 4 + N * (12 + 12 + 4 + 4)
    if family == "spread_charge":  # density written; position and charge in
        return G * 4 + N * 16
    if family == "near_field":
        return N * (16 + 12 + 12)
    if family == "cell_list":
        return N * (12 + 4 * 4)
    if family == "update":
        return N * (12 * 4)
    return None


def kernel_breakdown(dg, h, x, qd, step0, steps=3):
    """Per-step time of every kernel family (CUDA events on the launching
    streams), measured outside the timed region to pick the dominant one."""
    from paper_2204_14167_gb300 import _lib
    out = {}
    step = step0
    for fam in _lib.PROBE_FAMILIES:
        dg.probe(h, fam)
        for _ in range(steps):
            h.step(x, qd, step0=step, nsteps=1)
            step += 1
        t, n = dg.probe_read(h)
        out[fam] = t / steps
    dg.probe(h, None)
    return out, step


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the production-form measurements")
    ap.add_argument("--profile-batched", action="store_true",
                    help="run only batched-replica steps (for ncu)")
    ap.add_argument("--profile", action="store_true",
                    help="only W warm-up steps and K steps of the workload (for ncu), no timing output")
    ap.add_argument("--transform-shape", default="",
                    help="with --profile: x pairs, x threads, z tile (as tuned by the bench) instead of tuning")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
    elif args.profile_batched:
        run_profile_batched(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
