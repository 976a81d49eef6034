"""Benchmark of the radiative-equilibrium hot path on one B300 (or N, one process per GPU).

A step is one radiative-equilibrium iteration over the whole workload: opacities, sublayer
optical depths, two-stream coefficients, 1 + n_scat down/up passes, Gauss-point and bin sums,
and the FP64 temperature step (helios_flux_sweep + helios_temp_update).  The workload is the
full-size single atmosphere: 100 layers (1e-6..1e3 bar) x 3000 wavenumber bins
(0.3-200 um) x 20 Gauss points, Rayleigh-like scattering, seeded synthetic k-table.
Each GPU process runs its own copy of that atmosphere (atmospheres are independent; no
collective on the data path): weak scaling.

value: Gcell/s, cell = (atmosphere, layer, bin, g) of one full RE iteration.
L2 is flushed (a 256 MB write) before every timed step; only the step is inside the events.

--impl reference: the FP64 CPU oracle (test infrastructure) timed on the host cores on a
bounded sample of the same workload, same metric and unit.
"""
import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RE-converged atmospheres/s & flux-sweep Gcell/s, batched+surrogate vs plain"
UNIT = "Gcell/s"
WORKLOAD = "full-size single atmosphere: 100 layers x 3000 bins x 20 g, scattering, 5 passes/step"


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ---- replicas: one process per GPU, each with its own atmospheres; the process group carries
# only the barriers around the timed region and the max-over-ranks time (atmospheres are
# independent, so there is no collective on the data path)
def init_replicas(world, local, backend="nccl"):
    if world > 1:
        import torch
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    """The largest of every rank's value of x (the job's time is its slowest rank's)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world, device):
    """The sum of every rank's value of x (units processed by the whole job)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_ids(rank, per_rank):
    """The atmospheres rank `rank` owns: disjoint shards of per_rank consecutive seeds."""
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# DRAM traffic (read + write) of one sweep-kernel launch on the full-size single atmosphere, from
# the ncu capture summarised in profiles/sweep_kernel_full_single_atmosphere.md, valid only for the
# kernel source it was taken on (sha256 prefix of csrc/helios_kernels.cuh); null otherwise.
SWEEP_TRAFFIC = {"kernels_sha256": "abf436c89c4d6f59", "bytes_per_launch": 63123200}


def kernel_source_hash():
    """Hash of the sweep kernel's source and its launch configuration (the recorded DRAM traffic
    holds only while both are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("helios_kernels.cuh", "helios_api.cu"):
        h.update(open(os.path.join(ROOT, "paper_1606_05474_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def algorithmic_counts(wl, n_passes):
    """Algorithmic work of one RE step (see the design notes, roofline section).

    bytes: warm-start upward fluxes read and written (4 B per column point), the k-table rows
    the profile touches (counted from the actual (iP, iT) corners), bolometric outputs.
    fp32: per sublayer 24 coefficient operations once per step plus 4 fused multiply-adds per
    pass (down and up recurrences); sfu: 3 per sublayer (exp, 2 reciprocals)."""
    cells = wl.cells
    subs = sum(2 * a.n_layers * a.n_bins for a in wl.atms) * wl.G
    pts = sum((2 * a.n_layers + 1) * a.n_bins for a in wl.atms) * wl.G
    fp32 = subs * (24 + 4 * n_passes)
    sfu = subs * 3
    return cells, pts, fp32, sfu


def touched_table_bytes(plan, wl, T):
    """Bytes of the k-table rows (iP, iT corners) the current profile touches, from the library's
    own index output (helios_interp_opacity)."""
    _, idx, _ = plan.interp_opacity(T, want_kappa=False)
    idx = idx.cpu().numpy()
    tot = 0
    for a in range(plan.A):
        rows = set()
        for iP, iT in idx[plan.pt_off[a]:plan.pt_off[a + 1]]:
            for dp in (0, 1):
                for dt in (0, 1):
                    rows.add((int(iP) + dp, int(iT) + dt))
        tot += len(rows) * int(plan.L[a]) * wl.G * 4
    return tot


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    init_replicas(world, local)
    import synth
    import paper_1606_05474_b300 as hp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = synth.config2()
    wl.atms[0].T_init = synth.perturbed_profile(wl.atms[0], 11 + rank, amp=200.0)
    ctx = hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(col_lanes=args.col_lanes))
    n_passes = plan.info.passes
    lanes = 32 if args.col_lanes == 32 else 16       # automatic: 16 lanes for 24..119 layers
    T = torch.from_numpy(np.asarray(wl.atms[0].T_init, np.float64)).to(dev)
    T0 = T.clone()
    state = plan.new_state()
    Fu = torch.empty(plan.info.interfaces, dtype=torch.float64, device=dev)
    Fd = torch.empty_like(Fu)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(warm):
        plan.re_step(T, state, warm=warm, out=(Fu, Fd))

    # warm-up (the first step starts the coupled stream from zero)
    step(False)
    for _ in range(args.warmup - 1):
        step(True)
    torch.cuda.synchronize()
    # prep, sweep groups, finalize (unless fused), post
    n_launch_per_step = 2 + plan.info.sweep_launches + (0 if plan.info.fused_finalize else 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)                                     # let the sampler attach before timing
    barrier(world)
    torch.cuda.synchronize()
    t_wall = time.time()
    for k in range(args.steps):
        flush.zero_()                                   # evict L2 between timed steps
        ev[k][0].record(stream)
        step(True)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.time() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # the sweep kernel's own time: the same steps again with events around the sweep launches
    # (kept out of the timed loop above: the events split the step's chain of dependent launches)
    n_sweep = min(args.steps, 500)
    plan.set_timing(n_sweep)
    for _ in range(n_sweep):
        flush.zero_()
        step(True)
    torch.cuda.synchronize()
    sweep_ms = list(plan.sweep_times(n_sweep))
    plan.set_timing(0)
    total_ms = float(np.sum(step_ms))
    total_ms = max_over_ranks(total_ms, world, dev)

    cells, pts, fp32, sfu = algorithmic_counts(wl, n_passes)
    value = cells * args.steps * world / (total_ms * 1e-3) / 1e9

    # ---- end to end: host temperatures in, host temperatures and status out, every step
    Th = torch.empty(plan.info.layers, dtype=torch.float64).pin_memory()
    Th.copy_(T.cpu())
    Sh = torch.empty(plan.A, dtype=torch.int32).pin_memory()
    e2e_ms = []
    e2e_steps = min(args.steps, 200)
    for k in range(e2e_steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        T.copy_(Th, non_blocking=True)
        step(True)
        Th.copy_(T, non_blocking=True)
        Sh.copy_(state["status"], non_blocking=True)
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
    e2e_total = float(np.sum(e2e_ms))
    e2e_total = max_over_ranks(e2e_total, world, dev)
    e2e_value = cells * e2e_steps * world / (e2e_total * 1e-3) / 1e9

    # ---- one full radiative-equilibrium solve from the start profile (context)
    solve = None
    if not args.no_solve:
        Ts = T0.clone()
        torch.cuda.synchronize()
        t0 = time.time()
        iters, status = plan.solve_re(Ts)
        torch.cuda.synchronize()
        dt = time.time() - t0
        solve = {"wall_s": round(dt, 4), "iters": int(iters.item()), "status": int(status.item()),
                 "atm_per_s": round(1.0 / dt, 3), "tol": 1e-7}

    # ---- the exact column solve (the limit of the passes, Sect. 2.2.3) against 1 + 4 passes, the
    # RE solve with it, and the post-processing spectrum (isothermal layers, Sect. 3) with
    # 1 + 80 passes against the exact solve; each sweep timed cold-start after an L2 flush
    direct = None
    if not args.no_solve:
        def time_sweeps(pl, Tt, npass, reps=20):
            pl.flux_sweep(Tt, n_passes=npass, warm=False, want_toa=True)
            pl.set_timing(reps)
            for _ in range(reps):
                flush.zero_()
                pl.flux_sweep(Tt, n_passes=npass, warm=False, want_toa=True)
            torch.cuda.synchronize()
            return round(float(np.median(pl.sweep_times(reps))), 5)
        Tc = Ts.clone()
        ms_dir, ms_pass = time_sweeps(plan, Tc, hp.DIRECT), time_sweeps(plan, Tc, n_passes)
        pd = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(direct=1))
        Td = T0.clone()
        torch.cuda.synchronize()
        t0 = time.time()
        it_d, st_d = pd.solve_re(Td)
        torch.cuda.synchronize()
        dt_d = time.time() - t0
        pp = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(iso_layers=1))
        # Sect. 2.6: the same 1 + 4 passes with the tabulated Planck and transmission functions
        pt = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(tabulate=1))
        ms_tab = time_sweeps(pt, Tc, n_passes)
        del pt
        direct = {"sweep_ms_exact": ms_dir, "sweep_ms_passes": ms_pass, "passes": n_passes,
                  "sweep_ms_passes_tabulated_functions": ms_tab,
                  "re_solve_exact": {"wall_s": round(dt_d, 4), "iters": int(it_d.item()), "status": int(st_d.item()),
                                     "max_dT_vs_passes_K": round(float((Td - Ts).abs().max()), 4)},
                  "post_processing_spectrum_ms": {"isothermal_layers_81_passes": time_sweeps(pp, Tc, 81),
                                                  "isothermal_layers_exact": time_sweeps(pp, Tc, hp.DIRECT)}}
        del pd, pp

    if rank != 0:
        return
    P = peaks()
    hbm = P.get("hbm_gbs", 6400.0)
    sweep_avg = float(np.mean(sweep_ms))
    warm_bytes = 2 * 4 * pts                        # read + write of the warm-start upward fluxes
    table_bytes = touched_table_bytes(plan, wl, T)
    alg_bytes = warm_bytes + table_bytes + 16 * plan.info.interfaces
    achieved = alg_bytes / (sweep_avg * 1e-3) / 1e9
    # FP32 and MUFU peaks measured on this device (helios_measure_peaks): T instructions/s
    fp32_tflops, sfu_tops = hp.measure_peaks(ctx)
    fp32_peak = fp32_tflops / 2.0                        # an FMA counts once as an instruction
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweep / f64 temperature step", "data": "synthetic",
        "config": {"workload": WORKLOAD, "atmospheres_per_gpu": 1, "layers": 100, "bins": 3000, "g": 20,
                   "passes_per_step": n_passes, "cells_per_step_per_gpu": cells, "l2": "flushed before every step",
                   "parallelism": f"replicas x{world}", "lanes_per_column": lanes},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4),
                     "traffic": (SWEEP_TRAFFIC["bytes_per_launch"]
                                 if kernel_source_hash() == SWEEP_TRAFFIC["kernels_sha256"] else None),
                     "kernel": "sweep_kernel<7> (32 lanes)" if lanes == 32 else "sweep_kernel<13> (16 lanes)",
                     "kernel_ms": round(sweep_avg, 5),
                     "algorithmic_bytes": int(alg_bytes), "peak_source": "measured",
                     "fp32_frac": round(fp32 / (sweep_avg * 1e-3) / 1e12 / fp32_peak, 4),
                     "sfu_frac": round(sfu / (sweep_avg * 1e-3) / 1e12 / sfu_tops, 4),
                     "fp32_peak_measured_tinst_s": round(fp32_peak, 2), "sfu_peak_measured_tops": round(sfu_tops, 3)},
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": int(8 * plan.info.layers),
                "d2h_bytes_per_step": int(8 * plan.info.layers + 4 * plan.A)},
        "gpu_launches": n_launch_per_step * args.steps,
        "clocks": clk,
        "re_solve": solve,
        "exact_column_solve": direct,
        "wall_s": round(wall, 3),
    }
    if not args.no_cpu_baseline and world == 1:            # rank 0 at N = 1 only
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds)
    print(json.dumps(line), flush=True)


def run_gpu_batched(args):
    """Batched ragged atmospheres (layers U{50..200}, bins U{300..3000}, 20 g, scattering), all in
    flight at once: one RE step = one flux evaluation of every atmosphere + the temperature step.
    The working set (warm-start fluxes of every column, tens of GB) is far larger than L2."""
    import torch
    rank, world, local = dist_env()
    init_replicas(world, local)
    import synth
    import paper_1606_05474_b300 as hp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    t0 = time.time()
    ids = replica_ids(rank, args.atmospheres)
    wl = synth.config3(A=len(ids), atm_ids=ids)
    t_gen = time.time() - t0
    ctx = hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    t0 = time.time()
    cache = os.environ.get("HELIOS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "helios_tune.json"))
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    tuned = hp.autotune(ctx, wl.atms, wl.tables, kap, cache_path=cache)
    t_tune = time.time() - t0
    t0 = time.time()
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, tuned)
    t_plan = time.time() - t0
    T = torch.from_numpy(np.concatenate([a.T_init for a in wl.atms])).to(dev)
    state = plan.new_state()
    Fu = torch.empty(plan.info.interfaces, dtype=torch.float64, device=dev)
    Fd = torch.empty_like(Fu)
    plan.set_timing(args.steps)
    stream = torch.cuda.current_stream(dev)

    def step(warm):
        plan.re_step(T, state, warm=warm, out=(Fu, Fd))

    step(False)
    for _ in range(args.warmup - 1):
        step(True)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step(True)
    b.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = a.elapsed_time(b)
    total_ms = max_over_ranks(total_ms, world, dev)
    sweep_ms = float(np.mean(plan.sweep_times(args.steps)))
    n_passes = plan.info.passes
    cells, pts, fp32, sfu = algorithmic_counts(wl, n_passes)
    value = cells * args.steps * world / (total_ms * 1e-3) / 1e9
    if rank != 0:
        return
    P = peaks()
    hbm = P.get("hbm_gbs", 6400.0)
    warm_bytes = 2 * 4 * pts
    table_bytes = touched_table_bytes(plan, wl, T)
    alg_bytes = warm_bytes + table_bytes + 16 * plan.info.interfaces
    achieved = alg_bytes / (sweep_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweep / f64 temperature step", "data": "synthetic",
        "config": {"workload": f"batched ragged: {len(wl.atms)} atmospheres per GPU, layers U{{50..200}}, "
                               "bins U{300..3000} x 20 g, scattering, 64-table pool",
                   "cells_per_step_per_gpu": cells, "l2": "working set far larger than L2 (no flush)",
                   "tuned": {"bins_per_item": tuned.bins_per_item, "persistent": tuned.persistent},
                   "parallelism": f"replicas x{world}", "lanes_per_column": "16 for 24..119 layers, else 32"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4), "traffic": None, "kernel": "sweep_kernel (all lane chunks)",
                     "kernel_ms": round(sweep_ms, 3), "algorithmic_bytes": int(alg_bytes), "peak_source": "measured"},
        "gpu_launches": (2 + plan.info.sweep_launches + (0 if plan.info.fused_finalize else 1)) * args.steps,
        "clocks": clk,
        "setup_s": {"inputs": round(t_gen, 2), "autotune": round(t_tune, 2), "plan": round(t_plan, 2)},
        "workspace_gb": round(plan.info.workspace_bytes / 1e9, 2),
    }
    print(json.dumps(line), flush=True)


def run_gpu_learned(args):
    """Batched radiative-equilibrium solves of held-out planets from the isothermal start (plain)
    and from the learned initial profile (surrogate): RE-converged atmospheres per second.  The
    planets are the learned-initialiser family (100 layers 1e-6..1e3 bar, 20 g, Rayleigh-like
    scattering, opacity a metallicity- and C/O-weighted mixture of two seeded tables) on the
    paper's radiative-equilibrium resolution of 300 bins (Sect. 3).  The surrogate is trained on
    converged plain solutions of other planets of the family; its inference is inside the timed
    region, plan set-up is not."""
    import torch
    rank, world, local = dist_env()
    init_replicas(world, local)
    import synth
    import paper_1606_05474_b300 as hp
    from paper_1606_05474_b300.learned import LearnedInitializer, features
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    n_tr, n_te = args.train, args.test
    wl = synth.learned_dataset(n_tr + n_te, L=args.bins, n=100, first=rank * (n_tr + n_te))
    ctx = hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    prm = hp.default_params(max_iter=20000)
    tr_atms, te_atms = wl.atms[:n_tr], wl.atms[n_tr:]

    def solve(atms, starts):
        plan = hp.Plan(ctx, atms, wl.tables, kap, prm)
        T = torch.from_numpy(np.concatenate(starts)).to(dev)
        torch.cuda.synchronize()
        t = time.time()
        iters, status = plan.solve_re(T)
        torch.cuda.synchronize()
        dt = time.time() - t
        return np.array(plan.split_layers(T.cpu().numpy())), iters.cpu().numpy(), status.cpu().numpy(), dt

    Ttr, it_tr, st_tr, t_tr = solve(tr_atms, [a.T_init for a in tr_atms])
    ok = st_tr == 1
    init = LearnedInitializer(ctx, seed=1, max_batch=max(256, n_te))
    t = time.time()
    losses = init.fit(features(tr_atms)[ok], Ttr[ok], epochs=args.epochs, batch=256, lr=2e-3)
    torch.cuda.synchronize()
    t_fit = time.time() - t
    Tp, it_p, st_p, t_plain = solve(te_atms, [a.T_init for a in te_atms])
    t = time.time()
    starts, used = init.initial_profiles(features(te_atms), [a.n_layers for a in te_atms],
                                         [a.T_init for a in te_atms])
    t_inf = time.time() - t
    Ts, it_s, st_s, t_sur = solve(te_atms, starts)
    t_sur += t_inf
    # whole job: atmospheres converged on every rank over the slowest rank's time
    n_conv_p = sum_over_ranks(int((st_p == 1).sum()), world, dev)
    n_conv_s = sum_over_ranks(int((st_s == 1).sum()), world, dev)
    t_plain_job = max_over_ranks(t_plain, world, dev)
    t_sur_job = max_over_ranks(t_sur, world, dev)
    if rank != 0:
        return
    both = (st_p == 1) & (st_s == 1)
    T0 = np.array([a.T_init for a in te_atms])
    rms_iso = np.sqrt(((T0 - Tp) ** 2).mean(axis=1))[both]
    rms_ml = np.sqrt(((np.array(starts) - Tp) ** 2).mean(axis=1))[both]
    dT = np.abs(Ts - Tp)[both]
    flop_fwd = 2 * (6 * 256 + 2 * 256 * 256 + 256 * 100)
    n_fit = int(ok.sum()) * args.epochs
    line = {
        "metric": "RE-converged atmospheres/s, batched + surrogate vs plain", "value": round(n_conv_s / t_sur_job, 3),
        "unit": "atm/s", "n_gpus": world, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 sweep / f64 temperature step / bf16 MLP", "data": "synthetic",
        "config": {"workload": f"learned-initialiser family: {n_te} held-out planets, 100 layers x {args.bins} bins x 20 g, "
                               f"scattering, 2-table mixtures; surrogate trained on {int(ok.sum())} converged planets",
                   "tol": prm.tol, "max_iter": prm.max_iter, "parallelism": f"replicas x{world}"},
        "plain": {"atm_per_s": round(n_conv_p / t_plain_job, 3), "wall_s": round(t_plain, 3),
                  "converged": int((st_p == 1).sum()), "iters_median": float(np.median(it_p)),
                  "iters_mean": round(float(it_p.mean()), 1)},
        "surrogate": {"atm_per_s": round(n_conv_s / t_sur_job, 3), "wall_s": round(t_sur, 3),
                      "inference_s": round(t_inf, 4), "converged": int((st_s == 1).sum()),
                      "iters_median": float(np.median(it_s)), "iters_mean": round(float(it_s.mean()), 1),
                      "used_learned_start": int(used.sum())},
        "initial_guess_rms_K": {"isothermal_median": round(float(np.median(rms_iso)), 2),
                                "learned_median": round(float(np.median(rms_ml)), 2),
                                "learned_max": round(float(rms_ml.max()), 2)},
        "final_T_agreement_K": {"median_of_max": round(float(np.median(dT.max(axis=1))), 4),
                                "p95_all_layers": round(float(np.quantile(dT, 0.95)), 4),
                                "max": round(float(dT.max()), 3)},
        "training": {"solve_s": round(t_tr, 2), "fit_s": round(t_fit, 2), "loss_first": float(losses[0]),
                     "loss_last": float(losses[-1]), "samples": int(ok.sum()), "epochs": args.epochs,
                     "mlp_tflops": round(3 * flop_fwd * n_fit / t_fit / 1e12, 4)},
    }
    print(json.dumps(line), flush=True)


def run_gpu_spectrum(args):
    """Post-processing emission spectrum (Sect. 3): the full-size atmosphere (100 layers x 3000
    bins x 20 g, scattering) on isothermal layers, from a cold start, with 1 + 80 scattering
    passes (Sect. 2.2.3) and with their limit, the exact column solve.  A step is one spectrum;
    L2 is flushed before every step; CUDA events on the launching stream."""
    import torch
    rank, world, local = dist_env()
    init_replicas(world, local)
    import synth
    import paper_1606_05474_b300 as hp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    wl = synth.config2()
    T0 = synth.perturbed_profile(wl.atms[0], 21 + rank, amp=200.0)
    ctx = hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(iso_layers=1))
    T = torch.from_numpy(np.asarray(T0, np.float64)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    for name, npass in (("exact", hp.DIRECT), ("passes_81", 81)):
        for _ in range(args.warmup):
            plan.emission_spectrum(T, n_passes=npass)
        plan.set_timing(args.steps)
        torch.cuda.synchronize()
        barrier(world)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            plan.emission_spectrum(T, n_passes=npass)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        total = max_over_ranks(float(np.sum([a.elapsed_time(b) for a, b in ev])), world, dev)
        res[name] = {"ms_per_spectrum": round(total / args.steps, 5),
                     "sweep_ms": round(float(np.median(plan.sweep_times(args.steps))), 5)}
    if rank != 0:
        return
    cells = plan.info.cells
    P = peaks()
    fp32_peak = hp.measure_peaks(ctx)[0] / 2.0           # measured, T FP32 instructions/s
    # algorithmic FP32 instructions of the exact solve per cell: 2 sublayers x (24 for the
    # coefficients + 14 for the three recurrences and G_up = rho G_dn + u)
    fp32 = 2 * (24 + 14) * cells
    achieved = fp32 / (res["exact"]["sweep_ms"] * 1e-3) / 1e12
    line = {
        "metric": "post-processing emission spectra/s (isothermal layers, exact column solve)",
        "value": round(world * 1e3 / res["exact"]["ms_per_spectrum"], 3), "unit": "spectra/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["exact"]["ms_per_spectrum"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweep / f64 sums",
        "data": "synthetic",
        "config": {"workload": "full-size atmosphere on 100 isothermal layers x 3000 bins x 20 g, scattering, cold start",
                   "cells": cells, "l2": "flushed before every step", "parallelism": f"replicas x{world}"},
        "exact": res["exact"], "passes_81": res["passes_81"],
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_peak, 2),
                     "unit": "T FP32 inst/s", "frac": round(achieved / fp32_peak, 4), "traffic": None,
                     "kernel": "sweep_kernel<7, 2, true> (exact column solve)",
                     "peak_source": "measured (helios_measure_peaks: independent FMA chains on every SM)"},
        "gpu_launches": 3 * 2 * args.steps,                      # prep, sweep, finalize per spectrum
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(seconds=12.0, wl=None):
    """The FP64 oracle on the same workload on the host cores: whole RE steps, as many as fit."""
    import oracle
    import synth
    wl = wl or synth.config2()
    atm = oracle.Atm.from_workload(wl)
    st = oracle.State(atm, synth.perturbed_profile(wl.atms[0], 11, amp=200.0))
    p = oracle.params()
    K = oracle.passes(atm, p)
    t0 = time.time()
    steps = 0
    while True:
        r = oracle.flux_sweep(atm, st.T, n_passes=K, warm=st.warm, warm_valid=steps > 0)
        oracle.temp_update(atm, st, r["Fup"], r["Fdn"], p)
        steps += 1
        if time.time() - t0 > seconds:
            break
    dt = time.time() - t0
    v = wl.cells * steps / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full RE steps of the same atmosphere ({wl.cells} cells each), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    wl = synth.config2()
    atm = oracle.Atm.from_workload(wl)
    st = oracle.State(atm, synth.perturbed_profile(wl.atms[0], 11, amp=200.0))
    p = oracle.params()
    K = oracle.passes(atm, p)
    # a bounded sample per step: every 10th bin of the workload (300 of 3000 bins), whole column
    sub = synth.config2(L=300)
    satm = oracle.Atm.from_workload(sub)
    sst = oracle.State(satm, st.T.copy())
    def one(i):
        r = oracle.flux_sweep(satm, sst.T, n_passes=K, warm=sst.warm, warm_valid=i > 0)
        oracle.temp_update(satm, sst, r["Fup"], r["Fdn"], p)
    for i in range(args.warmup):
        one(i)
    t0 = time.time()
    for i in range(args.steps):
        one(args.warmup + i)
    dt = time.time() - t0
    v = sub.cells * args.steps / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "300 of the 3000 bins per step (bins equal in wavenumber)"},
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} RE steps on 300 bins x 100 layers x 20 g"},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single", choices=["single", "batched", "learned", "spectrum"])
    ap.add_argument("--atmospheres", type=int, default=4096)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--col-lanes", type=int, default=0, choices=[0, 16, 32],
                    help="lanes per column of the iterated sweep (16: two Gauss points per warp; 0: automatic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--train", type=int, default=2048, help="learned workload: training planets")
    ap.add_argument("--test", type=int, default=512, help="learned workload: held-out planets")
    ap.add_argument("--bins", type=int, default=300, help="learned workload: bins per planet")
    ap.add_argument("--epochs", type=int, default=300, help="learned workload: training epochs")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_gpu_batched(args)
    elif args.workload == "learned":
        run_gpu_learned(args)
    elif args.workload == "spectrum":
        run_gpu_spectrum(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
