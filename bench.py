"""Benchmark of the radiative-equilibrium hot path on one B300 (or N, one process per GPU).

Metric: RE-converged atmospheres/s and flux-sweep Gcell/s, batched + surrogate vs plain.

Default (the headline line):
- value: the batched solver step -- one radiative-equilibrium iteration (opacities, sublayer
  optical depths, two-stream coefficients, 1 + 4 scattering passes, Gauss-point and bin sums,
  FP64 temperature step) of 4096 ragged atmospheres (layers U{50..200}, bins U{300..3000} x 20 g,
  Rayleigh-like scattering, a pool of 64 seeded k-tables) with autotuned launches, in Gcell/s
  (cell = atmosphere x layer x bin x g of one full iteration).  W untimed steps, then K timed
  steps between CUDA events on the launching stream; the working set (151 GB) is far larger than
  L2, so no flush is needed.
- surrogate_vs_plain: converged atmospheres per second of held-out planets of the learned-
  initialiser family, solved in one batched graph-captured solve from the isothermal start
  (plain) and from the learned network's profile (surrogate, inference inside the timed region),
  both to eq. (29), and the multiple between them.
- single_atmosphere: the full-size single atmosphere (100 layers x 3000 bins x 20 g, scattering):
  per-step times with L2 flushed, back-to-back steady state, the sweep kernel, end to end, one full
  solve, the exact column solve and the post-processing spectrum.
- plain_single_atmosphere: the plain single atmosphere (50 layers x 30 bins x 8 g, pure
  absorption; latency-bound): microseconds per RE iteration back to back and inside one
  graph-captured solve, and (in the cpu_baseline leg) the oracle on one host core and on all of
  them: its full solve of this atmosphere and one full-size flux evaluation.
- roofline: the sweep kernel of the batched step against the three floors of its work (HBM bytes,
  FP32 instructions, SFU operations); the FP32 and SFU counts per cell come from the op-counting
  build of the oracle on a bounded sample of the same workload (taken in the cpu_baseline leg).
- cpu_baseline: the FP64 oracle on the host cores on a bounded sample of the batched workload.

--workload batched|learned|single|spectrum prints the line of one part alone; --workload precision
solves the 64-atmosphere high-resolution precision-stress workload (minutes).
--impl reference: the FP64 CPU oracle timed on the host cores on the headline's workload and
metric (bounded sample per step).
"""
import argparse
import dataclasses
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
BATCHED_WORKLOAD = ("batched ragged: {A} atmospheres per GPU, layers U{{50..200}}, bins U{{300..3000}} x 20 g, "
                    "Rayleigh-like scattering, 1 + 4 passes per step, pool of 64 k-tables, autotuned")
SINGLE_WORKLOAD = "full-size single atmosphere: 100 layers x 3000 bins x 20 g, scattering, 5 passes/step"


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
        time.sleep(0.4)                                 # let the sampler attach before timing

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


# DRAM traffic (read + write) per cell of the sweep kernel, from ncu captures of the same command
# on smaller cases (the summaries under profiles/ give each command), valid only for the kernel
# source they were taken on (sha256 prefix of the kernels and the launch code); null otherwise.
SWEEP_TRAFFIC = {"kernels_sha256": "86227aafd4f8eac1", "bytes_per_cell": {"single": 10.14, "batched": 17.40}}


def kernel_source_hash():
    """Hash of the sweep kernel's source and its launch configuration (the recorded DRAM traffic
    holds only while both are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("helios_kernels.cuh", "helios_api.cu"):
        h.update(open(os.path.join(ROOT, "paper_1606_05474_b300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(key, cells):
    if SWEEP_TRAFFIC["kernels_sha256"] != kernel_source_hash() or key not in SWEEP_TRAFFIC["bytes_per_cell"]:
        return None
    return int(SWEEP_TRAFFIC["bytes_per_cell"][key] * cells)


def touched_table_bytes(plan, wl, T):
    """Bytes of the k-table rows (iP, iT corners) the current profiles touch, from the library's
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


def sweep_bytes(plan, wl, T):
    """Algorithmic DRAM bytes of one flux evaluation: the warm-start upward fluxes read and written
    (4 B per column point each way), the k-table rows the profiles touch, the bolometric outputs."""
    pts = sum((2 * a.n_layers + 1) * a.n_bins for a in wl.atms) * wl.G
    return 2 * 4 * pts + touched_table_bytes(plan, wl, T) + 16 * int(plan.info.interfaces)


def fp32_peak_derived(dev_index, sm_max_mhz):
    """FP32 instruction peak from unit counts and the maximum SM clock: SMs x 128 FP32 lanes x f."""
    import torch
    sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
    return sms * 128 * sm_max_mhz * 1e6 / 1e12


def roofline(sweep_ms, cells, alg_bytes, counts, fp32_peak, sfu_peak, hbm, traffic, kernel, clocks_mhz):
    """The sweep against its three floors: algorithmic HBM bytes at the measured copy bandwidth,
    algorithmic FP32 instructions at the FP32 pipe's peak, SFU operations at the measured MUFU
    rate.  The binding term is the largest floor; `frac` is achieved / peak in that term."""
    t = sweep_ms * 1e-3
    terms = {"hbm": {"work": alg_bytes, "unit": "GB/s", "peak": hbm, "achieved": alg_bytes / t / 1e9}}
    if counts:
        fp32 = counts["fp32_per_cell"] * cells
        sfu = counts["sfu_per_cell"] * cells
        terms["alu"] = {"work": fp32, "unit": "T FP32 inst/s", "peak": fp32_peak, "achieved": fp32 / t / 1e12}
        terms["sfu"] = {"work": sfu, "unit": "T SFU op/s", "peak": sfu_peak, "achieved": sfu / t / 1e12}
    for v in terms.values():
        v["frac"] = round(v["achieved"] / v["peak"], 4)
        v["floor_ms"] = round(sweep_ms * v["frac"], 5)
        v["achieved"] = round(v["achieved"], 3)
    bound = max(terms, key=lambda k: terms[k]["floor_ms"])
    b = terms[bound]
    return {"bound": "alu" if bound in ("alu", "sfu") else bound, "binding_term": bound, "achieved": b["achieved"],
            "peak": b["peak"], "unit": b["unit"], "frac": b["frac"], "traffic": traffic, "kernel": kernel,
            "kernel_ms": round(sweep_ms, 5), "algorithmic_bytes": int(alg_bytes),
            "terms": {k: {kk: vv for kk, vv in v.items() if kk != "work"} for k, v in terms.items()},
            "peak_source": {"hbm": "measured (MEASURED_PEAKS.json)",
                            "alu": f"derived: SMs x 128 FP32 lanes x {clocks_mhz:.0f} MHz (max SM clock)",
                            "sfu": "measured on the device (helios_measure_peaks: MUFU ex2 chains on every SM)"},
            "counts_source": counts.get("source") if counts else None,
            "fp32_per_cell": counts.get("fp32_per_cell") if counts else None,
            "sfu_per_cell": counts.get("sfu_per_cell") if counts else None}


# ---------------------------------------------------------------------------------------------
# batched solver step (the headline value)
# ---------------------------------------------------------------------------------------------
def tune_cache_path():
    """The autotuner's cache file (HELIOS_TUNE_CACHE, else ~/.cache/helios_tune.json): a second run
    on the same batch reuses the choice instead of timing the candidates again."""
    cache = os.environ.get("HELIOS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "helios_tune.json"))
    os.makedirs(os.path.dirname(cache), exist_ok=True)
    return cache


def run_batched(args, world, rank, local, dev):
    import torch
    import synth
    import paper_1606_05474_b300 as hp
    t0 = time.time()
    ids = replica_ids(rank, args.atmospheres)
    wl = synth.config3(A=len(ids), atm_ids=ids)
    t_gen = time.time() - t0
    ctx = hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    t0 = time.time()
    tuned = hp.autotune(ctx, wl.atms, wl.tables, kap, cache_path=tune_cache_path())
    t_tune = time.time() - t0
    t0 = time.time()
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, tuned)
    t_plan = time.time() - t0
    T = torch.from_numpy(np.concatenate([a.T_init for a in wl.atms])).to(dev)
    state = plan.new_state()
    Fu = torch.empty(plan.info.interfaces, dtype=torch.float64, device=dev)
    Fd = torch.empty_like(Fu)
    stream = torch.cuda.current_stream(dev)

    def step(warm):
        plan.re_step(T, state, warm=warm, out=(Fu, Fd))

    step(False)
    for _ in range(args.warmup - 1):
        step(True)
    torch.cuda.synchronize()
    plan.set_timing(args.steps)
    clocks = ClockSampler(local)
    clocks.start()
    barrier(world)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        step(True)
    b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    total_ms = max_over_ranks(a.elapsed_time(b), world, dev)
    sweep_ms = float(np.mean(plan.sweep_times(args.steps)))
    plan.set_timing(0)
    cells = wl.cells
    value = cells * args.steps * world / (total_ms * 1e-3) / 1e9

    # end to end through helios_re_step_host: the temperatures of every atmosphere from pinned host
    # memory in, the new temperatures and statuses back to the host, every step
    Th = torch.empty(int(plan.info.layers), dtype=torch.float64).pin_memory()
    Th.copy_(T.cpu())
    Sh = torch.empty(plan.A, dtype=torch.int32).pin_memory()
    Td = torch.empty_like(T)
    torch.cuda.synchronize()
    barrier(world)
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a2.record(stream)
    for _ in range(args.steps):
        plan.re_step_host(Th, Td, state, Sh, warm=True)
        torch.cuda.current_stream(dev).synchronize()        # the host reads the step's result
    b2.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(a2.elapsed_time(b2), world, dev)
    e2e = {"value": round(cells * args.steps * world / (e2e_ms * 1e-3) / 1e9, 3), "unit": UNIT,
           "h2d_bytes_per_step": int(8 * plan.info.layers), "d2h_bytes_per_step": int(8 * plan.info.layers + 4 * plan.A),
           "path": "helios_re_step_host (host temperatures in, temperatures + statuses out, host waits every step)"}
    out = {"value": value, "total_ms": total_ms, "sweep_ms": sweep_ms, "cells": cells, "clocks": clk, "e2e": e2e,
           "launches_per_step": 2 + plan.info.sweep_launches + (0 if plan.info.fused_finalize else 1),
           "tuned": {"bins_per_item": tuned.bins_per_item, "persistent": tuned.persistent},
           "setup_s": {"inputs": round(t_gen, 2), "autotune": round(t_tune, 2), "plan": round(t_plan, 2)},
           "workspace_gb": round(plan.info.workspace_bytes / 1e9, 2), "A": len(ids),
           "alg_bytes": sweep_bytes(plan, wl, T) if rank == 0 else None, "ctx": ctx}
    del plan, kap
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------------------
# surrogate vs plain: converged atmospheres per second
# ---------------------------------------------------------------------------------------------
def run_learned(args, world, rank, local, dev, ctx=None):
    import torch
    import synth
    import paper_1606_05474_b300 as hp
    from paper_1606_05474_b300.learned import LearnedInitializer, features
    n_tr, n_te = args.train, args.test
    wl = synth.learned_dataset(n_tr + n_te, L=args.bins, n=100, first=rank * (n_tr + n_te))
    ctx = ctx or hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    prm = hp.default_params(max_iter=20000)
    tr_atms, te_atms = wl.atms[:n_tr], wl.atms[n_tr:]
    inf = {}
    init = None

    def solve(atms, starts, pre=None):
        plan = hp.Plan(ctx, atms, wl.tables, kap, prm)
        T = torch.from_numpy(np.concatenate(starts)).to(dev)
        torch.cuda.synchronize()
        barrier(world)
        t = time.time()
        if pre is not None:
            T = pre(plan)
        iters, status = plan.solve_re(T)
        torch.cuda.synchronize()
        dt = time.time() - t
        out = np.array(plan.split_layers(T.cpu().numpy())), iters.cpu().numpy(), status.cpu().numpy(), dt
        if pre is not None:
            inf["starts"] = np.array(init.initial_profiles(plan, features(atms), [a.T_init for a in atms])[0])
        return out

    Ttr, it_tr, st_tr, t_tr = solve(tr_atms, [a.T_init for a in tr_atms])
    ok = st_tr == 1
    # a throwaway network's single epoch first: the first use of the network's kernels in a process
    # carries one-time costs (seconds, varying) that are not training
    LearnedInitializer(ctx, seed=2, max_batch=256).fit(features(tr_atms)[ok][:256], Ttr[ok][:256], epochs=1)
    torch.cuda.synchronize()
    init = LearnedInitializer(ctx, seed=1, max_batch=max(256, n_te))    # noqa: F841 (used by solve)
    t = time.time()
    losses = init.fit(features(tr_atms)[ok], Ttr[ok], epochs=args.epochs, batch=256, lr=2e-3)
    torch.cuda.synchronize()
    t_fit = time.time() - t
    if init.net.error():
        raise RuntimeError("a tensor-core product of the network gave up waiting: its results are invalid")
    Tp, it_p, st_p, t_plain = solve(te_atms, [a.T_init for a in te_atms])

    def predict(plan):
        # inference inside the timed region: features -> network -> profiles on the plan's layers
        t = time.time()
        T, used = init.initial_profiles_device(plan, features(te_atms), [a.T_init for a in te_atms])
        torch.cuda.synchronize()
        inf["s"], inf["used"] = time.time() - t, used
        return T

    Ts, it_s, st_s, t_sur = solve(te_atms, [a.T_init for a in te_atms], pre=predict)
    n_conv_p = sum_over_ranks(int((st_p == 1).sum()), world, dev)
    n_conv_s = sum_over_ranks(int((st_s == 1).sum()), world, dev)
    t_plain_job = max_over_ranks(t_plain, world, dev)
    t_sur_job = max_over_ranks(t_sur, world, dev)
    both = (st_p == 1) & (st_s == 1)
    T0 = np.array([a.T_init for a in te_atms])
    starts = inf["starts"]
    rms_iso = np.sqrt(((T0 - Tp) ** 2).mean(axis=1))[both]
    rms_ml = np.sqrt(((np.array(starts) - Tp) ** 2).mean(axis=1))[both]
    dT = np.abs(Ts - Tp)[both]
    flop_fwd = 2 * (6 * 256 + 2 * 256 * 256 + 256 * 100)
    n_fit = int(ok.sum()) * args.epochs
    plain_aps, sur_aps = n_conv_p / t_plain_job, n_conv_s / t_sur_job
    return {
        "workload": (f"learned-initialiser family: {n_te} held-out planets per GPU, 100 layers x {args.bins} bins x 20 g, "
                     f"scattering, 2-table mixtures; network trained on {int(ok.sum())} converged planets "
                     f"(the stated size is 20k planets at 3000 bins; this run is smaller so that the benchmark "
                     f"finishes in minutes)"),
        "unit": "atm/s", "tol": prm.tol, "multiple": round(sur_aps / plain_aps, 3),
        "plain": {"atm_per_s": round(plain_aps, 3), "wall_s": round(t_plain, 3), "converged": int((st_p == 1).sum()),
                  "iters_median": float(np.median(it_p)), "iters_mean": round(float(it_p.mean()), 1)},
        "surrogate": {"atm_per_s": round(sur_aps, 3), "wall_s": round(t_sur, 3),
                      "inference_s": round(inf["s"], 4), "converged": int((st_s == 1).sum()),
                      "iters_median": float(np.median(it_s)), "iters_mean": round(float(it_s.mean()), 1),
                      "used_learned_start": int(np.sum(inf["used"]))},
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


# ---------------------------------------------------------------------------------------------
# full-size single atmosphere
# ---------------------------------------------------------------------------------------------
def run_single(args, world, rank, local, dev, ctx=None, steps=200):
    import torch
    import synth
    import paper_1606_05474_b300 as hp
    wl = synth.config2()
    wl.atms[0].T_init = synth.perturbed_profile(wl.atms[0], 11 + rank, amp=200.0)
    ctx = ctx or hp.Context(local)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(col_lanes=args.col_lanes))
    n_passes = plan.info.passes
    T = torch.from_numpy(np.asarray(wl.atms[0].T_init, np.float64)).to(dev)
    T0 = T.clone()
    state = plan.new_state()
    Fu = torch.empty(plan.info.interfaces, dtype=torch.float64, device=dev)
    Fd = torch.empty_like(Fu)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(warm):
        plan.re_step(T, state, warm=warm, out=(Fu, Fd))

    step(False)
    for _ in range(max(3, args.warmup) - 1):
        step(True)
    torch.cuda.synchronize()
    # (i) per step, L2 flushed before each (the flush is outside the events; the dirty warm-start
    # lines of the previous step are written back during the flush, not inside the next step)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        step(True)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    flushed_ms = float(np.mean([x.elapsed_time(y) for x, y in ev]))
    # (ii) steady state: back-to-back steps between one event pair, no flush (each step pays for
    # its own warm-start write-back)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        step(True)
    b.record(stream)
    torch.cuda.synchronize()
    steady_ms = a.elapsed_time(b) / steps
    # (iii) the sweep kernel alone (events around the sweep launches; a separate pass, since inside
    # the timed loops the events would split the step's chain of dependent launches)
    plan.set_timing(steps)
    for _ in range(steps):
        flush.zero_()
        step(True)
    torch.cuda.synchronize()
    sweep_flushed = float(np.mean(plan.sweep_times(steps)))
    for _ in range(steps):
        step(True)
    torch.cuda.synchronize()
    sweep_steady = float(np.mean(plan.sweep_times(steps)))
    plan.set_timing(0)
    # (iv) end to end through helios_re_step_host, the host waiting for every step's result
    Th = torch.empty(int(plan.info.layers), dtype=torch.float64).pin_memory()
    Th.copy_(T.cpu())
    Sh = torch.empty(plan.A, dtype=torch.int32).pin_memory()
    Td = torch.empty_like(T)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        plan.re_step_host(Th, Td, state, Sh, warm=True)
        stream.synchronize()
    e2e_ms = (time.perf_counter() - t) * 1e3 / steps
    # the same without the copies (host waits every step): what the copies add vs the wait
    t = time.perf_counter()
    for _ in range(steps):
        step(True)
        stream.synchronize()
    sync_ms = (time.perf_counter() - t) * 1e3 / steps
    cells = wl.cells
    # (v) one full radiative-equilibrium solve from the start profile (graph-captured device loop)
    Ts = T0.clone()
    torch.cuda.synchronize()
    t0 = time.time()
    iters, status = plan.solve_re(Ts)
    torch.cuda.synchronize()
    dt = time.time() - t0
    solve = {"wall_s": round(dt, 4), "iters": int(iters.item()), "status": int(status.item()),
             "atm_per_s": round(1.0 / dt, 3), "tol": 1e-7}

    # (vi) the exact column solve (the limit of the passes, Sect. 2.2.3) against 1 + 4 passes, and
    # the post-processing spectrum (isothermal layers, Sect. 3) with 1 + 80 passes against the exact
    # solve; each sweep timed cold-start after an L2 flush
    def time_sweeps(pl, Tt, npass, reps=20):
        pl.flux_sweep(Tt, n_passes=npass, warm=False, want_toa=True)
        pl.set_timing(reps)
        for _ in range(reps):
            flush.zero_()
            pl.flux_sweep(Tt, n_passes=npass, warm=False, want_toa=True)
        torch.cuda.synchronize()
        r = round(float(np.median(pl.sweep_times(reps))), 5)
        pl.set_timing(0)
        return r
    Tc = Ts.clone()
    ms_dir, ms_pass = time_sweeps(plan, Tc, hp.DIRECT), time_sweeps(plan, Tc, n_passes)
    pp = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(iso_layers=1))
    pt = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(tabulate=1))
    direct = {"sweep_ms_exact": ms_dir, "sweep_ms_passes": ms_pass, "passes": n_passes,
              "sweep_ms_passes_tabulated_functions": time_sweeps(pt, Tc, n_passes),
              "post_processing_spectrum_ms": {"isothermal_layers_81_passes": time_sweeps(pp, Tc, 81),
                                              "isothermal_layers_exact": time_sweeps(pp, Tc, hp.DIRECT)}}
    del pp, pt
    out = {"workload": SINGLE_WORKLOAD, "cells_per_step": cells,
           "gcell_s_l2_flushed": round(cells / (flushed_ms * 1e-3) / 1e9, 3), "ms_per_step_l2_flushed": round(flushed_ms, 5),
           "gcell_s_steady": round(cells / (steady_ms * 1e-3) / 1e9, 3), "ms_per_step_steady": round(steady_ms, 5),
           "sweep_ms_l2_flushed": round(sweep_flushed, 5), "sweep_ms_steady": round(sweep_steady, 5),
           "e2e": {"value": round(cells / (e2e_ms * 1e-3) / 1e9, 3), "unit": UNIT, "ms_per_step": round(e2e_ms, 4),
                   "ms_per_step_without_copies": round(sync_ms, 4),
                   "h2d_bytes_per_step": int(8 * plan.info.layers), "d2h_bytes_per_step": int(8 * plan.info.layers + 4),
                   "path": "helios_re_step_host, host waits every step (wall clock)"},
           "re_solve": solve, "exact_column_solve": direct, "passes_per_step": n_passes,
           "l2": "flushed (256 MB write) before every step of the flushed figures"}
    out["alg_bytes"] = sweep_bytes(plan, wl, T) if rank == 0 else None
    del plan
    return out


# ---------------------------------------------------------------------------------------------
# CPU leg: the FP64 oracle on a bounded sample of the workload, and its op counts
# ---------------------------------------------------------------------------------------------
def _sub_atmosphere(wl, a, l0, nb):
    """Bins l0 .. l0+nb-1 of atmosphere a (with the matching slice of its table)."""
    import synth
    atm = wl.atms[a]
    tab = wl.tables[atm.table_id]
    st = dataclasses.replace(tab, L=nb, kappa32=np.ascontiguousarray(tab.kappa32[:, :, l0:l0 + nb, :]), kappa64=None)
    sa = dataclasses.replace(atm, nu_edges=atm.nu_edges[l0:l0 + nb + 1].copy(), omega0=atm.omega0[l0:l0 + nb].copy(),
                             g0=atm.g0[l0:l0 + nb].copy(), table_id=0)
    return synth.Workload(name="sample", atms=[sa], tables=[st])


def oracle_counts(wl, atm_ids, chunks=3, nb=8, T_of=None):
    """FP32 and SFU instructions per cell of one flux evaluation (1 + 4 passes), from the
    op-counting build of the oracle on chunks of nb bins spread over the spectrum of the given
    atmospheres."""
    from oracle import opcount
    fp32 = sfu = cells = 0
    for a in atm_ids:
        L = wl.atms[a].n_bins
        for c in range(chunks):
            l0 = min(L - nb, (c * L) // chunks)
            sw = _sub_atmosphere(wl, a, l0, nb)
            T = T_of(a) if T_of else wl.atms[a].T_init
            r = opcount.flux_evaluation(sw.atms[0], sw.tables[0], T, 1 + wl.n_scat)
            fp32 += r["fp32"]; sfu += r["sfu"]; cells += r["cells"]
    return {"fp32_per_cell": round(fp32 / cells, 3), "sfu_per_cell": round(sfu / cells, 3),
            "source": f"op-counting build of the FP64 oracle (oracle/opcount.cpp) on {len(atm_ids)} atmospheres x "
                      f"{chunks} chunks of {nb} bins ({cells} cells), 1 + {wl.n_scat} passes"}


def run_plain(args, dev, ctx, steps=200):
    """The plain single atmosphere (50 layers x 30 bins x 8 g, pure absorption, one pass per step):
    latency-bound (240 columns, far below one wave), so microseconds per RE iteration -- back to
    back through helios_re_step, and inside one graph-captured solve from the isothermal start --
    not a roofline."""
    import torch
    import synth
    import paper_1606_05474_b300 as hp
    wl = synth.config1()
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params())
    T = torch.from_numpy(np.asarray(wl.atms[0].T_init, np.float64)).to(dev)
    T0 = T.clone()
    state = plan.new_state()
    stream = torch.cuda.current_stream(dev)
    plan.re_step(T, state, warm=False)
    for _ in range(max(3, args.warmup)):
        plan.re_step(T, state, warm=True)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        plan.re_step(T, state, warm=True)
    b.record(stream)
    torch.cuda.synchronize()
    step_us = a.elapsed_time(b) * 1e3 / steps
    Ts = T0.clone()
    plan.solve_re(Ts)                                   # first solve: graph capture
    Ts = T0.clone()
    torch.cuda.synchronize()
    t0 = time.time()
    iters, status = plan.solve_re(Ts)
    torch.cuda.synchronize()
    dt = time.time() - t0
    return {"workload": "plain single atmosphere: 50 layers x 30 bins x 8 g, pure absorption, 1 pass per step, "
                        "isothermal 1000 K start", "cells_per_step": wl.cells,
            "us_per_step_back_to_back": round(step_us, 2),
            "re_solve": {"wall_s": round(dt, 4), "iters": int(iters.item()), "status": int(status.item()),
                         "us_per_iteration": round(dt * 1e6 / max(1, int(iters.item())), 2),
                         "atm_per_s": round(1.0 / dt, 2), "tol": 1e-7}}


def oracle_timings(gpu_iters_config2=None):
    """The FP64 oracle on one host core and on all of them: a full RE solve of the plain single
    atmosphere from its isothermal start, and one flux evaluation (1 + 4 passes) of the full-size
    single atmosphere; a converged full-size atmosphere is estimated as that evaluation's time
    times the GPU solve's iteration count (a full oracle solve takes tens of minutes)."""
    import oracle
    import synth
    wl1 = synth.config1()
    a1 = oracle.Atm.from_workload(wl1)
    wl2 = synth.config2()
    a2 = oracle.Atm.from_workload(wl2)
    T2 = synth.perturbed_profile(wl2.atms[0], 11, amp=200.0)
    all_cores = oracle.max_threads()
    out = {"kind": "oracle", "cores_all": all_cores}
    for tag, nt in (("1_core", 1), ("all_cores", all_cores)):
        oracle.set_threads(nt)
        st = oracle.State(a1, wl1.atms[0].T_init)
        t0 = time.time()
        rc, it, _ = oracle.solve_re(a1, st)
        t1 = time.time()
        oracle.flux_sweep(a2, T2, n_passes=5)
        t2 = time.time()
        out[tag] = {"plain_single_solve_s": round(t1 - t0, 3), "plain_single_iters": it, "plain_single_status": rc,
                    "full_size_eval_s": round(t2 - t1, 3)}
        if gpu_iters_config2:
            out[tag]["full_size_converged_s_estimate"] = round((t2 - t1) * gpu_iters_config2, 1)
    oracle.set_threads(all_cores)
    return out


def cpu_baseline(wl, a=0, seconds=12.0):
    """The FP64 oracle on the host cores: whole RE steps (flux evaluation + temperature step) of
    atmosphere a of the workload, as many as fit in `seconds`."""
    import oracle
    atm = oracle.Atm.from_workload(wl, a)
    st = oracle.State(atm, wl.atms[a].T_init)
    p = oracle.params()
    K = oracle.passes(atm, p)
    cells = atm.n * atm.L * atm.G
    t0 = time.time()
    steps = 0
    while True:
        r = oracle.flux_sweep(atm, st.T, n_passes=K, warm=st.warm, warm_valid=steps > 0)
        oracle.temp_update(atm, st, r["Fup"], r["Fdn"], p)
        steps += 1
        if time.time() - t0 > seconds:
            break
    dt = time.time() - t0
    cores = oracle.max_threads()                    # the OpenMP threads the oracle's loops used
    return {"value": round(cells * steps / dt / 1e9, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{steps} full RE steps of atmosphere {a} of the workload ({atm.n} layers x {atm.L} bins x "
                      f"{atm.G} g = {cells} cells each), {dt:.1f} s"}


# ---------------------------------------------------------------------------------------------
def headline(args):
    import torch
    rank, world, local = dist_env()
    init_replicas(world, local)
    import synth
    import paper_1606_05474_b300 as hp
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    want = args.workload
    bat = run_batched(args, world, rank, local, dev) if want in ("headline", "batched") else None
    ctx = bat["ctx"] if bat else hp.Context(local)
    lrn = run_learned(args, world, rank, local, dev, ctx) if want in ("headline", "learned") else None
    sgl = run_single(args, world, rank, local, dev, ctx) if want in ("headline", "single") else None
    pln = run_plain(args, dev, ctx) if want in ("headline", "single") and rank == 0 else None
    if rank != 0:
        return
    P = peaks()
    hbm = P.get("hbm_gbs", 6400.0)
    sm_max = P.get("sm_max_mhz", 2032.0)
    fp32_peak = fp32_peak_derived(local, sm_max)
    fp32_meas, sfu_peak = hp.measure_peaks(ctx)
    base = {"n_gpus": world, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 sweep / f64 temperature step / bf16 MLP", "data": "synthetic"}
    counts = cpu = None
    if want in ("headline", "batched"):
        wl3 = synth.config3(A=64, atm_ids=list(range(0, 4096, 64)))     # the first table pool, sampled
        if not args.no_cpu_baseline and world == 1:
            cpu = cpu_baseline(wl3, 0, seconds=args.cpu_seconds)
            counts = oracle_counts(wl3, [0, 16, 32, 48])
        line = {"metric": METRIC, "value": round(bat["value"], 3), "unit": UNIT,
                "ms_per_step": round(bat["total_ms"] / args.steps, 4), **base,
                "config": {"workload": BATCHED_WORKLOAD.format(A=bat["A"]), "cells_per_step_per_gpu": bat["cells"],
                           "l2": "working set (151 GB) far larger than L2; no flush", "tuned": bat["tuned"],
                           "parallelism": f"replicas x{world}"},
                "roofline": roofline(bat["sweep_ms"], bat["cells"], bat["alg_bytes"], counts, fp32_peak, sfu_peak, hbm,
                                     measured_traffic("batched", bat["cells"]), "sweep_kernel (all launch groups)",
                                     sm_max),
                "e2e": bat["e2e"], "gpu_launches": bat["launches_per_step"] * args.steps, "clocks": bat["clocks"],
                "setup_s": bat["setup_s"], "workspace_gb": bat["workspace_gb"],
                "fp32_peak_measured_tinst_s": round(fp32_meas / 2.0, 2)}
        if cpu:
            line["cpu_baseline"] = cpu
    elif want == "learned":
        line = {"metric": METRIC, "value": lrn["surrogate"]["atm_per_s"], "unit": "atm/s", **base,
                "config": {"workload": lrn["workload"]}}
    else:
        line = {"metric": METRIC, "value": sgl["gcell_s_l2_flushed"], "unit": UNIT,
                "ms_per_step": sgl["ms_per_step_l2_flushed"], **base, "config": {"workload": SINGLE_WORKLOAD}}
    if lrn:
        line["surrogate_vs_plain"] = lrn
    if sgl:
        wl2 = synth.config2()
        sc = oracle_counts(wl2, [0], chunks=4, nb=10, T_of=lambda a: synth.perturbed_profile(wl2.atms[0], 11, amp=200.0)) \
            if not args.no_cpu_baseline and world == 1 else None
        sgl["roofline_sweep_l2_flushed"] = roofline(sgl["sweep_ms_l2_flushed"], sgl["cells_per_step"], sgl.pop("alg_bytes"),
                                                   sc, fp32_peak, sfu_peak, hbm,
                                                   measured_traffic("single", sgl["cells_per_step"]),
                                                   "sweep_kernel<13, 2, false, 16>", sm_max)
        line["single_atmosphere"] = sgl
    if pln:
        if not args.no_cpu_baseline and world == 1:
            pln["oracle_host"] = oracle_timings(sgl["re_solve"]["iters"] if sgl else None)
        line["plain_single_atmosphere"] = pln
    print(json.dumps(line), flush=True)


def run_profile(args):
    """A short run for profilers: the chosen workload's plan, W warm-up and K timed RE steps
    through helios_re_step, nothing else (no extra sections, no CPU leg).  The batched plan's
    autotuning comes from the tuner's cache when an earlier run filled it, so that a profiled run
    launches the steps' kernels only."""
    import torch
    import synth
    import paper_1606_05474_b300 as hp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    if args.workload == "batched":
        wl = synth.config3(A=args.atmospheres, atm_ids=list(range(args.atmospheres)))
    else:
        wl = synth.config2()
        wl.atms[0].T_init = synth.perturbed_profile(wl.atms[0], 11, amp=200.0)
    ctx = hp.Context(0)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    prm = hp.default_params(col_lanes=args.col_lanes)
    if args.workload == "batched":
        prm = hp.autotune(ctx, wl.atms, wl.tables, kap, prm, cache_path=tune_cache_path())
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, prm)
    T = torch.from_numpy(np.concatenate([a.T_init for a in wl.atms])).to(dev)
    state = plan.new_state()
    for k in range(args.warmup + args.steps):
        plan.re_step(T, state, warm=k > 0)
    torch.cuda.synchronize()
    print(json.dumps({"profile_run": args.workload, "steps": args.steps, "warmup": args.warmup,
                      "atmospheres": len(wl.atms), "sweep_launches_per_step": plan.info.sweep_launches}))


def run_precision(args):
    """The high-resolution precision-stress workload at its stated size: 64 atmospheres x 200 layers
    x 30000 bins x 20 g with scattering, iterated to radiative equilibrium (eq. 29, tol 1e-7) on the
    GPU in one batched, graph-captured solve.  Reports converged atmospheres per second and the
    iteration statistics (the FP64 checks of sampled atmospheres are in the precision tests)."""
    import torch
    import synth
    import paper_1606_05474_b300 as hp
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    t0 = time.time()
    wl = synth.config5(A=64)
    t_gen = time.time() - t0
    ctx = hp.Context(0)
    kap = [torch.from_numpy(t.kappa32).to(dev) for t in wl.tables]
    plan = hp.Plan(ctx, wl.atms, wl.tables, kap, hp.default_params(max_iter=20000))
    T = torch.from_numpy(np.concatenate([a.T_init for a in wl.atms])).to(dev)
    torch.cuda.synchronize()
    t0 = time.time()
    iters, status = plan.solve_re(T)
    torch.cuda.synchronize()
    dt = time.time() - t0
    it, st = iters.cpu().numpy(), status.cpu().numpy()
    Tg = np.array(plan.split_layers(T.cpu().numpy()))
    line = {"metric": METRIC, "value": round(float((st == 1).sum()) / dt, 4), "unit": "atm/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 sweep / f64 temperature step", "data": "synthetic",
            "config": {"workload": "precision stress: 64 atmospheres x 200 layers x 30000 bins x 20 g, scattering, "
                                   "one solve to eq. (29) at tol 1e-7", "cells_per_evaluation": wl.cells},
            "wall_s": round(dt, 2), "converged": int((st == 1).sum()), "status_counts": np.bincount(st, minlength=4).tolist(),
            "iterations": {"min": int(it.min()), "median": float(np.median(it)), "max": int(it.max())},
            "T_range_K": [round(float(Tg.min()), 1), round(float(Tg.max()), 1)],
            "workspace_gb": round(plan.info.workspace_bytes / 1e9, 2), "inputs_s": round(t_gen, 2)}
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
    line = {
        "metric": "post-processing emission spectra/s (isothermal layers, exact column solve)",
        "value": round(world * 1e3 / res["exact"]["ms_per_spectrum"], 3), "unit": "spectra/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["exact"]["ms_per_spectrum"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 sweep / f64 sums",
        "data": "synthetic",
        "config": {"workload": "full-size atmosphere on 100 isothermal layers x 3000 bins x 20 g, scattering, cold start",
                   "cells": plan.info.cells, "l2": "flushed before every step", "parallelism": f"replicas x{world}"},
        "exact": res["exact"], "passes_81": res["passes_81"],
        "gpu_launches": 3 * 2 * args.steps,                      # prep, sweep, finalize per spectrum
    }
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The FP64 oracle on the host cores on the headline's workload (the batched ragged
    atmospheres), same metric and unit: each step is one RE iteration (flux evaluation + temperature
    step) of one atmosphere of the batch, cycling through atmospheres 0, 1, 2, ... (each with its own
    iteration state) -- a bounded sample of the batched step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    A = 8
    wl = synth.config3(A=A, atm_ids=list(range(A)))
    atms = [oracle.Atm.from_workload(wl, a) for a in range(A)]
    states = [oracle.State(atm, wl.atms[a].T_init) for a, atm in enumerate(atms)]
    p = oracle.params()
    done = [0] * A

    def one(i):
        a = i % A
        atm, st = atms[a], states[a]
        r = oracle.flux_sweep(atm, st.T, n_passes=oracle.passes(atm, p), warm=st.warm, warm_valid=done[a] > 0)
        oracle.temp_update(atm, st, r["Fup"], r["Fdn"], p)
        done[a] += 1
        return atm.n * atm.L * atm.G

    for i in range(args.warmup):
        one(i)
    t0 = time.time()
    cells = 0
    for i in range(args.steps):
        cells += one(args.warmup + i)
    dt = time.time() - t0
    v = cells / dt / 1e9
    cores = oracle.max_threads()                    # the OpenMP threads the oracle's loops used
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": BATCHED_WORKLOAD.format(A=4096),
                       "sample": f"each step: one RE iteration of one of the batch's first {A} atmospheres, in turn"},
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} RE iterations over atmospheres 0..{A - 1} of the batched workload "
                                       f"({cells} cells), {dt:.1f} s"},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline", choices=["headline", "single", "batched", "learned", "spectrum", "precision"])
    ap.add_argument("--atmospheres", type=int, default=4096)
    ap.add_argument("--col-lanes", type=int, default=0, choices=[0, 16, 32],
                    help="single atmosphere: lanes per column of the iterated sweep (0: automatic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--train", type=int, default=2048, help="surrogate vs plain: training planets per GPU")
    ap.add_argument("--test", type=int, default=512, help="surrogate vs plain: held-out planets per GPU")
    ap.add_argument("--bins", type=int, default=300, help="surrogate vs plain: bins per planet")
    ap.add_argument("--epochs", type=int, default=300, help="surrogate vs plain: training epochs")
    ap.add_argument("--profile", action="store_true",
                    help="a short run for profilers: warm-up + timed RE steps of the workload, nothing else")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile(args)
    elif args.workload == "spectrum":
        run_gpu_spectrum(args)
    elif args.workload == "precision":
        run_precision(args)
    else:
        headline(args)


if __name__ == "__main__":
    main()
