"""Benchmark: Newton steps per second on truncated power series in multiple
double arithmetic, one GB300 per rank.

Workload (default): quad double, real, n = 64 equations and unknowns,
16 monomials of 2..8 distinct variables per equation plus 64 x_i, series of
degree d = 31, planted solution; one "step" is one Newton step (evaluation
and differentiation, Householder QR of A0 and its inverse, forward
substitution over the 32 coefficient blocks, update and norms).  The timed
steps run as solves of 7 steps (the workload's step count) from the start
series, one mdn_newton call each, with CUDA events around every solve and
the L2 flushed between solves.

Output: one JSON line (rank 0).  ``value`` is Newton steps/s over all ranks
from CUDA events around each timed step (inputs resident in HBM, L2 flushed
between steps); ``e2e`` times whole solves through the public API with the
start series copied from pinned host memory and the solution copied back;
``roofline`` reports the phase with the largest share of device time: the
method's md multiply-adds of that phase per second, against the peak of the
pipe it runs on (integer instructions, measured at the start of the run by
peaks/peak_probe.cu), with the FP64-equivalent fraction and the paper's
Table 2 convention beside it; ``cpu_baseline`` times the CPU oracle on a
bounded sample (all host threads, and one step on a single thread).

``--impl reference`` times the CPU oracle (the plain multiple double
implementation the tests check the GPU against) on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2301_12659_gb300 import flops as F  # noqa: E402
from paper_2301_12659_gb300 import workloads as wl  # noqa: E402

# Roofline denominators: the peaks of the FP64 and integer pipes are measured
# at the start of every run by the microbenchmarks of
# paper_2301_12659_gb300/peaks/peak_probe.cu (PEAKS below), and reported in
# the JSON line.  The evaluation, the QR and the forward substitution
# compute md values in integer limbs (extended floats and fixed-point
# accumulators), so their pipe is the integer one: its peak is the measured
# rate of an even IMAD/LOP3 mix (the instruction kinds of that arithmetic).
# The method's work is counted in md multiply-adds (flops.method_counts);
# one real md multiply-add in integer limbs costs this many integer thread
# instructions (operand conversions and the accumulator included), measured
# with ncu on ed_kernel (profiles/ed_kernel_int_per_fma.md):
XF_INT_OPS_PER_FMA = {2: 169.6, 4: 406.6, 8: 957.7}
NUM_SMS = 152
PEAKS = {}

METRIC = "Newton steps/s (qd, n=64, d=31)"


def metric_of(cfg) -> str:
    """The metric name: the quad double workload's own, else named by its sizes."""
    if cfg.name == "qd-real-n64-d31":
        return METRIC
    prec = {1: "d", 2: "dd", 4: "qd", 8: "od"}[cfg.K] + (" complex" if cfg.C == 2 else "")
    return f"Newton steps/s ({prec}, n={cfg.n}, d={cfg.d})"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=70)
    ap.add_argument("--warmup", type=int, default=7)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="qd-real-n64-d31", choices=sorted({**wl.CONFIGS, **wl.EXTRA_CONFIGS}))
    ap.add_argument("--e2e-solves", type=int, default=5)
    ap.add_argument("--cpu-sample-steps", type=int, default=14)
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the CPU oracle (0: all cores; 1 times it single-threaded)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-single-thread", default="on", choices=["on", "off"],
                    help="also time one oracle step on a single host thread")
    ap.add_argument("--table4", action="store_true",
                    help="instead: Newton on the paper's Table 4 workloads (one- and two-column systems, "
                         "n=1024, 64 coefficients, octo double, 24 staggered steps) with per-phase times")
    ap.add_argument("--peaks", action="store_true",
                    help="instead: measure and print the FP64 and integer pipe peaks (peak_probe.cu)")
    ap.add_argument("--batched", default="on", choices=["on", "off"],
                    help="also time the batched workload (4096 quad double systems) and the same systems one by one")
    ap.add_argument("--adjoint", default="on", choices=["on", "off"],
                    help="also time the adjoint gradient of the double double n=64, d=31 workload")
    ap.add_argument("--one-by-one-sample", type=int, default=512,
                    help="systems of the batch solved one by one (stratified by size class; 0: all)")
    ap.add_argument("--batch-count", type=int, default=0,
                    help="systems of the batched workload (0: all 4096; fewer for profiling captures)")
    ap.add_argument("--staggered", default="on", choices=["on", "off"],
                    help="also time solves with staggered orders and the QR once")
    ap.add_argument("--ed-context", action="store_true",
                    help="instead: time the evaluation and differentiation of the paper's one-column "
                         "workload (n=1024 monomials x_0...x_i, 64 coefficients, octo double) against Table 5")
    ap.add_argument("--late-updates", type=int, default=0, metavar="FIRST_STAGE",
                    help="stated-accuracy variant: stages k >= FIRST_STAGE form their updates in K/2 limbs")
    return ap.parse_args()


# DRAM bytes (read + write) per launch of the phase's main kernel from one ncu
# capture of the unchanged kernels (profiles/ncu_qr_ed_fsub_qd-real-n64-d31.md:
# qr_kernel and fsub_kernel as they are now, ed_kernel from the earlier
# capture, unchanged since); absent entries report null.
NCU_TRAFFIC = {
    ("qd-real-n64-d31", "qr"): 438016 + 2816,
    ("qd-real-n64-d31", "evaluate"): 1294976,
    ("qd-real-n64-d31", "forward"): 4722944 + 6144,
}


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def aggregate_over_ranks(total_ms: float, steps: int, device=None):
    """Replicas: every rank ran `steps` Newton steps of its own copy of the
    workload (no collective on the data path).  Returns (max time over ranks
    in ms, whole-job steps/s = world * steps / max time)."""
    world = 1
    t_max = float(total_ms)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            import torch
            world = dist.get_world_size()
            t = torch.tensor([t_max], dtype=torch.float64, device=device)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_max = float(t.item())
    except ImportError:
        pass
    return t_max, world * steps / (t_max * 1e-3)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm and CPU baseline: the CPU oracle
# ---------------------------------------------------------------------------
def oracle_sample(cfg, nsteps, threads=0):
    """Time `nsteps` oracle Newton steps on the workload (host cores; all of
    them unless `threads` > 0)."""
    from oracle import oracle
    if threads > 0:
        oracle.set_threads(threads)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    t0 = time.perf_counter()
    oracle.newton(s, x0, nsteps)
    dt = time.perf_counter() - t0
    return dt, oracle.get_threads()


def oracle_single_thread_step(cfg):
    """Seconds of one oracle Newton step on one host thread, at the series
    that 5 steps reached (all host threads for those)."""
    from oracle import oracle
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x5, _ = oracle.newton(s, x0, 5)
    all_threads = oracle.get_threads()
    oracle.set_threads(1)
    t0 = time.perf_counter()
    oracle.newton(s, x5, 1)
    dt = time.perf_counter() - t0
    oracle.set_threads(all_threads)
    return dt


def run_reference(args, cfg):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import oracle
    if args.cpu_threads > 0:
        oracle.set_threads(args.cpu_threads)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = oracle.planted_constant(s, xstar)
    x = x0
    for i in range(args.warmup):
        x, _ = oracle.newton(s, x0 if i % cfg.steps == 0 else x, 1)
    times = []
    x = x0
    for i in range(args.steps):
        t0 = time.perf_counter()
        x, _ = oracle.newton(s, x0 if i % cfg.steps == 0 else x, 1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    v = args.steps / total
    cores = oracle.get_threads()
    line = {
        "impl": "reference", "metric": metric_of(cfg), "value": v, "unit": "steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(cfg),
        "data": "synthetic", "config": config_dict(cfg, args),
        "cpu_baseline": {"value": v, "unit": "steps/s", "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} oracle Newton steps of the workload on {cores} host threads"},
        "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def dtype_name(cfg):
    return {1: "f64", 2: "f64x2 (double double)", 4: "f64x4 (quad double)", 8: "f64x8 (octo double)"}[cfg.K] + \
        (" complex" if cfg.C == 2 else "")


def config_dict(cfg, args):
    late = {"late_updates": {"first_stage": args.late_updates, "limbs": cfg.K // 2}} if args.late_updates else {}
    return {**late, "workload": cfg.name, "limbs": cfg.K, "complex": cfg.C == 2, "n": cfg.n, "degree": cfg.d,
            "monomials_per_equation": cfg.mono_per_eq, "vars_per_monomial": [cfg.kmin, cfg.kmax],
            "newton_steps_per_solve": cfg.steps, "parallelism": f"replicas x{args.gpus}",
            "l2": "flushed between timed solves (256 MiB write); steps run in solves of "
                  f"{cfg.steps} from the start series"}


# ---------------------------------------------------------------------------
# the batched workload and the adjoint (extra objects of the JSON line)
# ---------------------------------------------------------------------------
def run_batched(args, dev):
    """4096 independent quad double systems in one persistent launch (graph
    replay), against the same systems solved one by one through mdn_newton
    (a stratified sample, each run for the number of updates the batch gave
    it, scaled by the class counts)."""
    import torch
    from paper_2301_12659_gb300 import autotune
    from paper_2301_12659_gb300 import mdnewton as md

    bcfg = wl.BATCH_CONFIGS["qd-real-batch4096"]
    t0 = time.perf_counter()
    items = wl.batch_planted_systems(bcfg, args.batch_count or None)
    gen_s = time.perf_counter() - t0
    threads, bps, entry = autotune.batch_tiles(items, bcfg.max_steps, bcfg.tol)
    systems = [s for s, _, _ in items]
    b = md.Batch(systems, threads, bps)
    b.set_constant(-b.evaluate(b.pack([xs for _, xs, _ in items])))
    x0 = b.pack([x0 for _, _, x0 in items])
    x = torch.empty_like(x0)
    b.solve(x0, bcfg.max_steps, bcfg.tol, x)  # warm-up: captures the graph
    times = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, steps, flags = b.solve(x0, bcfg.max_steps, bcfg.tol, x)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = min(times)
    worst = 0.0
    xs = b.unpack(x)
    for q in range(0, len(items), 64):  # leading-limb spot check against the plant
        worst = max(worst, float(np.max(np.abs(xs[q][0] - items[q][1][0]))))
    cst = b.unpack(b.cst)
    # one by one, on a stratified sample
    idx = (list(range(len(systems))) if args.one_by_one_sample <= 0 or args.one_by_one_sample >= len(systems)
           else autotune._stratified(systems, args.one_by_one_sample, seed=1))
    per_class = {}
    for q in idx:
        s = systems[q]
        s.cst = cst[q]
        nw = md.Newton(s)
        nw.set_series(items[q][2])
        nw.newton(max(1, int(steps[q])))
        torch.cuda.synchronize()
        nw.set_series(items[q][2])
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        md.mdn_newton(nw.ctx, max(1, int(steps[q])), 0.0)
        e1.record()
        torch.cuda.synchronize()
        per_class.setdefault((s.n, s.d), []).append(e0.elapsed_time(e1))
        nw.close()
    counts = {}
    for s in systems:
        counts[(s.n, s.d)] = counts.get((s.n, s.d), 0) + 1
    # algorithmic work of the updates applied (one evaluation, QR and forward
    # substitution per update; the stopping evaluations not counted): FP64
    # operations of md.cuh's algorithms, and the method's md multiply-adds
    ops, mfma = 0.0, 0.0
    for q, s in enumerate(systems):
        ops += float(steps[q]) * F.step_counts(s.monomial_sizes(), s.n, s.D, s.K, s.C)["fp64_ops"]
        mc = F.method_counts(s.monomial_sizes(), s.n, s.D, s.C)
        mfma += float(steps[q]) * mc["real_factor"] * (mc["evaluate"] + mc["qr"] + mc["updates"] + mc["qhb"] + mc["bs"])
    one_ms = sum(counts[c] * float(np.mean(v)) for c, v in per_class.items())
    spread = {f"n={c[0]},d={c[1]}": {"in_batch": counts[c], "timed": len(v), "ms_mean": float(np.mean(v)),
                                     "ms_min": float(np.min(v)), "ms_max": float(np.max(v))}
              for c, v in sorted(per_class.items())}
    b.close()
    return {
        "workload": bcfg.name, "systems": len(items), "solves_per_s": len(items) / (ms * 1e-3),
        "ms_per_batch": ms, "tiles": {"threads_per_block": threads, "blocks_per_sm": bps,
                                      "source": "autotuner cache" if "timings" in entry else "tuned"},
        "updates": int(np.sum(steps)), "converged": int(np.sum(flags == md.BATCH_CONVERGED)),
        "max_leading_limb_error_vs_plant_sampled": worst, "gpu_launches_per_batch": 1,
        "one_by_one": {"solves_per_s": len(items) / (one_ms * 1e-3), "ms_total_estimate": one_ms,
                       "sample": f"{len(idx)} of the {len(items)} systems (stratified by (n, d)), each through "
                                 "mdn_newton for the number of updates the batch applied to it; class means "
                                 "scaled by the class counts",
                       "per_class": spread},
        "speedup_vs_one_by_one": one_ms / ms, "generate_s": gen_s,
        "roofline": {"bound": "alu", "kernel": "batch_kernel", "md_fma_per_launch": mfma,
                     "md_fma_per_s": mfma / (ms * 1e-3),
                     "achieved": mfma * XF_INT_OPS_PER_FMA[bcfg.K] / (ms * 1e-3) / 1e12,
                     "peak": PEAKS["int_mix"]["ops_per_s"] / 1e12, "unit": "integer Tops/s",
                     "frac": mfma * XF_INT_OPS_PER_FMA[bcfg.K] / (ms * 1e-3) / PEAKS["int_mix"]["ops_per_s"],
                     "peak_source": "IMAD/LOP3 mix of peak_probe.cu, measured in this run",
                     "work": "the method's md multiply-adds of the updates applied x integer instructions per "
                             "multiply-add (ncu, ed_kernel); the products of the evaluation run in integer limbs, "
                             "the QR and the forward substitution in FP64 md operations",
                     "fp64_equivalent": {"ops_per_launch": ops, "achieved": ops / (ms * 1e-3) / 1e12,
                                         "peak": PEAKS["fp64_fma"]["ops_per_s"] / 1e12, "unit": "FP64 Tops/s",
                                         "frac": ops / (ms * 1e-3) / PEAKS["fp64_fma"]["ops_per_s"]}},
        "l2": "working set larger than L2 (GBs of Jacobians)",
    }


def run_staggered(nw, cfg, x0_dev, xs_dev, plain_solve_ms):
    """Solves with staggered orders and the QR once (Sections 4 and 5.3):
    order-1 steps with a QR each until x_0 is accurate, then orders
    1 -> 2 -> 4 -> 7 -> ... -> d+1 reusing the last QR, to the plant."""
    import torch
    from paper_2301_12659_gb300 import mdnewton as md

    first = {2: 4, 4: 5, 8: 6}.get(cfg.K, 5)
    L, growth = 1, 0
    while L < cfg.d + 1:
        L, growth = min(cfg.d + 1, L + 1 + L // 2), growth + 1
    steps = first + growth + 2
    nw.set_stagger(first)
    times = []
    for rep in range(4):
        nw.set_series(x0_dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        md.mdn_newton(nw.ctx, steps, 0.0)
        e1.record()
        torch.cuda.synchronize()
        if rep:
            times.append(e0.elapsed_time(e1))
    err = (nw.series() - xs_dev)[0].abs().max().item()
    nw.set_stagger(0)
    ms = statistics.median(times)
    return {"first_order_steps": first, "steps_per_solve": steps, "solve_ms": ms, "plain_solve_ms": plain_solve_ms,
            "speedup_vs_plain_solve": plain_solve_ms / ms, "max_leading_limb_error_vs_plant": err}


def run_adjoint(args, dev):
    """Gradient of the Fabry-ratio loss of the converged dd n=64 d=31 series
    with respect to every coefficient series (mdn_fabry_loss + mdn_adjoint)."""
    import torch
    from paper_2301_12659_gb300 import mdnewton as md

    acfg = wl.ADJOINT_CONFIG
    s, xstar, x0 = wl.planted_system(acfg)
    s.cst = None
    nw = md.Newton(s)
    nw.set_constant(-nw.evaluate(xstar, want_A=False))
    nw.set_series(x0)
    nw.newton(acfg.steps)
    x = nw.series()
    loss, g = nw.fabry_loss(x)
    grad = nw.adjoint(x, g)
    torch.cuda.synchronize()
    md.mdn_profile(nw.ctx, 1)
    reps = 10
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        loss, g = nw.fabry_loss(x)
        grad = nw.adjoint(x, g)
    e1.record()
    torch.cuda.synchronize()
    _, phase_ms, _ = md.mdn_profile(nw.ctx, 0)
    ms = e0.elapsed_time(e1) / reps
    counts = F.adjoint_counts(s.monomial_sizes(), s.n, s.D, s.K, s.C)
    qr_ms = float(phase_ms[md.PHASES.index("qr")]) / reps
    out = {"workload": acfg.name, "gradients_per_s": 1e3 / ms, "ms_per_gradient": ms,
           "roofline": {"bound": "alu", "fp64_ops_per_gradient": counts["fp64_ops"],
                        "frac": counts["fp64_ops"] / (ms * 1e-3) / PEAKS["fp64_fma"]["ops_per_s"],
                        "dominant_kernel": "qr",
                        "qr_frac": counts["qr_fp64_ops"] / (qr_ms * 1e-3) / PEAKS["fp64_fma"]["ops_per_s"]
                        if qr_ms > 0 else None,
                        "peak": PEAKS["fp64_fma"]["ops_per_s"] / 1e12, "unit": "FP64 Tops/s",
                        "note": "FP64-equivalent: the md algorithms' FP64 operation count against the FP64 "
                                "pipe; the QR, the evaluation and the solve run in integer limbs"},
           "gradient_entries": int(grad.numel() // acfg.K), "loss_leading": float(loss[0]),
           "phases_ms_per_gradient": {p: float(v) / reps for p, v in zip(md.PHASES, phase_ms)}}
    nw.close()
    return out


def measure_peaks():
    """The FP64 and integer pipe peaks of this GPU, measured now."""
    from paper_2301_12659_gb300 import peaks
    PEAKS.clear()
    PEAKS.update(peaks.measure())
    return PEAKS


def phase_rooflines(cfg, s, ms_per_step):
    """Per phase (evaluation, QR of A0, forward substitution): the method's
    md multiply-adds per step (flops.method_counts; the QR counts its
    (2/3) n^3 multiply-adds, not the inverse this library forms from it),
    their rate, the paper-convention GFLOPS (Table 2 multiplication
    weights) and the fraction of the measured integer pipe peak (integer
    instructions per md multiply-add from ncu; where no figure exists for
    the limb count, the FP64-equivalent fraction of the measured FP64 peak
    is the main one)."""
    m = F.method_counts(s.monomial_sizes(), s.n, s.D, s.C)
    work = {"evaluate": m["evaluate"], "qr": m["qr"], "forward": m["updates"] + m["qhb"] + m["bs"]}
    kernel = {"evaluate": "ed_kernel", "qr": "qr_kernel", "forward": "fsub_kernel"}
    real = m["real_factor"]
    cost = XF_INT_OPS_PER_FMA.get(cfg.K)
    fp64_per_fma = F.md_ops(cfg.K)["acc_fma"]
    int_peak = PEAKS["int_mix"]["ops_per_s"]
    fp64_peak = PEAKS["fp64_fma"]["ops_per_s"]
    out = {}
    for p, w in work.items():
        t = ms_per_step[p] * 1e-3
        if t <= 0:
            continue
        rate = w * real / t  # real md multiply-adds per second
        fp64 = {"achieved": rate * fp64_per_fma / 1e12, "peak": fp64_peak / 1e12, "unit": "FP64 Tops/s",
                "frac": rate * fp64_per_fma / fp64_peak,
                "note": f"{fp64_per_fma} FP64 operations per md multiply-add of md.cuh's algorithms"}
        r = {"bound": "alu", "kernel": kernel[p], "md_fma_per_step": w * real, "md_fma_per_s": rate,
             "paper_gflops": w * real * F.PAPER_MUL_COST[cfg.K] / t / 1e9, "fp64_equivalent": fp64}
        if cost:
            r.update({"achieved": rate * cost / 1e12, "peak": int_peak / 1e12, "unit": "integer Tops/s",
                      "frac": rate * cost / int_peak,
                      "peak_source": "IMAD/LOP3 mix of peak_probe.cu, measured in this run",
                      "work": f"method md multiply-adds x {cost:g} integer instructions per multiply-add "
                              "(ncu, ed_kernel)"})
        else:
            r.update({k: fp64[k] for k in ("achieved", "peak", "unit", "frac")})
            r["peak_source"] = "FP64 FMA of peak_probe.cu, measured in this run"
            r["work"] = "method md multiply-adds x FP64 operations per multiply-add (an equivalent)"
        out[p] = r
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args, cfg):
    import torch
    from paper_2301_12659_gb300 import mdnewton as md

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    measure_peaks()
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = None
    nw = md.Newton(s)
    if args.late_updates:
        nw.set_late_updates(args.late_updates, cfg.K // 2)
    # constant term planting x*: minus the system at x* (evaluated here)
    cst = -nw.evaluate(xstar, want_A=False)
    nw.set_constant(cst)
    x0_dev = torch.as_tensor(x0, device=dev)
    # correctness check of this run: recover the plant within the tolerance
    nw.set_series(x0_dev)
    nw.newton(cfg.steps)
    xs_dev = torch.as_tensor(xstar, device=dev)
    x = nw.series()
    diff = (x - xs_dev)[0].abs().max().item()  # leading limbs: a coarse check only
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(local)

    def solve_chunks(total):
        # Newton steps in solves of cfg.steps from the start series (the last
        # one shorter); each solve is one mdn_newton call
        out, left = [], total
        while left > 0:
            out.append(min(cfg.steps, left))
            left -= out[-1]
        return out

    def run_solve(nsteps):
        nw.set_series(x0_dev)
        st, done, _ = md.mdn_newton(nw.ctx, nsteps, 0.0)
        if st != md.MDN_OK or done != nsteps:
            raise md.MdnError(st, md.mdn_last_error(nw.ctx))

    for c in solve_chunks(args.warmup):
        run_solve(c)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    md.mdn_profile(nw.ctx, 1)
    evs = []
    t_wall = time.perf_counter()
    for c in solve_chunks(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_solve(c)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    _, phase_ms, launches = md.mdn_profile(nw.ctx, 0)
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    t_max, value = aggregate_over_ranks(total_ms, args.steps, device=dev)
    if world > 1:
        torch.distributed.barrier()

    # end to end: whole solves from pinned host memory through the API
    x0_host = torch.from_numpy(x0).pin_memory()
    x_host = torch.empty_like(x0_host).pin_memory()
    hist = None
    e2e_ms = []
    for rep in range(args.e2e_solves + 1):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        x0_dev.copy_(x0_host, non_blocking=True)
        nw.set_series(x0_dev)
        st, done, hist = md.mdn_newton(nw.ctx, cfg.steps, 0.0)
        x_out = nw.series()
        x_host.copy_(x_out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = world * cfg.steps / (statistics.median(e2e_ms) * 1e-3)
    nbytes = x0.nbytes

    # roofline of the phase with the largest share of device time, in the
    # method's work (md multiply-adds, flops.method_counts) against the
    # measured peak of the pipe it runs on
    counts = F.step_counts(s.monomial_sizes(), s.n, s.D, s.K, s.C)
    steps_timed = args.steps
    share = {p: float(ms) for p, ms in zip(md.PHASES, phase_ms)}
    roof = phase_rooflines(cfg, s, {p: share[p] / steps_timed for p in md.PHASES})
    dom = max(("evaluate", "qr", "forward"), key=lambda p: share[p])
    main_roof = dict(roof[dom])
    main_roof["traffic"] = NCU_TRAFFIC.get((cfg.name, dom))
    line = {
        "metric": metric_of(cfg), "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(cfg), "data": "synthetic",
        "config": config_dict(cfg, args),
        "roofline": main_roof,
        "phases_ms_per_step": {p: share[p] / steps_timed for p in md.PHASES},
        "phase_rooflines": roof,
        "peaks": PEAKS,
        "step_fp64_ops": counts["fp64_ops"], "step_paper_flops": counts["paper_flops"],
        "e2e": {"value": e2e_value, "unit": "steps/s", "h2d_bytes_per_step": nbytes / cfg.steps,
                "d2h_bytes_per_step": (nbytes + 24 * cfg.steps) / cfg.steps,
                "solve_ms": statistics.median(e2e_ms)},
        "gpu_launches": int(np.sum(launches)),
        "clocks": clk,
        "check": {"max_leading_limb_error_vs_plant": diff, "final_norm_f": float(hist[-1, 0]) if hist is not None else None},
        "wall_s_timed_region": t_wall,
    }
    if args.staggered == "on" and not args.late_updates:
        line["staggered"] = run_staggered(nw, cfg, x0_dev, xs_dev, total_ms / args.steps * cfg.steps)
    if args.batched == "on":
        line["batched"] = run_batched(args, dev)
    if args.adjoint == "on":
        line["adjoint"] = run_adjoint(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, cores = oracle_sample(cfg, args.cpu_sample_steps, args.cpu_threads)
        line["cpu_baseline"] = {"value": args.cpu_sample_steps / dt, "unit": "steps/s", "cores": cores,
                                "kind": "oracle", "host_cpus": os.cpu_count(),
                                "sample": f"{args.cpu_sample_steps} oracle Newton steps from the start series"}
        if args.cpu_single_thread:
            dt1 = oracle_single_thread_step(cfg)
            line["cpu_baseline"]["single_thread"] = {
                "value": 1.0 / dt1, "unit": "steps/s", "cores": 1, "kind": "oracle",
                "sample": "1 oracle Newton step at the series after 5 steps (a late step, whose full-width "
                          "coefficients make it the costliest of a solve) on one host thread"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    nw.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_ed_context(args):
    """Evaluation and differentiation of one column of 1024 monomials with a
    triangular exponent matrix of ones, 64 coefficients, real octo double:
    the workload of the paper's Table 5, reported in the paper's convention
    (3k-5 products per monomial of k variables, 64^2 multiplications per
    product, 1742 flops per octo double multiplication) beside this
    library's own FP64 operation count."""
    import torch
    from paper_2301_12659_gb300 import mdnewton as md

    measure_peaks()
    n, d, K = 1024, 63, 8
    D = d + 1
    s, x = wl.one_column_system(n, d, K)
    nw = md.Newton(s)
    xd = torch.as_tensor(x, device="cuda")
    f = torch.empty((K, 1, n, D), dtype=torch.float64, device="cuda")
    A = torch.empty((K, 1, D, n, n), dtype=torch.float64, device="cuda")
    md.mdn_evaluate(nw.ctx, xd, f, A)
    torch.cuda.synchronize()
    times = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = md.mdn_evaluate(nw.ctx, xd, f, A)
        e1.record()
        torch.cuda.synchronize()
        if st != md.MDN_OK:
            raise md.MdnError(st, md.mdn_last_error(nw.ctx))
        times.append(e0.elapsed_time(e1))
    ms = min(times)
    sizes = s.monomial_sizes()
    paper_flops = float(sum(max(0, 3 * int(k) - 5) for k in sizes)) * D * D * 1742.0
    ops = F.ed_counts(sizes, D, K, 1)["fp64_ops"]
    line = {"context": "the paper's Table 5 workload: one column of 1024 monomials, triangular exponents, "
                       "64 coefficients, real octo double; evaluation and differentiation only",
            "ms": ms, "paper_convention_gflops": paper_flops / (ms * 1e-3) / 1e9,
            "paper_table5_gflops_order64": {"P100": 554.654, "V100": 1658.382, "A100": 2568.016},
            "fp64_ops": ops, "fp64_frac": ops / (ms * 1e-3) / PEAKS["fp64_fma"]["ops_per_s"],
            "check_f0_leading": float(f[0, 0, n - 1, 0])}
    print(json.dumps(line), flush=True)
    nw.close()


# Table 4 of the paper (V100, octo double, n = 1024, 64 coefficients, 24 Newton
# steps): kernel seconds by kind and the wall time, one and two columns.
TABLE4_V100 = {
    1: {"convolutions": 121.386, "qr": 24.451, "qhb": 5.849, "bs": 17.053, "updates": 111.474,
        "residuals": 125.122, "all_kernels": 405.334, "wall": 1129.794},
    2: {"convolutions": 244.535, "qr": 24.123, "qhb": 6.139, "bs": 17.884, "updates": 124.080,
        "residuals": 137.963, "all_kernels": 554.723, "wall": 1808.480},
}


def run_table4(args):
    """The paper's Table 4 runs: Newton on the one- and two-column systems of
    Section 3 at n = 1024 with 64 coefficients in real octo double, 24 steps
    with staggered orders (6 steps on x_0 alone, each with its QR of A_0,
    then 1 -> 2 -> 4 -> 7 -> ... -> 64 coefficients reusing the last QR:
    Sections 4 and 5.3).  Device seconds per phase (mdn_profile) in the
    paper's kernel categories, beside its V100 row (context: another GPU)."""
    import torch
    from paper_2301_12659_gb300 import mdnewton as md

    torch.cuda.set_device(dist_info()[2])
    measure_peaks()
    out = {"context": "the paper's Table 4 workloads: one- and two-column systems of Section 3, n = 1024, "
                      "64 coefficients, real octo double, 24 Newton steps with staggered orders and the QR once",
           "runs": []}
    steps, first = 24, 6
    for columns in (1, 2):
        s, x0 = wl.section3_system(1024, 63, 8, columns)
        nw = md.Newton(s)
        nw.set_stagger(first)
        x0d = torch.as_tensor(x0, device="cuda")
        nw.set_series(x0d)
        md.mdn_newton(nw.ctx, 2, 0.0)  # warm-up (module loads, first launches)
        torch.cuda.synchronize()
        nw.set_series(x0d)
        md.mdn_profile(nw.ctx, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        st, done, hist = md.mdn_newton(nw.ctx, steps, 0.0)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        _, phase_ms, launches = md.mdn_profile(nw.ctx, 0)
        alpha = s.meta["alpha"]
        x = nw.series()[0, 0].cpu().numpy()
        fact = np.array([float(np.prod(np.arange(1, j + 1))) for j in range(s.D)])
        ref = alpha[:, None] ** np.arange(s.D)[None, :] / fact[None, :]
        ph = {p: float(v) / 1e3 for p, v in zip(md.PHASES, phase_ms)}
        out["runs"].append({
            "columns": columns, "status": md.STATUS.get(st, st), "steps": done,
            "device_s": e0.elapsed_time(e1) / 1e3, "wall_s": wall,
            "newton_steps_per_s": done / (e0.elapsed_time(e1) / 1e3),
            "phases_s": {"convolutions (evaluate + assemble)": ph["evaluate"] + ph["assemble"],
                         "qr (QR of A_0 with Q^H and R^{-1}, forming A_0^{-1})": ph["qr"],
                         "updates + residuals (forward substitution, fused monitor)": ph["forward"],
                         "update of x and norms": ph["update"]},
            "gpu_launches": int(np.sum(launches)),
            "final_norms": [float(v) for v in hist[-1]],
            "leading_limb_error_vs_exp_alpha_t": float(np.max(np.abs(x - ref))),
            "paper_v100_seconds": TABLE4_V100[columns],
        })
        nw.close()
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.table4:
        run_table4(args)
        return
    if args.peaks:
        import torch
        torch.cuda.set_device(dist_info()[2])
        print(json.dumps({"peaks": measure_peaks()}), flush=True)
        return
    if args.ed_context:
        run_ed_context(args)
        return
    cfg = {**wl.CONFIGS, **wl.EXTRA_CONFIGS}[args.config]
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
