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
``roofline`` reports the phase with the largest share of device time against
the integer pipe peak (its md multiply-adds x the integer instructions one
costs in integer limbs); ``cpu_baseline`` times the CPU oracle on a bounded
sample.

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

# FP64 pipe peak of one GB300: 152 SMs x 1.684 FP64 lane operations per clock
# per SM (measured: one warp instruction per 64 cycles per sub-partition,
# ~76 with all four busy) x the 2070 MHz maximum SM clock.
FP64_LANES_PER_CLK_PER_SM = 1.684
NUM_SMS = 152
SM_MAX_MHZ = 2070.0
FP64_PEAK_OPS = NUM_SMS * FP64_LANES_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6
# Integer pipe peak: 152 SMs x 64 integer lane operations per clock per SM
# (measured: IMAD and LOP3 each) x 2070 MHz.  The evaluation, the QR and the
# forward substitution compute md values in integer limbs (extended floats
# and fixed-point accumulators), so their roofline is this pipe.
INT_LANES_PER_CLK_PER_SM = 64
INT_PEAK_OPS = NUM_SMS * INT_LANES_PER_CLK_PER_SM * SM_MAX_MHZ * 1e6
# Integer thread instructions per md multiply-add in integer limbs, by
# limbs (real data): measured with ncu on ed_kernel at the quad double
# workload, 2.591e9 integer instructions for 12 070 x 528 = 6.37e6
# multiply-adds (operand conversions and the accumulator included).
XF_INT_OPS_PER_FMA = {4: 406.6}

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
    ap.add_argument("--config", default="qd-real-n64-d31", choices=sorted(wl.CONFIGS))
    ap.add_argument("--e2e-solves", type=int, default=5)
    ap.add_argument("--cpu-sample-steps", type=int, default=14)
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the CPU oracle (0: all cores; 1 times it single-threaded)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched", default="on", choices=["on", "off"],
                    help="also time the batched workload (4096 quad double systems) and the same systems one by one")
    ap.add_argument("--adjoint", default="on", choices=["on", "off"],
                    help="also time the adjoint gradient of the double double n=64, d=31 workload")
    ap.add_argument("--one-by-one-sample", type=int, default=48)
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
# capture of the unchanged kernels (profiles/ncu_qr_ed_fsub_qd-real-n64-d31.md);
# absent entries report null.
NCU_TRAFFIC = {
    ("qd-real-n64-d31", "qr"): 603904 + 8448,
    ("qd-real-n64-d31", "evaluate"): 1294848,
    ("qd-real-n64-d31", "forward"): 4622592 + 42368,
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
    idx = autotune._stratified(systems, args.one_by_one_sample, seed=1)
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
    # algorithmic FP64 operations of the updates applied (one evaluation, QR
    # and forward substitution per update; the stopping evaluations not counted)
    ops = 0.0
    for q, s in enumerate(systems):
        ops += float(steps[q]) * F.step_counts(s.monomial_sizes(), s.n, s.D, s.K, s.C)["fp64_ops"]
    one_ms = sum(counts[c] * float(np.mean(v)) for c, v in per_class.items())
    b.close()
    return {
        "workload": bcfg.name, "systems": len(items), "solves_per_s": len(items) / (ms * 1e-3),
        "ms_per_batch": ms, "tiles": {"threads_per_block": threads, "blocks_per_sm": bps,
                                      "source": "autotuner cache" if "timings" in entry else "tuned"},
        "updates": int(np.sum(steps)), "converged": int(np.sum(flags == md.BATCH_CONVERGED)),
        "max_leading_limb_error_vs_plant_sampled": worst, "gpu_launches_per_batch": 1,
        "one_by_one": {"solves_per_s": len(items) / (one_ms * 1e-3), "ms_total_estimate": one_ms,
                       "sample": f"{len(idx)} systems stratified by (n, d), each through mdn_newton for the "
                                 "number of updates the batch applied to it, scaled by the class counts"},
        "speedup_vs_one_by_one": one_ms / ms, "generate_s": gen_s,
        "roofline": {"bound": "alu", "kernel": "batch_kernel", "ops_per_launch": ops,
                     "achieved": ops / (ms * 1e-3) / 1e12, "peak": FP64_PEAK_OPS / 1e12, "unit": "FP64 Tops/s",
                     "frac": ops / (ms * 1e-3) / FP64_PEAK_OPS},
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
                        "frac": counts["fp64_ops"] / (ms * 1e-3) / FP64_PEAK_OPS,
                        "dominant_kernel": "qr",
                        "qr_frac": counts["qr_fp64_ops"] / (qr_ms * 1e-3) / FP64_PEAK_OPS if qr_ms > 0 else None,
                        "peak": FP64_PEAK_OPS / 1e12, "unit": "FP64 Tops/s",
                        "note": "FP64-equivalent: the md algorithms' FP64 operation count against the FP64 "
                                "pipe; the QR, the evaluation and the solve run in integer limbs"},
           "gradient_entries": int(grad.numel() // acfg.K), "loss_leading": float(loss[0]),
           "phases_ms_per_gradient": {p: float(v) / reps for p, v in zip(md.PHASES, phase_ms)}}
    nw.close()
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

    # roofline of the phase with the largest share of device time
    counts = F.step_counts(s.monomial_sizes(), s.n, s.D, s.K, s.C)
    steps_timed = args.steps
    share = {p: float(ms) for p, ms in zip(md.PHASES, phase_ms)}
    md_fma = {"evaluate": counts["evaluate"]["md_fma"], "qr": counts["solve"]["qr_md_fma"],
              "forward": counts["solve"]["forward_md_fma"]}
    dom = max(md_fma, key=lambda p: share[p])
    dom_launch_ms = share[dom] / steps_timed
    eval_ms = share["evaluate"] / steps_timed
    unit_cost = XF_INT_OPS_PER_FMA.get(cfg.K) if cfg.C == 1 else None
    if unit_cost:
        # algorithmic md multiply-adds x integer instructions per multiply-add
        per_phase_ops = {p: v * unit_cost for p, v in md_fma.items()}
        peak, unit = INT_PEAK_OPS, "int Tops/s"
        peak_source = "derived: 152 SMs x 64 integer lanes/clk/SM (measured IMAD/LOP3) x 2070 MHz"
        work = f"{md_fma[dom]} md multiply-adds x {unit_cost:g} integer instructions each (ncu, ed_kernel)"
    else:
        # no measured integer cost for these limbs: the FP64 operations the md
        # algorithms would take, against the FP64 pipe (an equivalent, which
        # exceeds 1 where the kernels run in integer limbs instead)
        per_phase_ops = {"evaluate": counts["evaluate"]["fp64_ops"], "qr": counts["solve"]["qr_fp64_ops"],
                         "forward": counts["solve"]["forward_fp64_ops"]}
        peak, unit = FP64_PEAK_OPS, "FP64-equivalent Tops/s"
        peak_source = "derived: 152 SMs x 1.684 FP64 lanes/clk/SM (measured) x 2070 MHz"
        work = ("FP64 operations of the md algorithms (flops.py); the evaluation, QR and forward "
                "substitution run in integer limbs, so this is an equivalent, not a pipe fraction")
    achieved = per_phase_ops[dom] / (dom_launch_ms * 1e-3)
    line = {
        "metric": metric_of(cfg), "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype_name(cfg), "data": "synthetic",
        "config": config_dict(cfg, args),
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved / 1e12, "peak": peak / 1e12,
                     "unit": unit, "frac": achieved / peak,
                     "traffic": NCU_TRAFFIC.get((cfg.name, dom)),
                     "peak_source": peak_source, "ops_per_launch": per_phase_ops[dom], "work": work},
        "phases_ms_per_step": {p: share[p] / steps_timed for p in md.PHASES},
        "evaluate_roofline_frac": (per_phase_ops["evaluate"] / (eval_ms * 1e-3)) / peak if eval_ms > 0 else None,
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
                                "kind": "oracle",
                                "sample": f"{args.cpu_sample_steps} oracle Newton steps from the start series"}
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
            "fp64_ops": ops, "fp64_frac": ops / (ms * 1e-3) / FP64_PEAK_OPS,
            "check_f0_leading": float(f[0, 0, n - 1, 0])}
    print(json.dumps(line), flush=True)
    nw.close()


def main():
    args = parse()
    if args.ed_context:
        run_ed_context(args)
        return
    cfg = wl.CONFIGS[args.config]
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
