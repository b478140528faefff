"""Tile autotuner of the batched solver (mdn_batch_*).

The tiles are the block size (threads per block) and the number of resident
blocks per SM of the persistent kernel.  For a batch, the tuner times one
solve of a stratified sample of its systems (every size class in proportion)
for every candidate the kernel's register count admits, keeps the fastest,
and caches the choice in a JSON file keyed by GPU name, limbs, real/complex
and the batch's size classes.  Later runs read the cache.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned", "batch_tiles.json")
CANDIDATES = [(128, 0), (128, 1), (128, 2), (256, 0), (256, 1), (512, 0)]


def signature(systems) -> str:
    K, C = systems[0].K, systems[0].C
    classes = sorted({(s.n, s.d) for s in systems})
    return f"K{K}C{C}|" + ",".join(f"{n}x{d}" for n, d in classes)


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _load() -> dict:
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _stratified(systems, count: int, seed: int = 0):
    """Indices of about `count` systems, every (n, d) class in proportion."""
    rng = np.random.default_rng(seed)
    by = {}
    for q, s in enumerate(systems):
        by.setdefault((s.n, s.d), []).append(q)
    frac = min(1.0, count / max(1, len(systems)))
    pick = []
    for qs in by.values():
        k = max(1, int(round(frac * len(qs))))
        pick.extend(rng.choice(qs, size=min(k, len(qs)), replace=False).tolist())
    return sorted(pick)


def tune(items, max_steps: int, tol: float, sample: int = 4096, candidates=CANDIDATES, log=None):
    """Times every admissible candidate on a sample of `items` ((system,
    x*, x0) triples; the constant terms are planted here) and returns
    (threads, blocks_per_sm, table of timings).  The objective is the
    throughput of a whole batch, so the sample must hold many systems per
    resident block: on small samples the slowest single system decides and
    fewer, larger blocks win (measured: 512 systems favour 256 x 1, the full
    4096 favour 128 x 4)."""
    import torch
    from . import mdnewton as md

    idx = _stratified([s for s, _, _ in items], sample)
    sub = [items[q] for q in idx]
    systems = [s for s, _, _ in sub]
    table = []
    best = None
    for threads, bps in candidates:
        try:
            b = md.Batch(systems, threads, bps)
        except md.MdnError:
            continue
        xstar = b.pack([xs for _, xs, _ in sub])
        b.set_constant(-b.evaluate(xstar))
        x0 = b.pack([x0 for _, _, x0 in sub])
        x = torch.empty_like(x0)
        b.solve(x0, max_steps, tol, x)  # warm-up (captures the graph)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        b.solve(x0, max_steps, tol, x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        t, k = b.tiles()
        table.append({"threads": t, "blocks_per_sm": k, "ms": ms})
        if log:
            log(f"tiles {t} x {k}: {ms:.1f} ms on {len(sub)} systems")
        if best is None or ms < best[2]:
            best = (t, k, ms)
        b.close()
    if best is None:
        raise RuntimeError("no admissible tiles")
    return best[0], best[1], table


def batch_tiles(items, max_steps: int, tol: float, retune: bool = False, log=None):
    """Cached tiles for this batch on this GPU (tuned and stored if absent)."""
    key = f"{_gpu_name()}|{signature([s for s, _, _ in items])}"
    cache = _load()
    if not retune and key in cache:
        e = cache[key]
        return e["threads"], e["blocks_per_sm"], e
    t0 = time.time()
    threads, bps, table = tune(items, max_steps, tol, sample=min(len(items), 2048), log=log)
    entry = {"threads": threads, "blocks_per_sm": bps, "timings": table, "tuned_s": round(time.time() - t0, 1)}
    cache[key] = entry
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    except OSError:
        pass
    return threads, bps, entry


def main():
    """Tune the tiles of the batched quad double workload on the whole batch
    and store them in the cache (python -m paper_2301_12659_gb300.autotune)."""
    import argparse

    from . import workloads as wl

    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", default="qd-real-batch4096", choices=sorted(wl.BATCH_CONFIGS))
    ap.add_argument("--sample", type=int, default=0, help="systems timed per candidate (0: all)")
    args = ap.parse_args()
    cfg = wl.BATCH_CONFIGS[args.batch]
    items = wl.batch_planted_systems(cfg)
    key = f"{_gpu_name()}|{signature([s for s, _, _ in items])}"
    t0 = time.time()
    threads, bps, table = tune(items, cfg.max_steps, cfg.tol, sample=args.sample or len(items), log=print)
    cache = _load()
    cache[key] = {"threads": threads, "blocks_per_sm": bps, "timings": table, "tuned_s": round(time.time() - t0, 1),
                  "sample": args.sample or len(items)}
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    print(json.dumps({"key": key, "threads": threads, "blocks_per_sm": bps}))


if __name__ == "__main__":
    main()
