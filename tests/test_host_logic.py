"""Host-side logic that needs no GPU: the stratified sample of the tile
autotuner, the paper's one-column workload, the bench's metric names, and
the evaluation's product schedule executed symbolically."""
import numpy as np
import pytest

from paper_2301_12659_gb300 import autotune
from paper_2301_12659_gb300 import workloads as wl


def test_stratified_sample_keeps_every_class_in_proportion():
    cfg = wl.BATCH_CONFIGS["qd-real-batch4096"]
    systems = [s for s, _, _ in wl.batch_planted_systems(cfg, 240)]
    idx = autotune._stratified(systems, 60, seed=3)
    assert idx == sorted(set(idx)) and len(idx) >= 12
    classes = {(s.n, s.d) for s in systems}
    assert {(systems[q].n, systems[q].d) for q in idx} == classes
    assert autotune._stratified(systems, 60, seed=3) == idx          # reproducible
    assert len(autotune._stratified(systems, 10 ** 6)) == len(systems)  # all when asked for more
    sig = autotune.signature(systems)
    assert sig.startswith("K4C1|") and sig.count(",") == len(classes) - 1


def test_one_column_system_structure():
    s, x = wl.one_column_system(40, 9, 4)
    s.check()
    k = np.diff(s.vptr)
    assert np.array_equal(k, np.arange(1, 41))                  # monomial i has i+1 variables
    for m in range(40):
        assert np.array_equal(s.vidx[s.vptr[m]:s.vptr[m + 1]], np.arange(m + 1))
    assert np.all(s.coeff[0, 0, :, 0] == 1) and np.all(s.coeff[0, 0, :, 1:] == 0) and np.all(s.coeff[1:] == 0)
    alpha = x[0, 0, :, 1]
    assert np.all((np.abs(alpha) >= 0.9) & (np.abs(alpha) <= 1.0))
    assert np.all(x[0, 0, :, 0] == 1) and np.all(x[1:] == 0)
    assert np.allclose(x[0, 0, :, 3], alpha ** 3 / 6)


def test_bench_metric_names():
    import bench
    assert bench.metric_of(wl.CONFIGS["qd-real-n64-d31"]) == "Newton steps/s (qd, n=64, d=31)"
    assert bench.metric_of(wl.CONFIGS["od-complex-n128-d63"]) == "Newton steps/s (od complex, n=128, d=63)"


def _library():
    """The C-ABI library, built for sm_103a if needed (loading it needs no GPU;
    mdn_ed_schedule makes no CUDA call)."""
    from paper_2301_12659_gb300 import build
    from paper_2301_12659_gb300 import mdnewton as md
    build.build()
    md.load()
    return md


SLOT_C, SLOT_X, SLOT_F, SLOT_B, SLOT_V, SLOT_P = 1, 2, 3, 4, 5, 6
OP_NONE, OP_PRODUCT, OP_COPY = 0, 1, 2


def _run_schedule(ops, k):
    """Execute a product schedule with each series replaced by the multiset
    of its factors (c and the positions 1..k): a truncated product of series
    is then the union of the factor multisets, so the table computes the
    right products exactly when every slot ends with the right multiset.
    Returns the slots written and the number of products."""
    from collections import Counter
    known = {(SLOT_C, 0): Counter({"c": 1})}
    for q in range(k):
        known[(SLOT_X, q)] = Counter({q + 1: 1})
    written, products = set(), 0
    for wave in ops:
        new = {}
        for op, dst, a, b in wave.tolist():
            if op == OP_NONE:
                continue
            sa, sd = (a >> 16, a & 0xffff), (dst >> 16, dst & 0xffff)
            assert sa in known, f"reads {sa} before it is written"
            assert sd not in known and sd not in new, f"writes {sd} twice"
            if op == OP_PRODUCT:
                sb = (b >> 16, b & 0xffff)
                assert sb in known, f"reads {sb} before it is written"
                new[sd] = known[sa] + known[sb]
                products += 1
            else:
                assert op == OP_COPY
                new[sd] = known[sa].copy()
        # a product reads only what earlier waves wrote: the groups of one
        # wave run at the same time
        known.update(new)
        written.update(new)
    return known, written, products


@pytest.mark.parametrize("groups", [1, 2, 3, 5, 8, 16, 32])
def test_ed_schedule_computes_the_value_and_every_partial(groups):
    """The evaluation's product table (Section 5.1: forward, backward and
    cross products; the coefficient series enters as F_0) leaves c x_1..x_k
    in the value slot and c times all factors but x_p in partial slot p, with
    3k-3 products for k >= 2 (the paper's 3k-5 without a coefficient, plus
    two), scratch slots F_1..F_{k-2} and B_2..B_{k-1} only, and no more
    waves than the products or the dependency chain force."""
    from collections import Counter
    md = _library()
    for k in list(range(1, 19)) + [31, 64, 300]:
        ops = md.mdn_ed_schedule(k, groups)
        assert ops.shape[1:] == (groups, 4)
        known, written, products = _run_schedule(ops, k)
        full = Counter({"c": 1, **{q: 1 for q in range(1, k + 1)}})
        assert known[(SLOT_V, 0)] == full
        for p in range(k):
            assert known[(SLOT_P, p)] == full - Counter({p + 1: 1}), (k, p)
        assert products == (1 if k == 1 else 3 * k - 3)
        for kind, idx in written:
            assert kind in (SLOT_F, SLOT_B, SLOT_V, SLOT_P)
            if kind == SLOT_F:
                assert 1 <= idx <= k - 2
            elif kind == SLOT_B:
                assert 2 <= idx <= k - 1
            elif kind == SLOT_P:
                assert 0 <= idx < k
        # the forward chain c x_1 ... x_k has k dependent products
        waves = ops.shape[0]
        assert waves >= max(-(-products // groups), k if k > 1 else 1)
        if groups >= 3 * k - 3 and k > 1:
            assert waves == k, (k, groups, waves)


def test_ed_schedule_of_the_four_variable_example():
    """The paper's n = 4 example (Section 5.1): with x_1 x_2 x_3 x_4 and a
    coefficient c the three columns are c x_1, F_1 x_2, F_2 x_3, F_3 x_4
    (forward); x_4 x_3, B_2 x_2 (backward); c B_3, F_1 B_2, F_2 x_4 (cross)."""
    md = _library()
    ops = md.mdn_ed_schedule(4, 32)
    prods = sorted(tuple(r) for r in ops.reshape(-1, 4).tolist() if r[0] == OP_PRODUCT)
    s = lambda kind, idx: (kind << 16) | idx
    expect = sorted([
        (OP_PRODUCT, s(SLOT_F, 1), s(SLOT_C, 0), s(SLOT_X, 0)),
        (OP_PRODUCT, s(SLOT_F, 2), s(SLOT_F, 1), s(SLOT_X, 1)),
        (OP_PRODUCT, s(SLOT_P, 3), s(SLOT_F, 2), s(SLOT_X, 2)),   # F_3 = the partial wrt x_4
        (OP_PRODUCT, s(SLOT_V, 0), s(SLOT_P, 3), s(SLOT_X, 3)),
        (OP_PRODUCT, s(SLOT_B, 2), s(SLOT_X, 3), s(SLOT_X, 2)),
        (OP_PRODUCT, s(SLOT_B, 3), s(SLOT_B, 2), s(SLOT_X, 1)),
        (OP_PRODUCT, s(SLOT_P, 0), s(SLOT_C, 0), s(SLOT_B, 3)),
        (OP_PRODUCT, s(SLOT_P, 1), s(SLOT_F, 1), s(SLOT_B, 2)),
        (OP_PRODUCT, s(SLOT_P, 2), s(SLOT_F, 2), s(SLOT_X, 3)),
    ])
    assert prods == expect
    assert ops.shape[0] == 4


def _bench(args, env_extra=None):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ)
    env.update(env_extra or {})
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *args], capture_output=True, text=True,
                       timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    return [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]


def test_reference_arm_prints_one_line_of_the_contract():
    """bench.py --impl reference times the CPU oracle on the workload's
    metric and prints one JSON line with the reference arm's keys."""
    lines = _bench(["--impl", "reference", "--config", "dd-real-n8-d15", "--steps", "3", "--warmup", "3"])
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["metric"] == "Newton steps/s (dd, n=8, d=15)"
    assert d["unit"] == "steps/s" and d["higher_is_better"] is True and d["steps"] == 3 and d["warmup"] == 3
    assert d["value"] > 0 and d["vs_baseline"] is None and d["config"]["workload"] == "dd-real-n8-d15"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the ranks other than 0 exit without work or output."""
    lines = _bench(["--impl", "reference", "--config", "dd-real-n8-d15", "--steps", "3", "--warmup", "3"],
                   {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert lines == []


def test_autotuner_cache_is_keyed_by_gpu_and_size_classes(tmp_path, monkeypatch):
    """batch_tiles reads the cache entry of (GPU, limbs, real/complex, size
    classes) when present, and otherwise tunes once and stores the choice."""
    cfg = wl.small_config(4, 1, n=4, d=7, mono_per_eq=2, kmin=1, kmax=3, index=960)
    cfg2 = wl.small_config(4, 1, n=8, d=7, mono_per_eq=2, kmin=1, kmax=3, index=961)
    items = [wl.planted_system(cfg), wl.planted_system(cfg2), wl.planted_system(cfg)]
    assert autotune.signature([s for s, _, _ in items]) == "K4C1|4x7,8x7"
    monkeypatch.setattr(autotune, "CACHE", str(tmp_path / "tiles.json"))
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "GPU-A")
    calls = []

    def fake_tune(its, max_steps, tol, sample=4096, candidates=None, log=None):
        calls.append(len(its))
        return 256, 1, [{"threads": 256, "blocks_per_sm": 1, "ms": 1.0}]

    monkeypatch.setattr(autotune, "tune", fake_tune)
    t, b, e = autotune.batch_tiles(items, 12, 1e-50)
    assert (t, b) == (256, 1) and calls == [3]
    t, b, e = autotune.batch_tiles(items, 12, 1e-50)  # cached: no second tuning
    assert (t, b) == (256, 1) and calls == [3]
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "GPU-B")  # another GPU tunes again
    autotune.batch_tiles(items, 12, 1e-50)
    assert calls == [3, 3]
    import json
    keys = sorted(json.load(open(tmp_path / "tiles.json")))
    assert keys == ["GPU-A|K4C1|4x7,8x7", "GPU-B|K4C1|4x7,8x7"]


def test_cpu_baseline_thread_count():
    """The CPU baseline leg times the oracle on all host cores by default
    and on the number of threads asked for otherwise; it reports the count
    it used."""
    import bench
    from oracle import oracle
    cfg = wl.CONFIGS["dd-real-n8-d15"]
    all_cores = oracle.get_threads()
    try:
        dt, cores = bench.oracle_sample(cfg, 2, threads=1)
        assert cores == 1 and dt > 0
    finally:
        oracle.set_threads(all_cores)
    lines = _bench(["--impl", "reference", "--config", "dd-real-n8-d15", "--steps", "3", "--warmup", "3",
                    "--cpu-threads", "1"])
    assert lines[0]["cpu_baseline"]["cores"] == 1
