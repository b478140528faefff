"""Host-side logic that needs no GPU: the stratified sample of the tile
autotuner, the paper's one-column workload, the bench's metric names."""
import numpy as np

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
