"""Host logic of the batched workload: seeded, reproducible systems of the
stated recipe (size classes, distinct variables, diagonal term, planted
start), and the packing of series that the batch calls expect."""
import numpy as np

from paper_2301_12659_gb300 import workloads as wl


def test_batch_systems_follow_the_recipe():
    cfg = wl.BATCH_CONFIGS["qd-real-batch4096"]
    items = wl.batch_planted_systems(cfg, 48)
    again = wl.batch_planted_systems(cfg, 3)
    for (a, xa, x0a), (b, xb, x0b) in zip(items, again):
        assert np.array_equal(a.vidx, b.vidx) and np.array_equal(a.coeff, b.coeff) and np.array_equal(x0a, x0b)
    seen = set()
    for s, xstar, x0 in items:
        s.check()
        assert s.n in cfg.n_choices and s.d in cfg.d_choices
        seen.add((s.n, s.d))
        k = np.diff(s.vptr)
        diag = s.meta["diag_monomials"]
        assert len(diag) == s.n and np.all(k[diag] == 1)
        assert np.all(s.vidx[s.vptr[diag]] == np.arange(s.n))
        assert np.all(s.coeff[0, 0, diag, 0] == s.n) and np.all(s.coeff[0, 0, diag, 1:] == 0)
        reg = np.setdiff1d(np.arange(s.M), diag)
        assert len(reg) == cfg.mono_per_eq * s.n
        assert np.all((k[reg] >= cfg.kmin) & (k[reg] <= min(cfg.kmax, s.n)))
        for m in reg:
            v = s.vidx[s.vptr[m]:s.vptr[m + 1]]
            assert len(set(v.tolist())) == len(v)  # distinct variables
        assert np.all(np.bincount(s.eq, minlength=s.n) == cfg.mono_per_eq + 1)
        # start: x*_0 plus noise of at most 1e-3, higher coefficients zero
        assert np.all(np.abs(x0[0, :, :, 0] - xstar[0, :, :, 0]) <= cfg.noise)
        assert np.all(x0[:, :, :, 1:] == 0) and np.all(x0[1:] == 0)
    assert len(seen) >= 8  # the size classes mix
