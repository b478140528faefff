"""mdn_evaluate_static: the evaluation for callers that cannot allocate device
memory (plug-ins inside an application whose own pool reserves the device
memory up front, loops that must not allocate after start-up because
cudaMalloc can block on the device).  Its
scratch is a static device array of the library, so nothing is allocated per
call.  Checked against the workspace evaluation (mdn_evaluate) on two calls
in a row, within the per-precision tolerances of the other GPU tests.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2301_12659_gb300 import workloads as wl
from tests import metrics as mt
from tests.gpu_util import TOL, need_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def md():
    return need_gpu()


CASES = [
    wl.CONFIGS["qd-real-n64-d31"],
    wl.CONFIGS["dd-real-n8-d15"],
    wl.small_config(8, 2, n=7, d=12, mono_per_eq=3, kmin=1, kmax=5, index=950),
    wl.small_config(4, 1, n=5, d=0, mono_per_eq=2, kmin=1, kmax=3, index=951),
]


@pytest.mark.parametrize("cfg", CASES, ids=lambda c: c.name)
def test_static_evaluation_matches_workspace_evaluation(md, cfg):
    import torch
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = wl.random_md((s.n, s.D), s.K, s.C, 17, unit_circle=(s.C == 2))
    nw = md.Newton(s)
    dev = nw.cst.device
    eq = torch.as_tensor(s.eq, device=dev)
    vptr = torch.as_tensor(s.vptr, device=dev)
    vidx = torch.as_tensor(s.vidx, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    for rep in range(2):
        x = torch.as_tensor(wl.random_md((s.n, s.D), s.K, s.C, 40 + rep, unit_circle=(s.C == 2)), device=dev)
        f_ref = to_np(nw.evaluate(x, want_A=False))
        f = torch.full_like(nw.cst, np.nan)
        st = md.mdn_evaluate_static(s.K, s.C - 1, s.n, s.d, s.M, int(s.vptr[-1]), eq, vptr, vidx, nw.coeff,
                                    nw.cst, x, f, stream)
        assert st == md.MDN_OK
        assert mt.matrix_rel_error(to_np(f), f_ref) <= TOL[s.K]


def test_static_evaluation_rejects_sizes_beyond_its_array(md):
    import torch
    # complex octo double, n = 128, d = 63 needs 2 MiB + 256 bytes > MDN_STATIC_SCRATCH_BYTES
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    idx = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = md.mdn_evaluate_static(8, 1, 128, 63, 1, 1, idx, idx, idx, dummy, dummy, dummy, dummy,
                                torch.cuda.current_stream().cuda_stream)
    assert st == md.MDN_ETOOLARGE


@pytest.mark.parametrize("bad", ["eq", "var_idx", "var_ptr"])
def test_static_evaluation_rejects_indices_out_of_range(md, bad):
    """An equation index, a variable index or a CSR offset out of range is
    found on the device and reported as MDN_EINVAL (the kernel checks each
    index before it uses it)."""
    import torch
    cfg = wl.small_config(2, 1, n=5, d=7, mono_per_eq=2, kmin=1, kmax=3, index=952)
    s, xstar, x0 = wl.planted_system(cfg)
    s.cst = wl.random_md((s.n, s.D), s.K, s.C, 18)
    eq, vptr, vidx = s.eq.copy(), s.vptr.copy(), s.vidx.copy()
    if bad == "eq":
        eq[3] = s.n
    elif bad == "var_idx":
        vidx[4] = s.n + 2
    else:
        vptr[2] = vptr[-1] + 7
    dev = torch.device("cuda")
    t = lambda a: torch.as_tensor(a, device=dev)
    coeff, cst = t(s.coeff), t(s.cst)
    x = t(wl.random_md((s.n, s.D), s.K, s.C, 41))
    f = torch.zeros_like(cst)
    st = md.mdn_evaluate_static(s.K, s.C - 1, s.n, s.d, s.M, int(s.vptr[-1]), t(eq), t(vptr), t(vidx), coeff, cst, x,
                                f, torch.cuda.current_stream().cuda_stream)
    assert st == md.MDN_EINVAL
