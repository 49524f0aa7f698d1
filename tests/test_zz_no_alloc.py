"""The allocation-free solver entry point, gipc_pcg_noalloc, against gipc_pcg.

gipc_pcg_noalloc serves callers that may not allocate device memory (a framework that
owns all device memory through its own pool, or a latency-critical loop where cudaMalloc
would synchronise the device): it keeps the solver's vectors in a fixed array of the
library instead of context scratch.  Both entry points are called through the C ABI on
the same inputs; results must agree to the 1e-10 relative tolerance of the PCG tests, on
two calls in a row (the second on a different system, so stale contents of the shared
array would show).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

from test_oracle_pcg import spd_system  # noqa: E402

RTOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2308_09400_gb300 as g
    from paper_2308_09400_gb300 import _abi
    return g, _abi


def _bsr(_abi, R, n, prec, keep):
    dt = torch.float64 if prec == 0 else torch.float32
    rowptr = torch.tensor(R["rowptr"].astype(np.int32), device="cuda")
    colidx = torch.tensor(R["colidx"].astype(np.int32), device="cuda")
    vals = torch.tensor(np.asarray(R["vals"]).reshape(-1, 9), device="cuda").to(dt)
    keep += [rowptr, colidx, vals]
    return _abi.Bsr(n, len(R["colidx"]), len(R["colidx"]), rowptr.data_ptr(), colidx.data_ptr(),
                    vals.data_ptr(), prec)


def _solve(_abi, ctx, bsr, b, iters, fixed=None):
    x = torch.zeros_like(b)
    prm = _abi.PcgParams(0.0, iters, 0)
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    fx = ctypes.c_void_p(fixed.data_ptr()) if fixed is not None else ctypes.c_void_p(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if ctx is None:
        st = _abi.lib().gipc_pcg_noalloc(ctypes.byref(bsr), ctypes.c_void_p(b.data_ptr()),
                                         ctypes.c_void_p(x.data_ptr()), fx, ctypes.byref(prm), ctypes.byref(it),
                                         ctypes.byref(rel), stream)
    else:
        st = _abi.lib().gipc_pcg(ctx.handle, ctypes.byref(bsr), ctypes.c_void_p(b.data_ptr()),
                                 ctypes.c_void_p(x.data_ptr()), fx, ctypes.byref(prm), ctypes.byref(it),
                                 ctypes.byref(rel), stream)
    assert st == 0, _abi.lib().gipc_last_error()
    torch.cuda.synchronize()
    return x.cpu().numpy(), it.value, rel.value


def test_noalloc_matches_context_solver_on_two_calls(lib):
    g, _abi = lib
    ctx = g.Context()
    keep = []
    cases = [(6000, 20000, 4000, 0, None), (2500, 7000, 900, 1, 5)]   # (n, stencils, tets, prec, fixed stride)
    for call, (n, k, T, prec, stride) in enumerate(cases):
        R, b, _, _ = spd_system(n, k, T, seed=70 + call)
        bsr = _bsr(_abi, R, n, prec, keep)
        bt = torch.tensor(b, device="cuda")
        fixed = None
        if stride:
            f = np.zeros(n, np.uint8)
            f[::stride] = 1
            fixed = torch.tensor(f, device="cuda")
        xr, itr, relr = _solve(_abi, ctx, bsr, bt, 30, fixed)
        xn, itn, reln = _solve(_abi, None, bsr, bt, 30, fixed)
        assert itn == itr == 30
        assert np.abs(xn - xr).max() <= RTOL * np.abs(xr).max()
        assert reln == pytest.approx(relr, rel=RTOL)
    ctx.close()


def test_noalloc_rejects_systems_beyond_its_limit(lib):
    g, _abi = lib
    n = g.PCG_NOALLOC_MAX_N + 1
    bsr = _abi.Bsr(n, 0, 0, 0, 0, 0, 0)
    prm = _abi.PcgParams(0.0, 5, 0)
    st = _abi.lib().gipc_pcg_noalloc(ctypes.byref(bsr), None, None, None, ctypes.byref(prm), None, None, None)
    assert st == -1
    assert b"32768" in _abi.lib().gipc_last_error()
