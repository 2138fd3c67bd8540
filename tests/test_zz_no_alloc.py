"""mf_dot_noalloc: the allocation-free inner products, for callers that cannot let the library
allocate device memory (their own memory pool, latency-critical loops, no mf_ctx).  Called
through the C ABI, it must agree with mf_dot on two calls in a row; its workspace is a shared
static device array, so the second call must not see anything left over from the first.
This file is collected last so that a failure here never hides the other tests."""
import ctypes as C

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, _lib, build_library
    build_library()
    return Context(0), _lib


def _vecs(seed, n, nvec, dtype):
    X = np.stack([syn.uniform_pm1(seed + k, n) for k in range(nvec)])
    Y = np.stack([syn.uniform_pm1(seed + 100 + k, n) for k in range(nvec)])
    return (torch.tensor(X.ravel(), device="cuda", dtype=dtype),
            torch.tensor(Y.ravel(), device="cuda", dtype=dtype))


def _bound(x, y, nvec):
    a = x.abs().double().reshape(nvec, -1)
    b = y.abs().double().reshape(nvec, -1)
    return (a * b).sum(dim=1).cpu().numpy()


def test_noalloc_matches_mf_dot_on_two_calls_in_a_row(setup):
    ctx, lib = setup
    L = lib.load()
    code = {torch.float64: lib.MF_F64, torch.float32: lib.MF_F32}
    # call 1 uses more vector pairs than call 2, so stale partials would show up in call 2
    for seed, n, nvec, dt in ((1, 777_777, 7, torch.float64), (2, 123_457, 3, torch.float64),
                              (3, 500_001, 5, torch.float32)):
        x, y = _vecs(seed, n, nvec, dt)
        ref = torch.empty(nvec, dtype=torch.float64, device="cuda")
        got = torch.empty(nvec, dtype=torch.float64, device="cuda")
        lib.check(L.mf_dot(ctx.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), n, n, nvec, code[dt],
                           C.c_void_p(ref.data_ptr())))
        lib.check(L.mf_dot_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), n, n, nvec, code[dt],
                                   C.c_void_p(got.data_ptr()), C.c_void_p(1)))   # cudaStreamLegacy
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        # same fixed grid and summation order as mf_dot: equal bit for bit
        assert np.array_equal(g, r), (seed, g, r, np.abs(g - r) / _bound(x, y, nvec))


def test_noalloc_rejects_more_pairs_than_its_workspace(setup):
    ctx, lib = setup
    L = lib.load()
    x = torch.zeros(17 * 8, dtype=torch.float64, device="cuda")
    out = torch.empty(17, dtype=torch.float64, device="cuda")
    st = L.mf_dot_noalloc(C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()), 8, 8, 17, lib.MF_F64,
                          C.c_void_p(out.data_ptr()), None)
    assert st == lib.MF_EINVAL
    assert b"nvec" in L.mf_last_error()
