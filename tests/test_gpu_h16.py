"""Packed 16-bit (fp16x2 / bf16x2) operator applies and their use inside defect correction."""
import numpy as np
import pytest

import synthetic as syn
from problems import band_octree, heat, helmholtz, reinit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# normwise error of one apply against the fp64 oracle, relative to || |A| |u| ||: a few units of
# the format's rounding (2^-11 for fp16, 2^-8 for bf16) times the depth of the cell computation
TOL = {"f16": 4e-3, "bf16": 3e-2}


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def check_packed(P, arith, nrhs):
    n = P["n"]
    U = np.stack([syn.uniform_pm1(20 + r, n) for r in range(nrhs)]).astype(np.float32).astype(np.float64)
    u = torch.tensor(U.ravel(), dtype=torch.float32, device="cuda")
    v = P["op"].apply(u, nrhs=nrhs, arith=arith).cpu().numpy().astype(np.float64).reshape(nrhs, n)
    absA = abs(P["A"])
    for r in range(nrhs):
        ref = P["A"] @ U[r]
        err = np.linalg.norm(v[r] - ref) / np.linalg.norm(absA @ np.abs(U[r]))
        assert err <= TOL[arith], (arith, r, err)


@pytest.mark.parametrize("arith", ["f16", "bf16"])
def test_packed_apply_heat_and_helmholtz(ctx, arith):
    check_packed(heat(8, ctx, coef_mode=1), arith, 2)
    check_packed(helmholtz(6, ctx, coef_mode=1), arith, 3)     # odd: one idle lane


@pytest.mark.parametrize("arith", ["f16", "bf16"])
def test_packed_apply_octree_reinit(ctx, arith):
    check_packed(reinit(band_octree(), ctx, coef_mode=1), arith, 4)


@pytest.mark.parametrize("arith", ["f16", "bf16"])
def test_defect_correction_with_packed_inner_applies(ctx, arith):
    P = reinit(band_octree(), ctx, coef_mode=1)
    b = np.stack([syn.uniform_pm1(s, P["n"]) for s in range(1, 5)])
    x, info = P["op"].solve(torch.tensor(b.ravel(), device="cuda"), nrhs=4, solver="defect_correction",
                            precond="chebyshev", tol=1e-10, inner_arith=arith)
    assert info["status"] == 0, info
    X = x.cpu().numpy().reshape(4, P["n"])
    for r in range(4):
        res = np.linalg.norm(b[r] - P["A"] @ X[r]) / np.linalg.norm(b[r])
        assert res <= 1e-10 * (1 + 1e-3), (arith, r, res, info)


def test_packed_apply_rejects_convection(ctx):
    from paper_2501_18781_gb300._lib import MFError
    P = heat(4, ctx, with_beta=True)
    with pytest.raises(MFError):
        P["op"].apply(torch.zeros(P["n"], dtype=torch.float32, device="cuda"), arith="bf16")
