"""Operator apply, transpose and diagonal on the GPU against the oracle's assembled matrices.

FP64 bar: |v_gpu - v_oracle|_i <= 1e-12 (|A| |u|)_i for every i (componentwise, robust to
summation order).  FP32 bar: 2e-5 (|A| |u|)_i (single-precision contractions with O(100)
roundings per entry).  Sizes span several 8x4x4-cell blocks with ragged tails."""
import numpy as np
import pytest

import synthetic as syn
from problems import band_octree, componentwise_ok, heat, helmholtz, oseen, reinit, schur_fp16_bound, schur_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def check_apply(P, seed=1, nrhs=1, rtol64=1e-12, rtol32=2e-5, transpose=False):
    n = P["n"]
    A = P["A"].T.tocsr() if transpose else P["A"]
    absA = abs(A)
    U = np.stack([syn.uniform_pm1(seed + r, n) for r in range(nrhs)])
    src = torch.tensor(U.ravel(), device="cuda")
    out64 = P["op"].apply(src, nrhs=nrhs, transpose=transpose).cpu().numpy().reshape(nrhs, n)
    outdf = P["op"].apply(src, nrhs=nrhs, transpose=transpose, arith="df64").cpu().numpy().reshape(nrhs, n)
    out32 = P["op"].apply(src.float(), nrhs=nrhs, transpose=transpose).cpu().numpy().astype(np.float64).reshape(nrhs, n)
    for r in range(nrhs):
        ref = A @ U[r]
        bound = absA @ np.abs(U[r])
        ok, worst = componentwise_ok(out64[r], ref, bound, rtol64)
        assert ok, f"fp64 componentwise error {worst:.3e} (rhs {r})"
        okd, worstd = componentwise_ok(outdf[r], ref, bound, rtol64)
        assert okd, f"double-float componentwise error {worstd:.3e} (rhs {r})"
        ok32, worst32 = componentwise_ok(out32[r], ref, bound, rtol32)
        assert ok32, f"fp32 componentwise error {worst32:.3e} (rhs {r})"
    return worst, worstd, worst32


@pytest.mark.parametrize("n", [1, 3, 10])
@pytest.mark.parametrize("mode", [0, 1])
def test_helmholtz_uniform(ctx, n, mode):
    P = helmholtz(n, ctx, coef_mode=mode)
    check_apply(P)


def test_helmholtz_sine_heaviside(ctx):
    P = helmholtz(9, ctx, heaviside="sine", coef_mode=1)
    check_apply(P)
    P0 = helmholtz(9, ctx, heaviside="sine", coef_mode=0)
    check_apply(P0, rtol32=1e-4)


def test_helmholtz_batched_rhs(ctx):
    P = helmholtz(10, ctx)
    check_apply(P, nrhs=3)


@pytest.mark.parametrize("mode", [0, 1])
def test_heat_k_of_T_with_dirichlet(ctx, mode):
    P = heat(10, ctx, coef_mode=mode)
    check_apply(P)
    # Dirichlet rows return the input
    u = torch.tensor(syn.uniform_pm1(3, P["n"]), device="cuda")
    v = P["op"].apply(u).cpu().numpy()
    d = P["dm"].dirichlet
    assert np.array_equal(v[d], u.cpu().numpy()[d])


@pytest.mark.parametrize("case", [("helmholtz", 3, 0), ("helmholtz", 5, 1), ("heat", 4, 0), ("heat", 7, 1)])
def test_q2_line_per_thread_kernel(ctx, case):
    """The degree-2 instance of the line-per-thread kernel (nine threads per cell, coefficients from
    the Q2 Gauss-point tables) against the oracle: fp64 at 1e-12 and fp32 at 2e-5 componentwise, with
    the Dirichlet bottom face of the heat operator and two right-hand sides per call; then the
    one-thread-per-cell kernel again on the same operator."""
    from paper_2501_18781_gb300 import MFError
    kind, n, mode = case
    P = (heat if kind == "heat" else helmholtz)(n, ctx, coef_mode=mode)
    op = P["op"]
    op.set_variant("q2_line", 1)
    check_apply(P, nrhs=2)
    assert op.variant.endswith("/f32/tabulated/line-per-thread"), op.variant
    op.apply(torch.zeros(P["n"], dtype=torch.float64, device="cuda"))
    assert op.variant.endswith("/f64/tabulated/line-per-thread"), op.variant
    op.set_variant("q2_line", 0)
    check_apply(P)
    assert "line-per-thread" not in op.variant
    with pytest.raises(MFError):
        op.set_variant("q2_line", 2)
    with pytest.raises(MFError):
        op.set_variant("no_such_variant", 1)


def test_heat_convection_kq_and_transpose(ctx):
    P = heat(9, ctx, with_beta=True, kq=True)
    check_apply(P)
    check_apply(P, transpose=True)


def test_oseen_q2q1(ctx):
    P = oseen(9, ctx)
    check_apply(P, rtol32=5e-5)


@pytest.mark.parametrize("dtype,rtol", [("f64", 1e-12), ("f32", 2e-5)])
def test_oseen_coupling_blocks(ctx, dtype, rtol):
    """B^T p and B u alone against the oracle's assembled off-diagonal blocks."""
    P = oseen(5, ctx)
    A = P["A"].tocsr()
    N = 3 * P["dmu"].n_dofs
    B, BT = A[N:, :N], A[:N, N:]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    p = syn.uniform_pm1(3, A.shape[0] - N)
    u = syn.uniform_pm1(4, N)
    if dtype == "f32":
        p, u = p.astype(np.float32).astype(np.float64), u.astype(np.float32).astype(np.float64)
    g = P["op"].coupling("grad", torch.tensor(p, dtype=tdt, device="cuda")).cpu().double().numpy()
    ok, worst = componentwise_ok(g, BT @ p, abs(BT) @ abs(p), rtol)
    assert ok, worst
    assert np.all(g[np.tile(P["dmu"].dirichlet, 3)] == 0.0)
    d = P["op"].coupling("div", torch.tensor(u, dtype=tdt, device="cuda")).cpu().double().numpy()
    ok, worst = componentwise_ok(d, B @ u, abs(B) @ abs(u), rtol)
    assert ok, worst


@pytest.mark.parametrize("n", [1, 2, 5])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_oseen_schur_complement_approximation(ctx, n, dtype):
    """B D^-1 B^T p (D: the 3 x 3 nodal blocks of A_uu) against the same product of the oracle's
    assembled blocks.  fp64: the coupling kernels and block Jacobi, 1e-12 componentwise.  fp32: the
    block-triangular preconditioner's own operator, assembled as a 125-point stencil from the 1D
    couplings of B and stored as row-scaled fp16, so its bound adds the storage error.  n = 1 and 2
    put every node on or next to the boundary."""
    P = oseen(n, ctx)
    nu = P["dmu"].n_dofs
    S, Sabs = schur_reference(P["A"], nu)
    p = syn.uniform_pm1(8 + n, S.shape[0])
    if dtype == "f32":
        p = p.astype(np.float32).astype(np.float64)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    got = P["op"].coupling("schur", torch.tensor(p, dtype=tdt, device="cuda")).cpu().double().numpy()
    ref, bound = S @ p, Sabs @ np.abs(p)
    if dtype == "f64":
        ok, worst = componentwise_ok(got, ref, bound, 1e-12)
    else:
        ok, worst = componentwise_ok(got, ref, 5e-5 * bound + schur_fp16_bound(S, p, n), 1.0)
    assert ok, worst


@pytest.mark.parametrize("mode", [0, 1])
def test_helmholtz_octree_hanging_nodes(ctx, mode):
    P = helmholtz(0, ctx, octree=band_octree(), coef_mode=mode)
    assert P["map"].n_constraints > 0
    check_apply(P)


@pytest.mark.parametrize("mode", [0, 1])
def test_reinit_octree_multi_rhs(ctx, mode):
    P = reinit(band_octree(), ctx, coef_mode=mode)
    check_apply(P, nrhs=2, rtol32=5e-5)


@pytest.mark.parametrize("which", ["helmholtz", "heat_beta", "octree", "reinit"])
def test_diagonal(ctx, which):
    if which == "helmholtz":
        P = helmholtz(10, ctx)
    elif which == "heat_beta":
        P = heat(7, ctx, with_beta=True, kq=True)
    elif which == "octree":
        P = helmholtz(0, ctx, octree=band_octree())
    else:
        P = reinit(band_octree(), ctx)
    d = P["op"].diagonal().cpu().numpy()
    ref = P["A"].diagonal()
    assert np.max(np.abs(d - ref) / np.abs(ref)) <= 1e-12


def test_laser_load_and_parameter_derivatives(ctx):
    from oracle import assemble as asm
    P = heat(8, ctx)
    lz = P["wl"].params["laser"]
    f, dF = P["op"].laser_load(lz["power"], lz["radius"], lz["x0"], lz["y0"], lz["absorptivity"], derivatives=True)
    ref = asm.laser_rhs(P["dm"], **lz)
    dref = asm.laser_rhs(P["dm"], **lz, derivatives=True)
    scale = np.abs(ref).max()
    assert np.abs(f.cpu().numpy() - ref).max() <= 1e-13 * scale
    for k in range(4):
        assert np.abs(dF[k].cpu().numpy() - dref[k]).max() <= 1e-12 * np.abs(dref[k]).max()


def test_launch_count_increases(ctx):
    P = helmholtz(4, ctx)
    before = ctx.launch_count()
    P["op"].apply(torch.ones(P["n"], dtype=torch.float64, device="cuda"))
    assert ctx.launch_count() > before


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_dot_products_against_fp64_numpy(ctx, dt):
    n, nvec = 1_000_003, 3
    X = np.stack([syn.uniform_pm1(10 + k, n) for k in range(nvec)])
    Y = np.stack([syn.uniform_pm1(20 + k, n) for k in range(nvec)])
    tdt = torch.float64 if dt == "f64" else torch.float32
    x = torch.tensor(X.ravel(), device="cuda", dtype=tdt)
    y = torch.tensor(Y.ravel(), device="cuda", dtype=tdt)
    out = ctx.dot(x, y, nvec).cpu().numpy()
    Xs, Ys = x.cpu().double().numpy().reshape(nvec, n), y.cpu().double().numpy().reshape(nvec, n)
    ref = np.array([np.dot(Xs[k], Ys[k]) for k in range(nvec)])
    bound = np.array([np.dot(np.abs(Xs[k]), np.abs(Ys[k])) for k in range(nvec)])
    assert np.all(np.abs(out - ref) <= 1e-13 * bound)
    again = ctx.dot(x, y, nvec).cpu().numpy()
    assert np.array_equal(out, again)     # fixed-grid reduction: bit-reproducible
