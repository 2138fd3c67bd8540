"""Q3/Q4 Helmholtz operators (Gauss-Lobatto support points, (k+1)^3 Gauss points) on the GPU against
the oracle's assembled matrices: applies componentwise (fp64 1e-12, fp32 5e-5 of (|A||u|)_i), the
diagonal, Jacobi- and Chebyshev-preconditioned CG by the oracle's true residual, and the
combinations the boundary rejects."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import mesh as omesh
from problems import componentwise_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def _problem(ctx, k, n, heaviside="tanh"):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    dm = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), k)
    eps = 1.0 / (2 * n)
    phi = syn.initial_level_set(syn.sphere_distance(*dm.dof_coords().T), eps)
    A = asm.helmholtz_matrix(dm, phi, 1.0, 1000.0, 1.0, heaviside, eps)
    m = DofMap(Mesh.uniform(ctx, n), k, 0)
    op = Operator(ctx, "helmholtz", [m], mass_coef=1.0, a_liquid=1000.0, a_gas=1.0, eps=eps,
                  heaviside=0 if heaviside == "tanh" else 1)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    assert m.n_dofs == dm.n_dofs
    return dm, A, op


@pytest.mark.parametrize("k", [3, 4])
@pytest.mark.parametrize("n", [1, 3, 4])
def test_qk_apply_matches_oracle(ctx, k, n):
    dm, A, op = _problem(ctx, k, n)
    u = syn.uniform_pm1(k + n, dm.n_dofs)
    ref, bound = A @ u, abs(A) @ np.abs(u)
    v = op.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    ok, worst = componentwise_ok(v, ref, bound, 1e-12)
    assert ok, worst
    v32 = op.apply(torch.tensor(u, device="cuda").float()).cpu().double().numpy()
    ok, worst = componentwise_ok(v32, ref, bound, 5e-5)
    assert ok, worst
    assert op.variant.startswith(f"helmholtz_q{k}/")


def test_qk_sine_heaviside_and_strided_batch(ctx):
    dm, A, op = _problem(ctx, 3, 3, heaviside="sine")
    n, ld = dm.n_dofs, dm.n_dofs + 11
    U = np.zeros((2, ld))
    U[0, :n], U[1, :n] = syn.uniform_pm1(1, n), syn.uniform_pm1(2, n)
    out = op.apply(torch.tensor(U.ravel(), device="cuda"), nrhs=2).cpu().numpy().reshape(2, ld)
    for r in range(2):
        ok, worst = componentwise_ok(out[r, :n], A @ U[r, :n], abs(A) @ np.abs(U[r, :n]), 1e-12)
        assert ok, (r, worst)


@pytest.mark.parametrize("k", [3, 4])
def test_qk_diagonal(ctx, k):
    dm, A, op = _problem(ctx, k, 3)
    d = op.diagonal().cpu().numpy()
    assert np.abs(d - A.diagonal()).max() <= 1e-12 * np.abs(A.diagonal()).max()


@pytest.mark.parametrize("k,precond", [(3, "jacobi"), (4, "jacobi"), (3, "chebyshev")])
def test_qk_cg_reaches_tolerance_on_the_oracle_matrix(ctx, k, precond):
    dm, A, op = _problem(ctx, k, 4)
    b = syn.uniform_pm1(7, dm.n_dofs)
    x, info = op.solve(torch.tensor(b, device="cuda"), solver="cg", precond=precond, tol=1e-10)
    assert info["status"] == 0, info
    res = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1e-10 * (1 + 1e-3), (res, info)


def test_qk_rejections(ctx):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    from paper_2501_18781_gb300._lib import MFError
    mesh = Mesh.uniform(ctx, 2)
    with pytest.raises(MFError):
        Operator(ctx, "helmholtz", [DofMap(mesh, 3, 1 << 4)], mass_coef=1.0, a_liquid=2.0, a_gas=1.0)
    with pytest.raises(MFError):
        Operator(ctx, "heat", [DofMap(mesh, 4, 0)], rhocp=1.0, dt=1.0, k0=1.0, t_boil=1.0)
    _, _, op = _problem(ctx, 3, 2)
    with pytest.raises(MFError):
        op.apply(torch.zeros(op.n, dtype=torch.float64, device="cuda"), arith="df64")
    with pytest.raises(MFError):
        DofMap(Mesh.octree(ctx, 2, 0, np.array([[0, i, j, k] for k in range(2) for j in range(2) for i in range(2)],
                                                np.int32)), 3, 0)


@pytest.mark.parametrize("n", [1, 3, 6])
def test_q3_tensor_core_apply_matches_oracle(ctx, n):
    """tcgen05 dense form with bf16 hi/lo operands (three products, fp32 accumulation): tiles of 128
    cells, here 1 cell, one partial tile (27 cells) and two tiles with a ragged tail (216 cells)."""
    dm, A, op = _problem(ctx, 3, n)
    u = syn.uniform_pm1(11 + n, dm.n_dofs).astype(np.float32).astype(np.float64)
    ref, bound = A @ u, abs(A) @ np.abs(u)
    v = op.apply(torch.tensor(u, device="cuda").float(), arith="tc").cpu().double().numpy()
    ok, worst = componentwise_ok(v, ref, bound, 5e-5)
    assert ok, worst
    assert op.variant == "helmholtz_q3/uniform/f32/tcgen05-bf16x3/dense"
    # a strided batch of two
    ld = dm.n_dofs + 5
    U = np.zeros((2, ld), np.float32)
    U[0, :dm.n_dofs], U[1, :dm.n_dofs] = u, -0.5 * u
    out = op.apply(torch.tensor(U.ravel(), device="cuda"), nrhs=2, arith="tc").cpu().double().numpy().reshape(2, ld)
    for r, s in ((0, 1.0), (1, -0.5)):
        ok, worst = componentwise_ok(out[r, :dm.n_dofs], s * ref, abs(s) * bound, 5e-5)
        assert ok, (r, worst)


def test_tensor_core_apply_rejects_q4(ctx):
    from paper_2501_18781_gb300._lib import MFError
    _, _, op = _problem(ctx, 4, 2)
    with pytest.raises(MFError):
        op.apply(torch.zeros(op.n, dtype=torch.float32, device="cuda"), arith="tc")


@pytest.mark.parametrize("inner", ["f32", "tc"])
def test_q3_defect_correction_with_cuda_core_or_tensor_core_inner_applies(ctx, inner):
    """fp64 outer residual, fp32 Chebyshev-CG inner solve whose applies run on the CUDA cores or on
    the tensor cores: the oracle's true residual reaches 1e-10."""
    dm, A, op = _problem(ctx, 3, 4)
    b = syn.uniform_pm1(9, dm.n_dofs)
    x, info = op.solve(torch.tensor(b, device="cuda"), solver="defect_correction", precond="chebyshev",
                       inner_arith=inner, tol=1e-10)
    assert info["status"] == 0, info
    res = np.linalg.norm(b - A @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1e-10 * (1 + 1e-3), (res, info)
    assert info["outer_iterations"] >= 2


def test_tensor_core_inner_arithmetic_needs_q3_and_defect_correction(ctx):
    from paper_2501_18781_gb300._lib import MFError
    dm, A, op = _problem(ctx, 3, 2)
    b = torch.ones(dm.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(MFError):
        op.solve(b, solver="cg", precond="jacobi", inner_arith="tc")
    _, _, op4 = _problem(ctx, 4, 2)
    with pytest.raises(MFError):
        op4.solve(torch.ones(op4.n, dtype=torch.float64, device="cuda"), solver="defect_correction",
                  precond="chebyshev", inner_arith="tc")


def test_q3_autotune_picks_an_fp32_kernel_and_keeps_parity(ctx):
    """After mf_autotune the plain fp32 apply runs whichever Q3 kernel was faster; either passes."""
    dm, A, op = _problem(ctx, 3, 6)
    op.autotune()
    u = syn.uniform_pm1(5, dm.n_dofs).astype(np.float32).astype(np.float64)
    v = op.apply(torch.tensor(u, device="cuda").float()).cpu().double().numpy()
    ok, worst = componentwise_ok(v, A @ u, abs(A) @ np.abs(u), 5e-5)
    assert ok, worst
    assert op.variant in ("helmholtz_q3/uniform/f32/tabulated/line-per-thread",
                          "helmholtz_q3/uniform/f32/tcgen05-bf16x3/dense")
