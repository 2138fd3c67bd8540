"""Krylov solves on the GPU, checked on the TRUE residual computed with the oracle's own
assembled matrix: ||b - A_oracle x_gpu|| <= tol ||b|| (1 + 1e-3); adjoint gradients against
the oracle and against central finite differences of the GPU heat step."""
import numpy as np
import pytest

import synthetic as syn
from problems import band_octree, heat, helmholtz, oseen, reinit

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def true_residual(A, b, x):
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


def solve_and_check(P, b, nrhs=1, tol=1e-10, **kw):
    n = P["n"]
    x, info = P["op"].solve(torch.tensor(b.ravel(), device="cuda"), nrhs=nrhs, tol=tol, **kw)
    assert info["status"] == 0, info
    X = x.cpu().numpy().reshape(nrhs, n)
    B = b.reshape(nrhs, n)
    for r in range(nrhs):
        res = true_residual(P["A"], B[r], X[r])
        assert res <= tol * (1 + 1e-3), (r, res, info)
    return info


@pytest.mark.parametrize("precond", ["jacobi", "chebyshev", "none"])
def test_cg_helmholtz(ctx, precond):
    P = helmholtz(10, ctx)
    info = solve_and_check(P, syn.uniform_pm1(1, P["n"]), solver="cg", precond=precond)
    assert info["iterations"] > 0


def test_cg_graph_capture_batched(ctx):
    P = helmholtz(8, ctx)
    b = np.stack([syn.uniform_pm1(s, P["n"]) for s in (1, 2, 3)])
    solve_and_check(P, b, nrhs=3, solver="cg", precond="jacobi", use_graph=True)


def test_chebyshev_lambda_max_matches_oracle_lanczos(ctx):
    from oracle import krylov
    P = helmholtz(8, ctx)
    _, info = P["op"].solve(torch.tensor(syn.uniform_pm1(1, P["n"]), device="cuda"), solver="cg",
                            precond="chebyshev")
    A = P["A"]
    lam = krylov.lanczos_lambda_max(lambda v: A @ v, A.diagonal(), syn.uniform_pm1(9, P["n"]), steps=60)
    # 20 Lanczos steps from another start vector: within a few percent of the converged value
    assert abs(info["lambda_max"] / 1.1 - lam) <= 0.05 * lam


def test_gmres_heat_with_convection(ctx):
    P = heat(7, ctx, with_beta=True, kq=True)
    b = syn.uniform_pm1(2, P["n"])
    b[P["dm"].dirichlet] = 0.0
    solve_and_check(P, b, solver="gmres", precond="jacobi", restart=30)


def test_gmres_oseen_block_jacobi(ctx):
    P = oseen(4, ctx)
    b = syn.uniform_pm1(1, P["n"])
    mask = np.concatenate([np.tile(P["dmu"].dirichlet, 3), np.zeros(P["dmp"].n_dofs, bool)])
    b[mask] = 0.0
    solve_and_check(P, b, solver="gmres", precond="block_jacobi", restart=50, maxit=20000)


@pytest.mark.parametrize("n", [4, 7])
def test_fgmres_oseen_block_triangular(ctx, n):
    P = oseen(n, ctx)
    b = syn.uniform_pm1(2, P["n"])
    mask = np.concatenate([np.tile(P["dmu"].dirichlet, 3), np.zeros(P["dmp"].n_dofs, bool)])
    b[mask] = 0.0
    info = solve_and_check(P, b, solver="gmres", precond="block_triangular", restart=50, maxit=400)
    # the inner velocity GMRES and Schur CG make the outer iteration count nearly mesh independent
    assert info["iterations"] <= 60, info


def test_fgmres_oseen_block_triangular_replayed_as_a_graph(ctx):
    """use_graph records the preconditioner call once and replays it: the same solution to the
    oracle's tolerance, the same outer iteration count, and the launch count of the replayed
    kernels equal to that of the direct calls."""
    P = oseen(7, ctx)
    b = syn.uniform_pm1(3, P["n"])
    mask = np.concatenate([np.tile(P["dmu"].dirichlet, 3), np.zeros(P["dmp"].n_dofs, bool)])
    b[mask] = 0.0
    kw = dict(solver="gmres", precond="block_triangular", restart=50, maxit=400)
    solve_and_check(P, b, **kw)  # builds the operator's fp32 tables, once
    l0 = ctx.launch_count()
    direct = solve_and_check(P, b, **kw)
    l1 = ctx.launch_count()
    replayed = solve_and_check(P, b, use_graph=True, **kw)
    l2 = ctx.launch_count()
    assert replayed["iterations"] == direct["iterations"], (direct, replayed)
    assert l2 - l1 == l1 - l0


def test_block_triangular_needs_gmres(ctx):
    from paper_2501_18781_gb300._lib import MFError
    P = oseen(3, ctx)
    b = torch.ones(P["n"], dtype=torch.float64, device="cuda")
    with pytest.raises(MFError):
        P["op"].solve(b, solver="cg", precond="block_triangular")


def test_chebyshev_bounds_kept_on_the_operator_until_a_field_changes(ctx):
    """The Lanczos estimate of lambda_max is run by the first Chebyshev solve and reused by later
    solves of the same operator (the same step count and inner arithmetic give the same estimate):
    a second solve reports the same lambda_max and launches 20 fp32 applies fewer; after a field is
    set again (even to the same values) the estimate is recomputed, and every solve still meets the
    oracle's true residual."""
    P = heat(6, ctx)
    op = P["op"]
    b = syn.uniform_pm1(4, P["n"])
    b[P["dm"].dirichlet] = 0.0
    kw = dict(solver="defect_correction", precond="chebyshev", inner_tol=1e-4, inner_maxit=100)

    def counted(**extra):
        l0 = ctx.launch_count()
        info = solve_and_check(P, b, **kw, **extra)
        return info, ctx.launch_count() - l0

    i1, l1 = counted()
    i2, l2 = counted()
    assert i2["lambda_max"] == i1["lambda_max"]
    assert i2["iterations"] == i1["iterations"]
    assert l1 - l2 >= 20, (l1, l2)
    i3, l3 = counted(lanczos_steps=10)          # another step count: estimated again
    assert l3 > l2
    op.set_field("t_prev", torch.tensor(P["T_prev"], device="cuda"))
    i4, l4 = counted()
    assert l4 - l2 >= 20 and abs(i4["lambda_max"] - i1["lambda_max"]) <= 1e-6 * i1["lambda_max"]


def test_defect_correction_mixed_precision_heat(ctx):
    P = heat(10, ctx)
    b = syn.uniform_pm1(4, P["n"])
    b[P["dm"].dirichlet] = 0.0
    info = solve_and_check(P, b, solver="defect_correction", precond="chebyshev", inner_tol=1e-4,
                           inner_maxit=100)
    assert info["outer_iterations"] >= 2


def test_repeated_solves_on_pooled_work_vectors(ctx):
    """The solvers' work vectors come from the context's block pool, so a repeated solve runs on the
    blocks the previous one left, with its values still in them: a solver that read a work vector
    before writing it would start from those.  Each repeat must meet the tolerance on the oracle's
    true residual in the same number of iterations (one more or fewer allowed: the atomic scatter
    of the applies sums in a run-dependent order) and agree with the first to the solve's accuracy."""
    for P, kw in ((helmholtz(6, ctx), dict(solver="cg", precond="chebyshev", use_graph=True)),
                  (heat(5, ctx, with_beta=True, kq=True), dict(solver="gmres", precond="jacobi", restart=20)),
                  (heat(5, ctx, with_beta=True, kq=True), dict(solver="defect_correction", precond="jacobi",
                                                               fp64_arith="df64"))):
        b = syn.uniform_pm1(21, P["n"])
        b[P["dm"].dirichlet] = 0.0
        xs = []
        for _ in range(3):
            x, info = P["op"].solve(torch.tensor(b, device="cuda"), tol=1e-10, **kw)
            assert info["status"] == 0, (kw, info)
            xs.append((x.cpu().numpy(), info["iterations"]))
        for x, it in xs:
            assert abs(it - xs[0][1]) <= 1, kw
            assert true_residual(P["A"], b, x) <= 1e-10 * (1 + 1e-3), kw
            assert np.abs(x - xs[0][0]).max() <= 1e-7 * np.abs(xs[0][0]).max(), kw


def test_defect_correction_batched_reinit_octree(ctx):
    P = reinit(band_octree(), ctx)
    b = np.stack([syn.uniform_pm1(s, P["n"]) for s in range(1, 5)])
    solve_and_check(P, b, nrhs=4, solver="defect_correction", precond="chebyshev")


def test_cg_octree_helmholtz(ctx):
    P = helmholtz(0, ctx, octree=band_octree())
    solve_and_check(P, syn.uniform_pm1(5, P["n"]), solver="cg", precond="jacobi")


def _gradient_case(ctx, n=4):
    from oracle import heat as oheat
    P = heat(n, ctx, with_beta=True, kq=True)
    wl = P["wl"]
    p = wl.params
    dm = P["dm"]
    x = dm.dof_coords()
    ztop = wl.hi[2]
    laser = dict(power=200.0, radius=150e-6, x0=0.0, y0=0.0, absorptivity=0.35)
    th_prev = syn.heat_initial_temperature(*x.T, 150e-6, ztop) - p["t_ref"]
    th_prev[dm.dirichlet] = 0
    target = syn.heat_target_temperature(*x.T, ztop, 5, r=160e-6) - p["t_ref"]
    return P, laser, th_prev, target


@pytest.mark.parametrize("solver", ["gmres", "defect_correction"])
def test_heat_adjoint_gradient_matches_oracle(ctx, solver):
    """defect_correction: fp32 inner GMRES on the convective operator and on its transpose (the
    adjoint solve), outer residuals in double-float."""
    from oracle import heat as oheat
    P, laser, th_prev, target = _gradient_case(ctx)
    p = P["wl"].params
    st = oheat.HeatStep(P["dm"], p["rhocp"], p["dt"], kq=P["kq"], beta=P["beta"])
    cells = oheat.box_cells(P["dm"], 200e-6, 200e-6)
    J, gl, gk, th, lam = oheat.gradients(st, th_prev, target, laser, cells)
    lz = (laser["power"], laser["radius"], laser["x0"], laser["y0"], laser["absorptivity"])
    kw = dict(solver="gmres", precond="jacobi", tol=1e-13, restart=50) if solver == "gmres" else \
        dict(solver="defect_correction", precond="jacobi", tol=1e-12, restart=30, maxit=20, fp64_arith="df64")
    Jg, glg, gkg, thg, lamg = P["op"].heat_step_gradient(lz, torch.tensor(th_prev, device="cuda"),
                                                         torch.tensor(target, device="cuda"), 200e-6, 200e-6, **kw)
    assert abs(Jg - J) <= 1e-9 * abs(J)
    assert np.allclose(glg, gl, rtol=1e-8, atol=1e-10 * np.abs(gl).max())
    gkg = gkg.cpu().numpy().reshape(gk.shape)
    assert np.abs(gkg - gk).max() <= 1e-8 * np.abs(gk).max()


def test_heat_adjoint_gradient_matches_central_differences(ctx):
    P, laser, th_prev, target = _gradient_case(ctx)
    tp, tt = torch.tensor(th_prev, device="cuda"), torch.tensor(target, device="cuda")
    kw = dict(solver="gmres", precond="jacobi", tol=1e-13, restart=50)
    names = ["power", "radius", "x0", "y0"]
    lz = [laser[k] for k in names] + [laser["absorptivity"]]
    J0, g, gk, _, _ = P["op"].heat_step_gradient(lz, tp, tt, 200e-6, 200e-6, **kw)
    for i, k in enumerate(names):
        step = 1e-6 * (abs(lz[i]) if k in ("power", "radius") else laser["radius"])
        a, b = list(lz), list(lz)
        a[i] += step
        b[i] -= step
        Ja = P["op"].heat_step_gradient(a, tp, tt, 200e-6, 200e-6, with_kq=False, **kw)[0]
        Jb = P["op"].heat_step_gradient(b, tp, tt, 200e-6, 200e-6, with_kq=False, **kw)[0]
        fd = (Ja - Jb) / (2 * step)
        assert abs(g[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * max(abs(v) for v in g)), (k, g[i], fd)
    # k_q: largest-magnitude entries, perturbing the per-Gauss-point field
    gk = gk.cpu().numpy()
    kq = P["kq"].ravel().copy()
    for flat in np.argsort(-np.abs(gk))[:2]:
        hh = 1e-6 * kq[flat]
        vals = []
        for sgn in (1, -1):
            k2 = kq.copy()
            k2[flat] += sgn * hh
            P["op"].set_field("k_qpoint", torch.tensor(k2, device="cuda"))
            vals.append(P["op"].heat_step_gradient(lz, tp, tt, 200e-6, 200e-6, with_kq=False, **kw)[0])
        P["op"].set_field("k_qpoint", torch.tensor(kq, device="cuda"))
        fd = (vals[0] - vals[1]) / (2 * hh)
        assert abs(gk[flat] - fd) <= 1e-6 * abs(fd), (flat, gk[flat], fd)


def test_cg_with_double_float_applies_reaches_fp64_tolerance(ctx):
    P = helmholtz(10, ctx)
    solve_and_check(P, syn.uniform_pm1(6, P["n"]), solver="cg", precond="chebyshev", fp64_arith="df64")
    Pg = heat(6, ctx, with_beta=True, kq=True)
    b = syn.uniform_pm1(7, Pg["n"])
    b[Pg["dm"].dirichlet] = 0.0
    solve_and_check(Pg, b, solver="gmres", precond="jacobi", fp64_arith="df64")


def test_autograd_function_matches_adjoint_and_central_differences(ctx):
    from paper_2501_18781_gb300.autograd import heat_step_objective
    P, laser, th_prev, target = _gradient_case(ctx)
    tp, tt = torch.tensor(th_prev, device="cuda"), torch.tensor(target, device="cuda")
    kw = dict(solver="gmres", precond="jacobi", tol=1e-13, restart=50)
    lz = torch.tensor([laser["power"], laser["radius"], laser["x0"], laser["y0"]], dtype=torch.float64,
                      requires_grad=True)
    kq = torch.tensor(P["kq"].ravel(), device="cuda", requires_grad=True)
    J = heat_step_objective(P["op"], lz, kq, tp, tt, 200e-6, 200e-6, **kw)
    J.backward()
    _, g, gk, _, _ = P["op"].heat_step_gradient(list(lz.detach().tolist()) + [0.35], tp, tt, 200e-6, 200e-6, **kw)
    assert np.allclose(lz.grad.numpy(), g, rtol=1e-12)
    assert torch.allclose(kq.grad, gk, rtol=1e-12)
    # central difference on the radius through the Function's forward
    step = 1e-6 * laser["radius"]
    with torch.no_grad():
        a, b = lz.detach().clone(), lz.detach().clone()
        a[1] += step
        b[1] -= step
        fd = (heat_step_objective(P["op"], a, kq.detach(), tp, tt, 200e-6, 200e-6, **kw)
              - heat_step_objective(P["op"], b, kq.detach(), tp, tt, 200e-6, 200e-6, **kw)) / (2 * step)
    assert abs(lz.grad[1].item() - fd.item()) <= 1e-6 * abs(fd.item())
