"""Edge cases through the C ABI on the GPU: arguments the boundary must reject before any launch,
zero right-hand sides (alone and inside a batch), the method's degenerate cases against the oracle
(a constant level set makes the reinit normal vanish, leaving (1/dtau) M; a single-phase Oseen
operator without convection is the Stokes operator sigma rho M + 2 mu eps:eps), one-cell meshes of
every operator, an octree with no refinement, and strided batches whose padding stays untouched."""
import ctypes as C

import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import mesh as omesh
from problems import DIRICHLET_BOTTOM, OSEEN_FACES, componentwise_ok, heat, helmholtz, oseen

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _check_fp64(A, op, seed=1, rtol=1e-12):
    u = syn.uniform_pm1(seed, A.shape[0])
    v = op.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    ok, worst = componentwise_ok(v, A @ u, abs(A) @ np.abs(u), rtol)
    assert ok, worst


def test_boundary_rejects_bad_arguments(ctx):
    from paper_2501_18781_gb300 import _lib
    lib = _lib.load()
    P = helmholtz(3, ctx)
    n = P["n"]
    u = torch.ones(2 * n, dtype=torch.float64, device="cuda")
    v = torch.full((2 * n,), 7.0, dtype=torch.float64, device="cuda")
    h = P["op"].h
    assert lib.mf_apply(h, _ptr(u), _ptr(v), 0, n, _lib.MF_F64) == _lib.MF_EINVAL          # empty batch
    assert lib.mf_apply(h, _ptr(u), _ptr(v), 1, n - 1, _lib.MF_F64) == _lib.MF_EINVAL      # ld < n
    assert lib.mf_apply(h, None, _ptr(v), 1, n, _lib.MF_F64) == _lib.MF_EINVAL
    assert lib.mf_apply(h, _ptr(u), _ptr(v), 1, n, 99) != _lib.MF_OK                        # unknown dtype
    assert lib.mf_apply_transpose(h, _ptr(u), _ptr(v), 0, n, _lib.MF_F64) == _lib.MF_EINVAL
    torch.cuda.synchronize()
    assert torch.all(v == 7.0)                                                              # nothing launched
    sp = _lib.SolverParams()
    info = _lib.SolveInfo()
    for nrhs in (0, 65):
        assert lib.mf_solve(h, C.byref(sp), _ptr(u), _ptr(v), nrhs, C.byref(info)) == _lib.MF_EINVAL
    short = torch.zeros(n - 1, dtype=torch.float64, device="cuda")
    assert lib.mf_operator_set_field(h, _lib.MF_FIELD_PHI, _ptr(short), _lib.MF_F64, n - 1) == _lib.MF_EINVAL


def test_zero_right_hand_sides(ctx):
    """x = 0 exactly, at iteration 0, for a zero b; a zero column of a batch does not disturb the
    others (CG, defect correction) and GMRES returns at once."""
    P = helmholtz(5, ctx)
    n, A = P["n"], P["A"]
    x, info = P["op"].solve(torch.zeros(n, dtype=torch.float64, device="cuda"), solver="cg", precond="jacobi")
    assert info["status"] == 0 and info["iterations"] == 0 and torch.all(x == 0)
    B = np.stack([syn.uniform_pm1(1, n), np.zeros(n), syn.uniform_pm1(3, n)])
    for solver, prec in (("cg", "jacobi"), ("cg", "chebyshev"), ("defect_correction", "chebyshev")):
        x, info = P["op"].solve(torch.tensor(B.ravel(), device="cuda"), nrhs=3, solver=solver, precond=prec,
                                tol=1e-10)
        assert info["status"] == 0, (solver, info)
        X = x.cpu().numpy().reshape(3, n)
        assert np.all(X[1] == 0.0), solver
        for r in (0, 2):
            assert np.linalg.norm(B[r] - A @ X[r]) <= 1e-10 * (1 + 1e-3) * np.linalg.norm(B[r]), (solver, r)
    H = heat(4, ctx, with_beta=True, kq=True)
    x, info = H["op"].solve(torch.zeros(H["n"], dtype=torch.float64, device="cuda"), solver="gmres",
                            precond="jacobi")
    assert info["status"] == 0 and info["iterations"] == 0 and torch.all(x == 0)
    O = oseen(3, ctx)
    x, info = O["op"].solve(torch.zeros(O["n"], dtype=torch.float64, device="cuda"), solver="gmres",
                            precond="block_triangular")
    assert info["status"] == 0 and info["iterations"] == 0 and torch.all(x == 0)


@pytest.mark.parametrize("mesh", ["uniform", "octree"])
def test_reinit_constant_level_set_is_scaled_mass(ctx, mesh):
    """grad phi_h = 0: the normal is set to 0, the n-n diffusion drops out and A = M / dtau, in
    every arithmetic and both coefficient modes."""
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    if mesh == "uniform":
        dm = omesh.uniform_dofmap(3, (0, 0, 0), (1, 1, 1), 2)
        m = DofMap(Mesh.uniform(ctx, 3), 2, 0)
        eps = 2.0 / 3
    else:
        d = lambda x, y, z: syn.deformed_sphere_distance(x, y, z, 3)
        leaves = syn.refine_band_leaves(4, 2, d, 1.0 / 64)
        dm = omesh.octree_dofmap(leaves, 4, 2)
        m = DofMap(Mesh.octree(ctx, 4, 2, leaves), 2, 0)
        eps = 1.0 / 8
    dtau = 0.01
    phi = np.full(dm.n_dofs, 0.3)
    A = asm.reinit_matrix(dm, phi, eps, dtau)
    M = asm.mass_matrix(dm) / dtau
    assert abs(A - M).max() <= 1e-14 * abs(M).max()        # the oracle's own reduction
    u = syn.uniform_pm1(5, dm.n_dofs)
    ref, bound = M @ u, abs(M) @ np.abs(u)
    for mode in (0, 1):
        op = Operator(ctx, "reinit", [m], eps=eps, dtau=dtau, coef_mode=mode)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        v = op.apply(torch.tensor(u, device="cuda")).cpu().numpy()
        ok, worst = componentwise_ok(v, ref, bound, 1e-12)
        assert ok, (mode, worst)
        v32 = op.apply(torch.tensor(u, device="cuda").float()).cpu().double().numpy()
        ok, worst = componentwise_ok(v32, ref, bound, 2e-5)
        assert ok, (mode, worst)


def test_single_phase_oseen_without_convection_is_stokes(ctx):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    n, sigma, rho, mu = 4, 50.0, 4087.0, 5e-3
    dmu = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 2, OSEEN_FACES)
    dmp = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 1, 0)
    phi, beta = np.ones(dmu.n_dofs), np.zeros((3, dmu.n_dofs))
    A = asm.oseen_matrix(dmu, dmp, phi, beta, sigma, rho, 4.087, mu, 1e-5)
    mesh = Mesh.uniform(ctx, n)
    op = Operator(ctx, "oseen", [DofMap(mesh, 2, OSEEN_FACES), DofMap(mesh, 1, 0)], sigma=sigma, rho_l=rho,
                  rho_g=4.087, mu_l=mu, mu_g=1e-5, eps=0.5)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
    _check_fp64(A, op)
    # the velocity block is symmetric once convection is gone
    nu3 = 3 * dmu.n_dofs
    Auu = A[:nu3, :nu3]
    assert abs(Auu - Auu.T).max() <= 1e-12 * abs(Auu).max()


def test_one_cell_meshes(ctx):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    H = heat(1, ctx)
    _check_fp64(H["A"], H["op"])
    assert H["dm"].dirichlet.sum() == 9                      # the bottom face of one Q2 cell
    O = oseen(1, ctx)
    _check_fp64(O["A"], O["op"])
    dm = omesh.uniform_dofmap(1, (0, 0, 0), (1, 1, 1), 2)
    x = dm.dof_coords()
    phi = syn.initial_level_set(syn.sphere_distance(*x.T), 0.5)
    op = Operator(ctx, "reinit", [DofMap(Mesh.uniform(ctx, 1), 2, 0)], eps=0.5, dtau=0.1)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    _check_fp64(asm.reinit_matrix(dm, phi, 0.5, 0.1), op)


def test_octree_without_refinement_matches_the_uniform_operator(ctx):
    """Every leaf on level 0 of a 5^3 base mesh declared with 2 levels: no hanging nodes, and the
    operator is the uniform one (DoFs in the octree's own order)."""
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    base = 5
    ii, jj, kk = np.meshgrid(np.arange(base), np.arange(base), np.arange(base), indexing="ij")
    leaves = np.stack([np.zeros(base ** 3), ii.ravel(), jj.ravel(), kk.ravel()], axis=1).astype(np.int32)
    for levels in (0, 2):
        dm = omesh.octree_dofmap(leaves, base, levels)
        assert dm.n_dofs == (2 * base + 1) ** 3
        x = dm.dof_coords()
        eps = 2.0 / base
        phi = syn.initial_level_set(syn.sphere_distance(*x.T), eps)
        A = asm.helmholtz_matrix(dm, phi, 1.0, 1000.0, 1.0, "tanh", eps)
        m = DofMap(Mesh.octree(ctx, base, levels, leaves), 2, 0)
        assert m.n_dofs == dm.n_dofs and m.n_constraints == 0
        op = Operator(ctx, "helmholtz", [m], mass_coef=1.0, a_liquid=1000.0, a_gas=1.0, eps=eps)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        _check_fp64(A, op)
        # the same operator as on the uniform mesh, up to the DoF order
        du = omesh.uniform_dofmap(base, (0, 0, 0), (1, 1, 1), 2)
        xu = du.dof_coords()
        key = lambda X: np.lexsort(np.round(X * 4 * base).astype(np.int64).T)
        perm_o, perm_u = key(x), key(xu)
        Au = asm.helmholtz_matrix(du, syn.initial_level_set(syn.sphere_distance(*xu.T), eps), 1.0, 1000.0, 1.0,
                                  "tanh", eps)
        D = A[perm_o][:, perm_o] - Au[perm_u][:, perm_u]
        assert abs(D).max() <= 1e-12 * abs(Au).max()


def _line(P):
    P["op"].set_variant("q2_line", 1)   # the nine-threads-per-cell kernel
    return P


def test_strided_batches_leave_the_padding_alone(ctx):
    from paper_2501_18781_gb300 import _lib
    lib = _lib.load()
    for P, dt, code, rtol in ((heat(4, ctx, with_beta=True, kq=True), torch.float64, _lib.MF_F64, 1e-12),
                              (_line(heat(4, ctx)), torch.float64, _lib.MF_F64, 1e-12),
                              (_line(helmholtz(3, ctx)), torch.float32, _lib.MF_F32, 2e-5),
                              (helmholtz(4, ctx), torch.float32, _lib.MF_F32, 2e-5),
                              (heat(5, ctx), torch.float64, _lib.MF_DF64, 1e-12),
                              (heat(5, ctx, with_beta=True, kq=True), torch.float64, _lib.MF_DF64, 1e-12)):
        n, ld, R = P["n"], P["n"] + 37, 3
        U = np.zeros((R, ld))
        for r in range(R):
            U[r, :n] = syn.uniform_pm1(10 + r, n)
        U[:, n:] = 5.0
        src = torch.tensor(U.ravel(), dtype=dt, device="cuda")
        dst = torch.full((R * ld,), -3.0, dtype=dt, device="cuda")
        for fn, A in ((lib.mf_apply, P["A"]), (lib.mf_apply_transpose, P["A"].T.tocsr())):
            dst.fill_(-3.0)
            assert fn(P["op"].h, _ptr(src), _ptr(dst), R, ld, code) == _lib.MF_OK
            V = dst.cpu().double().numpy().reshape(R, ld)
            assert np.all(V[:, n:] == -3.0)
            for r in range(R):
                u = U[r, :n].astype(np.float32).astype(np.float64) if dt == torch.float32 else U[r, :n]
                ok, worst = componentwise_ok(V[r, :n], A @ u, abs(A) @ np.abs(u), rtol)
                assert ok, (r, worst)
