"""Pins of the oracle against what the mathematics and the paper fix (no GPU)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic as syn
from oracle import assemble as asm
from oracle import basis, coeffs, heat, krylov, mesh

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ----------------------------------------------------------------------------- basis / quadrature

def test_gauss_rules_closed_form():
    g = gold("gauss_rules.json")
    x2, w2 = basis.gauss_rule_01(2)
    assert np.allclose(x2, [0.5 - np.sqrt(3) / 6, 0.5 + np.sqrt(3) / 6], atol=1e-15)
    assert np.allclose(w2, g["two"]["weights"], atol=1e-15)
    x3, w3 = basis.gauss_rule_01(3)
    assert np.allclose(x3, [0.5 - np.sqrt(15) / 10, 0.5, 0.5 + np.sqrt(15) / 10], atol=1e-15)
    assert np.allclose(w3, [5 / 18, 8 / 18, 5 / 18], atol=1e-15)


@pytest.mark.parametrize("npts", [2, 3])
def test_tensor_gauss_exact_for_degree_2n_minus_1(npts):
    """int_{[0,1]^3} x^a y^b z^c = 1/((a+1)(b+1)(c+1)) for a, b, c <= 2 npts - 1."""
    _, _, w = basis.tensor_tables(1, npts)
    x, _ = basis.gauss_rule_01(npts)
    pts = np.array([[x[a], x[b], x[c]] for c in range(npts) for b in range(npts) for a in range(npts)])
    top = 2 * npts - 1
    for a in range(top + 1):
        for b in range(top + 1):
            for c in range(top + 1):
                val = np.sum(w * pts[:, 0] ** a * pts[:, 1] ** b * pts[:, 2] ** c)
                assert abs(val - 1.0 / ((a + 1) * (b + 1) * (c + 1))) < 1e-15
    # and not exact one degree higher (so the rule really has npts points)
    val = np.sum(w * pts[:, 0] ** (top + 1))
    assert abs(val - 1.0 / (top + 2)) > 1e-8


def test_lagrange_hanging_weights():
    g = gold("lagrange_hanging_weights.json")
    L, _ = basis.lagrange_1d(2, np.array([0.25, 0.75]))
    assert np.array_equal(L[:, 0], g["q2_at_quarter"])
    assert np.array_equal(L[:, 1], g["q2_at_three_quarters"])
    L1, _ = basis.lagrange_1d(1, np.array([0.5]))
    assert np.array_equal(L1[:, 0], g["q1_at_half"])


def test_partition_of_unity_and_derivative_sum():
    N, G, _ = basis.tensor_tables(2, 3)
    assert np.allclose(N.sum(axis=1), 1.0, atol=1e-15)
    assert np.allclose(G.sum(axis=1), 0.0, atol=1e-13)


def test_element_matrices_are_tensor_products_of_1d_rationals():
    """Constant-coefficient Q2 element mass = h^3 M1 x M1 x M1, stiffness = h (K1 x M1 x M1 + ...)
    with the exact 1D matrices; the x-fastest local numbering makes x the last kron factor."""
    g = gold("q2_1d_matrices.json")
    M1 = np.array(g["mass_times_30"]) / 30.0
    K1 = np.array(g["stiffness_times_3"]) / 3.0
    h = 0.37
    dm = mesh.uniform_dofmap(1, (0, 0, 0), (h, h, h), 2)
    one = np.ones((1, 27))
    Me = asm.scalar_element_matrices(dm, one)[0]
    Ke = asm.scalar_element_matrices(dm, 0 * one, diff=one)[0]
    Mk = np.kron(M1, np.kron(M1, M1)) * h ** 3
    Kk = (np.kron(K1, np.kron(M1, M1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(M1, np.kron(M1, K1))) * h
    assert np.abs(Me - Mk).max() <= 1e-15 * np.abs(Mk).max()
    assert np.abs(Ke - Kk).max() <= 1e-14 * np.abs(Kk).max()


def test_q1_tables_against_1d_rationals():
    g = gold("q2_1d_matrices.json")
    M1 = np.array(g["q1_mass_times_6"]) / 6.0
    K1 = np.array(g["q1_stiffness"], dtype=float)
    N, G, w = basis.tensor_tables(1, 2)
    Me = np.einsum("q,qi,qj->ij", w, N, N)
    Ke = np.einsum("q,qid,qjd->ij", w, G, G)
    assert np.allclose(Me, np.kron(M1, np.kron(M1, M1)), atol=1e-16)
    assert np.allclose(Ke, np.kron(K1, np.kron(M1, M1)) + np.kron(M1, np.kron(K1, M1))
                       + np.kron(M1, np.kron(M1, K1)), atol=1e-15)


# ----------------------------------------------------------------------------- coefficient laws

def test_heaviside_laws():
    phi = np.linspace(-1.2, 1.2, 2001)
    H = coeffs.heaviside_tanh(phi)
    assert H.min() == 0.0 and H.max() == 1.0 and np.all(np.diff(H) >= 0)
    # tanh reading: H(phi(d)) = 1 / (1 + exp(-d / eps))
    eps = 0.01
    d = np.linspace(-0.05, 0.05, 101)
    assert np.allclose(coeffs.heaviside_tanh(np.tanh(d / (2 * eps))), 1 / (1 + np.exp(-d / eps)), atol=1e-15)
    Hs = coeffs.heaviside_sine(np.tanh(d / (2 * eps)), eps)
    # eq. (heaviside): H(0) = 1/2, 0 / 1 beyond -+3 eps, continuous at the ends, monotone
    assert coeffs.heaviside_sine(np.array([0.0]), eps)[0] == 0.5
    assert np.all(Hs[d <= -3 * eps] == 0) and np.all(Hs[d >= 3 * eps] == 1)
    assert np.all(np.diff(Hs) >= -1e-15)
    dd = np.array([-3 * eps * (1 - 1e-9), 3 * eps * (1 - 1e-9)])
    assert np.allclose(coeffs.heaviside_sine(np.tanh(dd / (2 * eps)), eps), [0, 1], atol=1e-8)


def test_density_and_viscosity_laws():
    t = gold("ti64_table.json")
    for k in ("rho_l", "rho_g", "mu_l", "mu_g", "cp_l", "k_l", "t_boil"):
        assert syn.TI64[k] == t[k]
    H = np.array([0.0, 1.0, 0.5])
    rho = coeffs.reciprocal_density(H, t["rho_l"], t["rho_g"])
    assert rho[0] == t["rho_g"] and rho[1] == t["rho_l"]
    assert abs(rho[2] - 2 / (1 / t["rho_l"] + 1 / t["rho_g"])) < 1e-12
    mu = coeffs.arithmetic_mix(H, t["mu_l"], t["mu_g"])
    assert mu[0] == t["mu_g"] and mu[1] == t["mu_l"] and abs(mu[2] - 0.5 * (t["mu_l"] + t["mu_g"])) < 1e-18


def test_laser_flux_total_power_and_derivatives():
    P, r, x0, y0, chi = 200.0, 50e-6, 3e-6, -4e-6, 0.35
    # integral over the plane = chi P (Gaussian normalisation of eq. laser_gauss)
    s = np.linspace(-6 * r, 6 * r, 1201)
    X, Y = np.meshgrid(s + x0, s + y0)
    q = coeffs.laser_flux(X, Y, P, r, x0, y0, chi)
    tot = np.trapezoid(np.trapezoid(q, s, axis=1), s)
    assert abs(tot - chi * P) < 1e-9 * chi * P
    # closed-form parameter derivatives against central differences
    xs, ys = np.array([10e-6, -30e-6, 55e-6]), np.array([0.0, 20e-6, -41e-6])
    D = coeffs.laser_flux_parameter_derivatives(xs, ys, P, r, x0, y0, chi)
    base = dict(power=P, radius=r, x0=x0, y0=y0)
    for i, k in enumerate(["power", "radius", "x0", "y0"]):
        step = 1e-6 * (abs(base[k]) if k in ("power", "radius") else r)
        a, b = dict(base), dict(base)
        a[k] += step
        b[k] -= step
        fd = (coeffs.laser_flux(xs, ys, a["power"], a["radius"], a["x0"], a["y0"], chi)
              - coeffs.laser_flux(xs, ys, b["power"], b["radius"], b["x0"], b["y0"], chi)) / (2 * step)
        assert np.allclose(D[i], fd, rtol=1e-6, atol=1e-9 * np.abs(D[i]).max())


# ----------------------------------------------------------------------------- assembled operators

def _sphere_phi(dm, eps):
    x = dm.dof_coords()
    return syn.initial_level_set(syn.sphere_distance(*x.T), eps)


def test_mass_row_sums_equal_volume_uniform_and_octree():
    dm = mesh.uniform_dofmap(3, (0, 0, 0), (0.5, 0.5, 0.5), 2)
    assert abs(asm.mass_matrix(dm).sum() - 0.125) < 1e-15
    dmo = _small_octree()
    M = asm.mass_matrix(dmo)
    assert abs(M.sum() - 1.0) < 1e-14
    # each element's mass sums to its volume
    Ae = asm.scalar_element_matrices(dmo, np.ones((dmo.n_cells, 27)))
    assert np.allclose(Ae.sum(axis=(1, 2)), dmo.cell_h ** 3, rtol=1e-14)


def _small_octree():
    leaves = [[0, i, j, k] for k in range(2) for j in range(2) for i in range(2) if (i, j, k) != (0, 0, 0)]
    leaves += [[1, i, j, k] for k in range(2) for j in range(2) for i in range(2)]
    return mesh.octree_dofmap(np.array(leaves), 2, 1)


def _band_octree():
    d = lambda x, y, z: syn.deformed_sphere_distance(x, y, z, 3)
    leaves = syn.refine_band_leaves(4, 2, d, 1.0 / 64)
    assert syn.is_two_to_one_balanced(leaves, 4, 2)
    return mesh.octree_dofmap(leaves, 4, 2)


def test_neumann_laplacian_nullspace_with_variable_coefficient():
    for dm in (mesh.uniform_dofmap(4, (0, 0, 0), (1, 1, 1), 2), _band_octree()):
        phi = _sphere_phi(dm, 0.125)
        m, a = asm.helmholtz_coefficients(dm, phi, 1.0, 1000.0, 1.0)
        K = asm.assemble_scalar(dm, 0 * m, diff=a)
        r = K @ np.ones(dm.n_dofs)
        assert np.abs(r).max() <= 1e-13 * np.abs(K).max()
        assert abs(K - K.T).max() <= 1e-15 * np.abs(K).max()


def test_hanging_constraints_reproduce_global_q2_polynomials_exactly():
    dm = _band_octree()
    assert (dm.hang_of_point >= 0).sum() > 100
    p = lambda x: ((1 + x[:, 0] - 2 * x[:, 0] ** 2) * (0.5 + x[:, 1] - x[:, 1] ** 2) * (0.3 + x[:, 2] ** 2)
                   + x[:, 0] * x[:, 1] * x[:, 2] ** 2)
    u = p(dm.dof_coords())
    allp = dm.lo + dm.points * (dm.hspan / dm.R)
    assert np.abs(dm.C @ u - p(allp)).max() <= 1e-14


def test_octree_fe_function_is_continuous_across_every_face():
    """Evaluate a random FE function from both sides of every face shared by two leaves
    (including coarse-fine faces) at points of the smaller face: the traces must agree."""
    dm = _band_octree()
    u = syn.uniform_pm1(11, dm.n_dofs)
    ul = asm.local_values(dm, u)
    lo = dm.cell_origin
    hi = dm.cell_origin + dm.cell_h[:, None]
    rng = np.random.default_rng(0)
    checked = 0
    centers = lo + 0.5 * dm.cell_h[:, None]
    for c in rng.choice(dm.n_cells, 300, replace=False):
        for ax in range(3):
            # neighbour across the + face of cell c
            pt = centers[c].copy()
            pt[ax] = hi[c, ax] + 1e-9
            if pt[ax] >= 1.0:
                continue
            nb = np.nonzero(np.all((lo <= pt) & (pt < hi), axis=1))[0][0]
            # sample points on the smaller of the two faces
            small = c if dm.cell_h[c] <= dm.cell_h[nb] else nb
            s = rng.random((5, 2))
            for st in s:
                x = np.empty(3)
                o = [d for d in range(3) if d != ax]
                x[o[0]] = lo[small, o[0]] + st[0] * dm.cell_h[small]
                x[o[1]] = lo[small, o[1]] + st[1] * dm.cell_h[small]
                x[ax] = hi[c, ax]
                vals = []
                for cell in (c, nb):
                    xi = (x - lo[cell]) / dm.cell_h[cell]
                    L = [basis.lagrange_1d(2, np.array([xi[d]]))[0][:, 0] for d in range(3)]
                    Nv = np.einsum("c,b,a->cba", L[2], L[1], L[0]).ravel()
                    vals.append(Nv @ ul[cell])
                assert abs(vals[0] - vals[1]) <= 1e-13
                checked += 1
    assert checked > 200


def test_l2_projection_reproduces_q2_polynomial_on_octree():
    dm = _band_octree()
    p = lambda x: (1 + x[..., 0] - 2 * x[..., 1] ** 2) * (0.5 + x[..., 2] ** 2)
    xq = asm.qpoint_coords(dm)
    N, _, w = basis.tensor_tables(2, 3)
    fe = np.einsum("cq,q,qi->ci", p(xq) * dm.cell_h[:, None] ** 3, w, N)
    f_all = np.bincount(dm.cell_points.ravel(), weights=fe.ravel(), minlength=dm.points.shape[0])
    b = dm.C.T @ f_all
    u = spla.spsolve(asm.mass_matrix(dm).tocsc(), b)
    assert np.abs(u - p(dm.dof_coords())).max() <= 1e-11


@pytest.mark.parametrize("degree", [2])
def test_manufactured_solution_converges_at_rate_k_plus_1(degree):
    """-div grad u + u = f on the unit cube with homogeneous Neumann data,
    u = cos(pi x) cos(pi y) cos(pi z): L2 error rate k + 1, H1 seminorm rate k."""
    ue = lambda x: np.cos(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1]) * np.cos(np.pi * x[..., 2])
    errs, h1 = [], []
    N, G, w = basis.tensor_tables(degree, degree + 1)
    for n in (2, 4, 8):
        dm = mesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), degree)
        nq = (degree + 1) ** 3
        A = asm.assemble_scalar(dm, np.ones((dm.n_cells, nq)), diff=np.ones((dm.n_cells, nq)))
        xq = asm.qpoint_coords(dm)
        f = (1 + 3 * np.pi ** 2) * ue(xq)
        fe = np.einsum("cq,q,qi->ci", f * dm.cell_h[:, None] ** 3, w, N)
        b = np.bincount(dm.cell_points.ravel(), weights=fe.ravel(), minlength=dm.n_dofs)
        u = spla.spsolve(A.tocsc(), b)
        val, grad = asm.field_at_qpoints(dm, u)
        e = val - ue(xq)
        errs.append(np.sqrt(np.sum(e ** 2 * w * dm.cell_h[:, None] ** 3)))
        gx = -np.pi * np.stack([np.sin(np.pi * xq[..., 0]) * np.cos(np.pi * xq[..., 1]) * np.cos(np.pi * xq[..., 2]),
                                np.cos(np.pi * xq[..., 0]) * np.sin(np.pi * xq[..., 1]) * np.cos(np.pi * xq[..., 2]),
                                np.cos(np.pi * xq[..., 0]) * np.cos(np.pi * xq[..., 1]) * np.sin(np.pi * xq[..., 2])], -1)
        h1.append(np.sqrt(np.sum(np.sum((grad - gx) ** 2, -1) * w * dm.cell_h[:, None] ** 3)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    rates1 = np.log2(np.array(h1[:-1]) / np.array(h1[1:]))
    assert rates[-1] > degree + 1 - 0.25, rates
    assert rates1[-1] > degree - 0.25, rates1


def test_convection_orientation_and_skew_symmetry():
    """C u for u = x and beta = e_x is int N_i (the mass row sum); for constant beta, C + C^T
    vanishes on rows whose support avoids the boundary."""
    dm = mesh.uniform_dofmap(4, (0, 0, 0), (1, 1, 1), 2)
    nq = 27
    conv = np.zeros((dm.n_cells, nq, 3))
    conv[..., 0] = 1.0
    C = asm.assemble_scalar(dm, np.zeros((dm.n_cells, nq)), conv=conv)
    x = dm.dof_coords()
    rowsum = np.asarray(asm.mass_matrix(dm).sum(axis=1)).ravel()
    assert np.allclose(C @ x[:, 0], rowsum, atol=1e-15)
    interior = np.all((x > 0.25 + 1e-12) & (x < 0.75 - 1e-12), axis=1)
    S = (C + C.T).tocsr()
    assert np.abs(S[interior]).max() <= 1e-15


def test_reinit_operator_acts_only_along_the_normal():
    """For phi depending on z only, n = e_z, so (n . grad u) vanishes for u = u(x, y): the
    operator reduces to M / dtau on such functions."""
    dm = mesh.uniform_dofmap(3, (0, 0, 0), (1, 1, 1), 2)
    x = dm.dof_coords()
    phi = np.tanh((0.5 - x[:, 2]) / 0.2)
    A = asm.reinit_matrix(dm, phi, eps=0.05, dtau=0.1)
    M = asm.mass_matrix(dm)
    u = np.sin(2 * x[:, 0]) + x[:, 1] ** 2
    assert np.allclose(A @ u, (M @ u) / 0.1, atol=1e-14 * np.abs(M @ u).max() / 0.1)
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()


def test_oseen_pins():
    n = 2
    dmu = mesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 2)
    dmp = mesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 1)
    x = dmu.dof_coords()
    nu = dmu.n_dofs
    phi = np.ones(nu)  # pure liquid: rho = rho_l, mu = mu_l
    zero = np.zeros((3, nu))
    # viscous part alone annihilates rigid rotations u = (-y, x, 0)
    A = asm.oseen_matrix(dmu, dmp, phi, zero, 0.0, 2.0, 1.0, 3.0, 1.0)
    u = np.concatenate([-x[:, 1], x[:, 0], np.zeros(nu), np.zeros(dmp.n_dofs)])
    assert np.abs(A @ u).max() <= 1e-13
    # but not a shear u = (y, 0, 0)
    u2 = np.concatenate([x[:, 1], np.zeros(2 * nu), np.zeros(dmp.n_dofs)])
    assert np.abs((A @ u2)[:3 * nu]).max() > 1e-3
    # divergence block: B (x, 0, 0) = -int psi_i (minus the Q1 mass row sums)
    u3 = np.concatenate([x[:, 0], np.zeros(2 * nu), np.zeros(dmp.n_dofs)])
    Bu = (A @ u3)[3 * nu:]
    assert np.allclose(Bu, -np.asarray(asm.mass_matrix(dmp).sum(axis=1)).ravel(), atol=1e-15)
    # convection with beta = e_x on u = (x, 0, 0) gives rho int N_i in the first block
    beta = np.zeros((3, nu))
    beta[0] = 1.0
    A0 = asm.oseen_matrix(dmu, dmp, phi, zero, 0.0, 2.0, 1.0, 0.0, 0.0)
    A1 = asm.oseen_matrix(dmu, dmp, phi, beta, 0.0, 2.0, 1.0, 0.0, 0.0)
    r = ((A1 - A0) @ u3)[:nu]
    assert np.allclose(r, 2.0 * np.asarray(asm.mass_matrix(dmu).sum(axis=1)).ravel(), atol=1e-15)
    # symmetric without convection
    assert abs(A - A.T).max() <= 1e-15 * abs(A).max()


# ----------------------------------------------------------------------------- solvers

def _spd(n=60, seed=0, lo=1e-2):
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    lam = np.geomspace(lo, 10.0, n)
    return Q @ np.diag(lam) @ Q.T, lam


def test_cg_and_gmres_reach_the_true_residual():
    A, _ = _spd()
    b = syn.uniform_pm1(3, A.shape[0])
    x, it, rr = krylov.cg(lambda v: A @ v, b, krylov.jacobi(np.diag(A)), 1e-10)
    assert np.linalg.norm(b - A @ x) <= 1e-10 * np.linalg.norm(b)
    A, _ = _spd(lo=1.0)
    rng = np.random.default_rng(1)
    An = A + 0.3 * rng.standard_normal(A.shape) / np.sqrt(A.shape[0])
    x, it, rr = krylov.gmres(lambda v: An @ v, b, krylov.jacobi(np.diag(An)), 20, 1e-10)
    assert np.linalg.norm(b - An @ x) <= 1e-10 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(An, b), rtol=1e-7, atol=1e-8)


def test_chebyshev_is_the_chebyshev_residual_polynomial():
    """With D = I the preconditioner is p(A) and 1 - lambda p(lambda) = T_k((theta - lambda)/delta) / T_k(theta/delta)."""
    A, lam = _spd(40, 2)
    lmin, lmax, k = 0.5, 10.5, 4
    P = krylov.chebyshev(lambda v: A @ v, np.ones(40), lmin, lmax, k)
    w, Q = np.linalg.eigh(A)
    theta, delta = 0.5 * (lmax + lmin), 0.5 * (lmax - lmin)
    Tk = lambda t: np.cosh(k * np.arccosh(t)) if np.all(np.abs(t) >= 1) else np.polynomial.chebyshev.chebval(t, [0] * k + [1])
    T = np.polynomial.chebyshev.chebval
    expect = 1 - T((theta - w) / delta, [0] * (k + 1) + [1]) / T(theta / delta, [0] * (k + 1) + [1])
    for j in range(5):
        z = P(Q[:, j])
        assert abs(Q[:, j] @ A @ z - expect[j]) < 1e-12


def test_lanczos_lambda_max():
    A, lam = _spd(30, 4)
    D = np.diag(A)
    est = krylov.lanczos_lambda_max(lambda v: A @ v, D, syn.uniform_pm1(5, 30), steps=30)
    S = A / np.sqrt(np.outer(D, D))
    assert abs(est - np.linalg.eigvalsh(S)[-1]) < 1e-10


# ----------------------------------------------------------------------------- heat step adjoint

def test_heat_adjoint_gradients_match_central_differences():
    wl = syn.scaled(syn.HEAT_ADJOINT, 4)
    p = wl.params
    dm = mesh.uniform_dofmap(wl.n, wl.lo, wl.hi, 2, dirichlet_faces=heat.DIRICHLET_BOTTOM)
    x = dm.dof_coords()
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    kq = syn.kq_field(dm.n_cells * 27, wl.seed, p["k0"]).reshape(dm.n_cells, 27)
    ztop = wl.hi[2]
    laser = dict(power=200.0, radius=150e-6, x0=0.0, y0=0.0, absorptivity=0.35)
    th_prev = syn.heat_initial_temperature(*x.T, 150e-6, ztop) - p["t_ref"]
    th_prev[dm.dirichlet] = 0
    target = syn.heat_target_temperature(*x.T, ztop, 5, r=160e-6) - p["t_ref"]
    cells = heat.box_cells(dm, 200e-6, 200e-6)
    st = heat.HeatStep(dm, p["rhocp"], p["dt"], kq=kq, beta=beta)
    J, gl, gk, _, _ = heat.gradients(st, th_prev, target, laser, cells)

    def J_of(lz, kq2=None):
        s2 = st if kq2 is None else heat.HeatStep(dm, p["rhocp"], p["dt"], kq=kq2, beta=beta)
        th = s2.solve(s2.rhs(th_prev, lz))
        return heat.objective(dm, th, target, cells)[0]

    for i, k in enumerate(["power", "radius", "x0", "y0"]):
        step = 1e-6 * (abs(laser[k]) if k in ("power", "radius") else laser["radius"])
        a, b = dict(laser), dict(laser)
        a[k] += step
        b[k] -= step
        fd = (J_of(a) - J_of(b)) / (2 * step)
        assert abs(gl[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gl).max()), (k, gl[i], fd)
    big = np.argsort(-np.abs(gk).ravel())[:3]
    for flat in big:
        c, q = divmod(int(flat), 27)
        k2, k3 = kq.copy(), kq.copy()
        hh = 1e-6 * kq[c, q]
        k2[c, q] += hh
        k3[c, q] -= hh
        fd = (J_of(laser, k2) - J_of(laser, k3)) / (2 * hh)
        assert abs(gk[c, q] - fd) <= 1e-6 * abs(fd), (c, q, gk[c, q], fd)


def test_splitmix64_reference_vector():
    g = gold("splitmix64.json")
    out = syn.splitmix64(g["seed"], 5)
    assert [int(v) for v in out] == [int(v) for v in g["first_outputs"]]
    u = syn.uniform_pm1(1, 100000)
    assert u.min() >= -1 and u.max() < 1 and abs(u.mean()) < 0.01
