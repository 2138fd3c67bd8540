"""Element matrices by full quadrature and global CSR assembly (Appendix B).

Every element matrix is the plain triple sum A_e[i, j] = sum_q w_q |J| f(N_i, N_j)(x_q)
over all (k+1)^3 Gauss points, with every shape function and gradient evaluated
directly at every point (``basis.tensor_tables``): no sum factorisation.  Cells are
axis-aligned cubes of edge h, so x = x0 + h xi, |J| = h^3 and grad = grad_xi / h.
The global matrix over all lattice nodes is condensed to the free DoFs as C^T A C;
Dirichlet DoFs get identity rows and columns.  Coefficients that depend on a
nodal field (phi, T, beta) are evaluated from the finite element interpolant of
that field at the Gauss point.
"""
import numpy as np
import scipy.sparse as sp

from .basis import tensor_tables, face_tables
from . import coeffs as co

CHUNK = 4096


def local_values(dm, u):
    """Cell-local node values (ncell, nb) of the free-DoF vector u, through C."""
    return (dm.C @ u)[dm.cell_points]


def field_at_qpoints(dm, u, npts=None):
    """FE interpolant of u at the Gauss points: values (ncell, nq), gradients (ncell, nq, 3)."""
    k = dm.degree
    N, G, _ = tensor_tables(k, npts or k + 1)
    ul = local_values(dm, u)
    val = ul @ N.T
    grad = np.einsum("qid,ci->cqd", G, ul) / dm.cell_h[:, None, None]
    return val, grad


def qpoint_coords(dm, npts=None):
    """Physical coordinates (ncell, nq, 3) of the Gauss points."""
    from .basis import gauss_rule_01
    n = npts or dm.degree + 1
    x, _ = gauss_rule_01(n)
    xi = np.array([[x[a], x[b], x[c]] for c in range(n) for b in range(n) for a in range(n)])
    return dm.cell_origin[:, None, :] + dm.cell_h[:, None, None] * xi[None, :, :]


def _condense(dm, A_full):
    C = dm.C
    A = (C.T @ A_full @ C).tocsr()
    return _dirichlet_identity(A, dm.dirichlet)


def _dirichlet_identity(A, mask):
    if not mask.any():
        return A.tocsr()
    keep = sp.diags((~mask).astype(np.float64))
    return (keep @ A @ keep + sp.diags(mask.astype(np.float64))).tocsr()


def scalar_element_matrices(dm, mass, diff=None, diff_tensor=None, conv=None, cells=None):
    """Element matrices (nc, nb, nb) of
        a(u, v) = int mass u v + grad v . D grad u + v (conv . grad u)
    with per-Gauss-point coefficients mass (ncell, nq), isotropic diff (ncell, nq) or
    tensor diff_tensor (ncell, nq, 3, 3), and conv (ncell, nq, 3)."""
    k = dm.degree
    N, G, w = tensor_tables(k, k + 1)
    cells = np.arange(dm.n_cells) if cells is None else cells
    h = dm.cell_h[cells]
    MM = np.einsum("qi,qj->qij", N, N).reshape(N.shape[0], -1)
    KK = np.einsum("qid,qjd->qij", G, G).reshape(N.shape[0], -1)
    nb = N.shape[1]
    A = (mass[cells] * w * h[:, None] ** 3) @ MM
    if diff is not None:
        A = A + (diff[cells] * w * h[:, None]) @ KK
    A = A.reshape(-1, nb, nb)
    if diff_tensor is not None:
        DG = np.einsum("cqde,qje->cqdj", diff_tensor[cells], G)
        A = A + np.einsum("q,c,qid,cqdj->cij", w, h, G, DG)
    if conv is not None:
        bG = np.einsum("cqd,qjd->cqj", conv[cells], G)
        A = A + np.einsum("q,c,qi,cqj->cij", w, h ** 2, N, bG)
    return A


def assemble_scalar(dm, mass, diff=None, diff_tensor=None, conv=None):
    """Global condensed CSR matrix of the scalar form above."""
    M = dm.points.shape[0]
    parts = []
    for s in range(0, dm.n_cells, CHUNK):
        cells = np.arange(s, min(s + CHUNK, dm.n_cells))
        Ae = scalar_element_matrices(dm, mass, diff, diff_tensor, conv, cells)
        p = dm.cell_points[cells]
        nb = p.shape[1]
        rows = np.repeat(p, nb, axis=1).ravel()
        cols = np.tile(p, (1, nb)).ravel()
        parts.append(sp.csr_matrix((Ae.ravel(), (rows, cols)), shape=(M, M)))
    A_full = parts[0]
    for P in parts[1:]:
        A_full = A_full + P
    return _condense(dm, A_full)


# ----------------------------------------------------------------------------- operators

def helmholtz_coefficients(dm, phi, mass_coef, a_liquid, a_gas, heaviside="tanh", eps=None):
    """Helmholtz workload: int c u v + a(phi) grad u . grad v, a = eq. (muEff) with H(phi_h)."""
    ph, _ = field_at_qpoints(dm, phi)
    H = co.heaviside_tanh(ph) if heaviside == "tanh" else co.heaviside_sine(ph, eps)
    a = co.arithmetic_mix(H, a_liquid, a_gas)
    return np.full_like(a, mass_coef), a


def helmholtz_matrix(dm, phi, mass_coef, a_liquid, a_gas, heaviside="tanh", eps=None):
    m, a = helmholtz_coefficients(dm, phi, mass_coef, a_liquid, a_gas, heaviside, eps)
    return assemble_scalar(dm, m, diff=a)


def heat_coefficients(dm, rhocp, dt, k0=None, t_boil=None, T_prev=None, kq=None, beta=None):
    """Heat-step form: int (rho c_p / dt) u v + k grad u . grad v + rho c_p v beta . grad u,
    with k = k(T_h^n) at the Gauss points, or the given per-Gauss-point k_q (ncell, nq)."""
    nq = (dm.degree + 1) ** 3
    m = np.full((dm.n_cells, nq), rhocp / dt)
    if kq is None:
        Th, _ = field_at_qpoints(dm, T_prev)
        kq = co.conductivity_of_temperature(Th, k0, t_boil)
    conv = None
    if beta is not None:
        bq = np.stack([field_at_qpoints(dm, beta[c])[0] for c in range(3)], axis=-1)
        conv = rhocp * bq
    return m, kq, conv


def heat_matrix(dm, rhocp, dt, k0=None, t_boil=None, T_prev=None, kq=None, beta=None):
    m, kq, conv = heat_coefficients(dm, rhocp, dt, k0, t_boil, T_prev, kq, beta)
    return assemble_scalar(dm, m, diff=kq, conv=conv)


def reinit_coefficients(dm, phi, eps, dtau):
    """Reinitialisation diffusion part: int u v / dtau + eps (n . grad u)(n . grad v),
    n = grad phi_h / |grad phi_h| (zero where |grad phi_h| < 1e-12 / h)."""
    _, g = field_at_qpoints(dm, phi)
    nrm = np.linalg.norm(g, axis=-1)
    small = nrm < 1e-12 / dm.cell_h[:, None]
    n = np.where(small[..., None], 0.0, g / np.where(small, 1.0, nrm)[..., None])
    D = eps * np.einsum("cqd,cqe->cqde", n, n)
    m = np.full(nrm.shape, 1.0 / dtau)
    return m, D


def reinit_matrix(dm, phi, eps, dtau):
    m, D = reinit_coefficients(dm, phi, eps, dtau)
    return assemble_scalar(dm, m, diff_tensor=D)


def mass_matrix(dm, cells=None):
    """Unit-coefficient mass matrix (optionally of a subset of cells), no Dirichlet rows."""
    nq = (dm.degree + 1) ** 3
    m = np.zeros((dm.n_cells, nq))
    sel = np.arange(dm.n_cells) if cells is None else cells
    m[sel] = 1.0
    M = dm.points.shape[0]
    Ae = scalar_element_matrices(dm, m)
    p = dm.cell_points
    nb = p.shape[1]
    A_full = sp.csr_matrix((Ae.ravel(), (np.repeat(p, nb, axis=1).ravel(), np.tile(p, (1, nb)).ravel())),
                           shape=(M, M))
    return (dm.C.T @ A_full @ dm.C).tocsr()


def oseen_matrix(dmu, dmp, phi, beta, sigma, rho_l, rho_g, mu_l, mu_g, T=None, solid=None, darcy=None,
                 trace_correction=False):
    """Linearised incompressible Navier-Stokes (Oseen) operator of eq. (momentum_balance)
    and eq. (continuity) with Q2 velocity and Q1 pressure on one uniform mesh:
        [[ (sigma rho + K) M + C_rho(beta) + int tau(u):grad v,  B^T ],
         [ B,                                                    0   ]],
        (B u, q) = -int q div u,  tau = 2 mu (eps(u) - tr(eps(u)) n n)  (trace_correction)
                                  or 2 mu eps(u),
    rho(phi) by eq. (rhoEff) and mu(phi) by eq. (muEff) with the tanh Heaviside; with ``solid``
    (dict rho_s, mu_s, t_solidus, t_liquidus) and the nodal temperature T, the three-phase laws
    eqs. (solid_liquid_gas_density), (solid_liquid_gas_property) with H_s(f_s(T)); with ``darcy``
    (dict C, b) the damping of eq. (darcy_damping_force) in the dense phase, K = H K_d(f_s(T)),
    moved to the left-hand side.  n = grad phi_h / |grad phi_h| (0 where |grad phi_h| < 1e-12/h).
    Velocity Dirichlet DoFs (all three components) get identity rows/columns."""
    N, G, w = tensor_tables(2, 3)
    P, _, _ = tensor_tables(1, 3)
    ph, gph = field_at_qpoints(dmu, phi)
    H = co.heaviside_tanh(ph)
    if T is not None and (solid is not None or darcy is not None):
        Tq, _ = field_at_qpoints(dmu, T)
    if solid is not None:
        fs = co.solid_fraction(Tq, solid["t_solidus"], solid["t_liquidus"])
        Hs = co.heaviside_solid(fs)
        rho = co.three_phase_density(H, Hs, solid["rho_s"], rho_l, rho_g)
        mu = co.three_phase_mix(H, Hs, solid["mu_s"], mu_l, mu_g)
    else:
        rho = co.reciprocal_density(H, rho_l, rho_g)
        mu = co.arithmetic_mix(H, mu_l, mu_g)
    mass = sigma * rho
    if darcy is not None:
        fs = co.solid_fraction(Tq, darcy["t_solidus"], darcy["t_liquidus"])
        mass = mass + H * co.darcy_coefficient(fs, darcy["C"], darcy["b"])
    if trace_correction:
        gn = np.sqrt(np.sum(gph ** 2, axis=-1))
        small = gn < 1e-12 / dmu.cell_h[:, None]
        nrm = np.where(small[..., None], 0.0, gph / np.where(small, 1.0, gn)[..., None])
    bq = np.stack([field_at_qpoints(dmu, beta[c])[0] for c in range(3)], axis=-1)
    h = dmu.cell_h
    nu, nc = dmu.n_dofs, dmu.n_cells
    rows, cols, vals = [], [], []
    for s in range(0, nc, CHUNK):
        cs = np.arange(s, min(s + CHUNK, nc))
        hc = h[cs]
        wm = mass[cs] * w * hc[:, None] ** 3
        wc = rho[cs] * w * hc[:, None] ** 2
        wv = mu[cs] * w * hc[:, None]
        Mss = np.einsum("cq,qi,qj->cij", wm, N, N)
        bG = np.einsum("cqd,qjd->cqj", bq[cs], G)
        Conv = np.einsum("cq,qi,cqj->cij", wc, N, bG)
        Lap = np.einsum("cq,qid,qjd->cij", wv, G, G)
        pu = dmu.cell_points[cs]
        pp = dmp.cell_points[cs]
        if trace_correction:
            nG = np.einsum("cqd,qid->cqi", nrm[cs], G)           # n . grad N_i (reference)
        for c in range(3):
            for d in range(3):
                Ae = np.einsum("cq,qi,qj->cij", wv, G[:, :, d], G[:, :, c])
                if c == d:
                    Ae = Ae + Mss + Conv + Lap
                if trace_correction:
                    # -2 mu (div u)(n . grad v . n): row comp c (test N_i e_c), column comp d (N_j e_d)
                    Ae = Ae - 2.0 * np.einsum("cq,cq,cqi,qj->cij", wv, nrm[cs][:, :, c], nG, G[:, :, d])
                rows.append(np.repeat(pu + c * nu, 27, axis=1).ravel())
                cols.append(np.tile(pu + d * nu, (1, 27)).ravel())
                vals.append(Ae.ravel())
            # B: pressure rows, velocity component-c columns; and its transpose
            Be = -np.einsum("q,c,qi,qj->cij", w, hc ** 2, P, G[:, :, c])
            r = np.repeat(pp + 3 * nu, 27, axis=1).ravel()
            cc = np.tile(pu + c * nu, (1, 8)).ravel()
            rows += [r, cc]
            cols += [cc, r]
            vals += [Be.ravel(), Be.ravel()]
    n = 3 * nu + dmp.n_dofs
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    mask = np.concatenate([np.tile(dmu.dirichlet, 3), np.zeros(dmp.n_dofs, dtype=bool)])
    return _dirichlet_identity(A, mask)


def laser_rhs(dm, power, radius, x0, y0, absorptivity, derivatives=False):
    """Top-face load vector int_{z = z_max} q(x, y) v dA of eq. (laser_gauss) with the
    (k+1)^2-point Gauss rule on each top face; with ``derivatives`` also the four load
    vectors of dq/dP, dq/dr, dq/dx0, dq/dy0 (shape (4, n))."""
    Nf, wf, xq = face_tables(dm.degree, dm.degree + 1)
    n = dm.degree + 1
    ztop = dm.lo[2] + dm.hspan[2]
    top = np.nonzero(np.isclose(dm.cell_origin[:, 2] + dm.cell_h, ztop, rtol=0, atol=1e-12 * dm.hspan[2]))[0]
    h = dm.cell_h[top]
    px = dm.cell_origin[top, 0][:, None] + h[:, None] * np.array([xq[a] for b in range(n) for a in range(n)])[None]
    py = dm.cell_origin[top, 1][:, None] + h[:, None] * np.array([xq[b] for b in range(n) for a in range(n)])[None]
    M = dm.points.shape[0]
    if derivatives:
        q = co.laser_flux_parameter_derivatives(px, py, power, radius, x0, y0, absorptivity)
    else:
        q = co.laser_flux(px, py, power, radius, x0, y0, absorptivity)[None]
    out = []
    for qq in q:
        fe = np.einsum("cp,p,pi->ci", qq * h[:, None] ** 2, wf, Nf)
        f_full = np.bincount(dm.cell_points[top].ravel(), weights=fe.ravel(), minlength=M)
        f = dm.C.T @ f_full
        f[dm.dirichlet] = 0.0
        out.append(f)
    return np.array(out) if derivatives else out[0]
