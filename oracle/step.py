"""One time step of the overall solution algorithm (Algorithm algo:meltpooldg) on one uniform
mesh, by plain assembly and direct sparse solves (test infrastructure: only tests, smoke() and the
bench's CPU leg use this package).

Fields: velocity Q2 (three components), pressure Q1, level set phi and temperature T as Q2 fields
on the velocity lattice.  All Gauss-point quantities come from the finite element interpolants with
every basis function evaluated directly (``basis.tensor_tables``), all loads are full-quadrature
integrals condensed through C^T, all systems are assembled (``assemble``) and solved with
``scipy.sparse.linalg.spsolve``.

The step, in the algorithm's order:
 1. predictors x* = 2 x^n - x^(n-1) for u, T, phi (extrapolate; x^(n-1) = x^n gives x* = x^n);
 2. level set:
    * transport velocity of variant 1 (eq. transport_vel_local_continuous) at the Gauss points,
      u_G = u*_h + mdot(T*_h) / rho(phi*_h) n(phi*_h);
    * advection (eq. transport) by backward Euler: (M/dt + C(u_G)) phi_a = M phi^n / dt;
    * Olsson's reinitialisation, n_r from phi_a, K_r pseudo-time steps of
      (M/dtau + eps N_{n_r}) psi^(k+1) = M psi^k / dtau + F(psi^k),
      F_i = int (1 - psi_h^2)/2 n_r . grad N_i, psi^0 = phi_a, phi^(n+1) = psi^(K_r);
    * geometry: n_G = grad phi_h / |grad phi_h| and kappa = -div n_G of phi^(n+1)_h;
 3. heat (eq. heat_transfer): properties (rho c_p)(phi^(n+1)), k(phi^(n+1)) by eq. (muEff);
    s = evaporative cooling with mdot(T*) (eq. vapor_heat_loss) + interface laser flux
    (eq. laser_gauss); backward Euler
      (M_{rho c_p/dt} + K_k + C_{rho c_p}(u*)) T^(n+1) = M_{rho c_p/dt} T^n + s,
    Dirichlet DoFs keep T^n (their columns lifted to the right-hand side);
 4. Navier-Stokes (eqs. continuity, momentum_balance), linearised about beta = u*, sigma = 1/dt:
    the melt-pool Oseen operator of ``assemble.oseen_matrix`` with phi^(n+1), T^(n+1); velocity
    load sigma M_rho u^n + rho g + surface tension (eq. surface_tension) + hybrid recoil force;
    pressure rows -int q sdot (B = -div, continuity div u = sdot of eq. evaporDil); velocity
    Dirichlet rows 0.

Readings (the paper leaves these open; each is listed with the design notes):
* one mesh, phi and T in Q2 on the velocity lattice (the paper's level-set and heat meshes are
  finer Q1 meshes);
* backward Euler for every field; the explicit couplings use the predictors (mdot of the
  transport velocity and of the cooling from T*) or the fields just computed (recoil, dilation,
  surface tension from T^(n+1) and phi^(n+1));
* Olsson's conservative reinitialisation written for phi in [-1, 1]: the stationary profile
  tanh(d / (2 eps)) balances the flux (1 - phi^2)/2 n against eps (grad phi . n) n; the
  compressive part is explicit, its boundary term dropped (|psi| = 1 there);
* curvature and normal straight from phi^(n+1)_h (the paper's filtered projection, S8, is out of
  scope): kappa = -(tr Hess - n^T Hess n) / |grad phi_h|, 0 where grad phi_h vanishes;
* the laser factor is <n_G . e_L> with n_G = grad phi / |grad phi| pointing into the dense phase
  and e_L the beam direction (the printed <-n_G . e_L> with this n_G would switch the laser off
  wherever the beam meets the melt); d_L is the distance to the beam axis through x_L;
* surface tension alpha(T) = max(alpha_0 - alpha_1 (T - T_alpha), alpha_res), grad alpha =
  -alpha_1 grad T_h where the first branch is active, else 0.
"""
import numpy as np
import scipy.sparse.linalg as sla

from . import assemble as asm
from . import coeffs as co
from . import interface as oi
from .basis import tensor_tables


# ----------------------------------------------------------------------------- Gauss-point fields

def hessian_at_qpoints(dm, u):
    """Hessian (ncell, nq, 3, 3) of the Q2 interpolant of u at the Gauss points, from the second
    derivatives of the 1D Lagrange polynomials (a quadratic l_a has the constant l_a'')."""
    from .basis import gauss_rule_01, lagrange_1d, lagrange_nodes
    k = dm.degree
    xq, _ = gauss_rule_01(k + 1)
    L, dL = lagrange_1d(k, xq)
    nodes = lagrange_nodes(k)
    d2 = np.zeros((k + 1, xq.size))
    for a in range(k + 1):
        # l_a'' of the product formula: sum over ordered pairs of factors that are differentiated
        for m in range(k + 1):
            for l in range(k + 1):
                if m == a or l == a or l == m:
                    continue
                term = np.full(xq.size, 1.0 / ((nodes[a] - nodes[m]) * (nodes[a] - nodes[l])))
                for b in range(k + 1):
                    if b not in (a, m, l):
                        term = term * (xq - nodes[b]) / (nodes[a] - nodes[b])
                d2[a] += term
    n1 = k + 1
    nq, nb = n1 ** 3, n1 ** 3
    Hb = np.zeros((nq, nb, 3, 3))
    for qc in range(n1):
        for qb in range(n1):
            for qa in range(n1):
                q = qa + n1 * (qb + n1 * qc)
                for c in range(n1):
                    for b in range(n1):
                        for a in range(n1):
                            i = a + n1 * (b + n1 * c)
                            v = [(L[a, qa], dL[a, qa], d2[a, qa]), (L[b, qb], dL[b, qb], d2[b, qb]),
                                 (L[c, qc], dL[c, qc], d2[c, qc])]
                            for d in range(3):
                                for e in range(3):
                                    order = [0, 0, 0]
                                    order[d] += 1
                                    order[e] += 1
                                    Hb[q, i, d, e] = v[0][order[0]] * v[1][order[1]] * v[2][order[2]]
    ul = asm.local_values(dm, u)
    return np.einsum("qide,ci->cqde", Hb, ul) / dm.cell_h[:, None, None, None] ** 2


def normal_and_curvature(dm, phi):
    """n_G = grad phi_h / |grad phi_h| and kappa = -div n_G at the Gauss points (0 where
    |grad phi_h| < 1e-12 / h)."""
    _, g = asm.field_at_qpoints(dm, phi)
    Hs = hessian_at_qpoints(dm, phi)
    gn = np.linalg.norm(g, axis=-1)
    small = gn < 1e-12 / dm.cell_h[:, None]
    safe = np.where(small, 1.0, gn)
    n = np.where(small[..., None], 0.0, g / safe[..., None])
    tr = np.trace(Hs, axis1=-2, axis2=-1)
    nHn = np.einsum("cqd,cqde,cqe->cq", n, Hs, n)
    kappa = np.where(small, 0.0, -(tr - nHn) / safe)
    return n, kappa


def mass_flux(T, ev):
    if ev["model"] == "knight":
        return oi.mass_flux_knight(T, ev["p_amb"], ev["h_v"], ev["molar_mass"], ev["t_boil"], ev["sticking"])
    return oi.mass_flux_tanasawa(T, ev["tanasawa"], ev["t_boil"])


def transport_velocity(dm, u, T, phi, prm):
    """Eq. (transport_vel_local_continuous), variant 1, at the Gauss points (ncell, nq, 3):
    u_G = u_h + mdot(T_h) / rho(phi_h) n_G(phi_h), rho by eq. (rhoEff)."""
    uq = np.stack([asm.field_at_qpoints(dm, u[c])[0] for c in range(3)], axis=-1)
    Tq, _ = asm.field_at_qpoints(dm, T)
    ph, g = asm.field_at_qpoints(dm, phi)
    gn = np.linalg.norm(g, axis=-1)
    small = gn < 1e-12 / dm.cell_h[:, None]
    n = np.where(small[..., None], 0.0, g / np.where(small, 1.0, gn)[..., None])
    rho = co.reciprocal_density(co.heaviside_tanh(ph), prm["rho_l"], prm["rho_g"])
    return uq + (mass_flux(Tq, prm["evaporation"]) / rho)[..., None] * n


def surface_tension_density(n, kappa, T, gradT, delta_rho, st):
    """Eq. (surface_tension) at points: (alpha kappa n + (I - n n) grad alpha) delta_rho."""
    lin = st["alpha0"] - st["alpha1"] * (T - st["t_alpha"])
    active = lin > st["alpha_res"]
    alpha = np.where(active, lin, st["alpha_res"])
    galpha = np.where(active[..., None], -st["alpha1"] * gradT, 0.0)
    tang = galpha - np.sum(n * galpha, axis=-1)[..., None] * n
    return (alpha * kappa)[..., None] * n * delta_rho[..., None] + tang * delta_rho[..., None]


def laser_density(x, n, delta_rhocp, laser):
    """Eq. (laser_gauss) at points x (..., 3): 2 chi P / (pi r^2) <n_G . e_L> exp(-2 d_L^2 / r^2)
    delta_rhocp, d_L the distance to the beam axis through x_L along e_L (unit)."""
    eL = np.asarray(laser["direction"], float)
    r = x - np.asarray(laser["focus"], float)
    perp = r - (r @ eL)[..., None] * eL          # the component off the axis (no cancellation)
    d2 = np.sum(perp * perp, axis=-1)
    q0 = 2.0 * laser["absorptivity"] * laser["power"] / (np.pi * laser["radius"] ** 2)
    return q0 * np.maximum(n @ eL, 0.0) * np.exp(-2.0 * d2 / laser["radius"] ** 2) * delta_rhocp


# ----------------------------------------------------------------------------- loads

def load(dm, s=None, V=None, dirichlet_zero=False):
    """f_i = int s N_i + V . grad N_i over every cell (s: (ncell, nq), V: (ncell, nq, 3)),
    condensed through C^T; Dirichlet rows set to 0 if asked."""
    N, G, w = tensor_tables(dm.degree, dm.degree + 1)
    h = dm.cell_h
    loc = np.zeros((dm.n_cells, N.shape[1]))
    if s is not None:
        loc += np.einsum("cq,qi->ci", s * w * h[:, None] ** 3, N)
    if V is not None:
        loc += np.einsum("cqd,qid->ci", V * (w * h[:, None] ** 2)[..., None], G)
    f = np.bincount(dm.cell_points.ravel(), weights=loc.ravel(), minlength=dm.points.shape[0])
    f = dm.C.T @ f
    if dirichlet_zero:
        f[dm.dirichlet] = 0.0
    return f


def compressive_flux(dm, psi, nrm):
    """F_i = int (1 - psi_h^2)/2 n . grad N_i with the given Gauss-point normals (ncell, nq, 3)."""
    pq, _ = asm.field_at_qpoints(dm, psi)
    return load(dm, V=(0.5 * (1.0 - pq * pq))[..., None] * nrm)


def _normal(dm, phi):
    _, g = asm.field_at_qpoints(dm, phi)
    gn = np.linalg.norm(g, axis=-1)
    small = gn < 1e-12 / dm.cell_h[:, None]
    return np.where(small[..., None], 0.0, g / np.where(small, 1.0, gn)[..., None])


# ----------------------------------------------------------------------------- the step

def _sources(prm):
    ev = prm["evaporation"]
    return dict(rho_l=prm["rho_l"], rho_g=prm["rho_g"], rhocp_l=prm["rhocp_l"], rhocp_g=prm["rhocp_g"],
                heaviside="tanh", eps=prm["eps"], model=ev["model"], p_amb=ev["p_amb"], h_v=ev["h_v"],
                molar_mass=ev["molar_mass"], t_boil=ev["t_boil"], sticking=ev["sticking"],
                tanasawa=ev["tanasawa"], recoil=True)


def predictors(state):
    """Step 1: x* = 2 x^n - x^(n-1) for u, T and phi."""
    return (2.0 * state["u"] - state["u_prev"], 2.0 * state["T"] - state["T_prev"],
            2.0 * state["phi"] - state["phi_prev"])


def advection_system(dmphi, phi_n, u_s, T_s, phi_s, prm):
    """Step 2, advection: (M/dt + C(u_G)) phi_a = M phi^n / dt with u_G of variant 1."""
    dt = prm["dt"]
    uG = transport_velocity(dmphi, u_s, T_s, phi_s, prm)
    A = asm.assemble_scalar(dmphi, np.full(uG.shape[:2], 1.0 / dt), conv=uG)
    return A, load(dmphi, s=asm.field_at_qpoints(dmphi, phi_n)[0] / dt), uG


def reinitialise(dmphi, phi_a, prm):
    """Step 2, reinitialisation: K_r pseudo-time steps with the normal of phi_a."""
    nr = _normal(dmphi, phi_a)
    A = asm.reinit_matrix(dmphi, phi_a, prm["eps"], prm["dtau"])
    psi = phi_a
    for _ in range(prm["reinit_steps"]):
        rhs = load(dmphi, s=asm.field_at_qpoints(dmphi, psi)[0] / prm["dtau"]) + compressive_flux(dmphi, psi, nr)
        psi = sla.spsolve(A.tocsc(), rhs)
    return psi, A


def heat_system(maps, T_n, u_s, T_s, phi_new, prm):
    """Step 3: the heat matrix A_T (Dirichlet rows identity), the right-hand side with the
    Dirichlet columns lifted, r = s + M_{rho c_p/dt} T^n - A_all T^n (Dirichlet rows 0), the
    right-hand side of the update T^(n+1) - T^n, and A_all (the form without Dirichlet rows)."""
    dmu, dmp, dmphi, dmT = maps
    dt = prm["dt"]
    ph, gph = asm.field_at_qpoints(dmT, phi_new)
    H = co.heaviside_tanh(ph)
    rhocp = co.arithmetic_mix(H, prm["rhocp_l"], prm["rhocp_g"])
    kq = co.arithmetic_mix(H, prm["k_l"], prm["k_g"])
    uq = np.stack([asm.field_at_qpoints(dmT, u_s[c])[0] for c in range(3)], axis=-1)
    coef = dict(diff=kq, conv=rhocp[..., None] * uq)
    A_T = asm.assemble_scalar(dmT, rhocp / dt, **coef)
    A_all = asm.assemble_scalar(dmphi, rhocp / dt, **coef)     # the same form without Dirichlet rows
    _, _, f_cool = oi.interface_sources(dmu, dmp, phi_new, T_s, _sources(prm))
    b = load(dmT, s=rhocp / dt * asm.field_at_qpoints(dmT, T_n)[0]) + f_cool
    if prm.get("laser") is not None:
        n_G, _ = normal_and_curvature(dmT, phi_new)
        d_rhocp = oi.delta_smoothed(ph, gph, "tanh") * rhocp * rhocp * oi.c_rhocp(prm["rhocp_l"], prm["rhocp_g"])
        b = b + load(dmT, s=laser_density(asm.qpoint_coords(dmT), n_G, d_rhocp, prm["laser"]))
    # Dirichlet DoFs keep T^n; the eliminated columns move to the right-hand side (lifting)
    D = dmT.dirichlet
    rhs = b - A_all @ np.where(D, T_n, 0.0)
    rhs[D] = T_n[D]
    r = b - A_all @ T_n
    r[D] = 0.0
    return A_T, rhs, r, A_all


def flow_system(maps, u_n, u_s, phi_new, T_new, prm):
    """Step 4: the melt-pool Oseen matrix and its right-hand side [f_u; -f_dilation]."""
    dmu, dmp = maps[0], maps[1]
    sigma = 1.0 / prm["dt"]
    A = asm.oseen_matrix(dmu, dmp, phi_new, u_s, sigma, prm["rho_l"], prm["rho_g"], prm["mu_l"], prm["mu_g"],
                         T=T_new, solid=prm.get("solid"), darcy=prm.get("darcy"),
                         trace_correction=prm.get("trace_correction", False))
    ph, gph = asm.field_at_qpoints(dmu, phi_new)
    H = co.heaviside_tanh(ph)
    Tq, gT = asm.field_at_qpoints(dmu, T_new)
    if prm.get("solid") is not None:
        s = prm["solid"]
        Hs = co.heaviside_solid(co.solid_fraction(Tq, s["t_solidus"], s["t_liquidus"]))
        rho = co.three_phase_density(H, Hs, s["rho_s"], prm["rho_l"], prm["rho_g"])
    else:
        rho = co.reciprocal_density(H, prm["rho_l"], prm["rho_g"])
    d_rho = oi.delta_smoothed(ph, gph, "tanh") * co.reciprocal_density(H, prm["rho_l"], prm["rho_g"]) * \
        oi.c_rho(prm["rho_l"], prm["rho_g"])
    n_G, kappa = normal_and_curvature(dmu, phi_new)
    f_st = surface_tension_density(n_G, kappa, Tq, gT, d_rho, prm["surface_tension"])
    f_rec, f_dil, _ = oi.interface_sources(dmu, dmp, phi_new, T_new, _sources(prm))
    g = np.asarray(prm.get("gravity", (0.0, 0.0, 0.0)), float)
    f_u = []
    for c in range(3):
        unq, _ = asm.field_at_qpoints(dmu, u_n[c])
        f_u.append(load(dmu, s=sigma * rho * unq + rho * g[c] + f_st[..., c], dirichlet_zero=True))
    return A, np.concatenate([np.concatenate(f_u) + f_rec, -f_dil])


def step(maps, state, prm, keep=False):
    """One step.  maps = (dmu, dmp, dmphi, dmT): Q2 velocity (Dirichlet faces of u), Q1
    pressure, Q2 level set (no Dirichlet) and Q2 temperature (Dirichlet faces of T), all uniform on
    one mesh.  state: u, u_prev (3, n); T, T_prev, phi, phi_prev (n).  prm: dt, eps, rho_l, rho_g,
    mu_l, mu_g, rhocp_l, rhocp_g, k_l, k_g, evaporation (model, p_amb, h_v, molar_mass, t_boil,
    sticking, tanasawa), surface_tension (alpha0, alpha1, t_alpha, alpha_res), gravity (3), laser
    (power, radius, absorptivity, focus, direction) or None, reinit_steps, dtau, solid / darcy
    (dicts or None), trace_correction.  Returns u (3, n), p, T, phi (and the intermediate fields
    and systems with keep)."""
    dmu, dmp, dmphi, dmT = maps
    u_s, T_s, phi_s = predictors(state)
    A_adv, b_adv, uG = advection_system(dmphi, state["phi"], u_s, T_s, phi_s, prm)
    phi_a = sla.spsolve(A_adv.tocsc(), b_adv)
    phi_new, A_re = reinitialise(dmphi, phi_a, prm)
    A_T, rhs_T, r_T, _ = heat_system(maps, state["T"], u_s, T_s, phi_new, prm)
    T_new = sla.spsolve(A_T.tocsc(), rhs_T)
    A_ns, rhs = flow_system(maps, state["u"], u_s, phi_new, T_new, prm)
    x = sla.spsolve(A_ns.tocsc(), rhs)
    nu = dmu.n_dofs
    out = dict(u=x[:3 * nu].reshape(3, nu), p=x[3 * nu:], T=T_new, phi=phi_new)
    if keep:
        out.update(phi_adv=phi_a, u_star=u_s, T_star=T_s, phi_star=phi_s, u_gamma=uG, b_adv=b_adv, rhs_T=rhs_T,
                   r_T=r_T, rhs_ns=rhs, A_adv=A_adv, A_re=A_re, A_T=A_T, A_ns=A_ns)
    return out
