"""Pins of the oracle's melt-pool time step (Algorithm algo:meltpooldg) and of its new pieces:
curvature and normal on quadrics the Q2 space reproduces exactly, the surface tension of eq.
(surface_tension) and the laser flux of eq. (laser_gauss) in closed-form configurations, the
absorbed laser power chi P in the mesh limit, the conservation identities of Olsson's compressive
flux, and whole steps whose exact discrete solution is known (linear advection, hydrostatics,
energy balance, quiescent states)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import coeffs as co
from oracle import interface as oi
from oracle import mesh as omesh
from oracle import step as st

TI = syn.TI64


def _unit(n, faces=0, degree=2):
    return omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), degree, faces)


def test_hessian_of_a_quadratic_is_exact():
    dm = _unit(3)
    x, y, z = dm.dof_coords().T
    Hs = st.hessian_at_qpoints(dm, x * y + 2 * y * z - z * z + 3 * x * x)
    ref = np.array([[6.0, 1.0, 0.0], [1.0, 0.0, 2.0], [0.0, 2.0, -2.0]])
    assert np.abs(Hs - ref).max() <= 1e-11


@pytest.mark.parametrize("shape", ["sphere", "cylinder", "plane"])
def test_normal_and_curvature_of_quadrics(shape):
    """phi = 1 - s |x - c|^2 (in the Q2 space): n = -(x - c)/r pointing into phi > 0, kappa = 2/r;
    the cylinder gives 1/rho; a linear phi gives its constant direction and kappa = 0."""
    dm = _unit(3)
    X = dm.dof_coords()
    c = np.array([0.41, 0.53, 0.47])
    xq = asm.qpoint_coords(dm)
    if shape == "sphere":
        phi = 1.0 - 2.0 * np.sum((X - c) ** 2, axis=1)
        r = xq - c
    elif shape == "cylinder":
        phi = 1.0 - 2.0 * np.sum((X[:, :2] - c[:2]) ** 2, axis=1)
        r = np.concatenate([xq[..., :2] - c[:2], np.zeros(xq.shape[:-1] + (1,))], axis=-1)
    else:
        a = np.array([0.3, -0.4, 1.2])
        phi = X @ a + 0.1
    n, kappa = st.normal_and_curvature(dm, phi)
    if shape == "plane":
        assert np.abs(n - a / np.linalg.norm(a)).max() <= 1e-13
        assert np.abs(kappa).max() <= 1e-11
        return
    rn = np.linalg.norm(r, axis=-1)
    assert np.abs(n + r / rn[..., None]).max() <= 1e-12
    expect = (2.0 if shape == "sphere" else 1.0) / rn
    assert np.abs(kappa / expect - 1.0).max() <= 1e-11


def test_surface_tension_closed_forms():
    st_p = dict(alpha0=1.493, alpha1=5.5e-4, t_alpha=1928.0, alpha_res=0.01)
    rng = np.random.default_rng(4)
    # flat interface (kappa = 0, n = -e_z), T = T0 + 7 x: pure Marangoni force -alpha_1 7 e_x delta
    n = np.tile([0.0, 0.0, -1.0], (5, 1))
    dl = rng.uniform(0.5, 2.0, 5)
    f = st.surface_tension_density(n, np.zeros(5), np.full(5, 2500.0), np.tile([7.0, 0.0, 3.0], (5, 1)), dl, st_p)
    assert np.allclose(f, np.stack([-5.5e-4 * 7.0 * dl, 0 * dl, 0 * dl], axis=1), rtol=1e-14, atol=0)
    # hot enough for the residual coefficient: alpha = alpha_res, no Marangoni term
    f = st.surface_tension_density(n, np.full(5, 3.0), np.full(5, 5000.0), np.tile([7.0, 1.0, 3.0], (5, 1)), dl,
                                   st_p)
    assert np.allclose(f, (0.01 * 3.0 * dl)[:, None] * n, rtol=1e-14, atol=0)
    # in general n . f = alpha kappa delta (the Marangoni part is tangential)
    nn = rng.normal(size=(7, 3))
    nn /= np.linalg.norm(nn, axis=1)[:, None]
    T = rng.uniform(1500, 3000, 7)
    kap = rng.normal(size=7)
    dl = rng.uniform(0.5, 2.0, 7)
    f = st.surface_tension_density(nn, kap, T, rng.normal(size=(7, 3)), dl, st_p)
    alpha = 1.493 - 5.5e-4 * (T - 1928.0)
    assert np.allclose(np.sum(f * nn, axis=1), alpha * kap * dl, rtol=1e-12, atol=0)


def test_laser_density_closed_forms():
    las = dict(power=200.0, radius=50e-6, absorptivity=0.35, focus=(1e-5, -2e-5, 7.0), direction=(0, 0, -1))
    x = np.array([[1e-5, -2e-5, 0.0], [6e-5, -2e-5, 1e-4], [1e-5, 3e-5, -2e-4]])
    q0 = 2 * 0.35 * 200.0 / (np.pi * 2.5e-9)
    down = np.tile([0.0, 0.0, -1.0], (3, 1))
    got = st.laser_density(x, down, np.ones(3), las)
    assert np.allclose(got, q0 * np.exp(-2.0 * np.array([0.0, 1.0, 1.0])), rtol=1e-14)
    assert np.all(st.laser_density(x, -down, np.ones(3), las) == 0.0)   # melt above the gas: no heating
    # a tilted beam: distance to the axis, and the factor n . e_L
    th = 0.3
    las2 = dict(las, focus=(0.0, 0.0, 0.0), direction=(np.sin(th), 0.0, -np.cos(th)))
    p = np.array([[0.0, 4e-5, 0.0]])
    assert st.laser_density(p, down[:1], np.ones(1), las2)[0] == pytest.approx(
        q0 * np.cos(th) * np.exp(-2.0 * (4e-5 / 5e-5) ** 2), rel=1e-13)


def test_absorbed_laser_power_tends_to_chi_P():
    """A flat interface under a centred beam: the load sums to int q = chi P (the Gaussian's tail
    outside the 600 um box is e^-72) up to the discretisation of delta_rhocp, which halves and more
    with every refinement."""
    L = 3e-4
    las = dict(power=200.0, radius=50e-6, absorptivity=0.35, focus=(0, 0, 0), direction=(0, 0, -1))
    errs = []
    for n in (16, 24):
        dm = omesh.uniform_dofmap(n, (-L, -L, -L), (L, L, L), 2)
        eps = 2 * (2 * L / n)
        phi = np.tanh(-dm.dof_coords()[:, 2] / (2 * eps))
        ph, g = asm.field_at_qpoints(dm, phi)
        rhocp = co.arithmetic_mix(co.heaviside_tanh(ph), TI["rho_l"] * TI["cp_l"], TI["rho_g"] * TI["cp_g"])
        d = oi.delta_smoothed(ph, g, "tanh") * rhocp ** 2 * oi.c_rhocp(TI["rho_l"] * TI["cp_l"],
                                                                        TI["rho_g"] * TI["cp_g"])
        nG, _ = st.normal_and_curvature(dm, phi)
        f = st.load(dm, s=st.laser_density(asm.qpoint_coords(dm), nG, d, las))
        errs.append(abs(f.sum() / 70.0 - 1.0))
    assert errs[1] < 1e-2 and errs[1] < 0.25 * errs[0], errs


def test_compressive_flux_identities():
    """F_i = int (1 - psi^2)/2 n . grad N_i: sum_i F_i = 0 (conservation), and with x_i the DoF
    coordinates sum_i z_i F_i = int (1 - psi^2)/2 n_z, here for psi = a + b z in closed form."""
    dm = _unit(3)
    z = dm.dof_coords()[:, 2]
    a, b = -0.3, 0.8
    nrm = np.broadcast_to(np.array([0.2, -0.3, 0.9]), (dm.n_cells, 27, 3))
    F = st.compressive_flux(dm, a + b * z, nrm)
    assert abs(F.sum()) <= 1e-15
    exact = 0.9 / 2.0 * (1.0 - (a * a + a * b + b * b / 3.0))
    assert (z @ F) == pytest.approx(exact, rel=1e-13)


def test_transport_velocity_reductions():
    dm = _unit(3)
    X = dm.dof_coords()
    u = np.stack([0.3 + 0 * X[:, 0], X[:, 1], -X[:, 2]])
    phi = np.tanh((0.55 - X[:, 2]) / 0.2)
    T = 2500.0 + 800.0 * X[:, 0]
    base = dict(rho_l=TI["rho_l"], rho_g=TI["rho_g"])
    ev0 = dict(model="tanasawa", tanasawa=0.0, t_boil=3133.0)
    uq = np.stack([asm.field_at_qpoints(dm, u[c])[0] for c in range(3)], axis=-1)
    assert np.array_equal(st.transport_velocity(dm, u, T, phi, dict(base, evaporation=ev0)), uq)
    ev = dict(model="knight", p_amb=101325.0, h_v=TI["h_v"], molar_mass=TI["molar_mass"], t_boil=3133.0, sticking=1.0)
    uG = st.transport_velocity(dm, 0 * u, T, phi, dict(base, evaporation=ev))
    # the evaporation part points along grad phi_h (into the melt; the Q2 interpolant of tanh is
    # not monotone, so grad phi_h changes sign in the saturated cells) ...
    _, g = asm.field_at_qpoints(dm, phi)
    assert np.abs(uG[..., :2]).max() <= 1e-12 * np.abs(uG).max()
    assert np.all(uG[..., 2] * g[..., 2] > 0)
    # ... with magnitude mdot / rho, which grows towards the gas by rho_l / rho_g at most
    Tq, _ = asm.field_at_qpoints(dm, T)
    m = oi.mass_flux_knight(Tq, 101325.0, TI["h_v"], TI["molar_mass"], 3133.0)
    ratio = np.abs(uG[..., 2]) / m
    assert ratio.min() >= 1.0 / TI["rho_l"] * (1 - 1e-12) and ratio.max() <= 1.0 / TI["rho_g"] * (1 + 1e-12)


# ----------------------------------------------------------------------------- whole steps

def _params(**kw):
    p = dict(dt=1e-3, eps=0.25, rho_l=TI["rho_l"], rho_g=TI["rho_g"], mu_l=TI["mu_l"], mu_g=TI["mu_g"],
             rhocp_l=TI["rho_l"] * TI["cp_l"], rhocp_g=TI["rho_g"] * TI["cp_g"], k_l=TI["k_l"], k_g=TI["k_g"],
             evaporation=dict(model="tanasawa", tanasawa=0.0, p_amb=0.0, h_v=TI["h_v"],     # no recoil either
                              molar_mass=TI["molar_mass"], t_boil=3133.0, sticking=1.0),
             surface_tension=dict(alpha0=0.0, alpha1=0.0, t_alpha=1928.0, alpha_res=0.0),
             gravity=(0.0, 0.0, 0.0), laser=None, reinit_steps=0, dtau=0.125, solid=None, darcy=None)
    p.update(kw)
    return p


def _maps(n, u_faces=0b011111, t_faces=1 << 4):
    return _unit(n, u_faces), _unit(n, 0, 1), _unit(n), _unit(n, t_faces)


def _state(nu, u=None, T=1000.0, phi=None):
    u = np.zeros((3, nu)) if u is None else u
    T = np.full(nu, T) if np.isscalar(T) else T
    return dict(u=u, u_prev=u, T=T, T_prev=T, phi=phi, phi_prev=phi)


def test_linear_level_set_is_advected_exactly():
    """u_G constant (mdot = 0), phi linear: backward Euler keeps phi linear and the Galerkin solution
    is the exact phi - dt u . grad phi (the form's residual vanishes pointwise)."""
    maps = _maps(3)
    X = maps[2].dof_coords()
    a = np.array([0.2, -0.1, 0.4])
    u = np.tile(np.array([0.3, -0.2, 0.1])[:, None], (1, X.shape[0]))
    s = _state(X.shape[0], u=u, phi=X @ a - 0.3)
    s["u_prev"] = 0.5 * u                      # the predictor 2u - u_prev = 1.5 u is what advects
    out = st.step(maps, s, _params(dt=0.1), keep=True)
    expect = X @ a - 0.3 - 0.1 * (1.5 * np.array([0.3, -0.2, 0.1])) @ a
    assert np.abs(out["phi_adv"] - expect).max() <= 1e-13


def test_reinitialisation_sharpens_a_wide_profile_and_conserves_mass():
    maps = _maps(6)
    dm = maps[2]
    z = dm.dof_coords()[:, 2]
    eps = 1.0 / 12
    wide = np.tanh((0.5 - z) / (4 * eps))
    target = np.tanh((0.5 - z) / (2 * eps))
    M = asm.mass_matrix(dm)
    s = _state(dm.n_dofs, phi=wide)
    errs, mass = [], []
    for k in (0, 2, 6):
        out = st.step(maps, s, _params(eps=eps, dtau=0.5 / 12, reinit_steps=k))
        errs.append(np.abs(out["phi"] - target).max())
        mass.append((M @ out["phi"]).sum())
    assert errs[2] < errs[1] < errs[0]
    assert max(abs(m - mass[0]) for m in mass) <= 1e-12 * np.abs(M @ np.abs(wide)).sum()


def test_hydrostatic_pressure_is_exact():
    """One phase at rest under gravity, walls on five faces and an open top: u = 0 and
    p = rho |g| (z_top - z) (linear, in Q1) solve the discrete system exactly."""
    maps = _maps(3)
    dmu, dmp = maps[0], maps[1]
    s = _state(dmu.n_dofs, phi=np.ones(dmu.n_dofs))
    out = st.step(maps, s, _params(gravity=(0.0, 0.0, -9.81)))
    zp = dmp.dof_coords()[:, 2]
    scale = TI["rho_l"] * 9.81
    # exact up to the LU's rounding on a saddle-point system with sigma rho / mu ~ 1e6
    assert np.abs(out["u"]).max() <= 1e-9 * scale
    assert np.abs(out["p"] - TI["rho_l"] * 9.81 * (1.0 - zp)).max() <= 1e-9 * scale


def test_energy_balance_of_the_heat_step():
    """No Dirichlet face, fluid at rest, laser on and cooling by Tanasawa: the heat step's sum over
    all rows is int rho c_p (T^(n+1) - T^n) / dt = int (laser + cooling) (Neumann: K 1 = 0)."""
    L = 3e-4
    maps = [omesh.uniform_dofmap(6, (-L, -L, -L), (L, L, L), d, f) for d, f in ((2, 0b011111), (1, 0), (2, 0), (2, 0))]
    dmT = maps[3]
    x = dmT.dof_coords()
    eps = 2 * (2 * L / 6)
    phi = np.tanh(-x[:, 2] / (2 * eps))
    T = 2800.0 + 600.0 * np.exp(-(x[:, 0] ** 2 + x[:, 1] ** 2) / (1e-4) ** 2)
    las = dict(power=200.0, radius=50e-6, absorptivity=0.35, focus=(0, 0, 0), direction=(0, 0, -1))
    ev = dict(model="tanasawa", tanasawa=2e-3, p_amb=101325.0, h_v=TI["h_v"], molar_mass=TI["molar_mass"],
              t_boil=3133.0, sticking=1.0)
    prm = _params(dt=1e-6, eps=eps, laser=las, evaporation=ev)
    out = st.step(maps, _state(dmT.n_dofs, T=T, phi=phi), prm, keep=True)
    ph, _ = asm.field_at_qpoints(dmT, out["phi"])
    rhocp = co.arithmetic_mix(co.heaviside_tanh(ph), prm["rhocp_l"], prm["rhocp_g"])
    dT = asm.field_at_qpoints(dmT, out["T"] - T)[0]
    stored = np.sum(rhocp * dT * (asm.tensor_tables(2, 3)[2] * dmT.cell_h[:, None] ** 3)) / 1e-6
    src = out["rhs_T"].sum() - st.load(dmT, s=rhocp / 1e-6 * asm.field_at_qpoints(dmT, T)[0]).sum()
    assert stored == pytest.approx(src, rel=1e-9)
    assert src > 0.0                            # the beam out-heats the cooling


def test_quiescent_state_stays_put():
    """No flow, no evaporation, no laser, no surface tension or gravity, uniform T equal to its
    Dirichlet value: phi, T unchanged, u = 0, p = 0."""
    maps = _maps(4)
    z = maps[2].dof_coords()[:, 2]
    phi = np.tanh((0.5 - z) / 0.5)
    out = st.step(maps, _state(maps[0].n_dofs, T=1200.0, phi=phi), _params())
    assert np.abs(out["phi"] - phi).max() <= 1e-13
    assert np.abs(out["T"] - 1200.0).max() <= 1e-10
    assert np.abs(out["u"]).max() == 0.0 and np.abs(out["p"]).max() == 0.0


def test_update_form_of_the_heat_solve_equals_the_lifted_form():
    """T^n + A_T^-1 r (r: Dirichlet rows 0) is the lifted solution A_T^-1 rhs, with a Dirichlet face,
    convection and a non-uniform T^n."""
    import scipy.sparse.linalg as sla
    maps = _maps(4)
    X = maps[3].dof_coords()
    T = 900.0 + 400.0 * X[:, 0] * X[:, 2] + 50.0 * X[:, 1]
    phi = np.tanh((0.6 - X[:, 2]) / 0.3)
    u = np.stack([X[:, 1] - 0.5, 0.5 - X[:, 0], 0.2 + 0 * X[:, 2]])
    prm = _params(dt=0.05)
    A, rhs, r, _ = st.heat_system(maps, T, u, T, phi, prm)
    lifted = sla.spsolve(A.tocsc(), rhs)
    assert np.array_equal(lifted[maps[3].dirichlet], T[maps[3].dirichlet])
    assert np.abs(T + sla.spsolve(A.tocsc(), r) - lifted).max() <= 1e-12 * np.abs(T).max()
