"""One melt-pool time step (Algorithm algo:meltpooldg) on the GPU against the oracle, stage by
stage: the predictors bit for bit; the Gauss-point transport velocity and every load vector
componentwise (each recomputed by the oracle from the GPU's own inputs of that stage, so the
comparison is not blurred by the solver tolerance of earlier stages); every solve by the oracle's
true residual; the reinitialisation by the oracle's direct solves from the GPU's advected field;
and the whole step against the oracle's whole step.  Also the heat operator's Gauss-point
rho_cp and convection fields against the assembled matrix, and exact hydrostatics."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import mesh as omesh
from oracle import step as ost
from problems import componentwise_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TI = syn.TI64
U_FACES, T_FACES = 0b011111, 1 << 4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def _cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def test_heat_operator_with_gauss_point_rho_cp_and_velocity(ctx):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    n, dt = 5, 1e-3
    dm = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 2, T_FACES)
    nq = dm.n_cells * 27
    rc = 1.0 + 3.0 * syn.uniform_01(3, nq).reshape(dm.n_cells, 27)
    kq = syn.kq_field(nq, 4, 2.0).reshape(dm.n_cells, 27)
    bq = syn.uniform_pm1(5, 3 * nq).reshape(dm.n_cells, 27, 3)
    A = asm.assemble_scalar(dm, rc / dt, diff=kq, conv=rc[..., None] * bq)
    op = Operator(ctx, "heat", [DofMap(Mesh.uniform(ctx, n), 2, T_FACES)], rhocp=7.0, dt=dt, coef_mode=1)
    keep = [_cuda(kq.ravel()), _cuda(rc.ravel()), _cuda(bq.ravel())]
    for name, t in zip(("k_qpoint", "rhocp_qpoint", "beta_qpoint"), keep):
        op.set_field(name, t)
    u = syn.uniform_pm1(6, dm.n_dofs)
    for transpose in (False, True):
        M = A.T.tocsr() if transpose else A
        v = op.apply(_cuda(u), transpose=transpose).cpu().numpy()
        ok, worst = componentwise_ok(v, M @ u, abs(M) @ np.abs(u), 1e-12)
        assert ok, (transpose, worst)
        # double-float: the convective kernel with the value coefficient per Gauss point
        v = op.apply(_cuda(u), transpose=transpose, arith="df64").cpu().numpy()
        ok, worst = componentwise_ok(v, M @ u, abs(M) @ np.abs(u), 1e-12)
        assert ok, (transpose, "df64", worst)
        assert op.variant.endswith("/conv-T" if transpose else "/conv") and "/df64/" in op.variant, op.variant
        v32 = op.apply(_cuda(u).float(), transpose=transpose).cpu().double().numpy()
        ok, worst = componentwise_ok(v32, M @ u, abs(M) @ np.abs(u), 2e-5)
        assert ok, (transpose, worst)
    d = op.diagonal().cpu().numpy()
    free = ~dm.dirichlet
    assert np.abs(d[free] - A.diagonal()[free]).max() <= 1e-12 * np.abs(A.diagonal()).max()
    with pytest.raises(Exception):
        op.apply(_cuda(u).float(), arith="bf16")


@pytest.mark.parametrize("arith", ["f64", "df64"])
def test_defect_correction_on_the_convective_heat_operator(ctx, arith):
    """Mixed-precision defect correction on the nonsymmetric heat operator of the melt-pool step
    (rho_cp, k and the velocity per Gauss point): fp32 inner GMRES, outer residuals in fp64 or
    double-float; the true residual from the oracle's assembled matrix meets the tolerance."""
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    n, dt = 6, 1e-3
    dm = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), 2, T_FACES)
    nq = dm.n_cells * 27
    rc = 1.0 + 3.0 * syn.uniform_01(13, nq).reshape(dm.n_cells, 27)
    kq = syn.kq_field(nq, 14, 2.0).reshape(dm.n_cells, 27)
    bq = 20.0 * syn.uniform_pm1(15, 3 * nq).reshape(dm.n_cells, 27, 3)
    A = asm.assemble_scalar(dm, rc / dt, diff=kq, conv=rc[..., None] * bq)
    op = Operator(ctx, "heat", [DofMap(Mesh.uniform(ctx, n), 2, T_FACES)], rhocp=7.0, dt=dt, coef_mode=1)
    keep = [_cuda(kq.ravel()), _cuda(rc.ravel()), _cuda(bq.ravel())]
    for name, t in zip(("k_qpoint", "rhocp_qpoint", "beta_qpoint"), keep):
        op.set_field(name, t)
    b = syn.uniform_pm1(16, dm.n_dofs)
    b[dm.dirichlet] = 0.0
    x, info = op.solve(_cuda(b), solver="defect_correction", precond="jacobi", tol=1e-10, restart=30, maxit=20,
                       fp64_arith=arith)
    assert info["status"] == 0 and info["outer_iterations"] >= 2, info
    r = b - A @ x.cpu().numpy()
    assert np.linalg.norm(r) <= (1e-10 + 1e-13) * np.linalg.norm(b), (np.linalg.norm(r) / np.linalg.norm(b), info)
    with pytest.raises(Exception):
        op.solve(_cuda(b), solver="defect_correction", precond="chebyshev", tol=1e-10)


def _workload(n, **over):
    wl = syn.scaled(syn.MELTPOOL_STEP, n)
    p = dict(wl.params)
    p.update(over)
    ev = {k: syn.EVAPORATION[k] for k in ("p_amb", "h_v", "molar_mass", "t_boil", "sticking", "tanasawa")}
    prm = dict(dt=p["dt"], eps=wl.eps, rho_l=TI["rho_l"], rho_g=TI["rho_g"], mu_l=TI["mu_l"], mu_g=TI["mu_g"],
               rhocp_l=TI["rho_l"] * TI["cp_l"], rhocp_g=TI["rho_g"] * TI["cp_g"], k_l=TI["k_l"], k_g=TI["k_g"],
               evaporation=dict(model=p.get("model", "knight"), **ev), surface_tension=p["surface_tension"],
               gravity=p["gravity"], laser=p["laser"], reinit_steps=p["reinit_steps"], dtau=p["dtau_cells"] * wl.h,
               solid=p["solid"], darcy=p["darcy"], trace_correction=p["trace_correction"])
    return wl, prm


def _gpu_step(ctx, wl, prm, tol, flow_tol):
    from paper_2501_18781_gb300 import DofMap, MeltPoolStep, Mesh
    from paper_2501_18781_gb300 import _lib
    mesh = Mesh.uniform(ctx, wl.n, wl.lo, wl.hi)
    maps = [DofMap(mesh, 2, U_FACES), DofMap(mesh, 1, 0), DofMap(mesh, 2, 0), DofMap(mesh, 2, T_FACES)]
    ev = prm["evaporation"]
    flags = (_lib.MF_OSEEN_THREE_PHASE if prm["solid"] else 0) | (_lib.MF_OSEEN_DARCY if prm["darcy"] else 0) | \
        (_lib.MF_OSEEN_TRACE_CORRECTION if prm["trace_correction"] else 0)
    sol, dar = prm["solid"] or {}, prm["darcy"] or {}
    st = prm["surface_tension"]
    step = MeltPoolStep(
        ctx, maps,
        evaporation=dict(mass_flux=ev["model"], p_ambient=ev["p_amb"], latent_heat=ev["h_v"],
                         molar_mass=ev["molar_mass"], t_boil=ev["t_boil"], sticking=ev["sticking"],
                         tanasawa_coef=ev["tanasawa"], gas_constant=8.314),
        laser=prm["laser"], gravity=prm["gravity"], dt=prm["dt"], eps=prm["eps"], rho_l=prm["rho_l"],
        rho_g=prm["rho_g"], mu_l=prm["mu_l"], mu_g=prm["mu_g"], rhocp_l=prm["rhocp_l"], rhocp_g=prm["rhocp_g"],
        k_l=prm["k_l"], k_g=prm["k_g"], oseen_flags=flags, rho_s=sol.get("rho_s", 0.0), mu_s=sol.get("mu_s", 0.0),
        t_solidus=sol.get("t_solidus", dar.get("t_solidus", 0.0)),
        t_liquidus=sol.get("t_liquidus", dar.get("t_liquidus", 0.0)), darcy_c=dar.get("C", 0.0),
        darcy_b=dar.get("b", 1.0), alpha0=st["alpha0"], alpha1=st["alpha1"], t_alpha=st["t_alpha"],
        alpha_res=st["alpha_res"], reinit_steps=prm["reinit_steps"], dtau=prm["dtau"], tol=tol, flow_tol=flow_tol,
        maxit=5000)
    return step, maps


def _oracle_maps(wl):
    return [omesh.uniform_dofmap(wl.n, wl.lo, wl.hi, d, f) for d, f in ((2, U_FACES), (1, 0), (2, 0), (2, T_FACES))]


def _max_ok(v, ref, rtol):
    err = np.abs(v - ref).max()
    return err <= rtol * np.abs(ref).max(), err / max(np.abs(ref).max(), 1e-300)


def test_meltpool_step_stage_by_stage(ctx):
    tol, flow_tol = 1e-12, 1e-11
    wl, prm = _workload(5)
    maps = _oracle_maps(wl)
    dmu, dmp, dmphi, dmT = maps
    x = dmu.dof_coords()
    s = syn.meltpool_state(*x.T, wl.seed, wl.lo, wl.hi, wl.eps)
    step, _ = _gpu_step(ctx, wl, prm, tol, flow_tol)
    out, info = step.advance({k: _cuda(v.ravel()) for k, v in s.items()}, trace=True)
    assert info["status"] == 0, info
    g = {k: v.cpu().numpy() for k, v in out.items()}
    nu, nc = dmu.n_dofs, dmu.n_cells
    # 1. predictors, bit for bit
    us, Ts, phis = ost.predictors(s)
    assert np.array_equal(g["u_star"], us.ravel()) and np.array_equal(g["T_star"], Ts)
    assert np.array_equal(g["phi_star"], phis)
    # 2. advection: transport velocity and load from the same inputs, then the true residual
    A_adv, b_adv, uG = ost.advection_system(dmphi, s["phi"], us, Ts, phis, prm)
    ok, err = _max_ok(g["u_gamma"].reshape(nc, 27, 3), uG, 1e-12)
    assert ok, err
    M = asm.mass_matrix(dmphi)
    ok, worst = componentwise_ok(g["b_advection"], b_adv, abs(M) @ np.abs(s["phi"]) / prm["dt"], 1e-12)
    assert ok, worst
    phia = g["phi_advected"]
    assert np.linalg.norm(b_adv - A_adv @ phia) <= tol * (1 + 1e-3) * np.linalg.norm(b_adv)
    # 2. reinitialisation: the oracle's direct solves from the GPU's advected field
    phi_re, _ = ost.reinitialise(dmphi, phia, prm)
    ok, err = _max_ok(g["phi"], phi_re, 1e-10)
    assert ok, err
    # 3. heat: the update's right-hand side from the GPU's phi^(n+1), then the true residual
    A_T, rhs_T, r_T, A_all = ost.heat_system(maps, s["T"], us, Ts, g["phi"], prm)
    bound = abs(A_all) @ np.abs(s["T"]) + np.abs(r_T)
    ok, worst = componentwise_ok(g["r_heat"], r_T, bound, 1e-12)
    assert ok, worst
    assert np.array_equal(g["T"][dmT.dirichlet], s["T"][dmT.dirichlet])
    # the solve, in the update form it ran in, with the right-hand side it was given (r is a
    # difference of terms ~1e5 times larger at a 0.01 us step, so the two r agree only to the
    # rounding of those terms, as checked above); then T^(n+1) in the lifted form, where that
    # difference and storing T^n + delta in fp64 (up to 2^-52 |A_T| |T|) set the floor
    r_g = g["r_heat"]
    assert np.linalg.norm(r_g - A_T @ g["T_update"]) <= tol * (1 + 1e-3) * np.linalg.norm(r_g)
    floor = 2.0 ** -52 * np.linalg.norm(abs(A_T) @ np.abs(g["T"])) + np.linalg.norm(r_g - r_T)
    assert np.linalg.norm(rhs_T - A_T @ g["T"]) <= tol * (1 + 1e-3) * np.linalg.norm(r_g) + floor
    # 4. flow: the load from the GPU's phi^(n+1) and T^(n+1), then the true residual
    A_ns, b_ns = ost.flow_system(maps, s["u"], us, g["phi"], g["T"], prm)
    ok, worst = componentwise_ok(g["b_flow"], b_ns, np.abs(b_ns) + 1e-6 * np.abs(b_ns).max(), 1e-10)
    assert ok, worst
    xg = np.concatenate([g["u"].ravel(), g["p"]])
    assert np.linalg.norm(b_ns - A_ns @ xg) <= flow_tol * (1 + 1e-3) * np.linalg.norm(b_ns)
    # the whole step against the oracle's (direct solves throughout)
    ref = ost.step(maps, s, prm)
    for k in ("phi", "T"):
        ok, err = _max_ok(g[k], ref[k], 1e-8)
        assert ok, (k, err)
    ok, err = _max_ok(xg, np.concatenate([ref["u"].ravel(), ref["p"]]), 1e-6)
    assert ok, err
    assert info["advection_iterations"] > 0 and info["heat_iterations"] > 0 and info["flow_iterations"] > 0
    assert info["reinit_iterations"] >= prm["reinit_steps"]


def test_meltpool_step_tanasawa_without_laser_first_step(ctx):
    """Tanasawa mass flux, no laser, no three-phase/Darcy, x^(n-1) = x^n (first step): final fields
    against the oracle's whole step."""
    tol, flow_tol = 1e-12, 1e-11
    wl, prm = _workload(4, laser=None, solid=None, darcy=None, model="tanasawa", trace_correction=False)
    maps = _oracle_maps(wl)
    x = maps[0].dof_coords()
    s = syn.meltpool_state(*x.T, wl.seed, wl.lo, wl.hi, wl.eps)
    for k in ("u", "T", "phi"):
        s[k + "_prev"] = s[k]
    step, _ = _gpu_step(ctx, wl, prm, tol, flow_tol)
    out, info = step.advance({k: _cuda(v.ravel()) for k, v in s.items()})
    assert info["status"] == 0, info
    ref = ost.step(maps, s, prm)
    for k in ("phi", "T"):
        ok, err = _max_ok(out[k].cpu().numpy(), ref[k], 1e-8)
        assert ok, (k, err)
    ok, err = _max_ok(np.concatenate([out["u"].cpu().numpy().ravel(), out["p"].cpu().numpy()]),
                      np.concatenate([ref["u"].ravel(), ref["p"]]), 1e-6)
    assert ok, err


def test_meltpool_step_hydrostatics(ctx):
    """Liquid everywhere, at rest, gravity only (no evaporation, no laser, no surface tension): the
    discrete solution is u = 0, p = rho |g| (z_top - z) exactly, and T, phi do not move.

    The bars on u and p are derived, not fitted: the oracle checks that the hydrostatic state x*
    solves its assembled flow system K0 x* = b0 (phi = 1, T = 800) to rounding.  The GPU's flow
    stage sees the phi and T its own level-set and heat solves returned (equal to 1 and 800 up to
    those solves' tolerance), so the oracle assembles that system, K x = b - r, from the GPU's
    outputs, and checks the true residual |r| <= tol |b| (tol = 1e-12, the flow solve's tolerance).
    Then x - x* = K^-1 (b - K x* - r), so |x_i - x*_i| <= |row i of K^-1|_2 (|b - K x*| + tol |b|):
    the bound is formed from the dense inverse of the 2312 x 2312 system (|b - K x*| vanishes
    when phi and T came back exact).  (At the 0.01 us step sigma rho h^2 / mu = 2.6e6 makes K
    mass-dominated and its pressure Schur complement a scaled Laplacian; the bound comes to about
    5e-4 rho |g| L for p and 1.2e-3 |g| dt for u.)"""
    wl, prm = _workload(4, laser=None, solid=None, darcy=None, trace_correction=False, reinit_steps=0)
    prm["evaporation"].update(model="tanasawa", tanasawa=0.0, p_amb=0.0)
    prm["surface_tension"] = dict(alpha0=0.0, alpha1=0.0, t_alpha=0.0, alpha_res=0.0)
    maps = _oracle_maps(wl)
    nu = maps[0].n_dofs
    s = dict(u=np.zeros((3, nu)), u_prev=np.zeros((3, nu)), T=np.full(nu, 800.0), T_prev=np.full(nu, 800.0),
             phi=np.ones(nu), phi_prev=np.ones(nu))
    step, _ = _gpu_step(ctx, wl, prm, 1e-12, 1e-12)
    out, info = step.advance({k: _cuda(v.ravel()) for k, v in s.items()})
    assert info["status"] == 0, info
    zp = maps[1].dof_coords()[:, 2]
    A0, b0 = ost.flow_system(maps, s["u"], s["u"], s["phi"], s["T"], prm)
    xs = np.concatenate([np.zeros(3 * nu), TI["rho_l"] * 9.81 * (wl.hi[2] - zp)])
    assert np.linalg.norm(b0 - A0 @ xs) <= 1e-13 * np.linalg.norm(b0)            # x* is the discrete solution
    phi_g, T_g = out["phi"].cpu().numpy(), out["T"].cpu().numpy()
    A_ns, b_ns = ost.flow_system(maps, s["u"], s["u"], phi_g, T_g, prm)         # the system the GPU solved
    x = np.concatenate([out["u"].cpu().numpy().ravel(), out["p"].cpu().numpy()])
    tol = 1e-12 * (1 + 1e-3)
    assert np.linalg.norm(b_ns - A_ns @ x) <= tol * np.linalg.norm(b_ns)          # the GPU's true residual
    rs = np.linalg.norm(b_ns - A_ns @ xs)
    bound = np.linalg.norm(np.linalg.inv(A_ns.toarray()), axis=1) * (rs + tol * np.linalg.norm(b_ns))
    assert np.all(np.abs(x - xs) <= bound + 2.0 ** -52 * np.abs(xs)), np.max(np.abs(x - xs) / bound)
    assert np.array_equal(out["T"].cpu().numpy(), s["T"]) or np.abs(out["T"].cpu().numpy() - 800.0).max() <= 1e-9
    assert np.abs(out["phi"].cpu().numpy() - 1.0).max() <= 1e-12


def test_meltpool_create_rejects_inconsistent_maps(ctx):
    from paper_2501_18781_gb300 import DofMap, MeltPoolStep, Mesh
    from paper_2501_18781_gb300._lib import MFError
    wl, prm = _workload(3)
    mesh = Mesh.uniform(ctx, 3, wl.lo, wl.hi)
    ev = dict(mass_flux="knight", p_ambient=1e5, latent_heat=TI["h_v"], molar_mass=TI["molar_mass"], t_boil=3133.0,
              sticking=1.0)
    good = dict(dt=1e-6, eps=wl.eps, rho_l=1.0, rho_g=1.0e-3, mu_l=1.0, mu_g=1e-2, rhocp_l=1.0, rhocp_g=1.0, k_l=1.0,
                k_g=1.0, tol=1e-10, flow_tol=1e-10)
    bad_maps = [DofMap(mesh, 2, U_FACES), DofMap(mesh, 1, 0), DofMap(mesh, 2, T_FACES), DofMap(mesh, 2, T_FACES)]
    with pytest.raises(MFError):
        MeltPoolStep(ctx, bad_maps, evaporation=ev, **good)
    maps = [DofMap(mesh, 2, U_FACES), DofMap(mesh, 1, 0), DofMap(mesh, 2, 0), DofMap(mesh, 2, T_FACES)]
    with pytest.raises(MFError):
        MeltPoolStep(ctx, maps, evaporation=ev, **dict(good, dt=0.0))
    with pytest.raises(MFError):
        MeltPoolStep(ctx, maps, evaporation=ev, **dict(good, reinit_steps=2, dtau=0.0))
