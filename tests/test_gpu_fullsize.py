"""Parity at the benchmark sizes, in the launch configuration bench.py times: sampled output rows
against the oracle's patch rows (uniform meshes), the whole vector where the oracle finishes in
seconds (16^3 Helmholtz), and size-independent properties on the 12.3M-DoF octree."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import patch
from problems import DIRICHLET_BOTTOM, OSEEN_FACES, componentwise_ok

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def _lattice_sample(n, count, seed, dirichlet):
    """Free Q2 DoFs: random ones plus the corners/edges/faces of the lattice (ragged boundary rows)."""
    L = 2 * n + 1
    rng = np.random.default_rng(seed)
    pick = list(rng.choice(L ** 3, count, replace=False))
    for x in (0, 1, L // 2, L - 2, L - 1):
        for y in (0, 1, L - 1):
            for z in (0, 1, L - 2, L - 1):
                pick.append(x + L * (y + L * z))
    pick = np.unique(np.array(pick))
    return pick[~dirichlet[pick]], pick[dirichlet[pick]]


def test_oseen_64_apply_sampled_rows(ctx):
    import bench
    n = 64
    wl = syn.scaled(syn.OSEEN_INTERFACE, n)
    p = wl.params
    op, mu, mp, mesh = bench.build_oseen(ctx, n)   # the benchmark operator (autotuned kernel)
    x = mu.coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    dirichlet = mu.export(cell_map=False, constraints=False, coords=False)["dirichlet"].astype(bool)
    nu, npr = mu.n_dofs, mp.n_dofs
    u = syn.uniform_pm1(11, op.n)
    sigma = 1.0 / (p["dt_cfl"] * wl.h)
    args = (sigma, p["rho_l"], p["rho_g"], p["mu_l"], p["mu_g"])
    build = lambda du, dp, nod: asm.oseen_matrix(du, dp, nod["phi"], nod["beta"], *args)
    free, dir_rows = _lattice_sample(n, 40, 5, dirichlet)
    rows = np.concatenate([free, nu + free[::3], 2 * nu + free[::3],
                           3 * nu + np.random.default_rng(6).choice(npr, 25, replace=False), [3 * nu, op.n - 1]])
    nodal = {"phi": phi, "beta": beta}
    uu = u.astype(np.float32).astype(np.float64)       # exact in every arithmetic tested
    ref = patch.oseen_rows(n, wl.lo, wl.hi, rows, build, nodal, uu, dirichlet)
    bound = patch.oseen_rows(n, wl.lo, wl.hi, rows, build, nodal, uu, dirichlet, absolute=True)
    for arith, rtol in (("f64", 1e-12), ("df64", 1e-12), ("f32", 5e-5)):
        t = torch.tensor(uu, device="cuda", dtype=torch.float32 if arith == "f32" else torch.float64)
        v = op.apply(t, arith="df64" if arith == "df64" else None).cpu().double().numpy()
        ok, worst = componentwise_ok(v[rows], ref, bound, rtol)
        assert ok, (arith, worst)
        for c in range(3):   # Dirichlet rows are identities
            assert np.all(v[c * nu + dir_rows] == uu[c * nu + dir_rows].astype(v.dtype))


def test_oseen_64_fgmres_true_residual(ctx):
    """The 64^3 Oseen solve as bench.py runs it (FGMRES(50), block-triangular preconditioner with
    the assembled fp16 Schur stencil, the call replayed as a CUDA graph): the residual b - A x,
    recomputed with the fp64 apply that the sampled-row test pins against the oracle and reduced by
    torch, is at most 1e-10 |b|, the reported residual agrees with it, and the Dirichlet velocity
    rows of x equal b's (zero here) exactly."""
    import bench
    op, mu, mp, mesh = bench.build_oseen(ctx, 64)
    b = syn.uniform_pm1(1, op.n)
    d = mu.export(cell_map=False, constraints=False, coords=False)["dirichlet"].astype(bool)
    mask = np.concatenate([np.tile(d, 3), np.zeros(mp.n_dofs, bool)])
    b[mask] = 0
    bt = torch.tensor(b, device="cuda")
    for arith in ("f64", "df64"):   # outer applies on the fp64 pipes or in double-float
        x, info = op.solve(bt, solver="gmres", precond="block_triangular", restart=50, maxit=400, tol=1e-10,
                           use_graph=True, fp64_arith=arith)
        assert info["status"] == 0, (arith, info)
        r = bt - op.apply(x)
        rel = (torch.linalg.vector_norm(r) / torch.linalg.vector_norm(bt)).item()
        assert rel <= 1e-10 * (1 + 1e-3), (arith, rel, info)
        # the reported residual is ||b - A' x|| / ||b|| with A' the apply of the solve's arithmetic: by the
        # triangle inequality it lies within ||A' x - A x|| / ||b|| of the recomputed one
        delta = _apply_gap(op, bt, x, arith)
        assert delta <= 1e-11, (arith, delta)   # a tenth of the tolerance: the solve saw its residual
        assert abs(rel - info["rel_residual"]) <= 1e-3 * max(rel, info["rel_residual"]) + delta, (arith, rel, info)
        assert np.all(x.cpu().numpy()[mask] == 0.0)
        assert 0 < info["inner_steps"] <= 30 * info["iterations"]


def _heat_case(n, wl, kq=False, beta=False):
    p = wl.params
    from oracle import mesh as omesh
    dm = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2, DIRICHLET_BOTTOM)
    x = dm.dof_coords()
    T_prev = syn.heat_initial_temperature(*x.T, p["laser"]["radius"], wl.hi[2])
    b = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi)) if beta else None
    k = syn.kq_field(dm.n_cells * 27, wl.seed, p["k0"]).reshape(dm.n_cells, 27) if kq else None
    return dm, T_prev, b, k


def _heat_operator(ctx, n, wl, T_prev, b, k, coef_mode=1):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    p = wl.params
    m = DofMap(Mesh.uniform(ctx, n, wl.lo, wl.hi), 2, DIRICHLET_BOTTOM)
    op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"], coef_mode=coef_mode)
    keep = [torch.tensor(T_prev, device="cuda")]
    op.set_field("t_prev", keep[0])
    if b is not None:
        keep.append(torch.tensor(b.ravel(), device="cuda"))
        op.set_field("beta", keep[-1])
    if k is not None:
        keep.append(torch.tensor(k.ravel(), device="cuda"))
        op.set_field("k_qpoint", keep[-1])
    op._keep = keep
    return op


def test_heat_128_apply_sampled_rows(ctx):
    n = 128
    wl = syn.scaled(syn.HEAT_LASER, n)
    p = wl.params
    dm, T_prev, _, _ = _heat_case(n, wl)
    op = _heat_operator(ctx, n, wl, T_prev, None, None, coef_mode=1)   # as in the heat-step benchmark
    free, dir_rows = _lattice_sample(n, 60, 7, dm.dirichlet)
    build = lambda d, nod, cw: asm.heat_matrix(d, p["rhocp"], p["dt"], k0=p["k0"], t_boil=p["t_boil"], T_prev=nod["T"])
    uu = syn.uniform_pm1(12, dm.n_dofs).astype(np.float32).astype(np.float64)
    ref = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"T": T_prev}, uu, dm.dirichlet)
    bound = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"T": T_prev}, uu, dm.dirichlet, absolute=True)
    for arith, rtol in (("f64", 1e-12), ("df64", 1e-12), ("f32", 2e-5)):
        t = torch.tensor(uu, device="cuda", dtype=torch.float32 if arith == "f32" else torch.float64)
        v = op.apply(t, arith="df64" if arith == "df64" else None).cpu().double().numpy()
        ok, worst = componentwise_ok(v[free], ref, bound, rtol)
        assert ok, (arith, worst)
        assert np.all(v[dir_rows] == uu[dir_rows].astype(v.dtype))


def test_heat_adjoint_64_sampled_rows(ctx):
    n = 64
    wl = syn.scaled(syn.HEAT_ADJOINT, n)
    p = wl.params
    dm, T_prev, b, k = _heat_case(n, wl, kq=True, beta=True)
    op = _heat_operator(ctx, n, wl, T_prev, b, k)
    free, _ = _lattice_sample(n, 60, 8, dm.dirichlet)
    build = lambda d, nod, cw: asm.heat_matrix(d, p["rhocp"], p["dt"], kq=cw["kq"], beta=nod["beta"])
    u = syn.uniform_pm1(13, dm.n_dofs)
    ut = torch.tensor(u, device="cuda")
    for tr in (True, False):   # the adjoint rows, then the forward rows; fp64 pipes and double-float
        kw = dict(cellwise={"kq": k}, transpose=tr)
        ref = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"beta": b}, u, dm.dirichlet, **kw)
        bound = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"beta": b}, u, dm.dirichlet, absolute=True, **kw)
        for arith in (None, "df64"):
            v = op.apply(ut, transpose=tr, arith=arith).cpu().numpy()
            ok, worst = componentwise_ok(v[free], ref, bound, 1e-12)
            assert ok, (tr, arith, worst)
            if arith == "df64":
                assert op.variant.endswith("/conv-T" if tr else "/conv"), op.variant


def test_helmholtz_16_whole_vector(ctx):
    from problems import helmholtz
    P = helmholtz(16, ctx)
    u = syn.uniform_pm1(1, P["n"])
    v = P["op"].apply(torch.tensor(u, device="cuda")).cpu().numpy()
    ok, worst = componentwise_ok(v, P["A"] @ u, abs(P["A"]) @ np.abs(u), 1e-12)
    assert ok, worst


def test_reinit_octree_full_size_properties(ctx):
    """32^3 + 3 levels (12.3M DoFs), 8 right-hand sides in one launch: symmetry, the constant vector
    (the n-n diffusion annihilates it, so sum(A 1) = |Omega| / dtau through the partition of unity
    of the constrained space), batched = one-at-a-time, fp32 close to fp64."""
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    wl = syn.REINIT_OCTREE
    d = lambda X, Y, Z: syn.deformed_sphere_distance(X, Y, Z, wl.seed)
    leaves = syn.refine_band_leaves(wl.n, wl.levels, d, wl.eps)
    m = DofMap(Mesh.octree(ctx, wl.n, wl.levels, leaves), 2, 0)
    x = m.coords()
    phi = syn.initial_level_set(syn.deformed_sphere_distance(*x.T, wl.seed), wl.eps)
    dtau = 0.5 / (wl.n << wl.levels)
    op = Operator(ctx, "reinit", [m], eps=wl.eps, dtau=dtau)
    ph = torch.tensor(phi, device="cuda")
    op.set_field("phi", ph)
    N, R = m.n_dofs, wl.nrhs
    assert N > 10_000_000 and m.n_constraints > 0
    U = torch.tensor(np.concatenate([syn.uniform_pm1(s, N) for s in range(1, R + 1)]), device="cuda")
    V = op.apply(U, nrhs=R)
    for r in (0, R - 1):
        single = op.apply(U[r * N:(r + 1) * N].contiguous())
        assert torch.allclose(single, V[r * N:(r + 1) * N], rtol=1e-13, atol=1e-13 * single.abs().max().item())
    a = (U[:N] * V[N:2 * N]).sum().item()
    b = (U[N:2 * N] * V[:N]).sum().item()
    assert abs(a - b) <= 1e-12 * (U[:N].abs() * V[N:2 * N].abs()).sum().item()
    one = op.apply(torch.ones(N, dtype=torch.float64, device="cuda"))
    assert one.sum().item() == pytest.approx(1.0 / dtau, rel=1e-12)
    V32 = op.apply(U.float(), nrhs=R).double()
    assert ((V32 - V).norm() / V.norm()).item() < 5e-6


def test_meltpool_step_64_properties(ctx):
    """The 64^3 melt-pool step as bench.py runs it (11.0M unknowns): every solve reaches 1e-10; the
    Dirichlet temperatures keep T^n and the wall velocities stay 0, both exactly (identity rows and
    zero right-hand sides); the reinitialisation conserves int phi (sum_i F_i = 0 for the
    compressive flux, N_n 1 = 0 for the diffusion) up to the CG residual, and keeps phi bounded; the
    temperature moves by a fraction of a kelvin at 0.01 us."""
    import bench
    import torch
    from paper_2501_18781_gb300 import Operator
    wl, maps, state, step = bench.build_meltpool_step(ctx, 64)
    out, info = step.advance(state, trace=True)
    assert info["status"] == 0, info
    for k in ("advection", "reinit", "heat", "flow"):
        assert info[k + "_residual"] <= 1e-10 * (1 + 1e-3), (k, info)
    dT = maps[3].export(cell_map=False, constraints=False, coords=False)["dirichlet"]
    du = maps[0].export(cell_map=False, constraints=False, coords=False)["dirichlet"]
    T, Tn = out["T"].cpu().numpy(), state["T"].cpu().numpy()
    assert dT.any() and np.array_equal(T[dT], Tn[dT])
    u = out["u"].cpu().numpy()
    assert du.any() and np.all(u[:, du] == 0.0)
    assert np.isfinite(T).all() and np.isfinite(u).all() and np.isfinite(out["p"].cpu().numpy()).all()
    assert np.abs(T - Tn).max() < 1.0
    # int phi_h = sum_i phi_i int N_i, with int N_i = (M 1)_i from a pure mass operator
    mass = Operator(ctx, "helmholtz", [maps[2]], mass_coef=1.0, a_liquid=0.0, a_gas=0.0)
    mass.set_field("phi", out["phi"])
    w = mass.apply(torch.ones(maps[2].n_dofs, dtype=torch.float64, device="cuda"))
    i_adv, i_new = (w * out["phi_advected"]).sum().item(), (w * out["phi"]).sum().item()
    assert abs(i_new - i_adv) <= 1e-8 * (w * out["phi_advected"].abs()).sum().item()
    assert out["phi"].abs().max().item() <= 1.05


@pytest.mark.parametrize("k,n", [(3, 64), (4, 48)])
def test_qk_bench_size_sampled_rows(ctx, k, n):
    """Q3 on 64^3 and Q4 on 48^3 cells (7,189,057 DoFs each, as bench.py builds them): sampled rows
    against the oracle's degree-k patch rows, fp64 1e-12, fp32 5e-5, and Q3 on the tensor cores 5e-5."""
    import torch
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    m = DofMap(Mesh.uniform(ctx, n), k, 0)
    eps = 1.0 / (2 * n)
    phi = syn.initial_level_set(syn.sphere_distance(*m.coords().T), eps)
    op = Operator(ctx, "helmholtz", [m], mass_coef=1.0, a_liquid=1000.0, a_gas=1.0, eps=eps)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    L = k * n + 1
    rng = np.random.default_rng(20 + k)
    rows = list(rng.choice(m.n_dofs, 50, replace=False))
    for x in (0, 1, L // 2, L - 2, L - 1):
        for y in (0, k, L - 1):
            for z in (0, 1, L - 1):
                rows.append(x + L * (y + L * z))
    rows = np.unique(np.array(rows))
    uu = syn.uniform_pm1(30 + k, m.n_dofs).astype(np.float32).astype(np.float64)
    build = lambda d, nod, cw: asm.helmholtz_matrix(d, nod["phi"], 1.0, 1000.0, 1.0, "tanh", eps)
    none = np.zeros(m.n_dofs, bool)
    ref = patch.scalar_rows(n, (0, 0, 0), (1, 1, 1), rows, build, {"phi": phi}, uu, none, degree=k)
    bound = patch.scalar_rows(n, (0, 0, 0), (1, 1, 1), rows, build, {"phi": phi}, uu, none, degree=k, absolute=True)
    cases = [("f64", torch.float64, None, 1e-12), ("f32", torch.float32, None, 5e-5)]
    if k == 3:
        cases.append(("tc", torch.float32, "tc", 5e-5))
    for name, dt, arith, rtol in cases:
        v = op.apply(torch.tensor(uu, device="cuda", dtype=dt), arith=arith).cpu().double().numpy()
        ok, worst = componentwise_ok(v[rows], ref, bound, rtol)
        assert ok, (name, worst)


def _apply_gap(op, b, x, arith):
    """||A' x - A x|| / ||b|| for A' the fp64-accurate apply in ``arith`` ("df64" or the fp64 pipes) and A
    the fp64 apply: the most by which a residual the solver reports from A' can differ from the one
    recomputed from A.  Both applies are pinned componentwise to 1e-12 (|A| |x|)_i, and ||A| |x|| / ||b||
    is large for the Oseen system, so the gap is held to a tenth of the solve tolerance: then the
    residual the solver stopped on is the true one to 10 %."""
    if arith != "df64":
        return 0.0
    d = op.apply(x, arith="df64") - op.apply(x)
    return (torch.linalg.vector_norm(d) / torch.linalg.vector_norm(b)).item()


def _true_residual(op, b, x, nrhs=1):
    """Per right-hand side ||b - A x|| / ||b|| with A the fp64 apply that the sampled-row tests pin
    against the oracle, reduced by torch."""
    r = (b - op.apply(x, nrhs=nrhs)).view(nrhs, -1)
    return (torch.linalg.vector_norm(r, dim=1) / torch.linalg.vector_norm(b.view(nrhs, -1), dim=1)).cpu().numpy()


def test_heat_128_step_solves_true_residual(ctx):
    """The 128^3 heat-step solves exactly as bench.py times them (laser load plus (rho c_p/dt) M theta^n
    as right-hand side; fp64 CG with Chebyshev(4) and fp32-inner defect correction, graph-replayed):
    the residual recomputed with the pinned fp64 apply is at most 1e-10 |b|, agrees with the reported
    one, and the Dirichlet rows of x are exactly 0.  Also the seeded uniform right-hand side."""
    import bench
    op, m, T_prev = bench.build_heat(ctx, 128)
    d = torch.tensor(m.export(cell_map=False, constraints=False, coords=False)["dirichlet"], device="cuda")
    b = bench.heat_step_rhs(ctx, m, T_prev, 128)
    assert torch.all(b[d] == 0) and b.abs().max().item() > 0
    br = torch.tensor(syn.uniform_pm1(1, m.n_dofs), device="cuda")
    br[d] = 0
    for rhs in (b, br):
        for name, kw in bench.HEAT_SOLVERS.items():
            x, info = op.solve(rhs, tol=1e-10, use_graph=True, **kw)
            assert info["status"] == 0, (name, info)
            rel = _true_residual(op, rhs, x)[0]
            assert rel <= 1e-10 * (1 + 1e-3), (name, rel, info)
            delta = _apply_gap(op, rhs, x, kw.get("fp64_arith"))
            assert delta <= 1e-11, (name, delta)   # a tenth of the tolerance
            assert abs(rel - info["rel_residual"]) <= 1e-2 * max(rel, info["rel_residual"]) + delta, (name, rel, info)
            assert torch.all(x[d] == 0)


def test_heat_128_laser_rhs_sampled_rows(ctx):
    """The heat-step right-hand side the bench solves, checked at sampled rows against the oracle:
    (rho c_p / dt) (M theta^n)_i from the patch rows of the oracle's mass form plus the oracle's laser
    load (its top-face rows, computed on the 2 x 2 x 2-cell patch with the same Gauss face rule)."""
    import bench
    from oracle import mesh as omesh
    n = 128
    wl = syn.scaled(syn.HEAT_LASER, n)
    p = wl.params
    op, m, T_prev = bench.build_heat(ctx, n, autotune=False)
    b = bench.heat_step_rhs(ctx, m, T_prev, n).cpu().numpy()
    dirichlet = m.export(cell_map=False, constraints=False, coords=False)["dirichlet"].astype(bool)
    theta = T_prev.cpu().numpy() - p["t_ref"]
    free, _ = _lattice_sample(n, 40, 9, dirichlet)
    L = 2 * n + 1
    top = free[free // (L * L) >= L - 2]
    rng = np.random.default_rng(3)
    rows = np.unique(np.concatenate([free, top, L * L * (L - 1) + rng.choice(L * L, 30, replace=False)]))
    rows = rows[~dirichlet[rows]]
    mass = lambda d, nod, cw: asm.assemble_scalar(d, np.full((d.n_cells, 27), p["rhocp"] / p["dt"]))
    ref = patch.scalar_rows(n, wl.lo, wl.hi, rows, mass, {}, theta, dirichlet)
    bound = patch.scalar_rows(n, wl.lo, wl.hi, rows, mass, {}, theta, dirichlet, absolute=True)
    lz = p["laser"]
    # the laser load of a row from the top cells of its patch (only top-face rows are nonzero)
    for s, r in enumerate(rows):
        coord = (r % L, (r // L) % L, r // (L * L))
        if coord[2] != L - 1:
            continue
        c0 = [patch._first_cell(c, 2, n) for c in coord]
        dm, idx = patch._patch(n, wl.lo, wl.hi, c0, 2)
        f = asm.laser_rhs(dm, lz["power"], lz["radius"], lz["x0"], lz["y0"], lz["absorptivity"])
        loc = int(np.nonzero(idx == r)[0][0])
        ref[s] += f[loc]
        bound[s] += abs(f[loc])
    ok, worst = componentwise_ok(b[rows], ref, bound, 1e-12)
    assert ok, worst


def test_reinit_octree_8rhs_mixed_solve_true_residual(ctx):
    """The 8-right-hand-side mixed-precision solve of the 12.3M-DoF octree as bench.py times it
    (fp32-inner defect correction, Chebyshev, graph-replayed): every column's residual, recomputed with
    the fp64 batched apply and reduced by torch, is at most 1e-10 of its right-hand side."""
    import bench
    op, m = bench.build_reinit_octree(ctx)
    R = syn.REINIT_OCTREE.nrhs
    B = torch.tensor(np.concatenate([syn.uniform_pm1(s, m.n_dofs) for s in range(1, R + 1)]), device="cuda")
    X, info = op.solve(B, nrhs=R, solver="defect_correction", precond="chebyshev", tol=1e-10, use_graph=True)
    assert info["status"] == 0, info
    rel = _true_residual(op, B, X, nrhs=R)
    assert np.all(rel <= 1e-10 * (1 + 1e-3)), rel


def test_heat_adjoint_64_gradients_match_central_differences(ctx):
    """The gradient workload at its own size (Q2 on 64^3, 2,146,689 DoFs, convection and a
    per-Gauss-point k_q, the 200 W / 50 um beam, the 100 um objective box): the adjoint gradients with
    respect to the four laser parameters and to the largest-magnitude k_q entries agree with central
    differences of the objective at step 1e-6 (relative to the parameter) to 1e-6."""
    import bench
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    wl = syn.HEAT_ADJOINT
    p = wl.params
    m = DofMap(Mesh.uniform(ctx, wl.n, wl.lo, wl.hi), 2, DIRICHLET_BOTTOM)
    x = m.coords()
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    kq = syn.kq_field(m.n_cells * 27, wl.seed, p["k0"])
    op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"])
    bt = torch.tensor(beta.ravel(), device="cuda")
    op.set_field("beta", bt)
    op.set_field("k_qpoint", torch.tensor(kq, device="cuda"))
    lz = p["laser"]
    th_prev = syn.heat_initial_temperature(*x.T, lz["radius"], wl.hi[2]) - p["t_ref"]
    target = syn.heat_target_temperature(*x.T, wl.hi[2], wl.seed + 4) - p["t_ref"]
    tp, tt = torch.tensor(th_prev, device="cuda"), torch.tensor(target, device="cuda")
    kw = dict(solver="gmres", precond="jacobi", tol=1e-13, restart=50)
    names = ["power", "radius", "x0", "y0"]
    lzl = [lz[k] for k in names] + [lz["absorptivity"]]
    box = (p["box_half"], p["box_depth"])
    J0, g, gk, _, _ = op.heat_step_gradient(lzl, tp, tt, *box, **kw)
    assert J0 > 0
    for i, k in enumerate(names):
        step = p["fd_step"] * (abs(lzl[i]) if k in ("power", "radius") else lz["radius"])
        a, b = list(lzl), list(lzl)
        a[i] += step
        b[i] -= step
        Ja = op.heat_step_gradient(a, tp, tt, *box, with_kq=False, **kw)[0]
        Jb = op.heat_step_gradient(b, tp, tt, *box, with_kq=False, **kw)[0]
        fd = (Ja - Jb) / (2 * step)
        assert abs(g[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * max(abs(v) for v in g)), (k, g[i], fd)
    gk = gk.cpu().numpy()
    for flat in np.argsort(-np.abs(gk))[:3]:
        hh = p["fd_step"] * kq[flat]
        vals = []
        for sgn in (1, -1):
            k2 = kq.copy()
            k2[flat] += sgn * hh
            op.set_field("k_qpoint", torch.tensor(k2, device="cuda"))
            vals.append(op.heat_step_gradient(lzl, tp, tt, *box, with_kq=False, **kw)[0])
        fd = (vals[0] - vals[1]) / (2 * hh)
        assert abs(gk[flat] - fd) <= 1e-6 * abs(fd), (flat, gk[flat], fd)


def test_reinit_octree_full_size_maps_and_sampled_rows(ctx):
    """The 12.3M-DoF octree of the batched reinitialisation (base 32^3 + 3 levels) against the
    oracle's own construction from the same leaf list: the integer cell map, the constraint rows and
    the DoF coordinates bit for bit, then rows of the 8-right-hand-side launch as bench.py times it
    (fp64 1e-12, fp32 5e-5 componentwise) at DoFs on leaves of every level and at the masters of
    every class of hanging node (edge, face, chained), each row of C^T A C formed from the cells
    around it by the oracle's full-quadrature element matrices.

    Rows are compared where the operator is determined by phi to better than the bar: every Gauss
    point of the row's cells has h |grad phi_h| >= 1e-4, or below 1e-14 (n = 0 on both sides of the
    1e-12 / h cut-off).  In the saturated tail of tanh(d / 2 eps) in between, n = grad phi_h / |grad
    phi_h| is set by the rounding of phi: perturbing phi by one ulp moves the oracle's own rows there
    by up to 3.6e-6 of |A||u|, so two correct fp64 evaluations differ by that much; those rows are
    covered by the size-independent properties of test_reinit_octree_full_size_properties."""
    import dataclasses
    import bench
    from oracle import mesh as omesh
    wl = syn.REINIT_OCTREE
    eps = 2.0 / (wl.n << wl.levels)
    dtau = 0.5 / (wl.n << wl.levels)
    d = lambda X, Y, Z: syn.deformed_sphere_distance(X, Y, Z, wl.seed)
    leaves = syn.refine_band_leaves(wl.n, wl.levels, d, eps)
    dm = omesh.octree_dofmap(leaves, wl.n, wl.levels)
    op, m = bench.build_reinit_octree(ctx)
    # integer maps, bit for bit
    e = m.export()
    cm, rp, cols, w = dm.export()
    assert m.n_dofs == dm.n_dofs and m.n_cells == dm.n_cells
    assert np.array_equal(e["cell_map"], cm) and np.array_equal(e["con_rowptr"], rp)
    assert np.array_equal(e["con_cols"], cols) and np.array_equal(e["con_w"], w)
    x = dm.dof_coords()
    assert np.array_equal(e["coords"], x)
    del e, cm
    phi = syn.initial_level_set(syn.deformed_sphere_distance(*x.T, wl.seed), eps)
    def sub_map(cells):
        return dataclasses.replace(dm, cell_points=dm.cell_points[cells], cell_h=dm.cell_h[cells],
                                   cell_origin=dm.cell_origin[cells], cell_level=dm.cell_level[cells])

    def emat(cells):
        sub = sub_map(cells)
        mq, D = asm.reinit_coefficients(sub, phi, eps, dtau)
        return asm.scalar_element_matrices(sub, mq, diff_tensor=D)

    import scipy.sparse as sp
    nc, nb = dm.cell_points.shape
    incid = sp.csr_matrix((np.ones(nc * nb), (dm.cell_points.ravel(), np.repeat(np.arange(nc), nb))),
                          shape=(dm.points.shape[0], nc))
    CT = dm.C.T.tocsr()

    def determined(i):
        cells = np.unique(incid[CT.indices[CT.indptr[i]:CT.indptr[i + 1]]].indices)
        sub = sub_map(cells)
        _, g = asm.field_at_qpoints(sub, phi)
        hg = np.linalg.norm(g, axis=-1) * sub.cell_h[:, None]
        return bool(np.all((hg >= 1e-4) | (hg < 1e-14)))

    # sampled rows: DoFs on leaves of each level, masters of each class of hanging node
    rng = np.random.default_rng(17)
    rows = []
    for lev in range(wl.levels + 1):
        cells = np.nonzero(dm.cell_level == lev)[0]
        pts = dm.cell_points[rng.choice(cells, 40)].ravel()
        free = dm.free_of_point[pts]
        cand = [i for i in rng.choice(free[free >= 0], 60, replace=False) if determined(i)]
        assert len(cand) >= 4, lev
        rows.append(np.array(cand[:8]))
    hang = np.nonzero(dm.hang_of_point >= 0)[0]
    Ch = dm.C[hang].tocsr()
    nm = np.diff(Ch.indptr)
    for cls in np.unique(nm):
        sel = np.nonzero(nm == cls)[0]
        for t in rng.choice(sel, min(3, sel.size), replace=False):
            rows.append(np.array([i for i in Ch.indices[Ch.indptr[t]:Ch.indptr[t + 1]][:3] if determined(i)], dtype=np.int64))
    rows = np.unique(np.concatenate(rows))

    R = wl.nrhs
    U = np.concatenate([syn.uniform_pm1(s, dm.n_dofs) for s in range(1, R + 1)])
    U = U.astype(np.float32).astype(np.float64)         # exact in both arithmetics
    refs = {}
    for r in (0, R - 1):
        u = U[r * dm.n_dofs:(r + 1) * dm.n_dofs]
        refs[r] = (patch.constrained_rows(dm, rows, emat, u), patch.constrained_rows(dm, rows, emat, u, absolute=True))
    for arith, rtol in (("f64", 1e-12), ("df64", 1e-12), ("f32", 5e-5)):
        t = torch.tensor(U, device="cuda", dtype=torch.float32 if arith == "f32" else torch.float64)
        V = op.apply(t, nrhs=R, arith="df64" if arith == "df64" else None).cpu().double().numpy()
        if arith == "df64":
            assert op.variant == "reinit/octree/df64/tabulated/planes", op.variant
        for r, (ref, bound) in refs.items():
            ok, worst = componentwise_ok(V[r * dm.n_dofs + rows], ref, bound, rtol)
            assert ok, (arith, r, worst)
