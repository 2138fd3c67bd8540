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
    x, info = op.solve(bt, solver="gmres", precond="block_triangular", restart=50, maxit=400, tol=1e-10,
                       use_graph=True)
    assert info["status"] == 0, info
    r = bt - op.apply(x)
    rel = (torch.linalg.vector_norm(r) / torch.linalg.vector_norm(bt)).item()
    assert rel <= 1e-10 * (1 + 1e-3), (rel, info)
    assert abs(rel - info["rel_residual"]) <= 1e-3 * max(rel, info["rel_residual"]), (rel, info)
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
    for arith, rtol in (("f64", 1e-12), ("f32", 2e-5)):
        t = torch.tensor(uu, device="cuda", dtype=torch.float32 if arith == "f32" else torch.float64)
        v = op.apply(t).cpu().double().numpy()
        ok, worst = componentwise_ok(v[free], ref, bound, rtol)
        assert ok, (arith, worst)
        assert np.all(v[dir_rows] == uu[dir_rows].astype(v.dtype))


def test_heat_adjoint_64_transpose_sampled_rows(ctx):
    n = 64
    wl = syn.scaled(syn.HEAT_ADJOINT, n)
    p = wl.params
    dm, T_prev, b, k = _heat_case(n, wl, kq=True, beta=True)
    op = _heat_operator(ctx, n, wl, T_prev, b, k)
    free, _ = _lattice_sample(n, 60, 8, dm.dirichlet)
    build = lambda d, nod, cw: asm.heat_matrix(d, p["rhocp"], p["dt"], kq=cw["kq"], beta=nod["beta"])
    u = syn.uniform_pm1(13, dm.n_dofs)
    v = op.apply(torch.tensor(u, device="cuda"), transpose=True).cpu().numpy()
    kw = dict(cellwise={"kq": k}, transpose=True)
    ref = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"beta": b}, u, dm.dirichlet, **kw)
    bound = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"beta": b}, u, dm.dirichlet, absolute=True, **kw)
    ok, worst = componentwise_ok(v[free], ref, bound, 1e-12)
    assert ok, worst


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
