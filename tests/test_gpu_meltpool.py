"""The Oseen operator with the melt-pool terms (three-phase density and viscosity, Darcy damping,
trace-corrected viscous stress) on the GPU against the oracle's assembled matrix."""
import numpy as np
import pytest

import synthetic as syn
from oracle import assemble as asm
from oracle import mesh as omesh
from problems import OSEEN_FACES, componentwise_ok, schur_fp16_bound, schur_reference

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TS, TL = 1933.0, 2200.0
SOLID = dict(rho_s=5000.0, mu_s=2e-2, t_solidus=TS, t_liquidus=TL)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_18781_gb300 import Context, build_library
    build_library()
    return Context(0)


def meltpool(n, ctx, flags, darcy_c=1e6, with_temperature=True):
    from paper_2501_18781_gb300 import DofMap, Mesh, Operator
    from paper_2501_18781_gb300._lib import MF_OSEEN_DARCY, MF_OSEEN_THREE_PHASE, MF_OSEEN_TRACE_CORRECTION
    wl = syn.scaled(syn.OSEEN_INTERFACE, n)
    p = wl.params
    dmu = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2, OSEEN_FACES)
    dmp = omesh.uniform_dofmap(n, wl.lo, wl.hi, 1, 0)
    x = dmu.dof_coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    T = syn.interface_temperature(*x.T, t_base=1500.0)   # solid far away, melt and vapour near the spot
    sigma = 1.0 / (p["dt_cfl"] * wl.h)
    darcy = dict(C=darcy_c, b=1.0, t_solidus=TS, t_liquidus=TL)
    A = asm.oseen_matrix(dmu, dmp, phi, beta, sigma, p["rho_l"], p["rho_g"], p["mu_l"], p["mu_g"], T=T,
                         solid=SOLID if "three" in flags else None, darcy=darcy if "darcy" in flags else None,
                         trace_correction="trace" in flags)
    bits = (MF_OSEEN_THREE_PHASE if "three" in flags else 0) | (MF_OSEEN_DARCY if "darcy" in flags else 0) | \
        (MF_OSEEN_TRACE_CORRECTION if "trace" in flags else 0)
    mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
    mu_, mp_ = DofMap(mesh, 2, OSEEN_FACES), DofMap(mesh, 1, 0)
    op = Operator(ctx, "oseen", [mu_, mp_], sigma=sigma, rho_l=p["rho_l"], rho_g=p["rho_g"], mu_l=p["mu_l"],
                  mu_g=p["mu_g"], eps=wl.eps, rho_s=SOLID["rho_s"], mu_s=SOLID["mu_s"], t_solidus=TS, t_liquidus=TL,
                  darcy_c=darcy_c, darcy_b=1.0, oseen_flags=bits)
    op.set_field("phi", torch.tensor(phi, device="cuda"))
    op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
    if with_temperature:
        op.set_field("t_prev", torch.tensor(T, device="cuda"))
    return dict(A=A, op=op, n=A.shape[0], dmu=dmu, dmp=dmp)


@pytest.mark.parametrize("flags", [("three",), ("darcy",), ("trace",), ("three", "darcy", "trace")])
def test_meltpool_oseen_apply_matches_oracle(ctx, flags):
    P = meltpool(5, ctx, flags)
    u = syn.uniform_pm1(5, P["n"])
    ref = P["A"] @ u
    bound = abs(P["A"]) @ np.abs(u)
    v = P["op"].apply(torch.tensor(u, device="cuda")).cpu().numpy()
    ok, worst = componentwise_ok(v, ref, bound, 1e-12)
    assert ok, (flags, worst)
    vd = P["op"].apply(torch.tensor(u, device="cuda"), arith="df64").cpu().numpy()   # double-float
    ok, worst = componentwise_ok(vd, ref, bound, 1e-12)
    assert ok, (flags, "df64", worst)
    assert P["op"].variant.startswith("oseen_q2q1/df64/") and P["op"].variant.endswith("/meltpool"), P["op"].variant
    u32 = u.astype(np.float32)
    v32 = P["op"].apply(torch.tensor(u32, device="cuda")).cpu().numpy().astype(np.float64)
    ok, worst = componentwise_ok(v32, P["A"] @ u32.astype(np.float64), abs(P["A"]) @ np.abs(u32.astype(np.float64)),
                                 5e-5)
    assert ok, (flags, "fp32", worst)
    assert "meltpool" in P["op"].variant


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_meltpool_schur_complement_approximation(ctx, dtype):
    """B D^-1 B^T p with the melt-pool terms (the trace correction makes the nodal blocks D
    nonsymmetric) against the oracle's assembled blocks; fp32 is the preconditioner's row-scaled
    fp16 stencil, whose bound adds the storage error."""
    P = meltpool(3, ctx, ("three", "darcy", "trace"))
    nu = P["dmu"].n_dofs
    Auu = P["A"].tocsr()[:3 * nu, :3 * nu]
    i = np.arange(nu)
    d01 = np.asarray(Auu[i, nu + i]).ravel() - np.asarray(Auu[nu + i, i]).ravel()
    assert np.abs(d01).max() > 0  # the nodal blocks are nonsymmetric
    S, Sabs = schur_reference(P["A"], nu)
    p = syn.uniform_pm1(12, S.shape[0])
    if dtype == "f32":
        p = p.astype(np.float32).astype(np.float64)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    got = P["op"].coupling("schur", torch.tensor(p, dtype=tdt, device="cuda")).cpu().double().numpy()
    ref, bound = S @ p, Sabs @ np.abs(p)
    if dtype == "f64":
        ok, worst = componentwise_ok(got, ref, bound, 1e-12)
    else:
        ok, worst = componentwise_ok(got, ref, 5e-5 * bound + schur_fp16_bound(S, p, 3), 1.0)
    assert ok, worst


def test_meltpool_oseen_solve_with_block_preconditioner(ctx):
    """The Darcy-damped velocity block needs more inner GMRES steps than the defaults: with 10,
    restarted FGMRES(50) takes about 300 iterations in exact arithmetic, and the run-to-run
    rounding of the atomic scatter moves the count between 300 and past 600; with 20 steps and
    the Schur CG to 0.05 it converges within the first restart cycle (34 iterations in fp64)."""
    P = meltpool(6, ctx, ("three", "darcy", "trace"))
    b = syn.uniform_pm1(6, P["n"])
    b[np.concatenate([np.tile(P["dmu"].dirichlet, 3), np.zeros(P["dmp"].n_dofs, bool)])] = 0.0
    x, info = P["op"].solve(torch.tensor(b, device="cuda"), solver="gmres", precond="block_triangular", restart=50,
                            maxit=400, tol=1e-10, velocity_steps=20, schur_maxit=50, schur_tol=0.05)
    assert info["status"] == 0, info
    assert info["iterations"] <= 100, info
    res = np.linalg.norm(b - P["A"] @ x.cpu().numpy()) / np.linalg.norm(b)
    assert res <= 1e-10 * (1 + 1e-3), (res, info)


def test_meltpool_rejects_missing_temperature(ctx):
    """Three-phase and Darcy terms need the nodal temperature: without it every arithmetic refuses."""
    from paper_2501_18781_gb300._lib import MFError
    for flags in (("darcy",), ("three",)):
        P = meltpool(3, ctx, flags, with_temperature=False)
        u = torch.tensor(syn.uniform_pm1(1, P["n"]), device="cuda")
        for arith in (None, "df64"):
            with pytest.raises(MFError):
                P["op"].apply(u, arith=arith)
