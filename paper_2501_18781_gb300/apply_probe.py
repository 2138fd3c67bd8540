"""Build one benchmark workload and apply its operator a few times (for profilers such as ncu).

    python -m paper_2501_18781_gb300.apply_probe heat [n] [f32|f64|df64] [inkernel|tabulated]
    python -m paper_2501_18781_gb300.apply_probe oseen [n] [f32|f64|df64]
    python -m paper_2501_18781_gb300.apply_probe reinit [base] [levels] [f32|f64|df64] [nrhs]
    python -m paper_2501_18781_gb300.apply_probe oseen_solve [n] [maxit]
    python -m paper_2501_18781_gb300.apply_probe helmholtz_qk [k] [n] [f32|f64|tc]

Inputs come from the seeded generators in ``synthetic``; every apply runs in libmfgb.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def _apply(op, n, prec, nrhs=1, reps=4):
    import torch
    import synthetic as syn
    u = torch.tensor(syn.uniform_pm1(1, n * nrhs), device="cuda")
    if prec == "f32":
        u = u.float()
    v = torch.empty_like(u)
    for _ in range(reps):
        op.apply(u, v, nrhs=nrhs, arith="df64" if prec == "df64" else None)
    torch.cuda.synchronize()
    print(op.variant, n, "x", nrhs)


def main(argv):
    import numpy as np
    import torch
    import synthetic as syn
    from . import Context, DofMap, Mesh, Operator, build_library
    build_library()
    ctx = Context(0)
    kind = argv[0] if argv else "heat"
    if kind == "heat":
        n = int(argv[1]) if len(argv) > 1 else 128
        prec = argv[2] if len(argv) > 2 else "f32"
        mode = 0 if (len(argv) <= 3 or argv[3] == "inkernel") else 1
        wl = syn.scaled(syn.HEAT_LASER, n)
        p = wl.params
        m = DofMap(Mesh.uniform(ctx, n, wl.lo, wl.hi), 2, 1 << 4)
        x = m.coords()
        T = syn.heat_initial_temperature(*x.T, p["laser"]["radius"], wl.hi[2])
        op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"],
                      coef_mode=mode)
        op.set_field("t_prev", torch.tensor(T, device="cuda"))
        _apply(op, m.n_dofs, prec)
    elif kind in ("oseen", "oseen_solve"):
        n = int(argv[1]) if len(argv) > 1 else 64
        prec = argv[2] if (len(argv) > 2 and kind == "oseen") else "f64"
        wl = syn.scaled(syn.OSEEN_INTERFACE, n)
        p = wl.params
        mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
        mu, mp = DofMap(mesh, 2, 0b011111), DofMap(mesh, 1, 0)
        x = mu.coords()
        t1, t2 = syn.wavy_plane_phases(wl.seed)
        phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
        beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
        op = Operator(ctx, "oseen", [mu, mp], sigma=1.0 / (p["dt_cfl"] * wl.h), rho_l=p["rho_l"], rho_g=p["rho_g"],
                      mu_l=p["mu_l"], mu_g=p["mu_g"], eps=wl.eps)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
        op.autotune()
        if kind == "oseen":
            _apply(op, op.n, prec)
        else:
            # flexible GMRES with the block-triangular preconditioner, capped at maxit iterations
            maxit = int(argv[2]) if len(argv) > 2 else 400
            b = syn.uniform_pm1(1, op.n)
            d = mu.export(cell_map=False, constraints=False, coords=False)["dirichlet"]
            b[np.concatenate([np.tile(d, 3), np.zeros(mp.n_dofs, bool)])] = 0
            bt = torch.tensor(b, device="cuda")
            for _ in range(2):
                _, info = op.solve(bt, solver="gmres", precond="block_triangular", maxit=maxit, tol=1e-10)
            torch.cuda.synchronize()
            print(op.variant, n, info)
    elif kind == "helmholtz_qk":
        k = int(argv[1]) if len(argv) > 1 else 3
        n = int(argv[2]) if len(argv) > 2 else 64
        prec = argv[3] if len(argv) > 3 else "f32"
        m = DofMap(Mesh.uniform(ctx, n), k, 0)
        eps = 1.0 / (2 * n)
        phi = syn.initial_level_set(syn.sphere_distance(*m.coords().T), eps)
        op = Operator(ctx, "helmholtz", [m], mass_coef=1.0, a_liquid=1000.0, a_gas=1.0, eps=eps)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        u = torch.tensor(syn.uniform_pm1(1, m.n_dofs), device="cuda")
        if prec != "f64":
            u = u.float()
        v = torch.empty_like(u)
        for _ in range(4):
            op.apply(u, v, arith="tc" if prec == "tc" else None)
        torch.cuda.synchronize()
        print(op.variant, m.n_dofs)
    elif kind == "reinit":
        base = int(argv[1]) if len(argv) > 1 else 16
        levels = int(argv[2]) if len(argv) > 2 else 3
        prec = argv[3] if len(argv) > 3 else "f32"
        nrhs = int(argv[4]) if len(argv) > 4 else 1
        eps = 2.0 / (base << levels)
        d = lambda X, Y, Z: syn.deformed_sphere_distance(X, Y, Z, 1)
        leaves = syn.refine_band_leaves(base, levels, d, eps)
        m = DofMap(Mesh.octree(ctx, base, levels, leaves), 2, 0)
        x = m.coords()
        phi = syn.initial_level_set(syn.deformed_sphere_distance(*x.T, 1), eps)
        op = Operator(ctx, "reinit", [m], eps=eps, dtau=0.5 / (base << levels), coef_mode=1)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        _apply(op, m.n_dofs, prec, nrhs)
    else:
        raise SystemExit(f"unknown workload {kind}")


if __name__ == "__main__":
    main(sys.argv[1:])
