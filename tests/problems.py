"""Shared builders for the parity tests: the same seeded workload as an oracle CSR matrix
and as a library operator on the GPU."""
import numpy as np

import synthetic as syn
from oracle import assemble as asm
from oracle import heat as oheat
from oracle import mesh as omesh

DIRICHLET_BOTTOM = 1 << 4
OSEEN_FACES = 0b011111  # all faces but z+


def componentwise_ok(v, ref, bound, rtol):
    """|v - ref|_i <= rtol * bound_i (bound = |A| |u|, plus a tiny floor)."""
    err = np.abs(v - ref)
    floor = 1e-300 + 1e-15 * np.max(bound)
    worst = np.max(err / (bound + floor))
    return worst <= rtol, worst


def schur_reference(A, nu):
    """The oracle's B D^-1 B^T (D: the 3 x 3 nodal blocks of A_uu) from an assembled Oseen matrix
    with 3 nu velocity unknowns first: returns (S, |B| |D^-1| |B^T|) as sparse matrices."""
    import scipy.sparse as sp
    A = A.tocsr()
    N = 3 * nu
    B, BT, Auu = A[N:, :N], A[:N, N:], A[:N, :N]
    i = np.arange(nu)
    D = np.empty((nu, 3, 3))
    for d in range(3):
        for e in range(3):
            D[:, d, e] = np.asarray(Auu[d * nu + i, e * nu + i]).ravel()
    Dinv = np.linalg.inv(D)
    rows = np.concatenate([d * nu + i for d in range(3) for e in range(3)])
    cols = np.concatenate([e * nu + i for d in range(3) for e in range(3)])
    Dsp = sp.csr_matrix((np.concatenate([Dinv[:, d, e] for d in range(3) for e in range(3)]), (rows, cols)),
                        shape=(N, N))
    return (B @ Dsp @ BT).tocsr(), (abs(B) @ abs(Dsp) @ abs(BT)).tocsr()


def schur_fp16_bound(S, p, n):
    """Error bound of the fp32 Schur stencil whose entries are stored as fp16 scaled by their row's
    largest magnitude: per entry at most half an fp16 unit of 1, 2^-12 of the row maximum, so per
    row 2^-12 max_o |S_io| times the sum of |p| over the 5 x 5 x 5 box of grid nodes (n + 1 per
    axis) around the row's node."""
    m = n + 1
    P = np.abs(p).reshape(m, m, m)
    box = np.zeros_like(P)
    for dz in range(-2, 3):
        for dy in range(-2, 3):
            for dx in range(-2, 3):
                sh = np.zeros_like(P)
                sh[max(0, -dz):m - max(0, dz), max(0, -dy):m - max(0, dy), max(0, -dx):m - max(0, dx)] = \
                    P[max(0, dz):m - max(0, -dz), max(0, dy):m - max(0, -dy), max(0, dx):m - max(0, -dx)]
                box += sh
    rowmax = np.asarray(abs(S).max(axis=1).todense()).ravel()
    return 2.0 ** -12 * rowmax * box.ravel()


def helmholtz(n, ctx=None, heaviside="tanh", coef_mode=0, octree=None):
    wl = syn.scaled(syn.HELMHOLTZ_SPHERE, n)
    if octree is None:
        dm = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2)
        eps = wl.eps
    else:
        leaves, base, levels = octree
        dm = omesh.octree_dofmap(leaves, base, levels)
        eps = 2.0 / (base << levels)
    x = dm.dof_coords()
    phi = syn.initial_level_set(syn.sphere_distance(*x.T), eps)
    p = wl.params
    A = asm.helmholtz_matrix(dm, phi, p["mass"], p["a_liquid"], p["a_gas"], heaviside, eps)
    out = dict(dm=dm, A=A, phi=phi, eps=eps, n=dm.n_dofs)
    if ctx is not None:
        import torch
        from paper_2501_18781_gb300 import DofMap, Mesh, Operator
        if octree is None:
            mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
        else:
            mesh = Mesh.octree(ctx, octree[1], octree[2], octree[0])
        m = DofMap(mesh, 2, 0)
        op = Operator(ctx, "helmholtz", [m], mass_coef=p["mass"], a_liquid=p["a_liquid"], a_gas=p["a_gas"],
                      heaviside=0 if heaviside == "tanh" else 1, eps=eps, coef_mode=coef_mode)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        out.update(op=op, map=m, mesh=mesh)
    return out


def heat(n, ctx=None, with_beta=False, kq=False, coef_mode=0):
    wl = syn.scaled(syn.HEAT_ADJOINT if kq or with_beta else syn.HEAT_LASER, n)
    p = wl.params
    dm = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2, DIRICHLET_BOTTOM)
    x = dm.dof_coords()
    ztop = wl.hi[2]
    T_prev = syn.heat_initial_temperature(*x.T, p["laser"]["radius"], ztop)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi)) if with_beta else None
    kqv = syn.kq_field(dm.n_cells * 27, wl.seed, p["k0"]).reshape(dm.n_cells, 27) if kq else None
    A = asm.heat_matrix(dm, p["rhocp"], p["dt"], k0=p["k0"], t_boil=p["t_boil"], T_prev=T_prev, kq=kqv, beta=beta)
    out = dict(dm=dm, A=A, T_prev=T_prev, beta=beta, kq=kqv, wl=wl, n=dm.n_dofs)
    if ctx is not None:
        import torch
        from paper_2501_18781_gb300 import DofMap, Mesh, Operator
        mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
        m = DofMap(mesh, 2, DIRICHLET_BOTTOM)
        op = Operator(ctx, "heat", [m], rhocp=p["rhocp"], dt=p["dt"], k0=p["k0"], t_boil=p["t_boil"],
                      coef_mode=coef_mode)
        op.set_field("t_prev", torch.tensor(T_prev, device="cuda"))
        if beta is not None:
            op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
        if kqv is not None:
            op.set_field("k_qpoint", torch.tensor(kqv.ravel(), device="cuda"))
        out.update(op=op, map=m, mesh=mesh)
    return out


def oseen(n, ctx=None):
    wl = syn.scaled(syn.OSEEN_INTERFACE, n)
    p = wl.params
    dmu = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2, OSEEN_FACES)
    dmp = omesh.uniform_dofmap(n, wl.lo, wl.hi, 1, 0)
    x = dmu.dof_coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    sigma = 1.0 / (p["dt_cfl"] * wl.h)
    A = asm.oseen_matrix(dmu, dmp, phi, beta, sigma, p["rho_l"], p["rho_g"], p["mu_l"], p["mu_g"])
    out = dict(dmu=dmu, dmp=dmp, A=A, phi=phi, beta=beta, sigma=sigma, n=A.shape[0])
    if ctx is not None:
        import torch
        from paper_2501_18781_gb300 import DofMap, Mesh, Operator
        mesh = Mesh.uniform(ctx, n, wl.lo, wl.hi)
        mu_, mp_ = DofMap(mesh, 2, OSEEN_FACES), DofMap(mesh, 1, 0)
        op = Operator(ctx, "oseen", [mu_, mp_], sigma=sigma, rho_l=p["rho_l"], rho_g=p["rho_g"], mu_l=p["mu_l"],
                      mu_g=p["mu_g"], eps=wl.eps)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        op.set_field("beta", torch.tensor(beta.ravel(), device="cuda"))
        out.update(op=op, maps=(mu_, mp_), mesh=mesh)
    return out


def reinit(octree, ctx=None, seed=1, coef_mode=0):
    leaves, base, levels = octree
    dm = omesh.octree_dofmap(leaves, base, levels)
    h_min = 1.0 / (base << levels)
    eps = 2.0 * h_min
    x = dm.dof_coords()
    phi = syn.initial_level_set(syn.deformed_sphere_distance(*x.T, seed), eps)
    dtau = 0.5 * h_min
    A = asm.reinit_matrix(dm, phi, eps, dtau)
    out = dict(dm=dm, A=A, phi=phi, eps=eps, dtau=dtau, n=dm.n_dofs)
    if ctx is not None:
        import torch
        from paper_2501_18781_gb300 import DofMap, Mesh, Operator
        mesh = Mesh.octree(ctx, base, levels, leaves)
        m = DofMap(mesh, 2, 0)
        op = Operator(ctx, "reinit", [m], eps=eps, dtau=dtau, coef_mode=coef_mode)
        op.set_field("phi", torch.tensor(phi, device="cuda"))
        out.update(op=op, map=m, mesh=mesh)
    return out


def band_octree(base=4, levels=2, eps=1.0 / 64, seed=3):
    d = lambda x, y, z: syn.deformed_sphere_distance(x, y, z, seed)
    return syn.refine_band_leaves(base, levels, d, eps), base, levels
