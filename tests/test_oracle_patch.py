"""The oracle's patch rows (one row of a full-size operator from a 2x2x2-cell patch) reproduce the
rows of the fully assembled oracle matrices: heat with Dirichlet rows, per-Gauss-point k and the
convection transpose, and the Oseen saddle-point operator (velocity and pressure rows)."""
import numpy as np

import synthetic as syn
from oracle import assemble as asm
from oracle import mesh as omesh
from oracle import patch

from problems import DIRICHLET_BOTTOM, OSEEN_FACES


def test_heat_rows_with_dirichlet_kq_and_transpose():
    n = 4
    wl = syn.scaled(syn.HEAT_ADJOINT, n)
    p = wl.params
    dm = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2, DIRICHLET_BOTTOM)
    x = dm.dof_coords()
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    kq = syn.kq_field(dm.n_cells * 27, wl.seed, p["k0"]).reshape(dm.n_cells, 27)
    A = asm.heat_matrix(dm, p["rhocp"], p["dt"], kq=kq, beta=beta).tocsr()
    u = syn.uniform_pm1(3, dm.n_dofs)
    free = np.random.default_rng(0).choice(np.nonzero(~dm.dirichlet)[0], 150, replace=False)
    build = lambda d, nod, cw: asm.heat_matrix(d, p["rhocp"], p["dt"], kq=cw["kq"], beta=nod["beta"])
    for tr in (False, True):
        got = patch.scalar_rows(n, wl.lo, wl.hi, free, build, {"beta": beta}, u, dm.dirichlet,
                                cellwise={"kq": kq}, transpose=tr)
        ref = ((A.T if tr else A) @ np.where(dm.dirichlet, 0.0, u))[free]
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_oseen_rows_velocity_and_pressure():
    n = 4
    wl = syn.scaled(syn.OSEEN_INTERFACE, n)
    p = wl.params
    dmu = omesh.uniform_dofmap(n, wl.lo, wl.hi, 2, OSEEN_FACES)
    dmp = omesh.uniform_dofmap(n, wl.lo, wl.hi, 1, 0)
    x = dmu.dof_coords()
    t1, t2 = syn.wavy_plane_phases(wl.seed)
    phi = syn.initial_level_set(syn.wavy_plane_distance(*x.T, t1, t2), wl.eps)
    beta = np.array(syn.convection_field(*x.T, wl.seed, wl.lo, wl.hi))
    sigma = 1.0 / (p["dt_cfl"] * wl.h)
    args = (sigma, p["rho_l"], p["rho_g"], p["mu_l"], p["mu_g"])
    A = asm.oseen_matrix(dmu, dmp, phi, beta, *args).tocsr()
    nu = dmu.n_dofs
    u = syn.uniform_pm1(4, A.shape[0])
    mask = np.concatenate([np.tile(dmu.dirichlet, 3), np.zeros(dmp.n_dofs, bool)])
    rows = np.sort(np.concatenate([np.random.default_rng(1).choice(np.nonzero(~mask[:3 * nu])[0], 120, replace=False),
                                   3 * nu + np.arange(dmp.n_dofs)[::4]]))
    build = lambda du, dp, nod: asm.oseen_matrix(du, dp, nod["phi"], nod["beta"], *args)
    got = patch.oseen_rows(n, wl.lo, wl.hi, rows, build, {"phi": phi, "beta": beta}, u, dmu.dirichlet)
    ref = (A @ np.where(mask, 0.0, u))[rows]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    bound = patch.oseen_rows(n, wl.lo, wl.hi, rows[:20], build, {"phi": phi, "beta": beta}, u, dmu.dirichlet,
                             absolute=True)
    assert np.allclose(bound, (abs(A) @ np.abs(np.where(mask, 0.0, u)))[rows[:20]], rtol=1e-13)


def test_q3_q4_helmholtz_rows():
    """Degree-k patches (Gauss-Lobatto nodes): Q3 and Q4 Helmholtz rows against the assembled matrix,
    including every corner, edge and face class of the lattice."""
    for k in (3, 4):
        n = 3
        dm = omesh.uniform_dofmap(n, (0, 0, 0), (1, 1, 1), k)
        phi = syn.initial_level_set(syn.sphere_distance(*dm.dof_coords().T), 1.0 / 6)
        A = asm.helmholtz_matrix(dm, phi, 1.0, 1000.0, 1.0, "tanh", 1.0 / 6).tocsr()
        u = syn.uniform_pm1(4 + k, dm.n_dofs)
        L = k * n + 1
        rows = np.unique(np.concatenate([np.random.default_rng(k).choice(dm.n_dofs, 60, replace=False),
                                         [0, L - 1, L * L - 1, dm.n_dofs - 1, L // 2 + L * (L // 2)]]))
        build = lambda d, nod, cw: asm.helmholtz_matrix(d, nod["phi"], 1.0, 1000.0, 1.0, "tanh", 1.0 / 6)
        got = patch.scalar_rows(n, (0, 0, 0), (1, 1, 1), rows, build, {"phi": phi}, u, dm.dirichlet, degree=k)
        ref = (A @ u)[rows]
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max(), k


def test_constrained_rows_match_the_assembled_octree_operator():
    """Rows of C^T A C from the cells around each row (octree with hanging nodes on two levels)
    equal the rows of the fully assembled and condensed oracle matrix, for free DoFs next to
    hanging nodes, on coarse and fine leaves; the absolute form bounds |C^T A C| |u|."""
    d = lambda x, y, z: syn.deformed_sphere_distance(x, y, z, 3)
    leaves = syn.refine_band_leaves(4, 2, d, 1.0 / 64)
    dm = omesh.octree_dofmap(leaves, 4, 2)
    eps = 1.0 / 64
    phi = syn.initial_level_set(syn.deformed_sphere_distance(*dm.dof_coords().T, 3), eps)
    m, D = asm.reinit_coefficients(dm, phi, eps, 0.5 / 16)
    A = asm.assemble_scalar(dm, m, diff_tensor=D).tocsr()
    u = syn.uniform_pm1(5, dm.n_dofs)
    # DoFs that master some hanging node, plus random ones
    masters = np.unique(dm.C[dm.hang_of_point >= 0].indices)
    rng = np.random.default_rng(2)
    rows = np.unique(np.concatenate([rng.choice(masters, 60, replace=False), rng.choice(dm.n_dofs, 60, replace=False)]))
    emat = lambda cells: asm.scalar_element_matrices(dm, m, diff_tensor=D, cells=cells)
    got = patch.constrained_rows(dm, rows, emat, u)
    ref = (A @ u)[rows]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    bound = patch.constrained_rows(dm, rows, emat, u, absolute=True)
    assert np.all(bound >= (abs(A) @ np.abs(u))[rows] * (1 - 1e-13))
