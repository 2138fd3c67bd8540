"""Rows of full-size operators one at a time, from patches of 2 x 2 x 2 cells (test
infrastructure: only tests, smoke() and the bench's CPU leg use this package).

Row i of an assembled finite element operator involves only the cells that contain node i, and on
a uniform mesh those cells lie in a block of 2 x 2 x 2 cells around the node.  The oracle
assembles that block as a mesh of its own (same cell size, the nodal fields restricted to it, no
Dirichlet rows) with the plain full-quadrature routines of ``assemble`` and reads the node's row
(or, for the transpose, its column: the column of node i is complete in the same patch).  Columns
of DoFs that are Dirichlet in the full problem are removed by zeroing those input values; rows of
Dirichlet DoFs are identities and are not computed here.

Lattice conventions are those of ``mesh.uniform_dofmap``: a Q_k lattice of k n + 1 nodes per axis,
DoF index x + L (y + L z), cell index i + n (j + n k).
"""
import numpy as np

from . import mesh as omesh


def _first_cell(coord, k, n):
    """First of the two patch cells along one axis for lattice coordinate ``coord`` of a Q_k
    lattice: the node's cells are coord/k - 1 and coord/k (vertex) or floor(coord/k) (interior)."""
    c = (coord - 1) // k if k > 0 else coord
    return int(min(max(c, 0), n - 2))


def _patch(n, lo, hi, c0, degree):
    h = (np.asarray(hi, float) - np.asarray(lo, float)) / n
    plo = np.asarray(lo, float) + h * np.asarray(c0)
    dm = omesh.uniform_dofmap(2, plo, plo + 2 * h, degree, 0)
    L, Lp = degree * n + 1, 2 * degree + 1
    r = np.arange(Lp)
    gx, gy, gz = np.meshgrid(degree * c0[0] + r, degree * c0[1] + r, degree * c0[2] + r, indexing="ij")
    idx = (gx + L * (gy + L * gz)).transpose(2, 1, 0).ravel()   # patch DoF order: x fastest
    return dm, idx


def _cells(n, c0):
    a = np.arange(2)
    ci, cj, ck = np.meshgrid(c0[0] + a, c0[1] + a, c0[2] + a, indexing="ij")
    return (ci + n * (cj + n * ck)).transpose(2, 1, 0).ravel()     # patch cell order: i fastest


def scalar_rows(n, lo, hi, dofs, build, nodal, u, dirichlet, cellwise=None, transpose=False, absolute=False,
                degree=2):
    """(A u)_i (or (A^T u)_i) for the Q_k DoFs ``dofs`` (k = ``degree``) of a uniform n^3 mesh of [lo, hi].
    ``build(dm, nodal, cellwise)`` assembles the operator on a patch from the nodal fields (dict of
    arrays over the patch DoFs) and the per-cell fields (dict of (8, ...) arrays); ``dirichlet`` is
    the full problem's Dirichlet mask (nodal arrays are indexed on their last axis).  With
    ``absolute``, (|A| |u|)_i instead."""
    L = degree * n + 1
    out = np.empty(len(dofs))
    for s, d in enumerate(dofs):
        coord = (d % L, (d // L) % L, d // (L * L))
        c0 = [_first_cell(c, degree, n) for c in coord]
        dm, idx = _patch(n, lo, hi, c0, degree)
        cells = _cells(n, c0)
        A = build(dm, {k: v[..., idx] for k, v in nodal.items()},
                  {k: v[cells] for k, v in (cellwise or {}).items()}).tocsr()
        us = np.where(dirichlet[idx], 0.0, u[idx])
        local = int(np.nonzero(idx == d)[0][0])
        vec = A.T.tocsr()[local] if transpose else A[local]
        out[s] = np.ravel(abs(vec) @ np.abs(us) if absolute else vec @ us)[0]
    return out


def oseen_rows(n, lo, hi, rows, build, nodal, u, dirichlet_u, absolute=False):
    """(A u)_r of the Oseen operator (three Q2 velocity blocks, then the Q1 pressure block) for the
    row indices ``rows`` of the full vector; ``build(dmu, dmp, nodal)`` assembles it on a patch
    from the nodal fields (dict of (..., n_u) arrays over the patch's velocity DoFs)."""
    L, Lp = 2 * n + 1, n + 1
    nu, npr = L ** 3, Lp ** 3
    out = np.empty(len(rows))
    for s, r in enumerate(rows):
        if r < 3 * nu:
            comp, d = divmod(r, nu)
            coord = (d % L, (d // L) % L, d // (L * L))
            c0 = [_first_cell(c, 2, n) for c in coord]
        else:
            d = r - 3 * nu
            coord = (d % Lp, (d // Lp) % Lp, d // (Lp * Lp))
            c0 = [_first_cell(c, 1, n) for c in coord]
        dmu, idx = _patch(n, lo, hi, c0, 2)
        dmp, pidx = _patch(n, lo, hi, c0, 1)
        A = build(dmu, dmp, {k: v[..., idx] for k, v in nodal.items()}).tocsr()
        uu = [np.where(dirichlet_u[idx], 0.0, u[c * nu + idx]) for c in range(3)]
        us = np.concatenate(uu + [u[3 * nu + pidx]])
        if r < 3 * nu:
            local = comp * len(idx) + int(np.nonzero(idx == d)[0][0])
        else:
            local = 3 * len(idx) + int(np.nonzero(pidx == d)[0][0])
        row = A[local]
        out[s] = np.ravel(abs(row) @ np.abs(us) if absolute else row @ us)[0]
    return out


def constrained_rows(dm, dofs, element_matrices, u, absolute=False):
    """(C^T A C u)_i for the free DoFs ``dofs`` of an octree (or uniform) DoF map ``dm`` without
    assembling the whole operator.  Row i of C^T A C u is sum_p C[p, i] (A C u)_p over the lattice
    points p whose constraint row holds DoF i (i itself, and the hanging points that interpolate from
    it); (A C u)_p sums the element contributions of the cells that contain p.  So only those cells'
    element matrices are formed, by ``element_matrices(cells)`` -> (len(cells), nb, nb) (the plain
    full-quadrature routines of ``assemble``).  Dirichlet columns are removed by zeroing u there;
    Dirichlet rows are identities and are not computed here.  With ``absolute``, (|C|^T |A| |C| |u|)_i,
    an upper bound of (|C^T A C| |u|)_i."""
    import scipy.sparse as sp
    M = dm.points.shape[0]
    nc, nb = dm.cell_points.shape  # incidence of lattice points in cells
    incid = sp.csr_matrix((np.ones(nc * nb), (dm.cell_points.ravel(), np.repeat(np.arange(nc), nb))),
                          shape=(M, nc))
    CT = dm.C.T.tocsr()
    us = np.where(dm.dirichlet, 0.0, u)
    Cu = (abs(dm.C) @ np.abs(us)) if absolute else dm.C @ us
    out = np.empty(len(dofs))
    for s, i in enumerate(dofs):
        pts = CT.indices[CT.indptr[i]:CT.indptr[i + 1]]
        wts = CT.data[CT.indptr[i]:CT.indptr[i + 1]]
        order = np.argsort(pts)
        pts, wts = pts[order], (np.abs(wts) if absolute else wts)[order]
        cells = np.unique(incid[pts].indices)
        Ae = element_matrices(cells)
        cp = dm.cell_points[cells]
        ul = Cu[cp]                                             # (ncells, nb)
        pos = np.minimum(np.searchsorted(pts, cp), len(pts) - 1)
        wl = np.where(pts[pos] == cp, wts[pos], 0.0)            # C[p_a(e), i] per local row
        if absolute:
            out[s] = np.einsum("ea,eab,eb->", wl, np.abs(Ae), ul)
        else:
            out[s] = np.einsum("ea,eab,eb->", wl, Ae, ul)
    return out
