"""Node lattices, DoF numbering and hanging-node constraints (Appendix B: continuous
Lagrange elements on adaptively refined hexahedral meshes).

Conventions of the library that the oracle reproduces independently:
* Nodes live on the lattice of spacing h_finest / k.  Free nodes are numbered in
  lexicographic (z, y, x) order of their integer lattice coordinates.
* A node that lies on the closure of a leaf K without being one of K's nodes is
  hanging; its value is the interpolant of K's Q_k function at that point, so its
  weights are products of 1D Lagrange values l_a(xi) with xi in {0, 1/4, 1/2, 3/4, 1}
  (dyadic, exact in binary64).  Masters that hang themselves are replaced
  recursively; equal masters are summed and exact zeros dropped.
* Uniform meshes order cells lexicographically (x fastest); octree leaves by the
  Morton code of their anchor on the finest level (bit b of x, y, z goes to bit
  3b, 3b+1, 3b+2).
* Dirichlet faces are bits 0..5 = x-, x+, y-, y+, z-, z+.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .basis import lagrange_1d


@dataclass
class DofMap:
    degree: int
    R: int                    # lattice intervals per axis (points 0..R)
    lo: np.ndarray            # domain lower corner
    hspan: np.ndarray         # domain edge lengths
    cell_level: np.ndarray    # (ncell,)
    cell_h: np.ndarray        # (ncell,) physical edge length
    cell_origin: np.ndarray   # (ncell, 3) physical lower corner
    cell_points: np.ndarray   # (ncell, nb) index into ``points``
    points: np.ndarray        # (M, 3) lattice coords of every node of every cell
    C: sp.csr_matrix          # (M, n_dofs) node values from free DoFs
    free_of_point: np.ndarray # (M,) free index or -1
    hang_of_point: np.ndarray # (M,) hanging rank or -1
    n_dofs: int
    dirichlet: np.ndarray     # (n_dofs,) bool

    @property
    def n_cells(self):
        return self.cell_points.shape[0]

    def dof_coords(self):
        """Physical coordinates of the free DoFs, in DoF order (for k >= 3, uniform meshes: lattice
        coordinate k c + a sits at the support point xi_a of cell c)."""
        free = np.nonzero(self.free_of_point >= 0)[0]
        order = np.argsort(self.free_of_point[free])
        p = self.points[free[order]]
        if self.degree <= 2:
            return self.lo + p.astype(np.float64) * (self.hspan / self.R)
        from .basis import lagrange_nodes
        k, n = self.degree, self.R // self.degree
        c = np.minimum(p // k, n - 1)
        return self.lo + (c + lagrange_nodes(k)[p - k * c]) * (self.hspan / n)

    def export(self):
        """Integer cell map (free index, or -(1 + hanging rank)) and the constraint rows
        (CSR: row pointer, master DoF indices ascending, weights) of the hanging nodes."""
        cm = np.where(self.free_of_point[self.cell_points] >= 0,
                      self.free_of_point[self.cell_points],
                      -1 - self.hang_of_point[self.cell_points]).astype(np.int32)
        hang = np.nonzero(self.hang_of_point >= 0)[0]
        hang = hang[np.argsort(self.hang_of_point[hang])]
        rows = self.C[hang].tocsr()
        rows.sort_indices()
        return cm, rows.indptr.astype(np.int64), rows.indices.astype(np.int32), rows.data.copy()


def _keys(points, R):
    p = points.astype(np.int64)
    return p[:, 2] * (R + 1) * (R + 1) + p[:, 1] * (R + 1) + p[:, 0]


def _dirichlet_of_points(points, R, face_mask):
    m = np.zeros(points.shape[0], dtype=bool)
    for ax in range(3):
        if face_mask >> (2 * ax) & 1:
            m |= points[:, ax] == 0
        if face_mask >> (2 * ax + 1) & 1:
            m |= points[:, ax] == R
    return m


def uniform_dofmap(n, lo, hi, degree, dirichlet_faces=0):
    """Q_k DoF map of a uniform n^3 mesh of the box [lo, hi]: every lattice node is free."""
    k = degree
    R = k * n
    lo = np.asarray(lo, dtype=np.float64)
    hspan = np.asarray(hi, dtype=np.float64) - lo
    nb = (k + 1) ** 3
    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    # lexicographic cells, x fastest
    cells = np.stack([ci.transpose(2, 1, 0).ravel(), cj.transpose(2, 1, 0).ravel(),
                      ck.transpose(2, 1, 0).ravel()], axis=1)
    loc = np.array([[a, b, c] for c in range(k + 1) for b in range(k + 1) for a in range(k + 1)])
    pts = cells[:, None, :] * k + loc[None, :, :]                 # (ncell, nb, 3)
    keys = pts[..., 2] * (R + 1) ** 2 + pts[..., 1] * (R + 1) + pts[..., 0]
    M = (R + 1) ** 3
    pz, py, px = np.meshgrid(np.arange(R + 1), np.arange(R + 1), np.arange(R + 1), indexing="ij")
    points = np.stack([px.ravel(), py.ravel(), pz.ravel()], axis=1)
    dmask = _dirichlet_of_points(points, R, dirichlet_faces)
    h = hspan[0] / n
    return DofMap(degree=k, R=R, lo=lo, hspan=hspan,
                  cell_level=np.zeros(n ** 3, dtype=np.int32),
                  cell_h=np.full(n ** 3, h), cell_origin=lo + cells * h,
                  cell_points=keys.reshape(-1, nb), points=points,
                  C=sp.identity(M, format="csr"), free_of_point=np.arange(M),
                  hang_of_point=np.full(M, -1), n_dofs=M, dirichlet=dmask)


def morton3(x, y, z, bits=21):
    """Interleave the bits of x, y, z (x in bit 0)."""
    code = np.zeros(np.shape(x), dtype=np.int64)
    x, y, z = (np.asarray(v, dtype=np.int64) for v in (x, y, z))
    for b in range(bits):
        code |= ((x >> b) & 1) << (3 * b)
        code |= ((y >> b) & 1) << (3 * b + 1)
        code |= ((z >> b) & 1) << (3 * b + 2)
    return code


def octree_dofmap(leaves, base, levels, degree=2, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0),
                  dirichlet_faces=0):
    """Q_k DoF map of a 2:1-balanced leaf list (rows level, i, j, k on the level grid of a
    base^3 root mesh of the box [lo, hi]) with hanging-node constraints."""
    k = degree
    L = levels
    leaves = np.asarray(leaves, dtype=np.int64)
    lev = leaves[:, 0]
    nf = base << L
    R = k * nf
    order = np.argsort(morton3(leaves[:, 1] << (L - lev), leaves[:, 2] << (L - lev),
                               leaves[:, 3] << (L - lev)), kind="stable")
    leaves, lev = leaves[order], lev[order]
    step = (1 << (L - lev))                                   # node spacing in lattice units
    anchor = leaves[:, 1:4] * (k * step)[:, None]
    loc = np.array([[a, b, c] for c in range(k + 1) for b in range(k + 1) for a in range(k + 1)])
    pts = anchor[:, None, :] + loc[None, :, :] * step[:, None, None]
    flat = pts.reshape(-1, 3)
    keys = _keys(flat, R)
    ukeys, inv = np.unique(keys, return_inverse=True)
    points = np.stack([ukeys % (R + 1), (ukeys // (R + 1)) % (R + 1), ukeys // (R + 1) ** 2], axis=1)
    M = ukeys.size
    cell_points = inv.reshape(pts.shape[0], -1)

    # hanging points: on the closure of a leaf, at half its node spacing, but node of another leaf
    masters = {}   # point index -> dict(point index -> weight)
    half = np.array([[p, q, r] for r in range(2 * k + 1) for q in range(2 * k + 1)
                     for p in range(2 * k + 1)])
    on_boundary = np.any((half == 0) | (half == 2 * k), axis=1)
    odd = np.any(half % 2 == 1, axis=1)
    cand = half[on_boundary & odd]                             # candidate offsets (in half spacings)
    L1, _ = lagrange_1d(k, np.arange(2 * k + 1) / (2.0 * k))   # L1[a, p] = l_a(p / 2k)
    for c in np.nonzero(lev < L)[0]:
        hs = step[c] // 2
        cpts = anchor[c][None, :] + cand * hs
        ck = _keys(cpts, R)
        pos = np.searchsorted(ukeys, ck)
        pos = np.minimum(pos, M - 1)
        found = ukeys[pos] == ck
        for t in np.nonzero(found)[0]:
            pidx = pos[t]
            p, q, r = cand[t]
            w = {}
            for li in range(cell_points.shape[1]):
                a, b, cc = loc[li]
                val = L1[a, p] * L1[b, q] * L1[cc, r]
                if val != 0.0:
                    w[cell_points[c, li]] = val
            if pidx in masters:
                assert masters[pidx] == w, "inconsistent hanging interpolation"
            masters[pidx] = w

    # resolve chains: substitute hanging masters until only free masters remain
    def resolve(pidx, depth=0):
        assert depth < 64
        out = {}
        for m, wm in masters[pidx].items():
            if m in masters:
                for mm, wmm in resolve(m, depth + 1).items():
                    out[mm] = out.get(mm, 0.0) + wm * wmm
            else:
                out[m] = out.get(m, 0.0) + wm
        return {m: w for m, w in out.items() if w != 0.0}

    is_hang = np.zeros(M, dtype=bool)
    is_hang[list(masters.keys())] = True
    free_of_point = np.full(M, -1, dtype=np.int64)
    free_pts = np.nonzero(~is_hang)[0]                        # already in key order
    free_of_point[free_pts] = np.arange(free_pts.size)
    hang_of_point = np.full(M, -1, dtype=np.int64)
    hang_pts = np.nonzero(is_hang)[0]
    hang_of_point[hang_pts] = np.arange(hang_pts.size)

    rows, cols, vals = [free_pts], [np.arange(free_pts.size)], [np.ones(free_pts.size)]
    for pidx in hang_pts:
        res = resolve(pidx)
        ms = np.array(sorted(res.keys()), dtype=np.int64)
        rows.append(np.full(ms.size, pidx))
        cols.append(free_of_point[ms])
        vals.append(np.array([res[m] for m in ms]))
    C = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(M, free_pts.size))
    lo = np.asarray(lo, dtype=np.float64)
    hspan = np.asarray(hi, dtype=np.float64) - lo
    h = hspan[0] / (base << lev)
    dmask = _dirichlet_of_points(points[free_pts], R, dirichlet_faces)
    return DofMap(degree=k, R=R, lo=lo, hspan=hspan, cell_level=lev.astype(np.int32),
                  cell_h=h, cell_origin=lo + leaves[:, 1:4] * h[:, None],
                  cell_points=cell_points, points=points, C=C,
                  free_of_point=free_of_point, hang_of_point=hang_of_point,
                  n_dofs=int(free_pts.size), dirichlet=dmask)
