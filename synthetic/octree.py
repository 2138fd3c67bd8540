"""Adaptive leaf lists on the unit cube: band refinement around a level-set zero and
full (face, edge and corner) 2:1 balancing.  A leaf is (level, i, j, k) with
0 <= i, j, k < base * 2**level."""
import numpy as np


def _block_max(grid, s):
    n = grid.shape[0] // s
    return grid.reshape(n, s, n, s, n, s).max(axis=(1, 3, 5))


def _upsample(coarse, s):
    return np.repeat(np.repeat(np.repeat(coarse, s, axis=0), s, axis=1), s, axis=2)


def refine_band_leaves(base, levels, distance, eps):
    """Refine a level-l cell (l < levels) when |d(centre)| < 4 eps + (sqrt(3)/2) h_l, then
    2:1-balance.  ``distance(x, y, z)`` is vectorised.  Returns int32 (n, 4) leaves sorted
    by (level, k, j, i)."""
    from scipy.ndimage import maximum_filter
    nf = base << levels
    lev = np.zeros((nf, nf, nf), dtype=np.int8)  # [i, j, k] -> level of the covering leaf
    for l in range(levels):
        n = base << l
        s = nf // n
        h = 1.0 / n
        c = (np.arange(n) + 0.5) * h
        X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
        leaf_here = lev[::s, ::s, ::s] == l
        near = np.abs(distance(X, Y, Z)) < 4.0 * eps + 0.5 * np.sqrt(3.0) * h
        mark = leaf_here & near
        lev = np.maximum(lev, _upsample(mark.astype(np.int8) * np.int8(l + 1), s))
    changed = True
    while changed:
        changed = False
        dil = maximum_filter(lev, size=3, mode="nearest")
        for l in range(levels - 1):
            s = nf // (base << l)
            leaf_here = lev[::s, ::s, ::s] == l
            need = leaf_here & (_block_max(dil, s) >= l + 2)
            if need.any():
                lev = np.maximum(lev, _upsample(need.astype(np.int8) * np.int8(l + 1), s))
                changed = True
    out = []
    for l in range(levels + 1):
        s = nf // (base << l)
        ii, jj, kk = np.nonzero(lev[::s, ::s, ::s] == l)
        order = np.lexsort((ii, jj, kk))
        out.append(np.stack([np.full(ii.size, l), ii[order], jj[order], kk[order]], axis=1))
    return np.concatenate(out).astype(np.int32)


def is_two_to_one_balanced(leaves, base, levels):
    """True if the leaves tile the cube exactly once and any two leaves whose closures
    touch differ by at most one level."""
    nf = base << levels
    lev = np.full((nf, nf, nf), -1, dtype=np.int8)
    cover = np.zeros((nf, nf, nf), dtype=np.int32)
    for l, i, j, k in leaves:
        s = nf // (base << int(l))
        sl = (slice(i * s, (i + 1) * s), slice(j * s, (j + 1) * s), slice(k * s, (k + 1) * s))
        lev[sl] = l
        cover[sl] += 1
    if not np.all(cover == 1):
        return False
    from scipy.ndimage import maximum_filter, minimum_filter
    hi = maximum_filter(lev, size=3, mode="nearest")
    lo = minimum_filter(lev, size=3, mode="nearest")
    return bool(np.all(hi - lev <= 1) and np.all(lev - lo <= 1))
