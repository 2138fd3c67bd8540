"""Q_k Lagrange bases and tensor Gauss rules (Appendix B).

Everything is evaluated directly from its definition: a 1D Lagrange polynomial as a
product over the other nodes, a 3D shape function as the product of three 1D ones.
Local node and point numbering is x fastest: i = a + (k+1) b + (k+1)^2 c.
"""
import numpy as np


def gauss_rule_01(npts):
    """Gauss-Legendre points and weights mapped to [0, 1] (numpy's leggauss on [-1, 1])."""
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_nodes(k):
    """Support points on [0, 1]: {0, 1} for k = 1, {0, 1/2, 1} for k = 2 (equispaced and
    Gauss-Lobatto coincide), and the Gauss-Lobatto points for k >= 3: the ends and the roots of
    P_k', the derivative of the Legendre polynomial of degree k (numpy's root finder)."""
    if k <= 2:
        return np.linspace(0.0, 1.0, k + 1)
    inner = np.sort(np.polynomial.legendre.Legendre.basis(k).deriv().roots().real)
    return np.concatenate([[0.0], 0.5 * (inner + 1.0), [1.0]])


def lagrange_1d(k, x):
    """Values L[a, p] = l_a(x_p) and derivatives dL[a, p] = l_a'(x_p) of the degree-k
    Lagrange polynomials, from the product formula l_a(x) = prod_{b != a} (x - x_b)/(x_a - x_b)."""
    nodes = lagrange_nodes(k)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    L = np.ones((k + 1, x.size))
    dL = np.zeros((k + 1, x.size))
    for a in range(k + 1):
        for b in range(k + 1):
            if b != a:
                L[a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        # derivative of the product: sum over the factor that is differentiated
        for m in range(k + 1):
            if m == a:
                continue
            term = np.full(x.size, 1.0 / (nodes[a] - nodes[m]))
            for b in range(k + 1):
                if b != a and b != m:
                    term = term * (x - nodes[b]) / (nodes[a] - nodes[b])
            dL[a] += term
    return L, dL


def tensor_tables(k, npts):
    """Shape values N[q, i], reference gradients G[q, i, d] and weights w[q] of the
    tensor Gauss rule with npts^3 points on the unit reference cube."""
    xq, wq = gauss_rule_01(npts)
    L, dL = lagrange_1d(k, xq)
    nb, nq = (k + 1) ** 3, npts ** 3
    N = np.zeros((nq, nb))
    G = np.zeros((nq, nb, 3))
    w = np.zeros(nq)
    for qc in range(npts):
        for qb in range(npts):
            for qa in range(npts):
                q = qa + npts * (qb + npts * qc)
                w[q] = wq[qa] * wq[qb] * wq[qc]
                for c in range(k + 1):
                    for b in range(k + 1):
                        for a in range(k + 1):
                            i = a + (k + 1) * (b + (k + 1) * c)
                            N[q, i] = L[a, qa] * L[b, qb] * L[c, qc]
                            G[q, i, 0] = dL[a, qa] * L[b, qb] * L[c, qc]
                            G[q, i, 1] = L[a, qa] * dL[b, qb] * L[c, qc]
                            G[q, i, 2] = L[a, qa] * L[b, qb] * dL[c, qc]
    return N, G, w


def face_tables(k, npts):
    """Shape values on the top face zeta = 1 of the reference cube: Nf[p, i] for the
    npts^2 face Gauss points (x fastest) and weights wf[p]."""
    xq, wq = gauss_rule_01(npts)
    L, _ = lagrange_1d(k, xq)
    Ltop, _ = lagrange_1d(k, np.array([1.0]))
    nb = (k + 1) ** 3
    Nf = np.zeros((npts * npts, nb))
    wf = np.zeros(npts * npts)
    for qb in range(npts):
        for qa in range(npts):
            p = qa + npts * qb
            wf[p] = wq[qa] * wq[qb]
            for c in range(k + 1):
                for b in range(k + 1):
                    for a in range(k + 1):
                        i = a + (k + 1) * (b + (k + 1) * c)
                        Nf[p, i] = L[a, qa] * L[b, qb] * Ltop[c, 0]
    return Nf, wf, xq
