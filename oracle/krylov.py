"""Textbook Krylov solvers and preconditioners in fp64 (Appendix B: preconditioned CG for
symmetric and GMRES for nonsymmetric systems, after Saad, Iterative Methods for Sparse
Linear Systems, 2nd ed.).  Every routine takes the operator as a callable v -> A v.

Readings: the stopping rule is ||b - A x_k||_2 <= tol ||b||_2 with x_0 = 0 (GMRES with
right preconditioning, so its Arnoldi residual estimate is the unpreconditioned residual);
Chebyshev acceleration of Jacobi follows Saad's Algorithm 12.1 with ``degree`` operator
applications; lambda_max of D^-1 A comes from Lanczos on the symmetric D^-1/2 A D^-1/2.
"""
import numpy as np


def jacobi(diag):
    inv = 1.0 / diag
    return lambda r: inv * r


def cg(A, b, M=None, tol=1e-10, maxit=10000):
    """Preconditioned conjugate gradients (Saad Algorithm 9.1).  Convergence is confirmed on the
    true residual b - A x.  Returns x, iterations, ||b - A x||/||b||."""
    M = M or (lambda r: r)
    x = np.zeros_like(b)
    r = b.copy()
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    z = M(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        Ap = A(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        rn = np.linalg.norm(r)
        if rn <= tol * bn:
            # confirm with the true residual; restart from it if the recursion drifted
            r = b - A(x)
            rn = np.linalg.norm(r)
            if rn <= tol * bn:
                return x, it, rn / bn
            z = M(r)
            p = z.copy()
            rz = r @ z
            continue
        z = M(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, np.linalg.norm(r) / bn


def gmres(A, b, M=None, restart=50, tol=1e-10, maxit=5000):
    """Restarted GMRES(m) with right preconditioning, modified Gram-Schmidt and Givens
    rotations (Saad Algorithms 6.9/9.5).  Returns x, iterations, ||b - A x||/||b||."""
    M = M or (lambda r: r)
    n = b.size
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0, 0.0
    it = 0
    while it < maxit:
        r = b - A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bn:
            return x, it, beta / bn
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        Hm = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(restart):
            Z[j] = M(V[j])
            w = A(Z[j])
            for i in range(j + 1):
                Hm[i, j] = w @ V[i]
                w = w - Hm[i, j] * V[i]
            Hm[j + 1, j] = np.linalg.norm(w)
            if Hm[j + 1, j] != 0.0:
                V[j + 1] = w / Hm[j + 1, j]
            for i in range(j):
                t = cs[i] * Hm[i, j] + sn[i] * Hm[i + 1, j]
                Hm[i + 1, j] = -sn[i] * Hm[i, j] + cs[i] * Hm[i + 1, j]
                Hm[i, j] = t
            den = np.hypot(Hm[j, j], Hm[j + 1, j])
            cs[j], sn[j] = Hm[j, j] / den, Hm[j + 1, j] / den
            Hm[j, j] = den
            Hm[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * bn or it >= maxit:
                break
        y = np.linalg.solve(np.triu(Hm[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ y
    r = b - A(x)
    return x, it, np.linalg.norm(r) / bn


def chebyshev(A, diag, lam_min, lam_max, degree):
    """Chebyshev acceleration of the Jacobi iteration for A z = r from z_0 = 0 on the
    interval [lam_min, lam_max] of D^-1 A (Saad Algorithm 12.1), ``degree`` applications of A.
    Returns the preconditioner r -> z."""
    inv = 1.0 / diag
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    sigma = theta / delta

    def apply(r):
        rho = 1.0 / sigma
        d = inv * r / theta
        z = np.zeros_like(r)
        res = r.copy()
        for _ in range(degree):
            z = z + d
            res = res - A(d)
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (inv * res)
            rho = rho_new
        return z + d
    return apply


def lanczos_lambda_max(A, diag, v0, steps=20):
    """Largest Ritz value of D^-1/2 A D^-1/2 after ``steps`` Lanczos steps from v0."""
    s = 1.0 / np.sqrt(diag)
    op = lambda v: s * A(s * v)
    v = v0 / np.linalg.norm(v0)
    v_prev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(steps):
        w = op(v) - beta * v_prev
        alpha = w @ v
        w = w - alpha * v
        alphas.append(alpha)
        beta = np.linalg.norm(w)
        if beta == 0.0:
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:m - 1], 1) + np.diag(betas[:m - 1], -1)
    return float(np.linalg.eigvalsh(T)[-1])
