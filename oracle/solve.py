"""Dense LU and restarted GMRES (oracle; test infrastructure).

Sec. 5.1 solves the CFIE systems by GMRES restarted after 30 iterations.  Here: x0 = 0, no
preconditioner, modified Gram-Schmidt Arnoldi, Givens rotations on the Hessenberg matrix, stop when
||b - A x||_2 <= tol ||b||_2 (the residual estimate of the least-squares problem, checked against
the true residual at every restart).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def lu_solve(A, b):
    return scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), b)


def gmres(matvec, b, tol=1e-8, restart=30, max_iter=1000):
    """Restarted GMRES for one right-hand side.  Returns (x, iterations, relative residual)."""
    b = np.asarray(b, dtype=complex)
    n = b.shape[0]
    x = np.zeros(n, dtype=complex)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    it = 0
    r = b.copy()
    beta = np.linalg.norm(r)
    while it < max_iter:
        V = np.zeros((restart + 1, n), dtype=complex)
        H = np.zeros((restart + 1, restart), dtype=complex)
        cs = np.zeros(restart, dtype=complex)
        sn = np.zeros(restart, dtype=complex)
        g = np.zeros(restart + 1, dtype=complex)
        V[0] = r / beta
        g[0] = beta
        j_used = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + np.conj(cs[i]) * H[i + 1, j]
                H[i, j] = t
            a, c = H[j, j], H[j + 1, j]
            den = np.sqrt(abs(a) ** 2 + abs(c) ** 2)
            # rotation [[c, s], [-conj(s), conj(c)]] with c = conj(a)/den, s = conj(b)/den maps
            # (a, b) to (den, 0)
            cs[j] = np.conj(a) / den if den else 1.0
            sn[j] = np.conj(c) / den if den else 0.0
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_used = j + 1
            if abs(g[j + 1]) <= tol * bnorm or it >= max_iter:
                break
        y = scipy.linalg.solve_triangular(H[:j_used, :j_used], g[:j_used])
        x = x + V[:j_used].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bnorm:
            break
    return x, it, beta / bnorm
