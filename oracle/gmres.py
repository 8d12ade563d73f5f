"""Textbook GMRES (the paper solves Eq. (2.30) with "standard GMRES", Sec. 2.5).

Arnoldi with modified Gram-Schmidt, Givens rotations on the Hessenberg
matrix, x0 = 0, stop when the residual estimate |s_{j+1}| <= tol * |g|
(the paper gives no tolerance or restart; unrestarted unless `restart`).

Parity status: pinned (dense LU solve of the same matrix).
"""
from __future__ import annotations

import numpy as np


def gmres(apply, b, tol=1e-13, max_iter=300, restart=None, x0=None):
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    info = {"iterations": 0, "residuals": [], "converged": False}
    if bnorm == 0.0:
        info["converged"] = True
        return x, info
    m = max_iter if restart is None else min(restart, max_iter)
    total = 0
    while total < max_iter:
        r = b - apply(x) if total > 0 or x0 is not None else b.copy()
        beta = float(np.linalg.norm(r))
        if beta <= tol * bnorm:
            info["converged"] = True
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        s = np.zeros(m + 1)
        s[0] = beta
        V[0] = r / beta
        k_done = 0
        for j in range(m):
            w = apply(V[j])
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                           # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            s[j + 1] = -sn[j] * s[j]
            s[j] = cs[j] * s[j]
            total += 1
            k_done = j + 1
            info["residuals"].append(abs(s[j + 1]) / bnorm)
            if abs(s[j + 1]) <= tol * bnorm or total >= max_iter:
                break
        y = np.zeros(k_done)
        for i in range(k_done - 1, -1, -1):              # back substitution
            y[i] = (s[i] - np.dot(H[i, i + 1:k_done], y[i + 1:k_done])) / H[i, i]
        x = x + V[:k_done].T @ y
        if info["residuals"][-1] <= tol:
            info["converged"] = True
            break
    info["iterations"] = total
    return x, info
