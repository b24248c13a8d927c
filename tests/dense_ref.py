"""Independent dense references for tiny grids (numpy/scipy only).

* the assembled Kronecker sum K = A_d (+) ... (+) A_1 (Section 1, eq. kronsum),
* phi_l(X) from scipy's expm of an augmented block matrix,
* the unsplit third-order exponential Runge-Kutta scheme EXPRK3 with the
  tableau the paper uses (Section 2.4, eq. exprk3), with dense phi(tau K).
None of this calls the oracle or the CUDA library.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def kron_sum(As):
    ns = [A.shape[0] for A in As]
    N = int(np.prod(ns))
    K = np.zeros((N, N))
    for mu in range(len(As)):
        M = np.ones((1, 1))
        for nu in range(len(As)):
            M = np.kron(As[nu] if nu == mu else np.eye(ns[nu]), M)
        K += M
    return K


def dense_phi(X, ell):
    n = X.shape[0]
    if ell == 0:
        return sla.expm(X)
    M = np.zeros(((ell + 1) * n, (ell + 1) * n))
    M[:n, :n] = X
    for b in range(ell):
        M[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = np.eye(n)
    return sla.expm(M)[:n, ell * n:(ell + 1) * n]


def g_model(model, p, u, v):
    if model == "schnakenberg":
        gam, a, b = p
        return gam * (a - u + u * u * v), gam * (b - u * u * v)
    if model == "fhn":
        eps, a1, a0 = p
        return u - u ** 3 - v, eps * (u - a1 * v - a0)
    if model == "linear":
        return np.zeros_like(u), np.zeros_like(v)
    raise ValueError(model)


def exprk3_dense(U0, Ks, model, p, tau, m):
    """m steps of unsplit EXPRK3 (c2 = 1/3, c3 = 2/3, a32 = 4/3 phi_2(c3 .),
    b2 = 0, b3 = 3/2 phi_2) on the block system [K_1 0; 0 K_2]."""
    shape = U0.shape
    N = U0[0].size
    u = U0.reshape(2, N).copy()
    ph = []
    for K in Ks:
        ph.append({
            "p1_3": dense_phi(tau / 3 * K, 1),
            "p1_23": dense_phi(2 * tau / 3 * K, 1),
            "p2_23": dense_phi(2 * tau / 3 * K, 2),
            "p1_1": dense_phi(tau * K, 1),
            "p2_1": dense_phi(tau * K, 2),
        })

    def g(w):
        return np.stack(g_model(model, p, w[0], w[1]))

    for _ in range(m):
        G = g(u)
        F = np.stack([Ks[c] @ u[c] for c in range(2)]) + G
        u2 = np.stack([u[c] + tau / 3 * ph[c]["p1_3"] @ F[c] for c in range(2)])
        D2 = g(u2) - G
        u3 = np.stack([u[c] + 2 * tau / 3 * ph[c]["p1_23"] @ F[c]
                       + 4 * tau / 3 * ph[c]["p2_23"] @ D2[c] for c in range(2)])
        D3 = g(u3) - G
        u = np.stack([u[c] + tau * ph[c]["p1_1"] @ F[c]
                      + 1.5 * tau * ph[c]["p2_1"] @ D3[c] for c in range(2)])
    return u.reshape(shape)


def etd2rk_dense(U0, Ks, model, p, tau, m):
    """m steps of unsplit ETD2RK (Section 1, eq. ETD2RK) with dense phi(tau K)."""
    shape = U0.shape
    N = U0[0].size
    u = U0.reshape(2, N).copy()
    p1 = [dense_phi(tau * K, 1) for K in Ks]
    p2 = [dense_phi(tau * K, 2) for K in Ks]

    def g(w):
        return np.stack(g_model(model, p, w[0], w[1]))

    for _ in range(m):
        G = g(u)
        F = np.stack([Ks[c] @ u[c] for c in range(2)]) + G
        u2 = np.stack([u[c] + tau * p1[c] @ F[c] for c in range(2)])
        D = g(u2) - G
        u = np.stack([u2[c] + tau * p2[c] @ D[c] for c in range(2)])
    return u.reshape(shape)
