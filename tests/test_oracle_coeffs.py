"""Pins of the oracle's split coefficients (Tables 1 and 3) against facts
other than their closed forms: the order-condition systems of Section 2,
the printed Groebner bases, and third-order behaviour against dense
phi_l(tau K) of an assembled Kronecker sum."""
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")
f = math.factorial


def order_residuals(d, ell, ell_i, eta, alpha, third=False):
    """Residuals of the order conditions for the split
    phi_l(tau sum A_mu) ~ sum_i eta_i (x)_mu phi_{l_i}(alpha_{i,mu} tau A_mu):
    matching the Taylor coefficient of prod_mu A_mu^{k_mu} (Section 2.1
    eq. phi1phi22d, Section 2.2 eq. phi1phi2nd, Section 2.3 eq.
    phi1phi2nd3t and the additional third-order conditions)."""
    k = len(eta)
    res = []
    # degree 0
    res.append(sum(eta[i] / f(ell_i[i]) ** d for i in range(k)) - 1 / f(ell))
    for mu in range(d):
        res.append(sum(eta[i] * alpha[i][mu] / (f(ell_i[i]) ** (d - 1) * f(ell_i[i] + 1))
                       for i in range(k)) - 1 / f(ell + 1))
        res.append(sum(eta[i] * alpha[i][mu] ** 2 / (f(ell_i[i]) ** (d - 1) * f(ell_i[i] + 2))
                       for i in range(k)) - 1 / f(ell + 2))
    for mu in range(d):
        for nu in range(mu + 1, d):
            res.append(sum(eta[i] * alpha[i][mu] * alpha[i][nu]
                           / (f(ell_i[i]) ** (d - 2) * f(ell_i[i] + 1) ** 2)
                           for i in range(k)) - 2 / f(ell + 2))
    if third:
        for mu in range(d):
            res.append(sum(eta[i] * alpha[i][mu] ** 3 / (f(ell_i[i]) ** (d - 1) * f(ell_i[i] + 3))
                           for i in range(k)) - 1 / f(ell + 3))
        for mu in range(d):
            for nu in range(mu + 1, d):
                for xi in range(nu + 1, d):
                    res.append(sum(eta[i] * alpha[i][mu] * alpha[i][nu] * alpha[i][xi]
                                   / (f(ell_i[i]) ** (d - 3) * f(ell_i[i] + 1) ** 3)
                                   for i in range(k)) - 6 / f(ell + 3))
    return np.array(res)


@pytest.mark.parametrize("ell", [1, 2])
def test_table1_real_solves_two_term_2d_system(ell):
    ell_i, eta, alpha = O.coeffs(2, ell)
    assert ell_i == [1, 2]
    r = order_residuals(2, ell, ell_i, eta, alpha)
    assert len(r) == 6
    assert np.max(np.abs(r)) < 1e-14


@pytest.mark.parametrize("d", [3, 4])
@pytest.mark.parametrize("ell", [1, 2])
def test_table3_solves_three_term_system(d, ell):
    ell_i, eta, alpha = O.coeffs(d, ell)
    assert ell_i == [1, 2, 1]
    r = order_residuals(d, ell, ell_i, eta, alpha, third=True)
    assert np.max(np.abs(r)) < 1e-13


def test_table3_a_dropped_factor_fails():
    # sanity of the pin itself: perturbing eta_2 by the 2^(d-3) factor breaks it
    ell_i, eta, alpha = O.coeffs(4, 1)
    eta = eta.copy()
    eta[1] /= 2.0
    r = order_residuals(4, 1, ell_i, eta, alpha, third=True)
    assert np.max(np.abs(r)) > 1e-3


def _groebner():
    rows = []
    with open(os.path.join(GOLD, "groebner_table3.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            ell, const, terms = [s.strip() for s in line.split("|")]
            rows.append((int(ell), float(const),
                         [(float(t.split(":")[0]), t.split(":")[1]) for t in terms.split()]))
    return rows


@pytest.mark.parametrize("ell", [1, 2])
def test_table3_zeros_of_printed_groebner_basis(ell):
    ell_i, eta, alpha = O.coeffs(3, ell)
    env = {"eta1": eta[0], "eta2": eta[1], "eta3": eta[2],
           "a1": alpha[0][0], "a2": alpha[1][0], "a3": alpha[2][0]}
    env["eta3^2"] = eta[2] ** 2
    polys = [p for p in _groebner() if p[0] == ell]
    assert len(polys) == 6
    for _, c0, terms in polys:
        val = c0 + sum(c * env[m] for c, m in terms)
        scale = abs(c0) + sum(abs(c * env[m]) for c, m in terms)
        assert abs(val) / scale < 1e-14
    # all directions share the same alpha for Table 3
    assert np.allclose(alpha, alpha[:, :1])


def dense_phi(X, ell):
    """phi_ell(X) from the exponential of an augmented block matrix:
    exp([[X, I, 0], [0, 0, I], [0, 0, 0]]) has phi_1(X), phi_2(X) in its
    first block row (independent of the oracle)."""
    n = X.shape[0]
    if ell == 0:
        return sla.expm(X)
    M = np.zeros(((ell + 1) * n, (ell + 1) * n))
    M[:n, :n] = X
    for b in range(ell):
        M[b * n:(b + 1) * n, (b + 1) * n:(b + 2) * n] = np.eye(n)
    return sla.expm(M)[:n, ell * n:(ell + 1) * n]


def split_phi_dense(As, tau, ell):
    """Assembled split approximation sum_i eta_i phi(alpha tau A_d) (x) ... (x) phi(alpha tau A_1)."""
    d = len(As)
    ell_i, eta, alpha = O.coeffs(d, ell)
    total = 0
    for i in range(len(eta)):
        M = np.ones((1, 1))
        for mu in range(d):
            # Kronecker order A_d (x) ... (x) A_1: the mode-1 factor is rightmost
            M = np.kron(dense_phi(alpha[i][mu] * tau * As[mu], ell_i[i]), M)
        total = total + eta[i] * M
    return total


def kron_sum(As):
    d = len(As)
    ns = [A.shape[0] for A in As]
    N = int(np.prod(ns))
    K = np.zeros((N, N))
    for mu in range(d):
        M = np.ones((1, 1))
        for nu in range(d):
            M = np.kron(As[nu] if nu == mu else np.eye(ns[nu]), M)
        K += M
    return K


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("ell", [1, 2])
def test_split_is_third_order(d, ell):
    rng = np.random.default_rng(5 + d + ell)
    As = [rng.standard_normal((3, 3)) for _ in range(d)]
    K = kron_sum(As)
    errs = []
    # d = 4 sums four random directions: halve tau to stay past the pre-asymptotic range
    taus = [0.1, 0.05, 0.025] if d < 4 else [0.05, 0.025, 0.0125]
    for tau in taus:
        E = split_phi_dense(As, tau, ell) - dense_phi(tau * K, ell)
        errs.append(np.linalg.norm(E, 2))
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(7.0 < r < 9.5 for r in ratios), ratios
