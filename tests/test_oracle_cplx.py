"""Pins of the oracle's complex variant EXPRK3DS_CPLX (Table 2, Algorithm 1):
the two-term order conditions of Section 2.2 in complex arithmetic, the
complex phi against scipy's expm of augmented matrices, and observed order 3
of the step (real part of each split action) against the unsplit EXPRK3."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

from tests.dense_ref import exprk3_dense, kron_sum

f = math.factorial
FHN = (0.1, 2.0, -0.1)


@pytest.mark.parametrize("d", [2, 3, 4])
@pytest.mark.parametrize("ell", [1, 2])
def test_table2_solves_two_term_system(d, ell):
    eta, alpha = O.coeffs_cplx(d, ell)
    li = (1, 2)
    res = [sum(eta[i] / f(li[i]) ** d for i in range(2)) - 1 / f(ell),
           sum(eta[i] * alpha[i] / (f(li[i]) ** (d - 1) * f(li[i] + 1)) for i in range(2)) - 1 / f(ell + 1),
           sum(eta[i] * alpha[i] ** 2 / (f(li[i]) ** (d - 1) * f(li[i] + 2)) for i in range(2)) - 1 / f(ell + 2),
           sum(eta[i] * alpha[i] ** 2 / (f(li[i]) ** (d - 2) * f(li[i] + 1) ** 2) for i in range(2)) - 2 / f(ell + 2)]
    assert np.max(np.abs(res)) < 1e-13


def test_complex_phi_against_augmented_expm():
    rng = np.random.default_rng(2)
    X = (rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6))) * 3.0 - 4.0 * np.eye(6)
    ph = O.phi_cplx(X, 2)
    n = 6
    M = np.zeros((3 * n, 3 * n), dtype=complex)
    M[:n, :n] = X
    M[:n, n:2 * n] = np.eye(n)
    M[n:2 * n, 2 * n:] = np.eye(n)
    E = sla.expm(M)
    for ell, ref in ((0, E[:n, :n]), (1, E[:n, n:2 * n]), (2, E[:n, 2 * n:])):
        assert np.linalg.norm(ph[ell] - ref) / np.linalg.norm(ref) < 1e-12


@pytest.mark.parametrize("dims,ms", [((6, 6, 6), (64, 128, 256)), ((8, 7), (256, 512, 1024))])
def test_cplx_step_observed_order_three(dims, ms):
    Ds = [inputs.fd_neumann(n, -1.0, 1.0) for n in dims]
    As = [[dl * D for D in Ds] for dl in (1.0, 42.1887)]
    U0 = inputs.initial_state("fhn", dims, seed=1)
    T = 0.2
    ref = exprk3_dense(U0, [kron_sum(As[c]) for c in range(2)], "fhn", FHN, T / 8192, 8192)
    errs = []
    for m in ms:
        P = O.phi_set_cplx(dims, As, T / m)
        got = O.step_cplx(dims, As, P, "fhn", FHN, T / m, U0, m)
        errs.append(max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2)))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.7 <= s <= 3.4 for s in slopes), (errs, slopes)
