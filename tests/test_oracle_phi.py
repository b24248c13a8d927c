"""Pins of the oracle's phi_l of small matrices (Section 1 definition,
evaluated by scaling / Taylor / modified squaring) against independent
evaluations: scalar closed forms, eigendecomposition of the symmetrisable
finite-difference matrix, and scipy's expm of an augmented block matrix."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

from tests.test_oracle_coeffs import dense_phi


def scalar_phi(z, ell):
    """phi_ell(z) by closed form, with the (cancellation-free) series for |z| < 1."""
    z = np.asarray(z, dtype=np.float64)
    out = np.empty_like(z)
    small = np.abs(z) < 1.0
    zs = z[small]
    out[small] = sum(zs ** k / math.factorial(k + ell) for k in range(30))
    zb = z[~small]
    if ell == 0:
        out[~small] = np.exp(zb)
    elif ell == 1:
        out[~small] = np.expm1(zb) / zb
    elif ell == 2:
        out[~small] = (np.expm1(zb) - zb) / zb ** 2
    elif ell == 3:
        out[~small] = (np.expm1(zb) - zb - zb ** 2 / 2) / zb ** 3
    return out


def rel(A, B):
    return np.linalg.norm(A - B) / np.linalg.norm(B)


@pytest.mark.parametrize("zmax", [4000.0, 731.5, 12.0, 0.4])
def test_diagonal_matches_scalar_closed_forms(zmax):
    z = np.array([-zmax, -12.0, -1.0, -1e-3, 0.0, 1e-4, 0.3, 0.4])
    z = z[np.abs(z) <= zmax]
    ph = O.phi(np.diag(z), 3)
    # squaring count used for this matrix; each squaring can double the
    # relative error of every entry (the usual scaling-and-squaring bound)
    s = max(0, int(np.ceil(np.log2(2 * np.abs(z).max()))))
    for ell in range(4):
        ref = scalar_phi(z, ell)
        got = np.diag(ph[ell])
        ok = np.abs(ref) > 1e-280
        relerr = np.abs(got - ref)[ok] / np.abs(ref)[ok]
        assert np.max(relerr) <= 16 * 2.0 ** s * 2.2e-16, (ell, np.max(relerr))
        off = ph[ell] - np.diag(np.diag(ph[ell]))
        assert np.max(np.abs(off)) == 0.0


@pytest.mark.parametrize("n,scale", [(16, 1e-3 * 1.3 * 42.19), (64, 1e-3 * 1.6 * 42.19), (64, 1e-4 * 2.5 * 10)])
def test_fd_matrix_eigendecomposition(n, scale):
    """A = scale * D with D the Neumann FD matrix; W^(1/2) D W^(-1/2) is
    symmetric for W = diag(1/2, 1, ..., 1, 1/2), so phi(A) = V phi(L) V^-1
    exactly, with V from eigh."""
    D = inputs.fd_neumann(n, -1.0, 1.0)
    w = np.ones(n)
    w[0] = w[-1] = 0.5
    S = np.sqrt(w)[:, None] * D / np.sqrt(w)[None, :]
    assert np.allclose(S, S.T, rtol=0, atol=1e-9 * np.abs(D).max())
    lam, V = np.linalg.eigh(0.5 * (S + S.T))
    X = scale * D
    ph = O.phi(X, 2)
    for ell in range(3):
        ref = (V * scalar_phi(scale * lam, ell)) @ V.T
        ref = ref / np.sqrt(w)[:, None] * np.sqrt(w)[None, :]
        assert rel(ph[ell], ref) < 1e-13, (ell, rel(ph[ell], ref))


@pytest.mark.parametrize("n,scale", [(5, 0.3), (8, 7.0), (12, 150.0), (20, 300.0)])
def test_random_nonsymmetric_against_augmented_expm(n, scale):
    X = inputs.random_matrix(n, seed=3, stream=n) * scale / n
    X -= scale * 0.5 * np.eye(n)      # bias towards the stable half-plane like tau*A
    ph = O.phi(X, 2)
    for ell in range(3):
        ref = dense_phi(X, ell)
        assert rel(ph[ell], ref) < 1e-12, (ell, rel(ph[ell], ref))


def test_squaring_identity_consistency():
    # phi_l(2Y) from two different scalings must agree (oracle vs itself at a
    # scale where no squaring is needed is checked by the tests above)
    X = inputs.random_matrix(6, seed=9) * 0.1
    a = O.phi(X, 2)
    b = O.phi(2 * X, 2)
    ref1 = 0.5 * (a[0] @ a[1] + a[1])
    ref2 = 0.25 * (a[0] @ a[2] + a[1] + a[2])
    assert rel(b[1], ref1) < 1e-14
    assert rel(b[2], ref2) < 1e-14
