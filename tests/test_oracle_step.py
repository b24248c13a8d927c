"""Pins of the oracle's EXPRK3DS_REAL step (Algorithms 1 and 2):
observed third order against the unsplit EXPRK3 with dense phi(tau K),
fourth-order local error of the linear (g = 0) step against expm(tau K),
and invariance of the homogeneous Schnakenberg steady state."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

from tests.dense_ref import exprk3_dense, kron_sum

FHN = (0.1, 2.0, -0.1)
SCHNAK = (1000.0, 0.1, 0.9)


def problem(dims, lo, hi, delta):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    As = [[delta[c] * D for D in Ds] for c in range(2)]
    return As


def split_run(dims, As, model, p, tau, m, U0):
    P = O.phi_set(dims, As, tau)
    return O.step(dims, As, P, model, p, tau, U0, m)


def relerr(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(2))


@pytest.mark.parametrize("dims,ms", [((6, 6, 6), (64, 128, 256)), ((8, 7), (256, 512, 1024)),
                                     ((4, 4, 4, 4), (32, 64, 128))])
def test_observed_order_three(dims, ms):
    """FHN on [-1,1]^d, T = 0.2, U[-1,1) data.  Reference: unsplit EXPRK3 with
    dense phi(tau K) at 8192 steps.  The step counts keep tau * rho(A_v)
    at or below about 3, past the pre-asymptotic regime."""
    delta = (1.0, 42.1887)
    As = problem(dims, -1.0, 1.0, delta)
    U0 = inputs.initial_state("fhn", dims, seed=1)
    T = 0.2
    Ks = [kron_sum(As[c]) for c in range(2)]
    ref = exprk3_dense(U0, Ks, "fhn", FHN, T / 8192, 8192)
    errs = [relerr(split_run(dims, As, "fhn", FHN, T / m, m, U0), ref) for m in ms]
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.8 <= s <= 3.4 for s in slopes), (errs, slopes)


@pytest.mark.parametrize("dims", [(5, 6), (4, 5, 3), (3, 4, 3, 3)])
def test_linear_step_local_error_fourth_order(dims):
    """g = 0: one step is U + tau S_f^{(1)}(K U), a third-order split of
    tau phi_1(tau K) K U = (exp(tau K) - I) U, so the local error is O(tau^4)."""
    delta = (1.0, 3.0)
    As = problem(dims, 0.0, 1.0, delta)
    U0 = inputs.initial_state("fhn", dims, seed=2)
    errs = []
    for tau in (1e-3, 5e-4, 2.5e-4):
        got = split_run(dims, As, "linear", (0.0,), tau, 1, U0)
        ref = np.stack([(sla.expm(tau * kron_sum(As[c])) @ U0[c].ravel()).reshape(U0[c].shape)
                        for c in range(2)])
        errs.append(np.abs(got - ref).max())
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    assert all(13.0 < r < 19.0 for r in ratios), (errs, ratios)


@pytest.mark.parametrize("dims", [(8, 8), (4, 5, 3)])
def test_schnakenberg_equilibrium_is_fixed(dims):
    a, b = SCHNAK[1], SCHNAK[2]
    ue, ve = inputs.schnakenberg_equilibrium(a, b)
    U0 = np.stack([np.full(tuple(reversed(dims)), ue), np.full(tuple(reversed(dims)), ve)])
    As = problem(dims, 0.0, 1.0, (1.0, 10.0))
    got = split_run(dims, As, "schnakenberg", SCHNAK, 1e-3, 5, U0)
    assert np.abs(got - U0).max() < 1e-13


def test_d2_uses_algorithm1_with_two_terms():
    # the d = 2 phi-set has 2 terms (Table 1), the d = 3 one has 3 (Table 3)
    assert O.lib().orc_phi_set_size(2, O._dims((4, 5))) == 2 * 5 * 2 * (16 + 25)
    assert O.lib().orc_phi_set_size(3, O._dims((4, 5, 3))) == 2 * 5 * 3 * (16 + 25 + 9)


def test_phi_set_entries_are_the_named_functions():
    """Spot-check the phi-set layout against phi_{l_i}(c_s tau alpha A) built
    from scipy: slot 2 is P_{i,3}^{(2)}, term 2 uses phi_2 (Algorithm 2)."""
    dims = (4, 5, 3)
    As = problem(dims, -1.0, 1.0, (1.0, 42.1887))
    tau = 1e-3
    P = O.phi_set(dims, As, tau)
    blocks = O.phi_set_blocks(dims, P)
    ell_i, eta, alpha = O.coeffs(3, 2)
    from tests.dense_ref import dense_phi
    for c in range(2):
        for i in range(3):
            for mu in range(3):
                ref = dense_phi(2 * tau / 3 * alpha[i][mu] * As[c][mu], ell_i[i])
                got = blocks[c][2][i][mu]
                assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()
