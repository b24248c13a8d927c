"""Pins of the oracle's mu-mode product, Tucker operator and Kronecker-sum
action against explicit Kronecker matrices (Section 2 eq. krontomu and
Section 2.4 eq. kronsumv), and of the exactness of the Tucker form of
exp(tau K) (Section 2 eq. expTucker) against dense expm of the assembled K."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

from tests.test_oracle_coeffs import kron_sum


def vec(T):
    # mode-1-fastest storage is already column-stacking order
    return np.ascontiguousarray(T).ravel()


def kron_chain(Ls):
    """L_d (x) ... (x) L_1 for Ls = [L_1, ..., L_d]."""
    M = np.ones((1, 1))
    for L in Ls:
        M = np.kron(L, M)
    return M


DIMS = [(2, 3), (5, 4), (3, 4, 2), (4, 2, 5), (2, 3, 2, 3)]


@pytest.mark.parametrize("dims", DIMS)
def test_mode_product_equals_kronecker_with_identities(dims):
    X = inputs.random_tensor(dims, seed=1)
    for mu in range(1, len(dims) + 1):
        L = inputs.random_matrix(dims[mu - 1], seed=2, stream=mu)
        Ls = [L if nu == mu - 1 else np.eye(dims[nu]) for nu in range(len(dims))]
        ref = kron_chain(Ls) @ vec(X)
        got = vec(O.mode_product(X, mu, L))
        assert np.max(np.abs(got - ref)) < 1e-14 * max(1, np.abs(ref).max()) * dims[mu - 1]


@pytest.mark.parametrize("dims", DIMS)
def test_tucker_equals_kronecker_product(dims):
    X = inputs.random_tensor(dims, seed=4)
    Ls = [inputs.random_matrix(n, seed=5, stream=q) for q, n in enumerate(dims)]
    ref = kron_chain(Ls) @ vec(X)
    got = vec(O.tucker(X, Ls))
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()


def test_tucker_transposed_order_matters():
    # a swapped Kronecker order must not pass: guards the mode/index convention
    dims = (3, 4)
    X = inputs.random_tensor(dims, seed=4)
    L1 = inputs.random_matrix(3, seed=5, stream=0)
    L2 = inputs.random_matrix(4, seed=5, stream=1)
    ref = kron_chain([L1, L2]) @ vec(X)
    wrong = np.kron(L1, L2) @ vec(X)
    got = vec(O.tucker(X, [L1, L2]))
    assert np.allclose(got, ref) and not np.allclose(got, wrong)


@pytest.mark.parametrize("dims", DIMS)
def test_kronsum_equals_assembled_K(dims):
    X = inputs.random_tensor(dims, seed=6)
    As = [inputs.random_matrix(n, seed=7, stream=q) for q, n in enumerate(dims)]
    K = kron_sum(As)
    ref = K @ vec(X)
    got = vec(O.kronsum(X, As))
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("dims", [(6, 5), (4, 5, 3)])
def test_exp_tucker_is_exact(dims):
    """exp(tau K) v = vec(V x_1 exp(tau A_1) ... x_d exp(tau A_d)), with the
    small exponentials from the oracle's phi_0 and the big one from scipy."""
    tau = 0.7e-2
    As = [inputs.fd_neumann(n, 0.0, 1.0) * (1.0 + q) for q, n in enumerate(dims)]
    X = inputs.random_tensor(dims, seed=8)
    Es = [O.phi(tau * A, 0)[0] for A in As]
    got = vec(O.tucker(X, Es))
    ref = sla.expm(tau * kron_sum(As)) @ vec(X)
    assert np.max(np.abs(got - ref)) < 1e-13 * np.abs(ref).max()
