"""Pins of the oracle's step adjoint (the exact transpose of one EXPRK3DS_REAL
step): for the linear model against the assembled step matrix, and for the
nonlinear models against central finite differences of the forward step, in
both the state and the reaction parameters."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

FHN = (0.1, 2.0, -0.1)
SCHNAK = (1000.0, 0.1, 0.9)


def setup(dims, lo, hi, delta, tau):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    As = [[dl * D for D in Ds] for dl in delta]
    return As, O.phi_set(dims, As, tau)


@pytest.mark.parametrize("dims", [(4, 3), (3, 2, 4)])
def test_linear_adjoint_is_transpose_of_assembled_step(dims):
    tau = 2e-3
    As, P = setup(dims, 0.0, 1.0, (1.0, 3.0), tau)
    shape = (2,) + tuple(reversed(dims))
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = O.step(dims, As, P, "linear", (0.0,), tau, e.reshape(shape), 1).ravel()
    rng = np.random.default_rng(3)
    for _ in range(3):
        w = rng.standard_normal(shape)
        got, dp = O.step_adjoint(dims, As, P, "linear", (0.0,), tau, np.zeros(shape), w)
        assert np.allclose(got.ravel(), M.T @ w.ravel(), rtol=0, atol=1e-13 * np.abs(M).max() * n)
        assert np.all(dp == 0.0)


@pytest.mark.parametrize("model,p,dims,lo,hi,delta,tau", [
    ("fhn", FHN, (5, 4, 3), -1.0, 1.0, (1.0, 42.1887), 1e-3),
    ("schnakenberg", SCHNAK, (6, 5), 0.0, 1.0, (1.0, 10.0), 1e-4),
])
def test_nonlinear_adjoint_matches_finite_differences(model, p, dims, lo, hi, delta, tau):
    As, P = setup(dims, lo, hi, delta, tau)
    U = inputs.initial_state(model, dims, seed=4, a=0.1, b=0.9)
    rng = np.random.default_rng(7)
    w = rng.standard_normal(U.shape)
    lam, dp = O.step_adjoint(dims, As, P, model, p, tau, U, w)
    L = lambda UU, pp=p: float(np.sum(O.step(dims, As, P, model, pp, tau, UU, 1) * w))
    # state directions
    for _ in range(3):
        v = rng.standard_normal(U.shape)
        h = 1e-6
        fd = (L(U + h * v) - L(U - h * v)) / (2 * h)
        assert abs(fd - np.sum(lam * v)) <= 1e-6 * max(1.0, abs(fd))
    # reaction parameters (the phi-matrices do not depend on them)
    for q in range(3):
        h = 1e-6 * max(1.0, abs(p[q]))
        pp_p = list(p); pp_p[q] += h
        pp_m = list(p); pp_m[q] -= h
        fd = (L(U, tuple(pp_p)) - L(U, tuple(pp_m))) / (2 * h)
        assert abs(fd - dp[q]) <= 1e-6 * max(1.0, abs(fd)), (q, fd, dp[q])


@pytest.mark.parametrize("model,p,dims,lo,hi,delta,tau", [
    ("fhn", FHN, (5, 4, 3), -1.0, 1.0, (1.0, 42.1887), 1e-3),
    ("schnakenberg", SCHNAK, (6, 5), 0.0, 1.0, (1.0, 10.0), 1e-4),
])
def test_adjoint_diffusion_scaling_matches_finite_differences(model, p, dims, lo, hi, delta, tau):
    """dL/ds_c with A_{c,mu} -> s_c A_{c,mu}: through K and through every
    phi-matrix (dP/ds = phi_{l-1}(Z) - l phi_l(Z)); against central FD of the
    forward step with the phi-set rebuilt at s_c = 1 +- h."""
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    As = [[dl * D for D in Ds] for dl in delta]
    P = O.phi_set(dims, As, tau)
    U = inputs.initial_state(model, dims, seed=4, a=0.1, b=0.9)
    w = np.random.default_rng(8).standard_normal(U.shape)
    _, _, dsc = O.step_adjoint(dims, As, P, model, p, tau, U, w, with_scale=True)
    for c in range(2):
        h = 1e-6
        vals = []
        for sgn in (1, -1):
            sc = [1.0, 1.0]
            sc[c] += sgn * h
            Ash = [[sc[cc] * A for A in As[cc]] for cc in range(2)]
            Ph = O.phi_set(dims, Ash, tau)
            vals.append(float(np.sum(O.step(dims, Ash, Ph, model, p, tau, U, 1) * w)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dsc[c]) <= 1e-6 * max(1.0, abs(fd)), (c, fd, dsc[c])
