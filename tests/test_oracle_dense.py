"""Pins of the oracle's unsplit EXPRK3 (orc_step_dense: eq. exprk3 with dense
phi(c tau K)) against an independent dense reference (scipy's expm of
augmented block matrices, tests/dense_ref.py), and of its relation to the
split step: the splitting error of EXPRK3DS shrinks like tau^3 per unit time."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

from tests.dense_ref import exprk3_dense, kron_sum

FHN = (0.1, 2.0, -0.1)
SCHNAK = (1000.0, 0.1, 0.9)


def problem(dims, lo, hi, delta):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    return [[dl * D for D in Ds] for dl in delta]


def relmax(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(2))


@pytest.mark.parametrize("model,p,dims,lo,hi,delta,tau,m", [
    ("schnakenberg", SCHNAK, (6, 5), 0.0, 1.0, (1.0, 10.0), 1e-3, 4),
    ("fhn", FHN, (4, 3, 5), -1.0, 1.0, (1.0, 42.1887), 1e-3, 3),
    ("fhn", FHN, (3, 3, 2, 3), -1.0, 1.0, (1.0, 5.0), 1e-3, 2),
])
def test_dense_step_matches_scipy_reference(model, p, dims, lo, hi, delta, tau, m):
    As = problem(dims, lo, hi, delta)
    U0 = inputs.initial_state(model, dims, seed=4)
    got = O.step_dense(dims, As, model, p, tau, U0, m)
    ref = exprk3_dense(U0, [kron_sum(As[c]) for c in range(2)], model, p, tau, m)
    assert relmax(got, ref) < 1e-12


def test_split_error_is_third_order_against_dense():
    """Same step count T / m for both schemes: the split-minus-unsplit
    difference at T falls like m^-3."""
    dims = (6, 5, 4)
    As = problem(dims, -1.0, 1.0, (1.0, 42.1887))
    U0 = inputs.initial_state("fhn", dims, seed=1)
    T = 0.1
    errs = []
    for m in (32, 64, 128):
        tau = T / m
        dense = O.step_dense(dims, As, "fhn", FHN, tau, U0, m)
        split = O.step(dims, As, O.phi_set(dims, As, tau), "fhn", FHN, tau, U0, m)
        errs.append(relmax(split, dense))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(2.6 <= s <= 3.5 for s in slopes), (errs, slopes)
