"""Pins of the oracle's ETD2RKDS step (ETD2RK of Section 1 with the
second-order split of eq. secondord): observed order 2 against the unsplit
ETD2RK with dense phi(tau K) (a wrong l!^(d-1) weight drops it to order 1),
and the phi-set's blocks against scipy's expm of augmented matrices."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

from tests.dense_ref import etd2rk_dense, kron_sum

FHN = (0.1, 2.0, -0.1)


def problem(dims, delta):
    Ds = [inputs.fd_neumann(n, -1.0, 1.0) for n in dims]
    return [[dl * D for D in Ds] for dl in delta]


@pytest.mark.parametrize("dims,ms", [((6, 6, 6), (128, 256, 512)), ((8, 7), (256, 512, 1024))])
def test_etd2rkds_observed_order_two(dims, ms):
    As = problem(dims, (1.0, 42.1887))
    U0 = inputs.initial_state("fhn", dims, seed=1)
    T = 0.2
    ref = etd2rk_dense(U0, [kron_sum(As[c]) for c in range(2)], "fhn", FHN, T / 8192, 8192)
    errs = []
    for m in ms:
        P = O.phi_set2(dims, As, T / m)
        got = O.step2(dims, As, P, "fhn", FHN, T / m, U0, m)
        errs.append(max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2)))
    slopes = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(1.8 <= s <= 2.3 for s in slopes), (errs, slopes)


def test_phi_set2_layout_and_values():
    dims = (4, 5, 3)
    As = problem(dims, (1.0, 3.0))
    tau = 1e-2
    P = O.phi_set2(dims, As, tau)
    off = 0
    from tests.dense_ref import dense_phi
    for c in range(2):
        for l in (1, 2):
            for mu, n in enumerate(dims):
                blk = P[off:off + n * n].reshape(n, n).T
                assert np.abs(blk - dense_phi(tau * As[c][mu], l)).max() < 1e-13
                off += n * n
    assert off == P.size
