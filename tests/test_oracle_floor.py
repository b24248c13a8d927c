"""FP64 rounding floor of the oracle on the 64^2 Schnakenberg workload (100
steps): the same computation with every mode-product sum taken in ascending
and in descending order.  The Turing instability amplifies rounding (linear
growth rate ~57/s at these parameters, e^5.7 over T = 0.1), so the floor is
measured, not assumed; it bounds how closely any FP64 implementation can
track the oracle."""
import numpy as np

from oracle import oracle as O
from paper_2310_07551_gb300 import configs, inputs


def test_schnakenberg_64_floor():
    w = configs.WORKLOADS["schnak2d_64"]
    Ds = [inputs.fd_neumann(n, w.lo, w.hi) for n in w.dims]
    As = [[dl * D for D in Ds] for dl in w.delta]
    U0 = inputs.initial_state("schnakenberg", w.dims, seed=w.seed)
    floor, a = O.noise_floor(w.dims, As, "schnakenberg", w.params, w.tau, U0, w.steps)
    print("FP64 floor, Schnakenberg 64^2, 100 steps:", floor)
    # a reordering changes the result (the switch is live) but only at rounding level
    assert 0.0 < floor < 1e-12
    # the default order is restored afterwards
    P = O.phi_set(w.dims, As, w.tau)
    b = O.step(w.dims, As, P, "schnakenberg", w.params, w.tau, U0, w.steps)
    assert np.array_equal(a, b)
