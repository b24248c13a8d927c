"""GPU parity of the unsplit EXPRK3 (DS_EXPRK3_DENSE: eq. exprk3 with dense
phi(c tau K)) against the oracle's orc_step_dense, and its use as the
reference for the splitting error of EXPRK3DS_REAL."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

pytestmark = pytest.mark.gpu

FHN = (0.1, 2.0, -0.1)
SCHNAK = (1000.0, 0.1, 0.9)


@pytest.fixture(scope="module")
def ds():
    from paper_2310_07551_gb300 import ds as _ds
    _ds.lib()
    return _ds


def problem(dims, lo, hi, delta):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    return [[dl * D for D in Ds] for dl in delta]


def relmax(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(2))


@pytest.mark.parametrize("model,p,dims,lo,hi,delta,tau,m", [
    ("schnakenberg", SCHNAK, (16, 12), 0.0, 1.0, (1.0, 10.0), 1e-3, 5),
    ("fhn", FHN, (9, 7, 6), -1.0, 1.0, (1.0, 42.1887), 1e-3, 4),
    ("fhn", FHN, (5, 4, 3, 3), -1.0, 1.0, (1.0, 5.0), 1e-3, 3),
])
def test_dense_matches_oracle(ds, model, p, dims, lo, hi, delta, tau, m):
    As = problem(dims, lo, hi, delta)
    U0 = inputs.initial_state(model, dims, seed=6)
    ref = O.step_dense(dims, As, model, p, tau, U0, m)
    ps = ds.PhiSet(dims, As, tau, scheme="exprk3_dense")
    plan = ds.Plan(ps, model, p, "f64")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, m)
    plan.sync(U, check_state=True)
    assert relmax(U.cpu().numpy(), ref) < 1e-12


def test_dense_phi_matrix_and_limits(ds):
    dims = (6, 5)
    As = problem(dims, 0.0, 1.0, (1.0, 10.0))
    ps = ds.PhiSet(dims, As, 1e-3, scheme="exprk3_dense")
    P = ps.get(1, 4, 0, 0)                       # phi_2(tau K_v)
    assert P.shape == (30, 30)
    # phi_2(0) = I / 2 and phi_2 of a small matrix is close to it
    assert np.abs(P - 0.5 * np.eye(30)).max() < 0.5
    with pytest.raises(ds.DsError):
        ds.Plan(ps, "schnakenberg", SCHNAK, "bf16x6")
    with pytest.raises(ds.DsError) as e:
        big = (80, 60)
        ds.PhiSet(big, problem(big, 0.0, 1.0, (1.0, 10.0)), 1e-3, scheme="exprk3_dense")
    assert e.value.status == ds.DS_ERR_UNSUPPORTED


def test_splitting_error_measured_online(ds):
    """A dense and a split plan side by side: their difference after m steps
    equals the oracle's (split minus dense) to rounding."""
    dims = (12, 10)
    As = problem(dims, 0.0, 1.0, (1.0, 10.0))
    U0 = inputs.initial_state("schnakenberg", dims, seed=2)
    tau, m = 1e-3, 10
    out = {}
    for scheme in ("exprk3ds_real", "exprk3_dense"):
        ps = ds.PhiSet(dims, As, tau, scheme=scheme)
        plan = ds.Plan(ps, "schnakenberg", SCHNAK, "f64")
        U = torch.from_numpy(U0.copy()).cuda()
        plan.integrate(U, m)
        plan.sync()
        out[scheme] = U.cpu().numpy()
    gpu_diff = out["exprk3ds_real"] - out["exprk3_dense"]
    ref_diff = (O.step(dims, As, O.phi_set(dims, As, tau), "schnakenberg", SCHNAK, tau, U0, m)
                - O.step_dense(dims, As, "schnakenberg", SCHNAK, tau, U0, m))
    scale = np.abs(ref_diff).max()
    assert scale > 0
    assert np.abs(gpu_diff - ref_diff).max() < 1e-6 * scale + 1e-12
