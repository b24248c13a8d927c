"""GPU parity of the FP64 path against the CPU oracle, through the C ABI.

Tolerance: <= 1e-12 relative (max-norm) for steps, <= 1e-13 for single
operators.  Sizes span several 64x64 tiles and ragged tails."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_07551_gb300 import configs, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    from paper_2310_07551_gb300 import ds as _ds
    _ds.lib()
    return _ds


def problem(dims, lo, hi, delta):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    return [[delta[c] * D for D in Ds] for c in range(2)]


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("dims,tau", [((64, 64), 1e-3), ((24, 20, 16), 1e-3), ((70, 33), 1e-4),
                                      ((12, 10, 9, 7), 1e-3)])
def test_phi_setup_matches_oracle(ds, dims, tau):
    As = problem(dims, -1.0, 1.0, (1.0, 42.1887))
    ref = O.phi_set_blocks(dims, O.phi_set(dims, As, tau))
    ps = ds.PhiSet(dims, As, tau)
    k = 2 if len(dims) == 2 else 3
    worst = 0.0
    for c in range(2):
        for q in range(5):
            for i in range(k):
                for mu in range(len(dims)):
                    got = ps.get(c, q, i, mu)
                    worst = max(worst, relmax(got, ref[c][q][i][mu]))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("dims", [(70, 65), (33, 70, 9), (128, 64, 40), (2, 3, 5), (17, 9, 12, 6)])
@pytest.mark.parametrize("transpose", [0, 1])
def test_tucker_f64_matches_oracle(ds, dims, transpose):
    X = inputs.random_tensor(dims, seed=3)
    Ls = [inputs.random_matrix(n, seed=4, stream=q) for q, n in enumerate(dims)]
    ref = O.tucker(X, [L.T if transpose else L for L in Ls])
    got = ds.tucker(torch.from_numpy(X).cuda(), [torch.from_numpy(L).cuda() for L in Ls],
                    transpose=bool(transpose)).cpu().numpy()
    assert relmax(got, ref) < 1e-13


def test_kronsum_matches_oracle(ds):
    dims = (40, 33, 17)
    As = problem(dims, 0.0, 1.0, (1.0, 3.0))
    ps = ds.PhiSet(dims, As, 1e-3)
    X = inputs.random_tensor(dims, seed=5)
    for c in range(2):
        got = ps.kronsum(c, torch.from_numpy(X).cuda()).cpu().numpy()
        ref = O.kronsum(X, As[c])
        assert relmax(got, ref) < 1e-13


def run_both(ds, dims, lo, hi, delta, model, p, tau, U0, m, integrate=True):
    As = problem(dims, lo, hi, delta)
    ref = O.step(dims, As, O.phi_set(dims, As, tau), model, p, tau, U0, m)
    ps = ds.PhiSet(dims, As, tau)
    plan = ds.Plan(ps, model, p, "f64")
    U = torch.from_numpy(U0.copy()).cuda()
    if integrate:
        plan.integrate(U, m)
    else:
        for _ in range(m):
            plan.step(U)
    plan.sync(U, check_state=True)
    return U.cpu().numpy(), ref, plan


def test_schnakenberg_64_full_horizon(ds):
    """Tolerance: max(1e-12, 10 x the oracle's FP64 floor), the floor being the
    difference between the oracle run with ascending and with descending
    summation in every mode product (Turing-unstable growth amplifies
    rounding over the horizon)."""
    w = configs.WORKLOADS["schnak2d_64"]
    U0 = inputs.initial_state("schnakenberg", w.dims, seed=w.seed)
    got, ref, _ = run_both(ds, w.dims, w.lo, w.hi, w.delta, "schnakenberg", w.params, w.tau, U0, w.steps)
    floor, _ = O.noise_floor(w.dims, problem(w.dims, w.lo, w.hi, w.delta), "schnakenberg", w.params,
                             w.tau, U0, w.steps)
    errs = [relmax(got[c], ref[c]) for c in range(2)]
    assert max(errs) <= max(1e-12, 10 * floor), (errs, floor)


@pytest.mark.parametrize("dims", [(20, 18, 16), (33, 9, 70), (12, 10, 9, 7)])
def test_fhn_3d_steps(ds, dims):
    U0 = inputs.initial_state("fhn", dims, seed=1)
    got, ref, plan = run_both(ds, dims, -1.0, 1.0, (1.0, 42.1887), "fhn", (0.1, 2.0, -0.1), 1e-3, U0, 5)
    assert max(relmax(got[c], ref[c]) for c in range(2)) < 1e-12
    assert plan.kernels_per_step > 0


def test_step_and_integrate_agree_bitwise(ds):
    dims = (24, 17)
    U0 = inputs.initial_state("schnakenberg", dims, seed=2)
    a, _, _ = run_both(ds, dims, 0.0, 1.0, (1.0, 10.0), "schnakenberg", (1000.0, 0.1, 0.9), 1e-3, U0, 3, True)
    b, _, _ = run_both(ds, dims, 0.0, 1.0, (1.0, 10.0), "schnakenberg", (1000.0, 0.1, 0.9), 1e-3, U0, 3, False)
    assert np.array_equal(a, b)


def test_linear_model_and_dense_A(ds):
    """Non-tridiagonal A takes the dense mode-product route for K."""
    dims = (9, 7)
    As = [[inputs.random_matrix(n, seed=6, stream=10 * c + q, scale=3.0) for q, n in enumerate(dims)]
          for c in range(2)]
    U0 = inputs.initial_state("fhn", dims, seed=3)
    tau = 1e-3
    ref = O.step(dims, As, O.phi_set(dims, As, tau), "linear", (0.0,), tau, U0, 4)
    ps = ds.PhiSet(dims, As, tau)
    plan = ds.Plan(ps, "linear", (0.0,), "f64")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, 4)
    plan.sync()
    assert relmax(U.cpu().numpy(), ref) < 1e-12


def test_invalid_arguments(ds):
    dims = (8, 8)
    As = problem(dims, 0.0, 1.0, (1.0, 10.0))
    with pytest.raises(ds.DsError) as e:
        ds.PhiSet(dims, As, -1.0)
    assert e.value.status == ds.DS_ERR_INVALID_ARG
    bad = [[A.copy() for A in row] for row in As]
    bad[1][0][2, 2] = np.nan
    with pytest.raises(ds.DsError) as e:
        ds.PhiSet(dims, bad, 1e-3)
    assert e.value.status == ds.DS_ERR_NONFINITE
    ps = ds.PhiSet(dims, As, 1e-3)
    with pytest.raises(ds.DsError) as e:
        ds.Plan(ps, "schnakenberg", (1000.0, 0.1, float("inf")))
    assert e.value.status == ds.DS_ERR_INVALID_ARG


def test_nonfinite_state_is_reported(ds):
    dims = (8, 8)
    As = problem(dims, 0.0, 1.0, (1.0, 10.0))
    ps = ds.PhiSet(dims, As, 1e-3)
    plan = ds.Plan(ps, "schnakenberg", (1000.0, 0.1, 0.9))
    U = torch.from_numpy(inputs.initial_state("schnakenberg", dims, seed=1)).cuda()
    U[0, 3, 3] = float("nan")
    plan.step(U)
    with pytest.raises(ds.DsError) as e:
        plan.sync(U, check_state=True)
    assert e.value.status == ds.DS_ERR_NONFINITE
