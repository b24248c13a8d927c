"""Edge cases of the GPU paths: zero steps, the homogeneous steady state,
the smallest grids the tensor-core path accepts (n_mu = 8), and a long,
narrow problem (n_1 = 256, n_2 = 8: few output tiles, where the autotuner
considers split-K and narrow tiles)."""
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


@pytest.mark.parametrize("precision", ["f64", "bf16x6", "bf16x6c", "f32"])
def test_zero_steps_leave_the_state_untouched(ds, precision):
    dims = (16, 8, 8)
    ps = ds.PhiSet(dims, problem(dims, -1.0, 1.0, (1.0, 42.1887)), 1e-3)
    plan = ds.Plan(ps, "fhn", FHN, precision)
    U0 = torch.from_numpy(inputs.initial_state("fhn", dims, seed=1)).cuda()
    U = U0.clone()
    plan.integrate(U, 0)
    plan.sync()
    assert torch.equal(U, U0)
    if precision == "f64":
        ck = plan.integrate_ckpt(U, 0, 5)
        plan.sync()
        assert ck.shape[0] == 0 and torch.equal(U, U0)


@pytest.mark.parametrize("precision,tol", [("f64", 1e-13), ("bf16x6", 1e-9), ("bf16x6c", 1e-9), ("f32", 1e-6)])
def test_homogeneous_steady_state_stays_fixed(ds, precision, tol):
    """(a + b, b / (a + b)^2) is a fixed point: K u = 0 for a constant field
    (rows of the Neumann matrices sum to 0) and g vanishes there."""
    dims = (24, 16)
    a, b = SCHNAK[1], SCHNAK[2]
    ue, ve = inputs.schnakenberg_equilibrium(a, b)
    U0 = np.stack([np.full((16, 24), ue), np.full((16, 24), ve)])
    ps = ds.PhiSet(dims, problem(dims, 0.0, 1.0, (1.0, 10.0)), 1e-3)
    plan = ds.Plan(ps, "schnakenberg", SCHNAK, precision)
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, 10)
    plan.sync(U, check_state=True)
    assert np.abs(U.cpu().numpy() - U0).max() < tol


@pytest.mark.parametrize("dims", [(8, 8), (8, 8, 8), (8, 8, 8, 8)])
@pytest.mark.parametrize("precision", ["bf16x6", "bf16x6c", "f16x10"])
def test_smallest_tensor_core_grids(ds, dims, precision):
    """One tile, mostly padding.  Bounds: 2e-5, the FP32-class per-config
    bound of the split-BF16 precisions on white-noise FHN data (not the
    workloads' 1e-6 target); 2e-7 for f16x10 (d <= 3)."""
    if precision == "f16x10" and len(dims) > 3:
        pytest.skip("DS_PREC_F16X10 plans take d = 2 or 3")
    As = problem(dims, -1.0, 1.0, (1.0, 5.0))
    U0 = inputs.initial_state("fhn", dims, seed=2)
    tau, m = 1e-3, 3
    ref = O.step(dims, As, O.phi_set(dims, As, tau), "fhn", FHN, tau, U0, m)
    plan = ds.Plan(ds.PhiSet(dims, As, tau), "fhn", FHN, precision)
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, m)
    plan.sync(U, check_state=True)
    assert relmax(U.cpu().numpy(), ref) < (2e-7 if precision == "f16x10" else 2e-5)


def test_long_narrow_problem(ds):
    """n_1 = 256 with n_2 = 8: few output tiles against a 256-long K; the
    autotuner may split K (deterministic part-ordered reduction)."""
    dims = (256, 8)
    As = problem(dims, 0.0, 1.0, (1.0, 10.0))
    U0 = inputs.initial_state("schnakenberg", dims, seed=3)
    tau, m = 1e-4, 2
    ref = O.step(dims, As, O.phi_set(dims, As, tau), "schnakenberg", SCHNAK, tau, U0, m)
    plan = ds.Plan(ds.PhiSet(dims, As, tau), "schnakenberg", SCHNAK, "bf16x6")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, m)
    plan.sync(U, check_state=True)
    assert relmax(U.cpu().numpy(), ref) < 1e-6
