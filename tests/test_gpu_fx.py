"""GPU parity of the DS_PREC_F16X10 path (fixed-head FP16 operands on the
tensor cores for the Tucker group on F) against the FP64 oracle, through the
C ABI.

Error model: a tensor (or a phi-matrix row) is held as four FP16 parts
with a fixed-point head, 2^E (h + s1 + s2 + s3): the representation keeps
~2^-35 of the tensor's (row's) largest entry.  Head-by-head products are
summed exactly in FP32 (multiples of 256 below 2^32); the other nine
products go to three more accumulators by weight class, so the tensor
core's truncating accumulation acts on small partial sums only.  A Tucker
operator therefore errs by ~2^-33 of the Tucker operator of the absolute
values, and a step by ~1e-9..1e-8 of the state: the tolerances below are
stated from that, well inside the workload target of 1e-6 relative (maximum
norm, per component)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_07551_gb300 import configs, inputs

pytestmark = pytest.mark.gpu

FHN_P = (0.1, 2.0, -0.1)
FHN_DELTA = (1.0, 42.1887)
SCHNAK_P = (1000.0, 0.1, 0.9)


@pytest.fixture(scope="module")
def ds():
    from paper_2310_07551_gb300 import ds as _ds
    _ds.lib()
    return _ds


def problem(dims, lo, hi, delta):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    return [[delta[c] * D for D in Ds] for c in range(2)]


def relmax(a, b):
    return max(np.abs(a[c] - b[c]).max() / np.abs(b[c]).max() for c in range(2))


SHAPES = [(64, 64), (136, 40), (32, 24, 16), (64, 48, 40), (40, 33, 70), (256, 256), (96, 72, 20),
          (24, 16, 12, 10)]


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("transpose", [0, 1])
def test_tucker_f16x10_matches_oracle(ds, dims, transpose):
    X = inputs.random_tensor(dims, seed=11)
    Ls = [inputs.random_matrix(n, seed=12, stream=q) for q, n in enumerate(dims)]
    Lu = [L.T if transpose else L for L in Ls]
    ref = O.tucker(X, Lu)
    scale = O.tucker(np.abs(X), [np.abs(L) for L in Lu])
    got = ds.tucker(torch.from_numpy(X).cuda(), [torch.from_numpy(L).cuda() for L in Ls],
                    transpose=bool(transpose), precision="f16x10").cpu().numpy()
    err = np.max(np.abs(got - ref) / scale)
    print("tucker f16x10", dims, transpose, err)
    assert err < 2e-8, err


def test_tucker_f16x10_is_far_more_accurate_than_bf16x6(ds):
    """Same operands: the FX operator's error is at least 100 times below the
    split-BF16 one (2^-35-class operands and exact head accumulation against
    24-bit operands with truncating FP32 accumulation)."""
    dims = (256, 256)
    X = inputs.random_tensor(dims, seed=13)
    Ls = [inputs.random_matrix(n, seed=14, stream=q) for q, n in enumerate(dims)]
    ref = O.tucker(X, Ls)
    scale = O.tucker(np.abs(X), [np.abs(L) for L in Ls])
    Xd, Ld = torch.from_numpy(X).cuda(), [torch.from_numpy(L).cuda() for L in Ls]
    e_fx = np.max(np.abs(ds.tucker(Xd, Ld, precision="f16x10").cpu().numpy() - ref) / scale)
    e_bf = np.max(np.abs(ds.tucker(Xd, Ld, precision="bf16x6").cpu().numpy() - ref) / scale)
    print("f16x10", e_fx, "bf16x6", e_bf)
    assert e_fx * 100 < e_bf, (e_fx, e_bf)


def run(ds, dims, lo, hi, delta, model, p, tau, U0, m, precision="f16x10"):
    As = problem(dims, lo, hi, delta)
    ref = O.step(dims, As, O.phi_set(dims, As, tau), model, p, tau, U0, m)
    ps = ds.PhiSet(dims, As, tau)
    plan = ds.Plan(ps, model, p, precision)
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, m)
    plan.sync(U, check_state=True)
    return U.cpu().numpy(), ref


@pytest.mark.parametrize("precision", ["f16x10", "f16x13"])
@pytest.mark.parametrize("dims,m", [((32, 24, 16), 5), ((40, 33, 70), 3), ((64, 48, 40), 3), ((96, 72, 20), 2)])
def test_fhn_3d_f16x10_step_matches_oracle(ds, dims, m, precision):
    """White-noise FHN data (the stiff case where FP32-class contractions err
    by ~1e-5): the FX F group brings the step to the 1e-8 class (f16x13:
    every group FX, double-float stages)."""
    U0 = inputs.initial_state("fhn", dims, seed=1)
    got, ref = run(ds, dims, -1.0, 1.0, FHN_DELTA, "fhn", FHN_P, 1e-3, U0, m, precision)
    err = relmax(got, ref)
    print("fhn3d", precision, "rel err", dims, err)
    assert err < 2e-7, err


@pytest.mark.parametrize("precision", ["f16x10", "f16x13"])
@pytest.mark.parametrize("dims,m", [((64, 64), 20), ((136, 40), 10)])
def test_schnakenberg_2d_f16x10_step_matches_oracle(ds, dims, m, precision):
    U0 = inputs.initial_state("schnakenberg", dims, seed=1)
    got, ref = run(ds, dims, 0.0, 1.0, (1.0, 10.0), "schnakenberg", SCHNAK_P, 1e-4, U0, m, precision)
    err = relmax(got, ref)
    print("schnak2d", precision, "rel err", dims, err)
    assert err < 1e-7, err


def test_f16x10_calibration_is_per_state_and_deterministic(ds):
    """ds_integrate on one state in two calls equals one call (the scales
    carry over between calls on the same state), and ds_step on a second
    state, which recalibrates at its first step, gives the same bits as
    ds_integrate on the first."""
    dims = (40, 33, 70)
    As = problem(dims, -1.0, 1.0, FHN_DELTA)
    U0 = inputs.initial_state("fhn", dims, seed=2)
    ps = ds.PhiSet(dims, As, 1e-3)
    plan = ds.Plan(ps, "fhn", FHN_P, "f16x10")
    A = torch.from_numpy(U0.copy()).cuda()
    B = torch.from_numpy(U0.copy()).cuda()
    C = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(A, 4)
    plan.integrate(B, 2)
    plan.integrate(B, 2)
    for _ in range(4):
        plan.step(C)
    plan.sync()
    assert torch.equal(A, B)
    assert torch.equal(A, C)


def test_f16x10_reports_a_tensor_that_outgrew_its_scale(ds):
    """Scales come from the previous step on the same state; a state scaled
    by 4096 in place between calls puts F far beyond the FP16 range of its
    parts (which allows ~32x growth), and ds_plan_sync reports it
    (DS_ERR_NONFINITE).  A new state pointer recalibrates and runs clean."""
    dims = (32, 24, 16)
    As = problem(dims, -1.0, 1.0, FHN_DELTA)
    U0 = inputs.initial_state("fhn", dims, seed=3)
    ps = ds.PhiSet(dims, As, 1e-3)
    plan = ds.Plan(ps, "fhn", FHN_P, "f16x10")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, 1)
    plan.sync()
    U.mul_(4096.0)
    plan.integrate(U, 1)
    with pytest.raises(ds.DsError) as e:
        plan.sync()
    assert e.value.status == ds.DS_ERR_NONFINITE
    V = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(V, 2)
    plan.sync(V, check_state=True)


def test_f16x10_plan_rejects_d4(ds):
    dims = (16, 12, 10, 9)
    As = problem(dims, -1.0, 1.0, FHN_DELTA)
    ps = ds.PhiSet(dims, As, 1e-3)
    with pytest.raises(ds.DsError) as e:
        ds.Plan(ps, "fhn", FHN_P, "f16x10")
    assert e.value.status == ds.DS_ERR_UNSUPPORTED


def test_f16x10_settling_state_keeps_its_range(ds):
    """Instance 36 of the 64-instance Schnakenberg workload (128 x 256):
    as the state settles, max |F| falls by ~1e5 and then, at step ~362,
    grows 65-fold within one step (where the maximum moves).  The exponent
    floor keeps every FX tensor in range: 1500 steps run without an overflow
    report and stay within 1e-6 of the FP64 path."""
    inst = configs.batch_instances()[36]
    Ds = [inputs.fd_neumann(n, 0.0, 1.0) for n in inst.dims]
    As = [[dl * D for D in Ds] for dl in inst.delta]
    ps = ds.PhiSet(inst.dims, As, inst.tau)
    U0 = inputs.initial_state("schnakenberg", inst.dims, seed=7 + 36, a=inst.params[1], b=inst.params[2])
    pfx = ds.Plan(ps, "schnakenberg", inst.params, "f16x10")
    p64 = ds.Plan(ps, "schnakenberg", inst.params, "f64")
    Ua = torch.from_numpy(U0.copy()).cuda()
    Ub = torch.from_numpy(U0.copy()).cuda()
    pfx.integrate(Ua, 1500)
    p64.integrate(Ub, 1500)
    pfx.sync(Ua, check_state=True)
    p64.sync(Ub, check_state=True)
    err = max(float((Ua[c] - Ub[c]).abs().max() / Ub[c].abs().max()) for c in range(2))
    print("settling schnakenberg f16x10 vs f64 at step 1500", err)
    assert err <= 1e-6, err
