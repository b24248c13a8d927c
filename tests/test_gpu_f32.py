"""GPU parity of the FP32 CUDA-core path (DS_PREC_F32) against the FP64
oracle: plain FP32 mode products (FP32 FMA, round to nearest) and FP64 state.
Tolerances follow FP32 rounding: a mode product errs by about n 2^-24 of
sum |a||b| at worst."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ds():
    from paper_2310_07551_gb300 import ds as _ds
    _ds.lib()
    return _ds


@pytest.mark.parametrize("dims", [(70, 65), (33, 70, 9), (64, 48, 40)])
def test_tucker_f32_matches_oracle(ds, dims):
    X = inputs.random_tensor(dims, seed=3)
    Ls = [inputs.random_matrix(n, seed=4, stream=q) for q, n in enumerate(dims)]
    ref = O.tucker(X, Ls)
    scale = O.tucker(np.abs(X), [np.abs(L) for L in Ls])
    got = ds.tucker(torch.from_numpy(X).cuda(), [torch.from_numpy(L).cuda() for L in Ls],
                    precision="f32").cpu().numpy()
    assert np.max(np.abs(got - ref) / scale) < 1e-5


def test_fhn_3d_f32_steps(ds):
    dims = (40, 33, 70)
    Ds = [inputs.fd_neumann(n, -1.0, 1.0) for n in dims]
    As = [[dl * D for D in Ds] for dl in (1.0, 42.1887)]
    U0 = inputs.initial_state("fhn", dims, seed=1)
    ref = O.step(dims, As, O.phi_set(dims, As, 1e-3), "fhn", (0.1, 2.0, -0.1), 1e-3, U0, 3)
    ps = ds.PhiSet(dims, As, 1e-3)
    plan = ds.Plan(ps, "fhn", (0.1, 2.0, -0.1), "f32")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, 3)
    plan.sync(U, check_state=True)
    got = U.cpu().numpy()
    err = max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2))
    print("fhn3d f32 rel err", err)
    assert err < 1e-5
