"""GPU parity of the ETD2RKDS scheme (ETD2RK with the second-order split,
FP64) against the oracle: phi-set blocks <= 1e-13, steps <= 1e-12."""
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


@pytest.mark.parametrize("model,p,dims,lo,hi,delta,tau,m", [
    ("schnakenberg", SCHNAK, (64, 64), 0.0, 1.0, (1.0, 10.0), 1e-4, 20),
    ("fhn", FHN, (20, 18, 16), -1.0, 1.0, (1.0, 42.1887), 1e-3, 5),
    ("fhn", FHN, (33, 70), -1.0, 1.0, (1.0, 42.1887), 1e-3, 5),
])
def test_etd2rkds_matches_oracle(ds, model, p, dims, lo, hi, delta, tau, m):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    As = [[dl * D for D in Ds] for dl in delta]
    P = O.phi_set2(dims, As, tau)
    U0 = inputs.initial_state(model, dims, seed=2)
    ref = O.step2(dims, As, P, model, p, tau, U0, m)
    ps = ds.PhiSet(dims, As, tau, scheme="etd2rkds")
    # phi blocks: [c][l-1][mu]
    off = 0
    for c in range(2):
        for slot in range(2):
            for mu, n in enumerate(dims):
                blk = P[off:off + n * n].reshape(n, n).T
                got = ps.get(c, slot, 0, mu)
                assert np.abs(got - blk).max() <= 1e-13 * np.abs(blk).max()
                off += n * n
    plan = ds.Plan(ps, model, p, "f64")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, m)
    plan.sync(U, check_state=True)
    got = U.cpu().numpy()
    assert max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2)) < 1e-12
    assert plan.kernels_per_step == 2 + 2 * 2 * len(dims) + 1


def test_etd2rkds_is_fp64_only(ds):
    dims = (16, 16)
    Ds = [inputs.fd_neumann(n, 0.0, 1.0) for n in dims]
    ps = ds.PhiSet(dims, [[D for D in Ds], [10 * D for D in Ds]], 1e-4, scheme="etd2rkds")
    with pytest.raises(ds.DsError) as e:
        ds.Plan(ps, "schnakenberg", SCHNAK, "bf16x6")
    assert e.value.status == ds.DS_ERR_UNSUPPORTED
