"""GPU parity of the complex-coefficient scheme EXPRK3DS_CPLX (Table 2,
Algorithm 1; FP64) against the oracle: complex phi blocks <= 1e-13 (via the
real 2n x 2n embedding on the GPU), steps <= 1e-12."""
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
    ("fhn", FHN, (20, 18, 16), -1.0, 1.0, (1.0, 42.1887), 1e-3, 4),
    ("schnakenberg", SCHNAK, (40, 33), 0.0, 1.0, (1.0, 10.0), 1e-4, 10),
])
def test_cplx_matches_oracle(ds, model, p, dims, lo, hi, delta, tau, m):
    Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
    As = [[dl * D for D in Ds] for dl in delta]
    P = O.phi_set_cplx(dims, As, tau)
    ps = ds.PhiSet(dims, As, tau, scheme="exprk3ds_cplx")
    off = 0
    worst = 0.0
    for c in range(2):
        for q in range(5):
            for i in range(2):
                for mu, n in enumerate(dims):
                    blk = P[off:off + n * n].reshape(n, n).T
                    got = ps.get(c, q, i, mu, 0) + 1j * ps.get(c, q, i, mu, 1)
                    worst = max(worst, np.abs(got - blk).max() / np.abs(blk).max())
                    off += n * n
    assert worst < 1e-13, worst
    U0 = inputs.initial_state(model, dims, seed=3)
    ref = O.step_cplx(dims, As, P, model, p, tau, U0, m)
    plan = ds.Plan(ps, model, p, "f64")
    U = torch.from_numpy(U0.copy()).cuda()
    plan.integrate(U, m)
    plan.sync(U, check_state=True)
    got = U.cpu().numpy()
    assert max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2)) < 1e-12
