"""DS_ERR_TIMEOUT: every pipeline wait of the tensor-core kernel is bounded.
The test hook DS_WAIT_LIMIT_CYCLES shortens that bound for the plans created
while it is set, so waits that would complete give up instead: the kernel
records the timeout in the plan's status word, drains its copies and MMAs
(those waits keep the full bound) and returns.  ds_plan_sync reports
DS_ERR_TIMEOUT, and a plan created afterwards on the same device runs clean.
No fault and no hang: the wait that gives up is an ordinary bounded wait."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_07551_gb300 import inputs

pytestmark = pytest.mark.gpu

P = (0.1, 2.0, -0.1)


def test_short_wait_limit_reports_timeout_and_next_plan_is_clean(monkeypatch):
    from paper_2310_07551_gb300 import ds
    ds.lib()
    # a shape no other test uses: the tuner's per-shape choices made under
    # the short limit stay with this shape
    dims = (72, 40, 24)
    Ds = [inputs.fd_neumann(n, -1.0, 1.0) for n in dims]
    As = [[dl * D for D in Ds] for dl in (1.0, 42.1887)]
    U0 = inputs.initial_state("fhn", dims, seed=4)
    ps = ds.PhiSet(dims, As, 1e-3)

    monkeypatch.setenv("DS_WAIT_LIMIT_CYCLES", "200")
    bad = ds.Plan(ps, "fhn", P, "bf16x6")
    monkeypatch.delenv("DS_WAIT_LIMIT_CYCLES")
    U = torch.from_numpy(U0.copy()).cuda()
    bad.integrate(U, 1)
    with pytest.raises(ds.DsError) as e:
        bad.sync()
    assert e.value.status == ds.DS_ERR_TIMEOUT
    assert "gave up" in str(e.value)
    bad.close()

    good = ds.Plan(ps, "fhn", P, "f16x10")
    V = torch.from_numpy(U0.copy()).cuda()
    good.integrate(V, 2)
    good.sync(V, check_state=True)
    ref = O.step(dims, As, O.phi_set(dims, As, 1e-3), "fhn", P, 1e-3, U0, 2)
    got = V.cpu().numpy()
    err = max(np.abs(got[c] - ref[c]).max() / np.abs(ref[c]).max() for c in range(2))
    assert err < 2e-7, err
