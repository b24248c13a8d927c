"""GPU adjoint step (ds_step_backward) and the checkpointed autograd horizon.

* one adjoint step against the oracle's adjoint (<= 1e-12 relative), for the
  stencil (tridiagonal A) and the dense-A routes, d = 2 and 3;
* the differentiation workload: FHN 96^3, FP64, 200 steps, checkpoints every
  20 steps; loss = mean squared mismatch of u_T against a target made by the
  forward solver with hidden (delta_v, eps, alpha0) = nominal x (1.05, 0.9,
  1.2); gradients w.r.t. delta_v (through K and every phi-matrix), eps,
  alpha0 and the initial state (3 seeded directions) against central finite
  differences, h = 1e-6; one adjoint step, including d/d delta, against the
  oracle's adjoint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2310_07551_gb300 import configs, inputs

pytestmark = pytest.mark.gpu

FHN = (0.1, 2.0, -0.1)
SCHNAK = (1000.0, 0.1, 0.9)


@pytest.fixture(scope="module")
def ds():
    from paper_2310_07551_gb300 import ds as _ds
    _ds.lib()
    return _ds


def relmax(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("model,p,dims,lo,hi,delta,tau,dense", [
    ("fhn", FHN, (20, 18, 16), -1.0, 1.0, (1.0, 42.1887), 1e-3, False),
    ("schnakenberg", SCHNAK, (33, 40), 0.0, 1.0, (1.0, 10.0), 1e-4, False),
    ("fhn", FHN, (9, 7), -1.0, 1.0, (1.0, 3.0), 1e-3, True),
])
def test_adjoint_step_matches_oracle(ds, model, p, dims, lo, hi, delta, tau, dense):
    if dense:
        As = [[inputs.random_matrix(n, seed=8, stream=10 * c + q, scale=3.0) for q, n in enumerate(dims)]
              for c in range(2)]
    else:
        Ds = [inputs.fd_neumann(n, lo, hi) for n in dims]
        As = [[dl * D for D in Ds] for dl in delta]
    U = inputs.initial_state(model, dims, seed=5)
    lam = inputs.random_tensor((int(np.prod(dims)) * 2,), seed=6).reshape(U.shape)
    P = O.phi_set(dims, As, tau)
    ref, dref, sref = O.step_adjoint(dims, As, P, model, p, tau, U, lam, with_scale=True)
    ps = ds.PhiSet(dims, As, tau)
    plan = ds.Plan(ps, model, p, "f64")
    dp = torch.zeros(3, dtype=torch.float64, device="cuda")
    dsc = torch.zeros(2, dtype=torch.float64, device="cuda")
    got = plan.step_backward(torch.from_numpy(U).cuda(), torch.from_numpy(lam).cuda(), dp, dsc)
    plan.sync()
    assert relmax(got.cpu().numpy(), ref) < 1e-12
    assert np.allclose(dp.cpu().numpy(), dref, rtol=1e-11, atol=1e-12 * np.abs(dref).max())
    assert np.allclose(dsc.cpu().numpy(), sref, rtol=1e-10, atol=1e-12 * np.abs(sref).max())


def test_adjoint_rejects_reduced_precision_plan(ds):
    dims = (16, 16)
    Ds = [inputs.fd_neumann(n, 0.0, 1.0) for n in dims]
    ps = ds.PhiSet(dims, [[D for D in Ds], [10 * D for D in Ds]], 1e-4)
    plan = ds.Plan(ps, "schnakenberg", SCHNAK, "bf16x6")
    U = torch.zeros((2, 16, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(ds.DsError) as e:
        plan.step_backward(U, U.clone())
    assert e.value.status == ds.DS_ERR_UNSUPPORTED


def test_differentiation_workload_fhn96(ds):
    from paper_2310_07551_gb300.adjoint import integrate
    w = configs.WORKLOADS["fhn3d_96"]
    nsteps, ckpt = w.steps, 20
    Ds = [inputs.fd_neumann(n, w.lo, w.hi) for n in w.dims]
    As = [[dl * D for D in Ds] for dl in w.delta]
    ps = ds.PhiSet(w.dims, As, w.tau)
    U0 = torch.from_numpy(inputs.initial_state("fhn", w.dims, seed=w.seed)).cuda()
    # target from hidden parameters
    hid_delta = (w.delta[0], w.delta[1] * 1.05)
    hid_p = (w.params[0] * 0.9, w.params[1], w.params[2] * 1.2)
    ps_h = ds.PhiSet(w.dims, [[dl * D for D in Ds] for dl in hid_delta], w.tau)
    plan_h = ds.Plan(ps_h, "fhn", hid_p, "f64")
    target = U0.clone()
    plan_h.integrate(target, nsteps)
    plan_h.sync()
    u_target = target[0].clone()

    def loss_of(UT):
        return ((UT[0] - u_target) ** 2).mean()

    plans = {}

    def plan_for(p):
        key = tuple(p)
        if key not in plans:
            plans[key] = ds.Plan(ps, "fhn", key, "f64")
        return plans[key]

    p0 = torch.tensor(w.params, dtype=torch.float64)
    U0g = U0.clone().requires_grad_(True)
    pg = p0.clone().requires_grad_(True)
    sg = torch.ones(2, dtype=torch.float64, requires_grad=True)
    L = loss_of(integrate(U0g, pg, plan_for(w.params), nsteps, ckpt, s=sg))
    L.backward()
    gU, gp = U0g.grad, pg.grad
    g_delta_v = float(sg.grad[1]) / w.delta[1]      # dL/d delta_v

    def L_at(U, p):
        X = U.clone()
        pl = plan_for(p)
        pl.integrate(X, nsteps)
        pl.sync()
        return float(loss_of(X))

    h = 1e-6
    for q in (0, 2):          # eps, alpha0
        pp = list(w.params); pm = list(w.params)
        pp[q] += h; pm[q] -= h
        fd = (L_at(U0, pp) - L_at(U0, pm)) / (2 * h)
        assert abs(fd - float(gp[q])) <= 1e-6 * abs(fd) + 1e-14, (q, fd, float(gp[q]))
    # delta_v: rebuild the phi-set at delta_v (1 +- h)
    vals = []
    for sgn in (1, -1):
        dv = w.delta[1] * (1 + sgn * h)
        ps_d = ds.PhiSet(w.dims, [[w.delta[0] * D for D in Ds], [dv * D for D in Ds]], w.tau)
        pl = ds.Plan(ps_d, "fhn", w.params, "f64")
        X = U0.clone()
        pl.integrate(X, nsteps)
        pl.sync()
        vals.append(float(loss_of(X)))
    fd = (vals[0] - vals[1]) / (2 * h * w.delta[1])
    assert abs(fd - g_delta_v) <= 1e-6 * abs(fd) + 1e-14, (fd, g_delta_v)
    g = torch.Generator(device="cpu").manual_seed(11)
    for _ in range(3):
        v = torch.randn(U0.shape, generator=g, dtype=torch.float64).cuda()
        fd = (L_at(U0 + h * v, w.params) - L_at(U0 - h * v, w.params)) / (2 * h)
        an = float((gU * v).sum())
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-14, (fd, an)


def test_integrate_ckpt_matches_integrate(ds):
    dims = (24, 20, 18)
    Ds = [inputs.fd_neumann(n, -1.0, 1.0) for n in dims]
    ps = ds.PhiSet(dims, [[D for D in Ds], [42.1887 * D for D in Ds]], 1e-3)
    plan = ds.Plan(ps, "fhn", FHN, "f64")
    U0 = torch.from_numpy(inputs.initial_state("fhn", dims, seed=3)).cuda()
    U = U0.clone()
    ck = plan.integrate_ckpt(U, 11, 4)            # checkpoints after 4 and 8 steps
    assert ck.shape == (2,) + tuple(U0.shape)
    R = U0.clone()
    for j in range(2):
        plan.integrate(R, 4)
        plan.sync()
        assert torch.equal(ck[j], R)
    plan.integrate(R, 3)
    plan.sync()
    assert torch.equal(U, R)
    with pytest.raises(ds.DsError):
        plan.integrate_ckpt(U, 5, 0)
