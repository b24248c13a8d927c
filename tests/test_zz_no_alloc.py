"""ds_tucker_static: the Tucker entry point for callers that cannot allocate
device memory (allocator callbacks, hosts that forbid allocation after
start-up, plugins whose framework owns the device heap).  It runs the same
kernels as the allocating entry point ds_tucker on the same data, so the two
must agree bit for bit, call after call, while its intermediates live in the
library's fixed device array.

Kept in a file of its own that collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_static_tucker_matches_ds_tucker_on_two_calls_in_a_row():
    from paper_2310_07551_gb300 import ds, inputs
    ds.lib()
    # two calls in a row, the second with another shape and other data, so a
    # stale intermediate left by the first call would show up in the second
    for call, dims in enumerate([(64, 48, 40), (96, 70)]):
        X = torch.from_numpy(inputs.random_tensor(dims, seed=30 + call)).cuda()
        Ls = [torch.from_numpy(inputs.random_matrix(n, seed=31 + call, stream=q)).cuda()
              for q, n in enumerate(dims)]
        for transpose in (False, True):
            ref = ds.tucker(X, Ls, transpose=transpose)
            got = ds.tucker_static(X, Ls, transpose=transpose)
            torch.cuda.synchronize()
            assert torch.equal(got, ref), (call, transpose)


def test_static_tucker_matches_the_oracle():
    from oracle import oracle as O
    from paper_2310_07551_gb300 import ds, inputs
    dims = (40, 24, 18)
    X = inputs.random_tensor(dims, seed=36)
    Ls = [inputs.random_matrix(n, seed=37, stream=q) for q, n in enumerate(dims)]
    ref = O.tucker(X, Ls)
    got = ds.tucker_static(torch.from_numpy(X).cuda(), [torch.from_numpy(L).cuda() for L in Ls]).cpu().numpy()
    rel = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert rel < 1e-13, rel


def test_static_tucker_flat_grid_at_the_launch_limits():
    """(2, 2, 256, 512): the mode-2 product has 131,072 outer slices, more
    than one launch's 65,535 grid rows, and 524,288 points fit the static
    scratch; the result must still be the allocating entry point's."""
    from paper_2310_07551_gb300 import ds, inputs
    dims = (2, 2, 256, 512)
    X = torch.from_numpy(inputs.random_tensor(dims, seed=38)).cuda()
    Ls = [torch.from_numpy(inputs.random_matrix(n, seed=39, stream=q)).cuda() for q, n in enumerate(dims)]
    ref = ds.tucker(X, Ls)
    got = ds.tucker_static(X, Ls)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)


def test_static_tucker_rejects_grids_beyond_its_scratch():
    from paper_2310_07551_gb300 import ds
    X = torch.zeros((2, 1024, 1024), dtype=torch.float64, device="cuda")   # 2,097,152 points
    Ls = [torch.eye(n, dtype=torch.float64, device="cuda") for n in (1024, 1024, 2)]
    with pytest.raises(ds.DsError) as e:
        ds.tucker_static(X, Ls)
    assert e.value.status == ds.DS_ERR_INVALID_ARG
    assert "1048576" in str(e.value)
