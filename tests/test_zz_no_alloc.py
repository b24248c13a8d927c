"""ds_tucker_static: the Tucker entry point for callers that cannot allocate
device memory (allocator callbacks, hosts that forbid allocation after
start-up, plugins whose framework owns the device heap).  It must give the
result of the allocating entry point ds_tucker, call after call, while its
intermediates live in the library's fixed device array.

Kept in a file of its own that collects last."""
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
            rel = float((got - ref).abs().max() / ref.abs().max())
            assert rel < 1e-13, (call, transpose, rel)


def test_static_tucker_rejects_grids_beyond_its_scratch():
    from paper_2310_07551_gb300 import ds
    X = torch.zeros((2, 1024, 1024), dtype=torch.float64, device="cuda")   # 2,097,152 points
    Ls = [torch.eye(n, dtype=torch.float64, device="cuda") for n in (1024, 1024, 2)]
    with pytest.raises(ds.DsError) as e:
        ds.tucker_static(X, Ls)
    assert e.value.status == ds.DS_ERR_INVALID_ARG
    assert "1048576" in str(e.value)
