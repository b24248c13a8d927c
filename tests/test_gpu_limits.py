"""FP64 Tucker operator on flat grids whose mode products exceed one launch's
grid limits (more than 65,535 outer slices, or more than 65,535 row tiles of
fibres): the library cuts such products into launches that fit, and the
result must be the oracle's (Section 2, eq. krontomu: a mode product is a
matrix product of the unfolded tensor)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [
    (2, 2, 256, 512),     # mode 2: 131,072 outer slices in the batch dimension
    (2, 256, 256, 128),   # mode 1: 8,388,608 fibres = 131,072 row tiles of 64
])
def test_tucker_f64_beyond_one_launch_matches_the_oracle(dims):
    from oracle import oracle as O
    from paper_2310_07551_gb300 import ds, inputs
    X = inputs.random_tensor(dims, seed=41)
    Ls = [inputs.random_matrix(n, seed=42, stream=q, scale=1.0 / np.sqrt(n)) for q, n in enumerate(dims)]
    ref = O.tucker(X, Ls)
    got = ds.tucker(torch.from_numpy(X).cuda(), [torch.from_numpy(L).cuda() for L in Ls]).cpu().numpy()
    rel = float(np.abs(got - ref).max() / np.abs(ref).max())
    assert rel < 1e-12, rel
