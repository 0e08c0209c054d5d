"""The allocation-free weight-gradient entry point (petgem_nn_conv3d_wgrad_noalloc) against the
allocating one (petgem_nn_conv3d_wgrad), through the C ABI.

Collected last (file name) so that it also runs after every other GPU test in one process, and
it passes alone.  Two calls in a row on different grids and channel counts: the second must not
see the first's partial sums or error flag left in the shared scratch.  Both entry points run the
same split-K kernel with the same split count, so the bar is the convolution tests' 1e-4 of the
largest entry (in practice the two agree exactly).
"""
import numpy as np
import pytest

from paper_1808_00186_gb300 import api

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1808_00186_gb300 import build
    build.build()
    api.load()
    torch.cuda.set_device(0)


def rel_max(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def inputs(grid, cin, cout, seed):
    rng = np.random.default_rng(seed)
    V = grid[0] * grid[1] * grid[2]
    x = torch.as_tensor(rng.normal(size=(V, cin)).astype(np.float32)).to(torch.bfloat16).cuda()
    dy = torch.as_tensor(rng.normal(size=(V, cout)).astype(np.float32)).to(torch.bfloat16).cuda()
    return x, dy


def test_noalloc_wgrad_matches_allocating_entry_point_twice_in_a_row():
    stream = torch.cuda.current_stream().cuda_stream
    # 48 x 50 x 52 = 124,800 voxels is near the scratch limit (31 split-K slices); 9 x 7 x 5 uses one.
    cases = [((48, 50, 52), 32, 32, 1), ((9, 7, 5), 16, 32, 2)]
    outs = []
    for grid, cin, cout, seed in cases:
        x, dy = inputs(grid, cin, cout, seed)
        ref = torch.empty((27, cout, cin), dtype=torch.float32, device="cuda")
        api.petgem_nn_conv3d_wgrad(stream, grid, cin, cout, x, dy, ref)
        got = torch.full((27, cout, cin), float("nan"), dtype=torch.float32, device="cuda")
        api.petgem_nn_conv3d_wgrad_noalloc(stream, grid, cin, cout, x, dy, got)
        outs.append((got.cpu().numpy(), ref.cpu().numpy()))
    for got, ref in outs:
        assert np.isfinite(got).all()
        assert np.abs(ref).max() > 0
        assert rel_max(got, ref) <= 1e-4


def test_noalloc_wgrad_rejects_grids_beyond_its_scratch():
    stream = torch.cuda.current_stream().cuda_stream
    grid = (64, 64, 33)  # 135,168 voxels > the limit
    assert grid[0] * grid[1] * grid[2] > api.NOALLOC_MAX_VOXELS
    x, dy = inputs(grid, 16, 16, 3)
    dw = torch.zeros((27, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(api.PetgemError) as e:
        api.petgem_nn_conv3d_wgrad_noalloc(stream, grid, 16, 16, x, dy, dw)
    assert e.value.status == api.ERR_UNSUPPORTED
    assert torch.count_nonzero(dw).item() == 0
