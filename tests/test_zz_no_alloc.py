"""sph_cell_sort_noalloc, the allocation-free cell sort, called through the C ABI.

Its users are callers that cannot let a library allocate device memory (HBM
already held by their own caching allocator, no tolerance for the device
synchronisation of cudaMalloc, or an outside memory manager).  Its output must
equal sph_cell_sort's (index work: bit-exact) on two calls in a row, since the
calls share one scratch array that keeps the previous call's contents.

This file is collected last so a failure here cannot hide the other tests.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2512_09904_b300 import build
    build.build()
    from paper_2512_09904_b300 import sph
    return torch, sph


def _device_memory_in_use(torch):
    """(bytes the driver reports in use on the device, bytes in use in the
    device's default stream-ordered pool): a cudaMalloc or a
    cudaMallocAsync inside the call would move one of them."""
    from cuda.bindings import runtime as rt
    free, total = torch.cuda.mem_get_info()
    err, pool = rt.cudaDeviceGetDefaultMemPool(torch.cuda.current_device())
    assert err == rt.cudaError_t.cudaSuccess
    err, used = rt.cudaMemPoolGetAttribute(pool, rt.cudaMemPoolAttr.cudaMemPoolAttrUsedMemCurrent)
    assert err == rt.cudaError_t.cudaSuccess
    return total - free, int(used)


def _sort(torch, sph, fn, pos, origin, cellw, ncell, check_noalloc=False):
    n = len(pos)
    d_pos = torch.tensor(pos, dtype=torch.float64, device="cuda")
    d_perm = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    d_cs = torch.full((int(np.prod(ncell)) + 1,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    before = _device_memory_in_use(torch)
    fn(d_pos.data_ptr(), n, origin, cellw, ncell, d_perm.data_ptr(), d_cs.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    if check_noalloc:
        assert _device_memory_in_use(torch) == before
    return d_perm.cpu().numpy()[:n], d_cs.cpu().numpy()


def test_noalloc_matches_allocating_sort_twice(env):
    torch, sph = env
    rng = np.random.default_rng(404)
    # the first call on the device may load the library's module there (lazy
    # loading), which places the fixed scratch array: take it before measuring
    _sort(torch, sph, sph.sph_cell_sort_noalloc, np.zeros((1, 3)), np.zeros(3), np.ones(3), (1, 1, 1))
    # two different calls in a row: the second must not see the first's leftovers
    calls = [(300001, (64, 40, 30), 1.0), (120000, (17, 90, 11), 2.5)]
    for n, ncell, L in calls:
        pos = rng.uniform(-0.02 * L, 1.02 * L, size=(n, 3))
        origin = np.zeros(3)
        cellw = L / np.asarray(ncell, np.float64)
        ref = _sort(torch, sph, sph.sph_cell_sort, pos, origin, cellw, ncell)
        got = _sort(torch, sph, sph.sph_cell_sort_noalloc, pos, origin, cellw, ncell, check_noalloc=True)
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    torch, sph = env
    # the size check comes before any device access: small buffers suffice
    d_pos = torch.zeros(3, dtype=torch.float64, device="cuda")
    d_perm = torch.zeros(1, dtype=torch.int32, device="cuda")
    d_cs = torch.zeros(2, dtype=torch.int32, device="cuda")
    args = (d_perm.data_ptr(), d_cs.data_ptr(), torch.cuda.current_stream().cuda_stream)
    with pytest.raises(sph.SphError) as e:
        sph.sph_cell_sort_noalloc(d_pos.data_ptr(), sph.NOALLOC_MAX_N + 1, np.zeros(3), np.ones(3), (1, 1, 1), *args)
    assert e.value.status == sph.SPH_EINVAL
    assert "SPH_NOALLOC_MAX_N" in str(e.value)
    with pytest.raises(sph.SphError) as e:
        sph.sph_cell_sort_noalloc(d_pos.data_ptr(), 1, np.zeros(3), np.ones(3), (1024, 1024, 2), *args)
    assert e.value.status == sph.SPH_EINVAL
    # the entry point still works after the rejections
    got = _sort(torch, sph, sph.sph_cell_sort_noalloc, np.array([[0.5, 0.5, 0.5], [0.1, 0.1, 0.1]]),
                np.zeros(3), np.full(3, 0.5), (2, 2, 2))
    assert got[0].tolist() == [1, 0] and got[1].tolist() == [0, 1, 1, 1, 1, 1, 1, 1, 2]
