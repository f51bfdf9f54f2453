"""nep_jacobi_svd_noalloc: the Jacobi SVD for callers that cannot allocate device memory.

Runs last (file name) so that a run stopping at the first failure has run everything else.
The variant must give the results of nep_jacobi_svd on the same input, call after call,
even though every call reuses the same fixed block of device memory.
"""
import numpy as np
import pytest

from tests.gpu_util import from_dev_c128, to_dev, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bnd():
    from paper_1910_11712_gb300 import binding
    binding.load(build_if_missing=True)
    return binding


def _svd(bnd, torch, A, noalloc):
    rows, cols = A.shape
    Ad = to_dev(np.asfortranarray(A), torch)
    Wd = torch.zeros(cols * cols * 2, dtype=torch.float64, device="cuda")
    sd = torch.zeros(cols, dtype=torch.float64, device="cuda")
    (bnd.jacobi_svd_noalloc if noalloc else bnd.jacobi_svd)(rows, cols, Ad, Wd, sd)
    torch.cuda.synchronize()
    U = from_dev_c128(Ad).reshape(cols, rows).T
    W = from_dev_c128(Wd).reshape(cols, cols).T
    return U, W, sd.cpu().numpy()


def test_noalloc_svd_matches_allocating_entry_point_twice(bnd):
    torch = torch_cuda()
    rng = np.random.default_rng(2024)
    # two calls in a row with different shapes: the second reuses the block the first left dirty
    for shape in [(128, 128), (90, 60)]:
        A = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        U0, W0, s0 = _svd(bnd, torch, A, noalloc=False)
        U1, W1, s1 = _svd(bnd, torch, A, noalloc=True)
        ref = np.linalg.svd(A, compute_uv=False)
        # same tolerances as the Jacobi SVD parity test
        assert np.abs(s1 - s0).max() <= 1e-13 * ref[0] * max(shape)
        assert np.abs(s1 - ref).max() <= 1e-13 * ref[0] * max(shape)
        assert np.abs(A @ W1 - U1 * s1[None, :]).max() <= 1e-12 * ref[0]
        assert np.abs(W1.conj().T @ W1 - np.eye(shape[1])).max() <= 1e-12
        assert np.abs(np.abs(W1) - np.abs(W0)).max() <= 1e-10


def test_noalloc_svd_rejects_sizes_beyond_the_fixed_block(bnd):
    torch = torch_cuda()
    rows, cols = 400, 300  # 400*300 + 300*300 > 131072
    Ad = torch.zeros(rows * cols * 2, dtype=torch.float64, device="cuda")
    Wd = torch.zeros(cols * cols * 2, dtype=torch.float64, device="cuda")
    sd = torch.zeros(cols, dtype=torch.float64, device="cuda")
    with pytest.raises(bnd.NepError) as e:
        bnd.jacobi_svd_noalloc(rows, cols, Ad, Wd, sd)
    assert e.value.code == bnd.NEP_ERR_ARG
    assert "exceeds the fixed scratch" in str(e.value)


def _device_memory_state():
    """(free device bytes, used and reserved bytes of the device's default stream-ordered pool),
    read through the CUDA runtime the library itself links."""
    import ctypes
    rt = ctypes.CDLL("libcudart.so.13")
    dev = ctypes.c_int()
    assert rt.cudaGetDevice(ctypes.byref(dev)) == 0
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used, reserved = ctypes.c_uint64(), ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, 7, ctypes.byref(used)) == 0      # cudaMemPoolAttrUsedMemCurrent
    assert rt.cudaMemPoolGetAttribute(pool, 5, ctypes.byref(reserved)) == 0  # cudaMemPoolAttrReservedMemCurrent
    free, total = ctypes.c_size_t(), ctypes.c_size_t()
    assert rt.cudaMemGetInfo(ctypes.byref(free), ctypes.byref(total)) == 0
    return free.value, used.value, reserved.value


def test_noalloc_svd_allocates_no_device_memory(bnd):
    """The promise itself: around a call (after a first one has loaded the kernels), neither the
    device's free memory nor the default memory pool's use changes. The inputs and outputs are
    allocated beforehand."""
    torch = torch_cuda()
    rows, cols = 120, 100
    rng = np.random.default_rng(11)
    A = rng.standard_normal((rows, cols)) + 1j * rng.standard_normal((rows, cols))
    Ad = to_dev(np.asfortranarray(A), torch)
    Wd = torch.zeros(cols * cols * 2, dtype=torch.float64, device="cuda")
    sd = torch.zeros(cols, dtype=torch.float64, device="cuda")
    bnd.jacobi_svd_noalloc(rows, cols, Ad, Wd, sd)
    torch.cuda.synchronize()
    before = _device_memory_state()
    for _ in range(2):
        bnd.jacobi_svd_noalloc(rows, cols, Ad, Wd, sd)
    torch.cuda.synchronize()
    assert _device_memory_state() == before
