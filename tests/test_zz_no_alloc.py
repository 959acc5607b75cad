"""afsai_apply_static: the preconditioner application for callers that
cannot allocate device memory (their memory belongs to another allocator,
or cudaMalloc/cudaFree would synchronise a latency-critical path).  It keeps
the intermediate G r in a fixed 2^20-double device array instead of
allocating.  This file is collected last on purpose.

Checks, through the C ABI: two calls in a row give the same z as
afsai_apply (within the rounding bound the apply tests use); the second
call changes neither the device's free memory, nor the use of its default
stream-ordered memory pool (both read from the CUDA driver), nor the use of
the library's own memory pool (afsai_pool_stats); the first call works in a fresh process (the array
was loaded by afsai_setup); n above the array's size is rejected with
EINVAL."""
import ctypes
import numpy as np
import pytest

from paper_2010_14175_gb300 import matgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_14175_gb300 import afsai

    afsai.load()
    return afsai


class _DriverMemory:
    """Free device memory (cuMemGetInfo) and the bytes in use in the current
    device's default memory pool (cuMemPoolGetAttribute), read through the
    CUDA driver library for the context torch made current."""

    USED_MEM_CURRENT = 0x7  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT
    RESERVED_MEM_CURRENT = 0x5  # CU_MEMPOOL_ATTR_RESERVED_MEM_CURRENT

    def __init__(self, device):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), device) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def snapshot(self):
        free, total = ctypes.c_size_t(), ctypes.c_size_t()
        assert self.cu.cuMemGetInfo_v2(ctypes.byref(free), ctypes.byref(total)) == 0
        used, reserved = ctypes.c_uint64(), ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.USED_MEM_CURRENT, ctypes.byref(used)) == 0
        assert self.cu.cuMemPoolGetAttribute(self.pool, self.RESERVED_MEM_CURRENT, ctypes.byref(reserved)) == 0
        return {"free": free.value, "pool_used": used.value, "pool_reserved": reserved.value}


def _bound(G, r):
    import scipy.sparse as sp

    absG = abs(sp.csr_matrix(G))
    return 64 * np.finfo(float).eps * (absG.T @ (absG @ np.abs(r)))


@pytest.mark.parametrize("name,make,kiter,s,eps,g_prec", [
    ("hetero20_fp64", lambda: mg.diffusion7_hetero(20, 4), 5, 2, 1e-3, 0),
    ("elast6_fp64", lambda: mg.elasticity_hex(6, 17), 10, 3, 1e-3, 0),
    ("poisson16_fp32", lambda: mg.poisson7(16), 5, 2, 1e-3, 1),
])
def test_static_apply_matches_apply_twice(gpu, name, make, kiter, s, eps, g_prec):
    import torch

    afsai = gpu
    A = make()
    M = afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(kiter, s, eps, 0, g_prec))
    rp, ci, va = M.export()
    G = (va, ci, rp)
    rng = np.random.default_rng(5)
    mem = _DriverMemory(torch.cuda.current_device())
    for call in range(2):  # the array keeps the previous call's contents
        r = rng.standard_normal(A.n)
        rd = torch.from_numpy(r).cuda()
        z_static = torch.full((A.n,), np.nan, dtype=torch.float64, device="cuda")
        z_ref = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        before = (mem.snapshot(), afsai.pool_stats())
        afsai.afsai_apply_static(M, rd, z_static)
        torch.cuda.synchronize()
        after = (mem.snapshot(), afsai.pool_stats())
        if call == 1:
            assert after == before, (before, after)
        afsai.afsai_apply(M, rd, z_ref)
        torch.cuda.synchronize()
        zs, zr = z_static.cpu().numpy(), z_ref.cpu().numpy()
        import scipy.sparse as sp

        Gs = sp.csr_matrix(G, shape=(A.n, A.n))
        tol = _bound(Gs, r) if g_prec == 0 else 1e-5 * (abs(Gs).T @ (abs(Gs) @ np.abs(r)))
        assert np.all(np.isfinite(zs)), f"call {call}"
        assert np.all(np.abs(zs - zr) <= tol + 1e-300), f"call {call}"
    M.close()


def test_static_apply_rejects_n_above_capacity(gpu):
    import torch

    afsai = gpu
    n = (1 << 20) + 1
    A = mg.laplace1d(n)
    M = afsai.afsai_setup(afsai.DeviceCSR.from_host(A), afsai.params(0, 1, 1e-3))
    r = torch.ones(n, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(afsai.AfsaiError) as e:
        afsai.afsai_apply_static(M, r, z)
    assert e.value.status == afsai.EINVAL
    assert "2^20" in str(e.value) or "1048576" in str(e.value)
    M.close()
