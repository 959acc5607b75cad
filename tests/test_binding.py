"""The Python binding refuses arguments that would make the library's
kernels read or write the wrong memory (no GPU needed): host tensors (there
is no CPU path), other dtypes, non-contiguous or wrongly sized tensors."""

import numpy as np
import pytest
import torch

from paper_2010_14175_gb300 import afsai
from paper_2010_14175_gb300 import matgen as mg


class FakeDevice:
    """Stands in for a CUDA tensor (this test runs without a GPU)."""

    def __init__(self, dtype, numel, contiguous=True):
        self.is_cuda = True
        self.dtype = dtype
        self._numel = numel
        self._contiguous = contiguous

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contiguous

    def data_ptr(self):
        return 0x7F0000001000


def test_host_tensors_are_refused():
    A = mg.poisson7(3)
    host = afsai.DeviceCSR(A.n, torch.from_numpy(A.rowptr), torch.from_numpy(A.col), torch.from_numpy(A.val))
    with pytest.raises(ValueError, match="CUDA tensor"):
        host.c()
    with pytest.raises(ValueError, match="CUDA tensor"):
        afsai._vec(torch.zeros(A.n, dtype=torch.float64), A.n, "x")
    with pytest.raises(ValueError, match="CUDA tensor"):
        afsai._vec(np.zeros(A.n), A.n, "x")


def test_dtype_shape_and_layout_checks():
    n = 10
    assert afsai._vec(FakeDevice(torch.float64, n), n, "x").value == 0x7F0000001000
    with pytest.raises(ValueError, match="float64"):
        afsai._vec(FakeDevice(torch.float32, n), n, "x")
    with pytest.raises(ValueError, match="10 entries"):
        afsai._vec(FakeDevice(torch.float64, n - 1), n, "x")
    with pytest.raises(ValueError, match="contiguous"):
        afsai._vec(FakeDevice(torch.float64, n, contiguous=False), n, "x")
    # a CSR whose arrays have the right types and lengths passes; a short
    # row pointer array or int64 columns do not
    ok = afsai.DeviceCSR(n, FakeDevice(torch.int32, n + 1), FakeDevice(torch.int32, 30), FakeDevice(torch.float64, 30))
    csr = ok.c()
    assert (csr.n, csr.nnz) == (n, 30)
    short = afsai.DeviceCSR(n, FakeDevice(torch.int32, n), FakeDevice(torch.int32, 30), FakeDevice(torch.float64, 30))
    with pytest.raises(ValueError, match="rowptr"):
        short.c()
    wide = afsai.DeviceCSR(n, FakeDevice(torch.int32, n + 1), FakeDevice(torch.int64, 30), FakeDevice(torch.float64, 30))
    with pytest.raises(ValueError, match="int32"):
        wide.c()
