"""C ABI checks that need no GPU: the library builds for sm_103a, loads,
exports every entry point include/afsai.h declares, and the ctypes
structures of the binding match the C layout compiled from the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "afsai.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"AFSAI_API\s+[\w\s\*]+?\b(\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_14175_gb300 import afsai

    return afsai.load()


def test_library_exports_every_declared_function(lib):
    from paper_2010_14175_gb300 import afsai

    names = declared_functions()
    assert len(names) >= 12
    assert set(names) == set(afsai.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", afsai.library_path()], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, re.M))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert getattr(lib, n) is not None


def test_library_is_sm103a_only(lib):
    from paper_2010_14175_gb300 import build

    # one -gencode pair, sm_103a only, for every translation unit and the link
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_calls(lib):
    from paper_2010_14175_gb300 import afsai

    assert lib.afsai_version().decode().startswith("afsai-gb300")
    # argument checks run before any CUDA call
    st = lib.afsai_setup(None, None, None, None)
    assert st == afsai.EINVAL
    assert b"NULL" in lib.afsai_last_error()
    assert lib.afsai_get_info(None, None) == afsai.EINVAL
    lib.afsai_destroy(None)


def test_struct_layout_matches_header(tmp_path):
    from paper_2010_14175_gb300 import afsai

    src = tmp_path / "layout.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "afsai.h"
int main(void) {
  printf("%zu %zu %zu %zu\\n", sizeof(afsai_csr), sizeof(afsai_params), sizeof(afsai_info), sizeof(pcg_info));
  printf("%zu %zu %zu %zu\\n", offsetof(afsai_csr, val), offsetof(afsai_params, chol_prec), offsetof(pcg_info, solve_ms),
         offsetof(afsai_params, block_power));
  return 0;
}
""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    sizes = [int(v) for v in out]
    assert sizes[0] == ctypes.sizeof(afsai.Csr)
    assert sizes[1] == ctypes.sizeof(afsai.Params)
    assert sizes[2] == ctypes.sizeof(afsai.Info)
    assert sizes[3] == ctypes.sizeof(afsai.PcgInfo)
    assert sizes[4] == afsai.Csr.val.offset
    assert sizes[5] == afsai.Params.chol_prec.offset
    assert sizes[6] == afsai.PcgInfo.solve_ms.offset
    assert sizes[7] == afsai.Params.block_power.offset


@pytest.mark.parametrize("bad,status", [
    (dict(kiter=-1), "EINVAL"), (dict(s=0), "EINVAL"), (dict(eps=-1e-3), "EINVAL"), (dict(eps=float("nan")), "EINVAL"),
    (dict(exit_mode=2), "EINVAL"), (dict(g_prec=3), "EINVAL"), (dict(chol_prec=2), "EINVAL"),
    (dict(block_rows=-1), "EINVAL"), (dict(block_power=65), "EINVAL"), (dict(kiter=64, s=2), "ENOTSUP"),
])
def test_setup_parameter_checks_before_any_device_call(lib, bad, status):
    """afsai_setup rejects bad parameters on the host, before it touches the
    CSR or the device (so this runs without a GPU)."""
    from paper_2010_14175_gb300 import afsai

    p = dict(kiter=5, s=2, eps=1e-3, exit_mode=0, g_prec=0, chol_prec=0, block_rows=0, block_power=1)
    p.update(bad)
    prm = afsai.params(**p)
    A = afsai.Csr()  # never read: the parameters are checked first
    out = ctypes.c_void_p()
    st = lib.afsai_setup(ctypes.byref(A), ctypes.byref(prm), None, ctypes.byref(out))
    assert st == getattr(afsai, status)
    assert out.value is None
    assert lib.afsai_last_error()


def test_batch_and_server_argument_checks_on_the_host(lib):
    """afsai_batch_solve and the server entry points reject bad arguments
    and bad set-up parameters on the host, before any device call."""
    from paper_2010_14175_gb300 import afsai

    good = afsai.params(5, 2, 1e-3)
    bad = afsai.params(5, 0, 1e-3)  # s < 1
    bounded = afsai.params(5, 2, 1e-3, block_rows=64)
    A = afsai.Csr()
    ptrs = (ctypes.c_void_p * 1)(0x1000)  # never dereferenced: the checks come first

    def batch(nsys, prm, rtol=1e-8, maxit=100):
        return lib.afsai_batch_solve(nsys, ctypes.addressof(A), ctypes.byref(prm), ctypes.addressof(ptrs),
                                     ctypes.addressof(ptrs), rtol, maxit, None, None, None)

    assert batch(0, good) == afsai.EINVAL
    assert batch(1, bad) == afsai.EINVAL
    assert batch(1, bounded) == afsai.ENOTSUP
    assert batch(1, good, rtol=-1.0) == afsai.EINVAL
    assert batch(1, good, maxit=-1) == afsai.EINVAL

    out = ctypes.c_void_p()
    assert lib.serve_create(0, 8, ctypes.byref(good), 100, 4, ctypes.byref(out)) == afsai.EINVAL
    assert lib.serve_create(1 << 30, 0, ctypes.byref(good), 100, 4, ctypes.byref(out)) == afsai.EINVAL
    assert lib.serve_create(1 << 30, 8, ctypes.byref(bad), 100, 4, ctypes.byref(out)) == afsai.EINVAL
    assert lib.serve_create(1 << 30, 8, ctypes.byref(bounded), 100, 4, ctypes.byref(out)) == afsai.ENOTSUP
    assert out.value is None
    mid = ctypes.c_int32()
    assert lib.serve_register(None, ctypes.byref(A), ctypes.byref(mid)) == afsai.EINVAL
    ticket = ctypes.c_int64()
    assert lib.serve_submit(None, 0, None, 1, 1e-8, ctypes.byref(ticket)) == afsai.EINVAL
