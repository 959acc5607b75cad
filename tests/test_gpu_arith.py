"""The lane-per-row dense solves of the FP64 set-up compute square roots and
divisions on the integer pipes (GB300 issues FP64 at 1/64 of the FP32 rate);
they must return the IEEE round-to-nearest results bit for bit, or the FP64
set-up would drift from the plain definition.  The library's self-check
compares them with the hardware operations on operands drawn on the device:
random and structured significands, mid-range and extreme exponents
(subnormal and overflowing quotients take the fallback), near-exact
quotients, zero numerators, exact squares and their neighbours."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_14175_gb300 import afsai

    afsai.load()
    return afsai


@pytest.mark.parametrize("seed", [1, 20101417, 2**63 + 5])
def test_integer_pipe_div_sqrt_match_ieee(gpu, seed):
    nd, ns = gpu.check_arith(1 << 26, seed)
    assert (nd, ns) == (0, 0)


def test_check_arith_arguments(gpu):
    with pytest.raises(gpu.AfsaiError):
        gpu.check_arith(-1, 1)
    assert gpu.check_arith(0, 1) == (0, 0)
