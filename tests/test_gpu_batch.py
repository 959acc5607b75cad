"""Batched form: many uneven SPD systems in one set-up launch and one
graph-captured PCG loop (afsai_batch_solve), against the CPU oracle.

Bars: every system converges to the true residual 1e-8; its iteration
count is the oracle's +-1 (different summation order of the dot products);
its solution matches the oracle's within the solve tolerance; and a
system's result is bit-for-bit the same alone and inside the batch (its
reductions never mix with other systems)."""
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


def _run(afsai, systems, prm, rtol=1e-8):
    import torch

    As = [afsai.DeviceCSR.from_host(A) for A, _, _ in systems]
    bs = [torch.from_numpy(b).cuda() for _, b, _ in systems]
    xs = [torch.zeros_like(b) for b in bs]
    infos, binfo = afsai.afsai_batch_solve(As, prm, bs, xs, rtol=rtol, maxit=5000)
    return [x.cpu().numpy() for x in xs], infos, binfo


@pytest.fixture(scope="module")
def systems():
    # 24 uneven systems (n from 50 to 3000), every stencil type
    return mg.batch_workload(24, nmin=50, nmax=3000)


def test_batch_matches_oracle(gpu, oracle_mod, systems):
    kiter, s, eps = 8, 2, 1e-3
    xs, infos, binfo = _run(gpu, systems, gpu.params(kiter, s, eps))
    assert binfo["converged"] == len(systems)
    for (A, b, kind), x, inf in zip(systems, xs, infos):
        G = oracle_mod.afsai_setup(A, kiter, s, eps)
        xo, it_o, _, _ = oracle_mod.pcg(A, G, b, rtol=1e-8)
        assert inf["converged"] == 1 and inf["relres_true"] <= 1.05e-8, (kind, inf)
        assert abs(inf["iters"] - it_o) <= 1, (kind, A.n, inf["iters"], it_o)
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def test_batch_result_same_alone_and_in_mix(gpu, systems):
    prm = gpu.params(8, 2, 1e-3)
    xs_mix, inf_mix, _ = _run(gpu, systems, prm)
    for k in (0, 5, len(systems) - 1):
        xs_alone, inf_alone, _ = _run(gpu, [systems[k]], prm)
        assert inf_alone[0]["iters"] == inf_mix[k]["iters"]
        assert np.array_equal(xs_alone[0], xs_mix[k])
    # a different mix (reversed order, subset)
    sub = systems[::-2]
    xs_sub, inf_sub, _ = _run(gpu, sub, prm)
    for j, k in enumerate(range(len(systems) - 1, -1, -2)):
        assert np.array_equal(xs_sub[j], xs_mix[k])


@pytest.mark.parametrize("g_prec,chol_prec", [(1, 1), (2, 1)])
def test_batch_mixed_precision(gpu, oracle_mod, systems, g_prec, chol_prec):
    kiter, s, eps = 8, 2, 1e-3
    xs, infos, binfo = _run(gpu, systems, gpu.params(kiter, s, eps, 0, g_prec, chol_prec))
    assert binfo["converged"] == len(systems)
    for (A, b, kind), inf in zip(systems, infos):
        G = oracle_mod.afsai_setup(A, kiter, s, eps)
        _, it_o, _, _ = oracle_mod.pcg(A, G, b, rtol=1e-8)
        assert inf["relres_true"] <= 1.05e-8
        assert inf["iters"] <= int(np.ceil(1.10 * it_o)) + 1, (kind, A.n, inf["iters"], it_o)
