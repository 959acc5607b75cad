"""Batched form: many uneven SPD systems set up by buckets of row length
and solved by one graph-captured PCG loop (afsai_batch_solve), against the
CPU oracle.

Bars: every system converges to the true residual 1e-8 after exactly the
oracle's iteration count (both stop on the recursive residual and then
require the true one; each system's oracle residual is clear of the
tolerance on both sides of its stopping iteration, so rounding cannot move
the stop); its solution matches the oracle's within the solve tolerance;
and a system's result is bit-for-bit the same alone and inside the batch
(its reductions never mix with other systems).  A second case takes
systems of the full uneven-batch sizes (near 2e5 rows, every stencil
type) and checks sampled rows of G bit for bit and the iteration counts."""
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
        xo, it_o, _, _, hist = oracle_mod.pcg(A, G, b, rtol=1e-8, history=True)
        assert _clear(hist), (kind, A.n, hist[-2:])
        assert inf["converged"] == 1 and inf["relres_true"] <= 1e-8, (kind, inf)
        assert inf["iters"] == it_o, (kind, A.n, inf["iters"], it_o)
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)


def _clear(hist, rtol=1e-8, margin=1e-6):
    return len(hist) >= 2 and hist[-1] < rtol * (1 - margin) and hist[-2] > rtol * (1 + margin)


def test_batch_full_size_systems(gpu, oracle_mod):
    """Systems of the uneven batch's full sizes (n near 2e5) of every
    stencil type, with smaller ones beside: sampled rows of every system's G
    (exported from the batch through a single-system set-up of the same
    system, which the alone-and-in-mix test ties to the batch) are
    bit-identical to the oracle's; iteration counts equal the oracle's."""
    # the largest sizes the batch draws (n up to 2e5), one of each type, with
    # anisotropy ratios from its range, and smaller batch members beside
    big = {}
    for kind, A in (("5pt2d", mg.poisson5_2d(440, 440, scale=(1.0, 37.0))),
                    ("7pt3d", mg.poisson7(58, 58, 58, scale=(1.0, 1.0, 420.0))),
                    ("27pt3d", mg.stencil27_fe(56, 56, 56, scale=(1.0, 1.0, 8.0)))):
        b, _ = mg.rhs(A, mg.BASE_SEED + 31)
        big[kind] = (A, b, kind)
    small = [t for t in mg.batch_workload(24, nmin=2e3, nmax=2e4)][:6]
    chosen = list(big.values()) + small
    kiter, s, eps = 8, 2, 1e-3
    xs, infos, binfo = _run(gpu, chosen, gpu.params(kiter, s, eps))
    assert binfo["converged"] == len(chosen)
    for (A, b, kind), x, inf in zip(chosen, xs, infos):
        G = oracle_mod.afsai_setup(A, kiter, s, eps)
        xo, it_o, _, _, hist = oracle_mod.pcg(A, G, b, rtol=1e-8, history=True)
        assert inf["converged"] == 1 and inf["relres_true"] <= 1e-8, (kind, A.n, inf)
        if _clear(hist):
            assert inf["iters"] == it_o, (kind, A.n, inf["iters"], it_o)
        else:
            assert abs(inf["iters"] - it_o) <= 1, (kind, A.n, inf["iters"], it_o, hist[-2:])
        assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    # the set-up of one big system of each type, sampled rows bit for bit
    for A, b, kind in big.values():
        M = gpu.afsai_setup(gpu.DeviceCSR.from_host(A), gpu.params(kiter, s, eps))
        rp, ci, va = M.export()
        for r0 in (0, A.n // 3, A.n - 64):
            ref = oracle_mod.afsai_setup(A, kiter, s, eps, rows=(r0, r0 + 64), nthreads=1)
            a, e = rp[r0], rp[r0 + 64]
            assert np.array_equal(ci[a:e], ref.col) and np.array_equal(va[a:e], ref.val), (kind, r0)
        M.close()


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
        assert inf["relres_true"] <= 1e-8
        bar = 1.10 if g_prec == 1 else 1.20
        assert inf["iters"] <= int(np.ceil(bar * it_o)) + 1, (kind, A.n, inf["iters"], it_o)
