"""Serving form: continuous batching of solve requests (serve_* C ABI).

Bars: every request converges to the true residual 1e-8 with the oracle's
iteration count (exactly, where the oracle's residual is clear of the
tolerance at its stop); requests submitted while others run are admitted
while those are still on the GPU and overlap with them; each result is
bit-for-bit the same alone and in the mix; the preconditioner of a matrix
is built once (on the set-up thread) and reused; a small memory budget
queues requests instead of failing them."""
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


@pytest.fixture(scope="module")
def pool():
    return [A for A, _, _ in mg.batch_workload(6, seed=mg.BASE_SEED + 9, nmin=300, nmax=4000)]


def _rhs(A, k, nrhs):
    rng = np.random.default_rng(1000 + k)
    return rng.uniform(-1, 1, size=(nrhs, A.n))


def test_server_mix_matches_alone_and_oracle(gpu, oracle_mod, pool):
    afsai = gpu
    prm = afsai.params(8, 2, 1e-3)
    # alone: one server, one request at a time
    alone = {}
    S = afsai.Server(2 << 30, 64, prm)
    ids = [S.register(A) for A in pool]
    for k in range(8):
        m = k % len(pool)
        b = _rhs(pool[m], k, 1 + k % 3)
        x, infos, res = S.wait(S.submit(ids[m], b))
        alone[k] = x
    S.close()
    # mix: all submitted at once to a fresh server
    S = afsai.Server(2 << 30, 64, prm)
    ids = [S.register(A) for A in pool]
    tickets = {}
    for k in range(8):
        m = k % len(pool)
        tickets[k] = (m, S.submit(ids[m], _rhs(pool[m], k, 1 + k % 3)))
    results = {k: S.wait(t) for k, (m, t) in tickets.items()}
    st = S.stats()
    S.close()
    assert st["requests_done"] == 8 and st["solves"] == sum(1 + k % 3 for k in range(8))
    for k, (m, _) in tickets.items():
        x, infos, res = results[k]
        assert res["converged"] == 1 and res["max_relres_true"] <= 1e-8
        assert np.array_equal(x, alone[k]), f"request {k}: mix differs from alone"
        A = pool[m]
        G = oracle_mod.afsai_setup(A, 8, 2, 1e-3)
        b = _rhs(A, k, 1 + k % 3)
        for j in range(b.shape[0]):
            xo, it_o, _, _, hist = oracle_mod.pcg(A, G, b[j], rtol=1e-8, history=True)
            if hist[-1] < 1e-8 * (1 - 1e-6) and hist[-2] > 1e-8 * (1 + 1e-6):
                assert infos[j]["iters"] == it_o, (k, j, infos[j]["iters"], it_o)
            else:
                assert abs(infos[j]["iters"] - it_o) <= 1
            assert infos[j]["relres_true"] <= 1e-8
            assert np.linalg.norm(x[j] - xo) <= 1e-6 * np.linalg.norm(xo)


def test_server_overlap_reuse_and_budget(gpu, pool):
    afsai = gpu
    prm = afsai.params(8, 2, 1e-3)
    # budget just above the matrices + one preconditioner + a few vectors:
    # requests must queue and still complete
    need = sum(4 * (A.n + 1) + 12 * A.nnz for A in pool)
    nmax = max(A.n for A in pool)
    budget = need + 2 * (nmax * 17 * 12 * 2 + 24 * nmax) + 3 * 7 * 8 * nmax
    S = afsai.Server(budget, 16, prm)
    ids = [S.register(A) for A in pool]
    ts = [S.submit(ids[k % len(pool)], _rhs(pool[k % len(pool)], k, 1)) for k in range(12)]
    out = [S.wait(t) for t in ts]
    st = S.stats()
    S.close()
    assert all(r[2]["converged"] == 1 for r in out)
    assert st["peak_mem_bytes"] <= budget
    # a preconditioner evicted for memory is built again at a later request:
    # at most one set-up per request
    assert sum(1 for r in out if r[2]["setup_ms"] > 0.0) <= len(out)
    # plenty of memory: later requests of a matrix reuse its G, and requests overlap
    S = afsai.Server(4 << 30, 64, prm)
    ids = [S.register(A) for A in pool]
    ts = [S.submit(ids[k % len(pool)], _rhs(pool[k % len(pool)], k, 2)) for k in range(18)]
    out = [S.wait(t) for t in ts]
    st = S.stats()
    S.close()
    paid = [r[2]["setup_ms"] > 0 for r in out]
    assert sum(paid) == len(pool)  # one set-up per matrix
    assert st["steps"] < sum(r[2]["max_iters"] for r in out) / 4  # requests shared steps


def test_server_admits_while_others_run(gpu, pool):
    """A long request is on the GPU; requests submitted after it started are
    admitted while it still runs (mid-flight admission: their admission
    time precedes its completion, on the host clock of the submits plus the
    server's own queue and latency times), and every result equals the
    result of the same request served alone."""
    import time

    afsai = gpu
    prm = afsai.params(8, 2, 1e-3)
    big = mg.poisson7(64, 64, 64, scale=(1.0, 1.0, 300.0))
    b_big = _rhs(big, 99, 1)
    S = afsai.Server(8 << 30, 64, prm)
    big_id = S.register(big)
    ids = [S.register(A) for A in pool]
    # the preconditioners exist before the timed part (one request each)
    for m in range(len(pool)):
        S.wait(S.submit(ids[m], _rhs(pool[m], 500 + m, 1)))
    S.wait(S.submit(big_id, _rhs(big, 98, 1), rtol=1e-4))
    t_sub_big = time.perf_counter()
    t_big = S.submit(big_id, b_big, rtol=1e-12)
    t0 = time.time()
    while S.stats()["running"] == 0:
        assert time.time() - t0 < 30
        time.sleep(0.0002)
    late, t_sub_late = [], []
    for k in range(6):
        t_sub_late.append(time.perf_counter())
        late.append(S.submit(ids[k % len(pool)], _rhs(pool[k % len(pool)], k, 1)))
    late_res = [S.wait(t) for t in late]
    big_res = S.wait(t_big)
    st = S.stats()
    S.close()
    big_done = t_sub_big + big_res[2]["latency_ms"] / 1e3
    admitted = [ts + r[2]["queue_ms"] / 1e3 for ts, r in zip(t_sub_late, late_res)]
    assert all(a < big_done for a in admitted), (admitted, big_done)
    assert all(r[2]["converged"] == 1 and r[2]["max_relres_true"] <= 1e-8 for r in late_res)
    assert big_res[2]["converged"] == 1 and big_res[2]["max_relres_true"] <= 1e-12
    # alone
    S = afsai.Server(8 << 30, 64, prm)
    big_id = S.register(big)
    ids = [S.register(A) for A in pool]
    x_big = S.wait(S.submit(big_id, b_big, rtol=1e-12))[0]
    for k, r in enumerate(late_res):
        x_alone = S.wait(S.submit(ids[k % len(pool)], _rhs(pool[k % len(pool)], k, 1)))[0]
        assert np.array_equal(x_alone, r[0]), k
    S.close()
    assert np.array_equal(x_big, big_res[0])
