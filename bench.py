"""Benchmark: aFSAI set-up + PCG to relative residual 1e-8 on one GB300.

Workload (default): heterogeneous diffusion, cell-centred 7-point stencil on
a 256^3 grid (n = 16,777,216, 117,047,296 nonzeros), lognormal coefficient
(sigma 2, smoothed over 8 cells), harmonic face means; aFSAI kiter = 5,
s = 2, eps = 1e-3; seeded right-hand side b = A x*, x* ~ U[-1, 1].  A step
is one whole solve in the FP64 form: aFSAI set-up (pattern search, gather,
Cholesky, scaling, G^T) followed by PCG from x = 0 until ||r|| <= 1e-8 ||b||
(and the true residual too), with A and b resident in device memory.  The
metric is seconds per solve (lower is better).  --workload elast48 runs the
48^3 elasticity problem instead.

Other keys of the JSON line:
  forms        the other precision forms on the same input (FP32 G, BF16 G,
               the mixed form with FP32 Cholesky + one FP64 refinement step,
               and Jacobi), seconds per solve, iterations and the error of
               their G against the FP64 G
  e2e          the same solve through afsai_solve_host from pinned host
               buffers (H2D of A and b, D2H of x inside the timed region)
  roofline     the dominant kernel against its roof (measured with CUDA
               events on the launching stream inside the timed region)
  cpu_baseline the FP64 CPU oracle on a bounded sample of the same solve,
               at all cores and at one thread, scaled to seconds per solve
  clocks       SM clocks and throttle reasons sampled during the timed region

--impl reference times the CPU oracle (the only reference this method has:
the paper's code is not public) on the host cores: its timed steps add up
to one whole oracle solve of the workload.
Multi-GPU (--gpus N under torchrun): every rank solves its own copy of the
workload (independent problems, no collective on the data path); value is
the max-over-ranks time divided by the number of solves of all ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "aFSAI set-up+PCG s/solve to relres 1e-8 (FP64; mixed reported beside)"
WORKLOAD_NAMES = {"elast48": "elasticity_hex48", "hetero256": "hetero_diffusion7_256", "poisson20": "poisson7_20",
                  "batch512": "batch_uneven", "serve": "serve_poisson_arrivals", "poisson_sweep": "poisson7_sweep"}
# precision forms: storage/arithmetic of G and of the row Cholesky solves
FORMS = {
    "fp64": dict(g_prec=0, chol_prec=0, desc="FP64 G, FP64 Cholesky"),
    "mixed": dict(g_prec=1, chol_prec=1, desc="FP32 G, FP32 Cholesky + one FP64 refinement step"),
    "g32": dict(g_prec=1, chol_prec=0, desc="FP32 G, FP64 Cholesky"),
    "bf16": dict(g_prec=2, chol_prec=1, desc="BF16 G, FP32 Cholesky + one FP64 refinement step"),
    # the paper's comparison preconditioner (Section 5.2): kiter = 0 keeps
    # the diagonal pattern, G^T G = diag(A)^{-1}
    "jacobi": dict(g_prec=0, chol_prec=0, kiter=0, desc="Jacobi (aFSAI with kiter = 0), FP64"),
    # locality bound of the distributed set-up (Section 4): 64 row stripes,
    # stripe graph of G inside lower(Ahat^k)
    "local64k1": dict(g_prec=0, chol_prec=0, stripes=64, power=1,
                      desc="FP64, candidates bounded to lower(Ahat^1) over 64 row stripes"),
    "local64k2": dict(g_prec=0, chol_prec=0, stripes=64, power=2,
                      desc="FP64, candidates bounded to lower(Ahat^2) over 64 row stripes"),
    "local64k0": dict(g_prec=0, chol_prec=0, stripes=64, power=0,
                      desc="FP64, candidates bounded to each row's own stripe of 64 (block-diagonal aFSAI)"),
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def source_digest(paths):
    import hashlib

    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel_key, units):
    """DRAM bytes per launch of `kernel_key` from the committed ncu record,
    scaled to `units` rows; None if absent or the kernel source changed."""
    try:
        rec = json.load(open(TRAFFIC_FILE))[kernel_key]
    except Exception:
        return None, "no ncu record"
    if rec.get("source_digest") != source_digest(rec["sources"]):
        return None, "kernel changed since the ncu capture"
    # units = 1: the record is per launch, scaled to the full-size workload
    # by its own factor (rows of the full problem / rows of the capture)
    scale = rec.get("scale_to_full", 1.0) if units == 1 else units / rec["units"]
    return rec["dram_bytes"] * scale, (f"ncu {rec['capture']}: {rec['dram_bytes']:.4g} B over {rec['units']} rows, "
                                       f"scaled x{scale:.4g}")



def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=None, help="grid size override (testing only)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the other precision forms")
    ap.add_argument("--workload", default="hetero256",
                    choices=["elast48", "hetero256", "poisson20", "batch512", "serve", "poisson_sweep"])
    ap.add_argument("--requests", type=int, default=2000, help="timed requests of the serve workload")
    ap.add_argument("--warm-requests", type=int, default=200)
    ap.add_argument("--nsys", type=int, default=512, help="systems of the batch512 workload")
    ap.add_argument("--form", default="fp64", choices=list(FORMS), help="precision form of the timed line")
    ap.add_argument("--extra-forms", default=None,
                    help="comma list of other forms reported beside (default: mixed; hetero256: g32,bf16,mixed)")
    return ap.parse_args()


def dist_init(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "gb300" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(v, world, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        # raw samples: $BENCH_CLOCKS_DIR (default: the system temp folder)
        import tempfile

        self.path = os.path.join(os.environ.get("BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def setup_flops(rowptr_G, steps, s, nnz_row_avg):
    """Algorithmic FP64 flops of the set-up: per row and step k with pattern
    size m_k: m_k^3/3 (Cholesky) + 2 m_k^2 (triangular solves) +
    2 nnz_row |P_{k-1}| (Kaporin gradient), with m_k = min(1 + k s, m_final)."""
    m_final = np.diff(rowptr_G).astype(np.float64)
    total = 0.0
    kmax = int(steps.max()) if steps.size else 0
    for k in range(1, kmax + 1):
        act = steps >= k
        mk = np.minimum(1 + k * s, m_final[act])
        mprev = np.minimum(1 + (k - 1) * s, m_final[act])
        total += float(np.sum(mk ** 3 / 3.0 + 2 * mk ** 2 + 2 * nnz_row_avg * mprev))
    return total


def setup_touched_bytes(rowptr_G, steps, s, nnz_row_avg):
    """Bytes the set-up touches without cache reuse: per row and step the
    rows of A read by the gradient (|P_{k-1}| of them) and by the gather
    (the s new ones), 12 B per entry plus 8 B of row pointers, plus the
    written row of G (12 B per entry)."""
    m_final = np.diff(rowptr_G).astype(np.float64)
    total = float(np.sum(m_final)) * 12.0
    kmax = int(steps.max()) if steps.size else 0
    for k in range(1, kmax + 1):
        act = steps >= k
        mprev = np.minimum(1 + (k - 1) * s, m_final[act])
        mk = np.minimum(1 + k * s, m_final[act])
        total += float(np.sum((mprev + (mk - mprev)) * (12.0 * nnz_row_avg + 8.0)))
    return total


def g_difference(G_ref, G_other, n):
    """||G - G_ref||_F / ||G_ref||_F, the largest entrywise relative
    difference on entries present in both, and the fraction of rows whose
    pattern equals the reference's."""
    import scipy.sparse as sp

    def csr(t):
        rp, ci, va = t
        return sp.csr_matrix((np.asarray(va, dtype=np.float64), ci, rp), shape=(n, n))

    R, O = csr(G_ref), csr(G_other)
    D = O - R
    rel_fro = float(sp.linalg.norm(D) / sp.linalg.norm(R))
    lr, lo = np.diff(R.indptr), np.diff(O.indptr)
    row = np.repeat(np.arange(n), lr)
    eq = lr[row] == lo[row]
    e = np.arange(R.nnz)
    match = np.zeros(R.nnz, dtype=bool)
    idx = e[eq] + (O.indptr[row[eq]] - R.indptr[row[eq]])
    match[eq] = R.indices[eq] == O.indices[idx]
    bad_rows = np.zeros(n, dtype=bool)
    np.logical_or.at(bad_rows, row[~match], True)
    same_rows = int(np.count_nonzero((lr == lo) & ~bad_rows))
    # largest entrywise relative difference over the rows whose pattern is
    # the reference's (entries align one to one there)
    good = (lr == lo) & ~bad_rows
    sel = good[row]
    max_rel = None
    if sel.any():
        o_idx = e[sel] + (O.indptr[row[sel]] - R.indptr[row[sel]])
        rvals = np.asarray(R.data, dtype=np.float64)[sel]
        max_rel = float(np.max(np.abs(np.asarray(O.data, dtype=np.float64)[o_idx] - rvals) / np.abs(rvals)))
    return {"rel_frobenius": rel_fro, "max_rel_same_pattern_rows": max_rel, "rows_same_pattern": same_rows / n}


def pcg_iteration_bytes(A, sinfo, form):
    """Algorithmic bytes of one PCG iteration: A (12 B/entry + row
    pointers), G and G^T ((4 + w) B/entry + row pointers, w the G value
    size) and ~140 B per row of vector traffic."""
    w = {0: 8, 1: 4, 2: 2}[FORMS[form]["g_prec"]]
    return 12 * A.nnz + 2 * (4 + w) * sinfo["nnz_G"] + 12 * A.n + 140 * A.n


def _measured_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0  # fallback figure of the pool


MEASURED_HBM_GBS = _measured_hbm()


def spmv_bytes(n, nnz, val_bytes=8, x_bytes=8, y_bytes=8):
    """Compulsory bytes of y = A x: values, columns, row pointers, x once,
    y once."""
    return nnz * (val_bytes + 4) + 4 * (n + 1) + n * x_bytes + n * y_bytes


FP64_DFMA_PER_S = 152 * 2 * 2.07e9  # derived FP64 peak: SMs x DFMA/clk x max clock (no measured FP64 figure)


def setup_roofline(key, flops, kern_ms, rp, steps, p, A, form):
    """The set-up kernels against their roof: the FP64 ALU for the FP64
    Cholesky (algorithmic flops), the measured HBM bandwidth for the FP32
    Cholesky (method-touched bytes)."""
    traffic, traffic_note = measured_traffic(key, A.n)
    if FORMS[form]["chol_prec"] == 0:
        r = {"kernel": key, "bound": "alu", "achieved": flops / (kern_ms * 1e-3) / 1e12,
             "peak": 2 * FP64_DFMA_PER_S / 1e12, "unit": "TFLOP/s", "traffic": traffic, "traffic_note": traffic_note,
             "kernel_ms": kern_ms, "algorithmic_flops": flops,
             "peak_source": "FP64 ALU: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived from unit counts)"}
    else:
        touched = setup_touched_bytes(rp, steps, p["s"], A.nnz / A.n)
        r = {"kernel": key, "bound": "hbm", "achieved": touched / (kern_ms * 1e-3) / 1e9, "peak": MEASURED_HBM_GBS,
             "unit": "GB/s", "traffic": traffic, "traffic_note": traffic_note, "kernel_ms": kern_ms,
             "algorithmic_bytes": touched, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    r["frac"] = r["achieved"] / r["peak"]
    return r


def pcg_kernel_table(A, nnz_G, form, kms):
    """Roofline of each PCG kernel from its in-graph device time (ms):
    algorithmic bytes (matrix entries and row pointers once, each vector
    read or written once) and FP64 fmas; the binding roof is the larger of
    bytes / measured HBM bandwidth and fmas / derived FP64 rate."""
    n, nnzA = A.n, A.nnz
    w = {0: 8, 1: 4, 2: 2}[FORMS[form]["g_prec"]]
    f64g = FORMS[form]["g_prec"] == 0
    rows = [
        # key, kernel, bytes, FP64 fmas
        ("pcg_A", "k_spmv_A_dot (q = A p, p.q)", 12 * nnzA + 4 * (n + 1) + 8 * n + 8 * n, nnzA + n),
        ("pcg_xr", "k_update_xr (x, r update, r.r)", 48 * n, 3 * n),
        ("pcg_G", "k_spmv_G (t = G r)", (4 + w) * nnz_G + 4 * (n + 1) + 8 * n + 8 * n, nnz_G if f64g else 0),
        ("pcg_Gt", "k_spmv_Gt_dot (z = G^T t, r.z)", (4 + w) * nnz_G + 4 * (n + 1) + 3 * 8 * n,
         (nnz_G if f64g else 0) + n),
        ("pcg_p", "k_update_p (p = z + beta p)", 24 * n, n),
    ]
    out = []
    for (key, name, by, dfma), ms in zip(rows, kms):
        ms = float(ms)
        if by / (MEASURED_HBM_GBS * 1e9) >= dfma / FP64_DFMA_PER_S:
            ach = by / (ms * 1e-3) / 1e9 if ms > 0 else None
            rec = {"bound": "hbm", "achieved": ach, "peak": MEASURED_HBM_GBS, "unit": "GB/s"}
        else:
            ach = 2 * dfma / (ms * 1e-3) / 1e12 if ms > 0 else None
            rec = {"bound": "alu", "achieved": ach, "peak": 2 * FP64_DFMA_PER_S / 1e12, "unit": "TFLOP/s"}
        rec.update({"key": key, "kernel": name, "ms": ms, "bytes": by, "dfma": dfma,
                    "frac": (rec["achieved"] / rec["peak"]) if rec["achieved"] else None})
        out.append(rec)
    return out


def make_workload(name, scale):
    from paper_2010_14175_gb300 import matgen as mg

    A, b, xs, p = mg.workload(name, scale=scale)
    return A, b, p


def job_value(ms_total, steps, world):
    """Seconds per solve of the whole job: the max-over-ranks time of the
    timed region divided by the solves of all ranks (each rank solves its
    own copy of the workload: replicas, weak scaling)."""
    return ms_total / 1e3 / (steps * world)


def _cpu_model():
    try:
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def _middle_rows(n, frac):
    k = max(1, int(n * frac))
    r0 = max(0, n // 2 - k // 2)
    return r0, min(n, r0 + k)


def cpu_oracle_sample(A, b, p, iters, setup_frac_1t=1 / 32, pcg_iters_all=2, pcg_iters_1t=1):
    """The CPU oracle (as it stands) on a bounded sample of one solve, at
    all cores and at one thread, scaled to seconds per solve:
      all cores  the full oracle set-up (timed; its G serves the PCG
                 timings) + `pcg_iters_all` oracle PCG iterations (timed),
                 scaled to `iters` iterations;
      one thread the set-up of a block of rows from the middle of the
                 matrix (`setup_frac_1t` of the rows; rows are independent)
                 scaled to all rows + `pcg_iters_1t` PCG iterations scaled
                 to `iters`.
    `iters` is the FP64 iteration count of the solve being compared."""
    import oracle

    cores = oracle.num_threads()
    t0 = time.perf_counter()
    G = oracle.afsai_setup(A, p["kiter"], p["s"], p["eps"])
    t_setup = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.pcg(A, G, b, rtol=1e-300, maxit=pcg_iters_all)
    t_it = (time.perf_counter() - t0) / pcg_iters_all
    all_cores = t_setup + t_it * iters
    before = oracle.set_threads(1)
    try:
        r0, r1 = _middle_rows(A.n, setup_frac_1t)
        t0 = time.perf_counter()
        oracle.afsai_setup(A, p["kiter"], p["s"], p["eps"], rows=(r0, r1), nthreads=1)
        t_setup1 = (time.perf_counter() - t0) * A.n / (r1 - r0)
        t0 = time.perf_counter()
        oracle.pcg(A, G, b, rtol=1e-300, maxit=pcg_iters_1t)
        t_it1 = (time.perf_counter() - t0) / pcg_iters_1t
    finally:
        oracle.set_threads(before)
    one = t_setup1 + t_it1 * iters
    return {
        "value": all_cores, "unit": "s/solve", "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
        "sample": (f"all {cores} cores: full oracle set-up ({t_setup:.2f} s, measured) + {pcg_iters_all} oracle PCG "
                   f"iterations ({t_it * 1e3:.0f} ms each) scaled to {iters} iterations; the iteration count is "
                   f"that of the FP64 solve timed on the GPU"),
        "one_thread": {"value": one, "unit": "s/solve", "cores": 1,
                       "sample": (f"set-up of rows [{r0}, {r1}) at one thread ({t_setup1:.1f} s scaled to all "
                                  f"{A.n} rows) + {pcg_iters_1t} PCG iteration(s) at one thread "
                                  f"({t_it1 * 1e3:.0f} ms each) scaled to {iters} iterations")},
        "extrapolated": True,
    }


def run_reference(args, rank, world):
    """--impl reference: the CPU oracle, as it stands, on the host cores
    (rank 0 only; the other ranks return at once).  The K timed steps
    together make up ONE whole oracle solve of the workload, measured and
    not extrapolated: step k runs the oracle set-up of the k-th of K row
    blocks (rows are independent, so the blocks add up to the full
    set-up), and step 0 also runs the oracle's PCG from x = 0 to the 1e-8
    stopping rule with the full G (built once before the timed steps).
    value = the sum of the K step times = seconds for one whole solve."""
    if rank != 0:
        return None
    import oracle

    A, b, p = make_workload(args.workload, args.scale)
    K = max(1, args.steps)
    G = oracle.afsai_setup(A, p["kiter"], p["s"], p["eps"])  # the PCG's G (untimed)
    bounds = [(A.n * k) // K for k in range(K + 1)]
    for w in range(args.warmup):  # a small block each
        r0, r1 = _middle_rows(A.n, min(0.01, 1.0 / K))
        oracle.afsai_setup(A, p["kiter"], p["s"], p["eps"], rows=(r0, r1))
    times, iters, rt = [], None, None
    for k in range(K):
        t0 = time.perf_counter()
        if bounds[k + 1] > bounds[k]:
            oracle.afsai_setup(A, p["kiter"], p["s"], p["eps"], rows=(bounds[k], bounds[k + 1]))
        if k == 0:
            _, iters, _, rt = oracle.pcg(A, G, b, rtol=1e-8, maxit=20000)
        times.append(time.perf_counter() - t0)
    value = float(sum(times))
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": value * 1e3 / K, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
        "config": {"workload": WORKLOAD_NAMES[args.workload] + "_fp64", "n": A.n, "nnz": A.nnz,
                   "kiter": p["kiter"], "s": p["s"], "eps": p["eps"], "rtol": 1e-8, "oracle_iters": iters,
                   "oracle_relres_true": rt},
        "cpu_baseline": {"value": value, "unit": "s/solve", "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
                         "extrapolated": False,
                         "sample": (f"one whole oracle solve split over the {K} timed steps: the set-up of "
                                    f"{K} row blocks (one per step) and the PCG to 1e-8 ({iters} iterations, "
                                    f"in step 0)")},
        "e2e": {"value": value, "unit": "s/solve", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return line


def run_batch(args, rank, world, local):
    """Batched form: nsys uneven systems (2D 5-point, 3D 7-point, 3D 27-point,
    anisotropy up to 1e3, n log-uniform in [2e3, 2e5]) solved by one
    afsai_batch_solve per step; value = seconds per system solve.  Reported
    beside: the same batch in FP64, and the plain FP64 GPU path solving the
    systems one after another (afsai_setup + pcg_solve each)."""
    import torch

    from paper_2010_14175_gb300 import afsai, matgen as mg

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    afsai.load()
    systems = mg.batch_workload(args.nsys)
    As = [afsai.DeviceCSR.from_host(A, device=dev) for A, _, _ in systems]
    bs = [torch.from_numpy(b).to(dev) for _, b, _ in systems]
    xs = [torch.zeros_like(b) for b in bs]
    stream = torch.cuda.current_stream(dev)
    kiter, s_, eps = 8, 2, 1e-3
    form = args.form if args.form != "fp64" or args.extra_forms == "none" else "mixed"

    def prm_of(f):
        return afsai.params(kiter, s_, eps, 0, FORMS[f]["g_prec"], FORMS[f]["chol_prec"])

    def batch_once(f):
        for x in xs:
            x.zero_()
        return afsai.afsai_batch_solve(As, prm_of(f), bs, xs, rtol=1e-8, maxit=20000, stream=stream)

    for _ in range(args.warmup):
        batch_once(form)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = afsai.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    binfos = []
    for _ in range(args.steps):
        infos, binfo = batch_once(form)
        binfos.append(binfo)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = afsai.kernel_launches() - launches0
    clk = clocks.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev) / args.steps
    nsys = len(systems)
    value = ms / 1e3 / (nsys * world)
    iters = np.array([i["iters"] for i in infos])
    worst = max(i["relres_true"] for i in infos)
    ntot = sum(A.n for A, _, _ in systems)
    nnz = sum(A.nnz for A, _, _ in systems)
    w = {0: 8, 1: 4, 2: 2}[FORMS[form]["g_prec"]]
    nnzg = binfos[-1]["nnz_G"]
    # batched PCG bytes: every system's iterations x its per-iteration bytes
    by = 0.0
    for (A, _, _), it in zip(systems, iters):
        by += it * (12 * A.nnz + 2 * (4 + w) * nnzg * A.n / ntot + 152 * A.n)
    solve_ms = float(np.median([b["solve_ms"] for b in binfos]))
    setup_ms = float(np.median([b["setup_ms"] for b in binfos]))
    roof = {"kernel": "batched PCG (kb_* kernels)", "bound": "hbm", "achieved": by / (solve_ms * 1e-3) / 1e9,
            "peak": MEASURED_HBM_GBS, "unit": "GB/s", "frac": None, "traffic": None,
            "traffic_note": "no ncu record for the batched kernels", "algorithmic_bytes": by,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    extra = {}
    if args.extra_forms != "none":
        # the same batch in FP64
        batch_once("fp64")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        inf64, b64 = batch_once("fp64")
        e1.record(stream)
        torch.cuda.synchronize()
        extra["batched_fp64"] = {"value": e0.elapsed_time(e1) / 1e3 / nsys, "unit": "s/solve",
                                 "max_iters": b64["max_iters"], "setup_ms": b64["setup_ms"],
                                 "solve_ms": b64["solve_ms"]}
        it64 = np.array([i["iters"] for i in inf64])
        extra["iters_vs_fp64_max_ratio"] = float(np.max(iters / np.maximum(it64, 1)))
        # plain FP64 GPU path, one system after another (engines tuned in a first pass)
        def sequential():
            for A, b, x in zip(As, bs, xs):
                x.zero_()
                M = afsai.afsai_setup(A, prm_of("fp64"), stream)
                afsai.pcg_solve(A, M, b, x, rtol=1e-8, maxit=20000, stream=stream)
                M.close()
        sequential()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sequential()
        torch.cuda.synchronize()
        extra["sequential_fp64"] = {"value": (time.perf_counter() - t0) / nsys, "unit": "s/solve",
                                    "desc": "afsai_setup + pcg_solve per system, FP64, one after another"}
    # end to end from pinned host buffers: every system's A and b copied in,
    # the batched solve, every x read back, inside the timed region
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        host = [(pin(np.asarray(A.rowptr, np.int32)), pin(np.asarray(A.col, np.int32)),
                 pin(np.asarray(A.val, np.float64)), pin(np.asarray(b, np.float64))) for A, b, _ in systems]
        xh = [torch.zeros(A.n, dtype=torch.float64).pin_memory() for A, _, _ in systems]

        def e2e_once():
            Ads, bds, xds = [], [], []
            for (A, _, _), (rp, ci, va, bh) in zip(systems, host):
                Ads.append(afsai.DeviceCSR(A.n, rp.to(dev, non_blocking=True), ci.to(dev, non_blocking=True),
                                           va.to(dev, non_blocking=True)))
                bds.append(bh.to(dev, non_blocking=True))
                xds.append(torch.zeros_like(bds[-1]))
            afsai.afsai_batch_solve(Ads, prm_of(form), bds, xds, rtol=1e-8, maxit=20000, stream=stream)
            for xd, xo in zip(xds, xh):
                xo.copy_(xd, non_blocking=True)
            torch.cuda.synchronize()

        e2e_once()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_once()
        te = (time.perf_counter() - t0) / args.steps
        e2e = {"value": te / nsys, "unit": "s/solve",
               "h2d_bytes_per_step": int(sum(4 * (A.n + 1) + 12 * A.nnz + 8 * A.n for A, _, _ in systems)),
               "d2h_bytes_per_step": int(sum(8 * A.n for A, _, _ in systems))}
    # the CPU oracle on a bounded sample of the batch: whole solves (set-up
    # and PCG to 1e-8) of every 32nd system, all cores, scaled by rows
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle

        sample = systems[::32]
        t0 = time.perf_counter()
        for A, b, _ in sample:
            Go = oracle.afsai_setup(A, kiter, s_, eps)
            oracle.pcg(A, Go, b, rtol=1e-8, maxit=20000)
        ts = time.perf_counter() - t0
        rows_s = sum(A.n for A, _, _ in sample)
        cpu = {"value": ts / rows_s * ntot / nsys, "unit": "s/solve", "cores": oracle.num_threads(), "kind": "oracle",
               "cpu": _cpu_model(), "extrapolated": True,
               "sample": f"whole FP64 oracle solves of {len(sample)} of the {nsys} systems (every 32nd, "
                         f"{rows_s} rows, {ts:.1f} s), scaled by rows to the batch and divided by {nsys} systems"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if form == "fp64" else "f64+f32", "data": "synthetic (seeded generator)",
            "config": {"workload": f"batch_uneven_{nsys}_{form}", "nsys": nsys, "total_rows": ntot, "total_nnz": nnz,
                       "kiter": kiter, "s": s_, "eps": eps, "rtol": 1e-8, "form": FORMS[form]["desc"],
                       "l2": "inputs larger than L2", "parallelism": f"replicas x{world}"},
            "setup_ms": setup_ms, "solve_ms": solve_ms, "pcg_iters_max": int(iters.max()),
            "pcg_iters_median": float(np.median(iters)), "relres_true_max": worst,
            "converged": binfos[-1]["converged"], "graph_launches": binfos[-1]["graph_launches"],
            "setup_rows_per_s": ntot / (setup_ms * 1e-3), "gpu_launches": int(launches), "roofline": roof,
            "forms": extra, "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_serve(args, rank, world, local):
    """Serving form: a pool of 64 matrices from the uneven-batch
    distribution; requests pick a matrix uniformly and bring 1..8
    right-hand sides; arrivals are a Poisson process at 70% of the
    server's measured capacity (solves/s when saturated); G is built at a
    matrix's first request and reused.  Reports p50/p99 latency (submit ->
    completion, measured by the server) and solves/s, beside the plain FP64
    path serving the same requests one at a time."""
    import torch

    from paper_2010_14175_gb300 import afsai, matgen as mg

    torch.cuda.set_device(local)
    afsai.load()
    rng = np.random.Generator(np.random.PCG64(mg.BASE_SEED + 5))
    pool = [A for A, _, _ in mg.batch_workload(64, seed=mg.BASE_SEED + 4)]
    form = args.form if args.form != "fp64" else "mixed"
    f = FORMS[form]
    prm = afsai.params(8, 2, 1e-3, 0, f["g_prec"], f["chol_prec"])
    S = afsai.Server(150 << 30, 512, prm, maxit=20000, iters_per_step=4)
    ids = [S.register(A) for A in pool]

    def make_request():
        m = int(rng.integers(0, len(pool)))
        nrhs = int(rng.integers(1, 9))
        return m, rng.uniform(-1, 1, size=(nrhs, pool[m].n))

    def drain(tickets):
        done = []
        while tickets:
            keep = []
            for t in tickets:
                r = S.poll(t)
                if r is None:
                    keep.append(t)
                else:
                    done.append(r)
            tickets = keep
            if tickets:
                time.sleep(0.0005)
        return done

    # capacity: saturate the server (all matrices' G built by a first pass);
    # one untimed burst, then the median of three timed bursts of 256
    # requests (a single burst varied by 1.5x from run to run, and the
    # arrival rate, hence the load, follows it)
    drain([S.submit(ids[m], np.ones(pool[m].n)) for m in range(len(pool))])
    caps = []
    for k in range(4):
        burst = [make_request() for _ in range(256)]
        t0 = time.perf_counter()
        drain([S.submit(ids[m], b) for m, b in burst])
        if k > 0:
            caps.append(sum(b.shape[0] for _, b in burst) / (time.perf_counter() - t0))
    capacity = float(np.median(caps))  # solves/s
    mean_rhs = 4.5
    lam = 0.7 * capacity / mean_rhs  # requests/s
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = afsai.kernel_launches()

    def poisson_run(nreq, trace=None):
        outstanding, done = [], []
        t_next = time.perf_counter()
        start = t_next
        for _ in range(nreq):
            t_next += rng.exponential(1.0 / lam)
            m, b = make_request()
            if trace is not None:
                trace.append((t_next - start, m, b))
            while True:
                now = time.perf_counter()
                if now >= t_next:
                    break
                keep = []
                for t in outstanding:
                    r = S.poll(t)
                    if r is None:
                        keep.append(t)
                    else:
                        done.append(r)
                outstanding = keep
                if t_next - now > 0.0005:
                    time.sleep(min(0.0005, t_next - now))
            outstanding.append(S.submit(ids[m], b))
        done += drain(outstanding)
        return done, time.perf_counter() - start

    poisson_run(args.warm_requests)
    trace = []
    done, wall = poisson_run(args.requests, trace)
    launches = afsai.kernel_launches() - launches0
    clk = clocks.stop()
    st = S.stats()
    S.close()
    lat = np.array([r[2]["latency_ms"] for r in done])
    qms = np.array([r[2]["queue_ms"] for r in done])
    sms = np.array([r[2]["setup_ms"] for r in done])
    solves = sum(r[2]["nrhs"] for r in done)
    worst = max(r[2]["max_relres_true"] for r in done)
    conv = all(r[2]["converged"] == 1 for r in done)
    # the plain FP64 path serving the SAME arrival trace one request at a
    # time (G cached per matrix): each request's service time is measured
    # (pcg_solve per right-hand side, b copied in and x read back), and it
    # starts when it has arrived and the previous one has finished, so its
    # latency includes its queueing
    Ad = [afsai.DeviceCSR.from_host(A) for A in pool]
    Ms = {}
    for m in set(m for _, m, _ in trace):
        Ms[m] = afsai.afsai_setup(Ad[m], afsai.params(8, 2, 1e-3))
    torch.cuda.synchronize()
    lat_seq, svc = [], []
    clock_free = 0.0
    for arr, m, b in trace:
        t1 = time.perf_counter()
        for j in range(b.shape[0]):
            bd = torch.from_numpy(b[j]).cuda()
            x = torch.zeros_like(bd)
            afsai.pcg_solve(Ad[m], Ms[m], bd, x, rtol=1e-8, maxit=20000)
            x.cpu()
        service = time.perf_counter() - t1
        svc.append(service * 1e3)
        start = max(arr, clock_free)
        clock_free = start + service
        lat_seq.append((clock_free - arr) * 1e3)
    seq_solves = sum(b.shape[0] for _, _, b in trace) / (sum(svc) / 1e3)
    for Mm in Ms.values():
        Mm.close()
    if rank == 0:
        line = {
            "metric": METRIC + "; serve p50/p99 ms", "value": float(np.percentile(lat, 50)) / 1e3, "unit": "s/request",
            "n_gpus": world, "steps": args.requests, "warmup": args.warm_requests,
            "ms_per_step": float(np.percentile(lat, 50)), "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic (seeded generator, Poisson arrivals)",
            "config": {"workload": f"serve_pool64_{form}", "arrival_rate_req_s": lam, "capacity_solves_s": capacity,
                       "load": 0.7, "nrhs": "U{1..8}", "pool": 64, "budget_gb": 150, "iters_per_step": 4,
                       "form": FORMS[form]["desc"], "parallelism": f"replicas x{world}"},
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "solves_per_s": solves / wall, "requests": len(done),
            "queue_ms": {"p50": float(np.percentile(qms, 50)), "p99": float(np.percentile(qms, 99))},
            "setup_ms": {"p50": float(np.percentile(sms, 50)), "p99": float(np.percentile(sms, 99)),
                         "requests_paying": int((sms > 0).sum())},
            "all_converged": conv, "relres_true_max": worst, "server_steps": st["steps"],
            "peak_mem_gb": st["peak_mem_bytes"] / 2 ** 30, "gpu_launches": int(launches),
            "sequential_fp64": {"solves_per_s": seq_solves, "p50_ms": float(np.percentile(lat_seq, 50)),
                                "p99_ms": float(np.percentile(lat_seq, 99)),
                                "service_p50_ms": float(np.percentile(svc, 50)),
                                "service_p99_ms": float(np.percentile(svc, 99)), "requests": len(trace),
                                "desc": "the same arrival trace served one request at a time by pcg_solve per "
                                        "right-hand side (G cached): latency = queueing + measured service"},
            "p99_vs_sequential": float(np.percentile(lat, 99)) / float(np.percentile(lat_seq, 99)),
            "roofline": None, "e2e": {"value": float(np.percentile(lat, 50)) / 1e3, "unit": "s/request",
                                      "h2d_bytes_per_step": None, "d2h_bytes_per_step": None},
            "cpu_baseline": None, "clocks": clk,
        }
        print(json.dumps(line), flush=True)


def run_sweep(args, rank, world, local):
    """Single-GPU size sweep of the 7-point Poisson problem (the analogue of
    the paper's weak-scaling study, which keeps 121^3 = 1,771,561 rows per
    GPU): set-up time per row and PCG time per iteration against n, FP64
    and mixed forms.  The JSON line's value is the s/solve of the 121^3 case."""
    import torch

    from paper_2010_14175_gb300 import afsai, matgen as mg

    torch.cuda.set_device(local)
    afsai.load()
    rows = []
    value = None
    for N in (32, 64, 96, 121, 160, 200):
        A = mg.poisson7(N)
        b, _ = mg.rhs(A, mg.BASE_SEED + N)
        Ad = afsai.DeviceCSR.from_host(A)
        bd = torch.from_numpy(b).cuda()
        x = torch.zeros_like(bd)
        rec = {"N": N, "n": A.n}
        for form in ("fp64", "mixed"):
            f = FORMS[form]
            prm = afsai.params(5, 2, 1e-3, 0, f["g_prec"], f["chol_prec"])
            ts, ss, its = [], [], []
            reps = max(3, args.steps)  # median of at least three timed solves per size
            for rep in range(args.warmup + reps):
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                M = afsai.afsai_setup(Ad, prm)
                inf = afsai.pcg_solve(Ad, M, bd, x, rtol=1e-8, maxit=20000)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                if rep >= args.warmup:
                    ts.append(t1 - t0)
                    ss.append(M.info()["setup_ms"])
                    its.append(inf)
                M.close()
            rec[form] = {"s_per_solve": float(np.median(ts)), "setup_ns_per_row": float(np.median(ss)) * 1e6 / A.n,
                         "iters": its[-1]["iters"], "us_per_iter": its[-1]["solve_ms"] * 1e3 / max(1, its[-1]["iters"]),
                         "relres_true": its[-1]["relres_true"]}
        rows.append(rec)
        if N == 121:
            value = rec["fp64"]["s_per_solve"]
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                          "dtype": "f64", "data": "synthetic (7-point Poisson, Dirichlet)",
                          "config": {"workload": "poisson7_sweep", "kiter": 5, "s": 2, "eps": 1e-3, "rtol": 1e-8},
                          "sweep": rows, "roofline": None, "e2e": None, "cpu_baseline": None}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_init(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch512":
        run_batch(args, rank, world, local)
        return
    if args.workload == "serve":
        run_serve(args, rank, world, local)
        return
    if args.workload == "poisson_sweep":
        run_sweep(args, rank, world, local)
        return
    import torch

    from paper_2010_14175_gb300 import afsai

    assert torch.cuda.is_available(), "bench needs a GPU"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    afsai.load()
    A, b, p = make_workload(args.workload, args.scale)
    Ad = afsai.DeviceCSR.from_host(A, device=dev)
    bd = torch.from_numpy(b).to(dev)
    x = torch.zeros_like(bd)
    stream = torch.cuda.current_stream(dev)

    def prm_of(form):
        f = FORMS[form]
        br = -(-A.n // f["stripes"]) if "stripes" in f else 0
        return afsai.params(f.get("kiter", p["kiter"]), p["s"], p["eps"], 0, f["g_prec"], f["chol_prec"], br,
                            f.get("power", 1))

    def one_solve(prm_):
        x.zero_()
        M = afsai.afsai_setup(Ad, prm_, stream)
        info = afsai.pcg_solve(Ad, M, bd, x, rtol=1e-8, maxit=20000, stream=stream)
        return M, M.info(), info

    prm = prm_of(args.form)
    for _ in range(args.warmup):
        M, sinfo, pinfo = one_solve(prm)
        M.close()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = afsai.kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    setup_ms, solve_ms, iters, kernel_ms, pcg_kernel_ms = [], [], [], [], []
    ev0.record(stream)
    last = None
    for _ in range(args.steps):
        M, sinfo, pinfo = one_solve(prm)
        setup_ms.append(sinfo["setup_ms"])
        kernel_ms.append(sinfo["kernel_ms"])
        pcg_kernel_ms.append(pinfo.get("kernel_ms", [0.0] * 5))
        solve_ms.append(pinfo["solve_ms"])
        iters.append(pinfo["iters"])
        if last is not None:
            last[0].close()
        last = (M, sinfo, pinfo)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = afsai.kernel_launches() - launches0
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, world, dev)
    M, sinfo, pinfo = last
    value = job_value(ms_total, args.steps, world)

    # the set-up's pattern-search kernels, timed together with CUDA events
    # around their launches (the gather and solve kernels of every step)
    kern_ms = float(np.mean(kernel_ms))
    rp, ci, va = M.export()
    psi, steps = M.rows()
    flops = setup_flops(rp, steps, p["s"], A.nnz / A.n)
    skey = f"setup/{args.workload}/{args.form}"
    setup_roof = setup_roofline(skey, flops, kern_ms, rp, steps, p, A, args.form)
    # each PCG kernel, timed with CUDA event nodes around the first iteration
    # of the solve's graph (on the solve's stream), averaged over the timed
    # solves, against its own roof (algorithmic bytes and FP64 fmas)
    kms = np.mean(np.array(pcg_kernel_ms, dtype=np.float64), axis=0)
    kernels = pcg_kernel_table(A, sinfo["nnz_G"], args.form, kms)
    # the dominant kernel of the solve: the largest device time per solve
    # among the PCG kernels (x iterations) and the set-up kernels together
    n_it = int(np.median(iters))
    top = max(kernels, key=lambda k: k["ms"])
    if kern_ms >= top["ms"] * n_it:
        roof = dict(setup_roof)
        roof["share_of_solve"] = kern_ms / (value * 1e3)
    else:
        traffic, traffic_note = measured_traffic(f"{top['key']}/{args.workload}/{args.form}", 1)
        roof = {"kernel": top["kernel"], "bound": top["bound"], "achieved": top["achieved"], "peak": top["peak"],
                "unit": top["unit"], "frac": top["frac"], "traffic": traffic, "traffic_note": traffic_note,
                "kernel_ms": top["ms"], "algorithmic_bytes": top["bytes"], "algorithmic_dfma": top["dfma"],
                "launches_per_solve": n_it, "share_of_solve": top["ms"] * n_it / (value * 1e3),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if top["bound"] == "hbm"
                else "FP64 ALU: 152 SMs x 2 DFMA/clk x 2.07 GHz (derived from unit counts)"}

    # preconditioner application z = G^T (G r) through the C ABI: algorithmic
    # bytes (G and G^T entries and row pointers, r gathered, t written and
    # gathered, z written) against the measured HBM copy bandwidth
    w_g = {0: 8, 1: 4, 2: 2}[FORMS[args.form]["g_prec"]]
    apply_bytes = 2 * (4 + w_g) * sinfo["nnz_G"] + 8 * (A.n + 1) + 32 * A.n
    rv = torch.rand(A.n, dtype=torch.float64, device=dev)
    zv = torch.empty_like(rv)
    for _ in range(3):
        afsai.afsai_apply(M, rv, zv, stream)
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(20):
        afsai.afsai_apply(M, rv, zv, stream)
    a1.record(stream)
    torch.cuda.synchronize()
    apply_us = a0.elapsed_time(a1) * 1e3 / 20
    apply_rec = {"us": apply_us, "bytes": apply_bytes, "gbs": apply_bytes / (apply_us * 1e-6) / 1e9,
                 "peak_gbs": MEASURED_HBM_GBS,
                 "frac": apply_bytes / (apply_us * 1e-6) / 1e9 / MEASURED_HBM_GBS}
    G64 = (rp.copy(), ci.copy(), va.copy())
    M.close()

    extra = {}
    if not args.no_mixed:
        names = args.extra_forms.split(",") if args.extra_forms else (
            ["g32", "bf16", "mixed", "jacobi"] if args.workload == "hetero256" else ["mixed", "jacobi"])
        for form in [f for f in names if f and f != args.form and f != "none"]:
            pf = prm_of(form)
            for _ in range(2):
                Mm, sm_, pm_ = one_solve(pf)
                Mm.close()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                Mm, sm_, pm_ = one_solve(pf)
                Mm.close()
            e1.record(stream)
            torch.cuda.synchronize()
            extra[form] = {"value": e0.elapsed_time(e1) / 1e3 / args.steps, "unit": "s/solve", "iters": pm_["iters"],
                           "relres_true": pm_["relres_true"], "desc": FORMS[form]["desc"],
                           "setup_ms": sm_["setup_ms"], "solve_ms": pm_["solve_ms"],
                           "iters_vs_fp64": pm_["iters"] / max(1, int(np.median(iters)))}
            if args.form == "fp64" and FORMS[form].get("kiter", 1) != 0:
                # error of this form's G against the FP64 G of the same input
                Mm, _, _ = one_solve(pf)
                extra[form]["g_vs_fp64"] = g_difference(G64, Mm.export(), A.n)
                Mm.close()

    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        Ah = type(A)(A.n, pin(A.rowptr).numpy(), pin(A.col).numpy(), pin(A.val).numpy())
        bh = pin(b).numpy()
        xh = torch.zeros(A.n, dtype=torch.float64).pin_memory().numpy()
        afsai.afsai_solve_host(Ah, prm, bh, xh, rtol=1e-8, maxit=20000, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            afsai.afsai_solve_host(Ah, prm, bh, xh, rtol=1e-8, maxit=20000, stream=stream)
        torch.cuda.synchronize()
        te = (time.perf_counter() - t0) / args.steps
        e2e = {"value": te, "unit": "s/solve", "h2d_bytes_per_step": int(4 * (A.n + 1) + 12 * A.nnz + 8 * A.n),
               "d2h_bytes_per_step": int(8 * A.n)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(A, b, p, int(np.median(iters)))

    if rank == 0:
        n_it = int(np.median(iters))
        line = {
            "metric": METRIC, "value": value, "unit": "s/solve", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.form == "fp64" else "f64+f32",
            "data": "synthetic (seeded generator)",
            "config": {"workload": WORKLOAD_NAMES[args.workload] + "_" + args.form, "n": A.n, "nnz": A.nnz,
                       "kiter": p["kiter"], "s": p["s"], "eps": p["eps"], "rtol": 1e-8,
                       "form": FORMS[args.form]["desc"],
                       "l2": "inputs larger than L2 (A is %.0f MB)" % (A.nnz * 12e-6),
                       "parallelism": f"replicas x{world}"},
            "setup_ms": float(np.median(setup_ms)), "solve_ms": float(np.median(solve_ms)), "pcg_iters": n_it,
            "relres_true": pinfo["relres_true"], "nnz_G": sinfo["nnz_G"],
            "setup_rows_per_s": A.n / (float(np.median(setup_ms)) * 1e-3),
            "solve_gbs": pcg_iteration_bytes(A, sinfo, args.form) * n_it / (float(np.median(solve_ms)) * 1e-3) / 1e9,
            "gpu_launches": int(launches), "roofline": roof, "setup_roofline": setup_roof,
            "pcg_kernels": [{k: v for k, v in r.items() if k != "key"} for r in kernels],
            "forms": extra, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk,
            "apply": apply_rec,
            # SpMV engines the timed run used (AFSAI_SPMV_MODES="a,g,gt" pins them for a profile)
            "spmv_engines": {"A": afsai.spmv_engine(0, A.n, A.nnz, 0),
                             "G": afsai.spmv_engine(1, A.n, sinfo["nnz_G"], FORMS[args.form]["g_prec"]),
                             "Gt": afsai.spmv_engine(2, A.n, sinfo["nnz_G"], FORMS[args.form]["g_prec"])},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
