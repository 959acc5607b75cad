"""Seeded synthetic SPD matrices and right-hand sides for aFSAI-PCG.

This module is shared by the CPU oracle tests and the CUDA path as a source
of INPUTS only: it builds sparse symmetric positive definite matrices in CSR
(int32 row pointers and columns, float64 values, columns sorted ascending,
full symmetric storage with the diagonal present) and seeded right-hand sides.
It contains none of the method's arithmetic (no pattern search, no
factorisation, no Krylov iteration).

The paper's matrices (Section 5, Table "tab-matrices") are not public; the
generators below stand in for them with the same structure:

* ``poisson7``       - 7-point Laplacian on a box, Dirichlet (homogeneous
  diffusion, the stand-in for the paper's Poisson matrix).
* ``elasticity_hex`` - trilinear hexahedral linear elasticity with a lognormal
  Young's modulus per element and one clamped face (stand-in for the
  geomechanics / mechanics matrices).
* ``diffusion7_hetero`` - cell-centred 7-point diffusion with a smoothed
  lognormal coefficient and harmonic face averages (stand-in for the
  heterogeneous-media diffusion matrices).
* ``poisson5_2d`` / ``poisson7_aniso`` / ``elasticity-free 27-point`` - the
  batched mix of uneven systems.

Grid ordering is natural lexicographic with x fastest (the pattern search is
ordering dependent through the j < i restriction).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

BASE_SEED = 20101417


@dataclasses.dataclass
class CSR:
    """Host CSR matrix: int32 rowptr/col, float64 val, sorted columns."""

    n: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n))


def from_scipy(M) -> CSR:
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    if M.nnz >= 2**31:
        raise ValueError("nnz does not fit int32 row pointers")
    return CSR(
        n=M.shape[0],
        rowptr=np.ascontiguousarray(M.indptr, dtype=np.int32),
        col=np.ascontiguousarray(M.indices, dtype=np.int32),
        val=np.ascontiguousarray(M.data, dtype=np.float64),
    )


def rhs(A: CSR, seed: int, nrhs: int = 1):
    """x* ~ U[-1, 1] from a PCG64 stream, and b = A x* (scipy matvec)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = (A.n,) if nrhs == 1 else (A.n, nrhs)
    xs = rng.uniform(-1.0, 1.0, size=shape)
    b = A.to_scipy() @ xs
    return np.ascontiguousarray(b), np.ascontiguousarray(xs)


# --------------------------------------------------------------------------
# Structured stencils
# --------------------------------------------------------------------------

def _stencil_csr(n, offsets_and_vals, diag):
    """Assemble a CSR matrix from per-row (column, value) lists given as
    arrays of shape (n,) with -1 for absent neighbours; columns must be
    supplied in ascending order per row."""
    cols = np.stack([c for c, _ in offsets_and_vals], axis=1)
    vals = np.stack([v for _, v in offsets_and_vals], axis=1)
    present = cols >= 0
    counts = present.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2**31:
        raise ValueError("nnz does not fit int32 row pointers")
    col = cols[present].astype(np.int32)
    val = vals[present].astype(np.float64)
    del diag
    return CSR(n=n, rowptr=rowptr.astype(np.int32), col=col, val=val)


def poisson7(nx: int, ny: int | None = None, nz: int | None = None, scale=(1.0, 1.0, 1.0)) -> CSR:
    """7-point Laplacian on nx*ny*nz interior nodes, Dirichlet boundary.

    With scale=(1,1,1): diagonal 6, off-diagonals -1.  ``scale`` gives
    per-axis coefficients (anisotropy): the diagonal is 2*sum(scale)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    n = nx * ny * nz
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    sx, sy, sz = (float(s) for s in scale)
    entries = []
    for (ok, off, c) in (
        (z > 0, -nx * ny, sz),
        (y > 0, -nx, sy),
        (x > 0, -1, sx),
    ):
        entries.append((np.where(ok, idx + off, -1), np.full(n, -c)))
    entries.append((idx, np.full(n, 2.0 * (sx + sy + sz))))
    for (ok, off, c) in (
        (x < nx - 1, 1, sx),
        (y < ny - 1, nx, sy),
        (z < nz - 1, nx * ny, sz),
    ):
        entries.append((np.where(ok, idx + off, -1), np.full(n, -c)))
    return _stencil_csr(n, entries, None)


def poisson5_2d(nx: int, ny: int | None = None, scale=(1.0, 1.0)) -> CSR:
    """5-point Laplacian on nx*ny interior nodes, Dirichlet."""
    ny = nx if ny is None else ny
    n = nx * ny
    idx = np.arange(n, dtype=np.int64)
    x = idx % nx
    y = idx // nx
    sx, sy = (float(s) for s in scale)
    entries = [
        (np.where(y > 0, idx - nx, -1), np.full(n, -sy)),
        (np.where(x > 0, idx - 1, -1), np.full(n, -sx)),
        (idx, np.full(n, 2.0 * (sx + sy))),
        (np.where(x < nx - 1, idx + 1, -1), np.full(n, -sx)),
        (np.where(y < ny - 1, idx + nx, -1), np.full(n, -sy)),
    ]
    return _stencil_csr(n, entries, None)


def laplace1d(n: int) -> CSR:
    """tridiag(-1, 2, -1) of order n (Dirichlet 1D Laplacian)."""
    idx = np.arange(n, dtype=np.int64)
    entries = [
        (np.where(idx > 0, idx - 1, -1), np.full(n, -1.0)),
        (idx, np.full(n, 2.0)),
        (np.where(idx < n - 1, idx + 1, -1), np.full(n, -1.0)),
    ]
    return _stencil_csr(n, entries, None)


# --------------------------------------------------------------------------
# Heterogeneous diffusion (cell-centred finite volumes)
# --------------------------------------------------------------------------

def _box_filter_axis(z: np.ndarray, axis: int, width: int) -> np.ndarray:
    """Moving average over ``width`` cells along ``axis`` with clamped
    (edge-replicated) ends; window [x - width//2 + 1, x + width//2]."""
    lo = width // 2 - 1
    hi = width // 2
    pad = [(0, 0)] * z.ndim
    pad[axis] = (lo + 1, hi)
    zp = np.pad(z, pad, mode="edge")
    c = np.cumsum(zp, axis=axis, dtype=np.float64)
    nlen = z.shape[axis]
    upper = np.take(c, np.arange(width, width + nlen), axis=axis)
    lower = np.take(c, np.arange(0, nlen), axis=axis)
    return (upper - lower) / width


def lognormal_field(shape, seed: int, sigma: float, smooth: int) -> np.ndarray:
    """k = exp(sigma * zs) where zs is N(0,1) noise box-filtered over
    ``smooth`` cells per axis and re-standardised to mean 0, std 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(size=shape)
    if smooth > 1:
        for ax in range(len(shape)):
            z = _box_filter_axis(z, ax, smooth)
    z = (z - z.mean()) / z.std()
    return np.exp(sigma * z)


def diffusion7_hetero(N: int, seed: int, sigma: float = 2.0, smooth: int = 8) -> CSR:
    """Cell-centred 7-point diffusion on N^3 unit cells.

    Coefficient: lognormal (``lognormal_field``).  Interior faces carry the
    harmonic mean 2 k1 k2 / (k1 + k2); Dirichlet boundary faces carry 2 k
    (half-cell distance).  A_ii = sum of the face transmissibilities of cell
    i, A_ij = -T_ij."""
    k = lognormal_field((N, N, N), seed, sigma, smooth)  # indexed [z, y, x]
    n = N ** 3
    kf = k.reshape(-1)

    def harm(a, b):
        return 2.0 * a * b / (a + b)

    # transmissibility to the +x, +y, +z neighbour (0 where absent)
    tx = np.zeros((N, N, N))
    tx[:, :, :-1] = harm(k[:, :, :-1], k[:, :, 1:])
    ty = np.zeros((N, N, N))
    ty[:, :-1, :] = harm(k[:, :-1, :], k[:, 1:, :])
    tz = np.zeros((N, N, N))
    tz[:-1, :, :] = harm(k[:-1, :, :], k[1:, :, :])
    diag = np.zeros((N, N, N))
    diag += tx
    diag[:, :, 1:] += tx[:, :, :-1]
    diag += ty
    diag[:, 1:, :] += ty[:, :-1, :]
    diag += tz
    diag[1:, :, :] += tz[:-1, :, :]
    # Dirichlet faces of the box: 2k each
    diag[:, :, 0] += 2.0 * k[:, :, 0]
    diag[:, :, -1] += 2.0 * k[:, :, -1]
    diag[:, 0, :] += 2.0 * k[:, 0, :]
    diag[:, -1, :] += 2.0 * k[:, -1, :]
    diag[0, :, :] += 2.0 * k[0, :, :]
    diag[-1, :, :] += 2.0 * k[-1, :, :]
    del k, kf

    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = (idx // N) % N
    z = idx // (N * N)
    txf, tyf, tzf = tx.reshape(-1), ty.reshape(-1), tz.reshape(-1)
    NN = N * N
    entries = [
        (np.where(z > 0, idx - NN, -1), -np.roll(tzf, NN)),
        (np.where(y > 0, idx - N, -1), -np.roll(tyf, N)),
        (np.where(x > 0, idx - 1, -1), -np.roll(txf, 1)),
        (idx, diag.reshape(-1)),
        (np.where(x < N - 1, idx + 1, -1), -txf),
        (np.where(y < N - 1, idx + N, -1), -tyf),
        (np.where(z < N - 1, idx + NN, -1), -tzf),
    ]
    return _stencil_csr(n, entries, None)


# --------------------------------------------------------------------------
# Linear elasticity, trilinear hexahedra
# --------------------------------------------------------------------------

def _hex8_reference_stiffness(nu: float) -> np.ndarray:
    """24x24 stiffness of a unit cube Q1 element for E = 1, 2x2x2 Gauss.

    Local node a = ax + 2*ay + 4*az with (ax, ay, az) in {0,1}^3; local dof
    3*a + component."""
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=np.float64)
    gp = np.array([0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0)])
    K = np.zeros((24, 24))
    for px in gp:
        for py in gp:
            for pz in gp:
                # shape function N_a = prod over axes of (c ? t : 1 - t)
                dN = np.zeros((8, 3))
                for a in range(8):
                    cx, cy, cz = corners[a]
                    fx = px if cx else 1 - px
                    fy = py if cy else 1 - py
                    fz = pz if cz else 1 - pz
                    gx = 1.0 if cx else -1.0
                    gy = 1.0 if cy else -1.0
                    gz = 1.0 if cz else -1.0
                    dN[a] = (gx * fy * fz, fx * gy * fz, fx * fy * gz)
                B = np.zeros((6, 24))
                for a in range(8):
                    dx, dy, dz = dN[a]
                    c = 3 * a
                    B[0, c] = dx
                    B[1, c + 1] = dy
                    B[2, c + 2] = dz
                    B[3, c] = dy
                    B[3, c + 1] = dx
                    B[4, c + 1] = dz
                    B[4, c + 2] = dy
                    B[5, c] = dz
                    B[5, c + 2] = dx
                K += B.T @ D @ B * (1.0 / 8.0)  # Gauss weights 1/2 per axis on [0,1]
    return 0.5 * (K + K.T)


def elasticity_hex(ne: int, seed: int, sigma: float = 1.0, nu: float = 0.3) -> CSR:
    """Q1 hex linear elasticity on ne^3 unit elements, (ne+1)^3 nodes, 3 dofs
    per node (node-major, x fastest).  Young's modulus per element is
    exp(sigma * N(0,1)).  The z = 0 face is clamped by symmetric elimination:
    its dofs' rows and columns are zeroed and the diagonal set to 1, so
    n = 3 (ne+1)^3."""
    nn = ne + 1
    n = 3 * nn ** 3
    rng = np.random.Generator(np.random.PCG64(seed))
    E = np.exp(sigma * rng.standard_normal(size=ne ** 3))
    Kref = _hex8_reference_stiffness(nu)
    e = np.arange(ne ** 3, dtype=np.int64)
    ex = e % ne
    ey = (e // ne) % ne
    ez = e // (ne * ne)
    base = ex + nn * ey + nn * nn * ez
    loc = np.array([(a & 1) + nn * ((a >> 1) & 1) + nn * nn * ((a >> 2) & 1) for a in range(8)], dtype=np.int64)
    nodes = base[:, None] + loc[None, :]  # (nel, 8)
    dofs = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 24)  # (nel, 24)
    rows = np.repeat(dofs, 24, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 24)).reshape(-1)
    vals = (E[:, None] * Kref.reshape(1, -1)).reshape(-1)
    # clamp the z = 0 face by symmetric elimination
    clamped = np.zeros(n, dtype=bool)
    clamped[: 3 * nn * nn] = True
    keep = ~(clamped[rows] | clamped[cols])
    cd = np.nonzero(clamped)[0]
    rows = np.concatenate([rows[keep], cd]).astype(np.int32)
    cols = np.concatenate([cols[keep], cd]).astype(np.int32)
    vals = np.concatenate([vals[keep], np.ones(cd.size)])
    del keep
    K = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
    del rows, cols, vals
    K.sum_duplicates()
    # exact symmetry: element matrices are symmetric, but duplicate sums may
    # round differently for (r, c) and (c, r)
    K = 0.5 * (K + K.T)
    return from_scipy(K)


def stencil27_fe(nx: int, ny: int | None = None, nz: int | None = None, scale=(1.0, 1.0, 1.0)) -> CSR:
    """Scalar Q1 (trilinear) finite-element Laplacian on (nx+1)^3 elements:
    a 27-point stencil on nx*ny*nz interior nodes with Dirichlet boundary.
    ``scale`` is a per-axis conductivity (anisotropy)."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    # 1D linear-element mass (m) and stiffness (k) matrices on unit spacing
    m1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    sx, sy, sz = (float(s) for s in scale)
    Ke = (sx * np.kron(np.kron(m1, m1), k1) + sy * np.kron(np.kron(m1, k1), m1) + sz * np.kron(np.kron(k1, m1), m1))
    # element nodes ordered a = ax + 2 ay + 4 az  (kron order: z outer, x inner)
    ex_n, ey_n, ez_n = nx + 1, ny + 1, nz + 1  # elements per axis
    Nx, Ny, Nz = nx + 2, ny + 2, nz + 2  # nodes incl. boundary
    e = np.arange(ex_n * ey_n * ez_n, dtype=np.int64)
    ex = e % ex_n
    ey = (e // ex_n) % ey_n
    ez = e // (ex_n * ey_n)
    base = ex + Nx * ey + Nx * Ny * ez
    loc = np.array([(a & 1) + Nx * ((a >> 1) & 1) + Nx * Ny * ((a >> 2) & 1) for a in range(8)], dtype=np.int64)
    nodes = base[:, None] + loc[None, :]
    rows = np.repeat(nodes, 8, axis=1).reshape(-1)
    cols = np.tile(nodes, (1, 8)).reshape(-1)
    vals = np.tile(Ke.reshape(-1), e.size)
    Nall = Nx * Ny * Nz
    K = sp.coo_matrix((vals, (rows, cols)), shape=(Nall, Nall)).tocsr()
    gx = np.arange(Nall) % Nx
    gy = (np.arange(Nall) // Nx) % Ny
    gz = np.arange(Nall) // (Nx * Ny)
    interior = (gx > 0) & (gx < Nx - 1) & (gy > 0) & (gy < Ny - 1) & (gz > 0) & (gz < Nz - 1)
    ii = np.nonzero(interior)[0]
    K = K[ii][:, ii]
    K = 0.5 * (K + K.T)
    return from_scipy(K)


# --------------------------------------------------------------------------
# Small random SPD matrices for brute-force tests
# --------------------------------------------------------------------------

def random_spd(n: int, density: float, seed: int, dense: bool = False) -> CSR:
    """Symmetric, strictly diagonally dominant (hence SPD) sparse matrix with
    off-diagonal values U[-1,1] on a random symmetric pattern of the given
    density; the diagonal is 1 + sum |off-diagonals| + U[0,1].  With
    ``dense=True``: A = Q^T Q + n I for Q with N(0,1) entries (generic, no
    zero entries)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if dense:
        Q = rng.standard_normal(size=(n, n))
        A = Q.T @ Q + n * np.eye(n)
        A = 0.5 * (A + A.T)
        return from_scipy(sp.csr_matrix(A))
    mask = rng.random(size=(n, n)) < density
    mask = np.triu(mask, 1)
    vals = rng.uniform(-1.0, 1.0, size=(n, n)) * mask
    off = vals + vals.T
    d = 1.0 + np.abs(off).sum(axis=1) + rng.random(n)
    A = off + np.diag(d)
    return from_scipy(sp.csr_matrix(A))


# --------------------------------------------------------------------------
# Named workloads
# --------------------------------------------------------------------------

WORKLOADS = {
    # name: (description, kiter, s, eps)
    "poisson20": ("3D 7-point Poisson 20^3 Dirichlet, n=8000", 5, 2, 1e-3),
    "elast48": ("3D Q1 hex elasticity 48^3 elements, lognormal E (sigma=1), nu=0.3, z=0 face clamped, n=352947", 10, 3, 1e-3),
    "hetero256": ("heterogeneous 7-point diffusion 256^3, lognormal k (sigma=2, 8-cell smoothing), harmonic faces, n=16777216", 5, 2, 1e-3),
}


def workload(name: str, scale: int | None = None):
    """Return (A, b, xstar, params dict) of a named workload.  ``scale``
    overrides the grid size for reduced-size variants of the same recipe."""
    if name == "poisson20":
        N = 20 if scale is None else scale
        A = poisson7(N)
        seed = BASE_SEED + 0
    elif name == "elast48":
        ne = 48 if scale is None else scale
        A = elasticity_hex(ne, BASE_SEED + 1)
        seed = BASE_SEED + 1
    elif name == "hetero256":
        N = 256 if scale is None else scale
        A = diffusion7_hetero(N, BASE_SEED + 2)
        seed = BASE_SEED + 2
    else:
        raise KeyError(name)
    _, kiter, s, eps = WORKLOADS[name]
    b, xs = rhs(A, seed + 1000)
    return A, b, xs, dict(kiter=kiter, s=s, eps=eps)


# --------------------------------------------------------------------------
# Batch of uneven systems (the batched and served forms)
# --------------------------------------------------------------------------

def batch_system(k: int, seed: int, nmin: float = 2e3, nmax: float = 2e5):
    """System k of the uneven batch: n ~ log-uniform[nmin, nmax], type
    uniform over {2D 5-point, 3D 7-point, 3D 27-point (Q1 FE)}, anisotropy
    rho ~ log-uniform[1, 1e3] on the last axis, Dirichlet boundary; the
    grid side is round(n^(1/d)).  Returns (A, type name)."""
    rng = np.random.Generator(np.random.PCG64([seed, k]))
    n_target = math.exp(rng.uniform(math.log(nmin), math.log(nmax)))
    kind = int(rng.integers(0, 3))
    rho = math.exp(rng.uniform(0.0, math.log(1e3)))
    if kind == 0:
        side = max(2, int(round(n_target ** 0.5)))
        return poisson5_2d(side, side, scale=(1.0, rho)), "5pt2d"
    side = max(2, int(round(n_target ** (1.0 / 3.0))))
    if kind == 1:
        return poisson7(side, side, side, scale=(1.0, 1.0, rho)), "7pt3d"
    return stencil27_fe(side, side, side, scale=(1.0, 1.0, rho)), "27pt3d"


def batch_workload(nsys: int, seed: int = BASE_SEED + 3, nmin: float = 2e3, nmax: float = 2e5):
    """nsys systems of the uneven batch with seeded right-hand sides."""
    out = []
    for k in range(nsys):
        A, kind = batch_system(k, seed, nmin, nmax)
        b, _ = rhs(A, seed * 1000 + k)
        out.append((A, b, kind))
    return out
