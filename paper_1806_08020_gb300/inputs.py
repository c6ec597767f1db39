"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module builds matrices and start vectors only; it holds none of the
method's arithmetic (no GMRES, no roots, no Arnoldi).  Everything is plain
numpy so that both sides of every parity test draw identical inputs.

Matrices are returned as :class:`CSR` (int64 row pointers, int32 column
indices sorted within each row, float64 values).

Problem families (the paper's Section 4-8 examples and the scaled configs):

* 2-D / 3-D constant-coefficient convection-diffusion, ``-lap(u) + beta*u_x``
  on the unit square / cube, homogeneous Dirichlet boundary, central
  differences on an ``N`` (``N^2``, ``N^3``) interior grid, ``h = 1/(N+1)``,
  lexicographic ordering with x fastest (Example 1's operator family).
* Example 1's two-region operator (bottom half ``-lap u + 20 u_x``, top half
  ``-100 lap u + 2000 u_x``).
* Diagonal test matrices of Examples 4, 6 and 7 and the Figure 1 spectrum.
* Random nonsymmetric banded matrices for the request-stream workload.
* Rotation blocks with a fanned-out complex spectrum (Example 2's stand-in).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 20181806


@dataclass
class CSR:
    """Compressed sparse row matrix: row i holds colind/vals[rowptr[i]:rowptr[i+1]]."""

    n: int
    rowptr: np.ndarray  # int64, n+1
    colind: np.ndarray  # int32, nnz
    vals: np.ndarray  # float64, nnz

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        np.add.at(d, (rows, self.colind), self.vals)
        return d


def _from_stencil(n: int, offsets: list[int], coef: np.ndarray, valid: np.ndarray) -> CSR:
    """Assemble CSR from per-row stencil columns.

    ``offsets`` are column offsets sorted ascending; ``coef[i, s]`` and
    ``valid[i, s]`` give the value and presence of entry (i, i+offsets[s]).
    """
    cols = np.arange(n, dtype=np.int64)[:, None] + np.asarray(offsets, dtype=np.int64)[None, :]
    counts = valid.sum(axis=1)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    colind = cols[valid].astype(np.int32)
    vals = np.ascontiguousarray(coef[valid], dtype=np.float64)
    return CSR(n, rowptr, colind, vals)


def convection_diffusion_2d(N: int, beta: float, scale_top: float | None = None,
                            beta_top: float | None = None) -> CSR:
    """5-point central-difference ``-u_xx - u_yy + beta*u_x`` on an N x N grid.

    Unknown (i, j) (x index i, y index j, both 0-based) has row i + N*j.
    With ``scale_top``/``beta_top`` the rows with y >= 1/2 use the operator
    ``-scale_top*lap(u) + beta_top*u_x`` instead (Example 1's two regions).
    """
    n = N * N
    h = 1.0 / (N + 1)
    idx = np.arange(n)
    ix = idx % N
    iy = idx // N
    diff = np.ones(n)
    conv = np.full(n, float(beta))
    if scale_top is not None:
        top = (iy + 1) * h >= 0.5
        diff[top] = scale_top
        conv[top] = beta_top
    offs = [-N, -1, 0, 1, N]
    coef = np.empty((n, 5))
    coef[:, 0] = -diff / h**2
    coef[:, 1] = -diff / h**2 - conv / (2 * h)
    coef[:, 2] = 4 * diff / h**2
    coef[:, 3] = -diff / h**2 + conv / (2 * h)
    coef[:, 4] = -diff / h**2
    valid = np.ones((n, 5), dtype=bool)
    valid[:, 0] = iy > 0
    valid[:, 1] = ix > 0
    valid[:, 3] = ix < N - 1
    valid[:, 4] = iy < N - 1
    return _from_stencil(n, offs, coef, valid)


def example1_matrix(N: int) -> CSR:
    """Example 1 (Section 4): bottom half -lap u + 20 u_x, top half -100 lap u + 2000 u_x."""
    return convection_diffusion_2d(N, 20.0, scale_top=100.0, beta_top=2000.0)


def convection_diffusion_3d(N: int, beta: float) -> CSR:
    """7-point central-difference ``-lap(u) + beta*u_x`` on an N^3 grid (row i + N*j + N^2*k)."""
    n = N * N * N
    h = 1.0 / (N + 1)
    idx = np.arange(n, dtype=np.int64)
    ix = idx % N
    iy = (idx // N) % N
    iz = idx // (N * N)
    offs = [-N * N, -N, -1, 0, 1, N, N * N]
    c = 1.0 / h**2
    cb = beta / (2 * h)
    row = np.array([-c, -c, -c - cb, 6 * c, -c + cb, -c, -c])
    coef = np.broadcast_to(row, (n, 7))
    valid = np.ones((n, 7), dtype=bool)
    valid[:, 0] = iz > 0
    valid[:, 1] = iy > 0
    valid[:, 2] = ix > 0
    valid[:, 4] = ix < N - 1
    valid[:, 5] = iy < N - 1
    valid[:, 6] = iz < N - 1
    return _from_stencil(n, offs, coef, valid)


def diagonal(d: np.ndarray) -> CSR:
    d = np.asarray(d, dtype=np.float64)
    n = d.size
    return CSR(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), d.copy())


def example4_diag() -> np.ndarray:
    """Example 4 (Section 5): diag(1, 2, ..., 1000)."""
    return np.arange(1, 1001, dtype=np.float64)


def example6_diag() -> np.ndarray:
    """Example 6 (Section 6.2): diag(1, 2, ..., 10000)."""
    return np.arange(1, 10001, dtype=np.float64)


def example7_diag() -> np.ndarray:
    """Example 7 (Section 7): 0.1, 0.2, ..., 9.9, 10, 11, ..., 9909, 20000 (n = 10000)."""
    small = np.arange(1, 100) / 10.0
    mid = np.arange(10, 9910, dtype=np.float64)
    return np.concatenate([small, mid, [20000.0]])


def figure1_diag() -> np.ndarray:
    """Figure 1 / Table 1 (Sections 2, 3): 20 log-spaced in [1e-3, 0.9], 80 uniform in [1, 2]."""
    return np.concatenate([np.logspace(-3, np.log10(0.9), 20), np.linspace(1.0, 2.0, 80)])


def banded_random(n: int, w: int, seed: int) -> CSR:
    """Random nonsymmetric banded matrix (request-stream workload).

    Full band of half-width ``w`` (2w off-diagonals per interior row), off-diagonal
    entries N(0,1)/sqrt(w), diagonal U[0, 10] plus 1e-3 * (row index).
    """
    rng = np.random.default_rng([seed, 7])
    offs = list(range(-w, w + 1))
    coef = rng.standard_normal((n, 2 * w + 1)) / np.sqrt(w)
    coef[:, w] = rng.uniform(0.0, 10.0, n) + 1e-3 * np.arange(n)
    cols = np.arange(n)[:, None] + np.arange(-w, w + 1)[None, :]
    valid = (cols >= 0) & (cols < n)
    return _from_stencil(n, offs, coef, valid)


def rotation_blocks(nb: int, bmax: float, seed: int) -> CSR:
    """Stand-in for Example 2's complex spectrum (Af23560 is not available):
    n = 2 nb, 2 x 2 blocks [[a_i, b_i], [-b_i, a_i]] (eigenvalues a_i +- i b_i)
    with a_i uniform in [0.05, 10] (sorted) and b_i uniform in [0, bmax] times
    sqrt(a_i / 10), so the spectrum fans out into large imaginary parts away
    from the origin, plus a weak coupling: each row i also gets 0.01 * N(0,1)
    at column (i + 7 + (i * 7919) % (n - 7)) % n (never in its own block)."""
    rng = np.random.default_rng([seed, 2])
    n = 2 * nb
    a = np.sort(rng.uniform(0.05, 10.0, nb))
    b = rng.uniform(0.0, bmax, nb) * np.sqrt(a / 10.0)
    cw = 0.01 * rng.standard_normal(n)
    rows, cols, vals = [], [], []
    for i in range(n):
        blk = i // 2
        j0 = 2 * blk
        far = (i + 7 + (i * 7919) % (n - 7)) % n
        ent = {j0: a[blk] if i == j0 else -b[blk], j0 + 1: b[blk] if i == j0 else a[blk]}
        if far // 2 != blk:
            ent[far] = ent.get(far, 0.0) + cw[i]
        for j in sorted(ent):
            rows.append(i)
            cols.append(j)
            vals.append(ent[j])
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, np.asarray(rows) + 1, 1)
    return CSR(n, np.cumsum(rowptr).astype(np.int64), np.asarray(cols, dtype=np.int32),
               np.asarray(vals, dtype=np.float64))


def start_vector(n: int, seed: int, stream: int) -> np.ndarray:
    """Seeded N(0,1) start vector; stream 0 builds the polynomial, stream 1 starts Arnoldi."""
    return np.random.default_rng([seed, stream]).standard_normal(n)


# ----------------------------------------------------------------------------
# Workload recipes (sizes and parameters of the five configurations)
# ----------------------------------------------------------------------------

def plain_small() -> dict:
    """n = 2500 2-D CD (beta = 20), d = 10, Arnoldi(30, 15), nev = 10, FP64."""
    A = convection_diffusion_2d(50, 20.0)
    return dict(name="cd2d_N50_beta20_d10_m30_k15_nev10", A=A, d=10, m=30, k=15, nev=10,
                rtol=1e-8, seed=BASE_SEED)


def plain_large() -> dict:
    """n = 1e6 2-D CD (beta = 100), d = 50, Arnoldi(50, 25), nev = 20, FP64."""
    A = convection_diffusion_2d(1000, 100.0)
    return dict(name="cd2d_N1000_beta100_d50_m50_k25_nev20", A=A, d=50, m=50, k=25, nev=20,
                rtol=1e-8, seed=BASE_SEED + 1)


def precision_3d(N: int = 160) -> dict:
    """n = N^3 3-D CD (beta = 50), double polynomial 10 x 20, m = 40, nev = 16 (k = nev + 5)."""
    A = convection_diffusion_3d(N, 50.0)
    return dict(name=f"cd3d_N{N}_beta50_d10x20_m40_k21_nev16", A=A, d1=10, d2=20, m=40, k=21,
                nev=16, rtol=1e-8, seed=BASE_SEED + 2)


def batch_instances(count: int = 64, seed: int = BASE_SEED + 3, side_lo: int = 64,
                    side_hi: int = 512) -> list[dict]:
    """Uneven batch: grid side U{64..512}, beta U[1, 200], d U{20..80}, m = 30, nev = 8, k = 13."""
    rng = np.random.default_rng([seed, 11])
    out = []
    for i in range(count):
        N = int(rng.integers(side_lo, side_hi + 1))
        beta = float(rng.uniform(1.0, 200.0))
        d = int(rng.integers(20, 81))
        out.append(dict(N=N, beta=beta, d=d, m=30, k=13, nev=8, rtol=1e-8,
                        seed=BASE_SEED + 1000 * (i + 1)))
    return out


def request_stream(count: int = 2000, rate: float = 50.0, seed: int = BASE_SEED + 4,
                   n_lo: float = 1e4, n_hi: float = 2e6) -> list[dict]:
    """Poisson request stream: arrival times, n log-uniform, half-band U{5..25},
    nev U{4..32}, d U{10..100}, k = nev + 5, m = max(30, 2k)."""
    rng = np.random.default_rng([seed, 13])
    t = np.cumsum(rng.exponential(1.0 / rate, count))
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        w = int(rng.integers(5, 26))
        nev = int(rng.integers(4, 33))
        d = int(rng.integers(10, 101))
        k = nev + 5
        out.append(dict(arrival=float(t[i]), n=n, w=w, nev=nev, d=d, k=k, m=max(30, 2 * k),
                        rtol=1e-8, seed=BASE_SEED + 1000 * (i + 1)))
    return out
