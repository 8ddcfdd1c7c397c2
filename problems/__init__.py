"""Seeded synthetic test problems shared by the CPU oracle and the GPU path.

This module only builds inputs: matrices (CSR arrays, stencil face
coefficients, dense model matrices), right-hand sides and initial guesses.
It holds none of the conjugate gradient arithmetic; both the oracle and the
CUDA library consume what it returns.

Problems (all symmetric positive definite):

* constant-coefficient Poisson, 5-point (2D) / 7-point (3D), Dirichlet-0
  boundary, no h^2 scaling: diagonal 2*dim + shift, off-diagonal -1;
* variable-coefficient diffusion: one coefficient c_f > 0 per cell face,
  boundary faces included, A = sum_f c_f (e_a - e_b)(e_a - e_b)^T over
  interior faces plus c_f e_a e_a^T over boundary faces; c_f = exp(sigma z_f),
  z_f ~ N(0, 1);
* the model problem of Section 4 (Eq. 4.1): eigenvalues
  lambda_i = lambda_1 + (i-1)/(n-1) (lambda_n - lambda_1) rho^(n-i),
  Haar-random orthogonal eigenvectors; and its diagonal form;
* random small integer SPD matrices B B^T + I for exact-arithmetic checks.

Grid ordering is lexicographic with x fastest: index = x + nx*(y + ny*z).
"""
from __future__ import annotations

import dataclasses
from fractions import Fraction
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20190503


def rng_for(tag: str, base: int = BASE_SEED) -> np.random.Generator:
    """A PCG64 generator whose seed is derived from ``base`` and a config tag."""
    sub = sum((i + 1) * ord(c) for i, c in enumerate(tag))
    return np.random.Generator(np.random.PCG64([base, sub]))


# ----------------------------------------------------------------------------
# structured grids
# ----------------------------------------------------------------------------

def _dims3(dims: Sequence[int]) -> Tuple[int, int, int]:
    if len(dims) == 2:
        return int(dims[0]), int(dims[1]), 1
    if len(dims) == 3:
        return int(dims[0]), int(dims[1]), int(dims[2])
    raise ValueError("dims must have length 2 or 3")


def face_shapes(dims: Sequence[int]) -> List[Tuple[int, ...]]:
    """Shapes (C order, slowest axis first) of the per-direction face arrays.

    2D (nx, ny): x-faces (ny, nx+1), y-faces (ny+1, nx).
    3D (nx, ny, nz): x-faces (nz, ny, nx+1), y-faces (nz, ny+1, nx),
    z-faces (nz+1, ny, nx).  Face index i along its own axis sits between
    cells i-1 and i; faces 0 and n are boundary faces.
    """
    if len(dims) == 2:
        nx, ny = dims
        return [(ny, nx + 1), (ny + 1, nx)]
    nx, ny, nz = dims
    return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]


def face_coefficients(dims: Sequence[int], sigma: float,
                      rng: np.random.Generator) -> List[np.ndarray]:
    """Log-normal face coefficients c_f = exp(sigma * z_f), z_f ~ N(0, 1)."""
    return [np.exp(sigma * rng.standard_normal(sh)) for sh in face_shapes(dims)]


def flat_faces(faces: Sequence[np.ndarray]) -> np.ndarray:
    """Concatenate per-direction face arrays into the layout the library takes."""
    return np.ascontiguousarray(np.concatenate([np.ravel(f) for f in faces]))


def _faces_or_const(dims, faces):
    if faces is not None:
        return [np.asarray(f, dtype=np.float64) for f in faces]
    return [np.ones(sh) for sh in face_shapes(dims)]


def stencil_csr(dims: Sequence[int], faces: Optional[Sequence[np.ndarray]] = None,
                shift: float = 0.0):
    """CSR arrays (row_ptr int32, col_idx int32, vals float64) of the grid operator.

    With ``faces=None`` this is the constant-coefficient Poisson matrix
    (diagonal 2*dim + shift, off-diagonals -1).  Columns are sorted within
    each row.  Built vectorised: every row has up to 2*dim+1 candidate
    entries in increasing column order, and absent neighbours are masked.
    """
    nx, ny, nz = _dims3(dims)
    dim = len(dims)
    n = nx * ny * nz
    fc = _faces_or_const(dims, faces)
    if dim == 2:
        fx = fc[0].reshape(1, ny, nx + 1)
        fy = fc[1].reshape(1, ny + 1, nx)
        fz = None
    else:
        fx, fy, fz = fc
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x = x.ravel(); y = y.ravel(); z = z.ravel()
    idx = np.arange(n, dtype=np.int64)
    # coefficient of the face on each side of every cell
    cxm = fx[z, y, x]; cxp = fx[z, y, x + 1]
    cym = fy[z, y, x]; cyp = fy[z, y + 1, x]
    diag = cxm + cxp + cym + cyp
    if dim == 3:
        czm = fz[z, y, x]; czp = fz[z + 1, y, x]
        diag = diag + czm + czp
    diag = diag + shift
    cand_cols = []
    cand_vals = []
    cand_mask = []
    if dim == 3:
        cand_cols.append(idx - nx * ny); cand_vals.append(-czm); cand_mask.append(z > 0)
    cand_cols.append(idx - nx); cand_vals.append(-cym); cand_mask.append(y > 0)
    cand_cols.append(idx - 1); cand_vals.append(-cxm); cand_mask.append(x > 0)
    cand_cols.append(idx); cand_vals.append(diag); cand_mask.append(np.ones(n, bool))
    cand_cols.append(idx + 1); cand_vals.append(-cxp); cand_mask.append(x < nx - 1)
    cand_cols.append(idx + nx); cand_vals.append(-cyp); cand_mask.append(y < ny - 1)
    if dim == 3:
        cand_cols.append(idx + nx * ny); cand_vals.append(-czp); cand_mask.append(z < nz - 1)
    C = np.stack(cand_cols, axis=1)
    V = np.stack(cand_vals, axis=1)
    M = np.stack(cand_mask, axis=1)
    counts = M.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("nnz exceeds int32 range")
    col_idx = C[M].astype(np.int32)
    vals = V[M].astype(np.float64)
    return row_ptr.astype(np.int32), col_idx, vals


def poisson_csr(dims: Sequence[int], shift: float = 0.0):
    """Constant-coefficient 5/7-point Poisson matrix in CSR."""
    return stencil_csr(dims, None, shift)


def stencil_apply(dims: Sequence[int], v: np.ndarray,
                  faces: Optional[Sequence[np.ndarray]] = None,
                  shift: float = 0.0) -> np.ndarray:
    """y = A v for the grid operator, used only to build right-hand sides."""
    nx, ny, nz = _dims3(dims)
    dim = len(dims)
    fc = _faces_or_const(dims, faces)
    if dim == 2:
        fx = fc[0].reshape(1, ny, nx + 1)
        fy = fc[1].reshape(1, ny + 1, nx)
    else:
        fx, fy, fz = fc
    u = np.asarray(v, dtype=np.float64).reshape(nz, ny, nx)
    up = np.zeros((nz + 2, ny + 2, nx + 2))
    up[1:-1, 1:-1, 1:-1] = u
    c = up[1:-1, 1:-1, 1:-1]
    out = fx[:, :, :-1] * (c - up[1:-1, 1:-1, :-2]) + fx[:, :, 1:] * (c - up[1:-1, 1:-1, 2:])
    out = out + fy[:, :-1, :] * (c - up[1:-1, :-2, 1:-1]) + fy[:, 1:, :] * (c - up[1:-1, 2:, 1:-1])
    if dim == 3:
        out = out + fz[:-1] * (c - up[:-2, 1:-1, 1:-1]) + fz[1:] * (c - up[2:, 1:-1, 1:-1])
    out = out + shift * c
    return out.reshape(-1)


def csr_apply(row_ptr, col_idx, vals, v):
    """y = A v for CSR arrays (scipy), used only to build right-hand sides."""
    import scipy.sparse as sp
    n = len(row_ptr) - 1
    A = sp.csr_matrix((vals, col_idx, row_ptr), shape=(n, n))
    return A @ np.asarray(v, dtype=np.float64)


# ----------------------------------------------------------------------------
# the model problem of Section 4 (Eq. 4.1) and its diagonal form
# ----------------------------------------------------------------------------

def model_eigenvalues(n: int, rho: float, kappa: Optional[float] = None,
                      lam1: Optional[float] = None, lamn: Optional[float] = None) -> np.ndarray:
    """lambda_1 = 1/kappa (or lam1), lambda_n = 1 (or lamn), Eq. 4.1 in between."""
    if lam1 is None:
        lam1 = 1.0 / kappa
    if lamn is None:
        lamn = 1.0
    i = np.arange(1, n + 1, dtype=np.float64)
    lam = lam1 + ((i - 1) / (n - 1)) * (lamn - lam1) * rho ** (n - i)
    lam[0] = lam1
    lam[-1] = lamn
    return lam


def haar_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian, R-diagonal signs fixed."""
    G = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    return Q * np.sign(np.diag(R))


@dataclasses.dataclass
class DenseProblem:
    A: np.ndarray
    b: np.ndarray
    x_star: np.ndarray
    lam: np.ndarray


def model_problem(n: int = 48, rho: float = 0.8, kappa: float = 1e3,
                  rng: Optional[np.random.Generator] = None) -> DenseProblem:
    """Dense A = Q diag(lambda) Q^T with b chosen so that x* has entries 1/sqrt(n)."""
    if rng is None:
        rng = rng_for(f"model_{n}_{rho}_{kappa}")
    lam = model_eigenvalues(n, rho, kappa)
    Q = haar_orthogonal(n, rng)
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    x_star = np.full(n, 1.0 / np.sqrt(n))
    b = A @ x_star
    return DenseProblem(A, b, x_star, lam)


def dense_lowrank_spd(n: int, rank: int, rng: np.random.Generator) -> DenseProblem:
    """Dense SPD A = diag(delta) + U U^T / n, delta ~ U[1, 2], U Gaussian n x rank
    (a dense matrix built in O(n^2 rank)); x* ~ U(-1, 1), b = A x*."""
    delta = rng.uniform(1.0, 2.0, n)
    U = rng.standard_normal((n, rank))
    A = (U @ U.T) / n
    A[np.diag_indices(n)] += delta
    x_star = rng.uniform(-1.0, 1.0, n)
    return DenseProblem(A, A @ x_star, x_star, np.empty(0))


def model_problem_on_device(n: int, rho: float, kappa: float, device: str = "cuda"):
    """The Eq. 4.1 model problem built on a GPU with torch (for sizes where a
    host QR takes minutes, e.g. Section 5's n = 10752): the Gaussian is drawn
    on the host from the seeded generator, Q from its QR (R-diagonal signs
    fixed), A = Q diag(lambda) Q^T symmetrised, x* = 1/sqrt(n), b = A x*.
    Returns (A, b, x_star) as FP64 tensors on `device`."""
    import torch
    rng = rng_for(f"model_{n}_{rho}_{kappa}")
    G = torch.from_numpy(rng.standard_normal((n, n))).to(device)
    Q, R = torch.linalg.qr(G)
    del G
    Q = Q * torch.sign(torch.diagonal(R))
    del R
    lam = torch.from_numpy(model_eigenvalues(n, rho, kappa)).to(device)
    A = (Q * lam) @ Q.T
    del Q
    A = 0.5 * (A + A.T)
    x_star = torch.full((n,), 1.0 / np.sqrt(n), dtype=torch.float64, device=device)
    return A.contiguous(), A @ x_star, x_star


def strakos_diagonal(n: int = 100_000, lam1: float = 1e-3, lamn: float = 1e3,
                     rho: float = 0.8) -> Tuple[np.ndarray, np.ndarray]:
    """Diagonal of the Eq. 4.1 spectrum and b = A (1/sqrt(n)) 1."""
    lam = model_eigenvalues(n, rho, lam1=lam1, lamn=lamn)
    b = lam * (1.0 / np.sqrt(n))
    return lam, b


# ----------------------------------------------------------------------------
# right-hand sides
# ----------------------------------------------------------------------------

def xtrue_uniform(n: int, rng: np.random.Generator) -> np.ndarray:
    return rng.uniform(-1.0, 1.0, size=n)


# ----------------------------------------------------------------------------
# exact-arithmetic inputs
# ----------------------------------------------------------------------------

def random_int_spd(n: int, rng: np.random.Generator, lo: int = -3, hi: int = 3) -> np.ndarray:
    """Integer SPD matrix B B^T + I (object array of Fractions)."""
    B = rng.integers(lo, hi + 1, size=(n, n))
    A = B @ B.T + np.eye(n, dtype=np.int64)
    return np.array([[Fraction(int(v)) for v in row] for row in A], dtype=object)


def int_spd_with_eigs(eigs: Sequence[int], rng: np.random.Generator) -> np.ndarray:
    """H diag(eigs) H with a rational Householder H = I - 2 v v^T / v^T v.

    The result is rational, symmetric, with exactly the given eigenvalues.
    """
    n = len(eigs)
    v = rng.integers(-3, 4, size=n)
    while not np.any(v):
        v = rng.integers(-3, 4, size=n)
    vv = sum(int(t) * int(t) for t in v)
    H = np.empty((n, n), dtype=object)
    for i in range(n):
        for j in range(n):
            H[i, j] = Fraction(int(i == j)) - Fraction(2 * int(v[i]) * int(v[j]), vv)
    D = np.empty((n, n), dtype=object)
    for i in range(n):
        for j in range(n):
            D[i, j] = Fraction(int(eigs[i])) if i == j else Fraction(0)
    return H.dot(D).dot(H)


def fraction_vector(vals) -> np.ndarray:
    return np.array([Fraction(int(v)) if not isinstance(v, Fraction) else v for v in vals],
                    dtype=object)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class GridProblem:
    """A grid operator with its CSR form (optional) and a right-hand side."""
    dims: Tuple[int, ...]
    faces: Optional[List[np.ndarray]]
    shift: float
    b: np.ndarray
    x_true: Optional[np.ndarray]
    csr: Optional[Tuple[np.ndarray, np.ndarray, np.ndarray]] = None

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    def face_array(self) -> Optional[np.ndarray]:
        return None if self.faces is None else flat_faces(self.faces)


def grid_problem(dims: Sequence[int], tag: str, sigma: Optional[float] = None,
                 shift: float = 0.0, with_csr: bool = True, rhs: str = "xtrue") -> GridProblem:
    """Poisson (sigma=None) or log-normal diffusion (sigma) with a seeded rhs.

    rhs="xtrue": x_true ~ U(-1, 1), b = A x_true.  rhs="uniform": b ~ U(-1, 1).
    """
    dims = tuple(int(d) for d in dims)
    rng = rng_for(tag)
    faces = face_coefficients(dims, sigma, rng) if sigma is not None else None
    n = int(np.prod(dims))
    if rhs == "xtrue":
        x_true = xtrue_uniform(n, rng)
        b = stencil_apply(dims, x_true, faces, shift)
    elif rhs == "uniform":
        x_true = None
        b = rng.uniform(-1.0, 1.0, size=n)
    else:
        raise ValueError(rhs)
    csr = stencil_csr(dims, faces, shift) if with_csr else None
    return GridProblem(dims, faces, shift, b, x_true, csr)


def poisson2d_64(**kw) -> GridProblem:
    """2D 5-point Poisson on a 64 x 64 interior grid (n = 4096)."""
    return grid_problem((64, 64), "poisson2d_64", **kw)


def poisson3d(nside: int = 256, **kw) -> GridProblem:
    """3D 7-point Poisson on an nside^3 grid."""
    return grid_problem((nside,) * 3, f"poisson3d_{nside}", **kw)


def varcoef3d(nside: int = 128, sigma: float = 2.0, **kw) -> GridProblem:
    """3D variable-coefficient diffusion with log-normal face coefficients."""
    return grid_problem((nside,) * 3, f"varcoef3d_{nside}", sigma=sigma, **kw)


def varcoef2d(nside: int = 512, sigma: float = 2.0, **kw) -> GridProblem:
    """2D variable-coefficient diffusion (the differentiation workload)."""
    return grid_problem((nside,) * 2, f"varcoef2d_{nside}", sigma=sigma, **kw)


@dataclasses.dataclass
class BatchSpec:
    sides: np.ndarray
    shifts: np.ndarray
    seed_tag: str

    def system(self, i: int) -> GridProblem:
        s = int(self.sides[i])
        return grid_problem((s, s), f"{self.seed_tag}_{i}", shift=float(self.shifts[i]),
                            with_csr=False, rhs="uniform")


def batch_spec(count: int = 512, side_lo: int = 32, side_hi: int = 448,
               shift_hi: float = 0.1, tag: str = "batch") -> BatchSpec:
    """Sides ~ U{side_lo..side_hi}, diagonal shifts ~ U[0, shift_hi]."""
    rng = rng_for(f"{tag}_{count}_{side_lo}_{side_hi}")
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    shifts = rng.uniform(0.0, shift_hi, size=count)
    return BatchSpec(sides, shifts, f"{tag}_{count}_{side_lo}_{side_hi}")
