"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds only random-input recipes (no step of the solver).  Both the CUDA
path and the CPU oracle take their inputs from here.

Recipes:
* ``gaussian``      iid N(0,1) entries (random matrices of Sec. V-B).
* ``conditioned``   A = U diag(s) V^T with s geometric from 1 to 1/kappa and U, V
                    random orthogonal.  For N a power of two U and V are products of
                    three randomised Walsh-Hadamard rounds (H D_1 H D_2 H D_3), applied
                    in O(N^2 log N) so that the matrix is exact to float64 rounding
                    without an O(N^3) float64 product; otherwise they are the Q factors
                    of Gaussian matrices with the R-diagonal sign fix (Haar).
* ``worst_case_max``   the tile form of the growth example of Sec. III-A.
* ``block_diag_dominant`` random off-diagonal tiles with dominant diagonal tiles (Sec. III-B).
* ``scale_diag_tiles`` multiplies the diagonal tile of chosen panels by a factor.
* ``special``       the formula-defined special matrices of Table III.

Matrices are returned as torch tensors whose storage is column-major (stride (1, N)),
the layout the C interface takes; ``.numpy()`` of such a tensor is the same matrix.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def colmajor_empty(N, M=None, dtype=torch.float64, device="cpu"):
    M = N if M is None else M
    return torch.empty((M, N), dtype=dtype, device=device).t()


def gaussian(N, seed, device="cpu", dtype=torch.float64):
    """iid N(0,1) N x N matrix, column-major storage."""
    g = _gen(seed, device)
    return torch.randn((N, N), generator=g, device=device, dtype=dtype).t()


def ones_rhs(A):
    """b = A * ones(N), accumulated in float64."""
    return (A.to(torch.float64) @ torch.ones(A.shape[1], 1, dtype=torch.float64,
                                              device=A.device)).reshape(-1)


def _fwht_rows_(M):
    """In-place normalised Walsh-Hadamard transform of every row of M (N a power of two)."""
    rows, N = M.shape
    h = 1
    scale = 1.0 / math.sqrt(2.0)
    while h < N:
        V = M.view(rows, N // (2 * h), 2, h)
        a = V[:, :, 0, :].clone()
        b = V[:, :, 1, :]
        V[:, :, 0, :].add_(b)
        V[:, :, 1, :].mul_(-1.0).add_(a)
        M.mul_(scale)
        h *= 2
    return M


def _random_signs(N, g, device):
    return (torch.randint(0, 2, (N,), generator=g).to(torch.float64) * 2.0 - 1.0).to(device)


def conditioned(N, kappa, seed, device="cpu"):
    """A = U diag(s) V^T, s_i = kappa^(-i/(N-1)), U and V random orthogonal (float64).

    For N a power of two the random signs and the singular values are drawn on the host
    and only the exact transforms (sign flips, additions, one scaling per level) run on
    ``device``, so the matrix is bit-identical on the host and on a GPU."""
    if N >= 2 and (N & (N - 1)) == 0:
        g = _gen(seed, "cpu")
        i = torch.arange(N, dtype=torch.float64)
        s = torch.pow(torch.tensor(float(kappa), dtype=torch.float64), -i / max(N - 1, 1))
        s = s.to(device)
        # Row-major work array R holds A^T while the transforms are applied:
        # A = U S V^T  <=>  A^T = V S U^T.  Start from S (diagonal), then
        # A^T = V (S U^T): right-multiply by U^T = (H D1 H D2 H D3)^T = D3 H D2 H D1 H,
        # then left-multiply by V = H E1 H E2 H E3.
        R = torch.diag(s)
        d = [_random_signs(N, g, device) for _ in range(6)]
        # right-multiplication by D3 H D2 H D1 H acts on rows of R: R <- R D3 H D2 H D1 H
        R.mul_(d[2].view(1, N)); _fwht_rows_(R)
        R.mul_(d[1].view(1, N)); _fwht_rows_(R)
        R.mul_(d[0].view(1, N)); _fwht_rows_(R)
        # left-multiplication by V = H E1 H E2 H E3: transpose, act on rows, transpose back
        Rt = R.t().contiguous()
        del R
        # (V X)^T = X^T V^T = X^T E3 H E2 H E1 H
        Rt.mul_(d[5].view(1, N)); _fwht_rows_(Rt)
        Rt.mul_(d[4].view(1, N)); _fwht_rows_(Rt)
        Rt.mul_(d[3].view(1, N)); _fwht_rows_(Rt)
        # Rt now holds (V S U^T)^T = U S V^T = A in row-major; return column-major view of A
        return Rt.t().contiguous().t()
    g = _gen(seed, device)
    i = torch.arange(N, dtype=torch.float64, device=device)
    s = torch.pow(torch.tensor(float(kappa), dtype=torch.float64, device=device),
                  -i / max(N - 1, 1))
    G1 = torch.randn((N, N), generator=g, device=device, dtype=torch.float64)
    G2 = torch.randn((N, N), generator=g, device=device, dtype=torch.float64)
    U = _haar(G1)
    V = _haar(G2)
    A = (U * s.view(1, N)) @ V.t()
    return A.t().contiguous().t()


def _haar(G):
    Q, R = torch.linalg.qr(G)
    return Q * torch.sign(torch.diagonal(R)).view(1, -1)


def worst_case_max(n, nb, alpha):
    """Tile form of the growth example of Sec. III-A.

    A_kk = alpha^-1 I (k < n), A_ik = -I (i > k), last tile column = I, zeros elsewhere.
    """
    N = n * nb
    A = np.zeros((N, N))
    I = np.eye(nb)
    for k in range(n):
        for i in range(n):
            blk = (slice(i * nb, (i + 1) * nb), slice(k * nb, (k + 1) * nb))
            if k == n - 1:
                A[blk] = I
            elif i == k:
                A[blk] = I / alpha
            elif i > k:
                A[blk] = -I
    return torch.from_numpy(np.asfortranarray(A)).t().contiguous().t()


def block_diag_dominant(n, nb, seed, slack=1.01):
    """Random off-diagonal tiles; A_jj = c_j I with c_j = slack * sum_{i != j} ||A_ij||_1."""
    rng = np.random.default_rng(seed)
    N = n * nb
    A = rng.standard_normal((N, N))
    for j in range(n):
        cs = slice(j * nb, (j + 1) * nb)
        tot = 0.0
        for i in range(n):
            if i != j:
                tot += float(np.max(np.sum(np.abs(A[i * nb:(i + 1) * nb, cs]), axis=0)))
        A[cs, cs] = np.eye(nb) * (slack * tot)
    return torch.from_numpy(A).t().contiguous().t()


SPECIAL = ("house", "parter", "ris", "lehmer", "hilb", "orthogo", "demmel")


def special(name, N, seed=0):
    """Formula-defined special matrices of Table III (1-based i, j), column-major float64:

    house    I - beta v v^T with v ~ N(0, 1) (seeded) and beta = 2 / (v^T v)
    parter   1 / (i - j + 0.5)                      (Toeplitz; singular values near pi)
    ris      0.5 / (n - i - j + 1.5)                (Hankel; eigenvalues near -pi/2, pi/2)
    lehmer   i / j for j >= i, symmetric            (positive definite, tridiagonal inverse)
    hilb     1 / (i + j - 1)
    orthogo  sqrt(2 / (n + 1)) sin(i j pi / (n + 1))  (symmetric orthogonal)
    demmel   D (I + 1e-7 R), D = diag(10^(14 (k - 1) / n)), R ~ U(0, 1) (seeded)
    """
    i = np.arange(1, N + 1, dtype=np.float64).reshape(-1, 1)
    j = np.arange(1, N + 1, dtype=np.float64).reshape(1, -1)
    rng = np.random.default_rng(seed)
    if name == "house":
        v = rng.standard_normal(N)
        A = np.eye(N) - (2.0 / float(v @ v)) * np.outer(v, v)
    elif name == "parter":
        A = 1.0 / (i - j + 0.5)
    elif name == "ris":
        A = 0.5 / (N - i - j + 1.5)
    elif name == "lehmer":
        A = np.minimum(i, j) / np.maximum(i, j)
    elif name == "hilb":
        A = 1.0 / (i + j - 1.0)
    elif name == "orthogo":
        A = np.sqrt(2.0 / (N + 1)) * np.sin(i * j * np.pi / (N + 1))
    elif name == "demmel":
        d = 10.0 ** (14.0 * np.arange(N) / N)
        A = d.reshape(-1, 1) * (np.eye(N) + 1e-7 * rng.random((N, N)))
    else:
        raise ValueError(f"unknown special matrix {name}")
    return torch.from_numpy(np.asfortranarray(A)).t().contiguous().t()


def choose_panels(n, frac, seed):
    """round(frac * n) distinct panel indices chosen by seed (sorted)."""
    rng = np.random.default_rng(seed + 7919)
    cnt = int(round(frac * n))
    return sorted(int(v) for v in rng.choice(n, size=cnt, replace=False))


def scale_diag_tiles(A, nb, panels, factor):
    """Multiply the diagonal tile of each listed panel of A by ``factor`` (copy)."""
    B = A.clone()
    for k in panels:
        s = slice(k * nb, (k + 1) * nb)
        B[s, s] *= factor
    return B


def batch_sizes(count, nmin, nmax, seed):
    """Uniform integer sizes in [nmin, nmax] (inclusive)."""
    rng = np.random.default_rng(seed)
    return [int(v) for v in rng.integers(nmin, nmax + 1, size=count)]
