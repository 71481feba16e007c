"""Plain CPU oracle of the hybrid LU-QR solver (Faverge, Herrmann, Langou, Lowery,
Robert, Dongarra, "Designing LU-QR hybrid solvers for performance and stability").

THIS MODULE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import it.  The GPU library never calls it and
it never calls the GPU library; the two share no code.

It is a deliberately slow, step-by-step restatement of the paper's method in
float64 (or float32 for the emulation of the low-precision factorisation):

* Alg. 1 (hybrid step loop), Eq. 1 (factor / apply / eliminate / update),
* Alg. 2 (LU step, variant A1: GETRF, TRSM, SWPTRSM, GEMM) and variant A2 of Sec. II-B
  (GEQRT of the diagonal tile, TRSM with its U, ORMQR apply, GEMM); the diagonal-domain
  Factor of Sec. II-B (pivoting across several tiles of the panel),
* Alg. 3 + Alg. 4(a)/(b) (QR step with TS or TT elimination kernels),
* Eq. 2 (Max), Eq. 3 (Sum) and Eq. 4 (MUMPS) robustness criteria (Sec. III), with the
  exact inverse norm or the Hager-Higham estimate, and the random choice of Sec. V-B,
* Sec. II-D "Solving systems of linear equations": the transformations are applied
  to the augmented matrix (A, b), followed by one N-by-N triangular solve, or
  replayed on a new right-hand side in a second pass,
* Sec. II-D "No restriction on N": native ragged last tile.

Householder reflectors are applied one at a time (never through a compact-WY T
factor), pivots are searched with a plain arg-max, and the triangular solves are
scalar loops, so that every kernel can be checked against its textbook definition
by eye.  Readings of points the paper leaves open are listed in ``READINGS``.

Parity status: every function here is pinned by tests/test_oracle_*.py.  The MUMPS
criterion is pinned to the closed forms of both readings (default: LU iff alpha >=
max_j away(j)/local(j); cumulative: a log-domain prefix-sum threshold) and to a
hand-worked 2x2-tile example; which reading the paper intends stays open, because it
prints no MUMPS numbers (only alpha = 2.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Codes shared (by value, not by code) with the C interface.
# ---------------------------------------------------------------------------
DEC_QR = 0
DEC_LU = 1

CRIT_MAX = 0       # Eq. 2
CRIT_SUM = 1       # Eq. 3
CRIT_MUMPS = 2     # Eq. 4
CRIT_FORCE_LU = 3  # alpha = infinity limit (Sec. V-B, "LU NoPiv" inside the tile)
CRIT_FORCE_QR = 4  # alpha = 0 limit (Sec. V-B)
CRIT_RANDOM = 5    # random choice, LU with probability alpha/100 (Sec. V-B, Fig. 2 fourth row)

_M64 = (1 << 64) - 1


def splitmix64_at(seed, i):
    """Output i (0-based) of the SplitMix64 generator started at state `seed` (Steele, Lea
    and Flood 2014): the state advances by 0x9E3779B97F4A7C15 per output, and each output
    is the state mixed by two xor-shift-multiply rounds and a final xor-shift."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def random_draw(seed, k):
    """u_k in [0, 1): the top 53 bits of SplitMix64 output k, times 2^-53 (exact)."""
    return float(splitmix64_at(seed, k) >> 11) * 2.0 ** -53

TREE_FLAT_TS = 0   # eliminator(i,k) = k, Alg. 4(a)
TREE_BINARY_TT = 1  # pairwise binary reduction, Alg. 4(b)
TREE_GROUPED = 2   # flat TS inside groups of g tiles, binary TT across group heads

INJECT_SCALE = 2.0 ** -27   # run-time tile-row scaling used to force a QR step

READINGS = {
    "pivot": "partial pivoting inside the diagonal tile only; pivot = first row of maximal |a|; "
             "domain=d: across tiles k..k+d-1 (Sec. II-B variant), exchanges applied to "
             "columns k.. only (earlier multipliers stay, as the replay applies steps in order)",
    "inverse_norm": "||A_kk^-1||_1 computed exactly from the L and U factors (X = U^-1 L^-1 P); "
                    "norm_mode=1: the Hager-Higham estimate (a lower bound, so the test admits "
                    "LU at least as often)",
    "lu_variant": "A1 (GETRF of the tile) by default; A2 factors the tile by GEQRT, a zero "
                  "diagonal entry of R playing the zero pivot's part",
    "random_choice": "Sec. V-B's random choice: LU with probability alpha/100, u_k = SplitMix64 "
                     "output k of the seed, top 53 bits times 2^-53, LU iff u_k < alpha/100; a "
                     "zero pivot still selects QR",
    "tree_per_step": "the elimination tree may change from step to step (Alg. 3 leaves it free); "
                     "a two-tree policy switches below a number of sub-diagonal tiles",
    "tie": ">= in Eq. 2-4 selects LU",
    "zero_pivot": "an exact zero pivot in the diagonal GETRF selects QR (FORCE_LU raises Singular)",
    "alpha_zero": "alpha = 0 selects QR at every step, the last one included",
    "last_step": "at k = n the sub-diagonal max/sum is 0: LU iff the tile is nonsingular",
    "mumps_r2": "est(j) = away(j) * (pivot(j) / local(j)); LU iff alpha*pivot(j) >= est(j) for all j",
    "mumps_r1": "est(j) = away(j) * prod_{l<j} pivot(l)/local(l) (mumps_mode=1)",
    "householder": "LAPACK dlarfg: beta = -sign(a0)*sqrt(a0^2+|x|^2), sign(0)=+1, tau=(beta-a0)/beta, v=x/(a0-beta); tau=0 if x=0",
    "loop_bounds": "Alg. 4 'j = k+1 to n-1' is read as j = k+1..n plus the right-hand side",
    "geqrt_once": "a tile is triangularised by GEQRT once, when it first takes part in an elimination",
    "ragged": "the last tile row/column has N-(n-1)nb entries; kernels take rectangular tiles",
    "inject": "run-time injection scales tile row k of [A^(k) | b^(k)] by 2^-27 before the criterion",
}


class NonFinite(Exception):
    """A NaN or Inf was met in the panel at step ``step`` (0-based)."""

    def __init__(self, step):
        super().__init__(f"non-finite panel at step {step}")
        self.step = step


class Singular(Exception):
    """An exact zero pivot where one cannot be tolerated (FORCE_LU, back solve)."""

    def __init__(self, step, row):
        super().__init__(f"singular at step {step}, row {row}")
        self.step = step
        self.row = row


# ---------------------------------------------------------------------------
# LU kernels (Alg. 2, Sec. II-A)
# ---------------------------------------------------------------------------
def getrf(T):
    """GETRF: P T = L U with partial pivoting over the rows of T, in place.

    T is the diagonal tile (square) or, for the diagonal-domain variant, the stacked
    tiles of the domain (tall: the pivot search covers every row below).
    Returns (piv, zero_row): piv[r] is the row exchanged with row r at elimination
    step r (0-based LAPACK ipiv convention); zero_row is the first r whose pivot is
    exactly zero (that column is then left unscaled), or -1.
    """
    p = min(T.shape)
    piv = np.arange(p)
    zero_row = -1
    for r in range(p):
        s = r + int(np.argmax(np.abs(T[r:, r])))
        piv[r] = s
        if s != r:
            T[[r, s], :] = T[[s, r], :]
        if T[r, r] == 0.0:
            if zero_row < 0:
                zero_row = r
            continue
        T[r + 1:, r] = T[r + 1:, r] / T[r, r]
        T[r + 1:, r + 1:] -= np.outer(T[r + 1:, r], T[r, r + 1:])
    return piv, zero_row


def apply_row_swaps(C, piv):
    """C <- P C for the ipiv sequence produced by getrf (swaps applied in order)."""
    for r in range(len(piv)):
        s = piv[r]
        if s != r:
            C[[r, s], :] = C[[s, r], :]


def unit_lower_solve(LU, C):
    """C <- L^-1 C, L unit lower triangular stored strictly below the diagonal of LU."""
    p = LU.shape[0]
    for r in range(p):
        C[r + 1:, :] -= np.outer(LU[r + 1:, r], C[r, :])


def upper_solve(LU, C):
    """C <- U^-1 C, U upper triangular stored in the upper triangle of LU."""
    p = LU.shape[0]
    for r in reversed(range(p)):
        C[r, :] = C[r, :] / LU[r, r]
        C[:r, :] -= np.outer(LU[:r, r], C[r, :])


def trsm_right_upper(X, LU):
    """Eliminate: X <- X U^-1 (Alg. 2, TRSM on A_ik)."""
    p = LU.shape[0]
    for c in range(p):
        X[:, c] = X[:, c] / LU[c, c]
        X[:, c + 1:] -= np.outer(X[:, c], LU[c, c + 1:])


def swptrsm(C, LU, piv):
    """Apply: C <- L^-1 P C (Alg. 2, SWPTRSM on A_kj and on the right-hand side)."""
    apply_row_swaps(C, piv)
    unit_lower_solve(LU, C)


def gemm_update(C, A, B):
    """Update: C <- C - A B (Alg. 2, GEMM)."""
    C -= A @ B


# ---------------------------------------------------------------------------
# Householder kernels (Alg. 4)
# ---------------------------------------------------------------------------
def householder(a0, x):
    """Reflector H = I - tau [1; v][1; v]^T with H [a0; x] = [beta; 0].

    LAPACK dlarfg convention: beta = -sign(a0) * sqrt(a0^2 + |x|^2) with sign(0) = +1,
    tau = (beta - a0) / beta, v = x / (a0 - beta); tau = 0 and H = I when x = 0.
    """
    ss = float(np.sum(x * x)) if x.size else 0.0
    if ss == 0.0:
        return a0, 0.0, np.zeros_like(x)
    nrm = math.sqrt(float(a0) * float(a0) + ss)
    beta = -nrm if a0 >= 0.0 else nrm
    tau = (beta - a0) / beta
    v = x / (a0 - beta)
    return beta, tau, v


def geqrt(T):
    """GEQRT: T = Q R in place (R upper, reflector tails strictly below the diagonal).

    Returns tau (length min(rows, cols)).  Reflector j acts on rows j..end.
    """
    p, q = T.shape
    kk = min(p, q)
    tau = np.zeros(kk, dtype=T.dtype)
    for j in range(kk):
        beta, t, v = householder(T[j, j], T[j + 1:, j].copy())
        T[j, j] = beta
        T[j + 1:, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < q:
            w = T[j, j + 1:] + v @ T[j + 1:, j + 1:]
            T[j, j + 1:] -= t * w
            T[j + 1:, j + 1:] -= t * np.outer(v, w)
    return tau


def unmqr(V, tau, C):
    """UNMQR: C <- Q^T C for the reflectors left in V by geqrt (H_0 applied first)."""
    for j in range(len(tau)):
        t = tau[j]
        if t == 0.0:
            continue
        v = V[j + 1:, j]
        w = C[j, :] + v @ C[j + 1:, :]
        C[j, :] -= t * w
        C[j + 1:, :] -= t * np.outer(v, w)


def tsqrt(R, A):
    """TSQRT: QR of [R; A] with R upper triangular (the eliminator) and A full.

    R is overwritten by the new triangle, A by the reflector tails (reflector j is
    [e_j; A[:, j]] in the stacked coordinates).  Returns tau.
    """
    q = R.shape[1]
    tau = np.zeros(q, dtype=R.dtype)
    for j in range(q):
        beta, t, v = householder(R[j, j], A[:, j].copy())
        R[j, j] = beta
        A[:, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < q:
            w = R[j, j + 1:] + v @ A[:, j + 1:]
            R[j, j + 1:] -= t * w
            A[:, j + 1:] -= t * np.outer(v, w)
    return tau


def tsmqr(V2, tau, C1, C2):
    """TSMQR: [C1; C2] <- Q^T [C1; C2] for the reflectors of a tsqrt (row j of C1 pairs with C2)."""
    for j in range(len(tau)):
        t = tau[j]
        if t == 0.0:
            continue
        v = V2[:, j]
        w = C1[j, :] + v @ C2
        C1[j, :] -= t * w
        C2 -= t * np.outer(v, w)


def ttqrt(R1, R2):
    """TTQRT: QR of [R1; R2] with both upper triangular (R2 may be upper trapezoidal).

    Reflector j only involves rows 0..j of R2, so R2 stays upper triangular and
    holds the reflector tails on exit.  Returns tau.
    """
    q = R1.shape[1]
    p = R2.shape[0]
    tau = np.zeros(q, dtype=R1.dtype)
    for j in range(q):
        rows = min(j + 1, p)
        beta, t, v = householder(R1[j, j], R2[:rows, j].copy())
        R1[j, j] = beta
        R2[:rows, j] = v
        tau[j] = t
        if t != 0.0 and j + 1 < q:
            w = R1[j, j + 1:] + v @ R2[:rows, j + 1:]
            R1[j, j + 1:] -= t * w
            R2[:rows, j + 1:] -= t * np.outer(v, w)
    return tau


def ttmqr(V2, tau, C1, C2):
    """TTMQR: [C1; C2] <- Q^T [C1; C2] for the reflectors of a ttqrt."""
    p = C2.shape[0]
    for j in range(len(tau)):
        t = tau[j]
        if t == 0.0:
            continue
        rows = min(j + 1, p)
        v = V2[:rows, j]
        w = C1[j, :] + v @ C2[:rows, :]
        C1[j, :] -= t * w
        C2[:rows, :] -= t * np.outer(v, w)


# ---------------------------------------------------------------------------
# Criterion inputs (Sec. III-D) and the decision (Eq. 2, 3, 4)
# ---------------------------------------------------------------------------
def norm1(T):
    """||T||_1: maximum column absolute sum, accumulated in float64."""
    if T.size == 0:
        return 0.0
    return float(np.max(np.sum(np.abs(T.astype(np.float64)), axis=0)))


def inv_norm1(LU, piv):
    """||A_kk^-1||_1 from the GETRF factors: X = U^-1 L^-1 P, max column abs sum (float64)."""
    p = LU.shape[0]
    L64 = LU.astype(np.float64)
    X = np.eye(p)
    apply_row_swaps(X, piv)
    unit_lower_solve(L64, X)
    upper_solve(L64, X)
    return norm1(X)


def inv_norm1_qr(QR, tau):
    """||A_kk^-1||_1 from a GEQRT of the tile (LU variant A2): X = U^-1 Q^T, max column
    abs sum (float64)."""
    p = QR.shape[0]
    Q64 = QR.astype(np.float64)
    X = np.eye(p)
    unmqr(Q64, np.asarray(tau, dtype=np.float64), X)
    upper_solve(Q64, X)
    return norm1(X)


def _solve_t(L64, piv, x):
    """A^-T x for A = P^T L U: U^-T, then L^-T (unit), then P^T (swaps in reverse order)."""
    p = L64.shape[0]
    w = np.array(x, dtype=np.float64)
    for r in range(p):                      # U^T w = x, forward
        w[r] = (w[r] - np.dot(L64[:r, r], w[:r])) / L64[r, r]
    for r in reversed(range(p)):            # L^T v = w, backward, unit diagonal
        w[r] = w[r] - np.dot(L64[r + 1:, r], w[r + 1:])
    for r in reversed(range(p)):
        s = piv[r]
        if s != r:
            w[[r, s]] = w[[s, r]]
    return w


def _solve(L64, piv, x):
    """A^-1 x for A = P^T L U: P, then L^-1 (unit), then U^-1."""
    y = np.array(x, dtype=np.float64).reshape(-1, 1)
    apply_row_swaps(y, piv)
    unit_lower_solve(L64, y)
    upper_solve(L64, y)
    return y[:, 0]


def _sign(v):
    return np.where(v >= 0.0, 1.0, -1.0)


def inv_norm1_est(LU, piv):
    """Estimate of ||A_kk^-1||_1 in O(nb^2) per iteration (the paper's Sec. III-D uses an
    iterative estimate; this is the Hager (1984) / Higham (1988) 1-norm estimator).

    f(x) = ||A^-1 x||_1 is convex, so its maximum over the unit 1-norm ball is reached at a
    vertex e_j and equals the largest column sum of |A^-1|.  Starting from the centre
    x = e/n, each iteration takes the sub-gradient z = A^-T sign(A^-1 x) and moves to the
    vertex e_j of the largest |z_j|; it stops when the sign vector repeats, the value stops
    growing, the best vertex stays the same, or after five iterations.  A last probe with
    the alternating vector x_i = (-1)^i (1 + i/(n-1)) guards against unlucky paths; its
    value 2||A^-1 x||_1 / (3n) is taken when larger.  Every value is ||A^-1 w||_1 for some
    ||w||_1 <= 1, so the estimate never exceeds the exact norm (up to rounding)."""
    p = LU.shape[0]
    L64 = LU.astype(np.float64)
    if p == 1:
        return abs(1.0 / L64[0, 0])
    y = _solve(L64, piv, np.full(p, 1.0 / p))
    est = float(np.sum(np.abs(y)))
    xi = _sign(y)
    z = _solve_t(L64, piv, xi)
    j = int(np.argmax(np.abs(z)))
    it = 2
    while True:
        e = np.zeros(p)
        e[j] = 1.0
        y = _solve(L64, piv, e)
        est_old = est
        est = float(np.sum(np.abs(y)))
        if np.array_equal(_sign(y), xi) or est <= est_old:
            break
        xi = _sign(y)
        z = _solve_t(L64, piv, xi)
        jlast = j
        j = int(np.argmax(np.abs(z)))
        if abs(z[jlast]) == abs(z[j]) or it >= 5:
            break
        it += 1
    i = np.arange(p, dtype=np.float64)
    alt = np.where(np.arange(p) % 2 == 0, 1.0, -1.0) * (1.0 + i / (p - 1))
    t = 2.0 * float(np.sum(np.abs(_solve(L64, piv, alt)))) / (3.0 * p)
    return max(est, t)


@dataclass
class StepDecision:
    dec: int
    margin: float
    lhs: float = float("nan")
    rhs: float = float("nan")


def decide(criterion, alpha, LU, piv, zero_row, norms_below, local_max, away_max,
           mumps_mode=0, norm_mode=0, seed=0, k=0, qr_tau=None):
    """Robustness test of Sec. III.

    Max (Eq. 2):   alpha * (1/||A_kk^-1||_1) >= max_{i>k} ||A_ik||_1
    Sum (Eq. 3):   alpha * (1/||A_kk^-1||_1) >= sum_{i>k} ||A_ik||_1 (ascending i)
    MUMPS (Eq. 4): for all j, alpha * pivot(j) >= estimate_max(j)
    The margin is log2(lhs/rhs) (minimum over j for MUMPS).
    """
    if criterion == CRIT_FORCE_LU:
        return StepDecision(DEC_LU, math.inf)
    if criterion == CRIT_FORCE_QR or alpha == 0.0:
        return StepDecision(DEC_QR, -math.inf)
    if zero_row >= 0:
        return StepDecision(DEC_QR, -math.inf, 0.0)
    if criterion == CRIT_RANDOM:
        lhs = alpha / 100.0
        rhs = random_draw(seed, k)
        return StepDecision(DEC_LU if rhs < lhs else DEC_QR, _log2_ratio(lhs, rhs), lhs, rhs)
    if criterion in (CRIT_MAX, CRIT_SUM):
        if qr_tau is not None:        # LU variant A2: the tile was factored by GEQRT
            inv = inv_norm1_qr(LU, qr_tau)
        else:
            inv = inv_norm1(LU, piv) if norm_mode == 0 else inv_norm1_est(LU, piv)
        lhs = alpha * (1.0 / inv)
        if criterion == CRIT_MAX:
            rhs = max(norms_below) if len(norms_below) else 0.0
        else:
            rhs = 0.0
            for v in norms_below:
                rhs = rhs + v
        margin = _log2_ratio(lhs, rhs)
        return StepDecision(DEC_LU if lhs >= rhs else DEC_QR, margin, lhs, rhs)
    if criterion == CRIT_MUMPS:
        ok = True
        margin = math.inf
        gprod = 1.0
        for j in range(LU.shape[0]):
            pj = abs(float(LU[j, j]))
            lj = float(local_max[j])
            if lj == 0.0:
                return StepDecision(DEC_QR, -math.inf)
            if mumps_mode == 0:
                est = float(away_max[j]) * (pj / lj)
            else:
                est = float(away_max[j]) * gprod
                gprod = gprod * (pj / lj)
            lhs = alpha * pj
            if not lhs >= est:
                ok = False
            margin = min(margin, _log2_ratio(lhs, est))
        return StepDecision(DEC_LU if ok else DEC_QR, margin)
    raise ValueError(f"unknown criterion {criterion}")


def _log2_ratio(lhs, rhs):
    if rhs == 0.0:
        return math.inf if lhs > 0.0 else (0.0 if lhs == 0.0 else -math.inf)
    if lhs == 0.0:
        return -math.inf
    if math.isinf(lhs):
        return math.inf
    return math.log2(lhs / rhs)


# ---------------------------------------------------------------------------
# Elimination lists (Alg. 3; the tree is a free parameter of the paper)
# ---------------------------------------------------------------------------
def elimination_ops(k, n, tree, group=4):
    """Ordered QR-step operations for panel k over tile rows k..n-1 (0-based).

    ("geqrt", i): triangularise tile (i,k) and apply its Q^T to row i (UNMQR).
    ("ts", i, e): tile (i,k) (square) is eliminated by triangle (e,k): TSQRT + TSMQR.
    ("tt", i, e): triangle (i,k) is eliminated by triangle (e,k): TTQRT + TTMQR.
    """
    m = n - 1 - k
    ops = []
    if tree == TREE_FLAT_TS:
        ops.append(("geqrt", k))
        for i in range(k + 1, n):
            ops.append(("ts", i, k))
    elif tree == TREE_BINARY_TT:
        for i in range(k, n):
            ops.append(("geqrt", i))
        step = 1
        while step <= m:
            for d in range(step, m + 1, 2 * step):
                ops.append(("tt", k + d, k + d - step))
            step *= 2
    elif tree == TREE_GROUPED:
        g = max(1, int(group))
        heads = list(range(k, n, g))
        for h in heads:
            ops.append(("geqrt", h))
            for i in range(h + 1, min(h + g, n)):
                ops.append(("ts", i, h))
        step = 1
        H = len(heads)
        while step < H:
            for d in range(step, H, 2 * step):
                ops.append(("tt", heads[d], heads[d - step]))
            step *= 2
    else:
        raise ValueError(f"unknown tree {tree}")
    return ops


# ---------------------------------------------------------------------------
# Flop model (Table I, unit nb^3)
# ---------------------------------------------------------------------------
def step_flops(dec, m, nb):
    """Table I: LU = 2/3 + (n-1) + (n-1) + 2(n-1)^2, QR = 4/3 + 2(n-1) + 2(n-1) + 4(n-1)^2."""
    if dec == DEC_LU:
        units = 2.0 / 3.0 + 2.0 * m + 2.0 * m * m
    else:
        units = 4.0 / 3.0 + 4.0 * m + 4.0 * m * m
    return units * float(nb) ** 3


def normalized_gflops(N, seconds):
    """Sec. V-A: normalized GFLOP/s = (2/3) N^3 / time."""
    return (2.0 / 3.0) * float(N) ** 3 / seconds / 1e9


def true_gflops(N, seconds, f_lu):
    """Table II caption: true flops = (2/3 f_LU + 4/3 (1 - f_LU)) N^3."""
    return ((2.0 / 3.0) * f_lu + (4.0 / 3.0) * (1.0 - f_lu)) * float(N) ** 3 / seconds / 1e9


# ---------------------------------------------------------------------------
# The factorization (Alg. 1)
# ---------------------------------------------------------------------------
@dataclass
class Factorization:
    N: int
    nb: int
    n: int
    nrhs: int
    aug: np.ndarray                  # N x (N + nrhs): transformed [A | b]
    dec: np.ndarray                  # uint8[n]
    margin: np.ndarray               # float64[n]
    lhs: np.ndarray
    rhs: np.ndarray
    piv: dict = field(default_factory=dict)       # k -> ipiv (LU steps)
    taus: dict = field(default_factory=dict)      # (k, op) -> tau
    ops: dict = field(default_factory=dict)       # k -> elimination list (QR steps)
    injected: tuple = ()
    flops: float = 0.0
    growth: list = field(default_factory=list)    # max_{i,j>=k} ||A_ij^(k)||_1 per step
    norms: dict = field(default_factory=dict)     # k -> ||A_ik^(k)||_1, i = k..n-1
    domain_piv: dict = field(default_factory=dict)  # k -> (tiles, ipiv) of a domain LU step
    lu_tau: dict = field(default_factory=dict)      # k -> tau of an A2 LU step (GEQRT)

    @property
    def U(self):
        return np.triu(self.aug[:, :self.N])

    @property
    def c(self):
        return self.aug[:, self.N:]


def tile_bounds(i, nb, N):
    return i * nb, min((i + 1) * nb, N)


def factor(A, b, nb, criterion, alpha, tree=TREE_FLAT_TS, group=4, mumps_mode=0,
           forced=None, inject=(), dtype=np.float64, track_growth=False, on_step=None,
           norm_mode=0, seed=0, domain=1, lu_variant="A1", tree_small=TREE_FLAT_TS,
           tree_switch=0):
    """Run Alg. 1 on the augmented matrix [A | b] and return the Factorization.

    A: N x N; b: None, N or N x nrhs.  dtype float32 emulates the whole factorization
    in single precision (criterion norms and the comparison stay float64).
    ``forced``: optional per-step decisions replacing the criterion (replay).
    ``inject``: steps whose tile row is scaled by 2^-27 before the criterion.
    ``on_step(k, aug_before, fact)``: test hook called before each step.
    ``norm_mode``: 0 exact ||A_kk^-1||_1, 1 the Hager-Higham estimate (inv_norm1_est).
    ``seed``: SplitMix64 seed of CRIT_RANDOM's per-step draws.
    ``domain``: tiles of the diagonal domain (Sec. II-B variant): the Factor step pivots
    across tiles k .. k+domain-1 of the panel (a tall GETRF on a scratch copy); the
    criterion sees the pivoted panel; an LU step first applies the domain's row
    exchanges to columns k.. of those rows (and b), then runs Alg. 2 on the pivoted
    diagonal tile.  1 = pivoting inside the diagonal tile only.
    ``tree_small``, ``tree_switch``: steps with fewer than tree_switch sub-diagonal tiles
    eliminate along tree_small, the others along ``tree`` (Alg. 3 leaves the tree free at
    every step); tree_switch = 0 uses ``tree`` throughout.
    ``lu_variant``: "A1" (Alg. 2: GETRF of the tile) or "A2" (Sec. II-B: GEQRT of the
    tile; Eliminate A_ik U^-1, Apply Q^T A_kj, the same Update; a QR decision continues
    from that GEQRT).
    """
    assert lu_variant in ("A1", "A2")
    assert lu_variant == "A1" or (domain == 1 and norm_mode == 0)
    A = np.asarray(A)
    N = A.shape[0]
    assert A.shape == (N, N) and N >= 1 and nb >= 1
    if b is None:
        bb = np.zeros((N, 0))
    else:
        bb = np.asarray(b).reshape(N, -1)
    nrhs = bb.shape[1]
    aug = np.empty((N, N + nrhs), dtype=dtype)
    aug[:, :N] = A
    aug[:, N:] = bb
    n = (N + nb - 1) // nb
    W = N + nrhs
    fact = Factorization(N=N, nb=nb, n=n, nrhs=nrhs, aug=aug,
                         dec=np.zeros(n, dtype=np.uint8), margin=np.zeros(n),
                         lhs=np.full(n, np.nan), rhs=np.full(n, np.nan),
                         injected=tuple(sorted(set(int(s) for s in inject))))
    inject_set = set(fact.injected)
    for k in range(n):
        r0, r1 = tile_bounds(k, nb, N)
        if k in inject_set:
            aug[r0:r1, r0:W] *= dtype(INJECT_SCALE)
        if on_step is not None:
            on_step(k, aug, fact)
        m = n - 1 - k
        # -- criterion inputs on the panel A^(k)_{ik}, i >= k (Sec. III-D)
        norms = []
        for i in range(k, n):
            a0, a1 = tile_bounds(i, nb, N)
            T = aug[a0:a1, r0:r1]
            if not np.all(np.isfinite(T)):
                raise NonFinite(k)
            norms.append(norm1(T))
        fact.norms[k] = np.array(norms)
        if track_growth:
            fact.growth.append(max(norm1(aug[a0:a1, c0:c1])
                                   for i in range(k, n) for j in range(k, n)
                                   for (a0, a1) in [tile_bounds(i, nb, N)]
                                   for (c0, c1) in [tile_bounds(j, nb, N)]))
        dd = min(max(int(domain), 1), n - k)
        if dd > 1:
            # -- factor across the diagonal domain: tall GETRF of a scratch copy of the
            #    stacked tiles k .. k+dd-1; the criterion sees the pivoted panel
            q1 = tile_bounds(k + dd - 1, nb, N)[1]
            S = aug[r0:q1, r0:r1].copy()
            dpiv, zero_row = getrf(S)
            panel = aug[r0:N, r0:r1].copy()
            apply_row_swaps(panel[:q1 - r0], dpiv)
            norms = [norm1(panel[a0 - r0:a1 - r0]) for i in range(k, n)
                     for (a0, a1) in [tile_bounds(i, nb, N)]]
            fact.norms[k] = np.array(norms)
            Akk = panel[:r1 - r0]
            LU = S[:r1 - r0].copy()
            piv = np.arange(r1 - r0)
            away_src = panel[r1 - r0:]
        else:
            Akk = aug[r0:r1, r0:r1]
            away_src = aug[r1:N, r0:r1]
        local_max = np.max(np.abs(Akk.astype(np.float64)), axis=0)
        if m > 0:
            away_max = np.max(np.abs(away_src.astype(np.float64)), axis=0)
        else:
            away_max = np.zeros(r1 - r0)
        qr_tau = None
        if dd == 1 and lu_variant == "A2":
            # -- factor (variant A2): GEQRT of a scratch copy of the diagonal tile
            LU = Akk.copy()
            qr_tau = geqrt(LU)
            piv = np.arange(r1 - r0)
            zd = np.flatnonzero(np.diag(LU) == 0.0)
            zero_row = int(zd[0]) if len(zd) else -1
        elif dd == 1:
            # -- factor: GETRF of a scratch copy of the diagonal tile (Alg. 1, "Factor")
            LU = Akk.copy()
            piv, zero_row = getrf(LU)
        # -- check (Alg. 1, "Check")
        if forced is not None:
            d = int(forced[k])
            sd = StepDecision(d, math.inf if d == DEC_LU else -math.inf)
        else:
            sd = decide(criterion, alpha, LU, piv, zero_row, norms[1:], local_max,
                        away_max, mumps_mode, norm_mode, seed, k, qr_tau)
        if sd.dec == DEC_LU and zero_row >= 0:
            raise Singular(k, r0 + zero_row)
        fact.dec[k] = sd.dec
        fact.margin[k] = sd.margin
        fact.lhs[k] = sd.lhs
        fact.rhs[k] = sd.rhs
        fact.flops += step_flops(sd.dec, m, nb)
        if sd.dec == DEC_LU:
            if dd > 1:
                apply_row_swaps(aug[r0:q1, r0:W], dpiv)
                fact.domain_piv[k] = (dd, dpiv)
            if qr_tau is not None:
                _lu_step_a2(aug, k, nb, N, W, LU, qr_tau)
                fact.lu_tau[k] = qr_tau
            else:
                _lu_step(aug, k, n, nb, N, W, LU, piv)
            fact.piv[k] = piv
        else:
            tree_k = tree_small if (tree_switch > 0 and m < tree_switch) else tree
            ops = elimination_ops(k, n, tree_k, group)
            fact.ops[k] = ops
            _qr_step(aug, k, nb, N, W, ops, fact.taus)
    return fact


def _lu_step(aug, k, n, nb, N, W, LU, piv):
    """Alg. 2 (variant A1) on the augmented matrix."""
    r0, r1 = tile_bounds(k, nb, N)
    aug[r0:r1, r0:r1] = LU                                   # Factor (commit scratch LU)
    if r1 < N:
        trsm_right_upper(aug[r1:N, r0:r1], LU)              # Eliminate: A_ik U^-1
    if r1 < W:
        swptrsm(aug[r0:r1, r1:W], LU, piv)                  # Apply: L^-1 P A_kj (and b_k)
    if r1 < N and r1 < W:
        gemm_update(aug[r1:N, r1:W], aug[r1:N, r0:r1], aug[r0:r1, r1:W])  # Update


def _lu_step_a2(aug, k, nb, N, W, QR, tau):
    """LU step, variant A2 (Sec. II-B): Factor by GEQRT (V below, U on and above the
    diagonal), Eliminate A_ik U^-1, Apply Q^T A_kj (and b_k), Update as in A1."""
    r0, r1 = tile_bounds(k, nb, N)
    aug[r0:r1, r0:r1] = QR
    if r1 < N:
        trsm_right_upper(aug[r1:N, r0:r1], QR)
    if r1 < W:
        unmqr(QR, tau, aug[r0:r1, r1:W])
    if r1 < N and r1 < W:
        gemm_update(aug[r1:N, r1:W], aug[r1:N, r0:r1], aug[r0:r1, r1:W])


def _qr_step(aug, k, nb, N, W, ops, taus):
    """Alg. 3 with the kernels of Alg. 4 along the given elimination list."""
    c0, c1 = tile_bounds(k, nb, N)
    for op in ops:
        if op[0] == "geqrt":
            i = op[1]
            a0, a1 = tile_bounds(i, nb, N)
            t = geqrt(aug[a0:a1, c0:c1])
            unmqr(aug[a0:a1, c0:c1], t, aug[a0:a1, c1:W])
            taus[(k, op)] = t
        else:
            kind, i, e = op
            a0, a1 = tile_bounds(i, nb, N)
            e0, e1 = tile_bounds(e, nb, N)
            R = aug[e0:e1, c0:c1]
            V = aug[a0:a1, c0:c1]
            if kind == "ts":
                t = tsqrt(R, V)
                tsmqr(V, t, aug[e0:e1, c1:W], aug[a0:a1, c1:W])
            else:
                t = ttqrt(R, V)
                ttmqr(V, t, aug[e0:e1, c1:W], aug[a0:a1, c1:W])
            taus[(k, op)] = t


# ---------------------------------------------------------------------------
# Solves (Sec. II-D)
# ---------------------------------------------------------------------------
def back_substitution(U, c):
    """Solve U x = c with U upper triangular (scalar back substitution)."""
    N = U.shape[0]
    x = np.array(c, dtype=np.float64, copy=True).reshape(N, -1)
    Uf = U.astype(np.float64)
    for r in reversed(range(N)):
        if Uf[r, r] == 0.0:
            raise Singular(-1, r)
        if r + 1 < N:
            x[r, :] -= Uf[r, r + 1:] @ x[r + 1:, :]
        x[r, :] = x[r, :] / Uf[r, r]
    return x


def apply_transforms(fact, b):
    """Second pass: replay every step's transformation on a new right-hand side."""
    N, nb, n = fact.N, fact.nb, fact.n
    aug = fact.aug
    y = np.array(b, dtype=aug.dtype, copy=True).reshape(N, -1)
    inj = set(fact.injected)
    for k in range(n):
        r0, r1 = tile_bounds(k, nb, N)
        if k in inj:
            y[r0:r1] *= aug.dtype.type(INJECT_SCALE)
        if fact.dec[k] == DEC_LU:
            LU = aug[r0:r1, r0:r1]
            if k in fact.domain_piv:
                dd, dpiv = fact.domain_piv[k]
                apply_row_swaps(y[r0:tile_bounds(k + dd - 1, nb, N)[1]], dpiv)
            if k in fact.lu_tau:
                unmqr(LU, fact.lu_tau[k], y[r0:r1])
            else:
                swptrsm(y[r0:r1], LU, fact.piv[k])
            if r1 < N:
                y[r1:N] -= aug[r1:N, r0:r1] @ y[r0:r1]
        else:
            for op in fact.ops[k]:
                t = fact.taus[(k, op)]
                if op[0] == "geqrt":
                    a0, a1 = tile_bounds(op[1], nb, N)
                    unmqr(aug[a0:a1, r0:r1], t, y[a0:a1])
                else:
                    kind, i, e = op
                    a0, a1 = tile_bounds(i, nb, N)
                    e0, e1 = tile_bounds(e, nb, N)
                    if kind == "ts":
                        tsmqr(aug[a0:a1, r0:r1], t, y[e0:e1], y[a0:a1])
                    else:
                        ttmqr(aug[a0:a1, r0:r1], t, y[e0:e1], y[a0:a1])
    return y


def solve(A, b, nb, criterion, alpha, **kw):
    """Factor the augmented system and back-substitute; returns (x, Factorization)."""
    fact = factor(A, b, nb, criterion, alpha, **kw)
    x = back_substitution(fact.U, fact.c)
    return x, fact


def replay_solve(fact, b):
    """Solve A x = b from a finished Factorization by replaying its transforms."""
    y = apply_transforms(fact, b)
    return back_substitution(fact.U, y)


# ---------------------------------------------------------------------------
# Accuracy measures (Sec. V-A and the normwise backward error)
# ---------------------------------------------------------------------------
def backward_error(A, x, b):
    """eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64).reshape(A.shape[0], -1)
    b = np.asarray(b, dtype=np.float64).reshape(A.shape[0], -1)
    r = b - A @ x
    nA = np.max(np.sum(np.abs(A), axis=1))
    return float(np.max(np.abs(r)) / (nA * np.max(np.abs(x)) + np.max(np.abs(b))))


def hpl3(A, x, b):
    """Sec. V-A: HPL3 = ||Ax - b||_inf / (||A||_inf ||x||_inf * eps * N), eps = 2^-53."""
    A = np.asarray(A, dtype=np.float64)
    N = A.shape[0]
    x = np.asarray(x, dtype=np.float64).reshape(N, -1)
    b = np.asarray(b, dtype=np.float64).reshape(N, -1)
    r = A @ x - b
    nA = np.max(np.sum(np.abs(A), axis=1))
    return float(np.max(np.abs(r)) / (nA * np.max(np.abs(x)) * 2.0 ** -53 * N))
