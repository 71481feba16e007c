// Plain threaded CPU restatement of the hybrid LU-QR oracle, for the large sizes.
//
// THIS FILE IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
// baseline of the benchmark use it (through oracle/luqr_oracle_mt.py).  It shares no code,
// header or constant table with the GPU library, and it never calls it.
//
// It computes what oracle/luqr_oracle.py computes, step for step, for the options that
// the large configurations use (Max / Sum / MUMPS / forced / random criteria, exact
// inverse norm, flat-TS / binary-TT / grouped trees, run-time injection, replayed
// decisions, float64 or float32 storage, native ragged last tile):
//   * Alg. 1: per panel k, the tile norms ||A_ik||_1 (float64 sums), the column maxima
//     of the MUMPS test, GETRF of a scratch copy of A_kk (partial pivoting inside the
//     tile, first row of maximal |a|), the exact ||A_kk^-1||_1 = max column sum of
//     U^-1 L^-1 P, and the decision of Eq. 2 (Max), Eq. 3 (Sum) or Eq. 4 (MUMPS);
//   * Alg. 2 (LU step, variant A1): commit, TRSM A_ik U^-1, SWPTRSM L^-1 P A_kj, GEMM;
//   * Alg. 3 with Alg. 4(a)/(b) (QR step): GEQRT, UNMQR, TSQRT/TSMQR, TTQRT/TTMQR
//     along the elimination list of the tree, reflectors applied one at a time
//     (LAPACK dlarfg convention), never through a compact-WY T;
//   * Sec. II-D: the transformations act on the augmented matrix [A | b]; then one
//     N x N back substitution.
//
// Threads only split work that the algorithm leaves independent: the columns of the
// trailing matrix (every transformation of a step acts on each column separately, the
// paper's "for j = k+1 .. n" loops), and the rows of the TRSM.  Each column sees exactly
// the same operations in the same order whatever the thread count, so results do not
// depend on it.  Dot products are plain sequential sums; built with -O3 -ffp-contract=off,
// no fast-math and no BLAS, so the same source gives the same bits on every host.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

enum { DEC_QR = 0, DEC_LU = 1, DEC_NONE = 255 };
enum { CRIT_MAX = 0, CRIT_SUM = 1, CRIT_MUMPS = 2, CRIT_FORCE_LU = 3, CRIT_FORCE_QR = 4,
       CRIT_RANDOM = 5 };
enum { TREE_FLAT_TS = 0, TREE_BINARY_TT = 1, TREE_GROUPED = 2 };
enum { OK = 0, E_INVALID = -1, E_SINGULAR = -4, E_NONFINITE = -5 };
enum { OP_GEQRT = 0, OP_TS = 1, OP_TT = 2 };

struct Op {
  int kind, i, e;
};

// Elimination list of panel k (Alg. 3; the tree is a free parameter of the paper).
std::vector<Op> elimination_ops(int k, int n, int tree, int group) {
  std::vector<Op> ops;
  const int m = n - 1 - k;
  if (tree == TREE_FLAT_TS) {
    ops.push_back({OP_GEQRT, k, k});
    for (int i = k + 1; i < n; ++i) ops.push_back({OP_TS, i, k});
  } else if (tree == TREE_BINARY_TT) {
    for (int i = k; i < n; ++i) ops.push_back({OP_GEQRT, i, i});
    for (int step = 1; step <= m; step *= 2)
      for (int d = step; d <= m; d += 2 * step) ops.push_back({OP_TT, k + d, k + d - step});
  } else {
    const int g = std::max(1, group);
    std::vector<int> heads;
    for (int h = k; h < n; h += g) heads.push_back(h);
    for (int h : heads) {
      ops.push_back({OP_GEQRT, h, h});
      for (int i = h + 1; i < std::min(h + g, n); ++i) ops.push_back({OP_TS, i, h});
    }
    const int H = (int)heads.size();
    for (int step = 1; step < H; step *= 2)
      for (int d = step; d < H; d += 2 * step) ops.push_back({OP_TT, heads[d], heads[d - step]});
  }
  return ops;
}

// Runs fn(lo, hi) over [b, e) split into `threads` contiguous chunks (multiples of `gran`).
template <typename F>
void parallel_range(int64_t b, int64_t e, int threads, int64_t gran, F&& fn) {
  const int64_t len = e - b;
  if (len <= 0) return;
  int t = std::max(1, threads);
  const int64_t units = (len + gran - 1) / gran;
  if (units < t) t = (int)units;
  if (t <= 1) {
    fn(b, e);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(t);
  for (int q = 0; q < t; ++q) {
    const int64_t lo = b + std::min(len, (units * q / t) * gran);
    const int64_t hi = b + std::min(len, (units * (q + 1) / t) * gran);
    if (lo < hi) pool.emplace_back([&fn, lo, hi] { fn(lo, hi); });
  }
  for (auto& th : pool) th.join();
}

uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
  // output i of SplitMix64 (Steele, Lea and Flood 2014) started at state `seed`
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double log2_ratio(double lhs, double rhs) {
  if (rhs == 0.0) return lhs > 0.0 ? INFINITY : (lhs == 0.0 ? 0.0 : -INFINITY);
  if (lhs == 0.0) return -INFINITY;
  if (std::isinf(lhs)) return INFINITY;
  return std::log2(lhs / rhs);
}

template <typename R>
struct Aug {
  R* a;
  int64_t ld, N, W;
  int nb, n;
  int64_t t0(int i) const { return (int64_t)i * nb; }
  int64_t t1(int i) const { return std::min<int64_t>((int64_t)(i + 1) * nb, N); }
  R* col(int64_t c) const { return a + c * ld; }
};

// ---------------------------------------------------------------- Householder kernels
// Reflector H = I - tau [1; v][1; v]^T with H [a0; x] = [beta; 0] (LAPACK dlarfg):
// beta = -sign(a0) sqrt(a0^2 + |x|^2), sign(0) = +1, tau = (beta - a0) / beta,
// v = x / (a0 - beta); tau = 0 (H = I) when x = 0.  x is overwritten by v, a0 by beta.
template <typename R>
R householder(R& a0, R* x, int64_t len) {
  R ss = 0;
  for (int64_t r = 0; r < len; ++r) ss += x[r] * x[r];
  if (ss == (R)0) {
    for (int64_t r = 0; r < len; ++r) x[r] = 0;
    return (R)0;
  }
  const double a = (double)a0;
  const double nrm = std::sqrt(a * a + (double)ss);
  const double beta = a >= 0.0 ? -nrm : nrm;
  const R tau = (R)((beta - a) / beta);
  const R den = (R)(a - beta);
  for (int64_t r = 0; r < len; ++r) x[r] = x[r] / den;
  a0 = (R)beta;
  return tau;
}

// Applies reflector (v of length len, tau t) to the pair (c1[j], c2[0..len)) of each of
// NC columns c1 + q*ld, c2 + q*ld:  w = c1[j] + v . c2;  c1[j] -= t w;  c2 -= t (v w).
// The columns are independent; each keeps its own sequential dot.
template <int NC, typename R>
void apply_reflector_n(const R* v, int64_t len, R t, R* c1, R* c2, int64_t ld) {
  R acc[NC];
  for (int q = 0; q < NC; ++q) acc[q] = 0;
  for (int64_t r = 0; r < len; ++r) {
    const R vr = v[r];
    for (int q = 0; q < NC; ++q) acc[q] += vr * c2[r + q * ld];
  }
  for (int q = 0; q < NC; ++q) {
    const R w = c1[q * ld] + acc[q];
    c1[q * ld] -= t * w;
    R* c = c2 + q * ld;
    for (int64_t r = 0; r < len; ++r) c[r] -= t * (v[r] * w);
  }
}

template <typename R>
void apply_reflector(const R* v, int64_t len, R t, R* c1, R* c2, int64_t ld, int nc) {
  switch (nc) {
    case 4: apply_reflector_n<4>(v, len, t, c1, c2, ld); break;
    case 3: apply_reflector_n<3>(v, len, t, c1, c2, ld); break;
    case 2: apply_reflector_n<2>(v, len, t, c1, c2, ld); break;
    default: apply_reflector_n<1>(v, len, t, c1, c2, ld); break;
  }
}

// GEQRT of the p x q tile at (r0, c0): R on and above the diagonal, reflector tails below.
template <typename R>
void geqrt(const Aug<R>& A, int64_t r0, int64_t p, int64_t c0, int64_t q, R* tau) {
  const int64_t kk = std::min(p, q);
  for (int64_t j = 0; j < kk; ++j) {
    R* cj = A.col(c0 + j) + r0;
    const R t = householder(cj[j], cj + j + 1, p - j - 1);
    tau[j] = t;
    if (t != (R)0)
      for (int64_t jj = j + 1; jj < q; jj += 4)
        apply_reflector(cj + j + 1, p - j - 1, t, A.col(c0 + jj) + r0 + j,
                        A.col(c0 + jj) + r0 + j + 1, A.ld, (int)std::min<int64_t>(4, q - jj));
  }
}

// TSQRT: QR of [R; V] with R (rows e0..) upper triangular and V (p rows at a0) full.
template <typename R>
void tsqrt(const Aug<R>& A, int64_t e0, int64_t a0, int64_t p, int64_t c0, int64_t q, R* tau) {
  for (int64_t j = 0; j < q; ++j) {
    R* cj = A.col(c0 + j);
    const R t = householder(cj[e0 + j], cj + a0, p);
    tau[j] = t;
    if (t != (R)0)
      for (int64_t jj = j + 1; jj < q; jj += 4) {
        R* cc = A.col(c0 + jj);
        apply_reflector(cj + a0, p, t, cc + e0 + j, cc + a0, A.ld, (int)std::min<int64_t>(4, q - jj));
      }
  }
}

// TTQRT: QR of [R1; R2], both upper triangular (R2: p rows, may be trapezoidal);
// reflector j involves rows 0..min(j+1, p)-1 of R2 only.
template <typename R>
void ttqrt(const Aug<R>& A, int64_t e0, int64_t a0, int64_t p, int64_t c0, int64_t q, R* tau) {
  for (int64_t j = 0; j < q; ++j) {
    const int64_t rows = std::min<int64_t>(j + 1, p);
    R* cj = A.col(c0 + j);
    const R t = householder(cj[e0 + j], cj + a0, rows);
    tau[j] = t;
    if (t != (R)0)
      for (int64_t jj = j + 1; jj < q; jj += 4) {
        R* cc = A.col(c0 + jj);
        apply_reflector(cj + a0, rows, t, cc + e0 + j, cc + a0, A.ld,
                        (int)std::min<int64_t>(4, q - jj));
      }
  }
}

// Q^T of one elimination-list operation applied to columns [lo, hi) of the trailing
// matrix (UNMQR for a GEQRT tile, TSMQR / TTMQR for a TS / TT pair).
template <typename R>
void apply_op(const Aug<R>& A, const Op& op, int64_t c0, int64_t q, const R* tau, int64_t lo,
              int64_t hi) {
  const int64_t a0 = A.t0(op.i), p = A.t1(op.i) - a0, e0 = A.t0(op.e);
  for (int64_t c = lo; c < hi; c += 4) {
    const int nc = (int)std::min<int64_t>(4, hi - c);
    R* base = A.col(c);
    if (op.kind == OP_GEQRT) {
      const int64_t kk = std::min(p, q);
      for (int64_t j = 0; j < kk; ++j) {
        if (tau[j] == (R)0) continue;
        apply_reflector(A.col(c0 + j) + a0 + j + 1, p - j - 1, tau[j], base + a0 + j,
                        base + a0 + j + 1, A.ld, nc);
      }
    } else {
      for (int64_t j = 0; j < q; ++j) {
        if (tau[j] == (R)0) continue;
        const int64_t len = op.kind == OP_TS ? p : std::min<int64_t>(j + 1, p);
        apply_reflector(A.col(c0 + j) + a0, len, tau[j], base + e0 + j, base + a0, A.ld, nc);
      }
    }
  }
}

// ---------------------------------------------------------------- LU kernels (Alg. 2)
// GETRF of the p x p column-major scratch tile T (leading dimension p): P T = L U with
// partial pivoting (first row of maximal |a|).  piv[r] = row exchanged with r at step r.
// Returns the first r whose pivot is exactly zero (that column is left unscaled), or -1.
template <typename R>
int getrf(R* T, int p, int* piv) {
  int zero_row = -1;
  for (int r = 0; r < p; ++r) {
    int s = r;
    R best = std::fabs(T[r + (int64_t)r * p]);
    for (int i = r + 1; i < p; ++i)
      if (std::fabs(T[i + (int64_t)r * p]) > best) {
        best = std::fabs(T[i + (int64_t)r * p]);
        s = i;
      }
    piv[r] = s;
    if (s != r)
      for (int c = 0; c < p; ++c) std::swap(T[r + (int64_t)c * p], T[s + (int64_t)c * p]);
    const R d = T[r + (int64_t)r * p];
    if (d == (R)0) {
      if (zero_row < 0) zero_row = r;
      continue;
    }
    for (int i = r + 1; i < p; ++i) T[i + (int64_t)r * p] = T[i + (int64_t)r * p] / d;
    for (int c = r + 1; c < p; ++c) {
      const R u = T[r + (int64_t)c * p];
      for (int i = r + 1; i < p; ++i) T[i + (int64_t)c * p] -= T[i + (int64_t)r * p] * u;
    }
  }
  return zero_row;
}

// One column x (length p) <- L^-1 P x, L unit lower triangular below the diagonal of LU.
template <typename R, typename S>
void swp_lower_col(const S* LU, int64_t ldlu, int p, const int* piv, R* x) {
  for (int r = 0; r < p; ++r)
    if (piv[r] != r) std::swap(x[r], x[piv[r]]);
  for (int r = 0; r < p; ++r) {
    const R xr = x[r];
    const S* l = LU + (int64_t)r * ldlu;
    for (int i = r + 1; i < p; ++i) x[i] -= (R)l[i] * xr;
  }
}

// ||A_kk^-1||_1 from the GETRF factors: X = U^-1 L^-1 P column by column, max column
// absolute sum, all in float64 (the factors are widened first).
template <typename R>
double inv_norm1(const R* LU, int p, const int* piv) {
  std::vector<double> L((size_t)p * p), x(p);
  for (size_t q = 0; q < L.size(); ++q) L[q] = (double)LU[q];
  double best = 0.0;
  for (int c = 0; c < p; ++c) {
    std::fill(x.begin(), x.end(), 0.0);
    x[c] = 1.0;
    swp_lower_col<double, double>(L.data(), p, p, piv, x.data());
    for (int r = p - 1; r >= 0; --r) {
      x[r] = x[r] / L[r + (size_t)r * p];
      const double xr = x[r];
      for (int i = 0; i < r; ++i) x[i] -= L[i + (size_t)r * p] * xr;
    }
    double s = 0.0;
    for (int r = 0; r < p; ++r) s += std::fabs(x[r]);
    best = std::max(best, s);
  }
  return best;
}

struct StepDecision {
  int dec;
  double margin, lhs, rhs;
};

// Robustness test of Sec. III: Eq. 2 (Max), Eq. 3 (Sum), Eq. 4 (MUMPS), the forced
// limits and the random choice of Sec. V-B.  Margin = log2(lhs / rhs) (min over j for
// MUMPS).
template <typename R>
StepDecision decide(int criterion, double alpha, const R* LU, int p, const int* piv, int zero_row,
                    const std::vector<double>& below, const std::vector<double>& local,
                    const std::vector<double>& away, int mumps_mode, uint64_t seed, int k) {
  const double nan = NAN;
  if (criterion == CRIT_FORCE_LU) return {DEC_LU, INFINITY, nan, nan};
  if (criterion == CRIT_FORCE_QR || alpha == 0.0) return {DEC_QR, -INFINITY, nan, nan};
  if (zero_row >= 0) return {DEC_QR, -INFINITY, 0.0, nan};
  if (criterion == CRIT_RANDOM) {
    const double lhs = alpha / 100.0;
    const double rhs = (double)(splitmix64_at(seed, (uint64_t)k) >> 11) * std::ldexp(1.0, -53);
    return {rhs < lhs ? DEC_LU : DEC_QR, log2_ratio(lhs, rhs), lhs, rhs};
  }
  if (criterion == CRIT_MAX || criterion == CRIT_SUM) {
    const double inv = inv_norm1(LU, p, piv);
    const double lhs = alpha * (1.0 / inv);
    double rhs = 0.0;
    if (criterion == CRIT_MAX) {
      for (double v : below) rhs = std::max(rhs, v);
    } else {
      for (double v : below) rhs = rhs + v;
    }
    return {lhs >= rhs ? DEC_LU : DEC_QR, log2_ratio(lhs, rhs), lhs, rhs};
  }
  // MUMPS (Eq. 4): for every column j, alpha * |pivot(j)| >= estimate_max(j)
  bool ok = true;
  double margin = INFINITY, gprod = 1.0;
  for (int j = 0; j < p; ++j) {
    const double pj = std::fabs((double)LU[j + (int64_t)j * p]);
    const double lj = local[j];
    if (lj == 0.0) return {DEC_QR, -INFINITY, nan, nan};
    double est;
    if (mumps_mode == 0) {
      est = away[j] * (pj / lj);
    } else {
      est = away[j] * gprod;
      gprod = gprod * (pj / lj);
    }
    const double lhs = alpha * pj;
    if (!(lhs >= est)) ok = false;
    margin = std::min(margin, log2_ratio(lhs, est));
  }
  return {ok ? DEC_LU : DEC_QR, margin, nan, nan};
}

// LU step (Alg. 2, variant A1) on the augmented matrix.
template <typename R>
void lu_step(const Aug<R>& A, int k, const std::vector<R>& LU, const int* piv, int threads) {
  const int64_t r0 = A.t0(k), r1 = A.t1(k), p = r1 - r0, N = A.N, W = A.W;
  for (int64_t c = 0; c < p; ++c)                                   // Factor: commit
    std::memcpy(A.col(r0 + c) + r0, LU.data() + c * p, sizeof(R) * p);
  // Eliminate: A_ik <- A_ik U^-1 (rows are independent)
  parallel_range(r1, N, threads, 64, [&](int64_t lo, int64_t hi) {
    for (int64_t c = 0; c < p; ++c) {
      R* xc = A.col(r0 + c);
      const R d = LU[c + c * p];
      for (int64_t r = lo; r < hi; ++r) xc[r] = xc[r] / d;
      for (int64_t cc = c + 1; cc < p; ++cc) {
        const R u = LU[c + cc * p];
        R* xcc = A.col(r0 + cc);
        for (int64_t r = lo; r < hi; ++r) xcc[r] -= xc[r] * u;
      }
    }
  });
  // Apply (L^-1 P on A_kj and b_k), then Update A_ij -= A_ik A_kj, column by column
  parallel_range(r1, W, threads, 4, [&](int64_t lo, int64_t hi) {
    for (int64_t c = lo; c < hi; ++c) swp_lower_col<R, R>(LU.data(), p, (int)p, piv, A.col(c) + r0);
    std::vector<R> acc(A.nb);
    for (int i = k + 1; i < A.n; ++i) {
      const int64_t a0 = A.t0(i), pa = A.t1(i) - a0;
      for (int64_t c = lo; c < hi; ++c) {
        R* cc = A.col(c);
        std::fill(acc.begin(), acc.begin() + pa, (R)0);
        for (int64_t q = 0; q < p; ++q) {
          const R b = cc[r0 + q];
          const R* a = A.col(r0 + q) + a0;
          for (int64_t r = 0; r < pa; ++r) acc[r] += a[r] * b;
        }
        for (int64_t r = 0; r < pa; ++r) cc[a0 + r] -= acc[r];
      }
    }
  });
}

// QR step (Alg. 3 with the kernels of Alg. 4) along the elimination list of the tree.
// The panel is factored op by op (consecutive ops on disjoint tiles, e.g. the GEQRTs or
// one TT level of the binary tree, commute exactly and run side by side); then every
// trailing column receives the ops' Q^T in list order.
template <typename R>
void qr_step(const Aug<R>& A, int k, const std::vector<Op>& ops, int threads) {
  const int64_t c0 = A.t0(k), q = A.t1(k) - c0;
  std::vector<R> tau(ops.size() * (size_t)q, (R)0);
  size_t o = 0;
  while (o < ops.size()) {
    size_t e = o;
    std::vector<char> used(A.n, 0);
    while (e < ops.size() && !used[ops[e].i] && !used[ops[e].e]) {
      used[ops[e].i] = used[ops[e].e] = 1;
      ++e;
    }
    parallel_range((int64_t)o, (int64_t)e, threads, 1, [&](int64_t lo, int64_t hi) {
      for (int64_t x = lo; x < hi; ++x) {
        const Op& op = ops[x];
        const int64_t a0 = A.t0(op.i), p = A.t1(op.i) - a0, e0 = A.t0(op.e);
        R* t = tau.data() + x * q;
        if (op.kind == OP_GEQRT) geqrt(A, a0, p, c0, q, t);
        else if (op.kind == OP_TS) tsqrt(A, e0, a0, p, c0, q, t);
        else ttqrt(A, e0, a0, p, c0, q, t);
      }
    });
    o = e;
  }
  parallel_range(A.t1(k), A.W, threads, 4, [&](int64_t lo, int64_t hi) {
    for (size_t x = 0; x < ops.size(); ++x) apply_op(A, ops[x], c0, q, tau.data() + x * q, lo, hi);
  });
}

// Alg. 1 on the augmented matrix [A | b] (column-major, leading dimension ld >= N, W
// columns).  Runs steps 0 .. min(n, max_steps) - 1; dec / margin / lhs / rhs get one entry
// per step (DEC_NONE / NaN past the last step run).
template <typename R>
int factor(R* aug, int64_t ld, int64_t N, int64_t W, int nb, int criterion, double alpha, int tree,
           int group, int tree_small, int tree_switch, int mumps_mode, const uint8_t* forced, const int* inject, int n_inject,
           uint64_t seed, int threads, int max_steps, uint8_t* dec, double* margin, double* lhs,
           double* rhs, int* where, int* steps_done) {
  if (!aug || N < 1 || nb < 1 || ld < N || W < N || criterion < CRIT_MAX ||
      criterion > CRIT_RANDOM || !(alpha >= 0.0) || tree < 0 || tree > 2 || tree_small < 0 ||
      tree_small > 2 || tree_switch < 0)
    return E_INVALID;
  const int n = (int)((N + nb - 1) / nb);
  Aug<R> A{aug, ld, N, W, nb, n};
  std::vector<char> injected(n, 0);
  for (int q = 0; q < n_inject; ++q)
    if (inject[q] >= 0 && inject[q] < n) injected[inject[q]] = 1;
  for (int k = 0; k < n; ++k) {
    dec[k] = DEC_NONE;
    margin[k] = lhs[k] = rhs[k] = NAN;
  }
  where[0] = where[1] = -1;
  *steps_done = 0;
  const int kend = max_steps >= 0 ? std::min(n, max_steps) : n;
  const R scale = (R)std::ldexp(1.0, -27);
  for (int k = 0; k < kend; ++k) {
    const int64_t r0 = A.t0(k), r1 = A.t1(k), p = r1 - r0;
    if (injected[k])   // run-time injection: tile row k of [A^(k) | b^(k)] times 2^-27
      parallel_range(r0, W, threads, 4, [&](int64_t lo, int64_t hi) {
        for (int64_t c = lo; c < hi; ++c)
          for (int64_t r = r0; r < r1; ++r) A.col(c)[r] *= scale;
      });
    // criterion inputs on the panel A^(k)_{ik}, i >= k (Sec. III-D), in float64
    std::vector<double> norms(n - k), local(p, 0.0), away(p, 0.0);
    for (int i = k; i < n; ++i) {
      const int64_t a0 = A.t0(i), a1 = A.t1(i);
      double best = 0.0;
      for (int64_t c = 0; c < p; ++c) {
        const R* x = A.col(r0 + c);
        double s = 0.0;
        for (int64_t r = a0; r < a1; ++r) {
          if (!std::isfinite((double)x[r])) {
            where[0] = k;
            return E_NONFINITE;
          }
          s += std::fabs((double)x[r]);
          if (i == k) local[c] = std::max(local[c], std::fabs((double)x[r]));
          else away[c] = std::max(away[c], std::fabs((double)x[r]));
        }
        best = std::max(best, s);
      }
      norms[i - k] = best;
    }
    // Factor: GETRF of a scratch copy of the diagonal tile (Alg. 1)
    std::vector<R> LU((size_t)p * p);
    for (int64_t c = 0; c < p; ++c)
      std::memcpy(LU.data() + c * p, A.col(r0 + c) + r0, sizeof(R) * p);
    std::vector<int> piv(p);
    const int zero_row = getrf(LU.data(), (int)p, piv.data());
    // Check (Alg. 1)
    StepDecision sd;
    if (forced) {
      const int d = forced[k];
      sd = {d, d == DEC_LU ? INFINITY : -INFINITY, NAN, NAN};
    } else {
      std::vector<double> below(norms.begin() + 1, norms.end());
      sd = decide(criterion, alpha, LU.data(), (int)p, piv.data(), zero_row, below, local, away,
                  mumps_mode, seed, k);
    }
    if (sd.dec == DEC_LU && zero_row >= 0) {
      where[0] = k;
      where[1] = (int)(r0 + zero_row);
      return E_SINGULAR;
    }
    dec[k] = (uint8_t)sd.dec;
    margin[k] = sd.margin;
    lhs[k] = sd.lhs;
    rhs[k] = sd.rhs;
    if (sd.dec == DEC_LU) lu_step(A, k, LU, piv.data(), threads);
    else   // the tree of this step: tree_small below tree_switch sub-diagonal tiles
      qr_step(A, k,
              elimination_ops(k, n, (tree_switch > 0 && n - 1 - k < tree_switch) ? tree_small : tree,
                              group),
              threads);
    *steps_done = k + 1;
  }
  return OK;
}

// Back substitution U x = c (U the upper triangle of the first N columns, c the columns
// N .. N+nrhs-1 of the factored augmented matrix), in float64.  Bottom row first; an
// exact zero on the diagonal returns E_SINGULAR with where[1] = its row.
template <typename R>
int backsolve(const R* aug, int64_t ld, int64_t N, int64_t nrhs, double* x, int64_t ldx,
              int* where) {
  for (int64_t j = 0; j < nrhs; ++j) {
    double* xj = x + j * ldx;
    const R* c = aug + (N + j) * ld;
    for (int64_t r = 0; r < N; ++r) xj[r] = (double)c[r];
    for (int64_t r = N - 1; r >= 0; --r) {
      const R* u = aug + r * ld;
      if (u[r] == (R)0) {
        where[1] = (int)r;
        return E_SINGULAR;
      }
      xj[r] = xj[r] / (double)u[r];
      const double xr = xj[r];
      for (int64_t i = 0; i < r; ++i) xj[i] -= (double)u[i] * xr;
    }
  }
  return OK;
}

}  // namespace

extern "C" {

int luqr_oracle_mt_factor_f64(double* aug, int64_t ld, int64_t N, int64_t W, int nb, int criterion,
                              double alpha, int tree, int group, int tree_small,
                              int tree_switch, int mumps_mode,
                              const uint8_t* forced, const int* inject, int n_inject, uint64_t seed,
                              int threads, int max_steps, uint8_t* dec, double* margin, double* lhs,
                              double* rhs, int* where, int* steps_done) {
  return factor<double>(aug, ld, N, W, nb, criterion, alpha, tree, group, tree_small,
                        tree_switch, mumps_mode, forced,
                        inject, n_inject, seed, threads, max_steps, dec, margin, lhs, rhs, where,
                        steps_done);
}

int luqr_oracle_mt_factor_f32(float* aug, int64_t ld, int64_t N, int64_t W, int nb, int criterion,
                              double alpha, int tree, int group, int tree_small,
                              int tree_switch, int mumps_mode,
                              const uint8_t* forced, const int* inject, int n_inject, uint64_t seed,
                              int threads, int max_steps, uint8_t* dec, double* margin, double* lhs,
                              double* rhs, int* where, int* steps_done) {
  return factor<float>(aug, ld, N, W, nb, criterion, alpha, tree, group, tree_small,
                        tree_switch, mumps_mode, forced,
                       inject, n_inject, seed, threads, max_steps, dec, margin, lhs, rhs, where,
                       steps_done);
}

int luqr_oracle_mt_backsolve_f64(const double* aug, int64_t ld, int64_t N, int64_t nrhs, double* x,
                                 int64_t ldx, int* where) {
  return backsolve<double>(aug, ld, N, nrhs, x, ldx, where);
}

int luqr_oracle_mt_backsolve_f32(const float* aug, int64_t ld, int64_t N, int64_t nrhs, double* x,
                                 int64_t ldx, int* where) {
  return backsolve<float>(aug, ld, N, nrhs, x, ldx, where);
}

int luqr_oracle_mt_hardware_threads(void) {
  const unsigned t = std::thread::hardware_concurrency();
  return t ? (int)t : 1;
}

}  // extern "C"
