// Batched hybrid LU-QR solves: one persistent launch factors and solves many independent
// systems of uneven order.  Each CTA repeatedly claims the next system from a queue
// ordered largest first (longest-processing-time order), copies it into its own padded
// scratch slot, runs Alg. 1 with in-kernel decisions (Eq. 2-4), the LU step of Alg. 2 and
// the QR step of Alg. 3 / Alg. 4(a) (flat TS tree), back-substitutes the augmented right-
// hand side (Sec. II-D) and, in FP32 mode, refines the solution with FP64 residuals until
// the normwise backward error reaches the tolerance.  Tiles are nb x nb with nb in
// {32, 64} chosen per system; every tile operation works on shared-memory copies.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/luqr.h"
#include "internal.cuh"

namespace luqr {
namespace {

constexpr int BT = 256;          // threads per CTA
constexpr int NBMAX = 64;
constexpr int LDS = NBMAX + 1;   // shared-memory tile leading dimension
constexpr int TILE = NBMAX * LDS;

struct BatchArgs {
  const double* const* A;   // per system, column-major N x N (lda = N), read only
  double* const* b;         // per system, length N; receives x
  const double* const* b0;  // per system, the batch's own copy of the right-hand side
  const int* N;             // orders
  const int* nbs;           // tile size per system (32 or 64)
  const int* order;         // processing order (largest first)
  int count;
  int criterion, mumps_mode;
  double alpha;
  int fp32;                 // 0: FP64 factorization; 1: FP32 factorization + FP64 refinement
  double tol;
  int max_iter;
  void* slots;              // per-CTA scratch
  size_t slot_bytes;
  int64_t ldw;              // padded leading dimension of the workspace (max Npad)
  int nmax;                 // max tiles per system
  uint8_t* dec;             // count x nmax decisions (LUQR_DEC_*), 255 = unused
  int* iters;               // refinement iterations per system
  double* eta;              // final backward error per system
  int* status;              // per system status
  int* counter;             // work queue head
};

// ------------------------------------------------------------------ small tile helpers
template <typename T>
__device__ void tload(T* S, const T* G, int64_t ldg, int nb) {
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int r = idx % nb, c = idx / nb;
    S[r + c * LDS] = G[r + (int64_t)c * ldg];
  }
}
template <typename T>
__device__ void tstore(const T* S, T* G, int64_t ldg, int nb) {
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int r = idx % nb, c = idx / nb;
    G[r + (int64_t)c * ldg] = S[r + c * LDS];
  }
}

// out (op)= opA(A) opB(B) on nb x nb shared tiles.  opA: 0 = A, 1 = A^T.  maskA: 0 none,
// 1 unit lower (A's own row > col kept, 1 on the diagonal), 2 upper (row <= col kept).
// mode: 0 out = P, 1 out = out - P, 2 out = init + P (init a shared tile).
template <typename T>
__device__ __forceinline__ T fetchA(const T* A, int transA, int maskA, int r, int q) {
  const int pr = transA ? q : r, pc = transA ? r : q;
  if (maskA == 1) {
    if (pr == pc) return (T)1;
    if (pr < pc) return (T)0;
  } else if (maskA == 2) {
    if (pr > pc) return (T)0;
  }
  return A[pr + pc * LDS];
}

template <typename T>
__device__ void tgemm(T* out, const T* A, int transA, int maskA, const T* B, int mode,
                      const T* init, int nb) {
  const int bs = nb / 16;                 // 4 (nb = 64) or 2 (nb = 32) outputs per side
  const int nblk = 16 * 16;
  for (int blk = threadIdx.x; blk < nblk; blk += BT) {
    const int r0 = (blk % 16) * bs, c0 = (blk / 16) * bs;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
    for (int q = 0; q < nb; ++q) {
      T a[4], bq[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = i < bs ? fetchA(A, transA, maskA, r0 + i, q) : (T)0;
#pragma unroll
      for (int j = 0; j < 4; ++j) bq[j] = j < bs ? B[q + (c0 + j) * LDS] : (T)0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bq[j];
    }
    for (int i = 0; i < bs; ++i)
      for (int j = 0; j < bs; ++j) {
        T* o = &out[(r0 + i) + (c0 + j) * LDS];
        if (mode == 0) *o = acc[i][j];
        else if (mode == 1) *o -= acc[i][j];
        else *o = init[(r0 + i) + (c0 + j) * LDS] + acc[i][j];
      }
  }
  __syncthreads();
}

// G (global, ld) -= A B with A, B shared tiles (LU trailing update of one tile).
template <typename T>
__device__ void tgemm_global_sub(T* G, int64_t ldg, const T* A, const T* B, int nb) {
  const int bs = nb / 16;
  for (int blk = threadIdx.x; blk < 256; blk += BT) {
    const int r0 = (blk % 16) * bs, c0 = (blk / 16) * bs;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (T)0;
    for (int q = 0; q < nb; ++q) {
      T a[4], bq[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = i < bs ? A[(r0 + i) + q * LDS] : (T)0;
#pragma unroll
      for (int j = 0; j < 4; ++j) bq[j] = j < bs ? B[q + (c0 + j) * LDS] : (T)0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bq[j];
    }
    for (int j = 0; j < bs; ++j)
      for (int i = 0; i < bs; ++i) G[(r0 + i) + (int64_t)(c0 + j) * ldg] -= acc[i][j];
  }
  __syncthreads();
}

// P S = L U of a shared tile (pivot: first row of maximal |a|); returns the first zero
// pivot row or -1.  piv in shared memory.
template <typename T>
__device__ int tgetrf(T* S, int* piv, int nb, int* s_int) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_int[1] = -1;
  __syncthreads();
  for (int r = 0; r < nb; ++r) {
    if (warp == 0) {
      double bv = -1.0;
      int bi = nb;
      for (int rr = r + lane; rr < nb; rr += 32) {
        const double v = fabs((double)S[rr + r * LDS]);
        if (v > bv) { bv = v; bi = rr; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (bi >= nb) bi = r;
      if (lane == 0) { piv[r] = bi; s_int[0] = bi; }
    }
    __syncthreads();
    const int p = s_int[0];
    if (p != r)
      for (int c = tid; c < nb; c += BT) {
        const T t = S[r + c * LDS];
        S[r + c * LDS] = S[p + c * LDS];
        S[p + c * LDS] = t;
      }
    __syncthreads();
    const T d = S[r + r * LDS];
    if (d != (T)0) {
      for (int rr = r + 1 + tid; rr < nb; rr += BT) S[rr + r * LDS] = S[rr + r * LDS] / d;
      __syncthreads();
      const int m = nb - r - 1;
      for (int idx = tid; idx < m * m; idx += BT) {
        const int rr = r + 1 + idx % m, cc = r + 1 + idx / m;
        S[rr + cc * LDS] -= S[rr + r * LDS] * S[r + cc * LDS];
      }
    } else if (tid == 0 && s_int[1] < 0) {
      s_int[1] = r;
    }
    __syncthreads();
  }
  return s_int[1];
}

// ||A_kk^-1||_1 from the shared LU factors (FP64); vec: 8 warps x nb doubles scratch.
template <typename T>
__device__ double tinvnorm(const T* S, const int* piv, int nb, double* vec, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double best = 0.0;
  double* y = vec + warp * NBMAX;
  for (int c = warp; c < nb; c += BT / 32) {
    int pos = c;
    for (int r = 0; r < nb; ++r) {
      const int p = piv[r];
      if (pos == r) pos = p;
      else if (pos == p) pos = r;
    }
    for (int row = lane; row < nb; row += 32) y[row] = (row == pos) ? 1.0 : 0.0;
    __syncwarp();
    for (int r = pos; r < nb - 1; ++r) {
      const double yr = y[r];
      if (yr != 0.0)
        for (int row = r + 1 + lane; row < nb; row += 32) y[row] -= (double)S[row + r * LDS] * yr;
      __syncwarp();
    }
    for (int r = nb - 1; r >= 0; --r) {
      if (lane == 0) y[r] = y[r] / (double)S[r + r * LDS];
      __syncwarp();
      const double xr = y[r];
      if (xr != 0.0)
        for (int row = lane; row < r; row += 32) y[row] -= (double)S[row + r * LDS] * xr;
      __syncwarp();
    }
    double sum = 0.0;
    for (int row = lane; row < nb; row += 32) sum += fabs(y[row]);
    sum = warp_sum_d(sum);
    best = fmax(best, sum);
    __syncwarp();
  }
  if (lane == 0) red[warp] = best;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < BT / 32; ++w) m = fmax(m, red[w]);
  __syncthreads();
  return m;
}

// Householder QR of a shared tile (GEQRT, dlarfg convention), full compact-WY T (nb x nb)
// in Tm; tau in tau_s.  Also serves TSQRT when Rtop != nullptr: then the reflector of
// column j is [e_j; S[:, j]] with R's row j on top.
template <typename T>
__device__ void thouse(T* S, T* Rtop, T* Tm, T* tau_s, T* G, int nb) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool pair = Rtop != nullptr;
  for (int j = 0; j < nb; ++j) {
    const int r0 = pair ? 0 : j + 1;
    if (warp == 0) {
      T part = (T)0;
      for (int r = r0 + lane; r < nb; r += 32) {
        const T v = S[r + j * LDS];
        part += v * v;
      }
      const T ss = warp_sum<T>(part);
      const T a0 = pair ? Rtop[j + j * LDS] : S[j + j * LDS];
      T beta, tau, inv;
      if (ss == (T)0) {
        beta = a0; tau = (T)0; inv = (T)0;
      } else {
        const T nrm = sqrt(a0 * a0 + ss);
        beta = (a0 >= (T)0) ? -nrm : nrm;
        tau = (beta - a0) / beta;
        inv = (T)1 / (a0 - beta);
      }
      for (int r = r0 + lane; r < nb; r += 32) S[r + j * LDS] = S[r + j * LDS] * inv;
      __syncwarp();
      if (lane == 0) {
        if (pair) Rtop[j + j * LDS] = beta; else S[j + j * LDS] = beta;
        tau_s[j] = tau;
      }
    }
    __syncthreads();
    const T tau = tau_s[j];
    if (tau != (T)0) {
      for (int c = j + 1 + warp; c < nb; c += BT / 32) {
        T s = (T)0;
        for (int r = r0 + lane; r < nb; r += 32) s += S[r + j * LDS] * S[r + c * LDS];
        s = warp_sum<T>(s);
        const T top = pair ? Rtop[j + c * LDS] : S[j + c * LDS];
        const T wc = top + s;
        __syncwarp();
        if (lane == 0) {
          if (pair) Rtop[j + c * LDS] -= tau * wc; else S[j + c * LDS] -= tau * wc;
        }
        for (int r = r0 + lane; r < nb; r += 32) S[r + c * LDS] -= tau * S[r + j * LDS] * wc;
      }
    }
    __syncthreads();
  }
  // G = V^T V (strictly upper part), then T by the forward recurrence
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int bcol = idx % nb, j = idx / nb;
    if (bcol >= j) continue;
    T sacc = pair ? (T)0 : S[j + bcol * LDS];   // single: v_j has its unit at row j
    for (int r = pair ? 0 : j + 1; r < nb; ++r) sacc += S[r + bcol * LDS] * S[r + j * LDS];
    G[bcol + j * LDS] = sacc;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int r = idx % nb, c = idx / nb;
    Tm[r + c * LDS] = (T)0;
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const T tj = tau_s[j];
    T val = (T)0;
    if ((int)threadIdx.x < j) {
      T s = (T)0;
      for (int q = threadIdx.x; q < j; ++q) s += Tm[threadIdx.x + q * LDS] * G[q + j * LDS];
      val = -tj * s;
    }
    __syncthreads();
    if ((int)threadIdx.x < j) Tm[threadIdx.x + j * LDS] = val;
    else if ((int)threadIdx.x == j) Tm[j + j * LDS] = tj;
    __syncthreads();
  }
}

// Q^T C for a single tile's reflectors: W = V^T C; W = T^T W; C -= V W (V unit lower).
template <typename T>
__device__ void tunmqr(const T* V, const T* Tm, T* C, T* W, T* W2, int nb) {
  tgemm<T>(W, V, 1, 1, C, 0, nullptr, nb);
  tgemm<T>(W2, Tm, 1, 0, W, 0, nullptr, nb);
  tgemm<T>(C, V, 0, 1, W2, 1, nullptr, nb);
}

// [C1; C2] <- Q^T [C1; C2] for a TS pair: W = C1 + V2^T C2; W2 = T^T W; C1 -= W2; C2 -= V2 W2.
template <typename T>
__device__ void ttsmqr(const T* V2, const T* Tm, T* C1, T* C2, T* W, T* W2, int nb) {
  tgemm<T>(W, V2, 1, 0, C2, 2, C1, nb);
  tgemm<T>(W2, Tm, 1, 0, W, 0, nullptr, nb);
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int r = idx % nb, c = idx / nb;
    C1[r + c * LDS] -= W2[r + c * LDS];
  }
  __syncthreads();
  tgemm<T>(C2, V2, 0, 0, W2, 1, nullptr, nb);
}

// Vector versions for the second pass (one right-hand side, shared-memory segments).
template <typename T>
__device__ void vunmqr(const T* V, const T* Tm, T* y, T* w, T* w2, int nb) {
  for (int j = threadIdx.x; j < nb; j += BT) {
    T s = y[j];
    for (int r = j + 1; r < nb; ++r) s += V[r + j * LDS] * y[r];
    w[j] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nb; j += BT) {
    T s = (T)0;
    for (int a = 0; a <= j; ++a) s += Tm[a + j * LDS] * w[a];
    w2[j] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += BT) {
    T s = w2[r];
    for (int j = 0; j < r; ++j) s += V[r + j * LDS] * w2[j];
    y[r] -= s;
  }
  __syncthreads();
}

template <typename T>
__device__ void vtsmqr(const T* V2, const T* Tm, T* y1, T* y2, T* w, T* w2, int nb) {
  for (int j = threadIdx.x; j < nb; j += BT) {
    T s = y1[j];
    for (int r = 0; r < nb; ++r) s += V2[r + j * LDS] * y2[r];
    w[j] = s;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nb; j += BT) {
    T s = (T)0;
    for (int a = 0; a <= j; ++a) s += Tm[a + j * LDS] * w[a];
    w2[j] = s;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < nb; r += BT) {
    T s = (T)0;
    for (int j = 0; j < nb; ++j) s += V2[r + j * LDS] * w2[j];
    y2[r] -= s;
    y1[r] -= w2[r];
  }
  __syncthreads();
}

template <typename T>
struct Slot {
  T* W;          // Npad x (Npad + 1) tiles + augmented column
  T* Tst;        // per step, per tile: nb x LDS compact-WY T (flat tree: tile k is GEQRT, i>k TS)
  int* piv;      // per step: nb pivots
  double* x;     // FP64 solution (refinement)
  double* r;     // FP64 residual
  T* y;          // factorization-precision right-hand side (Npad)
};

template <typename T>
__device__ Slot<T> slot_of(const BatchArgs& a, int nmax) {
  unsigned char* base = static_cast<unsigned char*>(a.slots) + (size_t)blockIdx.x * a.slot_bytes;
  Slot<T> s;
  const size_t ldw = (size_t)a.ldw;
  s.W = reinterpret_cast<T*>(base);
  size_t off = ldw * (ldw + 1) * sizeof(T);
  off = (off + 255) & ~(size_t)255;
  s.Tst = reinterpret_cast<T*>(base + off);
  off += (size_t)nmax * nmax * TILE * sizeof(T);
  off = (off + 255) & ~(size_t)255;
  s.piv = reinterpret_cast<int*>(base + off);
  off += (size_t)nmax * NBMAX * sizeof(int);
  off = (off + 255) & ~(size_t)255;
  s.x = reinterpret_cast<double*>(base + off);
  off += ldw * sizeof(double);
  s.r = reinterpret_cast<double*>(base + off);
  off += ldw * sizeof(double);
  off = (off + 255) & ~(size_t)255;
  s.y = reinterpret_cast<T*>(base + off);
  return s;
}

// Replays the stored steps on y (Npad, factorization precision) and back-substitutes.
template <typename T>
__device__ void replay_solve(const BatchArgs& a, const Slot<T>& sl, const uint8_t* dec, int n,
                             int nb, T* S0, T* S1, T* Tm, T* vv) {
  const int64_t ldw = a.ldw;
  T* w = vv;
  T* w2 = vv + NBMAX;
  T* ytile = vv + 2 * NBMAX;
  T* ytile2 = vv + 3 * NBMAX;
  for (int k = 0; k < n; ++k) {
    const int64_t r0 = (int64_t)k * nb;
    tload<T>(S0, sl.W + r0 + r0 * ldw, ldw, nb);
    for (int i = threadIdx.x; i < nb; i += BT) ytile[i] = sl.y[r0 + i];
    __syncthreads();
    if (dec[k] == DEC_LU) {
      if (threadIdx.x == 0) {
        const int* pv = sl.piv + k * NBMAX;
        for (int r = 0; r < nb; ++r) {
          const int p = pv[r];
          if (p != r) { const T t = ytile[r]; ytile[r] = ytile[p]; ytile[p] = t; }
        }
        for (int r = 0; r < nb; ++r)
          for (int q = r + 1; q < nb; ++q) ytile[q] -= S0[q + r * LDS] * ytile[r];
      }
      __syncthreads();
      for (int i = k + 1; i < n; ++i) {
        for (int rr = threadIdx.x; rr < nb; rr += BT) {
          T s = (T)0;
          for (int q = 0; q < nb; ++q) s += sl.W[(int64_t)i * nb + rr + (r0 + q) * ldw] * ytile[q];
          sl.y[(int64_t)i * nb + rr] -= s;
        }
      }
    } else {
      const T* Tk = sl.Tst + ((size_t)k * a.nmax + k) * TILE;
      for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
        const int rr = idx % nb, c = idx / nb;
        Tm[rr + c * LDS] = Tk[rr + c * LDS];
      }
      __syncthreads();
      vunmqr<T>(S0, Tm, ytile, w, w2, nb);
      for (int i = k + 1; i < n; ++i) {
        tload<T>(S1, sl.W + (int64_t)i * nb + r0 * ldw, ldw, nb);
        const T* Ti = sl.Tst + ((size_t)k * a.nmax + i) * TILE;
        for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
          const int rr = idx % nb, c = idx / nb;
          Tm[rr + c * LDS] = Ti[rr + c * LDS];
        }
        for (int q = threadIdx.x; q < nb; q += BT) ytile2[q] = sl.y[(int64_t)i * nb + q];
        __syncthreads();
        vtsmqr<T>(S1, Tm, ytile, ytile2, w, w2, nb);
        for (int q = threadIdx.x; q < nb; q += BT) sl.y[(int64_t)i * nb + q] = ytile2[q];
        __syncthreads();
      }
    }
    for (int i = threadIdx.x; i < nb; i += BT) sl.y[r0 + i] = ytile[i];
    __syncthreads();
  }
  // back substitution U x = y, tile by tile from the bottom
  for (int k = n - 1; k >= 0; --k) {
    const int64_t r0 = (int64_t)k * nb;
    if (threadIdx.x == 0) {
      for (int r = nb - 1; r >= 0; --r) {
        T s = sl.y[r0 + r];
        for (int q = r + 1; q < nb; ++q) s -= sl.W[r0 + r + (r0 + q) * ldw] * sl.y[r0 + q];
        sl.y[r0 + r] = s / sl.W[r0 + r + (r0 + r) * ldw];
      }
    }
    __syncthreads();
    for (int rr = threadIdx.x; rr < (int)r0; rr += BT) {
      T s = (T)0;
      for (int q = 0; q < nb; ++q) s += sl.W[rr + (r0 + q) * ldw] * sl.y[r0 + q];
      sl.y[rr] -= s;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(BT, sizeof(T) == 4 ? 2 : 1) k_batched(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char bsm[];
  T* S0 = reinterpret_cast<T*>(bsm);
  T* S1 = S0 + TILE;
  T* S2 = S1 + TILE;
  T* S3 = S2 + TILE;
  T* Tm = S3 + TILE;
  T* Wm = Tm + TILE;
  T* vv = Wm + TILE;                                     // 4 * NBMAX
  T* tau_s = vv + 4 * NBMAX;                             // NBMAX
  double* dvec = reinterpret_cast<double*>(tau_s + NBMAX);   // 10 * NBMAX: local, away, 8 warps
  double* red = dvec + 10 * NBMAX;                       // 32
  int* piv_s = reinterpret_cast<int*>(red + 32);         // NBMAX
  int* s_int = piv_s + NBMAX;                            // 8
  __shared__ int s_sys;
  const Slot<T> sl = slot_of<T>(a, a.nmax);
  const int64_t ldw = a.ldw;
  for (;;) {
    if (threadIdx.x == 0) {
      s_sys = atomicAdd(a.counter, 1);
      for (int q = 0; q < 8; ++q) s_int[q] = 0;   // per-system flags start cleared
    }
    __syncthreads();
    const int qi = s_sys;
    __syncthreads();
    if (qi >= a.count) break;
    const int sys = a.order[qi];
    const int N = a.N[sys], nb = a.nbs[sys];
    const int n = (N + nb - 1) / nb, Np = n * nb;
    const double* A = a.A[sys];
    double* bx = a.b[sys];
    const double* b0 = a.b0[sys];
    uint8_t* dec = a.dec + (size_t)sys * a.nmax;
    int st = 0;
    // ---- pack [A | b] into the padded workspace (identity on the padded diagonal)
    for (int64_t idx = threadIdx.x; idx < (int64_t)Np * (Np + 1); idx += BT) {
      const int r = (int)(idx % Np), c = (int)(idx / Np);
      double v;
      if (c < Np) v = (r < N && c < N) ? A[r + (int64_t)c * N] : (r == c ? 1.0 : 0.0);
      else v = r < N ? b0[r] : 0.0;
      sl.W[r + (int64_t)c * ldw] = (T)v;
    }
    __syncthreads();
    for (int k = 0; k < n && st == 0; ++k) {
      const int64_t r0 = (int64_t)k * nb;
      const int m = n - 1 - k;
      // ---- criterion inputs (Sec. III-D): tile 1-norms, MUMPS column maxima, NaN/Inf
      for (int c = threadIdx.x; c < nb; c += BT) { dvec[c] = 0.0; dvec[NBMAX + c] = 0.0; }
      if (threadIdx.x == 0) s_int[2] = 0;
      __syncthreads();
      double nmax_below = 0.0, nsum_below = 0.0;
      for (int i = k; i < n; ++i) {
        double cs = 0.0;
        if (threadIdx.x < nb) {
          const int c = threadIdx.x;
          double sum = 0.0, mx = 0.0;
          for (int r = 0; r < nb; ++r) {
            const double v = fabs((double)sl.W[(int64_t)i * nb + r + (r0 + c) * ldw]);
            if (!isfinite(v)) s_int[2] = 1;
            sum += v;
            mx = fmax(mx, v);
          }
          cs = sum;
          if (i == k) dvec[c] = mx;
          else dvec[NBMAX + c] = fmax(dvec[NBMAX + c], mx);
        }
        // block max of the column sums = ||A_ik||_1
        double v = warp_max_d(threadIdx.x < nb ? cs : 0.0);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        double tn = 0.0;
        for (int w = 0; w < BT / 32; ++w) tn = fmax(tn, red[w]);
        __syncthreads();
        if (i > k) { nmax_below = fmax(nmax_below, tn); nsum_below = nsum_below + tn; }
      }
      // ---- GETRF of a shared copy of the diagonal tile, inverse norm, decision
      tload<T>(S0, sl.W + r0 + r0 * ldw, ldw, nb);
      __syncthreads();
      const int zr = tgetrf<T>(S0, piv_s, nb, s_int);
      double inv = 0.0;
      const bool need_inv = (a.criterion == LUQR_MAX || a.criterion == LUQR_SUM) && a.alpha != 0.0 && zr < 0;
      if (need_inv) inv = tinvnorm<T>(S0, piv_s, nb, dvec + 2 * NBMAX, red);
      if (threadIdx.x == 0) {
        uint8_t d;
        const int crit = a.criterion;
        if (s_int[2]) {
          d = DEC_ABORT;
          s_int[3] = LUQR_ERR_NONFINITE;
        } else if (crit == LUQR_FORCE_LU) {
          d = DEC_LU;
        } else if (crit == LUQR_FORCE_QR || a.alpha == 0.0 || zr >= 0) {
          d = DEC_QR;
        } else if (crit == LUQR_MAX || crit == LUQR_SUM) {
          const double L = a.alpha * (1.0 / inv);
          const double R = crit == LUQR_MAX ? nmax_below : nsum_below;
          d = (L >= R) ? DEC_LU : DEC_QR;
        } else {
          bool ok = true;
          double gprod = 1.0;
          for (int j = 0; j < nb; ++j) {
            const double pj = fabs((double)S0[j + j * LDS]);
            const double lj = dvec[j], aj = dvec[NBMAX + j];
            if (lj == 0.0) { ok = false; break; }
            double est;
            if (a.mumps_mode == 0) est = aj * (pj / lj);
            else { est = aj * gprod; gprod = gprod * (pj / lj); }
            if (!(a.alpha * pj >= est)) ok = false;
          }
          d = ok ? DEC_LU : DEC_QR;
        }
        if (d == DEC_LU && zr >= 0) { d = DEC_ABORT; s_int[3] = LUQR_ERR_SINGULAR; }
        dec[k] = d;
        s_int[4] = d;
        if (d == DEC_ABORT) s_int[5] = s_int[3];
        else s_int[5] = 0;
      }
      __syncthreads();
      const int d = s_int[4];
      st = s_int[5];
      (void)m;
      if (d == DEC_ABORT) break;
      if (d == DEC_LU) {
        // Alg. 2: commit LU, TRSM the tiles below, SWPTRSM the row (and b), GEMM the rest
        tstore<T>(S0, sl.W + r0 + r0 * ldw, ldw, nb);
        for (int q = threadIdx.x; q < nb; q += BT) sl.piv[k * NBMAX + q] = piv_s[q];
        __syncthreads();
        for (int i = k + 1; i < n; ++i) {
          T* X = sl.W + (int64_t)i * nb + r0 * ldw;
          tload<T>(S1, X, ldw, nb);
          __syncthreads();
          for (int c = 0; c < nb; ++c) {
            for (int rr = threadIdx.x; rr < nb; rr += BT) S1[rr + c * LDS] = S1[rr + c * LDS] / S0[c + c * LDS];
            __syncthreads();
            const int mc = nb - c - 1;
            for (int idx = threadIdx.x; idx < nb * mc; idx += BT) {
              const int rr = idx % nb, cc = c + 1 + idx / nb;
              S1[rr + cc * LDS] -= S1[rr + c * LDS] * S0[c + cc * LDS];
            }
            __syncthreads();
          }
          tstore<T>(S1, X, ldw, nb);
          __syncthreads();
        }
        for (int j = k + 1; j <= n; ++j) {   // column tiles of row k, then the b column
          const int w = (j < n) ? nb : 1;
          T* Cg = sl.W + r0 + (int64_t)j * nb * ldw;
          for (int idx = threadIdx.x; idx < nb * w; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            S1[rr + c * LDS] = Cg[rr + (int64_t)c * ldw];
          }
          __syncthreads();
          if ((int)threadIdx.x < w) {
            const int c = threadIdx.x;
            for (int r = 0; r < nb; ++r) {
              const int p = piv_s[r];
              if (p != r) { const T t = S1[r + c * LDS]; S1[r + c * LDS] = S1[p + c * LDS]; S1[p + c * LDS] = t; }
            }
            for (int r = 0; r < nb; ++r)
              for (int q = r + 1; q < nb; ++q) S1[q + c * LDS] -= S0[q + r * LDS] * S1[r + c * LDS];
          }
          __syncthreads();
          for (int idx = threadIdx.x; idx < nb * w; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            Cg[rr + (int64_t)c * ldw] = S1[rr + c * LDS];
          }
          __syncthreads();
        }
        for (int i = k + 1; i < n; ++i) {
          tload<T>(S1, sl.W + (int64_t)i * nb + r0 * ldw, ldw, nb);
          __syncthreads();
          for (int j = k + 1; j < n; ++j) {
            tload<T>(S2, sl.W + r0 + (int64_t)j * nb * ldw, ldw, nb);
            __syncthreads();
            tgemm_global_sub<T>(sl.W + (int64_t)i * nb + (int64_t)j * nb * ldw, ldw, S1, S2, nb);
          }
          // b column: b_i -= A_ik b_k
          for (int rr = threadIdx.x; rr < nb; rr += BT) {
            T s = (T)0;
            for (int q = 0; q < nb; ++q) s += S1[rr + q * LDS] * sl.W[r0 + q + (int64_t)Np * ldw];
            sl.W[(int64_t)i * nb + rr + (int64_t)Np * ldw] -= s;
          }
          __syncthreads();
        }
      } else {
        // Alg. 3 / Alg. 4(a), flat tree: GEQRT(k), UNMQR on row k; TSQRT(i, k), TSMQR rows (k, i)
        tload<T>(S0, sl.W + r0 + r0 * ldw, ldw, nb);
        __syncthreads();
        thouse<T>(S0, nullptr, Tm, tau_s, Wm, nb);
        tstore<T>(S0, sl.W + r0 + r0 * ldw, ldw, nb);
        {
          T* Tk = sl.Tst + ((size_t)k * a.nmax + k) * TILE;
          for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            Tk[rr + c * LDS] = Tm[rr + c * LDS];
          }
        }
        __syncthreads();
        for (int j = k + 1; j <= n; ++j) {
          const int w = (j < n) ? nb : 1;
          T* Cg = sl.W + r0 + (int64_t)j * nb * ldw;
          for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            S1[rr + c * LDS] = c < w ? Cg[rr + (int64_t)c * ldw] : (T)0;
          }
          __syncthreads();
          tunmqr<T>(S0, Tm, S1, Wm, S2, nb);
          for (int idx = threadIdx.x; idx < nb * w; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            Cg[rr + (int64_t)c * ldw] = S1[rr + c * LDS];
          }
          __syncthreads();
        }
        // R (upper part of the diagonal tile) eliminates every tile below; it is re-read
        // for each TSQRT so that S0 can serve as a product workspace during the TSMQRs
        for (int i = k + 1; i < n; ++i) {
          T* Ai = sl.W + (int64_t)i * nb + r0 * ldw;
          T* Rg = sl.W + r0 + r0 * ldw;
          for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            S0[rr + c * LDS] = rr <= c ? Rg[rr + (int64_t)c * ldw] : (T)0;
          }
          tload<T>(S1, Ai, ldw, nb);
          __syncthreads();
          thouse<T>(S1, S0, Tm, tau_s, Wm, nb);
          for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            if (rr <= c) Rg[rr + (int64_t)c * ldw] = S0[rr + c * LDS];
          }
          tstore<T>(S1, Ai, ldw, nb);
          T* Ti = sl.Tst + ((size_t)k * a.nmax + i) * TILE;
          for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
            const int rr = idx % nb, c = idx / nb;
            Ti[rr + c * LDS] = Tm[rr + c * LDS];
          }
          __syncthreads();
          for (int j = k + 1; j <= n; ++j) {
            const int w = (j < n) ? nb : 1;
            T* C1g = sl.W + r0 + (int64_t)j * nb * ldw;
            T* C2g = sl.W + (int64_t)i * nb + (int64_t)j * nb * ldw;
            for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
              const int rr = idx % nb, c = idx / nb;
              S2[rr + c * LDS] = c < w ? C1g[rr + (int64_t)c * ldw] : (T)0;
              S3[rr + c * LDS] = c < w ? C2g[rr + (int64_t)c * ldw] : (T)0;
            }
            __syncthreads();
            ttsmqr<T>(S1, Tm, S2, S3, Wm, S0, nb);
            for (int idx = threadIdx.x; idx < nb * w; idx += BT) {
              const int rr = idx % nb, c = idx / nb;
              C1g[rr + (int64_t)c * ldw] = S2[rr + c * LDS];
              C2g[rr + (int64_t)c * ldw] = S3[rr + c * LDS];
            }
            __syncthreads();
          }
        }
        __syncthreads();
      }
    }
    // ---- back substitution of the augmented column, then FP64 refinement (FP32 mode)
    double eta = NAN;
    int its = 0;
    if (st == 0) {
      for (int i = threadIdx.x; i < Np; i += BT) sl.y[i] = sl.W[i + (int64_t)Np * ldw];
      __syncthreads();
      // back substitution only (transforms already applied to the augmented column)
      for (int k = n - 1; k >= 0; --k) {
        const int64_t r0 = (int64_t)k * nb;
        if (threadIdx.x == 0) {
          for (int r = nb - 1; r >= 0; --r) {
            T s = sl.y[r0 + r];
            for (int q = r + 1; q < nb; ++q) s -= sl.W[r0 + r + (r0 + q) * ldw] * sl.y[r0 + q];
            const T dd = sl.W[r0 + r + (r0 + r) * ldw];
            if (dd == (T)0) { s_int[6] = 1; s = (T)0; }
            sl.y[r0 + r] = dd != (T)0 ? s / dd : (T)0;
          }
        }
        __syncthreads();
        for (int rr = threadIdx.x; rr < (int)r0; rr += BT) {
          T s = (T)0;
          for (int q = 0; q < nb; ++q) s += sl.W[rr + (r0 + q) * ldw] * sl.y[r0 + q];
          sl.y[rr] -= s;
        }
        __syncthreads();
      }
      for (int i = threadIdx.x; i < N; i += BT) sl.x[i] = (double)sl.y[i];
      __syncthreads();
      for (its = 1; its <= a.max_iter + 1; ++its) {
        // r = b - A x (FP64), eta = ||r|| / (||A|| ||x|| + ||b||)
        double rmax = 0.0, xmax = 0.0, bmax = 0.0, amax = 0.0;
        for (int i = threadIdx.x; i < N; i += BT) {
          double s = b0[i], ra = 0.0;
          for (int c = 0; c < N; ++c) {
            const double av = A[i + (int64_t)c * N];
            s -= av * sl.x[c];
            ra += fabs(av);
          }
          sl.r[i] = s;
          rmax = fmax(rmax, fabs(s));
          xmax = fmax(xmax, fabs(sl.x[i]));
          bmax = fmax(bmax, fabs(b0[i]));
          amax = fmax(amax, ra);
        }
        double vals[4] = {rmax, xmax, bmax, amax};
        for (int q = 0; q < 4; ++q) {
          double v = warp_max_d(vals[q]);
          if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) + 8 * q] = v;
        }
        __syncthreads();
        double R[4] = {0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
          for (int w = 0; w < BT / 32; ++w) R[q] = fmax(R[q], red[w + 8 * q]);
        __syncthreads();
        eta = R[0] / (R[3] * R[1] + R[2]);
        if (!a.fp32 || !(eta > a.tol) || its > a.max_iter) break;
        // d = solve(r / ||r||) in the factorization's precision; x += ||r|| d
        const double sc = R[0] > 0.0 ? R[0] : 1.0;
        for (int i = threadIdx.x; i < Np; i += BT) sl.y[i] = (T)(i < N ? sl.r[i] / sc : 0.0);
        __syncthreads();
        replay_solve<T>(a, sl, dec, n, nb, S0, S1, Tm, vv);
        for (int i = threadIdx.x; i < N; i += BT) sl.x[i] += sc * (double)sl.y[i];
        __syncthreads();
      }
      if (s_int[6]) st = LUQR_ERR_SINGULAR;
    }
    if (st == 0)
      for (int i = threadIdx.x; i < N; i += BT) bx[i] = sl.x[i];
    if (threadIdx.x == 0) {
      a.status[sys] = st;
      a.iters[sys] = its;
      a.eta[sys] = eta;
      s_int[6] = 0;
    }
    __syncthreads();
  }
}


template <typename T>
size_t batched_smem() {
  return sizeof(T) * (6 * (size_t)TILE + 5 * NBMAX) + sizeof(double) * (10 * NBMAX + 32) +
         sizeof(int) * (NBMAX + 8) + 64;
}

}  // namespace
}  // namespace luqr

using namespace luqr;

struct luqr_batched {
  int count = 0, nmax = 0, fp32 = 0;
  int64_t ldw = 0;
  size_t slot_bytes = 0;
  int slots = 0;
  BatchArgs args{};
  void* dev = nullptr;      // metadata block
  void* slot_mem = nullptr;
  double* b0_mem = nullptr; // copies of the right-hand sides (runs are repeatable)
  cudaGraphExec_t graph = nullptr;   // captured counter reset + persistent launch
};

namespace {
void batched_free(luqr_batched* p) {
  if (!p) return;
  if (p->dev) cudaFree(p->dev);
  if (p->slot_mem) cudaFree(p->slot_mem);
  if (p->b0_mem) cudaFree(p->b0_mem);
  if (p->graph) cudaGraphExecDestroy(p->graph);
  delete p;
}
}  // namespace

extern "C" int luqr_batched_create(const double* const* dA, double* const* db, const int* N,
                                   const int* nb, int count, int criterion, double alpha,
                                   const luqr_options* opt, double tol, int max_iter,
                                   luqr_batched_t* out) {
  if (!out) return LUQR_ERR_INVALID;
  *out = nullptr;
  if (!dA || !db || !N || !nb || count < 1) return LUQR_ERR_INVALID;
  if (criterion < LUQR_MAX || criterion > LUQR_FORCE_QR || !(alpha >= 0.0) || max_iter < 0 ||
      !(tol >= 0.0))
    return LUQR_ERR_INVALID;
  luqr_options o{};
  if (opt) o = *opt;
  if (o.precision < 0 || o.precision > 1 || o.mumps_mode < 0 || o.mumps_mode > 1) return LUQR_ERR_INVALID;
  if (o.norm_mode != 0) return LUQR_ERR_INVALID;   // the batched criterion uses the exact norm
  if (o.lu_variant != 0 || o.domain > 1) return LUQR_ERR_INVALID;  // batched: A1, tile pivoting
  int nmax = 0;
  int64_t npmax = 0;
  for (int i = 0; i < count; ++i) {
    if (N[i] < 1 || N[i] > 8192 || (nb[i] != 32 && nb[i] != 64) || !dA[i] || !db[i]) return LUQR_ERR_INVALID;
    const int n = (N[i] + nb[i] - 1) / nb[i];
    nmax = std::max(nmax, n);
    npmax = std::max<int64_t>(npmax, (int64_t)n * nb[i]);
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return N[x] > N[y]; });
  luqr_batched* p = new (std::nothrow) luqr_batched();
  if (!p) return LUQR_ERR_NOMEM;
  p->count = count;
  p->nmax = nmax;
  p->fp32 = o.precision == LUQR_PREC_FP32;
  p->ldw = npmax;
  const size_t elt = p->fp32 ? sizeof(float) : sizeof(double);
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  size_t sb = al((size_t)npmax * (npmax + 1) * elt);
  sb += al((size_t)nmax * nmax * TILE * elt);
  sb += al((size_t)nmax * NBMAX * sizeof(int));
  sb += al(2 * (size_t)npmax * sizeof(double));
  sb += al((size_t)npmax * elt);
  p->slot_bytes = sb;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // as many persistent CTAs as fit at once (two per SM for FP32 tiles)
  int per_sm = 1;
  if (p->fp32) {
    ensure_dyn_smem<k_batched<float>>(batched_smem<float>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<float>, BT, batched_smem<float>());
  } else {
    ensure_dyn_smem<k_batched<double>>(batched_smem<double>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched<double>, BT, batched_smem<double>());
  }
  cudaGetLastError();
  p->slots = std::min(count, std::max(1, sms) * std::max(1, per_sm));
  // metadata block: A ptrs, b ptrs, N, nb, order, dec, iters, eta, status, counter
  size_t off = 0;
  const size_t oA = off; off = al(off + sizeof(void*) * count);
  const size_t oB = off; off = al(off + sizeof(void*) * count);
  const size_t oB0 = off; off = al(off + sizeof(void*) * count);
  const size_t oN = off; off = al(off + sizeof(int) * count);
  const size_t oNB = off; off = al(off + sizeof(int) * count);
  const size_t oO = off; off = al(off + sizeof(int) * count);
  const size_t oD = off; off = al(off + (size_t)count * nmax);
  const size_t oI = off; off = al(off + sizeof(int) * count);
  const size_t oE = off; off = al(off + sizeof(double) * count);
  const size_t oS = off; off = al(off + sizeof(int) * count);
  const size_t oC = off; off = al(off + sizeof(int));
  int64_t total_n = 0;
  for (int i = 0; i < count; ++i) total_n += N[i];
  cudaError_t e = cudaMalloc(&p->dev, off);
  if (e == cudaSuccess) e = cudaMalloc(&p->slot_mem, p->slot_bytes * p->slots);
  if (e == cudaSuccess) e = cudaMalloc(&p->b0_mem, sizeof(double) * (size_t)total_n);
  if (e != cudaSuccess) {
    batched_free(p);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LUQR_ERR_NOMEM : LUQR_ERR_CUDA;
  }
  unsigned char* d = static_cast<unsigned char*>(p->dev);
  cudaMemcpy(d + oA, dA, sizeof(void*) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(d + oB, db, sizeof(void*) * count, cudaMemcpyHostToDevice);
  {
    std::vector<const double*> b0p(count);
    int64_t o0 = 0;
    for (int i = 0; i < count; ++i) {
      b0p[i] = p->b0_mem + o0;
      cudaMemcpy(p->b0_mem + o0, db[i], sizeof(double) * N[i], cudaMemcpyDeviceToDevice);
      o0 += N[i];
    }
    cudaMemcpy(d + oB0, b0p.data(), sizeof(void*) * count, cudaMemcpyHostToDevice);
  }
  cudaMemcpy(d + oN, N, sizeof(int) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(d + oNB, nb, sizeof(int) * count, cudaMemcpyHostToDevice);
  cudaMemcpy(d + oO, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice);
  cudaMemset(d + oD, 255, (size_t)count * nmax);
  BatchArgs& a = p->args;
  a.A = reinterpret_cast<const double* const*>(d + oA);
  a.b = reinterpret_cast<double* const*>(d + oB);
  a.b0 = reinterpret_cast<const double* const*>(d + oB0);
  a.N = reinterpret_cast<const int*>(d + oN);
  a.nbs = reinterpret_cast<const int*>(d + oNB);
  a.order = reinterpret_cast<const int*>(d + oO);
  a.count = count;
  a.criterion = criterion;
  a.mumps_mode = o.mumps_mode;
  a.alpha = alpha;
  a.fp32 = p->fp32;
  a.tol = tol;
  a.max_iter = max_iter;
  a.slots = p->slot_mem;
  a.slot_bytes = p->slot_bytes;
  a.ldw = npmax;
  a.nmax = nmax;
  a.dec = reinterpret_cast<uint8_t*>(d + oD);
  a.iters = reinterpret_cast<int*>(d + oI);
  a.eta = reinterpret_cast<double*>(d + oE);
  a.status = reinterpret_cast<int*>(d + oS);
  a.counter = reinterpret_cast<int*>(d + oC);
  if (cudaGetLastError() != cudaSuccess) { batched_free(p); return LUQR_ERR_CUDA; }
  *out = p;
  return LUQR_OK;
}

extern "C" int luqr_batched_run(luqr_batched_t p, void* stream) {
  if (!p) return LUQR_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaMemsetAsync(p->args.counter, 0, sizeof(int), s);
  if (p->fp32) {
    const size_t sm = batched_smem<float>();
    ensure_dyn_smem<k_batched<float>>(sm);
    ProfScope ps_("k_batched", s);
    k_batched<float><<<p->slots, BT, sm, s>>>(p->args);
  } else {
    const size_t sm = batched_smem<double>();
    ensure_dyn_smem<k_batched<double>>(sm);
    ProfScope ps_("k_batched", s);
    k_batched<double><<<p->slots, BT, sm, s>>>(p->args);
  }
  return cudaGetLastError() == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}

extern "C" int luqr_batched_run_graph(luqr_batched_t p, void* stream) {
  if (!p) return LUQR_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!p->graph) {
    const size_t sm = p->fp32 ? batched_smem<float>() : batched_smem<double>();
    if (p->fp32) ensure_dyn_smem<k_batched<float>>(sm);
    else ensure_dyn_smem<k_batched<double>>(sm);
    // capture on a private stream so that the caller's stream is never in capture mode
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemsetAsync(p->args.counter, 0, sizeof(int), cs);
      if (p->fp32) k_batched<float><<<p->slots, BT, sm, cs>>>(p->args);
      else k_batched<double><<<p->slots, BT, sm, cs>>>(p->args);
      e = cudaStreamEndCapture(cs, &g);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      p->graph = nullptr;
      cudaGetLastError();
      return LUQR_ERR_CUDA;
    }
  }
  ProfScope ps_("k_batched", s);
  return cudaGraphLaunch(p->graph, s) == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}

extern "C" int luqr_batched_results(luqr_batched_t p, uint8_t* dec, int* status, int* iters,
                                    double* eta, int* nmax_out) {
  if (!p) return LUQR_ERR_INVALID;
  if (cudaDeviceSynchronize() != cudaSuccess) return LUQR_ERR_CUDA;
  if (nmax_out) *nmax_out = p->nmax;
  const BatchArgs& a = p->args;
  if (dec && cudaMemcpy(dec, a.dec, (size_t)p->count * p->nmax, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  if (status && cudaMemcpy(status, a.status, sizeof(int) * p->count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  if (iters && cudaMemcpy(iters, a.iters, sizeof(int) * p->count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  if (eta && cudaMemcpy(eta, a.eta, sizeof(double) * p->count, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  return LUQR_OK;
}

extern "C" void luqr_batched_destroy(luqr_batched_t p) {
  if (!p) return;
  cudaDeviceSynchronize();
  batched_free(p);
}
