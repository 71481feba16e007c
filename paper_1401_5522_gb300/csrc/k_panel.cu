// Panel-side kernels of one step of the hybrid LU-QR factorization:
// pack/pad, run-time injection, criterion inputs (Sec. III-D), the diagonal GETRF on
// a scratch copy (Alg. 1 "Factor"), ||A_kk^-1||_1 from the L and U factors, and the
// robustness test (Eq. 2, 3, 4) that writes the step's decision to device memory.
#include "internal.cuh"

namespace luqr {

// ---------------------------------------------------------------- pack / pad
// W (Npad x Wc, column-major) <- [A, b] padded with an identity block (Sec. II-D).
template <typename T>
__global__ void k_pack(const double* __restrict__ A, int64_t lda, const double* __restrict__ b,
                       int64_t N, int64_t Npad, int64_t Wc, T* __restrict__ W, int64_t ldw) {
  for (int64_t c = blockIdx.y; c < Wc; c += gridDim.y)
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < Npad;
         r += (int64_t)gridDim.x * blockDim.x) {
      double v;
      if (c < Npad)
        v = (r < N && c < N) ? A[r + c * lda] : (r == c ? 1.0 : 0.0);
      else
        v = (b != nullptr && r < N) ? b[r] : 0.0;
      W[r + c * ldw] = (T)v;
    }
}

template <typename T>
void launch_pack(const double* A, int64_t lda, const double* b, int64_t N, int64_t Npad,
                 int64_t Wc, T* W, int64_t ldw, cudaStream_t s) {
  int bx = (int)((Npad + 255) / 256);
  if (bx > 64) bx = 64;
  dim3 grid(bx, (unsigned)(Wc < 65535 ? Wc : 65535));
  {
    ProfScope ps_("k_pack", s);
    k_pack<T><<<grid, 256, 0, s>>>(A, lda, b, N, Npad, Wc, W, ldw);
  }
}

// ---------------------------------------------------------------- injection
template <typename T>
__global__ void k_scale_rows(T* W, int64_t ldw, int64_t row0, int rows, int64_t col0,
                             int64_t col1, double scale) {
  for (int64_t c = col0 + blockIdx.x; c < col1; c += gridDim.x)
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
      T* p = &W[row0 + r + c * ldw];
      *p = (T)((double)*p * scale);
    }
}

template <typename T>
void launch_scale_rows(T* W, int64_t ldw, int64_t row0, int rows, int64_t col0, int64_t col1,
                       double scale, cudaStream_t s) {
  int64_t nc = col1 - col0;
  if (nc <= 0) return;
  int g = (int)(nc < 4096 ? nc : 4096);
  {
    ProfScope ps_("k_scale_rows", s);
    k_scale_rows<T><<<g, 256, 0, s>>>(W, ldw, row0, rows, col0, col1, scale);
  }
}

// ---------------------------------------------------------------- criterion inputs
// Block i-k: ||A_ik||_1 (max column abs sum, FP64 accumulation) and the column maxima
// used by the MUMPS criterion (local for i = k, away for i > k).  Non-finite entries
// raise the status' nonfinite flag.
template <typename T>
__global__ void k_panel_stats(const T* __restrict__ W, int64_t ldw, int k, int nb,
                              double* __restrict__ norms_k, unsigned long long* __restrict__ local,
                              unsigned long long* __restrict__ away, int* status) {
  const int i = k + blockIdx.x;
  const T* tile = W + (int64_t)i * nb + (int64_t)k * nb * ldw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  double best = 0.0;
  bool bad = false;
  for (int c = warp; c < nb; c += nw) {
    const T* col = tile + (int64_t)c * ldw;
    double sum = 0.0, mx = 0.0;
    for (int r = lane; r < nb; r += 32) {
      double v = fabs((double)col[r]);
      if (!isfinite(v)) bad = true;
      sum += v;
      mx = fmax(mx, v);
    }
    sum = warp_sum_d(sum);
    mx = warp_max_d(mx);
    if (lane == 0) {
      best = fmax(best, sum);
      unsigned long long bits = (unsigned long long)__double_as_longlong(mx);
      if (i == k)
        local[c] = bits;
      else
        atomicMax(&away[c], bits);   // non-negative doubles order like their bit patterns
    }
  }
  if (bad) atomicOr(&status[ST_NONFINITE], 1);
  __shared__ double red[32];
  if (lane == 0) red[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, red[w]);
    norms_k[i] = m;
  }
}

template <typename T>
void launch_panel_stats(const T* W, int64_t ldw, int k, int n, int nb, double* norms_k,
                        unsigned long long* local, unsigned long long* away, int* status,
                        cudaStream_t s) {
  cudaMemsetAsync(away, 0, sizeof(unsigned long long) * nb, s);
  {
    ProfScope ps_("k_panel_stats", s);
    k_panel_stats<T><<<n - k, 256, 0, s>>>(W, ldw, k, nb, norms_k, local, away, status);
  }
}

// ---------------------------------------------------------------- diagonal GETRF
// S <- A_kk, then P S = L U in place with partial pivoting inside the tile: the pivot
// of column r is the first row of maximal |S[r:, r]|.  An exact zero pivot leaves the
// column unscaled and is recorded (first one) in status[ST_ZERO_ROW].
//
// Blocked right-looking order (same operations per element as the column loop, up to
// the summation order of the trailing update): for each panel of GP columns
//   (a) the panel rows jb.. are factored in shared memory (warp 0 searches the pivot),
//   (b) the panel's row exchanges are applied to the other columns as one gather,
//   (c) U12 <- L11^-1 A12 (one thread per column),
//   (d) A22 <- A22 - L21 U12 with U12 staged in shared memory per column chunk.
constexpr int GP = 32;        // panel width
constexpr int GT = 512;       // threads
constexpr int GCH = 64;       // column chunk of the trailing update

template <typename T>
__global__ void __launch_bounds__(GT) k_getrf(const T* __restrict__ W, int64_t ldw, int k, int nb,
                                              T* __restrict__ S, int* __restrict__ piv,
                                              int* status, int gbuf_elems) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* P = reinterpret_cast<T*>(smem_raw);          // nb x GP panel, row stride GP+1
  T* U12 = P + (size_t)nb * (GP + 1);              // GP x GCH chunk, row stride GCH
  T* gbuf = U12 + GP * GCH;                        // gather buffer, gbuf_elems values
  int* perm = reinterpret_cast<int*>(gbuf + gbuf_elems);   // nb
  int* moved = perm + nb;                          // <= 2*GP moved rows
  __shared__ int s_nmoved, s_zero;
  __shared__ T s_piv_val;
  const T* A = W + (int64_t)k * nb + (int64_t)k * nb * ldw;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int PST = GP + 1;
  for (int idx = tid; idx < nb * nb; idx += GT) {
    const int r = idx % nb, c = idx / nb;
    S[idx] = A[r + (int64_t)c * ldw];
  }
  if (tid == 0) s_zero = -1;
  __syncthreads();
  for (int jb = 0; jb < nb; jb += GP) {
    const int nr = nb - jb;
    // ---- (a) panel factorization in shared memory
    for (int idx = tid; idx < nr * GP; idx += GT) {
      const int r = idx % nr, j = idx / nr;
      P[r * PST + j] = S[(jb + r) + (jb + j) * nb];
    }
    for (int i = tid; i < nr; i += GT) perm[i] = i;
    __syncthreads();
    for (int j = 0; j < GP; ++j) {
      if (warp == 0) {
        // |a| compares exactly in the working precision
        T bv = (T)-1;
        int bi = nr;
        for (int r = j + lane; r < nr; r += 32) {
          const T v = fabs(P[r * PST + j]);
          if (v > bv) { bv = v; bi = r; }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if (bi >= nr) bi = j;                 // no comparable entry (NaN): keep the row
        if (bi != j)
          for (int c = lane; c < GP; c += 32) {
            const T tmp = P[j * PST + c];
            P[j * PST + c] = P[bi * PST + c];
            P[bi * PST + c] = tmp;
          }
        __syncwarp();
        if (lane == 0) {
          piv[jb + j] = jb + bi;
          const int tmp = perm[j];
          perm[j] = perm[bi];
          perm[bi] = tmp;
          s_piv_val = P[j * PST + j];
          if (P[j * PST + j] == (T)0 && s_zero < 0) s_zero = jb + j;
        }
      }
      __syncthreads();
      const T d = s_piv_val;
      if (d != (T)0) {
        // one thread per row below the pivot: its multiplier, then its entries right of j
        // (the pivot row is final after the barrier; no other thread touches this row)
        for (int r = j + 1 + tid; r < nr; r += GT) {
          const T l = P[r * PST + j] / d;
          P[r * PST + j] = l;
          for (int c = j + 1; c < GP; ++c) P[r * PST + c] -= l * P[j * PST + c];
        }
      }
      __syncthreads();
    }
    for (int idx = tid; idx < nr * GP; idx += GT) {
      const int r = idx % nr, j = idx / nr;
      S[(jb + r) + (jb + j) * nb] = P[r * PST + j];
    }
    // ---- (b) gather the moved rows of the columns outside the panel (the moved rows are
    //      listed by all threads at once, their order does not matter: a permutation)
    if (tid == 0) s_nmoved = 0;
    __syncthreads();
    for (int i = tid; i < nr; i += GT)
      if (perm[i] != i) moved[atomicAdd(&s_nmoved, 1)] = i;   // at most 2*GP rows move
    __syncthreads();
    const int nm = s_nmoved;
    const int nother = nb - GP;   // columns outside the panel
    // as many columns per pass as the gather buffer holds (every column at nb = 256 FP32)
    const int gcw = nm > 0 ? max(1, gbuf_elems / nm) : nother;
    for (int c0 = 0; c0 < nother; c0 += gcw) {
      const int cw = min(gcw, nother - c0);
      for (int idx = tid; idx < nm * cw; idx += GT) {
        const int a = idx % nm, cc = idx / nm;
        int col = c0 + cc;
        col = col < jb ? col : col + GP;
        gbuf[idx] = S[(jb + perm[moved[a]]) + col * nb];
      }
      __syncthreads();
      for (int idx = tid; idx < nm * cw; idx += GT) {
        const int a = idx % nm, cc = idx / nm;
        int col = c0 + cc;
        col = col < jb ? col : col + GP;
        S[(jb + moved[a]) + col * nb] = gbuf[idx];
      }
      __syncthreads();
    }
    // ---- (c) U12 <- L11^-1 A12 and (d) A22 -= L21 U12, per chunk of trailing columns
    for (int c0 = jb + GP; c0 < nb; c0 += GCH) {
      const int cw = min(GCH, nb - c0);
      if (tid < cw) {
        T u[GP];
#pragma unroll
        for (int r = 0; r < GP; ++r) u[r] = S[(jb + r) + (c0 + tid) * nb];
#pragma unroll
        for (int r = 0; r < GP; ++r) {
#pragma unroll
          for (int q = r + 1; q < GP; ++q) u[q] -= P[q * PST + r] * u[r];
        }
#pragma unroll
        for (int r = 0; r < GP; ++r) {
          S[(jb + r) + (c0 + tid) * nb] = u[r];
          U12[r * GCH + tid] = u[r];
        }
      }
      __syncthreads();
      const int mr = nr - GP;
      const int rt = (mr + 3) / 4, ct = (cw + 3) / 4;
      for (int idx = tid; idx < rt * ct; idx += GT) {
        const int rb = (idx % rt) * 4, cb = (idx / rt) * 4;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) acc[i][jj] = (T)0;
        for (int q = 0; q < GP; ++q) {
          T a[4], bq[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = (rb + i < mr) ? P[(GP + rb + i) * PST + q] : (T)0;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) bq[jj] = (cb + jj < cw) ? U12[q * GCH + cb + jj] : (T)0;
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) acc[i][jj] += a[i] * bq[jj];
        }
#pragma unroll
        for (int jj = 0; jj < 4; ++jj)
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (rb + i < mr && cb + jj < cw) S[(jb + GP + rb + i) + (c0 + cb + jj) * nb] -= acc[i][jj];
      }
      __syncthreads();
    }
  }
  if (tid == 0) status[ST_ZERO_ROW] = s_zero;
}

// Gather buffer of k_getrf: every moved row (at most 2*GP) of every column outside the panel
// when that fits in a CTA's shared memory, else the largest multiple of 2*GP rows that does.
template <typename T>
int getrf_gbuf(int nb) {
  const size_t base = sizeof(T) * ((size_t)nb * (GP + 1) + (size_t)GP * GCH) +
                      sizeof(int) * (size_t)(nb + 2 * GP) + 16;
  const size_t want = (size_t)2 * GP * (nb - GP);
  const size_t room = base < (size_t)SMEM_MAX ? ((size_t)SMEM_MAX - base) / sizeof(T) : 0;
  const size_t g = want < room ? want : room / (2 * GP) * (2 * GP);
  return (int)(g > (size_t)2 * GP ? g : (size_t)2 * GP);
}
template <typename T>
size_t getrf_smem(int nb) {
  return sizeof(T) * ((size_t)nb * (GP + 1) + (size_t)GP * GCH + (size_t)getrf_gbuf<T>(nb)) +
         sizeof(int) * (size_t)(nb + 2 * GP);
}

template <typename T>
void launch_getrf(const T* W, int64_t ldw, int k, int nb, T* S, int* piv_s, int* status,
                  cudaStream_t s) {
  ensure_dyn_smem<k_getrf<T>>(getrf_smem<T>(nb));
  {
    ProfScope ps_("k_getrf", s);
    k_getrf<T><<<1, GT, getrf_smem<T>(nb), s>>>(W, ldw, k, nb, S, piv_s, status,
                                                 getrf_gbuf<T>(nb));
  }
}

// ---------------------------------------------------------------- ||A_kk^-1||_1
// X = U^-1 L^-1 P (FP64 arithmetic on the stored factors); colsum[c] = sum_r |X[r, c]|.
// One warp per column c (two per CTA): the column is substituted in shared memory, step
// by step, with the factor's columns staged INV_CH at a time through cp.async (the next
// group in flight) and shared by the CTA's warps.  FP64 arithmetic runs at 2 FMA per clock
// per SM on this part, so the columns are spread over nb/2 CTAs.  Skipped when the tile
// has a zero pivot.
constexpr int INV_CH = 8;
constexpr int INV_WARPS = 2;

template <typename T>
__global__ void __launch_bounds__(32 * INV_WARPS) k_invnorm(const T* __restrict__ S, int nb,
                                                           const int* __restrict__ piv,
                                                           double* __restrict__ colsum,
                                                           const int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* xs_all = reinterpret_cast<double*>(smem_raw);                 // INV_WARPS x nb
  T* colbuf = reinterpret_cast<T*>(xs_all + (size_t)INV_WARPS * nb);    // 2 x INV_CH x nb
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x * INV_WARPS + warp;
  if (status[ST_ZERO_ROW] >= 0) {
    if (lane == 0 && c < nb) colsum[c] = INFINITY;
    return;
  }
  double* ys = xs_all + (size_t)warp * nb;
  int pos = c;   // row of the single 1 of column c of P
  for (int r = 0; r < nb; ++r) {
    const int p = piv[r];
    if (pos == r) pos = p;
    else if (pos == p) pos = r;
  }
  for (int row = lane; row < nb; row += 32) ys[row] = (row == pos) ? 1.0 : 0.0;
  auto fetch = [&](int first, int slot) {
    T* dst = colbuf + (size_t)slot * INV_CH * nb;
    for (int idx = tid; idx < INV_CH * nb; idx += 32 * INV_WARPS) {
      const int cc = idx / nb, i = idx - cc * nb, col = first + cc;
      if (col >= 0 && col < nb) cp_async(&dst[idx], &S[i + (int64_t)col * nb]);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int nch = nb / INV_CH;
  // y <- L^-1 y (unit lower), columns r = 0 .. nb-2
  fetch(0, 0);
  for (int g = 0; g < nch; ++g) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    fetch((g + 1) * INV_CH, (g + 1) & 1);
    const T* base = colbuf + (size_t)(g & 1) * INV_CH * nb;
    for (int cc = 0; cc < INV_CH; ++cc) {
      const int r = g * INV_CH + cc;
      if (r >= nb - 1 || c >= nb) break;
      __syncwarp();
      const double yr = ys[r];
      if (r < pos || yr == 0.0) continue;
      const T* col = base + (size_t)cc * nb;
      for (int row = r + 1 + lane; row < nb; row += 32) ys[row] -= (double)col[row] * yr;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  // x <- U^-1 y, columns r = nb-1 .. 0; group g holds columns [nb-(g+1)*CH, nb-g*CH)
  fetch(nb - INV_CH, 0);
  for (int g = 0; g < nch; ++g) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    fetch(nb - (g + 2) * INV_CH, (g + 1) & 1);
    const T* base = colbuf + (size_t)(g & 1) * INV_CH * nb;
    if (c < nb) {
      // reciprocals of the group's diagonal entries first, off the dependency chain
      double dinv = 0.0;
      if (lane < INV_CH) {
        const int r = nb - (g + 1) * INV_CH + lane;
        dinv = 1.0 / (double)base[(size_t)lane * nb + r];
      }
      for (int cc = INV_CH - 1; cc >= 0; --cc) {
        const int r = nb - (g + 1) * INV_CH + cc;
        const T* col = base + (size_t)cc * nb;
        const double inv = __shfl_sync(0xffffffffu, dinv, cc);
        __syncwarp();
        if (lane == 0) ys[r] = ys[r] * inv;
        __syncwarp();
        const double xr = ys[r];
        if (xr != 0.0)
          for (int row = lane; row < r; row += 32) ys[row] -= (double)col[row] * xr;
      }
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  if (c < nb) {
    double sum = 0.0;
    for (int row = lane; row < nb; row += 32) sum += fabs(ys[row]);
    sum = warp_sum_d(sum);
    if (lane == 0) colsum[c] = sum;
  }
}

template <typename T>
void launch_invnorm(const T* S, int nb, const int* piv_s, double* colsum, const int* status,
                    cudaStream_t s) {
  const size_t smem = sizeof(double) * INV_WARPS * (size_t)nb + sizeof(T) * 2 * INV_CH * (size_t)nb;
  ensure_dyn_smem<k_invnorm<T>>(smem);
  ProfScope ps_("k_invnorm", s);
  k_invnorm<T><<<(nb + INV_WARPS - 1) / INV_WARPS, 32 * INV_WARPS, smem, s>>>(S, nb, piv_s,
                                                                             colsum, status);
}

// ---------------------------------------------------------------- ||A_kk^-1||_1 estimate
// Hager-Higham estimator of ||A^-1||_1 for A = P^T L U (norm_mode = 1; the paper's
// Sec. III-D uses an iterative O(nb^2) estimate): maximise the convex f(x) = ||A^-1 x||_1
// over the unit 1-norm ball by moving from the centre e/nb to the vertex e_j of the
// largest |z_j|, z = A^-T sign(A^-1 x); stop when the sign vector repeats, the value stops
// growing, the vertex stays, or after five iterations; finally probe the alternating
// vector x_i = (-1)^i (1 + i/(nb-1)) and keep 2||A^-1 x||_1 / (3 nb) when larger.  One CTA;
// every solve is blocked by 32: a warp solves the diagonal block with shuffles, the block
// then updates the remaining rows.  FP64 arithmetic on the stored factors.  The estimate
// goes to colsum[0] (the other entries are 0), so the decision kernel is unchanged.
constexpr int EST_T = 256;

__device__ double est_block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < EST_T / 32; ++w) t += red[w];
  return t;
}

// First index of the largest |z_i|.
__device__ int est_block_argmax(const double* z, int nb, double* redv, int* redi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double bv = -1.0;
  int bi = nb;
  for (int i = threadIdx.x; i < nb; i += EST_T) {
    const double a = fabs(z[i]);
    if (a > bv) { bv = a; bi = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, bv, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
  }
  __syncthreads();
  if (lane == 0) { redv[warp] = bv; redi[warp] = bi; }
  __syncthreads();
  double rv = -1.0;
  int ri = nb;
  for (int w = 0; w < EST_T / 32; ++w)
    if (redv[w] > rv || (redv[w] == rv && redi[w] < ri)) { rv = redv[w]; ri = redi[w]; }
  return ri;
}

// v <- A^-1 v = U^-1 L^-1 P v  (perm: (P v)[i] = v[perm[i]])
template <typename T>
__device__ void est_solve(const T* __restrict__ S, int nb, double* v, double* tmp,
                          const int* perm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < nb; i += EST_T) tmp[i] = v[perm[i]];
  __syncthreads();
  for (int i = tid; i < nb; i += EST_T) v[i] = tmp[i];
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 32) {            // L y = P v, unit lower, forward
    if (warp == 0) {
      double a[32];   // row b0+lane of the diagonal block, loaded before the dependent chain
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = (double)S[(b0 + lane) + (int64_t)(b0 + j) * nb];
      double yi = v[b0 + lane];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const double yj = __shfl_sync(0xffffffffu, yi, j);
        if (lane > j) yi -= a[j] * yj;
      }
      v[b0 + lane] = yi;
    }
    __syncthreads();
    for (int i = b0 + 32 + tid; i < nb; i += EST_T) {
      double acc = 0.0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) acc += (double)S[i + (int64_t)(b0 + j) * nb] * v[b0 + j];
      v[i] -= acc;
    }
    __syncthreads();
  }
  for (int b0 = nb - 32; b0 >= 0; b0 -= 32) {      // U x = y, backward
    if (warp == 0) {
      double a[32];   // row b0+lane of the diagonal block (a[lane] is the pivot)
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = (double)S[(b0 + lane) + (int64_t)(b0 + j) * nb];
      double xi = v[b0 + lane];
#pragma unroll
      for (int j = 31; j >= 0; --j) {
        if (lane == j) xi = xi / a[j];
        const double xj = __shfl_sync(0xffffffffu, xi, j);
        if (lane < j) xi -= a[j] * xj;
      }
      v[b0 + lane] = xi;
    }
    __syncthreads();
    for (int i = tid; i < b0; i += EST_T) {
      double acc = 0.0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) acc += (double)S[i + (int64_t)(b0 + j) * nb] * v[b0 + j];
      v[i] -= acc;
    }
    __syncthreads();
  }
}

// v <- A^-T v = P^T L^-T U^-T v
template <typename T>
__device__ void est_solve_t(const T* __restrict__ S, int nb, double* v, double* tmp,
                            const int* perm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int b0 = 0; b0 < nb; b0 += 32) {            // U^T w = v, forward (column i of U)
    if (warp == 0) {
      double a[32];   // column b0+lane of the diagonal block (a[lane] is the pivot)
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = (double)S[(b0 + j) + (int64_t)(b0 + lane) * nb];
      double wi = v[b0 + lane];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (lane == j) wi = wi / a[j];
        const double wj = __shfl_sync(0xffffffffu, wi, j);
        if (lane > j) wi -= a[j] * wj;
      }
      v[b0 + lane] = wi;
    }
    __syncthreads();
    for (int i = b0 + 32 + tid; i < nb; i += EST_T) {
      const T* col = S + (int64_t)i * nb + b0;
      double acc = 0.0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) acc += (double)col[j] * v[b0 + j];
      v[i] -= acc;
    }
    __syncthreads();
  }
  for (int b0 = nb - 32; b0 >= 0; b0 -= 32) {      // L^T u = w, backward, unit
    if (warp == 0) {
      double a[32];   // column b0+lane of the diagonal block
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = (double)S[(b0 + j) + (int64_t)(b0 + lane) * nb];
      double ui = v[b0 + lane];
#pragma unroll
      for (int j = 31; j >= 0; --j) {
        const double uj = __shfl_sync(0xffffffffu, ui, j);
        if (lane < j) ui -= a[j] * uj;
      }
      v[b0 + lane] = ui;
    }
    __syncthreads();
    for (int i = tid; i < b0; i += EST_T) {
      const T* col = S + (int64_t)i * nb + b0;
      double acc = 0.0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) acc += (double)col[j] * v[b0 + j];
      v[i] -= acc;
    }
    __syncthreads();
  }
  for (int i = tid; i < nb; i += EST_T) tmp[perm[i]] = v[i];
  __syncthreads();
  for (int i = tid; i < nb; i += EST_T) v[i] = tmp[i];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(EST_T) k_invnorm_est(const T* __restrict__ S, int nb,
                                                       const int* __restrict__ piv,
                                                       double* __restrict__ colsum,
                                                       const int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* v = reinterpret_cast<double*>(smem_raw);   // nb
  double* z = v + nb;                                  // nb
  double* tmp = z + nb;                                // nb
  double* red = tmp + nb;                              // 32
  int* perm = reinterpret_cast<int*>(red + 32);        // nb
  int* redi = perm + nb;                               // 32
  signed char* xi = reinterpret_cast<signed char*>(redi + 32);   // nb
  const int tid = threadIdx.x;
  if (status[ST_ZERO_ROW] >= 0) {
    for (int c = tid; c < nb; c += EST_T) colsum[c] = INFINITY;
    return;
  }
  if (tid == 0) {
    for (int i = 0; i < nb; ++i) perm[i] = i;
    for (int r = 0; r < nb; ++r) {
      const int p = piv[r];
      if (p != r) { const int t = perm[r]; perm[r] = perm[p]; perm[p] = t; }
    }
  }
  for (int i = tid; i < nb; i += EST_T) v[i] = 1.0 / nb;
  __syncthreads();
  est_solve<T>(S, nb, v, tmp, perm);
  double part = 0.0;
  for (int i = tid; i < nb; i += EST_T) part += fabs(v[i]);
  double est = est_block_sum(part, red);
  for (int i = tid; i < nb; i += EST_T) {
    xi[i] = v[i] >= 0.0 ? 1 : -1;
    z[i] = v[i] >= 0.0 ? 1.0 : -1.0;
  }
  __syncthreads();
  est_solve_t<T>(S, nb, z, tmp, perm);
  int j = est_block_argmax(z, nb, red, redi);
  for (int it = 2;; ++it) {
    for (int i = tid; i < nb; i += EST_T) v[i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    est_solve<T>(S, nb, v, tmp, perm);
    part = 0.0;
    bool same = true;
    for (int i = tid; i < nb; i += EST_T) {
      part += fabs(v[i]);
      same = same && ((v[i] >= 0.0 ? 1 : -1) == xi[i]);
    }
    const double est_old = est;
    est = est_block_sum(part, red);
    const bool all_same = __syncthreads_and(same ? 1 : 0) != 0;
    if (all_same || est <= est_old) break;
    for (int i = tid; i < nb; i += EST_T) {
      xi[i] = v[i] >= 0.0 ? 1 : -1;
      z[i] = v[i] >= 0.0 ? 1.0 : -1.0;
    }
    __syncthreads();
    est_solve_t<T>(S, nb, z, tmp, perm);
    const int jlast = j;
    j = est_block_argmax(z, nb, red, redi);
    if (fabs(z[jlast]) == fabs(z[j]) || it >= 5) break;
  }
  for (int i = tid; i < nb; i += EST_T)
    v[i] = ((i & 1) ? -1.0 : 1.0) * (1.0 + (double)i / (double)(nb - 1));
  __syncthreads();
  est_solve<T>(S, nb, v, tmp, perm);
  part = 0.0;
  for (int i = tid; i < nb; i += EST_T) part += fabs(v[i]);
  const double t = 2.0 * est_block_sum(part, red) / (3.0 * nb);
  if (t > est) est = t;
  for (int c = tid; c < nb; c += EST_T) colsum[c] = (c == 0) ? est : 0.0;
}

template <typename T>
void launch_invnorm_est(const T* S, int nb, const int* piv_s, double* colsum, const int* status,
                        cudaStream_t s) {
  const size_t smem = sizeof(double) * (3 * (size_t)nb + 32) + sizeof(int) * ((size_t)nb + 32) +
                      (size_t)nb;
  ensure_dyn_smem<k_invnorm_est<T>>(smem);
  ProfScope ps_("k_invnorm_est", s);
  k_invnorm_est<T><<<1, EST_T, smem, s>>>(S, nb, piv_s, colsum, status);
}

// ---------------------------------------------------------------- decision
__device__ double log2_ratio(double lhs, double rhs) {
  if (rhs == 0.0) return lhs > 0.0 ? INFINITY : (lhs == 0.0 ? 0.0 : -INFINITY);
  if (lhs == 0.0) return -INFINITY;
  if (isinf(lhs)) return INFINITY;
  return log2(lhs / rhs);
}

// Output i (0-based) of the SplitMix64 generator whose state starts at `seed` (Steele, Lea
// and Flood, 2014): state advanced by the golden-ratio increment, then two xor-shift /
// multiply rounds and a final xor-shift.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed,
                                                           unsigned long long i) {
  unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Single thread: Eq. 2 (Max), Eq. 3 (Sum), Eq. 4 (MUMPS) with the readings listed in the
// oracle (">=" selects LU, alpha = 0 or a zero pivot selects QR, last step compares to 0),
// and the random choice of Sec. V-B (LU with probability alpha/100).
template <typename T>
__global__ void k_decide(DecideArgs a, const T* __restrict__ S) {
  if (threadIdx.x != 0) return;
  int* st = a.status;
  const int k = a.k;
  if (st[ST_CODE] != 0) { a.dec[k] = DEC_ABORT; return; }
  if (st[ST_NONFINITE]) {
    st[ST_CODE] = -5; st[ST_STEP] = k; st[ST_ROW] = -1;
    a.dec[k] = DEC_ABORT;
    return;
  }
  const int zr = st[ST_ZERO_ROW];
  uint8_t d;
  double mg, L = NAN, R = NAN;
  const int crit = a.criterion;
  if (a.forced) {
    d = a.forced[k];
    mg = (d == DEC_LU) ? INFINITY : -INFINITY;
  } else if (crit == 3) {
    d = DEC_LU; mg = INFINITY;
  } else if (crit == 4 || a.alpha == 0.0) {
    d = DEC_QR; mg = -INFINITY;
  } else if (zr >= 0) {
    d = DEC_QR; mg = -INFINITY; L = 0.0;
  } else if (crit == 5) {
    L = a.alpha / 100.0;
    R = (double)(splitmix64_at(a.seed, (unsigned long long)k) >> 11) * 0x1.0p-53;
    d = (R < L) ? DEC_LU : DEC_QR;
    mg = log2_ratio(L, R);
  } else if (crit == 0 || crit == 1) {
    double inv = 0.0;
    for (int c = 0; c < a.nb; ++c) inv = fmax(inv, a.colsum[c]);
    L = a.alpha * (1.0 / inv);
    R = 0.0;
    if (crit == 0) {
      for (int i = k + 1; i < a.n; ++i) R = fmax(R, a.norms_k[i]);
    } else {
      for (int i = k + 1; i < a.n; ++i) R = R + a.norms_k[i];
    }
    d = (L >= R) ? DEC_LU : DEC_QR;
    mg = log2_ratio(L, R);
  } else {   // MUMPS, Eq. 4
    bool ok = true;
    mg = INFINITY;
    double gprod = 1.0;
    d = DEC_LU;
    for (int j = 0; j < a.nb; ++j) {
      const double pj = fabs((double)S[j + j * a.nb]);
      const double lj = __longlong_as_double((long long)a.local[j]);
      const double aj = __longlong_as_double((long long)a.away[j]);
      if (lj == 0.0) { ok = false; mg = -INFINITY; break; }
      double est;
      if (a.mumps_mode == 0) {
        est = aj * (pj / lj);
      } else {
        est = aj * gprod;
        gprod = gprod * (pj / lj);
      }
      const double lhs = a.alpha * pj;
      if (!(lhs >= est)) ok = false;
      mg = fmin(mg, log2_ratio(lhs, est));
    }
    d = ok ? DEC_LU : DEC_QR;
  }
  if (d == DEC_LU && zr >= 0) {
    st[ST_CODE] = -4; st[ST_STEP] = k; st[ST_ROW] = k * a.nb + zr;
    d = DEC_ABORT;
  }
  a.dec[k] = d;
  a.margin[k] = mg;
  a.lhs[k] = L;
  a.rhs[k] = R;
}

template <typename T>
void launch_decide(const DecideArgs& a, const T* S, cudaStream_t s) {
  {
    ProfScope ps_("k_decide", s);
    k_decide<T><<<1, 32, 0, s>>>(a, S);
  }
}

#define INST(T)                                                                                  \
  template void launch_pack<T>(const double*, int64_t, const double*, int64_t, int64_t, int64_t, \
                               T*, int64_t, cudaStream_t);                                       \
  template void launch_scale_rows<T>(T*, int64_t, int64_t, int, int64_t, int64_t, double,        \
                                     cudaStream_t);                                              \
  template void launch_panel_stats<T>(const T*, int64_t, int, int, int, double*,                 \
                                      unsigned long long*, unsigned long long*, int*,            \
                                      cudaStream_t);                                             \
  template void launch_getrf<T>(const T*, int64_t, int, int, T*, int*, int*, cudaStream_t);      \
  template void launch_invnorm<T>(const T*, int, const int*, double*, const int*, cudaStream_t); \
  template void launch_invnorm_est<T>(const T*, int, const int*, double*, const int*,           \
                                      cudaStream_t);                                            \
  template void launch_decide<T>(const DecideArgs&, const T*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace luqr
