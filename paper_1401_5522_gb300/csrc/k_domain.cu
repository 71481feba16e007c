// Diagonal-domain pivoting (Sec. II-B, the variant the paper's experiments use): the Factor
// step searches its pivots over the d tiles k .. k+d-1 of the panel instead of the diagonal
// tile alone.
//   * a tall GETRF (partial pivoting, first row of maximal |a|) of a scratch copy of the
//     d*nb x nb domain; its top nb x nb rows are L11 and U of the pivoted diagonal tile;
//   * the criterion sees the pivoted panel: a copy of panel k with the domain rows permuted
//     gives the tile norms and the MUMPS column maxima;
//   * an LU step first applies the domain's row exchanges to columns k.. of those rows (and
//     b), then runs the tile LU step with identity pivots; the second pass repeats the
//     exchanges on its right-hand sides.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace luqr {

constexpr int DT = 256;   // threads of the domain kernels

// Tall GETRF of the rows x nb domain (rows = d*nb) starting at (k*nb, k*nb) of W, on a
// scratch copy St (leading dimension rows).  dpiv[j] = row (0-based within the domain)
// exchanged with row j at elimination step j; piv_s gets the identity (the diagonal tile is
// already pivoted); status[ST_ZERO_ROW] = first j with an exact zero pivot, or -1.  One CTA;
// the scratch stays in L2.
template <typename T>
__global__ void __launch_bounds__(DT) k_getrf_tall(const T* __restrict__ W, int64_t ld, int k,
                                                   int nb, int rows, T* __restrict__ St,
                                                   int* __restrict__ dpiv, int* __restrict__ piv_s,
                                                   int* status) {
  __shared__ double s_val[DT / 32];
  __shared__ int s_idx[DT / 32];
  __shared__ int s_p, s_zero;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const T* A = W + (int64_t)k * nb + (int64_t)k * nb * ld;
  for (int64_t idx = tid; idx < (int64_t)rows * nb; idx += DT) {
    const int r = (int)(idx % rows), c = (int)(idx / rows);
    St[idx] = A[r + (int64_t)c * ld];
  }
  for (int j = tid; j < nb; j += DT) piv_s[j] = j;
  if (tid == 0) s_zero = -1;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    T* cj = St + (int64_t)j * rows;
    // pivot: first row of maximal |a| in rows j .. rows-1
    double bv = -1.0;
    int bi = rows;
    for (int r = j + tid; r < rows; r += DT) {
      const double a = fabs((double)cj[r]);
      if (a > bv) { bv = a; bi = r; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, bv, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { s_val[warp] = bv; s_idx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double v = s_val[0];
      int p = s_idx[0];
      for (int w = 1; w < DT / 32; ++w)
        if (s_val[w] > v || (s_val[w] == v && s_idx[w] < p)) { v = s_val[w]; p = s_idx[w]; }
      s_p = p;
      dpiv[j] = p;
    }
    __syncthreads();
    const int p = s_p;
    if (p != j)
      for (int c = tid; c < nb; c += DT) {
        T* col = St + (int64_t)c * rows;
        const T t = col[j];
        col[j] = col[p];
        col[p] = t;
      }
    __syncthreads();
    const T d = cj[j];
    if (d == (T)0) {
      if (tid == 0 && s_zero < 0) s_zero = j;
      __syncthreads();
      continue;
    }
    for (int r = j + 1 + tid; r < rows; r += DT) cj[r] = cj[r] / d;
    __syncthreads();
    const int nr = rows - j - 1, ncl = nb - j - 1;
    for (int64_t idx = tid; idx < (int64_t)nr * ncl; idx += DT) {
      const int r = j + 1 + (int)(idx % nr), c = j + 1 + (int)(idx / nr);
      T* col = St + (int64_t)c * rows;
      col[r] -= cj[r] * col[j];
    }
    __syncthreads();
  }
  if (tid == 0) status[ST_ZERO_ROW] = s_zero;
}

// Final position map of the exchange sequence: row j of the pivoted domain is original
// row perm[j] (rows 0 .. rows-1 of the domain).
__device__ void domain_perm(const int* __restrict__ dpiv, int nb, int rows, int* perm) {
  for (int j = threadIdx.x; j < rows; j += blockDim.x) perm[j] = j;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int j = 0; j < nb; ++j) {
      const int p = dpiv[j];
      if (p != j) { const int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
    }
  __syncthreads();
}

// P (rows k*nb .. Npad-1 of one nb-column panel, leading dimension ldp, indexed like W) <-
// panel k of W with the domain rows permuted.
template <typename T>
__global__ void __launch_bounds__(DT) k_domain_panel(const T* __restrict__ W, int64_t ld, int k,
                                                     int nb, int rows, int64_t Npad,
                                                     const int* __restrict__ dpiv,
                                                     T* __restrict__ P, int64_t ldp) {
  extern __shared__ int perm[];
  domain_perm(dpiv, nb, rows, perm);
  const int64_t r0 = (int64_t)k * nb;
  const int c = blockIdx.x;
  const T* src = W + (r0 + c) * ld;
  T* dst = P + (int64_t)c * ldp;
  for (int64_t r = r0 + threadIdx.x; r < Npad; r += DT) {
    const int64_t j = r - r0;
    dst[r] = (j < rows) ? src[r0 + perm[j]] : src[r];
  }
}

// Columns [c0, c1) of M (rows k*nb ..): the domain's row exchanges, gated on dec[k] = LU.
template <typename T>
__global__ void __launch_bounds__(DT) k_domain_swap(T* __restrict__ M, int64_t ld, int k, int nb,
                                                    int rows, int64_t c0, int64_t c1,
                                                    const int* __restrict__ dpiv,
                                                    const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_LU) return;
  extern __shared__ int perm[];
  T* buf = reinterpret_cast<T*>(perm + ((rows + 3) & ~3));
  domain_perm(dpiv, nb, rows, perm);
  const int64_t r0 = (int64_t)k * nb;
  for (int64_t c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
    T* col = M + r0 + c * ld;
    for (int j = threadIdx.x; j < rows; j += DT) buf[j] = col[j];
    __syncthreads();
    for (int j = threadIdx.x; j < rows; j += DT) col[j] = buf[perm[j]];
    __syncthreads();
  }
}

template <typename T>
void launch_getrf_tall(const T* W, int64_t ld, int k, int nb, int rows, T* St, int* dpiv,
                       int* piv_s, int* status, cudaStream_t s) {
  ProfScope ps_("k_getrf_tall", s);
  k_getrf_tall<T><<<1, DT, 0, s>>>(W, ld, k, nb, rows, St, dpiv, piv_s, status);
}

template <typename T>
void launch_domain_panel(const T* W, int64_t ld, int k, int nb, int rows, int64_t Npad,
                         const int* dpiv, T* P, int64_t ldp, cudaStream_t s) {
  ProfScope ps_("k_domain_panel", s);
  k_domain_panel<T><<<nb, DT, sizeof(int) * rows, s>>>(W, ld, k, nb, rows, Npad, dpiv, P, ldp);
}

template <typename T>
void launch_domain_swap(T* M, int64_t ld, int k, int nb, int rows, int64_t c0, int64_t c1,
                        const int* dpiv, const uint8_t* dec, cudaStream_t s) {
  if (c1 <= c0) return;
  const size_t smem = sizeof(int) * (size_t)((rows + 3) & ~3) + sizeof(T) * (size_t)rows;
  const int64_t cols = c1 - c0;
  const int grid = (int)(cols < 1024 ? cols : 1024);
  ProfScope ps_("k_domain_swap", s);
  k_domain_swap<T><<<grid, DT, smem, s>>>(M, ld, k, nb, rows, c0, c1, dpiv, dec);
}

#define DINST(T)                                                                               \
  template void launch_getrf_tall<T>(const T*, int64_t, int, int, int, T*, int*, int*, int*,   \
                                     cudaStream_t);                                            \
  template void launch_domain_panel<T>(const T*, int64_t, int, int, int, int64_t, const int*,  \
                                       T*, int64_t, cudaStream_t);                             \
  template void launch_domain_swap<T>(T*, int64_t, int, int, int, int64_t, int64_t,            \
                                      const int*, const uint8_t*, cudaStream_t);
DINST(double)
DINST(float)

}  // namespace luqr
