// LU step variant A2 (Sec. II-B): the diagonal tile is factored by GEQRT instead of GETRF.
//
// Factor: A_kk = Q R on a scratch copy (the library's GEQRT kernel, run on the scratch tile).
// Check: ||A_kk^-1||_1 = ||R^-1 Q^T||_1 for Eq. 2 and 3; |R_jj| are the pivots of Eq. 4; an
// exact zero on R's diagonal plays the zero pivot's part (QR is selected).
// LU step: the scratch V and R are committed to the tile; Eliminate A_ik <- A_ik R^-1 (the
// TRSM of variant A1, on R); Apply A_kj <- Q^T A_kj (UNMQR with the tile's V and T, or for
// the FP32 tensor-core update an explicit X = Q^T); Update as A1.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace luqr {

// Identity pivots (no row exchange in A2) and the first exact zero on R's diagonal.
template <typename T>
__global__ void k_a2_prep(const T* __restrict__ S, int nb, int* __restrict__ piv, int* status) {
  for (int j = threadIdx.x; j < nb; j += blockDim.x) piv[j] = j;
  if (threadIdx.x == 0) {
    int zr = -1;
    for (int j = 0; j < nb; ++j)
      if (S[j + (int64_t)j * nb] == (T)0) { zr = j; break; }
    status[ST_ZERO_ROW] = zr;
  }
}

// gate[k] = DEC_QR exactly when dec[k] = DEC_LU, so that the QR-gated UNMQR kernel applies
// the Q^T of an A2 LU step.
__global__ void k_a2_gate(const uint8_t* __restrict__ dec, uint8_t* __restrict__ gate, int k) {
  if (threadIdx.x == 0) gate[k] = (dec[k] == DEC_LU) ? DEC_QR : DEC_LU;
}

// Column c of Q^T (mode 1: written to X, nb x nb column-major) or of R^-1 Q^T (mode 0: its
// absolute sum to colsum[c]) for the GEQRT factors in S (leading dimension lds): V unit lower triangular below the
// diagonal, R on and above; tau_j on the diagonal of the compact-WY T blocks (IB x IB block
// of columns jb.. stored at Tslot[a + (jb + j) * IB]).  x = e_c; reflectors j = 0 .. nb-1 in
// order: w = x_j + v_j . x(j+1:), x_j -= tau_j w, x(j+1:) -= tau_j v_j w; then (mode 0) the
// backward substitution with R.  One warp per column, FP64 arithmetic.  Mode 0 is gated on
// dec[k] (runs before the decision: gate array may be all DEC_QR) and skipped when R has an
// exact zero on its diagonal (colsum = inf).
constexpr int QT_WARPS = 4;

template <typename T>
__global__ void __launch_bounds__(32 * QT_WARPS) k_qt_cols(const T* __restrict__ S, int64_t lds,
                                                          int nb, const T* __restrict__ Tslot,
                                                          int mode,
                                                          double* __restrict__ colsum,
                                                          T* __restrict__ X, const int* status,
                                                          const uint8_t* __restrict__ gate, int k) {
  if (gate[k] != DEC_QR) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * QT_WARPS + warp;
  if (c >= nb) return;
  if (mode == 0 && status[ST_ZERO_ROW] >= 0) {
    if (lane == 0) colsum[c] = INFINITY;
    return;
  }
  double* x = reinterpret_cast<double*>(smem_raw) + (size_t)warp * nb;
  for (int r = lane; r < nb; r += 32) x[r] = (r == c) ? 1.0 : 0.0;
  __syncwarp();
  for (int j = 0; j < nb; ++j) {
    const double tau = (double)Tslot[(j % IB) + (size_t)j * IB];
    if (tau == 0.0) continue;
    const T* v = S + (int64_t)j * lds;
    double part = 0.0;
    for (int r = j + 1 + lane; r < nb; r += 32) part += (double)v[r] * x[r];
    const double w = warp_sum_d(part) + x[j];
    __syncwarp();
    if (lane == 0) x[j] -= tau * w;
    for (int r = j + 1 + lane; r < nb; r += 32) x[r] -= tau * ((double)v[r] * w);
    __syncwarp();
  }
  if (mode == 1) {
    for (int r = lane; r < nb; r += 32) X[r + (int64_t)c * nb] = (T)x[r];
    return;
  }
  for (int r = nb - 1; r >= 0; --r) {
    const T* u = S + (int64_t)r * lds;
    if (lane == 0) x[r] = x[r] / (double)u[r];
    __syncwarp();
    const double xr = x[r];
    if (xr != 0.0)
      for (int i = lane; i < r; i += 32) x[i] -= (double)u[i] * xr;
    __syncwarp();
  }
  double sum = 0.0;
  for (int r = lane; r < nb; r += 32) sum += fabs(x[r]);
  sum = warp_sum_d(sum);
  if (lane == 0) colsum[c] = sum;
}

template <typename T>
void launch_a2_prep(const T* S, int nb, int* piv, int* status, cudaStream_t s) {
  ProfScope ps_("k_a2_prep", s);
  k_a2_prep<T><<<1, 256, 0, s>>>(S, nb, piv, status);
}

void launch_a2_gate(const uint8_t* dec, uint8_t* gate, int k, cudaStream_t s) {
  ProfScope ps_("k_a2_gate", s);
  k_a2_gate<<<1, 32, 0, s>>>(dec, gate, k);
}

template <typename T>
void launch_qt_cols(const T* S, int64_t lds, int nb, const T* Tslot, int mode, double* colsum,
                    T* X, const int* status, const uint8_t* gate, int k, cudaStream_t s) {
  const size_t smem = sizeof(double) * QT_WARPS * (size_t)nb;
  ensure_dyn_smem<k_qt_cols<T>>(smem);
  ProfScope ps_(mode == 0 ? "k_qt_invnorm" : "k_qt_explicit", s);
  k_qt_cols<T><<<(nb + QT_WARPS - 1) / QT_WARPS, 32 * QT_WARPS, smem, s>>>(
      S, lds, nb, Tslot, mode, colsum, X, status, gate, k);
}

template void launch_a2_prep<float>(const float*, int, int*, int*, cudaStream_t);
template void launch_a2_prep<double>(const double*, int, int*, int*, cudaStream_t);
template void launch_qt_cols<float>(const float*, int64_t, int, const float*, int, double*,
                                    float*, const int*, const uint8_t*, int, cudaStream_t);
template void launch_qt_cols<double>(const double*, int64_t, int, const double*, int, double*,
                                     double*, const int*, const uint8_t*, int, cudaStream_t);

}  // namespace luqr
