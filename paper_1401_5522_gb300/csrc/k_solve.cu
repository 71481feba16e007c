// Triangular solve of the factored system (Sec. II-D: "an N-by-N triangular solve is
// needed") and the FP64 helpers of iterative refinement: residual r = b - A x, norms
// for the normwise backward error, and x <- x + d.
#include "internal.cuh"

namespace luqr {

// ---------------------------------------------------------------- back substitution
// One block per right-hand side: x_k <- U_kk^-1 x_k for diagonal tile k (in place).
// The tile is processed in 32-row blocks from the bottom: warp 0 solves the 32 x 32
// triangle with shuffles, then all threads update the rows above.
template <typename T>
__global__ void __launch_bounds__(256) k_trsv_diag(Mat<const T> U, int k, int nb, Mat<T> X, int nrhs,
                                                   int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  __shared__ int s_bad;
  const int j = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t r0 = (int64_t)k * nb;
  for (int r = tid; r < nb; r += blockDim.x) xs[r] = X(r0 + r, j);
  if (tid == 0) s_bad = -1;
  __syncthreads();
  for (int bb = nb / 32 - 1; bb >= 0; --bb) {
    const int b0 = bb * 32;
    if (warp == 0) {
      // lane l holds row b0+l of the 32 x 32 diagonal block (all loads issued at once)
      T u[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) u[r] = U(r0 + b0 + lane, r0 + b0 + r);
      T x = xs[b0 + lane];
      int bad = -1;
#pragma unroll
      for (int r = 31; r >= 0; --r) {
        const T d = __shfl_sync(0xffffffffu, u[r], r);
        if (d == (T)0) { bad = b0 + r; break; }
        if (lane == r) x = x / d;
        const T xr = __shfl_sync(0xffffffffu, x, r);
        if (lane < r) x -= u[r] * xr;
      }
      xs[b0 + lane] = x;
      if (lane == 0 && bad >= 0) s_bad = bad;
    }
    __syncthreads();
    if (s_bad >= 0) break;
    for (int i = tid; i < b0; i += blockDim.x) {
      T acc = (T)0;
#pragma unroll 8
      for (int q = 0; q < 32; ++q) acc += U(r0 + i, r0 + b0 + q) * xs[b0 + q];
      xs[i] -= acc;
    }
    __syncthreads();
  }
  if (s_bad >= 0) {
    if (tid == 0 && atomicCAS(&status[ST_CODE], 0, -4) == 0) {
      status[ST_STEP] = k;
      status[ST_ROW] = (int)(r0 + s_bad);
    }
    return;
  }
  for (int r = tid; r < nb; r += blockDim.x) X(r0 + r, j) = xs[r];
}

template <typename T>
void launch_trsv_diag(Mat<const T> U, int k, int nb, Mat<T> X, int nrhs, int* status,
                      cudaStream_t s) {
  {
    ProfScope ps_("k_trsv_diag", s);
    k_trsv_diag<T><<<nrhs, 256, nb * sizeof(T), s>>>(U, k, nb, X, nrhs, status);
  }
}

// X[0:k*nb, :] -= U[0:k*nb, k*nb:(k+1)*nb] X[k*nb:(k+1)*nb, :]
template <typename T>
__global__ void k_trsv_update(Mat<const T> U, int k, int nb, Mat<T> X, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xk = reinterpret_cast<T*>(smem_raw);
  const int64_t r0 = (int64_t)k * nb;
  const int j = blockIdx.y;
  for (int c = threadIdx.x; c < nb; c += blockDim.x) xk[c] = X(r0 + c, j);
  __syncthreads();
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= r0) return;
  T s = (T)0;
  for (int c = 0; c < nb; ++c) s += U(row, r0 + c) * xk[c];
  X(row, j) -= s;
}

template <typename T>
void launch_trsv_update(Mat<const T> U, int k, int nb, Mat<T> X, int nrhs, cudaStream_t s) {
  const int64_t rows = (int64_t)k * nb;
  if (rows <= 0) return;
  dim3 grid((unsigned)((rows + 127) / 128), (unsigned)nrhs);
  {
    ProfScope ps_("k_trsv_update", s);
    k_trsv_update<T><<<grid, 128, nb * sizeof(T), s>>>(U, k, nb, X, nrhs);
  }
}

// ---------------------------------------------------------------- conversions
// dst (Npad x nrhs) <- src / scale (rows >= N set to 0); scale may be null (1).
template <typename T>
__global__ void k_convert_in(const double* __restrict__ src, int64_t lds, int64_t N, int64_t Npad,
                             const double* __restrict__ scale, T* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  const double inv = scale ? (scale[0] > 0.0 ? 1.0 / scale[0] : 1.0) : 1.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < Npad;
       r += (int64_t)gridDim.x * blockDim.x)
    dst[r + j * ldd] = (T)(r < N ? src[r + j * lds] * inv : 0.0);
}

template <typename T>
void launch_convert_in(const double* src, int64_t lds, int64_t N, int64_t Npad, int nrhs,
                       const double* scale, T* dst, int64_t ldd, cudaStream_t s) {
  int bx = (int)((Npad + 255) / 256);
  if (bx > 1024) bx = 1024;
  {
    ProfScope ps_("k_convert_in", s);
    k_convert_in<T><<<dim3(bx, nrhs), 256, 0, s>>>(src, lds, N, Npad, scale, dst, ldd);
  }
}

template <typename T>
__global__ void k_convert_out(const T* __restrict__ src, int64_t lds, int64_t N,
                              double* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x)
    dst[r + j * ldd] = (double)src[r + j * lds];
}

template <typename T>
void launch_convert_out(const T* src, int64_t lds, int64_t N, int nrhs, double* dst, int64_t ldd,
                        cudaStream_t s) {
  int bx = (int)((N + 255) / 256);
  if (bx > 1024) bx = 1024;
  {
    ProfScope ps_("k_convert_out", s);
    k_convert_out<T><<<dim3(bx, nrhs), 256, 0, s>>>(src, lds, N, dst, ldd);
  }
}

// ---------------------------------------------------------------- residual (FP64)
// partial[c][row] = sum_{j in chunk c} A[row, j] x[j]; then r = b - sum_c partial[c] (fixed order).
constexpr int RES_ROWS = 256;
constexpr int RES_COLS = 512;

__global__ void k_residual_partial(const double* __restrict__ A, int64_t lda, int64_t N,
                                   const double* __restrict__ x, double* __restrict__ partial) {
  __shared__ double xs[RES_COLS];
  const int64_t c0 = (int64_t)blockIdx.y * RES_COLS;
  const int64_t row = (int64_t)blockIdx.x * RES_ROWS + threadIdx.x;
  const int nc = (int)min((int64_t)RES_COLS, N - c0);
  for (int c = threadIdx.x; c < nc; c += blockDim.x) xs[c] = x[c0 + c];
  __syncthreads();
  if (row >= N) return;
  const double* a = A + row + c0 * lda;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int c = 0;
  for (; c + 4 <= nc; c += 4) {
    s0 += a[(int64_t)c * lda] * xs[c];
    s1 += a[(int64_t)(c + 1) * lda] * xs[c + 1];
    s2 += a[(int64_t)(c + 2) * lda] * xs[c + 2];
    s3 += a[(int64_t)(c + 3) * lda] * xs[c + 3];
  }
  for (; c < nc; ++c) s0 += a[(int64_t)c * lda] * xs[c];
  partial[blockIdx.y * N + row] = (s0 + s1) + (s2 + s3);
}

__global__ void k_residual_reduce(const double* __restrict__ partial, int nchunk, int64_t N,
                                  const double* __restrict__ b, double* __restrict__ r) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < N;
       row += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[c * N + row];
    r[row] = b[row] - s;
  }
}

void launch_residual(const double* A, int64_t lda, int64_t N, const double* x, const double* b,
                     double* r, double* partial, int nchunk, cudaStream_t s) {
  dim3 grid((unsigned)((N + RES_ROWS - 1) / RES_ROWS), (unsigned)nchunk);
  {
    ProfScope ps_("k_residual_partial", s);
    k_residual_partial<<<grid, RES_ROWS, 0, s>>>(A, lda, N, x, partial);
  }
  int bx = (int)((N + 255) / 256);
  if (bx > 2048) bx = 2048;
  {
    ProfScope ps_("k_residual_reduce", s);
    k_residual_reduce<<<bx, 256, 0, s>>>(partial, nchunk, N, b, r);
  }
}

// ||A||_inf: partial row sums over column chunks, then the max over rows of their sum.
__global__ void k_rowabs_partial(const double* __restrict__ A, int64_t lda, int64_t N,
                                 double* __restrict__ partial) {
  const int64_t c0 = (int64_t)blockIdx.y * RES_COLS;
  const int64_t row = (int64_t)blockIdx.x * RES_ROWS + threadIdx.x;
  if (row >= N) return;
  const int nc = (int)min((int64_t)RES_COLS, N - c0);
  const double* a = A + row + c0 * lda;
  double s = 0.0;
  for (int c = 0; c < nc; ++c) s += fabs(a[(int64_t)c * lda]);
  partial[blockIdx.y * N + row] = s;
}

__global__ void k_rowabs_max(const double* __restrict__ partial, int nchunk, int64_t N,
                             double* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t row = threadIdx.x; row < N; row += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[c * N + row];
    m = fmax(m, s);
  }
  m = warp_max_d(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    out[0] = t;
  }
}

void launch_row_abs_sum_max(const double* A, int64_t lda, int64_t N, double* partial, int nchunk,
                            double* out, cudaStream_t s) {
  dim3 grid((unsigned)((N + RES_ROWS - 1) / RES_ROWS), (unsigned)nchunk);
  {
    ProfScope ps_("k_rowabs_partial", s);
    k_rowabs_partial<<<grid, RES_ROWS, 0, s>>>(A, lda, N, partial);
  }
  {
    ProfScope ps_("k_rowabs_max", s);
    k_rowabs_max<<<1, 1024, 0, s>>>(partial, nchunk, N, out);
  }
}

__global__ void k_vec_absmax(const double* __restrict__ v, int64_t N, double* __restrict__ out) {
  __shared__ double red[32];
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(v[i]));
  m = warp_max_d(m);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    out[0] = t;
  }
}

void launch_vec_absmax(const double* v, int64_t N, double* out, cudaStream_t s) {
  {
    ProfScope ps_("k_vec_absmax", s);
    k_vec_absmax<<<1, 1024, 0, s>>>(v, N, out);
  }
}

// x <- x + scale * d (d in the factorization's precision)
template <typename T>
__global__ void k_axpy_update(double* __restrict__ x, const T* __restrict__ d, int64_t N,
                              const double* __restrict__ scale) {
  const double sc = scale ? scale[0] : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] += sc * (double)d[i];
}

template <typename T>
void launch_axpy_update(double* x, const T* d, int64_t N, const double* scale, cudaStream_t s) {
  int bx = (int)((N + 255) / 256);
  if (bx > 1024) bx = 1024;
  {
    ProfScope ps_("k_axpy_update", s);
    k_axpy_update<T><<<bx, 256, 0, s>>>(x, d, N, scale);
  }
}

// ---------------------------------------------------------------- GMRES helpers (FP64)
// out = A v (column-major A); same chunked two-pass scheme as the residual.
__global__ void k_matvec_reduce(const double* __restrict__ partial, int nchunk, int64_t N,
                                double* __restrict__ out) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < N;
       row += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[c * N + row];
    out[row] = s;
  }
}

void launch_matvec(const double* A, int64_t lda, int64_t N, const double* v, double* out,
                   double* partial, int nchunk, cudaStream_t s) {
  dim3 grid((unsigned)((N + RES_ROWS - 1) / RES_ROWS), (unsigned)nchunk);
  {
    ProfScope ps_("k_residual_partial", s);
    k_residual_partial<<<grid, RES_ROWS, 0, s>>>(A, lda, N, v, partial);
  }
  int bx = (int)((N + 255) / 256);
  if (bx > 2048) bx = 2048;
  {
    ProfScope ps_("k_matvec_reduce", s);
    k_matvec_reduce<<<bx, 256, 0, s>>>(partial, nchunk, N, out);
  }
}

// dots[i] = V[:, i] . w for i < cnt (V column-major, ldv); one block per i.
__global__ void k_multidot(const double* __restrict__ V, int64_t ldv, int64_t N,
                           const double* __restrict__ w, double* __restrict__ dots) {
  __shared__ double red[32];
  const double* v = V + (int64_t)blockIdx.x * ldv;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += v[i] * w[i];
  s = warp_sum_d(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
    dots[blockIdx.x] = t;
  }
}

void launch_multidot(const double* V, int64_t ldv, int64_t N, int cnt, const double* w,
                     double* dots, cudaStream_t s) {
  if (cnt <= 0) return;
  {
    ProfScope ps_("k_multidot", s);
    k_multidot<<<cnt, 512, 0, s>>>(V, ldv, N, w, dots);
  }
}

// w <- alpha * (w - sum_{i<cnt} coef[i] V[:, i])  (coef on the device)
__global__ void k_multiaxpy(const double* __restrict__ V, int64_t ldv, int64_t N, int cnt,
                            const double* __restrict__ coef, double* __restrict__ w, double alpha) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x) {
    double acc = w[r];
    for (int i = 0; i < cnt; ++i) acc -= coef[i] * V[r + (int64_t)i * ldv];
    w[r] = alpha * acc;
  }
}

void launch_multiaxpy(const double* V, int64_t ldv, int64_t N, int cnt, const double* coef,
                      double* w, double alpha, cudaStream_t s) {
  int bx = (int)((N + 255) / 256);
  if (bx > 4096) bx = 4096;
  {
    ProfScope ps_("k_multiaxpy", s);
    k_multiaxpy<<<bx, 256, 0, s>>>(V, ldv, N, cnt, coef, w, alpha);
  }
}

#define INST(T)                                                                                 \
  template void launch_trsv_diag<T>(Mat<const T>, int, int, Mat<T>, int, int*, cudaStream_t);   \
  template void launch_trsv_update<T>(Mat<const T>, int, int, Mat<T>, int, cudaStream_t);       \
  template void launch_convert_in<T>(const double*, int64_t, int64_t, int64_t, int,             \
                                     const double*, T*, int64_t, cudaStream_t);                 \
  template void launch_convert_out<T>(const T*, int64_t, int64_t, int, double*, int64_t,        \
                                      cudaStream_t);                                            \
  template void launch_axpy_update<T>(double*, const T*, int64_t, const double*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace luqr
