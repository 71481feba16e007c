// LU step, variant A1 (Alg. 2): commit the scratch GETRF into A_kk, Apply (SWPTRSM,
// A_kj <- L^-1 P A_kj), Eliminate (TRSM, A_ik <- A_ik U^-1) and Update (GEMM,
// A_ij <- A_ij - A_ik A_kj).  Every kernel exits at once unless dec[k] selects it.
#include "internal.cuh"

namespace luqr {

template <typename T>
__global__ void k_lu_commit(T* __restrict__ W, int64_t ldw, int k, int nb, const T* __restrict__ S,
                            const int* __restrict__ piv_s, int* __restrict__ piv_k,
                            const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_LU) return;
  T* A = W + (int64_t)k * nb + (int64_t)k * nb * ldw;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < nb * nb; idx += gridDim.x * blockDim.x)
    A[idx % nb + (int64_t)(idx / nb) * ldw] = S[idx];
  if (blockIdx.x == 0)
    for (int r = threadIdx.x; r < nb; r += blockDim.x) piv_k[r] = piv_s[r];
}

template <typename T>
void launch_lu_commit(T* W, int64_t ldw, int k, int nb, const T* S, const int* piv_s, int* piv_k,
                      const uint8_t* dec, cudaStream_t s) {
  {
    ProfScope ps_("k_lu_commit", s);
    k_lu_commit<T><<<(nb * nb + 255) / 256 < 128 ? (nb * nb + 255) / 256 : 128, 256, 0, s>>>(
        W, ldw, k, nb, S, piv_s, piv_k, dec);
  }
}

// ---------------------------------------------------------------- SWPTRSM
// Block = slab of SWW columns of the tile row.  Cs[r][c] (row stride SWW+1).
constexpr int SWW = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_swptrsm(Mat<const T> LU, int nb, const int* __restrict__ piv,
                                                 Mat<T> C, int64_t row0, int64_t c0, int64_t c1,
                                                 const uint8_t* __restrict__ dec, int k) {
  if (dec[k] != DEC_LU) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Cs = reinterpret_cast<T*>(smem_raw);
  int* spiv = reinterpret_cast<int*>(Cs + (size_t)nb * (SWW + 1));
  const int ST = SWW + 1;
  const int64_t cb = c0 + (int64_t)blockIdx.x * SWW;
  const int w = (int)((c1 - cb) < SWW ? (c1 - cb) : SWW);
  const int tid = threadIdx.x;
  for (int r = tid; r < nb; r += blockDim.x) spiv[r] = piv[r];
  for (int idx = tid; idx < nb * w; idx += blockDim.x) {
    int r = idx % nb, c = idx / nb;
    cp_async(&Cs[r * ST + c], &C(row0 + r, cb + c));
  }
  cp_async_wait_all();
  __syncthreads();
  if (tid < w)
    for (int r = 0; r < nb; ++r) {
      int p = spiv[r];
      if (p != r) {
        T t = Cs[r * ST + tid];
        Cs[r * ST + tid] = Cs[p * ST + tid];
        Cs[p * ST + tid] = t;
      }
    }
  __syncthreads();
  const int c = tid & 31, rg = tid >> 5, ng = blockDim.x >> 5;
  for (int r = 0; r < nb - 1; ++r) {
    if (c < w) {
      const T xr = Cs[r * ST + c];
      for (int row = r + 1 + rg; row < nb; row += ng) Cs[row * ST + c] -= LU(row, r) * xr;
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * w; idx += blockDim.x) {
    int r = idx % nb, cc = idx / nb;
    C(row0 + r, cb + cc) = Cs[r * ST + cc];
  }
}

template <typename T>
void launch_swptrsm(Mat<const T> LU, int nb, const int* piv_k, Mat<T> C, int64_t row0, int64_t c0,
                    int64_t c1, const uint8_t* dec, int k, cudaStream_t s) {
  if (c1 <= c0) return;
  const int nblk = (int)((c1 - c0 + SWW - 1) / SWW);
  const size_t smem = (size_t)nb * (SWW + 1) * sizeof(T) + (size_t)nb * sizeof(int);
  ensure_dyn_smem<k_swptrsm<T>>(smem);
  {
    ProfScope ps_("k_swptrsm", s);
    k_swptrsm<T><<<nblk, 256, smem, s>>>(LU, nb, piv_k, C, row0, c0, c1, dec, k);
  }
}

// ---------------------------------------------------------------- L^-1 P (FP32)
// X = L^-1 P (nb x nb, column-major, ld nb) of the committed unit-lower factor of step k,
// so that the Apply of Alg. 2 on a wide tile row becomes one tensor-core product
// A_kj <- X A_kj.  One warp per column of X (two per CTA); the factor's columns come into
// shared memory 8 at a time through cp.async and are shared by the CTA's warps.
constexpr int LI_CH = 8;

__global__ void __launch_bounds__(64) k_lu_inverse(const float* __restrict__ W, int64_t ldw, int k,
                                                   int nb, const int* __restrict__ piv,
                                                   float* __restrict__ X,
                                                   const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_LU) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* ys_all = reinterpret_cast<float*>(smem_raw);          // 2 x nb
  float* colbuf = ys_all + 2 * (size_t)nb;                     // 2 x LI_CH x nb
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c = blockIdx.x * 2 + warp;
  const float* L = W + (int64_t)k * nb + (int64_t)k * nb * ldw;
  float* ys = ys_all + (size_t)warp * nb;
  int pos = c;   // row of the single 1 of column c of P
  for (int r = 0; r < nb; ++r) {
    const int p = piv[r];
    if (pos == r) pos = p;
    else if (pos == p) pos = r;
  }
  for (int row = lane; row < nb; row += 32) ys[row] = (row == pos) ? 1.f : 0.f;
  auto fetch = [&](int first, int slot) {
    float* dst = colbuf + (size_t)slot * LI_CH * nb;
    for (int idx = tid; idx < LI_CH * nb; idx += 64) {
      const int cc = idx / nb, i = idx - cc * nb, col = first + cc;
      if (col < nb) cp_async(&dst[idx], &L[i + (int64_t)col * ldw]);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int nch = nb / LI_CH;
  fetch(0, 0);
  for (int g = 0; g < nch; ++g) {
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    fetch((g + 1) * LI_CH, (g + 1) & 1);
    const float* base = colbuf + (size_t)(g & 1) * LI_CH * nb;
    for (int cc = 0; cc < LI_CH; ++cc) {
      const int r = g * LI_CH + cc;
      if (r >= nb - 1) break;
      __syncwarp();
      const float yr = ys[r];
      if (r < pos || yr == 0.f) continue;
      const float* col = base + (size_t)cc * nb;
      for (int row = r + 1 + lane; row < nb; row += 32) ys[row] -= col[row] * yr;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  for (int row = lane; row < nb; row += 32) X[row + (int64_t)c * nb] = ys[row];
}

void launch_lu_inverse(const float* W, int64_t ldw, int k, int nb, const int* piv_k, float* X,
                       const uint8_t* dec, cudaStream_t s) {
  const size_t smem = sizeof(float) * (2 * (size_t)nb + 2 * LI_CH * (size_t)nb);
  ensure_dyn_smem<k_lu_inverse>(smem);
  ProfScope ps_("k_lu_inverse", s);
  k_lu_inverse<<<nb / 2, 64, smem, s>>>(W, ldw, k, nb, piv_k, X, dec);
}

// ---------------------------------------------------------------- TRSM
// Block = TRB rows of the sub-diagonal panel, all nb columns in shared memory (row
// stride nb+1), U row c staged per column step.
constexpr int TRB = 32;

template <typename T>
__global__ void __launch_bounds__(256) k_trsm(Mat<const T> LU, int nb, Mat<T> X, int64_t r0,
                                              int64_t r1, int64_t xc, const uint8_t* __restrict__ dec,
                                              int k) {
  if (dec[k] != DEC_LU) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xs = reinterpret_cast<T*>(smem_raw);
  T* Us = Xs + TRB * (nb + 1);
  const int ST = nb + 1;
  const int64_t rb = r0 + (int64_t)blockIdx.x * TRB;
  const int h = (int)((r1 - rb) < TRB ? (r1 - rb) : TRB);
  const int tid = threadIdx.x;
  for (int idx = tid; idx < TRB * nb; idx += blockDim.x) {
    int r = idx % TRB, c = idx / TRB;
    if (r < h) cp_async(&Xs[r * ST + c], &X(rb + r, xc + c));
    else Xs[r * ST + c] = (T)0;
  }
  cp_async_wait_all();
  __syncthreads();
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < nb; ++c) {
    for (int j = c + tid; j < nb; j += blockDim.x) Us[j] = LU(c, j);
    __syncthreads();
    if (tid < TRB) Xs[tid * ST + c] = Xs[tid * ST + c] / Us[c];
    __syncthreads();
    for (int r = warp; r < TRB; r += nw) {
      const T xv = Xs[r * ST + c];
      for (int j = c + 1 + lane; j < nb; j += 32) Xs[r * ST + j] -= xv * Us[j];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < TRB * nb; idx += blockDim.x) {
    int r = idx % TRB, c = idx / TRB;
    if (r < h) X(rb + r, xc + c) = Xs[r * ST + c];
  }
}

template <typename T>
void launch_trsm(Mat<const T> LU, int nb, Mat<T> X, int64_t r0, int64_t r1, int64_t xc,
                 const uint8_t* dec, int k, cudaStream_t s) {
  if (r1 <= r0) return;
  const int nblk = (int)((r1 - r0 + TRB - 1) / TRB);
  const size_t smem = ((size_t)TRB * (nb + 1) + nb) * sizeof(T);
  ensure_dyn_smem<k_trsm<T>>(smem);
  {
    ProfScope ps_("k_trsm", s);
    k_trsm<T><<<nblk, 256, smem, s>>>(LU, nb, X, r0, r1, xc, dec, k);
  }
}

// ---------------------------------------------------------------- GEMM update
// C[M x Ncols] -= A[M x K] B[K x Ncols]; register-tiled, BK-deep shared-memory stages.
template <typename T>
struct GemmCfg;
template <>
struct GemmCfg<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };
template <>
struct GemmCfg<float> { static constexpr int BM = 128, BN = 128, BK = 8, TM = 8, TN = 8; };

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_update(Mat<const T> A, Mat<const T> B, Mat<T> C,
                                                     int64_t M, int64_t Ncols, int K,
                                                     const uint8_t* __restrict__ dec, int k,
                                                     uint8_t want) {
  if (dec[k] != want) return;
  using G = GemmCfg<T>;
  constexpr int BM = G::BM, BN = G::BN, BK = G::BK, TM = G::TM, TN = G::TN;
  __shared__ T As[2][BK][BM];
  __shared__ T Bs[2][BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = (T)0;

  auto load = [&](int buf, int kb) {
    for (int idx = tid; idx < BM * BK; idx += 256) {
      int r = idx % BM, kk = idx / BM;
      int64_t gr = m0 + r;
      int gk = kb + kk;
      As[buf][kk][r] = (gr < M && gk < K) ? A(gr, gk) : (T)0;
    }
    for (int idx = tid; idx < BN * BK; idx += 256) {
      int kk = idx % BK, c = idx / BK;
      int64_t gc = n0 + c;
      int gk = kb + kk;
      Bs[buf][kk][c] = (gc < Ncols && gk < K) ? B(gk, gc) : (T)0;
    }
  };
  load(0, 0);
  __syncthreads();
  int buf = 0;
  for (int kb = 0; kb < K; kb += BK) {
    if (kb + BK < K) load(buf ^ 1, kb + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    int64_t gc = n0 + tx * TN + j;
    if (gc >= Ncols) continue;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      int64_t gr = m0 + ty * TM + i;
      if (gr < M) C(gr, gc) -= acc[i][j];
    }
  }
}

template <typename T>
void launch_gemm_update(Mat<const T> A, Mat<const T> B, Mat<T> C, int64_t M, int64_t Ncols, int K,
                        const uint8_t* dec, int k, uint8_t want, cudaStream_t s) {
  if (M <= 0 || Ncols <= 0) return;
  using G = GemmCfg<T>;
  dim3 grid((unsigned)((Ncols + G::BN - 1) / G::BN), (unsigned)((M + G::BM - 1) / G::BM));
  {
    ProfScope ps_("k_gemm_update", s);
    k_gemm_update<T><<<grid, 256, 0, s>>>(A, B, C, M, Ncols, K, dec, k, want);
  }
}

#define INST(T)                                                                                   \
  template void launch_lu_commit<T>(T*, int64_t, int, int, const T*, const int*, int*,            \
                                    const uint8_t*, cudaStream_t);                                \
  template void launch_swptrsm<T>(Mat<const T>, int, const int*, Mat<T>, int64_t, int64_t,        \
                                  int64_t, const uint8_t*, int, cudaStream_t);                    \
  template void launch_trsm<T>(Mat<const T>, int, Mat<T>, int64_t, int64_t, int64_t,              \
                               const uint8_t*, int, cudaStream_t);                                \
  template void launch_gemm_update<T>(Mat<const T>, Mat<const T>, Mat<T>, int64_t, int64_t, int,  \
                                      const uint8_t*, int, uint8_t, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace luqr
