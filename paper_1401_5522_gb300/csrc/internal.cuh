// Internal declarations of the hybrid LU-QR library (not part of the C interface).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include <mutex>

#include "smem_record.h"

namespace luqr {

constexpr int IB = 32;              // inner block of the Householder kernels (T is IB x IB per block)
constexpr int NT = 256;             // threads of the tile kernels
constexpr int SMEM_MAX = 232448;    // opt-in dynamic shared memory per block (227 KB)

enum : uint8_t { DEC_QR = 0, DEC_LU = 1, DEC_ABORT = 2 };

// Device status word of a handle: {code, step, row, nonfinite, zero_row, ...}
enum { ST_CODE = 0, ST_STEP = 1, ST_ROW = 2, ST_NONFINITE = 3, ST_ZERO_ROW = 4, ST_WORDS = 8 };

// A column-major matrix view.
template <typename T>
struct Mat {
  T* p;
  int64_t ld;
  __host__ __device__ T& operator()(int64_t r, int64_t c) const { return p[r + c * ld]; }
};

// Rows [i0 + t*istride, +nb) for t < count; eliminator rows i - eoff.
struct TileList {
  int i0, istride, count, eoff;
};

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v);
template <>
__device__ __forceinline__ double warp_sum<double>(double v) { return warp_sum_d(v); }
template <>
__device__ __forceinline__ float warp_sum<float>(float v) { return warp_sum_f(v); }

__device__ __forceinline__ double warp_max_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over the whole block (blockDim.x multiple of 32); result valid in every thread.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red /* >= 32 */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum<T>(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = (T)0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// Asynchronous global -> shared copy of one element (cp.async, no register staging);
// many copies stay in flight per thread until cp_async_wait_all().
template <typename T>
__device__ __forceinline__ void cp_async(T* smem_dst, const T* gsrc) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem_dst);
  if constexpr (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(saddr), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Raises kernel K's dynamic shared-memory limit to `bytes` when a launch needs more than
// the limit already set on the current device (the record is per device and locked:
// smem_record.h).  The request is the launch's own size, so kernels that also use static
// shared memory stay within the per-block maximum.
template <auto K>
inline void ensure_dyn_smem(size_t bytes) {
  static SmemRecord rec;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  rec.ensure(dev, bytes, [](size_t b) {
    return cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) ==
           cudaSuccess;
  });
}

// ---------------------------------------------------------------- launch profiler
void prof_begin(const char* name, cudaStream_t s);
void prof_end(cudaStream_t s);
struct ProfScope {
  cudaStream_t s;
  ProfScope(const char* name, cudaStream_t st) : s(st) { prof_begin(name, st); }
  ~ProfScope() { prof_end(s); }
};

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_pack(const double* A, int64_t lda, const double* b, int64_t N, int64_t Npad,
                 int64_t Wc, T* W, int64_t ldw, cudaStream_t s);
template <typename T>
void launch_scale_rows(T* W, int64_t ldw, int64_t row0, int rows, int64_t col0, int64_t col1,
                       double scale, cudaStream_t s);
template <typename T>
void launch_panel_stats(const T* W, int64_t ldw, int k, int n, int nb, double* norms_k,
                        unsigned long long* local, unsigned long long* away, int* status,
                        cudaStream_t s);
template <typename T>
void launch_getrf(const T* W, int64_t ldw, int k, int nb, T* S, int* piv_s, int* status,
                  cudaStream_t s);
template <typename T>
void launch_invnorm(const T* S, int nb, const int* piv_s, double* colsum, const int* status,
                    cudaStream_t s);
template <typename T>
void launch_invnorm_est(const T* S, int nb, const int* piv_s, double* colsum, const int* status,
                        cudaStream_t s);

struct DecideArgs {
  int k, n, nb, criterion, mumps_mode;
  double alpha;
  const double* norms_k;             // indexed by tile row i
  const double* colsum;              // nb column sums of |A_kk^-1|
  const unsigned long long* local;   // nb column maxima of |A_kk| (double bits)
  const unsigned long long* away;    // nb column maxima of |A_ik|, i > k (double bits)
  const uint8_t* forced;             // device, may be null
  uint8_t* dec;
  double* margin;
  double* lhs;
  double* rhs;
  int* status;
  unsigned long long seed;           // LUQR_RANDOM draws
};
template <typename T>
void launch_decide(const DecideArgs& a, const T* S, cudaStream_t s);

template <typename T>
void launch_lu_commit(T* W, int64_t ldw, int k, int nb, const T* S, const int* piv_s,
                      int* piv_k, const uint8_t* dec, cudaStream_t s);
// C rows [row0, row0+nb), columns [c0, c1) <- L^-1 P C with L, P of the LU-factored tile LU.
template <typename T>
void launch_swptrsm(Mat<const T> LU, int nb, const int* piv_k, Mat<T> C, int64_t row0, int64_t c0,
                    int64_t c1, const uint8_t* dec, int k, cudaStream_t s);
// X rows [r0, r1), columns [xc, xc+nb) <- X U^-1.
template <typename T>
void launch_trsm(Mat<const T> LU, int nb, Mat<T> X, int64_t r0, int64_t r1, int64_t xc,
                 const uint8_t* dec, int k, cudaStream_t s);
// C[r0:r1, c0:c1] -= A[r0:r1, 0:K] * B[0:K, c0:c1]   (A, B given at their (r0,0)/(0,c0) origins)
template <typename T>
void launch_gemm_update(Mat<const T> A, Mat<const T> B, Mat<T> C, int64_t M, int64_t Ncols, int K,
                        const uint8_t* dec, int k, uint8_t want, cudaStream_t s);

// QR kernels; the V tiles live in the factored panel column kc of F.
template <typename T>
void launch_geqrt(Mat<T> F, int k, int nb, TileList tl, T* Tk, int n, const uint8_t* dec,
                  cudaStream_t s);
template <typename T>
void launch_unmqr(Mat<const T> F, int k, int nb, TileList tl, const T* Tk, int n, Mat<T> C,
                  int64_t c0, int64_t c1, const uint8_t* dec, cudaStream_t s);
template <typename T>
void launch_pair_qrt(Mat<T> F, int k, int nb, TileList tl, bool tri, T* Tk, int n,
                     const uint8_t* dec, cudaStream_t s);
template <typename T>
void launch_pair_apply(Mat<const T> F, int k, int nb, TileList tl, bool tri, const T* Tk, int n,
                       Mat<T> C, int64_t c0, int64_t c1, const uint8_t* dec, cudaStream_t s);

// Tensor-core (tcgen05, 3xTF32) contraction D = A B (FP32 in, FP32 accumulate) with a
// batch index z: operand t of the batch starts at base + t * stride (elements).
enum { TC_MASK_NONE = 0, TC_MASK_UNIT_LOWER = 1, TC_MASK_UPPER = 2 };
enum { TC_EPI_SUB = 0, TC_EPI_OUT = 1, TC_EPI_ADD_OUT = 2 };   // C -= D | C = D | C = D + C1
struct TcArgs {
  const float* A; int64_t lda; int64_t sA; int a_trans; int a_mask;
  const float* B; int64_t ldb; int64_t sB; int b_trans; int b_mask;
  float* C; int64_t ldc; int64_t sC;
  const float* C1; int64_t ldc1; int64_t sC1;
  int64_t M, N; int K; int epi;
  const uint8_t* dec; int k_step; uint8_t want;
  int* status;
  const unsigned char* Apk; int64_t sApk;   // packed A (launch_tc2)
  // packed A known to be triangular (exact zeros): 1 lower (A[m][q] = 0 for q > m), 2 upper
  // (A[m][q] = 0 for q < m); the persistent kernel skips the products of zero blocks
  int a_tri;
  // the C (EPI_SUB) or C1 (EPI_ADD_OUT) blocks an epilogue reads may be brought into shared
  // memory by bulk copies (set by launch_tc2 when every column segment is 16-byte aligned)
  int c_bulk;
  // budget of each bounded wait of the persistent kernel in clock cycles (0: the default,
  // about 0.5 s)
  long long wait_cycles;
};
// Test hook of the persistent tensor-core kernel: while >= 0, CTA 0 of every launch does not
// signal the arrival of its raw B chunk with this index, so the converters' wait on it runs
// out (see luqr_debug_tc_skip).
void tc_set_debug_skip(int chunk);
void launch_tc(const TcArgs& a, int batch, const char* name, cudaStream_t s);
// Packed-A form: pack A once (launch_tc_pack), then launch_tc2 with a.Apk/a.sApk set.
size_t tc_packed_bytes(int64_t M, int K);
void launch_tc_pack(const float* A, int64_t lda, int64_t sA, int a_trans, int a_mask, int64_t M,
                    int K, unsigned char* Apk, int64_t sApk, int batch, const uint8_t* dec, int k,
                    uint8_t want, cudaStream_t s);
void launch_tc2(const TcArgs& a, int batch, const char* name, cudaStream_t s);
void launch_tfull(const float* G, int64_t sG, const float* Tslots, int64_t sT, float* Tf,
                  int64_t sTf, int nb, int batch, const uint8_t* dec, int k, cudaStream_t s);
// C[M x N] -= A[M x K] B[K x N], FP32 column-major (single matrix).
void launch_gemm_tc(const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                    int64_t ldc, int64_t M, int64_t N, int K, const uint8_t* dec, int k,
                    uint8_t want, int* status, cudaStream_t s);

// Solves and refinement helpers.
template <typename T>
void launch_trsv_diag(Mat<const T> U, int k, int nb, Mat<T> X, int nrhs, int* status,
                      cudaStream_t s);
template <typename T>
void launch_trsv_update(Mat<const T> U, int k, int nb, Mat<T> X, int nrhs, cudaStream_t s);
template <typename T>
void launch_convert_in(const double* src, int64_t lds, int64_t N, int64_t Npad, int nrhs,
                       const double* scale, T* dst, int64_t ldd, cudaStream_t s);
template <typename T>
void launch_convert_out(const T* src, int64_t lds, int64_t N, int nrhs, double* dst, int64_t ldd,
                        cudaStream_t s);
void launch_residual(const double* A, int64_t lda, int64_t N, const double* x, const double* b,
                     double* r, double* partial, int nchunk, cudaStream_t s);
void launch_row_abs_sum_max(const double* A, int64_t lda, int64_t N, double* partial, int nchunk,
                            double* out, cudaStream_t s);
void launch_vec_absmax(const double* v, int64_t N, double* out, cudaStream_t s);
template <typename T>
void launch_axpy_update(double* x, const T* d, int64_t N, const double* scale, cudaStream_t s);
void launch_matvec(const double* A, int64_t lda, int64_t N, const double* v, double* out,
                   double* partial, int nchunk, cudaStream_t s);
void launch_multidot(const double* V, int64_t ldv, int64_t N, int cnt, const double* w,
                     double* dots, cudaStream_t s);
void launch_multiaxpy(const double* V, int64_t ldv, int64_t N, int cnt, const double* coef,
                      double* w, double alpha, cudaStream_t s);

// X = L^-1 P of an LU step's committed factor (k_lu.cu, FP32).
void launch_lu_inverse(const float* W, int64_t ldw, int k, int nb, const int* piv_k, float* X,
                       const uint8_t* dec, cudaStream_t s);

// Single-vector second pass in one persistent launch (k_replay.cu).  Task types; rows i
// (and e for pairs) are written, row r (GEMV) is read; ni / ne / nr are the numbers of
// earlier writes of those rows to wait for.
constexpr int LUQR_TIMEOUT_CODE = -6;   // LUQR_ERR_TIMEOUT
// RT_GEMV_TRSV: x_i -= A_{i,k} x_k (k = i + 1, the last update of row i in the back
// substitution) and then x_i <- U_ii^-1 x_i, in one task (the chain of the back substitution
// then takes one task per tile row instead of two).
enum : int { RT_SCALE = 0, RT_SINGLE = 1, RT_PAIR_TS = 2, RT_PAIR_TT = 3, RT_LUAPPLY = 4,
             RT_GEMV = 5, RT_TRSV = 6, RT_GEMV_TRSV = 7 };
struct ReplayTask {
  int type, k, i, e, r, ni, ne, nr;
  int gate;              // 0 always; 1 only if dec[k] = QR; 2 only if dec[k] = LU (a task whose
                         // branch was not taken still waits and signals, as a no-op)
};
template <typename T>
struct ReplayArgs {
  const T* W;            // factored workspace (column-major, leading dimension ld)
  int64_t ld;
  const T* Tbuf;         // T blocks, t_step elements per step
  size_t t_step;
  const int* piv_all;    // n x nb pivots of the LU steps
  const uint8_t* dec;    // decisions of the factorization
  T* x;                  // Npad vector, transformed in place
  const ReplayTask* tasks;
  int ntasks, nb;
  int* ctl;              // [0] next task, [1] abort flag (zero before the launch)
  int* done;             // n completed-write counters (zero before the launch)
  int* status;
  long long budget;      // clock64 cycles a wait may last
  int skip_signal;       // test hook: this task does not signal its completion (-1: none)
};
template <typename T>
bool replay_fits(int nb);
template <typename T>
void launch_replay(const ReplayArgs<T>& a, int grid, cudaStream_t s);
template <typename T>
int replay_blocks_per_sm(int nb);

// Diagonal-domain pivoting (k_domain.cu): tall GETRF of the rows x nb domain of panel k
// (exchanges to dpiv, identity to piv_s, zero pivot to the status word), the pivoted copy of
// panel k the criterion reads, and the exchanges on columns [c0, c1) of an LU step.
template <typename T>
void launch_getrf_tall(const T* W, int64_t ld, int k, int nb, int rows, T* St, int* dpiv,
                       int* piv_s, int* status, cudaStream_t s);
template <typename T>
void launch_domain_panel(const T* W, int64_t ld, int k, int nb, int rows, int64_t Npad,
                         const int* dpiv, T* P, int64_t ldp, cudaStream_t s);
template <typename T>
void launch_domain_swap(T* M, int64_t ld, int k, int nb, int rows, int64_t c0, int64_t c1,
                        const int* dpiv, const uint8_t* dec, cudaStream_t s);

// LU step variant A2 (k_a2.cu): identity pivots and R's first zero diagonal entry; the
// gate that lets the QR-gated UNMQR run on A2 LU steps; columns of Q^T (mode 1, to X) or the
// column sums of |R^-1 Q^T| (mode 0, to colsum) from GEQRT factors (leading dimension lds).
template <typename T>
void launch_a2_prep(const T* S, int nb, int* piv, int* status, cudaStream_t s);
void launch_a2_gate(const uint8_t* dec, uint8_t* gate, int k, cudaStream_t s);
template <typename T>
void launch_qt_cols(const T* S, int64_t lds, int nb, const T* Tslot, int mode, double* colsum,
                    T* X, const int* status, const uint8_t* gate, int k, cudaStream_t s);

// Decision predictor and speculation helpers (k_mlp.cu).
template <typename T>
void launch_features_spec(const T* W, int64_t ldw, int k, int n, int nb, double alpha,
                          int criterion, const double* norms_k, const unsigned long long* local,
                          const unsigned long long* away, const uint8_t* dec, const double* margin,
                          float* feat, int mode, const float* params, uint8_t* spec,
                          cudaStream_t s);
// After the decision of step k: qrfac / commit as below for QR; lufac[k] = LU when LU was
// chosen and not speculated (TRSM in place), lucmt[k] = LU when LU was chosen and the
// speculative TRSM on the shadow copy is committed (lu_spec: the LU branch is speculated).
void launch_spec_resolve(int k, const uint8_t* dec, const uint8_t* spec, uint8_t* qrfac,
                         uint8_t* commit, uint8_t* lufac, uint8_t* lucmt, bool lu_spec,
                         cudaStream_t s);
template <typename T>
void launch_gated_copy(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int cols,
                       const uint8_t* gate, int k, uint8_t want, const char* name, cudaStream_t s);

}  // namespace luqr
