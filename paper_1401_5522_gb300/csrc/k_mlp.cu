// Decision predictor: per-step features of the panel and a small MLP (16 -> 64 -> 64 -> 1,
// ReLU, logit > 0 means "LU step") with its own forward, gradient (binary cross-entropy
// with logits, mean over the batch) and Adam kernels.  The factorization uses the forward
// pass to start the predicted branch's panel work early; the exact criterion (Eq. 2-4)
// still decides every step.  Nothing here is in the paper.
#include <cuda_runtime.h>

#include "../../include/luqr.h"
#include "internal.cuh"

namespace luqr {
namespace {

constexpr int MF = 16, MH = 64, MP = 5313;
constexpr int O_W1 = 0, O_B1 = 1024, O_W2 = 1088, O_B2 = 5184, O_W3 = 5248, O_B3 = 5312;

struct Act {
  float z1[2], h1[2], z2[2], h2[2];
  float out;
};

// One warp evaluates one sample; lane l owns hidden units l and l + 32.
__device__ __forceinline__ void warp_forward(const float* P, const float* x, Act& a) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int j = lane + 32 * u;
    float s = P[O_B1 + j];
#pragma unroll
    for (int i = 0; i < MF; ++i) s += P[O_W1 + j * MF + i] * x[i];
    a.z1[u] = s;
    a.h1[u] = fmaxf(s, 0.f);
  }
  float s0 = P[O_B2 + lane], s1 = P[O_B2 + lane + 32];
  for (int i = 0; i < MH; ++i) {
    const float hi = __shfl_sync(0xffffffffu, a.h1[i >> 5], i & 31);
    s0 += P[O_W2 + lane * MH + i] * hi;
    s1 += P[O_W2 + (lane + 32) * MH + i] * hi;
  }
  a.z2[0] = s0;
  a.z2[1] = s1;
  a.h2[0] = fmaxf(s0, 0.f);
  a.h2[1] = fmaxf(s1, 0.f);
  float o = P[O_W3 + lane] * a.h2[0] + P[O_W3 + lane + 32] * a.h2[1];
  o = warp_sum_f(o);
  a.out = o + P[O_B3];
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float* __restrict__ params,
                                                     const float* __restrict__ X, float* __restrict__ Y,
                                                     int B) {
  __shared__ float P[MP];
  for (int i = threadIdx.x; i < MP; i += blockDim.x) P[i] = params[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int s = blockIdx.x * nw + warp; s < B; s += gridDim.x * nw) {
    Act a;
    warp_forward(P, X + (int64_t)s * MF, a);
    if ((threadIdx.x & 31) == 0) Y[s] = a.out;
  }
}

// Gradient of the mean binary cross-entropy: each block takes chunks of GB samples, keeps
// their activations and back-propagated errors in shared memory (one warp per sample in
// the forward and backward passes), then forms the parameter gradients as sums over the
// chunk's samples with one thread per parameter (no atomics); a block adds its totals to
// the global gradient once.
constexpr int GB = 64;

__global__ void __launch_bounds__(256) k_mlp_grad(const float* __restrict__ params,
                                                  const float* __restrict__ X,
                                                  const float* __restrict__ lab, int B,
                                                  float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ __align__(16) float sm[];
  float* P = sm;                     // MP
  float* xs = P + MP + 3;            // GB x MF
  float* h1 = xs + GB * MF;          // GB x MH (post-activation)
  float* h2 = h1 + GB * MH;          // GB x MH
  float* d1 = h2 + GB * MH;          // GB x MH (dL/dz1)
  float* d2 = d1 + GB * MH;          // GB x MH (dL/dz2)
  float* dz = d2 + GB * MH;          // GB
  __shared__ float Ls;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = tid; i < MP; i += blockDim.x) P[i] = params[i];
  if (tid == 0) Ls = 0.f;
  const float invB = 1.f / (float)B;
  // per-thread partial sums of the parameters it owns (parameters tid, tid+256, ...)
  constexpr int PPT = (MP + 255) / 256;
  float acc[PPT];
#pragma unroll
  for (int q = 0; q < PPT; ++q) acc[q] = 0.f;
  __syncthreads();
  for (int s0 = blockIdx.x * GB; s0 < B; s0 += gridDim.x * GB) {
    const int cnt = min(GB, B - s0);
    for (int i = tid; i < cnt * MF; i += blockDim.x) xs[i] = X[(int64_t)s0 * MF + i];
    __syncthreads();
    for (int sl = warp; sl < cnt; sl += nw) {
      Act a;
      warp_forward(P, xs + sl * MF, a);
      const float z = a.out, y = lab[s0 + sl];
      const float dzz = (1.f / (1.f + expf(-z)) - y) * invB;
      float dz2v[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int j = lane + 32 * u;
        h1[sl * MH + j] = a.h1[u];
        h2[sl * MH + j] = a.h2[u];
        dz2v[u] = a.z2[u] > 0.f ? dzz * P[O_W3 + j] : 0.f;
        d2[sl * MH + j] = dz2v[u];
      }
      // dL/dh1_i = sum_j W2[j][i] dz2_j, lanes split i
      float dh1[2] = {0.f, 0.f};
      for (int i = 0; i < MH; ++i) {
        float part = P[O_W2 + lane * MH + i] * dz2v[0] + P[O_W2 + (lane + 32) * MH + i] * dz2v[1];
        part = warp_sum_f(part);
        if ((i & 31) == lane) dh1[i >> 5] = part;
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) d1[sl * MH + lane + 32 * u] = a.z1[u] > 0.f ? dh1[u] : 0.f;
      if (lane == 0) {
        dz[sl] = dzz;
        atomicAdd(&Ls, (fmaxf(z, 0.f) - z * y + log1pf(expf(-fabsf(z)))) * invB);
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PPT; ++q) {
      const int p = tid + 256 * q;
      if (p >= MP) break;
      float g = 0.f;
      if (p < O_B1) {                       // W1[j][i] += d1[s][j] x[s][i]
        const int j = p / MF, i = p % MF;
        for (int sl = 0; sl < cnt; ++sl) g += d1[sl * MH + j] * xs[sl * MF + i];
      } else if (p < O_W2) {                // b1[j]
        const int j = p - O_B1;
        for (int sl = 0; sl < cnt; ++sl) g += d1[sl * MH + j];
      } else if (p < O_B2) {                // W2[j][i] += d2[s][j] h1[s][i]
        const int j = (p - O_W2) / MH, i = (p - O_W2) % MH;
        for (int sl = 0; sl < cnt; ++sl) g += d2[sl * MH + j] * h1[sl * MH + i];
      } else if (p < O_W3) {                // b2[j]
        const int j = p - O_B2;
        for (int sl = 0; sl < cnt; ++sl) g += d2[sl * MH + j];
      } else if (p < O_B3) {                // W3[j] += dz[s] h2[s][j]
        const int j = p - O_W3;
        for (int sl = 0; sl < cnt; ++sl) g += dz[sl] * h2[sl * MH + j];
      } else {                              // b3
        for (int sl = 0; sl < cnt; ++sl) g += dz[sl];
      }
      acc[q] += g;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    const int p = tid + 256 * q;
    if (p < MP && acc[q] != 0.f) atomicAdd(&grad[p], acc[q]);
  }
  if (tid == 0 && loss) atomicAdd(loss, Ls);
}

static size_t mlp_grad_smem() {
  return sizeof(float) * (MP + 3 + GB * MF + 4 * GB * MH + GB);
}

__global__ void k_mlp_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                           float* __restrict__ v, int t, float lr, float b1, float b2, float eps) {
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MP; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__device__ __forceinline__ float flog2(double v) {
  return (float)log2(fmax(v, 1e-300));
}

}  // namespace

// Features of step k (16 per step, FP32) computed from the panel statistics that precede
// the criterion and the diagonal of A_kk, and the predicted decision spec[k] (1 = LU):
// mode 1 evaluates the network (params), mode 2 repeats the previous decision, mode 0
// only logs the features.
template <typename T>
__global__ void k_features_spec(const T* __restrict__ W, int64_t ldw, int k, int n, int nb,
                                double alpha, int criterion, const double* __restrict__ norms_k,
                                const unsigned long long* __restrict__ local,
                                const unsigned long long* __restrict__ away,
                                const uint8_t* __restrict__ dec, const double* __restrict__ margin,
                                float* __restrict__ feat, int mode, const float* __restrict__ params,
                                uint8_t* __restrict__ spec) {
  __shared__ float P[MP];
  __shared__ float f[MF];
  const int lane = threadIdx.x & 31;
  if (mode == 1)
    for (int i = threadIdx.x; i < MP; i += blockDim.x) P[i] = params[i];
  if (threadIdx.x < 32) {
    const T* Akk = W + (int64_t)k * nb + (int64_t)k * nb * ldw;
    double lmax = 0.0, lmin = INFINITY, dmax = 0.0, dmin = INFINITY, rmax = -INFINITY, rsum = 0.0;
    for (int j = lane; j < nb; j += 32) {
      const double lj = __longlong_as_double((long long)local[j]);
      const double aj = __longlong_as_double((long long)away[j]);
      const double dj = fabs((double)Akk[(int64_t)j * (ldw + 1)]);
      lmax = fmax(lmax, lj);
      lmin = fmin(lmin, lj);
      dmax = fmax(dmax, dj);
      dmin = fmin(dmin, dj);
      const double r = (lj > 0.0) ? log2(fmax(aj, 1e-300) / lj) : 64.0;
      rmax = fmax(rmax, r);
      rsum += r;
    }
    for (int o = 16; o > 0; o >>= 1) {
      lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
      lmin = fmin(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
      dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      dmin = fmin(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
      rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
      rsum += __shfl_xor_sync(0xffffffffu, rsum, o);
    }
    double nmax = 0.0, nsum = 0.0;
    int nqr = 0;
    for (int i = k + 1 + lane; i < n; i += 32) { nmax = fmax(nmax, norms_k[i]); nsum += norms_k[i]; }
    for (int q = lane; q < k; q += 32) nqr += dec[q] == DEC_QR;
    for (int o = 16; o > 0; o >>= 1) {
      nmax = fmax(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
      nsum += __shfl_xor_sync(0xffffffffu, nsum, o);
      nqr += __shfl_xor_sync(0xffffffffu, nqr, o);
    }
    if (lane == 0) {
      auto cm = [](double m) {
        return (float)(isnan(m) ? 0.0 : fmax(-64.0, fmin(64.0, m)));
      };
      f[0] = flog2(norms_k[k]);
      f[1] = flog2(nmax);
      f[2] = flog2(nsum);
      f[3] = flog2(lmin);
      f[4] = flog2(dmax / fmax(lmax, 1e-300));
      f[5] = flog2(dmin / fmax(lmax, 1e-300));
      f[6] = (float)fmax(-64.0, fmin(64.0, rmax));
      f[7] = (float)fmax(-64.0, fmin(64.0, rsum / nb));
      f[8] = k > 0 ? (float)(dec[k - 1] == DEC_LU) : 0.5f;
      f[9] = k > 0 ? cm(margin[k - 1]) : 0.f;
      f[10] = k > 1 ? cm(margin[k - 2]) : 0.f;
      f[11] = (float)k / (float)n;
      f[12] = isinf(alpha) ? 64.f : flog2(alpha);
      f[13] = flog2((double)(n - k));
      f[14] = (float)criterion / 4.f;
      f[15] = k > 0 ? (float)nqr / (float)k : 0.f;
      if (feat)
        for (int q = 0; q < MF; ++q) feat[(size_t)k * MF + q] = f[q];
      if (mode == 2) spec[k] = k > 0 ? (dec[k - 1] == DEC_LU ? DEC_LU : DEC_QR) : DEC_LU;
    }
  }
  __syncthreads();
  if (mode == 1 && threadIdx.x < 32) {
    Act a;
    warp_forward(P, f, a);
    if (lane == 0) spec[k] = a.out > 0.f ? DEC_LU : DEC_QR;
  }
}

template <typename T>
void launch_features_spec(const T* W, int64_t ldw, int k, int n, int nb, double alpha,
                          int criterion, const double* norms_k, const unsigned long long* local,
                          const unsigned long long* away, const uint8_t* dec, const double* margin,
                          float* feat, int mode, const float* params, uint8_t* spec,
                          cudaStream_t s) {
  ProfScope ps_("k_features_spec", s);
  k_features_spec<T><<<1, 256, 0, s>>>(W, ldw, k, n, nb, alpha, criterion, norms_k, local, away,
                                       dec, margin, feat, mode, params, spec);
}
template void launch_features_spec<float>(const float*, int64_t, int, int, int, double, int,
                                          const double*, const unsigned long long*,
                                          const unsigned long long*, const uint8_t*,
                                          const double*, float*, int, const float*, uint8_t*,
                                          cudaStream_t);
template void launch_features_spec<double>(const double*, int64_t, int, int, int, double, int,
                                           const double*, const unsigned long long*,
                                           const unsigned long long*, const uint8_t*,
                                           const double*, float*, int, const float*, uint8_t*,
                                           cudaStream_t);

// ---------------------------------------------------------------- speculation helpers
// qrfac[k] = QR when the criterion chose QR and the step was not speculated (the panel is
// factored in place); commit[k] = QR when it chose QR and the speculative copy is used.
// lufac[k] = LU when it chose LU and the LU branch was not speculated (the panel's TRSM runs
// in place); lucmt[k] = LU when it chose LU and the speculative TRSM's copy is used.
__global__ void k_spec_resolve(int k, const uint8_t* __restrict__ dec,
                               const uint8_t* __restrict__ spec, uint8_t* __restrict__ qrfac,
                               uint8_t* __restrict__ commit, uint8_t* __restrict__ lufac,
                               uint8_t* __restrict__ lucmt, bool lu_spec) {
  const bool qr = dec[k] == DEC_QR, sp = spec[k] == DEC_QR;
  const bool lu = dec[k] == DEC_LU, splu = lu_spec && spec[k] == DEC_LU;
  qrfac[k] = (qr && !sp) ? DEC_QR : DEC_LU;
  commit[k] = (qr && sp) ? DEC_QR : DEC_LU;
  lufac[k] = (lu && !splu) ? DEC_LU : DEC_QR;
  lucmt[k] = (lu && splu) ? DEC_LU : DEC_QR;
}

void launch_spec_resolve(int k, const uint8_t* dec, const uint8_t* spec, uint8_t* qrfac,
                         uint8_t* commit, uint8_t* lufac, uint8_t* lucmt, bool lu_spec,
                         cudaStream_t s) {
  ProfScope ps_("k_spec_resolve", s);
  k_spec_resolve<<<1, 1, 0, s>>>(k, dec, spec, qrfac, commit, lufac, lucmt, lu_spec);
}

// dst(r, c) = src(r, c) for r < rows, c < cols when gate[k] == want (16-byte vectors when
// both leading dimensions and base addresses allow it).
template <typename T>
__global__ void k_gated_copy(const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                             int64_t ldd, int64_t rows, int cols, const uint8_t* __restrict__ gate,
                             int k, uint8_t want, bool vec) {
  if (gate[k] != want) return;
  const int c = blockIdx.y;
  const T* sc = src + (int64_t)c * lds;
  T* dc = dst + (int64_t)c * ldd;
  constexpr int V = 16 / sizeof(T);
  if (vec) {
    const int64_t nv = rows / V;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv;
         i += (int64_t)gridDim.x * blockDim.x)
      reinterpret_cast<float4*>(dc)[i] = reinterpret_cast<const float4*>(sc)[i];
    for (int64_t r = nv * V + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x)
      dc[r] = sc[r];
  } else {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows;
         r += (int64_t)gridDim.x * blockDim.x)
      dc[r] = sc[r];
  }
}

template <typename T>
void launch_gated_copy(const T* src, int64_t lds, T* dst, int64_t ldd, int64_t rows, int cols,
                       const uint8_t* gate, int k, uint8_t want, const char* name,
                       cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  const bool vec = ((uintptr_t)src % 16 == 0) && ((uintptr_t)dst % 16 == 0) &&
                   ((lds * (int64_t)sizeof(T)) % 16 == 0) && ((ldd * (int64_t)sizeof(T)) % 16 == 0);
  int64_t bx = (rows + 1023) / 1024;
  if (bx > 64) bx = 64;
  ProfScope ps_(name, s);
  k_gated_copy<T><<<dim3((unsigned)bx, (unsigned)cols), 256, 0, s>>>(src, lds, dst, ldd, rows, cols,
                                                                    gate, k, want, vec);
}
template void launch_gated_copy<float>(const float*, int64_t, float*, int64_t, int64_t, int,
                                       const uint8_t*, int, uint8_t, const char*, cudaStream_t);
template void launch_gated_copy<double>(const double*, int64_t, double*, int64_t, int64_t, int,
                                        const uint8_t*, int, uint8_t, const char*, cudaStream_t);

}  // namespace luqr

extern "C" int luqr_mlp_forward(const float* dparams, const float* dX, float* dlogits, int B,
                                void* stream) {
  if (B < 0 || (B > 0 && (!dparams || !dX || !dlogits))) return LUQR_ERR_INVALID;
  if (B == 0) return LUQR_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int blocks = (B + 7) / 8;
  if (blocks > 4096) blocks = 4096;
  {
    luqr::ProfScope ps_("k_mlp_forward", s);
    luqr::k_mlp_forward<<<blocks, 256, 0, s>>>(dparams, dX, dlogits, B);
  }
  return cudaGetLastError() == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}

extern "C" int luqr_mlp_grad(const float* dparams, const float* dX, const float* dlabels, int B,
                             float* dgrad, float* dloss, void* stream) {
  if (!dparams || !dX || !dlabels || !dgrad || B < 1) return LUQR_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int blocks = (B + luqr::GB - 1) / luqr::GB;
  if (blocks > 1024) blocks = 1024;
  {
    const size_t smem = luqr::mlp_grad_smem();
    luqr::ensure_dyn_smem<luqr::k_mlp_grad>(smem);
    luqr::ProfScope ps_("k_mlp_grad", s);
    luqr::k_mlp_grad<<<blocks, 256, smem, s>>>(dparams, dX, dlabels, B, dgrad, dloss);
  }
  return cudaGetLastError() == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}

extern "C" int luqr_mlp_adam(float* dparams, const float* dgrad, float* dm, float* dv, int t,
                             float lr, float beta1, float beta2, float eps, void* stream) {
  if (!dparams || !dgrad || !dm || !dv || t < 1) return LUQR_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  {
    luqr::ProfScope ps_("k_mlp_adam", s);
    luqr::k_mlp_adam<<<(luqr::MP + 255) / 256, 256, 0, s>>>(dparams, dgrad, dm, dv, t, lr, beta1,
                                                              beta2, eps);
  }
  return cudaGetLastError() == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}
