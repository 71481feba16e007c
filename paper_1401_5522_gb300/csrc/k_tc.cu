// Blackwell (sm_103a) tensor-core GEMM update C <- C - A B for FP32 matrices, the dense
// contraction of the trailing updates (Alg. 2 GEMM; QR updates expressed as GEMMs).
//
// FP32 operands are split 3xTF32 (x = hi + lo, hi = tf32(x), lo = tf32(x - hi)) while
// they are staged into shared memory, and each K=8 slice issues three tcgen05.mma
// kind::tf32 instructions (lo*hi, hi*lo, hi*hi) accumulating in FP32 in tensor memory
// (TMEM).  One CTA computes a 128 x 128 tile of C; K is consumed in 32-wide chunks,
// double-buffered: while the MMAs of chunk c run, the CTA stages chunk c+1.
//
// Shared-memory operand layout: K-major, no swizzle.  A "core matrix" is 8 rows x 16
// bytes (4 FP32 along K, 128 contiguous bytes); element (r, k) of a 128 x 32 chunk lives
// at (r/8)*SBO + (k/4)*LBO + (r%8)*16 + (k%4)*4 with LBO = 128 B (next core matrix along
// K) and SBO = 1024 B (next 8-row group).  MMA k-step s starts 2*LBO*s bytes in.
//
// Every wait on an mbarrier is bounded; on expiry the kernel records LUQR_ERR_TIMEOUT in
// the status word, waits (bounded) for its own MMAs, frees its TMEM and returns.
#include <algorithm>
#include <atomic>

#include "internal.cuh"

namespace luqr {

constexpr int TC_BM = 128;      // rows of a C tile (MMA M)
constexpr int TC_BN = 128;      // columns of a C tile (MMA N)
constexpr int TC_BK = 32;       // K chunk
constexpr int TC_THREADS = 256;
constexpr uint32_t TC_LBO = 128;
constexpr uint32_t TC_SBO = 1024;
constexpr int TC_CHUNK_BYTES = TC_BM * TC_BK * 4;           // 16 KB per operand copy
constexpr int TC_STAGE_BYTES = 4 * TC_CHUNK_BYTES;          // A hi/lo + B hi/lo
constexpr int TC_SMEM = 2 * TC_STAGE_BYTES + 128;           // two stages + barriers/TMEM addr
constexpr long long TC_SPIN_LIMIT = 20000000;               // bounded mbarrier polling

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;   // descriptor version for tcgen05
  return d;                 // base offset 0, no swizzle
}

// Instruction descriptor, kind::tf32: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

// Returns true once the phase with the given parity has completed; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long it = 0; it < TC_SPIN_LIMIT; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Epilogue of 32 consecutive columns gc0.. of one row: all loads of the row segment are
// issued before any store, so a thread keeps 32 independent loads in flight.
__device__ __forceinline__ void tc_epi32(const TcArgs& a, float* C, const float* C1, int64_t row,
                                         int64_t gc0, const float* v) {
  if (row >= a.M || gc0 >= a.N) return;
  const int64_t lim = a.N - gc0;
  float* Cr = C + row + gc0 * a.ldc;
  if (a.epi == TC_EPI_OUT) {
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < lim) Cr[(int64_t)i * a.ldc] = v[i];
    return;
  }
  float old[32];
  if (a.epi == TC_EPI_SUB) {
#pragma unroll
    for (int i = 0; i < 32; ++i) old[i] = (i < lim) ? Cr[(int64_t)i * a.ldc] : 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < lim) Cr[(int64_t)i * a.ldc] = old[i] - v[i];
  } else {
    const float* C1r = C1 + row + gc0 * a.ldc1;
#pragma unroll
    for (int i = 0; i < 32; ++i) old[i] = (i < lim) ? C1r[(int64_t)i * a.ldc1] : 0.f;
#pragma unroll
    for (int i = 0; i < 32; ++i)
      if (i < lim) Cr[(int64_t)i * a.ldc] = v[i] + old[i];
  }
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
  return (uint32_t)((r >> 3) * TC_SBO + (k >> 2) * TC_LBO + (r & 7) * 16 + (k & 3) * 4);
}

// Element of a (possibly transposed, possibly masked) operand.  The mask refers to the
// source matrix P's own row/column (pr, pc): unit-lower keeps pr > pc, puts 1 on the
// diagonal and 0 above (Householder V of GEQRT); upper keeps pr <= pc (V of TTQRT).
__device__ __forceinline__ float tc_fetch(const float* P, int64_t ld, int64_t pr, int64_t pc,
                                          int mask) {
  if (mask == TC_MASK_UNIT_LOWER) {
    if (pr == pc) return 1.f;
    if (pr < pc) return 0.f;
  } else if (mask == TC_MASK_UPPER) {
    if (pr > pc) return 0.f;
  }
  return P[pr + pc * ld];
}

__device__ __forceinline__ void tc_put(unsigned char* hi, unsigned char* lo, uint32_t off, float x) {
  const uint32_t h = tf32_bits(x);
  const uint32_t l = tf32_bits(x - __uint_as_float(h));
  *reinterpret_cast<uint32_t*>(hi + off) = h;
  *reinterpret_cast<uint32_t*>(lo + off) = l;
}

// Stages chunk [k0, k0 + 32) of the logical operands A (M x K) and B (K x N) into one
// stage of shared memory as hi/lo TF32 copies (zero outside the matrices).  All 32 global
// loads of a thread are issued before its shared-memory stores.
__device__ __forceinline__ void tc_stage(unsigned char* st, const TcArgs& a, const float* A,
                                         const float* B, int64_t m0, int64_t n0, int k0) {
  constexpr int PER = TC_BM * TC_BK / TC_THREADS;
  static_assert(TC_BN == TC_BM && PER * TC_THREADS == TC_BM * TC_BK, "staging map");
  unsigned char* ahi = st;
  unsigned char* alo = st + TC_CHUNK_BYTES;
  unsigned char* bhi = st + 2 * TC_CHUNK_BYTES;
  unsigned char* blo = st + 3 * TC_CHUNK_BYTES;
  float xa[PER], xb[PER];
  uint32_t oa[PER], ob[PER];
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int idx = threadIdx.x + u * TC_THREADS;
    int r, k;
    if (!a.a_trans) { r = idx % TC_BM; k = idx / TC_BM; }   // consecutive threads walk m
    else { k = idx % TC_BK; r = idx / TC_BK; }             // consecutive threads walk k
    const int64_t gr = m0 + r;
    const int gk = k0 + k;
    xa[u] = (gr < a.M && gk < a.K) ? (a.a_trans ? tc_fetch(A, a.lda, gk, gr, a.a_mask)
                                                : tc_fetch(A, a.lda, gr, gk, a.a_mask))
                                   : 0.f;
    oa[u] = kmajor_off(r, k);
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) {
    const int idx = threadIdx.x + u * TC_THREADS;
    int c, k;
    if (!a.b_trans) { k = idx % TC_BK; c = idx / TC_BK; }   // consecutive threads walk k
    else { c = idx % TC_BN; k = idx / TC_BN; }             // consecutive threads walk n
    const int64_t gc = n0 + c;
    const int gk = k0 + k;
    xb[u] = (gc < a.N && gk < a.K) ? (a.b_trans ? tc_fetch(B, a.ldb, gc, gk, a.b_mask)
                                                : tc_fetch(B, a.ldb, gk, gc, a.b_mask))
                                   : 0.f;
    ob[u] = kmajor_off(c, k);
  }
#pragma unroll
  for (int u = 0; u < PER; ++u) tc_put(ahi, alo, oa[u], xa[u]);
#pragma unroll
  for (int u = 0; u < PER; ++u) tc_put(bhi, blo, ob[u], xb[u]);
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc(TcArgs a) {
  if (a.dec != nullptr && a.dec[a.k_step] != a.want) return;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  unsigned char* stages = smem_tc;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_tc + 2 * TC_STAGE_BYTES);   // 2 barriers
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(smem_tc + 2 * TC_STAGE_BYTES + 64);
  int* last_commit = reinterpret_cast<int*>(smem_tc + 2 * TC_STAGE_BYTES + 96);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.y * TC_BM, n0 = (int64_t)blockIdx.x * TC_BN;
  const int64_t t = blockIdx.z;
  const float* A = a.A + t * a.sA;
  const float* B = a.B + t * a.sB;
  float* C = a.C + t * a.sC;
  const float* C1 = a.C1 ? a.C1 + t * a.sC1 : nullptr;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(taddr_slot)),
                 "r"(TC_BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    *last_commit = -1;
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_slot;
  const uint32_t idesc = make_idesc_tf32(TC_BM, TC_BN);
  const int nchunks = (a.K + TC_BK - 1) / TC_BK;
  bool ok = true;
  for (int c = 0; c < nchunks; ++c) {
    const int buf = c & 1;
    unsigned char* st = stages + buf * TC_STAGE_BYTES;
    if (c >= 2) {   // the MMAs that read this stage two chunks ago must be done
      if (!mbar_wait(&bars[buf], (uint32_t)(((c - 2) >> 1) & 1))) ok = false;
    }
    if (!__syncthreads_and(ok ? 1 : 0)) { ok = false; break; }
    tc_stage(st, a, A, B, m0, n0, c * TC_BK);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const uint32_t base = smem_u32(st);
#pragma unroll
      for (int s = 0; s < TC_BK / 8; ++s) {
        const uint32_t koff = (uint32_t)s * 2 * TC_LBO;
        const uint64_t ahi = make_desc(base + koff);
        const uint64_t alo = make_desc(base + TC_CHUNK_BYTES + koff);
        const uint64_t bhi = make_desc(base + 2 * TC_CHUNK_BYTES + koff);
        const uint64_t blo = make_desc(base + 3 * TC_CHUNK_BYTES + koff);
        const uint32_t acc0 = (c > 0 || s > 0) ? 1u : 0u;
        tc_mma(tmem, alo, bhi, idesc, acc0);
        tc_mma(tmem, ahi, blo, idesc, 1u);
        tc_mma(tmem, ahi, bhi, idesc, 1u);
      }
      tc_commit(&bars[buf]);
      *last_commit = c;
    }
  }
  // Wait for the last committed chunk's MMAs (a commit covers every earlier MMA of the
  // thread), also on the error path, so TMEM is released only when no MMA is in flight.
  __syncthreads();
  const int last = *last_commit;
  if (last >= 0) {
    if (!mbar_wait(&bars[last & 1], (uint32_t)((last >> 1) & 1))) ok = false;
  }
  tc_fence_after();
  const bool all_ok = __syncthreads_and(ok ? 1 : 0);
  if (all_ok) {
    // Epilogue: warp w reads TMEM lanes 32*(w%4).. (rows), columns half (w/4) of the tile.
    const int lane_base = (warp & 3) * 32;
    const int col_half = warp >> 2;
    const int64_t row = m0 + lane_base + lane;
    for (int cc = 0; cc < TC_BN / 2; cc += 32) {
      const int col0 = col_half * (TC_BN / 2) + cc;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)col0, v);
      tc_epi32(a, C, C1, row, n0 + col0, v);
    }
  } else if (tid == 0 && a.status != nullptr) {
    atomicCAS(&a.status[ST_CODE], 0, -6);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_BN));
  }
}

void launch_tc(const TcArgs& a, int batch, const char* name, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0 || batch <= 0) return;
  ensure_dyn_smem<k_gemm_tc>(TC_SMEM);
  dim3 grid((unsigned)((a.N + TC_BN - 1) / TC_BN), (unsigned)((a.M + TC_BM - 1) / TC_BM),
            (unsigned)batch);
  {
    ProfScope ps_(name, s);
    k_gemm_tc<<<grid, TC_THREADS, TC_SMEM, s>>>(a);
  }
}

void launch_gemm_tc(const float* A, int64_t lda, const float* B, int64_t ldb, float* C,
                    int64_t ldc, int64_t M, int64_t N, int K, const uint8_t* dec, int k,
                    uint8_t want, int* status, cudaStream_t s) {
  TcArgs a{};
  a.A = A; a.lda = lda; a.B = B; a.ldb = ldb; a.C = C; a.ldc = ldc;
  a.M = M; a.N = N; a.K = K; a.epi = TC_EPI_SUB;
  a.dec = dec; a.k_step = k; a.want = want; a.status = status;
  launch_tc(a, 1, "k_gemm_tc", s);
}

// ---------------------------------------------------------------- packed-A pipeline
// Second form of the contraction for operands shared by many output tiles (the V^T,
// V T^T and T^T tiles of a QR step): A is packed once into K-major no-swizzle core-matrix
// blocks (128 rows x 16 K, hi and lo TF32, 16 KB per block) and every CTA brings its
// blocks in with TMA bulk copies (cp.async.bulk, completion tracked by the mbarrier's
// transaction count).  The CTA tile is 256 x 256 (two M=128 accumulators, all 512 TMEM
// columns); K advances in 16-wide chunks through a 3-stage ring.
constexpr int P_BK = 16;
constexpr int P_BN = 256;
constexpr int P_STAGES = 3;
constexpr int P_ABLK = 128 * P_BK * 4;                 // 8 KB per hi or lo copy
constexpr int P_ASTAGE = 2 * 2 * P_ABLK;               // two M-halves x (hi, lo) = 32 KB
constexpr int P_BSTAGE = 2 * P_BN * P_BK * 4;          // hi + lo = 32 KB
constexpr int P_STAGE = P_ASTAGE + P_BSTAGE;           // 64 KB
constexpr int P_SMEM = P_STAGES * P_STAGE + 256;
constexpr uint32_t P_SBO = (P_BK / 4) * 128;           // 512 B between 8-row groups

__device__ __forceinline__ uint64_t make_desc_sbo(uint32_t saddr, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ uint32_t kmajor_off16(int r, int k) {
  return (uint32_t)((r >> 3) * P_SBO + (k >> 2) * TC_LBO + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Packs the logical operand A (M x K; transposed / masked like tc_fetch) of every batch item
// into blocks: block (mb, kc) of item t starts at Apk + t*sApk + (mb*nK + kc)*2*P_ABLK bytes,
// hi copy first, then lo.  One CTA per block.
__global__ void __launch_bounds__(256) k_tc_pack(const float* __restrict__ A, int64_t lda,
                                                 int64_t sA, int a_trans, int a_mask, int64_t M,
                                                 int K, unsigned char* __restrict__ Apk,
                                                 int64_t sApk, const uint8_t* __restrict__ dec,
                                                 int k_step, uint8_t want) {
  if (dec != nullptr && dec[k_step] != want) return;
  const int kc = blockIdx.x, mb = blockIdx.y;
  const int64_t t = blockIdx.z;
  const int nK = (K + P_BK - 1) / P_BK;
  const float* P = A + t * sA;
  unsigned char* hi = Apk + t * sApk + ((int64_t)mb * nK + kc) * 2 * P_ABLK;
  unsigned char* lo = hi + P_ABLK;
  for (int idx = threadIdx.x; idx < 128 * P_BK; idx += 256) {
    int r, k;
    if (a_trans) { k = idx % P_BK; r = idx / P_BK; } else { r = idx % 128; k = idx / 128; }
    const int64_t gr = (int64_t)mb * 128 + r;
    const int gk = kc * P_BK + k;
    float x = 0.f;
    if (gr < M && gk < K) x = a_trans ? tc_fetch(P, lda, gk, gr, a_mask) : tc_fetch(P, lda, gr, gk, a_mask);
    tc_put(hi, lo, kmajor_off16(r, k), x);
  }
}

// Stages a B chunk (K rows [k0, k0+16) x P_BN columns) with hi/lo splitting.
__device__ __forceinline__ void p_stage_b(unsigned char* bst, const TcArgs& a, const float* B,
                                          int64_t n0, int k0) {
  unsigned char* bhi = bst;
  unsigned char* blo = bst + P_BN * P_BK * 4;
  if (!a.b_trans && a.b_mask == TC_MASK_NONE) {
    // 4 consecutive K of one column per thread step: one 16-byte core-matrix row
    for (int idx = threadIdx.x; idx < P_BN * (P_BK / 4); idx += TC_THREADS) {
      const int q = idx % (P_BK / 4), c = idx / (P_BK / 4);
      const int64_t gc = n0 + c;
      const int gk = k0 + 4 * q;
      float x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        x[u] = (gc < a.N && gk + u < a.K) ? B[gk + u + gc * a.ldb] : 0.f;
      uint4 h, l;
      uint32_t* hp = reinterpret_cast<uint32_t*>(&h);
      uint32_t* lp = reinterpret_cast<uint32_t*>(&l);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        hp[u] = tf32_bits(x[u]);
        lp[u] = tf32_bits(x[u] - __uint_as_float(hp[u]));
      }
      const uint32_t off = kmajor_off16(c, 4 * q);
      *reinterpret_cast<uint4*>(bhi + off) = h;
      *reinterpret_cast<uint4*>(blo + off) = l;
    }
  } else {
    for (int idx = threadIdx.x; idx < P_BN * P_BK; idx += TC_THREADS) {
      int c, k;
      if (a.b_trans) { c = idx % P_BN; k = idx / P_BN; } else { k = idx % P_BK; c = idx / P_BK; }
      const int64_t gc = n0 + c;
      const int gk = k0 + k;
      float x = 0.f;
      if (gc < a.N && gk < a.K)
        x = a.b_trans ? tc_fetch(B, a.ldb, gc, gk, a.b_mask) : tc_fetch(B, a.ldb, gk, gc, a.b_mask);
      tc_put(bhi, blo, kmajor_off16(c, k), x);
    }
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_gemm_tc2(TcArgs a) {
  if (a.dec != nullptr && a.dec[a.k_step] != a.want) return;
  extern __shared__ __align__(1024) unsigned char smem_p[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_p + P_STAGES * P_STAGE);
  uint64_t* empty = full + P_STAGES;
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(empty + P_STAGES);
  int* last_commit = reinterpret_cast<int*>(taddr_slot + 1);
  int* pending_copy = last_commit + 1;   // chunk whose bulk copy was not seen complete
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.y * 256, n0 = (int64_t)blockIdx.x * P_BN;
  const int64_t t = blockIdx.z;
  const int nK = (a.K + P_BK - 1) / P_BK;
  const int mh = (a.M - m0) > 128 ? 2 : 1;     // M halves present in this tile
  const unsigned char* Apk = a.Apk + t * a.sApk;
  const float* B = a.B + t * a.sB;
  float* C = a.C + t * a.sC;
  const float* C1 = a.C1 ? a.C1 + t * a.sC1 : nullptr;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(taddr_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    *last_commit = -1;
    *pending_copy = -1;
    for (int q = 0; q < P_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_slot;
  const uint32_t idesc = make_idesc_tf32(128, P_BN);
  bool ok = true;
  for (int c = 0; c < nK; ++c) {
    const int st = c % P_STAGES;
    const uint32_t use = (uint32_t)(c / P_STAGES);
    unsigned char* sa = smem_p + st * P_STAGE;
    unsigned char* sb = sa + P_ASTAGE;
    if (c >= P_STAGES && !mbar_wait(&empty[st], (use - 1) & 1)) ok = false;
    if (!__syncthreads_and(ok ? 1 : 0)) { ok = false; break; }
    if (tid == 0) {
      const uint32_t bytes = (uint32_t)mh * 2 * P_ABLK;
      mbar_expect_tx(&full[st], bytes);
      for (int h = 0; h < mh; ++h) {
        const unsigned char* src = Apk + (((int64_t)(m0 / 128 + h) * nK + c) * 2 * P_ABLK);
        bulk_g2s(sa + h * 2 * P_ABLK, src, 2 * P_ABLK, &full[st]);
      }
    }
    p_stage_b(sb, a, B, n0, c * P_BK);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      if (!mbar_wait(&full[st], use & 1)) {
        ok = false;
        *pending_copy = c;
      } else {
        const uint32_t sbase = smem_u32(sb);
#pragma unroll
        for (int s8 = 0; s8 < P_BK / 8; ++s8) {
          const uint32_t koff = (uint32_t)s8 * 2 * TC_LBO;
          const uint64_t bhi = make_desc_sbo(sbase + koff, P_SBO);
          const uint64_t blo = make_desc_sbo(sbase + P_BN * P_BK * 4 + koff, P_SBO);
          for (int h = 0; h < mh; ++h) {
            const uint32_t abase = smem_u32(sa + h * 2 * P_ABLK);
            const uint64_t ahi = make_desc_sbo(abase + koff, P_SBO);
            const uint64_t alo = make_desc_sbo(abase + P_ABLK + koff, P_SBO);
            const uint32_t d = tmem + (uint32_t)(h * P_BN);
            const uint32_t acc0 = (c > 0 || s8 > 0) ? 1u : 0u;
            tc_mma(d, alo, bhi, idesc, acc0);
            tc_mma(d, ahi, blo, idesc, 1u);
            tc_mma(d, ahi, bhi, idesc, 1u);
          }
        }
        tc_commit(&empty[st]);
        *last_commit = c;
      }
    }
  }
  __syncthreads();
  const int last = *last_commit;
  if (last >= 0 && !mbar_wait(&empty[last % P_STAGES], (uint32_t)(last / P_STAGES) & 1)) ok = false;
  // a bulk copy that was not seen complete must land before shared memory is released
  if (tid == 0 && *pending_copy >= 0) {
    const int pc = *pending_copy;
    (void)mbar_wait(&full[pc % P_STAGES], (uint32_t)(pc / P_STAGES) & 1);
  }
  tc_fence_after();
  const bool all_ok = __syncthreads_and(ok ? 1 : 0);
  if (all_ok) {
    const int h = warp >> 2;                       // M half handled by this warp
    const int lane_base = (warp & 3) * 32;
    const int64_t row = m0 + h * 128 + lane_base + lane;
    if (h < mh) {
      for (int cc = 0; cc < P_BN; cc += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(h * P_BN + cc), v);
        tc_epi32(a, C, C1, row, n0 + cc, v);
      }
    }
  } else if (tid == 0 && a.status != nullptr) {
    atomicCAS(&a.status[ST_CODE], 0, -6);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// cp.async helpers of the streamed contraction below (16-byte copies, zero fill past the
// source bytes given).
__device__ __forceinline__ void cp_async16_zfill(void* sdst, const void* gsrc, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- bounded mbarrier waits
// Waits for the phase of the given parity; false when the CTA's fail flag is set (unless
// honour_fail is false) or the cycle budget runs out (then it sets the flag itself).
constexpr long long W_WAIT_CYCLES = 1000000000LL;   // ~0.5 s

__device__ __forceinline__ bool wwait(uint64_t* bar, uint32_t parity, volatile int* fail,
                                      bool honour_fail = true,
                                      long long budget = W_WAIT_CYCLES) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (honour_fail && *fail) return false;
    if (clock64() - t0 > budget) {
      *fail = 1;
      return false;
    }
  }
}
__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// ---------------------------------------------------------------- persistent form
// Persistent, warp-specialised form of the contraction: one CTA per SM walks the
// 256 x 128 output tiles of the launch, and two TMEM accumulators let the epilogue of tile
// i (warps 8-11) overlap the main loop of tile i+1.  Without the overlap every SM alternates
// between a tensor-bound main loop and an HBM-bound epilogue, and the two phases of all SMs
// line up.  Roles:
//   warp 0      raw B chunks (cp.async) into a 4-slot ring
//   warp 1      tcgen05.mma issue (one thread) into accumulator (tile parity)
//   warp 2      packed A chunks (cp.async.bulk) into a 3-stage ring
//   warp 3      C loader: the C (or C1) blocks an accumulating epilogue reads, one
//               128-row x 32-column segment at a time (a column per lane, one bulk copy of
//               512 bytes each), into a 3-slot ring running ahead of the epilogue
//   warps 4-7   TF32 hi/lo split of B into the stage
//   warps 8-11  epilogue: TMEM -> registers -> C, then free the accumulator
// Chunks are numbered across tiles (g = tile_iter * nK + c) for the ring slots and parities.
constexpr int T4_THREADS = 384;
constexpr int T4_BN = 128;
constexpr int T4_STG = 3;
constexpr int T4_RAW = 4;
constexpr int T4_ABYTES = 2 * 2 * P_ABLK;                   // two M halves x (hi, lo)
constexpr int T4_BBYTES = 2 * T4_BN * P_BK * 4;             // hi + lo
constexpr int T4_STAGE = T4_ABYTES + T4_BBYTES;             // 48 KB
constexpr int T4_RAWB = T4_BN * P_BK * 4;                   // 8 KB
constexpr int T4_CSLOTS = 3;
constexpr int T4_CBOX = 128 * 32 * 4;                        // 16 KB: one epilogue segment
constexpr int T4_SMEM = T4_STG * T4_STAGE + T4_RAW * T4_RAWB + T4_CSLOTS * T4_CBOX + 512;
static_assert(T4_SMEM <= SMEM_MAX, "persistent GEMM stages exceed the shared memory of a CTA");

__global__ void __launch_bounds__(T4_THREADS, 1) k_gemm_tc4(TcArgs a, int mtiles, int ntiles,
                                                     int total, int skip) {
  if (a.dec != nullptr && a.dec[a.k_step] != a.want) return;
  if (a.status != nullptr && a.status[ST_CODE] != 0) return;
  extern __shared__ __align__(1024) unsigned char smem_p4[];
  unsigned char* rawbase = smem_p4 + T4_STG * T4_STAGE;
  float* cbox = reinterpret_cast<float*>(rawbase + T4_RAW * T4_RAWB);   // T4_CSLOTS boxes
  uint64_t* raw_full =
      reinterpret_cast<uint64_t*>(rawbase + T4_RAW * T4_RAWB + T4_CSLOTS * T4_CBOX);
  uint64_t* raw_empty = raw_full + T4_RAW;
  uint64_t* a_full = raw_empty + T4_RAW;
  uint64_t* b_full = a_full + T4_STG;
  uint64_t* st_empty = b_full + T4_STG;
  uint64_t* acc_full = st_empty + T4_STG;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* c_full = acc_empty + 2;
  uint64_t* c_empty = c_full + T4_CSLOTS;
  uint32_t* taddr_slot = reinterpret_cast<uint32_t*>(c_empty + T4_CSLOTS);
  volatile int* fail = reinterpret_cast<volatile int*>(taddr_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nK = a.K / P_BK;
  // tiles of this CTA: tile = blockIdx.x + it * gridDim.x
  const int ntile_cta = (total - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  auto tile_of = [&](int it, int64_t& t, int64_t& m0, int64_t& n0) {
    const int tile = (int)blockIdx.x + it * (int)gridDim.x;
    const int per = mtiles * ntiles;
    t = tile / per;
    const int r = tile - (int)t * per;
    m0 = (int64_t)(r / ntiles) * 256;
    n0 = (int64_t)(r % ntiles) * T4_BN;
  };
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(taddr_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    *fail = 0;
    for (int q = 0; q < T4_RAW; ++q) {
      mbar_init(&raw_full[q], 32);
      mbar_init(&raw_empty[q], 4);
    }
    for (int q = 0; q < T4_STG; ++q) {
      mbar_init(&a_full[q], 1);
      mbar_init(&b_full[q], 4);
      mbar_init(&st_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], 4);
    }
    for (int q = 0; q < T4_CSLOTS; ++q) {
      mbar_init(&c_full[q], 1);
      mbar_init(&c_empty[q], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *taddr_slot;
  const long long budget = a.wait_cycles > 0 ? a.wait_cycles : W_WAIT_CYCLES;

  if (warp == 0) {
    // ---- raw B producer
    bool stop = false;
    for (int it = 0; it < ntile_cta && !stop; ++it) {
      int64_t t, m0, n0;
      tile_of(it, t, m0, n0);
      const float* B = a.B + t * a.sB;
      for (int c = 0; c < nK; ++c) {
        const int g = it * nK + c, slot = g % T4_RAW;
        bool ok = g < T4_RAW || wwait(&raw_empty[slot], (uint32_t)((g / T4_RAW) - 1) & 1, fail, true, budget);
        if (!__all_sync(0xffffffffu, ok ? 1 : 0)) { stop = true; break; }
        unsigned char* raw = rawbase + slot * T4_RAWB;
        const int k0 = c * P_BK;
        for (int idx = lane; idx < T4_BN * (P_BK / 4); idx += 32) {
          const int q = idx & 3, col = idx >> 2;
          const int64_t gc = n0 + col;
          const bool in = gc < a.N;
          const float* src = in ? B + (k0 + 4 * q) + gc * a.ldb : B;
          cp_async16_zfill(raw + idx * 16, src, in ? 16u : 0u);
        }
        if (g != skip || blockIdx.x != 0)   // skip: test hook, normally -1
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(
                           smem_u32(&raw_full[slot]))
                       : "memory");
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc_tf32(128, T4_BN);
      int last_g = -1;
      bool stop = false;
      for (int it = 0; it < ntile_cta && !stop; ++it) {
        int64_t t, m0, n0;
        tile_of(it, t, m0, n0);
        const int mh = (a.M - m0) > 128 ? 2 : 1;
        const int buf = it & 1;
        if (it >= 2 && !wwait(&acc_empty[buf], (uint32_t)((it / 2) - 1) & 1, fail, true, budget)) break;
        tc_fence_after();
        bool started[2] = {false, false};
        for (int c = 0; c < nK; ++c) {
          const int g = it * nK + c, st = g % T4_STG;
          const uint32_t ph = (uint32_t)(g / T4_STG) & 1;
          if (!wwait(&a_full[st], ph, fail, true, budget) || !wwait(&b_full[st], ph, fail, true, budget)) { stop = true; break; }
          tc_fence_after();
          unsigned char* sa = smem_p4 + st * T4_STAGE;
          const uint32_t sbase = smem_u32(sa + T4_ABYTES);
#pragma unroll
          for (int s8 = 0; s8 < P_BK / 8; ++s8) {
            const uint32_t koff = (uint32_t)s8 * 2 * TC_LBO;
            const uint64_t bhi = make_desc_sbo(sbase + koff, P_SBO);
            const uint64_t blo = make_desc_sbo(sbase + T4_BN * P_BK * 4 + koff, P_SBO);
            for (int h = 0; h < mh; ++h) {
              // rows [r0, r0 + 128) of a triangular A meet only part of K
              const int64_t r0 = m0 + h * 128, q0 = (int64_t)c * P_BK + s8 * 8;
              if ((a.a_tri == 1 && q0 >= r0 + 128) || (a.a_tri == 2 && q0 + 8 <= r0)) continue;
              const uint32_t abase = smem_u32(sa + h * 2 * P_ABLK);
              const uint64_t ahi = make_desc_sbo(abase + koff, P_SBO);
              const uint64_t alo = make_desc_sbo(abase + P_ABLK + koff, P_SBO);
              const uint32_t d = tmem + (uint32_t)(buf * 256 + h * T4_BN);
              const uint32_t acc0 = started[h] ? 1u : 0u;
              started[h] = true;
              tc_mma(d, alo, bhi, idesc, acc0);
              tc_mma(d, ahi, blo, idesc, 1u);
              tc_mma(d, ahi, bhi, idesc, 1u);
            }
          }
          tc_commit(&st_empty[st]);
          last_g = g;
        }
        if (stop) break;
        tc_commit(&acc_full[buf]);
      }
      if (last_g >= 0)
        wwait(&st_empty[last_g % T4_STG], (uint32_t)(last_g / T4_STG) & 1, fail, false, budget);
    }
  } else if (warp == 2) {
    // ---- packed A producer
    if (lane == 0) {
      int last_g = -1;
      bool stop = false;
      for (int it = 0; it < ntile_cta && !stop; ++it) {
        int64_t t, m0, n0;
        tile_of(it, t, m0, n0);
        const int mh = (a.M - m0) > 128 ? 2 : 1;
        const unsigned char* Apk = a.Apk + t * a.sApk;
        for (int c = 0; c < nK; ++c) {
          const int g = it * nK + c, st = g % T4_STG;
          if (g >= T4_STG && !wwait(&st_empty[st], (uint32_t)((g / T4_STG) - 1) & 1, fail, true, budget)) {
            stop = true;
            break;
          }
          unsigned char* sa = smem_p4 + st * T4_STAGE;
          mbar_expect_tx(&a_full[st], (uint32_t)mh * 2 * P_ABLK);
          for (int h = 0; h < mh; ++h) {
            const unsigned char* src = Apk + (((int64_t)(m0 / 128 + h) * nK + c) * 2 * P_ABLK);
            bulk_g2s(sa + h * 2 * P_ABLK, src, 2 * P_ABLK, &a_full[st]);
          }
          last_g = g;
        }
      }
      for (int q = last_g; q >= 0 && q > last_g - T4_STG; --q)
        wwait(&a_full[q % T4_STG], (uint32_t)(q / T4_STG) & 1, fail, false, budget);
    }
  } else if (warp == 3) {
    // ---- C loader (accumulating epilogues with aligned segments only)
    if (a.c_bulk && a.epi != TC_EPI_OUT) {
      const bool sub = a.epi == TC_EPI_SUB;
      const int64_t ldr = sub ? a.ldc : a.ldc1;
      int seg = 0;
      bool stop = false;
      for (int it = 0; it < ntile_cta && !stop; ++it) {
        int64_t t, m0, n0;
        tile_of(it, t, m0, n0);
        const float* Cr = sub ? a.C + t * a.sC : a.C1 + t * a.sC1;
        const int mh = (a.M - m0) > 128 ? 2 : 1;
        for (int h = 0; h < mh && !stop; ++h) {
          const int64_t r0 = m0 + h * 128;
          const int rows = (int)min((int64_t)128, a.M - r0);
          for (int cc = 0; cc < T4_BN; cc += 32, ++seg) {
            if (n0 + cc >= a.N) break;
            const int slot = seg % T4_CSLOTS;
            bool ok = seg < T4_CSLOTS ||
                      wwait(&c_empty[slot], (uint32_t)((seg / T4_CSLOTS) - 1) & 1, fail, true, budget);
            if (!__all_sync(0xffffffffu, ok ? 1 : 0)) { stop = true; break; }
            const int cols = (int)min((int64_t)32, a.N - (n0 + cc));
            if (lane == 0) mbar_expect_tx(&c_full[slot], (uint32_t)(rows * 4 * cols));
            __syncwarp();
            if (lane < cols)
              bulk_g2s(cbox + (size_t)slot * (T4_CBOX / 4) + lane * 128,
                       Cr + r0 + (n0 + cc + lane) * ldr, (uint32_t)(rows * 4), &c_full[slot]);
          }
        }
      }
      // copies still in flight land before the CTA exits
      for (int q = seg - 1; q >= 0 && q > seg - 1 - T4_CSLOTS; --q)
        wwait(&c_full[q % T4_CSLOTS], (uint32_t)(q / T4_CSLOTS) & 1, fail, false, budget);
    }
  } else if (warp >= 4 && warp < 8) {
    // ---- converters
    const int ct = tid - 128;
    bool stop = false;
    for (int it = 0; it < ntile_cta && !stop; ++it) {
      for (int c = 0; c < nK; ++c) {
        const int g = it * nK + c, slot = g % T4_RAW, st = g % T4_STG;
        bool ok = wwait(&raw_full[slot], (uint32_t)(g / T4_RAW) & 1, fail, true, budget);
        if (ok && g >= T4_STG) ok = wwait(&st_empty[st], (uint32_t)((g / T4_STG) - 1) & 1, fail, true, budget);
        if (!__all_sync(0xffffffffu, ok ? 1 : 0)) { stop = true; break; }
        const unsigned char* raw = rawbase + slot * T4_RAWB;
        unsigned char* bhi = smem_p4 + st * T4_STAGE + T4_ABYTES;
        unsigned char* blo = bhi + T4_BN * P_BK * 4;
        static_assert(T4_BN * (P_BK / 4) == 4 * 128, "four 16-byte pieces per converter thread");
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int idx = ct + 128 * j;
          const int q = idx & 3, col = idx >> 2;
          const float4 x = *reinterpret_cast<const float4*>(raw + idx * 16);
          uint4 hh, ll;
          hh.x = tf32_bits(x.x); ll.x = tf32_bits(x.x - __uint_as_float(hh.x));
          hh.y = tf32_bits(x.y); ll.y = tf32_bits(x.y - __uint_as_float(hh.y));
          hh.z = tf32_bits(x.z); ll.z = tf32_bits(x.z - __uint_as_float(hh.z));
          hh.w = tf32_bits(x.w); ll.w = tf32_bits(x.w - __uint_as_float(hh.w));
          const uint32_t off = kmajor_off16(col, 4 * q);
          *reinterpret_cast<uint4*>(bhi + off) = hh;
          *reinterpret_cast<uint4*>(blo + off) = ll;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive1(&raw_empty[slot]);
          mbar_arrive1(&b_full[st]);
        }
      }
    }
  } else if (warp >= 8) {
    // ---- epilogue (warp 8 + e owns TMEM lanes 32e..32e+31 of each half)
    const int e = warp - 8;
    const bool boxed = a.c_bulk && a.epi != TC_EPI_OUT;
    int seg = 0;
    bool stop = false;
    for (int it = 0; it < ntile_cta && !stop; ++it) {
      int64_t t, m0, n0;
      tile_of(it, t, m0, n0);
      const int mh = (a.M - m0) > 128 ? 2 : 1;
      const int buf = it & 1;
      bool ok = wwait(&acc_full[buf], (uint32_t)(it / 2) & 1, fail, true, budget);
      if (!__all_sync(0xffffffffu, ok ? 1 : 0)) break;
      tc_fence_after();
      float* C = a.C + t * a.sC;
      const float* C1 = a.C1 ? a.C1 + t * a.sC1 : nullptr;
      for (int h = 0; h < mh && !stop; ++h) {
        const int64_t row = m0 + h * 128 + e * 32 + lane;
        for (int cc = 0; cc < T4_BN; cc += 32, ++seg) {
          if (n0 + cc >= a.N) break;
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(e * 32) << 16) + (uint32_t)(buf * 256 + h * T4_BN + cc), v);
          if (!boxed) {
            tc_epi32(a, C, C1, row, n0 + cc, v);
            continue;
          }
          // the segment's old values come from the loader's box (column c at c * 128)
          const int slot = seg % T4_CSLOTS;
          ok = wwait(&c_full[slot], (uint32_t)(seg / T4_CSLOTS) & 1, fail, true, budget);
          if (!__all_sync(0xffffffffu, ok ? 1 : 0)) { stop = true; break; }
          const float* bx = cbox + (size_t)slot * (T4_CBOX / 4) + e * 32 + lane;
          if (row < a.M) {
            const int64_t lim = a.N - (n0 + cc);
            float* Cr = C + row + (n0 + cc) * a.ldc;
            if (a.epi == TC_EPI_SUB) {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (i < lim) Cr[(int64_t)i * a.ldc] = bx[i * 128] - v[i];
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i)
                if (i < lim) Cr[(int64_t)i * a.ldc] = v[i] + bx[i * 128];
            }
          }
          __syncwarp();
          if (lane == 0) mbar_arrive1(&c_empty[slot]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0 && !stop) mbar_arrive1(&acc_empty[buf]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *fail && a.status != nullptr) atomicCAS(&a.status[ST_CODE], 0, -6);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

static std::atomic<int> g_tc_skip{-1};
void tc_set_debug_skip(int chunk) { g_tc_skip.store(chunk < 0 ? -1 : chunk); }

size_t tc_packed_bytes(int64_t M, int K) {
  const int64_t mb = (M + 127) / 128, nK = (K + P_BK - 1) / P_BK;
  return (size_t)(mb * nK) * 2 * P_ABLK;
}

void launch_tc_pack(const float* A, int64_t lda, int64_t sA, int a_trans, int a_mask, int64_t M,
                    int K, unsigned char* Apk, int64_t sApk, int batch, const uint8_t* dec, int k,
                    uint8_t want, cudaStream_t s) {
  if (M <= 0 || K <= 0 || batch <= 0) return;
  dim3 grid((unsigned)((K + P_BK - 1) / P_BK), (unsigned)((M + 127) / 128), (unsigned)batch);
  {
    ProfScope ps_("k_tc_pack", s);
    k_tc_pack<<<grid, 256, 0, s>>>(A, lda, sA, a_trans, a_mask, M, K, Apk, sApk, dec, k, want);
  }
}

void launch_tc2(const TcArgs& a, int batch, const char* name, cudaStream_t s) {
  if (a.M <= 0 || a.N <= 0 || a.K <= 0 || batch <= 0) return;
  dim3 grid((unsigned)((a.N + P_BN - 1) / P_BN), (unsigned)((a.M + 255) / 256), (unsigned)batch);
  // a triangular A must leave every row some nonzero K (M <= K); else no skipping
  if (a.a_tri != 0 && a.M > a.K) {
    TcArgs b = a;
    b.a_tri = 0;
    launch_tc2(b, batch, name, s);
    return;
  }
  const bool vec = !a.b_trans && a.b_mask == TC_MASK_NONE && (a.K % P_BK) == 0 &&
                   (a.ldb % 4) == 0 && (a.sB % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(a.B) % 16) == 0;
  ProfScope ps_(name, s);
  if (vec) {
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (sms <= 0) sms = 1;
    }
    const int mtiles = (int)((a.M + 255) / 256), ntiles = (int)((a.N + T4_BN - 1) / T4_BN);
    const int64_t total = (int64_t)mtiles * ntiles * batch;
    // persistent over all but about a ninth of the SMs: the high-priority panel, look-ahead
    // and operand kernels of the next steps keep SMs of their own (a grid over every SM held
    // them off for whole launches; short-lived CTAs cost the pipeline fill and drain of each)
    const int ctas = (int)std::min<int64_t>(total, std::max(1, sms - sms / 9));
    // bulk copies of the accumulating epilogue's column segments need every segment start
    // 16-byte aligned and a whole number of 16 bytes per column
    TcArgs b = a;
    const bool sub = a.epi == TC_EPI_SUB;
    const float* Cr = sub ? a.C : a.C1;
    const int64_t ldr = sub ? a.ldc : a.ldc1, sr = sub ? a.sC : a.sC1;
    b.c_bulk = a.epi != TC_EPI_OUT && Cr != nullptr &&
               (reinterpret_cast<uintptr_t>(Cr) % 16) == 0 && (ldr % 4) == 0 &&
               (batch == 1 || (sr % 4) == 0) && (a.M % 4) == 0;
    ensure_dyn_smem<k_gemm_tc4>(T4_SMEM);
    k_gemm_tc4<<<ctas, T4_THREADS, T4_SMEM, s>>>(b, mtiles, ntiles, (int)total,
                                                  g_tc_skip.load(std::memory_order_relaxed));
  } else {
    ensure_dyn_smem<k_gemm_tc2>(P_SMEM);
    k_gemm_tc2<<<grid, TC_THREADS, P_SMEM, s>>>(a);
  }
}

// ---------------------------------------------------------------- full compact-WY T
// Tf (nb x nb, upper triangular, column-major, ld nb) such that Q = I - V Tf V^T for all
// nb reflectors of a tile, from the Gram matrix G = V^T V (upper part used) and the stored
// IB x IB diagonal blocks (T slot: block b at columns b*IB.., IB rows).  Built by recursive
// bisection of the nb/IB blocks: for a node whose leading blocks are A and trailing blocks
// B, Q = Q_A Q_B gives
//   Tf[A,A] = T_A,  Tf[B,B] = T_B,  Tf[A,B] = -T_A G[A,B] T_B.
// Nodes at depth d cover blocks [floor(i nblk / 2^d), floor((i+1) nblk / 2^d)); the deepest
// level goes first, so both children of a node are complete when it is formed.  The
// intermediate P = G[A,B] T_B is kept transposed in the node's block below the diagonal,
// Tf[B,A], and cleared after use (Tf is zero below the diagonal when the kernel ends).
// One CTA (256 threads) per tile; each product runs in 64 x 64 output tiles, 4 x 4 outputs
// per thread, operands staged in 32-deep chunks in shared memory.
constexpr int TF_T = 64, TF_Q = 32, TF_LD = TF_T + 4;

// out(i, j) = sum_{q in [qlo(i0), qhi(j0))} X(i, q) Y(q, j) for one 64 x 64 tile of an m x n
// product.  YQ: Y's consecutive q are contiguous in memory (else consecutive j).
template <bool YQ, class FX, class FY, class FO>
__device__ __forceinline__ void tf_tile(int m, int n, int i0, int j0, int q0, int q1, FX X, FY Y,
                                        FO out, float* Xs, float* Ys) {
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  // operands of the next chunk are loaded into registers while this chunk is multiplied
  constexpr int PER = TF_T * TF_Q / 256;
  float xr[PER], yr[PER];
  auto fetch = [&](int qc) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * 256;
      const int i = idx % TF_T, q = idx / TF_T;
      xr[u] = (i0 + i < m && qc + q < q1) ? X(i0 + i, qc + q) : 0.f;
      const int qy = YQ ? idx % TF_Q : idx / TF_T, j = YQ ? idx / TF_Q : idx % TF_T;
      yr[u] = (j0 + j < n && qc + qy < q1) ? Y(qc + qy, j0 + j) : 0.f;
    }
  };
  if (q0 < q1) fetch(q0);
  for (int qc = q0; qc < q1; qc += TF_Q) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int idx = tid + u * 256;
      Xs[(idx / TF_T) * TF_LD + idx % TF_T] = xr[u];
      const int qy = YQ ? idx % TF_Q : idx / TF_T, j = YQ ? idx / TF_Q : idx % TF_T;
      Ys[qy * TF_LD + j] = yr[u];
    }
    __syncthreads();
    if (qc + TF_Q < q1) fetch(qc + TF_Q);
#pragma unroll 8
    for (int q = 0; q < TF_Q; ++q) {
      const float4 xa = *reinterpret_cast<const float4*>(&Xs[q * TF_LD + ty * 4]);
      const float4 yb = *reinterpret_cast<const float4*>(&Ys[q * TF_LD + tx * 4]);
      const float xv[4] = {xa.x, xa.y, xa.z, xa.w}, yv[4] = {yb.x, yb.y, yb.z, yb.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xv[a], yv[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
      if (i < m && j < n) out(i, j, acc[a][b]);
    }
}

__global__ void __launch_bounds__(256) k_tfull(const float* __restrict__ G, int64_t sG,
                                               const float* __restrict__ Tslots, int64_t sT,
                                               float* __restrict__ Tf, int64_t sTf, int nb,
                                               const uint8_t* __restrict__ dec, int k) {
  if (dec[k] != DEC_QR) return;
  __shared__ __align__(16) float Xs[TF_Q * TF_LD];
  __shared__ __align__(16) float Ys[TF_Q * TF_LD];
  const int64_t t = blockIdx.x;
  const float* g = G + t * sG;
  const float* ts = Tslots + t * sT;
  float* tf = Tf + t * sTf;
  const int tid = threadIdx.x;
  const int nblk = nb / IB;
  // diagonal blocks from the T slots; zero below them
  for (int idx = tid; idx < nb * nb; idx += 256) {
    const int r = idx % nb, c = idx / nb, rb = r / IB, cb = c / IB;
    if (rb == cb) tf[idx] = (r <= c) ? ts[(r - cb * IB) + (int64_t)c * IB] : 0.f;
    else if (rb > cb) tf[idx] = 0.f;
  }
  __syncthreads();
  int D = 0;
  while ((1 << D) < nblk) ++D;
  for (int d = D - 1; d >= 0; --d) {
    for (int i = 0; i < (1 << d); ++i) {
      const int lo = (int)(((int64_t)i * nblk) >> d), hi = (int)(((int64_t)(i + 1) * nblk) >> d);
      const int mid = (int)(((int64_t)(2 * i + 1) * nblk) >> (d + 1));
      if (mid <= lo || hi <= mid) continue;
      const int a0 = lo * IB, b0 = mid * IB, ma = (mid - lo) * IB, nbB = (hi - mid) * IB;
      // P = G[A,B] T_B (T_B upper triangular: q <= j), stored as P^T in Tf[B,A]
      for (int i0 = 0; i0 < ma; i0 += TF_T)
        for (int j0 = 0; j0 < nbB; j0 += TF_T)
          tf_tile<true>(
              ma, nbB, i0, j0, 0, min(nbB, j0 + TF_T),
              [&](int ii, int q) { return g[(a0 + ii) + (int64_t)(b0 + q) * nb]; },
              [&](int q, int j) { return tf[(b0 + q) + (int64_t)(b0 + j) * nb]; },
              [&](int ii, int j, float v) { tf[(b0 + j) + (int64_t)(a0 + ii) * nb] = v; }, Xs, Ys);
      __syncthreads();
      // Tf[A,B] = -T_A P (T_A upper triangular: q >= i)
      for (int i0 = 0; i0 < ma; i0 += TF_T)
        for (int j0 = 0; j0 < nbB; j0 += TF_T)
          tf_tile<false>(
              ma, nbB, i0, j0, i0, ma,
              [&](int ii, int q) { return tf[(a0 + ii) + (int64_t)(a0 + q) * nb]; },
              [&](int q, int j) { return tf[(b0 + j) + (int64_t)(a0 + q) * nb]; },
              [&](int ii, int j, float v) { tf[(a0 + ii) + (int64_t)(b0 + j) * nb] = -v; }, Xs, Ys);
      __syncthreads();
      for (int idx = tid; idx < ma * nbB; idx += 256) {
        const int j = idx % nbB, ii = idx / nbB;
        tf[(b0 + j) + (int64_t)(a0 + ii) * nb] = 0.f;
      }
      __syncthreads();
    }
  }
}

void launch_tfull(const float* G, int64_t sG, const float* Tslots, int64_t sT, float* Tf,
                  int64_t sTf, int nb, int batch, const uint8_t* dec, int k, cudaStream_t s) {
  if (batch <= 0) return;
  {
    ProfScope ps_("k_tfull", s);
    k_tfull<<<batch, 256, 0, s>>>(G, sG, Tslots, sT, Tf, sTf, nb, dec, k);
  }
}

}  // namespace luqr

extern "C" int luqr_gemm_sub_f32(float* C, int64_t ldc, const float* A, int64_t lda,
                                 const float* B, int64_t ldb, int64_t M, int64_t N, int64_t K,
                                 int* dstatus, void* stream) {
  if (!C || !A || !B || M < 0 || N < 0 || K < 0 || K > (1 << 30) || ldc < M || lda < M ||
      ldb < K)
    return -1;
  luqr::launch_gemm_tc(A, lda, B, ldb, C, ldc, M, N, (int)K, nullptr, 0, 0, dstatus,
                       static_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
