// Second pass on one right-hand side in ONE persistent launch (Sec. II-D, "Solving systems":
// every stored step replayed on a new b, then the N x N triangular solve).
//
// The host lists the replay as tasks in program order (rq_build in luqr_api.cu):
//   RT_SCALE   x_k *= 2^-27                          (run-time injection at step k)
//   RT_SINGLE  x_i <- Q_ik^T x_i                      (GEQRT reflectors of tile (i, k); also
//                                                      the Q^T of an A2 LU step, tile (k, k))
//   RT_PAIR_*  [x_e; x_i] <- Q^T [x_e; x_i]            (TS / TT reflectors of tile (i, k))
//   RT_LUAPPLY x_k <- L^-1 P x_k                       (A1 LU step k)
//   RT_GEMV    x_i -= A_ik x_k                          (LU step k, i > k; back substitution,
//                                                      i < k, with the tiles of U)
//   RT_TRSV    x_k <- U_kk^-1 x_k                       (back substitution)
//   RT_GEMV_TRSV  x_i -= A_{i,i+1} x_{i+1}, then x_i <- U_ii^-1 x_i  (k = i + 1)
// Every task writes one or two tile rows of x and may read one more.  Per tile row r the
// kernel counts completed writes (done[r]); a task waits until every write that precedes it
// in program order has completed on each row it touches (the counts are precomputed).  Reads
// need no count of their own: every later writer of a row depends, through the back
// substitution, on all readers of that row.  CTAs claim tasks in program order from a
// device counter and a task waits only on earlier tasks, which running CTAs have claimed, so
// the launch always progresses, whatever number of CTAs is resident.  Waits are bounded by
// a clock64 budget; when one runs out the kernel records LUQR_ERR_TIMEOUT in the status
// word, raises an abort flag that stops every CTA, and returns.
#include <cuda_runtime.h>

#include "internal.cuh"

namespace luqr {


// Shared memory of one task: a ring of nbuf staged IB x nb V blocks and IB x IB T blocks,
// two nb segments of x, two IB work vectors.
template <typename T>
size_t replay_smem(int nb, int nbuf) {
  return sizeof(T) * (nbuf * (size_t)IB * nb + nbuf * IB * IB + 2 * (size_t)nb + 2 * IB);
}

// Ring depth of the launch: the deepest of 6, 4, 3, 2 that fits one CTA's shared memory
// (0: none fits).  FP32 tiles of 256 take 6 (about 218 KB), FP64 ones 3.
template <typename T>
int replay_nbuf(int nb) {
  for (int q : {6, 4, 3, 2})
    if (replay_smem<T>(nb, q) <= (size_t)SMEM_MAX) return q;
  return 0;
}

__device__ __forceinline__ void rp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void rp_wait_groups() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void rp_cp16(void* sdst, const void* gsrc) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(gsrc) : "memory");
}

__device__ __forceinline__ int rp_load_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Rows [lo, hi) of column j + jb of the reflector block jb: the nonzero part of V.
__device__ __forceinline__ int rp_lo(bool pair, int jb) { return pair ? 0 : jb; }
__device__ __forceinline__ int rp_hi(bool pair, bool tri, int jb, int nb) {
  return pair ? (tri ? jb + IB : nb) : nb;
}

// Issues the cp.async copies of inner block jb (its IB columns of V and its IB x IB T block)
// into buffer buf, as one commit group.
template <typename T>
__device__ void rp_stage(const T* __restrict__ V, int64_t ldv, const T* __restrict__ Tslot,
                         int nb, bool pair, bool tri, int jb, int buf, T* Vb, T* Tb) {
  constexpr int VEC = 16 / sizeof(T);
  const int tid = threadIdx.x;
  T* vs = Vb + (size_t)buf * IB * nb;
  const int r0 = rp_lo(pair, jb), rows = rp_hi(pair, tri, jb, nb) - r0, cpc = rows / VEC;
  for (int idx = tid; idx < IB * cpc; idx += NT) {
    const int j = idx / cpc, q = idx - j * cpc;
    rp_cp16(&vs[(size_t)j * nb + q * VEC], &V[r0 + q * VEC + (int64_t)(jb + j) * ldv]);
  }
  T* ts = Tb + buf * IB * IB;
  for (int idx = tid; idx < IB * IB / VEC; idx += NT)
    rp_cp16(&ts[idx * VEC], &Tslot[(size_t)jb * IB + idx * VEC]);
  rp_commit();
}

// Q^T of one tile (pair = 0: GEQRT reflectors, unit lower V) or one tile pair (pair = 1:
// reflector j is [e_j; V(:, j)], V upper triangular for TT) applied to the vector segments
// xs (row i) and xe (eliminator row), inner block by inner block:
//   w = V_b^T x_i (+ x_e(block rows) for pairs),  w2 = T_b^T w,  x_i -= V_b w2,  x_e -= w2,
// with the copies of the next NBUF - 1 blocks in flight (a ring of NBUF buffers, one commit
// group per block; block b lives in buffer b % NBUF).  Blocks 0 .. NBUF - 2 were staged
// before the call (while the task waited for its inputs).
template <typename T, int NBUF>
__device__ void rp_qr_vec(const T* __restrict__ V, int64_t ldv, const T* __restrict__ Tslot,
                          int nb, bool pair, bool tri, T* Vb, T* Tb, T* xs, T* xe, T* w, T* w2) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = NT / 32;
  const int nblk = nb / IB;
  auto lo = [&](int jb) { return rp_lo(pair, jb); };
  auto hi = [&](int jb) { return rp_hi(pair, tri, jb, nb); };
  auto stage = [&](int jb, int buf) { rp_stage<T>(V, ldv, Tslot, nb, pair, tri, jb, buf, Vb, Tb); };
  auto vval = [&](const T* vs, int jb, int r, int j) -> T {
    const int d = jb + j;
    if (!pair) {
      if (r < d) return (T)0;
      if (r == d) return (T)1;
    } else if (tri && r > d) {
      return (T)0;
    }
    return vs[(size_t)j * nb + (r - lo(jb))];
  };
  for (int blk = 0; blk < nblk; ++blk) {
    const int jb = blk * IB, b = blk % NBUF, nxt = blk + NBUF - 1;
    // the buffer of block nxt held block blk - 1, consumed before the last barrier
    if (nxt < nblk) stage(nxt * IB, nxt % NBUF);
    else rp_commit();
    rp_wait_groups<NBUF - 1>();   // block blk has landed
    __syncthreads();
    const T* vs = Vb + (size_t)b * IB * nb;
    const T* ts = Tb + b * IB * IB;
    const int r0 = lo(jb), r1 = hi(jb);
    // w = V_b^T x (+ x_e): each warp takes its IB / nw columns together (independent
    // accumulators, so the loads of one row serve several columns and overlap)
    static_assert(IB == 4 * (NT / 32), "four columns per warp");
    {
      T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll 2
      for (int r = r0 + lane; r < r1; r += 32) {
        const T xr = xs[r];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] += vval(vs, jb, r, warp + nw * c) * xr;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T sum = warp_sum<T>(acc[c]);
        const int j = warp + nw * c;
        if (lane == 0) w[j] = pair ? sum + xe[jb + j] : sum;
      }
    }
    __syncthreads();
    // w2 = T_b^T w: column c of T_b (T(a, c) at ts[c * IB + a], a <= c) is read by the lanes
    // of one warp (lane = a, consecutive words), then summed across the warp
    {
      T t[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = warp + nw * q;
        t[q] = (lane <= c) ? ts[(size_t)c * IB + lane] * w[lane] : (T)0;
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T acc = warp_sum<T>(t[q]);
        if (lane == 0) w2[warp + nw * q] = acc;
      }
    }
    __syncthreads();
    for (int r = r0 + tid; r < r1; r += NT) {   // x -= V_b w2, four partial sums per row
      T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
      for (int j = 0; j < IB; ++j) acc[j & 3] += vval(vs, jb, r, j) * w2[j];
      xs[r] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    if (pair && tid < IB) xe[jb + tid] -= w2[tid];
    __syncthreads();
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// x <- L^-1 P x for the GETRF factors of the diagonal tile (unit lower L below the diagonal,
// ld ldl): the exchanges in order, then 32-row blocks from the top: warp 0 solves the block
// with shuffles, all threads update the rows below it.
template <typename T>
__device__ void rp_lu_apply(const T* __restrict__ L, int64_t ldl, const int* __restrict__ piv,
                            int nb, T* xs) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0)
    for (int r = 0; r < nb; ++r) {
      const int p = piv[r];
      if (p != r) { const T t = xs[r]; xs[r] = xs[p]; xs[p] = t; }
    }
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 32) {
    if (warp == 0) {
      T l[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) l[c] = L[(b0 + lane) + (int64_t)(b0 + c) * ldl];
      T x = xs[b0 + lane];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const T xc = __shfl_sync(0xffffffffu, x, c);
        if (lane > c) x -= l[c] * xc;
      }
      xs[b0 + lane] = x;
    }
    __syncthreads();
    for (int r = b0 + 32 + tid; r < nb; r += NT) {   // four partial sums: loads overlap
      T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c & 3] += L[r + (int64_t)(b0 + c) * ldl] * xs[b0 + c];
      xs[r] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
  }
}

// x <- U^-1 x for the upper triangle of the diagonal tile (ld ldu), 32-row blocks from the
// bottom.  Returns the first row with an exact zero diagonal entry, or -1.
template <typename T>
__device__ int rp_trsv(const T* __restrict__ U, int64_t ldu, int nb, T* xs, int* s_bad) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) *s_bad = -1;
  __syncthreads();
  for (int bb = nb / 32 - 1; bb >= 0; --bb) {
    const int b0 = bb * 32;
    if (warp == 0) {
      T u[32];
#pragma unroll
      for (int r = 0; r < 32; ++r) u[r] = U[(b0 + lane) + (int64_t)(b0 + r) * ldu];
      T x = xs[b0 + lane];
      int bad = -1;
#pragma unroll
      for (int r = 31; r >= 0; --r) {
        // the diagonal and its reciprocal do not depend on x: only the multiply, the
        // broadcast and the update are on the dependency chain
        const T d = __shfl_sync(0xffffffffu, u[r], r);
        if (d == (T)0) { bad = b0 + r; break; }
        const T inv = (T)1 / d;
        if (lane == r) x = x * inv;
        const T xr = __shfl_sync(0xffffffffu, x, r);
        if (lane < r) x -= u[r] * xr;
      }
      xs[b0 + lane] = x;
      if (lane == 0 && bad >= 0) *s_bad = bad;
    }
    __syncthreads();
    if (*s_bad >= 0) return *s_bad;
    for (int i = tid; i < b0; i += NT) {   // four partial sums: loads overlap
      T acc[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
      for (int q = 0; q < 32; ++q) acc[q & 3] += U[i + (int64_t)(b0 + q) * ldu] * xs[b0 + q];
      xs[i] -= (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }
    __syncthreads();
  }
  return -1;
}

// xs (row i) -= A xk for the nb x nb tile A (ld lda).  Each thread owns 16 bytes of rows
// (VEC consecutive elements) in one of G column groups; a group walks its nb/G columns with
// 16-byte loads (many in flight per thread), and the G partial sums meet in shared memory
// (scratch, G x nb elements).
template <typename T>
__device__ void rp_gemv(const T* __restrict__ A, int64_t lda, int nb, const T* xk, T* xs,
                        T* scratch) {
  constexpr int VEC = 16 / sizeof(T);
  const int tpc = nb / VEC;                       // threads covering one column
  const int G = min(NT / tpc, nb);                // column groups
  const int cpg = nb / G;                         // columns per group
  const int tid = threadIdx.x, g = tid / tpc, lr = tid - g * tpc;
  if (g < G) {
    T acc[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) acc[v] = (T)0;
    const T* base = A + lr * VEC + (int64_t)(g * cpg) * lda;
    const T* xg = xk + g * cpg;
#pragma unroll 8
    for (int c = 0; c < cpg; ++c) {
      const T xc = xg[c];
      if constexpr (sizeof(T) == 4) {
        const float4 a4 = __ldg(reinterpret_cast<const float4*>(base + (int64_t)c * lda));
        acc[0] += a4.x * xc; acc[1] += a4.y * xc; acc[2] += a4.z * xc; acc[3] += a4.w * xc;
      } else {
        const double2 a2 = __ldg(reinterpret_cast<const double2*>(base + (int64_t)c * lda));
        acc[0] += a2.x * xc; acc[1] += a2.y * xc;
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) scratch[(size_t)g * nb + lr * VEC + v] = acc[v];
  }
  __syncthreads();
  for (int r = tid; r < nb; r += NT) {
    T sum = (T)0;
    for (int q = 0; q < G; ++q) sum += scratch[(size_t)q * nb + r];
    xs[r] -= sum;
  }
}

// L2 prefetch of `elems` elements at p (16-byte aligned, a multiple of 16 bytes).
template <typename T>
__device__ __forceinline__ void rp_prefetch(const T* p, int elems) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p),
               "r"((unsigned)(elems * (int)sizeof(T)))
               : "memory");
}

// Prefetches into L2 the part of a task's tile (and T slot) that the task reads and that is
// not already staged in shared memory: per column c, the rows the task touches (unit lower V
// and L: c.., upper V and U: ..c, full tiles otherwise), rounded out to 16 bytes.  The first
// staged_blocks inner blocks of a QR task are staged separately.  Every address lies inside
// the tile and slot.
template <typename T>
__device__ void rp_prefetch_task(int type, const T* tile, int64_t ld, int nb, const T* Tslot,
                                 int staged_blocks) {
  constexpr int VEC = 16 / (int)sizeof(T);
  for (int c = threadIdx.x + staged_blocks * IB; c < nb; c += NT) {
    int lo = 0, hi = nb;
    if (type == RT_SINGLE || type == RT_LUAPPLY) lo = c;
    if (type == RT_PAIR_TT || type == RT_TRSV) hi = c + 1;
    lo = lo / VEC * VEC;
    hi = min(nb, (hi + VEC - 1) / VEC * VEC);
    if (hi > lo) rp_prefetch<T>(tile + lo + (int64_t)c * ld, hi - lo);
  }
  if (Tslot != nullptr && (int)threadIdx.x < nb / IB - staged_blocks)
    rp_prefetch<T>(Tslot + (size_t)(threadIdx.x + staged_blocks) * IB * IB, IB * IB);
}

// Waits (thread 0) until *cnt >= need; false when the abort flag is raised or the clock64
// budget runs out (then the timeout is recorded and the abort flag raised).
__device__ bool rp_wait(const int* cnt, int need, long long budget, int* abort_flag, int* status,
                        int k) {
  if (rp_load_acquire(cnt) >= need) return true;
  const long long t0 = clock64();
  unsigned ns = 32;
  while (rp_load_acquire(cnt) < need) {
    if (*(volatile int*)abort_flag) return false;
    if (clock64() - t0 > budget) {
      if (atomicCAS(&status[ST_CODE], 0, LUQR_TIMEOUT_CODE) == 0) {
        status[ST_STEP] = k;
        status[ST_ROW] = -1;
      }
      atomicExch(abort_flag, 1);
      return false;
    }
    __nanosleep(ns);
    if (ns < 256) ns *= 2;
  }
  return true;
}

template <typename T, int NBUF>
__global__ void __launch_bounds__(NT) k_replay(ReplayArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = a.nb;
  T* Vb = reinterpret_cast<T*>(smem_raw);           // NBUF x (IB x nb)
  T* Tb = Vb + NBUF * (size_t)IB * nb;              // NBUF x (IB x IB)
  T* xs = Tb + NBUF * IB * IB;                      // nb: row i
  T* xe = xs + nb;                                  // nb: eliminator row / read row
  T* w = xe + nb;                                   // IB
  T* w2 = w + IB;                                   // IB
  __shared__ int s_task, s_go, s_bad;
  const int tid = threadIdx.x;
  int* next = a.ctl;
  int* abort_flag = a.ctl + 1;
  for (;;) {
    if (tid == 0) s_task = *(volatile int*)abort_flag ? -1 : atomicAdd(next, 1);
    __syncthreads();
    const int t = s_task;
    if (t < 0 || t >= a.ntasks) break;
    const ReplayTask q = a.tasks[t];
    const uint8_t dk = a.dec[q.k];
    const bool run = q.gate == 0 || (q.gate == 1 && dk == DEC_QR) || (q.gate == 2 && dk == DEC_LU);
    const T* tile = a.W + (int64_t)q.i * nb + (int64_t)q.k * nb * a.ld;
    const T* Tstep = a.Tbuf + (size_t)q.k * a.t_step;
    const bool qr = q.type == RT_SINGLE || q.type == RT_PAIR_TS || q.type == RT_PAIR_TT;
    const bool pair = q.type == RT_PAIR_TS || q.type == RT_PAIR_TT;
    const T* Tslot = qr ? Tstep + ((size_t)q.i * 2 + (pair ? 1 : 0)) * IB * nb : nullptr;
    if (run && q.type != RT_SCALE) {
      // the factor data do not depend on x: stage a QR task's first inner block and start
      // the rest of its tile towards L2 while thread 0 waits for the task's inputs
      // a QR task's first NBUF - 1 inner blocks into the ring (one commit group each, empty
      // groups past the last block keep the count uniform), the rest towards L2
      if (qr)
        for (int blk = 0; blk < NBUF - 1; ++blk) {
          if (blk * IB < nb)
            rp_stage<T>(tile, a.ld, Tslot, nb, pair, q.type == RT_PAIR_TT, blk * IB, blk, Vb, Tb);
          else
            rp_commit();
        }
      if (q.type == RT_GEMV_TRSV) {
        rp_prefetch_task<T>(RT_GEMV, tile, a.ld, nb, nullptr, 0);
        rp_prefetch_task<T>(RT_TRSV, a.W + (int64_t)q.i * nb * (1 + a.ld), a.ld, nb, nullptr, 0);
      } else {
        rp_prefetch_task<T>(q.type, tile, a.ld, nb, Tslot, qr ? NBUF - 1 : 0);
      }
    }
    if (tid == 0) {
      bool ok = rp_wait(a.done + q.i, q.ni, a.budget, abort_flag, a.status, q.k);
      if (ok && q.e >= 0) ok = rp_wait(a.done + q.e, q.ne, a.budget, abort_flag, a.status, q.k);
      if (ok && q.r >= 0) ok = rp_wait(a.done + q.r, q.nr, a.budget, abort_flag, a.status, q.k);
      s_go = ok ? 1 : 0;
    }
    __syncthreads();
    if (!s_go) {
      asm volatile("cp.async.wait_all;" ::: "memory");
      break;
    }
    T* xi = a.x + (int64_t)q.i * nb;
    if (!run) {   // the branch not taken: keep the counts in program order, move no data
      if (tid == 0 && t != a.skip_signal) {
        __threadfence();
        atomicAdd(a.done + q.i, 1);
        if (q.e >= 0) atomicAdd(a.done + q.e, 1);
      }
      continue;
    }
    for (int r = tid; r < nb; r += NT) xs[r] = __ldcg(&xi[r]);
    if (q.e >= 0)
      for (int r = tid; r < nb; r += NT) xe[r] = __ldcg(&a.x[(int64_t)q.e * nb + r]);
    if (q.r >= 0)
      for (int r = tid; r < nb; r += NT) xe[r] = __ldcg(&a.x[(int64_t)q.r * nb + r]);
    __syncthreads();
    bool write_e = false;
    switch (q.type) {
      case RT_SCALE:
        for (int r = tid; r < nb; r += NT) xs[r] *= (T)0x1.0p-27;
        break;
      case RT_SINGLE:
        rp_qr_vec<T, NBUF>(tile, a.ld, Tslot, nb, false, false, Vb, Tb, xs, xe, w, w2);
        break;
      case RT_PAIR_TS:
      case RT_PAIR_TT:
        rp_qr_vec<T, NBUF>(tile, a.ld, Tslot, nb, true, q.type == RT_PAIR_TT, Vb, Tb, xs, xe, w,
                           w2);
        write_e = true;
        break;
      case RT_LUAPPLY:
        rp_lu_apply<T>(tile, a.ld, a.piv_all + (size_t)q.k * nb, nb, xs);
        break;
      case RT_GEMV:
        rp_gemv<T>(tile, a.ld, nb, xe, xs, Vb);
        break;
      case RT_TRSV: {
        const int bad = rp_trsv<T>(tile, a.ld, nb, xs, &s_bad);
        if (bad >= 0) {
          if (tid == 0 && atomicCAS(&a.status[ST_CODE], 0, -4) == 0) {
            a.status[ST_STEP] = q.k;
            a.status[ST_ROW] = q.k * nb + bad;
          }
        }
        break;
      }
      case RT_GEMV_TRSV: {
        rp_gemv<T>(tile, a.ld, nb, xe, xs, Vb);   // tile (i, i+1); xe holds x_{i+1}
        __syncthreads();
        const int bad = rp_trsv<T>(a.W + (int64_t)q.i * nb * (1 + a.ld), a.ld, nb, xs, &s_bad);
        if (bad >= 0) {
          if (tid == 0 && atomicCAS(&a.status[ST_CODE], 0, -4) == 0) {
            a.status[ST_STEP] = q.i;
            a.status[ST_ROW] = q.i * nb + bad;
          }
        }
        break;
      }
      default:
        break;
    }
    __syncthreads();
    for (int r = tid; r < nb; r += NT) __stcg(&xi[r], xs[r]);
    if (write_e)
      for (int r = tid; r < nb; r += NT) __stcg(&a.x[(int64_t)q.e * nb + r], xe[r]);
    __syncthreads();
    if (tid == 0 && t != a.skip_signal) {   // skip_signal: test hook, normally -1
      __threadfence();
      atomicAdd(a.done + q.i, 1);
      if (q.e >= 0) atomicAdd(a.done + q.e, 1);
    }
  }
}

template <typename T>
bool replay_fits(int nb) {
  return replay_nbuf<T>(nb) >= 2 && (nb % 32) == 0;
}

template <typename T, int NBUF>
void launch_replay_n(const ReplayArgs<T>& a, int grid, cudaStream_t s) {
  const size_t smem = replay_smem<T>(a.nb, NBUF);
  ensure_dyn_smem<k_replay<T, NBUF>>(smem);
  ProfScope ps_("k_replay", s);
  k_replay<T, NBUF><<<grid, NT, smem, s>>>(a);
}

template <typename T>
void launch_replay(const ReplayArgs<T>& a, int grid, cudaStream_t s) {
  switch (replay_nbuf<T>(a.nb)) {
    case 6: launch_replay_n<T, 6>(a, grid, s); break;
    case 4: launch_replay_n<T, 4>(a, grid, s); break;
    case 3: launch_replay_n<T, 3>(a, grid, s); break;
    default: launch_replay_n<T, 2>(a, grid, s); break;
  }
}

// Resident CTAs per SM of the launch (1 when its ring takes most of the shared memory).
template <typename T>
int replay_blocks_per_sm(int nb) {
  const int q = replay_nbuf<T>(nb);
  const size_t smem = replay_smem<T>(nb, q);
  int b = 0;
  cudaError_t e;
  switch (q) {
    case 6: ensure_dyn_smem<k_replay<T, 6>>(smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_replay<T, 6>, NT, smem); break;
    case 4: ensure_dyn_smem<k_replay<T, 4>>(smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_replay<T, 4>, NT, smem); break;
    case 3: ensure_dyn_smem<k_replay<T, 3>>(smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_replay<T, 3>, NT, smem); break;
    default: ensure_dyn_smem<k_replay<T, 2>>(smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_replay<T, 2>, NT, smem); break;
  }
  if (e != cudaSuccess) return 1;
  return b > 0 ? b : 1;
}

template bool replay_fits<float>(int);
template bool replay_fits<double>(int);
template void launch_replay<float>(const ReplayArgs<float>&, int, cudaStream_t);
template void launch_replay<double>(const ReplayArgs<double>&, int, cudaStream_t);
template int replay_blocks_per_sm<float>(int);
template int replay_blocks_per_sm<double>(int);

}  // namespace luqr
