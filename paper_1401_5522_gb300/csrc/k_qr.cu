// QR step (Alg. 3) with the kernels of Alg. 4: GEQRT / UNMQR on single tiles and
// TSQRT-TSMQR (square eliminated tile) or TTQRT-TTMQR (triangular eliminated tile) on
// tile pairs.  Reflectors follow the LAPACK dlarfg convention and are kept in
// compact-WY form per inner block of IB columns: Q_b = I - V T V^T with T (IB x IB)
// upper triangular (Schreiber-Van Loan forward recurrence); Q^T is applied as
// C <- C - V (T^T (V^T C)).  T blocks are stored IB x nb per tile for the second pass.
#include "internal.cuh"

#include <type_traits>

namespace luqr {

constexpr int VST = IB + 1;   // row stride of V / panel blocks in shared memory
constexpr int TST = IB + 1;   // row stride of T and Gram blocks

template <int SW>
struct Cst { static constexpr int v = SW + 1; };

// ---------------------------------------------------------------- FP32 tensor-core path
// For FP32 tiles the three products of apply_block run on the tensor cores with 3xTF32
// splitting: x = hi + lo with hi = tf32(x), lo = tf32(x - hi); a*b ~ ah*bh + ah*bl + al*bh
// (al*bl dropped), FP32 accumulation.  mma.sync m16n8k8 fragments (A row-major 16x8,
// B column-major 8x8): a0=(g,t) a1=(g+8,t) a2=(g,t+4) a3=(g+8,t+4); b0=(t,g) b1=(t+4,g);
// c0=(g,2t) c1=(g,2t+1) c2=(g+8,2t) c3=(g+8,2t+1) with g = lane/4, t = lane%4.
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void split3(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// d += a b with 3xTF32 on operands already split (small terms first).
__device__ __forceinline__ void mma3s(float* d, const uint32_t* ah, const uint32_t* al,
                                      const uint32_t* bh, const uint32_t* bl) {
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}
// Splits an A fragment (4 values) once, so that it serves every n-tile of a k-step.
__device__ __forceinline__ void split_a(const float* a, uint32_t* ah, uint32_t* al) {
#pragma unroll
  for (int i = 0; i < 4; ++i) split3(a[i], ah[i], al[i]);
}
// d += a b with 3xTF32, A pre-split.
__device__ __forceinline__ void mma3a(float* d, const uint32_t* ah, const uint32_t* al,
                                      const float* b) {
  uint32_t bh[2], bl[2];
  split3(b[0], bh[0], bl[0]);
  split3(b[1], bh[1], bl[1]);
  mma3s(d, ah, al, bh, bl);
}

// Stacked-operand helpers: rows 0..IB-1 come from the top block, rows IB.. from the bottom.
__device__ __forceinline__ float vstk(const float* Vtop, const float* Vbot, bool unit_top, int k,
                                      int j) {
  if (k >= IB) return Vbot[(k - IB) * VST + j];
  if (k == j) return 1.0f;
  return (unit_top && k > j) ? Vtop[k * VST + j] : 0.0f;
}

// XV: V is stored explicitly and contiguously, [Vtop; Vbot] = Vtop[0 .. IB + nbot) with its
// unit diagonal and the zeros above it written out (Vbot == Vtop + IB * VST), so its entries
// are plain loads instead of the stacked-operand selection.
template <int SW, bool XV = false>
__device__ void apply_block_mma(const float* Vtop, const float* Vbot, int nbot, const float* Ts,
                                float* Ctop, float* Cbot, float* Ws, float* W2s, bool unit_top) {
  constexpr int CST = SW + 1;
  constexpr int NTN = SW / 8;          // n-tiles of 8 columns
  constexpr int NPW = NTN / 4;         // n-tiles per warp in the 32-row products
  static_assert(NPW >= 1, "tensor-core path needs SW >= 32");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int K1 = IB + nbot;
  auto cstk = [&](int k, int c) -> float {
    return k < IB ? Ctop[k * CST + c] : Cbot[(k - IB) * CST + c];
  };
  auto vv = [&](int k, int j) -> float {
    if constexpr (XV) return Vtop[k * VST + j];
    else return vstk(Vtop, Vbot, unit_top, k, j);
  };
  // ---- W (IB x SW) = [Vtop; Vbot]^T [Ctop; Cbot]
  {
    const int m0 = (warp & 1) * 16;
    const int nbase = (warp >> 1) * NPW;
    float acc[NPW][4];
#pragma unroll
    for (int q = 0; q < NPW; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    for (int k0 = 0; k0 < K1; k0 += 8) {
      float a[4];
      a[0] = vv(k0 + t, m0 + g);
      a[1] = vv(k0 + t, m0 + g + 8);
      a[2] = vv(k0 + t + 4, m0 + g);
      a[3] = vv(k0 + t + 4, m0 + g + 8);
      uint32_t ah[4], al[4];
      split_a(a, ah, al);
#pragma unroll
      for (int q = 0; q < NPW; ++q) {
        const int n0 = (nbase + q) * 8;
        float b[2] = {cstk(k0 + t, n0 + g), cstk(k0 + t + 4, n0 + g)};
        mma3a(acc[q], ah, al, b);
      }
    }
#pragma unroll
    for (int q = 0; q < NPW; ++q) {
      const int n0 = (nbase + q) * 8;
      Ws[(m0 + g) * CST + n0 + 2 * t] = acc[q][0];
      Ws[(m0 + g) * CST + n0 + 2 * t + 1] = acc[q][1];
      Ws[(m0 + g + 8) * CST + n0 + 2 * t] = acc[q][2];
      Ws[(m0 + g + 8) * CST + n0 + 2 * t + 1] = acc[q][3];
    }
  }
  __syncthreads();
  // ---- W2 = T^T W (T upper triangular, stored with zeros below the diagonal)
  {
    const int m0 = (warp & 1) * 16;
    const int nbase = (warp >> 1) * NPW;
    float acc[NPW][4];
#pragma unroll
    for (int q = 0; q < NPW; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
#pragma unroll
    for (int k0 = 0; k0 < IB; k0 += 8) {
      float a[4] = {Ts[(k0 + t) * TST + m0 + g], Ts[(k0 + t) * TST + m0 + g + 8],
                    Ts[(k0 + t + 4) * TST + m0 + g], Ts[(k0 + t + 4) * TST + m0 + g + 8]};
      uint32_t ah[4], al[4];
      split_a(a, ah, al);
#pragma unroll
      for (int q = 0; q < NPW; ++q) {
        const int n0 = (nbase + q) * 8;
        float b[2] = {Ws[(k0 + t) * CST + n0 + g], Ws[(k0 + t + 4) * CST + n0 + g]};
        mma3a(acc[q], ah, al, b);
      }
    }
    // W2 is stored split: hi parts in W2s, lo parts in Ws (free once every warp has read W)
    __syncthreads();
    uint32_t* W2h = reinterpret_cast<uint32_t*>(W2s);
    uint32_t* W2l = reinterpret_cast<uint32_t*>(Ws);
#pragma unroll
    for (int q = 0; q < NPW; ++q) {
      const int n0 = (nbase + q) * 8;
      const int o[4] = {(m0 + g) * CST + n0 + 2 * t, (m0 + g) * CST + n0 + 2 * t + 1,
                        (m0 + g + 8) * CST + n0 + 2 * t, (m0 + g + 8) * CST + n0 + 2 * t + 1};
#pragma unroll
      for (int e = 0; e < 4; ++e) split3(acc[q][e], W2h[o[e]], W2l[o[e]]);
    }
  }
  __syncthreads();
  // ---- [Ctop; Cbot] -= [Vtop; Vbot] W2   (accumulator starts from C, A negated)
  {
    const int MT = K1 / 16;
    for (int mt = warp; mt < MT; mt += NT / 32) {
      const int m0 = mt * 16;
      float* rowA = (m0 < IB) ? Ctop + m0 * CST : Cbot + (m0 - IB) * CST;
      float acc[NTN][4];
#pragma unroll
      for (int q = 0; q < NTN; ++q) {
        const int n0 = q * 8;
        acc[q][0] = rowA[g * CST + n0 + 2 * t];
        acc[q][1] = rowA[g * CST + n0 + 2 * t + 1];
        acc[q][2] = rowA[(g + 8) * CST + n0 + 2 * t];
        acc[q][3] = rowA[(g + 8) * CST + n0 + 2 * t + 1];
      }
      const uint32_t* W2h = reinterpret_cast<const uint32_t*>(W2s);
      const uint32_t* W2l = reinterpret_cast<const uint32_t*>(Ws);
#pragma unroll
      for (int k0 = 0; k0 < IB; k0 += 8) {
        float a[4] = {-vv(m0 + g, k0 + t), -vv(m0 + g + 8, k0 + t), -vv(m0 + g, k0 + t + 4),
                      -vv(m0 + g + 8, k0 + t + 4)};
        uint32_t ah[4], al[4];
        split_a(a, ah, al);
#pragma unroll
        for (int q = 0; q < NTN; ++q) {
          const int n0 = q * 8;
          const int o0 = (k0 + t) * CST + n0 + g, o1 = (k0 + t + 4) * CST + n0 + g;
          const uint32_t bh[2] = {W2h[o0], W2h[o1]}, bl[2] = {W2l[o0], W2l[o1]};
          mma3s(acc[q], ah, al, bh, bl);
        }
      }
#pragma unroll
      for (int q = 0; q < NTN; ++q) {
        const int n0 = q * 8;
        rowA[g * CST + n0 + 2 * t] = acc[q][0];
        rowA[g * CST + n0 + 2 * t + 1] = acc[q][1];
        rowA[(g + 8) * CST + n0 + 2 * t] = acc[q][2];
        rowA[(g + 8) * CST + n0 + 2 * t + 1] = acc[q][3];
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- block application
// [Ctop; Cbot] <- (I - V T V^T)^T [Ctop; Cbot] for V = [Vtop; Vbot].
// Vtop is unit lower triangular (entries below its diagonal) when unit_top, else I.
// XV (tensor-core path only): V is explicit and contiguous as apply_block_mma states; the
// CUDA-core path reads the same matrix through unit_top.
template <typename T, int SW, bool XV = false>
__device__ void apply_block(const T* Vtop, const T* Vbot, int nbot, const T* Ts, T* Ctop, T* Cbot,
                            int w, T* Ws, T* W2s, bool unit_top) {
  if constexpr (std::is_same<T, float>::value && SW >= 32) {
    (void)w;
    apply_block_mma<SW, XV>(Vtop, Vbot, nbot, Ts, Ctop, Cbot, Ws, W2s, unit_top);
    return;
  }
  constexpr int CST = Cst<SW>::v;
  constexpr int JR = IB * SW / NT;
  static_assert(JR >= 1, "slab too narrow");
  const int tid = threadIdx.x;
  const int c = tid % SW, jg = tid / SW;
  if (c < w) {
    T acc[JR];
#pragma unroll
    for (int q = 0; q < JR; ++q) acc[q] = Ctop[(jg * JR + q) * CST + c];
    if (unit_top) {
      for (int a = 1; a < IB; ++a) {
        const T ca = Ctop[a * CST + c];
#pragma unroll
        for (int q = 0; q < JR; ++q) {
          const int j = jg * JR + q;
          if (a > j) acc[q] += Vtop[a * VST + j] * ca;
        }
      }
    }
    for (int r = 0; r < nbot; ++r) {
      const T cr = Cbot[r * CST + c];
      const T* vr = Vbot + r * VST + jg * JR;
#pragma unroll
      for (int q = 0; q < JR; ++q) acc[q] += vr[q] * cr;
    }
#pragma unroll
    for (int q = 0; q < JR; ++q) Ws[(jg * JR + q) * CST + c] = acc[q];
  }
  __syncthreads();
  if (c < w) {
#pragma unroll
    for (int q = 0; q < JR; ++q) {
      const int j = jg * JR + q;
      T s = (T)0;
      for (int a = 0; a <= j; ++a) s += Ts[a * TST + j] * Ws[a * CST + c];
      W2s[j * CST + c] = s;
    }
  }
  __syncthreads();
  constexpr int G = NT / SW;
  if (c < w) {
    for (int a = jg; a < IB; a += G) {
      T s = W2s[a * CST + c];
      if (unit_top)
        for (int j = 0; j < a; ++j) s += Vtop[a * VST + j] * W2s[j * CST + c];
      Ctop[a * CST + c] -= s;
    }
    for (int r = jg; r < nbot; r += G) {
      const T* vr = Vbot + r * VST;
      T s = (T)0;
#pragma unroll 8
      for (int j = 0; j < IB; ++j) s += vr[j] * W2s[j * CST + c];
      Cbot[r * CST + c] -= s;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Householder helpers
// Thread 0 forms the reflector of [a0; x] with sum(x^2) = ss (dlarfg convention).
template <typename T>
__device__ __forceinline__ void make_reflector(T a0, T ss, T* beta, T* tau, T* denom) {
  if (ss == (T)0) {
    *beta = a0; *tau = (T)0; *denom = (T)1;
  } else {
    const T nrm = sqrt(a0 * a0 + ss);
    const T b = (a0 >= (T)0) ? -nrm : nrm;
    *beta = b;
    *tau = (b - a0) / b;
    *denom = a0 - b;
  }
}

// Panel QR of IB columns with the block's T built alongside (dlarfg reflectors, the
// Schreiber-Van Loan recurrence T[0:j, j] = -tau_j T[0:j, 0:j] G[0:j, j], G = V^T V).
// SINGLE (GEQRT): the panel is Ps (nrows x IB); reflector j has a unit at row j and acts on
//   rows j.. ; the "top" row of step j is row j of Ps.
// pair (TS/TT):  the panel is [Rs; Ps]; reflector j is e_j in Rs plus rows [0, hi_j) of Ps
//   (hi_j = min(jb + j + 1, nrows) for TT, nrows for TS); the top row is row j of Rs.
// Thread (warp w, lane c) owns column c on rows r = w (mod 8), so the reductions over rows
// are 8 partials per column; the reflector columns stay unscaled (scale 1/(a0 - beta) kept
// in sinv) until the end of the panel, which removes one barrier per column.
// scratch: >= 8*IB + 8 + 2*IB + 2 elements.
template <typename T, bool SINGLE>
__device__ void panel_qr(T* Rs, T* Ps, int nrows, bool tri, int jb, T* tau_s, T* Ts, T* scratch) {
  static_assert(NT == 256 && IB == 32, "thread map assumes 8 warps x 32 columns");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  T* part = scratch;               // [8][IB] partial dot products
  T* nrm = part + 8 * IB;          // [8] partial squared norms of the next column
  T* wv = nrm + 8;                 // [IB] w_c (c > j) or G[c][j] (c < j)
  T* sinv = wv + IB;               // [IB] scale of each reflector column
  T* sc = sinv + IB;               // [2] tau, inv of the current column
  auto lo = [&](int j) { return SINGLE ? j + 1 : 0; };
  auto hi = [&](int j) { return SINGLE ? nrows : (tri ? min(jb + j + 1, nrows) : nrows); };
  auto top = [&](int j, int c) -> T& { return SINGLE ? Ps[j * VST + c] : Rs[j * VST + c]; };
  const int c = lane;
  // partial norm of column 0
  if (c == 0) {
    T sq = (T)0;
    for (int r = lo(0) + ((w - lo(0)) % 8 + 8) % 8; r < hi(0); r += 8) sq += Ps[r * VST] * Ps[r * VST];
    nrm[w] = sq;
  }
  __syncthreads();
  for (int j = 0; j < IB; ++j) {
    const int l0 = lo(j), h0 = hi(j);
    const int rs = l0 + ((w - l0) % 8 + 8) % 8;     // first row of this warp in [l0, h0)
    // [A] partial dots of the (unscaled) column j with every column
    {
      T d = (T)0;
      if (c != j)
        for (int r = rs; r < h0; r += 8) d += Ps[r * VST + j] * Ps[r * VST + c];
      part[w * IB + c] = d;
    }
    __syncthreads();
    // [B] warp 0: reflector, w_c / G column, T column
    if (w == 0) {
      T ss = (T)0;
#pragma unroll
      for (int q = 0; q < 8; ++q) ss += nrm[q];
      const T a0 = top(j, j);
      T beta, tau, denom;
      make_reflector<T>(a0, ss, &beta, &tau, &denom);
      const T inv = (tau == (T)0) ? (T)0 : (T)1 / denom;
      T dsum = (T)0;
#pragma unroll
      for (int q = 0; q < 8; ++q) dsum += part[q * IB + c];
      if (c > j) wv[c] = top(j, c) + inv * dsum;
      else if (c < j) wv[c] = sinv[c] * (inv * dsum + (SINGLE ? Ps[j * VST + c] : (T)0));
      __syncwarp();
      T tcol = (T)0;
      if (c < j) {
        T acc = (T)0;
        for (int b = c; b < j; ++b) acc += Ts[c * TST + b] * wv[b];
        tcol = -tau * acc;
      } else if (c == j) {
        tcol = tau;
      }
      Ts[c * TST + j] = tcol;
      if (c == 0) {
        top(j, j) = beta;
        tau_s[j] = tau;
        sinv[j] = inv;
        sc[0] = tau;
        sc[1] = inv;
      }
    }
    __syncthreads();
    // [C] update of the columns right of j; partial norm of column j+1
    {
      const T tau = sc[0], inv = sc[1];
      if (c > j && tau != (T)0) {
        const T f = tau * inv * wv[c];
        for (int r = rs; r < h0; r += 8) Ps[r * VST + c] -= f * Ps[r * VST + j];
        if (w == 0) top(j, c) -= tau * wv[c];
      }
      if (j + 1 < IB) {
        __syncwarp();
        if (c == j + 1) {
          const int l1 = lo(j + 1), h1 = hi(j + 1);
          T sq = (T)0;
          for (int r = l1 + ((w - l1) % 8 + 8) % 8; r < h1; r += 8) sq += Ps[r * VST + c] * Ps[r * VST + c];
          nrm[w] = sq;
        }
      }
    }
    __syncthreads();
  }
  // scale the reflector columns (column c: rows [lo(c), hi(c)); zero when tau = 0)
  for (int r = w; r < nrows; r += 8) {
    if (r >= lo(c) && r < hi(c)) {
      const T f = sinv[c];
      Ps[r * VST + c] = (f == (T)0) ? (T)0 : Ps[r * VST + c] * f;
    }
  }
  __syncthreads();
}

// Register form of panel_qr (same operations per element, same summation orders, so the
// same bits): thread (warp w, lane c) keeps rows w + 8q (q < RPT) of panel column c in
// registers; column j's values reach the other lanes by warp shuffles.  One block barrier
// per column: every warp reads the eight partial norms and dot products of column j,
// forms the reflector itself (identical inputs, identical results), updates its rows and
// writes the partials of column j+1 into the other half of a double buffer.  The G
// entries of each column are parked below the diagonal of Ts (G[c][j] at Ts[j][c]) and T
// is formed after the loop, one row per lane (T[c][j] = -tau_j sum_{b=c}^{j-1} T[c][b]
// G[b][j]: rows are independent); the parked entries are cleared afterwards.  For pairs,
// row j of R is read into registers during column j-1 (nobody writes it then), because
// warp 0 updates it during column j while the other warps still form the reflector.
// scratch: >= 2*8*IB + 2*8 + 2*IB + IB elements.
template <typename T, bool SINGLE, int RPT>
__device__ void panel_qr_reg(T* Rs, T* Ps, int nrows, bool tri, int jb, T* tau_s, T* Ts,
                             T* scratch) {
  static_assert(NT == 256 && IB == 32, "thread map assumes 8 warps x 32 columns");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  T* part = scratch;               // [2][8][IB] partial dots (double buffered by column)
  T* nrm = part + 2 * 8 * IB;      // [2][8] partial squared norms
  T* topbuf = nrm + 2 * 8;         // [2][IB] row j of the panel (single)
  T* sinv = topbuf + 2 * IB;       // [IB]
  auto lo = [&](int j) { return SINGLE ? j + 1 : 0; };
  auto hi = [&](int j) { return SINGLE ? nrows : (tri ? min(jb + j + 1, nrows) : nrows); };
  const int c = lane;
  T x[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = w + 8 * q;
    x[q] = (r < nrows) ? Ps[r * VST + c] : (T)0;
  }
  // partials of column 0 (its dots with every column, its partial norm, row 0 when single)
  {
    const int l0 = lo(0), h0 = hi(0);
    T d = (T)0, sq = (T)0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = w + 8 * q;
      const T xj = __shfl_sync(0xffffffffu, x[q], 0);
      if (r >= l0 && r < h0) {
        d += xj * x[q];
        sq += x[q] * x[q];
      }
      if (SINGLE && r == 0) topbuf[c] = x[q];
    }
    part[w * IB + c] = (c != 0) ? d : (T)0;
    if (c == 0) nrm[w] = sq;
  }
  T ra0 = (T)0, rc = (T)0;   // pairs: R[j][j] and R[j][c] as they stand before column j
  if (!SINGLE) {
    ra0 = Rs[0];
    rc = Rs[c];
  }
  __syncthreads();
#pragma unroll 1
  for (int j = 0; j < IB; ++j) {
    const int cur = j & 1, nxt = cur ^ 1;
    const int l0 = lo(j);
    const T* pc = part + cur * 8 * IB;
    // reflector of column j (every warp, identical arithmetic)
    T ss = (T)0, dsum = (T)0;
#pragma unroll
    for (int q = 0; q < 8; ++q) ss += nrm[cur * 8 + q];
#pragma unroll
    for (int q = 0; q < 8; ++q) dsum += pc[q * IB + c];
    const T a0 = SINGLE ? topbuf[cur * IB + j] : ra0;
    T beta, tau, denom;
    make_reflector<T>(a0, ss, &beta, &tau, &denom);
    const T inv = (tau == (T)0) ? (T)0 : (T)1 / denom;
    const T topc = SINGLE ? topbuf[cur * IB + c] : rc;
    const T wc = (c > j) ? topc + inv * dsum : (T)0;
    if (w == 0) {
      if (c < j) Ts[j * TST + c] = sinv[c] * (inv * dsum + (SINGLE ? topc : (T)0));
      if (c == 0) {
        tau_s[j] = tau;
        sinv[j] = inv;
      }
      if (!SINGLE) {
        if (c == j) Rs[j * VST + j] = beta;
        else if (c > j && tau != (T)0) Rs[j * VST + c] -= tau * wc;
      }
    }
    // update of the columns right of j on this warp's rows, then the partials of j+1.
    // Rows at or past hi(j) hold exact zeros in every column from j on (the zero padding
    // past nrows; for TT also the rows below the triangle, which no earlier reflector
    // reaches), so the update leaves them at zero and they add zeros to the sums: only
    // rows above the reflector need a test, and those exist only in GEQRT with r <= j < IB,
    // i.e. q < IB / 8.  Same bits as testing every row, for finite panels.
    const T f = tau * inv * wc;
    const bool upd = c > j && tau != (T)0;
    const int l1 = lo(j + 1);
    T d = (T)0, sq = (T)0;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int r = w + 8 * q;
      const T xj = __shfl_sync(0xffffffffu, x[q], j);
      if (SINGLE && q < IB / 8) {
        if (upd && r >= l0) x[q] -= f * xj;
        if (r == j) {
          if (c == j) x[q] = beta;
          else if (upd) x[q] -= tau * wc;
        }
      } else if (upd) {
        x[q] -= f * xj;
      }
    }
    if (j + 1 < IB) {
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int r = w + 8 * q;
        const T xj1 = __shfl_sync(0xffffffffu, x[q], j + 1);
        if (SINGLE && q < IB / 8) {
          if (r >= l1) {
            d += xj1 * x[q];
            sq += x[q] * x[q];
          }
          if (r == j + 1) topbuf[nxt * IB + c] = x[q];
        } else {
          d += xj1 * x[q];
          sq += x[q] * x[q];
        }
      }
      part[nxt * 8 * IB + w * IB + c] = (c != j + 1) ? d : (T)0;
      if (c == j + 1) nrm[nxt * 8 + w] = sq;
      if (!SINGLE) {
        ra0 = Rs[(j + 1) * VST + j + 1];
        rc = Rs[(j + 1) * VST + c];
      }
    }
    __syncthreads();
  }
  // T, one row per lane of warp 0 (reads G below the diagonal, writes on and above it).
  // Lane c runs only its own terms b = c .. j-1 of each entry, reading its row of T back
  // from shared memory (row c on and above the diagonal: written and read by lane c
  // alone, never one of the G entries below the diagonal that the other lanes read).
  if (w == 0) {
    const T* trow = Ts + c * TST;
#pragma unroll 1
    for (int j = c; j < IB; ++j) {
      const T* gj = Ts + j * TST;          // G[b][j] parked at Ts[j][b], b < j
      T acc = (T)0;
#pragma unroll 4
      for (int b = c; b < j; ++b) acc += trow[b] * gj[b];
      const T tj = tau_s[j];
      Ts[c * TST + j] = (j == c) ? tj : -tj * acc;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < IB; ++j)
      if (j < c) Ts[c * TST + j] = (T)0;
  }
  // scale the reflector columns and store the panel back
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int r = w + 8 * q;
    if (r < nrows) {
      T v = x[q];
      if (r >= lo(c) && r < hi(c)) {
        const T fs = sinv[c];
        v = (fs == (T)0) ? (T)0 : v * fs;
      }
      Ps[r * VST + c] = v;
    }
  }
  __syncthreads();
}

// Dispatches FP32 panels to the register form (FP64 shuffles and register pressure make the
// shared-memory form faster for doubles on this part).
template <typename T, bool SINGLE>
__device__ void panel_qr_any(T* Rs, T* Ps, int nrows, bool tri, int jb, T* tau_s, T* Ts,
                             T* scratch) {
  if constexpr (sizeof(T) == 8) {
    panel_qr<T, SINGLE>(Rs, Ps, nrows, tri, jb, tau_s, Ts, scratch);
    return;
  }
  if (nrows <= 64) panel_qr_reg<T, SINGLE, 8>(Rs, Ps, nrows, tri, jb, tau_s, Ts, scratch);
  else if (nrows <= 128) panel_qr_reg<T, SINGLE, 16>(Rs, Ps, nrows, tri, jb, tau_s, Ts, scratch);
  else if (nrows <= 256) panel_qr_reg<T, SINGLE, 32>(Rs, Ps, nrows, tri, jb, tau_s, Ts, scratch);
  else panel_qr_reg<T, SINGLE, 64>(Rs, Ps, nrows, tri, jb, tau_s, Ts, scratch);
}

// Row-fastest walk of an R x C index space by the CTA's NT threads, f(r, c) for every
// r < R, c < C: the same elements as idx = tid, tid + NT, ... < R*C with r = idx % R and
// c = idx / R, without a division per element (one at the start; afterwards idx + NT moves
// r by NT % R and c by NT / R, with one carry).
template <typename F>
__device__ __forceinline__ void walk_rc(int R, int C, F&& f) {
  int r = (int)threadIdx.x % R, c = (int)threadIdx.x / R;
  const int dr = NT % R, dc = NT / R;
  while (c < C) {
    f(r, c);
    r += dr;
    c += dc;
    if (r >= R) {
      r -= R;
      ++c;
    }
  }
}

// ---------------------------------------------------------------- shared memory plans
template <typename T, int SW>
struct Plan {
  static constexpr int CST = SW + 1;
  static size_t geqrt(int nb) {
    return sizeof(T) * ((size_t)nb * VST + (size_t)nb * CST + 2 * IB * TST + 2 * IB * CST + IB + 32 + 4);
  }
  static size_t unmqr(int nb) {
    return sizeof(T) * ((size_t)nb * CST + (size_t)nb * VST + IB * TST + 2 * IB * CST);
  }
  static size_t pair_qrt(int nb) {
    return sizeof(T) * ((size_t)IB * VST + (size_t)nb * VST + IB * CST + (size_t)nb * CST +
                        2 * IB * TST + 2 * IB * CST + IB + 32 + 4);
  }
  static size_t pair_apply(int nb) {
    return sizeof(T) * (2 * (size_t)nb * CST + (size_t)nb * VST + IB * TST + 2 * IB * CST);
  }
};

// ---------------------------------------------------------------- GEQRT
template <typename T, int SW>
__global__ void __launch_bounds__(NT) k_geqrt(Mat<T> F, int k, int nb, TileList tl, T* Tk,
                                              const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_QR) return;
  constexpr int CST = SW + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ps = reinterpret_cast<T*>(smem_raw);
  T* Cs = Ps + (size_t)nb * VST;
  T* Ts = Cs + (size_t)nb * CST;
  T* Gs = Ts + IB * TST;
  T* Ws = Gs + IB * TST;
  T* W2s = Ws + IB * CST;
  T* tau_s = W2s + IB * CST;
  T* red = tau_s + IB;
  T* bc = red + 32;
  const int i = tl.i0 + blockIdx.x * tl.istride;
  T* tile = F.p + (int64_t)i * nb + (int64_t)k * nb * F.ld;
  T* Tslot = Tk + ((size_t)i * 2 + 0) * IB * nb;
  const int tid = threadIdx.x;
  for (int jb = 0; jb < nb; jb += IB) {
    const int nrows = nb - jb;
    walk_rc(nrows, IB, [&](int r, int j) {
      cp_async(&Ps[r * VST + j], &tile[(jb + r) + (int64_t)(jb + j) * F.ld]);
    });
    cp_async_wait_all();
    __syncthreads();
    panel_qr_any<T, true>(nullptr, Ps, nrows, false, jb, tau_s, Ts, Gs);
    walk_rc(nrows, IB, [&](int r, int j) {
      tile[(jb + r) + (int64_t)(jb + j) * F.ld] = Ps[r * VST + j];
    });
    for (int idx = tid; idx < IB * IB; idx += NT) {
      const int a = idx % IB, j = idx / IB;
      Tslot[a + (size_t)(jb + j) * IB] = Ts[a * TST + j];
    }
    if (jb + IB < nb) {
      // R is stored: the top block becomes V's explicit unit-lower part for the updates
      __syncthreads();
      for (int idx = tid; idx < IB * IB; idx += NT) {
        const int a = idx % IB, j = idx / IB;
        if (a <= j) Ps[a * VST + j] = (a == j) ? (T)1 : (T)0;
      }
    }
    for (int cc = jb + IB; cc < nb; cc += SW) {
      const int w = min(SW, nb - cc);
      __syncthreads();
      walk_rc(nrows, SW, [&](int r, int c) {
        if (c < w) cp_async(&Cs[r * CST + c], &tile[(jb + r) + (int64_t)(cc + c) * F.ld]);
      });
      cp_async_wait_all();
      __syncthreads();
      apply_block<T, SW, true>(Ps, Ps + IB * VST, nrows - IB, Ts, Cs, Cs + IB * CST, w, Ws, W2s,
                               true);
      walk_rc(nrows, SW, [&](int r, int c) {
        if (c < w) tile[(jb + r) + (int64_t)(cc + c) * F.ld] = Cs[r * CST + c];
      });
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- UNMQR
template <typename T, int SW>
__global__ void __launch_bounds__(NT) k_unmqr(Mat<const T> F, int k, int nb, TileList tl,
                                              const T* Tk, Mat<T> C, int64_t c0, int64_t c1,
                                              const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_QR) return;
  constexpr int CST = SW + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Cs = reinterpret_cast<T*>(smem_raw);
  T* Vs = Cs + (size_t)nb * CST;
  T* Ts = Vs + (size_t)nb * VST;
  T* Ws = Ts + IB * TST;
  T* W2s = Ws + IB * CST;
  const int i = tl.i0 + blockIdx.y * tl.istride;
  const int64_t cb = c0 + (int64_t)blockIdx.x * SW;
  const int w = (int)min((int64_t)SW, c1 - cb);
  const T* V = F.p + (int64_t)i * nb + (int64_t)k * nb * F.ld;
  const T* Tslot = Tk + ((size_t)i * 2 + 0) * IB * nb;
  const int tid = threadIdx.x;
  T* Cg = C.p + (int64_t)i * nb + cb * C.ld;
  walk_rc(nb, SW, [&](int r, int c) {
    if (c < w) cp_async(&Cs[r * CST + c], &Cg[r + (int64_t)c * C.ld]);
  });
  for (int jb = 0; jb < nb; jb += IB) {
    const int nrows = nb - jb;
    walk_rc(nrows, IB, [&](int r, int j) {
      cp_async(&Vs[r * VST + j], &V[(jb + r) + (int64_t)(jb + j) * F.ld]);
    });
    for (int idx = tid; idx < IB * IB; idx += NT) {
      const int a = idx % IB, j = idx / IB;
      cp_async(&Ts[a * TST + j], &Tslot[a + (size_t)(jb + j) * IB]);
    }
    cp_async_wait_all();
    __syncthreads();
    apply_block<T, SW>(Vs, Vs + IB * VST, nrows - IB, Ts, Cs + jb * CST, Cs + (jb + IB) * CST, w,
                       Ws, W2s, true);
  }
  walk_rc(nb, SW, [&](int r, int c) {
    if (c < w) Cg[r + (int64_t)c * C.ld] = Cs[r * CST + c];
  });
}

// ---------------------------------------------------------------- TSQRT / TTQRT
template <typename T, int SW>
__global__ void __launch_bounds__(NT) k_pair_qrt(Mat<T> F, int k, int nb, TileList tl, bool tri,
                                                 T* Tk, const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_QR) return;
  constexpr int CST = SW + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Rs = reinterpret_cast<T*>(smem_raw);
  T* Ps = Rs + IB * VST;
  T* Ct = Ps + (size_t)nb * VST;
  T* Cb = Ct + IB * CST;
  T* Ts = Cb + (size_t)nb * CST;
  T* Gs = Ts + IB * TST;
  T* Ws = Gs + IB * TST;
  T* W2s = Ws + IB * CST;
  T* tau_s = W2s + IB * CST;
  T* red = tau_s + IB;
  T* bc = red + 32;
  const int i = tl.i0 + blockIdx.x * tl.istride;
  const int e = i - tl.eoff;
  T* R = F.p + (int64_t)e * nb + (int64_t)k * nb * F.ld;
  T* A = F.p + (int64_t)i * nb + (int64_t)k * nb * F.ld;
  T* Tslot = Tk + ((size_t)i * 2 + 1) * IB * nb;
  const int tid = threadIdx.x;
  for (int jb = 0; jb < nb; jb += IB) {
    const int rl = tri ? jb + IB : nb;
    for (int idx = tid; idx < IB * IB; idx += NT) {
      const int a = idx % IB, j = idx / IB;
      if (a <= j) cp_async(&Rs[a * VST + j], &R[(jb + a) + (int64_t)(jb + j) * F.ld]);
      else Rs[a * VST + j] = (T)0;
    }
    walk_rc(rl, IB, [&](int r, int j) {
      if (!tri || r <= jb + j) cp_async(&Ps[r * VST + j], &A[r + (int64_t)(jb + j) * F.ld]);
      else Ps[r * VST + j] = (T)0;
    });
    cp_async_wait_all();
    __syncthreads();
    panel_qr_any<T, false>(Rs, Ps, rl, tri, jb, tau_s, Ts, Gs);
    for (int idx = tid; idx < IB * IB; idx += NT) {
      const int a = idx % IB, j = idx / IB;
      if (a <= j) R[(jb + a) + (int64_t)(jb + j) * F.ld] = Rs[a * VST + j];
      Tslot[a + (size_t)(jb + j) * IB] = Ts[a * TST + j];
    }
    walk_rc(rl, IB, [&](int r, int j) {
      if (!tri || r <= jb + j) A[r + (int64_t)(jb + j) * F.ld] = Ps[r * VST + j];
    });
    if (jb + IB < nb) {
      // R is stored: Rs becomes the identity on top of V = [I; Ps] for the updates
      __syncthreads();
      for (int idx = tid; idx < IB * IB; idx += NT) {
        const int a = idx % IB, j = idx / IB;
        Rs[a * VST + j] = (a == j) ? (T)1 : (T)0;
      }
    }
    for (int cc = jb + IB; cc < nb; cc += SW) {
      const int w = min(SW, nb - cc);
      __syncthreads();
      for (int idx = tid; idx < IB * SW; idx += NT) {
        const int a = idx % IB, c = idx / IB;
        if (c < w) cp_async(&Ct[a * CST + c], &R[(jb + a) + (int64_t)(cc + c) * F.ld]);
      }
      walk_rc(rl, SW, [&](int r, int c) {
        if (c < w) cp_async(&Cb[r * CST + c], &A[r + (int64_t)(cc + c) * F.ld]);
      });
      cp_async_wait_all();
      __syncthreads();
      apply_block<T, SW, true>(Rs, Ps, rl, Ts, Ct, Cb, w, Ws, W2s, false);
      for (int idx = tid; idx < IB * SW; idx += NT) {
        const int a = idx % IB, c = idx / IB;
        if (c < w) R[(jb + a) + (int64_t)(cc + c) * F.ld] = Ct[a * CST + c];
      }
      walk_rc(rl, SW, [&](int r, int c) {
        if (c < w) A[r + (int64_t)(cc + c) * F.ld] = Cb[r * CST + c];
      });
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- TSMQR / TTMQR
template <typename T, int SW>
__global__ void __launch_bounds__(NT) k_pair_apply(Mat<const T> F, int k, int nb, TileList tl,
                                                   bool tri, const T* Tk, Mat<T> C, int64_t c0,
                                                   int64_t c1, const uint8_t* __restrict__ dec) {
  if (dec[k] != DEC_QR) return;
  constexpr int CST = SW + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* C1s = reinterpret_cast<T*>(smem_raw);
  T* C2s = C1s + (size_t)nb * CST;
  T* Vs = C2s + (size_t)nb * CST;
  T* Ts = Vs + (size_t)nb * VST;
  T* Ws = Ts + IB * TST;
  T* W2s = Ws + IB * CST;
  const int i = tl.i0 + blockIdx.y * tl.istride;
  const int e = i - tl.eoff;
  const int64_t cb = c0 + (int64_t)blockIdx.x * SW;
  const int w = (int)min((int64_t)SW, c1 - cb);
  const T* V = F.p + (int64_t)i * nb + (int64_t)k * nb * F.ld;
  const T* Tslot = Tk + ((size_t)i * 2 + 1) * IB * nb;
  T* C1g = C.p + (int64_t)e * nb + cb * C.ld;
  T* C2g = C.p + (int64_t)i * nb + cb * C.ld;
  const int tid = threadIdx.x;
  walk_rc(nb, SW, [&](int r, int c) {
    if (c < w) {
      cp_async(&C1s[r * CST + c], &C1g[r + (int64_t)c * C.ld]);
      cp_async(&C2s[r * CST + c], &C2g[r + (int64_t)c * C.ld]);
    }
  });
  for (int jb = 0; jb < nb; jb += IB) {
    const int rl = tri ? jb + IB : nb;
    walk_rc(rl, IB, [&](int r, int j) {
      if (!tri || r <= jb + j) cp_async(&Vs[r * VST + j], &V[r + (int64_t)(jb + j) * F.ld]);
      else Vs[r * VST + j] = (T)0;
    });
    for (int idx = tid; idx < IB * IB; idx += NT) {
      const int a = idx % IB, j = idx / IB;
      cp_async(&Ts[a * TST + j], &Tslot[a + (size_t)(jb + j) * IB]);
    }
    cp_async_wait_all();
    __syncthreads();
    apply_block<T, SW>(nullptr, Vs, rl, Ts, C1s + jb * CST, C2s, w, Ws, W2s, false);
  }
  walk_rc(nb, SW, [&](int r, int c) {
    if (c < w) {
      C1g[r + (int64_t)c * C.ld] = C1s[r * CST + c];
      C2g[r + (int64_t)c * C.ld] = C2s[r * CST + c];
    }
  });
}

// ---------------------------------------------------------------- one right-hand side
// ---------------------------------------------------------------- launchers
// The slab width SW is the widest of {64, 32, 16, 8} whose shared-memory plan fits.
enum PlanKind { PLAN_GEQRT, PLAN_UNMQR, PLAN_PAIR_QRT, PLAN_PAIR_APPLY };

template <typename T, int SW>
static size_t plan_bytes(PlanKind kind, int nb) {
  switch (kind) {
    case PLAN_GEQRT: return Plan<T, SW>::geqrt(nb);
    case PLAN_UNMQR: return Plan<T, SW>::unmqr(nb);
    case PLAN_PAIR_QRT: return Plan<T, SW>::pair_qrt(nb);
    default: return Plan<T, SW>::pair_apply(nb);
  }
}

// ncols: columns the launch updates; a narrow target (the second pass on a few right-hand
// sides) takes the narrowest slab that covers it instead of a mostly idle wide one.
template <typename T, typename Fn>
static void pick_sw(PlanKind kind, int nb, Fn&& fn, int64_t ncols = 1 << 30) {
  if (ncols <= 8) fn(std::integral_constant<int, 8>{});
  else if (ncols <= 16 && plan_bytes<T, 16>(kind, nb) <= (size_t)SMEM_MAX)
    fn(std::integral_constant<int, 16>{});
  else if (plan_bytes<T, 64>(kind, nb) <= (size_t)SMEM_MAX) fn(std::integral_constant<int, 64>{});
  else if (plan_bytes<T, 32>(kind, nb) <= (size_t)SMEM_MAX) fn(std::integral_constant<int, 32>{});
  else if (plan_bytes<T, 16>(kind, nb) <= (size_t)SMEM_MAX) fn(std::integral_constant<int, 16>{});
  else fn(std::integral_constant<int, 8>{});
}

template <typename T>
void launch_geqrt(Mat<T> F, int k, int nb, TileList tl, T* Tk, int n, const uint8_t* dec,
                  cudaStream_t s) {
  if (tl.count <= 0) return;
  (void)n;
  pick_sw<T>(PLAN_GEQRT, nb, [&](auto tag) {
    constexpr int SW = decltype(tag)::value;
    ensure_dyn_smem<k_geqrt<T, SW>>(Plan<T, SW>::geqrt(nb));
    {
      ProfScope ps_("k_geqrt", s);
      k_geqrt<T, SW><<<tl.count, NT, Plan<T, SW>::geqrt(nb), s>>>(F, k, nb, tl, Tk, dec);
    }
  });
}

template <typename T>
void launch_unmqr(Mat<const T> F, int k, int nb, TileList tl, const T* Tk, int n, Mat<T> C,
                  int64_t c0, int64_t c1, const uint8_t* dec, cudaStream_t s) {
  if (tl.count <= 0 || c1 <= c0) return;
  (void)n;
  pick_sw<T>(
      PLAN_UNMQR, nb,
      [&](auto tag) {
        constexpr int SW = decltype(tag)::value;
        ensure_dyn_smem<k_unmqr<T, SW>>(Plan<T, SW>::unmqr(nb));
        dim3 grid((unsigned)((c1 - c0 + SW - 1) / SW), (unsigned)tl.count);
        {
          ProfScope ps_("k_unmqr", s);
          k_unmqr<T, SW><<<grid, NT, Plan<T, SW>::unmqr(nb), s>>>(F, k, nb, tl, Tk, C, c0, c1,
                                                                   dec);
        }
      },
      c1 - c0);
}

template <typename T>
void launch_pair_qrt(Mat<T> F, int k, int nb, TileList tl, bool tri, T* Tk, int n,
                     const uint8_t* dec, cudaStream_t s) {
  if (tl.count <= 0) return;
  (void)n;
  pick_sw<T>(PLAN_PAIR_QRT, nb, [&](auto tag) {
    constexpr int SW = decltype(tag)::value;
    ensure_dyn_smem<k_pair_qrt<T, SW>>(Plan<T, SW>::pair_qrt(nb));
    {
      ProfScope ps_(tri ? "k_ttqrt" : "k_tsqrt", s);
      k_pair_qrt<T, SW><<<tl.count, NT, Plan<T, SW>::pair_qrt(nb), s>>>(F, k, nb, tl, tri, Tk, dec);
    }
  });
}

template <typename T>
void launch_pair_apply(Mat<const T> F, int k, int nb, TileList tl, bool tri, const T* Tk, int n,
                       Mat<T> C, int64_t c0, int64_t c1, const uint8_t* dec, cudaStream_t s) {
  if (tl.count <= 0 || c1 <= c0) return;
  (void)n;
  pick_sw<T>(
      PLAN_PAIR_APPLY, nb,
      [&](auto tag) {
        constexpr int SW = decltype(tag)::value;
        ensure_dyn_smem<k_pair_apply<T, SW>>(Plan<T, SW>::pair_apply(nb));
        dim3 grid((unsigned)((c1 - c0 + SW - 1) / SW), (unsigned)tl.count);
        {
          ProfScope ps_(tri ? "k_ttmqr" : "k_tsmqr", s);
          k_pair_apply<T, SW><<<grid, NT, Plan<T, SW>::pair_apply(nb), s>>>(F, k, nb, tl, tri, Tk,
                                                                           C, c0, c1, dec);
        }
      },
      c1 - c0);
}

#define INST(T)                                                                                  \
  template void launch_geqrt<T>(Mat<T>, int, int, TileList, T*, int, const uint8_t*,             \
                                cudaStream_t);                                                   \
  template void launch_unmqr<T>(Mat<const T>, int, int, TileList, const T*, int, Mat<T>,         \
                                int64_t, int64_t, const uint8_t*, cudaStream_t);                 \
  template void launch_pair_qrt<T>(Mat<T>, int, int, TileList, bool, T*, int, const uint8_t*,    \
                                   cudaStream_t);                                                \
  template void launch_pair_apply<T>(Mat<const T>, int, int, TileList, bool, const T*, int,      \
                                     Mat<T>, int64_t, int64_t, const uint8_t*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace luqr
