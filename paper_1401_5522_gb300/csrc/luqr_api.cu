// C interface and host-side step loop of the hybrid LU-QR solver (Alg. 1).
//
// The host enqueues, for every step k, the criterion kernels and BOTH branches
// (LU step of Alg. 2, QR step of Alg. 3/4); the decision lives only in device
// memory (dec[k]) and every branch kernel returns at once unless dec[k] selects it,
// so the factorization runs without a single host synchronisation.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/luqr.h"
#include "internal.cuh"

using namespace luqr;

struct luqr_handle {
  int64_t N = 0, Npad = 0, Wc = 0;
  int nb = 0, n = 0, prec = 0, criterion = 0, tree = 0, group = 4, mumps_mode = 0;
  int tree_small = 0, tree_switch = 0;   // per-step tree: below tree_switch sub-diagonal tiles
  int norm_mode = 0;   // 0 exact ||A_kk^-1||_1, 1 Hager-Higham estimate
  int lu_variant = 0;  // 0 A1 (GETRF of A_kk), 1 A2 (GEQRT of A_kk)
  int domain = 1;      // tiles of the diagonal pivot domain (1: the diagonal tile)
  void* St = nullptr;  // domain * nb x nb scratch of the tall GETRF
  int* dpiv_all = nullptr;  // n x nb row exchanges of the domain (0-based in the domain)
  uint8_t* gate_all = nullptr;  // n bytes of DEC_QR: runs QR-gated kernels unconditionally
  uint8_t* a2gate = nullptr;    // A2: DEC_QR at steps whose decision is LU
  unsigned long long seed = 0;   // LUQR_RANDOM
  double alpha = 0.0;
  bool has_rhs = false;
  cudaStream_t stream = nullptr;
  void* W = nullptr;        // Npad x Wc tiles (+ augmented column), column-major
  void* Tbuf = nullptr;     // n steps x n tiles x 2 kinds x (IB x nb) T blocks
  void* S = nullptr;        // nb x nb GETRF scratch
  int* piv_s = nullptr;
  int* piv_all = nullptr;   // n x nb pivots of LU steps
  double* norms = nullptr;  // n x n tile norms ||A_ik^(k)||_1 (row k holds step k)
  unsigned long long* local = nullptr;
  unsigned long long* away = nullptr;
  double* colsum = nullptr;
  uint8_t* dec = nullptr;
  double* margin = nullptr;
  double* lhs = nullptr;
  double* rhs = nullptr;
  int* status = nullptr;
  uint8_t* forced = nullptr;
  std::vector<char> injected;
  // look-ahead: the bulk trailing update of step k runs on upd_stream while the caller's
  // stream factors panel k+1 (events ev_fact / ev_rest order the two streams)
  cudaStream_t upd_stream = nullptr;
  std::vector<cudaEvent_t> ev_fact, ev_rest;
  cudaEvent_t ev_start = nullptr;
  // FP32 tensor-core trailing updates: W workspace (Npad x Wc, same layout as the trailing
  // matrix), Gram matrices, full compact-WY T and V T^T per tile (double-buffered by step)
  bool use_tc = false;      // tcgen05 GEMM for LU trailing updates
  bool use_tc_qr = false;   // tcgen05 GEMMs for QR trailing updates
  float* Wbuf = nullptr;
  float* Gbuf = nullptr;
  float* Tfull[2] = {nullptr, nullptr};
  float* Vt[2] = {nullptr, nullptr};
  unsigned char* Apk[2] = {nullptr, nullptr};   // packed QR operands (V^T, V T^T, T^T) per tile
  unsigned char* Lpk[2] = {nullptr, nullptr};   // packed LU panel (rows below the diagonal)
  float* Linv[2] = {nullptr, nullptr};          // X = L^-1 P of an LU step (nb x nb)
  unsigned char* Xpk[2] = {nullptr, nullptr};   // X packed for the tensor-core Apply
  size_t pk_tile = 0;                           // bytes of one packed nb x nb operand
  // decision predictor and speculation (spec_stream factors predicted-QR panels on the
  // shadow copy while the criterion runs on the panel stream)
  int speculate = 0;
  const float* mlp = nullptr;
  float* feat = nullptr;        // n x 16 features (when logged)
  uint8_t* spec = nullptr;      // predicted decision per step
  uint8_t* qrfac = nullptr;     // QR chosen and not speculated: factor in place
  uint8_t* cmt = nullptr;       // QR chosen and speculated: commit the shadow copy
  uint8_t* lufac = nullptr;     // LU chosen and not speculated: TRSM in place
  uint8_t* lucmt = nullptr;     // LU chosen and speculated: commit the shadow TRSM
  void* shadow = nullptr;       // Npad x nb copy of the panel column (same leading dimension)
  cudaStream_t spec_stream = nullptr;
  cudaStream_t panel_stream = nullptr;   // high priority; the caller's stream waits on it
  cudaStream_t la_stream = nullptr;      // look-ahead column, one tree level behind the panel
  cudaStream_t extra_stream = nullptr;   // tensor-core operand preparation of QR steps
  std::vector<cudaEvent_t> ev_lvl;       // per tile list of the current step (reused)
  std::vector<cudaEvent_t> ev_splvl;     // the same for the speculative chain
  std::vector<cudaEvent_t> ev_dec;       // per step: decision and speculation gates written
  std::vector<cudaEvent_t> ev_extra, ev_la;
  std::vector<cudaEvent_t> ev_stats, ev_spec, ev_getrf, ev_luspec;
  cudaEvent_t ev_end = nullptr;
  // second pass / refinement scratch
  void* rhs_ws = nullptr;
  int rhs_cap = 0;
  double* ref = nullptr;    // x, r, scalars, partial sums
  int ref_chunks = 0;
  double* gm = nullptr;     // GMRES: basis (N x (restart+1)), work vector, dot buffers
  // single-vector second pass in one persistent launch: the task list (both branches of
  // every step, gated on the device decision), its device copy and counters
  std::vector<ReplayTask> rq_host;
  ReplayTask* rq = nullptr;
  int* rq_ctl = nullptr;        // [0] next task, [1] abort flag, [2 .. 2+n) per-row counts
  int rq_grid = 0;
  int rq_skip = -1;             // test hook: task whose completion is never signalled
  bool rq_by_dec = false;       // the list holds only the branches taken (decisions known)
  long long wait_cycles = 1000000000LL;   // budget of a bounded device wait (about 0.5 s)
  double acc[4] = {NAN, NAN, NAN, NAN};   // last refinement: ||A||, ||r||, ||x||, ||b|| (inf-norms)
  int gm_restart = 0;
  size_t elt = 8;
};

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? LUQR_OK : (e == cudaErrorMemoryAllocation ? LUQR_ERR_NOMEM : LUQR_ERR_CUDA); }

template <typename T>
T* wsT(luqr_handle* h) { return static_cast<T*>(h->W); }

size_t t_block_elems(const luqr_handle* h) { return (size_t)IB * h->nb; }
size_t t_step_elems(const luqr_handle* h) { return (size_t)h->n * 2 * t_block_elems(h); }

// ---------------------------------------------------------------- QR step
// Enqueues the QR step of panel k along the handle's tree.  factor = true factors the
// panel tiles in F and applies to columns [c0, c1) of C; factor = false only applies
// the stored transformations to C (second pass).
// Tensor-core (FP32) helpers of the QR step: per tile of a tile list, G = V^T V, the full
// compact-WY T (k_tfull) and Vt = V T^T at factor time; at apply time
//   single (UNMQR):  W = V^T C;            C -= Vt W
//   pair (TS/TT):    W = C1 + V2^T C2;     C1 -= T^T W;   C2 -= Vt W
void tc_factor_extra(luqr_handle* h, int k, TileList tl, int kind, int mask, cudaStream_t s) {
  const int nb = h->nb;
  const int64_t ld = h->Npad, nb2 = (int64_t)nb * nb;
  float* W = static_cast<float*>(h->W);
  const float* V0 = W + (int64_t)tl.i0 * nb + (int64_t)k * nb * ld;
  const int64_t slot0 = ((int64_t)tl.i0 * 2 + kind) * nb2, sslot = (int64_t)tl.istride * 2 * nb2;
  float* Tf = h->Tfull[k & 1];
  float* Vt = h->Vt[k & 1];
  TcArgs a{};
  a.wait_cycles = h->wait_cycles;
  a.dec = h->dec; a.k_step = k; a.want = DEC_QR; a.status = h->status;
  a.M = nb; a.N = nb; a.K = nb; a.epi = TC_EPI_OUT;
  // G = V^T V
  a.A = V0; a.lda = ld; a.sA = (int64_t)tl.istride * nb; a.a_trans = 1; a.a_mask = mask;
  a.B = V0; a.ldb = ld; a.sB = (int64_t)tl.istride * nb; a.b_trans = 0; a.b_mask = mask;
  a.C = h->Gbuf + slot0; a.ldc = nb; a.sC = sslot;
  launch_tc(a, tl.count, "k_tc_gram", s);
  const float* Tsl = static_cast<const float*>(h->Tbuf) + (size_t)k * t_step_elems(h) +
                     ((size_t)tl.i0 * 2 + kind) * t_block_elems(h);
  launch_tfull(h->Gbuf + slot0, sslot, Tsl, (int64_t)tl.istride * 2 * (int64_t)t_block_elems(h),
               Tf + slot0, sslot, nb, tl.count, h->dec, k, s);
  // Vt = V T^T
  a.A = V0; a.lda = ld; a.sA = (int64_t)tl.istride * nb; a.a_trans = 0; a.a_mask = mask;
  a.B = Tf + slot0; a.ldb = nb; a.sB = sslot; a.b_trans = 1; a.b_mask = TC_MASK_NONE;
  a.C = Vt + slot0; a.ldc = nb; a.sC = sslot;
  launch_tc(a, tl.count, "k_tc_vt", s);
  // pack the A operands of the apply phase: V^T (0), V T^T (1), T^T (2, pairs only)
  unsigned char* pk = h->Apk[k & 1] + (((size_t)tl.i0 * 2 + kind) * 3) * h->pk_tile;
  const int64_t spk = (int64_t)tl.istride * 2 * 3 * (int64_t)h->pk_tile;
  launch_tc_pack(V0, ld, (int64_t)tl.istride * nb, 1, mask, nb, nb, pk, spk, tl.count, h->dec, k,
                 DEC_QR, s);
  launch_tc_pack(Vt + slot0, nb, sslot, 0, TC_MASK_NONE, nb, nb, pk + h->pk_tile, spk, tl.count,
                 h->dec, k, DEC_QR, s);
  if (kind == 1)
    launch_tc_pack(Tf + slot0, nb, sslot, 1, TC_MASK_NONE, nb, nb, pk + 2 * h->pk_tile, spk,
                   tl.count, h->dec, k, DEC_QR, s);
}

void tc_apply_single(luqr_handle* h, int k, TileList tl, Mat<float> C, int64_t c0, int64_t c1,
                     cudaStream_t s) {
  const int nb = h->nb;
  const int64_t ld = h->Npad;
  const int64_t rstride = (int64_t)tl.istride * nb;
  const unsigned char* pk = h->Apk[k & 1] + (((size_t)tl.i0 * 2 + 0) * 3) * h->pk_tile;
  const int64_t spk = (int64_t)tl.istride * 2 * 3 * (int64_t)h->pk_tile;
  TcArgs a{};
  a.wait_cycles = h->wait_cycles;
  a.dec = h->dec; a.k_step = k; a.want = DEC_QR; a.status = h->status;
  a.M = nb; a.N = c1 - c0; a.K = nb; a.sApk = spk;
  // W = V^T C  (V unit lower triangular: V^T upper)
  a.Apk = pk; a.a_tri = 2;
  a.B = C.p + (int64_t)tl.i0 * nb + c0 * C.ld; a.ldb = C.ld; a.sB = rstride;
  a.C = h->Wbuf + (int64_t)tl.i0 * nb + c0 * ld; a.ldc = ld; a.sC = rstride; a.epi = TC_EPI_OUT;
  launch_tc2(a, tl.count, "k_tc_unmqr_w", s);
  // C -= (V T^T) W  (lower triangular times lower triangular)
  a.Apk = pk + h->pk_tile; a.a_tri = 1;
  a.B = h->Wbuf + (int64_t)tl.i0 * nb + c0 * ld; a.ldb = ld; a.sB = rstride;
  a.C = C.p + (int64_t)tl.i0 * nb + c0 * C.ld; a.ldc = C.ld; a.sC = rstride; a.epi = TC_EPI_SUB;
  launch_tc2(a, tl.count, "k_tc_unmqr_c", s);
}

void tc_apply_pair(luqr_handle* h, int k, TileList tl, bool tri, Mat<float> C, int64_t c0,
                   int64_t c1, cudaStream_t s) {
  const int nb = h->nb;
  const int64_t ld = h->Npad;
  const int64_t rstride = (int64_t)tl.istride * nb;
  const int64_t i0r = (int64_t)tl.i0 * nb, e0r = (int64_t)(tl.i0 - tl.eoff) * nb;
  float* Wp = h->Wbuf + i0r + c0 * ld;
  const unsigned char* pk = h->Apk[k & 1] + (((size_t)tl.i0 * 2 + 1) * 3) * h->pk_tile;
  const int64_t spk = (int64_t)tl.istride * 2 * 3 * (int64_t)h->pk_tile;
  TcArgs a{};
  a.wait_cycles = h->wait_cycles;
  a.dec = h->dec; a.k_step = k; a.want = DEC_QR; a.status = h->status;
  a.M = nb; a.N = c1 - c0; a.K = nb; a.sApk = spk;
  // W = C1 + V2^T C2  (TT: V2 upper triangular, V2^T lower)
  a.Apk = pk; a.a_tri = tri ? 1 : 0;
  a.B = C.p + i0r + c0 * C.ld; a.ldb = C.ld; a.sB = rstride;
  a.C1 = C.p + e0r + c0 * C.ld; a.ldc1 = C.ld; a.sC1 = rstride;
  a.C = Wp; a.ldc = ld; a.sC = rstride; a.epi = TC_EPI_ADD_OUT;
  launch_tc2(a, tl.count, tri ? "k_tc_ttmqr_w" : "k_tc_tsmqr_w", s);
  a.C1 = nullptr;
  // C1 -= T^T W  (T^T lower triangular)
  a.Apk = pk + 2 * h->pk_tile; a.a_tri = 1;
  a.B = Wp; a.ldb = ld; a.sB = rstride;
  a.C = C.p + e0r + c0 * C.ld; a.ldc = C.ld; a.sC = rstride; a.epi = TC_EPI_SUB;
  launch_tc2(a, tl.count, tri ? "k_tc_ttmqr_c1" : "k_tc_tsmqr_c1", s);
  // C2 -= (V2 T^T) W
  a.Apk = pk + h->pk_tile; a.a_tri = 0;
  a.C = C.p + i0r + c0 * C.ld;
  launch_tc2(a, tl.count, tri ? "k_tc_ttmqr_c2" : "k_tc_tsmqr_c2", s);
}

// Visits the tile lists of step k's elimination tree in execution order:
// single(tl) for the tiles factored by GEQRT, pair(tl, tri) for the TS / TT levels.
template <typename FS, typename FP>
void for_each_tile_list(const luqr_handle* h, int k, FS&& single, FP&& pair) {
  const int n = h->n, m = n - 1 - k;
  // per-step tree: steps with fewer than tree_switch sub-diagonal tiles use tree_small
  const int tree = (h->tree_switch > 0 && m < h->tree_switch) ? h->tree_small : h->tree;
  if (tree == LUQR_TREE_FLAT_TS) {
    single(TileList{k, 1, 1, 0});
    for (int i = k + 1; i < n; ++i) pair(TileList{i, 1, 1, i - k}, false);
  } else if (tree == LUQR_TREE_BINARY_TT) {
    single(TileList{k, 1, m + 1, 0});
    for (int step = 1; step <= m; step *= 2) {
      const int count = (m - step) / (2 * step) + 1;
      pair(TileList{k + step, 2 * step, count, step}, true);
    }
  } else {
    const int g = h->group;
    const int H = (m + 1 + g - 1) / g;
    single(TileList{k, g, H, 0});
    for (int r = 1; r < g; ++r) {
      if (m + 1 - r <= 0) break;
      const int count = (m + 1 - r + g - 1) / g;
      pair(TileList{k + r, g, count, r}, false);
    }
    for (int step = 1; step < H; step *= 2) {
      const int count = (H - 1 - step) / (2 * step) + 1;
      pair(TileList{k + step * g, 2 * step * g, count, step * g}, true);
    }
  }
}

// Task list of the single-vector second pass (k_replay.cu), in program order: per step k the
// injection scaling, the QR branch (tile lists of the tree, gated on dec[k] = QR) and the LU
// branch (A1: L^-1 P on row k, A2: the tile's Q^T; then x_i -= A_ik x_k; gated on LU), then
// the back substitution from the last tile row up.  Each task carries, per row it writes
// or reads, the number of earlier writes of that row.
// dec (HOST, nullable): the factorization's decisions; when given, only the branch taken
// at each step is listed (no gated no-op tasks, which would hold CTAs until their step's
// tree completes).
void rq_build(luqr_handle* h, const uint8_t* dec = nullptr) {
  const int n = h->n;
  std::vector<int> wc(n, 0);
  std::vector<ReplayTask>& out = h->rq_host;
  out.clear();
  auto push = [&](int type, int k, int i, int e, int r, int gate) {
    ReplayTask t{type, k, i, e, r, wc[i], e >= 0 ? wc[e] : 0, r >= 0 ? wc[r] : 0, gate};
    out.push_back(t);
    ++wc[i];
    if (e >= 0) ++wc[e];
  };
  for (int k = 0; k < n; ++k) {
    if (h->injected[k]) push(RT_SCALE, k, k, -1, -1, 0);
    const bool want_qr = dec == nullptr || dec[k] == DEC_QR;
    const bool want_lu = dec == nullptr || dec[k] == DEC_LU;
    const int gq = dec ? 0 : 1, gl = dec ? 0 : 2;
    if (want_qr)
    for_each_tile_list(
        h, k,
        [&](TileList tl) {
          for (int t = 0; t < tl.count; ++t) push(RT_SINGLE, k, tl.i0 + t * tl.istride, -1, -1, gq);
        },
        [&](TileList tl, bool tri) {
          for (int t = 0; t < tl.count; ++t) {
            const int i = tl.i0 + t * tl.istride;
            push(tri ? RT_PAIR_TT : RT_PAIR_TS, k, i, i - tl.eoff, -1, gq);
          }
        });
    if (want_lu) {
      push(h->lu_variant == 1 ? RT_SINGLE : RT_LUAPPLY, k, k, -1, -1, gl);
      for (int i = k + 1; i < n; ++i) push(RT_GEMV, k, i, -1, k, gl);
    }
  }
  // back substitution: row k's solve takes the update from x_{k+1} with it; the other
  // updates from x_k are tasks of their own (row k-1's is the next fused solve)
  for (int k = n - 1; k >= 0; --k) {
    if (k == n - 1) push(RT_TRSV, k, k, -1, -1, 0);
    else push(RT_GEMV_TRSV, k + 1, k, -1, k + 1, 0);
    for (int i = k - 2; i >= 0; --i) push(RT_GEMV, k, i, -1, k, 0);
  }
  // Claim order: by depth in the dependency graph (1 + the deepest earlier writer of any row
  // the task touches), stable.  A task's dependencies are shallower, so the order stays a
  // topological one (per row, writes keep their program order and the counts stay valid),
  // and CTAs take tasks roughly when they become ready instead of holding a CTA on a task
  // whose step's tree has barely started.
  std::vector<int> depth(out.size()), lastw(n, 0);
  for (size_t t = 0; t < out.size(); ++t) {
    const ReplayTask& q = out[t];
    int d = lastw[q.i];
    if (q.e >= 0) d = std::max(d, lastw[q.e]);
    if (q.r >= 0) d = std::max(d, lastw[q.r]);
    depth[t] = d + 1;
    lastw[q.i] = depth[t];
    if (q.e >= 0) lastw[q.e] = depth[t];
  }
  std::vector<int> order(out.size());
  for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return depth[x] < depth[y]; });
  std::vector<ReplayTask> sorted(out.size());
  for (size_t t = 0; t < order.size(); ++t) sorted[t] = out[order[t]];
  out.swap(sorted);
}

// Enqueues the QR step of panel k along the handle's tree.  do_factor factors the panel
// tiles, do_apply applies the step's transformations to columns [c0, c1) of C.
// The factorization works on column k of fbase (default: the workspace; the shadow copy
// is passed with its base shifted by k*nb columns) and runs when fdec[k] == QR (default:
// the decision).  extras = false leaves the tensor-core operand preparation to
// enqueue_qr_extras.
// rec / wait (optional, one event per tile list in tree order): record after each tile
// list's factorization, or wait before each tile list's application.  vbase / adec
// (optional): where the application reads V (the shadow copy of a speculated panel, base
// shifted like fbase) and the gate it runs under.
template <typename T>
void enqueue_qr(luqr_handle* h, int k, Mat<T> C, int64_t c0, int64_t c1, bool do_factor,
                bool do_apply, cudaStream_t s, bool tc = false, T* fbase = nullptr,
                const uint8_t* fdec = nullptr, bool extras = true,
                const cudaEvent_t* rec = nullptr, const cudaEvent_t* wait = nullptr,
                const T* vbase = nullptr, const uint8_t* adec = nullptr) {
  const int n = h->n, nb = h->nb;
  Mat<T> F{fbase ? fbase : wsT<T>(h), h->Npad};
  // the application reads V from vbase (default: the workspace) and runs when adec[k] = QR
  Mat<const T> Fc{vbase ? vbase : wsT<T>(h), h->Npad};
  T* Tk = static_cast<T*>(h->Tbuf) + (size_t)k * t_step_elems(h);
  const uint8_t* dec = adec ? adec : h->dec;
  const uint8_t* fd = fdec ? fdec : h->dec;
  constexpr bool is_f32 = std::is_same<T, float>::value;
  tc = tc && is_f32 && h->use_tc_qr;
  int lvl = 0;
  auto single = [&](TileList tl) {
    if (wait) cudaStreamWaitEvent(s, wait[lvl], 0);
    if (do_factor) {
      launch_geqrt<T>(F, k, nb, tl, Tk, n, fd, s);
      if (tc && extras) tc_factor_extra(h, k, tl, 0, TC_MASK_UNIT_LOWER, s);
    }
    if (rec) cudaEventRecord(rec[lvl], s);
    ++lvl;
    if (do_apply) {
      if constexpr (is_f32) {
        if (tc) { tc_apply_single(h, k, tl, C, c0, c1, s); return; }
      }
      launch_unmqr<T>(Fc, k, nb, tl, Tk, n, C, c0, c1, dec, s);
    }
  };
  auto pair = [&](TileList tl, bool tri) {
    if (wait) cudaStreamWaitEvent(s, wait[lvl], 0);
    if (do_factor) {
      launch_pair_qrt<T>(F, k, nb, tl, tri, Tk, n, fd, s);
      if (tc && extras) tc_factor_extra(h, k, tl, 1, tri ? TC_MASK_UPPER : TC_MASK_NONE, s);
    }
    if (rec) cudaEventRecord(rec[lvl], s);
    ++lvl;
    if (do_apply) {
      if constexpr (is_f32) {
        if (tc) { tc_apply_pair(h, k, tl, tri, C, c0, c1, s); return; }
      }
      launch_pair_apply<T>(Fc, k, nb, tl, tri, Tk, n, C, c0, c1, dec, s);
    }
  };
  for_each_tile_list(h, k, single, pair);
}

// Tensor-core operand preparation of QR step k (Gram, full T, V T^T, packed operands) for
// a panel already factored in the workspace.  Every reflector block V stays untouched by
// the later levels of the tree (they only update R parts), so it can run after the chain.
void enqueue_qr_extras(luqr_handle* h, int k, cudaStream_t s) {
  if (!h->use_tc_qr) return;
  for_each_tile_list(
      h, k, [&](TileList tl) { tc_factor_extra(h, k, tl, 0, TC_MASK_UNIT_LOWER, s); },
      [&](TileList tl, bool tri) {
        tc_factor_extra(h, k, tl, 1, tri ? TC_MASK_UPPER : TC_MASK_NONE, s);
      });
}

// ---------------------------------------------------------------- LU step on a target
// tc_apply: the Apply (L^-1 P on tile row k) as an in-place tensor-core product with the
// step's packed X (prepared on the extra stream; only the bulk update uses it).  In place
// is safe because one CTA tile spans all nb rows (nb <= 256): its B columns are read in
// full before its epilogue writes them.
template <typename T>
void enqueue_lu_apply(luqr_handle* h, int k, Mat<T> C, int64_t c0, int64_t c1, cudaStream_t s,
                      bool tc = false, bool tc_apply = false) {
  const int nb = h->nb;
  const int64_t r0 = (int64_t)k * nb, r1 = r0 + nb, ld = h->Npad;
  T* W = wsT<T>(h);
  Mat<const T> LU{W + r0 + r0 * ld, ld};
  bool applied = false;
  if constexpr (std::is_same<T, float>::value) {
    if (tc_apply && h->Xpk[k & 1] != nullptr && c1 - c0 >= 64) {
      TcArgs a{};
      a.wait_cycles = h->wait_cycles;
      a.dec = h->dec; a.k_step = k; a.want = DEC_LU; a.status = h->status;
      a.M = nb; a.N = c1 - c0; a.K = nb;
      a.Apk = h->Xpk[k & 1];
      a.B = C.p + r0 + c0 * C.ld; a.ldb = C.ld;
      a.C = C.p + r0 + c0 * C.ld; a.ldc = C.ld; a.epi = TC_EPI_OUT;
      launch_tc2(a, 1, "k_tc_lu_apply", s);
      applied = true;
    }
  }
  if (!applied) {
    if (h->lu_variant == 1) {   // A2: Q^T of the tile's GEQRT (V below the diagonal, T slot)
      const T* Tk = static_cast<const T*>(h->Tbuf) + (size_t)k * t_step_elems(h);
      launch_unmqr<T>(Mat<const T>{W, ld}, k, nb, TileList{k, 1, 1, 0}, Tk, h->n, C, c0, c1,
                      h->a2gate, s);
    } else {
      launch_swptrsm<T>(LU, nb, h->piv_all + (size_t)k * nb, C, r0, c0, c1, h->dec, k, s);
    }
  }
  Mat<const T> Ablk{W + r1 + r0 * ld, ld};
  Mat<const T> Brow{C.p + r0 + c0 * C.ld, C.ld};
  Mat<T> Cblk{C.p + r1 + c0 * C.ld, C.ld};
  if constexpr (std::is_same<T, float>::value) {
    if (tc && h->use_tc) {
      TcArgs a{};
      a.wait_cycles = h->wait_cycles;
      a.dec = h->dec; a.k_step = k; a.want = DEC_LU; a.status = h->status;
      a.M = h->Npad - r1; a.N = c1 - c0; a.K = nb;
      a.Apk = h->Lpk[k & 1];   // packed by the factor phase (pack_lu_panel)
      a.B = Brow.p; a.ldb = C.ld;
      a.C = Cblk.p; a.ldc = C.ld; a.epi = TC_EPI_SUB;
      launch_tc2(a, 1, "k_tc_lu_gemm", s);
      return;
    }
  }
  launch_gemm_update<T>(Ablk, Brow, Cblk, h->Npad - r1, c1 - c0, nb, h->dec, k, DEC_LU, s);
}

template <typename T>
void enqueue_factor(luqr_handle* h) {
  // The panel chain runs on a high-priority internal stream so that its small kernels are
  // scheduled ahead of the bulk update's blocks; the caller's stream waits for both.
  cudaStream_t s = h->panel_stream, su = h->upd_stream, sp = h->spec_stream;
  cudaStream_t sl = h->la_stream, sx = h->extra_stream;
  const bool tcqr = std::is_same<T, float>::value && h->use_tc_qr;
  const int n = h->n, nb = h->nb;
  const int64_t ld = h->Npad;
  T* W = wsT<T>(h);
  T* S = static_cast<T*>(h->S);
  T* shadow = static_cast<T*>(h->shadow);
  Mat<T> F{W, ld};
  const bool need_inv = (h->forced == nullptr) &&
                        (h->criterion == LUQR_MAX || h->criterion == LUQR_SUM) && h->alpha != 0.0;
  const bool spec = h->speculate != 0;
  cudaEventRecord(h->ev_start, h->stream);
  cudaStreamWaitEvent(s, h->ev_start, 0);
  cudaStreamWaitEvent(su, h->ev_start, 0);
  cudaStreamWaitEvent(sl, h->ev_start, 0);
  cudaStreamWaitEvent(sx, h->ev_start, 0);
  if (spec) cudaStreamWaitEvent(sp, h->ev_start, 0);
  for (int k = 0; k < n; ++k) {
    const int64_t r0 = (int64_t)k * nb, r1 = r0 + nb;
    const int64_t la_end = std::min<int64_t>(r1 + nb, h->Npad);   // look-ahead column k+1
    // ---- panel k on the panel stream (column k is complete: see the waits below)
    if (h->injected[k]) {
      // the injected row spans every column >= k: wait for the previous bulk update
      if (k > 0) cudaStreamWaitEvent(s, h->ev_rest[k - 1], 0);
      launch_scale_rows<T>(W, ld, r0, nb, r0, h->Wc, std::ldexp(1.0, -27), s);
    }
    const int dd = std::min(h->domain, n - k);   // tiles of this step's pivot domain
    const bool lu_spec = spec && h->lu_variant == 0 && dd <= 1;
    int* dpiv_k = h->dpiv_all ? h->dpiv_all + (size_t)k * nb : nullptr;
    if (dd > 1) {
      // Factor over the diagonal domain: the exchanges reach every column >= k, so the
      // previous bulk update must be complete; the criterion reads the pivoted panel copy
      if (k > 0) cudaStreamWaitEvent(s, h->ev_rest[k - 1], 0);
      launch_getrf_tall<T>(W, ld, k, nb, dd * nb, static_cast<T*>(h->St), dpiv_k, h->piv_s,
                           h->status, s);
      launch_domain_panel<T>(W, ld, k, nb, dd * nb, h->Npad, dpiv_k, shadow, ld, s);
      launch_panel_stats<T>(shadow - (int64_t)k * nb * ld, ld, k, n, nb, h->norms + (size_t)k * n,
                            h->local, h->away, h->status, s);
      launch_gated_copy<T>(static_cast<T*>(h->St), dd * nb, S, nb, nb, nb, h->gate_all, k, DEC_QR,
                           "k_domain_top", s);
    } else {
      launch_panel_stats<T>(W, ld, k, n, nb, h->norms + (size_t)k * n, h->local, h->away,
                            h->status, s);
    }
    if (h->feat || spec)
      launch_features_spec<T>(W, ld, k, n, nb, h->alpha, h->criterion, h->norms + (size_t)k * n,
                              h->local, h->away, h->dec, h->margin, h->feat, h->speculate, h->mlp,
                              h->spec, s);
    if (spec) {
      // predicted QR: factor a copy of column k while GETRF and the criterion run
      cudaEventRecord(h->ev_stats[k], s);
      cudaStreamWaitEvent(sp, h->ev_stats[k], 0);
      launch_gated_copy<T>(W + r0 + r0 * ld, ld, shadow + r0, ld, h->Npad - r0, nb, h->spec, k,
                           DEC_QR, "k_spec_copy", sp);
      enqueue_qr<T>(h, k, F, 0, 0, true, false, sp, true, shadow - r0 * ld, h->spec, false,
                    r1 < la_end ? h->ev_splvl.data() : nullptr);
      cudaEventRecord(h->ev_spec[k], sp);
    }
    T* Tkk = static_cast<T*>(h->Tbuf) + (size_t)k * t_step_elems(h) +
             (size_t)k * 2 * t_block_elems(h);   // T slot of tile (k, k), GEQRT kind
    if (h->lu_variant == 1) {
      // Factor (variant A2): GEQRT of a scratch copy of A_kk; its T goes to the tile's slot
      launch_gated_copy<T>(W + r0 + r0 * ld, ld, S, nb, nb, nb, h->gate_all, k, DEC_QR,
                           "k_a2_copy", s);
      launch_geqrt<T>(Mat<T>{S, nb}, 0, nb, TileList{0, 1, 1, 0}, Tkk, n, h->gate_all, s);
      launch_a2_prep<T>(S, nb, h->piv_s, h->status, s);
      if (need_inv)
        launch_qt_cols<T>(S, nb, nb, Tkk, 0, h->colsum, nullptr, h->status, h->gate_all, k, s);
    } else {
      if (dd <= 1) launch_getrf<T>(W, ld, k, nb, S, h->piv_s, h->status, s);
      if (lu_spec) {
        // predicted LU: the panel's TRSM (A_ik U^-1, i > k) with the scratch LU on a copy of
        // the sub-diagonal tiles, while the inverse norm and the decision run
        cudaEventRecord(h->ev_getrf[k], s);
        cudaStreamWaitEvent(sp, h->ev_getrf[k], 0);
        if (r1 < h->Npad) {
          launch_gated_copy<T>(W + r1 + r0 * ld, ld, shadow + r1, ld, h->Npad - r1, nb, h->spec,
                               k, DEC_LU, "k_spec_copy_lu", sp);
          launch_trsm<T>(Mat<const T>{S, nb}, nb, Mat<T>{shadow, ld}, r1, h->Npad, 0, h->spec,
                         k, sp);
        }
        cudaEventRecord(h->ev_luspec[k], sp);
      }
      if (need_inv) {
        if (h->norm_mode == 1) launch_invnorm_est<T>(S, nb, h->piv_s, h->colsum, h->status, s);
        else launch_invnorm<T>(S, nb, h->piv_s, h->colsum, h->status, s);
      }
    }
    DecideArgs da{k,        n,         nb,       h->criterion, h->mumps_mode, h->alpha,
                  h->norms + (size_t)k * n, h->colsum, h->local, h->away,     h->forced,
                  h->dec,   h->margin, h->lhs,   h->rhs,       h->status};
    da.seed = h->seed;
    launch_decide<T>(da, S, s);
    if (spec) {
      launch_spec_resolve(k, h->dec, h->spec, h->qrfac, h->cmt, h->lufac, h->lucmt, lu_spec, s);
      cudaEventRecord(h->ev_dec[k], s);
    }
    if (h->lu_variant == 1) launch_a2_gate(h->dec, h->a2gate, k, s);
    if (dd > 1)   // an LU step applies the domain's exchanges to columns k.. and b first
      launch_domain_swap<T>(W, ld, k, nb, dd * nb, r0, h->Wc, dpiv_k, h->dec, s);
    // ---- factor the panel: LU (Alg. 2: commit + TRSM) or QR (GEQRT + TS/TT chain)
    launch_lu_commit<T>(W, ld, k, nb, S, h->piv_s, h->piv_all + (size_t)k * nb, h->dec, s);
    if (lu_spec) {   // the speculative TRSM is done (and S is free for the next step)
      cudaStreamWaitEvent(s, h->ev_luspec[k], 0);
      if (r1 < h->Npad)
        launch_gated_copy<T>(shadow + r1, ld, W + r1 + r0 * ld, ld, h->Npad - r1, nb, h->lucmt,
                             k, DEC_LU, "k_spec_commit_lu", s);
    }
    Mat<const T> LU{W + r0 + r0 * ld, ld};
    launch_trsm<T>(LU, nb, F, r1, h->Npad, r0, spec ? h->lufac : h->dec, k, s);
    if constexpr (std::is_same<T, float>::value) {
      if (h->use_tc && r1 < h->Npad)   // pack A_ik U^-1 for the tensor-core trailing GEMM
        launch_tc_pack(reinterpret_cast<float*>(W) + r1 + r0 * ld, ld, 0, 0, TC_MASK_NONE,
                       h->Npad - r1, nb, h->Lpk[k & 1], 0, 1, h->dec, k, DEC_LU, s);
    }
    // The QR chain of column k records one event per tree level (non-speculative runs), so
    // that the look-ahead stream applies level l to column k+1 while level l+1 factors.
    const bool piped = !spec && r1 < la_end;
    if (spec) {
      enqueue_qr<T>(h, k, F, 0, 0, true, false, s, true, nullptr, h->qrfac, false,
                    r1 < la_end ? h->ev_lvl.data() : nullptr);
      cudaStreamWaitEvent(s, h->ev_spec[k], 0);
      launch_gated_copy<T>(shadow + r0, ld, W + r0 + r0 * ld, ld, h->Npad - r0, nb, h->cmt, k,
                           DEC_QR, "k_spec_commit", s);
    } else {
      enqueue_qr<T>(h, k, F, 0, 0, true, false, s, true, nullptr, nullptr, !tcqr,
                    piped ? h->ev_lvl.data() : nullptr);
    }
    cudaEventRecord(h->ev_fact[k], s);
    // ---- tensor-core operands of the QR step (Gram, full T, V T^T, packing) off the
    //      panel's critical path; only the bulk update consumes them
    const bool lu_x = std::is_same<T, float>::value && h->Xpk[k & 1] != nullptr;
    if (tcqr || lu_x) {
      cudaStreamWaitEvent(sx, h->ev_fact[k], 0);
      if constexpr (std::is_same<T, float>::value) {
        if (tcqr) enqueue_qr_extras(h, k, sx);
        if (lu_x) {
          if (h->lu_variant == 1)   // A2: X = Q^T of the committed tile's GEQRT
            launch_qt_cols<float>(reinterpret_cast<const float*>(W) + r0 + r0 * ld, ld, nb,
                                  reinterpret_cast<const float*>(Tkk), 1, nullptr, h->Linv[k & 1],
                                  h->status, h->a2gate, k, sx);
          else
            launch_lu_inverse(reinterpret_cast<const float*>(W), ld, k, nb,
                              h->piv_all + (size_t)k * nb, h->Linv[k & 1], h->dec, sx);
          launch_tc_pack(h->Linv[k & 1], nb, 0, 0, TC_MASK_NONE, nb, nb, h->Xpk[k & 1], 0, 1,
                         h->dec, k, DEC_LU, sx);
        }
      }
      cudaEventRecord(h->ev_extra[k], sx);
    }
    // ---- bulk update of columns >= k+2 (and b) on the update stream
    if (la_end < h->Wc) {
      cudaStreamWaitEvent(su, h->ev_fact[k], 0);
      if (tcqr || lu_x) cudaStreamWaitEvent(su, h->ev_extra[k], 0);
      enqueue_lu_apply<T>(h, k, F, la_end, h->Wc, su, true, true);
      enqueue_qr<T>(h, k, F, la_end, h->Wc, false, true, su, true);
    }
    cudaEventRecord(h->ev_rest[k], su);
    // ---- look-ahead: column k+1 needs step k-1's bulk update, then step k's transform
    //      (CUDA-core QR kernels: they need only the stored V and the IB x IB T blocks)
    if (r1 < la_end && spec) {
      // speculation: once the decision is known, a QR step's transformations reach column
      // k+1 level by level behind whichever chain factors the panel (the speculative one,
      // V still in the shadow, or the in-place one); an LU step's after its TRSM
      cudaStreamWaitEvent(sl, h->ev_dec[k], 0);
      if (k > 0) cudaStreamWaitEvent(sl, h->ev_rest[k - 1], 0);
      enqueue_qr<T>(h, k, F, r1, la_end, false, true, sl, false, nullptr, nullptr, true, nullptr,
                    h->ev_splvl.data(), shadow - r0 * ld, h->cmt);
      enqueue_qr<T>(h, k, F, r1, la_end, false, true, sl, false, nullptr, nullptr, true, nullptr,
                    h->ev_lvl.data(), nullptr, h->qrfac);
      cudaStreamWaitEvent(sl, h->ev_fact[k], 0);
      enqueue_lu_apply<T>(h, k, F, r1, la_end, sl, true);
      cudaEventRecord(h->ev_la[k], sl);
      cudaStreamWaitEvent(s, h->ev_la[k], 0);
    } else if (r1 < la_end) {
      cudaStreamWaitEvent(sl, h->ev_lvl[0], 0);
      if (k > 0) cudaStreamWaitEvent(sl, h->ev_rest[k - 1], 0);
      enqueue_lu_apply<T>(h, k, F, r1, la_end, sl, true);
      enqueue_qr<T>(h, k, F, r1, la_end, false, true, sl, false, nullptr, nullptr, true, nullptr,
                    piped ? h->ev_lvl.data() : nullptr);
      cudaEventRecord(h->ev_la[k], sl);
      cudaStreamWaitEvent(s, h->ev_la[k], 0);
    }
  }
  cudaStreamWaitEvent(s, h->ev_rest[n - 1], 0);
  cudaEventRecord(h->ev_end, sx);
  cudaStreamWaitEvent(s, h->ev_end, 0);
  cudaEventRecord(h->ev_end, sl);
  cudaStreamWaitEvent(s, h->ev_end, 0);
  cudaEventRecord(h->ev_end, s);
  cudaStreamWaitEvent(h->stream, h->ev_end, 0);
}

template <typename T>
void enqueue_backsolve(luqr_handle* h, Mat<T> X, int nrhs) {
  Mat<const T> U{wsT<T>(h), h->Npad};
  for (int k = h->n - 1; k >= 0; --k) {
    launch_trsv_diag<T>(U, k, h->nb, X, nrhs, h->status, h->stream);
    launch_trsv_update<T>(U, k, h->nb, X, nrhs, h->stream);
  }
}

// Second pass: replay every step on X (Npad x nrhs, precision T), then back-substitute.
template <typename T>
void enqueue_replay(luqr_handle* h, Mat<T> X, int nrhs) {
  if (nrhs == 1 && h->rq != nullptr && h->elt == sizeof(T)) {
    cudaMemsetAsync(h->rq_ctl, 0, sizeof(int) * (2 + (size_t)h->n), h->stream);
    ReplayArgs<T> a{};
    a.W = wsT<T>(h); a.ld = h->Npad;
    a.Tbuf = static_cast<const T*>(h->Tbuf); a.t_step = t_step_elems(h);
    a.piv_all = h->piv_all; a.dec = h->dec; a.x = X.p;
    a.tasks = h->rq; a.ntasks = (int)h->rq_host.size(); a.nb = h->nb;
    a.ctl = h->rq_ctl; a.done = h->rq_ctl + 2; a.status = h->status;
    a.budget = h->wait_cycles; a.skip_signal = h->rq_skip;
    launch_replay<T>(a, h->rq_grid, h->stream);
    return;
  }
  for (int k = 0; k < h->n; ++k) {
    const int64_t r0 = (int64_t)k * h->nb;
    if (h->injected[k]) launch_scale_rows<T>(X.p, X.ld, r0, h->nb, 0, nrhs, std::ldexp(1.0, -27), h->stream);
    const int dd = std::min(h->domain, h->n - k);
    if (dd > 1)
      launch_domain_swap<T>(X.p, X.ld, k, h->nb, dd * h->nb, 0, nrhs,
                            h->dpiv_all + (size_t)k * h->nb, h->dec, h->stream);
    enqueue_lu_apply<T>(h, k, X, 0, nrhs, h->stream);
    enqueue_qr<T>(h, k, X, 0, nrhs, false, true, h->stream);
  }
  enqueue_backsolve<T>(h, X, nrhs);
}

// Rebuilds the second-pass task list from the decisions once they are known on the host
// (synchronises the handle's stream; called by the refinement drivers, which synchronise
// anyway).  The list only shrinks, so the device allocation is reused.
int rq_specialise(luqr_handle* h) {
  if (h->rq == nullptr || h->rq_by_dec) return LUQR_OK;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LUQR_ERR_CUDA;
  std::vector<uint8_t> dec(h->n);
  if (cudaMemcpy(dec.data(), h->dec, (size_t)h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  for (int k = 0; k < h->n; ++k)
    if (dec[k] != DEC_QR && dec[k] != DEC_LU) return LUQR_OK;   // aborted run: keep the gates
  rq_build(h, dec.data());
  if (cudaMemcpy(h->rq, h->rq_host.data(), sizeof(ReplayTask) * h->rq_host.size(),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return LUQR_ERR_CUDA;
  h->rq_by_dec = true;
  if (h->rq_skip >= (int)h->rq_host.size()) h->rq_skip = -1;
  return LUQR_OK;
}

int ensure_rhs(luqr_handle* h, int nrhs) {
  if (h->rhs_cap >= nrhs) return LUQR_OK;
  if (h->rhs_ws) cudaFree(h->rhs_ws);
  h->rhs_ws = nullptr;
  h->rhs_cap = 0;
  cudaError_t e = cudaMalloc(&h->rhs_ws, (size_t)h->Npad * nrhs * h->elt);
  if (e != cudaSuccess) return cuda_err(e);
  h->rhs_cap = nrhs;
  return LUQR_OK;
}

template <typename T>
int solve_impl(luqr_handle* h, double* db, int nrhs, int64_t ldb, const double* scale) {
  int st = ensure_rhs(h, nrhs);
  if (st) return st;
  T* X = static_cast<T*>(h->rhs_ws);
  launch_convert_in<T>(db, ldb, h->N, h->Npad, nrhs, scale, X, h->Npad, h->stream);
  enqueue_replay<T>(h, Mat<T>{X, h->Npad}, nrhs);
  return LUQR_OK;
}

void free_handle(luqr_handle* h) {
  if (!h) return;
  for (cudaEvent_t e : h->ev_fact) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_rest) if (e) cudaEventDestroy(e);
  if (h->ev_start) cudaEventDestroy(h->ev_start);
  for (cudaEvent_t e : h->ev_stats) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_spec) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_getrf) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_luspec) if (e) cudaEventDestroy(e);
  if (h->ev_end) cudaEventDestroy(h->ev_end);
  if (h->upd_stream) cudaStreamDestroy(h->upd_stream);
  if (h->spec_stream) cudaStreamDestroy(h->spec_stream);
  if (h->panel_stream) cudaStreamDestroy(h->panel_stream);
  if (h->la_stream) cudaStreamDestroy(h->la_stream);
  if (h->extra_stream) cudaStreamDestroy(h->extra_stream);
  for (cudaEvent_t e : h->ev_lvl) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_splvl) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_dec) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_extra) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : h->ev_la) if (e) cudaEventDestroy(e);
  void* ptrs[] = {h->W,      h->Tbuf,     h->S,        h->piv_s, h->piv_all, h->norms,
                  h->local,  h->away,     h->colsum,   h->dec,   h->margin,  h->lhs,
                  h->rhs,    h->status,   h->forced,   h->rhs_ws, h->ref,    h->Wbuf,
                  h->Gbuf,   h->Tfull[0], h->Tfull[1], h->Vt[0], h->Vt[1], h->gm,
                  h->Apk[0], h->Apk[1],   h->Lpk[0],   h->Lpk[1], h->feat, h->spec,
                  h->Linv[0], h->Linv[1], h->Xpk[0],   h->Xpk[1],
                  h->qrfac,  h->cmt,      h->lufac,    h->lucmt, h->shadow, h->gate_all,
                  h->a2gate, h->rq,
                  h->rq_ctl, h->St, h->dpiv_all};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete h;
}

int read_status(luqr_handle* h, int* st3) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return LUQR_ERR_CUDA;
  int buf[ST_WORDS];
  e = cudaMemcpy(buf, h->status, sizeof(buf), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return LUQR_ERR_CUDA;
  if (st3) { st3[0] = buf[ST_CODE]; st3[1] = buf[ST_STEP]; st3[2] = buf[ST_ROW]; }
  return buf[ST_CODE];
}

}  // namespace

// Preconditioner of GMRES-IR: out = M^-1 in with M the handle's factorization (second
// pass in the factorization's precision, input scaled by ||in||_inf on the device).
template <typename T>
void precond(luqr_handle* h, const double* in, double* out, double* scal) {
  launch_vec_absmax(in, h->N, scal, h->stream);
  solve_impl<T>(h, const_cast<double*>(in), 1, h->N, scal);
  cudaMemsetAsync(out, 0, sizeof(double) * h->N, h->stream);
  launch_axpy_update<T>(out, static_cast<T*>(h->rhs_ws), h->N, scal, h->stream);
}

template <typename T>
int refine_gmres_impl(luqr_handle* h, const double* dA, int64_t lda, const double* db, double* dx,
                      double tol, int max_iter, int restart, int* iters, double* eta) {
  cudaStream_t s = h->stream;
  const int64_t N = h->N;
  const int nchunk = (int)((N + 511) / 512);
  if (!h->ref || h->ref_chunks < nchunk) {
    if (h->ref) cudaFree(h->ref);
    h->ref = nullptr;
    cudaError_t e = cudaMalloc(&h->ref, sizeof(double) * ((size_t)N * (nchunk + 2) + 8));
    if (e != cudaSuccess) return cuda_err(e);
    h->ref_chunks = nchunk;
  }
  if (!h->gm || h->gm_restart < restart) {
    if (h->gm) cudaFree(h->gm);
    h->gm = nullptr;
    cudaError_t e = cudaMalloc(&h->gm, sizeof(double) * ((size_t)N * (restart + 2) + 4 * (restart + 2) + 16));
    if (e != cudaSuccess) return cuda_err(e);
    h->gm_restart = restart;
  }
  int st = ensure_rhs(h, 1);
  if (st) return st;
  double* r = h->ref;
  double* partial = r + N;
  double* scal = partial + (size_t)N * nchunk;   // [0] ||A|| [1] ||r|| [2] ||x|| [3] ||b|| [4] pc
  double* V = h->gm;                             // N x (restart + 1)
  double* tmp = V + (size_t)N * (restart + 1);   // N
  double* dots = tmp + N;                        // 2 x (restart + 2)
  double* dots2 = dots + (restart + 2);
  double* coef = dots2 + (restart + 2);
  launch_row_abs_sum_max(dA, lda, N, partial, nchunk, scal + 0, s);
  launch_vec_absmax(db, N, scal + 3, s);
  cudaMemsetAsync(dx, 0, sizeof(double) * N, s);
  cudaMemcpyAsync(r, db, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  std::vector<double> H((size_t)(restart + 1) * restart), g(restart + 1), cs(restart), sn(restart),
      hv(restart + 2), hv2(restart + 2), y(restart);
  int total = 0;
  double e_it = INFINITY, best = INFINITY;
  for (int outer = 0; outer <= max_iter; ++outer) {
    // z0 = M^-1 r, v0 = z0 / beta
    precond<T>(h, r, V, scal + 4);
    launch_multidot(V, N, N, 1, V, dots, s);
    double nrm2;
    cudaMemcpyAsync(&nrm2, dots, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return LUQR_ERR_CUDA;
    const double beta = std::sqrt(nrm2);
    int jend = 0;
    if (beta > 0.0 && std::isfinite(beta)) {
      launch_multiaxpy(V, N, N, 0, dots, V, 1.0 / beta, s);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      for (int j = 0; j < restart; ++j) {
        double* vj = V + (size_t)N * j;
        double* w = V + (size_t)N * (j + 1);
        launch_matvec(dA, lda, N, vj, tmp, partial, nchunk, s);
        precond<T>(h, tmp, w, scal + 4);
        // classical Gram-Schmidt, twice
        launch_multidot(V, N, N, j + 1, w, dots, s);
        launch_multiaxpy(V, N, N, j + 1, dots, w, 1.0, s);
        launch_multidot(V, N, N, j + 1, w, dots2, s);
        launch_multiaxpy(V, N, N, j + 1, dots2, w, 1.0, s);
        launch_multidot(w, N, N, 1, w, dots2 + j + 1, s);
        cudaMemcpyAsync(hv.data(), dots, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hv2.data(), dots2, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return LUQR_ERR_CUDA;
        ++total;
        double* Hj = H.data() + (size_t)j * (restart + 1);
        for (int i = 0; i <= j; ++i) Hj[i] = hv[i] + hv2[i];
        const double hn = std::sqrt(std::max(hv2[j + 1], 0.0));
        Hj[j + 1] = hn;
        if (hn > 0.0) launch_multiaxpy(V, N, N, 0, dots, w, 1.0 / hn, s);
        for (int i = 0; i < j; ++i) {   // previous rotations
          const double a = Hj[i], b = Hj[i + 1];
          Hj[i] = cs[i] * a + sn[i] * b;
          Hj[i + 1] = -sn[i] * a + cs[i] * b;
        }
        const double a = Hj[j], b = Hj[j + 1];
        const double rr = std::hypot(a, b);
        cs[j] = rr > 0.0 ? a / rr : 1.0;
        sn[j] = rr > 0.0 ? b / rr : 0.0;
        Hj[j] = rr;
        Hj[j + 1] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = cs[j] * g[j];
        jend = j + 1;
        if (std::fabs(g[j + 1]) <= 1e-10 * beta || hn == 0.0) break;
      }
      for (int i = jend - 1; i >= 0; --i) {   // back substitution on the rotated H
        double acc = g[i];
        for (int q = i + 1; q < jend; ++q) acc -= H[(size_t)q * (restart + 1) + i] * y[q];
        const double d = H[(size_t)i * (restart + 1) + i];
        y[i] = d != 0.0 ? acc / d : 0.0;
      }
      for (int i = 0; i < jend; ++i) y[i] = -y[i];
      cudaMemcpyAsync(coef, y.data(), sizeof(double) * jend, cudaMemcpyHostToDevice, s);
      launch_multiaxpy(V, N, N, jend, coef, dx, 1.0, s);   // x <- x + V y
    }
    launch_residual(dA, lda, N, dx, db, r, partial, nchunk, s);
    launch_vec_absmax(r, N, scal + 1, s);
    launch_vec_absmax(dx, N, scal + 2, s);
    double host[4];
    cudaMemcpyAsync(host, scal, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return LUQR_ERR_CUDA;
    e_it = host[1] / (host[0] * host[2] + host[3]);
    best = std::min(best, e_it);
    std::memcpy(h->acc, host, sizeof(host));
    if (!(e_it > tol) || jend == 0) break;
  }
  if (iters) *iters = total;
  if (eta) *eta = e_it;
  int code = read_status(h, nullptr);
  if (code) return code;
  return (e_it <= tol) ? LUQR_OK : LUQR_ERR_NOT_CONVERGED;
}

// ======================================================================= C ABI
extern "C" {

int luqr_factor(const double* dA, int64_t lda, double* db, int64_t N, int nb, int criterion,
                double alpha, const luqr_options* opt, void* stream, luqr_handle_t* out) {
  if (!out) return LUQR_ERR_INVALID;
  *out = nullptr;
  luqr_options o;
  std::memset(&o, 0, sizeof(o));
  if (opt) o = *opt;
  if (o.group <= 0) o.group = 4;
  if (!dA || N < 1 || nb < 32 || nb > 512 || (nb % 32) != 0 || lda < N) return LUQR_ERR_INVALID;
  if (!(alpha >= 0.0)) return LUQR_ERR_INVALID;   // rejects NaN too
  if (criterion < LUQR_MAX || criterion > LUQR_RANDOM) return LUQR_ERR_INVALID;
  if (o.tree < 0 || o.tree > 2 || o.precision < 0 || o.precision > 1) return LUQR_ERR_INVALID;
  if (o.tree_switch < 0 || o.tree_small < 0 || o.tree_small > 2) return LUQR_ERR_INVALID;
  if (o.fp32_kernels < 0 || o.fp32_kernels > 2) return LUQR_ERR_INVALID;
  if (o.mumps_mode < 0 || o.mumps_mode > 1 || o.n_inject < 0) return LUQR_ERR_INVALID;
  if (o.norm_mode < 0 || o.norm_mode > 1) return LUQR_ERR_INVALID;
  if (o.lu_variant < 0 || o.lu_variant > 1) return LUQR_ERR_INVALID;
  if (o.timeout_ms < 0) return LUQR_ERR_INVALID;
  if (o.domain < 0) return LUQR_ERR_INVALID;
  if (o.domain > 1 && (o.speculate != 0 || o.lu_variant != 0)) return LUQR_ERR_INVALID;
  if (o.lu_variant == 1 && (o.norm_mode != 0 || o.speculate != 0)) return LUQR_ERR_INVALID;
  if (o.speculate < 0 || o.speculate > 2 || (o.speculate == 1 && !o.mlp_params))
    return LUQR_ERR_INVALID;
  luqr_handle* h = new (std::nothrow) luqr_handle();
  if (!h) return LUQR_ERR_NOMEM;
  h->N = N;
  h->nb = nb;
  h->n = (int)((N + nb - 1) / nb);
  h->Npad = (int64_t)h->n * nb;
  h->has_rhs = db != nullptr;
  h->Wc = h->Npad + (h->has_rhs ? 1 : 0);
  h->prec = o.precision;
  h->elt = h->prec == LUQR_PREC_FP64 ? sizeof(double) : sizeof(float);
  h->criterion = criterion;
  h->alpha = alpha;
  h->tree = o.tree;
  h->tree_small = o.tree_small;
  h->tree_switch = o.tree_switch;
  h->group = o.group;
  h->mumps_mode = o.mumps_mode;
  h->norm_mode = o.norm_mode;
  h->lu_variant = o.lu_variant;
  h->domain = o.domain > 1 ? std::min(o.domain, h->n) : 1;
  h->seed = o.seed;
  h->stream = static_cast<cudaStream_t>(stream);
  h->injected.assign(h->n, 0);
  for (int q = 0; q < o.n_inject; ++q) {
    if (!o.inject) { free_handle(h); return LUQR_ERR_INVALID; }
    int k = o.inject[q];
    if (k < 0 || k >= h->n) { free_handle(h); return LUQR_ERR_INVALID; }
    h->injected[k] = 1;
  }
  const int n = h->n;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes);
  };
  A(&h->W, (size_t)h->Npad * h->Wc * h->elt);
  A(&h->Tbuf, (size_t)n * t_step_elems(h) * h->elt);
  A(&h->S, (size_t)nb * nb * h->elt);
  A((void**)&h->piv_s, sizeof(int) * nb);
  A((void**)&h->piv_all, sizeof(int) * (size_t)n * nb);
  A((void**)&h->norms, sizeof(double) * (size_t)n * n);
  A((void**)&h->local, sizeof(unsigned long long) * nb);
  A((void**)&h->away, sizeof(unsigned long long) * nb);
  A((void**)&h->colsum, sizeof(double) * nb);
  A((void**)&h->dec, (size_t)n);
  A((void**)&h->margin, sizeof(double) * n);
  A((void**)&h->lhs, sizeof(double) * n);
  A((void**)&h->rhs, sizeof(double) * n);
  A((void**)&h->status, sizeof(int) * ST_WORDS);
  if (o.forced) A((void**)&h->forced, (size_t)n);
  if (h->domain > 1) {
    A(&h->St, (size_t)h->domain * nb * nb * h->elt);
    A((void**)&h->dpiv_all, sizeof(int) * (size_t)n * nb);
    A(&h->shadow, (size_t)h->Npad * nb * h->elt);
  }
  if (h->lu_variant == 1 || h->domain > 1) A((void**)&h->gate_all, (size_t)n);
  if (h->lu_variant == 1) A((void**)&h->a2gate, (size_t)n);
  h->use_tc = (h->prec == LUQR_PREC_FP32) && (o.fp32_kernels != 1);
  h->use_tc_qr = (h->prec == LUQR_PREC_FP32) && (o.fp32_kernels != 1);
  h->pk_tile = tc_packed_bytes(nb, nb);
  if (h->use_tc) {
    for (int q = 0; q < 2; ++q) {
      A((void**)&h->Lpk[q], tc_packed_bytes(h->Npad, nb));
      if (nb <= 256) {
        A((void**)&h->Linv[q], sizeof(float) * (size_t)nb * nb);
        A((void**)&h->Xpk[q], tc_packed_bytes(nb, nb));
      }
    }
  }
  if (h->use_tc_qr) {
    for (int q = 0; q < 2; ++q) A((void**)&h->Apk[q], (size_t)n * 2 * 3 * h->pk_tile);
    const size_t slots = (size_t)n * 2 * nb * nb;
    A((void**)&h->Wbuf, sizeof(float) * (size_t)h->Npad * h->Wc);
    A((void**)&h->Gbuf, sizeof(float) * slots);
    for (int q = 0; q < 2; ++q) {
      A((void**)&h->Tfull[q], sizeof(float) * slots);
      A((void**)&h->Vt[q], sizeof(float) * slots);
    }
  }
  h->speculate = o.speculate;
  h->mlp = o.mlp_params;
  if (o.log_features || o.speculate) A((void**)&h->feat, sizeof(float) * 16 * (size_t)n);
  if (o.speculate) {
    A((void**)&h->spec, (size_t)n);
    A((void**)&h->qrfac, (size_t)n);
    A((void**)&h->cmt, (size_t)n);
    A((void**)&h->lufac, (size_t)n);
    A((void**)&h->lucmt, (size_t)n);
    A(&h->shadow, (size_t)h->Npad * nb * h->elt);
  }
  int prio_low = 0, prio_high = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&h->upd_stream, cudaStreamNonBlocking, prio_low);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&h->panel_stream, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess && o.speculate)
    e = cudaStreamCreateWithPriority(&h->spec_stream, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&h->la_stream, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess)
    e = cudaStreamCreateWithPriority(&h->extra_stream, cudaStreamNonBlocking, prio_high);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_end, cudaEventDisableTiming);
  h->ev_fact.assign(n, nullptr);
  h->ev_rest.assign(n, nullptr);
  for (int q = 0; q < n && e == cudaSuccess; ++q) {
    e = cudaEventCreateWithFlags(&h->ev_fact[q], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_rest[q], cudaEventDisableTiming);
  }
  h->ev_lvl.assign(n + 2, nullptr);
  h->ev_extra.assign(n, nullptr);
  h->ev_la.assign(n, nullptr);
  for (size_t q = 0; q < h->ev_lvl.size() && e == cudaSuccess; ++q)
    e = cudaEventCreateWithFlags(&h->ev_lvl[q], cudaEventDisableTiming);
  for (int q = 0; q < n && e == cudaSuccess; ++q) {
    e = cudaEventCreateWithFlags(&h->ev_extra[q], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_la[q], cudaEventDisableTiming);
  }
  if (o.speculate) {
    h->ev_stats.assign(n, nullptr);
    h->ev_spec.assign(n, nullptr);
    h->ev_getrf.assign(n, nullptr);
    h->ev_luspec.assign(n, nullptr);
    h->ev_dec.assign(n, nullptr);
    h->ev_splvl.assign(n + 2, nullptr);
    for (size_t q = 0; q < h->ev_splvl.size() && e == cudaSuccess; ++q)
      e = cudaEventCreateWithFlags(&h->ev_splvl[q], cudaEventDisableTiming);
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
      e = cudaEventCreateWithFlags(&h->ev_stats[q], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_spec[q], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_getrf[q], cudaEventDisableTiming);
      if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&h->ev_luspec[q], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_dec[q], cudaEventDisableTiming);
    }
  }
  if (o.timeout_ms > 0) h->wait_cycles = (long long)o.timeout_ms * 2070000LL;  // cycles at 2.07 GHz
  // single-vector second pass in one launch when its shared-memory plan fits
  const bool rq_ok = h->prec == LUQR_PREC_FP64 ? replay_fits<double>(nb) : replay_fits<float>(nb);
  if (e == cudaSuccess && rq_ok && h->domain == 1) {
    rq_build(h);
    A((void**)&h->rq, sizeof(ReplayTask) * h->rq_host.size());
    A((void**)&h->rq_ctl, sizeof(int) * (2 + (size_t)n));
    int sms = 0, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int bps = h->prec == LUQR_PREC_FP64 ? replay_blocks_per_sm<double>(nb)
                                              : replay_blocks_per_sm<float>(nb);
    // one CTA per SM: each claimed task stages and prefetches its tile while it waits, and
    // more waiting CTAs per SM would push other tasks' prefetched tiles out of L2
    h->rq_grid = (int)std::min<size_t>(h->rq_host.size(), (size_t)std::max(1, sms) * std::min(bps, 1));
    if (e == cudaSuccess)
      e = cudaMemcpy(h->rq, h->rq_host.data(), sizeof(ReplayTask) * h->rq_host.size(),
                     cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    free_handle(h);
    cudaGetLastError();
    return cuda_err(e);
  }
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->status, 0, sizeof(int) * ST_WORDS, s);
  cudaMemsetAsync(h->dec, DEC_ABORT, (size_t)n, s);
  cudaMemsetAsync(h->piv_all, 0, sizeof(int) * (size_t)n * nb, s);
  if (h->gate_all) cudaMemsetAsync(h->gate_all, DEC_QR, (size_t)n, s);
  if (h->a2gate) cudaMemsetAsync(h->a2gate, DEC_LU, (size_t)n, s);
  if (o.forced) cudaMemcpyAsync(h->forced, o.forced, (size_t)n, cudaMemcpyHostToDevice, s);
  if (h->prec == LUQR_PREC_FP64) {
    launch_pack<double>(dA, lda, db, N, h->Npad, h->Wc, wsT<double>(h), h->Npad, s);
    enqueue_factor<double>(h);
    if (h->has_rhs) {
      Mat<double> X{wsT<double>(h) + h->Npad * h->Npad, h->Npad};
      enqueue_backsolve<double>(h, X, 1);
      launch_convert_out<double>(X.p, h->Npad, N, 1, db, N, s);
    }
  } else {
    launch_pack<float>(dA, lda, db, N, h->Npad, h->Wc, wsT<float>(h), h->Npad, s);
    enqueue_factor<float>(h);
    if (h->has_rhs) {
      Mat<float> X{wsT<float>(h) + h->Npad * h->Npad, h->Npad};
      enqueue_backsolve<float>(h, X, 1);
      launch_convert_out<float>(X.p, h->Npad, N, 1, db, N, s);
    }
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaStreamSynchronize(s);
    free_handle(h);
    return LUQR_ERR_CUDA;
  }
  *out = h;
  return LUQR_OK;
}

int luqr_solve(luqr_handle_t h, double* db, int nrhs, int64_t ldb, void* stream) {
  if (!h || !db || nrhs < 1 || ldb < h->N) return LUQR_ERR_INVALID;
  h->stream = static_cast<cudaStream_t>(stream);
  int st;
  if (h->prec == LUQR_PREC_FP64) {
    st = solve_impl<double>(h, db, nrhs, ldb, nullptr);
    if (st) return st;
    launch_convert_out<double>(static_cast<double*>(h->rhs_ws), h->Npad, h->N, nrhs, db, ldb, h->stream);
  } else {
    st = solve_impl<float>(h, db, nrhs, ldb, nullptr);
    if (st) return st;
    launch_convert_out<float>(static_cast<float*>(h->rhs_ws), h->Npad, h->N, nrhs, db, ldb, h->stream);
  }
  return cudaGetLastError() == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}

int luqr_refine(luqr_handle_t h, const double* dA, int64_t lda, const double* db, double* dx,
                double tol, int max_iter, int* iters, double* eta, void* stream) {
  if (!h || !dA || !db || !dx || lda < h->N || max_iter < 0 || !(tol >= 0.0)) return LUQR_ERR_INVALID;
  h->stream = static_cast<cudaStream_t>(stream);
  if (int e0 = rq_specialise(h)) return e0;
  cudaStream_t s = h->stream;
  const int64_t N = h->N;
  const int nchunk = (int)((N + 511) / 512);
  if (!h->ref || h->ref_chunks < nchunk) {
    if (h->ref) cudaFree(h->ref);
    h->ref = nullptr;
    cudaError_t e = cudaMalloc(&h->ref, sizeof(double) * ((size_t)N * (nchunk + 2) + 8));
    if (e != cudaSuccess) return cuda_err(e);
    h->ref_chunks = nchunk;
  }
  double* r = h->ref;
  double* partial = r + N;
  double* scal = partial + (size_t)N * nchunk;   // [0] ||A||, [1] ||r||, [2] ||x||, [3] ||b||
  double* xbest = scal + 8;                       // best iterate so far (N)
  int st = ensure_rhs(h, 1);
  if (st) return st;
  launch_row_abs_sum_max(dA, lda, N, partial, nchunk, scal + 0, s);
  launch_vec_absmax(db, N, scal + 3, s);
  cudaMemsetAsync(dx, 0, sizeof(double) * N, s);
  cudaMemcpyAsync(r, db, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  launch_vec_absmax(r, N, scal + 1, s);
  double host[4];
  double best = INFINITY;
  int it = 0;
  for (; it <= max_iter; ++it) {
    // d = solve(r / ||r||) in the factorization's precision; x += ||r|| d
    if (h->prec == LUQR_PREC_FP64) {
      solve_impl<double>(h, r, 1, N, scal + 1);
      launch_axpy_update<double>(dx, static_cast<double*>(h->rhs_ws), N, scal + 1, s);
    } else {
      solve_impl<float>(h, r, 1, N, scal + 1);
      launch_axpy_update<float>(dx, static_cast<float*>(h->rhs_ws), N, scal + 1, s);
    }
    launch_residual(dA, lda, N, dx, db, r, partial, nchunk, s);
    launch_vec_absmax(r, N, scal + 1, s);
    launch_vec_absmax(dx, N, scal + 2, s);
    cudaMemcpyAsync(host, scal, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return LUQR_ERR_CUDA;
    const double e_it = host[1] / (host[0] * host[2] + host[3]);
    if (e_it < best) {
      best = e_it;
      cudaMemcpyAsync(xbest, dx, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
      std::memcpy(h->acc, host, sizeof(host));
    }
    if (!(e_it > tol)) {
      if (iters) *iters = it + 1;
      if (eta) *eta = e_it;
      int code = read_status(h, nullptr);
      return code ? code : LUQR_OK;
    }
  }
  // not converged: hand back the best iterate and its error
  if (std::isfinite(best))
    cudaMemcpyAsync(dx, xbest, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
  if (iters) *iters = it;
  if (eta) *eta = best;
  int code = read_status(h, nullptr);
  return code ? code : LUQR_ERR_NOT_CONVERGED;
}

int luqr_refine_gmres(luqr_handle_t h, const double* dA, int64_t lda, const double* db, double* dx,
                      double tol, int max_iter, int restart, int* iters, double* eta, void* stream) {
  if (!h || !dA || !db || !dx || lda < h->N || max_iter < 0 || restart < 1 || restart > 200 ||
      !(tol >= 0.0))
    return LUQR_ERR_INVALID;
  h->stream = static_cast<cudaStream_t>(stream);
  if (int e0 = rq_specialise(h)) return e0;
  if (h->prec == LUQR_PREC_FP64)
    return refine_gmres_impl<double>(h, dA, lda, db, dx, tol, max_iter, restart, iters, eta);
  return refine_gmres_impl<float>(h, dA, lda, db, dx, tol, max_iter, restart, iters, eta);
}

int luqr_debug_tc_skip(int chunk) {
  if (chunk < -1) return LUQR_ERR_INVALID;
  luqr::tc_set_debug_skip(chunk);
  return LUQR_OK;
}

int luqr_debug_replay_skip(luqr_handle_t h, int task) {
  if (!h || task < -1) return LUQR_ERR_INVALID;
  if (h->rq == nullptr || task >= (int)h->rq_host.size()) return LUQR_ERR_INVALID;
  h->rq_skip = task;
  return LUQR_OK;
}

int luqr_accuracy(luqr_handle_t h, double* eta, double* hpl3, double* norms) {
  if (!h) return LUQR_ERR_INVALID;
  if (!std::isfinite(h->acc[0])) return LUQR_ERR_INVALID;   // no refinement has run
  const double nA = h->acc[0], nr = h->acc[1], nx = h->acc[2], nb = h->acc[3];
  if (eta) *eta = nr / (nA * nx + nb);
  if (hpl3) *hpl3 = nr / (nA * nx * std::ldexp(1.0, -53) * (double)h->N);
  if (norms) std::memcpy(norms, h->acc, sizeof(h->acc));
  return LUQR_OK;
}

int luqr_features(luqr_handle_t h, float* feat, uint8_t* predicted, int* n_out) {
  if (!h || !h->feat) return LUQR_ERR_INVALID;
  int code = read_status(h, nullptr);
  if (feat && cudaMemcpy(feat, h->feat, sizeof(float) * 16 * (size_t)h->n,
                         cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  if (predicted) {
    if (h->spec) {
      if (cudaMemcpy(predicted, h->spec, (size_t)h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return LUQR_ERR_CUDA;
    } else {
      std::memset(predicted, LUQR_DEC_ABORTED, (size_t)h->n);
    }
  }
  if (n_out) *n_out = h->n;
  return code;
}

int luqr_decisions(luqr_handle_t h, uint8_t* dec, double* margin, int* n_out) {
  if (!h) return LUQR_ERR_INVALID;
  int code = read_status(h, nullptr);
  if (n_out) *n_out = h->n;
  if (dec && cudaMemcpy(dec, h->dec, (size_t)h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  if (margin && cudaMemcpy(margin, h->margin, sizeof(double) * h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  return code;
}

int luqr_step_stats(luqr_handle_t h, double* lhs, double* rhs) {
  if (!h) return LUQR_ERR_INVALID;
  int code = read_status(h, nullptr);
  if (lhs && cudaMemcpy(lhs, h->lhs, sizeof(double) * h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  if (rhs && cudaMemcpy(rhs, h->rhs, sizeof(double) * h->n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  return code;
}

int luqr_factor_data(luqr_handle_t h, double* host, int64_t ld) {
  if (!h || !host || ld < h->Npad) return LUQR_ERR_INVALID;
  int code = read_status(h, nullptr);
  const int64_t Np = h->Npad;
  std::vector<unsigned char> buf((size_t)Np * Np * h->elt);
  if (cudaMemcpy(buf.data(), h->W, buf.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return LUQR_ERR_CUDA;
  for (int64_t c = 0; c < Np; ++c)
    for (int64_t r = 0; r < Np; ++r) {
      const size_t idx = (size_t)r + (size_t)c * Np;
      host[r + c * ld] = h->prec == LUQR_PREC_FP64 ? reinterpret_cast<double*>(buf.data())[idx]
                                                   : (double)reinterpret_cast<float*>(buf.data())[idx];
    }
  return code;
}

int luqr_sync(luqr_handle_t h) {
  if (!h) return LUQR_ERR_INVALID;
  const int code = read_status(h, nullptr);
  if (code == LUQR_OK) {
    const int e0 = rq_specialise(h);
    if (e0) return e0;
  }
  return code;
}

int luqr_info(luqr_handle_t h, int* status, int* step, int* row) {
  if (!h) return LUQR_ERR_INVALID;
  int st3[3] = {0, 0, 0};
  int code = read_status(h, st3);
  if (code == LUQR_ERR_CUDA && st3[0] == 0) return LUQR_ERR_CUDA;
  if (status) *status = st3[0];
  if (step) *step = st3[0] ? st3[1] : -1;
  if (row) *row = st3[0] ? st3[2] : -1;
  return LUQR_OK;
}

int luqr_dims(luqr_handle_t h, int* n, int64_t* npad, int* precision) {
  if (!h) return LUQR_ERR_INVALID;
  if (n) *n = h->n;
  if (npad) *npad = h->Npad;
  if (precision) *precision = h->prec;
  return LUQR_OK;
}

void luqr_destroy(luqr_handle_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

const char* luqr_status_string(int status) {
  switch (status) {
    case LUQR_OK: return "ok";
    case LUQR_ERR_INVALID: return "invalid argument";
    case LUQR_ERR_NOMEM: return "device allocation failed";
    case LUQR_ERR_CUDA: return "CUDA runtime error";
    case LUQR_ERR_SINGULAR: return "singular: exact zero pivot";
    case LUQR_ERR_NONFINITE: return "non-finite value in a panel";
    case LUQR_ERR_TIMEOUT: return "bounded device wait expired";
    case LUQR_ERR_NOT_CONVERGED: return "iterative refinement did not converge";
    default: return "unknown status";
  }
}

const char* luqr_version(void) { return "luqr-gb300 0.1.0 (sm_103a)"; }

}  // extern "C"
