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
#include <vector>

#include "../../include/luqr.h"
#include "internal.cuh"

using namespace luqr;

struct luqr_handle {
  int64_t N = 0, Npad = 0, Wc = 0;
  int nb = 0, n = 0, prec = 0, criterion = 0, tree = 0, group = 4, mumps_mode = 0;
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
  // second pass / refinement scratch
  void* rhs_ws = nullptr;
  int rhs_cap = 0;
  double* ref = nullptr;    // x, r, scalars, partial sums
  int ref_chunks = 0;
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
template <typename T>
void enqueue_qr(luqr_handle* h, int k, Mat<T> C, int64_t c0, int64_t c1, bool factor) {
  cudaStream_t s = h->stream;
  const int n = h->n, nb = h->nb, m = n - 1 - k;
  Mat<T> F{wsT<T>(h), h->Npad};
  Mat<const T> Fc{wsT<T>(h), h->Npad};
  T* Tk = static_cast<T*>(h->Tbuf) + (size_t)k * t_step_elems(h);
  const uint8_t* dec = h->dec;
  auto single = [&](TileList tl) {
    if (factor) launch_geqrt<T>(F, k, nb, tl, Tk, n, dec, s);
    launch_unmqr<T>(Fc, k, nb, tl, Tk, n, C, c0, c1, dec, s);
  };
  auto pair = [&](TileList tl, bool tri) {
    if (factor) launch_pair_qrt<T>(F, k, nb, tl, tri, Tk, n, dec, s);
    launch_pair_apply<T>(Fc, k, nb, tl, tri, Tk, n, C, c0, c1, dec, s);
  };
  if (h->tree == LUQR_TREE_FLAT_TS) {
    single(TileList{k, 1, 1, 0});
    for (int i = k + 1; i < n; ++i) pair(TileList{i, 1, 1, i - k}, false);
  } else if (h->tree == LUQR_TREE_BINARY_TT) {
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

// ---------------------------------------------------------------- LU step on a target
template <typename T>
void enqueue_lu_apply(luqr_handle* h, int k, Mat<T> C, int64_t c0, int64_t c1) {
  cudaStream_t s = h->stream;
  const int nb = h->nb;
  const int64_t r0 = (int64_t)k * nb, r1 = r0 + nb, ld = h->Npad;
  T* W = wsT<T>(h);
  Mat<const T> LU{W + r0 + r0 * ld, ld};
  launch_swptrsm<T>(LU, nb, h->piv_all + (size_t)k * nb, C, r0, c0, c1, h->dec, k, s);
  Mat<const T> Ablk{W + r1 + r0 * ld, ld};
  Mat<const T> Brow{C.p + r0 + c0 * C.ld, C.ld};
  Mat<T> Cblk{C.p + r1 + c0 * C.ld, C.ld};
  launch_gemm_update<T>(Ablk, Brow, Cblk, h->Npad - r1, c1 - c0, nb, h->dec, k, DEC_LU, s);
}

template <typename T>
void enqueue_factor(luqr_handle* h) {
  cudaStream_t s = h->stream;
  const int n = h->n, nb = h->nb;
  const int64_t ld = h->Npad;
  T* W = wsT<T>(h);
  T* S = static_cast<T*>(h->S);
  Mat<T> F{W, ld};
  const bool need_inv = (h->forced == nullptr) &&
                        (h->criterion == LUQR_MAX || h->criterion == LUQR_SUM) && h->alpha != 0.0;
  for (int k = 0; k < n; ++k) {
    const int64_t r0 = (int64_t)k * nb, r1 = r0 + nb;
    if (h->injected[k]) launch_scale_rows<T>(W, ld, r0, nb, r0, h->Wc, std::ldexp(1.0, -27), s);
    launch_panel_stats<T>(W, ld, k, n, nb, h->norms + (size_t)k * n, h->local, h->away, h->status,
                          s);
    launch_getrf<T>(W, ld, k, nb, S, h->piv_s, h->status, s);
    if (need_inv) launch_invnorm<T>(S, nb, h->piv_s, h->colsum, h->status, s);
    DecideArgs da{k,        n,         nb,       h->criterion, h->mumps_mode, h->alpha,
                  h->norms + (size_t)k * n, h->colsum, h->local, h->away,     h->forced,
                  h->dec,   h->margin, h->lhs,   h->rhs,       h->status};
    launch_decide<T>(da, S, s);
    // ---- LU branch (Alg. 2)
    launch_lu_commit<T>(W, ld, k, nb, S, h->piv_s, h->piv_all + (size_t)k * nb, h->dec, s);
    Mat<const T> LU{W + r0 + r0 * ld, ld};
    launch_trsm<T>(LU, nb, F, r1, h->Npad, r0, h->dec, k, s);
    enqueue_lu_apply<T>(h, k, F, r1, h->Wc);
    // ---- QR branch (Alg. 3 + Alg. 4)
    enqueue_qr<T>(h, k, F, r1, h->Wc, true);
  }
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
  for (int k = 0; k < h->n; ++k) {
    const int64_t r0 = (int64_t)k * h->nb;
    if (h->injected[k]) launch_scale_rows<T>(X.p, X.ld, r0, h->nb, 0, nrhs, std::ldexp(1.0, -27), h->stream);
    enqueue_lu_apply<T>(h, k, X, 0, nrhs);
    enqueue_qr<T>(h, k, X, 0, nrhs, false);
  }
  enqueue_backsolve<T>(h, X, nrhs);
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
  void* ptrs[] = {h->W,     h->Tbuf,   h->S,    h->piv_s, h->piv_all, h->norms, h->local,
                  h->away,  h->colsum, h->dec,  h->margin, h->lhs,    h->rhs,   h->status,
                  h->forced, h->rhs_ws, h->ref};
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
  if (criterion < LUQR_MAX || criterion > LUQR_FORCE_QR) return LUQR_ERR_INVALID;
  if (o.tree < 0 || o.tree > 2 || o.precision < 0 || o.precision > 1) return LUQR_ERR_INVALID;
  if (o.mumps_mode < 0 || o.mumps_mode > 1 || o.n_inject < 0) return LUQR_ERR_INVALID;
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
  h->group = o.group;
  h->mumps_mode = o.mumps_mode;
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
  if (e != cudaSuccess) {
    free_handle(h);
    cudaGetLastError();
    return cuda_err(e);
  }
  cudaStream_t s = h->stream;
  cudaMemsetAsync(h->status, 0, sizeof(int) * ST_WORDS, s);
  cudaMemsetAsync(h->dec, DEC_ABORT, (size_t)n, s);
  cudaMemsetAsync(h->piv_all, 0, sizeof(int) * (size_t)n * nb, s);
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
  cudaStream_t s = h->stream;
  const int64_t N = h->N;
  const int nchunk = (int)((N + 511) / 512);
  if (!h->ref || h->ref_chunks < nchunk) {
    if (h->ref) cudaFree(h->ref);
    h->ref = nullptr;
    cudaError_t e = cudaMalloc(&h->ref, sizeof(double) * ((size_t)N * (nchunk + 1) + 8));
    if (e != cudaSuccess) return cuda_err(e);
    h->ref_chunks = nchunk;
  }
  double* r = h->ref;
  double* partial = r + N;
  double* scal = partial + (size_t)N * nchunk;   // [0] ||A||, [1] ||r||, [2] ||x||, [3] ||b||
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
    best = std::min(best, e_it);
    if (!(e_it > tol)) {
      if (iters) *iters = it + 1;
      if (eta) *eta = e_it;
      int code = read_status(h, nullptr);
      return code ? code : LUQR_OK;
    }
  }
  if (iters) *iters = it;
  if (eta) *eta = best;
  int code = read_status(h, nullptr);
  return code ? code : LUQR_ERR_NOT_CONVERGED;
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
  return read_status(h, nullptr);
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
