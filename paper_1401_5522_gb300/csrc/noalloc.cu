// Allocation-free robustness test of one panel.
//
// Some callers cannot call cudaMalloc: code running under a strict device-memory budget
// or inside a pre-reserved memory pool owned by a host application, and real-time paths
// that must not block on the allocator (cudaMalloc can synchronise the device).  luqr_panel_test_noalloc gives them the factorization's
// per-step decision (panel statistics, scratch GETRF of the diagonal tile, exact inverse
// norm and the Eq. 2-4 comparison) without any device allocation: its scratch lives in a
// fixed file-scope device array sized for nb <= LUQR_NOALLOC_MAX_NB and panels of at most
// LUQR_NOALLOC_MAX_TILES tiles.  Every GPU that loads the library keeps that array until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/luqr.h"
#include "internal.cuh"

namespace luqr {
namespace {

constexpr int NA_MAX_NB = LUQR_NOALLOC_MAX_NB;
constexpr int NA_MAX_TILES = LUQR_NOALLOC_MAX_TILES;

constexpr size_t na_align(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t NA_OFF_S = 0;                                                     // nb x nb tile
constexpr size_t NA_OFF_PIV = na_align(NA_OFF_S + sizeof(double) * NA_MAX_NB * NA_MAX_NB);
constexpr size_t NA_OFF_COLSUM = na_align(NA_OFF_PIV + sizeof(int) * NA_MAX_NB);
constexpr size_t NA_OFF_LOCAL = na_align(NA_OFF_COLSUM + sizeof(double) * NA_MAX_NB);
constexpr size_t NA_OFF_AWAY = na_align(NA_OFF_LOCAL + sizeof(unsigned long long) * NA_MAX_NB);
constexpr size_t NA_OFF_NORMS = na_align(NA_OFF_AWAY + sizeof(unsigned long long) * NA_MAX_NB);
constexpr size_t NA_OFF_LHS = na_align(NA_OFF_NORMS + sizeof(double) * NA_MAX_TILES);
constexpr size_t NA_OFF_RHS = na_align(NA_OFF_LHS + sizeof(double));
constexpr size_t NA_OFF_STATUS = na_align(NA_OFF_RHS + sizeof(double));
constexpr size_t NA_BYTES = na_align(NA_OFF_STATUS + sizeof(int) * ST_WORDS);

// The scratch itself.  In host code this name is only a stand-in for the device object:
// its device address comes from cudaGetSymbolAddress (below), never from the host symbol.
__device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device (set up once per device).
int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LUQR_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (g_na_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) return LUQR_ERR_CUDA;
    g_na_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_na_ptr[dev];
  return LUQR_OK;
}

}  // namespace
}  // namespace luqr

extern "C" int luqr_panel_test_noalloc(const double* dpanel, int64_t ld, int64_t rows, int nb,
                                       int criterion, double alpha, int mumps_mode,
                                       uint8_t* ddec, double* dmargin, void* stream) {
  using namespace luqr;
  // An error left pending by an earlier, unrelated launch is not ours to report or clear:
  // refuse to run on top of it.
  if (cudaPeekAtLastError() != cudaSuccess) return LUQR_ERR_CUDA;
  if (!dpanel || !ddec || !dmargin) return LUQR_ERR_INVALID;
  if (nb < 32 || nb > NA_MAX_NB || (nb % 32) != 0) return LUQR_ERR_INVALID;
  if (rows < nb || (rows % nb) != 0 || rows / nb > NA_MAX_TILES || ld < rows) return LUQR_ERR_INVALID;
  if (criterion < LUQR_MAX || criterion > LUQR_FORCE_QR || !(alpha >= 0.0)) return LUQR_ERR_INVALID;
  if (mumps_mode < 0 || mumps_mode > 1) return LUQR_ERR_INVALID;
  unsigned char* base = nullptr;
  const int st = scratch_address(&base);
  if (st != LUQR_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* S = reinterpret_cast<double*>(base + NA_OFF_S);
  int* piv = reinterpret_cast<int*>(base + NA_OFF_PIV);
  double* colsum = reinterpret_cast<double*>(base + NA_OFF_COLSUM);
  unsigned long long* local = reinterpret_cast<unsigned long long*>(base + NA_OFF_LOCAL);
  unsigned long long* away = reinterpret_cast<unsigned long long*>(base + NA_OFF_AWAY);
  double* norms = reinterpret_cast<double*>(base + NA_OFF_NORMS);
  double* lhs = reinterpret_cast<double*>(base + NA_OFF_LHS);
  double* rhs = reinterpret_cast<double*>(base + NA_OFF_RHS);
  int* status = reinterpret_cast<int*>(base + NA_OFF_STATUS);
  const int n = (int)(rows / nb);
  // The array keeps the previous call's contents: clear what must start at zero (the
  // status word; the away maxima are cleared by the statistics launch itself).
  if (cudaMemsetAsync(status, 0, sizeof(int) * ST_WORDS, s) != cudaSuccess) return LUQR_ERR_CUDA;
  launch_panel_stats<double>(dpanel, ld, 0, n, nb, norms, local, away, status, s);
  launch_getrf<double>(dpanel, ld, 0, nb, S, piv, status, s);
  if (criterion == LUQR_MAX || criterion == LUQR_SUM) launch_invnorm<double>(S, nb, piv, colsum, status, s);
  DecideArgs da{0,     n,      nb,    criterion, mumps_mode, alpha, norms, colsum,
                local, away,   nullptr, ddec,    dmargin,    lhs,   rhs,   status};
  launch_decide<double>(da, S, s);
  return cudaGetLastError() == cudaSuccess ? LUQR_OK : LUQR_ERR_CUDA;
}
