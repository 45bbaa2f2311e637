// Allocation-free Gram matrix: the entry point pou_gram_noalloc of pou.h.
//
// pou_gram needs a caller-provided device workspace for the per-split FP64
// partial sums.  Some callers cannot provide one: hosts that hand this
// library a fixed device-memory budget, and loops that must not call
// cudaMalloc once they run (it can synchronise the device and stall every
// stream).  This variant keeps the partial sums in a fixed buffer of static
// device memory instead, which every GPU that loads the library holds until
// the process exits.  The buffer's device address is looked up once per
// device and kept; that assumes the device's primary context (no
// cudaDeviceReset, no other driver context on the device).
#include "pou.h"
#include "pou_internal.cuh"

#include <mutex>

namespace {

constexpr size_t kScratchBytes = POU_GRAM_NOALLOC_MAX_BYTES;
constexpr int kMaxDevices = 64;

// Split partial sums of every pou_gram_noalloc call on this device.  Host code
// must not use this name as an address: it resolves the device address once
// per device with cudaGetSymbolAddress (below).
__device__ __align__(256) double g_gram_scratch[kScratchBytes / sizeof(double)];

std::mutex g_mu;
double* g_addr[kMaxDevices] = {nullptr};

// Device address of g_gram_scratch on the current device, looked up on the
// first call made with that device current.
pou_status scratch_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return POU_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return POU_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return POU_ECUDA;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return POU_OK;
}

template <typename T>
pou_status gram_noalloc(long long Ng, int N, const void* A, double dV, double* S, cudaStream_t s) {
  using namespace pou;
  int nsplit, npair;
  i64 ntiles;
  gram_layout<T>(Ng, N, false, &nsplit, &npair, &ntiles);
  const int ST = gram_supertile<T>();
  const size_t per_split = (size_t)npair * ST * ST * sizeof(double);
  const size_t fit = kScratchBytes / per_split;
  if (fit < 1) return POU_EINVAL;  // one split does not fit the fixed buffer
  if ((size_t)nsplit > fit) nsplit = (int)fit;
  double* scratch = nullptr;
  const pou_status st = scratch_address(&scratch);
  if (st != POU_OK) return st;
  GramArgs<T> g{};
  g.A = static_cast<const T*>(A);
  g.ng = Ng;
  g.N = N;
  g.split = scratch;
  launch_gram_nsplit<T>(g, nsplit, s);
  GramReduceArgs r{};
  r.split = scratch;
  r.nsplit = nsplit;
  r.npair = npair;
  r.ST = ST;
  r.N = N;
  r.dV = dV;
  r.S = S;
  launch_gram_reduce(r, s);
  return cudaGetLastError() == cudaSuccess ? POU_OK : POU_ECUDA;
}

}  // namespace

extern "C" pou_status pou_gram_noalloc(int dtype, long long Ng, int N, const void* A, double dV, double* S,
                                       void* stream) {
  if ((dtype != POU_DT_F64 && dtype != POU_DT_F32) || Ng < 1 || N < 1 || N > POU_MAX_N || !A || !S)
    return POU_EINVAL;
  if (!pou::device_accessible(A) || !pou::device_accessible(S)) return POU_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (dtype == POU_DT_F64) return gram_noalloc<double>(Ng, N, A, dV, S, s);
  return gram_noalloc<float>(Ng, N, A, dV, S, s);
}
