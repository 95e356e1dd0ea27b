// G = Y^T Y without any device allocation.
//
// sscg_gram allocates (and frees) its block-partial buffer on every call.
// Some callers cannot allow that: programs that fix their device-memory
// budget at start-up and forbid allocation afterwards, and hosts whose own
// memory manager owns the device memory, where a cudaMalloc/cudaFree inside a
// library call would bypass that manager, and cudaFree would also wait for the
// whole device.  sscg_gram_noalloc computes the same Gram matrix with the same
// kernels, taking the partial sums from a fixed array in this file instead.
//
// The scratch array is a file-scope __device__ array: every device that loads
// the library holds it (kGramNoAllocDoubles doubles, 1.36 MB) until the
// process exits, and all calls on a device share it.
#include <mutex>

#include "sscg_internal.cuh"

namespace sscg {
namespace {

// One partial sum per (block, pair): at most gram_blocks() = kGramMaxBlocks
// blocks, and kMaxPairs = 561 pairs for 33 columns.  The row count does not
// enter: longer inputs give each block more rows.
constexpr size_t kGramNoAllocDoubles = (size_t)kGramMaxBlocks * kMaxPairs;
static_assert(kGramNoAllocDoubles == (size_t)304 * 561, "scratch size stated in include/sscg.h");

static __device__ __align__(256) double g_gram_scratch[kGramNoAllocDoubles];

// Device address of g_gram_scratch, looked up once per device ordinal.  A
// device reset (cudaDeviceReset) reloads the module at another address, so
// the cached pointer is then stale: the entry point must not be used on a
// device after it was reset.
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

}  // namespace
}  // namespace sscg

using namespace sscg;

extern "C" int sscg_gram_noalloc(const double* Y, int64_t n, int64_t ldy, int ncols, double* G,
                                 void* cuda_stream) {
  if (!Y || !G || n <= 0 || ldy < n) return SSCG_ERR_INVALID_ARG;
  if (ncols < 1 || ncols > kMaxCols) return SSCG_ERR_INVALID_ARG;  // scratch holds partials for <= 33 columns
  const int nb = gram_blocks(n);
  if (nb > kGramMaxBlocks || (size_t)nb * kMaxPairs > kGramNoAllocDoubles) return SSCG_ERR_INVALID_ARG;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SSCG_ERR_CUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (g_scratch_ptr[dev] == nullptr) {
      // first call on this device: resolve the array's device address with
      // this device current (host code cannot use the symbol itself)
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_gram_scratch) != cudaSuccess || p == nullptr) return SSCG_ERR_CUDA;
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_scratch_ptr[dev];
  }
  // Every partial the reduction reads is written earlier in the same call,
  // so nothing in the scratch has to be cleared.
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (launch_gram(Y, n, ldy, nullptr, ncols, nullptr, scratch, nb, G, ncols, false, st) != cudaSuccess)
    return SSCG_ERR_CUDA;
  return SSCG_OK;
}
