// tdc_syev_tridiag_noalloc: the full solve for small orders with its workspace in a
// fixed device array owned by the library, for callers that cannot allocate device
// memory (see include/tdc.h).
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/tdc.h"
#include "tdc_internal.cuh"

namespace tdc {

int syev_core(int64_t n, const double* d, const double* e, double* lambda, double* Q, int64_t ldq,
              const tdc_opts* opts, void* ws, size_t ws_bytes, int* dev_status, void* stream,
              bool profile_accounting);

namespace {

constexpr int64_t kMaxOrder = TDC_NOALLOC_MAX_N;
constexpr size_t kScratchBytes = TDC_NOALLOC_SCRATCH_BYTES;

// The scratch lives for as long as the library is loaded, once on every device that
// loads it.  In host code the symbol is only a handle: its device address comes from
// cudaGetSymbolAddress, looked up once per device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceScratch {
  void* ptr = nullptr;
  bool ready = false;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

}  // namespace
}  // namespace tdc

extern "C" int tdc_syev_tridiag_noalloc(int64_t n, const double* d, const double* e, double* lambda,
                                        double* Q, int64_t ldq, int* dev_status, void* stream) {
  using namespace tdc;
  if (n < 1 || n > kMaxOrder) return -1;
  if (!d) return -2;
  if (!e && n > 1) return -3;
  if (!lambda) return -4;
  if (!Q) return -5;
  if (ldq < n) return -6;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 4;
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    DeviceScratch& ds = g_scratch_addr[dev];
    if (!ds.ready) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return 4;
      ds.ptr = p;
      ds.ready = true;
    }
    scratch = ds.ptr;
  }
  tdc_opts o;
  tdc_default_opts(&o);
  if (tdc_workspace_bytes(n, &o) > kScratchBytes) return 3;
  return syev_core(n, d, e, lambda, Q, ldq, &o, scratch, kScratchBytes, dev_status, stream, false);
}
