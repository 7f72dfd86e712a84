// hrp_potrs_noalloc: the triangular solves of hrp_potrs without any device allocation.
//
// Who needs it: code that must not call cudaMalloc at the point where it solves, for
// example a solver step running inside a region where the application forbids new
// device allocations (a framework that owns all device memory through its own pool, a
// latency-critical loop where cudaMalloc's implicit device synchronization is not
// acceptable, or a plugin that is given buffers but no allocator).  hrp_potrs takes its
// scratch from a handle, which allocates it; this entry point instead uses one
// file-scope device array, reserved in every GPU that loads the library until the
// process exits.
//
// Scratch layout (kScratchBytes, fixed): the solve's workspace for n_max (inverses of the
// 64 x 64 diagonal blocks and the two mailboxes of the sweeps, which every call empties
// itself), the sweep ticket and an error word.
// A bounded wait inside a sweep that expires leaves NaN in the rows of B it could not
// solve (and, through the products, in every row that depends on them): that NaN is
// how a caller of this entry point sees the failure.
#include <mutex>

#include "hrp_internal.cuh"

namespace hrp {
namespace {

constexpr int kNoAllocMaxN = 8192;                                   // largest order accepted
constexpr size_t kWorkBytes = potrs_workspace_bytes(kNoAllocMaxN);   // 6 MiB
constexpr size_t kTicketOffset = kWorkBytes;
constexpr size_t kErrOffset = kTicketOffset + sizeof(int);
constexpr size_t kScratchBytes = (kErrOffset + sizeof(unsigned) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_potrs_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;   // device address of g_potrs_scratch on this device
};
constexpr int kMaxDevices = 64;
DeviceScratch g_dev[kMaxDevices];
std::mutex g_mu;

}  // namespace
}  // namespace hrp

using namespace hrp;

extern "C" hrp_status hrp_potrs_noalloc(int n, int nrhs, const double* dL, int ldl, double* dB, int ldb,
                                        void* stream) {
  if (n < 0 || n > kNoAllocMaxN) return HRP_ERR_INVALID_ARG;   // beyond the fixed scratch
  if (nrhs < 0) return HRP_ERR_INVALID_ARG;
  if (n > 0 && !dL) return HRP_ERR_INVALID_ARG;
  if (ldl < (n > 1 ? n : 1)) return HRP_ERR_INVALID_ARG;
  if (n > 0 && nrhs > 0 && !dB) return HRP_ERR_INVALID_ARG;
  if (ldb < (n > 1 ? n : 1)) return HRP_ERR_INVALID_ARG;
  if (n == 0 || nrhs == 0) return HRP_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HRP_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceScratch& d = g_dev[dev];
    if (!d.ready) {
      // once per device, with that device current: the device address of the array (its
      // host-side name is only a stand-in), then a zeroed ticket and error word
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_potrs_scratch) != cudaSuccess) return HRP_ERR_CUDA;
      if (cudaMemset(static_cast<unsigned char*>(p) + kTicketOffset, 0, kScratchBytes - kTicketOffset) != cudaSuccess)
        return HRP_ERR_CUDA;
      d.base = static_cast<unsigned char*>(p);
      d.ready = true;
    }
    base = d.base;
  }
  cudaError_t e = launch_potrs(dL, ldl, dB, ldb, n, nrhs, false, base, reinterpret_cast<int*>(base + kTicketOffset),
                               reinterpret_cast<unsigned*>(base + kErrOffset), s);
  return e == cudaSuccess ? HRP_OK : HRP_ERR_CUDA;
}
