// Householder QR entry point that performs no device allocation.
//
// cpqr_house_qr() allocates its scratch (the working copy of the matrix when it
// does not fit in the cluster's shared memory, and a status word) with
// cudaMalloc on every call.  Some callers cannot do that: a host application
// that has handed all device memory to its own pool and forbids allocations
// behind its back, a latency-critical loop where cudaMalloc / cudaFree would
// stall (they can synchronise the device), or a deployment that must have a
// fixed memory footprint known at load time.  cpqr_house_qr_noalloc() runs the
// same kernel with its scratch in the file-scope array below instead.
#include <mutex>

#include "../../include/cpqr.h"
#include "common.cuh"

namespace {

// Scratch for one call: the working rows (at most CPQR_NOALLOC_QR_MAX_ELEMS doubles) and the
// status word.  Every GPU that loads the library holds it until the process exits.
constexpr size_t kScratchDoubles = (size_t)CPQR_NOALLOC_QR_MAX_ELEMS + 32;
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the array's device address and the context it was looked up in.  A device reset
// (cudaDeviceReset) destroys that context and unloads the module; the next call, made in the new
// context, then looks the address up again instead of using a stale one.
double* g_scratch_addr[kMaxDevices] = {};
void* g_scratch_ctx[kMaxDevices] = {};

typedef int (*cu_ctx_get_current_fn)(void**);  // CUresult cuCtxGetCurrent(CUcontext*)

// The current context's handle through the driver entry point (no link-time driver dependency).
void* current_context() {
  static cu_ctx_get_current_fn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<cu_ctx_get_current_fn>(f);
  }();
  void* c = nullptr;
  if (!fn || fn(&c) != 0) return nullptr;
  return c;
}

// Device address of the scratch array on the current device, looked up once per device and
// context.  The lookup loads the library's module into the context if it is not loaded yet.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  void* ctx = current_context();  // null before the runtime has made a context current
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the primary context current if needed
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<double*>(p);
    g_scratch_ctx[dev] = current_context();
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" cpqr_status cpqr_house_qr_noalloc(const double* A_dev, int64_t M, int32_t R, double* Q_dev,
                                             double* R_dev, void* stream) {
  if (!A_dev || !Q_dev || !R_dev || R < 1 || R > CPQR_MAXR || M < R) return CPQR_EINVAL;
  if (M * (int64_t)R > (int64_t)CPQR_NOALLOC_QR_MAX_ELEMS) return CPQR_EINVAL;  // beyond the fixed scratch
  double* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return CPQR_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* work = scratch;                                                            // M x R rows
  unsigned int* status = reinterpret_cast<unsigned int*>(scratch + CPQR_NOALLOC_QR_MAX_ELEMS);  // 1 word
  // the status word must start at zero; the rows are fully written by the kernel before use
  if (cudaMemsetAsync(status, 0, sizeof(unsigned int), st) != cudaSuccess) return CPQR_ECUDA;
  if (cpqr::launch_house_qr(A_dev, M, R, Q_dev, R_dev, work, status, st) != cudaSuccess) return CPQR_ECUDA;
  // the kernel's status word: a timed-out cluster wait or a zero column (partial results)
  unsigned int hs = 0;
  if (cudaMemcpyAsync(&hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st) != cudaSuccess) return CPQR_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CPQR_ECUDA;
  return cpqr::status_of_device_word(hs);
}
