// spcg_gram_apply_noalloc: the fused pass w = A^T (A p) without any device
// allocation, for callers that cannot allocate device memory themselves or
// let a library do it (for example code that runs while a caching allocator
// owns the device memory pool, inside a memory-capped sandbox, or between
// phases where an allocation would synchronise the device).
//
// Its scratch (the per-CTA partial sums and the status word of the pass) is
// a file-scope __device__ array of fixed size, loaded with this library and
// kept by every GPU that loads it until the process exits.  Host code cannot
// use the array's name as a device address: on the host it names a shadow
// object.  The address is looked up once per device with
// cudaGetSymbolAddress, with that device current, by the first call on that
// device.  A failed lookup is not remembered: the next call on that device
// tries again.
//
// All calls share the array and it keeps the last call's contents: the
// status word is cleared on the caller's stream before each launch, and the
// partial sums are fully rewritten by each pass.  Calls that overlap on the
// GPU (on different streams without ordering between them) race on the
// array and may return wrong results.
#include <mutex>

#include "common.cuh"
#include "internal.hpp"

namespace spcg {
spcg_status launch_gram_with_scratch(const PassGeom& g, const double* p, double* w,
                                     double* partials, int ldp, int grid, DevScalars* scal,
                                     cudaStream_t st);
}

namespace {

constexpr int kNoAllocMaxCtas = 160;          // at most one CTA per SM (148 on B300)
constexpr size_t kScalarBytes = 256;
constexpr size_t kNoAllocScratchBytes =
    kScalarBytes + (size_t)kNoAllocMaxCtas * SPCG_MAX_D * sizeof(double);   // 1,310,976 B

static_assert(sizeof(spcg::DevScalars) <= kScalarBytes, "scalar block outgrew its slot");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
// Per-device result of the one-time lookup.  Only a successful lookup is
// kept: an error (for example one left behind by an unrelated asynchronous
// launch) is returned to that call, and the next call tries again.
struct DeviceSlot {
  std::mutex mu;
  void* addr = nullptr;
  int sms = 0;
};
DeviceSlot g_slots[kMaxDevices];

// The scratch array's device address and the SM count on device `dev`
// (the current device).
cudaError_t device_slot(int dev, void** addr, int* sms) {
  DeviceSlot& slot = g_slots[dev];
  std::lock_guard<std::mutex> lock(slot.mu);
  if (!slot.addr) {
    void* a = nullptr;
    int n = 0;
    cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      return e;
    }
    slot.sms = n;
    slot.addr = a;
  }
  *addr = slot.addr;
  *sms = slot.sms;
  return cudaSuccess;
}

}  // namespace

using namespace spcg;

extern "C" spcg_status spcg_gram_apply_noalloc(const double* A, int64_t m, int32_t d,
                                               int64_t lda, const double* p, double* w,
                                               void* stream) {
  if (d < 1 || d > SPCG_MAX_D || m < 0 || !p || !w || (m > 0 && (!A || lda < d)))
    return SPCG_E_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return from_cuda(cudaErrorInvalidDevice);
  if (dev < 0 || dev >= kMaxDevices) return SPCG_E_INVALID_ARG;
  void* scratch = nullptr;
  int sms = 0;
  if (device_slot(dev, &scratch, &sms) != cudaSuccess || !scratch) return SPCG_E_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  if (m == 0) {
    SPCG_CK(cudaMemsetAsync(w, 0, (size_t)d * sizeof(double), st));
    SPCG_CK(cudaStreamSynchronize(st));
    return SPCG_OK;
  }
  PassGeom g;
  SPCG_TRY(make_pass_geom(A, m, d, lda, &g));
  int grid = sms < kNoAllocMaxCtas ? sms : kNoAllocMaxCtas;
  if (grid > g.ntiles) grid = g.ntiles;
  if (grid < 1) grid = 1;
  int ni = 1;
  while (ni * 32 < d) ni <<= 1;
  const int ldp = ni * 32;   // <= SPCG_MAX_D
  DevScalars* scal = reinterpret_cast<DevScalars*>(scratch);
  double* partials = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + kScalarBytes);
  SPCG_CK(cudaMemsetAsync(scal, 0, sizeof(DevScalars), st));
  SPCG_TRY(launch_gram_with_scratch(g, p, w, partials, ldp, grid, scal, st));
  int status = 0;
  SPCG_CK(cudaMemcpyAsync(&status, &scal->status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SPCG_CK(cudaStreamSynchronize(st));
  if (status == DEV_TIMEOUT) return SPCG_E_TIMEOUT;
  if (status != DEV_OK) return SPCG_E_CUDA;
  return SPCG_OK;
}
