// Arithmetic peak probe: the rate at which this GPU retires fused
// multiply-adds of one type, measured by a kernel that does nothing else.
// The plain FP64 path of SPCG is bound by FP64 FMA issue (two FMAs per
// element of X in every fused pass), so its roofline denominator is this
// measured FP64 rate rather than a nominal figure.
//
// Each thread runs kChains independent recurrences a <- a * b + c (b slightly
// below one, so the values stay finite and never become subnormal), enough
// chains per warp to cover the FMA pipe's latency; the grid fills every SM
// several times over.  Only the FMAs are counted: 2 flops each.
#include "common.cuh"
#include "internal.hpp"

namespace spcg {

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 8;

template <typename T>
__global__ void __launch_bounds__(kProbeThreads) k_fma_probe(int iters, T b, T c, T* out) {
  T a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  // a data-dependent store keeps the loop live; it is never taken for the
  // arguments the host passes (the recurrences stay near c / (1 - b))
  if (s == (T)-1) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
spcg_status run_probe(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0;
  SPCG_CK(cudaGetDevice(&dev));
  SPCG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = sms * kProbeBlocksPerSm;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SPCG_CK(cudaEventCreate(&e0));
  cudaError_t err = cudaEventCreate(&e1);
  float ms = 0.f;
  if (err == cudaSuccess) {
    // warm-up launch (module load, clocks), then the timed one
    k_fma_probe<T><<<grid, kProbeThreads, 0, st>>>(iters / 8 + 1, (T)0.9999999, (T)1e-3, nullptr);
    err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) {
      k_fma_probe<T><<<grid, kProbeThreads, 0, st>>>(iters, (T)0.9999999, (T)1e-3, nullptr);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err != cudaSuccess) return from_cuda(err);
  if (!(ms > 0.f)) return SPCG_E_CUDA;
  const double fmas = (double)grid * kProbeThreads * (double)iters * kChains;
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return SPCG_OK;
}

}  // namespace

}  // namespace spcg

extern "C" spcg_status spcg_probe_fma_tflops(int32_t dtype, int32_t iters, double* tflops_out,
                                             void* stream) {
  if (!tflops_out || iters < 1 || (dtype != 0 && dtype != 1)) return SPCG_E_INVALID_ARG;
  *tflops_out = 0.0;
  cudaStream_t st = (cudaStream_t)stream;
  return dtype == 0 ? spcg::run_probe<double>(iters, tflops_out, st)
                    : spcg::run_probe<float>(iters, tflops_out, st);
}
