// Measured arithmetic peaks of the device for the roofline of the FMM's SIMT kernels: chains
// of fused multiply-adds in FP32 or FP64, enough independent chains per thread and enough
// resident warps per SM that the FMA pipe, not latency, bounds the run.
#include "internal.h"

namespace lpb {

constexpr int PK_CHAINS = 8, PK_UNROLL = 32, PK_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PK_THREADS) k_fma_chain(T *sink, int iters, T a, T b) {
  T x[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < PK_UNROLL; ++r)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += x[k];
  if (s == (T)-1.0) sink[0] = s;  // never true for these inputs; keeps the chains alive
}

template <typename T>
static double fma_peak(cudaStream_t st) {
  int dev = 0, sms = 0;
  LPB_CUDA(cudaGetDevice(&dev));
  LPB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  T *sink = nullptr;
  LPB_CUDA(cudaMalloc(&sink, sizeof(T)));
  cudaEvent_t e0, e1;
  LPB_CUDA(cudaEventCreate(&e0));
  LPB_CUDA(cudaEventCreate(&e1));
  const int blocks = sms * 8;  // 64 resident warps per SM
  // FP64 runs far slower on this part; size both runs to a few tens of milliseconds
  const int iters = sizeof(T) == 4 ? 4096 : 256;
  float ms = 0.f;
  for (int rep = 0; rep < 3; ++rep) {  // first launch warms up clocks and caches
    LPB_CUDA(cudaEventRecord(e0, st));
    k_fma_chain<T><<<blocks, PK_THREADS, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
    LPB_LAUNCH();
    LPB_CUDA(cudaEventRecord(e1, st));
    LPB_CUDA(cudaEventSynchronize(e1));
    LPB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  const double flops = 2.0 * PK_CHAINS * PK_UNROLL * (double)iters * blocks * PK_THREADS;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace lpb

extern "C" int lpbfmm_measure_peak(int which, double *tflops) {
  using namespace lpb;
  if (!tflops || which < 0 || which > 1) return LPBFMM_ERR_ARG;
  cudaStream_t st = nullptr;
  int rc = LPBFMM_OK;
  try {
    LPB_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    *tflops = which == LPBFMM_PEAK_FP32_FMA ? fma_peak<float>(st) : fma_peak<double>(st);
  } catch (const CudaError &e) {
    fprintf(stderr, "lpbfmm: CUDA error %s at %s\n", cudaGetErrorString(e.e), e.where);
    rc = e.e == cudaErrorMemoryAllocation ? LPBFMM_ERR_OOM : LPBFMM_ERR_CUDA;
  }
  if (st) cudaStreamDestroy(st);
  return rc;
}
