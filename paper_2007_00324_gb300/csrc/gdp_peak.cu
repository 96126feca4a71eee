// FP64 throughput of the device, measured: the denominator of the FP64
// roofline of the refinement kernels (their predicates, circumcentres and
// split points are FP64; GB300's FP64 rate is a small fraction of its FP32
// rate, so this bound is measured rather than taken from a data sheet).
//
// Every thread runs eight independent chains of fused multiply-adds, enough
// to cover the FMA latency with the warps resident on each SM; the values
// stay bounded and non-negative (0 < a < 1, b > 0) and feed a store that
// depends on all of them and never happens, so no chain can be removed.
#include <cuda_runtime.h>

#include "gdp.h"

namespace {

constexpr int PK_BS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_BS) k_fp64_fma(double* out, int iters, double a, double b) {
  const int gt = blockIdx.x * blockDim.x + threadIdx.x;
  double x[PK_CHAINS];
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) x[c] = 1e-3 * (double)(gt + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < PK_CHAINS; ++c) x[c] = __fma_rn(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < PK_CHAINS; ++c) s += x[c];
  if (s < 0.0) out[gt] = s;   // never true (every chain stays >= 0); keeps every chain live
}

}  // namespace

extern "C" int gdp_measure_fp64_peak(void* cuda_stream, double* tflops) {
  if (!tflops) return GDP_ERR_INPUT;
  *tflops = 0.0;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return GDP_ERR_CUDA;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int grid = n_sm * 8, iters = 4096;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return GDP_ERR_CUDA;
  }
  int st = GDP_OK;
  float best = 0.0f;
  for (int rep = 0; rep < 4 && st == GDP_OK; ++rep) {   // the first launch warms up
    cudaEventRecord(e0, s);
    k_fp64_fma<<<grid, PK_BS, 0, s>>>(nullptr, iters, 0.999999, 1e-7);
    cudaEventRecord(e1, s);
    float ms = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = GDP_ERR_CUDA;
      break;
    }
    if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (cudaGetLastError() != cudaSuccess) st = GDP_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == GDP_OK && best > 0.0f) {
    const double flops = 2.0 * PK_CHAINS * (double)iters * grid * PK_BS;
    *tflops = flops / (best * 1e-3) / 1e12;
  }
  return st;
}
