// peak.cu -- the arithmetic peaks that the roofline of the batched product is
// measured against: FP32 FMA throughput (scalar and packed-pair instructions)
// and FP64 FMA throughput of this device, from chains of independent FMAs in
// registers (no memory traffic inside the timed loop).
#include <algorithm>

#include "cpm_internal.cuh"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;  // independent FMA chains per thread

// MODE 0: FP32 FMA, 1: FP32 packed-pair FMA (two FMAs per instruction), 2: FP64 FMA
template <int MODE>
__global__ void __launch_bounds__(PK_THREADS) fma_peak_kernel(int iters, float a, float b, float *out) {
  const float seed = 1.0f + 1e-3f * (float)(threadIdx.x & 31);
  float acc = 0.0f;
  if constexpr (MODE == 0) {
    float x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = seed + (float)k;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) acc += x[k];
  } else if constexpr (MODE == 1) {
    float2 x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = make_float2(seed + (float)k, seed - (float)k);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) acc += x[k].x + x[k].y;
  } else {
    double x[PK_CHAINS];
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) x[k] = (double)seed + (double)k;
    const double ad = a, bd = b;
    for (int it = 0; it < iters; ++it)
#pragma unroll
      for (int k = 0; k < PK_CHAINS; ++k) x[k] = fma(x[k], ad, bd);
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) acc += (float)x[k];
  }
  out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = acc;  // keeps the chains live
}

template <int MODE>
cpm_status time_mode(int nsm, int iters, float *out, double *tflops) {
  const unsigned g = (unsigned)nsm * 8;  // 8 blocks of 256 threads per SM
  cudaEvent_t e0, e1;
  CPM_CUDA_TRY(cudaEventCreate(&e0));
  CPM_CUDA_TRY(cudaEventCreate(&e1));
  fma_peak_kernel<MODE><<<g, PK_THREADS>>>(16, 0.999999f, 1e-7f, out);  // warm-up
  cudaEventRecord(e0);
  fma_peak_kernel<MODE><<<g, PK_THREADS>>>(iters, 0.999999f, 1e-7f, out);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cpm_internal_cuda_err(e);
  const double fmas = (double)g * PK_THREADS * PK_CHAINS * (double)iters * (MODE == 1 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return CPM_OK;
}

}  // namespace

extern "C" cpm_status cpm_measure_fma_peak(double *fp32_tflops, double *fp32_pair_tflops, double *fp64_tflops) {
  int dev = 0, nsm = 0;
  CPM_CUDA_TRY(cudaGetDevice(&dev));
  CPM_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  float *out = nullptr;
  const size_t n = (size_t)nsm * 8 * PK_THREADS;
  CPM_CUDA_TRY(cudaMalloc(&out, sizeof(float) * n));
  double t0 = 0.0, t1 = 0.0, t2 = 0.0;
  cpm_status rc = time_mode<0>(nsm, 1 << 15, out, &t0);
  if (rc == CPM_OK) rc = time_mode<1>(nsm, 1 << 14, out, &t1);
  if (rc == CPM_OK) rc = time_mode<2>(nsm, 1 << 11, out, &t2);
  cudaFree(out);
  if (rc) return rc;
  if (fp32_tflops) *fp32_tflops = t0;
  if (fp32_pair_tflops) *fp32_pair_tflops = t1;
  if (fp64_tflops) *fp64_tflops = t2;
  return CPM_OK;
}
