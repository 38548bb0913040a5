// peak_probe.cu -- measurement utility, not part of the method: the FP32
// FMA throughput of the current GPU, the denominator of the inverse search's
// roofline (an FP32 / instruction-issue bound kernel, not a dense contraction).
//
// Every thread runs eight independent FMA chains (enough independent work to
// cover the FMA latency at full occupancy); the grid is a multiple of the SM
// count. flops = 2 x 8 x iterations x threads, timed with CUDA events on the
// given stream around one launch after one warm-up launch.
#include "bdis_internal.cuh"

namespace {

__global__ void __launch_bounds__(256) fma_probe_kernel(float *out, int iters, float a, float b) {
  float x0 = threadIdx.x * 1e-3f, x1 = x0 + 0.1f, x2 = x0 + 0.2f, x3 = x0 + 0.3f;
  float x4 = x0 + 0.4f, x5 = x0 + 0.5f, x6 = x0 + 0.6f, x7 = x0 + 0.7f;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
    x0 = fmaf(x0, a, b);
    x1 = fmaf(x1, a, b);
    x2 = fmaf(x2, a, b);
    x3 = fmaf(x3, a, b);
    x4 = fmaf(x4, a, b);
    x5 = fmaf(x5, a, b);
    x6 = fmaf(x6, a, b);
    x7 = fmaf(x7, a, b);
  }
  const float s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == 1234.5f) out[blockIdx.x] = s;  // keeps the chains live; never true in practice
}

}  // namespace

extern "C" bdis_status bdis_probe_fp32_tflops(int iterations, double *tflops, void *stream) {
  if (!tflops || iterations < 1 || iterations > (1 << 24)) return BDIS_E_INVALID_ARG;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int threads = 256, blocks = sms * 8;
  cudaEvent_t a = nullptr, b = nullptr;
  e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  fma_probe_kernel<<<blocks, threads, 0, st>>>(nullptr, iterations, 0.9999f, 1e-4f);  // warm-up
  cudaEventRecord(a, st);
  fma_probe_kernel<<<blocks, threads, 0, st>>>(nullptr, iterations, 0.9999f, 1e-4f);
  cudaEventRecord(b, st);
  e = cudaEventSynchronize(b);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  const double flops = 2.0 * 8.0 * (double)iterations * threads * (double)blocks;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return BDIS_OK;
}
