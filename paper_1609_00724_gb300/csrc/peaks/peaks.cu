// Peak-rate microbenchmarks of this GPU for the roofline denominators of the
// tracer kernels: the FP32 FMA pipe and L2 read bandwidth. Measurement
// utilities of the benchmark, not part of the method (the paper has no
// counterpart); they read no clock or power setting and change none. Each
// entry point times its kernel with CUDA events on `stream` after one warm-up
// launch and returns the rate of the fastest of `reps` launches.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

// FP32 FMA throughput: every thread runs CHAINS independent FMA chains of
// `iters` steps (the chains hide the FMA latency), so the pipe, not the
// dependency, sets the rate. The result is written only when it cannot be
// known in advance, so the compiler keeps every FMA.
constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) fma_kernel(int iters, float seed, float* out) {
  float v[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) v[c] = seed + (float)(threadIdx.x * CHAINS + c) * 1e-7f;
  const float a = 0.999999f, b = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) v[c] = fmaf(v[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += v[c];
  if (s == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// L2 read bandwidth: a grid-stride sweep of float4 loads over a buffer small
// enough to stay resident in L2, `sweeps` times per launch.
__global__ void __launch_bounds__(512) l2_read_kernel(const float4* __restrict__ buf, int64_t n4, int sweeps,
                                                      float* out) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int s = 0; s < sweeps; ++s)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);  // cached in L2 only
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  const float t = acc.x + acc.y + acc.z + acc.w;
  if (t == 12345.678f) out[0] = t;
}

int sms_of_current(int* sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess ? 0 : -1;
}

}  // namespace

extern "C" {

// FP32 FMA rate in TFLOP/s (an FMA counts 2 FLOP) over the whole GPU; *ms the
// fastest launch's duration. Returns 0 or -1 on a CUDA error.
int qslpk_fp32_fma(int iters, int reps, void* stream_, double* tflops, double* ms) {
  cudaStream_t stream = (cudaStream_t)stream_;
  int sms = 0;
  if (sms_of_current(&sms)) return -1;
  const int threads = 256, blocks = sms * 8;
  float* out = nullptr;
  if (cudaMallocAsync((void**)&out, sizeof(float) * threads * blocks, stream) != cudaSuccess) return -1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_kernel<<<blocks, threads, 0, stream>>>(iters, 1.0f, out);
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, stream);
    fma_kernel<<<blocks, threads, 0, stream>>>(iters, 1.0f + r * 1e-6f, out);
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(out, stream);
  cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return -1;
  const double flop = 2.0 * CHAINS * 16.0 * (double)iters * threads * blocks;
  *ms = best;
  *tflops = flop / (best * 1e-3) / 1e12;
  return 0;
}

// L2 read rate in GB/s over a `bytes` buffer (kept in L2 after a first sweep).
int qslpk_l2_read(int64_t bytes, int sweeps, int reps, void* stream_, double* gbs, double* ms) {
  cudaStream_t stream = (cudaStream_t)stream_;
  int sms = 0;
  if (sms_of_current(&sms)) return -1;
  const int64_t n4 = bytes / 16;
  float4* buf = nullptr;
  float* out = nullptr;
  if (cudaMallocAsync((void**)&buf, n4 * 16, stream) != cudaSuccess) return -1;
  if (cudaMallocAsync((void**)&out, sizeof(float), stream) != cudaSuccess) return -1;
  cudaMemsetAsync(buf, 0, n4 * 16, stream);
  const int threads = 512, blocks = sms * 4;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  l2_read_kernel<<<blocks, threads, 0, stream>>>(buf, n4, 1, out);
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, stream);
    l2_read_kernel<<<blocks, threads, 0, stream>>>(buf, n4, sweeps, out);
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    if (t < best) best = t;
  }
  const cudaError_t e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(buf, stream);
  cudaFreeAsync(out, stream);
  cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return -1;
  *ms = best;
  *gbs = (double)n4 * 16.0 * sweeps / (best * 1e-3) / 1e9;
  return 0;
}

}  // extern "C"
