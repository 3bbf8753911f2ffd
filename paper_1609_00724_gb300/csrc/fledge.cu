// FLEDGE map (Sec. "Adaptive refinements" of arXiv:1609.00724): gradient
// magnitude of the Sobel operator applied to a 2D or 3D field-line-length map.
// Unnormalised separable Sobel ([-1,0,1] derivative along the axis, [1,2,1]
// smoothing along the others), half-sample-symmetric boundary, index units;
// non-finite lengths count as the largest finite length of the map.
//
// HBM-bound: one read and one write per point. Each CTA stages its tile plus a
// one-point halo in shared memory (plain per-CTA loads; consecutive threads
// read consecutive addresses) and evaluates the stencil from there.
#include <cstring>

#include "qsl_internal.cuh"

namespace qsl {
namespace {

// Order-preserving map of floats to unsigned ints for atomicMax.
__device__ __forceinline__ unsigned f2ord(float f) {
  unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void max_finite_kernel(const float* __restrict__ L, int64_t n, unsigned* out) {
  unsigned best = 0;  // below every finite value
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float v = L[i];
    if (isfinite(v)) best = max(best, f2ord(v));
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

__device__ __forceinline__ int refl(int i, int n) { return i < 0 ? -i - 1 : (i >= n ? 2 * n - i - 1 : i); }

__device__ __forceinline__ float fetch(const float* __restrict__ L, int64_t idx, float fill) {
  float v = __ldg(L + idx);
  return isfinite(v) ? v : fill;
}

constexpr int TX2 = 32, TY2 = 8;

__global__ void __launch_bounds__(TX2* TY2) sobel2d_kernel(const float* __restrict__ L, int n0, int n1,
                                                         const unsigned* fill_bits, float* __restrict__ S) {
  __shared__ float t[TY2 + 2][TX2 + 2];
  const float fill = *fill_bits ? ord2f(*fill_bits) : 0.0f;
  int i1b = blockIdx.x * TX2, i0b = blockIdx.y * TY2;
  for (int k = threadIdx.y * TX2 + threadIdx.x; k < (TY2 + 2) * (TX2 + 2); k += TX2 * TY2) {
    int r = k / (TX2 + 2), c = k % (TX2 + 2);
    int i0 = refl(i0b + r - 1, n0), i1 = refl(i1b + c - 1, n1);
    i0 = min(max(i0, 0), n0 - 1);
    i1 = min(max(i1, 0), n1 - 1);
    t[r][c] = fetch(L, (int64_t)i0 * n1 + i1, fill);
  }
  __syncthreads();
  int i0 = i0b + threadIdx.y, i1 = i1b + threadIdx.x;
  if (i0 >= n0 || i1 >= n1) return;
  int r = threadIdx.y + 1, c = threadIdx.x + 1;
  float g0 = (t[r + 1][c - 1] - t[r - 1][c - 1]) + 2.0f * (t[r + 1][c] - t[r - 1][c]) + (t[r + 1][c + 1] - t[r - 1][c + 1]);
  float g1 = (t[r - 1][c + 1] - t[r - 1][c - 1]) + 2.0f * (t[r][c + 1] - t[r][c - 1]) + (t[r + 1][c + 1] - t[r + 1][c - 1]);
  S[(int64_t)i0 * n1 + i1] = sqrtf(g0 * g0 + g1 * g1);
}

constexpr int TX3 = 32, TY3 = 4, TZ3 = 4;

__global__ void __launch_bounds__(TX3* TY3) sobel3d_kernel(const float* __restrict__ L, int n0, int n1, int n2,
                                                         const unsigned* fill_bits, float* __restrict__ S) {
  // tile over (i1, i2) with a 1-point halo, marching along i0 with a rolling
  // window of three planes
  __shared__ float t[3][TY3 + 2][TX3 + 2];
  const float fill = *fill_bits ? ord2f(*fill_bits) : 0.0f;
  int i2b = blockIdx.x * TX3, i1b = blockIdx.y * TY3;
  int z0 = blockIdx.z * TZ3;
  int z1 = min(z0 + TZ3, n0);
  auto load_plane = [&](int slot, int i0) {
    int ii0 = refl(i0, n0);
    for (int k = threadIdx.y * TX3 + threadIdx.x; k < (TY3 + 2) * (TX3 + 2); k += TX3 * TY3) {
      int r = k / (TX3 + 2), c = k % (TX3 + 2);
      int i1 = refl(i1b + r - 1, n1), i2 = refl(i2b + c - 1, n2);
      i1 = min(max(i1, 0), n1 - 1);
      i2 = min(max(i2, 0), n2 - 1);
      t[slot][r][c] = fetch(L, ((int64_t)ii0 * n1 + i1) * n2 + i2, fill);
    }
  };
  load_plane(0, z0 - 1);
  load_plane(1, z0);
  for (int i0 = z0; i0 < z1; ++i0) {
    load_plane((i0 - z0 + 2) % 3, i0 + 1);
    __syncthreads();
    int pm = (i0 - z0) % 3, pc = (i0 - z0 + 1) % 3, pp = (i0 - z0 + 2) % 3;
    int r = threadIdx.y + 1, c = threadIdx.x + 1;
    // smoothing weights [1,2,1] on the two other axes; derivative [-1,0,1]
    float g0 = 0, g1 = 0, g2 = 0;
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        float w = (a == 0 ? 2.0f : 1.0f) * (b == 0 ? 2.0f : 1.0f);
        g0 += w * (t[pp][r + a][c + b] - t[pm][r + a][c + b]);
      }
#pragma unroll
    for (int a = -1; a <= 1; ++a)
#pragma unroll
      for (int b = -1; b <= 1; ++b) {
        int plane = a < 0 ? pm : (a == 0 ? pc : pp);
        float w = (a == 0 ? 2.0f : 1.0f) * (b == 0 ? 2.0f : 1.0f);
        g1 += w * (t[plane][r + 1][c + b] - t[plane][r - 1][c + b]);
        g2 += w * (t[plane][r + b][c + 1] - t[plane][r + b][c - 1]);
      }
    int i1 = i1b + threadIdx.y, i2 = i2b + threadIdx.x;
    if (i1 < n1 && i2 < n2) S[((int64_t)i0 * n1 + i1) * n2 + i2] = sqrtf(g0 * g0 + g1 * g1 + g2 * g2);
    __syncthreads();
  }
}

}  // namespace

int fledge_device(const float* L, int ndim, const int64_t* shape, float* S, cudaStream_t stream) {
  int64_t n = 1;
  for (int i = 0; i < ndim; ++i) n *= shape[i];
  unsigned* fill = nullptr;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&fill, sizeof(unsigned), stream));
  QSL_CHECK_CUDA(cudaMemsetAsync(fill, 0, sizeof(unsigned), stream));
  int dev = 0, sms = 0;
  QSL_CHECK_CUDA(cudaGetDevice(&dev));
  QSL_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (n > 0) {
    int b = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8);
    max_finite_kernel<<<b, 256, 0, stream>>>(L, n, fill);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
    if (ndim == 2) {
      dim3 grid((unsigned)((shape[1] + TX2 - 1) / TX2), (unsigned)((shape[0] + TY2 - 1) / TY2));
      sobel2d_kernel<<<grid, dim3(TX2, TY2), 0, stream>>>(L, (int)shape[0], (int)shape[1], fill, S);
      qsl::count_launch();
    } else {
      dim3 grid((unsigned)((shape[2] + TX3 - 1) / TX3), (unsigned)((shape[1] + TY3 - 1) / TY3),
                (unsigned)((shape[0] + TZ3 - 1) / TZ3));
      sobel3d_kernel<<<grid, dim3(TX3, TY3), 0, stream>>>(L, (int)shape[0], (int)shape[1], (int)shape[2], fill,
                                                         S);
                                                         qsl::count_launch();
    }
    QSL_CHECK_CUDA(cudaGetLastError());
  }
  QSL_CHECK_CUDA(cudaFreeAsync(fill, stream));
  return QSL_OK;
}

}  // namespace qsl

extern "C" int qsl_fledge(const float* length, int ndim, const int64_t* shape, float* s_out, int mem,
                          void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (ndim != 2 && ndim != 3) {
    qsl::set_error("ndim must be 2 or 3");
    return QSL_EINVAL;
  }
  if (!shape) {
    qsl::set_error("shape is NULL");
    return QSL_EINVAL;
  }
  int64_t n = 1;
  for (int i = 0; i < ndim; ++i) {
    if (shape[i] < 1 || shape[i] > (1 << 30)) {
      qsl::set_error("shape[%d] = %lld out of range", i, (long long)shape[i]);
      return QSL_EINVAL;
    }
    n *= shape[i];
  }
  if (!length || !s_out) {
    qsl::set_error("length/s_out is NULL");
    return QSL_EINVAL;
  }
  if (mem == QSL_MEM_DEVICE) return qsl::fledge_device(length, ndim, shape, s_out, stream);
  if (mem != QSL_MEM_HOST) {
    qsl::set_error("bad mem %d", mem);
    return QSL_EINVAL;
  }
  float *dL = nullptr, *dS = nullptr;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&dL, n * sizeof(float), stream));
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&dS, n * sizeof(float), stream));
  QSL_CHECK_CUDA(cudaMemcpyAsync(dL, length, n * sizeof(float), cudaMemcpyHostToDevice, stream));
  int rc = qsl::fledge_device(dL, ndim, shape, dS, stream);
  if (rc) return rc;
  QSL_CHECK_CUDA(cudaMemcpyAsync(s_out, dS, n * sizeof(float), cudaMemcpyDeviceToHost, stream));
  QSL_CHECK_CUDA(cudaFreeAsync(dL, stream));
  QSL_CHECK_CUDA(cudaFreeAsync(dS, stream));
  QSL_CHECK_CUDA(cudaStreamSynchronize(stream));
  return QSL_OK;
}
