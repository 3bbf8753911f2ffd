// Learned refinement proposal: a 3-layer CNN over coarse (FLEDGE, log10 Q)
// tiles that marks coarse cells where FLL-jump refinement will be needed.
// conv3x3 2->32 + ReLU, conv3x3 32->32 + ReLU, conv3x3 32->1 (logit); loss:
// binary cross-entropy with a positive-class weight. Weights are BF16 for the
// forward and backward passes (FP32 master copy, Adam in FP32); every
// contraction accumulates in FP32. Activations are NCHW float32.
//
// Kernels: one output pixel per thread with all output channels in registers,
// the input tile (+1 halo) and the layer's weights staged in shared memory;
// the weight gradient reduces over pixels per block and adds into FP32
// gradients with one atomic per weight and block.
#include <cuda_bf16.h>

#include <cstring>
#include <vector>

#include "qsl_internal.cuh"

namespace {

constexpr int T = 16;          // output tile edge
constexpr int TH = T + 2;      // with halo
constexpr int C1 = 2, C2 = 32; // input and hidden channels
constexpr int NW1 = 32 * 2 * 9, NB1 = 32, NW2 = 32 * 32 * 9, NB2 = 32, NW3 = 32 * 9, NB3 = 1;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NW1, OFF_W2 = OFF_B1 + NB1, OFF_B2 = OFF_W2 + NW2, OFF_W3 = OFF_B2 + NB2,
              OFF_B3 = OFF_W3 + NW3, NPAR = OFF_B3 + NB3;

// y[n][co][p] = act(b[co] + sum_{ci,k} w[co][ci][k] x[n][ci][p + k - 1])  (zero padding)
// TRANSPOSE: the data gradient of a convolution: w read as w[ci][co][8 - k]
// (channels swapped, kernel flipped), no bias; MASK: multiply by (m > 0).
template <int CIN, int COUT, bool RELU, bool TRANSPOSE, bool BIAS>
__global__ void __launch_bounds__(T* T) conv3x3_kernel(const float* __restrict__ x, const __nv_bfloat16* __restrict__ w,
                                                      const float* __restrict__ b, const float* __restrict__ mask,
                                                      float* __restrict__ y, int H, int W) {
  extern __shared__ float sm[];
  float* xs = sm;                    // CIN x TH x TH
  float* ws = sm + CIN * TH * TH;    // COUT x CIN x 9 (as used)
  const int n = blockIdx.z;
  const int ox = blockIdx.x * T, oy = blockIdx.y * T;
  const int tid = threadIdx.x;
  const size_t plane = (size_t)H * W;
  const float* xn = x + (size_t)n * CIN * plane;
  for (int i = tid; i < CIN * TH * TH; i += T * T) {
    int c = i / (TH * TH), r = (i / TH) % TH, q = i % TH;
    int gy = oy + r - 1, gx = ox + q - 1;
    xs[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xn[c * plane + (size_t)gy * W + gx] : 0.0f;
  }
  for (int i = tid; i < COUT * CIN * 9; i += T * T) {
    int co = i / (CIN * 9), ci = (i / 9) % CIN, k = i % 9;
    float v;
    if (TRANSPOSE)
      v = __bfloat162float(w[(ci * COUT + co) * 9 + (8 - k)]);  // weights stored [CIN'=COUT][COUT'=CIN]
    else
      v = __bfloat162float(w[(co * CIN + ci) * 9 + k]);
    ws[i] = v;
  }
  __syncthreads();
  const int tx = tid % T, ty = tid / T;
  const int gx = ox + tx, gy = oy + ty;
  float acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co) acc[co] = BIAS ? b[co] : 0.0f;
#pragma unroll 1
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float v = xs[(ci * TH + ty + k / 3) * TH + tx + k % 3];
#pragma unroll
      for (int co = 0; co < COUT; ++co) acc[co] = fmaf(v, ws[(co * CIN + ci) * 9 + k], acc[co]);
    }
  }
  if (gx < W && gy < H) {
    float* yn = y + (size_t)n * COUT * plane + (size_t)gy * W + gx;
    const float* mn = mask ? mask + (size_t)n * COUT * plane + (size_t)gy * W + gx : nullptr;
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
      float v = acc[co];
      if (RELU) v = fmaxf(v, 0.0f);
      if (mn && !(mn[co * plane] > 0.0f)) v = 0.0f;
      yn[co * plane] = v;
    }
  }
}

// dW[co][ci][k] += sum_p dy[n][co][p] x[n][ci][p + k - 1]; dB[co] += sum_p dy.
// One block per (tile, image); threads own weights (strided), pixels in smem.
template <int CIN, int COUT>
__global__ void __launch_bounds__(T* T) conv3x3_wgrad_kernel(const float* __restrict__ x, const float* __restrict__ dy,
                                                            float* __restrict__ dw, float* __restrict__ db, int H,
                                                            int W) {
  extern __shared__ float sm[];
  float* xs = sm;                  // CIN x TH x TH
  float* ds = sm + CIN * TH * TH;  // COUT x T x T
  const int n = blockIdx.z;
  const int ox = blockIdx.x * T, oy = blockIdx.y * T;
  const int tid = threadIdx.x;
  const size_t plane = (size_t)H * W;
  const float* xn = x + (size_t)n * CIN * plane;
  const float* dn = dy + (size_t)n * COUT * plane;
  for (int i = tid; i < CIN * TH * TH; i += T * T) {
    int c = i / (TH * TH), r = (i / TH) % TH, q = i % TH;
    int gy = oy + r - 1, gx = ox + q - 1;
    xs[i] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? xn[c * plane + (size_t)gy * W + gx] : 0.0f;
  }
  for (int i = tid; i < COUT * T * T; i += T * T) {
    int c = i / (T * T), r = (i / T) % T, q = i % T;
    int gy = oy + r, gx = ox + q;
    ds[i] = (gy < H && gx < W) ? dn[c * plane + (size_t)gy * W + gx] : 0.0f;
  }
  __syncthreads();
  for (int wi = tid; wi < COUT * CIN * 9; wi += T * T) {
    int co = wi / (CIN * 9), ci = (wi / 9) % CIN, k = wi % 9;
    int ky = k / 3, kx = k % 3;
    float acc = 0.0f;
    for (int r = 0; r < T; ++r)
#pragma unroll 4
      for (int q = 0; q < T; ++q) acc = fmaf(ds[(co * T + r) * T + q], xs[(ci * TH + r + ky) * TH + q + kx], acc);
    atomicAdd(&dw[wi], acc);
  }
  if (tid < COUT) {
    float acc = 0.0f;
    for (int i = 0; i < T * T; ++i) acc += ds[tid * T * T + i];
    atomicAdd(&db[tid], acc);
  }
}

// Logit -> probability, and the BCE loss / logit gradient:
// loss = w y softplus(-z) + (1 - y) softplus(z), averaged over pixels.
__global__ void bce_kernel(const float* __restrict__ z, const float* __restrict__ yl, int64_t n, float pos_w,
                           float* __restrict__ dz, float* __restrict__ loss) {
  float acc = 0.0f;
  const float inv = 1.0f / (float)n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float zi = z[i], yi = yl[i];
    float sp_pos = fmaxf(zi, 0.0f) + log1pf(expf(-fabsf(zi)));  // softplus(z)
    float sp_neg = sp_pos - zi;                                  // softplus(-z)
    acc += pos_w * yi * sp_neg + (1.0f - yi) * sp_pos;
    float s = 1.0f / (1.0f + expf(-zi));
    dz[i] = (-pos_w * yi * (1.0f - s) + (1.0f - yi) * s) * inv;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc * inv);
}

__global__ void sigmoid_kernel(const float* __restrict__ z, int64_t n, float* __restrict__ p) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = 1.0f / (1.0f + expf(-z[i]));
}

__global__ void adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, __nv_bfloat16* __restrict__ wb, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

template <int CIN, int COUT, bool RELU, bool TRANSPOSE, bool BIAS>
int launch_conv(const float* x, const __nv_bfloat16* w, const float* b, const float* mask, float* y, int n, int H,
                int W, cudaStream_t s) {
  size_t smem = sizeof(float) * (CIN * TH * TH + COUT * CIN * 9);
  auto kern = conv3x3_kernel<CIN, COUT, RELU, TRANSPOSE, BIAS>;
  QSL_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((W + T - 1) / T, (H + T - 1) / T, n);
  kern<<<grid, T * T, smem, s>>>(x, w, b, mask, y, H, W);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

template <int CIN, int COUT>
int launch_wgrad(const float* x, const float* dy, float* dw, float* db, int n, int H, int W, cudaStream_t s) {
  size_t smem = sizeof(float) * (CIN * TH * TH + COUT * T * T);
  auto kern = conv3x3_wgrad_kernel<CIN, COUT>;
  QSL_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((W + T - 1) / T, (H + T - 1) / T, n);
  kern<<<grid, T * T, smem, s>>>(x, dy, dw, db, H, W);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

}  // namespace

struct qsl_cnn {
  float* w = nullptr;            // FP32 master parameters
  __nv_bfloat16* wb = nullptr;   // BF16 copy used by the passes
  float* m = nullptr;            // Adam moments
  float* v = nullptr;
  int64_t steps = 0;
  float* act = nullptr;          // activations of the largest batch seen
  size_t act_cap = 0;
};

namespace {

int ensure_act(qsl_cnn* c, size_t pixels, cudaStream_t s) {
  // a1, a2 (32 channels each), z (1), dz (1), d2 (32), d1 (32)
  size_t need = pixels * (32 + 32 + 1 + 1 + 32 + 32);
  if (need <= c->act_cap) return QSL_OK;
  if (c->act) QSL_CHECK_CUDA(cudaFreeAsync(c->act, s));
  c->act = nullptr;
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&c->act, need * sizeof(float), s));
  c->act_cap = need;
  return QSL_OK;
}

int forward(qsl_cnn* c, const float* x, int n, int H, int W, cudaStream_t s, float** a1, float** a2, float** z) {
  size_t P = (size_t)n * H * W;
  int rc = ensure_act(c, P, s);
  if (rc) return rc;
  *a1 = c->act;
  *a2 = *a1 + P * 32;
  *z = *a2 + P * 32;
  if ((rc = launch_conv<C1, C2, true, false, true>(x, c->wb + OFF_W1, c->w + OFF_B1, nullptr, *a1, n, H, W, s)))
    return rc;
  if ((rc = launch_conv<C2, C2, true, false, true>(*a1, c->wb + OFF_W2, c->w + OFF_B2, nullptr, *a2, n, H, W, s)))
    return rc;
  return launch_conv<C2, 1, false, false, true>(*a2, c->wb + OFF_W3, c->w + OFF_B3, nullptr, *z, n, H, W, s);
}

bool dims_ok(int n, int H, int W) { return n >= 1 && H >= 1 && W >= 1 && (int64_t)n * H * W <= (1ll << 31); }

// Network input of each z-slice of a coarse volume (one block per slice):
// channel 0 the FLEDGE map over its largest finite value in the slice
// (non-finite entries 0), channel 1 (log10 Q - 2) / 2 clamped to [-2, 3], a
// missing Q (NaN) counted as the floor Q = 2 and an infinite one as the top
// of the range.
__global__ void __launch_bounds__(256) features_kernel(const float* __restrict__ S, const float* __restrict__ Q,
                                                       int64_t plane, float* __restrict__ X) {
  __shared__ float red[256];
  const int z = blockIdx.x;
  const float* s = S + (size_t)z * plane;
  const float* q = Q + (size_t)z * plane;
  float m = 0.0f;
  for (int64_t i = threadIdx.x; i < plane; i += blockDim.x) {
    const float v = s[i];
    if (isfinite(v) && v > m) m = v;
  }
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const float smax = fmaxf(red[0], 1e-12f);
  float* x0 = X + (size_t)z * 2 * plane;
  float* x1 = x0 + plane;
  for (int64_t i = threadIdx.x; i < plane; i += blockDim.x) {
    const float v = s[i] / smax;
    x0[i] = isfinite(v) ? v : 0.0f;
    float qv = q[i];
    if (isnan(qv) || (isinf(qv) && qv < 0)) qv = 2.0f;  // no Q: the floor Q = 2
    x1[i] = isinf(qv) ? 3.0f : fminf(fmaxf((log10f(fmaxf(qv, 2.0f)) - 2.0f) * 0.5f, -2.0f), 3.0f);
  }
}

// out = 1 where any cell of the 3 x 3 x 3 neighbourhood (clipped to the
// volume; 3 x 3 for one slice) of `in` is nonzero.
__global__ void dilate_kernel(const uint8_t* __restrict__ in, int nz, int ny, int nx, uint8_t* __restrict__ out) {
  const int64_t n = (int64_t)nz * ny * nx;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((int64_t)nx * ny));
    uint8_t v = 0;
    for (int dz = -1; dz <= 1 && !v; ++dz) {
      const int zz = z + dz;
      if (zz < 0 || zz >= nz) continue;
      for (int dy = -1; dy <= 1 && !v; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= ny) continue;
        for (int dx = -1; dx <= 1; ++dx) {
          const int xx = x + dx;
          if (xx < 0 || xx >= nx) continue;
          if (in[((int64_t)zz * ny + yy) * nx + xx]) {
            v = 1;
            break;
          }
        }
      }
    }
    out[i] = v;
  }
}

}  // namespace

extern "C" {

int qsl_cnn_features(const float* S, const float* Q, int nz, int ny, int nx, float* X, void* stream_) {
  if (!S || !Q || !X || nz < 1 || ny < 1 || nx < 1) {
    qsl::set_error("qsl_cnn_features: bad arguments");
    return QSL_EINVAL;
  }
  features_kernel<<<nz, 256, 0, (cudaStream_t)stream_>>>(S, Q, (int64_t)ny * nx, X);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

int qsl_mask_dilate(const uint8_t* in, int nz, int ny, int nx, uint8_t* out, void* stream_) {
  if (!in || !out || in == out || nz < 1 || ny < 1 || nx < 1) {
    qsl::set_error("qsl_mask_dilate: bad arguments (in and out must differ)");
    return QSL_EINVAL;
  }
  const int64_t n = (int64_t)nz * ny * nx;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
  dilate_kernel<<<blocks, 256, 0, (cudaStream_t)stream_>>>(in, nz, ny, nx, out);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

int qsl_cnn_create(const float* params, qsl_cnn** out) {
  if (!params || !out) {
    qsl::set_error("NULL argument");
    return QSL_EINVAL;
  }
  qsl_cnn* c = new qsl_cnn();
  cudaError_t e = cudaMalloc((void**)&c->w, NPAR * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->wb, NPAR * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->m, NPAR * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->v, NPAR * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(c->w, params, NPAR * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->m, 0, NPAR * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(c->v, 0, NPAR * sizeof(float));
  if (e != cudaSuccess) {
    qsl::set_error("CNN allocation failed: %s", cudaGetErrorString(e));
    qsl_cnn_free(c);
    return QSL_ENOMEM;
  }
  to_bf16_kernel<<<(NPAR + 255) / 256, 256>>>(c->w, c->wb, NPAR);
  qsl::count_launch();
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
    qsl::set_error("CNN init failed: %s", cudaGetErrorString(e));
    qsl_cnn_free(c);
    return QSL_ECUDA;
  }
  *out = c;
  return QSL_OK;
}

int qsl_cnn_params(const qsl_cnn* c, float* params) {
  if (!c || !params) {
    qsl::set_error("NULL argument");
    return QSL_EINVAL;
  }
  QSL_CHECK_CUDA(cudaMemcpy(params, c->w, NPAR * sizeof(float), cudaMemcpyDeviceToHost));
  return QSL_OK;
}

int qsl_cnn_forward(qsl_cnn* c, const float* x, int n, int H, int W, float* prob, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if (!c || !x || !prob || !dims_ok(n, H, W)) {
    qsl::set_error("bad CNN forward arguments");
    return QSL_EINVAL;
  }
  float *a1, *a2, *z;
  int rc = forward(c, x, n, H, W, s, &a1, &a2, &z);
  if (rc) return rc;
  int64_t P = (int64_t)n * H * W;
  sigmoid_kernel<<<(int)std::min<int64_t>((P + 255) / 256, 4096), 256, 0, s>>>(z, P, prob);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

int qsl_cnn_loss_grad(qsl_cnn* c, const float* x, const float* y, int n, int H, int W, float pos_weight, float* loss,
                      float* grad, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if (!c || !x || !y || !loss || !grad || !dims_ok(n, H, W) || !(pos_weight > 0)) {
    qsl::set_error("bad CNN loss/gradient arguments");
    return QSL_EINVAL;
  }
  float *a1, *a2, *z;
  int rc = forward(c, x, n, H, W, s, &a1, &a2, &z);
  if (rc) return rc;
  size_t P = (size_t)n * H * W;
  float* dz = z + P;
  float* d2 = dz + P;
  float* d1 = d2 + P * 32;
  QSL_CHECK_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), s));
  QSL_CHECK_CUDA(cudaMemsetAsync(grad, 0, NPAR * sizeof(float), s));
  bce_kernel<<<(int)std::min<size_t>((P + 255) / 256, 4096), 256, 0, s>>>(z, y, (int64_t)P, pos_weight, dz, loss);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  // layer 3: dW3, dB3; d2 = conv^T(dz) masked by a2 > 0 (ReLU)
  if ((rc = launch_wgrad<C2, 1>(a2, dz, grad + OFF_W3, grad + OFF_B3, n, H, W, s))) return rc;
  if ((rc = launch_conv<1, C2, false, true, false>(dz, c->wb + OFF_W3, nullptr, a2, d2, n, H, W, s))) return rc;
  // layer 2
  if ((rc = launch_wgrad<C2, C2>(a1, d2, grad + OFF_W2, grad + OFF_B2, n, H, W, s))) return rc;
  if ((rc = launch_conv<C2, C2, false, true, false>(d2, c->wb + OFF_W2, nullptr, a1, d1, n, H, W, s))) return rc;
  // layer 1
  return launch_wgrad<C1, C2>(x, d1, grad + OFF_W1, grad + OFF_B1, n, H, W, s);
}

int qsl_cnn_adam_step(qsl_cnn* c, const float* grad, float lr, float beta1, float beta2, float eps, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if (!c || !grad || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) || !(beta2 >= 0 && beta2 < 1) || !(eps > 0)) {
    qsl::set_error("bad Adam arguments");
    return QSL_EINVAL;
  }
  c->steps += 1;
  float c1 = 1.0f - powf(beta1, (float)c->steps), c2 = 1.0f - powf(beta2, (float)c->steps);
  adam_kernel<<<(NPAR + 255) / 256, 256, 0, s>>>(c->w, c->m, c->v, grad, c->wb, NPAR, lr, beta1, beta2, eps, c1, c2);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

void qsl_cnn_free(qsl_cnn* c) {
  if (!c) return;
  if (c->act) cudaFree(c->act);
  cudaFree(c->w);
  cudaFree(c->wb);
  cudaFree(c->m);
  cudaFree(c->v);
  delete c;
}

int qsl_cnn_nparams(void) { return NPAR; }

}  // extern "C"
