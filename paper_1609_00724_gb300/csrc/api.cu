// C ABI of the GB300 QSL library: argument checking, device memory for host
// arguments, field packing and the tracing calls (see include/qsl.h).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include <map>
#include <mutex>

#include "qsl_internal.cuh"

namespace qsl {

static thread_local std::string g_err;
std::atomic<long long> g_launches{0};

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

#define QSL_FAIL(code, ...)        \
  do {                             \
    qsl::set_error(__VA_ARGS__);   \
    return code;                   \
  } while (0)

// Per-thread record of the last tracing call (for qsl_last_stats).
struct LastCall {
  DeviceStats* host = nullptr;  // pinned
  DeviceStats* dev = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int n_ev = 0;
  cudaStream_t stream = nullptr;
  int64_t lines = 0, retraced = 0;
  int64_t* retraced_host = nullptr;  // pinned
  LaunchShape shape{0, 0, 0};
  bool valid = false;
  int device = -1;
};
static thread_local LastCall g_last;

static int last_call_begin(cudaStream_t stream) {
  int dev = 0;
  QSL_CHECK_CUDA(cudaGetDevice(&dev));
  if (g_last.device != dev) {
    // per-thread, per-device bookkeeping buffers (small, kept until exit)
    QSL_CHECK_CUDA(cudaMallocHost((void**)&g_last.host, sizeof(DeviceStats)));
    QSL_CHECK_CUDA(cudaMallocHost((void**)&g_last.retraced_host, sizeof(int64_t)));
    QSL_CHECK_CUDA(cudaMalloc((void**)&g_last.dev, sizeof(DeviceStats)));
    for (int i = 0; i < 4; ++i) QSL_CHECK_CUDA(cudaEventCreate(&g_last.ev[i]));
    g_last.device = dev;
  }
  QSL_CHECK_CUDA(cudaMemsetAsync(g_last.dev, 0, sizeof(DeviceStats), stream));
  *g_last.retraced_host = 0;
  g_last.stream = stream;
  g_last.n_ev = 0;
  g_last.valid = true;
  return QSL_OK;
}

// ------------------------------------------------------------ options
void resolve_config(const qsl_field* f, const qsl_opts* o, TraceConfig* c) {
  bool use = true;
  for (int a = 0; a < 3; ++a)
    if (!(o->domain_lo[a] < o->domain_hi[a])) use = false;
  for (int a = 0; a < 3; ++a) {
    c->lo[a] = use ? o->domain_lo[a] : f->glo[a];
    c->hi[a] = use ? o->domain_hi[a] : f->ghi[a];
  }
  double ext[3];
  for (int a = 0; a < 3; ++a) ext[a] = c->hi[a] - c->lo[a];
  if (f->geom == QSL_GEOM_SPHERICAL) {  // physical extents at the outer radius
    ext[0] *= c->hi[2];
    ext[1] *= c->hi[2];
  }
  double d2 = ext[0] * ext[0] + ext[1] * ext[1] + ext[2] * ext[2];
  c->max_len = o->max_length > 0 ? o->max_length : 20.0 * std::sqrt(d2);
  c->cell = f->cell;
  c->geom = f->geom;
  c->tol_abs = o->tol_abs;
  c->tol_rel = o->tol_rel;
  c->h_init = o->h_init;
  c->h_max = o->h_max;
  c->h_min = o->h_min;
  c->euler_h = o->euler_h;
  c->land_tol = o->land_tol * (f->geom == QSL_GEOM_SPHERICAL ? f->cell_q : f->cell);
  c->max_steps = o->max_steps;
  c->integrator = o->integrator;
  c->length_only = o->length_only;
  c->timeout_ns = o->timeout_s > 0 ? (unsigned long long)(o->timeout_s * 1e9) : 0ull;
  c->interp_order = o->interp_order > 1 ? o->interp_order : 1;
}

int validate_opts(const qsl_field* f, const qsl_opts* o) {
  if (!f) QSL_FAIL(QSL_EINVAL, "field is NULL");
  if (!o) QSL_FAIL(QSL_EINVAL, "opts is NULL");
  if (o->integrator != QSL_RKCK54 && o->integrator != QSL_EULER && o->integrator != QSL_DOPRI5_CELL)
    QSL_FAIL(QSL_EINVAL, "bad integrator %d", o->integrator);
  if (o->q_form < 0 || o->q_form > 2) QSL_FAIL(QSL_EINVAL, "bad q_form %d", o->q_form);
  if (o->precision != QSL_FP32_MIXED && o->precision != QSL_FP64) QSL_FAIL(QSL_EINVAL, "bad precision %d", o->precision);
  if (!(o->tol_abs > 0) || !(o->tol_rel >= 0)) QSL_FAIL(QSL_EINVAL, "tolerances must be tol_abs > 0, tol_rel >= 0");
  if (!(o->h_init > 0) || !(o->h_max > 0) || !(o->h_min >= 0)) QSL_FAIL(QSL_EINVAL, "step bounds must be positive");
  if (o->integrator == QSL_EULER && !(o->euler_h > 0)) QSL_FAIL(QSL_EINVAL, "euler_h must be positive");
  if (o->max_steps < 1) QSL_FAIL(QSL_EINVAL, "max_steps must be >= 1");
  if (o->warps_per_block < 0 || o->warps_per_block > 8) QSL_FAIL(QSL_EINVAL, "warps_per_block must be 0..8");
  if (o->blocks_per_sm < 0 || o->blocks_per_sm > 32) QSL_FAIL(QSL_EINVAL, "blocks_per_sm must be 0..32");
  if (o->refill_min < 0 || o->refill_min > 32) QSL_FAIL(QSL_EINVAL, "refill_min must be 0..32");
  if (o->line_lanes != 0 && o->line_lanes != 1 && o->line_lanes != 3)
    QSL_FAIL(QSL_EINVAL, "line_lanes must be 0, 1 or 3");
  if (o->interp_order < 0 || o->interp_order > 3) QSL_FAIL(QSL_EINVAL, "interp_order must be 0..3");
  if (o->interp_order > 1 && !f->uniform)
    QSL_FAIL(QSL_EINVAL, "triquadratic and tricubic interpolation need a uniform grid");
  if (o->interp_order > 1 && o->integrator == QSL_DOPRI5_CELL)
    QSL_FAIL(QSL_EINVAL, "the cell-wise integrator is trilinear only; use QSL_RKCK54 or QSL_EULER");
  if (f->geom == QSL_GEOM_SPHERICAL && o->integrator == QSL_DOPRI5_CELL)
    QSL_FAIL(QSL_EINVAL, "spherical geometry runs with QSL_RKCK54 or QSL_EULER");
  return QSL_OK;
}

namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;
}  // namespace

cudaError_t alloc_async(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it == g_pools.end()) {
      cudaMemPoolProps props;
      memset(&props, 0, sizeof props);
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&pool, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      if (e != cudaSuccess) return e;
      g_pools[dev] = pool;
    } else {
      pool = it->second;
    }
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

int default_shape(const qsl_opts* o, int tangent, int precision, LaunchShape* s) {
  s->warps_per_block = o->warps_per_block > 0 ? o->warps_per_block : 4;
  if (o->blocks_per_sm > 0) {
    s->blocks_per_sm = o->blocks_per_sm;
  } else {
    // as many resident warps as registers allow (the launch clamps to the
    // occupancy of the chosen kernel)
    int w = 64;
    s->blocks_per_sm = w / s->warps_per_block;
    if (s->blocks_per_sm < 1) s->blocks_per_sm = 1;
  }
  s->refill_min = o->refill_min > 0 ? o->refill_min : 1;
  s->line_lanes = o->line_lanes;
  return QSL_OK;
}

// ------------------------------------------------------------ field packing
// Largest differences of rsqrt_fp64 / rcp_fp64 from 1 / sqrt(x) and 1 / x, in
// ulps of the latter, over the finite positive inputs (bit patterns of
// non-negative doubles order like their values, so atomicMax on them works).
__global__ void newton_check_kernel(const double* x, int64_t n, double* max_ulp) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    if (!(v > 0.0) || !isfinite(v)) continue;
    const double r1 = 1.0 / sqrt(v), r2 = 1.0 / v;
    const double u1 = fabs(rsqrt_fp64(v) - r1) / (nextafter(r1, INFINITY) - r1);
    const double u2 = fabs(rcp_fp64(v) - r2) / (nextafter(r2, INFINITY) - r2);
    atomicMax((unsigned long long*)&max_ulp[0], (unsigned long long)__double_as_longlong(u1));
    atomicMax((unsigned long long*)&max_ulp[1], (unsigned long long)__double_as_longlong(u2));
  }
}

template <class T>
__global__ void pack_kernel(const T* bx, const T* by, const T* bz, size_t n, int raw, float4* v32, double4_32a* v64,
                            int* bad) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    double B[3] = {(double)bx[i], (double)by[i], (double)bz[i]};
    if (!isfinite(B[0]) || !isfinite(B[1]) || !isfinite(B[2])) {
      atomicExch(bad, 1);
      B[0] = B[1] = B[2] = 0;
    }
    const double s2 = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const double rm = rsqrt_fp64(s2);  // 1 / |B|, 0 for B = 0
    const double m = s2 * rm;
    double o[3];
    for (int a = 0; a < 3; ++a) o[a] = raw ? B[a] : B[a] * rm;
    v32[i] = make_float4((float)o[0], (float)o[1], (float)o[2], (float)m);
    v64[i] = make_double4_32a(o[0], o[1], o[2], m);
  }
}

}  // namespace qsl

using namespace qsl;

extern "C" {

const char* qsl_last_error(void) { return g_err.c_str(); }

int64_t qsl_kernel_launches(void) { return (int64_t)g_launches.load(); }

void qsl_opts_default(qsl_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->integrator = QSL_RKCK54;
  o->q_form = QSL_Q_PERP;
  o->precision = QSL_FP32_MIXED;
  o->tol_abs = 1e-2;
  o->tol_rel = 1e-2;
  o->h_init = 0.1;
  o->h_max = 2.0;
  o->h_min = 1e-15;
  o->max_length = 0;
  o->max_steps = 1000000;
  o->euler_h = 0.2;
  o->retrace_q = 1e6;
  o->land_tol = 1e-12;
  o->timeout_s = 0;
  o->line_lanes = 0;
  o->interp_order = 1;
}

int qsl_load_field(const void* bx, const void* by, const void* bz, int dtype, int mem, int nx, int ny, int nz,
                   const double* xc, const double* yc, const double* zc, int interp_mode, void* stream_,
                   qsl_field** out) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (!out) QSL_FAIL(QSL_EINVAL, "out is NULL");
  *out = nullptr;
  if (!bx || !by || !bz || !xc || !yc || !zc) QSL_FAIL(QSL_EINVAL, "NULL array argument");
  if (dtype != QSL_F32 && dtype != QSL_F64) QSL_FAIL(QSL_EINVAL, "bad dtype %d", dtype);
  if (mem != QSL_MEM_HOST && mem != QSL_MEM_DEVICE) QSL_FAIL(QSL_EINVAL, "bad mem %d", mem);
  if (interp_mode != QSL_PAPER_NORMALIZE_FIRST && interp_mode != QSL_RAW_B)
    QSL_FAIL(QSL_EINVAL, "bad interp_mode %d", interp_mode);
  if (nx < 2 || ny < 2 || nz < 2) QSL_FAIL(QSL_EINVAL, "grid must have at least 2 vertices per axis");
  int n[3] = {nx, ny, nz};
  const double* ax[3] = {xc, yc, zc};
  qsl_field* f = new qsl_field();
  memset(f, 0, sizeof(*f));
  f->cell = INFINITY;
  f->uniform = 1;
  for (int a = 0; a < 3; ++a) {
    f->n[a] = n[a];
    double h0 = ax[a][1] - ax[a][0];
    for (int i = 0; i + 1 < n[a]; ++i) {
      double h = ax[a][i + 1] - ax[a][i];
      if (!(h > 0) || !std::isfinite(h)) {
        delete f;
        QSL_FAIL(QSL_EINVAL, "axis %d coordinates must be finite and strictly increasing", a);
      }
      f->cell = fmin(f->cell, h);
      // uniform when every vertex sits on org + i*h to 1e-12 of the span
      double span = ax[a][n[a] - 1] - ax[a][0];
      double pred = ax[a][0] + (ax[a][n[a] - 1] - ax[a][0]) * (double)(i + 1) / (n[a] - 1);
      if (fabs(ax[a][i + 1] - pred) > 1e-12 * span) f->uniform = 0;
      (void)h0;
    }
    f->glo[a] = ax[a][0];
    f->ghi[a] = ax[a][n[a] - 1];
    f->org[a] = ax[a][0];
    f->h[a] = (ax[a][n[a] - 1] - ax[a][0]) / (n[a] - 1);
  }
  f->mode = interp_mode;
  cudaGetDevice(&f->device);
  size_t N = (size_t)nx * ny * nz;
  size_t esz = dtype == QSL_F32 ? 4 : 8;
  const void* src[3] = {bx, by, bz};
  void* staged[3] = {nullptr, nullptr, nullptr};
  int* bad = nullptr;
  int bad_h = 0;
  // every buffer comes from the library's stream-ordered pool on `stream`, so
  // loading fields of the same size again reuses cached blocks (no driver
  // allocation); releases go back to the pool on the same stream
  auto fail = [&](int code) {
    cudaStreamSynchronize(stream);
    for (int a = 0; a < 3; ++a) {
      if (staged[a]) cudaFreeAsync(staged[a], stream);
      if (f->axis64[a]) cudaFreeAsync(f->axis64[a], stream);
      if (f->axis32[a]) cudaFreeAsync(f->axis32[a], stream);
    }
    if (bad) cudaFreeAsync(bad, stream);
    if (f->v32) cudaFreeAsync(f->v32, stream);
    if (f->v64) cudaFreeAsync(f->v64, stream);
    cudaStreamSynchronize(stream);
    delete f;
    return code;
  };
#define TRY(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      set_error("%s failed: %s", #call, cudaGetErrorString(e_));                              \
      return fail(e_ == cudaErrorMemoryAllocation ? QSL_ENOMEM : QSL_ECUDA);                   \
    }                                                                                          \
  } while (0)
  TRY(qsl::alloc_async((void**)&f->v32, N * sizeof(float4), stream));
  TRY(qsl::alloc_async((void**)&f->v64, N * sizeof(double4_32a), stream));
  TRY(qsl::alloc_async((void**)&bad, sizeof(int), stream));
  TRY(cudaMemsetAsync(bad, 0, sizeof(int), stream));
  for (int a = 0; a < 3; ++a) {
    TRY(qsl::alloc_async((void**)&f->axis64[a], n[a] * sizeof(double), stream));
    TRY(qsl::alloc_async((void**)&f->axis32[a], n[a] * sizeof(float), stream));
    TRY(cudaMemcpyAsync(f->axis64[a], ax[a], n[a] * sizeof(double), cudaMemcpyHostToDevice, stream));
    float* tmp = new float[n[a]];
    for (int i = 0; i < n[a]; ++i) tmp[i] = (float)ax[a][i];
    cudaError_t e = cudaMemcpyAsync(f->axis32[a], tmp, n[a] * sizeof(float), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);  // tmp is pageable and freed next
    delete[] tmp;
    TRY(e);
    if (mem == QSL_MEM_HOST) {
      TRY(qsl::alloc_async(&staged[a], N * esz, stream));
      TRY(cudaMemcpyAsync(staged[a], src[a], N * esz, cudaMemcpyHostToDevice, stream));
    }
  }
  const void* p[3];
  for (int a = 0; a < 3; ++a) p[a] = mem == QSL_MEM_HOST ? staged[a] : src[a];
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int blocks = (int)std::min<size_t>((N + 255) / 256, (size_t)sms * 32);
  if (dtype == QSL_F32)
    pack_kernel<float><<<blocks, 256, 0, stream>>>((const float*)p[0], (const float*)p[1], (const float*)p[2], N,
                                                   interp_mode == QSL_RAW_B, f->v32, f->v64, bad);
  else
    pack_kernel<double><<<blocks, 256, 0, stream>>>((const double*)p[0], (const double*)p[1],
                                                    (const double*)p[2], N, interp_mode == QSL_RAW_B, f->v32,
                                                    f->v64, bad);
  qsl::count_launch();
  TRY(cudaGetLastError());
  TRY(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, stream));
  for (int a = 0; a < 3; ++a)
    if (staged[a]) {
      TRY(cudaFreeAsync(staged[a], stream));
      staged[a] = nullptr;
    }
  TRY(cudaFreeAsync(bad, stream));
  bad = nullptr;
  TRY(cudaStreamSynchronize(stream));
  if (bad_h) {
    set_error("field contains non-finite values");
    return fail(QSL_ENONFINITE);
  }
#undef TRY
  *out = f;
  return QSL_OK;
}

void qsl_free_field(qsl_field* f) {
  if (!f) return;
  // work on any stream may still read the field: wait for the device to be
  // idle (as cudaFree does), then hand the blocks back to the pool
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != f->device) cudaSetDevice(f->device);
  cudaDeviceSynchronize();
  void* bufs[8] = {f->v32, f->v64, f->axis64[0], f->axis64[1], f->axis64[2], f->axis32[0], f->axis32[1], f->axis32[2]};
  for (void* b : bufs)
    if (b) cudaFreeAsync(b, 0);
  cudaStreamSynchronize(0);
  if (cur != f->device) cudaSetDevice(cur);
  delete f;
}

}  // extern "C"

namespace qsl {

// Common driver of qsl_trace_seeds / qsl_q_map_2d / qsl_q_volume_3d: the
// FP32 (or FP64) trace, then the FP64 retrace of lines above retrace_q.
// Device statistics of the last run_lines on this thread (valid after it
// returns; the stream orders readers after its kernels).
const DeviceStats* last_run_stats_dev() { return g_last.dev; }

int run_lines(const qsl_field* f, const SeedSource& src, int64_t S, const qsl_opts* o, const LineOutputs& out,
              cudaStream_t stream) {
  TraceConfig cfg;
  resolve_config(f, o, &cfg);
  int rc = last_call_begin(stream);
  if (rc) return rc;
  LaunchShape shape;
  default_shape(o, !o->length_only, o->precision, &shape);
  g_last.shape = shape;
  g_last.lines = S;
  rc = trace_and_assemble(f, src, S, nullptr, cfg, o->precision, shape, out, stream, g_last.dev, &g_last.ev[0]);
  if (rc) return rc;
  g_last.n_ev = 2;
  if (o->precision == QSL_FP32_MIXED && o->retrace_q > 0 && !o->length_only && S > 0) {
    int64_t* index = nullptr;
    int64_t* count = nullptr;
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&index, sizeof(int64_t) * S, stream));
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&count, sizeof(int64_t), stream));
    rc = select_retrace(src, S, out, o->retrace_q, index, count, stream);
    if (rc) return rc;
    LineOutputs o2 = out;
    o2.retraced = 1;
    LaunchShape sh2;
    default_shape(o, 1, QSL_FP64, &sh2);
    rc = trace_and_assemble(f, src, S, count, cfg, QSL_FP64, sh2, o2, stream, g_last.dev, &g_last.ev[2], index);
    if (rc) return rc;
    g_last.n_ev = 4;
    QSL_CHECK_CUDA(cudaMemcpyAsync(g_last.retraced_host, count, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
    QSL_CHECK_CUDA(cudaFreeAsync(index, stream));
    QSL_CHECK_CUDA(cudaFreeAsync(count, stream));
  }
  QSL_CHECK_CUDA(cudaMemcpyAsync(g_last.host, g_last.dev, sizeof(DeviceStats), cudaMemcpyDeviceToHost, stream));
  return QSL_OK;
}

// Device buffer that is either the caller's (device memory) or a staging copy.
struct Staged {
  void* dev = nullptr;
  void* user = nullptr;
  size_t bytes = 0;
  bool owned = false;
};

static int stage_out(void* user, size_t bytes, int mem, cudaStream_t s, Staged* st) {
  st->user = user;
  st->bytes = bytes;
  if (!user || mem == QSL_MEM_DEVICE) {
    st->dev = user;
    return QSL_OK;
  }
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&st->dev, bytes ? bytes : 1, s));
  st->owned = true;
  return QSL_OK;
}

static int stage_in(const void* user, size_t bytes, int mem, cudaStream_t s, Staged* st) {
  st->user = (void*)user;
  st->bytes = bytes;
  if (!user || mem == QSL_MEM_DEVICE) {
    st->dev = (void*)user;
    return QSL_OK;
  }
  QSL_CHECK_CUDA(qsl::alloc_async((void**)&st->dev, bytes ? bytes : 1, s));
  st->owned = true;
  if (bytes) QSL_CHECK_CUDA(cudaMemcpyAsync(st->dev, user, bytes, cudaMemcpyHostToDevice, s));
  return QSL_OK;
}

static int unstage(Staged* st, bool copy_back, cudaStream_t s) {
  if (!st->owned) return QSL_OK;
  if (copy_back && st->bytes)
    QSL_CHECK_CUDA(cudaMemcpyAsync(st->user, st->dev, st->bytes, cudaMemcpyDeviceToHost, s));
  QSL_CHECK_CUDA(cudaFreeAsync(st->dev, s));
  st->owned = false;
  return QSL_OK;
}

static int map_common(const qsl_field* f, const SeedSource& src, int64_t S, const qsl_opts* o, float* q,
                      float* length, uint8_t* faces, uint8_t* status, int mem, cudaStream_t stream) {
  int rc = validate_opts(f, o);
  if (rc) return rc;
  if (mem != QSL_MEM_HOST && mem != QSL_MEM_DEVICE) QSL_FAIL(QSL_EINVAL, "bad mem %d", mem);
  Staged sq, sl, sf, ss;
  if ((rc = stage_out(q, S * sizeof(float), mem, stream, &sq))) return rc;
  if ((rc = stage_out(length, S * sizeof(float), mem, stream, &sl))) return rc;
  if ((rc = stage_out(faces, S * 2, mem, stream, &sf))) return rc;
  if ((rc = stage_out(status, S, mem, stream, &ss))) return rc;
  LineOutputs out{};
  out.q = (float*)sq.dev;
  out.length = (float*)sl.dev;
  out.faces = (uint8_t*)sf.dev;
  out.status = (uint8_t*)ss.dev;
  out.q_form = o->q_form;
  out.skip_open = o->skip_open;
  // the FP64 retrace selects from the q output; give it a scratch one if absent
  Staged sq2;
  if (!out.q && o->precision == QSL_FP32_MIXED && o->retrace_q > 0 && !o->length_only) {
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&sq2.dev, S * sizeof(float) + 4, stream));
    sq2.owned = true;
    sq2.bytes = 0;
    out.q = (float*)sq2.dev;
  }
  rc = run_lines(f, src, S, o, out, stream);
  if (rc) return rc;
  if ((rc = unstage(&sq, true, stream)) || (rc = unstage(&sl, true, stream)) || (rc = unstage(&sf, true, stream)) ||
      (rc = unstage(&ss, true, stream)) || (rc = unstage(&sq2, false, stream)))
    return rc;
  if (mem == QSL_MEM_HOST) QSL_CHECK_CUDA(cudaStreamSynchronize(stream));
  return QSL_OK;
}

}  // namespace qsl

extern "C" {

int qsl_trace_seeds(const qsl_field* f, const double* seeds, int64_t S, const qsl_opts* o, qsl_line* out, int mem,
                    void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  int rc = validate_opts(f, o);
  if (rc) return rc;
  if (S < 0) QSL_FAIL(QSL_EINVAL, "S must be >= 0");
  if (S > 0 && (!seeds || !out)) QSL_FAIL(QSL_EINVAL, "seeds/out is NULL");
  if (mem != QSL_MEM_HOST && mem != QSL_MEM_DEVICE) QSL_FAIL(QSL_EINVAL, "bad mem %d", mem);
  Staged si, so;
  if ((rc = stage_in(seeds, S * 3 * sizeof(double), mem, stream, &si))) return rc;
  if ((rc = stage_out(out, S * sizeof(qsl_line), mem, stream, &so))) return rc;
  SeedSource src{};
  src.kind = SEEDS_ARRAY;
  src.xyz = (const double*)si.dev;
  LineOutputs lo{};
  lo.lines = (qsl_line*)so.dev;
  lo.q_form = QSL_Q_PERP;
  lo.skip_open = o->skip_open;
  rc = run_lines(f, src, S, o, lo, stream);
  if (rc) return rc;
  if ((rc = unstage(&so, true, stream)) || (rc = unstage(&si, false, stream))) return rc;
  if (mem == QSL_MEM_HOST) QSL_CHECK_CUDA(cudaStreamSynchronize(stream));
  return QSL_OK;
}

int qsl_q_map_2d(const qsl_field* f, const double center[3], const double u[3], const double v[3], int nu, int nv,
                 const qsl_opts* o, float* q, float* length, uint8_t* faces, uint8_t* status, int mem,
                 void* stream) {
  if (!center || !u || !v) QSL_FAIL(QSL_EINVAL, "center/u/v is NULL");
  if (nu < 0 || nv < 0) QSL_FAIL(QSL_EINVAL, "nu, nv must be >= 0");
  SeedSource src{};
  src.kind = SEEDS_PLANE;
  src.n[0] = nu;
  src.n[1] = nv;
  src.n[2] = 1;
  for (int k = 0; k < 3; ++k) {
    src.c[k] = center[k];
    src.u[k] = u[k];
    src.v[k] = v[k];
  }
  return map_common(f, src, (int64_t)nu * nv, o, q, length, faces, status, mem, (cudaStream_t)stream);
}

int qsl_q_volume_3d(const qsl_field* f, const double lo[3], const double hi[3], int nx, int ny, int nz,
                    const qsl_opts* o, float* q, float* length, uint8_t* faces, uint8_t* status, int mem,
                    void* stream) {
  if (!lo || !hi) QSL_FAIL(QSL_EINVAL, "lo/hi is NULL");
  if (nx < 0 || ny < 0 || nz < 0) QSL_FAIL(QSL_EINVAL, "lattice sizes must be >= 0");
  SeedSource src{};
  src.kind = SEEDS_VOLUME;
  src.n[0] = nx;
  src.n[1] = ny;
  src.n[2] = nz;
  for (int k = 0; k < 3; ++k) {
    src.c[k] = lo[k];
    src.u[k] = hi[k];
  }
  return map_common(f, src, (int64_t)nx * ny * nz, o, q, length, faces, status, mem, (cudaStream_t)stream);
}

int qsl_set_geometry(qsl_field* f, int geometry) {
  if (!f) QSL_FAIL(QSL_EINVAL, "field is NULL");
  double hmin = fmin(fmin(f->h[0], f->h[1]), f->h[2]);
  if (geometry == QSL_GEOM_CARTESIAN) {
    f->geom = QSL_GEOM_CARTESIAN;
    if (f->uniform) f->cell = hmin;  // (a spherical field had a physical cell edge here)
    f->cell_q = f->cell;
    return QSL_OK;
  }
  if (geometry != QSL_GEOM_SPHERICAL) QSL_FAIL(QSL_EINVAL, "bad geometry %d", geometry);
  if (!f->uniform) QSL_FAIL(QSL_EINVAL, "spherical geometry needs a uniform (phi, theta, r) grid");
  const double half_pi = 1.5707963267948966;
  if (!(f->glo[1] > -half_pi && f->ghi[1] < half_pi && f->glo[2] > 0))
    QSL_FAIL(QSL_EINVAL, "spherical grid needs latitudes inside (-pi/2, pi/2) and radii > 0");
  // step sizes are physical lengths: the smallest cell edge at the lowest radius
  double cmin = fmin(cos(f->glo[1]), cos(f->ghi[1]));
  f->cell = fmin(fmin(f->glo[2] * cmin * f->h[0], f->glo[2] * f->h[1]), f->h[2]);
  f->cell_q = hmin;
  f->geom = QSL_GEOM_SPHERICAL;
  return QSL_OK;
}

int qsl_check_fp64_newton(const double* x, int64_t n, double* max_ulp_out) {
  if (n < 1 || !x || !max_ulp_out) QSL_FAIL(QSL_EINVAL, "need n >= 1 and non-NULL pointers");
  double *dx = nullptr, *dm = nullptr;
  QSL_CHECK_CUDA(cudaMalloc((void**)&dx, sizeof(double) * n));
  QSL_CHECK_CUDA(cudaMalloc((void**)&dm, sizeof(double) * 2));
  QSL_CHECK_CUDA(cudaMemcpy(dx, x, sizeof(double) * n, cudaMemcpyHostToDevice));
  QSL_CHECK_CUDA(cudaMemset(dm, 0, sizeof(double) * 2));
  const int blocks = (int)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024);
  newton_check_kernel<<<blocks, 256>>>(dx, n, dm);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpy(max_ulp_out, dm, sizeof(double) * 2, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dm);
  if (e != cudaSuccess) QSL_FAIL(QSL_ECUDA, "%s", cudaGetErrorString(e));
  return QSL_OK;
}

int qsl_trim_pool(void) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  for (auto& kv : g_pools) QSL_CHECK_CUDA(cudaMemPoolTrimTo(kv.second, 0));
  return QSL_OK;
}

int qsl_last_stats(qsl_stats* s) {
  if (!s) QSL_FAIL(QSL_EINVAL, "out is NULL");
  memset(s, 0, sizeof(*s));
  if (!g_last.valid) QSL_FAIL(QSL_EINVAL, "no tracing call on this thread yet");
  QSL_CHECK_CUDA(cudaStreamSynchronize(g_last.stream));
  s->lines = g_last.lines;
  s->stage_evals = (int64_t)g_last.host->stage_evals;
  s->accepted = (int64_t)g_last.host->accepted;
  s->rejected = (int64_t)g_last.host->rejected;
  s->landing = (int64_t)g_last.host->landing;
  s->retraced = *g_last.retraced_host;
  double ms = 0;
  for (int i = 0; i + 1 < g_last.n_ev; i += 2) {
    float t = 0;
    QSL_CHECK_CUDA(cudaEventElapsedTime(&t, g_last.ev[i], g_last.ev[i + 1]));
    ms += t;
  }
  s->kernel_ms = ms;
  s->warps_per_block = g_last.shape.warps_per_block;
  s->blocks_per_sm = g_last.shape.blocks_per_sm;
  s->refill_min = g_last.shape.refill_min;
  if (g_last.host->timeouts) QSL_FAIL(QSL_ETIMEOUT, "device watchdog expired in %llu warps", g_last.host->timeouts);
  return QSL_OK;
}

}  // extern "C"
