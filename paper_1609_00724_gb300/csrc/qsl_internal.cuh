// Internal declarations of the GB300 QSL library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/qsl.h"

#include <atomic>

namespace qsl {

// Number of this library's kernel launches since load (qsl_kernel_launches).
extern std::atomic<long long> g_launches;
inline void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
#define QSL_CHECK_CUDA(call)                                                             \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      qsl::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? QSL_ENOMEM : QSL_ECUDA;                   \
    }                                                                                    \
  } while (0)

// ---------------------------------------------------------------- field
// Device view of a packed field. Vertex (i, j, k) is v[(k*ny + j)*nx + i].
template <class R>
struct V4;
template <>
struct V4<float> {
  typedef float4 type;
};
template <>
struct V4<double> {
  typedef double4_32a type;
};

template <class R>
struct FieldView {
  const typename V4<R>::type* v;
  const R* axis[3];   // vertex coordinates per axis (rectilinear grids)
  R org[3];           // first vertex per axis (uniform grids)
  R inv_h[3];         // 1 / spacing per axis (uniform grids)
  int n[3];
  int uniform;        // 1: all axes uniform (fast cell location)
  int raw;            // 1: QSL_RAW_B packing, 0: paper packing
  int order;          // interpolation: 1 trilinear, 2 triquadratic, 3 tricubic (uniform grids)
  int geom;           // 0 Cartesian; 1 spherical: axes (phi, theta, r), components (phi^, theta^, r^)
};

// Scale factors of the coordinates (a displacement dq_i is the physical
// length m_i dq_i): Cartesian 1; spherical (r cos(theta), r, 1), Eq. fl_sph.
template <class R>
__host__ __device__ __forceinline__ void sph_scale(R theta, R r, R* m) {
  m[0] = r * cos(theta);
  m[1] = r;
  m[2] = R(1);
}

// FP64 reciprocal square root and reciprocal without an FP64 square root or
// division (GB300's FP64 rate makes those the cost of the packing and the
// assembly kernels): Newton-Raphson iteration, x <- x (3 - s x^2) / 2 for
// 1 / sqrt(s) and x <- x (2 - s x) for 1 / s, started from the FP32 estimate;
// each step doubles the correct bits (about 23 -> 46 -> 92), so two reach FP64
// precision (within an ulp or two of the rounded result). Arguments outside
// the FP32 normal range take the FP64 operations; rsqrt_fp64(0) is 0.
__device__ __forceinline__ double rsqrt_fp64(double s) {
  if (!(s > 1e-30 && s < 1e30)) return s > 0.0 ? 1.0 / sqrt(s) : 0.0;
  double x = (double)rsqrtf((float)s);
  x = x * fma(-0.5 * s, x * x, 1.5);
  x = x * fma(-0.5 * s, x * x, 1.5);
  return x;
}

__device__ __forceinline__ double rcp_fp64(double s) {
  const double a = fabs(s);
  if (!(a > 1e-30 && a < 1e30)) return 1.0 / s;
  double x = (double)__frcp_rn((float)s);
  x = x * fma(-s, x, 2.0);
  x = x * fma(-s, x, 2.0);
  return x;
}

}  // namespace qsl

struct qsl_field {
  int n[3];
  int mode;
  int uniform;
  double cell;                 // smallest spacing over all axes
  double glo[3], ghi[3];       // grid extent
  double org[3], h[3];         // uniform spacing (valid when uniform)
  float4* v32;                 // packed vertices, FP32
  double4_32a* v64;                // packed vertices, FP64 (for FP64 tracing)
  double* axis64[3];           // device axis coordinates
  float* axis32[3];
  int device;
  int geom;                    // QSL_GEOM_CARTESIAN or QSL_GEOM_SPHERICAL
  double cell_q;               // smallest coordinate spacing (landing tolerance)
};

namespace qsl {

// Where the seeds of a tracing launch come from.
enum SeedKind { SEEDS_ARRAY = 0, SEEDS_PLANE = 1, SEEDS_VOLUME = 2, SEEDS_KEYS2 = 3, SEEDS_KEYS3 = 4 };

struct SeedSource {
  int kind;
  int bits;                 // Hilbert bits per axis (SEEDS_KEYS*)
  int n[3];                 // plane: (nu, nv, 1); volume and keys: lattice extent
  double c[3], u[3], v[3];  // plane: centre + axes; volume/keys3: lo (c) and hi (u)
  double inv_n[3];          // 1 / n[a] (filled where a launch item is made)
  const double* xyz;        // SEEDS_ARRAY: S x 3
  const uint64_t* keys;     // SEEDS_KEYS*: Hilbert keys
};

// Outputs of the assembly step (each optional).
struct LineOutputs {
  qsl_line* lines;
  float* q;
  float* length;
  uint8_t* faces;
  uint8_t* status;
  int q_form;
  int skip_open;
  int retraced;          // set QSL_FLAG_RETRACED on written seeds
};

struct DeviceStats {
  unsigned long long stage_evals, accepted, rejected, landing, lines, timeouts;
};

// Resolved tracing parameters (domain units).
struct TraceConfig {
  double lo[3], hi[3];
  double max_len;
  double cell;
  double tol_abs, tol_rel;
  double h_init, h_max, h_min, euler_h;
  double land_tol;       // domain units
  long long max_steps;
  int integrator;
  int length_only;
  unsigned long long timeout_ns;  // device watchdog per warp (%globaltimer), 0 = none
  int interp_order;  // 1, 2 or 3
  int geom;          // QSL_GEOM_CARTESIAN or QSL_GEOM_SPHERICAL
};

// Stream-ordered allocation from the library's own memory pool on the current
// device (created on first use, release threshold unlimited: freed blocks stay
// cached for the next call instead of going back to the driver at every
// synchronisation). Free with cudaFreeAsync.
cudaError_t alloc_async(void** p, size_t bytes, cudaStream_t s);

struct LaunchShape {
  int warps_per_block;
  int blocks_per_sm;
  int refill_min;
  int line_lanes;  // cell-wise tracer: 1 or 3 lanes per line, 0 = auto
};

// Runs the tracer over `n_seeds` seeds of `src` (n_seeds may live on the
// device: `n_seeds_dev` != nullptr overrides n_seeds as an upper bound), then
// assembles Q/FLL into `out`. Precision: 0 = FP32 trace, 1 = FP64 trace.
// ev (optional): two events recorded around the tracer kernel. index
// (optional, device): launch seed j traces seed index[j] (FP64 retrace lists).
// scratch (optional, device): 256 + end_record_bytes(precision) * 2 * n_seeds
// bytes of caller memory; allocated per call when null.
int trace_and_assemble(const qsl_field* f, const SeedSource& src, int64_t n_seeds, const int64_t* n_seeds_dev,
                       const TraceConfig& cfg, int precision, const LaunchShape& shape, const LineOutputs& out,
                       cudaStream_t stream, DeviceStats* stats_dev, cudaEvent_t* ev, const int64_t* index = nullptr,
                       void* scratch = nullptr);
size_t end_record_bytes(int precision);

// Selects seeds whose chosen Q exceeds `threshold` (or is not finite while
// L is) into `index` (device), count into count_dev (device).
int select_retrace(const SeedSource& src, int64_t n_seeds, const LineOutputs& out, double threshold,
                   int64_t* index, int64_t* count_dev, cudaStream_t stream);

void resolve_config(const qsl_field* f, const qsl_opts* o, TraceConfig* cfg);
int validate_opts(const qsl_field* f, const qsl_opts* o);
int default_shape(const qsl_opts* o, int tangent, int precision, LaunchShape* s);

}  // namespace qsl
