// Field-line and tangent-space tracer (Sec. "Algorithm" of arXiv:1609.00724)
// for sm_103a.
//
// Work unit = one direction of one seed (unit 2j: forward to lambda_F, unit
// 2j+1: backward to lambda_B), so the two halves of a line are load-balanced
// independently. Each warp is persistent: its 32 lanes trace 32 units, and
// lanes whose unit ends take the next units from a global queue (one atomic
// per warp refill), so uneven line lengths do not idle the warp. Every loop
// iteration performs exactly one Cash-Karp step evaluation (6 interpolations
// of B and grad B) per busy lane; accepting/rejecting, face landing and
// queue refill are per-lane bookkeeping around that common step.
//
// The field is a packed float4 (double4 for FP64) vertex array read through
// the read-only cache; consecutive units are spatially adjacent seeds, so the
// lanes of a warp start on neighbouring cells.
//
// After the trace, one thread per seed reads both ends and assembles Q in
// FP64 (Eq. finalQ and its footpoint/determinant forms).
#include <cstdio>
#include <type_traits>

#include "hilbert_dev.cuh"
#include "qsl_internal.cuh"

namespace qsl {
namespace {

constexpr int NO_FACE = 255;
constexpr int ST_RUNNING = -1;

// Cash & Karp (1990) embedded 5(4) coefficients (the stepper of Sec.
// "Integration methods").
constexpr double A21 = 1.0 / 5.0;
constexpr double A31 = 3.0 / 40.0, A32 = 9.0 / 40.0;
constexpr double A41 = 3.0 / 10.0, A42 = -9.0 / 10.0, A43 = 6.0 / 5.0;
constexpr double A51 = -11.0 / 54.0, A52 = 5.0 / 2.0, A53 = -70.0 / 27.0, A54 = 35.0 / 27.0;
constexpr double A61 = 1631.0 / 55296.0, A62 = 175.0 / 512.0, A63 = 575.0 / 13824.0, A64 = 44275.0 / 110592.0,
                 A65 = 253.0 / 4096.0;
constexpr double B1 = 37.0 / 378.0, B3 = 250.0 / 621.0, B4 = 125.0 / 594.0, B6 = 512.0 / 1771.0;
constexpr double E1 = 37.0 / 378.0 - 2825.0 / 27648.0, E3 = 250.0 / 621.0 - 18575.0 / 48384.0,
                 E4 = 125.0 / 594.0 - 13525.0 / 55296.0, E5 = -277.0 / 14336.0, E6 = 512.0 / 1771.0 - 0.25;

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double4_32a ldg4(const double4_32a* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1);
  double4_32a r;
  r.x = a.x;
  r.y = a.y;
  r.z = b.x;
  r.w = b.y;
  return r;
}

// ------------------------------------------------------------ interpolation
template <class R>
struct Interp {
  R b[3];     // interpolated rhs of Eq. fl
  R g[3][3];  // g[i][j] = d b_i / d x_j (Eq. dev)
  R m;        // |B|
};

template <class R>
__device__ __forceinline__ void locate_uniform(R x, R org, R inv_h, int n, int& i, R& u) {
  R f = (x - org) * inv_h;
  R fc = fmin(fmax(f, R(0)), R(n - 2));
  i = (int)floor(fc);
  if (i > n - 2) i = n - 2;
  u = f - R(i);
}

template <class R, class S>
__device__ __forceinline__ void locate_axis(const S* __restrict__ c, R x, int n, int& i, R& u, R& inv_h) {
  if (!(x > R(c[0]))) {
    i = 0;
  } else if (x >= R(c[n - 1])) {
    i = n - 2;
  } else {
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
      int mid = (lo + hi) >> 1;
      if (R(c[mid]) <= x) lo = mid; else hi = mid;
    }
    i = lo;
  }
  R c0 = R(c[i]), c1 = R(c[i + 1]);
  inv_h = R(1) / (c1 - c0);
  u = (x - c0) * inv_h;
}

// Fast power and division for the step-size controller (FP32 uses the
// hardware approximations; the controller is a heuristic either way).
__device__ __forceinline__ float cpow(float a, float e) { return __powf(a, e); }
__device__ __forceinline__ double cpow(double a, double e) { return pow(a, e); }
__device__ __forceinline__ float cdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double cdiv(double a, double b) { return a / b; }

// One component of the trilinear interpolant (Eq. interp with the trilinear
// kernels) and its derivatives in the local coordinates (u, v, w).
template <class R>
__device__ __forceinline__ void tri1(R v000, R v100, R v010, R v110, R v001, R v101, R v011, R v111, R u, R v,
                                     R w, R& val, R& du, R& dv, R& dw) {
  R e00 = v100 - v000, e10 = v110 - v010, e01 = v101 - v001, e11 = v111 - v011;
  R a00 = fma(u, e00, v000), a10 = fma(u, e10, v010), a01 = fma(u, e01, v001), a11 = fma(u, e11, v011);
  R d0 = fma(v, e10 - e00, e00), d1 = fma(v, e11 - e01, e01);
  du = fma(w, d1 - d0, d0);
  R f0 = a10 - a00, f1 = a11 - a01;
  R b0 = fma(v, f0, a00), b1 = fma(v, f1, a01);
  dv = fma(w, f1 - f0, f0);
  dw = b1 - b0;
  val = fma(w, dw, b0);
}

template <class R>
__device__ __forceinline__ R tri0(R v000, R v100, R v010, R v110, R v001, R v101, R v011, R v111, R u, R v, R w) {
  R a00 = fma(u, v100 - v000, v000), a10 = fma(u, v110 - v010, v010), a01 = fma(u, v101 - v001, v001),
    a11 = fma(u, v111 - v011, v011);
  R b0 = fma(v, a10 - a00, a00), b1 = fma(v, a11 - a01, a01);
  return fma(w, b1 - b0, b0);
}

// Taps of the higher-order kernels along one axis for a point in cell c at
// fraction u (Sec. "Interpolation schemes"; the cited methods, restated):
// order 3, Keys cubic convolution (a = -1/2) on vertices c-1..c+2; order 2,
// Dodgson's interpolating quadratic on the vertex m nearest the point and its
// two neighbours. w: weights, g: d w / d u; vertices clamped to [0, n-1].
// Returns the number of taps (4 or 3; a fourth tap of weight 0 pads order 2).
template <class R>
__device__ __forceinline__ int ho_taps(int order, int c, R u, int n, int* idx, R* w, R* g) {
  if (order == 3) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const R s = u - R(k - 1), a = fabs(s), sg = s < R(0) ? R(-1) : R(1);
      if (a <= R(1)) {
        w[k] = (R(1.5) * a - R(2.5)) * a * a + R(1);
        g[k] = sg * (R(4.5) * a - R(5)) * a;
      } else if (a < R(2)) {
        w[k] = ((R(-0.5) * a + R(2.5)) * a - R(4)) * a + R(2);
        g[k] = sg * ((R(-1.5) * a + R(5)) * a - R(4));
      } else {
        w[k] = R(0);
        g[k] = R(0);
      }
      idx[k] = min(max(c - 1 + k, 0), n - 1);
    }
    return 4;
  }
  const int m = c + (u >= R(0.5) ? 1 : 0);
  const R t = u - R(m - c);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R s = t - R(k - 1), a = fabs(s), sg = s < R(0) ? R(-1) : R(1);
    if (a <= R(0.5)) {
      w[k] = R(1) - R(2) * s * s;
      g[k] = R(-4) * s;
    } else if (a <= R(1.5)) {
      w[k] = (a - R(2.5)) * a + R(1.5);
      g[k] = sg * (R(2) * a - R(2.5));
    } else {
      w[k] = R(0);
      g[k] = R(0);
    }
    idx[k] = min(max(m - 1 + k, 0), n - 1);
  }
  w[3] = R(0);
  g[3] = R(0);
  idx[3] = idx[2];
  return 3;
}

// Value (4 stored components) and local-coordinate gradient of the
// higher-order interpolant: separable sums over the K^3 stencil vertices, K
// known at compile time so that the taps and the sums stay in registers.
template <class R, class S, bool GRAD, int K>
__device__ __forceinline__ void ho_sum_k(const FieldView<S>& F, const int* ci, const R* uu, R* val4, R (*d)[3]) {
  int ix[4], iy[4], iz[4];
  R wx[4], wy[4], wz[4], gx[4], gy[4], gz[4];
  ho_taps<R>(F.order, ci[0], uu[0], F.n[0], ix, wx, gx);
  ho_taps<R>(F.order, ci[1], uu[1], F.n[1], iy, wy, gy);
  ho_taps<R>(F.order, ci[2], uu[2], F.n[2], iz, wz, gz);
  typedef typename V4<S>::type V;
  const size_t sy = (size_t)F.n[0], sz = (size_t)F.n[0] * (size_t)F.n[1];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    val4[c] = R(0);
    if (GRAD && c < 3) d[c][0] = d[c][1] = d[c][2] = R(0);
  }
#pragma unroll 1
  for (int kz = 0; kz < K; ++kz) {
    // the z tap of this pass by selects (a rolled loop would index the arrays in local memory)
    const int izk = kz == 0 ? iz[0] : (kz == 1 ? iz[1] : (kz == 2 ? iz[2] : iz[3]));
    const R wzk = kz == 0 ? wz[0] : (kz == 1 ? wz[1] : (kz == 2 ? wz[2] : wz[3]));
    const R gzk = kz == 0 ? gz[0] : (kz == 1 ? gz[1] : (kz == 2 ? gz[2] : gz[3]));
#pragma unroll
    for (int ky = 0; ky < K; ++ky) {
      const size_t row = (size_t)izk * sz + (size_t)iy[ky] * sy;
      const R wyz = wy[ky] * wzk, gyz = gy[ky] * wzk, wgz = wy[ky] * gzk;
#pragma unroll
      for (int kx = 0; kx < K; ++kx) {
        const V q = ldg4(F.v + row + ix[kx]);
        const R f = wx[kx] * wyz;
        const R comp[4] = {R(q.x), R(q.y), R(q.z), R(q.w)};
#pragma unroll
        for (int c = 0; c < 4; ++c) val4[c] = fma(comp[c], f, val4[c]);
        if (GRAD) {
          const R fx = gx[kx] * wyz, fy = wx[kx] * gyz, fz = wx[kx] * wgz;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            d[c][0] = fma(comp[c], fx, d[c][0]);
            d[c][1] = fma(comp[c], fy, d[c][1]);
            d[c][2] = fma(comp[c], fz, d[c][2]);
          }
        }
      }
    }
  }
}

template <class R, class S, bool GRAD>
__device__ __forceinline__ void ho_sum(const FieldView<S>& F, const int* ci, const R* uu, R* val4, R (*d)[3]) {
  if (F.order == 3)
    ho_sum_k<R, S, GRAD, 4>(F, ci, uu, val4, d);
  else
    ho_sum_k<R, S, GRAD, 3>(F, ci, uu, val4, d);
}

// Interpolated b, grad b and |B| at a point. Storage type S (float/double),
// arithmetic R. Global frame (LOC = false): (x0, x1, x2) in domain units.
// Local frame (LOC = true, uniform grids): the point is vertex `ic` plus
// (x0, x1, x2) in cell units, so the cell and its local coordinates come from
// small exact numbers instead of a subtraction of nearly equal coordinates.
// HO = false compiles the trilinear path only (the cell-wise kernels, which
// are trilinear by construction).
template <class R, class S, bool GRAD, bool MAG, bool LOC = false, bool HO = true>
__device__ __forceinline__ void interp(const FieldView<S>& F, R x0, R x1, R x2, Interp<R>& I,
                                       const int* ic = nullptr) {
  int ci[3];
  R uu[3], sc[3];
  R xs[3] = {x0, x1, x2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (LOC) {
      R lim = R(F.n[a]);
      R fl = floor(fmin(fmax(xs[a], -lim), lim));
      int i = ic[a] + (int)fl;
      i = min(max(i, 0), F.n[a] - 2);
      uu[a] = xs[a] - R(i - ic[a]);
      ci[a] = i;
      sc[a] = R(F.inv_h[a]);
    } else if (F.uniform) {
      locate_uniform<R>(xs[a], R(F.org[a]), R(F.inv_h[a]), F.n[a], ci[a], uu[a]);
      sc[a] = R(F.inv_h[a]);
    } else {
      locate_axis<R, S>(F.axis[a], xs[a], F.n[a], ci[a], uu[a], sc[a]);
    }
  }
  R val[3], d[3][3];
  if (HO && F.order > 1) {
    R v4[4];
    ho_sum<R, S, GRAD>(F, ci, uu, v4, d);
    val[0] = v4[0];
    val[1] = v4[1];
    val[2] = v4[2];
    if (MAG || F.raw) I.m = v4[3];
  } else {
  typedef typename V4<S>::type V;
  const size_t sy = (size_t)F.n[0], sz = (size_t)F.n[0] * (size_t)F.n[1];
  const V* p = F.v + (size_t)ci[2] * sz + (size_t)ci[1] * sy + (size_t)ci[0];
  V q000 = ldg4(p), q100 = ldg4(p + 1), q010 = ldg4(p + sy), q110 = ldg4(p + sy + 1);
  V q001 = ldg4(p + sz), q101 = ldg4(p + sz + 1), q011 = ldg4(p + sz + sy), q111 = ldg4(p + sz + sy + 1);
  R u = uu[0], v = uu[1], w = uu[2];
#define QSL_TRI(C, K)                                                                                    \
  if (GRAD) {                                                                                            \
    tri1<R>(R(q000.C), R(q100.C), R(q010.C), R(q110.C), R(q001.C), R(q101.C), R(q011.C), R(q111.C), u, v, \
            w, val[K], d[K][0], d[K][1], d[K][2]);                                                       \
  } else {                                                                                               \
    val[K] = tri0<R>(R(q000.C), R(q100.C), R(q010.C), R(q110.C), R(q001.C), R(q101.C), R(q011.C),        \
                     R(q111.C), u, v, w);                                                                \
  }
  QSL_TRI(x, 0)
  QSL_TRI(y, 1)
  QSL_TRI(z, 2)
#undef QSL_TRI
  if (MAG || F.raw) {
    I.m = tri0<R>(R(q000.w), R(q100.w), R(q010.w), R(q110.w), R(q001.w), R(q101.w), R(q011.w), R(q111.w), u,
                  v, w);
  }
  }
  if (GRAD) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) d[i][j] *= sc[j];
  }
  if (!F.raw) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      I.b[i] = val[i];
      if (GRAD)
#pragma unroll
        for (int j = 0; j < 3; ++j) I.g[i][j] = d[i][j];
    }
  } else {
    // interpolate B, normalise at the point: b = B/|B|,
    // d b_i/d x_j = (dB_i/dx_j - b_i sum_k b_k dB_k/dx_j)/|B|
    R m2 = val[0] * val[0] + val[1] * val[1] + val[2] * val[2];
    R m = sqrt(m2);
    if (MAG) I.m = m;
    R rm = (m > R(0)) ? R(1) / m : R(0);
    R bh[3] = {val[0] * rm, val[1] * rm, val[2] * rm};
#pragma unroll
    for (int i = 0; i < 3; ++i) I.b[i] = bh[i];
    if (GRAD) {
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        R t = bh[0] * d[0][j] + bh[1] * d[1][j] + bh[2] * d[2][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) I.g[i][j] = (d[i][j] - bh[i] * t) * rm;
      }
    }
  }
}

// Spherical coordinates of the local-frame point vertex ic + y (cell units).
template <class R, class S>
__device__ __forceinline__ void sph_point(const FieldView<S>& F, const R* y, const int* ic, R* theta, R* r) {
  *theta = R(F.org[1]) + (R(ic[1]) + y[1]) / R(F.inv_h[1]);
  *r = R(F.org[2]) + (R(ic[2]) + y[2]) / R(F.inv_h[2]);
}

// SPH: spherical geometry (local frame): Eq. fl_sph for the position and
// Eq. dev_sph for the coordinate deviations, m_i d(dq_i)/dl = sum_j
// (d b_i / d q_j) dq_j with m = (r cos(theta), r, 1).
template <class R, class S, int NC, bool LOC, bool HO = false, bool SPH = false>
__device__ __forceinline__ void rhs(const FieldView<S>& F, const R* y, R* k, const int* ic) {
  Interp<R> I;
  interp<R, S, NC == 9, false, LOC, HO>(F, y[0], y[1], y[2], I, ic);
  R im[3] = {R(1), R(1), R(1)};
  if (SPH) {
    R th, rr, m[3];
    sph_point<R, S>(F, y, ic, &th, &rr);
    sph_scale<R>(th, rr, m);
    im[0] = R(1) / m[0];
    im[1] = R(1) / m[1];
  }
  if (LOC) {
    k[0] = I.b[0] * im[0] * R(F.inv_h[0]);
    k[1] = I.b[1] * im[1] * R(F.inv_h[1]);
    k[2] = I.b[2] * R(F.inv_h[2]);
  } else {
    k[0] = I.b[0];
    k[1] = I.b[1];
    k[2] = I.b[2];
  }
  if (NC == 9) {
#pragma unroll
    for (int v = 0; v < 2; ++v)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        k[3 + 3 * v + i] =
            (I.g[i][0] * y[3 + 3 * v] + I.g[i][1] * y[4 + 3 * v] + I.g[i][2] * y[5 + 3 * v]) * im[i];
  }
}

// One Cash-Karp step of signed size hh from y: the 5th-order increment dy
// (y_new = y + dy) and the embedded error estimate yerr.
template <class R, class S, int NC, bool LOC, bool HO = false, bool SPH = false>
__device__ __forceinline__ void ck_step(const FieldView<S>& F, const R* y, R hh, R* dy, R* yerr, const int* ic) {
  R k1[NC], k2[NC], k3[NC], k4[NC], k5[NC], k6[NC], t[NC];
  rhs<R, S, NC, LOC, HO, SPH>(F, y, k1, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i) t[i] = fma(hh, R(A21) * k1[i], y[i]);
  rhs<R, S, NC, LOC, HO, SPH>(F, t, k2, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i) t[i] = fma(hh, R(A31) * k1[i] + R(A32) * k2[i], y[i]);
  rhs<R, S, NC, LOC, HO, SPH>(F, t, k3, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i) t[i] = fma(hh, R(A41) * k1[i] + R(A42) * k2[i] + R(A43) * k3[i], y[i]);
  rhs<R, S, NC, LOC, HO, SPH>(F, t, k4, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i)
    t[i] = fma(hh, R(A51) * k1[i] + R(A52) * k2[i] + R(A53) * k3[i] + R(A54) * k4[i], y[i]);
  rhs<R, S, NC, LOC, HO, SPH>(F, t, k5, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i)
    t[i] = fma(hh, R(A61) * k1[i] + R(A62) * k2[i] + R(A63) * k3[i] + R(A64) * k4[i] + R(A65) * k5[i], y[i]);
  rhs<R, S, NC, LOC, HO, SPH>(F, t, k6, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    dy[i] = hh * (R(B1) * k1[i] + R(B3) * k3[i] + R(B4) * k4[i] + R(B6) * k6[i]);
    yerr[i] = hh * (R(E1) * k1[i] + R(E3) * k3[i] + R(E4) * k4[i] + R(E5) * k5[i] + R(E6) * k6[i]);
  }
}

template <class R, class S, int NC, bool LOC, bool HO = false, bool SPH = false>
__device__ __forceinline__ void euler_step(const FieldView<S>& F, const R* y, R hh, R* dy, R* yerr,
                                           const int* ic) {
  R k[NC];
  rhs<R, S, NC, LOC, HO, SPH>(F, y, k, ic);
#pragma unroll
  for (int i = 0; i < NC; ++i) {
    dy[i] = hh * k[i];
    yerr[i] = R(0);
  }
}

// ------------------------------------------------------------ seeds
__device__ __forceinline__ void seed_position(const SeedSource& s, int64_t g, double* x) {
  switch (s.kind) {
    case SEEDS_ARRAY:
      x[0] = s.xyz[3 * g];
      x[1] = s.xyz[3 * g + 1];
      x[2] = s.xyz[3 * g + 2];
      break;
    case SEEDS_PLANE: {
      int64_t i = g % s.n[0], j = g / s.n[0];
      double a = (i + 0.5) * s.inv_n[0] - 0.5, b = (j + 0.5) * s.inv_n[1] - 0.5;
      for (int k = 0; k < 3; ++k) x[k] = s.c[k] + a * s.u[k] + b * s.v[k];
      break;
    }
    case SEEDS_VOLUME: {
      int64_t i = g % s.n[0], r = g / s.n[0];
      int64_t j = r % s.n[1], k = r / s.n[1];
      int64_t id[3] = {i, j, k};
      for (int a = 0; a < 3; ++a) x[a] = s.c[a] + (id[a] + 0.5) * s.inv_n[a] * (s.u[a] - s.c[a]);
      break;
    }
    default:
      break;
  }
}

__device__ __forceinline__ void seed_of(const SeedSource& s, int64_t gi, double* x) {
  if (s.kind == SEEDS_KEYS2 || s.kind == SEEDS_KEYS3) {
    int nd = (s.kind == SEEDS_KEYS2) ? 2 : 3;
    uint32_t c[3] = {0, 0, 0};
    hilbert_coords_dev(s.keys[gi], nd, s.bits, c);
    if (nd == 2) {
      double a = (c[0] + 0.5) * s.inv_n[0] - 0.5, b = (c[1] + 0.5) * s.inv_n[1] - 0.5;
      for (int k = 0; k < 3; ++k) x[k] = s.c[k] + a * s.u[k] + b * s.v[k];
    } else {
      for (int a = 0; a < 3; ++a) x[a] = s.c[a] + (c[a] + 0.5) * s.inv_n[a] * (s.u[a] - s.c[a]);
    }
    return;
  }
  seed_position(s, gi, x);
}

// ------------------------------------------------------------ tracer kernel
template <class R>
struct EndRec {
  R x[3], d1[3], d2[3];
  R mu;
  int32_t face, status, steps, pad;
};

// One problem of a launch: a field, its tracing domain and step scales, and
// where its seeds come from. Single-problem launches carry one inline item;
// batch launches (many fields and cuts in one persistent launch) a table.
template <class R>
struct Item {
  FieldView<R> F;
  SeedSource src;
  R lo[3], hi[3];              // domain bounds: domain units (global frame) or grid-index units (local frame)
  double lo_d[3], hi_d[3];     // domain bounds in domain units
  R max_len, h_init, h_max, h_min, euler_h, land_tol;  // domain units
  double org_d[3], h_d[3], inv_h_d[3];  // uniform grids: first vertex, spacing, 1 / spacing (FP64)
  int64_t seed_start;          // global id of the item's first seed (outputs are concatenated in item order)
};

template <class R>
struct TraceParams {
  Item<R> item0;               // the problem of a single-problem launch
  const Item<R>* items;        // batch launches: device table sorted by seed_start, else nullptr
  int n_items;
  const int64_t* index;        // optional: unit seed j -> global seed id index[j] (FP64 retrace lists)
  int64_t n_units;             // 2 x seeds
  const int64_t* n_seeds_dev;  // optional device count of seeds
  EndRec<R>* ends;
  unsigned long long* head;
  DeviceStats* stats;
  R tol_abs, tol_rel;
  long long max_steps;
  int euler;
  int refill_min;
  unsigned long long timeout_ns;  // per-warp watchdog, 0 = none
  int* timeout_flag;
};

// Problem and seed of launch seed j: global id, item, position.
template <class R>
__device__ __forceinline__ const Item<R>* resolve_seed(const TraceParams<R>& P, int64_t j, int64_t* g, double* x) {
  int64_t s = P.index ? P.index[j] : j;
  const Item<R>* E = &P.item0;
  if (P.items) {
    int lo = 0, hi = P.n_items - 1;  // last item with seed_start <= s
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (P.items[mid].seed_start <= s) lo = mid; else hi = mid - 1;
    }
    E = &P.items[lo];
  }
  *g = s;
  seed_of(E->src, s - E->seed_start, x);
  return E;
}

// Outward signed distance of the point from face f: global frame, x in domain
// units; local frame, the point is vertex ic + x in cell units and lo/hi are
// grid-index coordinates (bound - ic is exact for grid-aligned domains).
// The distance is evaluated in "delta form" for the point y + d:
// (bound - y) - d, where bound - y is exact near the face, so its precision
// follows the step increment d rather than the coordinate (this keeps the
// landed lambda accurate for lines that graze the face).
template <class R, bool LOC>
__device__ __forceinline__ R face_g(const R* lo, const R* hi, const int* ic, int f, const R* y, const R* d) {
  int a = f >> 1;
  R bound = (f & 1) ? hi[a] : lo[a];
  if (LOC) bound -= R(ic[a]);
  R r = bound - y[a];
  R dd = d ? d[a] : R(0);
  return (f & 1) ? (dd - r) : (r - dd);
}

// face_g for a face id known only at run time: the axis components are
// picked by selects, so that the arrays stay in registers.
template <class R, bool LOC>
__device__ __forceinline__ R face_gs(const R* lo, const R* hi, const int* ic, int f, const R* y, const R* d) {
  const int a = f >> 1;
  const bool up = (f & 1) != 0;
  R bound = up ? (a == 0 ? hi[0] : (a == 1 ? hi[1] : hi[2])) : (a == 0 ? lo[0] : (a == 1 ? lo[1] : lo[2]));
  if (LOC) bound -= R(a == 0 ? ic[0] : (a == 1 ? ic[1] : ic[2]));
  const R r = bound - (a == 0 ? y[0] : (a == 1 ? y[1] : y[2]));
  const R dd = d ? (a == 0 ? d[0] : (a == 1 ? d[1] : d[2])) : R(0);
  return up ? (dd - r) : (r - dd);
}

// Exit face along the chord y -> y + d: the smallest crossing fraction,
// lowest face id on ties.
template <class R, bool LOC>
__device__ __forceinline__ int chord_face(const R* lo, const R* hi, const int* ic, const R* y, const R* d) {
  int face = -1;
  R tb = R(0);
#pragma unroll
  for (int f = 0; f < 6; ++f) {
    R g1 = face_g<R, LOC>(lo, hi, ic, f, y, d);
    if (g1 > R(0)) {
      R g0 = face_g<R, LOC>(lo, hi, ic, f, y, (const R*)nullptr);
      R t = g0 / (g0 - g1);
      if (face < 0 || t < tb) {
        face = f;
        tb = t;
      }
    }
  }
  return face < 0 ? 0 : face;
}

template <class R>
__device__ __forceinline__ R eps_of();
template <>
__device__ __forceinline__ float eps_of<float>() { return 1.1920928955078125e-07f; }
template <>
__device__ __forceinline__ double eps_of<double>() { return 2.220446049250313e-16; }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class R, int NC, bool LOC>
__device__ __forceinline__ void write_end(const TraceParams<R>& P, const Item<R>* E, int64_t unit, const R* y,
                                          const int* ic, R mu, int face, int status, int steps) {
  EndRec<R>& e = P.ends[unit];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (LOC)
      e.x[a] = (R)(E->org_d[a] + ((double)ic[a] + (double)y[a]) * E->h_d[a]);
    else
      e.x[a] = y[a];
  }
  if (status == QSL_LINE_OK && face != NO_FACE) {
    int a = face >> 1;
    e.x[a] = (R)((face & 1) ? E->hi_d[a] : E->lo_d[a]);  // exactly on the face
  }
  if (NC == 9)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      e.d1[i] = y[3 + i];
      e.d2[i] = y[6 + i];
    }
  e.mu = mu;
  e.face = (status == QSL_LINE_OK) ? face : NO_FACE;
  e.status = status;
  e.steps = steps;
}

// HO: higher-order interpolation (Sec. "Interpolation schemes"; uniform grids,
// local frame); a separate instantiation so the trilinear one keeps its
// registers.
template <class R, int NC, bool LOC, bool HO = false, bool SPH = false>
__global__ void __launch_bounds__(256) trace_kernel(const __grid_constant__ TraceParams<R> P) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  int64_t total = P.n_units;
  if (P.n_seeds_dev) {
    int64_t c = 2 * (*P.n_seeds_dev);
    total = c < total ? c : total;
  }
  // lanes of each warp that take work: all 32 when the units fill every
  // resident warp, fewer when they do not, so that a launch of few (and
  // typically long) lines spreads them over all warps and a lane's path is not
  // serialised behind the divergent paths of its neighbours
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t per_warp = (total + warps_total - 1) / warps_total;
  const int lanes = per_warp >= 32 ? 32 : (per_warp < 1 ? 1 : (int)per_warp);
  const bool usable = lane < lanes;
  const unsigned umask = lanes == 32 ? FULL : ((1u << lanes) - 1u);
  const int refill_min = P.refill_min < lanes ? P.refill_min : lanes;
  const Item<R>* E = &P.item0;

  bool active = false;
  bool exhausted = false;  // warp-uniform
  int64_t unit = 0;
  R y[NC];
  int ic[3] = {0, 0, 0};   // reference vertex of the local frame
  R mu = 0, muc = 0, h = 0, sgn = 1;
  int steps = 0, phase = 0;
  bool capped = false;
  // face landing state
  R la = 0, lb = 0, lga = 0, lgb = 0, lhm = 0, yh[3] = {0, 0, 0};
  int lface = 0, lside = 0, lit = 0, lround = 0;
  unsigned long long c_stage = 0, c_acc = 0, c_rej = 0, c_land = 0, c_lines = 0;
  int iter = 0;
  bool timed_out = false;
  const unsigned long long t_start = P.timeout_ns ? globaltimer() : 0ull;

  for (;;) {
    // ---- refill idle lanes from the global queue (one atomic per warp)
    if (!exhausted) {
      unsigned need = __ballot_sync(FULL, usable && !active);
      int nneed = __popc(need);
      if (nneed > 0 && (nneed >= refill_min || need == umask)) {
        int leader = __ffs(need) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(P.head, (unsigned long long)nneed);
        base = __shfl_sync(FULL, base, leader);
        if ((int64_t)(base + nneed) >= total) exhausted = true;
        if (usable && !active) {
          int64_t myu = (int64_t)base + __popc(need & lt_mask);
          if (myu < total) {
            unit = myu;
            active = true;
            c_lines += (myu & 1) == 0;
            // ---- initialise this unit
            int64_t g;
            double xd[3];
            E = resolve_seed(P, unit >> 1, &g, xd);
            sgn = (unit & 1) ? R(-1) : R(1);
            if (LOC) {
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                double fa = (xd[a] - E->org_d[a]) * E->inv_h_d[a];
                double fl = floor(fmin(fmax(fa, 0.0), (double)(E->F.n[a] - 2)));
                ic[a] = (int)fl;
                y[a] = (R)(fa - fl);
              }
            } else {
              y[0] = R(xd[0]);
              y[1] = R(xd[1]);
              y[2] = R(xd[2]);
            }
            mu = 0;
            muc = 0;
            steps = 0;
            phase = 0;
            lface = NO_FACE;
            int status = ST_RUNNING;
            bool outside = false;
#pragma unroll
            for (int f = 0; f < 6; ++f)
              if (face_g<R, LOC>(E->lo, E->hi, ic, f, y, (const R*)nullptr) > R(0)) outside = true;
            if (outside || !isfinite(xd[0]) || !isfinite(xd[1]) || !isfinite(xd[2])) {
              status = QSL_LINE_OUTSIDE;
            } else {
              Interp<R> I0;
              interp<R, R, false, false, LOC, HO>(E->F, y[0], y[1], y[2], I0, ic);
              R m0 = sqrt(I0.b[0] * I0.b[0] + I0.b[1] * I0.b[1] + I0.b[2] * I0.b[2]);
              if (!(m0 > R(0))) {
                status = QSL_LINE_NULL;
              } else {
                if (NC == 9) {
                  // Eq. ic: a, b orthonormal and orthogonal to B(x0); reading:
                  // e = axis of the smallest |b0| component (lowest on ties),
                  // a = normalise(e x b0), b = b0 x a.
                  R u0[3] = {I0.b[0] / m0, I0.b[1] / m0, I0.b[2] / m0};
                  int ax = 0;
                  if (fabs(u0[1]) < fabs(u0[ax])) ax = 1;
                  if (fabs(u0[2]) < fabs(u0[ax])) ax = 2;
                  R av[3];
                  if (ax == 0) { av[0] = 0; av[1] = -u0[2]; av[2] = u0[1]; }
                  else if (ax == 1) { av[0] = u0[2]; av[1] = 0; av[2] = -u0[0]; }
                  else { av[0] = -u0[1]; av[1] = u0[0]; av[2] = 0; }
                  R an = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
                  av[0] /= an;
                  av[1] /= an;
                  av[2] /= an;
                  y[3] = av[0];
                  y[4] = av[1];
                  y[5] = av[2];
                  y[6] = u0[1] * av[2] - u0[2] * av[1];
                  y[7] = u0[2] * av[0] - u0[0] * av[2];
                  y[8] = u0[0] * av[1] - u0[1] * av[0];
                  if (SPH) {
                    // physical vectors of the seed's frame to coordinate deviations
                    R th, rr, m[3];
                    sph_point<R, R>(E->F, y, ic, &th, &rr);
                    sph_scale<R>(th, rr, m);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                      y[3 + i] /= m[i];
                      y[6 + i] /= m[i];
                    }
                  }
                }
                // a seed on a face whose field points out of the domain ends
                // this side at once with zero length
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                  if (status == ST_RUNNING && face_g<R, LOC>(E->lo, E->hi, ic, f, y, (const R*)nullptr) == R(0)) {
                    R bn = I0.b[f >> 1] * sgn;
                    R outw = (f & 1) ? bn : -bn;
                    if (outw > R(0)) {
                      status = QSL_LINE_OK;
                      lface = f;
                    }
                  }
                }
              }
            }
            h = P.euler ? E->euler_h : E->h_init;
            if (status != ST_RUNNING) {
              write_end<R, NC, LOC>(P, E, unit, y, ic, R(0), lface, status, 0);
              active = false;
            }
          }
        }
      }
    }
    if (!__any_sync(FULL, active)) {
      if (exhausted) break;
      continue;
    }
    // ---- device watchdog
    if (P.timeout_ns && ((++iter & 63) == 0)) {
      if (globaltimer() - t_start > P.timeout_ns) timed_out = true;
    }
    if (!active) continue;

    int status = ST_RUNNING;
    if (timed_out) status = QSL_LINE_TIMEOUT;
    R hs = lhm;
    if (status == ST_RUNNING && phase == 0) {
      if (steps >= P.max_steps) status = QSL_LINE_MAXSTEPS;
      R room = E->max_len - mu;
      if (status == ST_RUNNING && !(room > R(0))) status = QSL_LINE_MAXLEN;
      R hcap = P.euler ? E->euler_h : E->h_max;
      hs = fmin(h, hcap);
      capped = false;
      if (room <= hs) {
        hs = room;
        capped = true;
      }
    }
    if (status == ST_RUNNING) {
      R dy[NC], yerr[NC];
      if (P.euler) {
        euler_step<R, R, NC, LOC, HO, SPH>(E->F, y, sgn * hs, dy, yerr, ic);
        c_stage += 1;
      } else {
        ck_step<R, R, NC, LOC, HO, SPH>(E->F, y, sgn * hs, dy, yerr, ic);
        c_stage += 6;
      }
      steps += 1;
      if (phase == 0) {
        R err = 0;
        bool finite = true;
        R sm[3] = {R(1), R(1), R(1)}, srr = R(0);
        if (SPH) {
          // spherical: errors and magnitudes as physical lengths, positions
          // against the radius (the distance from the centre)
          R th, rr;
          sph_point<R, R>(E->F, y, ic, &th, &rr);
          sph_scale<R>(th, rr, sm);
          srr = fmax(fabs(rr), fabs(rr + dy[2] / R(E->F.inv_h[2])));
        }
#pragma unroll
        for (int i = 0; i < NC; ++i) {
          R yn = y[i] + dy[i];
          if (!isfinite(yn)) finite = false;
          R e = fabs(yerr[i]), ya = fabs(y[i]), yb = fabs(yn);
          if (SPH) {
            const R mi = sm[i % 3];
            if (i < 3) {
              e *= mi / R(E->F.inv_h[i]);
              ya = yb = srr;
            } else {
              e *= mi;
              ya *= mi;
              yb *= mi;
            }
          } else if (LOC && i < 3) {
            // position error in domain units, scaled by |x| in domain units
            R hh = R(1) / R(E->F.inv_h[i]);
            R base = R(E->F.org[i]) + R(ic[i]) * hh;
            e *= hh;
            ya = fabs(base + y[i] * hh);
            yb = fabs(base + yn * hh);
          }
          R sc = P.tol_abs + P.tol_rel * fmax(ya, yb);
          err = fmax(err, cdiv(e, sc));
        }
        if (!finite) {
          status = QSL_LINE_NONFINITE;
        } else if (!P.euler && err > R(1)) {
          c_rej += 1;
          h = hs * fmax(R(0.2), R(0.9) * cpow(err, R(-0.25)));
          if (h < E->h_min) status = QSL_LINE_STALL;
        } else {
          c_acc += 1;
          bool inside = true;
#pragma unroll
          for (int f = 0; f < 6; ++f)
            if (face_g<R, LOC>(E->lo, E->hi, ic, f, y, dy) > R(0)) inside = false;
          if (inside) {
#pragma unroll
            for (int i = 0; i < NC; ++i) y[i] += dy[i];
            if (LOC) {
              // move the reference vertex with the line (exact shifts)
#pragma unroll
              for (int a = 0; a < 3; ++a) {
                R fl = floor(y[a]);
                int ni = min(max(ic[a] + (int)fl, 0), E->F.n[a] - 2);
                y[a] -= R(ni - ic[a]);
                ic[a] = ni;
              }
            }
            R t1 = hs - muc, t2 = mu + t1;  // compensated sum of the step lengths
            muc = (t2 - mu) - t1;
            mu = t2;
            if (capped) status = QSL_LINE_MAXLEN;
            else if (!P.euler) h = hs * ((err == R(0)) ? R(5) : fmin(R(5), R(0.9) * cpow(err, R(-0.2))));
          } else {
            // leave the domain: land exactly on the exit face
            phase = 1;
            yh[0] = dy[0];
            yh[1] = dy[1];
            yh[2] = dy[2];
            lface = chord_face<R, LOC>(E->lo, E->hi, ic, y, yh);
            la = 0;
            lb = hs;
            lga = face_gs<R, LOC>(E->lo, E->hi, ic, lface, y, (const R*)nullptr);
            lgb = face_gs<R, LOC>(E->lo, E->hi, ic, lface, y, yh);
            lside = 0;
            lit = 0;
            lround = 0;
            lhm = la + (lb - la) * lga / (lga - lgb);
            if (!(lga < R(0))) {
              // the step starts on this face and ends beyond it again (a line
              // curving back out): seek an inside point by halving first
              lside = 2;
              lhm = R(0.5) * lb;
            }
          }
        }
      } else {
        c_land += 1;
        lit += 1;
        R gm = face_gs<R, LOC>(E->lo, E->hi, ic, lface, y, dy);
        // converged when within the landing tolerance or at the resolution of
        // the step increment along the face normal
        R dn = fabs(lface >> 1 == 0 ? dy[0] : (lface >> 1 == 1 ? dy[1] : dy[2]));
        R gtol = fmax(E->land_tol, R(4) * eps_of<R>() * dn);
        if (lside == 2 && lit < 60 && isfinite(gm)) {
          // seeking an inside point below the outside step lb
          if (gm < R(0)) {
            la = lhm;
            lga = gm;
            lside = 0;
            lhm = la + (lb - la) * lga / (lga - lgb);
          } else {
            lb = lhm;
            lgb = gm;
            lhm = R(0.5) * lhm;
          }
        } else if (fabs(gm) <= gtol || lit >= 60 || !isfinite(gm) || !(lb - la > eps_of<R>() * lb)) {
          R worst = R(-1);
#pragma unroll
          for (int f = 0; f < 6; ++f)
            if (f != lface) worst = fmax(worst, face_g<R, LOC>(E->lo, E->hi, ic, f, y, dy));
          if (worst > gtol && lround < 8) {
            // the landed point is outside another face: that face was crossed first
            lround += 1;
            yh[0] = dy[0];
            yh[1] = dy[1];
            yh[2] = dy[2];
            R hi_h = lhm;
            lface = chord_face<R, LOC>(E->lo, E->hi, ic, y, yh);
            la = 0;
            lb = hi_h;
            lga = face_gs<R, LOC>(E->lo, E->hi, ic, lface, y, (const R*)nullptr);
            lgb = face_gs<R, LOC>(E->lo, E->hi, ic, lface, y, yh);
            lside = 0;
            lit = 0;
            lhm = la + (lb - la) * lga / (lga - lgb);
            if (!(lga < R(0))) {
              lside = 2;
              lhm = R(0.5) * lb;
            }
          } else {
#pragma unroll
            for (int i = 0; i < NC; ++i) y[i] += dy[i];
            R t1 = lhm - muc, t2 = mu + t1;
            muc = (t2 - mu) - t1;
            mu = t2;
            status = QSL_LINE_OK;
          }
        } else {
          if (gm > R(0)) {
            lb = lhm;
            lgb = gm;
            if (lside == 1) lga *= R(0.5);
            lside = 1;
          } else {
            la = lhm;
            lga = gm;
            if (lside == -1) lgb *= R(0.5);
            lside = -1;
          }
          lhm = la + (lb - la) * lga / (lga - lgb);
        }
      }
    }
    if (status != ST_RUNNING) {
      write_end<R, NC, LOC>(P, E, unit, y, ic, mu, lface, status, steps);
      active = false;
    }
  }
  // ---- statistics: one atomic per warp and counter
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_stage += __shfl_down_sync(FULL, c_stage, o);
    c_acc += __shfl_down_sync(FULL, c_acc, o);
    c_rej += __shfl_down_sync(FULL, c_rej, o);
    c_land += __shfl_down_sync(FULL, c_land, o);
    c_lines += __shfl_down_sync(FULL, c_lines, o);
  }
  unsigned any_to = __ballot_sync(FULL, timed_out);
  if (lane == 0 && P.stats) {
    atomicAdd(&P.stats->stage_evals, c_stage);
    atomicAdd(&P.stats->accepted, c_acc);
    atomicAdd(&P.stats->rejected, c_rej);
    atomicAdd(&P.stats->landing, c_land);
    atomicAdd(&P.stats->lines, c_lines);
    if (any_to) atomicAdd(&P.stats->timeouts, 1ull);
  }
  if (lane == 0 && any_to && P.timeout_flag) atomicExch(P.timeout_flag, 1);
}

// ------------------------------------------------------------ cell-wise Dormand-Prince tracer
// Dormand & Prince (1980) 5(4) pair with first-same-as-last stage and Hairer's
// 4th-order continuous extension (the paper lets any Boost.odeint stepper
// replace Cash-Karp, Sec. "Integration methods").
constexpr double DA21 = 1.0 / 5.0;
constexpr double DA31 = 3.0 / 40.0, DA32 = 9.0 / 40.0;
constexpr double DA41 = 44.0 / 45.0, DA42 = -56.0 / 15.0, DA43 = 32.0 / 9.0;
constexpr double DA51 = 19372.0 / 6561.0, DA52 = -25360.0 / 2187.0, DA53 = 64448.0 / 6561.0, DA54 = -212.0 / 729.0;
constexpr double DA61 = 9017.0 / 3168.0, DA62 = -355.0 / 33.0, DA63 = 46732.0 / 5247.0, DA64 = 49.0 / 176.0,
                 DA65 = -5103.0 / 18656.0;
constexpr double DB1 = 35.0 / 384.0, DB3 = 500.0 / 1113.0, DB4 = 125.0 / 192.0, DB5 = -2187.0 / 6784.0,
                 DB6 = 11.0 / 84.0;
constexpr double DE1 = 71.0 / 57600.0, DE3 = -71.0 / 16695.0, DE4 = 71.0 / 1920.0, DE5 = -17253.0 / 339200.0,
                 DE6 = 22.0 / 525.0, DE7 = -1.0 / 40.0;
constexpr double DD1 = -12715105075.0 / 11282082432.0, DD3 = 87487479700.0 / 32700410799.0,
                 DD4 = -10690763975.0 / 1880347072.0, DD5 = 701980252875.0 / 199316789632.0,
                 DD6 = -1453857185.0 / 822651844.0, DD7 = 69997945.0 / 29380423.0;

// Component c of (a, b, d) without indexing a local array (which would place
// it in local memory).
template <class R>
__device__ __forceinline__ R sel3(int c, R a, R b, R d) {
  return c == 0 ? a : (c == 1 ? b : d);
}

// Quotient for safeguarded iterations and step-size estimates: the fast
// single-precision division (FP64 keeps the IEEE one).
__device__ __forceinline__ float qdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }


// Increment of the continuous extension at fraction t of the step:
// y(t) - y0 = t (dy + s (bspl + t (c3 + s c4))), s = 1 - t, with
// bspl = h k1 - dy, c3 = dy - h k7 - bspl and c4 = h sum_i D_i k_i.
template <class R>
__device__ __forceinline__ R y_at(R t, R dy, R hk1, R hk7, R c4) {
  R s1 = R(1) - t;
  R bspl = hk1 - dy;
  R c3 = dy - hk7 - bspl;
  return t * (dy + s1 * (bspl + t * (c3 + s1 * c4)));
}

// Right-hand side inside one cell: the 24 corner values (3 components x 8
// corners, corner c = x + 2y + 4z) sit in shared memory with a stride of one
// block; (u, v, w) are the in-cell coordinates (may lie slightly outside
// [0, 1] within a step: the cell's trilinear polynomial is continued).
template <class R, int NC>
__device__ __forceinline__ void cell_rhs(const R* __restrict__ cs, int st, bool raw, R ihx, R ihy, R ihz,
                                         const R* y, R* k) {
  R u = y[0], v = y[1], w = y[2];
  R val[3], d[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R* p = cs + (8 * c) * st;
    tri1<R>(p[0], p[st], p[2 * st], p[3 * st], p[4 * st], p[5 * st], p[6 * st], p[7 * st], u, v, w, val[c], d[c][0],
            d[c][1], d[c][2]);
    d[c][0] *= ihx;
    d[c][1] *= ihy;
    d[c][2] *= ihz;
  }
  R g[3][3];
  if (!raw) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) g[i][j] = d[i][j];
  } else {
    R m = sqrt(val[0] * val[0] + val[1] * val[1] + val[2] * val[2]);
    R rm = (m > R(0)) ? R(1) / m : R(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) val[i] *= rm;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      R t = val[0] * d[0][j] + val[1] * d[1][j] + val[2] * d[2][j];
#pragma unroll
      for (int i = 0; i < 3; ++i) g[i][j] = (d[i][j] - val[i] * t) * rm;
    }
  }
  k[0] = val[0] * ihx;  // position in cell units
  k[1] = val[1] * ihy;
  k[2] = val[2] * ihz;
  if (NC == 9) {
#pragma unroll
    for (int v2 = 0; v2 < 2; ++v2)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        k[3 + 3 * v2 + i] = g[i][0] * y[3 + 3 * v2] + g[i][1] * y[4 + 3 * v2] + g[i][2] * y[5 + 3 * v2];
  }
}

// Lengths only, normalise-first field: the stage derivative of the lane's axis
// is component c of the trilinear interpolant, a polynomial in the in-cell
// coordinates, f = a0 + a1 u + a2 v + a3 w + a4 uv + a5 uw + a6 vw + a7 uvw
// (coefficients from the cell's 8 corner values, scaled by 1/h_c once per
// cell). Nested, it is three dependent FMAs after the shuffles, against the
// differences and interpolations of the corner form.
template <class R>
__device__ __forceinline__ void trilinear_coeffs(const R* cv, R ihc, R* a) {
  a[0] = cv[0] * ihc;
  a[1] = (cv[1] - cv[0]) * ihc;
  a[2] = (cv[2] - cv[0]) * ihc;
  a[3] = (cv[4] - cv[0]) * ihc;
  a[4] = ((cv[3] - cv[1]) - (cv[2] - cv[0])) * ihc;
  a[5] = ((cv[5] - cv[1]) - (cv[4] - cv[0])) * ihc;
  a[6] = ((cv[6] - cv[2]) - (cv[4] - cv[0])) * ihc;
  a[7] = (((cv[7] - cv[6]) - (cv[5] - cv[4])) - ((cv[3] - cv[2]) - (cv[1] - cv[0]))) * ihc;
}

// Right-hand side inside one cell from the coefficients of the cell's
// trilinear polynomials (8 per component c, corner form turned into
// a0 + a1 u + a2 v + a3 w + a4 uv + a5 uw + a6 vw + a7 uvw once per cell entry),
// held in shared memory as two 4-vectors per component with a stride of one
// block (six vector loads per stage, consecutive lanes on consecutive
// 16-byte words). Deviations are carried in
// cell units (du_j = dx_j / h_j). Normalise-first fields: the coefficients of
// component c are pre-scaled by 1/h_c, so the polynomial's value is the
// position derivative in cell units and its gradient in (u, v, w), applied to
// the deviations, their derivative in cell units; no scaling per stage. Raw
// fields (unscaled coefficients of B): b = B/|B| and its gradient
// (I - b b^T) grad B / |B| at the point, then the 1/h_c row scaling.
// Vector of 4 coefficients in shared memory (one 16-byte load per float4).
template <class R>
struct C4 {
  typedef typename V4<R>::type type;
};

template <class R, int NC>
__device__ __forceinline__ void cell_rhs_poly(const typename C4<R>::type* __restrict__ cs, int st, bool raw,
                                              const R* ih, const R* y, R* k) {
  const R u = y[0], v = y[1], w = y[2];
  R val[3], d[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const typename C4<R>::type lo = cs[(2 * c) * st], hi = cs[(2 * c + 1) * st];
    const R a0 = lo.x, a1 = lo.y, a2 = lo.z, a3 = lo.w, a4 = hi.x, a5 = hi.y, a6 = hi.z, a7 = hi.w;
    const R p0 = fma(a1, u, a0), p1 = fma(a4, u, a2), p2 = fma(a5, u, a3), p3 = fma(a7, u, a6);
    const R q1 = fma(p3, v, p2);
    val[c] = fma(q1, w, fma(p1, v, p0));
    if (NC == 9) {
      d[c][0] = fma(fma(a7, v, a5), w, fma(a4, v, a1));
      d[c][1] = fma(p3, w, p1);
      d[c][2] = q1;
    }
  }
  if (!raw) {
#pragma unroll
    for (int c = 0; c < 3; ++c) k[c] = val[c];
    if (NC == 9) {
#pragma unroll
      for (int v2 = 0; v2 < 2; ++v2)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          k[3 + 3 * v2 + i] = fma(d[i][0], y[3 + 3 * v2], fma(d[i][1], y[4 + 3 * v2], d[i][2] * y[5 + 3 * v2]));
    }
  } else {
    const R m = sqrt(val[0] * val[0] + val[1] * val[1] + val[2] * val[2]);
    const R rm = (m > R(0)) ? R(1) / m : R(0);
    R b[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) b[c] = val[c] * rm;
#pragma unroll
    for (int c = 0; c < 3; ++c) k[c] = b[c] * ih[c];
    if (NC == 9) {
      R g[3][3];
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const R t = b[0] * d[0][j] + b[1] * d[1][j] + b[2] * d[2][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) g[i][j] = (d[i][j] - b[i] * t) * rm;
      }
#pragma unroll
      for (int v2 = 0; v2 < 2; ++v2)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          k[3 + 3 * v2 + i] =
              ih[i] * fma(g[i][0], y[3 + 3 * v2], fma(g[i][1], y[4 + 3 * v2], g[i][2] * y[5 + 3 * v2]));
    }
  }
}

// Deviations of a line state from cell units to domain units (before its end
// record is written).
template <class R, int NC>
__device__ __forceinline__ void dev_to_domain(R* y, const R* hh3) {
  if (NC == 9) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      y[3 + i] *= hh3[i];
      y[6 + i] *= hh3[i];
    }
  }
}

template <class R, int NC>
__device__ __forceinline__ void cell_trace(const TraceParams<R>& P) {
  extern __shared__ __align__(32) unsigned char smem_raw[];
  typedef typename C4<R>::type CV;
  const int st = blockDim.x;
  CV* cs = reinterpret_cast<CV*>(smem_raw) + threadIdx.x;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  int64_t total = P.n_units;
  if (P.n_seeds_dev) {
    int64_t c = 2 * (*P.n_seeds_dev);
    total = c < total ? c : total;
  }
  // lanes of each warp that take work: all 32 when the units fill every
  // resident warp, fewer when they do not, so that a launch of few (and
  // typically long) lines spreads them over all warps and a lane's path is not
  // serialised behind the divergent paths of its neighbours
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t per_warp = (total + warps_total - 1) / warps_total;
  const int lanes = per_warp >= 32 ? 32 : (per_warp < 1 ? 1 : (int)per_warp);
  const bool usable = lane < lanes;
  const unsigned umask = lanes == 32 ? FULL : ((1u << lanes) - 1u);
  const int refill_min = P.refill_min < lanes ? P.refill_min : lanes;
  const Item<R>* E = &P.item0;
  R ih[3] = {R(1), R(1), R(1)}, hh3[3] = {R(1), R(1), R(1)};  // spacing of the lane's field
  const R band = R(16) * eps_of<R>();  // tolerance band of internal cell faces (cell units)
  R tiny = R(0);

  bool active = false, exhausted = false, kvalid = false;
  int64_t unit = 0;
  R y[NC], k1[NC];
  int ic[3] = {0, 0, 0};
  R mu = 0, muc = 0, h = 0, sgn = 1;
  int steps = 0, zc = 0;
  unsigned long long c_stage = 0, c_acc = 0, c_rej = 0, c_land = 0, c_lines = 0;
  int iter = 0;
  bool timed_out = false;
  const unsigned long long t_start = P.timeout_ns ? globaltimer() : 0ull;

  for (;;) {
    if (!exhausted) {
      unsigned need = __ballot_sync(FULL, usable && !active);
      int nneed = __popc(need);
      if (nneed > 0 && (nneed >= refill_min || need == umask)) {
        int leader = __ffs(need) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(P.head, (unsigned long long)nneed);
        base = __shfl_sync(FULL, base, leader);
        if ((int64_t)(base + nneed) >= total) exhausted = true;
        if (usable && !active) {
          int64_t myu = (int64_t)base + __popc(need & lt_mask);
          if (myu < total) {
            unit = myu;
            active = true;
            c_lines += (myu & 1) == 0;
            int64_t g;
            double xd[3];
            E = resolve_seed(P, unit >> 1, &g, xd);
            sgn = (unit & 1) ? R(-1) : R(1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              ih[a] = R(E->F.inv_h[a]);
              hh3[a] = R(1) / ih[a];
            }
            tiny = R(1e-4) * E->h_max;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              double fa = (xd[a] - E->org_d[a]) * E->inv_h_d[a];
              double fl = floor(fmin(fmax(fa, 0.0), (double)(E->F.n[a] - 2)));
              ic[a] = (int)fl;
              y[a] = (R)(fa - fl);
            }
            mu = 0;
            muc = 0;
            steps = 0;
            zc = 0;
            kvalid = false;
            int lface = NO_FACE;
            int status = ST_RUNNING;
            bool outside = false;
#pragma unroll
            for (int f = 0; f < 6; ++f)
              if (face_g<R, true>(E->lo, E->hi, ic, f, y, (const R*)nullptr) > R(0)) outside = true;
            if (outside || !isfinite(xd[0]) || !isfinite(xd[1]) || !isfinite(xd[2])) {
              status = QSL_LINE_OUTSIDE;
            } else {
              Interp<R> I0;
              interp<R, R, false, false, true, false>(E->F, y[0], y[1], y[2], I0, ic);
              R m0 = sqrt(I0.b[0] * I0.b[0] + I0.b[1] * I0.b[1] + I0.b[2] * I0.b[2]);
              if (!(m0 > R(0))) {
                status = QSL_LINE_NULL;
              } else {
                if (NC == 9) {
                  // Eq. ic (same construction as the Cash-Karp tracer)
                  R u0[3] = {I0.b[0] / m0, I0.b[1] / m0, I0.b[2] / m0};
                  int ax = 0;
                  if (fabs(u0[1]) < fabs(u0[ax])) ax = 1;
                  if (fabs(u0[2]) < fabs(u0[ax])) ax = 2;
                  R av[3];
                  if (ax == 0) { av[0] = 0; av[1] = -u0[2]; av[2] = u0[1]; }
                  else if (ax == 1) { av[0] = u0[2]; av[1] = 0; av[2] = -u0[0]; }
                  else { av[0] = -u0[1]; av[1] = u0[0]; av[2] = 0; }
                  R an = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
                  av[0] /= an;
                  av[1] /= an;
                  av[2] /= an;
                  y[3] = av[0];
                  y[4] = av[1];
                  y[5] = av[2];
                  y[6] = u0[1] * av[2] - u0[2] * av[1];
                  y[7] = u0[2] * av[0] - u0[0] * av[2];
                  y[8] = u0[0] * av[1] - u0[1] * av[0];
#pragma unroll
                  for (int i = 0; i < 3; ++i) {  // deviations in cell units
                    y[3 + i] *= ih[i];
                    y[6 + i] *= ih[i];
                  }
                }
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                  if (status == ST_RUNNING && face_g<R, true>(E->lo, E->hi, ic, f, y, (const R*)nullptr) == R(0)) {
                    R bn = I0.b[f >> 1] * sgn;
                    R outw = (f & 1) ? bn : -bn;
                    if (outw > R(0)) {
                      status = QSL_LINE_OK;
                      lface = f;
                    }
                  }
                }
              }
            }
            h = E->h_init;
            if (status != ST_RUNNING) {
              dev_to_domain<R, NC>(y, hh3);
              write_end<R, NC, true>(P, E, unit, y, ic, R(0), lface, status, 0);
              active = false;
            }
          }
        }
      }
    }
    if (!__any_sync(FULL, active)) {
      if (exhausted) break;
      continue;
    }
    if (P.timeout_ns && ((++iter & 63) == 0)) {
      if (globaltimer() - t_start > P.timeout_ns) timed_out = true;
    }
    if (!active) continue;

    int status = ST_RUNNING, lface = NO_FACE;
    if (timed_out) status = QSL_LINE_TIMEOUT;
    if (status == ST_RUNNING && steps >= P.max_steps) status = QSL_LINE_MAXSTEPS;
    R room = E->max_len - mu;
    if (status == ST_RUNNING && !(room > R(0))) status = QSL_LINE_MAXLEN;
    if (status == ST_RUNNING) {
      if (!kvalid) {
        // gather the 8 vertices of the current cell once; every stage of the
        // following steps in this cell reads them from shared memory
        typedef typename V4<R>::type V;
        const size_t sy = (size_t)E->F.n[0], sz = (size_t)E->F.n[0] * (size_t)E->F.n[1];
        const V* p = E->F.v + (size_t)ic[2] * sz + (size_t)ic[1] * sy + (size_t)ic[0];
        V q[8];
        q[0] = ldg4(p);
        q[1] = ldg4(p + 1);
        q[2] = ldg4(p + sy);
        q[3] = ldg4(p + sy + 1);
        q[4] = ldg4(p + sz);
        q[5] = ldg4(p + sz + 1);
        q[6] = ldg4(p + sz + sy);
        q[7] = ldg4(p + sz + sy + 1);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          R cv[8], co[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) cv[j] = R(c == 0 ? q[j].x : (c == 1 ? q[j].y : q[j].z));
          trilinear_coeffs<R>(cv, E->F.raw ? R(1) : ih[c], co);
          CV lo, hi;
          lo.x = co[0];
          lo.y = co[1];
          lo.z = co[2];
          lo.w = co[3];
          hi.x = co[4];
          hi.y = co[5];
          hi.z = co[6];
          hi.w = co[7];
          cs[(2 * c) * st] = lo;
          cs[(2 * c + 1) * st] = hi;
        }
        cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, y, k1);
        c_stage += 1;
        kvalid = true;
      }
      // planes of this cell (cell faces, or domain faces where they come first)
      R lo_pl[3], hi_pl[3];
      bool lo_dom[3], hi_dom[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R lr = E->lo[a] - R(ic[a]), hr = E->hi[a] - R(ic[a]);
        lo_dom[a] = lr >= R(0);
        hi_dom[a] = hr <= R(1);
        lo_pl[a] = lo_dom[a] ? lr : R(0);
        hi_pl[a] = hi_dom[a] ? hr : R(1);
      }
      // step: controller size, capped a little beyond the first plane along k1
      R tface = R(1e30);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        R vel = sgn * k1[a];
        if (vel > R(0)) tface = fmin(tface, qdiv(hi_pl[a] - y[a], vel));
        else if (vel < R(0)) tface = fmin(tface, qdiv(lo_pl[a] - y[a], vel));
      }
      R hs = fmin(fmin(h, E->h_max), room);
      bool capped = room <= fmin(h, E->h_max);
      R hf = R(1.25) * fmax(tface, R(0)) + tiny;
      if (hf < hs) {
        hs = hf;
        capped = false;
      }
      R hh = sgn * hs;
      // stage combinations with the step folded into the coefficients; each
      // stage's newest term is the last FMA
      const R c21 = hh * R(DA21), c31 = hh * R(DA31), c32 = hh * R(DA32), c41 = hh * R(DA41), c42 = hh * R(DA42),
              c43 = hh * R(DA43), c51 = hh * R(DA51), c52 = hh * R(DA52), c53 = hh * R(DA53), c54 = hh * R(DA54),
              c61 = hh * R(DA61), c62 = hh * R(DA62), c63 = hh * R(DA63), c64 = hh * R(DA64), c65 = hh * R(DA65);
      const R b1 = hh * R(DB1), b3 = hh * R(DB3), b4 = hh * R(DB4), b5 = hh * R(DB5), b6 = hh * R(DB6);
      R k2[NC], k3[NC], k4[NC], k5[NC], k6[NC], k7[NC], t[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) t[i] = fma(c21, k1[i], y[i]);
      cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, t, k2);
#pragma unroll
      for (int i = 0; i < NC; ++i) t[i] = fma(c32, k2[i], fma(c31, k1[i], y[i]));
      cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, t, k3);
#pragma unroll
      for (int i = 0; i < NC; ++i) t[i] = fma(c43, k3[i], fma(c42, k2[i], fma(c41, k1[i], y[i])));
      cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, t, k4);
#pragma unroll
      for (int i = 0; i < NC; ++i) t[i] = fma(c54, k4[i], fma(c53, k3[i], fma(c52, k2[i], fma(c51, k1[i], y[i]))));
      cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, t, k5);
#pragma unroll
      for (int i = 0; i < NC; ++i)
        t[i] = fma(c65, k5[i], fma(c64, k4[i], fma(c63, k3[i], fma(c62, k2[i], fma(c61, k1[i], y[i])))));
      cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, t, k6);
      R dy[NC];
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        dy[i] = fma(b6, k6[i], fma(b5, k5[i], fma(b4, k4[i], fma(b3, k3[i], b1 * k1[i]))));
        t[i] = y[i] + dy[i];
      }
      cell_rhs_poly<R, NC>(cs, st, E->F.raw, ih, t, k7);
      c_stage += 6;
      steps += 1;
      // the error estimate's and the continuous extension's weights, scaled by the step
      const R e1 = hh * R(DE1), e3 = hh * R(DE3), e4 = hh * R(DE4), e5 = hh * R(DE5), e6 = hh * R(DE6),
              e7 = hh * R(DE7);
      const R w1 = hh * R(DD1), w3 = hh * R(DD3), w4 = hh * R(DD4), w5 = hh * R(DD5), w6 = hh * R(DD6),
              w7 = hh * R(DD7);
      R err = 0;
      bool finite = true;
#pragma unroll
      for (int i = 0; i < NC; ++i) {
        R e = fabs(fma(e7, k7[i], fma(e6, k6[i], fma(e5, k5[i], fma(e4, k4[i], fma(e3, k3[i], e1 * k1[i]))))));
        if (!isfinite(t[i])) finite = false;
        R ya, yb;
        if (i < 3) {
          R base = R(E->F.org[i]) + R(ic[i]) * hh3[i];
          e *= hh3[i];
          ya = fabs(base + y[i] * hh3[i]);
          yb = fabs(base + t[i] * hh3[i]);
        } else {  // deviations, in domain units
          const R hc = hh3[i % 3];
          e *= hc;
          ya = fabs(y[i]) * hc;
          yb = fabs(t[i]) * hc;
        }
        err = fmax(err, cdiv(e, P.tol_abs + P.tol_rel * fmax(ya, yb)));
      }
      if (!finite) {
        status = QSL_LINE_NONFINITE;
      } else if (err > R(1)) {
        c_rej += 1;
        h = hs * fmax(R(0.2), R(0.9) * cpow(err, R(-0.25)));
        if (h < E->h_min) status = QSL_LINE_STALL;
      } else {
        c_acc += 1;
        R hnext = hs * ((err == R(0)) ? R(5) : fmin(R(5), R(0.9) * cpow(err, R(-0.2))));
        // First plane crossed within the step, on the dense output (4th-order
        // continuous extension): for every plane the step ends beyond, the
        // first sign change of dense(t) - plane over t = 1/4, 1/2, 3/4, 1
        // brackets the crossing, which safeguarded Newton then resolves; the
        // earliest crossing wins.
        R th = R(2);
        int ax_c = -1, up_c = 0;
        // planes the step ends beyond (bit 2a: lower plane of axis a, 2a+1: upper)
        unsigned cmask = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if ((lo_pl[a] - y[a]) - dy[a] > (lo_dom[a] ? R(0) : band)) cmask |= 1u << (2 * a);
          if (dy[a] - (hi_pl[a] - y[a]) > (hi_dom[a] ? R(0) : band)) cmask |= 2u << (2 * a);
        }
#pragma unroll 1
        while (cmask) {
          const int pl = __ffs(cmask) - 1;
          cmask &= cmask - 1;
          int a = pl >> 1, up = pl & 1;
          R ya = a == 0 ? y[0] : (a == 1 ? y[1] : y[2]);
          R dya = a == 0 ? dy[0] : (a == 1 ? dy[1] : dy[2]);
          R target = up ? (a == 0 ? hi_pl[0] : (a == 1 ? hi_pl[1] : hi_pl[2]))
                        : (a == 0 ? lo_pl[0] : (a == 1 ? lo_pl[1] : lo_pl[2]));
          R r = target - ya;  // exact near the plane
          R sg = up ? R(1) : R(-1);  // sg * f > 0 beyond the plane
          R k1a = a == 0 ? k1[0] : (a == 1 ? k1[1] : k1[2]);
          R k7a = a == 0 ? k7[0] : (a == 1 ? k7[1] : k7[2]);
          R c4 = fma(w7, k7a, fma(w6, sel3(a, k6[0], k6[1], k6[2]), fma(w5, sel3(a, k5[0], k5[1], k5[2]),
                 fma(w4, sel3(a, k4[0], k4[1], k4[2]), fma(w3, sel3(a, k3[0], k3[1], k3[2]), w1 * k1a)))));
          R bspl = hh * k1a - dya;
          R c3 = dya - hh * k7a - bspl;
          // The offset along the axis is t * P(t) with the cubic
          // P(t) = dya + (1 - t) (bspl + t (c3 + (1 - t) c4)). A step that
          // starts on the plane (r = 0: a seed on a domain face, or the face
          // just entered) has the trivial root t = 0; the crossing sought is
          // the root of P, so P is solved instead (the root t = 0 divided out).
          const bool defl = (r == R(0));
          // bracket the first crossing
          R ta = R(0), tb = R(1);
#pragma unroll
          for (int q = 1; q < 4; ++q) {
            R tq = R(0.25) * R(q);
            R s1 = R(1) - tq;
            R pq = dya + s1 * (bspl + tq * (c3 + s1 * c4));
            R f = defl ? pq : tq * pq - r;
            if (sg * f > R(0) && tb == R(1)) tb = tq;
            else if (tb == R(1)) ta = tq;
          }
          R t = ta + (tb - ta) * R(0.5);
          if (!defl) {
            // chord estimate inside the bracket as the first iterate
            R tl = qdiv(r, dya);
            if (tl > ta && tl < tb) t = tl;
          }
          for (int it = 0; it < 30; ++it) {
            R s1 = R(1) - t;
            R inner = c3 + s1 * c4;
            R mid = bspl + t * inner;
            R pv = dya + s1 * mid;
            R f = defl ? pv : t * pv - r;
            if (fabs(f) <= R(4) * eps_of<R>() * (fabs(r) + fabs(dya)) || !(tb - ta > R(2) * eps_of<R>())) break;
            if (sg * f > R(0)) tb = t;
            else ta = t;
            R dmid = inner - t * c4;
            R dp = s1 * dmid - mid;
            R df = defl ? dp : pv + t * dp;
            R tn = t - qdiv(f, df);
            t = (tn > ta && tn < tb) ? tn : R(0.5) * (ta + tb);
          }
          if (t < th) {
            th = t;
            ax_c = a;
            up_c = up;
          }
        }
        if (ax_c < 0) {
          // the step stays in the cell: accept it; k7 is the next k1
#pragma unroll
          for (int i = 0; i < NC; ++i) {
            y[i] += dy[i];
            k1[i] = k7[i];
          }
          R t1 = hs - muc, t2 = mu + t1;
          muc = (t2 - mu) - t1;
          mu = t2;
          h = hnext;
          zc = 0;
          if (capped) status = QSL_LINE_MAXLEN;
        } else {
          // advance to the plane on the dense output and snap onto it
#pragma unroll
          for (int i = 0; i < NC; ++i)
            y[i] += y_at<R>(th, dy[i], hh * k1[i], hh * k7[i],
                            fma(w7, k7[i], fma(w6, k6[i], fma(w5, k5[i], fma(w4, k4[i], fma(w3, k3[i], w1 * k1[i]))))));
          bool dom = up_c ? sel3(ax_c, hi_dom[0], hi_dom[1], hi_dom[2]) : sel3(ax_c, lo_dom[0], lo_dom[1], lo_dom[2]);
          R target = up_c ? sel3(ax_c, hi_pl[0], hi_pl[1], hi_pl[2]) : sel3(ax_c, lo_pl[0], lo_pl[1], lo_pl[2]);
          if (ax_c == 0) y[0] = target;
          else if (ax_c == 1) y[1] = target;
          else y[2] = target;
          R dl = th * hs;
          R t1 = dl - muc, t2 = mu + t1;
          muc = (t2 - mu) - t1;
          mu = t2;
          c_land += 1;
          if (dom) {
            status = QSL_LINE_OK;
            lface = 2 * ax_c + up_c;
          } else {
            // enter the neighbouring cell
            zc = (dl < tiny) ? zc + 1 : 0;
            int na = sel3(ax_c, ic[0], ic[1], ic[2]) + (up_c ? 1 : -1);
            if (zc > 3 || na < 0 || na > sel3(ax_c, E->F.n[0], E->F.n[1], E->F.n[2]) - 2) {
              // grazing a face back and forth: stay in this cell for one step
              // (the cell's polynomial continued across the face)
              zc = 0;
            } else {
              if (ax_c == 0) ic[0] = na;
              else if (ax_c == 1) ic[1] = na;
              else ic[2] = na;
              if (ax_c == 0) y[0] = up_c ? R(0) : R(1);
              else if (ax_c == 1) y[1] = up_c ? R(0) : R(1);
              else y[2] = up_c ? R(0) : R(1);
              kvalid = false;
            }
            h = fmax(hnext, hs);
          }
        }
      }
    }
    if (status != ST_RUNNING) {
      dev_to_domain<R, NC>(y, hh3);
      write_end<R, NC, true>(P, E, unit, y, ic, mu, lface, status, steps);
      active = false;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_stage += __shfl_down_sync(FULL, c_stage, o);
    c_acc += __shfl_down_sync(FULL, c_acc, o);
    c_rej += __shfl_down_sync(FULL, c_rej, o);
    c_land += __shfl_down_sync(FULL, c_land, o);
    c_lines += __shfl_down_sync(FULL, c_lines, o);
  }
  unsigned any_to = __ballot_sync(FULL, timed_out);
  if (lane == 0 && P.stats) {
    atomicAdd(&P.stats->stage_evals, c_stage);
    atomicAdd(&P.stats->accepted, c_acc);
    atomicAdd(&P.stats->rejected, c_rej);
    atomicAdd(&P.stats->landing, c_land);
    atomicAdd(&P.stats->lines, c_lines);
    if (any_to) atomicAdd(&P.stats->timeouts, 1ull);
  }
  if (lane == 0 && any_to && P.timeout_flag) atomicExch(P.timeout_flag, 1);
}

// The cell-wise kernel. FP32: at most 168 registers, so three blocks of 128
// threads stay resident per SM (the allocation granularity would make 170 a
// two-block kernel); FP64 keeps the compiler's choice (a cap would spill).
template <int NC>
__global__ void __maxnreg__(168) cell_kernel_f32(const __grid_constant__ TraceParams<float> P) {
  cell_trace<float, NC>(P);
}
template <int NC>
__global__ void __launch_bounds__(256) cell_kernel_f64(const __grid_constant__ TraceParams<double> P) {
  cell_trace<double, NC>(P);
}
template <int NC>
inline void (*cell_kernel_fn(float*))(const TraceParams<float>) {
  return cell_kernel_f32<NC>;
}
template <int NC>
inline void (*cell_kernel_fn(double*))(const TraceParams<double>) {
  return cell_kernel_f64<NC>;
}

// ------------------------------------------------------------ cooperative cell-wise tracer
// The cell-wise Dormand-Prince tracer with one line on a group of three lanes.
// Lane c of a group (c = 0, 1, 2) carries axis c of the position and of both
// deviations, interpolates component c of the field (value and gradient row c)
// from the cell's 8 corners held in its registers, and looks for crossings of
// the two planes of axis c; the group exchanges stage inputs with shuffles and
// reduces the error norm and the earliest crossing. A step's dependent chain is
// about a third of the one-lane kernel's, so launches of few (and typically
// long) lines - refinement passes, FP64 retraces - finish sooner. Ten groups
// per warp; lanes 30 and 31 take no work.
template <class R>
__device__ __forceinline__ R gbc(unsigned m, R v, int src) {
  return __shfl_sync(m, v, src);
}



// Stage derivative of the lane's components: k[0] = d(x_c)/dlambda (cell
// units), k[1], k[2] = row c of grad b applied to the two deviations.
template <class R, int NC>
__device__ __forceinline__ void coop_rhs(unsigned gm, int gb, const R* cv, bool raw, const R* ih, R ihc,
                                         const R* y, R* k) {
  R u = gbc(gm, y[0], gb), v = gbc(gm, y[0], gb + 1), w = gbc(gm, y[0], gb + 2);
  R val, d0, d1, d2;
  tri1<R>(cv[0], cv[1], cv[2], cv[3], cv[4], cv[5], cv[6], cv[7], u, v, w, val, d0, d1, d2);
  d0 *= ih[0];
  d1 *= ih[1];
  d2 *= ih[2];
  if (raw) {
    // interpolate B, normalise at the point: grad b = (I - b b^T) grad B / |B|
    R v0 = gbc(gm, val, gb), v1 = gbc(gm, val, gb + 1), v2 = gbc(gm, val, gb + 2);
    R m = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    R rm = (m > R(0)) ? R(1) / m : R(0);
    R nv = val * rm;
    R p0 = nv * d0, p1 = nv * d1, p2 = nv * d2;
    R t0 = gbc(gm, p0, gb) + gbc(gm, p0, gb + 1) + gbc(gm, p0, gb + 2);
    R t1 = gbc(gm, p1, gb) + gbc(gm, p1, gb + 1) + gbc(gm, p1, gb + 2);
    R t2 = gbc(gm, p2, gb) + gbc(gm, p2, gb + 1) + gbc(gm, p2, gb + 2);
    d0 = (d0 - nv * t0) * rm;
    d1 = (d1 - nv * t1) * rm;
    d2 = (d2 - nv * t2) * rm;
    val = nv;
  }
  k[0] = val * ihc;
  if constexpr (NC == 9) {
    R a0 = gbc(gm, y[1], gb), a1 = gbc(gm, y[1], gb + 1), a2 = gbc(gm, y[1], gb + 2);
    R b0 = gbc(gm, y[2], gb), b1 = gbc(gm, y[2], gb + 1), b2 = gbc(gm, y[2], gb + 2);
    k[1] = d0 * a0 + d1 * a1 + d2 * a2;
    k[2] = d0 * b0 + d1 * b1 + d2 * b2;
  }
}

template <class R>
__device__ __forceinline__ R coop_val_poly(unsigned gm, int gb, const R* a, R y0) {
  const R u = gbc(gm, y0, gb), v = gbc(gm, y0, gb + 1), w = gbc(gm, y0, gb + 2);
  const R p0 = fma(a[1], u, a[0]), p1 = fma(a[4], u, a[2]), p2 = fma(a[5], u, a[3]), p3 = fma(a[7], u, a[6]);
  return fma(fma(p3, v, p2), w, fma(p1, v, p0));
}

// The six new stages of one Dormand-Prince step of the lane's components
// (k2..k7; dy = the 5th-order increment, t = y + dy). POLY: stage derivatives
// from the cell polynomial (lengths only, normalise-first field), decided once
// per step so that the six stages form one straight-line sequence.
template <class R, int NC, bool POLY>
__device__ __forceinline__ void coop_stages(unsigned gm, int gb, const R* cv, const R* pc, bool raw, const R* ih,
                                           R ihc, R hh, const R* y, const R* k1, R* k2, R* k3, R* k4, R* k5, R* k6,
                                           R* k7, R* dy, R* t) {
  constexpr int ND = NC / 3;
  auto stage = [&](const R* tt, R* k) {
    if constexpr (POLY) k[0] = coop_val_poly<R>(gm, gb, pc, tt[0]);
    else coop_rhs<R, NC>(gm, gb, cv, raw, ih, ihc, tt, k);
  };
#pragma unroll
  for (int i = 0; i < ND; ++i) t[i] = fma(hh, R(DA21) * k1[i], y[i]);
  stage(t, k2);
#pragma unroll
  for (int i = 0; i < ND; ++i) t[i] = fma(hh, R(DA31) * k1[i] + R(DA32) * k2[i], y[i]);
  stage(t, k3);
#pragma unroll
  for (int i = 0; i < ND; ++i) t[i] = fma(hh, R(DA41) * k1[i] + R(DA42) * k2[i] + R(DA43) * k3[i], y[i]);
  stage(t, k4);
#pragma unroll
  for (int i = 0; i < ND; ++i)
    t[i] = fma(hh, R(DA51) * k1[i] + R(DA52) * k2[i] + R(DA53) * k3[i] + R(DA54) * k4[i], y[i]);
  stage(t, k5);
#pragma unroll
  for (int i = 0; i < ND; ++i)
    t[i] = fma(hh, R(DA61) * k1[i] + R(DA62) * k2[i] + R(DA63) * k3[i] + R(DA64) * k4[i] + R(DA65) * k5[i], y[i]);
  stage(t, k6);
#pragma unroll
  for (int i = 0; i < ND; ++i) {
    dy[i] = hh * (R(DB1) * k1[i] + R(DB3) * k3[i] + R(DB4) * k4[i] + R(DB5) * k5[i] + R(DB6) * k6[i]);
    t[i] = y[i] + dy[i];
  }
  stage(t, k7);
}

// End record of a group: lane c writes axis c, the group's first lane the rest.
template <class R, int NC>
__device__ __forceinline__ void write_end_coop(const TraceParams<R>& P, const Item<R>* E, int64_t unit, int c,
                                               const R* y, int icc, R mu, int face, int status, int steps) {
  EndRec<R>& e = P.ends[unit];
  R xv = (R)(E->org_d[c] + ((double)icc + (double)y[0]) * E->h_d[c]);
  if (status == QSL_LINE_OK && face != NO_FACE && (face >> 1) == c)
    xv = (R)((face & 1) ? E->hi_d[c] : E->lo_d[c]);  // exactly on the face
  e.x[c] = xv;
  if constexpr (NC == 9) {
    e.d1[c] = y[1];
    e.d2[c] = y[2];
  }
  if (c == 0) {
    e.mu = mu;
    e.face = (status == QSL_LINE_OK) ? face : NO_FACE;
    e.status = status;
    e.steps = steps;
  }
}

template <class R, int NC>
__global__ void __launch_bounds__(256) cell_coop_kernel(const __grid_constant__ TraceParams<R> P) {
  constexpr int ND = NC / 3;  // components per lane
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int grp = lane / 3;          // 0..9 (10 for lanes 30, 31)
  const int c = lane - 3 * grp;      // axis of this lane
  const int gb = 3 * grp;            // first lane of the group
  const unsigned gm = grp < 10 ? (7u << gb) : (3u << 30);  // lanes 30, 31 never take work
  int64_t total = P.n_units;
  if (P.n_seeds_dev) {
    int64_t cnt = 2 * (*P.n_seeds_dev);
    total = cnt < total ? cnt : total;
  }
  // groups of each warp that take work (spread over all resident warps when
  // the units do not fill them)
  const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t per_warp = (total + warps_total - 1) / warps_total;
  const int ngroups = per_warp >= 10 ? 10 : (per_warp < 1 ? 1 : (int)per_warp);
  const bool usable = grp < ngroups;
  unsigned lead_mask = 0;
  for (int g = 0; g < ngroups; ++g) lead_mask |= 1u << (3 * g);
  const int refill_min = P.refill_min < ngroups ? P.refill_min : ngroups;
  const Item<R>* E = &P.item0;
  R ih[3] = {R(1), R(1), R(1)};
  R ihc = R(1), hhc = R(1);
  const R band = R(16) * eps_of<R>();
  R tiny = R(0);

  bool active = false, exhausted = false, kvalid = false;
  int64_t unit = 0;
  R y[ND], k1[ND], cv[8];
  R pc[8];             // lengths only, normalise-first field: trilinear_coeffs of the cell
  bool poly = false;   // evaluate the stages on pc
  int ic[3] = {0, 0, 0};
  R mu = 0, muc = 0, h = 0, sgn = 1;
  int steps = 0, zc = 0;
  unsigned long long c_stage = 0, c_acc = 0, c_rej = 0, c_land = 0, c_lines = 0;
  int iter = 0;
  bool timed_out = false;
  const unsigned long long t_start = P.timeout_ns ? globaltimer() : 0ull;
#pragma unroll
  for (int i = 0; i < 8; ++i) cv[i] = R(0);

  for (;;) {
    if (!exhausted) {
      unsigned need = __ballot_sync(FULL, usable && c == 0 && !active);
      int nneed = __popc(need);
      if (nneed > 0 && (nneed >= refill_min || need == lead_mask)) {
        int leader = __ffs(need) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(P.head, (unsigned long long)nneed);
        base = __shfl_sync(FULL, base, leader);
        if ((int64_t)(base + nneed) >= total) exhausted = true;
        if (usable && ((need >> gb) & 1u)) {
          int64_t myu = (int64_t)base + __popc(need & ((1u << gb) - 1u));
          if (myu < total) {
            unit = myu;
            active = true;
            if (c == 0) c_lines += (myu & 1) == 0;
            int64_t g;
            double xd[3];
            E = resolve_seed(P, unit >> 1, &g, xd);
            sgn = (unit & 1) ? R(-1) : R(1);
#pragma unroll
            for (int a = 0; a < 3; ++a) ih[a] = R(E->F.inv_h[a]);
            ihc = sel3(c, ih[0], ih[1], ih[2]);
            hhc = R(1) / ihc;
            poly = NC == 3 && !E->F.raw;
            tiny = R(1e-4) * E->h_max;
            R yf[NC];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              double fa = (xd[a] - E->org_d[a]) * E->inv_h_d[a];
              double fl = floor(fmin(fmax(fa, 0.0), (double)(E->F.n[a] - 2)));
              ic[a] = (int)fl;
              yf[a] = (R)(fa - fl);
            }
            mu = 0;
            muc = 0;
            steps = 0;
            zc = 0;
            kvalid = false;
            int lface = NO_FACE;
            int status = ST_RUNNING;
            bool outside = false;
#pragma unroll
            for (int f = 0; f < 6; ++f)
              if (face_g<R, true>(E->lo, E->hi, ic, f, yf, (const R*)nullptr) > R(0)) outside = true;
            if (outside || !isfinite(xd[0]) || !isfinite(xd[1]) || !isfinite(xd[2])) {
              status = QSL_LINE_OUTSIDE;
            } else {
              Interp<R> I0;
              interp<R, R, false, false, true, false>(E->F, yf[0], yf[1], yf[2], I0, ic);
              R m0 = sqrt(I0.b[0] * I0.b[0] + I0.b[1] * I0.b[1] + I0.b[2] * I0.b[2]);
              if (!(m0 > R(0))) {
                status = QSL_LINE_NULL;
              } else {
                if constexpr (NC == 9) {
                  // Eq. ic (same construction as the other tracers)
                  R u0[3] = {I0.b[0] / m0, I0.b[1] / m0, I0.b[2] / m0};
                  int ax = 0;
                  if (fabs(u0[1]) < fabs(u0[ax])) ax = 1;
                  if (fabs(u0[2]) < fabs(u0[ax])) ax = 2;
                  R av[3];
                  if (ax == 0) { av[0] = 0; av[1] = -u0[2]; av[2] = u0[1]; }
                  else if (ax == 1) { av[0] = u0[2]; av[1] = 0; av[2] = -u0[0]; }
                  else { av[0] = -u0[1]; av[1] = u0[0]; av[2] = 0; }
                  R an = sqrt(av[0] * av[0] + av[1] * av[1] + av[2] * av[2]);
                  av[0] /= an;
                  av[1] /= an;
                  av[2] /= an;
                  yf[3] = av[0];
                  yf[4] = av[1];
                  yf[5] = av[2];
                  yf[6] = u0[1] * av[2] - u0[2] * av[1];
                  yf[7] = u0[2] * av[0] - u0[0] * av[2];
                  yf[8] = u0[0] * av[1] - u0[1] * av[0];
                }
#pragma unroll
                for (int f = 0; f < 6; ++f) {
                  if (status == ST_RUNNING && face_g<R, true>(E->lo, E->hi, ic, f, yf, (const R*)nullptr) == R(0)) {
                    R bn = I0.b[f >> 1] * sgn;
                    R outw = (f & 1) ? bn : -bn;
                    if (outw > R(0)) {
                      status = QSL_LINE_OK;
                      lface = f;
                    }
                  }
                }
              }
            }
#pragma unroll
            for (int i = 0; i < ND; ++i) y[i] = sel3(c, yf[3 * i], yf[3 * i + 1], yf[3 * i + 2]);
            h = E->h_init;
            if (status != ST_RUNNING) {
              write_end_coop<R, NC>(P, E, unit, c, y, sel3(c, ic[0], ic[1], ic[2]), R(0), lface, status, 0);
              active = false;
            }
          }
        }
      }
    }
    if (!__any_sync(FULL, active)) {
      if (exhausted) break;
      continue;
    }
    if (P.timeout_ns && ((++iter & 63) == 0)) {
      // warp-uniform, so that the lanes of a group agree
      if (__any_sync(FULL, globaltimer() - t_start > P.timeout_ns)) timed_out = true;
    }
    if (!active) continue;

    int status = ST_RUNNING, lface = NO_FACE;
    if (timed_out) status = QSL_LINE_TIMEOUT;
    if (status == ST_RUNNING && steps >= P.max_steps) status = QSL_LINE_MAXSTEPS;
    R room = E->max_len - mu;
    if (status == ST_RUNNING && !(room > R(0))) status = QSL_LINE_MAXLEN;
    if (status == ST_RUNNING) {
      if (!kvalid) {
        // component c of the cell's 8 vertices, into registers
        const size_t sy = (size_t)E->F.n[0], sz = (size_t)E->F.n[0] * (size_t)E->F.n[1];
        const R* p = reinterpret_cast<const R*>(E->F.v + (size_t)ic[2] * sz + (size_t)ic[1] * sy + (size_t)ic[0]) + c;
        cv[0] = __ldg(p);
        cv[1] = __ldg(p + 4);
        cv[2] = __ldg(p + 4 * sy);
        cv[3] = __ldg(p + 4 * sy + 4);
        cv[4] = __ldg(p + 4 * sz);
        cv[5] = __ldg(p + 4 * sz + 4);
        cv[6] = __ldg(p + 4 * (sz + sy));
        cv[7] = __ldg(p + 4 * (sz + sy) + 4);
        if constexpr (NC == 3) {
          if (poly) {
            trilinear_coeffs<R>(cv, ihc, pc);
            k1[0] = coop_val_poly<R>(gm, gb, pc, y[0]);
          } else {
            coop_rhs<R, NC>(gm, gb, cv, E->F.raw, ih, ihc, y, k1);
          }
        } else {
          coop_rhs<R, NC>(gm, gb, cv, E->F.raw, ih, ihc, y, k1);
        }
        c_stage += (c == 0);
        kvalid = true;
      }
      // the two planes of axis c (cell faces, or domain faces where they come first)
      const int icc = sel3(c, ic[0], ic[1], ic[2]);
      const R lr = E->lo[c] - R(icc), hr = E->hi[c] - R(icc);
      const bool lo_dom = lr >= R(0), hi_dom = hr <= R(1);
      const R lo_pl = lo_dom ? lr : R(0), hi_pl = hi_dom ? hr : R(1);
      // step: controller size, capped a little beyond the first plane along k1
      R tf = R(1e30);
      const R vel = sgn * k1[0];
      {
        if (vel > R(0)) tf = qdiv(hi_pl - y[0], vel);
        else if (vel < R(0)) tf = qdiv(lo_pl - y[0], vel);
      }
      const R tface = fmin(fmin(gbc(gm, tf, gb), gbc(gm, tf, gb + 1)), gbc(gm, tf, gb + 2));
      R hs = fmin(fmin(h, E->h_max), room);
      bool capped = room <= fmin(h, E->h_max);
      R hf = R(1.25) * fmax(tface, R(0)) + tiny;
      if (hf < hs) {
        hs = hf;
        capped = false;
      }
      const R hh = sgn * hs;
      R k2[ND], k3[ND], k4[ND], k5[ND], k6[ND], k7[ND], t[ND], dy[ND];
      if (NC == 3 && poly)
        coop_stages<R, NC, NC == 3>(gm, gb, cv, pc, E->F.raw, ih, ihc, hh, y, k1, k2, k3, k4, k5, k6, k7, dy, t);
      else
        coop_stages<R, NC, false>(gm, gb, cv, pc, E->F.raw, ih, ihc, hh, y, k1, k2, k3, k4, k5, k6, k7, dy, t);
      c_stage += (c == 0) ? 6 : 0;
      steps += 1;
      R err = 0;
      bool bad = false;
#pragma unroll
      for (int i = 0; i < ND; ++i) {
        R e = fabs(hh * (R(DE1) * k1[i] + R(DE3) * k3[i] + R(DE4) * k4[i] + R(DE5) * k5[i] + R(DE6) * k6[i] +
                         R(DE7) * k7[i]));
        if (!isfinite(t[i])) bad = true;
        R ya = fabs(y[i]), yb = fabs(t[i]);
        if (i == 0) {
          R base = R(E->F.org[c]) + R(icc) * hhc;
          e *= hhc;
          ya = fabs(base + y[0] * hhc);
          yb = fabs(base + t[0] * hhc);
        }
        err = fmax(err, cdiv(e, P.tol_abs + P.tol_rel * fmax(ya, yb)));
      }
      err = fmax(fmax(gbc(gm, err, gb), gbc(gm, err, gb + 1)), gbc(gm, err, gb + 2));
      bad = __any_sync(gm, bad);
      if (bad) {
        status = QSL_LINE_NONFINITE;
      } else if (err > R(1)) {
        c_rej += (c == 0);
        h = hs * fmax(R(0.2), R(0.9) * cpow(err, R(-0.25)));
        if (h < E->h_min) status = QSL_LINE_STALL;
      } else {
        c_acc += (c == 0);
        R hnext = hs * ((err == R(0)) ? R(5) : fmin(R(5), R(0.9) * cpow(err, R(-0.2))));
        // first crossing of this axis's planes within the step, on the dense
        // output (same bracket and safeguarded Newton as cell_trace, with the
        // root t = 0 divided out when the step starts on the plane)
        R thc = R(2);
        int upc = 0;
        const R c4 = hh * (R(DD1) * k1[0] + R(DD3) * k3[0] + R(DD4) * k4[0] + R(DD5) * k5[0] + R(DD6) * k6[0] +
                           R(DD7) * k7[0]);
        const R dya = dy[0];
        const R bspl = hh * k1[0] - dya;
        const R c3 = dya - hh * k7[0] - bspl;
#pragma unroll
        for (int up = 0; up < 2; ++up) {
          const R target = up ? hi_pl : lo_pl;
          const bool dom = up ? hi_dom : lo_dom;
          const R r = target - y[0];
          const R over = up ? (dya - r) : (r - dya);
          if (!(over > (dom ? R(0) : band))) continue;
          const R sg = up ? R(1) : R(-1);
          const bool defl = (r == R(0));
          R ta = R(0), tb = R(1);
#pragma unroll
          for (int q = 1; q < 4; ++q) {
            R tq = R(0.25) * R(q);
            R s1 = R(1) - tq;
            R pq = dya + s1 * (bspl + tq * (c3 + s1 * c4));
            R f = defl ? pq : tq * pq - r;
            if (sg * f > R(0) && tb == R(1)) tb = tq;
            else if (tb == R(1)) ta = tq;
          }
          R tt = ta + (tb - ta) * R(0.5);
          if (!defl) {
            R tl = qdiv(r, dya);
            if (tl > ta && tl < tb) tt = tl;
          }
          for (int it = 0; it < 30; ++it) {
            R s1 = R(1) - tt;
            R inner = c3 + s1 * c4;
            R mid = bspl + tt * inner;
            R pv = dya + s1 * mid;
            R f = defl ? pv : tt * pv - r;
            if (fabs(f) <= R(4) * eps_of<R>() * (fabs(r) + fabs(dya)) || !(tb - ta > R(2) * eps_of<R>())) break;
            if (sg * f > R(0)) tb = tt;
            else ta = tt;
            R dmid = inner - tt * c4;
            R dp = s1 * dmid - mid;
            R df = defl ? dp : pv + tt * dp;
            R tn = tt - qdiv(f, df);
            tt = (tn > ta && tn < tb) ? tn : R(0.5) * (ta + tb);
          }
          if (tt < thc) {
            thc = tt;
            upc = up;
          }
        }
        // earliest crossing over the group; ties go to the lower plane id
        const R q0 = gbc(gm, thc, gb), q1 = gbc(gm, thc, gb + 1), q2 = gbc(gm, thc, gb + 2);
        const int u0 = __shfl_sync(gm, upc, gb), u1 = __shfl_sync(gm, upc, gb + 1), u2 = __shfl_sync(gm, upc, gb + 2);
        R th = R(2);
        int ax_c = -1, up_c = 0;
        if (q0 < th) { th = q0; ax_c = 0; up_c = u0; }
        if (q1 < th) { th = q1; ax_c = 1; up_c = u1; }
        if (q2 < th) { th = q2; ax_c = 2; up_c = u2; }
        if (ax_c < 0) {
          // the step stays in the cell: accept it; k7 is the next k1
#pragma unroll
          for (int i = 0; i < ND; ++i) {
            y[i] += dy[i];
            k1[i] = k7[i];
          }
          R t1 = hs - muc, t2 = mu + t1;
          muc = (t2 - mu) - t1;
          mu = t2;
          h = hnext;
          zc = 0;
          if (capped) status = QSL_LINE_MAXLEN;
        } else {
          // advance to the plane on the dense output and snap onto it
#pragma unroll
          for (int i = 0; i < ND; ++i)
            y[i] += y_at<R>(th, dy[i], hh * k1[i], hh * k7[i],
                            hh * (R(DD1) * k1[i] + R(DD3) * k3[i] + R(DD4) * k4[i] + R(DD5) * k5[i] +
                                  R(DD6) * k6[i] + R(DD7) * k7[i]));
          const int my_dom = up_c ? hi_dom : lo_dom;
          const bool dom = __shfl_sync(gm, my_dom, gb + ax_c) != 0;
          if (c == ax_c) y[0] = up_c ? hi_pl : lo_pl;
          R dl = th * hs;
          R t1 = dl - muc, t2 = mu + t1;
          muc = (t2 - mu) - t1;
          mu = t2;
          c_land += (c == 0);
          if (dom) {
            status = QSL_LINE_OK;
            lface = 2 * ax_c + up_c;
          } else {
            // enter the neighbouring cell
            zc = (dl < tiny) ? zc + 1 : 0;
            int na = sel3(ax_c, ic[0], ic[1], ic[2]) + (up_c ? 1 : -1);
            if (zc > 3 || na < 0 || na > E->F.n[ax_c] - 2) {
              // grazing a face back and forth: stay in this cell for one step
              zc = 0;
            } else {
              if (ax_c == 0) ic[0] = na;
              else if (ax_c == 1) ic[1] = na;
              else ic[2] = na;
              if (c == ax_c) y[0] = up_c ? R(0) : R(1);
              kvalid = false;
            }
            h = fmax(hnext, hs);
          }
        }
      }
    }
    if (status != ST_RUNNING) {
      write_end_coop<R, NC>(P, E, unit, c, y, sel3(c, ic[0], ic[1], ic[2]), mu, lface, status, steps);
      active = false;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_stage += __shfl_down_sync(FULL, c_stage, o);
    c_acc += __shfl_down_sync(FULL, c_acc, o);
    c_rej += __shfl_down_sync(FULL, c_rej, o);
    c_land += __shfl_down_sync(FULL, c_land, o);
    c_lines += __shfl_down_sync(FULL, c_lines, o);
  }
  unsigned any_to = __ballot_sync(FULL, timed_out);
  if (lane == 0 && P.stats) {
    atomicAdd(&P.stats->stage_evals, c_stage);
    atomicAdd(&P.stats->accepted, c_acc);
    atomicAdd(&P.stats->rejected, c_rej);
    atomicAdd(&P.stats->landing, c_land);
    atomicAdd(&P.stats->lines, c_lines);
    if (any_to) atomicAdd(&P.stats->timeouts, 1ull);
  }
  if (lane == 0 && any_to && P.timeout_flag) atomicExch(P.timeout_flag, 1);
}

// ------------------------------------------------------------ lengths-only cell-wise tracer
// The cell-wise Dormand-Prince tracer for lengths only (refinement passes and
// lengths-only maps), one lane per line. Only the position is integrated, so
// inside a cell the right-hand side is three trilinear polynomials in the
// in-cell coordinates (normalise-first fields; raw fields normalise the three
// at the point), whose 24 coefficients stay in registers from the cell entry
// on: a stage is the polynomials' four independent first-level FMAs and three
// dependent ones per component, plus one FMA of the stage combination on its
// dependent chain (the earlier terms of each combination are summed while the
// previous stages run). No shuffles and no shared memory. While a step is
// integrated, the 8 corners of the cell the line is expected to enter next
// (across the first plane along the step's initial direction) are loaded, so
// a cell entry usually finds its corners in registers instead of waiting for
// the memory system.
template <class V>
__device__ __forceinline__ float vcomp(const V& q, int c) {
  return c == 0 ? q.x : (c == 1 ? q.y : q.z);
}

template <class R, class V>
__device__ __forceinline__ void len_coeffs(const V* q, bool raw, const R* ih, R (*a)[8]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R cv[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) cv[k] = R(c == 0 ? q[k].x : (c == 1 ? q[k].y : q[k].z));
    trilinear_coeffs<R>(cv, raw ? R(1) : ih[c], a[c]);
  }
}

// Stage derivative in cell units: ih_c b_c(u, v, w).
template <class R>
__device__ __forceinline__ void len_rhs(const R (*a)[8], bool raw, const R* ih, const R* t, R* k) {
  const R u = t[0], v = t[1], w = t[2];
  R val[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R p0 = fma(a[c][1], u, a[c][0]), p1 = fma(a[c][4], u, a[c][2]), p2 = fma(a[c][5], u, a[c][3]),
            p3 = fma(a[c][7], u, a[c][6]);
    val[c] = fma(fma(p3, v, p2), w, fma(p1, v, p0));
  }
  if (raw) {
    // interpolate B, normalise at the point
    const R m2 = val[0] * val[0] + val[1] * val[1] + val[2] * val[2];
    const R rm = m2 > R(0) ? rsqrt(m2) : R(0);
#pragma unroll
    for (int c = 0; c < 3; ++c) k[c] = val[c] * rm * ih[c];
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) k[c] = val[c];
  }
}

// Earliest crossing fraction t in (0, 1] of plane `target` by the axis
// component of the step's dense output, offset t P(t) with the cubic
// P(t) = dya + (1 - t)(bspl + t (c3 + (1 - t) c4)); sg = +1 for an upper plane.
// The same bracket (t = 1/4, 1/2, 3/4) and safeguarded Newton iteration as the
// other cell-wise kernels; a step that starts on the plane (r = 0) solves P = 0
// (the trivial root t = 0 divided out).
template <class R>
__device__ __forceinline__ R len_crossing(R r, R dya, R bspl, R c3, R c4, R sg) {
  const bool defl = (r == R(0));
  R ta = R(0), tb = R(1);
#pragma unroll
  for (int q = 1; q < 4; ++q) {
    R tq = R(0.25) * R(q);
    R s1 = R(1) - tq;
    R pq = dya + s1 * (bspl + tq * (c3 + s1 * c4));
    R f = defl ? pq : tq * pq - r;
    if (sg * f > R(0) && tb == R(1)) tb = tq;
    else if (tb == R(1)) ta = tq;
  }
  R t = ta + (tb - ta) * R(0.5);
  if (!defl) {
    R tl = qdiv(r, dya);
    if (tl > ta && tl < tb) t = tl;
  }
  for (int it = 0; it < 30; ++it) {
    R s1 = R(1) - t;
    R inner = c3 + s1 * c4;
    R mid = bspl + t * inner;
    R pv = dya + s1 * mid;
    R f = defl ? pv : t * pv - r;
    if (fabs(f) <= R(4) * eps_of<R>() * (fabs(r) + fabs(dya)) || !(tb - ta > R(2) * eps_of<R>())) break;
    if (sg * f > R(0)) tb = t;
    else ta = t;
    R dmid = inner - t * c4;
    R dp = s1 * dmid - mid;
    R df = defl ? dp : pv + t * dp;
    R tn = t - qdiv(f, df);
    t = (tn > ta && tn < tb) ? tn : R(0.5) * (ta + tb);
  }
  return t;
}

// One line direction of the lengths-only tracer, start to end, by one lane.
// The item's constants are copied into registers once (nothing in the step
// loop reads memory but the corners at a cell entry), the planes and the
// error-norm offsets of the current cell are formed at its entry, and the
// cell's vertex address moves by one stride per face crossed.
template <class R>
__device__ __forceinline__ void len_line(const TraceParams<R>& P, int64_t unit, unsigned long long* c_stage,
                                         unsigned long long* c_acc, unsigned long long* c_rej,
                                         unsigned long long* c_land, bool* timed_out,
                                         unsigned long long t_start) {
  typedef typename V4<R>::type V;
  constexpr bool PREFETCH = sizeof(R) == 4;  // FP64 corners would double the registers held
  int64_t g;
  double xd[3];
  const Item<R>* E = resolve_seed(P, unit >> 1, &g, xd);
  const R sgn = (unit & 1) ? R(-1) : R(1);
  // the item's constants, in registers
  const V* const fv = E->F.v;
  const bool raw = E->F.raw != 0;
  const int n0 = E->F.n[0], n1 = E->F.n[1], n2 = E->F.n[2];
  const int64_t sy = n0, sz = (int64_t)n0 * n1;
  const R ih[3] = {R(E->F.inv_h[0]), R(E->F.inv_h[1]), R(E->F.inv_h[2])};
  const R hh3[3] = {R(1) / ih[0], R(1) / ih[1], R(1) / ih[2]};
  const R org[3] = {R(E->F.org[0]), R(E->F.org[1]), R(E->F.org[2])};
  const R dlo[3] = {E->lo[0], E->lo[1], E->lo[2]}, dhi[3] = {E->hi[0], E->hi[1], E->hi[2]};
  const R max_len = E->max_len, h_max = E->h_max, h_min = E->h_min;
  const R tiny = R(1e-4) * h_max;
  const R band = R(16) * eps_of<R>();  // tolerance band of internal cell faces (cell units)
  const R tol_abs = P.tol_abs, tol_rel = P.tol_rel;
  const long long max_steps = P.max_steps;
  int ic[3];
  R y[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    double fa = (xd[ax] - E->org_d[ax]) * E->inv_h_d[ax];
    double fl = floor(fmin(fmax(fa, 0.0), (double)(E->F.n[ax] - 2)));
    ic[ax] = (int)fl;
    y[ax] = (R)(fa - fl);
  }
  int status = ST_RUNNING, lface = NO_FACE;
  {
    bool outside = false;
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if (face_g<R, true>(E->lo, E->hi, ic, f, y, (const R*)nullptr) > R(0)) outside = true;
    if (outside || !isfinite(xd[0]) || !isfinite(xd[1]) || !isfinite(xd[2])) {
      status = QSL_LINE_OUTSIDE;
    } else {
      Interp<R> I0;
      interp<R, R, false, false, true, false>(E->F, y[0], y[1], y[2], I0, ic);
      R m0 = sqrt(I0.b[0] * I0.b[0] + I0.b[1] * I0.b[1] + I0.b[2] * I0.b[2]);
      if (!(m0 > R(0))) {
        status = QSL_LINE_NULL;
      } else {
        // a seed on a face whose field points out of the domain ends this side
        // at once with zero length
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          if (status == ST_RUNNING && face_g<R, true>(E->lo, E->hi, ic, f, y, (const R*)nullptr) == R(0)) {
            R bn = I0.b[f >> 1] * sgn;
            R outw = (f & 1) ? bn : -bn;
            if (outw > R(0)) {
              status = QSL_LINE_OK;
              lface = f;
            }
          }
        }
      }
    }
  }
  if (status != ST_RUNNING) {
    write_end<R, 3, true>(P, E, unit, y, ic, R(0), lface, status, 0);
    return;
  }
  R mu = 0, muc = 0, h = E->h_init;
  int steps = 0, zc = 0;
  bool kvalid = false, pf_valid = false;
  int64_t cell = (int64_t)ic[2] * sz + (int64_t)ic[1] * sy + ic[0];  // vertex index of the cell's corner 000
  int64_t pf_cell = -1;
  R a[3][8], k1[3];
  R lo_pl[3], hi_pl[3], base[3];
  bool lo_dom[3], hi_dom[3];
  V pq[8];
  for (;;) {
    if (P.timeout_ns && ((steps & 63) == 63)) {
      if (globaltimer() - t_start > P.timeout_ns) *timed_out = true;
    }
    if (*timed_out) status = QSL_LINE_TIMEOUT;
    else if (steps >= max_steps) status = QSL_LINE_MAXSTEPS;
    const R room = max_len - mu;
    if (status == ST_RUNNING && !(room > R(0))) status = QSL_LINE_MAXLEN;
    if (status != ST_RUNNING) break;
    if (!kvalid) {
      // the cell's corners (prefetched when predicted) to its polynomials;
      // its planes (cell faces, or domain faces where they come first)
      V q[8];
      if (PREFETCH && pf_valid && pf_cell == cell) {
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = pq[k];
      } else {
        const V* p = fv + cell;
        q[0] = ldg4(p);
        q[1] = ldg4(p + 1);
        q[2] = ldg4(p + sy);
        q[3] = ldg4(p + sy + 1);
        q[4] = ldg4(p + sz);
        q[5] = ldg4(p + sz + 1);
        q[6] = ldg4(p + sz + sy);
        q[7] = ldg4(p + sz + sy + 1);
      }
      pf_valid = false;
      len_coeffs<R, V>(q, raw, ih, a);
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const R lr = dlo[ax] - R(ic[ax]), hr = dhi[ax] - R(ic[ax]);
        lo_dom[ax] = lr >= R(0);
        hi_dom[ax] = hr <= R(1);
        lo_pl[ax] = lo_dom[ax] ? lr : R(0);
        hi_pl[ax] = hi_dom[ax] ? hr : R(1);
        base[ax] = org[ax] + R(ic[ax]) * hh3[ax];
      }
      len_rhs<R>(a, raw, ih, y, k1);
      *c_stage += 1;
      kvalid = true;
    }
    // step: controller size, capped a little beyond the first plane along k1
    R tface = R(1e30);
    int pax = -1, pup = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const R vel = sgn * k1[ax];
      R tt = R(1e30);
      if (vel > R(0)) tt = qdiv(hi_pl[ax] - y[ax], vel);
      else if (vel < R(0)) tt = qdiv(lo_pl[ax] - y[ax], vel);
      if (tt < tface) {
        tface = tt;
        pax = ax;
        pup = vel > R(0);
      }
    }
    if (PREFETCH && pax >= 0) {
      // load the corners of the cell across that plane while the step runs
      const bool pdom = pup ? sel3(pax, hi_dom[0], hi_dom[1], hi_dom[2]) : sel3(pax, lo_dom[0], lo_dom[1], lo_dom[2]);
      const int na = sel3(pax, ic[0], ic[1], ic[2]) + (pup ? 1 : -1);
      const int nmax = sel3(pax, n0, n1, n2) - 2;
      const int64_t st = pax == 0 ? 1 : (pax == 1 ? sy : sz);
      const int64_t nc = cell + (pup ? st : -st);
      if (!pdom && na >= 0 && na <= nmax && !(pf_valid && pf_cell == nc)) {
        const V* p = fv + nc;
        pq[0] = ldg4(p);
        pq[1] = ldg4(p + 1);
        pq[2] = ldg4(p + sy);
        pq[3] = ldg4(p + sy + 1);
        pq[4] = ldg4(p + sz);
        pq[5] = ldg4(p + sz + 1);
        pq[6] = ldg4(p + sz + sy);
        pq[7] = ldg4(p + sz + sy + 1);
        pf_cell = nc;
        pf_valid = true;
      }
    }
    R hs = fmin(fmin(h, h_max), room);
    bool capped = room <= fmin(h, h_max);
    const R hf = R(1.25) * fmax(tface, R(0)) + tiny;
    if (hf < hs) {
      hs = hf;
      capped = false;
    }
    const R hh = sgn * hs;
    // stage combinations with the step folded into the coefficients; each
    // stage's newest term is the last FMA
    const R c21 = hh * R(DA21), c31 = hh * R(DA31), c32 = hh * R(DA32), c41 = hh * R(DA41), c42 = hh * R(DA42),
            c43 = hh * R(DA43), c51 = hh * R(DA51), c52 = hh * R(DA52), c53 = hh * R(DA53), c54 = hh * R(DA54),
            c61 = hh * R(DA61), c62 = hh * R(DA62), c63 = hh * R(DA63), c64 = hh * R(DA64), c65 = hh * R(DA65);
    const R b1 = hh * R(DB1), b3 = hh * R(DB3), b4 = hh * R(DB4), b5 = hh * R(DB5), b6 = hh * R(DB6);
    R k2[3], k3[3], k4[3], k5[3], k6[3], k7[3], t[3], dy[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = fma(c21, k1[i], y[i]);
    len_rhs<R>(a, raw, ih, t, k2);
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = fma(c32, k2[i], fma(c31, k1[i], y[i]));
    len_rhs<R>(a, raw, ih, t, k3);
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = fma(c43, k3[i], fma(c42, k2[i], fma(c41, k1[i], y[i])));
    len_rhs<R>(a, raw, ih, t, k4);
#pragma unroll
    for (int i = 0; i < 3; ++i) t[i] = fma(c54, k4[i], fma(c53, k3[i], fma(c52, k2[i], fma(c51, k1[i], y[i]))));
    len_rhs<R>(a, raw, ih, t, k5);
#pragma unroll
    for (int i = 0; i < 3; ++i)
      t[i] = fma(c65, k5[i], fma(c64, k4[i], fma(c63, k3[i], fma(c62, k2[i], fma(c61, k1[i], y[i])))));
    len_rhs<R>(a, raw, ih, t, k6);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dy[i] = fma(b6, k6[i], fma(b5, k5[i], fma(b4, k4[i], fma(b3, k3[i], b1 * k1[i]))));
      t[i] = y[i] + dy[i];
    }
    len_rhs<R>(a, raw, ih, t, k7);
    *c_stage += 6;
    steps += 1;
    R err = 0;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R e = fabs(hh * (R(DE1) * k1[i] + R(DE3) * k3[i] + R(DE4) * k4[i] + R(DE5) * k5[i] + R(DE6) * k6[i] +
                             R(DE7) * k7[i])) * hh3[i];
      if (!isfinite(t[i])) finite = false;
      const R ya = fabs(base[i] + y[i] * hh3[i]), yb = fabs(base[i] + t[i] * hh3[i]);
      err = fmax(err, cdiv(e, tol_abs + tol_rel * fmax(ya, yb)));
    }
    if (!finite) {
      status = QSL_LINE_NONFINITE;
      break;
    }
    if (err > R(1)) {
      *c_rej += 1;
      h = hs * fmax(R(0.2), R(0.9) * cpow(err, R(-0.25)));
      if (h < h_min) {
        status = QSL_LINE_STALL;
        break;
      }
      continue;
    }
    *c_acc += 1;
    const R hnext = hs * ((err == R(0)) ? R(5) : fmin(R(5), R(0.9) * cpow(err, R(-0.2))));
    // first plane crossed within the step on the dense output (4th-order
    // continuous extension); the earliest crossing wins, lower plane id on ties
    R th = R(2);
    int ax_c = -1, up_c = 0;
    unsigned cmask = 0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      if ((lo_pl[ax] - y[ax]) - dy[ax] > (lo_dom[ax] ? R(0) : band)) cmask |= 1u << (2 * ax);
      if (dy[ax] - (hi_pl[ax] - y[ax]) > (hi_dom[ax] ? R(0) : band)) cmask |= 2u << (2 * ax);
    }
#pragma unroll 1
    while (cmask) {
      const int pl = __ffs(cmask) - 1;
      cmask &= cmask - 1;
      const int ax = pl >> 1, up = pl & 1;
      const R ya = sel3(ax, y[0], y[1], y[2]);
      const R dya = sel3(ax, dy[0], dy[1], dy[2]);
      const R target = up ? sel3(ax, hi_pl[0], hi_pl[1], hi_pl[2]) : sel3(ax, lo_pl[0], lo_pl[1], lo_pl[2]);
      const R k1a = sel3(ax, k1[0], k1[1], k1[2]);
      const R k7a = sel3(ax, k7[0], k7[1], k7[2]);
      const R c4 = hh * (R(DD1) * k1a + R(DD3) * sel3(ax, k3[0], k3[1], k3[2]) + R(DD4) * sel3(ax, k4[0], k4[1], k4[2]) +
                         R(DD5) * sel3(ax, k5[0], k5[1], k5[2]) + R(DD6) * sel3(ax, k6[0], k6[1], k6[2]) + R(DD7) * k7a);
      const R bspl = hh * k1a - dya;
      const R c3 = dya - hh * k7a - bspl;
      const R tc = len_crossing<R>(target - ya, dya, bspl, c3, c4, up ? R(1) : R(-1));
      if (tc < th) {
        th = tc;
        ax_c = ax;
        up_c = up;
      }
    }
    if (ax_c < 0) {
      // the step stays in the cell: accept it; k7 is the next k1
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        y[i] += dy[i];
        k1[i] = k7[i];
      }
      R t1 = hs - muc, t2 = mu + t1;
      muc = (t2 - mu) - t1;
      mu = t2;
      h = hnext;
      zc = 0;
      if (capped) {
        status = QSL_LINE_MAXLEN;
        break;
      }
      continue;
    }
    // advance to the plane on the dense output and snap onto it
#pragma unroll
    for (int i = 0; i < 3; ++i)
      y[i] += y_at<R>(th, dy[i], hh * k1[i], hh * k7[i],
                      hh * (R(DD1) * k1[i] + R(DD3) * k3[i] + R(DD4) * k4[i] + R(DD5) * k5[i] + R(DD6) * k6[i] +
                            R(DD7) * k7[i]));
    const bool dom = up_c ? sel3(ax_c, hi_dom[0], hi_dom[1], hi_dom[2]) : sel3(ax_c, lo_dom[0], lo_dom[1], lo_dom[2]);
    const R target = up_c ? sel3(ax_c, hi_pl[0], hi_pl[1], hi_pl[2]) : sel3(ax_c, lo_pl[0], lo_pl[1], lo_pl[2]);
    if (ax_c == 0) y[0] = target;
    else if (ax_c == 1) y[1] = target;
    else y[2] = target;
    const R dl = th * hs;
    R t1 = dl - muc, t2 = mu + t1;
    muc = (t2 - mu) - t1;
    mu = t2;
    *c_land += 1;
    if (dom) {
      status = QSL_LINE_OK;
      lface = 2 * ax_c + up_c;
      break;
    }
    // enter the neighbouring cell
    zc = (dl < tiny) ? zc + 1 : 0;
    const int na = sel3(ax_c, ic[0], ic[1], ic[2]) + (up_c ? 1 : -1);
    if (zc > 3 || na < 0 || na > sel3(ax_c, n0, n1, n2) - 2) {
      // grazing a face back and forth: stay in this cell for one step (the
      // cell's polynomial continued across the face)
      zc = 0;
    } else {
      const int64_t st = ax_c == 0 ? 1 : (ax_c == 1 ? sy : sz);
      cell += up_c ? st : -st;
      if (ax_c == 0) {
        ic[0] = na;
        y[0] = up_c ? R(0) : R(1);
      } else if (ax_c == 1) {
        ic[1] = na;
        y[1] = up_c ? R(0) : R(1);
      } else {
        ic[2] = na;
        y[2] = up_c ? R(0) : R(1);
      }
      kvalid = false;
    }
    h = fmax(hnext, hs);
  }
  write_end<R, 3, true>(P, E, unit, y, ic, mu, lface, status, steps);
}

// The lengths-only kernel: lane l of global warp w traces units w + l W,
// w + (l + 32) W, ... (W warps in the grid), so the units of a launch spread
// over all warps before a warp takes a second one, and a lane runs its line
// to the end with no warp-wide operation in between.
template <class R>
__global__ void __launch_bounds__(256) cell_len_kernel(const __grid_constant__ TraceParams<R> P) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int64_t total = P.n_units;
  if (P.n_seeds_dev) {
    int64_t c = 2 * (*P.n_seeds_dev);
    total = c < total ? c : total;
  }
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long c_stage = 0, c_acc = 0, c_rej = 0, c_land = 0, c_lines = 0;
  bool timed_out = false;
  const unsigned long long t_start = P.timeout_ns ? globaltimer() : 0ull;
  for (int64_t unit = w + (int64_t)lane * W; unit < total; unit += 32 * W) {
    c_lines += (unit & 1) == 0;
    len_line<R>(P, unit, &c_stage, &c_acc, &c_rej, &c_land, &timed_out, t_start);
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_stage += __shfl_down_sync(FULL, c_stage, o);
    c_acc += __shfl_down_sync(FULL, c_acc, o);
    c_rej += __shfl_down_sync(FULL, c_rej, o);
    c_land += __shfl_down_sync(FULL, c_land, o);
    c_lines += __shfl_down_sync(FULL, c_lines, o);
  }
  unsigned any_to = __ballot_sync(FULL, timed_out);
  if (lane == 0 && P.stats) {
    atomicAdd(&P.stats->stage_evals, c_stage);
    atomicAdd(&P.stats->accepted, c_acc);
    atomicAdd(&P.stats->rejected, c_rej);
    atomicAdd(&P.stats->landing, c_land);
    atomicAdd(&P.stats->lines, c_lines);
    if (any_to) atomicAdd(&P.stats->timeouts, 1ull);
  }
  if (lane == 0 && any_to && P.timeout_flag) atomicExch(P.timeout_flag, 1);
}

// ------------------------------------------------------------ Cash-Karp lengths-only tracer
// The decision traces of the refinement passes (qsl_refine_spec.pass_stepper
// QSL_PASS_CASH_KARP): the paper's Cash-Karp stepper across cells (Sec.
// "Integration methods") on the position only, one lane per line direction,
// with the step control, error norm and face landing of trace_kernel. A stage
// takes its derivative from the trilinear polynomials of the cell its point
// lies in; those coefficients stay in registers while the following stages
// fall in the same cell (a step at the passes' step cap spans a few cells), so
// only a stage that enters another cell loads corners.
template <class R>
struct CkCell {
  int ci[3];    // lower vertex of the cached cell (absolute)
  R a[3][8];    // its polynomials (len_coeffs)
};

// Stage derivative in cell units at the local-frame point ic + t.
template <class R, class V>
__device__ __forceinline__ void ck_len_rhs(const V* fv, const int* n, int64_t sy, int64_t sz, bool raw,
                                           const R* ih, const int* ic, const R* t, CkCell<R>& C, R* k) {
  int ci[3];
  R uu[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R lim = R(n[a]);
    const R fl = floor(fmin(fmax(t[a], -lim), lim));
    int i = ic[a] + (int)fl;
    i = min(max(i, 0), n[a] - 2);
    uu[a] = t[a] - R(i - ic[a]);
    ci[a] = i;
  }
  if (ci[0] != C.ci[0] || ci[1] != C.ci[1] || ci[2] != C.ci[2]) {
    const V* p = fv + ((int64_t)ci[2] * sz + (int64_t)ci[1] * sy + ci[0]);
    V q[8];
    q[0] = ldg4(p);
    q[1] = ldg4(p + 1);
    q[2] = ldg4(p + sy);
    q[3] = ldg4(p + sy + 1);
    q[4] = ldg4(p + sz);
    q[5] = ldg4(p + sz + 1);
    q[6] = ldg4(p + sz + sy);
    q[7] = ldg4(p + sz + sy + 1);
    len_coeffs<R, V>(q, raw, ih, C.a);
    C.ci[0] = ci[0];
    C.ci[1] = ci[1];
    C.ci[2] = ci[2];
  }
  len_rhs<R>(C.a, raw, ih, uu, k);
}

// One Cash-Karp step of signed size hh from the local-frame point ic + y.
template <class R, class V>
__device__ __forceinline__ void ck_len_step(const V* fv, const int* n, int64_t sy, int64_t sz, bool raw,
                                            const R* ih, const int* ic, const R* y, R hh, CkCell<R>& C, R* dy,
                                            R* yerr) {
  R k1[3], k2[3], k3[3], k4[3], k5[3], k6[3], t[3];
  ck_len_rhs<R, V>(fv, n, sy, sz, raw, ih, ic, y, C, k1);
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = fma(hh, R(A21) * k1[i], y[i]);
  ck_len_rhs<R, V>(fv, n, sy, sz, raw, ih, ic, t, C, k2);
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = fma(hh, R(A31) * k1[i] + R(A32) * k2[i], y[i]);
  ck_len_rhs<R, V>(fv, n, sy, sz, raw, ih, ic, t, C, k3);
#pragma unroll
  for (int i = 0; i < 3; ++i) t[i] = fma(hh, R(A41) * k1[i] + R(A42) * k2[i] + R(A43) * k3[i], y[i]);
  ck_len_rhs<R, V>(fv, n, sy, sz, raw, ih, ic, t, C, k4);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    t[i] = fma(hh, R(A51) * k1[i] + R(A52) * k2[i] + R(A53) * k3[i] + R(A54) * k4[i], y[i]);
  ck_len_rhs<R, V>(fv, n, sy, sz, raw, ih, ic, t, C, k5);
#pragma unroll
  for (int i = 0; i < 3; ++i)
    t[i] = fma(hh, R(A61) * k1[i] + R(A62) * k2[i] + R(A63) * k3[i] + R(A64) * k4[i] + R(A65) * k5[i], y[i]);
  ck_len_rhs<R, V>(fv, n, sy, sz, raw, ih, ic, t, C, k6);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dy[i] = hh * (R(B1) * k1[i] + R(B3) * k3[i] + R(B4) * k4[i] + R(B6) * k6[i]);
    yerr[i] = hh * (R(E1) * k1[i] + R(E3) * k3[i] + R(E4) * k4[i] + R(E5) * k5[i] + R(E6) * k6[i]);
  }
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Asks L1 for the corner rows of the cell holding the local-frame point
// ic + t (clamped to the grid like a stage's cell, so the address is valid).
template <class R, class V>
__device__ __forceinline__ void ck_prefetch_cell(const V* fv, const int* n, int64_t sy, int64_t sz, const int* ic,
                                                 const R* t) {
  int cj[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R lim = R(n[a]);
    const R fl = floor(fmin(fmax(t[a], -lim), lim));
    cj[a] = min(max(ic[a] + (int)fl, 0), n[a] - 2);
  }
  const V* p = fv + ((int64_t)cj[2] * sz + (int64_t)cj[1] * sy + cj[0]);
  prefetch_l1(p);
  prefetch_l1(p + 1);
  prefetch_l1(p + sy);
  prefetch_l1(p + sy + 1);
  prefetch_l1(p + sz);
  prefetch_l1(p + sz + 1);
  prefetch_l1(p + sz + sy);
  prefetch_l1(p + sz + sy + 1);
}

// One line direction of the Cash-Karp lengths-only tracer, start to end, by
// one lane (trace_kernel's steps for NC = 3 in the local frame). After each
// accepted step the cells at a third, two thirds and the end of the next step
// (predicted along this step's increment) are requested from L1, so that the
// stages entering them find their corners there instead of waiting for L2.
template <class R>
__device__ __forceinline__ void ck_len_line(const TraceParams<R>& P, int64_t unit, unsigned long long* c_stage,
                                            unsigned long long* c_acc, unsigned long long* c_rej,
                                            unsigned long long* c_land, bool* timed_out,
                                            unsigned long long t_start) {
  typedef typename V4<R>::type V;
  int64_t g;
  double xd[3];
  const Item<R>* E = resolve_seed(P, unit >> 1, &g, xd);
  const R sgn = (unit & 1) ? R(-1) : R(1);
  const V* const fv = E->F.v;
  const bool raw = E->F.raw != 0;
  const int n[3] = {E->F.n[0], E->F.n[1], E->F.n[2]};
  const int64_t sy = n[0], sz = (int64_t)n[0] * n[1];
  const R ih[3] = {R(E->F.inv_h[0]), R(E->F.inv_h[1]), R(E->F.inv_h[2])};
  const R hh3[3] = {R(1) / ih[0], R(1) / ih[1], R(1) / ih[2]};
  const R org[3] = {R(E->F.org[0]), R(E->F.org[1]), R(E->F.org[2])};
  const R dlo[3] = {E->lo[0], E->lo[1], E->lo[2]}, dhi[3] = {E->hi[0], E->hi[1], E->hi[2]};
  const R max_len = E->max_len, h_max = E->h_max, h_min = E->h_min, land_tol = E->land_tol;
  const R tol_abs = P.tol_abs, tol_rel = P.tol_rel;
  const long long max_steps = P.max_steps;
  int ic[3];
  R y[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    double fa = (xd[ax] - E->org_d[ax]) * E->inv_h_d[ax];
    double fl = floor(fmin(fmax(fa, 0.0), (double)(n[ax] - 2)));
    ic[ax] = (int)fl;
    y[ax] = (R)(fa - fl);
  }
  int status = ST_RUNNING, lface = NO_FACE;
  {
    bool outside = false;
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if (face_g<R, true>(dlo, dhi, ic, f, y, (const R*)nullptr) > R(0)) outside = true;
    if (outside || !isfinite(xd[0]) || !isfinite(xd[1]) || !isfinite(xd[2])) {
      status = QSL_LINE_OUTSIDE;
    } else {
      Interp<R> I0;
      interp<R, R, false, false, true, false>(E->F, y[0], y[1], y[2], I0, ic);
      R m0 = sqrt(I0.b[0] * I0.b[0] + I0.b[1] * I0.b[1] + I0.b[2] * I0.b[2]);
      if (!(m0 > R(0))) {
        status = QSL_LINE_NULL;
      } else {
#pragma unroll
        for (int f = 0; f < 6; ++f) {
          if (status == ST_RUNNING && face_g<R, true>(dlo, dhi, ic, f, y, (const R*)nullptr) == R(0)) {
            R bn = I0.b[f >> 1] * sgn;
            R outw = (f & 1) ? bn : -bn;
            if (outw > R(0)) {
              status = QSL_LINE_OK;
              lface = f;
            }
          }
        }
      }
    }
  }
  if (status != ST_RUNNING) {
    write_end<R, 3, true>(P, E, unit, y, ic, R(0), lface, status, 0);
    return;
  }
  CkCell<R> C;
  C.ci[0] = C.ci[1] = C.ci[2] = -1;
  R mu = 0, muc = 0, h = E->h_init, hs = 0;
  int steps = 0, phase = 0;
  bool capped = false;
  R la = 0, lb = 0, lga = 0, lgb = 0, lhm = 0, yh[3] = {0, 0, 0};
  int lside = 0, lit = 0, lround = 0;
  for (;;) {
    if (P.timeout_ns && ((steps & 63) == 63)) {
      if (globaltimer() - t_start > P.timeout_ns) *timed_out = true;
    }
    if (*timed_out) status = QSL_LINE_TIMEOUT;
    hs = lhm;
    if (status == ST_RUNNING && phase == 0) {
      if (steps >= max_steps) status = QSL_LINE_MAXSTEPS;
      R room = max_len - mu;
      if (status == ST_RUNNING && !(room > R(0))) status = QSL_LINE_MAXLEN;
      hs = fmin(h, h_max);
      capped = false;
      if (room <= hs) {
        hs = room;
        capped = true;
      }
    }
    if (status != ST_RUNNING) break;
    R dy[3], yerr[3];
    ck_len_step<R, V>(fv, n, sy, sz, raw, ih, ic, y, sgn * hs, C, dy, yerr);
    *c_stage += 6;
    steps += 1;
    if (phase == 0) {
      R err = 0;
      bool finite = true;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        R yn = y[i] + dy[i];
        if (!isfinite(yn)) finite = false;
        // position error in domain units, scaled by |x| in domain units
        R base = org[i] + R(ic[i]) * hh3[i];
        R e = fabs(yerr[i]) * hh3[i];
        R ya = fabs(base + y[i] * hh3[i]);
        R yb = fabs(base + yn * hh3[i]);
        R sc = tol_abs + tol_rel * fmax(ya, yb);
        err = fmax(err, cdiv(e, sc));
      }
      if (!finite) {
        status = QSL_LINE_NONFINITE;
      } else if (err > R(1)) {
        *c_rej += 1;
        h = hs * fmax(R(0.2), R(0.9) * cpow(err, R(-0.25)));
        if (h < h_min) status = QSL_LINE_STALL;
      } else {
        *c_acc += 1;
        bool inside = true;
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if (face_g<R, true>(dlo, dhi, ic, f, y, dy) > R(0)) inside = false;
        if (inside) {
#pragma unroll
          for (int i = 0; i < 3; ++i) y[i] += dy[i];
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            R fl = floor(y[a]);
            int ni = min(max(ic[a] + (int)fl, 0), n[a] - 2);
            y[a] -= R(ni - ic[a]);
            ic[a] = ni;
          }
          R t1 = hs - muc, t2 = mu + t1;
          muc = (t2 - mu) - t1;
          mu = t2;
          if (capped) status = QSL_LINE_MAXLEN;
          else h = hs * ((err == R(0)) ? R(5) : fmin(R(5), R(0.9) * cpow(err, R(-0.2))));
          const R sc = fmin(h, h_max) / hs;
#pragma unroll
          for (int q = 1; q <= 3; ++q) {
            const R c = R(q) * R(1.0 / 3.0) * sc;
            const R tq[3] = {fma(c, dy[0], y[0]), fma(c, dy[1], y[1]), fma(c, dy[2], y[2])};
            ck_prefetch_cell<R, V>(fv, n, sy, sz, ic, tq);
          }
        } else {
          phase = 1;
          yh[0] = dy[0];
          yh[1] = dy[1];
          yh[2] = dy[2];
          lface = chord_face<R, true>(dlo, dhi, ic, y, yh);
          la = 0;
          lb = hs;
          lga = face_gs<R, true>(dlo, dhi, ic, lface, y, (const R*)nullptr);
          lgb = face_gs<R, true>(dlo, dhi, ic, lface, y, yh);
          lside = 0;
          lit = 0;
          lround = 0;
          lhm = la + (lb - la) * lga / (lga - lgb);
          if (!(lga < R(0))) {
            lside = 2;
            lhm = R(0.5) * lb;
          }
        }
      }
    } else {
      *c_land += 1;
      lit += 1;
      R gm = face_gs<R, true>(dlo, dhi, ic, lface, y, dy);
      R dn = fabs(lface >> 1 == 0 ? dy[0] : (lface >> 1 == 1 ? dy[1] : dy[2]));
      R gtol = fmax(land_tol, R(4) * eps_of<R>() * dn);
      if (lside == 2 && lit < 60 && isfinite(gm)) {
        if (gm < R(0)) {
          la = lhm;
          lga = gm;
          lside = 0;
          lhm = la + (lb - la) * lga / (lga - lgb);
        } else {
          lb = lhm;
          lgb = gm;
          lhm = R(0.5) * lhm;
        }
      } else if (fabs(gm) <= gtol || lit >= 60 || !isfinite(gm) || !(lb - la > eps_of<R>() * lb)) {
        R worst = R(-1);
#pragma unroll
        for (int f = 0; f < 6; ++f)
          if (f != lface) worst = fmax(worst, face_g<R, true>(dlo, dhi, ic, f, y, dy));
        if (worst > gtol && lround < 8) {
          lround += 1;
          yh[0] = dy[0];
          yh[1] = dy[1];
          yh[2] = dy[2];
          R hi_h = lhm;
          lface = chord_face<R, true>(dlo, dhi, ic, y, yh);
          la = 0;
          lb = hi_h;
          lga = face_gs<R, true>(dlo, dhi, ic, lface, y, (const R*)nullptr);
          lgb = face_gs<R, true>(dlo, dhi, ic, lface, y, yh);
          lside = 0;
          lit = 0;
          lhm = la + (lb - la) * lga / (lga - lgb);
          if (!(lga < R(0))) {
            lside = 2;
            lhm = R(0.5) * lb;
          }
        } else {
#pragma unroll
          for (int i = 0; i < 3; ++i) y[i] += dy[i];
          R t1 = lhm - muc, t2 = mu + t1;
          muc = (t2 - mu) - t1;
          mu = t2;
          status = QSL_LINE_OK;
        }
      } else {
        if (gm > R(0)) {
          lb = lhm;
          lgb = gm;
          if (lside == 1) lga *= R(0.5);
          lside = 1;
        } else {
          la = lhm;
          lga = gm;
          if (lside == -1) lgb *= R(0.5);
          lside = -1;
        }
        lhm = la + (lb - la) * lga / (lga - lgb);
      }
    }
    if (status != ST_RUNNING) break;
  }
  write_end<R, 3, true>(P, E, unit, y, ic, mu, lface, status, steps);
}

// The Cash-Karp lengths-only kernel: units spread over the warps as in
// cell_len_kernel, each lane runs its line to the end.
template <class R>
__global__ void __maxnreg__(168) ck_len_kernel(const __grid_constant__ TraceParams<R> P) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int64_t total = P.n_units;
  if (P.n_seeds_dev) {
    int64_t c = 2 * (*P.n_seeds_dev);
    total = c < total ? c : total;
  }
  const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  unsigned long long c_stage = 0, c_acc = 0, c_rej = 0, c_land = 0, c_lines = 0;
  bool timed_out = false;
  const unsigned long long t_start = P.timeout_ns ? globaltimer() : 0ull;
  for (int64_t unit = w + (int64_t)lane * W; unit < total; unit += 32 * W) {
    c_lines += (unit & 1) == 0;
    ck_len_line<R>(P, unit, &c_stage, &c_acc, &c_rej, &c_land, &timed_out, t_start);
  }
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c_stage += __shfl_down_sync(FULL, c_stage, o);
    c_acc += __shfl_down_sync(FULL, c_acc, o);
    c_rej += __shfl_down_sync(FULL, c_rej, o);
    c_land += __shfl_down_sync(FULL, c_land, o);
    c_lines += __shfl_down_sync(FULL, c_lines, o);
  }
  unsigned any_to = __ballot_sync(FULL, timed_out);
  if (lane == 0 && P.stats) {
    atomicAdd(&P.stats->stage_evals, c_stage);
    atomicAdd(&P.stats->accepted, c_acc);
    atomicAdd(&P.stats->rejected, c_rej);
    atomicAdd(&P.stats->landing, c_land);
    atomicAdd(&P.stats->lines, c_lines);
    if (any_to) atomicAdd(&P.stats->timeouts, 1ull);
  }
  if (lane == 0 && any_to && P.timeout_flag) atomicExch(P.timeout_flag, 1);
}

// ------------------------------------------------------------ assembly (FP64)
__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

struct EndTerms {
  double bmag, A, B, C, cross, Af, Bf, Cf, bn;
  bool foot_ok;
};

// B at a point for the assembly (|B| and the direction the deviations are
// projected against). FP32 field on a uniform grid: the cell and the in-cell
// fractions are found in FP64 (exact), the interpolation itself runs in FP32
// on the FP32 vertex values (relative error about 1e-7) and is widened; the
// deviation norms, the determinant and Q are then assembled in FP64. FP64
// fields and rectilinear grids interpolate in FP64.
template <class S>
__device__ __forceinline__ void interp_end(const FieldView<S>& F, const double* x, Interp<double>& I) {
  if (sizeof(S) == 4 && F.uniform) {
    int ic[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double fa = (x[a] - (double)F.org[a]) * (double)F.inv_h[a];
      const double fl = floor(fmin(fmax(fa, 0.0), (double)(F.n[a] - 2)));
      ic[a] = (int)fl;
      f[a] = (float)(fa - fl);
    }
    Interp<float> J;
    interp<float, S, false, true, true, true>(F, f[0], f[1], f[2], J, ic);
    I.b[0] = J.b[0];
    I.b[1] = J.b[1];
    I.b[2] = J.b[2];
    I.m = J.m;
  } else {
    interp<double, S, false, true>(F, x[0], x[1], x[2], I);
  }
}

template <class S>
__device__ void end_terms(const FieldView<S>& F, const double* x, const double* d1_in, const double* d2_in,
                          int face, bool have_face, EndTerms& r) {
  // deviations as physical vectors in the end's orthonormal frame (spherical
  // coordinates: (r cos(theta) dphi, r dtheta, dr))
  double sf[3] = {1.0, 1.0, 1.0};
  if (F.geom == QSL_GEOM_SPHERICAL) sph_scale<double>(x[1], x[2], sf);
  const double d1[3] = {d1_in[0] * sf[0], d1_in[1] * sf[1], d1_in[2] * sf[2]};
  const double d2[3] = {d2_in[0] * sf[0], d2_in[1] * sf[1], d2_in[2] * sf[2]};
  Interp<double> I;
  interp_end<S>(F, x, I);
  r.bmag = I.m;
  const double b2 = dot3(I.b, I.b);
  const double rm = b2 > 0.0 ? rsqrt_fp64(b2) : 1.0 / sqrt(b2);  // a null end gives NaN directions, as 1 / 0
  double u[3] = {I.b[0] * rm, I.b[1] * rm, I.b[2] * rm};
  // Sec. "Squashing factor calculation": dx_perp = dx - b (b.dx), b normalised
  double ud1 = dot3(u, d1), ud2 = dot3(u, d2);
  double ap[3], bp[3];
  for (int i = 0; i < 3; ++i) {
    ap[i] = d1[i] - u[i] * ud1;
    bp[i] = d2[i] - u[i] * ud2;
  }
  r.A = dot3(ap, ap);
  r.B = dot3(bp, bp);
  r.C = dot3(ap, bp);
  double cr[3] = {ap[1] * bp[2] - ap[2] * bp[1], ap[2] * bp[0] - ap[0] * bp[2], ap[0] * bp[1] - ap[1] * bp[0]};
  const double c2 = dot3(cr, cr);
  r.cross = c2 * rsqrt_fp64(c2);
  r.foot_ok = false;
  r.Af = r.Bf = r.Cf = r.bn = __longlong_as_double(0x7ff8000000000000ll);
  if (have_face && face != NO_FACE) {
    int a = face >> 1;
    if (u[a] != 0.0) {
      double af[3], bf[3];
      const double ru = rcp_fp64(u[a]);
      const double s1 = d1[a] * ru, s2 = d2[a] * ru;
      for (int i = 0; i < 3; ++i) {
        af[i] = d1[i] - u[i] * s1;
        bf[i] = d2[i] - u[i] * s2;
      }
      r.Af = dot3(af, af);
      r.Bf = dot3(bf, bf);
      r.Cf = dot3(af, bf);
      r.bn = I.m * fabs(u[a]);
      r.foot_ok = true;
    }
  }
}

template <class R>
struct AssembleParams {
  TraceParams<R> T;  // the launch's problems, seeds and end records
  LineOutputs out;
  int tangent;
};

template <class R>
__global__ void __launch_bounds__(128) assemble_kernel(const __grid_constant__ AssembleParams<R> P) {
  int64_t n = P.T.n_units / 2;
  if (P.T.n_seeds_dev) n = min(n, *P.T.n_seeds_dev);
  const double NaN = __longlong_as_double(0x7ff8000000000000ll);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    int64_t g;
    double x0[3];
    const Item<R>* E = resolve_seed(P.T, j, &g, x0);
    const FieldView<R>& FV = E->F;
    const EndRec<R>& ef = P.T.ends[2 * j];
    const EndRec<R>& eb = P.T.ends[2 * j + 1];
    double q_perp = NaN, q_foot = NaN, q_det = NaN, b0 = NaN, bf = NaN, bb = NaN, ff = NaN, fb = NaN;
    int sf = ef.status, sb = eb.status;
    double L = NaN;
    if (sf != QSL_LINE_OUTSIDE) L = (double)ef.mu + (double)eb.mu;
    if (sf != QSL_LINE_OUTSIDE && sf != QSL_LINE_NULL) {
      Interp<double> I0;
      interp_end<R>(FV, x0, I0);
      b0 = I0.m;
    }
    bool okf = (sf == QSL_LINE_OK || sf == QSL_LINE_MAXLEN);
    bool okb = (sb == QSL_LINE_OK || sb == QSL_LINE_MAXLEN);
    bool open = !(sf == QSL_LINE_OK && sb == QSL_LINE_OK && ef.face == 4 && eb.face == 4);
    if (P.tangent && okf && okb) {
      double xf[3], xb[3], d1f[3], d2f[3], d1b[3], d2b[3];
      for (int i = 0; i < 3; ++i) {
        xf[i] = ef.x[i];
        xb[i] = eb.x[i];
        d1f[i] = ef.d1[i];
        d2f[i] = ef.d2[i];
        d1b[i] = eb.d1[i];
        d2b[i] = eb.d2[i];
      }
      EndTerms tf, tb;
      end_terms<R>(FV, xf, d1f, d2f, ef.face, sf == QSL_LINE_OK, tf);
      end_terms<R>(FV, xb, d1b, d2b, eb.face, sb == QSL_LINE_OK, tb);
      bf = tf.bmag;
      bb = tb.bmag;
      double br = tf.A * tb.B + tb.A * tf.B - 2.0 * tb.C * tf.C;
      const double rb0 = rcp_fp64(b0), rb02 = rb0 * rb0;
      q_perp = bf * bb * rb02 * br;  // Eq. finalQ
      const double gd = (tf.A * tf.B - tf.C * tf.C) * (tb.A * tb.B - tb.C * tb.C);
      q_det = gd > 0.0 ? br * rsqrt_fp64(gd) : br / sqrt(gd);
      ff = bf * rb0 * tf.cross - 1.0;
      fb = bb * rb0 * tb.cross - 1.0;
      if (tf.foot_ok && tb.foot_ok) {
        double brf = tf.Af * tb.Bf + tb.Af * tf.Bf - 2.0 * tb.Cf * tf.Cf;
        q_foot = tf.bn * tb.bn * rb02 * brf;
      }
      if (P.out.skip_open && open) q_perp = q_foot = q_det = NaN;
    }
    uint8_t flags = (P.out.skip_open && open && P.tangent && okf && okb) ? QSL_FLAG_OPEN_SKIPPED : 0;
    if (P.out.retraced) flags |= QSL_FLAG_RETRACED;
    if (P.out.lines) {
      qsl_line& o = P.out.lines[g];
      o.q_perp = q_perp;
      o.q_foot = q_foot;
      o.q_det = q_det;
      o.b0 = b0;
      o.bf = bf;
      o.bb = bb;
      o.flux_f = ff;
      o.flux_b = fb;
      o.length = (float)L;
      o.lam_f = (float)ef.mu;
      o.lam_b = -(float)eb.mu;
      o.pad0 = 0;
      for (int i = 0; i < 3; ++i) {
        o.x_f[i] = (float)ef.x[i];
        o.x_b[i] = (float)eb.x[i];
      }
      o.steps = ef.steps + eb.steps;
      o.face_f = (uint8_t)ef.face;
      o.face_b = (uint8_t)eb.face;
      o.status_f = (uint8_t)sf;
      o.status_b = (uint8_t)sb;
    }
    double qsel = (P.out.q_form == QSL_Q_FOOT) ? q_foot : (P.out.q_form == QSL_Q_DET ? q_det : q_perp);
    if (P.out.q) P.out.q[g] = (float)qsel;
    if (P.out.length) P.out.length[g] = (float)L;
    if (P.out.faces) {
      P.out.faces[2 * g] = (uint8_t)ef.face;
      P.out.faces[2 * g + 1] = (uint8_t)eb.face;
    }
    if (P.out.status) P.out.status[g] = (uint8_t)((sf & 7) | ((sb & 7) << 3) | flags);
  }
}

// Seeds whose selected Q exceeds the threshold (or whose Q is not finite for
// a finite length) go to the FP64 retrace list.
__global__ void select_kernel(int64_t n, const float* q, const qsl_line* lines, int q_form, double thr,
                              int64_t* index, int64_t* count) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    double qv;
    if (q) {
      qv = q[j];
    } else {
      qv = (q_form == QSL_Q_FOOT) ? lines[j].q_foot : (q_form == QSL_Q_DET ? lines[j].q_det : lines[j].q_perp);
    }
    if (qv > thr) {
      unsigned long long k = atomicAdd((unsigned long long*)count, 1ull);
      index[k] = j;
    }
  }
}

template <class R>
FieldView<R> make_view(const qsl_field* f);
template <>
FieldView<float> make_view<float>(const qsl_field* f) {
  FieldView<float> v;
  v.v = f->v32;
  for (int a = 0; a < 3; ++a) {
    v.axis[a] = f->axis32[a];
    v.org[a] = (float)f->org[a];
    v.inv_h[a] = (float)(1.0 / f->h[a]);
    v.n[a] = f->n[a];
  }
  v.uniform = f->uniform;
  v.raw = f->mode == QSL_RAW_B;
  v.order = 1;
  v.geom = f->geom;
  return v;
}
template <>
FieldView<double> make_view<double>(const qsl_field* f) {
  FieldView<double> v;
  v.v = f->v64;
  for (int a = 0; a < 3; ++a) {
    v.axis[a] = f->axis64[a];
    v.org[a] = f->org[a];
    v.inv_h[a] = 1.0 / f->h[a];
    v.n[a] = f->n[a];
  }
  v.uniform = f->uniform;
  v.raw = f->mode == QSL_RAW_B;
  v.order = 1;
  v.geom = f->geom;
  return v;
}

// One problem of a launch from a field, its seed source and its resolved
// configuration (domain bounds, step scales in domain units).
template <class R>
Item<R> make_item(const qsl_field* f, const SeedSource& src, const TraceConfig& cfg, int64_t seed_start, bool loc) {
  Item<R> it;
  it.F = make_view<R>(f);
  it.F.order = cfg.interp_order;
  it.src = src;
  it.seed_start = seed_start;
  for (int a = 0; a < 3; ++a) {
    // reciprocals once here, so seeding multiplies instead of dividing in FP64
    it.src.inv_n[a] = src.n[a] > 0 ? 1.0 / (double)src.n[a] : 0.0;
    it.org_d[a] = f->org[a];
    it.h_d[a] = f->h[a];
    it.inv_h_d[a] = f->h[a] > 0 ? 1.0 / f->h[a] : 0.0;
    it.lo_d[a] = cfg.lo[a];
    it.hi_d[a] = cfg.hi[a];
    // the local frame measures positions in grid-index units
    it.lo[a] = loc ? (R)((cfg.lo[a] - f->org[a]) / f->h[a]) : (R)cfg.lo[a];
    it.hi[a] = loc ? (R)((cfg.hi[a] - f->org[a]) / f->h[a]) : (R)cfg.hi[a];
  }
  it.max_len = (R)cfg.max_len;
  it.h_init = (R)(cfg.h_init * cfg.cell);
  it.h_max = (R)(cfg.h_max * cfg.cell);
  it.h_min = (R)(cfg.h_min * cfg.cell);
  it.euler_h = (R)(cfg.euler_h * cfg.cell);
  // landing tolerance in the frame's units (cell units of the coarsest axis
  // in the local frame); the kernel also stops at the resolution of the step
  double lt = loc ? cfg.land_tol / fmax(fmax(f->h[0], f->h[1]), f->h[2]) : cfg.land_tol;
  it.land_tol = (R)lt;
  return it;
}

// Scratch of one tracing launch: the queue head and watchdog flag (16 bytes
// at offset 0) and one end record per unit from offset 256. `scratch` is
// either caller-provided (no-allocation entry point, captured plans) or
// allocated here.
template <class R, int NC>
int launch_trace(const Item<R>& item0, const Item<R>* items_dev, int n_items, bool loc, const int64_t* index,
                 int64_t n_seeds, const int64_t* n_seeds_dev, const TraceConfig& cfg, const LaunchShape& shape,
                 const LineOutputs& out, cudaStream_t stream, DeviceStats* stats_dev, cudaEvent_t* ev,
                 void* scratch) {
  int dev = 0, sms = 0;
  QSL_CHECK_CUDA(cudaGetDevice(&dev));
  QSL_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  size_t n_units = (size_t)(2 * n_seeds);
  const bool own = scratch == nullptr;
  if (own)
    QSL_CHECK_CUDA(qsl::alloc_async((void**)&scratch, 256 + sizeof(EndRec<R>) * (n_units ? n_units : 1), stream));
  unsigned long long* head = reinterpret_cast<unsigned long long*>(scratch);
  EndRec<R>* ends = reinterpret_cast<EndRec<R>*>(reinterpret_cast<unsigned char*>(scratch) + 256);
  QSL_CHECK_CUDA(cudaMemsetAsync(head, 0, 16, stream));
  TraceParams<R> P;
  P.item0 = item0;
  P.items = items_dev;
  P.n_items = n_items;
  P.index = index;
  P.n_units = 2 * n_seeds;
  P.n_seeds_dev = n_seeds_dev;
  P.ends = ends;
  P.head = head;
  P.stats = stats_dev;
  P.tol_abs = (R)cfg.tol_abs;
  P.tol_rel = (R)cfg.tol_rel;
  P.max_steps = cfg.max_steps;
  P.euler = cfg.integrator == QSL_EULER;
  P.refill_min = shape.refill_min > 0 ? shape.refill_min : 1;
  P.timeout_ns = cfg.timeout_ns;
  P.timeout_flag = reinterpret_cast<int*>(head + 1);
  int threads = 32 * shape.warps_per_block;
  // persistent kernel: never launch more blocks than can be resident at once
  const bool use_cell = loc && cfg.integrator == QSL_DOPRI5_CELL;
  // lengths only, unless three lanes per line are asked for: the one-lane
  // polynomial kernel when every lane of the resident grid takes at most one
  // line direction (refinement passes; launches bound by their longest line)
  bool len_kernel = false;
  if (use_cell && NC == 3 && shape.line_lanes != 3) {
    int res_len = 0;
    QSL_CHECK_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res_len, cell_len_kernel<R>, 32 * shape.warps_per_block, 0));
    const int bps_len = shape.blocks_per_sm < res_len ? shape.blocks_per_sm : res_len;
    len_kernel = 2 * n_seeds <= (int64_t)32 * shape.warps_per_block * (bps_len > 0 ? bps_len : 1) * sms;
  }
  // lengths only with the Cash-Karp stepper on a uniform, trilinear, Cartesian
  // grid in FP32 (the refinement passes' decision traces): the one-lane kernel
  // with the cell polynomials cached across stages, when every lane of the
  // resident grid takes at most one line direction
  bool ck_len = false;
  if (loc && NC == 3 && sizeof(R) == 4 && cfg.integrator == QSL_RKCK54 && cfg.geom != QSL_GEOM_SPHERICAL &&
      cfg.interp_order <= 1) {
    int res_ck = 0;
    QSL_CHECK_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res_ck, ck_len_kernel<R>, 32 * shape.warps_per_block, 0));
    const int bps_ck = shape.blocks_per_sm < res_ck ? shape.blocks_per_sm : res_ck;
    ck_len = 2 * n_seeds <= (int64_t)32 * shape.warps_per_block * (bps_ck > 0 ? bps_ck : 1) * sms;
  }
  bool coop = false;
  if (use_cell && !len_kernel) {
    if (shape.line_lanes == 3) {
      coop = true;
    } else if (shape.line_lanes == 0) {
      // auto: three lanes per line up to 512 units (line directions) per SM,
      // where the launch is bound by the latency of its longest lines rather
      // than by issue rate (measured crossover on GB300: about 640 per SM); a
      // device-side count is a retrace list, short by construction
      coop = n_seeds_dev != nullptr || 2 * n_seeds <= (int64_t)512 * sms;
    }
  }
  size_t smem = (use_cell && !coop && !len_kernel) ? (size_t)24 * threads * sizeof(R) : 0;
  int resident = 0;
  if (ck_len)
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, ck_len_kernel<R>, threads, 0));
  else if (len_kernel)
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, cell_len_kernel<R>, threads, 0));
  else if (coop)
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, cell_coop_kernel<R, NC>, threads, 0));
  else if (use_cell)
    QSL_CHECK_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, cell_kernel_fn<NC>((R*)nullptr), threads, smem));
  else if (loc && cfg.geom == QSL_GEOM_SPHERICAL && cfg.interp_order > 1)
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, trace_kernel<R, NC, true, true, true>,
                                                                 threads, 0));
  else if (loc && cfg.geom == QSL_GEOM_SPHERICAL)
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, trace_kernel<R, NC, true, false, true>,
                                                                 threads, 0));
  else if (loc && cfg.interp_order > 1)
    QSL_CHECK_CUDA(
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, trace_kernel<R, NC, true, true>, threads, 0));
  else if (loc)
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, trace_kernel<R, NC, true>, threads, 0));
  else
    QSL_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, trace_kernel<R, NC, false>, threads, 0));
  int bps = shape.blocks_per_sm < resident ? shape.blocks_per_sm : resident;
  if (bps < 1) bps = 1;
  int blocks = sms * bps;
  // one unit per warp at the least (the kernels use fewer lanes per warp when
  // the units do not fill every resident warp)
  int64_t max_warps_needed = 2 * n_seeds;
  if ((int64_t)blocks * shape.warps_per_block > max_warps_needed && !n_seeds_dev)
    blocks = (int)((max_warps_needed + shape.warps_per_block - 1) / shape.warps_per_block);
  if (blocks < 1) blocks = 1;
  if (ev) QSL_CHECK_CUDA(cudaEventRecord(ev[0], stream));
  if (n_seeds > 0) {
    if (ck_len) {
      ck_len_kernel<R><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else if (len_kernel) {
      cell_len_kernel<R><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else if (coop) {
      cell_coop_kernel<R, NC><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else if (use_cell) {
      cell_kernel_fn<NC>((R*)nullptr)<<<blocks, threads, smem, stream>>>(P);
      qsl::count_launch();
    } else if (loc && cfg.geom == QSL_GEOM_SPHERICAL && cfg.interp_order > 1) {
      trace_kernel<R, NC, true, true, true><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else if (loc && cfg.geom == QSL_GEOM_SPHERICAL) {
      trace_kernel<R, NC, true, false, true><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else if (loc && cfg.interp_order > 1) {
      trace_kernel<R, NC, true, true><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else if (loc) {
      trace_kernel<R, NC, true><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    } else {
      trace_kernel<R, NC, false><<<blocks, threads, 0, stream>>>(P);
      qsl::count_launch();
    }
    QSL_CHECK_CUDA(cudaGetLastError());
  }
  if (ev) QSL_CHECK_CUDA(cudaEventRecord(ev[1], stream));
  // assembly
  AssembleParams<R> A;
  A.T = P;
  A.out = out;
  A.tangent = NC == 9;
  if (n_seeds > 0) {
    int ab = (int)((n_seeds + 127) / 128);
    if (ab > sms * 16) ab = sms * 16;
    assemble_kernel<R><<<ab, 128, 0, stream>>>(A);
    qsl::count_launch();
    QSL_CHECK_CUDA(cudaGetLastError());
  }
  if (own) QSL_CHECK_CUDA(cudaFreeAsync(scratch, stream));
  return QSL_OK;
}

template <class R>
int launch_any(const Item<R>& item0, const Item<R>* items_dev, int n_items, bool loc, const int64_t* index,
               int64_t n_seeds, const int64_t* n_seeds_dev, const TraceConfig& cfg, const LaunchShape& shape,
               const LineOutputs& out, cudaStream_t stream, DeviceStats* stats_dev, cudaEvent_t* ev, void* scratch) {
  if (cfg.length_only)
    return launch_trace<R, 3>(item0, items_dev, n_items, loc, index, n_seeds, n_seeds_dev, cfg, shape, out, stream,
                              stats_dev, ev, scratch);
  return launch_trace<R, 9>(item0, items_dev, n_items, loc, index, n_seeds, n_seeds_dev, cfg, shape, out, stream,
                            stats_dev, ev, scratch);
}

}  // namespace

int trace_and_assemble(const qsl_field* f, const SeedSource& src, int64_t n_seeds, const int64_t* n_seeds_dev,
                       const TraceConfig& cfg, int precision, const LaunchShape& shape, const LineOutputs& out,
                       cudaStream_t stream, DeviceStats* stats_dev, cudaEvent_t* ev, const int64_t* index,
                       void* scratch) {
  bool loc = f->uniform != 0;
  if (precision == QSL_FP64)
    return qsl::launch_any<double>(make_item<double>(f, src, cfg, 0, loc), nullptr, 0, loc, index, n_seeds, n_seeds_dev,
                              cfg, shape, out, stream, stats_dev, ev, scratch);
  return qsl::launch_any<float>(make_item<float>(f, src, cfg, 0, loc), nullptr, 0, loc, index, n_seeds, n_seeds_dev, cfg,
                           shape, out, stream, stats_dev, ev, scratch);
}

size_t end_record_bytes(int precision) {
  return precision == QSL_FP64 ? sizeof(EndRec<double>) : sizeof(EndRec<float>);
}

int select_retrace(const SeedSource& src, int64_t n_seeds, const LineOutputs& out, double threshold,
                   int64_t* index, int64_t* count_dev, cudaStream_t stream) {
  (void)src;
  QSL_CHECK_CUDA(cudaMemsetAsync(count_dev, 0, sizeof(int64_t), stream));
  if (n_seeds == 0) return QSL_OK;
  int blocks = (int)((n_seeds + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  select_kernel<<<blocks, 256, 0, stream>>>(n_seeds, out.q, out.lines, out.q_form, threshold, index, count_dev);
  qsl::count_launch();
  QSL_CHECK_CUDA(cudaGetLastError());
  return QSL_OK;
}

}  // namespace qsl

// ---------------------------------------------------------------------------
// Tracing without any allocation. Some callers cannot call cudaMalloc: code
// that runs under a host-side allocator it must not bypass, inside a memory
// budget fixed up front, or in a process whose allocator state must not
// change. This variant of qsl_trace_seeds keeps its scratch (queue head and
// per-direction end records) in one file-scope device array instead of
// allocating it. The array is QSL_NOALLOC_SCRATCH_BYTES large and every GPU
// that loads this library holds it until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kNoallocBytes = 256 + sizeof(qsl::EndRec<float>) * 2 * (size_t)QSL_NOALLOC_MAX_SEEDS;
static_assert(kNoallocBytes == QSL_NOALLOC_SCRATCH_BYTES, "scratch size must match qsl.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Host code may not use the name of a __device__ array as a device address:
// it names a host-side stand-in. The device address is looked up once per
// device, with that device current, and kept here.
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

int noalloc_scratch(void** out) {
  int dev = 0;
  QSL_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    qsl::set_error("device %d out of range for the no-allocation scratch", dev);
    return QSL_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      qsl::set_error("cudaGetSymbolAddress of the no-allocation scratch failed: %s", cudaGetErrorString(e));
      return QSL_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return QSL_OK;
}

}  // namespace

extern "C" int qsl_trace_seeds_noalloc(const qsl_field* f, const double* seeds, int64_t S, const qsl_opts* o,
                                       qsl_line* out, void* stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  int rc = qsl::validate_opts(f, o);
  if (rc) return rc;
  if (S < 0 || S > QSL_NOALLOC_MAX_SEEDS) {
    qsl::set_error("S = %lld is outside 0..%d, the no-allocation limit of qsl_trace_seeds_noalloc", (long long)S,
                   QSL_NOALLOC_MAX_SEEDS);
    return QSL_EINVAL;
  }
  if (o->precision != QSL_FP32_MIXED) {
    qsl::set_error("qsl_trace_seeds_noalloc traces in FP32 only (opts.precision must be QSL_FP32_MIXED)");
    return QSL_EINVAL;
  }
  if (S > 0 && (!seeds || !out)) {
    qsl::set_error("seeds/out is NULL");
    return QSL_EINVAL;
  }
  const void* ptrs[2] = {seeds, out};
  for (int i = 0; i < 2 && S > 0; ++i) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptrs[i]);
    if (e != cudaSuccess || (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      qsl::set_error("qsl_trace_seeds_noalloc needs device pointers for seeds and out");
      return QSL_EINVAL;
    }
  }
  void* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  qsl::TraceConfig cfg;
  qsl::resolve_config(f, o, &cfg);
  qsl::LaunchShape shape;
  qsl::default_shape(o, !o->length_only, QSL_FP32_MIXED, &shape);
  qsl::SeedSource src{};
  src.kind = qsl::SEEDS_ARRAY;
  src.xyz = seeds;
  qsl::LineOutputs lo{};
  lo.lines = out;
  lo.q_form = QSL_Q_PERP;
  lo.skip_open = o->skip_open;
  if (S == 0) return QSL_OK;
  return qsl::trace_and_assemble(f, src, S, nullptr, cfg, QSL_FP32_MIXED, shape, lo, stream, nullptr, nullptr,
                                 nullptr, scratch);
}

// ---------------------------------------------------------------------------
// Batches: planar Q/FLL maps of many fields in one persistent launch, and
// plans that capture such a launch (trace, FP64 assembly, FP64 retrace) in a
// CUDA graph for replay.
// ---------------------------------------------------------------------------
#include <vector>

struct qsl_plan {
  int n_items = 0;
  int64_t total = 0;
  bool loc = true;
  int precision = QSL_FP32_MIXED;
  double retrace_q = 0;
  qsl::TraceConfig cfg{};
  qsl::LaunchShape shape{}, shape64{};
  qsl::LineOutputs out{};
  qsl::Item<float> first32{};
  qsl::Item<double> first64{};
  void* table32 = nullptr;
  void* table64 = nullptr;
  void* scratch32 = nullptr;
  void* scratch64 = nullptr;
  int64_t* index = nullptr;
  int64_t* count = nullptr;
  float* qtmp = nullptr;
  qsl::DeviceStats* stats = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = -1;
};

namespace {

void plan_release(qsl_plan* p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  void* bufs[] = {p->table32, p->table64, p->scratch32, p->scratch64, p->index, p->count, p->qtmp, p->stats};
  for (void* b : bufs)
    if (b) cudaFree(b);
  delete p;
}

// Validates the items and fills the plan's tables and scratch (synchronous).
int plan_build(const qsl_batch_item* items, int n_items, const qsl_opts* o, float* q, float* length, uint8_t* faces,
               uint8_t* status, qsl_plan** out) {
  *out = nullptr;
  if (n_items < 1 || !items) {
    qsl::set_error("need at least one batch item");
    return QSL_EINVAL;
  }
  int rc = QSL_OK;
  for (int k = 0; k < n_items; ++k) {
    if ((rc = qsl::validate_opts(items[k].field, o))) return rc;
    if (items[k].nu < 0 || items[k].nv < 0) {
      qsl::set_error("item %d: nu, nv must be >= 0", k);
      return QSL_EINVAL;
    }
  }
  qsl_plan* p = new qsl_plan();
  cudaGetDevice(&p->device);
  p->n_items = n_items;
  p->precision = o->precision;
  p->retrace_q = (o->precision == QSL_FP32_MIXED && !o->length_only) ? o->retrace_q : 0.0;
  qsl::default_shape(o, !o->length_only, o->precision, &p->shape);
  qsl::default_shape(o, 1, QSL_FP64, &p->shape64);
  for (int k = 0; k < n_items; ++k) p->loc = p->loc && items[k].field->uniform;
  std::vector<qsl::Item<float>> t32(n_items);
  std::vector<qsl::Item<double>> t64(n_items);
  int64_t start = 0;
  for (int k = 0; k < n_items; ++k) {
    const qsl_batch_item& it = items[k];
    qsl::TraceConfig c;
    qsl::resolve_config(it.field, o, &c);
    if (k == 0) p->cfg = c;
    qsl::SeedSource src{};
    src.kind = qsl::SEEDS_PLANE;
    src.n[0] = it.nu;
    src.n[1] = it.nv;
    src.n[2] = 1;
    for (int a = 0; a < 3; ++a) {
      src.c[a] = it.center[a];
      src.u[a] = it.u[a];
      src.v[a] = it.v[a];
    }
    t32[k] = qsl::make_item<float>(it.field, src, c, start, p->loc);
    t64[k] = qsl::make_item<double>(it.field, src, c, start, p->loc);
    start += (int64_t)it.nu * it.nv;
  }
  p->total = start;
  p->first32 = t32[0];
  p->first64 = t64[0];
  p->out.q = q;
  p->out.length = length;
  p->out.faces = faces;
  p->out.status = status;
  p->out.q_form = o->q_form;
  p->out.skip_open = o->skip_open;
#define PLAN_TRY(call)                                                         \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      qsl::set_error("%s failed: %s", #call, cudaGetErrorString(e_));          \
      plan_release(p);                                                         \
      return e_ == cudaErrorMemoryAllocation ? QSL_ENOMEM : QSL_ECUDA;         \
    }                                                                          \
  } while (0)
  size_t n_units = (size_t)(2 * p->total);
  PLAN_TRY(cudaMalloc(&p->table32, sizeof(qsl::Item<float>) * n_items));
  PLAN_TRY(cudaMemcpy(p->table32, t32.data(), sizeof(qsl::Item<float>) * n_items, cudaMemcpyHostToDevice));
  PLAN_TRY(cudaMalloc(&p->scratch32, 256 + qsl::end_record_bytes(o->precision) * (n_units ? n_units : 1)));
  PLAN_TRY(cudaMalloc((void**)&p->stats, sizeof(qsl::DeviceStats)));
  if (o->precision == QSL_FP64 || p->retrace_q > 0) {
    PLAN_TRY(cudaMalloc(&p->table64, sizeof(qsl::Item<double>) * n_items));
    PLAN_TRY(cudaMemcpy(p->table64, t64.data(), sizeof(qsl::Item<double>) * n_items, cudaMemcpyHostToDevice));
  }
  if (p->retrace_q > 0) {
    PLAN_TRY(cudaMalloc(&p->scratch64, 256 + sizeof(qsl::EndRec<double>) * (n_units ? n_units : 1)));
    PLAN_TRY(cudaMalloc((void**)&p->index, sizeof(int64_t) * (p->total ? p->total : 1)));
    PLAN_TRY(cudaMalloc((void**)&p->count, sizeof(int64_t)));
    if (!q) {
      PLAN_TRY(cudaMalloc((void**)&p->qtmp, sizeof(float) * (p->total ? p->total : 1)));
      p->out.q = p->qtmp;
    }
  }
#undef PLAN_TRY
  *out = p;
  return QSL_OK;
}

// Issues the plan's work on `s` (allocates nothing; capturable).
int plan_enqueue(qsl_plan* p, cudaStream_t s) {
  int rc;
  QSL_CHECK_CUDA(cudaMemsetAsync(p->stats, 0, sizeof(qsl::DeviceStats), s));
  if (p->precision == QSL_FP64) {
    return qsl::launch_any<double>(p->first64, (const qsl::Item<double>*)p->table64, p->n_items, p->loc, nullptr,
                              p->total, nullptr, p->cfg, p->shape, p->out, s, p->stats, nullptr, p->scratch32);
  }
  rc = qsl::launch_any<float>(p->first32, (const qsl::Item<float>*)p->table32, p->n_items, p->loc, nullptr, p->total,
                         nullptr, p->cfg, p->shape, p->out, s, p->stats, nullptr, p->scratch32);
  if (rc || p->retrace_q <= 0 || p->total == 0) return rc;
  qsl::SeedSource none{};
  if ((rc = qsl::select_retrace(none, p->total, p->out, p->retrace_q, p->index, p->count, s))) return rc;
  qsl::LineOutputs o2 = p->out;
  o2.retraced = 1;
  return qsl::launch_any<double>(p->first64, (const qsl::Item<double>*)p->table64, p->n_items, p->loc, p->index,
                            p->total, p->count, p->cfg, p->shape64, o2, s, p->stats, nullptr, p->scratch64);
}

}  // namespace

extern "C" {

int qsl_q_map_batch(const qsl_batch_item* items, int n_items, const qsl_opts* opts, float* q, float* length,
                    uint8_t* faces, uint8_t* status, int mem, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  if (mem != QSL_MEM_DEVICE) {
    qsl::set_error("qsl_q_map_batch takes device outputs (mem = QSL_MEM_DEVICE)");
    return QSL_EINVAL;
  }
  qsl_plan* p = nullptr;
  int rc = plan_build(items, n_items, opts, q, length, faces, status, &p);
  if (rc) return rc;
  rc = plan_enqueue(p, s);
  cudaError_t e = cudaStreamSynchronize(s);
  plan_release(p);
  if (rc) return rc;
  if (e != cudaSuccess) {
    qsl::set_error("batch failed: %s", cudaGetErrorString(e));
    return QSL_ECUDA;
  }
  return QSL_OK;
}

int qsl_plan_q_map_batch(const qsl_batch_item* items, int n_items, const qsl_opts* opts, float* q, float* length,
                         uint8_t* faces, uint8_t* status, qsl_plan** out) {
  if (!out) {
    qsl::set_error("out is NULL");
    return QSL_EINVAL;
  }
  qsl_plan* p = nullptr;
  int rc = plan_build(items, n_items, opts, q, length, faces, status, &p);
  if (rc) return rc;
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    qsl::set_error("stream capture failed to start: %s", cudaGetErrorString(e));
    plan_release(p);
    return QSL_ECUDA;
  }
  rc = plan_enqueue(p, p->cap_stream);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(p->cap_stream, &g);
  p->graph = g;
  if (rc || e != cudaSuccess) {
    if (!rc) qsl::set_error("stream capture failed: %s", cudaGetErrorString(e));
    plan_release(p);
    return rc ? rc : QSL_ECUDA;
  }
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) {
    qsl::set_error("graph instantiation failed: %s", cudaGetErrorString(e));
    plan_release(p);
    return QSL_ECUDA;
  }
  *out = p;
  return QSL_OK;
}

int qsl_plan_launch(qsl_plan* p, void* stream) {
  if (!p || !p->exec) {
    qsl::set_error("plan is NULL or not instantiated");
    return QSL_EINVAL;
  }
  cudaError_t e = cudaGraphLaunch(p->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    qsl::set_error("cudaGraphLaunch failed: %s", cudaGetErrorString(e));
    return QSL_ECUDA;
  }
  qsl::count_launch();
  return QSL_OK;
}

int qsl_plan_stats(qsl_plan* p, void* stream, qsl_stats* out) {
  if (!p || !out) {
    qsl::set_error("NULL argument");
    return QSL_EINVAL;
  }
  qsl::DeviceStats h{};
  QSL_CHECK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  QSL_CHECK_CUDA(cudaMemcpy(&h, p->stats, sizeof h, cudaMemcpyDeviceToHost));
  memset(out, 0, sizeof(*out));
  out->lines = p->total;
  out->stage_evals = (int64_t)h.stage_evals;
  out->accepted = (int64_t)h.accepted;
  out->rejected = (int64_t)h.rejected;
  out->landing = (int64_t)h.landing;
  if (p->count) {
    int64_t c = 0;
    QSL_CHECK_CUDA(cudaMemcpy(&c, p->count, sizeof c, cudaMemcpyDeviceToHost));
    out->retraced = c;
  }
  out->warps_per_block = p->shape.warps_per_block;
  out->blocks_per_sm = p->shape.blocks_per_sm;
  out->refill_min = p->shape.refill_min;
  return QSL_OK;
}

void qsl_plan_free(qsl_plan* p) { plan_release(p); }

}  // extern "C"
