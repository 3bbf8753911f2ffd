// QSL oracle: a plain, slow, FP64 CPU restatement of the QSL Squasher method
// (Tassev & Savcheva, arXiv:1609.00724).
//
// This file is TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the
// CPU-baseline leg of the benchmark load it. It shares no source, header, table or
// helper with the CUDA library; the two only see the same synthetic inputs.
//
// Every function names the passage of the paper it follows. Where the paper is
// silent, the reading taken is stated next to the code.
//
// Parity pins (tests/test_oracle_*.py): closed forms of the linear hyperbolic
// field, Q >= 2, flux conservation, equal Q from either footpoint and from a
// mid-line seed, Pariat-style finite-difference Q on tiny charge fields, the
// Cash-Karp order test, Hilbert bijection/adjacency, Sobel ramp constants,
// refinement special cases (tau = 0 gives the dense lattice; a step in L refines
// only along the step) and the converter on hand-made samples.
// Parity unpinned: which boundary set FLEDGE "should" find, and the value of tau.

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

const double NaN = std::numeric_limits<double>::quiet_NaN();

// ---------------------------------------------------------------------------
// Options (same meaning as the library's options; defined here independently)
// ---------------------------------------------------------------------------
struct Opts {
  int integrator;   // 0 = adaptive Cash-Karp 5(4) (Sec. "Integration methods"), 1 = fixed-step Euler
  int length_only;  // 1: integrate x only (FLEDGE fast path, Sec. "Illustrative examples" footnote)
  int skip_open;    // 1: open lines get Q = NaN (Sec. "Squashing factor calculation")
  int pad0;
  double tol_abs, tol_rel;  // step-error tolerances (the paper quotes 1e-2)
  double h_init, h_max, h_min;  // in units of the smallest grid spacing
  double max_length;        // <= 0: 20 x domain diagonal (fixed-maximum-length option)
  double max_steps;         // step attempts per direction
  double euler_h;           // Euler step in cells (paper: about 1/5)
  double lo[3], hi[3];      // tracing domain; lo >= hi means "grid extent"
  double land_tol;          // face landing tolerance in cells
  int nthreads;
  int pad1;
};

struct Field {
  int n[3];
  std::vector<double> c[3];  // per-axis vertex coordinates (rectilinear grid)
  std::vector<double> v;     // 4 doubles per vertex, x fastest
  int mode;                  // 0 = paper (normalise first), 1 = raw B
  double glo[3], ghi[3];
  double cell;               // smallest grid spacing over all axes
  int order = 1;             // interpolation: 1 trilinear, 2 triquadratic, 3 tricubic (uniform grids)
  int geom = 0;              // 0 Cartesian; 1 spherical: axes (phi, theta, r) = longitude, latitude
                             // (radians) and radius, field components in (phi^, theta^, r^)
  double cell_q = 0;         // smallest coordinate spacing (landing tolerance)
};

// Scale factors of the coordinates at point q: a coordinate displacement dq_i
// is a physical length m_i dq_i. Cartesian: 1; spherical (Sec. "Integrating
// field lines", Eq. fl_sph): (r cos(theta), r, 1).
inline void metric(const Field& F, const double* q, double* m) {
  if (F.geom == 1) {
    m[0] = q[2] * std::cos(q[1]);
    m[1] = q[2];
    m[2] = 1.0;
  } else {
    m[0] = m[1] = m[2] = 1.0;
  }
}

struct Stats {
  double stage_evals = 0, accepted = 0, rejected = 0, landing = 0;
};

// Line status codes (one per direction).
enum { ST_OK = 0, ST_MAXLEN = 1, ST_MAXSTEPS = 2, ST_STALL = 3, ST_OUTSIDE = 4, ST_NONFINITE = 5, ST_NULL = 6 };
const int NO_FACE = 255;

// ---------------------------------------------------------------------------
// Field packing (Sec. "Squashing factor calculation", footnote on normalising
// the field cubes before interpolation).
// paper mode: each vertex holds (B/|B|, |B|); a zero vertex holds (0,0,0,0).
// raw mode:   each vertex holds (B, |B|).
// ---------------------------------------------------------------------------
void pack_field(Field& F, const double* bx, const double* by, const double* bz) {
  size_t N = (size_t)F.n[0] * F.n[1] * F.n[2];
  F.v.assign(4 * N, 0.0);
  for (size_t i = 0; i < N; ++i) {
    double B[3] = {bx[i], by[i], bz[i]};
    double m = std::sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    for (int a = 0; a < 3; ++a) {
      if (F.mode == 0)
        F.v[4 * i + a] = (m > 0) ? B[a] / m : 0.0;
      else
        F.v[4 * i + a] = B[a];
    }
    F.v[4 * i + 3] = m;
  }
}

// ---------------------------------------------------------------------------
// Cell location (Sec. "Interpolation schemes"): c is the vertex of the cell
// containing x that lies closest to the array origin. Reading: the index is
// clamped to [0, n-2], so points on (or, during a trial step, beyond) the last
// vertex use the last cell and the kernels extrapolate linearly.
// ---------------------------------------------------------------------------
void locate(const Field& F, int a, double x, int* idx, double* frac, double* h) {
  const std::vector<double>& c = F.c[a];
  int n = F.n[a];
  int i;
  if (x <= c[0]) {
    i = 0;
  } else if (x >= c[n - 1]) {
    i = n - 2;
  } else {
    int lo = 0, hi = n - 1;  // invariant c[lo] <= x < c[hi]
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      if (c[mid] <= x) lo = mid; else hi = mid;
    }
    i = lo;
  }
  if (i > n - 2) i = n - 2;
  if (i < 0) i = 0;
  *idx = i;
  *h = c[i + 1] - c[i];
  *frac = (x - c[i]) / *h;
}

// Interpolated quantities at a point.
struct Interp {
  double b[3];     // right-hand side of the field-line equation (Eq. fl)
  double g[3][3];  // g[i][j] = d b_i / d x_j  (used by Eq. dev)
  double bmag;     // unnormalised |B| at the point
};

// Higher-order interpolation kernels of Sec. "Interpolation schemes" (the
// paper cites them; written here from their published definitions), as 1D
// weights w_k and dw_k/du for the stencil vertices idx_k along one axis. The
// point lies in cell c at fraction u; s is its offset from a vertex in units of
// the spacing. Stencil vertices beyond the grid are clamped to its edge.
//  order 3, Keys (1981) cubic convolution with a = -1/2, vertices c-1..c+2:
//    W(s) = 1.5|s|^3 - 2.5|s|^2 + 1 (|s| <= 1), -0.5|s|^3 + 2.5|s|^2 - 4|s| + 2
//    (1 < |s| < 2), 0 beyond;
//  order 2, Dodgson (1997) interpolating quadratic, the vertex m nearest the
//  point and its two neighbours:
//    W(s) = 1 - 2 s^2 (|s| <= 1/2), s^2 - 2.5|s| + 1.5 (1/2 < |s| <= 3/2), 0 beyond.
// Returns the number of taps.
int ho_weights(int order, int c, double u, int n, int* idx, double* w, double* dw) {
  if (order == 3) {
    for (int k = 0; k < 4; ++k) {
      double s = u - (k - 1);  // offset from vertex c - 1 + k
      double a = std::fabs(s), sg = s < 0 ? -1.0 : 1.0;
      if (a <= 1) {
        w[k] = 1.5 * a * a * a - 2.5 * a * a + 1;
        dw[k] = sg * (4.5 * a * a - 5 * a);
      } else if (a < 2) {
        w[k] = -0.5 * a * a * a + 2.5 * a * a - 4 * a + 2;
        dw[k] = sg * (-1.5 * a * a + 5 * a - 4);
      } else {
        w[k] = 0;
        dw[k] = 0;
      }
      idx[k] = std::min(std::max(c - 1 + k, 0), n - 1);
    }
    return 4;
  }
  int m = c + (u >= 0.5 ? 1 : 0);
  double t = u - (m - c);
  for (int k = 0; k < 3; ++k) {
    double s = t - (k - 1);  // offset from vertex m - 1 + k
    double a = std::fabs(s), sg = s < 0 ? -1.0 : 1.0;
    if (a <= 0.5) {
      w[k] = 1 - 2 * s * s;
      dw[k] = -4 * s;
    } else if (a <= 1.5) {
      w[k] = a * a - 2.5 * a + 1.5;
      dw[k] = sg * (2 * a - 2.5);
    } else {
      w[k] = 0;
      dw[k] = 0;
    }
    idx[k] = std::min(std::max(m - 1 + k, 0), n - 1);
  }
  return 3;
}

// Interpolation (Eq. interp with the kernels f_v of the field's order) and its
// analytic gradient (the gradient acts on the kernels only, Sec. "Field-line
// deviation using linearization").
void interp(const Field& F, const double* x, Interp* out, Stats* st) {
  if (st) st->stage_evals += 1;
  int ci[3];
  double u[3], h[3];
  for (int a = 0; a < 3; ++a) locate(F, a, x[a], &ci[a], &u[a], &h[a]);
  double val[4] = {0, 0, 0, 0};
  double grad[4][3] = {{0}};
  if (F.order > 1) {
    int idx[3][4];
    double w[3][4], dw[3][4];
    int K = 0;
    for (int a = 0; a < 3; ++a) K = ho_weights(F.order, ci[a], u[a], F.n[a], idx[a], w[a], dw[a]);
    for (int kz = 0; kz < K; ++kz)
      for (int ky = 0; ky < K; ++ky)
        for (int kx = 0; kx < K; ++kx) {
          double f = w[0][kx] * w[1][ky] * w[2][kz];
          double df[3] = {dw[0][kx] * w[1][ky] * w[2][kz] / h[0], w[0][kx] * dw[1][ky] * w[2][kz] / h[1],
                          w[0][kx] * w[1][ky] * dw[2][kz] / h[2]};
          size_t vi = ((size_t)idx[2][kz] * F.n[1] + idx[1][ky]) * F.n[0] + idx[0][kx];
          const double* p = &F.v[4 * vi];
          for (int k = 0; k < 4; ++k) {
            val[k] += p[k] * f;
            for (int j = 0; j < 3; ++j) grad[k][j] += p[k] * df[j];
          }
        }
  } else
  for (int vz = 0; vz < 2; ++vz)
    for (int vy = 0; vy < 2; ++vy)
      for (int vx = 0; vx < 2; ++vx) {
        int v[3] = {vx, vy, vz};
        double w1[3], dw1[3];  // 1D factor and its derivative per axis
        for (int a = 0; a < 3; ++a) {
          w1[a] = v[a] ? u[a] : (1.0 - u[a]);
          dw1[a] = (v[a] ? 1.0 : -1.0) / h[a];
        }
        double f = w1[0] * w1[1] * w1[2];
        double df[3] = {dw1[0] * w1[1] * w1[2], w1[0] * dw1[1] * w1[2], w1[0] * w1[1] * dw1[2]};
        size_t vi = ((size_t)(ci[2] + vz) * F.n[1] + (ci[1] + vy)) * F.n[0] + (ci[0] + vx);
        const double* p = &F.v[4 * vi];
        for (int k = 0; k < 4; ++k) {
          val[k] += p[k] * f;
          for (int j = 0; j < 3; ++j) grad[k][j] += p[k] * df[j];
        }
      }
  if (F.mode == 0) {
    // Paper mode: the interpolated normalised field is used as is (not unit).
    for (int i = 0; i < 3; ++i) {
      out->b[i] = val[i];
      for (int j = 0; j < 3; ++j) out->g[i][j] = grad[i][j];
    }
    out->bmag = val[3];
  } else {
    // Raw mode: interpolate B, then normalise at the point:
    // b = B/|B|,  d b_i/d x_j = (dB_i/dx_j - b_i sum_k b_k dB_k/dx_j) / |B|.
    double m = std::sqrt(val[0] * val[0] + val[1] * val[1] + val[2] * val[2]);
    out->bmag = m;
    if (!(m > 0)) {
      for (int i = 0; i < 3; ++i) {
        out->b[i] = 0;
        for (int j = 0; j < 3; ++j) out->g[i][j] = 0;
      }
      return;
    }
    double b[3] = {val[0] / m, val[1] / m, val[2] / m};
    for (int i = 0; i < 3; ++i) out->b[i] = b[i];
    for (int j = 0; j < 3; ++j) {
      double bd = b[0] * grad[0][j] + b[1] * grad[1][j] + b[2] * grad[2][j];
      for (int i = 0; i < 3; ++i) out->g[i][j] = (grad[i][j] - b[i] * bd) / m;
    }
  }
}

// ---------------------------------------------------------------------------
// Right-hand side: y = (x, dx1, dx2); dy/dl = s * (b(x), G dx1, G dx2)
// (Eq. fl and Eq. dev; s = +1 forward to lambda_F, -1 backward to lambda_B).
// ---------------------------------------------------------------------------
// Spherical geometry: Eq. fl_sph for the position, and Eq. dev_sph (the
// paper's form, which leaves out the terms of the metric factors' variation)
// for the coordinate deviations: m_i d(dq_i)/dl = sum_j (d b_i / d q_j) dq_j.
void rhs(const Field& F, int s, int ncomp, const double* y, double* dy, Stats* st) {
  Interp I;
  interp(F, y, &I, st);
  double m[3];
  metric(F, y, m);
  for (int i = 0; i < 3; ++i) dy[i] = s * I.b[i] / m[i];
  if (ncomp == 9) {
    for (int v = 0; v < 2; ++v) {
      const double* d = y + 3 + 3 * v;
      for (int i = 0; i < 3; ++i)
        dy[3 + 3 * v + i] = s * (I.g[i][0] * d[0] + I.g[i][1] * d[1] + I.g[i][2] * d[2]) / m[i];
    }
  }
}

// Cash & Karp (1990) embedded Runge-Kutta 5(4) tableau (the stepper the paper
// uses through Boost.odeint, Sec. "Integration methods"). Written from the
// published coefficients; the order test pins it.
const double CK_C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0, 7.0 / 8.0};
const double CK_A[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0}};
const double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0, 512.0 / 1771.0};
const double CK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0, 13525.0 / 55296.0, 277.0 / 14336.0, 1.0 / 4.0};

// One Cash-Karp step of size h from y: fifth-order solution in ynew, the
// difference to the embedded fourth-order solution in yerr.
void ck_step(const Field& F, int s, int ncomp, const double* y, double h, double* ynew, double* yerr,
             Stats* st) {
  double k[6][9], yt[9];
  for (int stage = 0; stage < 6; ++stage) {
    for (int i = 0; i < ncomp; ++i) {
      double acc = 0;
      for (int j = 0; j < stage; ++j) acc += CK_A[stage][j] * k[j][i];
      yt[i] = y[i] + h * acc;
    }
    rhs(F, s, ncomp, yt, k[stage], st);
  }
  for (int i = 0; i < ncomp; ++i) {
    double s5 = 0, s4 = 0;
    for (int j = 0; j < 6; ++j) {
      s5 += CK_B5[j] * k[j][i];
      s4 += CK_B4[j] * k[j][i];
    }
    ynew[i] = y[i] + h * s5;
    yerr[i] = h * (s5 - s4);
  }
}

// Fixed-step explicit Euler (Sec. "Integration methods").
void euler_step(const Field& F, int s, int ncomp, const double* y, double h, double* ynew, Stats* st) {
  double k[9];
  rhs(F, s, ncomp, y, k, st);
  for (int i = 0; i < ncomp; ++i) ynew[i] = y[i] + h * k[i];
}

void any_step(const Field& F, const Opts& o, int s, int ncomp, const double* y, double h, double* ynew,
              double* yerr, Stats* st) {
  if (o.integrator == 1) {
    euler_step(F, s, ncomp, y, h, ynew, st);
    for (int i = 0; i < ncomp; ++i) yerr[i] = 0;
  } else {
    ck_step(F, s, ncomp, y, h, ynew, yerr, st);
  }
}

// Outward signed distance of x from face f (0..5 = x-, x+, y-, y+, z-, z+).
inline double face_g(const double* lo, const double* hi, int f, const double* x) {
  int a = f >> 1;
  return (f & 1) ? (x[a] - hi[a]) : (lo[a] - x[a]);
}

struct End {
  double y[9];
  double mu;  // |lambda| travelled in this direction
  int face;
  int status;
  double steps;
};

// Land exactly on the face through which the line leaves the domain
// (Sec. "Squashing factor calculation": lines are followed until they reach the
// boundary). Reading: the exit face is the one crossed first along the chord of
// the accepted step; the step length that puts the line on that face is found
// by Illinois regula falsi on the step size, always stepping from the last
// inside state; if the landed point is outside another face, that face is taken
// instead and the search repeats on the shorter step.
void land(const Field& F, const Opts& o, const double* lo, const double* hi, int s, int ncomp,
          const double* y, double h_full, const double* y_full, End* e, Stats* st) {
  double tol = o.land_tol * (F.geom == 1 ? F.cell_q : F.cell);
  double hi_h = h_full;
  double yhi[9], ym[9], yerr[9];
  std::memcpy(yhi, y_full, sizeof(double) * ncomp);
  double hm = h_full;
  int face = -1;
  for (int round = 0; round < 8; ++round) {
    // exit face: smallest crossing fraction along the chord y -> yhi
    face = -1;
    double tbest = 0;
    for (int f = 0; f < 6; ++f) {
      double g1 = face_g(lo, hi, f, yhi);
      if (!(g1 > 0)) continue;
      double g0 = face_g(lo, hi, f, y);
      double t = g0 / (g0 - g1);
      if (face < 0 || t < tbest) {
        face = f;
        tbest = t;
      }
    }
    if (face < 0) {  // cannot happen: yhi is outside by construction
      std::memcpy(ym, yhi, sizeof(double) * ncomp);
      hm = hi_h;
      break;
    }
    double a = 0.0, b = hi_h;
    double ga = face_g(lo, hi, face, y), gb = face_g(lo, hi, face, yhi);
    if (!(ga < 0.0)) {
      // The step starts on this face (a seed on the face whose field points
      // into the domain) and ends beyond it again: the line's end is the
      // later crossing, not lambda = 0. Halve the step until a point inside
      // brackets that crossing; if none is found the line only grazes the face.
      double hh = hi_h;
      bool found = false;
      for (int k = 0; k < 60 && !found; ++k) {
        hh *= 0.5;
        any_step(F, o, s, ncomp, y, hh, ym, yerr, st);
        if (st) st->landing += 1;
        e->steps += 1;
        double gg = face_g(lo, hi, face, ym);
        if (gg < 0.0) {
          a = hh;
          ga = gg;
          found = true;
        } else {
          b = hh;
          gb = gg;
        }
      }
      if (!found) {
        a = 0.0;
        ga = 0.0;
        b = 0.0;
      }
    }
    int side = 0;
    hm = b;
    std::memcpy(ym, yhi, sizeof(double) * ncomp);
    for (int it = 0; it < 200; ++it) {
      hm = (b > a) ? a + (b - a) * ga / (ga - gb) : a;
      any_step(F, o, s, ncomp, y, hm, ym, yerr, st);
      if (st) st->landing += 1;
      e->steps += 1;
      double gm = face_g(lo, hi, face, ym);
      if (std::fabs(gm) <= tol) break;
      if (gm > 0) {
        b = hm;
        gb = gm;
        if (side == 1) ga *= 0.5;
        side = 1;
      } else {
        a = hm;
        ga = gm;
        if (side == -1) gb *= 0.5;
        side = -1;
      }
    }
    double worst = -1.0;
    for (int f = 0; f < 6; ++f)
      if (f != face) worst = std::max(worst, face_g(lo, hi, f, ym));
    if (worst > tol) {
      hi_h = hm;
      std::memcpy(yhi, ym, sizeof(double) * ncomp);
      continue;
    }
    break;
  }
  int ax = face >> 1;
  ym[ax] = (face & 1) ? hi[ax] : lo[ax];
  std::memcpy(e->y, ym, sizeof(double) * ncomp);
  e->mu += hm;
  e->face = face;
  e->status = ST_OK;
}

// Integrate one direction of one line (Eq. fl + Eq. dev with initial
// conditions Eq. ic) until it reaches a face, the maximum length, or a cutoff.
End trace_dir(const Field& F, const Opts& o, const double* lo, const double* hi, double max_len, int s,
              int ncomp, const double* y0, Stats* st) {
  End e;
  std::memcpy(e.y, y0, sizeof(double) * ncomp);
  e.mu = 0;
  e.face = NO_FACE;
  e.status = ST_OK;
  e.steps = 0;
  // A seed on a face whose field points out of the domain ends this side at
  // once with zero length (the reading of integrating until the line leaves the box).
  {
    Interp I;
    interp(F, y0, &I, nullptr);
    for (int f = 0; f < 6; ++f) {
      if (face_g(lo, hi, f, y0) == 0.0) {
        int a = f >> 1;
        double out = (f & 1) ? s * I.b[a] : -s * I.b[a];
        if (out > 0) {
          e.face = f;
          return e;
        }
      }
    }
  }
  double cell = F.cell;
  bool euler = (o.integrator == 1);
  double h = euler ? o.euler_h * cell : o.h_init * cell;
  double ynew[9], yerr[9];
  for (;;) {
    if (e.steps >= o.max_steps) {
      e.status = ST_MAXSTEPS;
      return e;
    }
    double room = max_len - e.mu;
    if (!(room > 0)) {
      e.status = ST_MAXLEN;
      return e;
    }
    double hcap = euler ? o.euler_h * cell : o.h_max * cell;
    bool capped_by_len = false;
    double hs = std::min(h, hcap);
    if (room <= hs) {
      hs = room;
      capped_by_len = true;
    }
    any_step(F, o, s, ncomp, e.y, hs, ynew, yerr, st);
    e.steps += 1;
    double err = 0;
    bool finite = true;
    if (F.geom == 1) {
      // spherical: errors and magnitudes as physical lengths (positions scaled
      // by the radius, the distance from the centre)
      double m[3];
      metric(F, e.y, m);
      double rr = std::max(std::fabs(e.y[2]), std::fabs(ynew[2]));
      for (int i = 0; i < ncomp; ++i) {
        if (!std::isfinite(ynew[i])) finite = false;
        double mi = m[i % 3];
        double mag = i < 3 ? rr : std::max(std::fabs(e.y[i]), std::fabs(ynew[i])) * mi;
        err = std::max(err, std::fabs(yerr[i]) * mi / (o.tol_abs + o.tol_rel * mag));
      }
    } else {
      for (int i = 0; i < ncomp; ++i) {
        if (!std::isfinite(ynew[i])) finite = false;
        double sc = o.tol_abs + o.tol_rel * std::max(std::fabs(e.y[i]), std::fabs(ynew[i]));
        err = std::max(err, std::fabs(yerr[i]) / sc);
      }
    }
    if (!finite) {
      e.status = ST_NONFINITE;
      return e;
    }
    if (!euler && err > 1.0) {
      if (st) st->rejected += 1;
      h = hs * std::max(0.2, 0.9 * std::pow(err, -0.25));
      if (h < o.h_min * cell) {
        e.status = ST_STALL;
        return e;
      }
      continue;
    }
    if (st) st->accepted += 1;
    bool inside = true;
    for (int f = 0; f < 6; ++f)
      if (face_g(lo, hi, f, ynew) > 0) inside = false;
    if (!inside) {
      land(F, o, lo, hi, s, ncomp, e.y, hs, ynew, &e, st);
      return e;
    }
    std::memcpy(e.y, ynew, sizeof(double) * ncomp);
    e.mu += hs;
    if (capped_by_len) {
      e.status = ST_MAXLEN;
      return e;
    }
    if (!euler) h = hs * ((err == 0.0) ? 5.0 : std::min(5.0, 0.9 * std::pow(err, -0.2)));
  }
}

struct LineOut {
  double q_perp, q_foot, q_det, b0, bf, bb, flux, flux_b;
  double L, lam_f, lam_b;
  double xf[3], xb[3];
  int face_f, face_b, st_f, st_b;
  double steps;
};

inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

void resolve_domain(const Field& F, const Opts& o, double* lo, double* hi, double* max_len) {
  bool use = o.lo[0] < o.hi[0] && o.lo[1] < o.hi[1] && o.lo[2] < o.hi[2];
  for (int a = 0; a < 3; ++a) {
    lo[a] = use ? o.lo[a] : F.glo[a];
    hi[a] = use ? o.hi[a] : F.ghi[a];
  }
  double e[3] = {hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]};
  if (F.geom == 1) {  // physical extents at the outer radius
    e[0] *= hi[2];
    e[1] *= hi[2];
  }
  double d = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
  *max_len = (o.max_length > 0) ? o.max_length : 20.0 * d;
}

// Ends of a line and their contributions to Q.
struct EndQ {
  double bmag;          // unnormalised |B| at the end
  double A, B, C;       // Gram entries of the perpendicular deviations a.a, b.b, a.b
  double cross;         // |a x b| of the perpendicular deviations
  double Af, Bf, Cf;    // Gram entries of the face-projected deviations
  double bn;            // |B . n| at the end face
  bool foot_ok;
};

// Perpendicular projection (Sec. "Squashing factor calculation":
// dx_perp = dx - b(b.dx) with b explicitly normalised) and the footpoint
// projection onto the end face along the field line (reading for Q_foot:
// dx_f = dx - b (dx.n)/(b.n)).
EndQ end_terms(const Field& F, const End& e, bool have_face) {
  EndQ r;
  Interp I;
  interp(F, e.y, &I, nullptr);
  r.bmag = I.bmag;
  double m = std::sqrt(dot3(I.b, I.b));
  double u[3] = {I.b[0] / m, I.b[1] / m, I.b[2] / m};
  double ap[3], bp[3];
  // deviations as physical vectors in the end's orthonormal frame
  double sf[3], d1[3], d2[3];
  metric(F, e.y, sf);
  for (int i = 0; i < 3; ++i) {
    d1[i] = e.y[3 + i] * sf[i];
    d2[i] = e.y[6 + i] * sf[i];
  }
  double ud1 = dot3(u, d1), ud2 = dot3(u, d2);
  for (int i = 0; i < 3; ++i) {
    ap[i] = d1[i] - u[i] * ud1;
    bp[i] = d2[i] - u[i] * ud2;
  }
  r.A = dot3(ap, ap);
  r.B = dot3(bp, bp);
  r.C = dot3(ap, bp);
  double cr[3];
  cross3(ap, bp, cr);
  r.cross = std::sqrt(dot3(cr, cr));
  r.foot_ok = false;
  r.Af = r.Bf = r.Cf = r.bn = NaN;
  if (have_face && e.face != NO_FACE) {
    int a = e.face >> 1;
    if (u[a] != 0.0) {
      double af[3], bf[3];
      for (int i = 0; i < 3; ++i) {
        af[i] = d1[i] - u[i] * (d1[a] / u[a]);
        bf[i] = d2[i] - u[i] * (d2[a] / u[a]);
      }
      r.Af = dot3(af, af);
      r.Bf = dot3(bf, bf);
      r.Cf = dot3(af, bf);
      r.bn = I.bmag * std::fabs(u[a]);
      r.foot_ok = true;
    }
  }
  return r;
}

// One seed: orthonormal initial deviations (Eq. ic), both directions, and the
// squashing factor by Eq. finalQ.
LineOut trace_line(const Field& F, const Opts& o, const double* x0, Stats* st) {
  LineOut r;
  double lo[3], hi[3], max_len;
  resolve_domain(F, o, lo, hi, &max_len);
  r.q_perp = r.q_foot = r.q_det = r.b0 = r.bf = r.bb = r.flux = r.flux_b = NaN;
  r.L = r.lam_f = r.lam_b = NaN;
  for (int i = 0; i < 3; ++i) r.xf[i] = r.xb[i] = NaN;
  r.face_f = r.face_b = NO_FACE;
  r.st_f = r.st_b = ST_OK;
  r.steps = 0;
  for (int f = 0; f < 6; ++f) {
    if (!(face_g(lo, hi, f, x0) <= 0)) {
      r.st_f = r.st_b = ST_OUTSIDE;
      return r;
    }
  }
  int ncomp = o.length_only ? 3 : 9;
  double y0[9];
  for (int i = 0; i < 3; ++i) y0[i] = x0[i];
  Interp I0;
  interp(F, x0, &I0, nullptr);
  double m0 = std::sqrt(dot3(I0.b, I0.b));
  r.b0 = I0.bmag;
  if (!(m0 > 0)) {
    r.st_f = r.st_b = ST_NULL;
    return r;
  }
  if (ncomp == 9) {
    // Reading of Eq. ic: the paper leaves (a, b) free up to orthonormality with
    // B(x0). Take e = the axis of the smallest |b0| component (lowest axis on
    // ties), a = normalise(e x b0), b = b0 x a.
    double u0[3] = {I0.b[0] / m0, I0.b[1] / m0, I0.b[2] / m0};
    int ax = 0;
    for (int a = 1; a < 3; ++a)
      if (std::fabs(u0[a]) < std::fabs(u0[ax])) ax = a;
    double e[3] = {0, 0, 0};
    e[ax] = 1;
    double av[3], bv[3];
    cross3(e, u0, av);
    double an = std::sqrt(dot3(av, av));
    for (int i = 0; i < 3; ++i) av[i] /= an;
    cross3(u0, av, bv);
    double m[3];
    metric(F, x0, m);  // physical vectors to coordinate deviations
    for (int i = 0; i < 3; ++i) {
      y0[3 + i] = av[i] / m[i];
      y0[6 + i] = bv[i] / m[i];
    }
  }
  End ef = trace_dir(F, o, lo, hi, max_len, +1, ncomp, y0, st);
  End eb = trace_dir(F, o, lo, hi, max_len, -1, ncomp, y0, st);
  r.st_f = ef.status;
  r.st_b = eb.status;
  r.face_f = ef.face;
  r.face_b = eb.face;
  r.steps = ef.steps + eb.steps;
  r.lam_f = ef.mu;
  r.lam_b = -eb.mu;
  r.L = ef.mu + eb.mu;
  for (int i = 0; i < 3; ++i) {
    r.xf[i] = ef.y[i];
    r.xb[i] = eb.y[i];
  }
  if (ncomp == 3) return r;
  bool okf = (ef.status == ST_OK || ef.status == ST_MAXLEN);
  bool okb = (eb.status == ST_OK || eb.status == ST_MAXLEN);
  if (!(okf && okb)) return r;
  EndQ qf = end_terms(F, ef, ef.status == ST_OK);
  EndQ qb = end_terms(F, eb, eb.status == ST_OK);
  r.bf = qf.bmag;
  r.bb = qb.bmag;
  double bracket = qf.A * qb.B + qb.A * qf.B - 2.0 * qb.C * qf.C;
  // Eq. finalQ
  r.q_perp = (r.bf * r.bb) / (r.b0 * r.b0) * bracket;
  // Same bracket over the true determinant of the Gram matrices (equal to
  // Eq. finalQ when flux is conserved exactly; >= 2 by construction).
  double detf = qf.A * qf.B - qf.C * qf.C, detb = qb.A * qb.B - qb.C * qb.C;
  r.q_det = bracket / std::sqrt(detf * detb);
  // Flux through the deviation parallelogram at the forward end, relative to
  // the seed (|a x b| = 1 there).
  r.flux = (r.bf / r.b0) * qf.cross - 1.0;
  r.flux_b = (r.bb / r.b0) * qb.cross - 1.0;
  if (qf.foot_ok && qb.foot_ok) {
    double bracket_f = qf.Af * qb.Bf + qb.Af * qf.Bf - 2.0 * qb.Cf * qf.Cf;
    r.q_foot = (qf.bn * qb.bn) / (r.b0 * r.b0) * bracket_f;
  }
  if (o.skip_open) {
    bool closed = (ef.status == ST_OK && eb.status == ST_OK && ef.face == 4 && eb.face == 4);
    if (!closed) r.q_perp = r.q_foot = r.q_det = NaN;
  }
  return r;
}

template <class Fn>
void parallel_for(int64_t n, int nthreads, Fn fn) {
  if (nthreads <= 0) nthreads = (int)std::thread::hardware_concurrency();
  if (nthreads <= 0) nthreads = 1;
  std::atomic<int64_t> next(0);
  const int64_t chunk = 64;
  auto worker = [&]() {
    for (;;) {
      int64_t b = next.fetch_add(chunk);
      if (b >= n) break;
      int64_t e = std::min(n, b + chunk);
      for (int64_t i = b; i < e; ++i) fn(i);
    }
  };
  if (nthreads == 1) {
    worker();
    return;
  }
  std::vector<std::thread> ts;
  for (int t = 0; t < nthreads; ++t) ts.emplace_back(worker);
  for (auto& t : ts) t.join();
}

// ---------------------------------------------------------------------------
// Hilbert curve (Sec. "Adaptive refinements"): Skilling (2004) "transpose"
// method, n dimensions, b bits per axis; the curve starts at the origin.
// The key's bits interleave the transposed words, most significant first,
// with axis 0 taking the highest bit of each group.
// ---------------------------------------------------------------------------
uint64_t hilbert_key(const uint32_t* coords, int ndim, int bits) {
  uint32_t X[3] = {0, 0, 0};
  for (int i = 0; i < ndim; ++i) X[i] = coords[i];
  if (bits > 0) {
    uint32_t top = 1u << (bits - 1);
    // undo the reflections/exchanges, from the top level down
    for (uint32_t q = top; q > 1; q >>= 1) {
      uint32_t p = q - 1;
      for (int i = 0; i < ndim; ++i) {
        if (X[i] & q) {
          X[0] ^= p;
        } else {
          uint32_t t = (X[0] ^ X[i]) & p;
          X[0] ^= t;
          X[i] ^= t;
        }
      }
    }
    // Gray encoding
    for (int i = 1; i < ndim; ++i) X[i] ^= X[i - 1];
    uint32_t t = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
      if (X[ndim - 1] & q) t ^= q - 1;
    for (int i = 0; i < ndim; ++i) X[i] ^= t;
  }
  uint64_t key = 0;
  for (int bit = bits - 1; bit >= 0; --bit)
    for (int i = 0; i < ndim; ++i) key = (key << 1) | ((X[i] >> bit) & 1u);
  return key;
}

void hilbert_coords(uint64_t key, int ndim, int bits, uint32_t* coords) {
  uint32_t X[3] = {0, 0, 0};
  int pos = ndim * bits - 1;
  for (int bit = bits - 1; bit >= 0; --bit)
    for (int i = 0; i < ndim; ++i, --pos) X[i] |= (uint32_t)((key >> pos) & 1u) << bit;
  if (bits > 0) {
    // Gray decoding
    uint32_t t = X[ndim - 1] >> 1;
    for (int i = ndim - 1; i > 0; --i) X[i] ^= X[i - 1];
    X[0] ^= t;
    // redo the exchanges/reflections, from the bottom level up
    uint32_t stop = 2u << (bits - 1);
    for (uint32_t q = 2; q != stop; q <<= 1) {
      uint32_t p = q - 1;
      for (int i = ndim - 1; i >= 0; --i) {
        if (X[i] & q) {
          X[0] ^= p;
        } else {
          uint32_t t2 = (X[0] ^ X[i]) & p;
          X[0] ^= t2;
          X[i] ^= t2;
        }
      }
    }
  }
  for (int i = 0; i < ndim; ++i) coords[i] = X[i];
}

// ---------------------------------------------------------------------------
// FLEDGE (Sec. "Adaptive refinements"): gradient magnitude of the Sobel
// operator applied to the field-line length map. Reading: unnormalised
// separable Sobel (derivative [-1,0,1] along the axis, smoothing [1,2,1] along
// each other axis), half-sample-symmetric ("reflect") boundary, index units.
// Non-finite lengths are replaced by the largest finite length of the map.
// ---------------------------------------------------------------------------
void sobel(const float* L, int ndim, const int64_t* shape, double* out) {
  int64_t n[3] = {1, 1, 1};
  for (int i = 0; i < ndim; ++i) n[i] = shape[i];  // shape[0] is the slowest axis
  // index space: axis 0 slowest
  int64_t N = n[0] * n[1] * n[2];
  double fill = -std::numeric_limits<double>::infinity();
  for (int64_t i = 0; i < N; ++i)
    if (std::isfinite(L[i])) fill = std::max(fill, (double)L[i]);
  if (!std::isfinite(fill)) fill = 0;
  auto at = [&](int64_t i0, int64_t i1, int64_t i2) -> double {
    auto refl = [](int64_t i, int64_t m) {
      if (i < 0) return -i - 1;
      if (i >= m) return 2 * m - i - 1;
      return i;
    };
    i0 = refl(i0, n[0]);
    i1 = refl(i1, n[1]);
    i2 = refl(i2, n[2]);
    double v = L[(i0 * n[1] + i1) * n[2] + i2];
    return std::isfinite(v) ? v : fill;
  };
  const double sm[3] = {1, 2, 1};
  const double dv[3] = {-1, 0, 1};
  for (int64_t i0 = 0; i0 < n[0]; ++i0)
    for (int64_t i1 = 0; i1 < n[1]; ++i1)
      for (int64_t i2 = 0; i2 < n[2]; ++i2) {
        double sum2 = 0;
        for (int ax = 0; ax < ndim; ++ax) {
          double g = 0;
          if (ndim == 2) {
            for (int a = -1; a <= 1; ++a)
              for (int b = -1; b <= 1; ++b) {
                double w = (ax == 0) ? dv[a + 1] * sm[b + 1] : sm[a + 1] * dv[b + 1];
                g += w * at(i0 + a, i1 + b, 0);
              }
          } else {
            for (int a = -1; a <= 1; ++a)
              for (int b = -1; b <= 1; ++b)
                for (int c = -1; c <= 1; ++c) {
                  double wa = (ax == 0) ? dv[a + 1] : sm[a + 1];
                  double wb = (ax == 1) ? dv[b + 1] : sm[b + 1];
                  double wc = (ax == 2) ? dv[c + 1] : sm[c + 1];
                  g += wa * wb * wc * at(i0 + a, i1 + b, i2 + c);
                }
          }
          sum2 += g * g;
        }
        out[(i0 * n[1] + i1) * n[2] + i2] = std::sqrt(sum2);
      }
}

}  // namespace

// ===========================================================================
// Exported C interface (host memory only).
// ===========================================================================
extern "C" {

typedef struct {
  double* q_perp; double* q_foot; double* q_det; double* b0; double* bf; double* bb; double* flux; double* flux_b;
  double* L; double* lam_f; double* lam_b; double* xf; double* xb;
  int32_t* face_f; int32_t* face_b; int32_t* st_f; int32_t* st_b; double* steps;
} qslref_lines;

typedef struct {
  double stage_evals, accepted, rejected, landing;
} qslref_stats;

void qslref_opts_default(Opts* o) {
  std::memset(o, 0, sizeof(Opts));
  o->integrator = 0;
  o->length_only = 0;
  o->skip_open = 0;
  o->tol_abs = 1e-2;
  o->tol_rel = 1e-2;
  o->h_init = 0.1;
  o->h_max = 2.0;
  o->h_min = 1e-15;
  o->max_length = 0;
  o->max_steps = 1e6;
  o->euler_h = 0.2;
  o->land_tol = 1e-12;
  o->nthreads = 0;
}

int qslref_sizeof_opts(void) { return (int)sizeof(Opts); }

// Interpolation order of a loaded field: 1 (trilinear), 2 (triquadratic) or
// 3 (tricubic; orders 2 and 3 need uniform spacing on every axis). Returns 0,
// or -1 for a bad order or a non-uniform grid.
int qslref_set_interp_order(void* field, int order) {
  Field* F = (Field*)field;
  if (order < 1 || order > 3) return -1;
  if (order > 1) {
    for (int a = 0; a < 3; ++a) {
      double h0 = F->c[a][1] - F->c[a][0];
      for (int i = 1; i + 1 < F->n[a]; ++i)
        if (std::fabs((F->c[a][i + 1] - F->c[a][i]) - h0) > 1e-9 * h0) return -1;
    }
  }
  F->order = order;
  return 0;
}

// Geometry of a loaded field: 0 Cartesian, 1 spherical (axes: longitude and
// latitude in radians, radius > 0; latitudes inside (-pi/2, pi/2)). Step sizes
// are physical lengths: the smallest cell edge becomes the smallest of
// r_min cos(theta) h_phi (over the grid's latitudes), r_min h_theta and h_r.
// Returns 0, or -1 for a bad geometry or a grid outside those ranges.
int qslref_set_geometry(void* field, int geom) {
  Field* F = (Field*)field;
  if (geom != 0 && geom != 1) return -1;
  double cq = std::numeric_limits<double>::infinity();
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i + 1 < F->n[a]; ++i) cq = std::min(cq, F->c[a][i + 1] - F->c[a][i]);
  F->cell_q = cq;
  if (geom == 1) {
    double th_lo = F->c[1][0], th_hi = F->c[1][F->n[1] - 1], r_lo = F->c[2][0];
    const double half_pi = 1.5707963267948966;
    if (!(th_lo > -half_pi && th_hi < half_pi && r_lo > 0)) return -1;
    double cmin = std::min(std::cos(th_lo), std::cos(th_hi));
    double c = std::numeric_limits<double>::infinity();
    for (int i = 0; i + 1 < F->n[0]; ++i) c = std::min(c, r_lo * cmin * (F->c[0][i + 1] - F->c[0][i]));
    for (int i = 0; i + 1 < F->n[1]; ++i) c = std::min(c, r_lo * (F->c[1][i + 1] - F->c[1][i]));
    for (int i = 0; i + 1 < F->n[2]; ++i) c = std::min(c, F->c[2][i + 1] - F->c[2][i]);
    F->cell = c;
  } else {
    F->cell = cq;
  }
  F->geom = geom;
  return 0;
}

void* qslref_load_field(const double* bx, const double* by, const double* bz, int nx, int ny, int nz,
                        const double* xc, const double* yc, const double* zc, int mode) {
  if (nx < 2 || ny < 2 || nz < 2) return nullptr;
  Field* F = new Field();
  F->n[0] = nx;
  F->n[1] = ny;
  F->n[2] = nz;
  const double* cs[3] = {xc, yc, zc};
  F->cell = std::numeric_limits<double>::infinity();
  for (int a = 0; a < 3; ++a) {
    F->c[a].assign(cs[a], cs[a] + F->n[a]);
    for (int i = 0; i + 1 < F->n[a]; ++i) {
      double h = F->c[a][i + 1] - F->c[a][i];
      if (!(h > 0)) {
        delete F;
        return nullptr;
      }
      F->cell = std::min(F->cell, h);
    }
    F->glo[a] = F->c[a][0];
    F->ghi[a] = F->c[a][F->n[a] - 1];
  }
  F->mode = mode;
  pack_field(*F, bx, by, bz);
  return F;
}

void qslref_free_field(void* f) { delete (Field*)f; }

// Interpolated rhs b (3), gradient g (9, row-major g[i][j] = d b_i/d x_j) and |B|.
void qslref_interp(const void* f, const double* x, double* b, double* g, double* bmag) {
  Interp I;
  interp(*(const Field*)f, x, &I, nullptr);
  for (int i = 0; i < 3; ++i) {
    b[i] = I.b[i];
    for (int j = 0; j < 3; ++j) g[3 * i + j] = I.g[i][j];
  }
  *bmag = I.bmag;
}

void qslref_trace_seeds(const void* fp, const double* seeds, int64_t S, const Opts* o, qslref_lines* out,
                        qslref_stats* stats) {
  const Field& F = *(const Field*)fp;
  int nth = o->nthreads;
  std::vector<double> ev(S), ac(S), rj(S), ld(S);
  parallel_for(S, nth, [&](int64_t i) {
    Stats st;
    LineOut r = trace_line(F, *o, seeds + 3 * i, &st);
    ev[i] = st.stage_evals;
    ac[i] = st.accepted;
    rj[i] = st.rejected;
    ld[i] = st.landing;
#define PUT(name) \
  if (out->name) out->name[i] = r.name;
    PUT(q_perp) PUT(q_foot) PUT(q_det) PUT(b0) PUT(bf) PUT(bb) PUT(flux) PUT(flux_b) PUT(L) PUT(lam_f) PUT(lam_b)
    PUT(face_f) PUT(face_b) PUT(st_f) PUT(st_b) PUT(steps)
#undef PUT
    for (int k = 0; k < 3; ++k) {
      if (out->xf) out->xf[3 * i + k] = r.xf[k];
      if (out->xb) out->xb[3 * i + k] = r.xb[k];
    }
  });
  if (stats) {
    stats->stage_evals = stats->accepted = stats->rejected = stats->landing = 0;
    for (int64_t i = 0; i < S; ++i) {
      stats->stage_evals += ev[i];
      stats->accepted += ac[i];
      stats->rejected += rj[i];
      stats->landing += ld[i];
    }
  }
}

// Trace one direction only and return the end state (x, dx1, dx2), mu, face
// and status. Used by the brute-force finite-difference pins.
void qslref_trace_dir(const void* fp, const double* y0, int s, int ncomp, const Opts* o, double* y_end,
                      double* mu, int32_t* face, int32_t* status) {
  const Field& F = *(const Field*)fp;
  double lo[3], hi[3], max_len;
  resolve_domain(F, *o, lo, hi, &max_len);
  End e = trace_dir(F, *o, lo, hi, max_len, s, ncomp, y0, nullptr);
  std::memcpy(y_end, e.y, sizeof(double) * ncomp);
  *mu = e.mu;
  *face = e.face;
  *status = e.status;
}

// Generic Cash-Karp step on the linear test ODE dy/dt = M y (n <= 9), used by
// the order pin; the tableau is the one the tracer uses.
void qslref_ck_linear_step(const double* M, int n, const double* y, double h, double* ynew, double* yerr) {
  double k[6][9], yt[9];
  for (int stage = 0; stage < 6; ++stage) {
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int j = 0; j < stage; ++j) acc += CK_A[stage][j] * k[j][i];
      yt[i] = y[i] + h * acc;
    }
    for (int i = 0; i < n; ++i) {
      double acc = 0;
      for (int j = 0; j < n; ++j) acc += M[i * n + j] * yt[j];
      k[stage][i] = acc;
    }
  }
  for (int i = 0; i < n; ++i) {
    double s5 = 0, s4 = 0;
    for (int j = 0; j < 6; ++j) {
      s5 += CK_B5[j] * k[j][i];
      s4 += CK_B4[j] * k[j][i];
    }
    ynew[i] = y[i] + h * s5;
    yerr[i] = h * (s5 - s4);
  }
}

void qslref_ck_c(double* c) { std::memcpy(c, CK_C, sizeof(CK_C)); }

// Planar slice seeds (Sec. "Code Overview": centre, orientation, axes span):
// pixel (i, j) sits at centre + ((i+0.5)/nu - 0.5) u + ((j+0.5)/nv - 0.5) v;
// output index j*nu + i (u fastest).
void qslref_plane_seeds(const double* c, const double* u, const double* v, int nu, int nv, double* out) {
  for (int j = 0; j < nv; ++j)
    for (int i = 0; i < nu; ++i) {
      double a = (i + 0.5) / nu - 0.5, b = (j + 0.5) / nv - 0.5;
      for (int k = 0; k < 3; ++k) out[3 * ((int64_t)j * nu + i) + k] = c[k] + a * u[k] + b * v[k];
    }
}

// Volume seeds: cell centres of an nx*ny*nz lattice over [lo, hi]; x fastest.
void qslref_volume_seeds(const double* lo, const double* hi, int nx, int ny, int nz, double* out) {
  int n[3] = {nx, ny, nz};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        int idx[3] = {i, j, k};
        int64_t o = ((int64_t)k * ny + j) * nx + i;
        for (int a = 0; a < 3; ++a) out[3 * o + a] = lo[a] + (idx[a] + 0.5) / n[a] * (hi[a] - lo[a]);
      }
}

void qslref_sobel(const float* L, int ndim, const int64_t* shape, double* out) { sobel(L, ndim, shape, out); }

uint64_t qslref_hilbert_key(const uint32_t* coords, int ndim, int bits) { return hilbert_key(coords, ndim, bits); }
void qslref_hilbert_coords(uint64_t key, int ndim, int bits, uint32_t* coords) {
  hilbert_coords(key, ndim, bits, coords);
}

}  // extern "C"

// ===========================================================================
// Adaptive refinement along a Hilbert curve and the Hilbert -> rectilinear
// converter (Sec. "Adaptive refinements").
// ===========================================================================
namespace {

struct RefineSpec {
  int ndim;            // 2: planar slice, 3: volume
  int coarse_order;    // p0
  int max_order;       // p (effective resolution 2^p per axis)
  int max_iters;
  int extent[3];       // effective lattice extent per axis (<= 2^p), multiple of 2^(p-p0)
  int shift;           // shifted-curve pass on/off
  int q_form;          // 0: Q_perp (Eq. finalQ), 1: Q_foot
  int out_order;       // converter output order (<= p)
  int pad;
  double center[3], u[3], v[3];  // planar slice
  double lo[3], hi[3];           // volume
  double tau;                    // threshold on |L_i - L_{i+1}|
  int criterion;                 // 0: FLL jump |L_i - L_{i+1}| > tau; 1: Q threshold
  int pad2;
  double q_threshold;            // criterion 1: refine a pair where a sample's Q exceeds it
  // Lengths the FLL-jump criterion compares for samples added by the passes
  // (the coarse samples' own lengths decide for them): 0 a lengths-only trace
  // by the Cash-Karp stepper (Sec. "Integration methods") at the run's
  // tolerance with the step cap pass_h_max; 1 a lengths-only trace with the
  // run's options; 2 the stored lengths themselves. The stored values are
  // always those of the trace with the run's options.
  int pass_stepper;
  int pad3;
  double pass_h_max;             // smallest grid spacings; 0: 4
};

struct Sample {
  uint64_t key;
  double q, L;
  double Ld;   // the length the FLL-jump criterion compares (see RefineSpec::pass_stepper)
  int face_f, face_b, st_f, st_b;
  int origin;  // pass that added it: 0 coarse pass, 2i + 1 / 2i + 2 pass A / B of iteration i
  int unsure;  // test hook: the evaluator could not determine the value
};

// Position of the centre of effective-lattice cell c.
void cell_position(const RefineSpec& s, const uint32_t* c, double* x) {
  if (s.ndim == 2) {
    double a = (c[0] + 0.5) / s.extent[0] - 0.5, b = (c[1] + 0.5) / s.extent[1] - 0.5;
    for (int k = 0; k < 3; ++k) x[k] = s.center[k] + a * s.u[k] + b * s.v[k];
  } else {
    for (int k = 0; k < 3; ++k) x[k] = s.lo[k] + (c[k] + 0.5) / s.extent[k] * (s.hi[k] - s.lo[k]);
  }
}

bool in_extent(const RefineSpec& s, const uint32_t* c) {
  for (int a = 0; a < s.ndim; ++a)
    if (c[a] >= (uint32_t)s.extent[a]) return false;
  return true;
}

// Evaluates (Q, L, faces, status) for every sample of a batch.
struct Evaluator {
  const Field* F = nullptr;
  const Opts* o = nullptr;
  void (*fn)(int64_t, const double*, double*, double*) = nullptr;  // test hook: (n, xyz, q, L)
  // test hook with the samples' keys: (n, xyz, keys, q, L, unsure); unsure[i] != 0
  // marks a sample whose value the caller cannot determine (see Arbiter)
  void (*fnk)(int64_t, const double*, const uint64_t*, double*, double*, int32_t*) = nullptr;
};

// Test hook of the refinement driver (no counterpart in the paper): pairs
// whose criterion value lies within a band of the threshold are decided by
// whether another run added their new cell in the same pass, read from that
// run's sorted keys and the pass that added each. A traced sample set whose
// values carry a known error can then be replayed from values without that
// error: with the band set to the error bound, the replay reproduces the set
// exactly when every decision the two runs disagree on lies within the bound.
//  - FLL jump: ambiguous when | |L_i - L_j| - tau | <= band_abs + band_rel * max(|L_i|, |L_j|).
//  - Q threshold: a sample is ambiguous when its Q is finite and
//    |Q / q_threshold - 1| <= band_rel; a pair is ambiguous when neither sample
//    is clearly above the threshold and one of them is ambiguous.
//  - Either criterion: a pair is ambiguous when the evaluator marks one of its
//    samples as undetermined (a line whose end changes under a perturbation of
//    its seed below the other run's error).
struct Arbiter {
  double band_abs, band_rel;
  const uint64_t* keys;   // sorted ascending
  const int32_t* origin;  // pass that added each of them (as Sample::origin)
  int64_t n;
};

// Region test for curve cells: lo[a] <= c[a] < hi[a] on every axis.
bool in_region(const uint32_t* c, int nd, const uint64_t* lo, const uint64_t* hi) {
  for (int a = 0; a < nd; ++a)
    if (c[a] < lo[a] || c[a] >= hi[a]) return false;
  return true;
}

// Reading of "halfway along the Hilbert curve" when the curve leaves the
// sampled region (a box clipped from the curve's cube, or the shifted lattice):
// the new sample is the in-region cell nearest to the midpoint key m along the
// curve, strictly between the pair's keys (the lower one on ties), found by
// skipping whole aligned blocks of the curve that lie outside the region.
// Returns false when the pair has no in-region cell between them.
bool nearest_in_region(uint64_t m, uint64_t k_lo, uint64_t k_hi, int nd, int bits, const uint64_t* lo,
                       const uint64_t* hi, uint64_t* out) {
  auto skip = [&](uint64_t k, int dir, uint64_t* res) -> bool {
    for (int guard = 0; guard < 4096; ++guard) {
      if (k <= k_lo || k >= k_hi) return false;
      uint32_t c[3] = {0, 0, 0};
      hilbert_coords(k, nd, bits, c);
      if (in_region(c, nd, lo, hi)) {
        *res = k;
        return true;
      }
      int lev = 0;
      while (lev < bits) {
        int l = lev + 1;
        bool outside = false;
        for (int a = 0; a < nd; ++a) {
          uint64_t b0 = ((uint64_t)c[a] >> l) << l;
          uint64_t b1 = b0 + ((uint64_t)1 << l);
          if (b1 <= lo[a] || b0 >= hi[a]) outside = true;
        }
        if (!outside) break;
        lev = l;
      }
      uint64_t blk = (uint64_t)1 << (nd * lev);
      uint64_t start = (k / blk) * blk;
      if (dir < 0) {
        if (start == 0) return false;
        k = start - 1;
      } else {
        k = start + blk;
      }
    }
    return false;
  };
  uint64_t a = 0, b = 0;
  bool ha = skip(m, -1, &a);
  bool hb = skip(m, +1, &b);
  if (ha && hb) {
    *out = (m - a <= b - m) ? a : b;
    return true;
  }
  if (ha) { *out = a; return true; }
  if (hb) { *out = b; return true; }
  return false;
}

// `pass`: the batch was added by a refinement pass (decision lengths per
// RefineSpec::pass_stepper); otherwise the coarse batch.
void trace_samples(const Evaluator& ev, const RefineSpec& s, std::vector<Sample>& v, bool pass) {
  if (v.empty()) return;
  std::vector<double> seeds(3 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    uint32_t c[3] = {0, 0, 0};
    hilbert_coords(v[i].key, s.ndim, s.max_order, c);
    cell_position(s, c, &seeds[3 * i]);
  }
  if (ev.fn || ev.fnk) {
    std::vector<double> q(v.size()), L(v.size());
    std::vector<int32_t> unsure(v.size(), 0);
    if (ev.fnk) {
      std::vector<uint64_t> keys(v.size());
      for (size_t i = 0; i < v.size(); ++i) keys[i] = v[i].key;
      ev.fnk((int64_t)v.size(), seeds.data(), keys.data(), q.data(), L.data(), unsure.data());
    } else {
      ev.fn((int64_t)v.size(), seeds.data(), q.data(), L.data());
    }
    for (size_t i = 0; i < v.size(); ++i) {
      v[i].q = q[i];
      v[i].L = L[i];
      v[i].Ld = L[i];
      v[i].face_f = v[i].face_b = NO_FACE;
      v[i].st_f = v[i].st_b = ST_OK;
      v[i].unsure = unsure[i];
    }
    return;
  }
  const Field& F = *ev.F;
  const Opts& o = *ev.o;
  const bool decide = pass && s.criterion == 0 && !o.length_only && s.pass_stepper != 2;
  Opts od = o;
  od.length_only = 1;
  if (s.pass_stepper == 0) {
    od.integrator = 0;
    od.h_max = s.pass_h_max > 0 ? s.pass_h_max : 4.0;
  }
  parallel_for((int64_t)v.size(), o.nthreads, [&](int64_t i) {
    LineOut r = trace_line(F, o, &seeds[3 * i], nullptr);
    v[i].q = (s.q_form == 1) ? r.q_foot : r.q_perp;
    v[i].L = r.L;
    v[i].Ld = decide ? trace_line(F, od, &seeds[3 * i], nullptr).L : r.L;
    v[i].face_f = r.face_f;
    v[i].face_b = r.face_b;
    v[i].st_f = r.st_f;
    v[i].st_b = r.st_b;
  });
}

void merge_in(std::vector<Sample>& all, std::vector<Sample>& add) {
  all.insert(all.end(), add.begin(), add.end());
  std::sort(all.begin(), all.end(), [](const Sample& a, const Sample& b) { return a.key < b.key; });
}

}  // namespace

extern "C" {

int qslref_sizeof_refine_spec(void) { return (int)sizeof(RefineSpec); }

// Refinement driver. Writes up to `capacity` samples sorted by key, returns the
// number of samples (or -needed when capacity is too small), and the number of
// iterations run in *iters_out. Per-iteration trace counts go to
// traced_per_iter (length max_iters + 1, entry 0 = coarse pass), if non-null.
//
// Reading of the paper's procedure: every sample sits at the centre of a cell
// of the effective lattice (2^p per axis); the coarse pass samples the cells
// whose indices are R/2 modulo R (R = 2^(p-p0)). One iteration is (A) flag
// every pair of samples adjacent along the curve with key gap > 1 and
// |L_i - L_{i+1}| > tau and add the cell halfway along the curve, floor of the
// mean key; (B) on the curve of order p+1 over the lattice shifted by S cells on
// every axis, S = 2^(p-1) + max(1, R/2) on even iterations and
// 2^(p-1) - max(1, R/2) on odd ones, the same flag rule, new cells mapped back
// by the inverse shift and kept when inside the lattice. Iterations stop when
// neither pass adds a sample.
// Refinement criterion of a pair of samples adjacent along the curve: the FLL
// jump the paper uses, or the alternative it compares against (Sec. "Adaptive
// refinements"): refine where Q exceeds a fixed threshold. A sample whose Q is
// not finite (a NaN of an open or cut-off line) does not trigger the latter.
static bool pair_flagged(const RefineSpec& s, const Sample& A, const Sample& B) {
  if (s.criterion == 1)
    return (std::isfinite(A.q) && A.q > s.q_threshold) || (std::isfinite(B.q) && B.q > s.q_threshold);
  return std::fabs(B.Ld - A.Ld) > s.tau;
}

// The decision with the test hook: the comparison, or, for a pair within the
// band, whether its new cell `cand` is in the arbiter's key set.
static bool pair_ambiguous(const RefineSpec& s, const Sample& A, const Sample& B, const Arbiter& arb) {
  if (A.unsure || B.unsure) return true;
  if (s.criterion == 1) {
    auto clear_above = [&](double q) { return std::isfinite(q) && q / s.q_threshold - 1.0 > arb.band_rel; };
    auto near = [&](double q) { return std::isfinite(q) && std::fabs(q / s.q_threshold - 1.0) <= arb.band_rel; };
    return !clear_above(A.q) && !clear_above(B.q) && (near(A.q) || near(B.q));
  }
  double d = std::fabs(B.Ld - A.Ld);
  double band = arb.band_abs + arb.band_rel * std::max(std::fabs(A.Ld), std::fabs(B.Ld));
  return std::fabs(d - s.tau) <= band;
}

// Whether the arbiter's run added cell k in pass `pass`.
static bool added_in(const Arbiter& arb, uint64_t k, int pass) {
  const uint64_t* it = std::lower_bound(arb.keys, arb.keys + arb.n, k);
  return it != arb.keys + arb.n && *it == k && arb.origin[it - arb.keys] == pass;
}

static int64_t refine_impl(const Evaluator& ev, const RefineSpec* sp, int64_t capacity, uint64_t* key,
                           double* q, double* L, int32_t* face_f, int32_t* face_b, int32_t* st_f,
                           int32_t* st_b, int32_t* iters_out, int64_t* traced_per_iter,
                           const Arbiter* arb = nullptr, int32_t* origin = nullptr) {
  const RefineSpec& s = *sp;
  int p = s.max_order, p0 = s.coarse_order, nd = s.ndim;
  uint32_t R = 1u << (p - p0);
  uint32_t r = R / 2;
  uint64_t rlo[3] = {0, 0, 0}, rhi[3] = {1, 1, 1};
  for (int a = 0; a < nd; ++a) rhi[a] = (uint64_t)s.extent[a];
  std::vector<Sample> all;
  // coarse pass
  {
    uint32_t nc[3] = {1, 1, 1};
    for (int a = 0; a < nd; ++a) nc[a] = (uint32_t)s.extent[a] / R;
    for (uint32_t k = 0; k < nc[2]; ++k)
      for (uint32_t j = 0; j < nc[1]; ++j)
        for (uint32_t i = 0; i < nc[0]; ++i) {
          uint32_t c[3] = {i * R + r, j * R + r, k * R + r};
          Sample smp{};
          smp.key = hilbert_key(c, nd, p);
          all.push_back(smp);
        }
    trace_samples(ev, s, all, false);
    std::sort(all.begin(), all.end(), [](const Sample& a, const Sample& b) { return a.key < b.key; });
    if (traced_per_iter) traced_per_iter[0] = (int64_t)all.size();
  }
  int it = 0;
  for (; it < s.max_iters; ++it) {
    int64_t added = 0;
    // (A) flag along the curve itself
    std::vector<Sample> add;
    for (size_t i = 0; i + 1 < all.size(); ++i) {
      uint64_t gap = all[i + 1].key - all[i].key;
      if (gap <= 1) continue;
      const bool amb = arb && pair_ambiguous(s, all[i], all[i + 1], *arb);
      if (amb || pair_flagged(s, all[i], all[i + 1])) {
        uint64_t m = all[i].key + gap / 2;
        uint64_t got;
        if (!nearest_in_region(m, all[i].key, all[i + 1].key, nd, p, rlo, rhi, &got)) continue;
        if (amb && !added_in(*arb, got, 2 * it + 1)) continue;
        Sample smp{};
        smp.key = got;
        smp.origin = 2 * it + 1;
        add.push_back(smp);
      }
    }
    trace_samples(ev, s, add, true);
    added += (int64_t)add.size();
    merge_in(all, add);
    // (B) flag along the shifted curve
    if (s.shift) {
      // Shift of the lattice on every axis, on a curve of order p+1: half the
      // lattice (so the region sits across the four top-level quadrants) plus
      // or minus half the coarse spacing, alternating between iterations.
      uint32_t half = 1u << (p - 1 >= 0 ? p - 1 : 0);
      uint32_t d = std::max<uint32_t>(1, R / 2);
      uint32_t S = (it % 2 == 0) ? half + d : half - std::min(half, d);
      std::vector<std::pair<uint64_t, size_t>> sk(all.size());
      for (size_t i = 0; i < all.size(); ++i) {
        uint32_t c[3] = {0, 0, 0};
        hilbert_coords(all[i].key, nd, p, c);
        for (int a = 0; a < nd; ++a) c[a] += S;
        sk[i] = {hilbert_key(c, nd, p + 1), i};
      }
      std::sort(sk.begin(), sk.end());
      std::vector<Sample> add2;
      for (size_t i = 0; i + 1 < sk.size(); ++i) {
        uint64_t gap = sk[i + 1].first - sk[i].first;
        const Sample& A = all[sk[i].second];
        const Sample& B = all[sk[i + 1].second];
        if (gap <= 1) continue;
        const bool amb = arb && pair_ambiguous(s, A, B, *arb);
        if (amb || pair_flagged(s, A, B)) {
          uint64_t m = sk[i].first + gap / 2;
          uint64_t slo[3], shi[3], got;
          for (int a = 0; a < 3; ++a) {
            slo[a] = rlo[a] + S;
            shi[a] = rhi[a] + S;
          }
          if (!nearest_in_region(m, sk[i].first, sk[i + 1].first, nd, p + 1, slo, shi, &got)) continue;
          uint32_t c[3] = {0, 0, 0};
          hilbert_coords(got, nd, p + 1, c);
          for (int a = 0; a < nd; ++a) c[a] -= S;
          Sample smp{};
          smp.key = hilbert_key(c, nd, p);
          smp.origin = 2 * it + 2;
          if (amb && !added_in(*arb, smp.key, 2 * it + 2)) continue;
          add2.push_back(smp);
        }
      }
      trace_samples(ev, s, add2, true);
      added += (int64_t)add2.size();
      merge_in(all, add2);
    }
    if (traced_per_iter) traced_per_iter[it + 1] = added;
    if (added == 0) break;
  }
  if (iters_out) *iters_out = it;
  int64_t n = (int64_t)all.size();
  if (n > capacity) return -n;
  for (int64_t i = 0; i < n; ++i) {
    key[i] = all[i].key;
    q[i] = all[i].q;
    L[i] = all[i].L;
    face_f[i] = all[i].face_f;
    face_b[i] = all[i].face_b;
    st_f[i] = all[i].st_f;
    st_b[i] = all[i].st_b;
    if (origin) origin[i] = all[i].origin;
  }
  return n;
}

int64_t qslref_refine(const void* fp, const Opts* o, const RefineSpec* sp, int64_t capacity, uint64_t* key,
                      double* q, double* L, int32_t* face_f, int32_t* face_b, int32_t* st_f, int32_t* st_b,
                      int32_t* iters_out, int64_t* traced_per_iter, int32_t* origin) {
  Evaluator ev;
  ev.F = (const Field*)fp;
  ev.o = o;
  return refine_impl(ev, sp, capacity, key, q, L, face_f, face_b, st_f, st_b, iters_out, traced_per_iter, nullptr,
                     origin);
}

// Same driver with the tracer replaced by a caller-supplied function of the
// sample positions (used to pin the refinement logic on analytic L maps).
int64_t qslref_refine_fn(void (*fn)(int64_t, const double*, double*, double*), const RefineSpec* sp,
                         int64_t capacity, uint64_t* key, double* q, double* L, int32_t* iters_out,
                         int64_t* traced_per_iter) {
  Evaluator ev;
  ev.fn = fn;
  std::vector<int32_t> dummy(4 * (size_t)std::max<int64_t>(capacity, 1));
  int32_t* d = dummy.data();
  size_t c = (size_t)std::max<int64_t>(capacity, 1);
  return refine_impl(ev, sp, capacity, key, q, L, d, d + c, d + 2 * c, d + 3 * c, iters_out, traced_per_iter);
}

// Replay of a sample set (test hook, see Arbiter): the driver with values from
// fn(n, xyz, keys, q, L), and pairs within the band of the threshold decided by
// membership of their new cell in tie_keys (sorted). Outputs as qslref_refine_fn.
int64_t qslref_refine_replay(void (*fn)(int64_t, const double*, const uint64_t*, double*, double*, int32_t*),
                             const RefineSpec* sp, double band_abs, double band_rel, const uint64_t* tie_keys,
                             const int32_t* tie_origin, int64_t n_tie, int64_t capacity, uint64_t* key,
                             double* q, double* L, int32_t* origin, int32_t* iters_out,
                             int64_t* traced_per_iter) {
  Evaluator ev;
  ev.fnk = fn;
  Arbiter arb{band_abs, band_rel, tie_keys, tie_origin, n_tie};
  std::vector<int32_t> dummy(4 * (size_t)std::max<int64_t>(capacity, 1));
  int32_t* d = dummy.data();
  size_t c = (size_t)std::max<int64_t>(capacity, 1);
  return refine_impl(ev, sp, capacity, key, q, L, d, d + c, d + 2 * c, d + 3 * c, iters_out, traced_per_iter,
                     &arb, origin);
}

// Hilbert -> rectilinear array converter (Sec. "Adaptive refinements").
// Output lattice: extent >> (p - out_order) per axis, x fastest. A cell holding
// samples gets their maximum (NaNs ignored unless all are NaN). An empty cell
// gets the value interpolated along the curve, linearly in key, between the
// nearest sample before and after the cell's key range, taken at the middle of
// that range; `log_interp` interpolates log10 of the values (used for Q).
void qslref_convert(const uint64_t* key, const double* val, int64_t n, int ndim, int max_order,
                    const int32_t* extent, int out_order, int log_interp, double* out) {
  int d = max_order - out_order;
  int64_t eo[3] = {1, 1, 1};
  for (int a = 0; a < ndim; ++a) eo[a] = extent[a] >> d;
  int64_t N = eo[0] * eo[1] * eo[2];
  std::vector<int64_t> count(N, 0);
  for (int64_t i = 0; i < N; ++i) out[i] = NaN;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t c[3] = {0, 0, 0};
    hilbert_coords(key[i], ndim, max_order, c);
    int64_t o = 0;
    for (int a = ndim - 1; a >= 0; --a) o = o * eo[a] + (c[a] >> d);
    count[o] += 1;
    if (std::isnan(out[o]) || val[i] > out[o]) out[o] = std::isnan(val[i]) ? out[o] : val[i];
  }
  uint64_t block = (uint64_t)1 << (ndim * d);
  for (int64_t o = 0; o < N; ++o) {
    if (count[o] > 0) continue;
    uint32_t c[3] = {0, 0, 0};
    int64_t rem = o;
    for (int a = 0; a < ndim; ++a) {
      c[a] = (uint32_t)((rem % eo[a]) << d);
      rem /= eo[a];
    }
    uint64_t k0 = (hilbert_key(c, ndim, max_order) / block) * block;
    uint64_t k1 = k0 + block;
    const uint64_t* it = std::lower_bound(key, key + n, k0);
    int64_t succ = (it - key);
    int64_t pred = succ - 1;
    if (succ >= n && pred < 0) continue;
    if (succ >= n) {
      out[o] = val[pred];
      continue;
    }
    if (pred < 0) {
      out[o] = val[succ];
      continue;
    }
    (void)k1;
    double kc = (double)k0 + 0.5 * (double)(block - 1);
    double t = (kc - (double)key[pred]) / ((double)key[succ] - (double)key[pred]);
    double a = val[pred], b = val[succ];
    if (log_interp) {
      double la = std::log10(a), lb = std::log10(b);
      out[o] = std::pow(10.0, (1 - t) * la + t * lb);
    } else {
      out[o] = (1 - t) * a + t * b;
    }
  }
}

}  // extern "C"
