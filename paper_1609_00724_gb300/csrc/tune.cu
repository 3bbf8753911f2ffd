// Autotuner of the tracer: picks the loosest step tolerance whose Q and length
// stay within stated bounds of an FP64 reference traced at tol 1e-10 on the
// same sample of seeds, then the launch shape (warps per block, resident
// blocks per SM, refill threshold of the work queue) and the step cap (the
// requested one, or 4 smallest spacings when that also meets the bounds; the
// cell-wise stepper otherwise often stops just short of a face on anisotropic
// grids). Each candidate is timed with CUDA events on the caller's stream;
// shapes on the sample repeated until one launch holds many waves of resident
// lines, so that the timing measures throughput, not the latency of the
// sample's longest line.
// Results are cached per (grid size, interpolation mode, integrator, q_form,
// length_only, requested tolerance decade).
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "qsl_internal.cuh"

namespace {

typedef std::tuple<int, int, int, int, int, int, int, int> TuneKey;
std::mutex g_tune_mu;
std::map<TuneKey, qsl_tune_report> g_tune_cache;

struct DevLines {
  qsl_line* p = nullptr;
  ~DevLines() {
    if (p) cudaFree(p);
  }
};

int time_trace(const qsl_field* f, const double* seeds, int64_t S, const qsl_opts* o, qsl_line* out,
               cudaStream_t s, double* ms_out) {
  cudaEvent_t e0, e1;
  QSL_CHECK_CUDA(cudaEventCreate(&e0));
  QSL_CHECK_CUDA(cudaEventCreate(&e1));
  QSL_CHECK_CUDA(cudaEventRecord(e0, s));
  int rc = qsl_trace_seeds(f, seeds, S, o, out, QSL_MEM_DEVICE, s);
  QSL_CHECK_CUDA(cudaEventRecord(e1, s));
  QSL_CHECK_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = ms;
  return rc;
}

// Worst relative errors of `got` against `ref` (Q below 1e6 and both ends on
// the same faces). Lengths: *el over lines of at least one cell (relative);
// *es over shorter lines, in units of one cell: a line shorter than a cell that
// leaves at a grazing angle has a length set by a cancellation in the FP32
// field samples, whatever the step tolerance, so it is held to the absolute
// bound of the parity bar and does not decide the tolerance.
void errors(const std::vector<qsl_line>& got, const std::vector<qsl_line>& ref, int q_form, double cell, double* eq,
            double* el, double* es, double* face_mismatch) {
  double wq = 0, wl = 0, ws = 0;
  int64_t fm = 0;
  for (size_t i = 0; i < ref.size(); ++i) {
    const qsl_line& a = got[i];
    const qsl_line& b = ref[i];
    if (a.face_f != b.face_f || a.face_b != b.face_b) {
      ++fm;
      continue;
    }
    double qa = q_form == QSL_Q_FOOT ? a.q_foot : (q_form == QSL_Q_DET ? a.q_det : a.q_perp);
    double qb = q_form == QSL_Q_FOOT ? b.q_foot : (q_form == QSL_Q_DET ? b.q_det : b.q_perp);
    if (std::isfinite(qb) && qb < 1e6) wq = fmax(wq, fabs(qa / qb - 1.0));
    if (std::isfinite(b.length)) {
      const double d = fabs((double)a.length - (double)b.length);
      if ((double)b.length >= cell) wl = fmax(wl, d / (double)b.length);
      else ws = fmax(ws, d / cell);
    }
  }
  *eq = wq;
  *el = wl;
  *es = ws;
  *face_mismatch = ref.empty() ? 0.0 : (double)fm / (double)ref.size();
}

}  // namespace

extern "C" int qsl_autotune(const qsl_field* f, const double* seeds, int64_t S, qsl_opts* opts,
                            qsl_tune_report* report, void* stream_) {
  cudaStream_t s = (cudaStream_t)stream_;
  int rc = qsl::validate_opts(f, opts);
  if (rc) return rc;
  if (S < 1 || !seeds) {
    qsl::set_error("autotune needs at least one sample seed (device memory)");
    return QSL_EINVAL;
  }
  TuneKey key(f->n[0], f->n[1], f->n[2], f->mode, opts->integrator, opts->q_form, opts->length_only,
              (int)std::lround(-std::log10(fmax(opts->tol_rel, 1e-30))));
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      opts->warps_per_block = it->second.warps_per_block;
      opts->blocks_per_sm = it->second.blocks_per_sm;
      opts->refill_min = it->second.refill_min;
      opts->tol_abs = opts->tol_rel = it->second.tol;
      opts->h_max = it->second.h_max;
      if (report) {
        *report = it->second;
        report->cached = 1;
      }
      return QSL_OK;
    }
  }
  DevLines d;
  QSL_CHECK_CUDA(cudaMalloc((void**)&d.p, sizeof(qsl_line) * S));
  std::vector<qsl_line> ref(S), got(S);
  // FP64 reference at tight tolerance
  qsl_opts r = *opts;
  r.precision = QSL_FP64;
  r.tol_abs = r.tol_rel = 1e-10;
  r.retrace_q = 0;
  double ms = 0;
  if ((rc = time_trace(f, seeds, S, &r, d.p, s, &ms))) return rc;
  QSL_CHECK_CUDA(cudaMemcpy(ref.data(), d.p, sizeof(qsl_line) * S, cudaMemcpyDeviceToHost));
  // tolerance: the loosest candidate within a fifth of the parity bar. The
  // candidates run the caller's precision policy (FP64 retrace of lines above
  // retrace_q included), and FP32 candidates stop at 1e-7: below that the
  // error estimate is FP32 rounding and the controller only shrinks steps.
  const double tols32[] = {1e-5, 1e-6, 1e-7};
  const double tols64[] = {1e-6, 1e-7, 1e-8, 1e-9};
  const bool fp64 = opts->precision == QSL_FP64;
  const double* tols = fp64 ? tols64 : tols32;
  const int n_tols = fp64 ? 4 : 3;
  qsl_opts base = *opts;
  double chosen_tol = tols[n_tols - 1], eq = 0, el = 0, es = 0, fm = 0;
  int passed = 0;
  for (int k = 0; k < n_tols; ++k) {
    qsl_opts c = base;
    c.tol_abs = c.tol_rel = tols[k];
    if ((rc = time_trace(f, seeds, S, &c, d.p, s, &ms))) return rc;
    QSL_CHECK_CUDA(cudaMemcpy(got.data(), d.p, sizeof(qsl_line) * S, cudaMemcpyDeviceToHost));
    errors(got, ref, opts->q_form, f->cell, &eq, &el, &es, &fm);
    if (eq <= 2e-4 && el <= 2e-6 && es <= 1e-5 && fm <= 1e-3) {
      chosen_tol = tols[k];
      passed = 1;
      break;
    }
  }
  // step cap: a larger one where it meets the same bounds at the chosen tolerance
  double hmaxes[2] = {opts->h_max, opts->h_max};
  int n_hmax = 1;
  if (opts->h_max < 4.0) {
    qsl_opts c = base;
    c.tol_abs = c.tol_rel = chosen_tol;
    c.h_max = 4.0;
    double eq4 = 0, el4 = 0, es4 = 0, fm4 = 0;
    if ((rc = time_trace(f, seeds, S, &c, d.p, s, &ms))) return rc;
    QSL_CHECK_CUDA(cudaMemcpy(got.data(), d.p, sizeof(qsl_line) * S, cudaMemcpyDeviceToHost));
    errors(got, ref, opts->q_form, f->cell, &eq4, &el4, &es4, &fm4);
    if (eq4 <= 2e-4 && el4 <= 2e-6 && es4 <= 1e-5 && fm4 <= 1e-3) hmaxes[n_hmax++] = 4.0;
  }
  // launch shape and step cap: fastest of the candidates at the chosen
  // tolerance (best of 2), on the sample repeated to at least 16 waves of
  // 12 resident warps per SM (copies far apart in the queue, so that a line
  // and its copies do not run side by side)
  int dev = 0, sms = 1;
  QSL_CHECK_CUDA(cudaGetDevice(&dev));
  QSL_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want_dirs = (int64_t)16 * sms * 12 * 32;
  const int64_t reps = (want_dirs + 2 * S - 1) / (2 * S);
  const int64_t ST = reps * S;
  DevLines dt;
  double* tiled = nullptr;
  struct DevFree {
    double* p;
    ~DevFree() {
      if (p) cudaFree(p);
    }
  } tiled_free{nullptr};
  if (reps > 1) {
    QSL_CHECK_CUDA(cudaMalloc((void**)&tiled, sizeof(double) * 3 * ST));
    tiled_free.p = tiled;
    QSL_CHECK_CUDA(cudaMalloc((void**)&dt.p, sizeof(qsl_line) * ST));
    for (int64_t k = 0; k < reps; ++k)
      QSL_CHECK_CUDA(cudaMemcpyAsync(tiled + 3 * S * k, seeds, sizeof(double) * 3 * S, cudaMemcpyDeviceToDevice, s));
  }
  const double* shape_seeds = reps > 1 ? tiled : seeds;
  qsl_line* shape_out = reps > 1 ? dt.p : d.p;
  const int wpb[] = {2, 4, 8};
  const int bps[] = {32, 2};
  const int refill[] = {1, 4, 8, 16};
  double best = 1e30;
  int bw = 4, bb = 32, br = 1;
  double bh = opts->h_max;
  for (int k = 0; k < n_hmax; ++k)
    for (int w : wpb)
      for (int b : bps)
        for (int rf : refill) {
          qsl_opts c = base;
          c.tol_abs = c.tol_rel = chosen_tol;
          c.h_max = hmaxes[k];
          c.warps_per_block = w;
          c.blocks_per_sm = b;
          c.refill_min = rf;
          double t1 = 0, t2 = 0;
          if ((rc = time_trace(f, shape_seeds, ST, &c, shape_out, s, &t1))) return rc;
          if ((rc = time_trace(f, shape_seeds, ST, &c, shape_out, s, &t2))) return rc;
          double t = fmin(t1, t2);
          if (t < best) {
            best = t;
            bw = w;
            bb = b;
            br = rf;
            bh = hmaxes[k];
          }
        }
  qsl_tune_report rep;
  memset(&rep, 0, sizeof rep);
  rep.warps_per_block = bw;
  rep.blocks_per_sm = bb;
  rep.refill_min = br;
  rep.tol = chosen_tol;
  rep.q_err = eq;
  rep.l_err = el;
  rep.l_err_subcell = es;
  rep.face_mismatch = fm;
  rep.sample_ms = best;
  rep.sample_seeds = S;
  rep.h_max = bh;
  rep.passed = passed;
  rep.shape_reps = (int32_t)reps;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = rep;
  }
  opts->warps_per_block = bw;
  opts->blocks_per_sm = bb;
  opts->refill_min = br;
  opts->tol_abs = opts->tol_rel = chosen_tol;
  opts->h_max = bh;
  if (report) *report = rep;
  return QSL_OK;
}
