/*
 * qsl.h — C ABI of the GB300 QSL engine: squashing factor Q, field-line length
 * (FLL) and FLEDGE maps of a gridded 3D magnetic field, after the method of
 * Tassev & Savcheva, "QSL Squasher: A Fast Quasi-Separatrix Layer Map
 * Calculator" (arXiv:1609.00724).
 *
 * Conventions shared by every call:
 *  - Return value: QSL_OK (0) or a negative QSL_E* code; qsl_last_error()
 *    gives a message (thread-local). Problems of single lines are status
 *    codes in the outputs, not call failures.
 *  - `mem` says where the caller's array arguments live: QSL_MEM_HOST or
 *    QSL_MEM_DEVICE (CUDA device memory of the current device). Small
 *    parameter arrays (axis coordinates, centre/axis vectors, shapes) are
 *    always host memory.
 *  - All outputs are caller-owned. Output pointers documented as optional may
 *    be NULL.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). With device
 *    memory, calls are asynchronous on that stream; with host memory they
 *    return after the results are in host memory. qsl_refine synchronises
 *    the stream once per refinement iteration (it reads a sample count).
 *  - Library scratch memory comes from the stream-ordered allocator
 *    (cudaMallocAsync) on `stream`; QSL_ENOMEM when it fails.
 *  - Every computation runs in this library's CUDA kernels on the current
 *    device; there is no CPU fallback.
 */
#ifndef QSL_H
#define QSL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------------- */
#define QSL_OK 0
#define QSL_EINVAL (-1)     /* bad argument (message says which)                   */
#define QSL_ENOMEM (-2)     /* device or host allocation failed                     */
#define QSL_ECUDA (-3)      /* a CUDA runtime call or kernel launch failed          */
#define QSL_ETIMEOUT (-4)   /* the device watchdog (qsl_opts.timeout_s) expired     */
#define QSL_ENONFINITE (-5) /* non-finite field values were given                   */
#define QSL_ECAPACITY (-6)  /* qsl_refine: sample capacity exhausted (partial result) */

/* ---- enumerations ----------------------------------------------------------- */
#define QSL_MEM_HOST 0
#define QSL_MEM_DEVICE 1

#define QSL_F32 0
#define QSL_F64 1

/* Interpolation of the field (Sec. "Interpolation schemes" and the footnote of
 * Sec. "Squashing factor calculation"): the paper normalises the field cubes
 * first and interpolates the unit vectors (the interpolant is then not unit);
 * RAW interpolates B and normalises at the point. */
#define QSL_PAPER_NORMALIZE_FIRST 0
#define QSL_RAW_B 1

/* Integrators (Sec. "Integration methods": the paper's adaptive Cash-Karp
 * stepper is one of several interchangeable embedded Runge-Kutta pairs). */
#define QSL_RKCK54 0 /* adaptive Cash-Karp 5(4), the paper's default          */
#define QSL_EULER 1  /* fixed-step explicit Euler, step qsl_opts.euler_h cells */
/* Adaptive Dormand-Prince 5(4) that never steps across a cell face: inside a
 * cell the trilinear field is a polynomial, so each step integrates a smooth
 * field from one 8-vertex gather, and its dense output (4th order) places the
 * line exactly on the next cell face. Same ODE as the paper; uniform grids
 * (other grids fall back to QSL_RKCK54). */
#define QSL_DOPRI5_CELL 2

/* Which Q the map calls return (qsl_line records hold all three). */
#define QSL_Q_PERP 0 /* Eq. finalQ with dx_perp = dx - b (b.dx)                   */
#define QSL_Q_FOOT 1 /* Eq. finalQ with deviations projected onto the end faces    */
#define QSL_Q_DET 2  /* Eq. finalQ's bracket over the true Gram determinants (>= 2) */

/* Precision policy. */
#define QSL_FP32_MIXED 0 /* FP32 tracing, FP64 Q assembly, FP64 retrace above retrace_q */
#define QSL_FP64 1       /* FP64 tracing and assembly everywhere                        */

/* Per-direction line status (3 bits). */
#define QSL_LINE_OK 0        /* reached a face of the domain                     */
#define QSL_LINE_MAXLEN 1    /* stopped at qsl_opts.max_length (Q at the cutoff)     */
#define QSL_LINE_MAXSTEPS 2  /* qsl_opts.max_steps step attempts used up          */
#define QSL_LINE_STALL 3     /* step size fell below qsl_opts.h_min               */
#define QSL_LINE_OUTSIDE 4   /* the seed lies outside the domain                  */
#define QSL_LINE_NONFINITE 5 /* the state became non-finite                       */
#define QSL_LINE_NULL 6      /* the interpolated field vanishes at the seed       */
#define QSL_LINE_TIMEOUT 7   /* the device watchdog stopped the launch            */

/* Map status byte: status_F | status_B << 3 | flags. */
#define QSL_FLAG_OPEN_SKIPPED 0x40 /* open line with skip_open: Q = NaN           */
#define QSL_FLAG_RETRACED 0x80     /* Q above retrace_q: traced again in FP64     */

/* Faces: 0..5 = x-, x+, y-, y+, z-, z+ of the domain; QSL_NO_FACE otherwise. */
#define QSL_NO_FACE 255

/* ---- options ----------------------------------------------------------------- */
typedef struct qsl_opts {
  int32_t integrator;  /* QSL_RKCK54 | QSL_EULER | QSL_DOPRI5_CELL                  */
  int32_t q_form;      /* QSL_Q_PERP | QSL_Q_FOOT | QSL_Q_DET (map outputs)          */
  int32_t precision;   /* QSL_FP32_MIXED | QSL_FP64                                  */
  int32_t skip_open;   /* 1: lines not closed on z- get Q = NaN (Sec. "Squashing factor calculation") */
  int32_t length_only; /* 1: integrate x only; Q outputs are NaN (FLEDGE fast path)   */
  int32_t warps_per_block; /* tracer launch shape; 0 = autotuned                        */
  int32_t blocks_per_sm;   /* tracer launch shape; 0 = autotuned                        */
  int32_t refill_min;      /* lanes idle before a warp refills from the queue; 0 = auto */
  double tol_abs, tol_rel; /* step error tolerances (paper: 1e-2)                       */
  double h_init, h_max, h_min; /* step bounds in units of the smallest grid spacing      */
  double max_length;       /* per direction, domain units; <= 0: 20 x domain diagonal  */
  int64_t max_steps;       /* step attempts per direction                               */
  double euler_h;          /* Euler step in cells (paper: about 1/5)                    */
  double retrace_q;        /* FP64 retrace threshold for QSL_FP32_MIXED; <= 0: never    */
  double domain_lo[3], domain_hi[3]; /* tracing box; lo >= hi on any axis: grid extent */
  double land_tol;         /* face landing tolerance in cells (FP32 stops at its resolution of the step) */
  double timeout_s;        /* device watchdog per launch; <= 0: none                    */
  int32_t line_lanes;      /* lanes per line of QSL_DOPRI5_CELL: 1 = one lane per line,
                              3 = a group of three lanes (one per axis), 0 = auto (three
                              up to 512 line directions per SM, where a launch is bound
                              by the latency of its longest lines; results agree to
                              rounding)                                                  */
  int32_t interp_order;    /* Sec. "Interpolation schemes": 1 (or 0) trilinear, 2 triquadratic
                              (Dodgson's interpolating quadratic, 27 vertices), 3 tricubic
                              (Keys cubic convolution, 64 vertices); 2 and 3 need a uniform
                              grid and QSL_RKCK54 or QSL_EULER; stencil vertices beyond the
                              grid are clamped to its edge                                */
} qsl_opts; /* 176 bytes */

/* Fills the defaults: RKCK54, Q_PERP, FP32_MIXED, tol 1e-2/1e-2, h_init 0.1,
 * h_max 2, h_min 1e-15 cells, max_length 20 x diagonal, max_steps 1e6,
 * euler_h 0.2, retrace_q 1e6, land_tol 1e-12, no watchdog, line_lanes 0 (auto),
 * interp_order 1. */
void qsl_opts_default(qsl_opts* opts);

/* ---- per-line record (qsl_trace_seeds) --------------------------------------- */
typedef struct qsl_line {
  double q_perp;  /* Eq. finalQ                                               */
  double q_foot;  /* Eq. finalQ with face-projected deviations and |B_n|      */
  double q_det;   /* bracket of Eq. finalQ / sqrt(det G_F det G_B)            */
  double b0, bf, bb;       /* |B| at the seed and at the two ends               */
  double flux_f, flux_b;   /* (B_e/B_0)|a_e x b_e| - 1 at each end               */
  float length;            /* lambda_F - lambda_B                                */
  float lam_f, lam_b;      /* lambda_F >= 0, lambda_B <= 0                       */
  float pad0;
  float x_f[3], x_b[3];    /* end points                                         */
  int32_t steps;           /* step attempts, both directions                     */
  uint8_t face_f, face_b;  /* end faces (QSL_NO_FACE at a cutoff)                */
  uint8_t status_f, status_b; /* QSL_LINE_* per direction                        */
} qsl_line; /* 112 bytes */

/* ---- statistics of the last tracing call on this thread ------------------------ */
typedef struct qsl_stats {
  int64_t lines;        /* seeds traced (both directions each)                 */
  int64_t stage_evals;  /* interpolations of B and grad B inside the tracer    */
  int64_t accepted, rejected, landing; /* step attempts by kind              */
  int64_t retraced;     /* seeds traced again in FP64                           */
  double kernel_ms;     /* device time of the tracer launches (CUDA events)     */
  int32_t warps_per_block, blocks_per_sm, refill_min, pad;
} qsl_stats;

/* Synchronises the stream of the last tracing call on this thread and copies
 * its counters. */
int qsl_last_stats(qsl_stats* out);

/* ---- field ------------------------------------------------------------------- */
typedef struct qsl_field qsl_field; /* opaque; library-owned device copy */

/* Loads B (three arrays nz x ny x nx, x fastest, dtype QSL_F32|QSL_F64, in
 * `mem`) sampled at the vertices of a rectilinear grid with strictly
 * increasing host coordinates xc[nx], yc[ny], zc[nz] (Sec. "Code Overview":
 * input cubes on a rectilinear grid), and packs it per vertex as float4:
 * (B/|B|, |B|) for QSL_PAPER_NORMALIZE_FIRST, (B, |B|) for QSL_RAW_B. A zero
 * vertex packs as (0,0,0,0). Every n >= 2. QSL_ENONFINITE if any component
 * is not finite. The handle owns its device memory until qsl_free_field. */
int qsl_load_field(const void* bx, const void* by, const void* bz, int dtype, int mem, int nx, int ny, int nz,
                   const double* xc, const double* yc, const double* zc, int interp_mode, void* stream,
                   qsl_field** out);
void qsl_free_field(qsl_field* field);

/* ---- tracing ----------------------------------------------------------------- */
/* Traces one field line per seed (seeds: S x 3 doubles in `mem`) forwards and
 * backwards to the domain faces (Sec. "Squashing factor calculation"),
 * integrating the field-line equation (Eq. fl) and the linearised deviation
 * equation (Eq. dev) for two orthonormal initial deviations (Eq. ic), and
 * writes one qsl_line per seed (`out`, S records in `mem`). S may be 0. */
int qsl_trace_seeds(const qsl_field* field, const double* seeds, int64_t S, const qsl_opts* opts, qsl_line* out,
                    int mem, void* stream);

/* Q / FLL map on a planar slice (Sec. "Code Overview": centre, orientation and
 * axes span): pixel (i, j), i < nu fastest, is seeded at
 *   center + ((i + 0.5)/nu - 0.5) u + ((j + 0.5)/nv - 0.5) v.
 * Outputs (each optional, nu*nv entries in `mem`): q (float, opts.q_form),
 * length (float), faces (2 bytes per pixel: face_F, face_B), status (byte). */
int qsl_q_map_2d(const qsl_field* field, const double center[3], const double u[3], const double v[3], int nu,
                 int nv, const qsl_opts* opts, float* q, float* length, uint8_t* faces, uint8_t* status, int mem,
                 void* stream);

/* Q / FLL volume: seeds at the cell centres of an nx x ny x nz lattice over the
 * box [lo, hi] (x fastest). Outputs as qsl_q_map_2d. */
int qsl_q_volume_3d(const qsl_field* field, const double lo[3], const double hi[3], int nx, int ny, int nz,
                    const qsl_opts* opts, float* q, float* length, uint8_t* faces, uint8_t* status, int mem,
                    void* stream);

/* FLEDGE map (Sec. "Adaptive refinements"): gradient magnitude of the Sobel
 * operator applied to a 2D or 3D length map `length` (shape[0] slowest, in
 * `mem`). Unnormalised separable Sobel ([-1,0,1] derivative, [1,2,1]
 * smoothing), half-sample-symmetric boundary, index units; non-finite lengths
 * count as the largest finite length of the map. s_out has the same shape. */
int qsl_fledge(const float* length, int ndim, const int64_t* shape, float* s_out, int mem, void* stream);

/* ---- Hilbert-curve refinement (Sec. "Adaptive refinements") ------------------- */
typedef struct qsl_refine_spec {
  int32_t ndim;          /* 2: planar slice (center, u, v); 3: volume (lo, hi)         */
  int32_t coarse_order;  /* p0: the coarse pass samples every 2^(p-p0)-th cell          */
  int32_t max_order;     /* p: effective lattice 2^p cells per axis (p <= 20 in 3D, 30 in 2D) */
  int32_t max_iters;     /* refinement iterations (each: curve pass + shifted pass)       */
  int32_t extent[3];     /* effective lattice extent per axis, <= 2^p, multiple of 2^(p-p0); 0: 2^p */
  int32_t shift;         /* 1: shifted-curve pass after each refinement pass                */
  int32_t out_order;     /* converter output order (<= p); 0: p                             */
  int32_t proposal_stride; /* with a proposal: the effective cells of a proposed coarse cell
                              that are sampled, every stride-th per axis at offset stride / 2
                              (stride 2 with out_order = p - 1: one sample per output cell);
                              0 or 1: every effective cell; a power of two <= 2^(p - p0)  */
  double center[3], u[3], v[3]; /* planar slice, as in qsl_q_map_2d                     */
  double lo[3], hi[3];          /* volume box                                             */
  double tau;                   /* refine a pair when |L_i - L_i+1| > tau; tau < 0: every pair */
  const uint8_t* proposal;      /* optional (device or host per `mem`): one byte per coarse
                                   cell, x fastest; nonzero cells are sampled (at the
                                   effective cells proposal_stride selects) before the
                                   first iteration                                     */
  int32_t criterion;            /* QSL_REFINE_FLL_JUMP (0): |L_i - L_i+1| > tau (the paper's);
                                   QSL_REFINE_Q_THRESHOLD (1): a pair is refined when either
                                   sample's Q (opts.q_form) is finite and > q_threshold, the
                                   alternative Sec. "Adaptive refinements" compares against */
  int32_t pass_stepper;         /* tracer of the FLL-jump decisions of the refinement passes
                                   (criterion QSL_REFINE_FLL_JUMP, opts.length_only == 0):
                                   QSL_PASS_CASH_KARP (0, default): lengths only, traced by the
                                     paper's Cash-Karp stepper across cells at opts' tolerance
                                     and the step cap pass_h_max; Cartesian fields;
                                   QSL_PASS_SAME (1): lengths only with opts' integrator when it
                                     is QSL_DOPRI5_CELL on a uniform grid, else as QSL_PASS_FULL;
                                   QSL_PASS_FULL (2): the passes trace with opts unchanged.
                                   With 0 and 1 one launch after the last iteration traces every
                                   pass sample with opts (deviation equations, FP64 retrace) and
                                   its values are the ones stored; the decision lengths only
                                   chose the samples. Other criteria, and 0 on spherical fields,
                                   trace as QSL_PASS_FULL.                                   */
  double q_threshold;
  double pass_h_max;            /* step cap of QSL_PASS_CASH_KARP in smallest grid spacings;
                                   0: 4                                                      */
} qsl_refine_spec;
#define QSL_REFINE_FLL_JUMP 0
#define QSL_REFINE_Q_THRESHOLD 1
#define QSL_PASS_CASH_KARP 0
#define QSL_PASS_SAME 1
#define QSL_PASS_FULL 2

typedef struct qsl_samples {
  int64_t capacity;  /* entries the arrays below can hold                           */
  int64_t count;     /* in: samples already present (resume); out: samples now       */
  uint64_t* key;     /* Hilbert keys at max_order, sorted ascending                    */
  float* q;          /* opts.q_form per sample                                         */
  float* length;
  uint8_t* faces;    /* 2 per sample (optional)                                        */
  uint8_t* status;   /* 1 per sample (optional)                                        */
  int32_t iters;     /* out: iterations run                                            */
  int32_t traced;    /* out: samples traced by this call (low 31 bits)                 */
  int32_t* origin;   /* optional (NULL): the pass of this call that added each sample:
                        0 the coarse pass or the proposal, 2i + 1 the pass along the
                        curve of iteration i, 2i + 2 its shifted-curve pass; entries
                        of resumed samples are kept                                    */
} qsl_samples;

/* Refines seeds along a Hilbert curve wherever the field-line length jumps by
 * more than tau between samples adjacent along the curve, then converts the
 * samples to the rectilinear output lattice (extent >> (p - out_order) per
 * axis, x fastest): a cell takes the maximum of its samples, an empty cell the
 * value interpolated along the curve (log10 for Q). q_grid / l_grid optional.
 * Samples sit at effective-cell centres; positions as in qsl_q_map_2d /
 * qsl_q_volume_3d over the effective lattice. With samples->count > 0 the
 * call resumes from those (sorted) samples instead of the coarse pass.
 * QSL_ECAPACITY when the capacity is reached (samples so far are valid).
 * With the FLL-jump criterion the refinement passes trace lengths only (the
 * criterion reads L) with the tracer spec->pass_stepper names, and the pass
 * samples' Q, L, end faces and status come from one trace with opts after the
 * last iteration. The coarse pass (and a proposal) always trace with opts. */
int qsl_refine(const qsl_field* field, const qsl_refine_spec* spec, const qsl_opts* opts, qsl_samples* samples,
               float* q_grid, float* l_grid, int mem, void* stream);

/* Time accounting of the last qsl_refine on this thread (no paper counterpart;
 * CUDA events on the call's stream). total_ms spans the whole call on the
 * device; coarse_ms the tracing of the coarse pass (and of a proposal);
 * passes_ms the tracing of the refinement passes (length-only with the
 * FLL-jump criterion); deferred_ms the one trace of all pass samples with the
 * deviation equations (FP64 assembly and retrace included) that follows the
 * last iteration with that criterion; the rest is sorting, merging, flagging,
 * conversion and host round trips. Synchronises that stream. QSL_EINVAL
 * before the first qsl_refine. */
typedef struct qsl_refine_stats {
  double total_ms, coarse_ms, passes_ms, deferred_ms;
  int64_t coarse_lines, pass_lines; /* seeds traced                                      */
  int64_t coarse_stage_evals, pass_stage_evals, deferred_stage_evals; /* FP32 tracer
                                       stage evaluations (the first 512 trace calls)     */
  int32_t passes, iters;            /* refinement pass trace calls, iterations           */
  int64_t coarse_landings, pass_landings, deferred_landings; /* plane crossings of the
                                       cell-wise tracers (cell entries and ends), same calls */
} qsl_refine_stats; /* 104 bytes */
int qsl_last_refine_stats(qsl_refine_stats* out);

/* ---- batches of fields and cuts: one persistent launch, captured plans ---------
 * Many planar cuts of many fields (each its own grid size) traced in one
 * persistent launch: the work queue spans all items, so uneven line lengths
 * and unequal items share the GPU. Item k's pixels are written at offset
 * sum_{i<k} nu_i*nv_i of the outputs (items concatenated in order, pixel
 * layout as qsl_q_map_2d). Mixed uniform and rectilinear fields trace with
 * QSL_RKCK54. */
typedef struct qsl_batch_item {
  const qsl_field* field;
  double center[3], u[3], v[3]; /* planar cut, as qsl_q_map_2d */
  int32_t nu, nv;
} qsl_batch_item;

/* One-shot batch: device outputs only (mem must be QSL_MEM_DEVICE). Returns
 * after the work completes. */
int qsl_q_map_batch(const qsl_batch_item* items, int n_items, const qsl_opts* opts, float* q, float* length,
                    uint8_t* faces, uint8_t* status, int mem, void* stream);

/* Plans: the batch (trace, FP64 assembly, selection and FP64 retrace of lines
 * above retrace_q with a device-side count) recorded once into a CUDA graph
 * with all scratch owned by the plan; qsl_plan_launch replays it on `stream`
 * with no allocation and no host synchronisation. Outputs (device memory) are
 * fixed at plan time; the fields must outlive the plan. */
typedef struct qsl_plan qsl_plan;
int qsl_plan_q_map_batch(const qsl_batch_item* items, int n_items, const qsl_opts* opts, float* q, float* length,
                         uint8_t* faces, uint8_t* status, qsl_plan** out);
int qsl_plan_launch(qsl_plan* plan, void* stream);
/* Synchronises `stream` and copies the counters of the plan's last replay. */
int qsl_plan_stats(qsl_plan* plan, void* stream, qsl_stats* out);
void qsl_plan_free(qsl_plan* plan);

/* ---- learned refinement proposal (an addition to the method; the paper has none) 
 * A 3-layer CNN over coarse tiles with 2 channels (normalised FLEDGE, log10 Q)
 * giving, per coarse cell, the probability that FLL-jump refinement
 * (Sec. "Adaptive refinements") will sample inside it:
 *   conv3x3 2->32 + ReLU, conv3x3 32->32 + ReLU, conv3x3 32->1 (logit),
 * zero padding, stride 1. Weights are BF16 in the passes (FP32 master copy and
 * Adam state); contractions accumulate in FP32. Parameters, flattened in this
 * order: w1[32][2][3][3], b1[32], w2[32][32][3][3], b2[32], w3[1][32][3][3],
 * b3[1] (QSL_CNN_NPARAMS floats). Tensors are NCHW float32 in device memory. */
#define QSL_CNN_NPARAMS (32 * 2 * 9 + 32 + 32 * 32 * 9 + 32 + 32 * 9 + 1)
typedef struct qsl_cnn qsl_cnn;
/* params: host array of QSL_CNN_NPARAMS floats (initial FP32 master). */
int qsl_cnn_create(const float* params, qsl_cnn** out);
/* Copies the FP32 master parameters to host memory. */
int qsl_cnn_params(const qsl_cnn* cnn, float* params);
/* prob[n][h][w] = sigmoid(logit) for x[n][2][h][w]. */
int qsl_cnn_forward(qsl_cnn* cnn, const float* x, int n, int h, int w, float* prob, void* stream);
/* Mean binary cross-entropy over pixels, pos_weight * y * softplus(-z) +
 * (1 - y) * softplus(z), and its gradient w.r.t. the parameters (device,
 * QSL_CNN_NPARAMS floats; overwritten). loss: one device float. */
int qsl_cnn_loss_grad(qsl_cnn* cnn, const float* x, const float* y, int n, int h, int w, float pos_weight,
                      float* loss, float* grad, void* stream);
/* One Adam update (bias-corrected) of the FP32 master from `grad`; refreshes
 * the BF16 weights. */
int qsl_cnn_adam_step(qsl_cnn* cnn, const float* grad, float lr, float beta1, float beta2, float eps, void* stream);
void qsl_cnn_free(qsl_cnn* cnn);
int qsl_cnn_nparams(void);
/* Network input (device, NCHW X[nz][2][ny][nx]) of the nz z-slices of a
 * coarse map or volume from its FLEDGE map S (qsl_fledge of the coarse
 * lengths) and Q (both [nz][ny][nx], device): channel 0 S over the largest
 * finite S of its slice (non-finite entries 0), channel 1 (log10 Q - 2) / 2
 * clamped to [-2, 3] (NaN Q counts as Q = 2). */
int qsl_cnn_features(const float* S, const float* Q, int nz, int ny, int nx, float* X, void* stream);
/* Proposal mask dilation (device bytes [nz][ny][nx]): out = 1 where any cell
 * of the 3 x 3 x 3 neighbourhood of `in`, clipped to the volume, is nonzero.
 * in and out must not alias. */
int qsl_mask_dilate(const uint8_t* in, int nz, int ny, int nx, uint8_t* out, void* stream);

/* ---- autotuner -----------------------------------------------------------------
 * Picks, on a sample of S seeds (device memory, S >= 1) of the caller's
 * workload:
 *  - the loosest tolerance in {1e-5, 1e-6, 1e-7} (FP32 tracing; FP64:
 *    {1e-6, ..., 1e-9}) whose Q (relative error <= 2e-4 for Q < 1e6), lengths
 *    (|dL| <= 2e-6 L for lines of at least the smallest spacing h) and end
 *    faces (<= 0.1 % of lines differ) agree with an FP64 trace of the same
 *    seeds at tol 1e-10 (a fifth of the 1e-3 / 1e-5 accuracy bar); lines
 *    shorter than h, whose length error is set by the FP32 field samples and
 *    not by the tolerance, are held to |dL| <= 1e-5 h. Candidates run the caller's precision
 *    policy, FP64 retrace above retrace_q included. When none passes, the
 *    tightest is taken and report->passed is 0;
 *  - the step cap: the requested h_max, or 4 smallest spacings when that also
 *    meets the bounds;
 *  - the fastest launch shape (warps per block 2/4/8, blocks per SM at most
 *    2 or as many as fit, refill threshold 1, 4, 8 or 16) and step cap at that
 *    tolerance, timed with CUDA events on `stream` on the sample repeated
 *    until one launch holds at least 16 x 384 line directions per SM (a
 *    throughput measurement; the sample's own launch is often as long as its
 *    longest line). The repeated sample and its records are allocated for
 *    the call (S x 3 doubles and S records per copy).
 * Writes the choice into *opts (tol_abs = tol_rel, h_max, warps_per_block,
 * blocks_per_sm, refill_min) and into *report (optional). The result is cached
 * per (grid size, interpolation mode, integrator, q_form, length_only, input
 * tolerance); a cached call does no GPU work. Synchronous. */
typedef struct qsl_tune_report {
  int32_t warps_per_block, blocks_per_sm, refill_min, cached;
  double tol;            /* chosen tolerance                                  */
  double q_err, l_err;   /* worst relative errors at that tolerance           */
  double face_mismatch;  /* fraction of sample lines with different end faces */
  double sample_ms;      /* time of the chosen shape on the sample repeated
                            shape_reps times (one launch)                      */
  int64_t sample_seeds;
  double h_max;          /* chosen step cap (units of the smallest spacing)   */
  int32_t passed;        /* 1: the chosen tolerance met the bounds; 0: none of
                            the candidates did and the tightest was taken      */
  int32_t shape_reps;    /* copies of the sample in each shape timing         */
  double l_err_subcell;  /* worst length error of lines shorter than one cell,
                            in cells (held to the full bar, 1e-5)              */
} qsl_tune_report;
int qsl_autotune(const qsl_field* field, const double* seeds, int64_t S, qsl_opts* opts, qsl_tune_report* report,
                 void* stream);

/* ---- tracing without allocation -------------------------------------------------
 * The paper has no counterpart to this entry point. It is qsl_trace_seeds for
 * callers that cannot allocate device memory (a host-side allocator or fixed
 * memory budget they must not bypass, or allocator state that must not change):
 * it calls no cudaMalloc, cudaFree or allocating library routine. Its scratch
 * (queue head and per-direction end records) is one file-scope device array of
 * QSL_NOALLOC_SCRATCH_BYTES (7 MiB + 256 B) that every GPU loading this library
 * holds until the process exits.
 *  - seeds (S x 3 doubles) and out (S records) must be device memory of the
 *    current device; 0 <= S <= QSL_NOALLOC_MAX_SEEDS, else QSL_EINVAL.
 *  - FP32 tracing only (opts->precision must be QSL_FP32_MIXED, else
 *    QSL_EINVAL); lines above retrace_q are not traced again in FP64 and
 *    qsl_last_stats does not report this call.
 *  - The first call on a device looks up the array's device address (with that
 *    device current); make it before any stream capture.
 *  - Every call shares the one array: calls whose work overlaps on the GPU
 *    (other streams, other host threads) race; serialise them.
 *  - Asynchronous on `stream`. */
#define QSL_NOALLOC_MAX_SEEDS 65536
#define QSL_NOALLOC_SCRATCH_BYTES (256 + 56 * 2 * 65536)
int qsl_trace_seeds_noalloc(const qsl_field* field, const double* seeds, int64_t S, const qsl_opts* opts,
                            qsl_line* out, void* stream);

/* Hilbert keys (Skilling's transpose method, curve starting at the origin) of
 * n cells with coords (n x ndim uint32, axis 0 first) at `bits` per axis
 * (ndim * bits <= 63), and the inverse. */
int qsl_hilbert_encode(const uint32_t* coords, int64_t n, int ndim, int bits, uint64_t* keys, int mem,
                       void* stream);
int qsl_hilbert_decode(const uint64_t* keys, int64_t n, int ndim, int bits, uint32_t* coords, int mem,
                       void* stream);

/* Hilbert -> rectilinear converter alone (the last step of qsl_refine): keys
 * sorted ascending at max_order, vals per key. */
int qsl_convert(const uint64_t* keys, const float* vals, int64_t n, int ndim, int max_order, const int32_t* extent,
                int out_order, int log_interp, float* out, int mem, void* stream);

/* Geometry of a loaded field (Sec. "Integrating field lines"):
 * QSL_GEOM_CARTESIAN (default) or QSL_GEOM_SPHERICAL. Spherical: the grid's
 * axes are longitude phi and latitude theta (radians, latitudes inside
 * (-pi/2, pi/2)) and radius r > 0, uniform on each axis; the three field
 * arrays are B_phi, B_theta, B_r in the local orthonormal basis. Field lines
 * follow Eq. fl_sph and the deviations Eq. dev_sph (the paper's form, without
 * the terms of the metric factors' variation); seeds and end points are
 * (phi, theta, r); planar seeds (qsl_q_map_2d) are planes in these
 * coordinates, so (0, 0, r0) + u = (dphi, 0, 0), v = (0, dtheta, 0) is the
 * spherical slice at radius r0. Eq. ic's vectors are orthonormal in the
 * seed's physical frame; Q uses the deviations as physical vectors in each
 * end's frame; step bounds are in units of the smallest physical cell edge
 * at the lowest radius; the step error is measured on physical lengths.
 * Runs with QSL_RKCK54 or QSL_EULER (any interpolation order). */
#define QSL_GEOM_CARTESIAN 0
#define QSL_GEOM_SPHERICAL 1
int qsl_set_geometry(qsl_field* field, int geometry);

/* Device memory: the library's temporary buffers (tracer scratch, refinement
 * work arrays, sort storage) come from its own stream-ordered pool on each
 * device, which keeps freed blocks cached for the next call (no return to the
 * driver at each synchronisation; peak about 100 bytes per refinement sample
 * of capacity). qsl_trim_pool hands the cached blocks back to the driver on
 * every device the library has used (no paper counterpart). Synchronous with
 * respect to nothing: blocks still in use by queued work stay allocated. */
int qsl_trim_pool(void);

/* Check of the library's FP64 Newton-Raphson reciprocal square root and
 * reciprocal (used by the field pack and the Q assembly; no paper
 * counterpart) against CUDA's 1 / sqrt(x) and 1 / x: x are n host values;
 * max_ulp_out (host, 2 doubles) receives the largest difference of each, in
 * units in the last place of CUDA's result, over the finite positive inputs.
 * Synchronous (default stream). QSL_EINVAL for n < 1 or NULL pointers. */
int qsl_check_fp64_newton(const double* x, int64_t n, double* max_ulp_out);

/* Kernels of this library launched by this process since the library was
 * loaded (all threads). Radix sorts and scans inside qsl_refine run CUB
 * kernels, which are not counted. */
int64_t qsl_kernel_launches(void);

/* Human-readable message of the last failing call on this thread. */
const char* qsl_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* QSL_H */
