"""Thin ctypes binding of libqsl.so (include/qsl.h), same names as the C ABI.

Argument marshalling only: arrays are torch tensors (device memory, current
stream) or numpy arrays (host memory); every step of the computation runs in
the library's CUDA kernels. Loading fails loudly when libqsl.so is missing.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsl.so")

QSL_OK, QSL_EINVAL, QSL_ENOMEM, QSL_ECUDA, QSL_ETIMEOUT, QSL_ENONFINITE, QSL_ECAPACITY = 0, -1, -2, -3, -4, -5, -6
QSL_MEM_HOST, QSL_MEM_DEVICE = 0, 1
QSL_F32, QSL_F64 = 0, 1
QSL_PAPER_NORMALIZE_FIRST, QSL_RAW_B = 0, 1
QSL_RKCK54, QSL_EULER, QSL_DOPRI5_CELL = 0, 1, 2
QSL_Q_PERP, QSL_Q_FOOT, QSL_Q_DET = 0, 1, 2
QSL_FP32_MIXED, QSL_FP64 = 0, 1
(QSL_LINE_OK, QSL_LINE_MAXLEN, QSL_LINE_MAXSTEPS, QSL_LINE_STALL, QSL_LINE_OUTSIDE, QSL_LINE_NONFINITE,
 QSL_LINE_NULL, QSL_LINE_TIMEOUT) = range(8)
QSL_FLAG_OPEN_SKIPPED, QSL_FLAG_RETRACED = 0x40, 0x80
QSL_NO_FACE = 255


class QslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("qsl error %d: %s" % (code, msg))
        self.code = code


class qsl_opts(C.Structure):
    _fields_ = [("integrator", C.c_int32), ("q_form", C.c_int32), ("precision", C.c_int32),
                ("skip_open", C.c_int32), ("length_only", C.c_int32), ("warps_per_block", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("refill_min", C.c_int32), ("tol_abs", C.c_double),
                ("tol_rel", C.c_double), ("h_init", C.c_double), ("h_max", C.c_double), ("h_min", C.c_double),
                ("max_length", C.c_double), ("max_steps", C.c_int64), ("euler_h", C.c_double),
                ("retrace_q", C.c_double), ("domain_lo", C.c_double * 3), ("domain_hi", C.c_double * 3),
                ("land_tol", C.c_double), ("timeout_s", C.c_double), ("line_lanes", C.c_int32),
                ("interp_order", C.c_int32)]


QSL_LINE_DTYPE = np.dtype([("q_perp", "<f8"), ("q_foot", "<f8"), ("q_det", "<f8"), ("b0", "<f8"), ("bf", "<f8"),
                           ("bb", "<f8"), ("flux_f", "<f8"), ("flux_b", "<f8"), ("length", "<f4"),
                           ("lam_f", "<f4"), ("lam_b", "<f4"), ("pad0", "<f4"), ("x_f", "<f4", (3,)),
                           ("x_b", "<f4", (3,)), ("steps", "<i4"), ("face_f", "u1"), ("face_b", "u1"),
                           ("status_f", "u1"), ("status_b", "u1")])
assert QSL_LINE_DTYPE.itemsize == 112


class qsl_stats(C.Structure):
    _fields_ = [("lines", C.c_int64), ("stage_evals", C.c_int64), ("accepted", C.c_int64), ("rejected", C.c_int64),
                ("landing", C.c_int64), ("retraced", C.c_int64), ("kernel_ms", C.c_double),
                ("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("refill_min", C.c_int32),
                ("pad", C.c_int32)]


class qsl_refine_stats(C.Structure):
    _fields_ = [("total_ms", C.c_double), ("coarse_ms", C.c_double), ("passes_ms", C.c_double),
                ("deferred_ms", C.c_double), ("coarse_lines", C.c_int64), ("pass_lines", C.c_int64),
                ("coarse_stage_evals", C.c_int64), ("pass_stage_evals", C.c_int64),
                ("deferred_stage_evals", C.c_int64), ("passes", C.c_int32), ("iters", C.c_int32),
                ("coarse_landings", C.c_int64), ("pass_landings", C.c_int64), ("deferred_landings", C.c_int64)]


class qsl_refine_spec(C.Structure):
    _fields_ = [("ndim", C.c_int32), ("coarse_order", C.c_int32), ("max_order", C.c_int32),
                ("max_iters", C.c_int32), ("extent", C.c_int32 * 3), ("shift", C.c_int32),
                ("out_order", C.c_int32), ("proposal_stride", C.c_int32), ("center", C.c_double * 3),
                ("u", C.c_double * 3),
                ("v", C.c_double * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("tau", C.c_double),
                ("proposal", C.c_void_p), ("criterion", C.c_int32), ("pass_stepper", C.c_int32),
                ("q_threshold", C.c_double), ("pass_h_max", C.c_double)]


QSL_REFINE_FLL_JUMP = 0
QSL_REFINE_Q_THRESHOLD = 1
QSL_PASS_CASH_KARP = 0
QSL_PASS_SAME = 1
QSL_PASS_FULL = 2


class qsl_samples(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("count", C.c_int64), ("key", C.c_void_p), ("q", C.c_void_p),
                ("length", C.c_void_p), ("faces", C.c_void_p), ("status", C.c_void_p), ("iters", C.c_int32),
                ("traced", C.c_int32), ("origin", C.c_void_p)]


class qsl_batch_item(C.Structure):
    _fields_ = [("field", C.c_void_p), ("center", C.c_double * 3), ("u", C.c_double * 3), ("v", C.c_double * 3),
                ("nu", C.c_int32), ("nv", C.c_int32)]


class qsl_tune_report(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("blocks_per_sm", C.c_int32), ("refill_min", C.c_int32),
                ("cached", C.c_int32), ("tol", C.c_double), ("q_err", C.c_double), ("l_err", C.c_double),
                ("face_mismatch", C.c_double), ("sample_ms", C.c_double), ("sample_seeds", C.c_int64),
                ("h_max", C.c_double), ("passed", C.c_int32), ("shape_reps", C.c_int32),
                ("l_err_subcell", C.c_double)]


_lib = None


def lib():
    """Loads libqsl.so (built in-tree by paper_1609_00724_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError("libqsl.so not found at %s: build it with `python -m paper_1609_00724_gb300.build`"
                      % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dp = C.c_void_p, C.c_int, C.c_int64, C.c_void_p
    L.qsl_last_error.restype = C.c_char_p
    L.qsl_check_fp64_newton.argtypes = [vp, i64, vp]
    L.qsl_opts_default.argtypes = [C.POINTER(qsl_opts)]
    L.qsl_load_field.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, dp, dp, dp, i32, vp, C.POINTER(vp)]
    L.qsl_free_field.argtypes = [vp]
    L.qsl_trace_seeds.argtypes = [vp, vp, i64, C.POINTER(qsl_opts), vp, i32, vp]
    L.qsl_q_map_2d.argtypes = [vp, dp, dp, dp, i32, i32, C.POINTER(qsl_opts), vp, vp, vp, vp, i32, vp]
    L.qsl_q_volume_3d.argtypes = [vp, dp, dp, i32, i32, i32, C.POINTER(qsl_opts), vp, vp, vp, vp, i32, vp]
    L.qsl_fledge.argtypes = [vp, i32, vp, vp, i32, vp]
    L.qsl_refine.argtypes = [vp, C.POINTER(qsl_refine_spec), C.POINTER(qsl_opts), C.POINTER(qsl_samples), vp, vp,
                             i32, vp]
    L.qsl_hilbert_encode.argtypes = [vp, i64, i32, i32, vp, i32, vp]
    L.qsl_hilbert_decode.argtypes = [vp, i64, i32, i32, vp, i32, vp]
    L.qsl_convert.argtypes = [vp, vp, i64, i32, i32, vp, i32, i32, vp, i32, vp]
    L.qsl_last_stats.argtypes = [C.POINTER(qsl_stats)]
    L.qsl_kernel_launches.restype = C.c_int64
    L.qsl_q_map_batch.argtypes = [C.POINTER(qsl_batch_item), i32, C.POINTER(qsl_opts), vp, vp, vp, vp, i32, vp]
    L.qsl_plan_q_map_batch.argtypes = [C.POINTER(qsl_batch_item), i32, C.POINTER(qsl_opts), vp, vp, vp, vp,
                                       C.POINTER(vp)]
    L.qsl_plan_launch.argtypes = [vp, vp]
    L.qsl_plan_stats.argtypes = [vp, vp, C.POINTER(qsl_stats)]
    L.qsl_plan_free.argtypes = [vp]
    L.qsl_cnn_create.argtypes = [vp, C.POINTER(vp)]
    L.qsl_cnn_params.argtypes = [vp, vp]
    L.qsl_cnn_forward.argtypes = [vp, vp, i32, i32, i32, vp, vp]
    L.qsl_cnn_loss_grad.argtypes = [vp, vp, vp, i32, i32, i32, C.c_float, vp, vp, vp]
    L.qsl_cnn_adam_step.argtypes = [vp, vp, C.c_float, C.c_float, C.c_float, C.c_float, vp]
    L.qsl_cnn_free.argtypes = [vp]
    L.qsl_cnn_features.argtypes = [vp, vp, i32, i32, i32, vp, vp]
    L.qsl_mask_dilate.argtypes = [vp, i32, i32, i32, vp, vp]
    L.qsl_autotune.argtypes = [vp, vp, i64, C.POINTER(qsl_opts), C.POINTER(qsl_tune_report), vp]
    L.qsl_trace_seeds_noalloc.argtypes = [vp, vp, i64, C.POINTER(qsl_opts), vp, vp]
    _lib = L
    return L


def _check(rc):
    if rc != QSL_OK:
        raise QslError(rc, lib().qsl_last_error().decode())
    return rc


# ------------------------------------------------------------------ marshalling
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _mem_of(*arrays):
    kinds = {(_is_torch(a) and a.is_cuda) for a in arrays if a is not None}
    if len(kinds) > 1:
        raise ValueError("mix of device and host arrays")
    return QSL_MEM_DEVICE if kinds == {True} else QSL_MEM_HOST


def _ptr(a):
    if a is None:
        return None
    if _is_torch(a):
        assert a.is_contiguous(), "tensor must be contiguous"
        return C.c_void_p(a.data_ptr())
    assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
    return C.c_void_p(a.ctypes.data)


def _stream(stream=None):
    if stream is not None:
        return C.c_void_p(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


def _d3(v):
    return (C.c_double * 3)(*[float(x) for x in v])


def qsl_opts_default(**kw):
    o = qsl_opts()
    lib().qsl_opts_default(C.byref(o))
    for k, v in kw.items():
        if k in ("domain_lo", "domain_hi"):
            getattr(o, k)[:] = [float(x) for x in v]
        else:
            setattr(o, k, v)
    return o


class Field:
    """Owned handle of a packed field (qsl_load_field / qsl_free_field)."""

    def __init__(self, handle, shape):
        self.handle = handle
        self.shape = shape

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsl_free_field(self.handle)
            self.handle = None


def qsl_load_field(bx, by, bz, xc, yc, zc, interp_mode=QSL_PAPER_NORMALIZE_FIRST, stream=None):
    """bx, by, bz: [nz, ny, nx] float32/float64 (torch CUDA tensors or numpy)."""
    mem = _mem_of(bx, by, bz)
    dt = str(bx.dtype)
    dtype = QSL_F64 if "64" in dt else QSL_F32
    nz, ny, nx = bx.shape
    ax = [np.ascontiguousarray(a, dtype=np.float64) for a in (xc, yc, zc)]
    h = C.c_void_p()
    _check(lib().qsl_load_field(_ptr(bx), _ptr(by), _ptr(bz), dtype, mem, nx, ny, nz,
                                *(a.ctypes.data_as(C.c_void_p) for a in ax), interp_mode, _stream(stream),
                                C.byref(h)))
    return Field(h, (nx, ny, nz))


def qsl_trace_seeds(field, seeds, opts, out=None, stream=None):
    """seeds: S x 3 float64. Returns a numpy record array (host seeds) or a
    torch uint8 tensor of S*112 bytes (device seeds)."""
    S = seeds.shape[0]
    mem = _mem_of(seeds)
    if out is None:
        if mem == QSL_MEM_DEVICE:
            import torch
            out = torch.empty(S * QSL_LINE_DTYPE.itemsize, dtype=torch.uint8, device=seeds.device)
        else:
            out = np.zeros(S, dtype=QSL_LINE_DTYPE)
    _check(lib().qsl_trace_seeds(field.handle, _ptr(seeds), S, C.byref(opts), _ptr(out), mem, _stream(stream)))
    return out


def _batch_items(items):
    """items: list of (Field, center, u, v, nu, nv)."""
    arr = (qsl_batch_item * len(items))()
    for k, (F, c, u, v, nu, nv) in enumerate(items):
        arr[k].field = F.handle.value if hasattr(F.handle, "value") else F.handle
        arr[k].center[:] = [float(x) for x in c]
        arr[k].u[:] = [float(x) for x in u]
        arr[k].v[:] = [float(x) for x in v]
        arr[k].nu, arr[k].nv = int(nu), int(nv)
    return arr


def qsl_q_map_batch(items, opts, q=None, length=None, faces=None, status=None, stream=None):
    """Maps of many (field, cut) items in one persistent launch; outputs are
    device tensors holding the items' pixels concatenated in order."""
    arr = _batch_items(items)
    _check(lib().qsl_q_map_batch(arr, len(items), C.byref(opts), _ptr(q), _ptr(length), _ptr(faces), _ptr(status),
                                 QSL_MEM_DEVICE, _stream(stream)))


class Plan:
    """A batch recorded into a CUDA graph (qsl_plan_q_map_batch)."""

    def __init__(self, items, opts, q=None, length=None, faces=None, status=None):
        self._keep = (items, q, length, faces, status)
        arr = _batch_items(items)
        h = C.c_void_p()
        _check(lib().qsl_plan_q_map_batch(arr, len(items), C.byref(opts), _ptr(q), _ptr(length), _ptr(faces),
                                          _ptr(status), C.byref(h)))
        self.handle = h

    def launch(self, stream=None):
        _check(lib().qsl_plan_launch(self.handle, _stream(stream)))

    def stats(self, stream=None):
        st = qsl_stats()
        _check(lib().qsl_plan_stats(self.handle, _stream(stream), C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_ if k != "pad"}

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsl_plan_free(self.handle)
            self.handle = None


def qsl_autotune(field, seeds, opts, stream=None):
    """Tunes opts in place on device sample seeds (S x 3 float64); returns the report."""
    rep = qsl_tune_report()
    _check(lib().qsl_autotune(field.handle, _ptr(seeds), seeds.shape[0], C.byref(opts), C.byref(rep),
                              _stream(stream)))
    return {k: getattr(rep, k) for k, _ in rep._fields_}


QSL_CNN_NPARAMS = 32 * 2 * 9 + 32 + 32 * 32 * 9 + 32 + 32 * 9 + 1


def qsl_cnn_features(S, Q, X, stream=None):
    """CNN input X [nz, 2, ny, nx] from FLEDGE S and Q ([nz, ny, nx] or [ny, nx]), device tensors."""
    nz, ny, nx = (1,) + tuple(S.shape) if S.dim() == 2 else tuple(S.shape)
    _check(lib().qsl_cnn_features(_ptr(S), _ptr(Q), nz, ny, nx, _ptr(X), _stream(stream)))
    return X


def qsl_mask_dilate(mask, out, stream=None):
    """3 x 3 x 3 dilation of a uint8 device mask ([nz, ny, nx] or [ny, nx])."""
    nz, ny, nx = (1,) + tuple(mask.shape) if mask.dim() == 2 else tuple(mask.shape)
    _check(lib().qsl_mask_dilate(_ptr(mask), nz, ny, nx, _ptr(out), _stream(stream)))
    return out


class Cnn:
    """The refinement-proposal CNN (qsl_cnn_*): forward, loss/gradient, Adam."""

    def __init__(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == QSL_CNN_NPARAMS
        h = C.c_void_p()
        _check(lib().qsl_cnn_create(p.ctypes.data_as(C.c_void_p), C.byref(h)))
        self.handle = h

    def params(self):
        out = np.zeros(QSL_CNN_NPARAMS, dtype=np.float32)
        _check(lib().qsl_cnn_params(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def forward(self, x, prob=None, stream=None):
        n, c, h, w = x.shape
        assert c == 2
        if prob is None:
            import torch
            prob = torch.empty((n, h, w), dtype=torch.float32, device=x.device)
        _check(lib().qsl_cnn_forward(self.handle, _ptr(x), n, h, w, _ptr(prob), _stream(stream)))
        return prob

    def loss_grad(self, x, y, pos_weight, loss, grad, stream=None):
        n, c, h, w = x.shape
        _check(lib().qsl_cnn_loss_grad(self.handle, _ptr(x), _ptr(y), n, h, w, C.c_float(pos_weight), _ptr(loss),
                                       _ptr(grad), _stream(stream)))

    def adam(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(lib().qsl_cnn_adam_step(self.handle, _ptr(grad), C.c_float(lr), C.c_float(beta1), C.c_float(beta2),
                                       C.c_float(eps), _stream(stream)))

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qsl_cnn_free(self.handle)
            self.handle = None


QSL_NOALLOC_MAX_SEEDS = 65536


def qsl_trace_seeds_noalloc(field, seeds, opts, out, stream=None):
    """Allocation-free variant of qsl_trace_seeds: seeds (S x 3 float64) and
    out (S * 112 bytes) must be CUDA tensors; S <= QSL_NOALLOC_MAX_SEEDS."""
    _check(lib().qsl_trace_seeds_noalloc(field.handle, _ptr(seeds), seeds.shape[0], C.byref(opts), _ptr(out),
                                         _stream(stream)))
    return out


def lines_to_numpy(raw):
    """Device qsl_line bytes (torch uint8) -> numpy record array."""
    return np.frombuffer(raw.cpu().numpy().tobytes(), dtype=QSL_LINE_DTYPE)


def qsl_q_map_2d(field, center, u, v, nu, nv, opts, q=None, length=None, faces=None, status=None, stream=None):
    mem = _mem_of(q, length, faces, status)
    _check(lib().qsl_q_map_2d(field.handle, _d3(center), _d3(u), _d3(v), nu, nv, C.byref(opts), _ptr(q),
                              _ptr(length), _ptr(faces), _ptr(status), mem, _stream(stream)))


def qsl_q_volume_3d(field, lo, hi, nx, ny, nz, opts, q=None, length=None, faces=None, status=None, stream=None):
    mem = _mem_of(q, length, faces, status)
    _check(lib().qsl_q_volume_3d(field.handle, _d3(lo), _d3(hi), nx, ny, nz, C.byref(opts), _ptr(q), _ptr(length),
                                 _ptr(faces), _ptr(status), mem, _stream(stream)))


def qsl_fledge(length, s_out, stream=None):
    mem = _mem_of(length, s_out)
    shape = np.array(list(length.shape), dtype=np.int64)
    _check(lib().qsl_fledge(_ptr(length), len(length.shape), shape.ctypes.data_as(C.c_void_p), _ptr(s_out), mem,
                            _stream(stream)))


def refine_spec(**kw):
    s = qsl_refine_spec()
    s.max_iters = 64
    s.shift = 1
    for k, v in kw.items():
        if k in ("extent", "center", "u", "v", "lo", "hi"):
            arr = getattr(s, k)
            for i, x in enumerate(v):
                arr[i] = x
        elif k == "proposal":
            s._proposal_keep = v
            s.proposal = _ptr(v).value if v is not None else None
        else:
            setattr(s, k, v)
    return s


def qsl_refine(field, spec, opts, key, q, length, faces=None, status=None, count=0, q_grid=None, l_grid=None,
               stream=None, origin=None):
    """Sample arrays (capacity = len(key)) are caller-owned; origin (optional,
    int32) receives the pass that added each sample. Returns (count, iters,
    traced, rc) and raises on errors other than QSL_ECAPACITY."""
    mem = _mem_of(key, q, length, faces, status, q_grid, l_grid, origin)
    smp = qsl_samples()
    smp.capacity = key.shape[0]
    smp.count = count
    smp.key, smp.q, smp.length = (_ptr(a).value for a in (key, q, length))
    smp.faces = _ptr(faces).value if faces is not None else None
    smp.status = _ptr(status).value if status is not None else None
    smp.origin = _ptr(origin).value if origin is not None else None
    rc = lib().qsl_refine(field.handle, C.byref(spec), C.byref(opts), C.byref(smp), _ptr(q_grid), _ptr(l_grid), mem,
                          _stream(stream))
    if rc not in (QSL_OK, QSL_ECAPACITY):
        _check(rc)
    return int(smp.count), int(smp.iters), int(smp.traced), rc


def qsl_hilbert_encode(coords, ndim, bits, keys, stream=None):
    mem = _mem_of(coords, keys)
    _check(lib().qsl_hilbert_encode(_ptr(coords), coords.shape[0], ndim, bits, _ptr(keys), mem, _stream(stream)))


def qsl_hilbert_decode(keys, ndim, bits, coords, stream=None):
    mem = _mem_of(coords, keys)
    _check(lib().qsl_hilbert_decode(_ptr(keys), keys.shape[0], ndim, bits, _ptr(coords), mem, _stream(stream)))


def qsl_convert(keys, vals, ndim, max_order, extent, out_order, log_interp, out, stream=None):
    mem = _mem_of(keys, vals, out)
    ext = np.zeros(3, dtype=np.int32)
    ext[:ndim] = extent[:ndim]
    _check(lib().qsl_convert(_ptr(keys), _ptr(vals), keys.shape[0], ndim, max_order,
                             ext.ctypes.data_as(C.c_void_p), out_order, int(log_interp), _ptr(out), mem,
                             _stream(stream)))


def qsl_kernel_launches():
    return int(lib().qsl_kernel_launches())


def qsl_last_stats():
    s = qsl_stats()
    _check(lib().qsl_last_stats(C.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_ if k != "pad"}


QSL_GEOM_CARTESIAN = 0
QSL_GEOM_SPHERICAL = 1


def qsl_set_geometry(field, geometry):
    """Sets the field's geometry (QSL_GEOM_CARTESIAN or QSL_GEOM_SPHERICAL)."""
    _check(lib().qsl_set_geometry(field.handle, int(geometry)))
    return field


def qsl_check_fp64_newton(x):
    """Largest differences (ulps) of the library's FP64 Newton-Raphson
    reciprocal square root and reciprocal from CUDA's, over host values x."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros(2)
    _check(lib().qsl_check_fp64_newton(_ptr(x), x.size, _ptr(out)))
    return {"rsqrt_ulp": float(out[0]), "rcp_ulp": float(out[1])}


def qsl_trim_pool():
    """Returns the library pool's cached device memory to the driver."""
    _check(lib().qsl_trim_pool())


def qsl_last_refine_stats():
    """Time accounting of the last qsl_refine on this thread (dict)."""
    s = qsl_refine_stats()
    _check(lib().qsl_last_refine_stats(C.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_}


EXPORTS = ["qsl_opts_default", "qsl_load_field", "qsl_free_field", "qsl_trace_seeds", "qsl_q_map_2d",
           "qsl_q_volume_3d", "qsl_fledge", "qsl_refine", "qsl_hilbert_encode", "qsl_hilbert_decode", "qsl_convert",
           "qsl_last_error", "qsl_last_stats", "qsl_trace_seeds_noalloc", "qsl_kernel_launches", "qsl_q_map_batch",
           "qsl_plan_q_map_batch", "qsl_plan_launch", "qsl_plan_stats", "qsl_plan_free", "qsl_autotune",
           "qsl_cnn_create", "qsl_cnn_params", "qsl_cnn_forward", "qsl_cnn_loss_grad", "qsl_cnn_adam_step",
           "qsl_cnn_free", "qsl_cnn_nparams", "qsl_last_refine_stats", "qsl_trim_pool", "qsl_set_geometry"]
