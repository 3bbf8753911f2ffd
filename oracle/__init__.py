"""ctypes wrapper of the FP64 QSL oracle (oracle/qslref.cpp).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's CPU
baseline leg import this package. It does not import the CUDA library and the
CUDA library does not import it.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

NO_FACE = 255
ST_OK, ST_MAXLEN, ST_MAXSTEPS, ST_STALL, ST_OUTSIDE, ST_NONFINITE, ST_NULL = range(7)


class Opts(C.Structure):
    _fields_ = [("integrator", C.c_int), ("length_only", C.c_int), ("skip_open", C.c_int), ("pad0", C.c_int),
                ("tol_abs", C.c_double), ("tol_rel", C.c_double), ("h_init", C.c_double), ("h_max", C.c_double),
                ("h_min", C.c_double), ("max_length", C.c_double), ("max_steps", C.c_double),
                ("euler_h", C.c_double), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("land_tol", C.c_double), ("nthreads", C.c_int), ("pad1", C.c_int)]


class RefineSpec(C.Structure):
    _fields_ = [("ndim", C.c_int), ("coarse_order", C.c_int), ("max_order", C.c_int), ("max_iters", C.c_int),
                ("extent", C.c_int * 3), ("shift", C.c_int), ("q_form", C.c_int), ("out_order", C.c_int),
                ("pad", C.c_int), ("center", C.c_double * 3), ("u", C.c_double * 3), ("v", C.c_double * 3),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("tau", C.c_double), ("criterion", C.c_int),
                ("pad2", C.c_int), ("q_threshold", C.c_double), ("pass_stepper", C.c_int), ("pad3", C.c_int),
                ("pass_h_max", C.c_double)]


class Lines(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("q_perp", "q_foot", "q_det", "b0", "bf", "bb", "flux", "flux_b", "L", "lam_f",
                                          "lam_b", "xf", "xb", "face_f", "face_b", "st_f", "st_b", "steps")]


class Stats(C.Structure):
    _fields_ = [("stage_evals", C.c_double), ("accepted", C.c_double), ("rejected", C.c_double),
                ("landing", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, dp, i32, i64, u64 = C.c_void_p, C.POINTER(C.c_double), C.c_int, C.c_int64, C.c_uint64
        L.qslref_load_field.restype = vp
        L.qslref_load_field.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp, i32]
        L.qslref_free_field.argtypes = [vp]
        L.qslref_interp.argtypes = [vp, vp, vp, vp, vp]
        L.qslref_trace_seeds.argtypes = [vp, vp, i64, C.POINTER(Opts), C.POINTER(Lines), C.POINTER(Stats)]
        L.qslref_trace_dir.argtypes = [vp, vp, i32, i32, C.POINTER(Opts), vp, vp, vp, vp]
        L.qslref_ck_linear_step.argtypes = [vp, i32, vp, C.c_double, vp, vp]
        L.qslref_plane_seeds.argtypes = [vp, vp, vp, i32, i32, vp]
        L.qslref_volume_seeds.argtypes = [vp, vp, i32, i32, i32, vp]
        L.qslref_sobel.argtypes = [vp, i32, vp, vp]
        L.qslref_hilbert_key.restype = u64
        L.qslref_hilbert_key.argtypes = [vp, i32, i32]
        L.qslref_hilbert_coords.argtypes = [u64, i32, i32, vp]
        L.qslref_refine.restype = i64
        L.qslref_refine.argtypes = [vp, C.POINTER(Opts), C.POINTER(RefineSpec), i64] + [vp] * 10
        L.qslref_refine_fn.restype = i64
        L.qslref_refine_fn.argtypes = [vp, C.POINTER(RefineSpec), i64, vp, vp, vp, vp, vp]
        L.qslref_refine_replay.restype = i64
        L.qslref_refine_replay.argtypes = [vp, C.POINTER(RefineSpec), C.c_double, C.c_double, vp, vp, i64, i64, vp,
                                           vp, vp, vp, vp, vp]
        L.qslref_convert.argtypes = [vp, vp, i64, i32, i32, vp, i32, i32, vp]
        assert L.qslref_sizeof_opts() == C.sizeof(Opts)
        assert L.qslref_sizeof_refine_spec() == C.sizeof(RefineSpec)
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def default_opts(**kw):
    o = Opts()
    lib().qslref_opts_default(C.byref(o))
    for k, v in kw.items():
        if k in ("lo", "hi"):
            getattr(o, k)[:] = list(v)
        else:
            setattr(o, k, v)
    return o


class Field:
    """Packed FP64 field on a rectilinear grid; b arrays are [nz, ny, nx] (x fastest)."""

    def __init__(self, bx, by, bz, xc, yc, zc, mode=0, order=1, geometry=0):
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (bx, by, bz, xc, yc, zc)]
        bx, by, bz, xc, yc, zc = self._keep
        nz, ny, nx = bx.shape
        assert (nx, ny, nz) == (len(xc), len(yc), len(zc))
        self.handle = lib().qslref_load_field(_p(bx), _p(by), _p(bz), nx, ny, nz, _p(xc), _p(yc), _p(zc), mode)
        if not self.handle:
            raise ValueError("oracle rejected the field")
        self.shape = (nx, ny, nz)
        self.mode = mode
        self._keep = None
        if order != 1 and lib().qslref_set_interp_order(self.handle, int(order)) != 0:
            raise ValueError("interpolation order %r needs 1..3 and, above 1, a uniform grid" % (order,))
        self.order = order
        if geometry != 0 and lib().qslref_set_geometry(self.handle, int(geometry)) != 0:
            raise ValueError("spherical geometry needs latitudes inside (-pi/2, pi/2) and radii > 0")
        self.geometry = geometry

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qslref_free_field(self.handle)
            self.handle = None

    def interp(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        b = np.zeros(3)
        g = np.zeros(9)
        m = np.zeros(1)
        lib().qslref_interp(self.handle, _p(x), _p(b), _p(g), _p(m))
        return b, g.reshape(3, 3), float(m[0])


def trace_seeds(field, seeds, opts=None, with_stats=False):
    """Traces each seed (S x 3) in both directions; returns a dict of arrays."""
    if opts is None:
        opts = default_opts()
    seeds = np.ascontiguousarray(seeds, dtype=np.float64).reshape(-1, 3)
    S = seeds.shape[0]
    out = {}
    lines = Lines()
    for name in ("q_perp", "q_foot", "q_det", "b0", "bf", "bb", "flux", "flux_b", "L", "lam_f", "lam_b", "steps"):
        out[name] = np.full(S, np.nan)
        setattr(lines, name, out[name].ctypes.data)
    for name in ("xf", "xb"):
        out[name] = np.full((S, 3), np.nan)
        setattr(lines, name, out[name].ctypes.data)
    for name in ("face_f", "face_b", "st_f", "st_b"):
        out[name] = np.zeros(S, dtype=np.int32)
        setattr(lines, name, out[name].ctypes.data)
    st = Stats()
    lib().qslref_trace_seeds(field.handle, _p(seeds), S, C.byref(opts), C.byref(lines), C.byref(st))
    if with_stats:
        return out, {"stage_evals": st.stage_evals, "accepted": st.accepted, "rejected": st.rejected,
                     "landing": st.landing}
    return out


def trace_dir(field, y0, s, opts=None):
    if opts is None:
        opts = default_opts()
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    n = y0.size
    y = np.zeros(n)
    mu = np.zeros(1)
    face = np.zeros(1, dtype=np.int32)
    status = np.zeros(1, dtype=np.int32)
    lib().qslref_trace_dir(field.handle, _p(y0), s, n, C.byref(opts), _p(y), _p(mu), _p(face), _p(status))
    return y, float(mu[0]), int(face[0]), int(status[0])


def ck_linear_step(M, y, h):
    M = np.ascontiguousarray(M, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    yn = np.zeros_like(y)
    ye = np.zeros_like(y)
    lib().qslref_ck_linear_step(_p(M), y.size, _p(y), C.c_double(h), _p(yn), _p(ye))
    return yn, ye


def plane_seeds(center, u, v, nu, nv):
    out = np.zeros((nv * nu, 3))
    c, uu, vv = (np.ascontiguousarray(a, dtype=np.float64) for a in (center, u, v))
    lib().qslref_plane_seeds(_p(c), _p(uu), _p(vv), nu, nv, _p(out))
    return out


def volume_seeds(lo, hi, nx, ny, nz):
    out = np.zeros((nx * ny * nz, 3))
    lo, hi = (np.ascontiguousarray(a, dtype=np.float64) for a in (lo, hi))
    lib().qslref_volume_seeds(_p(lo), _p(hi), nx, ny, nz, _p(out))
    return out


def q_map_2d(field, center, u, v, nu, nv, opts=None):
    r = trace_seeds(field, plane_seeds(center, u, v, nu, nv), opts)
    return {k: (a.reshape(nv, nu, *a.shape[1:])) for k, a in r.items()}


def q_volume_3d(field, lo, hi, nx, ny, nz, opts=None):
    r = trace_seeds(field, volume_seeds(lo, hi, nx, ny, nz), opts)
    return {k: (a.reshape(nz, ny, nx, *a.shape[1:])) for k, a in r.items()}


def fledge(L):
    """Sobel gradient magnitude of a 2D/3D length map (axis 0 slowest)."""
    L = np.ascontiguousarray(L, dtype=np.float32)
    shape = np.array(L.shape, dtype=np.int64)
    out = np.zeros(L.shape, dtype=np.float64)
    lib().qslref_sobel(_p(L), L.ndim, _p(shape), _p(out))
    return out


def hilbert_key(coords, ndim, bits):
    c = np.zeros(3, dtype=np.uint32)
    c[:ndim] = coords
    return int(lib().qslref_hilbert_key(_p(c), ndim, bits))


def hilbert_coords(key, ndim, bits):
    c = np.zeros(3, dtype=np.uint32)
    lib().qslref_hilbert_coords(C.c_uint64(int(key)), ndim, bits, _p(c))
    return tuple(int(x) for x in c[:ndim])


def refine_spec(**kw):
    s = RefineSpec()
    s.max_iters = 64
    s.shift = 1
    for k, v in kw.items():
        if k in ("extent", "center", "u", "v", "lo", "hi"):
            arr = getattr(s, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(s, k, v)
    if s.out_order == 0:
        s.out_order = s.max_order
    for a in range(s.ndim):
        if s.extent[a] == 0:
            s.extent[a] = 1 << s.max_order
    return s


def refine(field, spec, opts=None, capacity=None):
    if opts is None:
        opts = default_opts()
    if capacity is None:
        capacity = 1
        for a in range(spec.ndim):
            capacity *= spec.extent[a]
    arrs = {"key": np.zeros(capacity, dtype=np.uint64), "q": np.zeros(capacity), "L": np.zeros(capacity)}
    for n in ("face_f", "face_b", "st_f", "st_b", "origin"):
        arrs[n] = np.zeros(capacity, dtype=np.int32)
    iters = np.zeros(1, dtype=np.int32)
    per = np.zeros(spec.max_iters + 1, dtype=np.int64)
    n = lib().qslref_refine(field.handle, C.byref(opts), C.byref(spec), capacity, *(_p(arrs[k]) for k in (
        "key", "q", "L", "face_f", "face_b", "st_f", "st_b")), _p(iters), _p(per), _p(arrs["origin"]))
    if n < 0:
        raise RuntimeError("capacity too small: need %d" % -n)
    out = {k: a[:n].copy() for k, a in arrs.items()}
    out["iters"] = int(iters[0])
    out["traced_per_iter"] = per[:int(iters[0]) + 2].copy()
    return out


_EVAL_FN = C.CFUNCTYPE(None, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double))


def refine_fn(fn, spec, capacity=None):
    """Refinement driver with an analytic evaluator fn(xyz[n,3]) -> (q[n], L[n])."""
    if capacity is None:
        capacity = 1
        for a in range(spec.ndim):
            capacity *= spec.extent[a]

    def cb(n, xyz, q, L):
        x = np.ctypeslib.as_array(xyz, shape=(n, 3)).copy()
        qq, ll = fn(x)
        np.ctypeslib.as_array(q, shape=(n,))[:] = qq
        np.ctypeslib.as_array(L, shape=(n,))[:] = ll

    cfn = _EVAL_FN(cb)
    key = np.zeros(capacity, dtype=np.uint64)
    q = np.zeros(capacity)
    L = np.zeros(capacity)
    iters = np.zeros(1, dtype=np.int32)
    per = np.zeros(spec.max_iters + 1, dtype=np.int64)
    n = lib().qslref_refine_fn(C.cast(cfn, C.c_void_p), C.byref(spec), capacity, _p(key), _p(q), _p(L),
                               _p(iters), _p(per))
    if n < 0:
        raise RuntimeError("capacity too small: need %d" % -n)
    return {"key": key[:n].copy(), "q": q[:n].copy(), "L": L[:n].copy(), "iters": int(iters[0]),
            "traced_per_iter": per[:int(iters[0]) + 2].copy()}


_EVAL_KFN = C.CFUNCTYPE(None, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.POINTER(C.c_double),
                        C.POINTER(C.c_double), C.POINTER(C.c_int32))


def refine_replay(fn, spec, tie_keys=(), tie_origin=(), band_abs=0.0, band_rel=0.0, capacity=None):
    """Refinement driver (test hook) with values from fn(xyz[n,3], keys[n]) ->
    (q[n], L[n]) or (q[n], L[n], unsure[n]); a pair with an unsure sample, or
    whose criterion value lies within the band of the
    threshold (| |dL| - tau | <= band_abs + band_rel max(|L|), or Q within
    band_rel of q_threshold) is refined exactly when another run added its new
    cell in the same pass (tie_keys sorted, tie_origin the pass that added each:
    0 coarse pass, 2i+1 / 2i+2 pass A / B of iteration i). With values that
    carry no error, the band set to the error bound of the other run's values
    and that run's samples as the ties, the replay reproduces the other run's
    set when all their disagreements lie within the bound. Returns key, q, L,
    origin, iters."""
    if capacity is None:
        capacity = 1
        for a in range(spec.ndim):
            capacity *= spec.extent[a]
    tk = np.asarray(tie_keys, dtype=np.uint64)
    to = np.asarray(tie_origin, dtype=np.int32)
    assert tk.shape == to.shape
    order = np.argsort(tk, kind="stable")
    tk, to = np.ascontiguousarray(tk[order]), np.ascontiguousarray(to[order])

    def cb(n, xyz, keys, q, L, unsure):
        x = np.ctypeslib.as_array(xyz, shape=(n, 3)).copy()
        k = np.ctypeslib.as_array(keys, shape=(n,)).copy()
        r = fn(x, k)
        np.ctypeslib.as_array(q, shape=(n,))[:] = r[0]
        np.ctypeslib.as_array(L, shape=(n,))[:] = r[1]
        if len(r) > 2:
            np.ctypeslib.as_array(unsure, shape=(n,))[:] = np.asarray(r[2], dtype=np.int32)

    cfn = _EVAL_KFN(cb)
    key = np.zeros(capacity, dtype=np.uint64)
    q = np.zeros(capacity)
    L = np.zeros(capacity)
    origin = np.zeros(capacity, dtype=np.int32)
    iters = np.zeros(1, dtype=np.int32)
    per = np.zeros(spec.max_iters + 1, dtype=np.int64)
    n = lib().qslref_refine_replay(C.cast(cfn, C.c_void_p), C.byref(spec), float(band_abs), float(band_rel),
                                   _p(tk), _p(to), tk.size, capacity, _p(key), _p(q), _p(L), _p(origin), _p(iters),
                                   _p(per))
    if n < 0:
        raise RuntimeError("capacity too small: need %d" % -n)
    return {"key": key[:n].copy(), "q": q[:n].copy(), "L": L[:n].copy(), "origin": origin[:n].copy(),
            "iters": int(iters[0]), "traced_per_iter": per[:int(iters[0]) + 2].copy()}


def convert(keys, vals, ndim, max_order, extent, out_order, log_interp):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    ext = np.zeros(3, dtype=np.int32)
    ext[:ndim] = extent[:ndim]
    d = max_order - out_order
    shape = [int(ext[a]) >> d for a in range(ndim)][::-1]
    out = np.zeros(int(np.prod(shape)))
    lib().qslref_convert(_p(keys), _p(vals), keys.size, ndim, max_order, _p(ext), out_order, int(log_interp),
                         _p(out))
    return out.reshape(shape)
