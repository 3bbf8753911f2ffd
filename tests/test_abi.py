"""CPU checks of the C ABI: the library builds/loads and exports every
function that include/qsl.h declares (no compute calls without a GPU)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "qsl.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qsl_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_function():
    from paper_1609_00724_gb300 import build, qsl
    build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", qsl.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qsl_\w+)", out))
    decl = declared_functions()
    assert decl, "no declarations parsed"
    missing = [f for f in decl if f not in exported]
    assert not missing, missing
    L = qsl.lib()
    for f in decl:
        getattr(L, f)


def test_opts_default_and_struct_sizes():
    import ctypes as C

    from paper_1609_00724_gb300 import qsl
    o = qsl.qsl_opts_default()
    assert o.integrator == qsl.QSL_RKCK54 and o.tol_abs == 1e-2 and o.retrace_q == 1e6
    assert C.sizeof(qsl.qsl_opts) == 176
    assert C.sizeof(qsl.qsl_refine_stats) == 104
    assert C.sizeof(qsl.qsl_samples) == 72
    assert C.sizeof(qsl.qsl_refine_spec) == 200
    assert qsl.QSL_LINE_DTYPE.itemsize == 112
    assert qsl.lib().qsl_last_error() == b""


def test_peak_microbenchmarks_library_exports():
    """The benchmark's peak-rate microbenchmarks build into their own library."""
    from paper_1609_00724_gb300 import build
    path = build.build_peaks()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (qslpk_\w+)", out))
    assert {"qslpk_fp32_fma", "qslpk_l2_read"} <= exported, exported
