"""GPU test of qsl_trace_seeds_noalloc, the tracing entry point for callers
that cannot allocate device memory (it keeps its scratch in one static device
array). Its records must match qsl_trace_seeds on the same inputs, on two
calls in a row (the array keeps the previous call's contents).

This file is collected last, so a run that stops at the first failure has run
every other test before it."""
import numpy as np
import pytest
import torch

from paper_1609_00724_gb300 import inputs
from gpu_helpers import L_RTOL, Q_RTOL

pytestmark = pytest.mark.gpu


def _field(qsl):
    ch = inputs.random_charges(4, 2)
    gf = inputs.charge_field(ch, 48, dtype=torch.float32, device="cuda")
    return qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)


def _close(a, b, rtol):
    both = np.isfinite(a) & np.isfinite(b)
    assert np.array_equal(np.isfinite(a), np.isfinite(b))
    return np.all(np.abs(a[both] - b[both]) <= rtol * np.abs(b[both]))


@pytest.mark.parametrize("integrator", [0, 2])
def test_noalloc_matches_trace_seeds_twice(integrator):
    from paper_1609_00724_gb300 import qsl
    F = _field(qsl)
    o = qsl.qsl_opts_default(tol_abs=1e-7, tol_rel=1e-7, integrator=integrator, retrace_q=0.0)
    for call, (n, seed) in enumerate([(5000, 31), (777, 32)]):
        seeds = inputs.random_seeds(n, seed)
        seeds[: n // 4, 2] = 0.0
        sd = torch.as_tensor(seeds).cuda()
        want = qsl.lines_to_numpy(qsl.qsl_trace_seeds(F, sd, o))
        out = torch.empty(n * qsl.QSL_LINE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        got = qsl.lines_to_numpy(qsl.qsl_trace_seeds_noalloc(F, sd, o, out))
        assert np.array_equal(got["face_f"], want["face_f"]) and np.array_equal(got["face_b"], want["face_b"])
        assert np.array_equal(got["status_f"], want["status_f"]) and np.array_equal(got["status_b"], want["status_b"])
        assert _close(got["length"], want["length"], L_RTOL)
        ok = np.isfinite(want["q_perp"]) & (want["q_perp"] < 1e6)
        assert _close(got["q_perp"][ok], want["q_perp"][ok], Q_RTOL)
        assert _close(got["q_foot"], want["q_foot"], Q_RTOL)


def test_noalloc_leaves_device_memory_unchanged():
    """Free device memory (cudaMemGetInfo) is the same before and after two
    calls, once the first call has looked up the array's address and loaded
    the kernels; the same check catches qsl_trace_seeds, whose scratch comes
    from the library's stream-ordered pool (kept cached after the call), on a
    launch whose scratch (112 MB) is larger than any free space the pool's
    blocks can hold after a trim."""
    from paper_1609_00724_gb300 import qsl
    F = _field(qsl)
    o = qsl.qsl_opts_default(tol_abs=1e-7, tol_rel=1e-7, integrator=2, retrace_q=0.0)
    n = 5000
    sd = torch.as_tensor(inputs.random_seeds(n, 33)).cuda()
    out = torch.empty(n * qsl.QSL_LINE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n2 = 1 << 20
    sd2 = torch.as_tensor(inputs.random_seeds(n2, 34)).cuda()
    out2 = torch.empty(n2 * qsl.QSL_LINE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    qsl.qsl_trace_seeds_noalloc(F, sd, o, out)  # first call on this device
    torch.cuda.synchronize()
    qsl.qsl_trim_pool()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        qsl.qsl_trace_seeds_noalloc(F, sd, o, out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)
    qsl.qsl_trace_seeds(F, sd2, o, out=out2)
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 < free1
    qsl.qsl_trim_pool()


def test_noalloc_rejects_oversize_and_host_memory():
    from paper_1609_00724_gb300 import qsl
    F = _field(qsl)
    o = qsl.qsl_opts_default()
    n = qsl.QSL_NOALLOC_MAX_SEEDS + 1
    sd = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    out = torch.empty(n * qsl.QSL_LINE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_trace_seeds_noalloc(F, sd, o, out)
    assert e.value.code == qsl.QSL_EINVAL and "limit" in str(e.value)
    with pytest.raises(qsl.QslError) as e:
        qsl.qsl_trace_seeds_noalloc(F, np.zeros((4, 3)), o, np.zeros(4 * 112, dtype=np.uint8))
    assert e.value.code == qsl.QSL_EINVAL
    with pytest.raises(qsl.QslError):
        qsl.qsl_trace_seeds_noalloc(F, sd[:4], qsl.qsl_opts_default(precision=qsl.QSL_FP64), out[: 4 * 112])
