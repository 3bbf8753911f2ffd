"""GPU tests of the batch path: many fields of different sizes and cuts in one
persistent launch (qsl_q_map_batch) and its captured CUDA-graph plan."""
import numpy as np
import pytest
import torch

from paper_1609_00724_gb300 import inputs
from gpu_helpers import GPU_TOL, compare_lines

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qsl():
    from paper_1609_00724_gb300 import qsl as q
    q.lib()
    return q


def _items(qsl):
    specs = [(33, 2, 40, 37), (56, 3, 64, 64), (40, 4, 23, 71), (64, 5, 96, 50), (48, 6, 1, 9)]
    fields, items, gfs = [], [], []
    for n, seed, nu, nv in specs:
        ch = inputs.random_charges(4, seed)
        gf = inputs.charge_field(ch, n, dtype=torch.float32, device="cuda")
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
        fields.append(F)
        gfs.append(gf)
        items.append((F, (0.1, -0.05, 0.0), (1.8, 0.2, 0.0), (-0.1, 1.7, 0.0), nu, nv))
    return fields, items, gfs


@pytest.mark.parametrize("integ", [2, 0])
def test_batch_equals_per_item_maps_and_plan_replays(qsl, integ):
    fields, items, _ = _items(qsl)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, integrator=integ, retrace_q=1e3)
    N = sum(it[4] * it[5] for it in items)
    q, L = torch.empty(N, device="cuda"), torch.empty(N, device="cuda")
    fc = torch.empty(2 * N, dtype=torch.uint8, device="cuda")
    st = torch.empty(N, dtype=torch.uint8, device="cuda")
    qsl.qsl_q_map_batch(items, o, q, L, fc, st)
    torch.cuda.synchronize()
    off = 0
    for F, c, u, v, nu, nv in items:
        n = nu * nv
        q1, L1 = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
        f1 = torch.empty(2 * n, dtype=torch.uint8, device="cuda")
        s1 = torch.empty(n, dtype=torch.uint8, device="cuda")
        qsl.qsl_q_map_2d(F, c, u, v, nu, nv, o, q1, L1, f1, s1)
        torch.cuda.synchronize()
        # identical algorithm per line: identical results
        assert torch.equal(f1, fc[2 * off:2 * (off + n)]) and torch.equal(s1, st[off:off + n])
        assert torch.allclose(L1, L[off:off + n], rtol=1e-6, atol=0, equal_nan=True)
        assert torch.allclose(q1, q[off:off + n], rtol=1e-5, atol=0, equal_nan=True)
        off += n
    # captured plan: two replays give the batch's results
    q2, L2 = torch.full((N,), -1.0, device="cuda"), torch.full((N,), -1.0, device="cuda")
    plan = qsl.Plan(items, o, q=q2, length=L2)
    for _ in range(2):
        q2.fill_(-1.0)
        plan.launch()
        torch.cuda.synchronize()
        assert torch.allclose(q2, q, rtol=1e-6, equal_nan=True) and torch.allclose(L2, L, rtol=1e-6, equal_nan=True)
    s = plan.stats()
    assert s["lines"] == N and s["stage_evals"] > 0
    del plan


def test_batch_matches_oracle_sampled(qsl, oracle_mod):
    fields, items, gfs = _items(qsl)
    o = qsl.qsl_opts_default(tol_abs=GPU_TOL, tol_rel=GPU_TOL, integrator=qsl.QSL_DOPRI5_CELL)
    N = sum(it[4] * it[5] for it in items)
    q, L = torch.empty(N, device="cuda"), torch.empty(N, device="cuda")
    fc = torch.empty(2 * N, dtype=torch.uint8, device="cuda")
    qsl.qsl_q_map_batch(items, o, q, L, fc)
    torch.cuda.synchronize()
    q, L, fc = q.cpu().numpy(), L.cpu().numpy(), fc.cpu().numpy().reshape(-1, 2)
    off = 0
    for (F, c, u, v, nu, nv), gf in zip(items, gfs):
        n = nu * nv
        g = inputs.to_numpy64(gf)
        Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
        idx = inputs.subsample(n, 60, off + 1)
        seeds = oracle_mod.plane_seeds(c, u, v, nu, nv)[idx]
        ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
        gd = {"q_perp": q[off + idx], "L": L[off + idx], "face_f": fc[off + idx, 0], "face_b": fc[off + idx, 1]}
        compare_lines(gd, ref, 1.0 / (len(g.xc) - 1), (-1, -1, 0), (1, 1, 1))
        off += n


def test_autotune_picks_valid_shape_and_tolerance(qsl):
    fields, items, _ = _items(qsl)
    seeds = torch.as_tensor(inputs.random_seeds(2000, 5)).cuda()
    o = qsl.qsl_opts_default(integrator=qsl.QSL_DOPRI5_CELL)
    rep = qsl.qsl_autotune(items[1][0], seeds, o)
    assert rep["tol"] in (1e-5, 1e-6, 1e-7)
    assert rep["passed"] == 1
    assert rep["q_err"] <= 2e-4 and rep["l_err"] <= 2e-6 and rep["l_err_subcell"] <= 1e-5 and rep["cached"] == 0
    assert o.tol_rel == rep["tol"] and o.warps_per_block == rep["warps_per_block"]
    assert rep["h_max"] in (2.0, 4.0) and o.h_max == rep["h_max"]
    # shapes are timed on the sample repeated to at least 16 x 384 line
    # directions per SM (throughput, not the latency of the longest line)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert rep["shape_reps"] >= 1 and 2 * 2000 * rep["shape_reps"] >= 16 * 384 * sms
    o2 = qsl.qsl_opts_default(integrator=qsl.QSL_DOPRI5_CELL)
    rep2 = qsl.qsl_autotune(items[1][0], seeds, o2)
    assert rep2["cached"] == 1 and o2.refill_min == rep["refill_min"] and o2.h_max == rep["h_max"]


def test_config4_batch64_full_size_sampled(qsl, oracle_mod):
    """The 64-field batch at full size, as the bench runs it: 64 independently
    seeded 4-charge fields with grid edges n ~ U{64..256} and z = 0 cuts of
    m x m seeds, m ~ U{256..1024} (about 34 M seeds), autotuned on a sample of
    the first cut, in one persistent launch recorded into a CUDA graph and
    replayed twice; ten seeded pixels of every field against the FP64 oracle."""
    specs = inputs.batch64_specs()
    items, gfs = [], []
    for n, m, fseed in specs:
        gf = inputs.charge_field(inputs.random_charges(4, fseed), n, dtype=torch.float32, device="cuda", slab=64)
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
        items.append((F, (0, 0, 0), (2, 0, 0), (0, 2, 0), m, m))
        gfs.append(gf)
    N = sum(m * m for _, m, _ in specs)
    assert N > 30_000_000
    o = qsl.qsl_opts_default(integrator=qsl.QSL_DOPRI5_CELL, tol_abs=1e-7, tol_rel=1e-7)
    m0 = specs[0][1]
    pick = inputs.subsample(m0 * m0, 131072, 17)
    ii, jj = pick % m0, pick // m0
    sd = np.column_stack([-1 + (ii + 0.5) * 2 / m0, -1 + (jj + 0.5) * 2 / m0, np.zeros(len(pick))])
    rep = qsl.qsl_autotune(items[0][0], torch.as_tensor(sd).cuda(), o)
    print("autotune on the first cut (n = %d, m = %d):" % specs[0][:2], rep)
    assert rep["tol"] in (1e-5, 1e-6, 1e-7)
    q, L = torch.empty(N, device="cuda"), torch.empty(N, device="cuda")
    fc = torch.empty(2 * N, dtype=torch.uint8, device="cuda")
    plan = qsl.Plan(items, o, q=q, length=L, faces=fc)
    for _ in range(2):
        q.fill_(-1.0)
        plan.launch()
    torch.cuda.synchronize()
    assert plan.stats()["lines"] == N
    off = 0
    checked = 0
    for k, ((n, m, fseed), gf) in enumerate(zip(specs, gfs)):
        idx = inputs.subsample(m * m, 10, 500 + k)
        g = inputs.to_numpy64(gf)
        Fo = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
        seeds = oracle_mod.plane_seeds((0, 0, 0), (2, 0, 0), (0, 2, 0), m, m)[idx]
        ref = oracle_mod.trace_seeds(Fo, seeds, oracle_mod.default_opts(tol_abs=1e-11, tol_rel=1e-11))
        del Fo, g
        gd = {"q_perp": q[off + idx].cpu().numpy(), "L": L[off + idx].cpu().numpy(),
              "face_f": fc.view(-1, 2)[off + idx, 0].cpu().numpy(), "face_b": fc.view(-1, 2)[off + idx, 1].cpu().numpy()}
        rep_k = compare_lines(gd, ref, 1.0 / (n - 1), (-1, -1, 0), (1, 1, 1))
        checked += rep_k["q_checked"]
        off += m * m
    assert checked > 500
    del plan
