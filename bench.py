"""Benchmark: Q-points/s of a complete refined Q map (the QSL Squasher hot path).

Workload (one step): the potential field of 4 sub-photospheric point charges
(|q| ~ U(0.5, 1.5), alternating signs, depths ~ U(0.05, 0.2), (x, y) ~
U[-0.5, 0.5]^2, seed 2) sampled in FP32 on a 256^3 grid over [-1,1]^2 x [0,1];
field packing, the 1024 x 1024 photospheric (z = 0) coarse Q/FLL map, the
FLEDGE map of its lengths, FLL-jump refinement along the Hilbert curve (with
the shifted-curve pass) to 4096 x 4096 effective resolution, FP64 retrace of
lines with Q > 1e6, and the Hilbert -> rectilinear conversion of Q and FLL to
4096 x 4096. value = Q-points traced per step (coarse + refined) / step time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs an independent replica (its own field
seed); value sums all ranks' Q-points over the slowest rank's time.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Q-points/s (refined 4096^2-effective Q map, Q rel.err <= 1e-3 vs FP64 oracle)"
UNIT = "Q-points/s"
GRID_N = 256
COARSE = 1024
P0, P = 10, 12
TAU = 0.05
TOL = 1e-7
FIELD_SEED = 2

# Algorithmic FP32 work of one RK stage evaluation in the tangent tracer
# (paper mode, an FMA counts as 2 FLOP). Cash-Karp kernel: trilinear value +
# gradient of 3 components (99), cell location (9), gradient scaling (9),
# deviation right-hand sides (30), the stage's share of the combinations,
# error norm and controller (99). Cell-wise Dormand-Prince kernel: trilinear
# value + gradient (99), scaling (12), deviation right-hand sides (30), the
# stage's share of the combinations (414 per step) and error norm (144 per
# step) over 6.5 evaluations per step (85).
# DRAM bytes per launch of the two tracer phases of the default workload
# (4-charge field on 256^3, 1024^2 map refined to 4096^2):
# dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture of the
# current kernels (summaries under profiles/); None until captured. Coarse:
# one full-size launch, 435.2 MB read + 105.9 MB written. Passes: the average
# over one refined map's 27 launches, 28.4 MB read + 0.16 MB written.
TRAFFIC_COARSE_BYTES = 541.0e6
TRAFFIC_PASS_BYTES = 28.5e6
FLOP_PER_STAGE = {"ck": 246.0, "cell": 227.0}
# length-only stage evaluation: the cell-wise kernels (trilinear values of 3
# components 63, position scaling 3, the 3-component share of the stage
# combinations and error norm 29) and the Cash-Karp kernel of the refinement
# passes' decision traces (trilinear values 63, cell location 9, the
# 3-component share of the stage combinations, error norm and controller 32)
FLOP_PER_STAGE_LEN = {"cell": 95.0, "ck": 104.0}
# decision tracer of the refinement passes (qsl_refine_spec.pass_stepper) and
# its step cap in smallest grid spacings
PASS_STEPPER = 0
PASS_H_MAX = 4.0
# FP32 FMA pipe from unit counts (152 SMs x 128 lanes x 2 FLOP x 2.07 GHz):
# context only; the roofline divides by the rate measured in the same run
# (measure_peaks).
FP32_NOMINAL_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# the tolerance the autotuner picks on this workload (used where no GPU runs
# the tuner: the reference arm)
TUNED_TOL = 1e-5
# algorithmic gather of the cell-wise tracers: the 8 corner vertices of a cell
# (8 x 16 B) once per cell entered
GATHER_BYTES_PER_ENTRY = 128.0


def measure_peaks(local):
    """FP32 FMA and L2 read rates of this GPU from the package's own
    microbenchmarks (CUDA events, fastest of several launches), with the SM
    clock sampled meanwhile; no clock or power setting is read or changed."""
    import ctypes as C

    from paper_1609_00724_gb300 import build as _b
    lib = C.CDLL(_b.PEAKS_LIB)
    tf, ms_f, gb, ms_l = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    with ClockSampler(local) as clk:
        rc1 = lib.qslpk_fp32_fma(C.c_int(2048), C.c_int(5), None, C.byref(tf), C.byref(ms_f))
        rc2 = lib.qslpk_l2_read(C.c_int64(48 << 20), C.c_int(40), C.c_int(5), None, C.byref(gb), C.byref(ms_l))
        time.sleep(0.3)
    if rc1 or rc2:
        raise RuntimeError("peak microbenchmarks failed")
    c = clk.summary()
    out = {"fp32_tflops": tf.value, "fp32_ms": ms_f.value, "l2_read_gbs": gb.value, "l2_ms": ms_l.value,
           "l2_buffer_mb": 48, "clocks": c,
           "how": "libqslpeaks.so: 8 independent FMA chains per thread, 152x8 blocks of 256; float4 __ldcg sweeps "
                  "of a 48 MB buffer resident in L2, 152x4 blocks of 512; fastest of 5 launches (CUDA events)"}
    if c.get("sm_mhz"):
        out["fp32_flop_per_sm_cycle"] = tf.value * 1e12 / (c["sm_mhz"] * 1e6) / 152
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=GRID_N)
    ap.add_argument("--coarse", type=int, default=COARSE)
    ap.add_argument("--integrator", default="cell", choices=["cell", "ck"],
                    help="cell: cell-wise Dormand-Prince (default); ck: the paper's plain Cash-Karp")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (fixed tolerance and shape)")
    ap.add_argument("--config", default="refine2d",
                    choices=["refine2d", "hyperbolic", "volume", "batch64", "learned", "qcrit", "euler", "spherical",
                             "interp"],
                    help="refine2d: 1024^2 map refined to 4096^2 (default); volume: 512x512x256 Q/FLL/FLEDGE volume "
                         "of an 8-charge field on 384^3")
    ap.add_argument("--shape", default=None,
                    help="fixed launch shape 'warps_per_block,blocks_per_sm,refill_min' (skips the autotuner)")
    ap.add_argument("--hmax", type=float, default=None, help="fixed step cap in smallest spacings")
    ap.add_argument("--profile-refine", action="store_true",
                    help="one qsl_refine of the bench workload and its time accounting (for ncu captures)")
    ap.add_argument("--profile-map", action="store_true",
                    help="only run the coarse Q map (the tracer kernel) --steps times, for ncu captures")
    ap.add_argument("--profile-pass", type=int, default=0,
                    help="one refinement of the bench workload, then the samples that pass N added traced again "
                         "in lengths-only mode as one launch --steps times (the refinement-pass kernel), for ncu "
                         "captures")
    ap.add_argument("--pass-seeds", default=None,
                    help="with --profile-pass: file of that pass's seed positions; written by a run that finds it "
                         "missing, read (no refinement in the process) by one that finds it")
    return ap.parse_args()


def replica_seed(base, rank):
    """Seed of replica `rank`: each rank traces its own field (weak scaling)."""
    return base + 1000 * rank


def reduce_timing(torch, ms, units, world, device):
    """Whole-job figures over the replicas: the slowest rank's time and the sum
    of all ranks' units (all_reduce MAX / SUM; no-op for one rank)."""
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    n = torch.tensor([float(units)], device=device, dtype=torch.float64)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_field(seed, device, n):
    import torch

    from paper_1609_00724_gb300 import inputs
    ch = inputs.random_charges(4, seed)
    return inputs.charge_field(ch, n, dtype=torch.float32, device=device, slab=64)


INTEGRATOR = {"cell": 2, "ck": 0}
PEAK = {"fp32": FP32_NOMINAL_TFLOPS, "l2": None, "note": "nominal (not measured)"}
PEAKS_RUN = None
RUN = {"integrator": "cell", "tol": TOL}


def opts(qsl):
    o = qsl.qsl_opts_default(tol_abs=RUN["tol"], tol_rel=RUN["tol"], q_form=qsl.QSL_Q_PERP,
                             integrator=INTEGRATOR[RUN["integrator"]])
    if "shape" in RUN:
        o.warps_per_block, o.blocks_per_sm, o.refill_min = RUN["shape"]
    if "h_max" in RUN:
        o.h_max = RUN["h_max"]
    return o


def spec(qsl, coarse):
    p0 = int(np.log2(coarse))
    return qsl.refine_spec(ndim=2, coarse_order=p0, max_order=p0 + (P - P0), center=(0, 0, 0), u=(2, 0, 0),
                           v=(0, 2, 0), tau=TAU, shift=1, max_iters=64, pass_stepper=PASS_STEPPER,
                           pass_h_max=PASS_H_MAX)


def gpu_step(qsl, gf, bufs, coarse, stream_sync=True):
    """One full step on device-resident inputs. Returns (q_points, stats dict)."""
    import torch
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    o = opts(qsl)
    sp = spec(qsl, coarse)
    n, iters, traced, rc = qsl.qsl_refine(F, sp, o, bufs["key"], bufs["q"], bufs["L"], bufs["faces"], bufs["st"],
                                          0, bufs["qg"], bufs["lg"])
    # FLEDGE of the converted length map
    qsl.qsl_fledge(bufs["lg"].view(bufs["eff"], bufs["eff"]), bufs["sg"])
    if stream_sync:
        torch.cuda.synchronize()
    return traced, {"samples": n, "iters": iters, "rc": rc}


def alloc(torch, coarse, device):
    eff = coarse << (P - P0)
    cap = eff * eff
    return {"key": torch.empty(cap, dtype=torch.int64, device=device),
            "q": torch.empty(cap, dtype=torch.float32, device=device),
            "L": torch.empty(cap, dtype=torch.float32, device=device),
            "faces": torch.empty(2 * cap, dtype=torch.uint8, device=device),
            "st": torch.empty(cap, dtype=torch.uint8, device=device),
            "qg": torch.empty(cap, dtype=torch.float32, device=device),
            "lg": torch.empty(cap, dtype=torch.float32, device=device),
            "sg": torch.empty((eff, eff), dtype=torch.float32, device=device), "eff": eff}


WINDOW = 32  # coarse cells per side of one refinement window of the oracle baseline


def oracle_window_refine(oracle, Fo, tol, coarse, rng, nthreads):
    """The oracle's whole refinement (coarse pass, FLL-jump passes with their
    decision traces, tangent-space values) on one window of WINDOW x WINDOW
    coarse cells of the z = 0 map, at a seeded position, with the map's cell
    sizes (coarse spacing 2 / coarse, refined 2^(P - P0) times). Returns the
    samples it produced and the seconds it took."""
    nw = coarse // WINDOW
    i0, j0 = (int(v) for v in rng.integers(0, nw, size=2))
    w = 2.0 * WINDOW / coarse
    cx, cy = -1.0 + (i0 + 0.5) * w, -1.0 + (j0 + 0.5) * w
    p0 = int(np.log2(WINDOW))
    sp = oracle.refine_spec(ndim=2, coarse_order=p0, max_order=p0 + (P - P0), center=(cx, cy, 0.0), u=(w, 0, 0),
                            v=(0, w, 0), tau=TAU, shift=1, max_iters=64, pass_h_max=PASS_H_MAX)
    o = oracle.default_opts(tol_abs=tol, tol_rel=tol, nthreads=nthreads)
    t0 = time.perf_counter()
    r = oracle.refine(Fo, sp, o)
    return len(r["key"]), time.perf_counter() - t0


def oracle_refine_rate(gf_cpu, tol, coarse, budget_s=12.0, seed=99):
    """cpu_baseline of the refined map: the oracle's own refinement on seeded
    windows of the map (no input from the GPU run) until about budget_s
    seconds. Returns (samples/s, samples, windows, cores, seconds)."""
    import oracle
    from paper_1609_00724_gb300 import inputs
    g = inputs.to_numpy64(gf_cpu)
    Fo = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    cores = os.cpu_count() or 1
    rng = np.random.Generator(np.random.PCG64(seed))
    n, t, k = 0, 0.0, 0
    while t < budget_s:
        m, dt = oracle_window_refine(oracle, Fo, tol, coarse, rng, cores)
        n, t, k = n + m, t + dt, k + 1
    return n / t, n, k, cores, t


def oracle_rate_on(gf, seeds, tol, mode=0, budget_s=10.0, seed=99, order=1, geometry=0):
    """cpu_baseline of a bench mode: the FP64 oracle on seeded subsamples of
    `seeds` of the field gf (GridField, any device) at tolerance `tol`."""
    from paper_1609_00724_gb300 import inputs
    import oracle
    g = inputs.to_numpy64(gf)
    F = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=mode, order=order, geometry=geometry)
    cores = os.cpu_count() or 1
    o = oracle.default_opts(tol_abs=tol, tol_rel=tol, nthreads=cores)
    done, t_used, m, k = 0, 0.0, 64 * cores, seed
    while t_used < budget_s and done < len(seeds):
        idx = inputs.subsample(len(seeds), min(m, len(seeds)), k)
        t0 = time.perf_counter()
        oracle.trace_seeds(F, seeds[idx], o)
        t_used += time.perf_counter() - t0
        done += len(idx)
        k += 1
        m = min(4 * m, max(64, int(m * budget_s / max(t_used, 1e-3))))
    return {"value": done / t_used, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d seeded seeds of the workload, tol %g, %.1f s" % (done, tol, t_used)}


def sample_positions(qsl, keys, coarse):
    """z = 0 plane positions of refinement sample keys (effective lattice)."""
    eff = coarse << (P - P0)
    p = int(np.log2(eff))
    c = np.zeros((len(keys), 2), dtype=np.uint32)
    qsl.qsl_hilbert_decode(np.ascontiguousarray(keys), 2, p, c)
    return np.column_stack([(c[:, 0] + 0.5) / eff * 2 - 1, (c[:, 1] + 0.5) / eff * 2 - 1, np.zeros(len(keys))])


def parity_sample(qsl, gf, gf_cpu, coarse, n=200):
    """Coarse-map Q/FLL of the GPU path at the bench tolerance against the FP64
    oracle at tol 1e-11 on `n` seeded pixels."""
    import torch

    import oracle
    from paper_1609_00724_gb300 import inputs
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    N = coarse * coarse
    q = torch.empty(N, device="cuda")
    L = torch.empty(N, device="cuda")
    fc = torch.empty(2 * N, dtype=torch.uint8, device="cuda")
    qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), coarse, coarse, opts(qsl), q=q, length=L, faces=fc)
    torch.cuda.synchronize()
    idx = inputs.subsample(N, n, 7)
    g = inputs.to_numpy64(gf_cpu)
    Fo = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    seeds = oracle.plane_seeds([0, 0, 0], [2, 0, 0], [0, 2, 0], coarse, coarse)[idx]
    ref = oracle.trace_seeds(Fo, seeds, oracle.default_opts(tol_abs=1e-11, tol_rel=1e-11, nthreads=os.cpu_count()))
    qg, lg = q.cpu().numpy()[idx], L.cpu().numpy()[idx]
    fg = fc.cpu().numpy().reshape(-1, 2)[idx]
    ok = np.isfinite(ref["q_perp"]) & (ref["q_perp"] < 1e6)
    qe = np.abs(qg[ok] / ref["q_perp"][ok] - 1)
    # length error relative to max(L, one cell): sub-cell loops are held to an
    # absolute bound (their length is set by a cancellation in B_n)
    cell = float(min(np.min(np.diff(a)) for a in (g.xc, g.yc, g.zc)))
    pos = np.isfinite(ref["L"])
    le = np.abs(lg[pos] - ref["L"][pos]) / np.maximum(ref["L"][pos], cell)
    faces_eq = float(np.mean((fg[:, 0] == ref["face_f"]) & (fg[:, 1] == ref["face_b"])))
    return {"n": int(n), "q_max_rel": float(qe.max()), "q_p99_rel": float(np.quantile(qe, 0.99)),
            "l_max_rel": float(le.max()), "faces_equal": faces_eq}


def refined_parity(bufs, n_samples, gf_cpu, coarse, n=200):
    """Refined samples (keys off the coarse lattice, i.e. placed by the FLL-jump
    criterion near QSLs) of the last step against the FP64 oracle at tol 1e-11;
    lattice positions come from the oracle's own Hilbert decode."""
    import oracle
    from paper_1609_00724_gb300 import inputs
    eff = coarse << (P - P0)
    p = int(np.log2(eff))
    R = eff // coarse
    keys = bufs["key"][:n_samples].cpu().numpy()
    q = bufs["q"][:n_samples].cpu().numpy()
    L = bufs["L"][:n_samples].cpu().numpy()
    pick = inputs.subsample(n_samples, min(n_samples, 40 * n), 23)
    seeds, idx = [], []
    for i in pick:
        c = oracle.hilbert_coords(int(keys[i]), 2, p)
        if c[0] % R == R // 2 and c[1] % R == R // 2:
            continue  # coarse-lattice sample
        a, b = (c[0] + 0.5) / eff - 0.5, (c[1] + 0.5) / eff - 0.5
        seeds.append([2 * a, 2 * b, 0.0])
        idx.append(i)
        if len(idx) == n:
            break
    g = inputs.to_numpy64(gf_cpu)
    Fo = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    ref = oracle.trace_seeds(Fo, np.array(seeds), oracle.default_opts(tol_abs=1e-11, tol_rel=1e-11,
                                                                       nthreads=os.cpu_count()))
    idx = np.array(idx)
    ok = np.isfinite(ref["q_perp"]) & (ref["q_perp"] < 1e6)
    qe = np.abs(q[idx][ok] / ref["q_perp"][ok] - 1)
    cell = float(min(np.min(np.diff(a)) for a in (g.xc, g.yc, g.zc)))
    pos = np.isfinite(ref["L"])
    le = np.abs(L[idx][pos] - ref["L"][pos]) / np.maximum(ref["L"][pos], cell)
    return {"n": int(len(idx)), "q_checked": int(ok.sum()), "q_max_rel": float(qe.max()),
            "q_p99_rel": float(np.quantile(qe, 0.99)), "l_max_rel": float(le.max()),
            "q_median": float(np.median(ref["q_perp"][ok]))}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle (as it stands) on host cores, one
    bounded sample of the workload per step."""
    if rank != 0:
        return
    import torch

    import oracle
    from paper_1609_00724_gb300 import inputs
    gf = make_field(FIELD_SEED, "cpu", args.grid)
    g = inputs.to_numpy64(gf)
    F = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    cores = os.cpu_count() or 1
    per_step = 24  # refinement windows per step
    rng = np.random.Generator(np.random.PCG64(1000))
    for _ in range(args.warmup):
        oracle_window_refine(oracle, F, TUNED_TOL, args.coarse, rng, cores)
    rng = np.random.Generator(np.random.PCG64(2000))
    t, n = 0.0, 0
    for _ in range(args.steps):
        for _ in range(per_step):
            m, dt = oracle_window_refine(oracle, F, TUNED_TOL, args.coarse, rng, cores)
            n, t = n + m, t + dt
    value = n / t
    sample = ("the oracle's refinement of %d seeded %dx%d-coarse-cell windows per step of the 1024^2 z=0 map at its "
              "cell sizes (%d samples in all), tol %g (the tolerance the GPU arm's autotuner picks on this workload)"
              % (per_step, WINDOW, WINDOW, n, TUNED_TOL))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "4-charge potential field 256^3 FP32, 1024^2 z=0 map refined to 4096^2",
                       "oracle": "FP64 C++ (oracle/qslref.cpp)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    del torch


def run_hyperbolic(args, qsl, torch, dev, rank, world, local):
    """Config 1: the linear hyperbolic field B = (3x, -3y, 1) sampled in FP64 on
    64^3 over [-1, 1]^2 x [0, 1]; one step = the 256 x 256 z = 0 Q/FLL map
    (raw mode, exact for a linear field); the maps against the closed forms
    of the golden fixture (Q_foot = k^2 + k^-2 for top exits and the side-exit
    form, lengths by quadrature)."""
    from paper_1609_00724_gb300 import inputs
    gf = inputs.hyperbolic_field(64)
    t = [torch.as_tensor(a).to(dev) for a in (gf.bx, gf.by, gf.bz)]
    F = qsl.qsl_load_field(*t, gf.xc, gf.yc, gf.zc, interp_mode=qsl.QSL_RAW_B)
    n = 256
    N = n * n
    q = torch.empty(N, device=dev)
    L = torch.empty(N, device=dev)
    fc = torch.empty(2 * N, dtype=torch.uint8, device=dev)
    o = qsl.qsl_opts_default(tol_abs=RUN["tol"], tol_rel=RUN["tol"], q_form=qsl.QSL_Q_FOOT,
                             integrator=INTEGRATOR[RUN["integrator"]])

    def step():
        qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), n, n, o, q=q, length=L, faces=fc)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = qsl.qsl_kernel_launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 20)
    with ClockSampler(local) as clk:
        start.record()
        for _ in range(reps):
            step()
        end.record()
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    st = qsl.qsl_last_stats()
    ms_max, units = reduce_timing(torch, ms, N * reps, world, dev)
    g = np.loadtxt(os.path.join(ROOT, "tests", "golden", "hyperbolic_closed_forms.txt"))
    idx = g[:, 1].astype(int) * n + g[:, 0].astype(int)
    qh, Lh, fh = q.cpu().numpy()[idx], L.cpu().numpy()[idx], fc.cpu().numpy().reshape(-1, 2)[idx]
    line = {"metric": "Q-points/s (256^2 hyperbolic-field map, Q_foot against its closed form)",
            "value": units / (ms_max / 1000.0), "unit": UNIT, "n_gpus": world, "steps": reps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max / reps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "hyperbolic field (3x, -3y, 1) on 64^3 (FP64 samples), 256^2 z=0 map, raw mode",
                       "tol": RUN["tol"], "integrator": RUN["integrator"]},
            "clocks": clk.summary(), "gpu_launches": qsl.qsl_kernel_launches() - l0, "kernel_ms": st["kernel_ms"],
            "closed_form": {"pixels": int(len(idx)), "faces_equal": float(np.mean(fh[:, 0] == g[:, 7].astype(int))),
                            "q_foot_max_rel": float(np.max(np.abs(qh / g[:, 4] - 1))),
                            "l_max_rel": float(np.max(np.abs(Lh / g[:, 6] - 1)))}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        line["cpu_baseline"] = oracle_rate_on(gf, oracle.plane_seeds((0, 0, 0), (2, 0, 0), (0, 2, 0), n, n), RUN["tol"],
                                              mode=1)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_volume(args, qsl, torch, dev, rank, world, local):
    """Config 3: 8 charges on 384^3 (FP32); one step = Q/FLL at 512x512x256
    cell-centre seeds (FP32 trace, FP64 assembly, FP64 retrace above 1e6) and
    the 3D FLEDGE of the length volume."""
    from paper_1609_00724_gb300 import inputs
    ch = inputs.random_charges(8, replica_seed(3, rank))
    gf = inputs.charge_field(ch, 384, dtype=torch.float32, device=dev, slab=32)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
    nx, ny, nz = 512, 512, 256
    N = nx * ny * nz
    q = torch.empty(N, device=dev)
    L = torch.empty(N, device=dev)
    S = torch.empty((nz, ny, nx), device=dev)
    lo, hi = (-1.0, -1.0, 0.0), (1.0, 1.0, 1.0)

    def step():
        qsl.qsl_q_volume_3d(F, lo, hi, nx, ny, nz, opts(qsl), q=q, length=L)
        qsl.qsl_fledge(L.view(nz, ny, nx), S)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = qsl.qsl_kernel_launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record()
        for _ in range(args.steps):
            step()
        end.record()
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    st = qsl.qsl_last_stats()
    ms_max, units = reduce_timing(torch, ms, N * args.steps, world, dev)
    value = units / (ms_max / 1000.0)
    fps = FLOP_PER_STAGE[RUN["integrator"]]
    ach = st["stage_evals"] * fps / (st["kernel_ms"] / 1000.0) / 1e12
    line = {"metric": "Q-points/s (3D Q/FLL/FLEDGE volume)", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "8-charge potential field 384^3 FP32, 512x512x256 volume Q/FLL + 3D FLEDGE",
                       "tol": RUN["tol"], "integrator": RUN["integrator"], "retraced_last_step": st["retraced"],
                       "l2": "inputs larger than L2 (906 MB packed field)"},
            "clocks": clk.summary(), "gpu_launches": qsl.qsl_kernel_launches() - l0,
            "roofline": {"bound": "alu", "achieved": ach, "peak": PEAK["fp32"], "unit": "TFLOP/s",
                         "frac": ach / PEAK["fp32"], "traffic": None,
                         "kernel": "%s (512x512x256 volume, one launch)" % (
                             "cell_kernel_f32<9>" if RUN["integrator"] == "cell" else "trace_kernel<float,9>"),
                         "kernel_ms": st["kernel_ms"], "stage_evals": st["stage_evals"],
                         "flop_per_stage": fps,
                         "peak_note": "of measured: %s" % PEAK["note"]}}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        sub = inputs.subsample(N, 2_000_000, 5)
        ijk = np.column_stack([sub % nx, (sub // nx) % ny, sub // (nx * ny)]).astype(np.float64)
        sd = np.array(lo)[None] + (ijk + 0.5) / np.array([nx, ny, nz])[None] * (np.array(hi) - np.array(lo))[None]
        line["cpu_baseline"] = oracle_rate_on(gf, sd, RUN["tol"])
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, qsl, torch, dev, rank, world, local):
    """Config 4: 64 independently seeded 4-charge fields, grid edge n ~ U{64..256},
    each with a z=0 cut of m x m seeds, m ~ U{256..1024} (field i: seed
    4000 + i); all cuts in one persistent launch recorded into a CUDA graph
    (plan), with the launch shape and tolerance picked by the autotuner on a
    sample of the first cut."""
    from paper_1609_00724_gb300 import inputs
    items, fields = [], []
    for i, (n, m, fseed) in enumerate(inputs.batch64_specs()):
        if rank:  # replica r: its own draw of sizes and fields
            n, m, _ = inputs.batch64_specs(replica_seed(4, rank))[i]
        gf = inputs.charge_field(inputs.random_charges(4, replica_seed(fseed, rank)), n, dtype=torch.float32,
                                 device=dev, slab=64)
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
        if i == 0:
            gf0 = gf
        del gf
        fields.append(F)
        items.append((F, (0, 0, 0), (2, 0, 0), (0, 2, 0), m, m))
    N = sum(it[4] * it[5] for it in items)
    o = opts(qsl)
    # autotune on 131072 seeds of the first cut (several waves of the GPU)
    m0 = items[0][4]
    pick = inputs.subsample(m0 * m0, 131072, 17)
    ii, jj = pick % m0, pick // m0
    sd = np.column_stack([-1 + (ii + 0.5) * 2 / m0, -1 + (jj + 0.5) * 2 / m0, np.zeros(len(pick))])
    rep = qsl.qsl_autotune(items[0][0], torch.as_tensor(sd).to(dev), o)
    q = torch.empty(N, device=dev)
    L = torch.empty(N, device=dev)
    plan = qsl.Plan(items, o, q=q, length=L)
    for _ in range(max(args.warmup, 3)):
        plan.launch()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    l0 = qsl.qsl_kernel_launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        start.record()
        for _ in range(args.steps):
            plan.launch()
        end.record()
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    st = plan.stats()
    ms_max, units = reduce_timing(torch, ms, N * args.steps, world, dev)
    value = units / (ms_max / 1000.0)
    line = {"metric": "Q-points/s (64-field batch, one captured persistent launch)", "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "64 4-charge fields, n~U{64..256}^3, cuts m~U{256..1024}^2, %d seeds" % N,
                       "integrator": RUN["integrator"], "autotune": rep,
                       "l2": "inputs larger than L2 (%d packed fields)" % len(items)},
            "clocks": clk.summary(), "gpu_launches": qsl.qsl_kernel_launches() - l0,
            "stats_last_replay": st}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        m0 = items[0][4]
        line["cpu_baseline"] = oracle_rate_on(gf0, oracle.plane_seeds((0, 0, 0), (2, 0, 0), (0, 2, 0), m0, m0),
                                              o.tol_rel)
        line["cpu_baseline"]["sample"] += " (the first field's cut)"
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_euler(args, qsl, torch, dev, rank, world, local):
    """Fixed-step Euler (Sec. "Integration methods": step 1/5 of the smallest
    spacing) against the adaptive cell-wise Dormand-Prince path on the bench
    field's 1024^2 z = 0 map: map time (CUDA events) and each path's error
    against the FP64 oracle at tol 1e-11 on 200 seeded pixels."""
    import oracle
    from paper_1609_00724_gb300 import inputs
    c = args.coarse
    gf = make_field(replica_seed(FIELD_SEED, rank), dev, args.grid)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    N = c * c
    q = torch.empty(N, device=dev)
    L = torch.empty(N, device=dev)
    fc = torch.empty(2 * N, dtype=torch.uint8, device=dev)
    runs = {"euler": qsl.qsl_opts_default(integrator=qsl.QSL_EULER, euler_h=0.2),
            "adaptive_cell": opts(qsl)}
    idx = inputs.subsample(N, 200, 7)
    seeds = oracle.plane_seeds([0, 0, 0], [2, 0, 0], [0, 2, 0], c, c)[idx]
    g = inputs.to_numpy64(make_field(replica_seed(FIELD_SEED, rank), "cpu", args.grid))
    Fo = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    ref = oracle.trace_seeds(Fo, seeds, oracle.default_opts(tol_abs=1e-11, tol_rel=1e-11, nthreads=os.cpu_count()))
    cell = float(min(np.min(np.diff(a)) for a in (g.xc, g.yc, g.zc)))
    res = {}
    for name, o in runs.items():
        best = None
        for _ in range(3):
            qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), c, c, o, q=q, length=L, faces=fc)
            st = qsl.qsl_last_stats()
            best = st["kernel_ms"] if best is None else min(best, st["kernel_ms"])
        qg, lg = q.cpu().numpy()[idx], L.cpu().numpy()[idx]
        fg = fc.cpu().numpy().reshape(-1, 2)[idx]
        same = (fg[:, 0] == ref["face_f"]) & (fg[:, 1] == ref["face_b"])
        ok = same & np.isfinite(ref["q_perp"]) & (ref["q_perp"] < 1e6)
        qe = np.abs(qg[ok] / ref["q_perp"][ok] - 1)
        le = np.abs(lg[same] - ref["L"][same]) / np.maximum(ref["L"][same], cell)
        res[name] = {"map_ms": best, "q_points_per_s": N / (best / 1000.0), "stage_evals": st["stage_evals"],
                     "faces_equal": float(same.mean()), "q_rel_median": float(np.median(qe)),
                     "q_rel_p99": float(np.quantile(qe, 0.99)), "q_rel_max": float(qe.max()),
                     "l_rel_max": float(le.max())}
    line = {"metric": "Euler fixed-step map throughput / adaptive cell-wise throughput (errors vs FP64 oracle)",
            "value": res["euler"]["q_points_per_s"] / res["adaptive_cell"]["q_points_per_s"], "unit": "x",
            "n_gpus": world, "steps": 3, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "4-charge potential field %d^3 FP32, %d^2 z=0 Q map" % (args.grid, c),
                       "euler_h_cells": 0.2, "adaptive_tol": RUN["tol"], "parity_seeds": 200},
            "results": res}
    if rank == 0:
        print(json.dumps(line), flush=True)


def map_parity(oracle, Fo, seeds, idx, q, L, fc, cell, lo, hi, opts_ref):
    """Sampled pixels of a GPU map against the FP64 oracle (tol 1e-11): end
    faces, Q (Q < 1e6, same faces) and L relative to max(L, one cell)."""
    ref = oracle.trace_seeds(Fo, seeds[idx], opts_ref)
    qg, lg = q.cpu().numpy()[idx], L.cpu().numpy()[idx]
    fg = fc.cpu().numpy().reshape(-1, 2)[idx]
    same = (fg[:, 0] == ref["face_f"]) & (fg[:, 1] == ref["face_b"])
    ok = same & np.isfinite(ref["q_perp"]) & (ref["q_perp"] < 1e6)
    qe = np.abs(qg[ok] / ref["q_perp"][ok] - 1)
    le = np.abs(lg[same] - ref["L"][same]) / np.maximum(ref["L"][same], cell)
    return {"n": int(len(idx)), "faces_equal": float(same.mean()), "q_checked": int(ok.sum()),
            "q_max_rel": float(qe.max()) if qe.size else None, "l_max_rel": float(le.max()) if le.size else None}


def map_line(args, qsl, world, metric, workload, name_q, best_ms, N, st, flop, parity, cpu, extra):
    a = st["stage_evals"] * flop / (best_ms / 1000.0) / 1e12
    return {"metric": metric, "value": N / (best_ms / 1000.0), "unit": UNIT, "n_gpus": world, "steps": 3,
            "warmup": 1, "ms_per_step": best_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": dict({"workload": workload}, **extra),
            "roofline": {"bound": "alu", "achieved": a, "peak": PEAK["fp32"], "unit": "TFLOP/s",
                         "frac": a / PEAK["fp32"], "traffic": None, "kernel": name_q, "kernel_ms": best_ms,
                         "stage_evals": st["stage_evals"], "flop_per_stage": flop,
                         "peak_note": "of measured: FP32 FMA microbenchmark in this run"},
            "parity": parity, "cpu_baseline": cpu}


def run_spherical(args, qsl, torch, dev, rank, world, local):
    """Spherical geometry (Eq. fl_sph, Eq. dev_sph): a 6-charge potential field
    on a wedge (longitude and latitude +-0.4 and +-0.3 rad, radius 1 to 1.5;
    256 x 192 x 128 vertices), the spherical slice at r = 1 (the footpoints on
    the inner sphere) as a 1024 x 768 map, traced by the Cash-Karp kernel in
    FP32 with FP64 assembly at tol 1e-7: Q-points/s and errors against the
    FP64 oracle in spherical geometry on 200 seeded pixels."""
    import oracle
    from paper_1609_00724_gb300 import inputs
    ch = inputs.random_wedge_charges(6, replica_seed(7, rank))
    n = (256, 192, 128)
    gf = inputs.spherical_charge_field(ch, n, device=dev, slab=8)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    qsl.qsl_set_geometry(F, qsl.QSL_GEOM_SPHERICAL)
    nu, nv = 1024, 768
    N = nu * nv
    w = inputs.WEDGE
    c, u, v = (0.0, 0.0, 1.0), (w[0][1] - w[0][0], 0, 0), (0, w[1][1] - w[1][0], 0)
    q, L = torch.empty(N, device=dev), torch.empty(N, device=dev)
    fc = torch.empty(2 * N, dtype=torch.uint8, device=dev)
    tol = args.tol if args.tol is not None else 1e-7
    o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, integrator=qsl.QSL_RKCK54)
    best = None
    for _ in range(4):
        qsl.qsl_q_map_2d(F, c, u, v, nu, nv, o, q=q, length=L, faces=fc)
        st = qsl.qsl_last_stats()
        best = st["kernel_ms"] if best is None else min(best, st["kernel_ms"])
    torch.cuda.synchronize()
    parity, cpu = None, None
    if rank == 0:
        g = inputs.to_numpy64(gf)
        Fo = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0, geometry=1)
        seeds = oracle.plane_seeds(list(c), list(u), list(v), nu, nv)
        cell = float(min(np.min(np.diff(a)) for a in (g.xc, g.yc, g.zc)))
        parity = map_parity(oracle, Fo, seeds, inputs.subsample(N, 200, 7), q, L, fc, cell,
                            [a[0] for a in w], [a[1] for a in w],
                            oracle.default_opts(tol_abs=1e-11, tol_rel=1e-11, nthreads=os.cpu_count()))
        if not args.no_cpu_baseline:
            cpu = oracle_rate_on(gf, seeds, tol, geometry=1)
    line = map_line(args, qsl, world, "Q-points/s (spherical slice map, Cash-Karp)",
                    "6-charge potential field on a spherical wedge, 256x192x128 vertices, r = 1 slice %dx%d" % (nu, nv),
                    "trace_kernel<float,9,spherical>", best, N, st, FLOP_PER_STAGE["ck"] + 16.0, parity, cpu,
                    {"tol": tol, "integrator": "ck", "geometry": "spherical"})
    line["kernel_ms_per_map"] = best
    if rank == 0:
        print(json.dumps(line), flush=True)


# trilinear value and gradient of 3 components plus |B| (99 FLOP, as in the
# tangent stage count) against the separable K^3 stencils of the
# triquadratic (K = 3) and tricubic (K = 4) kernels: per vertex one weight
# product, 4 value FMAs, 3 gradient weights and 9 gradient FMAs (30 FLOP)
INTERP_FLOP = {1: 99.0, 2: 27 * 30.0, 3: 64 * 30.0}


def run_interp(args, qsl, torch, dev, rank, world, local):
    """Interpolation orders (Sec. "Interpolation schemes"): the bench field's
    1024^2 z = 0 map traced by the Cash-Karp kernel with trilinear,
    triquadratic and tricubic interpolation at tol 1e-7: map time, stage
    evaluations and each order's errors against the FP64 oracle with the same
    interpolation on 200 seeded pixels."""
    import oracle
    from paper_1609_00724_gb300 import inputs
    c = args.coarse
    gf = make_field(replica_seed(FIELD_SEED, rank), dev, args.grid)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    N = c * c
    q, L = torch.empty(N, device=dev), torch.empty(N, device=dev)
    fc = torch.empty(2 * N, dtype=torch.uint8, device=dev)
    tol = args.tol if args.tol is not None else 1e-7
    g = inputs.to_numpy64(make_field(replica_seed(FIELD_SEED, rank), "cpu", args.grid)) if rank == 0 else None
    seeds = oracle.plane_seeds([0, 0, 0], [2, 0, 0], [0, 2, 0], c, c)
    res = {}
    for order in (1, 2, 3):
        o = qsl.qsl_opts_default(tol_abs=tol, tol_rel=tol, integrator=qsl.QSL_RKCK54, interp_order=order)
        best = None
        for _ in range(3):
            qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), c, c, o, q=q, length=L, faces=fc)
            st = qsl.qsl_last_stats()
            best = st["kernel_ms"] if best is None else min(best, st["kernel_ms"])
        torch.cuda.synchronize()
        flop = FLOP_PER_STAGE["ck"] - INTERP_FLOP[1] + INTERP_FLOP[order]
        a = st["stage_evals"] * flop / (best / 1000.0) / 1e12
        r = {"map_ms": best, "q_points_per_s": N / (best / 1000.0), "stage_evals": st["stage_evals"],
             "flop_per_stage": flop, "tflops": a, "frac": a / PEAK["fp32"]}
        if rank == 0:
            Fo = oracle.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0, order=order)
            cell = float(min(np.min(np.diff(x)) for x in (g.xc, g.yc, g.zc)))
            r["parity"] = map_parity(oracle, Fo, seeds, inputs.subsample(N, 200, 7), q, L, fc, cell, (-1, -1, 0),
                                     (1, 1, 1), oracle.default_opts(tol_abs=1e-11, tol_rel=1e-11,
                                                                    nthreads=os.cpu_count()))
            if order == 3 and not args.no_cpu_baseline:
                r["cpu_baseline"] = oracle_rate_on(gf, seeds, tol, order=3)
        res[order] = r
    top = res[3]
    line = {"metric": "Q-points/s (1024^2 z=0 map, Cash-Karp, tricubic interpolation; other orders alongside)",
            "value": top["q_points_per_s"], "unit": UNIT, "n_gpus": world, "steps": 3, "warmup": 0,
            "ms_per_step": top["map_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "4-charge potential field %d^3 FP32, %d^2 z=0 Q map" % (args.grid, c),
                       "tol": tol, "integrator": "ck"},
            "roofline": {"bound": "alu", "achieved": top["tflops"], "peak": PEAK["fp32"], "unit": "TFLOP/s",
                         "frac": top["frac"], "traffic": None, "kernel": "trace_kernel<float,9,higher-order>",
                         "kernel_ms": top["map_ms"], "stage_evals": top["stage_evals"],
                         "flop_per_stage": top["flop_per_stage"],
                         "peak_note": "of measured: FP32 FMA microbenchmark in this run"},
            "cpu_baseline": top.get("cpu_baseline"), "orders": res}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_qcrit(args, qsl, torch, dev, rank, world, local):
    """Refinement criteria compared (Sec. "Adaptive refinements"): the FLL jump
    (tau 0.05) against a Q threshold (Q > 100), both refining the 1024^2 z = 0
    map of the bench field to 4096^2 with the same tolerance, against a dense
    4096^2 map traced at every effective cell: wall time, samples, iterations,
    and recall / precision of the cells with Q >= 100 (QSL cells) on the
    converted 4096^2 Q grids."""
    eff = args.coarse << (P - P0)
    gf = make_field(replica_seed(FIELD_SEED, rank), dev, args.grid)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    o = opts(qsl)
    qd = torch.empty(eff * eff, device=dev)
    Ld = torch.empty(eff * eff, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), eff, eff, o, q=qd, length=Ld)
    torch.cuda.synchronize()
    t_dense = time.perf_counter() - t0
    qsl_dense = torch.nan_to_num(qd, nan=0.0) >= 100.0
    bufs = alloc(torch, args.coarse, dev)
    res = {"dense": {"seconds": t_dense, "samples": eff * eff, "qsl_cells": int(qsl_dense.sum().item())}}
    p0 = int(np.log2(args.coarse))
    for name, kw in (("fll_jump", dict(criterion=qsl.QSL_REFINE_FLL_JUMP)),
                     ("q_threshold", dict(criterion=qsl.QSL_REFINE_Q_THRESHOLD, q_threshold=100.0))):
        sp = qsl.refine_spec(ndim=2, coarse_order=p0, max_order=p0 + (P - P0), center=(0, 0, 0), u=(2, 0, 0),
                             v=(0, 2, 0), tau=TAU, shift=1, max_iters=256, **kw)
        best = None
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            n, iters, traced, rc = qsl.qsl_refine(F, sp, o, bufs["key"], bufs["q"], bufs["L"], bufs["faces"],
                                                  bufs["st"], 0, bufs["qg"], bufs["lg"])
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        got = torch.nan_to_num(bufs["qg"], nan=0.0) >= 100.0
        tp = int((got & qsl_dense).sum().item())
        res[name] = {"seconds": best, "samples": int(n), "iters": int(iters), "rc": int(rc),
                     "qsl_recall": tp / max(1, int(qsl_dense.sum().item())),
                     "qsl_precision": tp / max(1, int(got.sum().item()))}
    line = {"metric": "refinement criteria: Q-threshold time / FLL-jump time (QSL-cell recall of each)",
            "value": res["q_threshold"]["seconds"] / res["fll_jump"]["seconds"], "unit": "x",
            "n_gpus": world, "steps": 1, "warmup": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "4-charge potential field %d^3 FP32, %d^2 z=0 map refined to %d^2; dense %d^2 "
                                   "reference" % (args.grid, args.coarse, eff, eff), "tau": TAU, "q_threshold": 100.0,
                       "tol": RUN["tol"], "qsl_cell": "Q >= 100"},
            "results": res}
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_learned(args, qsl, torch, dev, rank, world, local):
    """Config 5: the learned refinement proposal. Training: z-slices of
    tracer-generated volumes (random 4-12-charge fields on 128^3, coarse
    64 x 64 x 32 cell-centre volumes refined two orders by the plain
    criterion). Evaluation: an 8-charge field on 512^3, a coarse 256 x 256 x
    128 volume refined two orders (1024 x 1024 x 512 effective). Compared:
    wall time of the plain criterion with FP64 everywhere (and with FP32
    tracing) against the learned proposal (CNN on the coarse z-slices, mask
    dilated by one cell, the effective cells of a proposed coarse cell traced
    in one launch: all of them, or every other one per axis, which is one per
    output cell) with FP32 tracing and the plain criterion as fallback, run for
    a few iterations and to convergence; recall of the plain FP64 run's QSL
    pixels."""
    from paper_1609_00724_gb300 import inputs, learned
    n_vol = int(os.environ.get("QSL_LEARNED_VOLUMES", "160"))
    fb_iters = int(os.environ.get("QSL_LEARNED_FALLBACK_ITERS", "2"))
    o32 = opts(qsl)
    o64 = qsl.qsl_opts_default(tol_abs=RUN["tol"], tol_rel=RUN["tol"], integrator=INTEGRATOR[RUN["integrator"]],
                               precision=qsl.QSL_FP64)
    ot = qsl.qsl_opts_default(tol_abs=1e-6, tol_rel=1e-6, integrator=INTEGRATOR[RUN["integrator"]])
    tr_coarse = (64, 64, 32)
    X, Y, W, t_data = learned.make_training_volumes(n_vol, grid=128, coarse=tr_coarse, levels=2, tau=TAU,
                                                    seed0=5000, opts=ot, device=dev)
    nz_tr = tr_coarse[2]
    n_fit = int(0.9 * n_vol) * nz_tr
    t0 = time.perf_counter()
    net, hist, pw = learned.train(X[:n_fit], Y[:n_fit], epochs=12, batch=32, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    thr, frac, rec_cal = learned.calibrate_qsl(net, X[n_fit:], W[n_fit:], nz_tr, recall=0.995, dilate=True)
    del X, Y, W
    gf = inputs.charge_field(inputs.random_charges(8, 5), 512, dtype=torch.float32, device=dev, slab=16)
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc)
    del gf
    coarse = tuple(int(v) for v in os.environ.get("QSL_LEARNED_COARSE", "256,256,128").split(","))  # x, y, z
    cap = int(os.environ.get("QSL_LEARNED_CAPACITY", str(128 * 1024 * 1024)))
    spec = learned.volume_spec(coarse, 2, TAU)
    ext = [c * 4 for c in coarse]
    out_order = spec.max_order - 1
    res = {}

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t, r

    # plain criterion, FP64 everywhere (the reference of recall)
    smp = learned.Samples(cap, dev)
    dt, (n_p, it_p, tr_p, rc_p) = timed(lambda: smp.refine(F, spec, o64))
    res["plain_fp64"] = {"seconds": dt, "samples": n_p, "iters": it_p, "rc": rc_p}
    plain_keys = smp.key[:n_p].clone()
    qp = learned.converted_q(smp, 3, spec.max_order, ext, out_order)
    # QSL pixels: output cells holding a plain FP64 sample with Q >= 100
    hot = torch.nan_to_num(smp.q[:n_p], nan=0.0) >= 100.0
    cc = smp.coords(3, spec.max_order)[hot] >> 1
    eo = [e >> 1 for e in ext]
    qsl_cells = torch.unique(cc[:, 0] + eo[0] * (cc[:, 1] + eo[1] * cc[:, 2]))
    del smp, cc, hot
    # plain criterion with FP32 tracing (what the network is compared with)
    smp = learned.Samples(cap, dev)
    dt, (n_3, it_3, _, rc_3) = timed(lambda: smp.refine(F, spec, o32))
    res["plain_fp32"] = {"seconds": dt, "samples": n_3, "iters": it_3, "rc": rc_3}
    del smp

    ql_keep = {}

    def learned_run(max_iters, stride=1):
        s2 = learned.Samples(cap, dev)

        def go():
            s2.refine(F, learned.volume_spec(coarse, 2, TAU, max_iters=0), o32)
            L, Q, _ = learned.coarse_grids(s2, 3, spec.max_order, 2, coarse[::-1])
            if stride == "mixed":
                # the cells the network flags at every effective cell, the
                # ring the dilation adds at every other one per axis
                Xf = learned.features_slices(L, Q)
                core = learned.propose(net, Xf, thr, dilate=False)
                ring = (learned.propose(net, Xf, thr, dilate=True).bool() & ~core.bool()).to(torch.uint8)
                s2.refine(F, learned.volume_spec(coarse, 2, TAU, proposal=ring, max_iters=0, proposal_stride=2), o32)
                r = s2.refine(F, learned.volume_spec(coarse, 2, TAU, proposal=core, max_iters=max_iters), o32)
                return r, int(core.sum().item()) + int(ring.sum().item())
            budget = max(0, int(0.9 * (cap - s2.count) / (4 // stride) ** 3))
            mask = learned.propose(net, learned.features_slices(L, Q), thr, dilate=True)
            if int(mask.sum().item()) > budget:
                mask = learned.propose(net, learned.features_slices(L, Q), thr, budget=budget // 27, dilate=True)
            r = s2.refine(F, learned.volume_spec(coarse, 2, TAU, proposal=mask, max_iters=max_iters,
                                                 proposal_stride=stride), o32)
            return r, int(mask.sum().item())

        dt, ((n_l, it_l, tr_l, rc_l), ncells) = timed(go)
        lk = s2.key[:n_l]
        pos = torch.searchsorted(lk, plain_keys).clamp(max=n_l - 1)
        sample_recall = float((lk[pos] == plain_keys).float().mean().item())
        ql = learned.converted_q(s2, 3, spec.max_order, ext, out_order)
        ql_keep[(max_iters, stride)] = ql
        qsl_pix = torch.nan_to_num(ql.reshape(-1)[qsl_cells], nan=0.0) >= 100.0
        old_pix = torch.nan_to_num(qp, nan=0.0) >= 100.0
        old_recall = float(((torch.nan_to_num(ql, nan=0.0) >= 100.0) & old_pix).sum().item() /
                           max(1, int(old_pix.sum().item())))
        return {"seconds": dt, "samples": n_l, "iters": it_l, "rc": rc_l, "proposed_cells": ncells,
                "proposed_frac": ncells / float(np.prod(coarse)), "fallback_max_iters": max_iters,
                "proposal_stride": stride,
                "qsl_pixel_recall": float(qsl_pix.float().mean().item()), "sample_recall": sample_recall,
                "converted_qsl_recall": old_recall}

    runs = {"learned_fp32_bounded": (fb_iters, 1), "learned_fp32_full": (64, 1),
            "learned_fp32_stride2_bounded": (fb_iters, 2), "learned_fp32_stride2_full": (64, 2),
            "learned_fp32_mixed_bounded": (fb_iters, "mixed"), "learned_fp32_mixed_full": (64, "mixed")}
    for k, (mi, stv) in runs.items():
        res[k] = learned_run(mi, stv)
    dense = None
    if os.environ.get("QSL_LEARNED_DENSE") == "1":
        # a dense map of every effective cell (FP32), max-pooled to the output
        # lattice: which map shows the QSL cells of the dense truth
        torch.cuda.empty_cache()
        nx, ny, nz = ext
        qd = torch.empty(nx * ny * nz, device=dev)
        dt_d, _ = timed(lambda: qsl.qsl_q_volume_3d(F, (-1, -1, 0), (1, 1, 1), nx, ny, nz, o32, q=qd))
        qd = torch.nan_to_num(qd, nan=0.0).view(1, 1, nz, ny, nx)
        truth = torch.nn.functional.max_pool3d(qd, 2).reshape(-1) >= 100.0
        del qd
        dense = {"seconds": dt_d, "qsl_cells": int(truth.sum().item())}
        for k, qmap in [("plain_fp64", qp)] + [(k, ql_keep[v]) for k, v in runs.items()]:
            got = torch.nan_to_num(qmap, nan=0.0).reshape(-1) >= 100.0
            tp = int((got & truth).sum().item())
            dense[k] = {"recall": tp / max(1, dense["qsl_cells"]), "precision": tp / max(1, int(got.sum().item()))}
    meets = [k for k in runs if res[k]["qsl_pixel_recall"] >= 0.99]
    best = min(meets, key=lambda k: res[k]["seconds"]) if meets else "learned_fp32_full"
    line = {"metric": "refined-map wall time: learned proposal + FP32 vs plain FP64 at >= 99% QSL-pixel recall",
            "value": res["plain_fp64"]["seconds"] / res[best]["seconds"], "unit": "x speed-up",
            "n_gpus": world, "steps": 1, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "8-charge field 512^3, coarse 256x256x128 -> 1024x1024x512 effective",
                       "training": {"volumes": n_vol, "slices": n_vol * nz_tr, "data_s": t_data, "train_s": t_train,
                                    "final_loss": hist[-1], "pos_weight": pw, "threshold": thr,
                                    "proposed_frac_heldout": frac, "qsl_recall_heldout": rec_cal},
                       "tau": TAU, "tol": RUN["tol"], "qsl_pixel": "output cell (512x512x256) holding a plain FP64 "
                                                                   "sample with Q >= 100"},
            "headline": best, "recall_target_met": bool(meets),
            "vs_plain_fp32": res["plain_fp32"]["seconds"] / res[best]["seconds"],
            "qsl_pixels": int(qsl_cells.numel()), "results": res, "dense_truth": dense}
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    RUN["integrator"] = args.integrator
    RUN["tol"] = args.tol if args.tol is not None else TOL
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1609_00724_gb300 import qsl
    qsl.lib()
    global PEAKS_RUN
    PEAKS_RUN = measure_peaks(local)
    PEAK.update(fp32=PEAKS_RUN["fp32_tflops"], l2=PEAKS_RUN["l2_read_gbs"],
                note="%.1f TFLOP/s FP32, %.0f GB/s L2 read at a median %s MHz SM clock" % (
                    PEAKS_RUN["fp32_tflops"], PEAKS_RUN["l2_read_gbs"], PEAKS_RUN["clocks"].get("sm_mhz")))
    if args.shape:
        RUN["shape"] = tuple(int(v) for v in args.shape.split(","))
    if args.hmax:
        RUN["h_max"] = args.hmax
    if args.config != "refine2d":
        {"hyperbolic": run_hyperbolic, "volume": run_volume, "batch64": run_batch, "learned": run_learned,
         "qcrit": run_qcrit, "euler": run_euler, "spherical": run_spherical, "interp": run_interp}[args.config](
            args, qsl, torch, dev, rank, world, local)
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    field_seed = replica_seed(FIELD_SEED, rank)
    gf = make_field(field_seed, dev, args.grid)
    if args.profile_refine:
        bufs = alloc(torch, args.coarse, dev)
        for _ in range(args.steps):
            tr, info = gpu_step(qsl, gf, bufs, args.coarse)
        rs = qsl.qsl_last_refine_stats()
        print(json.dumps({"profile_refine": True, "grid": args.grid, "coarse": args.coarse, "tol": RUN["tol"],
                          "shape": RUN.get("shape"), "h_max": RUN.get("h_max"), "q_points": tr, **info, **rs}))
        return
    if args.profile_pass:
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
        it = None
        if args.pass_seeds and os.path.exists(args.pass_seeds):
            pos = np.load(args.pass_seeds)
        else:
            bufs = alloc(torch, args.coarse, dev)
            org = torch.full((bufs["key"].shape[0],), -1, dtype=torch.int32, device=dev)
            n, it, _, _ = qsl.qsl_refine(F, spec(qsl, args.coarse), opts(qsl), bufs["key"], bufs["q"], bufs["L"],
                                         bufs["faces"], bufs["st"], origin=org)
            sel = org[:n] == args.profile_pass
            pos = sample_positions(qsl, bufs["key"][:n][sel].cpu().numpy().view(np.uint64), args.coarse)
            del bufs, org
            torch.cuda.synchronize()
            qsl.qsl_trim_pool()
            if args.pass_seeds:
                np.save(args.pass_seeds, pos)
        sd = torch.as_tensor(pos).to(dev)
        ol = opts(qsl)
        ol.length_only = 1
        if PASS_STEPPER == 0:  # the decision traces of qsl_refine
            ol.integrator, ol.h_max = qsl.QSL_RKCK54, PASS_H_MAX
        for _ in range(args.steps):
            qsl.qsl_trace_seeds(F, sd, ol)
        st = qsl.qsl_last_stats()
        print(json.dumps({"profile_pass": args.profile_pass, "seeds": int(sd.shape[0]), "kernel_ms": st["kernel_ms"],
                          "stage_evals": st["stage_evals"], "landings": st["landing"], "iters": it}))
        return
    if args.profile_map:
        F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
        N = args.coarse * args.coarse
        qm, Lm = torch.empty(N, device=dev), torch.empty(N, device=dev)
        for _ in range(args.steps):
            qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), args.coarse, args.coarse, opts(qsl), q=qm, length=Lm)
        st = qsl.qsl_last_stats()
        print(json.dumps({"profile_map": True, "grid": args.grid, "coarse": args.coarse, "kernel_ms": st["kernel_ms"],
                          "stage_evals": st["stage_evals"], "retraced": st["retraced"]}))
        return
    bufs = alloc(torch, args.coarse, dev)
    # autotune (tolerance and launch shape) on 131072 seeds of the coarse map
    from paper_1609_00724_gb300 import inputs as _inp
    c = args.coarse
    pick = _inp.subsample(c * c, min(131072, c * c), 17)
    ii, jj = pick % c, pick // c
    sd = np.column_stack([-1 + (ii + 0.5) * 2 / c, -1 + (jj + 0.5) * 2 / c, np.zeros(len(pick))])
    F0 = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    tuned = opts(qsl)
    tune_rep = (qsl.qsl_autotune(F0, torch.as_tensor(sd).to(dev), tuned)
                if not (args.no_tune or args.shape) else None)
    del F0
    if tune_rep:
        RUN["tol"] = tuned.tol_rel
        RUN["shape"] = (tuned.warps_per_block, tuned.blocks_per_sm, tuned.refill_min)
        RUN["h_max"] = tuned.h_max

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3)):
        gpu_step(qsl, gf, bufs, args.coarse)
    # --- timed region: device-resident inputs (the field is 268 MB, larger than L2)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    traced_total = 0
    kernel_ms = []
    stage_evals = 0
    info = {}
    barrier()
    launches0 = qsl.qsl_kernel_launches()
    with ClockSampler(local) as clk:
        start.record()
        for _ in range(args.steps):
            tr, info = gpu_step(qsl, gf, bufs, args.coarse, stream_sync=False)
            traced_total += tr
        end.record()
        barrier()
    ms = start.elapsed_time(end)
    launches = qsl.qsl_kernel_launches() - launches0
    rs = qsl.qsl_last_refine_stats()  # the last timed step's qsl_refine
    ms_max, units = reduce_timing(torch, ms, traced_total, world, dev)
    value = units / (ms_max / 1000.0)

    # --- dominant kernel (tracer) timing over one more step: CUDA events recorded
    # by the library around each tracer launch on the launching stream
    F = qsl.qsl_load_field(gf.bx, gf.by, gf.bz, gf.xc, gf.yc, gf.zc, qsl.QSL_PAPER_NORMALIZE_FIRST)
    N = args.coarse * args.coarse
    qm = torch.empty(N, device=dev)
    Lm = torch.empty(N, device=dev)
    for _ in range(2):
        qsl.qsl_q_map_2d(F, (0, 0, 0), (2, 0, 0), (0, 2, 0), args.coarse, args.coarse, opts(qsl), q=qm, length=Lm)
    st = qsl.qsl_last_stats()
    kms = st["kernel_ms"]
    flop_per_stage = FLOP_PER_STAGE[RUN["integrator"]]
    achieved_tflops = st["stage_evals"] * flop_per_stage / (kms / 1000.0) / 1e12
    kname = "cell_kernel_f32<9>" if RUN["integrator"] == "cell" else "trace_kernel<float,9>"
    default_workload = args.grid == 256 and args.coarse == 1024 and RUN["integrator"] == "cell"
    peak_note = "of measured: %s in this run (%s)" % ("FP32 FMA microbenchmark" if PEAK["l2"] else "nominal",
                                                    PEAK["note"])

    def gather(entries, ms):
        """Algorithmic gather rate (8 corner vertices per cell entered) against the measured L2 read peak."""
        if not PEAK["l2"] or ms <= 0:
            return None
        a = entries * GATHER_BYTES_PER_ENTRY / (ms / 1000.0) / 1e9
        return {"bound": "l2", "achieved": a, "peak": PEAK["l2"], "unit": "GB/s", "frac": a / PEAK["l2"],
                "bytes_per_entry": GATHER_BYTES_PER_ENTRY, "entries": int(entries),
                "peak_note": "of measured: L2 read microbenchmark in this run"}

    roof_coarse = {"bound": "alu", "achieved": achieved_tflops, "peak": PEAK["fp32"], "unit": "TFLOP/s",
                   "frac": achieved_tflops / PEAK["fp32"],
                   "traffic": TRAFFIC_COARSE_BYTES if default_workload else None,
                   "kernel": kname + " (%d^2 coarse map, one launch)" % args.coarse, "kernel_ms": kms,
                   "stage_evals": st["stage_evals"], "accepted": st["accepted"], "rejected": st["rejected"],
                   "landings": st["landing"], "flop_per_stage": flop_per_stage, "peak_note": peak_note,
                   "gather": gather(st["landing"] + 2 * N, kms)}
    # refinement passes: few lines per launch, each launch as long as its
    # longest line (latency-bound); average over the step's passes, which
    # trace lengths only with the FLL-jump criterion
    pass_ms = rs["passes_ms"] / max(rs["passes"], 1)
    len_only = rs["deferred_ms"] > 0
    # the Cash-Karp decision traces read a cell's corners at every stage (the
    # kernel's cell cache skips repeats): one 8-vertex gather per stage
    ck_pass = len_only and PASS_STEPPER == 0
    if ck_pass:
        pass_flop, pass_kernel = FLOP_PER_STAGE_LEN["ck"], "trace_kernel<float,3> (Cash-Karp decision traces, "
    elif len_only:
        pass_flop, pass_kernel = FLOP_PER_STAGE_LEN["cell"], "cell_len_kernel<float> ("
    else:
        pass_flop = flop_per_stage
        pass_kernel = ("cell_coop_kernel<float,9>" if RUN["integrator"] == "cell" else kname) + " ("
    pass_tflops = (rs["pass_stage_evals"] * pass_flop / (rs["passes_ms"] / 1000.0) / 1e12
                   if rs["passes_ms"] > 0 else 0.0)
    roof_passes = {"bound": "alu", "achieved": pass_tflops, "peak": PEAK["fp32"], "unit": "TFLOP/s",
                   "frac": pass_tflops / PEAK["fp32"],
                   "traffic": TRAFFIC_PASS_BYTES if default_workload else None,
                   "kernel": pass_kernel + "%srefinement passes, %d per step)"
                   % ("length-only " if len_only else "", rs["passes"]), "kernel_ms": pass_ms,
                   "stage_evals": rs["pass_stage_evals"] // max(rs["passes"], 1), "flop_per_stage": pass_flop,
                   "peak_note": peak_note + "; launches are bound by the latency of their longest line, not by the "
                                            "pipe",
                   "gather": gather((rs["pass_stage_evals"] if ck_pass else rs["pass_landings"] + 2 * rs["pass_lines"])
                                    / max(rs["passes"], 1), pass_ms)}
    passes_dominate = rs["passes_ms"] > rs["coarse_ms"]
    step_breakdown = {"device_ms": rs["total_ms"], "coarse_trace_ms": rs["coarse_ms"],
                      "pass_trace_ms": rs["passes_ms"], "deferred_trace_ms": rs["deferred_ms"],
                      "passes": rs["passes"], "iters": rs["iters"], "pass_lines": rs["pass_lines"],
                      "other_ms": rs["total_ms"] - rs["coarse_ms"] - rs["passes_ms"] - rs["deferred_ms"]}

    # --- end to end through the C ABI with host buffers (pinned), copies inside:
    # field load, refinement with conversion, and the FLEDGE of the converted
    # length grid, as in the timed step; median of three runs
    eff = args.coarse << (P - P0)
    host = {k: torch.empty_like(v, device="cpu").pin_memory() for k, v in bufs.items() if k != "eff"}
    hb = [a.cpu().pin_memory() for a in (gf.bx, gf.by, gf.bz)]
    e2e_t = []
    for it in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Fh = qsl.qsl_load_field(hb[0].numpy(), hb[1].numpy(), hb[2].numpy(), gf.xc, gf.yc, gf.zc,
                                qsl.QSL_PAPER_NORMALIZE_FIRST)
        n_h, _, traced_h, _ = qsl.qsl_refine(Fh, spec(qsl, args.coarse), opts(qsl), host["key"].numpy(),
                                             host["q"].numpy(), host["L"].numpy(), host["faces"].numpy(),
                                             host["st"].numpy(), 0, host["qg"].numpy(), host["lg"].numpy())
        qsl.qsl_fledge(host["lg"].numpy().reshape(eff, eff), host["sg"].numpy())
        e2e_t.append(time.perf_counter() - t0)
        del Fh
    e2e_value = traced_h / float(np.median(e2e_t))
    h2d = sum(a.numel() * a.element_size() for a in hb) + eff * eff * 4  # the field; the length grid to FLEDGE
    d2h = n_h * (8 + 4 + 4 + 2 + 1) + 3 * eff * eff * 4  # samples; Q, L and FLEDGE grids

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "4-charge potential field %d^3 FP32, %d^2 z=0 Q map refined to %d^2 effective"
                                   % (args.grid, args.coarse, eff),
                       "tol": RUN["tol"], "integrator": RUN["integrator"], "tau": TAU,
                       "coarse_order": int(np.log2(args.coarse)), "max_order": int(np.log2(eff)),
                       "interp": "paper (normalise first)", "precision": "FP32 trace, FP64 Q",
                       "l2": "inputs larger than L2 (268 MB packed field)", "parallelism": "replicas x%d" % world,
                       "autotune": tune_rep,
                       "samples_per_step": info.get("samples"), "refine_iters": info.get("iters"),
                       "q_points_per_step": traced_total // max(args.steps, 1)},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                    "runs_s": e2e_t},
            "gpu_launches": launches,
            "roofline": roof_passes if passes_dominate else roof_coarse,
            "roofline_other": roof_coarse if passes_dominate else roof_passes,
            "peaks": PEAKS_RUN,
            "step_breakdown": step_breakdown}
    if rank == 0 and not args.no_cpu_baseline:
        gf_cpu = make_field(field_seed, "cpu", args.grid)
        n_s = int(info.get("samples") or 0)
        rate, nsm, nwin, cores, secs = oracle_refine_rate(gf_cpu, RUN["tol"], args.coarse)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "the oracle's refinement (coarse pass, FLL-jump passes, tangent-space "
                                          "values) of %d seeded %dx%d-coarse-cell windows of the map at its cell "
                                          "sizes, %d samples, tol %g (the autotuned GPU tolerance), %.1f s"
                                          % (nwin, WINDOW, WINDOW, nsm, RUN["tol"], secs)}
        line["parity"] = parity_sample(qsl, gf, gf_cpu, args.coarse)
        line["parity_refined"] = refined_parity(bufs, n_s, gf_cpu, args.coarse)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
