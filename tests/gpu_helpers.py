"""Shared helpers of the GPU parity tests (inputs and comparisons only)."""
import numpy as np

# parity bar: Q rel <= 1e-3 for Q < 1e6, length rel <= 1e-5 (with the length
# of one cell as the floor of the denominator: a sub-cell line leaving at a
# grazing angle has a length set by a cancellation in the field samples, so it
# is held to 1e-5 cells absolute), end-face labels exact for ends more than
# 1e-3 cells from a face edge
Q_RTOL = 1e-3
L_RTOL = 1e-5
EDGE_CELLS = 1e-3

# FP32 tracer tolerance used by the parity runs (the oracle runs at 1e-11)
GPU_TOL = 1e-7

# decision lengths of the refinement passes (lengths-only Cash-Karp across
# cells, step cap 4 smallest spacings) against the oracle's trace with the same
# method and settings: where the cap sets every step both take the same steps
# and meet L_RTOL; where the error estimate sets some steps (tight tolerances)
# the FP32 and FP64 runs step differently near cell faces and differ by the
# method's own error across the kinks of the trilinear field
D_RTOL = 1e-4


def min_spacing(gf):
    """Smallest grid spacing over the three axes of a GridField."""
    return float(min(np.min(np.diff(np.asarray(a, dtype=np.float64))) for a in (gf.xc, gf.yc, gf.zc)))


def length_err(L, Lr, cell):
    """Length error of the parity bar: |L - Lr| / max(Lr, cell)."""
    L = np.asarray(L, dtype=np.float64)
    Lr = np.asarray(Lr, dtype=np.float64)
    return np.abs(L - Lr) / np.maximum(Lr, cell)


def edge_distance(x, face, lo, hi):
    """Distance (domain units) of an end point on `face` to the nearest edge of that face."""
    ax = face // 2
    d = np.inf
    for a in range(3):
        if a == ax:
            continue
        d = min(d, x[a] - lo[a], hi[a] - x[a])
    return d


def compare_lines(gpu, ref, cell, lo, hi, q_key_gpu="q_perp", q_key_ref="q_perp", q_rtol=Q_RTOL, l_rtol=L_RTOL):
    """gpu: dict/record arrays from the CUDA path; ref: oracle dict; cell: the
    smallest grid spacing. Returns a report dict and raises AssertionError on a
    parity failure."""
    n = len(ref["L"])
    fails = []
    label_checked = 0
    q_checked = 0
    floored = 0  # lines shorter than one cell: their length error is taken against one cell
    worst_q = 0.0
    worst_l = 0.0
    for i in range(n):
        sf, sb = int(ref["st_f"][i]), int(ref["st_b"][i])
        away = True
        for key_x, key_face in (("xf", "face_f"), ("xb", "face_b")):
            f = int(ref[key_face][i])
            if f != 255 and edge_distance(ref[key_x][i], f, lo, hi) <= EDGE_CELLS * cell:
                away = False
        if away:
            label_checked += 1
            if int(gpu["face_f"][i]) != int(ref["face_f"][i]) or int(gpu["face_b"][i]) != int(ref["face_b"][i]):
                fails.append(("face", i, (gpu["face_f"][i], gpu["face_b"][i]), (ref["face_f"][i], ref["face_b"][i])))
                continue
        Lr = ref["L"][i]
        if np.isfinite(Lr):
            floored += int(Lr < cell)
            e = abs(gpu["L"][i] - Lr) / max(Lr, cell)
            worst_l = max(worst_l, e)
            if not e <= l_rtol:
                fails.append(("L", i, gpu["L"][i], Lr, e))
        qr = ref[q_key_ref][i]
        if np.isfinite(qr) and qr < 1e6 and away:
            q_checked += 1
            e = abs(gpu[q_key_gpu][i] / qr - 1)
            worst_q = max(worst_q, e)
            if not e <= q_rtol:
                fails.append(("Q", i, gpu[q_key_gpu][i], qr, e))
    rep = {"n": n, "labels_checked": label_checked, "q_checked": q_checked, "worst_q": worst_q, "worst_l": worst_l,
           "under_one_cell": floored, "fails": fails[:10], "n_fail": len(fails)}
    print("parity:", {k: v for k, v in rep.items() if k != "fails"}, rep["fails"][:4])
    assert not fails, rep
    return rep
