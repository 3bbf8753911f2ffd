"""Oracle pins for the Hilbert-curve refinement (Sec. "Adaptive refinements"),
driven by analytic length maps so that only the refinement logic is tested."""
import numpy as np
import pytest


def circle_map(x):
    r = np.hypot(x[:, 0] - 0.1, x[:, 1] + 0.05)
    return np.ones(len(x)), np.where(r < 0.5, 1.0, 0.0)


def smooth_map(x):
    return 2.0 + np.sin(3 * x[:, 0]) * np.cos(2 * x[:, 1]), x[:, 0] ** 2 + x[:, 1]


def _coarse_key_range(oracle_mod, ndim, p0, p, extent):
    R = 1 << (p - p0)
    keys = []
    for k in range(extent[2] // R if ndim == 3 else 1):
        for j in range(extent[1] // R):
            for i in range(extent[0] // R):
                c = (i * R + R // 2, j * R + R // 2, k * R + R // 2)[:ndim]
                keys.append(oracle_mod.hilbert_key(c, ndim, p))
    return min(keys), max(keys)


def test_negative_tau_gives_dense_lattice_2d(oracle_mod):
    """tau < 0 flags every pair: refinement fills every cell between the first
    and the last coarse sample along the curve (it only inserts between
    samples)."""
    k0, k1 = _coarse_key_range(oracle_mod, 2, 2, 4, (16, 16))
    for shift in (0, 1):
        sp = oracle_mod.refine_spec(ndim=2, coarse_order=2, max_order=4, center=(0, 0, 0), u=(2, 0, 0),
                                    v=(0, 2, 0), tau=-1.0, shift=shift)
        r = oracle_mod.refine_fn(smooth_map, sp)
        if shift == 0:
            assert list(r["key"]) == list(range(k0, k1 + 1))
        else:  # the shifted pass also reaches cells beyond the ends of the coarse range
            assert set(range(k0, k1 + 1)) <= set(int(k) for k in r["key"])


def test_negative_tau_gives_dense_lattice_3d_clipped(oracle_mod):
    """A 2:1 box: the order-3 curve is clipped to 8 x 8 x 4 cells."""
    sp = oracle_mod.refine_spec(ndim=3, coarse_order=1, max_order=3, extent=(8, 8, 4), lo=(-1, -1, 0),
                                hi=(1, 1, 1), tau=-1.0, shift=0)
    r = oracle_mod.refine_fn(lambda x: (np.ones(len(x)), x[:, 0] + 2 * x[:, 2]), sp)
    k0, k1 = _coarse_key_range(oracle_mod, 3, 1, 3, (8, 8, 4))
    want = sorted(k for k in range(k0, k1 + 1) if oracle_mod.hilbert_coords(k, 3, 3)[2] < 4)
    assert list(r["key"]) == want


def test_large_tau_keeps_coarse_samples_only(oracle_mod):
    sp = oracle_mod.refine_spec(ndim=2, coarse_order=3, max_order=6, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0),
                                tau=10.0)
    r = oracle_mod.refine_fn(smooth_map, sp)
    cells = [oracle_mod.hilbert_coords(k, 2, 6) for k in r["key"]]
    assert len(cells) == 64
    assert all(c[0] % 8 == 4 and c[1] % 8 == 4 for c in cells)  # index R/2 modulo R, R = 8
    assert r["iters"] == 0


def test_step_map_refines_only_along_the_step(oracle_mod):
    p0, p = 3, 7
    n = 1 << p
    sp = oracle_mod.refine_spec(ndim=2, coarse_order=p0, max_order=p, center=(0, 0, 0), u=(2, 0, 0),
                                v=(0, 2, 0), tau=0.5)
    r = oracle_mod.refine_fn(circle_map, sp)
    keys = r["key"].astype(np.int64)
    assert np.all(np.diff(keys) > 0)  # unique, sorted
    cells = np.array([oracle_mod.hilbert_coords(k, 2, p) for k in r["key"]])
    R = 1 << (p - p0)
    coarse = (cells[:, 0] % R == R // 2) & (cells[:, 1] % R == R // 2)
    assert coarse.sum() == (n // R) ** 2  # every coarse sample is kept
    # termination: no pair adjacent along the curve straddles the step with key gap > 1
    L = r["L"]
    straddle = np.abs(np.diff(L)) > 0.5
    assert np.all(np.diff(keys)[straddle] == 1)
    # every refined sample lies near the step: within sqrt(6 x coarse key gap) cells
    xy = -1 + (cells + 0.5) * 2.0 / n
    d = np.abs(np.hypot(xy[:, 0] - 0.1, xy[:, 1] + 0.05) - 0.5) * n / 2
    assert np.all(d[~coarse] <= np.sqrt(6 * R * R) + 1)


def test_shifted_curve_reduces_misses(oracle_mod):
    """The shifted-curve pass must find substantially more of the step's
    boundary cells than refinement along one curve (the misses the paper's
    shift is meant to remove)."""
    p0, p = 3, 7
    n = 1 << p
    cov = {}
    for shift in (0, 1):
        sp = oracle_mod.refine_spec(ndim=2, coarse_order=p0, max_order=p, center=(0, 0, 0), u=(2, 0, 0),
                                    v=(0, 2, 0), tau=0.5, shift=shift)
        r = oracle_mod.refine_fn(circle_map, sp)
        S = {oracle_mod.hilbert_coords(k, 2, p) for k in r["key"]}
        hit = tot = 0
        for i in range(n):
            for j in range(n):
                x, y = -1 + (i + 0.5) * 2 / n, -1 + (j + 0.5) * 2 / n
                if abs(np.hypot(x - 0.1, y + 0.05) - 0.5) < 1.0 / n:
                    tot += 1
                    hit += (i, j) in S
        cov[shift] = hit / tot
    assert cov[1] > 3 * cov[0]
    assert cov[1] > 0.7


def test_converter_on_refined_samples_keeps_sampled_values(oracle_mod):
    p0, p = 2, 5
    sp = oracle_mod.refine_spec(ndim=2, coarse_order=p0, max_order=p, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0),
                                tau=0.3)
    r = oracle_mod.refine_fn(smooth_map, sp)
    grid = oracle_mod.convert(r["key"], r["q"], 2, p, (32, 32, 0), p, True)
    for k, q in zip(r["key"], r["q"]):
        x, y = oracle_mod.hilbert_coords(k, 2, p)
        assert grid[y, x] == q
    assert np.all(np.isfinite(grid))
    lo, hi = r["q"].min(), r["q"].max()
    assert np.all((grid >= lo * (1 - 1e-12)) & (grid <= hi * (1 + 1e-12)))


def ring_q_map(x):
    """Q: a ridge of height 1000 on the circle r = 0.5 (width 0.03) over Q = 2;
    L is constant, so only the Q criterion can refine."""
    r = np.hypot(x[:, 0] - 0.1, x[:, 1] + 0.05)
    return 2.0 + 1000.0 * np.exp(-((r - 0.5) / 0.03) ** 2), np.ones(len(x))


def test_q_threshold_criterion_refines_the_high_q_region(oracle_mod):
    """Criterion 1 (the alternative the paper compares against): a pair of
    curve-adjacent samples is refined when either sample's Q exceeds the
    threshold. At termination no adjacent pair with key gap > 1 (on the curve,
    with the shifted pass off) has a sample above the threshold; every cell on
    the curve between two refined neighbours of a high-Q sample is traced; a
    threshold above max Q keeps only the coarse samples; the FLL criterion on
    the same constant-L map does not refine at all."""
    p0, p = 3, 7
    base = dict(ndim=2, coarse_order=p0, max_order=p, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), shift=0)
    sp = oracle_mod.refine_spec(criterion=1, q_threshold=100.0, tau=0.05, **base)
    r = oracle_mod.refine_fn(ring_q_map, sp)
    keys, q = r["key"].astype(np.int64), r["q"]
    assert len(keys) > 64 and r["iters"] > 0
    gap = np.diff(keys)
    hot = (q[:-1] > 100.0) | (q[1:] > 100.0)
    assert not np.any(hot & (gap > 1))
    # every traced cell with Q above the threshold has both curve neighbours traced
    ks = set(int(k) for k in keys)
    for k, qq in zip(keys, q):
        if qq > 100.0:
            assert (k == keys[0] or k - 1 in ks) and (k == keys[-1] or k + 1 in ks)
    # the high-Q cells found lie on the ridge
    xy = np.array([oracle_mod.hilbert_coords(int(k), 2, p) for k in keys[q > 100.0]])
    pos = (xy + 0.5) / (1 << p) * 2 - 1
    rr = np.hypot(pos[:, 0] - 0.1, pos[:, 1] + 0.05)
    assert np.all(np.abs(rr - 0.5) < 0.03 * np.sqrt(np.log(1000.0 / 98.0)) + 1e-9)
    # threshold above the maximum: coarse samples only
    r2 = oracle_mod.refine_fn(ring_q_map, oracle_mod.refine_spec(criterion=1, q_threshold=2000.0, tau=0.05, **base))
    assert len(r2["key"]) == (1 << p0) ** 2 and r2["iters"] == 0
    # the FLL criterion ignores Q
    r3 = oracle_mod.refine_fn(ring_q_map, oracle_mod.refine_spec(criterion=0, tau=0.05, **base))
    assert len(r3["key"]) == (1 << p0) ** 2


def ramp_map(x):
    """A steep smooth front: pair differences |dL| take a continuum of values,
    so some lie close to tau."""
    r = np.hypot(x[:, 0] - 0.1, x[:, 1] + 0.05)
    return 10.0 + 100.0 * np.tanh((r - 0.45) / 0.05), 1.0 + np.tanh((r - 0.45) / 0.05)


def _noisy(fn, eps, seed):
    """fn with a deterministic per-cell error of at most eps on q (relative) and L (absolute)."""
    def g(x, keys):
        q, L = fn(x)
        u = np.array([((int(k) * 2654435761 + seed) % 1000003) / 1000003.0 for k in keys])
        return q * (1 + eps * (2 * u - 1)), L + eps * (2 * u[::-1] - 1)
    return g


@pytest.mark.parametrize("ndim", [2, 3])
def test_replay_reproduces_a_noisy_run_from_exact_values(oracle_mod, ndim):
    """The replay hook of the refinement driver: a run on values with an error
    of at most eps is reproduced exactly by a run on the exact values when the
    pairs within 2 eps of tau are decided by the noisy run's sample set; without
    the band the two sets differ (the noise flips decisions), and with a zero
    band and no tie keys the replay is the plain driver."""
    if ndim == 2:
        kw = dict(ndim=2, coarse_order=3, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05)
    else:
        kw = dict(ndim=3, coarse_order=2, max_order=4, extent=(16, 16, 8), lo=(-1, -1, 0), hi=(1, 1, 1), tau=0.05)
    sp = oracle_mod.refine_spec(**kw)
    exact = lambda x, k: ramp_map(x)
    plain = oracle_mod.refine_fn(ramp_map, sp)
    r0 = oracle_mod.refine_replay(exact, sp)
    assert np.array_equal(r0["key"], plain["key"]) and r0["iters"] == plain["iters"]
    eps = 0.01
    noisy = oracle_mod.refine_replay(_noisy(ramp_map, eps, 7), sp)
    assert not np.array_equal(noisy["key"], plain["key"])
    rep = oracle_mod.refine_replay(exact, sp, noisy["key"], noisy["origin"], band_abs=2 * eps)
    assert np.array_equal(rep["key"], noisy["key"]) and np.array_equal(rep["origin"], noisy["origin"])
    # a band narrower than the error leaves decisions that only the noise explains
    narrow = oracle_mod.refine_replay(exact, sp, noisy["key"], noisy["origin"], band_abs=0.2 * eps)
    assert not np.array_equal(narrow["key"], noisy["key"])


def test_replay_q_threshold_band(oracle_mod):
    """Same for the Q-threshold criterion with a relative band on Q."""
    kw = dict(ndim=2, coarse_order=3, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05,
              criterion=1, q_threshold=60.0)
    sp = oracle_mod.refine_spec(**kw)
    exact = lambda x, k: ramp_map(x)
    plain = oracle_mod.refine_fn(ramp_map, sp)
    assert len(plain["key"]) > 64 * 1.5
    eps = 0.02
    noisy = oracle_mod.refine_replay(_noisy(ramp_map, eps, 3), sp)
    assert not np.array_equal(noisy["key"], plain["key"])
    rep = oracle_mod.refine_replay(exact, sp, noisy["key"], noisy["origin"], band_rel=1.01 * eps / (1 - eps))
    assert np.array_equal(rep["key"], noisy["key"])
    narrow = oracle_mod.refine_replay(exact, sp, noisy["key"], noisy["origin"], band_rel=0.1 * eps)
    assert not np.array_equal(narrow["key"], noisy["key"])


def test_replay_unsure_samples_follow_the_other_run(oracle_mod):
    """A pair with a sample the evaluator marks as undetermined is decided by
    the other run: values that differ arbitrarily at such samples (a line on a
    separatrix, whose length depends on the integration) still replay."""
    kw = dict(ndim=2, coarse_order=3, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05)
    sp = oracle_mod.refine_spec(**kw)
    odd = lambda k: np.array([(int(v) * 7919) % 13 == 0 for v in k])

    def jumpy(x, k):
        q, L = ramp_map(x)
        return q, np.where(odd(k), L + 0.3, L)

    other = oracle_mod.refine_replay(jumpy, sp)
    plain = oracle_mod.refine_replay(lambda x, k: ramp_map(x), sp)
    assert not np.array_equal(other["key"], plain["key"])
    rep = oracle_mod.refine_replay(lambda x, k: ramp_map(x) + (odd(k),), sp, other["key"], other["origin"])
    assert np.array_equal(rep["key"], other["key"]) and np.array_equal(rep["origin"], other["origin"])


def test_pass_decisions_use_lengths_only_traces(oracle_mod):
    """pass_stepper 0 (the default): the FLL-jump decisions on samples added by
    the passes compare lengths from a lengths-only Cash-Karp trace with the
    step cap pass_h_max, the coarse samples' decisions their own lengths, and
    the stored values are those of the run's options. The driver run that way
    equals the replay whose evaluator returns exactly those lengths, batch by
    batch; it differs from pass_stepper 2 (decisions on the stored lengths),
    and its stored lengths are the run's own traces of its keys."""
    import torch
    from paper_1609_00724_gb300 import inputs
    gf = inputs.charge_field(inputs.random_charges(4, 2), 24, dtype=torch.float32)
    g = inputs.to_numpy64(gf)
    F = oracle_mod.Field(g.bx, g.by, g.bz, g.xc, g.yc, g.zc, mode=0)
    tol, h_max = 1e-4, 8.0
    o = oracle_mod.default_opts(tol_abs=tol, tol_rel=tol)
    od = oracle_mod.default_opts(tol_abs=tol, tol_rel=tol, length_only=1, h_max=h_max)
    kw = dict(ndim=2, coarse_order=3, max_order=7, center=(0, 0, 0), u=(2, 0, 0), v=(0, 2, 0), tau=0.05)
    r0 = oracle_mod.refine(F, oracle_mod.refine_spec(pass_h_max=h_max, **kw), o)
    r2 = oracle_mod.refine(F, oracle_mod.refine_spec(pass_stepper=2, **kw), o)
    batches = []

    def decision_lengths(x, k):
        r = oracle_mod.trace_seeds(F, x, o)
        L = r["L"] if not batches else oracle_mod.trace_seeds(F, x, od)["L"]
        batches.append(len(k))
        return r["q_perp"], L

    rep = oracle_mod.refine_replay(decision_lengths, oracle_mod.refine_spec(**kw))
    assert np.array_equal(rep["key"], r0["key"]) and np.array_equal(rep["origin"], r0["origin"])
    assert batches[0] == 64 and len(batches) > 4
    assert len(np.setxor1d(r0["key"], r2["key"])) > 20
    c = np.array([oracle_mod.hilbert_coords(k, 2, 7) for k in r0["key"]], dtype=np.float64)
    x = np.column_stack([(c[:, 0] + 0.5) / 128 * 2 - 1, (c[:, 1] + 0.5) / 128 * 2 - 1, np.zeros(len(c))])
    assert np.array_equal(r0["L"], oracle_mod.trace_seeds(F, x, o)["L"])
