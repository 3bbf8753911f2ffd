"""Checks of the seeded input generators that feed both the CUDA path and
the oracle (they hold none of the method's arithmetic)."""
import numpy as np
import torch

from paper_1609_00724_gb300 import inputs


def test_spherical_wedge_field_components():
    """The wedge field's components are the Cartesian charge field along the
    local unit vectors of (longitude, latitude, radius): checked at random
    vertices against unit vectors taken from central differences of the
    coordinate map x(phi, theta, r) = r (cos th cos ph, cos th sin ph, sin th),
    and a direct Coulomb sum."""
    ch = inputs.random_wedge_charges(5, 11)
    n = (17, 13, 9)
    gf = inputs.spherical_charge_field(ch, n, dtype=torch.float64)
    bp, bt, br = (a.numpy() for a in (gf.bx, gf.by, gf.bz))
    rng = np.random.default_rng(3)

    def xyz(p, t, r):
        return r * np.array([np.cos(t) * np.cos(p), np.cos(t) * np.sin(p), np.sin(t)])

    for _ in range(20):
        i, j, k = rng.integers(0, n[0]), rng.integers(0, n[1]), rng.integers(0, n[2])
        p, t, r = gf.xc[i], gf.yc[j], gf.zc[k]
        x = xyz(p, t, r)
        d = x[None, :] - ch.pos
        B = (ch.q[:, None] * d / np.linalg.norm(d, axis=1)[:, None] ** 3).sum(axis=0)
        e = 1e-6
        units = []
        for a in range(3):
            lo, hi = [p, t, r], [p, t, r]
            lo[a] -= e
            hi[a] += e
            g = (xyz(*hi) - xyz(*lo)) / (2 * e)
            units.append(g / np.linalg.norm(g))
        want = [float(B @ u) for u in units]
        got = [bp[k, j, i], bt[k, j, i], br[k, j, i]]
        assert np.allclose(got, want, rtol=1e-7, atol=1e-9 * np.linalg.norm(B)), (got, want)


def test_wedge_charges_lie_below_the_inner_sphere():
    ch = inputs.random_wedge_charges(40, 5)
    rr = np.linalg.norm(ch.pos, axis=1)
    assert np.all(rr < inputs.WEDGE[2][0]) and np.all(rr > inputs.WEDGE[2][0] - 0.11)
    assert np.all(np.sign(ch.q) == np.where(np.arange(40) % 2 == 0, 1, -1))
