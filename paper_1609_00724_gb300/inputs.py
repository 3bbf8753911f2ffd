"""Seeded synthetic inputs: magnetic fields sampled on grids, and seed sets.

This module holds none of the QSL method's arithmetic. It only produces the
inputs that the CUDA library and the FP64 oracle both consume:

* the linear hyperbolic field B = (lam x, -lam y, B0) (its squashing factor has
  a closed form), sampled on a uniform grid;
* potential fields of sub-photospheric point charges, B = sum_i q_i (x - x_i) /
  |x - x_i|^3, evaluated in FP64 at the grid vertices and then cast;
* the same charge fields on a spherical wedge (axes longitude, latitude,
  radius; components along the local unit vectors), for spherical geometry;
* random seed points.

The paper's own workloads (the Titov-Demoulin flux rope and an NLFFF model of
SOL2010-04-08) are not available; these fields stand in for them.
Random numbers come from numpy's PCG64 with the stated seed.
"""
from dataclasses import dataclass

import numpy as np
import torch

BOX = ((-1.0, 1.0), (-1.0, 1.0), (0.0, 1.0))


@dataclass
class GridField:
    bx: object  # [nz, ny, nx] arrays (numpy or torch), x fastest
    by: object
    bz: object
    xc: np.ndarray  # vertex coordinates per axis (float64)
    yc: np.ndarray
    zc: np.ndarray

    @property
    def shape(self):
        return (len(self.xc), len(self.yc), len(self.zc))


def axes(n, box=BOX):
    """Uniform vertex coordinates with the box ends as first and last vertex."""
    if isinstance(n, int):
        n = (n, n, n)
    return tuple(np.linspace(box[a][0], box[a][1], n[a]) for a in range(3))


def hyperbolic_field(n=64, lam=3.0, b0=1.0, box=BOX, dtype=np.float64):
    """B = (lam x, -lam y, b0) sampled at the vertices (numpy arrays)."""
    xc, yc, zc = axes(n, box)
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    bx = (lam * X).astype(dtype)
    by = (-lam * Y).astype(dtype)
    bz = np.full_like(X, b0).astype(dtype)
    return GridField(bx, by, bz, xc, yc, zc)


@dataclass
class Charges:
    pos: np.ndarray  # (k, 3)
    q: np.ndarray    # (k,)


def random_charges(count, seed, strength=(0.5, 1.5), depth=(0.05, 0.2), xy=(-0.5, 0.5)):
    """`count` charges below z = 0 with alternating signs (+, -, +, ...),
    |q| ~ U(strength), depth ~ U(depth), (x, y) ~ U(xy)^2."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xy_ = rng.uniform(xy[0], xy[1], size=(count, 2))
    d = rng.uniform(depth[0], depth[1], size=count)
    mag = rng.uniform(strength[0], strength[1], size=count)
    sign = np.where(np.arange(count) % 2 == 0, 1.0, -1.0)
    pos = np.column_stack([xy_, -d])
    return Charges(pos=pos, q=sign * mag)


def charge_field(charges, n, box=BOX, dtype=torch.float32, device="cpu", slab=16):
    """Potential field of point charges at the grid vertices: evaluated in
    float64 (torch, on `device`), returned as torch tensors of `dtype`."""
    xc, yc, zc = axes(n, box)
    dev = torch.device(device)
    X = torch.as_tensor(xc, dtype=torch.float64, device=dev)
    Y = torch.as_tensor(yc, dtype=torch.float64, device=dev)
    Zs = torch.as_tensor(zc, dtype=torch.float64, device=dev)
    nx, ny, nz = len(xc), len(yc), len(zc)
    out = [torch.empty((nz, ny, nx), dtype=dtype, device=dev) for _ in range(3)]
    pos = torch.as_tensor(charges.pos, dtype=torch.float64, device=dev)
    q = torch.as_tensor(charges.q, dtype=torch.float64, device=dev)
    for z0 in range(0, nz, slab):
        Z = Zs[z0:z0 + slab]
        zz, yy, xx = torch.meshgrid(Z, Y, X, indexing="ij")
        acc = [torch.zeros_like(xx) for _ in range(3)]
        for i in range(pos.shape[0]):
            dx, dy, dz = xx - pos[i, 0], yy - pos[i, 1], zz - pos[i, 2]
            r2 = dx * dx + dy * dy + dz * dz
            w = q[i] / (r2 * torch.sqrt(r2))
            acc[0] += w * dx
            acc[1] += w * dy
            acc[2] += w * dz
        for a in range(3):
            out[a][z0:z0 + slab] = acc[a].to(dtype)
    return GridField(out[0], out[1], out[2], xc, yc, zc)


WEDGE = ((-0.4, 0.4), (-0.3, 0.3), (1.0, 1.5))  # longitude, latitude (radians), radius


def random_wedge_charges(count, seed, wedge=WEDGE, strength=(0.5, 1.5), depth=(0.03, 0.1)):
    """`count` charges below the wedge's inner sphere, alternating signs,
    |q| ~ U(strength), depth below r = wedge inner radius ~ U(depth), longitude
    and latitude ~ U over the inner half of the wedge; Cartesian positions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ph = rng.uniform(0.5 * wedge[0][0], 0.5 * wedge[0][1], size=count)
    th = rng.uniform(0.5 * wedge[1][0], 0.5 * wedge[1][1], size=count)
    rr = wedge[2][0] - rng.uniform(depth[0], depth[1], size=count)
    mag = rng.uniform(strength[0], strength[1], size=count)
    sign = np.where(np.arange(count) % 2 == 0, 1.0, -1.0)
    pos = np.column_stack([rr * np.cos(th) * np.cos(ph), rr * np.cos(th) * np.sin(ph), rr * np.sin(th)])
    return Charges(pos=pos, q=sign * mag)


def spherical_charge_field(charges, n, wedge=WEDGE, dtype=torch.float32, device="cpu", slab=16):
    """Potential field of Cartesian point charges on a spherical wedge grid:
    n = (n_phi, n_theta, n_r) uniform vertices over `wedge`; the field at each
    vertex is evaluated in FP64 and returned as its components along the local
    unit vectors (phi^, theta^, r^), as torch tensors [n_r, n_theta, n_phi] of
    `dtype`; the GridField's axes are the longitudes, latitudes and radii."""
    ax = [np.linspace(lo, hi, k) for (lo, hi), k in zip(wedge, n)]
    dev = torch.device(device)
    P = torch.as_tensor(ax[0], dtype=torch.float64, device=dev)
    T = torch.as_tensor(ax[1], dtype=torch.float64, device=dev)
    Rs = torch.as_tensor(ax[2], dtype=torch.float64, device=dev)
    out = [torch.empty((n[2], n[1], n[0]), dtype=dtype, device=dev) for _ in range(3)]
    pos = torch.as_tensor(charges.pos, dtype=torch.float64, device=dev)
    q = torch.as_tensor(charges.q, dtype=torch.float64, device=dev)
    for r0 in range(0, n[2], slab):
        rr, tt, pp = torch.meshgrid(Rs[r0:r0 + slab], T, P, indexing="ij")
        ct, st, cp, sp = torch.cos(tt), torch.sin(tt), torch.cos(pp), torch.sin(pp)
        x, y, z = rr * ct * cp, rr * ct * sp, rr * st
        acc = [torch.zeros_like(x) for _ in range(3)]
        for i in range(pos.shape[0]):
            dx, dy, dz = x - pos[i, 0], y - pos[i, 1], z - pos[i, 2]
            d2 = dx * dx + dy * dy + dz * dz
            w = q[i] / (d2 * torch.sqrt(d2))
            acc[0] += w * dx
            acc[1] += w * dy
            acc[2] += w * dz
        bx, by, bz = acc
        b_phi = -sp * bx + cp * by
        b_th = -st * cp * bx - st * sp * by + ct * bz
        b_r = ct * cp * bx + ct * sp * by + st * bz
        for a, v in enumerate((b_phi, b_th, b_r)):
            out[a][r0:r0 + slab] = v.to(dtype)
    return GridField(out[0], out[1], out[2], ax[0], ax[1], ax[2])


def to_numpy64(gf):
    """Same field as float64 numpy arrays (for the oracle)."""
    def cvt(a):
        if isinstance(a, torch.Tensor):
            return a.detach().to("cpu", torch.float64).numpy()
        return np.asarray(a, dtype=np.float64)
    return GridField(cvt(gf.bx), cvt(gf.by), cvt(gf.bz), gf.xc, gf.yc, gf.zc)


def random_seeds(count, seed, box=BOX, margin=0.0):
    """Uniform random points inside the box (shrunk by `margin` on each side)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.array([b[0] + margin for b in box])
    hi = np.array([b[1] - margin for b in box])
    return lo + rng.uniform(size=(count, 3)) * (hi - lo)


def subsample(n, count, seed):
    """Sorted random subset of range(n) of size min(count, n)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = min(count, n)
    return np.sort(rng.choice(n, size=count, replace=False))


def batch64_specs(seed=4, count=64):
    """The 64-field batch workload: (grid edge n, cut edge m, field seed) per
    field, n ~ U{64..256} and m ~ U{256..1024} drawn in turn from one PCG64
    stream with `seed`; field i's charges use seed 1000 * seed + i."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(rng.integers(64, 257))
        m = int(rng.integers(256, 1025))
        out.append((n, m, 1000 * seed + i))
    return out
