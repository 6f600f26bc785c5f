"""Seeded synthetic inputs: volumes of Gaussian tubes plus noise.

The paper shows its transform on artificial crossing tubes (Fig. 5) and on
vessel data (Figs. 6-7) that are not published; these generators stand in
for both. They hold none of the transform's arithmetic and serve the tests,
the benchmark and the oracle alike.

A tube contributes exp(-d^2 / (2 sigma^2)), d the distance to its centre
line; the volume is the sum over tubes plus i.i.d. Gaussian noise. Centre
lines are straight lines or Catmull-Rom cubics through four control points;
every second spline reuses a control point of the one before, so the tubes
cross.
"""
from __future__ import annotations

import numpy as np


def _splat(vol, pts, sigma):
    """vol += exp(-d^2/2 sigma^2), d = distance to the closest of ``pts``."""
    shape = np.array(vol.shape)
    r = int(np.ceil(3.5 * sigma))
    tube = np.zeros_like(vol)
    for p in pts:
        lo = np.maximum(np.floor(p).astype(int) - r, 0)
        hi = np.minimum(np.floor(p).astype(int) + r + 2, shape)
        if np.any(hi <= lo):
            continue
        z = np.arange(lo[0], hi[0])[:, None, None] - p[0]
        y = np.arange(lo[1], hi[1])[None, :, None] - p[1]
        x = np.arange(lo[2], hi[2])[None, None, :] - p[2]
        g = np.exp(-(z * z + y * y + x * x) / (2.0 * sigma * sigma))
        sl = tuple(slice(a, b) for a, b in zip(lo, hi))
        np.maximum(tube[sl], g, out=tube[sl])
    vol += tube


def _polyline(a, b, step=0.5):
    n = max(2, int(np.ceil(np.linalg.norm(b - a) / step)) + 1)
    s = np.linspace(0.0, 1.0, n)[:, None]
    return a[None, :] * (1 - s) + b[None, :] * s


def _catmull_rom(ctrl, step=0.5):
    """Uniform Catmull-Rom curve through the 4 control points (end points
    duplicated), sampled about every ``step`` voxels."""
    P = np.concatenate([ctrl[:1], ctrl, ctrl[-1:]], axis=0)
    out = []
    for i in range(1, len(P) - 2):
        p0, p1, p2, p3 = P[i - 1], P[i], P[i + 1], P[i + 2]
        n = max(4, int(np.ceil(2.0 * np.linalg.norm(p2 - p1) / step)))
        t = np.linspace(0.0, 1.0, n, endpoint=False)[:, None]
        out.append(0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t ** 2
                          + (-p0 + 3 * p1 - 3 * p2 + p3) * t ** 3))
    out.append(P[-2][None, :])
    return np.concatenate(out, axis=0)


def straight_tubes(shape, n_tubes=3, seed=0, sigma=(1.5, 3.0), noise=0.1):
    """Straight tubes through the centre (+-2 voxels), random directions."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    vol = np.zeros(shape, dtype=np.float64)
    c = (np.array(shape, dtype=np.float64) - 1.0) / 2.0
    span = float(np.linalg.norm(shape))
    for _ in range(n_tubes):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        o = c + rng.uniform(-2.0, 2.0, 3)
        s = rng.uniform(*sigma)
        _splat(vol, _polyline(o - span * d, o + span * d), s)
    vol += rng.normal(0.0, noise, shape)
    return vol.astype(np.float32)


def spline_tubes(shape, n_tubes=12, seed=0, radius=(1.0, 4.0), noise=0.2):
    """Catmull-Rom tubes through control points in [0.1 n, 0.9 n]^3."""
    rng = np.random.default_rng(seed)
    shape = tuple(int(s) for s in shape)
    vol = np.zeros(shape, dtype=np.float64)
    lo = 0.1 * np.array(shape, dtype=np.float64)
    hi = 0.9 * np.array(shape, dtype=np.float64)
    prev = None
    for t in range(n_tubes):
        ctrl = rng.uniform(lo, hi, size=(4, 3))
        if t % 2 == 1 and prev is not None:
            ctrl[rng.integers(1, 3)] = prev[rng.integers(1, 3)]
        prev = ctrl
        _splat(vol, _catmull_rom(ctrl), rng.uniform(*radius))
    vol += rng.normal(0.0, noise, shape)
    return vol.astype(np.float32)


def score_weights(shape, seed=1):
    """w ~ U(0, 1) of the differentiation workload's loss sum w |U|^2."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, shape).astype(np.float32)


# Named workloads: (volume generator kwargs, orientation subdivisions, L)
WORKLOADS = {
    "tubes32_no42": dict(shape=(32, 32, 32), kind="straight", n_tubes=3, noise=0.1,
                         subdiv=1, L=12),
    "splines128_no162": dict(shape=(128, 128, 128), kind="spline", n_tubes=12, noise=0.2,
                             subdiv=2, L=16),
    "splines128_no42": dict(shape=(128, 128, 128), kind="spline", n_tubes=12, noise=0.2,
                            subdiv=1, L=16),
    "splines256_no42": dict(shape=(256, 256, 256), kind="spline", n_tubes=40, noise=0.2,
                            subdiv=1, L=20),
    "splines96x8_no42": dict(shape=(96, 96, 96), kind="spline", n_tubes=12, noise=0.2,
                             subdiv=1, L=16, batch=8),
}


def workload_volume(name, seed=0, batch_index=0):
    w = WORKLOADS[name]
    if w["kind"] == "straight":
        return straight_tubes(w["shape"], w["n_tubes"], seed + batch_index, noise=w["noise"])
    return spline_tubes(w["shape"], w["n_tubes"], seed + batch_index, noise=w["noise"])
