"""Seeded synthetic inputs for PINS (optimal transport) workloads.

This module only draws inputs: point clouds, grid histograms, cost matrices and
marginals. It holds none of the solver's arithmetic, so both the FP64 CPU oracle
and the CUDA path can be fed from it without sharing any of the method.

Seeds follow one rule everywhere: ``20250205 + 1000 * family + instance`` with
NumPy's PCG64.

Families (sizes and distributions follow the paper's workloads, Section 5):

* ``family 0`` random assignment (Section 5.1.1): ``c_ij ~ U[0,1]``, ``a = b = 1/n``.
* ``family 1`` small points: m = n = 64, x, y iid U[0,1]^2, C = |x-y|^2 / max,
  a, b iid U(0.5, 1.5) normalised, eta = 1e-2.
* ``family 2`` dense Gaussian-mixture instance: 8 components (means U[0,1]^2,
  sigma 0.05, equal weights), x and y drawn independently, a, b ~ Dirichlet(1).
* ``family 3`` grid histograms on an s x s grid: sum of 5-20 Gaussian bumps
  (centre U[0,s)^2, width U[0.02,0.15]*s, amplitude U[0.5,1.5]) plus a 1e-6 floor,
  normalised; squared grid distance scaled by 1/(2 (s-1)^2).  Stands in for the
  DOTmark classes of Section 5.2, which are not available here.
* ``family 4`` stroke histograms: 1-3 thick polylines of 2-5 vertices rasterised
  at intensity 1.0 plus U(0, 1e-3) noise, shifted or rotated by up to 2 px, on
  grids s in {16, 28, 32, 48, 64}.  Stands in for the augmented-MNIST tiles of
  Section 5.1.1, which are not available here.
* ``family 5`` serving requests: n = round(exp U[ln 256, ln 16384]), m = n,
  Gaussian-mixture points as family 2 (fresh means per request), Dirichlet(1).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

BASE_SEED = 20250205


def rng_for(family: int, instance: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + 1000 * family + instance))


@dataclasses.dataclass
class Problem:
    """One OT instance.  ``kind`` is 'dense', 'points' or 'grid'.

    dense : C (m x n, row-major float64)
    points: x (m x d), y (n x d); C_ij = cost_scale * |x_i - y_j|^2
    grid  : source and target live on an s1 x s2 grid (m = n = s1 * s2), pixel
            i = i1 * s2 + i2; C_ij = cost_scale * ((i1-j1)^2 + (i2-j2)^2)
    """
    kind: str
    a: np.ndarray
    b: np.ndarray
    eta: float
    C: Optional[np.ndarray] = None
    x: Optional[np.ndarray] = None
    y: Optional[np.ndarray] = None
    cost_scale: float = 1.0
    grid: tuple = (0, 0)
    tol_marg: float = 1e-9
    name: str = ""

    @property
    def m(self) -> int:
        return int(self.a.shape[0])

    @property
    def n(self) -> int:
        return int(self.b.shape[0])

    def dense_cost(self) -> np.ndarray:
        """Materialise C (m x n float64).  For points and grids this is the
        definition of the streamed cost written out densely."""
        if self.kind == "dense":
            return self.C
        if self.kind == "points":
            diff = self.x[:, None, :] - self.y[None, :, :]
            return self.cost_scale * np.sum(diff * diff, axis=2)
        if self.kind == "grid":
            s1, s2 = self.grid
            idx = np.arange(s1 * s2)
            i1, i2 = idx // s2, idx % s2
            d1 = (i1[:, None] - i1[None, :]).astype(np.float64)
            d2 = (i2[:, None] - i2[None, :]).astype(np.float64)
            return self.cost_scale * (d1 * d1 + d2 * d2)
        raise ValueError(self.kind)


def _normalise(w: np.ndarray) -> np.ndarray:
    w = np.asarray(w, dtype=np.float64)
    return w / w.sum()


def max_sq_dist(x: np.ndarray, y: np.ndarray) -> float:
    """Exact max_ij |x_i - y_j|^2.  For a fixed x_i the farthest y_j is a vertex
    of the convex hull of y, so only hull vertices are scanned."""
    yy = y
    if y.shape[0] > 16 and y.shape[1] == 2:
        from scipy.spatial import ConvexHull
        yy = y[ConvexHull(y).vertices]
    best = 0.0
    for s in range(0, x.shape[0], 4096):
        d = x[s:s + 4096, None, :] - yy[None, :, :]
        best = max(best, float(np.max(np.sum(d * d, axis=2))))
    return best


def random_assignment(n: int, instance: int = 0, eta: float = 1e-2) -> Problem:
    """Section 5.1.1 synthetic family: c_ij ~ U[0,1], a = b = 1/n."""
    rng = rng_for(0, instance)
    C = rng.uniform(0.0, 1.0, size=(n, n))
    a = np.full(n, 1.0 / n)
    return Problem("dense", a, a.copy(), eta, C=C, name=f"assign-n{n}-i{instance}")


def small_points(instance: int = 0, m: int = 64, n: int = 64, eta: float = 1e-2,
                 tol_marg: float = 1e-10, as_dense: bool = True) -> Problem:
    """m = n = 64 uniform points in [0,1]^2, C normalised to max 1."""
    rng = rng_for(1, instance)
    x = rng.uniform(0.0, 1.0, size=(m, 2))
    y = rng.uniform(0.0, 1.0, size=(n, 2))
    a = _normalise(rng.uniform(0.5, 1.5, size=m))
    b = _normalise(rng.uniform(0.5, 1.5, size=n))
    scale = 1.0 / max_sq_dist(x, y)
    p = Problem("points", a, b, eta, x=x, y=y, cost_scale=scale, tol_marg=tol_marg,
                name=f"points-{m}x{n}-i{instance}")
    if as_dense:
        p = Problem("dense", a, b, eta, C=p.dense_cost(), x=x, y=y, cost_scale=scale,
                    tol_marg=tol_marg, name=p.name)
    return p


def gmm_points(rng: np.random.Generator, count: int, means: np.ndarray,
               sigma: float = 0.05) -> np.ndarray:
    comp = rng.integers(0, means.shape[0], size=count)
    return means[comp] + sigma * rng.standard_normal(size=(count, 2))


def gmm_instance(instance: int = 0, m: int = 4096, n: int = 4096, eta: float = 1e-2,
                 tol_marg: float = 1e-9, as_dense: bool = True, family: int = 2) -> Problem:
    """8-component 2-D Gaussian mixture (means U[0,1]^2, sigma 0.05); x and y are
    independent draws; a, b ~ Dirichlet(1); squared-Euclidean cost scaled to max 1."""
    rng = rng_for(family, instance)
    means = rng.uniform(0.0, 1.0, size=(8, 2))
    x = gmm_points(rng, m, means)
    y = gmm_points(rng, n, means)
    a = rng.dirichlet(np.ones(m))
    b = rng.dirichlet(np.ones(n))
    scale = 1.0 / max_sq_dist(x, y)
    p = Problem("points", a, b, eta, x=x, y=y, cost_scale=scale, tol_marg=tol_marg,
                name=f"gmm-{m}x{n}-i{instance}")
    if as_dense:
        C = np.empty((m, n))
        for s in range(0, m, 1024):
            d = x[s:s + 1024, None, :] - y[None, :, :]
            C[s:s + 1024] = scale * np.sum(d * d, axis=2)
        p = Problem("dense", a, b, eta, C=C, x=x, y=y, cost_scale=scale,
                    tol_marg=tol_marg, name=p.name)
    return p


def bump_histogram(rng: np.random.Generator, s: int) -> np.ndarray:
    """Sum of 5-20 Gaussian bumps on an s x s grid plus a 1e-6 floor, normalised."""
    k = int(rng.integers(5, 21))
    ii, jj = np.meshgrid(np.arange(s, dtype=np.float64), np.arange(s, dtype=np.float64),
                         indexing="ij")
    h = np.zeros((s, s))
    for _ in range(k):
        c1, c2 = rng.uniform(0.0, s, size=2)
        w = rng.uniform(0.02, 0.15) * s
        amp = rng.uniform(0.5, 1.5)
        h += amp * np.exp(-((ii - c1) ** 2 + (jj - c2) ** 2) / (2.0 * w * w))
    h += 1e-6
    return _normalise(h.ravel())


def grid_instance(s: int, instance: int = 0, eta: float = 1e-2,
                  tol_marg: float = 1e-9) -> Problem:
    rng = rng_for(3, instance + 100 * s)
    a = bump_histogram(rng, s)
    b = bump_histogram(rng, s)
    scale = 1.0 / (2.0 * (s - 1) ** 2)
    return Problem("grid", a, b, eta, cost_scale=scale, grid=(s, s), tol_marg=tol_marg,
                   name=f"grid-{s}-i{instance}")


def _rasterise_strokes(rng: np.random.Generator, s: int) -> np.ndarray:
    img = np.zeros((s, s))
    ii, jj = np.meshgrid(np.arange(s) + 0.5, np.arange(s) + 0.5, indexing="ij")
    thick = rng.uniform(1.5, 2.5) * s / 28.0
    for _ in range(int(rng.integers(1, 4))):
        nv = int(rng.integers(2, 6))
        pts = rng.uniform(0.15 * s, 0.85 * s, size=(nv, 2))
        for p0, p1 in zip(pts[:-1], pts[1:]):
            d = p1 - p0
            L2 = float(d @ d) + 1e-12
            t = np.clip(((ii - p0[0]) * d[0] + (jj - p0[1]) * d[1]) / L2, 0.0, 1.0)
            dist2 = (ii - p0[0] - t * d[0]) ** 2 + (jj - p0[1] - t * d[1]) ** 2
            img[dist2 <= (0.5 * thick) ** 2] = 1.0
    return img


def _shift_or_rotate(rng: np.random.Generator, img: np.ndarray) -> np.ndarray:
    """Random shift (|d| <= 2 px) or rotation about the centre whose corner
    displacement is at most 2 px; bilinear resampling, zero outside."""
    s = img.shape[0]
    ii, jj = np.meshgrid(np.arange(s, dtype=np.float64), np.arange(s, dtype=np.float64),
                         indexing="ij")
    if rng.uniform() < 0.5:
        di, dj = rng.uniform(-2.0, 2.0, size=2)
        si, sj = ii - di, jj - dj
    else:
        cmax = math.sqrt(2.0) * (s - 1) / 2.0
        th = rng.uniform(-1.0, 1.0) * (2.0 / cmax)
        c0 = (s - 1) / 2.0
        si = c0 + math.cos(th) * (ii - c0) + math.sin(th) * (jj - c0)
        sj = c0 - math.sin(th) * (ii - c0) + math.cos(th) * (jj - c0)
    i0 = np.floor(si).astype(int)
    j0 = np.floor(sj).astype(int)
    fi, fj = si - i0, sj - j0
    out = np.zeros_like(img)
    for oi, wi in ((0, 1.0 - fi), (1, fi)):
        for oj, wj in ((0, 1.0 - fj), (1, fj)):
            ri, rj = i0 + oi, j0 + oj
            ok = (ri >= 0) & (ri < s) & (rj >= 0) & (rj < s)
            out[ok] += (wi * wj)[ok] * img[ri[ok], rj[ok]]
    return out


STROKE_GRIDS = (16, 28, 32, 48, 64)


def stroke_pair(instance: int, eta: float = 1e-1, tol_marg: float = 1e-9,
                s: Optional[int] = None) -> Problem:
    rng = rng_for(4, instance)
    if s is None:
        s = int(STROKE_GRIDS[int(rng.integers(0, len(STROKE_GRIDS)))])
    hs = []
    for _ in range(2):
        img = _shift_or_rotate(rng, _rasterise_strokes(rng, s))
        img = img + rng.uniform(0.0, 1e-3, size=img.shape)
        hs.append(_normalise(img.ravel()))
    scale = 1.0 / (2.0 * (s - 1) ** 2)
    return Problem("grid", hs[0], hs[1], eta, cost_scale=scale, grid=(s, s),
                   tol_marg=tol_marg, name=f"strokes-{s}-i{instance}")


def serving_request(instance: int, eta: float = 1e-2, n_min: int = 256,
                    n_max: int = 16384) -> Problem:
    rng = rng_for(5, instance)
    n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    means = rng.uniform(0.0, 1.0, size=(8, 2))
    x = gmm_points(rng, n, means)
    y = gmm_points(rng, n, means)
    a = rng.dirichlet(np.ones(n))
    b = rng.dirichlet(np.ones(n))
    scale = 1.0 / max_sq_dist(x, y)
    return Problem("points", a, b, eta, x=x, y=y, cost_scale=scale, tol_marg=1e-9,
                   name=f"req-{n}-i{instance}")


def poisson_arrivals(rate: float, count: int, instance: int = 0) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream with the given rate."""
    rng = rng_for(5, 100000 + instance)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
