"""Seeded synthetic inputs for the dynamic-OT solver.

This module only draws and samples densities and obstacle masks; it holds none
of the method's arithmetic (no operators, no c vector, no solve).  Both the CUDA
path and the CPU oracle are fed from it, each doing its own set-up from the raw
density samples it returns.

Recipes (densities are sampled at cell centres (i + 1/2)/N of [0, 1]^D):
  gaussian_pair   isotropic Gaussian pdfs at mu0, mu1 with a constant floor
  mixture         1..5 pdf-normalised Gaussians, means U[0.15, 0.85]^D, sigma
                  U[0.03, 0.12] (isotropic) or U[0.05, 0.15]^D (anisotropic),
                  Dirichlet(1) weights; pdf values below `cut` set to exactly 0,
                  or a constant `floor` added
  rect_mask       union of 3..6 axis-aligned rectangles covering 8-12% of cells
  product_pair    separable (f(x) + eps)(f(y) + eps) densities whose W2^2 is the
                  sum of the 1D values (closed-form check)
  paper_example   the analytic 2D examples Ex-1 .. Ex-4 of Sec. 5 (Gaussians at
                  0.25 / 0.75, a Laplace-type bump, a quartic), each normalised
                  to unit mass on [0, 1]^2 and raised by the uniform floor delta
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class GridSpec:
    """D spatial axes with N cells each, T time intervals."""
    D: int
    T: int
    N: int

    @property
    def shape(self):
        return (self.N,) * self.D


# The four grid workloads, named by what they are.
GAUSS32 = GridSpec(2, 16, 32)        # 2D 32^2 x 16, two Gaussians + floor 1e-3
MIX256 = GridSpec(2, 64, 256)        # 2D 256^2 x 64, Gaussian mixtures with exact zeros
OBST128 = GridSpec(2, 32, 128)       # 2D 128^2 x 32, mixtures + rectangle obstacles
MIX3D64 = GridSpec(3, 32, 64)        # 3D 64^3 x 32, anisotropic mixtures + floor 1e-4
MIX1024 = GridSpec(2, 32, 1024)      # 2D 1024^2 x 32, mixtures as MIX256 (the scalability case)
EX128 = GridSpec(2, 32, 128)         # the paper's Ex-1 .. Ex-4 grid (n_0, n_1, n_2) = (32, 128, 128)


def cell_centres(N: int, D: int):
    x = (np.arange(N) + 0.5) / N
    return np.meshgrid(*([x] * D), indexing="ij")


def gaussian_pdf(X, mu, sig):
    """Product of 1D normal pdfs (diagonal covariance) at points X (list of arrays)."""
    D = len(X)
    sig = np.broadcast_to(np.asarray(sig, dtype=np.float64), (D,))
    out = np.ones_like(X[0])
    for d in range(D):
        out = out * np.exp(-0.5 * ((X[d] - mu[d]) / sig[d]) ** 2) / (np.sqrt(2 * np.pi) * sig[d])
    return out


def gaussian_pair(N=32, D=2, mu0=(0.3, 0.3), mu1=(0.7, 0.7), sig=0.1, floor=1e-3):
    """Two isotropic Gaussian pdfs plus a constant floor (not normalised)."""
    X = cell_centres(N, D)
    r0 = gaussian_pdf(X, mu0[:D], sig) + floor
    r1 = gaussian_pdf(X, mu1[:D], sig) + floor
    return r0, r1


def mixture(rng: np.random.Generator, N: int, D: int, kmin=1, kmax=5, sig_lo=0.03, sig_hi=0.12,
            anisotropic=False, cut=None, floor=None):
    """One Gaussian-mixture density sample (pdf units, not normalised)."""
    X = cell_centres(N, D)
    K = int(rng.integers(kmin, kmax + 1))
    w = rng.dirichlet(np.ones(K))
    out = np.zeros_like(X[0])
    for j in range(K):
        mu = rng.uniform(0.15, 0.85, size=D)
        sig = rng.uniform(sig_lo, sig_hi, size=D if anisotropic else 1)
        out += w[j] * gaussian_pdf(X, mu, sig)
    if cut is not None:
        out = np.where(out < cut, 0.0, out)
    if floor is not None:
        out = out + floor
    return out


def rect_mask(rng: np.random.Generator, N: int, D: int = 2, lo=0.08, hi=0.12, max_tries=1000):
    """Union of 3..6 axis-aligned rectangles covering a fraction in [lo, hi] of cells."""
    for _ in range(max_tries):
        m = np.zeros((N,) * D, dtype=bool)
        for _r in range(int(rng.integers(3, 7))):
            a = rng.integers(0, N, size=(2, D))
            lo_c, hi_c = a.min(axis=0), a.max(axis=0) + 1
            sl = tuple(slice(int(lo_c[d]), int(hi_c[d])) for d in range(D))
            m[sl] = True
        cov = m.mean()
        if lo <= cov <= hi:
            return m
    raise RuntimeError("could not draw an obstacle mask in the coverage window")


def mixture_pair(spec: GridSpec, seed: int, obstacles: bool = False):
    """(rho0, rho1, mask) for the Gaussian-mixture workloads.

    2D: 1..5 isotropic components, sigma U[0.03, 0.12], pdf < 1e-4 -> 0.
    3D: 2..4 anisotropic components, sigma U[0.05, 0.15]^3, floor 1e-4 added.
    obstacles=True draws a rectangle mask and zeros both densities on it."""
    rng = np.random.default_rng(seed)
    if spec.D == 3:
        kw = dict(kmin=2, kmax=4, sig_lo=0.05, sig_hi=0.15, anisotropic=True, floor=1e-4)
    else:
        kw = dict(kmin=1, kmax=5, sig_lo=0.03, sig_hi=0.12, cut=1e-4)
    mask = rect_mask(rng, spec.N, spec.D) if obstacles else None
    while True:
        r0 = mixture(rng, spec.N, spec.D, **kw)
        r1 = mixture(rng, spec.N, spec.D, **kw)
        if mask is not None:
            r0 = np.where(mask, 0.0, r0)
            r1 = np.where(mask, 0.0, r1)
        if r0.sum() > 0 and r1.sum() > 0:
            return r0, r1, mask


def product_pair(N: int, mu0=(0.35, 0.4), mu1=(0.65, 0.55), sig=(0.08, 0.1), eps=0.05):
    """2D densities (f0(x)+eps)(g0(y)+eps) -> (f1(x)+eps)(g1(y)+eps) with 1D Gaussian pdfs.

    Returns (rho0, rho1, (f0, g0, f1, g1)) with the 1D factors on the cell centres."""
    x = (np.arange(N) + 0.5) / N
    def g1d(m, s):
        return np.exp(-0.5 * ((x - m) / s) ** 2) / (np.sqrt(2 * np.pi) * s) + eps
    f0, g0 = g1d(mu0[0], sig[0]), g1d(mu0[1], sig[1])
    f1, g1 = g1d(mu1[0], sig[0]), g1d(mu1[1], sig[1])
    return np.outer(f0, g0), np.outer(f1, g1), (f0, g0, f1, g1)


def paper_example(k: int, N: int, delta: float = 0.0):
    """(rho0, rho1) of Ex-k, k = 1..4 (Sec. 5): the functions the examples define,
    sampled at the cell centres of an N x N grid, each scaled to unit mass on the
    unit square (mean 1) and raised by delta."""
    x = (np.arange(N) + 0.5) / N
    X1, X2 = np.meshgrid(x, x, indexing="ij")
    m1, m2 = 0.25, 0.75

    def gauss(a, b, chi):
        return np.exp((-(X1 - a) ** 2 - (X2 - b) ** 2) / (2.0 * chi ** 2))

    def four(chi):
        return gauss(m1, m1, chi) + gauss(m1, m2, chi) + gauss(m2, m1, chi) + gauss(m2, m2, chi)

    if k == 1:
        chi = np.sqrt(0.05)
        v0, v1 = gauss(m1, m2, chi), gauss(m2, m1, chi)
    elif k == 2:
        v0, v1 = gauss(m1, m1, 0.1), four(0.05)
    elif k == 3:
        v0, v1 = np.exp(-3.0 * np.abs(X1 - m1) - 5.0 * np.abs(X2 - m1)), four(0.05)
    elif k == 4:
        v0, v1 = (X1 - 0.5) ** 4 + (X2 - 0.5) ** 4, four(0.05)
    else:
        raise ValueError("k must be 1..4")
    return (v0 / v0.mean() + delta).ravel(), (v1 / v1.mean() + delta).ravel()


def workload(name: str, seed: int | None = None):
    """(spec, rho0, rho1, mask) for a named workload with its default seed."""
    if name == "gauss32":
        r0, r1 = gaussian_pair(32, 2)
        return GAUSS32, r0, r1, None
    if name == "mix256":
        r0, r1, m = mixture_pair(MIX256, 1002 if seed is None else seed)
        return MIX256, r0, r1, m
    if name == "obst128":
        r0, r1, m = mixture_pair(OBST128, 1003 if seed is None else seed, obstacles=True)
        return OBST128, r0, r1, m
    if name == "mix1024":
        r0, r1, m = mixture_pair(MIX1024, 1005 if seed is None else seed)
        return MIX1024, r0, r1, m
    if name == "mix3d64":
        r0, r1, m = mixture_pair(MIX3D64, 1004 if seed is None else seed)
        return MIX3D64, r0, r1, m
    if name in ("ex1", "ex2", "ex3", "ex4"):
        r0, r1 = paper_example(int(name[2]), EX128.N)
        return EX128, r0, r1, None
    raise KeyError(name)
