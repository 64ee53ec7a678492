"""Seeded synthetic inputs shared by the oracle checks, the GPU tests and bench.py.

This module holds no arithmetic of the method: it only draws observation sites,
observation values and run parameters.  The paper's datasets (Tangle, Ethanediol;
Sec. 6.3) are not available, so these fields stand in for them with the workload
shapes the paper reports (m = 50..500 observations, 64^3..1024^3 grids, an RBF
kernel whose length scale is ~0.1 of the domain, alpha = 1e-3, beta = 6, 1600 MC
samples; Sec. 6, Table 1, Sec. 7.3).

Field recipe: y = sum of Gaussian bumps a*exp(-|x-c|^2/(2w^2)) [+ 0.3 sin(pi(x+y+z))]
+ 0.01 N(0,1), observation sites uniform in [0,1]^3.  The draw order below is part
of the recipe: X, bump centres, bump widths, bump amplitudes, noise.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SE = 0
MATERN52 = 1


@dataclass
class Workload:
    name: str
    X: np.ndarray            # (m, 3) float64 observation sites
    y: np.ndarray            # (m,) float64 observation values
    kernel: int              # SE or MATERN52
    ell: tuple               # length scale per axis
    sf2: float               # signal variance
    sn2: float               # noise variance
    n: int                   # grid points per axis on [0,1]^3
    isovalues: list          # theta values
    max_depth: int           # octree depth D (2^D >= n-1)
    extra: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.X.shape[0])


def _field(rng, m, n_bumps, amp_lo, amp_hi, sinusoid):
    X = rng.random((m, 3))
    c = rng.random((n_bumps, 3))
    w = rng.uniform(0.1, 0.3, n_bumps)
    a = rng.uniform(amp_lo, amp_hi, n_bumps)
    d2 = ((X[:, None, :] - c[None, :, :]) ** 2).sum(-1)
    y = (a[None, :] * np.exp(-d2 / (2.0 * w[None, :] ** 2))).sum(-1)
    if sinusoid:
        y = y + 0.3 * np.sin(2.0 * math.pi * X.sum(-1) / 2.0)
    y = y + 0.01 * rng.standard_normal(m)
    return X, y


def depth_for(n: int) -> int:
    """Smallest D with 2^D >= n-1 cells per axis."""
    return max(0, int(math.ceil(math.log2(max(n - 1, 1)))))


def config1() -> Workload:
    """Plain dense method, FP64: m=64, SE l=0.2, 32^3 grid, theta = median(y)."""
    rng = np.random.default_rng(0)
    X, y = _field(rng, 64, 4, 0.5, 1.5, sinusoid=False)
    return Workload("m64_se_iso0.2_grid32", X, y, SE, (0.2, 0.2, 0.2), 1.0, 1e-4, 32,
                    [float(np.median(y))], depth_for(32))


def config2() -> Workload:
    """Paper scale: m=500, anisotropic SE (0.15,0.2,0.25), 128^3 grid, 3 isovalues, D=7."""
    rng = np.random.default_rng(1)
    X, y = _field(rng, 500, 16, -1.0, 1.0, sinusoid=True)
    th = [float(np.percentile(y, q)) for q in (25, 50, 75)]
    return Workload("m500_se_ard_grid128", X, y, SE, (0.15, 0.2, 0.25), 1.0, 1e-4, 128, th, 7)


def config3() -> Workload:
    """Precision study: m=2000, Matern-5/2 l=0.1, noise 1e-6, 256^3 grid, 64^3 sub-block."""
    rng = np.random.default_rng(2)
    X, y = _field(rng, 2000, 16, -1.0, 1.0, sinusoid=True)
    return Workload("m2000_matern52_grid256", X, y, MATERN52, (0.1, 0.1, 0.1), 1.0, 1e-6, 256,
                    [float(np.median(y))], 8, extra={"subblock": (96, 160)})


def config4(count: int = 64) -> list:
    """Batching: `count` models, m log-uniform in [100,2000], iso SE l in [0.05,0.3]."""
    rng = np.random.default_rng(3)
    out = []
    for i in range(count):
        m = int(round(math.exp(rng.uniform(math.log(100), math.log(2000)))))
        ell = float(rng.uniform(0.05, 0.3))
        n = int(rng.choice([64, 128, 256]))
        sub = np.random.default_rng(1000 + i)
        X, y = _field(sub, m, 16, -1.0, 1.0, sinusoid=True)
        out.append(Workload(f"batch{i}_m{m}_grid{n}", X, y, SE, (ell, ell, ell), 1.0, 1e-4, n,
                            [float(np.median(y))], depth_for(n)))
    return out


def config5() -> Workload:
    """Differentiation: m=500, SE (0.15,0.2,0.25), 128^3, theta=median(y), weights U(0,1)."""
    rng = np.random.default_rng(4)
    X, y = _field(rng, 500, 16, -1.0, 1.0, sinusoid=True)
    w = np.random.default_rng(5).random((127, 127, 127)).reshape(-1)
    return Workload("m500_se_ard_grid128_grad", X, y, SE, (0.15, 0.2, 0.25), 1.0, 1e-4, 128,
                    [float(np.median(y))], 7, extra={"cell_weights": w})


def small(seed: int, m: int, n: int, ell=(0.2, 0.2, 0.2), kernel=SE, sn2=1e-4,
          n_bumps=4, sinusoid=False) -> Workload:
    """A small field of the config-1 family, for parity tests with several tiles."""
    rng = np.random.default_rng(seed)
    X, y = _field(rng, m, n_bumps, -1.0, 1.0, sinusoid)
    return Workload(f"small{seed}_m{m}_grid{n}", X, y, kernel, tuple(ell), 1.0, sn2, n,
                    [float(np.median(y))], depth_for(n))


def _se(A, B, ell, sf2=1.0):
    d = (A[:, None, :] - B[None, :, :]) / np.asarray(ell, float)
    return sf2 * np.exp(-0.5 * (d ** 2).sum(-1))


def sgpr(seed: int = 6, m: int = 500, n_train: int = 4000, n: int = 128, ell=(0.15, 0.2, 0.25),
         noise: float = 1e-4, jitter: float = 1e-6) -> Workload:
    """A fitted sparse GP model (the stored {M, mu_M, A_M} of Sec. 3) on the paper-scale field.

    The paper fits its SGPR models with GPy (out of scope here).  Stand-in: n_train training
    points of the config-2 field recipe, m inducing sites drawn uniformly, and the inducing
    distribution that maximises the sparse-GP variational bound (Titsias 2009) for the given
    kernel and noise: S = (K_MM + K_MN K_NM / noise)^-1, mu_M = K_MM S K_MN y / noise,
    A_M = K_MM S K_MM, with K_MM = K(M, M) + jitter I.  Draw order: training sites and values (the
    field recipe), then the inducing sites."""
    rng = np.random.default_rng(seed)
    Xn, yn = _field(rng, n_train, 16, -1.0, 1.0, sinusoid=True)
    Xm = rng.random((m, 3))
    Kmm = _se(Xm, Xm, ell) + jitter * np.eye(m)
    Kmn = _se(Xm, Xn, ell)
    S = np.linalg.inv(Kmm + Kmn @ Kmn.T / noise)
    S = 0.5 * (S + S.T)
    mu = Kmm @ (S @ (Kmn @ yn)) / noise
    A = Kmm @ S @ Kmm
    A = 0.5 * (A + A.T)
    th = [float(np.percentile(yn, q)) for q in (25, 50, 75)]
    return Workload(f"sgpr_m{m}_train{n_train}_grid{n}", Xm, mu, SE, tuple(ell), 1.0, 0.0, n, th, depth_for(n),
                    extra={"A_M": A, "kmm_jitter": jitter, "train_X": Xn, "train_y": yn, "noise": noise})


def grid_points(n: int, lo=0.0, hi=1.0) -> np.ndarray:
    """Grid coordinates x_i = lo + i*(hi-lo)/(n-1), x-fastest order, (n^3, 3)."""
    g = lo + np.arange(n) * ((hi - lo) / (n - 1))
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1)
