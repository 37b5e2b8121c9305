"""Seeded workload recipes (inputs only; no GP arithmetic lives here).

Recipes, one per named workload:

* ``gp2k``   N=2048, d=32, 16-component mixture, 15 probes, rank-32
             preconditioner, M=512 test points.
* ``gp64k``  N=65,536, d=32, same mixture plus 5 % near-duplicate rows
             (x_j + N(0, (1e-3)^2 I), j a random earlier row), 31 probes,
             rank 64.
* ``gp1m``   N=1,048,576, d=64, 512 components with Pareto(1.2) sizes,
             targets at ~1e-4 scale with 20 % of rows below 1e-7 in
             magnitude, 15 probes, rank 100.
* ``gp256k`` N=262,144, d=64, same generator as ``gp1m``, 31 probes.
* ``serve``  two resident models (N=65,536 and N=1,048,576, d=64) and a
             stream of molecule-shaped prediction requests.

Mixture: centres ~ N(0, I_d), per-component isotropic std ~ U[0.2, 0.6].
Lengthscales ~ U[0.5, 2]^d, outputscale 1, noise sigma^2 = 1e-4.
Targets: f(x) = sum_{m<64} a_m cos(w_m.x + b_m), w_m ~ N(0, I),
b_m ~ U[0, 2 pi], a_m ~ N(0, 1); f is standardised and
y = scale * (f + e), e ~ N(0, 1e-4) (variance 1e-4).
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # (N, d) float32, row-major
    y: np.ndarray            # (N,) float32
    lengthscale: np.ndarray  # (d,) float64
    outputscale: float
    sigma2: float
    n_probes: int
    rank: int
    tol: float
    Xtest: Optional[np.ndarray] = None  # (M, d) float32

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]


def mixture_features(rng: np.random.Generator, n: int, d: int, n_comp: int,
                     sizes: str = "equal", std_range=(0.2, 0.6),
                     centres=None, stds=None):
    """Draw n points from a Gaussian mixture; returns (X, centres, stds)."""
    if centres is None:
        centres = rng.standard_normal((n_comp, d))
        stds = rng.uniform(std_range[0], std_range[1], size=n_comp)
    if sizes == "equal":
        comp = rng.integers(0, n_comp, size=n)
    elif sizes == "pareto":
        w = rng.pareto(1.2, size=n_comp) + 1.0
        w = w / w.sum()
        comp = rng.choice(n_comp, size=n, p=w)
    else:
        raise ValueError(sizes)
    X = centres[comp] + stds[comp, None] * rng.standard_normal((n, d))
    return X.astype(np.float32), centres, stds


def rff_targets(rng: np.random.Generator, X: np.ndarray, scale: float,
                n_feat: int = 64):
    """Smooth random targets: a standardised sum of random cosines."""
    n, d = X.shape
    W = rng.standard_normal((n_feat, d))
    b = rng.uniform(0.0, 2.0 * np.pi, size=n_feat)
    a = rng.standard_normal(n_feat)
    f = np.cos(X.astype(np.float64) @ W.T + b) @ a
    f = (f - f.mean()) / (f.std() + 1e-300)
    e = rng.normal(0.0, 1e-2, size=n)  # variance 1e-4
    return (scale * (f + e)).astype(np.float32)


def _near_duplicates(rng, X, frac):
    n = X.shape[0]
    m = int(round(frac * n))
    rows = rng.choice(np.arange(1, n), size=m, replace=False)
    rows.sort()
    for r in rows:
        j = rng.integers(0, r)
        X[r] = X[j] + rng.normal(0.0, 1e-3, size=X.shape[1])
    return X


CONFIGS = {
    "gp2k": dict(N=2048, d=32, n_comp=16, sizes="equal", n_probes=15,
                 rank=32, tol=1e-6, M=512, dup=0.0, yscale=1e-2,
                 small_y=0.0, seed=1),
    "gp64k": dict(N=65536, d=32, n_comp=16, sizes="equal", n_probes=31,
                  rank=64, tol=1e-4, M=256, dup=0.05, yscale=1e-2,
                  small_y=0.0, seed=2),
    "gp1m": dict(N=1048576, d=64, n_comp=512, sizes="pareto", n_probes=15,
                 rank=100, tol=1e-4, M=512, dup=0.0, yscale=1e-4,
                 small_y=0.2, seed=3),
    "gp256k": dict(N=262144, d=64, n_comp=512, sizes="pareto", n_probes=31,
                   rank=64, tol=1e-4, M=512, dup=0.0, yscale=1e-4,
                   small_y=0.2, seed=4),
}


def make_workload(name: str, N: Optional[int] = None, d: Optional[int] = None,
                  seed: Optional[int] = None) -> Workload:
    """Build a named workload; ``N``/``d`` override the size for scaled-down
    cases (the first N rows of the full recipe are drawn identically only
    when N is unchanged; overrides draw a fresh, smaller instance)."""
    cfg = dict(CONFIGS[name])
    if N is not None:
        cfg["N"] = N
    if d is not None:
        cfg["d"] = d
    if seed is not None:
        cfg["seed"] = seed
    rng = np.random.default_rng(cfg["seed"])
    n, dd = cfg["N"], cfg["d"]
    X, centres, stds = mixture_features(rng, n, dd, cfg["n_comp"], cfg["sizes"])
    if cfg["dup"] > 0:
        X = _near_duplicates(rng, X.astype(np.float64), cfg["dup"]).astype(np.float32)
    ell = rng.uniform(0.5, 2.0, size=dd)
    y = rff_targets(rng, X, cfg["yscale"])
    if cfg["small_y"] > 0:
        m = int(round(cfg["small_y"] * n))
        idx = rng.choice(n, size=m, replace=False)
        y[idx] = rng.uniform(-1e-7, 1e-7, size=m).astype(np.float32)
    Xt, _, _ = mixture_features(rng, cfg["M"], dd, cfg["n_comp"], cfg["sizes"],
                                centres=centres, stds=stds)
    return Workload(name=name, X=np.ascontiguousarray(X), y=y,
                    lengthscale=ell, outputscale=1.0, sigma2=1e-4,
                    n_probes=cfg["n_probes"], rank=cfg["rank"], tol=cfg["tol"],
                    Xtest=np.ascontiguousarray(Xt))


def molecule_request(rng: np.random.Generator, d: int, centres, stds,
                     n_occ_range=(2, 60)):
    """One synthetic molecule: n_occ diagonal and n_occ(n_occ-1)/2
    off-diagonal pair-feature rows drawn from the mixture."""
    n_occ = int(rng.integers(n_occ_range[0], n_occ_range[1] + 1))
    n_off = n_occ * (n_occ - 1) // 2
    Xd, _, _ = mixture_features(rng, n_occ, d, len(stds), "equal",
                                centres=centres, stds=stds)
    Xo, _, _ = mixture_features(rng, max(n_off, 0), d, len(stds), "equal",
                                centres=centres, stds=stds)
    return Xd, Xo
