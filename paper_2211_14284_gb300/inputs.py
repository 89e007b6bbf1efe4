"""Seeded synthetic inputs for the Riesz-map solvers.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no bases, no operators, no DOF numbering beyond a vector
length the caller supplies).  Both the CUDA path and the CPU oracle take their
inputs from here, so a test can feed the same problem to each.

Layouts
-------
* vertices: float64 array of shape ((n3+1)*(n2+1)*(n1+1), 3), vertex
  (a1, a2, a3) at row a1 + (n1+1)*(a2 + (n2+1)*a3), on the unit cube.
* per-cell coefficients: float64 array of length n1*n2*n3, cell (e1, e2, e3)
  at e1 + n1*(e2 + n2*e3).
* right-hand sides: float64 vector of the lattice length the caller passes.
  Entries that fall on Dirichlet DOFs are drawn too; the solvers ignore them.

The paper's meshes (extruded unstructured hexahedra, Sec. 5.1) exist only as
figures, so structured and randomly perturbed hexahedral meshes stand in.
"""

from __future__ import annotations

import numpy as np

BASE_SEED = 20221125


def rng(seed_offset: int) -> np.random.Generator:
    """PCG64 generator seeded with BASE_SEED + seed_offset."""
    return np.random.Generator(np.random.PCG64(BASE_SEED + int(seed_offset)))


def _dims(n):
    if np.isscalar(n):
        return (int(n), int(n), int(n))
    n1, n2, n3 = (int(v) for v in n)
    return (n1, n2, n3)


def vertices(n, perturb: float = 0.0, seed: int = 0) -> np.ndarray:
    """Vertices of a structured hex mesh of the unit cube.

    perturb > 0 moves every interior vertex by U(-perturb*h_d, perturb*h_d)
    along each coordinate d (h_d = 1/n_d); boundary vertices stay put, so the
    domain is still the unit cube.  perturb=0.1 is the "10% random
    interior-vertex perturbation" of the distorted-mesh workload.
    """
    n1, n2, n3 = _dims(n)
    a1, a2, a3 = np.meshgrid(np.arange(n1 + 1), np.arange(n2 + 1),
                             np.arange(n3 + 1), indexing="ij")
    # x fastest: transpose to (a3, a2, a1)
    a1 = a1.transpose(2, 1, 0).ravel()
    a2 = a2.transpose(2, 1, 0).ravel()
    a3 = a3.transpose(2, 1, 0).ravel()
    X = np.stack([a1 / n1, a2 / n2, a3 / n3], axis=1).astype(np.float64)
    if perturb > 0.0:
        g = rng(seed)
        h = np.array([1.0 / n1, 1.0 / n2, 1.0 / n3])
        shift = g.uniform(-1.0, 1.0, size=X.shape) * (perturb * h)
        interior = ((a1 > 0) & (a1 < n1) & (a2 > 0) & (a2 < n2)
                    & (a3 > 0) & (a3 < n3))
        X[interior] += shift[interior]
    return X


def constant_coefficient(n, value: float = 1.0) -> np.ndarray:
    n1, n2, n3 = _dims(n)
    return np.full(n1 * n2 * n3, float(value))


def loguniform_coefficient(n, lo: float, hi: float, seed: int) -> np.ndarray:
    """Piecewise-constant coefficient 10**U(log10 lo, log10 hi) per cell."""
    n1, n2, n3 = _dims(n)
    g = rng(seed)
    return 10.0 ** g.uniform(np.log10(lo), np.log10(hi), size=n1 * n2 * n3)


def lognormal_grf_coefficient(n, sigma: float = 1.0, ell: float = 0.1,
                              seed: int = 0) -> np.ndarray:
    """exp(g) per cell, g a zero-mean Gaussian random field at cell centres
    with squared-exponential covariance sigma^2 exp(-|x-y|^2 / (2 ell^2)).

    The covariance is separable, so g = (L3 (x) L2 (x) L1) xi with L_d the
    Cholesky factor of the 1D covariance at the cell centres (plus 1e-10
    jitter) and xi ~ N(0, I).
    """
    n1, n2, n3 = _dims(n)
    g = rng(seed)
    xi = g.standard_normal((n3, n2, n1))
    facs = []
    for nd in (n1, n2, n3):
        c = (np.arange(nd) + 0.5) / nd
        C = np.exp(-(c[:, None] - c[None, :]) ** 2 / (2.0 * ell * ell))
        facs.append(np.linalg.cholesky(C + 1e-10 * np.eye(nd)))
    L1, L2, L3 = facs
    f = np.einsum("ia,abc->ibc", L3, xi)
    f = np.einsum("jb,ibc->ijc", L2, f)
    f = np.einsum("kc,ijc->ijk", L1, f)
    return np.exp(sigma * f).ravel()


def annulus_coefficient(n, inside: float, outside: float, r_in: float = 0.15,
                        r_out: float = 0.3) -> np.ndarray:
    """Two-material piecewise-constant coefficient: `inside` on the cells whose
    centre lies in the annulus r_in <= r <= r_out around the vertical axis
    x = y = 1/2 of the unit cube (a wire), `outside` elsewhere (the air)."""
    n1, n2, n3 = _dims(n)
    e3, e2, e1 = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    x = (e1.ravel() + 0.5) / n1 - 0.5
    y = (e2.ravel() + 0.5) / n2 - 0.5
    r = np.sqrt(x * x + y * y)
    return np.where((r >= r_in) & (r <= r_out), float(inside), float(outside))


def normal_rhs(length: int, seed: int) -> np.ndarray:
    """N(0, 1) entries, one per lattice DOF (Dirichlet entries are ignored)."""
    return rng(seed).standard_normal(int(length))


def batched_hcurl_problems(count: int = 64, seed: int = 4):
    """Problem list of the batched H(curl) workload: n ~ U{4..12},
    p ~ U{3..12}, beta log-uniform in [0.1, 10], alpha = 1."""
    g = rng(seed)
    out = []
    for i in range(count):
        n = int(g.integers(4, 13))
        p = int(g.integers(3, 13))
        beta = float(10.0 ** g.uniform(-1.0, 1.0))
        out.append({"n": n, "p": p, "beta": beta, "alpha": 1.0,
                    "rhs_seed": 1000 + i})
    return out
