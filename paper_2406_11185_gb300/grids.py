"""Molecular integration grids: the input of the exchange-correlation step.

Sec. 1.2.2 (the EXC paragraph) evaluates the exchange-correlation energy by
numerical integration over grid points around the atoms.  This module only
generates such grids (points and weights).  It holds no density, functional or
basis-function arithmetic, so both the oracle and a device path can take its
output as input data.

* Per atom, a product grid: a radial Gauss-Chebyshev rule of the second kind
  on x in (-1, 1), mapped to r = R (1 + x) / (1 - x) (Becke, J. Chem. Phys. 88,
  2547 (1988)), times an angular rule that is Gauss-Legendre in cos(theta) and
  uniform in phi (exact for spherical harmonics of degree < 2 ntheta in theta
  and < nphi in phi).
* Becke's fuzzy-cell partition: a point of atom A's grid is weighted by
  w_A(r) = P_A(r) / sum_B P_B(r), P_A = prod_{B != A} s(mu_AB), with
  mu_AB = (|r - R_A| - |r - R_B|) / |R_A - R_B| and
  s(mu) = (1 - f(f(f(mu)))) / 2, f(x) = 3x/2 - x^3/2 (same paper).  The cell
  functions sum to one at every point, so the molecular grid integrates a
  function that is smooth away from the nuclei like the atomic grids do.
"""
from __future__ import annotations

import numpy as np


def radial_rule(nrad: int, R: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Points r_i and weights w_i with sum_i w_i g(r_i) ~ int_0^inf g(r) r^2 dr."""
    i = np.arange(1, nrad + 1)
    x = np.cos(i * np.pi / (nrad + 1))
    wx = np.pi / (nrad + 1) * np.sin(i * np.pi / (nrad + 1)) ** 2  # weight of sqrt(1 - x^2)
    r = R * (1.0 + x) / (1.0 - x)
    dr = 2.0 * R / (1.0 - x) ** 2
    return r, wx / np.sqrt(1.0 - x * x) * dr * r * r


def angular_rule(ntheta: int, nphi: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit vectors and weights with sum w f(u) ~ int f dOmega (total 4 pi)."""
    u, wu = np.polynomial.legendre.leggauss(ntheta)
    phi = 2.0 * np.pi * np.arange(nphi) / nphi
    st = np.sqrt(1.0 - u * u)
    dirs = np.stack([np.outer(st, np.cos(phi)), np.outer(st, np.sin(phi)), np.outer(u, np.ones(nphi))], axis=-1)
    w = np.outer(wu, np.full(nphi, 2.0 * np.pi / nphi))
    return dirs.reshape(-1, 3), w.reshape(-1)


def becke_partition(atoms: np.ndarray, points: np.ndarray) -> np.ndarray:
    """w[A, g]: Becke's cell function of atom A at every point (sums to 1 over A)."""
    atoms = np.asarray(atoms, dtype=np.float64)
    d = np.linalg.norm(points[None, :, :] - atoms[:, None, :], axis=-1)  # [natom, n]
    nat = len(atoms)
    P = np.ones((nat, len(points)))
    for a in range(nat):
        for b in range(nat):
            if a == b:
                continue
            mu = (d[a] - d[b]) / np.linalg.norm(atoms[a] - atoms[b])
            f = mu
            for _ in range(3):
                f = 1.5 * f - 0.5 * f ** 3
            P[a] *= 0.5 * (1.0 - f)
    return P / np.sum(P, axis=0, keepdims=True)


def molecular_grid(atoms, nrad: int = 60, ntheta: int = 18, nphi: int = 36,
                   R: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """Points [n, 3] (bohr) and weights [n] of the partitioned molecular grid:
    every atom's product grid, each point weighted by its own atom's cell
    function."""
    atoms = np.asarray(atoms, dtype=np.float64)
    r, wr = radial_rule(nrad, R)
    dirs, wa = angular_rule(ntheta, nphi)
    local = (r[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
    wloc = (wr[:, None] * wa[None, :]).reshape(-1)
    pts, wts = [], []
    for a, A in enumerate(atoms):
        p = local + A
        pts.append(p)
        wts.append(wloc * becke_partition(atoms, p)[a])
    return np.concatenate(pts), np.concatenate(wts)
