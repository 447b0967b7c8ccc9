"""Plain CPU oracle of the exchange-correlation step on a grid (the EXC
paragraph of Sec. 1.2.2: basis functions evaluated on grid points around the
atoms, the density and the exchange-correlation potential matrix obtained by
numerical integration).

TEST INFRASTRUCTURE ONLY, like the rest of this package.  The functional is
the local-density (Slater) exchange of a closed-shell density; the grid is an
input (``paper_2406_11185_gb300.grids``).  Everything is the plain definition
over all grid points and basis functions, without the paper's distance
screening or block sparsity:

    phi_mu(r_g)   Cartesian: sum_i c_i N(a_i, l) x^ax y^ay z^az exp(-a_i |r-A|^2),
                  spherical: the solid-harmonic combinations (oracle.cart2sph)
    rho(r_g)    = sum_{mu nu} D_mu,nu phi_mu(r_g) phi_nu(r_g)
    E_x         = sum_g w_g e_x(rho_g),      e_x(rho) = -(3/4) (3/pi)^(1/3) rho^(4/3)
    V^x_mu,nu   = sum_g w_g v_x(rho_g) phi_mu(r_g) phi_nu(r_g),
                  v_x = de_x/drho = -(3/pi)^(1/3) rho^(1/3)
"""
from __future__ import annotations

import math

import numpy as np

from . import cart2sph, cart_powers

_CX = 0.75 * (3.0 / math.pi) ** (1.0 / 3.0)


def _dfact(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def ao_values(mol, points) -> np.ndarray:
    """phi[g, mu] in the molecule's output basis (spherical iff mol.spherical)."""
    points = np.asarray(points, dtype=np.float64)
    cols = []
    for atom, l, exps, coefs in mol.shells:
        d = points - mol.atoms[atom]
        r2 = np.sum(d * d, axis=1)
        radial = np.zeros(len(points))
        for a, c in zip(exps, coefs):
            norm = (2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2) / math.sqrt(_dfact(2 * l - 1))
            radial += c * norm * np.exp(-a * r2)
        for px, py, pz in cart_powers(l):
            cols.append(radial * d[:, 0] ** px * d[:, 1] ** py * d[:, 2] ** pz)
    phi = np.stack(cols, axis=1)
    if mol.spherical:
        phi = phi @ cart2sph(mol).T
    return phi


def density(mol, D, points) -> np.ndarray:
    """rho(r_g) for the density matrix D in the molecule's output basis."""
    phi = ao_values(mol, points)
    return np.einsum("gm,mn,gn->g", phi, np.asarray(D, dtype=np.float64), phi)


def lda_exchange(mol, D, points, weights) -> tuple[float, np.ndarray]:
    """Slater exchange energy E_x and its potential matrix V^x of the
    closed-shell density D on the grid (points, weights)."""
    phi = ao_values(mol, points)
    rho = np.einsum("gm,mn,gn->g", phi, np.asarray(D, dtype=np.float64), phi)
    rho = np.maximum(rho, 0.0)
    w = np.asarray(weights, dtype=np.float64)
    ex = -_CX * rho ** (4.0 / 3.0)
    vx = -(4.0 / 3.0) * _CX * np.cbrt(rho)
    E = float(np.sum(w * ex))
    V = phi.T @ ((w * vx)[:, None] * phi)
    return E, 0.5 * (V + V.T)
