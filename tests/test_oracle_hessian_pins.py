"""Pins of the oracle's analytic second derivatives of E_JK = 1/2 tr(DJ) -
1/4 tr(DK) at fixed D with respect to the nuclear coordinates
(oracle.jk_hessian; the two-electron part of the Hessian task, Sec. 3):

* against fourth-order central differences of the oracle's analytic gradient
  (itself pinned against central differences of the energy), on an s/p/d
  molecule and on one with an f shell (raised powers up to l = 5);
* the translational sum rule: the energy at fixed D does not change when all
  atoms move together, so every column of the Hessian sums to zero over the
  atoms;
* symmetry.
All quartets are kept (thresh 0) with the Coulomb bounds of the reference
geometry, so the displaced geometries evaluate the same quartet set.
"""
import numpy as np
import pytest

import oracle
from paper_2406_11185_gb300 import synth


def _fd_hessian(mol, D, Q, h=1e-4):
    n3 = 3 * mol.natom
    fd = np.zeros((n3, n3))
    for i in range(n3):
        a, k = divmod(i, 3)
        g = []
        for step in (2, 1, -1, -2):
            m = synth.Molecule(mol.atoms.copy(), mol.heavy, mol.shells, mol.spherical)
            m.atoms[a, k] += step * h
            g.append(oracle.grad(m, D, 0.0, Q=Q).reshape(-1))
        fd[i] = (-g[0] + 8 * g[1] - 8 * g[2] + g[3]) / (12 * h)
    return fd


@pytest.mark.parametrize("recipe", [("3s2p1d", "2s1p", (1, 2), (0.1, 5e3), 1801, 5),
                                    ("1s1p1d1f", "1s1p", (1, 1), (0.3, 30.0), 1802, 4)])
def test_hessian_matches_gradient_differences(recipe):
    heavy, light, nprim, exps, seed, nocc = recipe
    mol = synth.make_molecule(seed, 1, 2 if light == "2s1p" else 1, heavy, light, nprim, exps, (1.4, 2.0), True,
                              "hessian pin")
    D = synth.make_density(mol, nocc, seed + 10000)
    Q = oracle.schwarz(mol)
    H = oracle.jk_hessian(mol, D, 0.0, Q=Q)
    scale = np.max(np.abs(H))
    assert np.max(np.abs(H - H.T)) <= 1e-14 * scale
    n = mol.natom
    assert np.max(np.abs(H.reshape(n, 3, n, 3).sum(axis=0))) <= 1e-9 * scale
    fd = _fd_hessian(mol, D, Q)
    assert np.max(np.abs(H - fd)) <= 1e-8 * scale
