"""Pins of the oracle's closed-shell SCF nuclear gradient (oracle.scf_gradient:
one-electron derivative integrals, the energy-weighted density term, the
two-electron gradient at fixed D and the nuclear repulsion; the single-point
force task of Sec. 3 around the J/K gradient):

* against central differences of the converged SCF energy, every coordinate
  of an s/p/d molecule;
* zero net force (the basis functions move with their atoms);
* two s Gaussians on two protons: dE/dR against differences of the
  closed-form energy built from the textbook s-type integrals (the symmetric
  occupied orbital is fixed by symmetry, so E(R) needs no SCF).
"""
import math

import numpy as np

import oracle
from paper_2406_11185_gb300 import synth

from .test_oracle_scf_pins import _mol, _s_integrals


def _light_molecule():
    mol = synth.make_molecule(1801, 1, 2, "3s2p1d", "2s1p", (1, 2), (0.1, 5e3), (1.4, 2.0), True, "force pin")
    Z = synth.nuclear_charges(mol)
    return mol, Z, int(round(Z.sum())) // 2


def test_scf_gradient_matches_energy_differences():
    mol, Z, nocc = _light_molecule()
    Q = oracle.schwarz(mol)
    _, g, r = oracle.scf_gradient(mol, Z, nocc, 0.0, Q=Q, e_tol=1e-13, g_tol=1e-10)
    assert r["converged"]
    h = 1e-3
    for a in range(mol.natom):
        for k in range(3):
            es = []
            for step in (2, 1, -1, -2):
                m = synth.Molecule(mol.atoms.copy(), mol.heavy, mol.shells, mol.spherical)
                m.atoms[a, k] += step * h
                es.append(oracle.scf(m, Z, nocc, 0.0, e_tol=1e-13, g_tol=1e-10)["energy"])
            fd = (-es[0] + 8 * es[1] - 8 * es[2] + es[3]) / (12 * h)
            assert abs(g[a, k] - fd) <= 1e-7 * max(1.0, abs(fd)), (a, k, g[a, k], fd)
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-10


def test_two_proton_force_closed_form():
    a = 0.4166

    def energy(R):
        centres = [[0.0, 0.0, 0.0], [0.0, 0.0, R]]
        S, T, V, G = _s_integrals(centres, [a, a], [1.0, 1.0])
        c = np.array([1.0, 1.0]) / math.sqrt(2 * (1 + S[0, 1]))
        return 2 * (c @ (T + V) @ c) + np.einsum("i,j,k,l,ijkl->", c, c, c, c, G) + 1.0 / R

    R, h = 1.4, 1e-4
    fd = (-energy(R + 2 * h) + 8 * energy(R + h) - 8 * energy(R - h) + energy(R - 2 * h)) / (12 * h)
    mol = _mol([[0.0, 0.0, 0.0], [0.0, 0.0, R]], [(0, 0, [a], [1.0]), (1, 0, [a], [1.0])])
    _, g, r = oracle.scf_gradient(mol, np.array([1.0, 1.0]), 1, 0.0, e_tol=1e-14, g_tol=1e-12)
    assert r["converged"]
    assert abs(g[1, 2] - fd) <= 1e-9 and abs(g[0, 2] + fd) <= 1e-9
    assert np.max(np.abs(g[:, :2])) <= 1e-12
