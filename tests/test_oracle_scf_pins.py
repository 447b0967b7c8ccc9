"""Pins of the oracle's one-electron integrals and of its SCF loop (the
restricted closed-shell Fock iteration around the J/K build, Eq. 1 of
Sec. 1.2.1 with F = H + J - 1/2 K).  Every reference here is independent of
the oracle's McMurchie-Davidson code:

* overlap and kinetic energy against Gauss-Hermite quadrature of the
  (differentiated) Gaussians;
* nuclear attraction against the t-integral form of 1/r with exact per-t
  quadrature, and one element with a compact f-f distribution against a
  30-digit mpmath evaluation;
* the SCF energy of one s Gaussian on a two-electron atom and of two s
  Gaussians on two protons against closed forms built from the textbook
  s-type integrals (the error function form of F_0);
* properties of a converged closed-shell SCF: idempotent density, electron
  count, vanishing commutator FDS - SDF and a stationary energy.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_11185_gb300 import synth

from . import brute


def _mol(atoms, shells, spherical=False):
    atoms = np.asarray(atoms, dtype=np.float64)
    return synth.Molecule(atoms, np.ones(len(atoms), dtype=bool),
                          [(a, l, np.asarray(e, float), np.asarray(c, float)) for a, l, e, c in shells], spherical)


@pytest.mark.parametrize("name,spherical", [("tiny", True), ("small_f3", False)])
def test_overlap_matches_quadrature(name, spherical):
    mol, _ = synth.config(name, spherical=spherical)
    S, _, _ = oracle.one_electron(mol, synth.nuclear_charges(mol))
    Sq = synth.overlap_matrix(mol)
    assert np.max(np.abs(S - Sq)) <= 1e-12 * np.max(np.abs(Sq))


def test_kinetic_matches_quadrature():
    mol, _ = synth.config("tiny_f", spherical=False)
    _, T, _ = oracle.one_electron(mol, synth.nuclear_charges(mol))
    Tq = brute.one_electron_cartesian(mol, synth.nuclear_charges(mol), "T")
    assert np.max(np.abs(T - Tq)) <= 1e-13 * np.max(np.abs(Tq))
    assert np.max(np.abs(T - T.T)) <= 1e-13 * np.max(np.abs(T))


def test_nuclear_attraction_matches_brute_force():
    # s, p, d and f shells on two centres and a third nucleus, moderate exponents
    atoms = [[0.0, 0.0, 0.0], [0.3, -1.1, 1.4], [1.5, 0.4, -0.6]]
    shells = [(0, 0, [3.1, 0.4], [0.6, 0.5]), (0, 1, [1.2], [1.0]), (1, 2, [0.9, 0.25], [0.7, 0.4]),
              (1, 3, [0.8], [1.0]), (0, 2, [2.2], [1.0])]
    mol = _mol(atoms, shells)
    Z = np.array([6.0, 1.0, 2.5])
    _, _, V = oracle.one_electron(mol, Z)
    Vb = brute.one_electron_cartesian(mol, Z, "V")
    assert np.max(np.abs(V - Vb)) <= 1e-11 * np.max(np.abs(Vb))


def test_nuclear_attraction_compact_f_shell_vs_mpmath():
    """A compact f-f distribution (exponent 1024) seen from a nucleus 1.7
    bohr away: an element set by high multipoles, evaluated to 30 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    A, C = np.zeros(3), np.array([0.9, -1.2, 0.8])
    e = 1024.35459669
    mol = _mol([A, C], [(0, 3, [e], [1.0])])
    _, _, V = oracle.one_electron(mol, np.array([0.0, 1.0]))
    pw = brute.cart_powers(3)
    i, j = 6, 7
    a2 = mp.mpf(2 * e)
    Am, Cm = [mp.mpf(x) for x in A], [mp.mpf(x) for x in C]

    def mom(k, q):  # int y^k exp(-q y^2) dy
        return mp.mpf(0) if k % 2 else mp.gamma((k + 1) / mp.mpf(2)) / q ** ((k + 1) / mp.mpf(2))

    def f(t):
        q = a2 + t * t
        v = mp.exp(-a2 * t * t / q * mp.fsum((x - y) ** 2 for x, y in zip(Am, Cm)))
        for k in range(3):
            R = (a2 * Am[k] + t * t * Cm[k]) / q
            m = pw[i][k] + pw[j][k]
            v *= mp.fsum(mp.binomial(m, n) * (R - Am[k]) ** (m - n) * mom(n, q) for n in range(m + 1))
        return v

    ref = -2 / mp.sqrt(mp.pi) * mp.quad(f, [0, 0.1, 0.5, 1, 2, 5, 20, 100, mp.inf]) * brute._prim_norm(e, 3) ** 2
    assert abs(V[i, j] - float(ref)) <= 1e-12 * abs(float(ref))


def _s_integrals(centres, alphas, charges):
    """Closed forms of normalised s Gaussians: S, T, V (all nuclei) and the
    ERI tensor (Boys F_0 by the error function)."""
    n = len(alphas)
    X = [np.asarray(c, float) for c in centres]
    N = [(2 * a / math.pi) ** 0.75 for a in alphas]
    F0 = lambda T: 1.0 if T < 1e-14 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    S, T, V = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            a, b = alphas[i], alphas[j]
            p, r2 = a + b, float(np.sum((X[i] - X[j]) ** 2))
            K = math.exp(-a * b / p * r2)
            P = (a * X[i] + b * X[j]) / p
            S[i, j] = (math.pi / p) ** 1.5 * K * N[i] * N[j]
            T[i, j] = a * b / p * (3 - 2 * a * b / p * r2) * S[i, j]
            V[i, j] = sum(-z * 2 * math.pi / p * K * F0(p * float(np.sum((P - np.asarray(c)) ** 2))) * N[i] * N[j]
                          for c, z in zip(centres, charges))
    G = np.zeros((n, n, n, n))
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for m in range(n):
                    a, b, c, d = alphas[i], alphas[j], alphas[k], alphas[m]
                    p, q = a + b, c + d
                    P = (a * X[i] + b * X[j]) / p
                    Q = (c * X[k] + d * X[m]) / q
                    Kab = math.exp(-a * b / p * float(np.sum((X[i] - X[j]) ** 2)))
                    Kcd = math.exp(-c * d / q * float(np.sum((X[k] - X[m]) ** 2)))
                    G[i, j, k, m] = (2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd *
                                     F0(p * q / (p + q) * float(np.sum((P - Q) ** 2))) * N[i] * N[j] * N[k] * N[m])
    return S, T, V, G


@pytest.mark.parametrize("a", [0.3, 0.768, 2.5])
def test_scf_one_gaussian_two_electron_atom(a):
    """E(a) = 3a - 4 Z sqrt(2a/pi) + 2 sqrt(a/pi) for one normalised s
    Gaussian doubly occupied on a nucleus of charge Z = 2."""
    mol = _mol([[0.0, 0.0, 0.0]], [(0, 0, [a], [1.0])])
    r = oracle.scf(mol, np.array([2.0]), 1, thresh=0.0)
    ref = 3 * a - 8 * math.sqrt(2 * a / math.pi) + 2 * math.sqrt(a / math.pi)
    assert r["converged"]
    assert abs(r["energy"] - ref) <= 1e-12 * abs(ref)


def test_scf_two_protons_closed_form():
    """Two s Gaussians on two protons: by symmetry the occupied orbital is
    (phi_1 + phi_2) / sqrt(2(1 + S12)), so E = 2 h + (ss|ss)_sigma + 1/R from
    the closed-form s integrals."""
    R, a = 1.4, 0.4166
    centres = [[0.0, 0.0, 0.0], [0.0, 0.0, R]]
    S, T, V, G = _s_integrals(centres, [a, a], [1.0, 1.0])
    c = np.array([1.0, 1.0]) / math.sqrt(2 * (1 + S[0, 1]))
    h = c @ (T + V) @ c
    J = np.einsum("i,j,k,l,ijkl->", c, c, c, c, G)
    ref = 2 * h + J + 1.0 / R
    mol = _mol(centres, [(0, 0, [a], [1.0]), (1, 0, [a], [1.0])])
    r = oracle.scf(mol, np.array([1.0, 1.0]), 1, thresh=0.0)
    assert r["converged"]
    assert abs(r["energy"] - ref) <= 1e-12 * abs(ref)


def test_scf_converged_density_properties():
    mol, opt = synth.config("tiny")
    Z = synth.nuclear_charges(mol)
    nocc = int(round(Z.sum())) // 2
    r = oracle.scf(mol, Z, nocc, thresh=opt["thresh"])
    D, S, F = r["D"], r["S"], r["F"]
    assert r["converged"]
    assert np.max(np.abs(D @ S @ D - 2 * D)) <= 1e-9
    assert abs(np.trace(D @ S) - 2 * nocc) <= 1e-10
    assert np.max(np.abs(F @ D @ S - S @ D @ F)) <= 1e-7
    # stationary: the energy changes only to second order under an
    # occupied-virtual rotation of the converged orbitals
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T
    _, C = np.linalg.eigh(X.T @ F @ X)
    C = X @ C

    def energy(theta):
        Cr = C.copy()
        o, v = nocc - 1, nocc
        Cr[:, o] = math.cos(theta) * C[:, o] + math.sin(theta) * C[:, v]
        Dr = 2 * Cr[:, :nocc] @ Cr[:, :nocc].T
        J, K = oracle.jk(mol, Dr, opt["thresh"])
        return float(np.sum(Dr * r["H"])) + oracle.energy(Dr, J, K) + r["e_nuc"]

    h = 1e-3
    e0, ep, em = energy(0.0), energy(h), energy(-h)
    assert abs(e0 - r["energy"]) <= 1e-10
    assert abs(ep - em) / (2 * h) <= 1e-5            # first derivative vanishes
    assert (ep + em - 2 * e0) / h ** 2 > 0.0         # a minimum along this rotation
