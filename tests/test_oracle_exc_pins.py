"""Pins of the exchange-correlation oracle (oracle.exc: basis functions on a
grid, the density and the Slater-exchange energy and potential matrix, the
EXC step of Sec. 1.2.2) and of the grid generator it takes as input.  Each
reference is independent of the code under test:

* grid: Becke's cell functions sum to one; the radial rule integrates
  r^2 exp(-a r^2) (closed form sqrt(pi) / (4 a^(3/2))) for a from 0.05 to 5e3;
  the angular rule integrates x^2, x^4 and x^2 y^2 over the sphere exactly;
* AO values: the grid integral of phi_mu phi_nu reproduces the overlap matrix
  of the C oracle (McMurchie-Davidson), and sum_g w_g rho_g = tr(D S);
* Slater exchange: for one normalised s Gaussian doubly occupied, the closed
  form -(3/4)(3/pi)^(1/3) 2^(4/3) (2a/pi)^2 (3 pi / (8a))^(3/2);
* the potential matrix is the derivative of the energy with respect to D
  (central differences along a random symmetric direction);
* the energy is unchanged under a rigid translation of molecule and grid.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import exc
from paper_2406_11185_gb300 import grids, synth


def test_becke_cells_sum_to_one():
    rng = np.random.default_rng(3)
    atoms = rng.uniform(-2, 2, size=(5, 3))
    pts = rng.uniform(-4, 4, size=(2000, 3))
    w = grids.becke_partition(atoms, pts)
    assert np.max(np.abs(w.sum(axis=0) - 1.0)) <= 1e-14
    assert np.all(w >= 0.0)
    # at a nucleus the cell of that atom has weight one
    near = grids.becke_partition(atoms, atoms + 1e-9)
    assert np.allclose(np.diag(near), 1.0, atol=1e-12)


@pytest.mark.parametrize("a", [0.05, 1.0, 100.0, 5000.0])
def test_radial_rule(a):
    r, w = grids.radial_rule(120)
    ref = math.sqrt(math.pi) / (4.0 * a ** 1.5)
    assert abs(float(np.sum(w * np.exp(-a * r * r))) - ref) <= 1e-7 * ref


def test_angular_rule():
    u, w = grids.angular_rule(6, 12)
    x, y, z = u[:, 0], u[:, 1], u[:, 2]
    assert abs(np.sum(w) - 4 * math.pi) <= 1e-13
    assert abs(np.sum(w * x * x) - 4 * math.pi / 3) <= 1e-13
    assert abs(np.sum(w * x ** 4) - 4 * math.pi / 5) <= 1e-13
    assert abs(np.sum(w * x * x * y * y) - 4 * math.pi / 15) <= 1e-13
    assert abs(np.sum(w * x * y * z)) <= 1e-13


@pytest.fixture(scope="module")
def tiny():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    P, W = grids.molecular_grid(mol.atoms, 60, 18, 36)
    return mol, D, P, W


def test_grid_overlap_matches_oracle(tiny):
    mol, D, P, W = tiny
    phi = exc.ao_values(mol, P)
    S = oracle.overlap(mol)
    Sg = phi.T @ (W[:, None] * phi)
    assert np.max(np.abs(Sg - S)) <= 2e-6 * np.max(np.abs(S))
    rho = exc.density(mol, D, P)
    assert abs(float(np.sum(W * rho)) - float(np.sum(D * S))) <= 1e-6 * float(np.sum(D * S))


@pytest.mark.parametrize("a", [0.3, 2.0, 40.0])
def test_slater_exchange_of_one_gaussian(a):
    mol = synth.Molecule(np.zeros((1, 3)), np.ones(1, dtype=bool), [(0, 0, np.array([a]), np.array([1.0]))],
                         True)
    D = np.array([[2.0]])
    P, W = grids.molecular_grid(mol.atoms, 120, 8, 8)
    E, V = exc.lda_exchange(mol, D, P, W)
    cx = 0.75 * (3 / math.pi) ** (1 / 3)
    ref = -cx * 2 ** (4 / 3) * (2 * a / math.pi) ** 2 * (3 * math.pi / (8 * a)) ** 1.5
    assert abs(E - ref) <= 1e-8 * abs(ref)


def test_potential_is_energy_derivative(tiny):
    mol, D, P, W = tiny
    rng = np.random.default_rng(5)
    X = rng.normal(size=D.shape)
    X = 0.5 * (X + X.T)
    h = 1e-5
    Ep, _ = exc.lda_exchange(mol, D + h * X, P, W)
    Em, _ = exc.lda_exchange(mol, D - h * X, P, W)
    _, V = exc.lda_exchange(mol, D, P, W)
    fd = (Ep - Em) / (2 * h)
    assert abs(fd - float(np.sum(V * X))) <= 1e-6 * abs(fd)


def test_energy_invariant_under_translation(tiny):
    mol, D, P, W = tiny
    E0, _ = exc.lda_exchange(mol, D, P, W)
    shift = np.array([0.7, -1.3, 2.1])
    mol2 = synth.Molecule(mol.atoms + shift, mol.heavy, mol.shells, mol.spherical)
    P2, W2 = grids.molecular_grid(mol2.atoms, 60, 18, 36)
    E1, _ = exc.lda_exchange(mol2, D, P2, W2)
    assert abs(E1 - E0) <= 1e-10 * abs(E0)
