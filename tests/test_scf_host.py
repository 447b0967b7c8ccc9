"""Host-side pieces of the SCF driver that need no GPU: the nuclear
repulsion energy and its gradient (against central differences and the
oracle's closed form)."""
import numpy as np

import oracle
from paper_2406_11185_gb300 import scf, synth


def test_nuclear_repulsion_and_gradient():
    rng = np.random.default_rng(11)
    X = rng.uniform(-3, 3, size=(6, 3))
    Z = rng.uniform(1, 8, size=6)
    mol = synth.Molecule(X, np.ones(6, dtype=bool), [], True)
    assert abs(scf.nuclear_repulsion(X, Z) - oracle.nuclear_repulsion(mol, Z)) <= 1e-12 * scf.nuclear_repulsion(X, Z)
    g = scf.nuclear_repulsion_gradient(X, Z)
    h = 1e-5
    for a in range(6):
        for k in range(3):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, k] += h
            Xm[a, k] -= h
            fd = (scf.nuclear_repulsion(Xp, Z) - scf.nuclear_repulsion(Xm, Z)) / (2 * h)
            assert abs(g[a, k] - fd) <= 1e-7 * max(1.0, abs(fd))
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-12 * np.max(np.abs(g))
