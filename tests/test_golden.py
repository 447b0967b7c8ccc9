"""The oracle reproduces its stored values for the 3-atom workload
(tests/golden/tiny_oracle.json, written by tests/golden/make_golden.py,
which calls only the oracle).  A change to the oracle's arithmetic shows up
here and must come with a regenerated fixture."""
import json
import os

import numpy as np

import oracle
from paper_2406_11185_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "tiny_oracle.json")


def test_oracle_matches_stored_tiny_values():
    ref = json.load(open(GOLDEN))
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    J, K = oracle.jk(mol, D, opt["thresh"])
    assert mol.nbf() == ref["nbf"]
    assert abs(oracle.energy(D, J, K) - ref["energy"]) <= 1e-11 * abs(ref["energy"])
    for got, key in ((np.diag(J), "J_diag"), (np.diag(K), "K_diag"), (J[0], "J_row0"), (K[0], "K_row0")):
        want = np.array(ref[key])
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want))), key
    g = oracle.grad(mol, D, opt["thresh"])
    assert np.max(np.abs(g - np.array(ref["grad"]))) <= 1e-12 * max(1.0, np.max(np.abs(g)))
