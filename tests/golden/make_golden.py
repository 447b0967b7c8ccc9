"""Writes the stored oracle values under tests/golden/.  It calls only
oracle/ and the seeded input generator; the paper prints no worked J/K
example, so these values pin the oracle against later changes to its own
arithmetic (tiny_oracle.json) and spare the GPU tests the oracle's slowest
runs (the other files), not a comparison with the paper.

    python tests/golden/make_golden.py [tiny] [small_f3] [c60] [c240]

* tiny_oracle.json: J, K, E_JK and the nuclear gradient of the 3-atom
  workload (1 heavy atom 3s2p1d + 2 H 2s1p, 24 spherical functions,
  thresh 1e-12).
* small_f3_grad.json: the nuclear gradient of the 5-atom f-shell molecule
  (2 heavy atoms 4s3p2d1f + 3 H 3s2p1d, 1-3 primitives, thresh 1e-12).
* c60_blocks.json / c240_blocks.json: sampled J and K blocks of the 60-atom
  (516 functions, thresh 1e-10) and 240-atom (2,064 functions, thresh 1e-10)
  molecules, each block computed straight from the definition over every
  ket pair (oracle.jk_blocks).
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2406_11185_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _write(name, out):
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, flush=True)


def tiny():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    J, K = oracle.jk(mol, D, opt["thresh"])
    g = oracle.grad(mol, D, opt["thresh"])
    _write("tiny_oracle.json", {
        "workload": "tiny: synth.config('tiny'), D = synth.make_density(mol, 5, 11001), thresh 1e-12",
        "nbf": int(mol.nbf()),
        "energy": oracle.energy(D, J, K),
        "J_diag": np.diag(J).tolist(),
        "K_diag": np.diag(K).tolist(),
        "J_row0": J[0].tolist(),
        "K_row0": K[0].tolist(),
        "grad": g.tolist(),
    })


def small_f3():
    mol, opt = synth.config("small_f3")
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    g = oracle.grad(mol, D, opt["thresh"])
    _write("small_f3_grad.json", {
        "workload": "small_f3: synth.config('small_f3'), spherical, D = synth.make_density(mol, 12, 11602), "
                    "thresh 1e-12",
        "nbf": int(mol.nbf()), "thresh": opt["thresh"], "grad": g.tolist(),
    })


def sample_pairs(mol, Q):
    """Shell pairs (a >= b) of the sampled blocks: for each class s-s, p-p,
    d-d on one shell and s-s, p-s, d-s, p-p, d-p, d-d across two atoms the
    first such pair in shell order, plus the pairs with the largest and the
    smallest Schwarz bound Q_ab."""
    L = [s[1] for s in mol.shells]
    at = [s[0] for s in mol.shells]
    n = len(L)
    pairs = []
    for la in range(3):  # diagonal blocks (a, a)
        a = next((i for i in range(n) if L[i] == la), None)
        if a is not None:
            pairs.append((a, a))
    for la, lb in ((0, 0), (1, 0), (2, 0), (1, 1), (2, 1), (2, 2)):  # two atoms
        hit = next(((a, b) for a in range(n) for b in range(a) if L[a] == la and L[b] == lb and at[a] != at[b]),
                   None)
        if hit is not None:
            pairs.append(hit)
    a, b = np.tril_indices(n)
    q = Q[a * (a + 1) // 2 + b]
    for k in (int(np.argmax(q)), int(np.argmin(q))):
        pairs.append((int(a[k]), int(b[k])))
    out = []
    for p in pairs:
        if p not in out:
            out.append(p)
    return out


def blocks(name):
    mol, opt = synth.config(name)
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    Q = oracle.schwarz(mol)
    pairs = sample_pairs(mol, Q)
    if name == "c240":  # each block sums over a million ket pairs: keep five
        pairs = [pairs[i] for i in (0, 2, 5, 8, len(pairs) - 2)]
    res = oracle.jk_blocks(mol, D, opt["thresh"], pairs, Q=Q)
    _write(f"{name}_blocks.json", {
        "workload": f"{name}: synth.config('{name}'), spherical, D = synth.make_density(mol, "
                    f"{synth.default_nocc(mol, opt['nocc'])}, {opt['dseed']}), thresh {opt['thresh']}",
        "nbf": int(mol.nbf()), "thresh": opt["thresh"],
        "pairs": [list(p) for p in pairs],
        "Q": [float(Q[max(p) * (max(p) + 1) // 2 + min(p)]) for p in pairs],
        "J": [jb.tolist() for jb, _ in res], "K": [kb.tolist() for _, kb in res],
    })


def main(argv):
    what = argv or ["tiny"]
    for w in what:
        if w == "tiny":
            tiny()
        elif w == "small_f3":
            small_f3()
        elif w in ("c60", "c240"):
            blocks(w)
        else:
            raise SystemExit(f"unknown fixture {w}")


if __name__ == "__main__":
    main(sys.argv[1:])
