"""GPU checks at the 60-atom size (24 heavy 3s2p1d + 36 H 2s1p, 516 spherical
functions, thresh 1e-10), where the oracle cannot build all of J and K:

* sampled J and K blocks against the oracle's (tests/golden/c60_blocks.json,
  written by tests/golden/make_golden.py, which calls only the oracle): the
  blocks cover s, p and d shells on one and on two atoms and the shell pairs
  with the largest and the smallest Schwarz bound;
* the nuclear gradient against central finite differences of the GPU energy
  (h = 1e-4 bohr) on 12 seeded coordinates, and the zero net force, in FP64
  and in mixed precision.

The builds run in the launch configuration the benchmark uses (autotuned
launch shapes).
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_11185_gb300 import adft, synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c60_blocks.json")


@pytest.fixture(scope="module")
def c60():
    mol, opt = synth.config("c60")
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    return mol, opt, D, b, Dt


def _blocks_err(mol, J, K, ref):
    sl = []
    o = 0
    for _, l, _, _ in mol.shells:
        sl.append(slice(o, o + 2 * l + 1))
        o += 2 * l + 1
    Jc, Kc = J.cpu().numpy(), K.cpu().numpy()
    ej, ek = [], []
    for (a, b), Jb, Kb in zip(ref["pairs"], ref["J"], ref["K"]):
        ej.append(np.max(np.abs(Jc[sl[a], sl[b]] - np.array(Jb))))
        ek.append(np.max(np.abs(Kc[sl[a], sl[b]] - np.array(Kb))))
    return np.array(ej), np.array(ek)


@pytest.mark.parametrize("precision,split", [("fp64", 0.0), ("mixed", 1e-5), ("mixed", 1e-3)])
def test_sampled_blocks_vs_stored_oracle(c60, precision, split):
    mol, opt, D, b, Dt = c60
    ref = json.load(open(GOLDEN))
    assert mol.nbf() == ref["nbf"] and ref["thresh"] == opt["thresh"]
    adft.adft_autotune(b, Dt, thresh=opt["thresh"], split=split, precision=precision)
    J, K = adft.adft_jk_build(b, Dt, thresh=opt["thresh"], split=split, precision=precision)
    ej, ek = _blocks_err(mol, J, K, ref)
    print(f"c60 {precision} split={split}: per block max|dJ| {np.array2string(ej, precision=1)} "
          f"max|dK| {np.array2string(ek, precision=1)}")
    if precision == "fp64":
        assert ej.max() <= 1e-10 and ek.max() <= 1e-10
    else:
        assert ej.max() <= 1e-6 and ek.max() <= 1e-6


def test_gradient_vs_finite_differences(c60):
    """Config 4: the FP64 and the mixed gradient against central finite
    differences of the FP64 GPU energy at fixed D (h = 1e-4 bohr) on 12
    seeded coordinates (<= 1e-6 Eh/bohr for FP64), and zero net force."""
    mol, opt, D, b, Dt = c60
    th = opt["thresh"]
    g64 = adft.adft_jk_grad(b, Dt, thresh=th, precision="fp64").cpu().numpy()
    gmx = adft.adft_jk_grad(b, Dt, thresh=th, precision="mixed", split=1e-5).cpu().numpy()
    rng = np.random.default_rng(60)
    picks = rng.choice(mol.natom * 3, size=12, replace=False)
    h = 1e-4
    fd = []
    for p in picks:
        a, k = divmod(int(p), 3)
        e = []
        for sgn in (1, -1):
            x = mol.atoms.copy()
            x[a, k] += sgn * h
            bb = adft.Basis.from_molecule(mol.with_atoms(x))
            e.append(adft.adft_jk_energy(bb, Dt, thresh=th, precision="fp64"))
            bb.close()
        fd.append((e[0] - e[1]) / (2 * h))
    fd = np.array(fd)
    e64 = np.max(np.abs(g64.reshape(-1)[picks] - fd))
    emx = np.max(np.abs(gmx.reshape(-1)[picks] - fd))
    net64 = np.max(np.abs(g64.sum(0)))
    netmx = np.max(np.abs(gmx.sum(0)))
    print(f"c60 gradient vs FD on 12 coordinates: fp64 {e64:.2e}, mixed {emx:.2e}; max|grad| "
          f"{np.max(np.abs(g64)):.2e}; net force fp64 {net64:.2e} mixed {netmx:.2e}; "
          f"max|g_mixed - g_fp64| {np.max(np.abs(gmx - g64)):.2e}")
    assert e64 <= 1e-6
    assert emx <= 1e-5
    assert net64 <= 1e-10 * max(1.0, np.max(np.abs(g64)))
    assert netmx <= 1e-7 * max(1.0, np.max(np.abs(gmx)))
