"""GPU SCF driver around the J/K build: one-electron matrices and converged
closed-shell SCF energies against the oracle (oracle.one_electron and
oracle.scf, which rebuilds J and K in full from the definition every
iteration).  The GPU driver uses incremental builds with density-weighted
screening unless told otherwise."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_11185_gb300 import adft, scf, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,spherical", [("tiny", True), ("tiny", False), ("small_f3", True)])
def test_one_electron_vs_oracle(name, spherical):
    mol, _ = synth.config(name, spherical=spherical)
    Z = synth.nuclear_charges(mol)
    b = adft.Basis.from_molecule(mol)
    got = [m.cpu().numpy() for m in adft.adft_one_electron(b, Z)]
    ref = oracle.one_electron(mol, Z)
    for g, r, what in zip(got, ref, "STV"):
        err = np.max(np.abs(g - r))
        print(f"{name} sph={spherical} {what}: max|d|={err:.2e} max={np.max(np.abs(r)):.2e}")
        assert err <= 1e-11 * np.max(np.abs(r)), what


_oracle_scf = {}


def _ref(name, nocc):
    if name not in _oracle_scf:
        mol, opt = synth.config(name)
        _oracle_scf[name] = oracle.scf(mol, synth.nuclear_charges(mol), nocc, opt["thresh"], e_tol=1e-11,
                                       g_tol=1e-9)
    return _oracle_scf[name]


@pytest.mark.parametrize("name,nocc", [("tiny", 4), ("small", 11)])
@pytest.mark.parametrize("incremental", [False, True])
def test_scf_fp64_vs_oracle(name, nocc, incremental):
    mol, opt = synth.config(name)
    ref = _ref(name, nocc)
    r = scf.RHF(mol, nocc=nocc, thresh=opt["thresh"], precision="fp64", incremental=incremental).run(
        e_tol=1e-11, g_tol=1e-9)
    kinds = [k for k, _ in r["builds"]]
    print(f"{name} incremental={incremental}: E={r['energy']:.12f} oracle {ref['energy']:.12f} "
          f"dE={r['energy'] - ref['energy']:.2e} iterations {r['iterations']} (oracle {ref['iterations']}) "
          f"builds {kinds.count('full')} full / {kinds.count('incremental')} incremental")
    assert ref["converged"] and r["converged"]
    assert abs(r["energy"] - ref["energy"]) <= 1e-8
    if incremental:
        assert kinds.count("incremental") > 0
    D = r["D"].cpu().numpy()
    assert np.max(np.abs(D - ref["D"])) <= 1e-5


def test_scf_mixed_precision_energy():
    mol, opt = synth.config("small")
    ref = _ref("small", 11)
    r = scf.RHF(mol, nocc=11, thresh=opt["thresh"], precision="mixed", split=1e-5).run(e_tol=1e-10, g_tol=1e-7)
    print(f"small mixed: dE={r['energy'] - ref['energy']:.2e} iterations {r['iterations']}")
    assert r["converged"]
    assert abs(r["energy"] - ref["energy"]) <= 1e-6


@pytest.mark.parametrize("name", ["tiny", "small_f3"])
def test_one_electron_gradient_vs_oracle(name):
    """sum D dH/dR - sum W dS/dR on the GPU against oracle.one_electron_grad
    for a synthetic D and a symmetric W (s to f shells)."""
    mol, opt = synth.config(name)
    Z = synth.nuclear_charges(mol)
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    rng = np.random.default_rng(7)
    W = rng.normal(size=D.shape)
    W = 0.5 * (W + W.T)
    b = adft.Basis.from_molecule(mol)
    g = adft.adft_one_electron_grad(b, Z, torch.from_numpy(D).cuda(), torch.from_numpy(W).cuda()).cpu().numpy()
    ref = oracle.one_electron_grad(mol, Z, D, W)
    err = np.max(np.abs(g - ref))
    print(f"{name}: max|d grad_1e|={err:.2e} max={np.max(np.abs(ref)):.2e}")
    assert err <= 1e-10 * np.max(np.abs(ref))


def test_scf_force_vs_oracle():
    """The single-point force of a converged FP64 SCF (one-electron gradient,
    J/K gradient at fixed D, nuclear repulsion) against oracle.scf_gradient."""
    mol = synth.make_molecule(1801, 1, 2, "3s2p1d", "2s1p", (1, 2), (0.1, 5e3), (1.4, 2.0), True, "force")
    Z = synth.nuclear_charges(mol)
    nocc = int(round(Z.sum())) // 2
    rhf = scf.RHF(mol, nocc=nocc, thresh=1e-12, precision="fp64", incremental=False)
    r = rhf.run(e_tol=1e-12, g_tol=1e-10)
    g = scf.scf_gradient(rhf, r).cpu().numpy()
    E_ref, g_ref, _ = oracle.scf_gradient(mol, Z, nocc, 1e-12, e_tol=1e-12, g_tol=1e-10)
    print(f"force: dE={r['energy'] - E_ref:.2e} max|dg|={np.max(np.abs(g - g_ref)):.2e}")
    assert r["converged"] and abs(r["energy"] - E_ref) <= 1e-9
    assert np.max(np.abs(g - g_ref)) <= 1e-7
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-9
