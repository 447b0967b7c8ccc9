"""GPU nuclear gradient of E_JK against the oracle's analytic gradient,
central finite differences of the GPU energy (h = 1e-4 bohr, <= 1e-6 Eh/bohr)
and the zero net force of translation invariance."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_11185_gb300 import adft, synth

pytestmark = pytest.mark.gpu


def _case(name):
    mol, opt = synth.config(name)
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    return mol, opt, D


_oracle_cache = {}


def _oracle_grad(name, mol, D, thresh):
    if name not in _oracle_cache:
        _oracle_cache[name] = oracle.grad(mol, D, thresh)
    return _oracle_cache[name]


# tiny: classes up to (dd|dd) on the cooperative two-pass kernels; tiny_f adds
# the f classes of the runtime-L kernel; small: 67 functions, many quartets
@pytest.mark.parametrize("name", ["tiny", "tiny_f", "small"])
def test_grad_fp64_vs_oracle(name):
    mol, opt, D = _case(name)
    b = adft.Basis.from_molecule(mol)
    g = adft.adft_jk_grad(b, torch.from_numpy(D).cuda(), thresh=opt["thresh"]).cpu().numpy()
    gr = _oracle_grad(name, mol, D, opt["thresh"])
    print(f"{name}: max|dgrad|={np.max(np.abs(g - gr)):.2e} max|grad|={np.max(np.abs(gr)):.2e} "
          f"net={np.max(np.abs(g.sum(0))):.2e}")
    assert np.max(np.abs(g - gr)) <= 1e-9
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-10 * max(1.0, np.max(np.abs(g)))


GOLDEN_F3 = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "small_f3_grad.json")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grad_small_f3_vs_stored_oracle(precision):
    """f classes with three and four distinct centres: the GPU gradient
    against the oracle's (stored by tests/golden/make_golden.py, which calls
    only the oracle)."""
    ref = json.load(open(GOLDEN_F3))
    mol, opt, D = _case("small_f3")
    assert mol.nbf() == ref["nbf"]
    b = adft.Basis.from_molecule(mol)
    g = adft.adft_jk_grad(b, torch.from_numpy(D).cuda(), thresh=ref["thresh"], precision=precision,
                          split=1e-5).cpu().numpy()
    gr = np.array(ref["grad"])
    err = np.max(np.abs(g - gr))
    print(f"small_f3 {precision}: max|dgrad|={err:.2e} max|grad|={np.max(np.abs(gr)):.2e} "
          f"net={np.max(np.abs(g.sum(0))):.2e}")
    assert err <= (1e-9 if precision == "fp64" else 1e-5)
    assert np.max(np.abs(g.sum(axis=0))) <= (1e-10 if precision == "fp64" else 1e-7) * max(1.0, np.max(np.abs(g)))


def test_grad_vs_finite_differences_of_gpu_energy():
    mol, opt, D = _case("small")
    Dt = torch.from_numpy(D).cuda()
    b = adft.Basis.from_molecule(mol)
    g = adft.adft_jk_grad(b, Dt, thresh=opt["thresh"]).cpu().numpy()
    h = 1e-4
    rng = np.random.default_rng(4)
    coords = [(int(rng.integers(mol.natom)), int(rng.integers(3))) for _ in range(6)]
    for a, k in coords:
        e = []
        for sgn in (1, -1):
            x = mol.atoms.copy()
            x[a, k] += sgn * h
            bb = adft.Basis.from_molecule(mol.with_atoms(x))
            e.append(adft.adft_jk_energy(bb, Dt, thresh=opt["thresh"]))
        fd = (e[0] - e[1]) / (2 * h)
        assert abs(fd - g[a, k]) <= 1e-6, (a, k, fd, g[a, k])
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-10 * max(1.0, np.max(np.abs(g)))


def test_grad_mixed_error_reported():
    mol, opt, D = _case("small")
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    g64 = adft.adft_jk_grad(b, Dt, thresh=opt["thresh"]).cpu().numpy()
    gmx = adft.adft_jk_grad(b, Dt, thresh=opt["thresh"], precision="mixed", split=1e-5).cpu().numpy()
    err = np.max(np.abs(gmx - g64))
    err_o = np.max(np.abs(gmx - _oracle_grad("small", mol, D, opt["thresh"])))
    print(f"mixed gradient: max|grad_mixed - grad_fp64| = {err:.2e}, vs oracle {err_o:.2e}")
    assert err <= 1e-5 and err_o <= 1e-5


def test_autograd_energy_backward_matches_gradient_kernel_and_oracle():
    mol, opt, D = _case("tiny")
    Dt = torch.from_numpy(D).cuda()
    coords = torch.tensor(mol.atoms, dtype=torch.float64, requires_grad=True)
    E = adft.jk_energy(Dt, coords, mol.shells, mol.spherical, thresh=opt["thresh"])
    E.backward()
    b = adft.Basis.from_molecule(mol)
    g_kernel = adft.adft_jk_grad(b, Dt, thresh=opt["thresh"]).cpu().numpy()
    g_oracle = _oracle_grad("tiny", mol, D, opt["thresh"])
    assert coords.grad is not None and coords.grad.shape == (mol.natom, 3)
    assert abs(E.item() - adft.adft_jk_energy(b, Dt, thresh=opt["thresh"])) <= 1e-12 * abs(E.item())
    # same kernels; only the order of the FP64 atomic additions may differ
    assert np.max(np.abs(coords.grad.numpy() - g_kernel)) <= 1e-12 * np.max(np.abs(g_kernel))
    assert np.max(np.abs(coords.grad.numpy() - g_oracle)) <= 1e-9
    # chain rule through a scaled loss
    coords.grad = None
    (3.0 * adft.jk_energy(Dt, coords, mol.shells, mol.spherical, thresh=opt["thresh"])).backward()
    assert np.max(np.abs(coords.grad.numpy() - 3.0 * g_kernel)) <= 3e-12 * np.max(np.abs(g_kernel))
