"""Edge cases of the GPU path against the oracle: zero density, a threshold
that screens out every quartet, a single atom (zero gradient), an s-only
basis (the (ss|ss) class alone) and shells at the maximum primitive count."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_11185_gb300 import adft, synth

pytestmark = pytest.mark.gpu

TOL_JK = 1e-10
TOL_GRAD = 1e-9
THRESH = 1e-12


def _edge_molecule(kind):
    if kind == "single_atom":  # one heavy atom 3s2p1d: every pair on one centre
        return synth.make_molecule(8101, 1, 0, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3), (1.9, 2.9))
    if kind == "s_only":  # 2 heavy (2s) + 2 H (1s): the (ss|ss) class alone
        return synth.make_molecule(8102, 2, 2, "2s", "1s", (1, 6), (0.1, 5e3), (1.4, 2.0))
    if kind == "max_prims":  # every shell at the largest primitive count the boundary accepts
        return synth.make_molecule(8103, 1, 1, "1s1p", "1s", (adft.ADFT_MAX_NPRIM, adft.ADFT_MAX_NPRIM),
                                   (0.05, 1e4), (1.4, 2.0))
    raise KeyError(kind)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_zero_density_gives_zero(precision):
    mol, opt = synth.config("tiny")
    b = adft.Basis.from_molecule(mol)
    Z = torch.zeros(b.nbf, b.nbf, dtype=torch.float64, device="cuda")
    J, K = adft.adft_jk_build(b, Z, thresh=opt["thresh"], precision=precision)
    assert torch.count_nonzero(J).item() == 0 and torch.count_nonzero(K).item() == 0
    assert adft.adft_jk_energy(b, Z, thresh=opt["thresh"], precision=precision) == 0.0
    g = adft.adft_jk_grad(b, Z, thresh=opt["thresh"], precision=precision)
    assert torch.count_nonzero(g).item() == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_everything_screened_out(precision):
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    thresh = 1e6  # above every Q_ab Q_cd
    assert float(np.max(b.schwarz())) ** 2 < thresh
    J, K = adft.adft_jk_build(b, Dt, thresh=thresh, precision=precision)
    st = adft.adft_jk_last_stats(b)
    assert st["quartets_fp64"] == 0 and st["quartets_fp32"] == 0 and st["quartets_total"] > 0
    assert st["prim_quartets_fp64"] == 0 and st["flops_fp64"] == 0.0
    assert torch.count_nonzero(J).item() == 0 and torch.count_nonzero(K).item() == 0
    g = adft.adft_jk_grad(b, Dt, thresh=thresh, precision=precision)
    assert torch.count_nonzero(g).item() == 0
    # the handle works normally afterwards
    J, K = adft.adft_jk_build(b, Dt, thresh=opt["thresh"], precision="fp64")
    Jr, Kr = oracle.jk(mol, D, opt["thresh"])
    assert np.max(np.abs(J.cpu().numpy() - Jr)) <= TOL_JK


@pytest.mark.parametrize("kind", ["single_atom", "s_only", "max_prims"])
def test_edge_molecules_vs_oracle(kind):
    mol = _edge_molecule(kind)
    D = synth.make_density(mol, max(1, mol.nbf() // 5), 5)
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    J, K = adft.adft_jk_build(b, Dt, thresh=THRESH, precision="fp64")
    Jr, Kr = oracle.jk(mol, D, THRESH)
    dj = np.max(np.abs(J.cpu().numpy() - Jr))
    dk = np.max(np.abs(K.cpu().numpy() - Kr))
    E = adft.adft_jk_energy(b, Dt, thresh=THRESH, precision="fp64")
    g = adft.adft_jk_grad(b, Dt, thresh=THRESH, precision="fp64").cpu().numpy()
    gr = oracle.grad(mol, D, THRESH)
    print(f"{kind}: nbf={mol.nbf()} max|dJ|={dj:.2e} max|dK|={dk:.2e} max|dgrad|={np.max(np.abs(g - gr)):.2e} "
          f"max|grad|={np.max(np.abs(g)):.2e}")
    assert dj <= TOL_JK and dk <= TOL_JK
    assert abs(E - oracle.energy(D, Jr, Kr)) <= 1e-9
    assert np.max(np.abs(g - gr)) <= TOL_GRAD
    if kind == "single_atom":  # the energy cannot depend on the position of a lone atom
        assert np.max(np.abs(g)) <= 1e-10


def test_threshold_below_primitive_drop_rejected():
    """Primitive pairs with bound products <= 1e-15 are dropped when the basis
    is created, so a threshold below 1e-12 (or 0) is refused, not silently
    approximated."""
    mol, opt = synth.config("tiny")
    D = torch.from_numpy(synth.make_density(mol, opt["nocc"], opt["dseed"])).cuda()
    b = adft.Basis.from_molecule(mol)
    for thr in (0.0, 1e-13):
        with pytest.raises(adft.AdftError) as e:
            adft.adft_jk_build(b, D, thresh=thr)
        assert e.value.status == adft.ADFT_ERR_ARG and "1e-12" in str(e.value)
    adft.adft_jk_build(b, D, thresh=1e-12)  # the smallest accepted threshold
