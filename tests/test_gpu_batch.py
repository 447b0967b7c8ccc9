"""Batched form: many molecules through one persistent launch per class pair
(and a captured CUDA graph), checked against the CPU oracle on small
molecules and against the single-molecule GPU path on larger ones."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_11185_gb300 import adft, synth

pytestmark = pytest.mark.gpu


def _small_batch():
    mols = []
    for i, (nh, nl) in enumerate([(1, 2), (2, 3), (1, 1), (3, 4)]):
        mols.append(synth.make_molecule(7100 + i, nh, nl, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3), (1.9, 2.9)))
    Ds = [synth.make_density(m, max(1, m.nbf() // 5), 7200 + i) for i, m in enumerate(mols)]
    return mols, Ds


def test_batch_vs_oracle():
    mols, Ds = _small_batch()
    thresh = 1e-12
    bases = [adft.Basis.from_molecule(m) for m in mols]
    bt = adft.Batch(bases)
    Dp = bt.pack([torch.from_numpy(D).cuda() for D in Ds])
    J, K, E, G = adft.adft_batch_jk(bt, Dp, thresh=thresh, precision="fp64", check=True, grad=True)
    Js, Ks = bt.unpack(J), bt.unpack(K)
    for i, (m, D) in enumerate(zip(mols, Ds)):
        Jr, Kr = oracle.jk(m, D, thresh)
        assert np.max(np.abs(Js[i].cpu().numpy() - Jr)) <= 1e-10
        assert np.max(np.abs(Ks[i].cpu().numpy() - Kr)) <= 1e-10
        assert abs(E[i].item() - oracle.energy(D, Jr, Kr)) <= 1e-9
        g = G[bt.grad_offsets[i]:bt.grad_offsets[i + 1]].reshape(-1, 3).cpu().numpy()
        gr = oracle.grad(m, D, thresh)
        assert np.max(np.abs(g - gr)) <= 1e-9


def test_batch_matches_single_molecule_path_and_graph_replay():
    mols = sorted(synth.batch_molecules(6, base_seed=5000), key=lambda m: m.natom)[:3]
    Ds = [synth.make_density(m, synth.default_nocc(m, None), 9000 + i) for i, m in enumerate(mols)]
    thresh, split = 1e-10, 1e-5
    bases = [adft.Basis.from_molecule(m) for m in mols]
    bt = adft.Batch(bases)
    Dt = [torch.from_numpy(D).cuda() for D in Ds]
    Dp = bt.pack(Dt)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r1 = adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed", check=False, grad=True)
        out = tuple(x.clone() for x in r1)
        r2 = adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed", check=False, grad=True,
                                out=r1)  # graph replay into the same buffers
    s.synchronize()
    for a, b in zip(out, r2):
        assert torch.max(torch.abs(a - b)).item() <= 1e-12 * max(1.0, torch.max(torch.abs(a)).item())
    Js, Ks = bt.unpack(r2[0]), bt.unpack(r2[1])
    for i, (b, D) in enumerate(zip(bases, Dt)):
        J, K = adft.adft_jk_build(b, D, thresh=thresh, split=split, precision="mixed")
        e = adft.adft_jk_energy(b, D, thresh=thresh, split=split, precision="mixed")
        g = adft.adft_jk_grad(b, D, thresh=thresh, split=split, precision="mixed")
        assert torch.max(torch.abs(Js[i] - J)).item() <= 1e-9
        assert torch.max(torch.abs(Ks[i] - K)).item() <= 1e-9
        assert abs(r2[2][i].item() - e) <= 1e-9
        gb = r2[3][bt.grad_offsets[i]:bt.grad_offsets[i + 1]].reshape(-1, 3)
        assert torch.max(torch.abs(gb - g)).item() <= 1e-8


def test_autotune_keeps_results():
    mol, opt = synth.config("small")
    D = torch.from_numpy(synth.make_density(mol, opt["nocc"], opt["dseed"])).cuda()
    b = adft.Basis.from_molecule(mol)
    J0, K0 = adft.adft_jk_build(b, D, thresh=opt["thresh"], precision="mixed")
    tab = adft.adft_autotune(b, D, thresh=opt["thresh"], precision="mixed")
    blocks, variant = tab % adft.TUNE_VARIANT_STRIDE, tab // adft.TUNE_VARIANT_STRIDE
    assert tab.shape == (2, 55) and np.all((blocks >= 1) & (blocks <= 8)) and np.all((variant >= 0) & (variant <= 3))
    J1, K1 = adft.adft_jk_build(b, D, thresh=opt["thresh"], precision="mixed")
    assert torch.max(torch.abs(J1 - J0)).item() <= 1e-12 * torch.max(torch.abs(J0)).item()
    assert torch.max(torch.abs(K1 - K0)).item() <= 1e-12 * torch.max(torch.abs(K0)).item()


def test_batch_tuning_from_sub_batch():
    """A table tuned on a sub-batch, installed with adft_batch_set_tuning,
    drops the captured graph and leaves the results unchanged."""
    mols, Ds = _small_batch()
    thresh, split = 1e-10, 1e-5
    bases = [adft.Basis.from_molecule(m) for m in mols]
    bt = adft.Batch(bases)
    Dt = [torch.from_numpy(D).cuda() for D in Ds]
    Dp = bt.pack(Dt)
    r0 = tuple(x.clone() for x in adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed",
                                                      grad=True))
    sub = adft.Batch(bases[:2])
    tab = adft.adft_batch_autotune(sub, sub.pack(Dt[:2]), thresh=thresh, split=split, precision="mixed")
    adft.adft_batch_set_tuning(bt, tab)
    bad = tab.copy()
    bad[0, 0] = 0  # zero blocks per SM
    with pytest.raises(adft.AdftError):
        adft.adft_batch_set_tuning(bt, bad)
    r1 = adft.adft_batch_jk(bt, Dp, thresh=thresh, split=split, precision="mixed", grad=True)
    for a, b in zip(r0, r1):
        assert torch.max(torch.abs(a - b)).item() <= 1e-11 * max(1.0, torch.max(torch.abs(a)).item())
