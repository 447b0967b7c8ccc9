"""GPU parity: the CUDA library through the C ABI against the CPU oracle,
element by element, on seeded synthetic molecules.

Tolerances: FP64 path max|dJ|, max|dK| <= 1e-10 and |dE| <= 1e-9 Eh; mixed
FP32/FP64 path |dE| <= 1e-6 Eh (its J/K errors are reported and bounded
loosely).  Quartets whose bound lies within round-off of the threshold may be
kept by one side and dropped by the other; their contribution is below
thresh * max|D| per element, far inside the tolerances.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_2406_11185_gb300 import adft, parallel, synth

pytestmark = pytest.mark.gpu

TOL_JK = 1e-10
TOL_E = 1e-9
TOL_E_MIXED = 1e-6


def _case(name, spherical=True, nocc=None):
    mol, opt = synth.config(name, spherical=spherical)
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"] if nocc is None else nocc), opt["dseed"])
    return mol, opt, D


_ref_cache = {}


def _oracle_jk(name, spherical, mol, D, thresh):
    key = (name, spherical, thresh)
    if key not in _ref_cache:
        J, K = oracle.jk(mol, D, thresh)
        _ref_cache[key] = (J, K, oracle.energy(D, J, K))
    return _ref_cache[key]


def _gpu_jk(mol, D, thresh, precision="fp64", split=1e-5):
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    J, K = adft.adft_jk_build(b, Dt, thresh=thresh, split=split, precision=precision)
    E = adft.adft_jk_energy(b, Dt, thresh=thresh, split=split, precision=precision)
    st = adft.adft_jk_last_stats(b)
    return J.cpu().numpy(), K.cpu().numpy(), E, st, b


# small_f3: f shells on two heavy atoms and d shells on three H atoms, so f
# classes with three and four distinct centres are covered
@pytest.mark.parametrize("name,spherical", [("tiny", True), ("tiny", False), ("small", True), ("tiny_f", True),
                                            ("tiny_f", False), ("small_f3", True), ("small_f3", False)])
def test_fp64_parity(name, spherical):
    mol, opt, D = _case(name, spherical)
    Jr, Kr, Er = _oracle_jk(name, spherical, mol, D, opt["thresh"])
    J, K, E, st, _ = _gpu_jk(mol, D, opt["thresh"])
    dj, dk = np.max(np.abs(J - Jr)), np.max(np.abs(K - Kr))
    print(f"{name} sph={spherical}: max|dJ|={dj:.2e} max|dK|={dk:.2e} |dE|={abs(E - Er):.2e} stats={st}")
    assert dj <= TOL_JK and dk <= TOL_JK
    assert abs(E - Er) <= TOL_E
    assert st["quartets_fp32"] == 0 and st["quartets_fp64"] > 0


@pytest.mark.parametrize("name,split", [("tiny_f", 1e-5), ("small", 1e-5), ("small", 1e-7), ("small_f3", 1e-5),
                                        ("small_f3", 1e-3)])
def test_mixed_precision_energy(name, split):
    mol, opt, D = _case(name)
    Jr, Kr, Er = _oracle_jk(name, True, mol, D, opt["thresh"])
    J, K, E, st, _ = _gpu_jk(mol, D, opt["thresh"], precision="mixed", split=split)
    dj, dk = np.max(np.abs(J - Jr)), np.max(np.abs(K - Kr))
    print(f"{name} split={split}: max|dJ|={dj:.2e} max|dK|={dk:.2e} |dE|={abs(E - Er):.2e} "
          f"fp64={st['quartets_fp64']} fp32={st['quartets_fp32']}")
    assert st["quartets_fp32"] > 0
    assert abs(E - Er) <= TOL_E_MIXED
    assert dj <= 1e-5 and dk <= 1e-5


def _variant_pairs(b, variant):
    """Class pairs X(X+1)/2 + Y of each band (0 FP64, 1 FP32) with a kernel
    variant `variant`: adft_set_tuning rejects a variant past a pair's count.
    The d-class pairs list their kernels as: the warp and the cooperative
    kernel (where both serve the pair; the cooperative one alone otherwise),
    then the row-blocked kernel with its busiest shape and with its
    occupancy-aware shape (where each plan fits and the two differ).  So
    variants 1-3 together cover every kernel but the default one."""
    found = {0: [], 1: []}
    for band in (0, 1):
        for cp in range(55):
            tab = np.full((2, 55), 2, dtype=np.int32)
            tab[band, cp] += variant * adft.TUNE_VARIANT_STRIDE
            try:
                adft.adft_set_tuning(b, tab)
                found[band].append(cp)
            except adft.AdftError:
                pass
    return found


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_alternative_kernel_variant_parity(variant, precision):
    mol, opt, D = _case("small")
    Jr, Kr, Er = _oracle_jk("small", True, mol, D, opt["thresh"])
    b = adft.Basis.from_molecule(mol)
    pairs = _variant_pairs(b, variant)
    # (dp|pp), (dp|ds), (dp|dp) have at least three kernels in both bands,
    # every d-class pair up to (dd|dp) at least two, and (dp|pp), (dp|dp)
    # four (both row-kernel shapes)
    if variant <= 2:
        assert {12, 13, 14} <= set(pairs[0]) and {12, 13, 14} <= set(pairs[1]), pairs
    if variant == 1:
        assert {19} <= set(pairs[0]) and {19} <= set(pairs[1]), pairs
    if variant == 3:
        assert {12, 14} <= set(pairs[0]) and {12, 14} <= set(pairs[1]), pairs
    tab = np.full((2, 55), 2, dtype=np.int32)
    for band in (0, 1):
        tab[band, pairs[band]] += variant * adft.TUNE_VARIANT_STRIDE
    adft.adft_set_tuning(b, tab)
    Dt = torch.from_numpy(D).cuda()
    J, K = adft.adft_jk_build(b, Dt, thresh=opt["thresh"], precision=precision)
    E = adft.adft_jk_energy(b, Dt, thresh=opt["thresh"], precision=precision)
    dj = np.max(np.abs(J.cpu().numpy() - Jr))
    dk = np.max(np.abs(K.cpu().numpy() - Kr))
    print(f"variant {variant} on {pairs} {precision}: max|dJ|={dj:.2e} max|dK|={dk:.2e} |dE|={abs(E - Er):.2e}")
    if precision == "fp64":
        assert dj <= TOL_JK and dk <= TOL_JK and abs(E - Er) <= TOL_E
    else:
        assert abs(E - Er) <= TOL_E_MIXED and dj <= 1e-5 and dk <= 1e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_primitive_screening_counts(precision):
    """A build reports the primitive quartets its kernels evaluated (after
    primitive-quartet screening); the plan reports the unscreened count."""
    mol, opt, D = _case("small")
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    adft.adft_jk_build(b, Dt, thresh=opt["thresh"], precision=precision)
    st = adft.adft_jk_last_stats(b)
    plan, _ = adft.adft_jk_plan(b, Dt, thresh=opt["thresh"], precision=precision)
    print(f"{precision}: evaluated {st} planned {plan}")
    for k in ("quartets_fp64", "quartets_fp32", "quartets_total"):
        assert st[k] == plan[k]
    for band in ("fp64", "fp32"):
        assert st[f"prim_quartets_{band}"] <= plan[f"prim_quartets_{band}"]
        assert st[f"flops_{band}"] <= plan[f"flops_{band}"] * (1 + 1e-9)
    assert st["prim_quartets_fp64"] > 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_class_pair_masks_sum_to_full_build(precision):
    """The sharded build: partial J, K, E and gradient over class-pair masks
    that partition the launches (3 ranks, assigned by measured kernel times)
    add up to the full build.  The ranks run one after the other on one GPU;
    no kernel waits on another."""
    mol, opt, D = _case("small")
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    kw = dict(thresh=opt["thresh"], split=1e-5, precision=precision)
    J, K = adft.adft_jk_build(b, Dt, **kw)
    E = adft.adft_jk_energy(b, Dt, **kw)
    g = adft.adft_jk_grad(b, Dt, **kw)
    _, ms = adft.adft_autotune(b, Dt, return_times=True, **kw)
    masks = parallel.assign_class_pairs(ms, 3)
    assert masks.sum() == np.count_nonzero(ms)
    Js, Ks, Es, gs = torch.zeros_like(J), torch.zeros_like(K), 0.0, torch.zeros_like(g)
    for m in masks:
        Jp, Kp = adft.adft_jk_build(b, Dt, pair_mask=m, **kw)
        Js += Jp
        Ks += Kp
        Es += adft.adft_jk_energy(b, Dt, pair_mask=m, **kw)
        gs += adft.adft_jk_grad(b, Dt, pair_mask=m, **kw)
    scale = torch.max(torch.abs(J)).item()
    assert torch.max(torch.abs(Js - J)).item() <= 1e-12 * scale
    assert torch.max(torch.abs(Ks - K)).item() <= 1e-12 * scale
    assert abs(Es - E) <= 1e-11 * abs(E)
    assert torch.max(torch.abs(gs - g)).item() <= 1e-11 * max(1.0, torch.max(torch.abs(g)).item())
    # an empty mask evaluates nothing
    J0, K0 = adft.adft_jk_build(b, Dt, pair_mask=np.zeros((2, 55), np.uint8), **kw)
    assert torch.count_nonzero(J0).item() == 0 and torch.count_nonzero(K0).item() == 0


def test_schwarz_bounds_match_oracle():
    mol, opt, D = _case("tiny_f")
    b = adft.Basis.from_molecule(mol)
    Qg = b.schwarz()
    Qr = oracle.schwarz(mol)
    assert np.max(np.abs(Qg - Qr) / np.maximum(Qr, 1e-300)) <= 1e-11


def test_screening_threshold_consistency():
    mol, opt, D = _case("small")
    Q = oracle.schwarz(mol)
    thr = float(np.quantile(np.outer(Q, Q), 0.5))
    Jr, Kr = oracle.jk(mol, D, thr, Q=Q)
    J, K, E, st, _ = _gpu_jk(mol, D, thr)
    npair = len(Q)
    assert 0 < st["quartets_fp64"] < npair * (npair + 1) // 2
    assert np.max(np.abs(J - Jr)) <= TOL_JK + thr * np.max(np.abs(D)) * 10
    assert np.max(np.abs(K - Kr)) <= TOL_JK + thr * np.max(np.abs(D)) * 10


def test_repeatability_and_symmetry():
    mol, opt, D = _case("small")
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    runs = [adft.adft_jk_build(b, Dt, thresh=opt["thresh"]) for _ in range(4)]
    J0, K0 = (x.cpu().numpy() for x in runs[0])
    for J, K in runs[1:]:
        assert np.max(np.abs(J.cpu().numpy() - J0)) <= 1e-13 * np.max(np.abs(J0))
        assert np.max(np.abs(K.cpu().numpy() - K0)) <= 1e-13 * np.max(np.abs(K0))
    assert np.max(np.abs(J0 - J0.T)) <= 1e-14 * np.max(np.abs(J0))
    assert np.max(np.abs(K0 - K0.T)) <= 1e-14 * np.max(np.abs(K0))


def test_bad_density_rejected():
    mol, opt, D = _case("tiny")
    b = adft.Basis.from_molecule(mol)
    A = D.copy()
    A[0, 1] += 1e-3
    with pytest.raises(adft.AdftError) as e:
        adft.adft_jk_build(b, torch.from_numpy(A).cuda(), thresh=opt["thresh"])
    assert e.value.status == adft.ADFT_ERR_ASYM_D
    A = D.copy()
    A[2, 2] = np.nan
    with pytest.raises(adft.AdftError) as e:
        adft.adft_jk_build(b, torch.from_numpy(A).cuda(), thresh=opt["thresh"])
    assert e.value.status == adft.ADFT_ERR_NONFINITE
    with pytest.raises(ValueError):
        adft.adft_jk_build(b, torch.from_numpy(D[:-1, :-1].copy()).cuda())
    # the handle still works afterwards
    J, K = adft.adft_jk_build(b, torch.from_numpy(D).cuda(), thresh=opt["thresh"])
    Jr, Kr, _ = _oracle_jk("tiny", True, mol, D, opt["thresh"])
    assert np.max(np.abs(J.cpu().numpy() - Jr)) <= TOL_JK


def test_abort_flag_reported():
    mol, opt, D = _case("tiny")
    b = adft.Basis.from_molecule(mol)
    Dt = torch.from_numpy(D).cuda()
    adft.adft_basis_set_abort(b, True)
    with pytest.raises(adft.AdftError) as e:
        adft.adft_jk_build(b, Dt, thresh=opt["thresh"])
    assert e.value.status == adft.ADFT_ERR_ABORTED
    adft.adft_basis_set_abort(b, False)
    J, K = adft.adft_jk_build(b, Dt, thresh=opt["thresh"])
    assert adft.adft_jk_status(b) == 0

