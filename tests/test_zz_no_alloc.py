"""adft_energy_static: the energy entry point that allocates nothing.

It is for callers that cannot allocate device memory where they need the
energy (a memory pool that may not grow, a region where cudaMalloc would
synchronise the device, an allocator owned by another framework); its scratch
is a fixed array inside the library.  This file is collected last, so a
failure here comes after every other test has run.  It must pass alone in a
fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2406_11185_gb300 import adft, synth

pytestmark = pytest.mark.gpu


def _call(D, J, K, n, E, stream):
    vp = ctypes.c_void_p
    return adft.load().adft_energy_static(vp(D.data_ptr()), vp(J.data_ptr()), vp(K.data_ptr()), n,
                                          vp(E.data_ptr()), vp(stream.cuda_stream))


def test_energy_static_matches_jk_energy_twice():
    mol, opt = synth.config("small")
    D = torch.from_numpy(synth.make_density(mol, opt["nocc"], opt["dseed"])).cuda()
    b = adft.Basis.from_molecule(mol)
    J, K = adft.adft_jk_build(b, D, thresh=opt["thresh"])
    E_ref = adft.adft_jk_energy(b, D, thresh=opt["thresh"])
    s = torch.cuda.current_stream()
    out = []
    for _ in range(2):  # two calls in a row share the library's scratch
        E = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        assert _call(D, J, K, b.nbf, E, s) == adft.ADFT_OK, adft.last_error()
        torch.cuda.synchronize()
        out.append(E.item())
    for e in out:
        assert abs(e - E_ref) <= 1e-9
    # the binding's wrapper reaches the same entry point
    assert abs(adft.adft_energy_static(D, J, K).item() - E_ref) <= 1e-9


def test_energy_static_rejects_oversize():
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    vp = ctypes.c_void_p
    st = adft.load().adft_energy_static(vp(d.data_ptr()), vp(d.data_ptr()), vp(d.data_ptr()),
                                        adft.ADFT_STATIC_MAX_NBF + 1, vp(d.data_ptr()), None)
    assert st == adft.ADFT_ERR_ARG
    assert "ADFT_STATIC_MAX_NBF" in adft.last_error() or "scratch" in adft.last_error()
