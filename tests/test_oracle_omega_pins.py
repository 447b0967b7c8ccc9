"""Pins of the oracle's long-range ERIs over erf(omega r12)/r12 (the operator
of the range-separated hybrid of the comparative benchmark, Sec. 4.1), each
against something other than the oracle's own formula:

* (ss|ss) against the Gaussian-geminal representation
  erf(omega r)/r = 2/sqrt(pi) int_0^omega exp(-t^2 r^2) dt, whose s-type
  integrand has a closed form, integrated by Gauss-Legendre quadrature;
* (p s|s s) and (d s|s s) against central differences of that (ss|ss) in the
  centre A (d/dA_x of exp(-a (x-A_x)^2) = 2a (x-A_x) exp(...));
* every Cartesian component of p to f blocks against the brute-force
  quadrature of tests/brute.py with its t-integral stopped at t = omega;
* the limits: omega -> infinity gives the Coulomb integral, omega -> 0 gives
  2 omega / sqrt(pi) times the product of the two overlap distributions;
* J of the attenuated operator: symmetric, and for a closed-shell density
  0 < tr(D J_omega) < tr(D J) (the attenuated kernel is positive and below
  the Coulomb kernel in Fourier space).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_11185_gb300 import synth

from . import brute


def _ss_geminal(centres, exps, omega, n=80):
    """Unnormalised [ss|ss] over erf(omega r)/r by t-quadrature of the
    closed-form Gaussian-geminal integrals."""
    A, B, C, D = [np.asarray(c, float) for c in centres]
    a, b, c, d = exps
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    Kab = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
    Kcd = math.exp(-c * d / q * float(np.sum((C - D) ** 2)))
    R2 = float(np.sum((P - Q) ** 2))
    x, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * omega * (x + 1.0)
    den = p * q + t * t * (p + q)
    g = (math.pi ** 2 / den) ** 1.5 * np.exp(-p * q * t * t * R2 / den)
    return 2.0 / math.sqrt(math.pi) * 0.5 * omega * float(np.sum(w * g)) * Kab * Kcd


_CENTRES = [[0.0, 0.0, 0.0], [0.4, -0.3, 0.9], [1.3, 0.8, -0.2], [0.7, 1.6, 0.5]]
_EXPS = [1.3, 0.45, 0.8, 2.2]


@pytest.mark.parametrize("omega", [0.1, 0.4, 1.5, 6.0])
def test_ssss_matches_geminal_quadrature(omega):
    got = oracle.prim_block((0, 0, 0, 0), _CENTRES, _EXPS, omega=omega)[0, 0, 0, 0]
    ref = _ss_geminal(_CENTRES, _EXPS, omega)
    assert abs(got - ref) <= 1e-13 * abs(ref)


@pytest.mark.parametrize("omega", [0.3, 2.0])
def test_ps_and_ds_match_finite_differences(omega):
    a, h = _EXPS[0], 1e-3

    def f(dx, dy=0.0):
        c = [list(x) for x in _CENTRES]
        c[0][0] += dx
        c[0][1] += dy
        return _ss_geminal(c, _EXPS, omega)

    # d/dA_x [ss|ss] = 2a [p_x s|ss]  (fourth-order central difference)
    d1 = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
    px = oracle.prim_block((1, 0, 0, 0), _CENTRES, _EXPS, omega=omega)[0, 0, 0, 0]
    assert abs(2 * a * px - d1) <= 1e-8 * abs(d1)
    # d2/dA_x dA_y [ss|ss] = 4a^2 [d_xy s|ss] (component xy is index 1)
    hh = 2e-3
    d2 = (f(hh, hh) - f(hh, -hh) - f(-hh, hh) + f(-hh, -hh)) / (4 * hh * hh)
    dxy = oracle.prim_block((2, 0, 0, 0), _CENTRES, _EXPS, omega=omega)[1, 0, 0, 0]
    assert abs(4 * a * a * dxy - d2) <= 1e-5 * abs(d2)


def test_large_omega_is_coulomb_and_small_omega_is_linear():
    ls = (2, 1, 1, 0)
    full = oracle.prim_block(ls, _CENTRES, _EXPS)
    big = oracle.prim_block(ls, _CENTRES, _EXPS, omega=1e7)
    assert np.max(np.abs(big - full)) <= 1e-9 * np.max(np.abs(full))
    # omega -> 0: erf(omega r)/r -> 2 omega / sqrt(pi), so [ss|ss]_omega / omega
    # -> 2/sqrt(pi) S_ab S_cd with S the overlap of the product Gaussians
    A, B, C, D = [np.asarray(c) for c in _CENTRES]
    a, b, c, d = _EXPS
    Sab = (math.pi / (a + b)) ** 1.5 * math.exp(-a * b / (a + b) * float(np.sum((A - B) ** 2)))
    Scd = (math.pi / (c + d)) ** 1.5 * math.exp(-c * d / (c + d) * float(np.sum((C - D) ** 2)))
    w = 1e-4
    small = oracle.prim_block((0, 0, 0, 0), _CENTRES, _EXPS, omega=w)[0, 0, 0, 0]
    assert abs(small / w - 2 / math.sqrt(math.pi) * Sab * Scd) <= 1e-6 * Sab * Scd


def test_attenuated_coulomb_energy_is_positive_and_below_coulomb():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, synth.default_nocc(mol, opt["nocc"]), opt["dseed"])
    J, K = oracle.jk(mol, D, opt["thresh"])
    Jw, Kw = oracle.jk(mol, D, opt["thresh"], omega=0.4)
    assert np.max(np.abs(Jw - Jw.T)) <= 1e-12 * np.max(np.abs(Jw))
    assert np.max(np.abs(Kw - Kw.T)) <= 1e-12 * np.max(np.abs(Kw))
    ej, ejw = float(np.sum(D * J)), float(np.sum(D * Jw))
    assert 0.0 < ejw < ej
    # omega -> infinity reproduces the Coulomb J and K
    Ji, Ki = oracle.jk(mol, D, opt["thresh"], omega=1e7)
    assert np.max(np.abs(Ji - J)) <= 1e-9 * np.max(np.abs(J))
    assert np.max(np.abs(Ki - K)) <= 1e-9 * np.max(np.abs(K))


@pytest.mark.parametrize("ls,omega", [((1, 1, 0, 0), 0.5), ((2, 1, 1, 0), 0.3), ((2, 2, 1, 1), 1.2),
                                      ((3, 0, 1, 0), 0.7)])
def test_blocks_match_brute_force(ls, omega):
    rng = np.random.default_rng(sum((i + 5) * l for i, l in enumerate(ls)) + 29)
    cen = [rng.normal(size=3) * 0.9 for _ in range(4)]
    ex = list(np.exp(rng.uniform(np.log(0.15), np.log(6.0), size=4)))
    ref = brute.prim_block(ls, cen, ex, omega=omega)
    got = oracle.prim_block(ls, cen, ex, omega=omega)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))
