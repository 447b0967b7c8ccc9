"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test checks the oracle against mathematics the paper's definitions fix:
closed forms, an independent brute-force quadrature, an arbitrary-precision
special-function library, invariances and identities.  A dropped term, a wrong
sign or index, or a transposed operand anywhere in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2406_11185_gb300 import synth

from . import brute

mp = pytest.importorskip("mpmath")


# ---------------------------------------------------------------------------
# Boys function F_m(T) = int_0^1 t^2m exp(-T t^2) dt


def _boys_mp(m, T):
    """F_m(T) = gamma(m+1/2, T) / (2 T^(m+1/2)) (lower incomplete gamma), 30 digits."""
    with mp.workdps(40):
        if T == 0:
            return mp.mpf(1) / (2 * m + 1)
        T = mp.mpf(T)
        return mp.gammainc(m + mp.mpf(0.5), 0, T) / (2 * T ** (m + mp.mpf(0.5)))


@pytest.mark.parametrize("T", [0.0, 1e-12, 1e-6, 0.01, 0.3, 1.0, 4.7, 12.0, 29.99, 30.0, 30.01, 47.0,
                               120.0, 1e3, 3.3e4, 1e6])
def test_boys_vs_incomplete_gamma(T):
    F = oracle.boys(17, T)
    for m in range(18):
        ref = float(_boys_mp(m, T))
        assert abs(F[m] - ref) <= 1e-14 * ref, (m, T, F[m], ref)


def test_boys_special_values():
    F = oracle.boys(16, 0.0)
    for m in range(17):
        assert F[m] == pytest.approx(1.0 / (2 * m + 1), rel=1e-15)
    for T in [0.5, 3.0, 17.0, 55.0]:
        F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        assert oracle.boys(0, T)[0] == pytest.approx(F0, rel=1e-14)
    # asymptotic form for T >> m: F_m ~ (2m-1)!! / 2^(m+1) sqrt(pi / T^(2m+1))
    T = 400.0
    F = oracle.boys(8, T)
    for m in range(9):
        df = 1.0
        for k in range(2 * m - 1, 0, -2):
            df *= k
        asym = df / 2 ** (m + 1) * math.sqrt(math.pi / T ** (2 * m + 1))
        assert F[m] == pytest.approx(asym, rel=1e-13)


def test_boys_recursions_consistent():
    for T in [0.2, 7.0, 29.0, 31.0, 90.0]:
        F = oracle.boys(14, T)
        e = math.exp(-T)
        for m in range(14):
            assert F[m] == pytest.approx((2 * T * F[m + 1] + e) / (2 * m + 1), rel=1e-13)


# ---------------------------------------------------------------------------
# primitive integrals


def test_ssss_closed_form():
    rng = np.random.default_rng(1)
    for _ in range(20):
        cen = [rng.normal(size=3) * 1.5 for _ in range(4)]
        a, b, c, d = np.exp(rng.uniform(np.log(0.05), np.log(1e4), size=4))
        p, q = a + b, c + d
        P = (a * cen[0] + b * cen[1]) / p
        Q = (c * cen[2] + d * cen[3]) / q
        kab = math.exp(-a * b / p * np.sum((cen[0] - cen[1]) ** 2))
        kcd = math.exp(-c * d / q * np.sum((cen[2] - cen[3]) ** 2))
        T = p * q / (p + q) * np.sum((P - Q) ** 2)
        F0 = float(_boys_mp(0, T))
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * kab * kcd * F0
        got = oracle.prim_block((0, 0, 0, 0), cen, (a, b, c, d))[0, 0, 0, 0]
        assert got == pytest.approx(ref, rel=1e-13, abs=1e-300)


@pytest.mark.parametrize("ls", [(1, 0, 0, 0), (0, 0, 0, 1), (1, 1, 0, 0), (1, 1, 1, 1), (2, 0, 1, 0),
                                (2, 2, 0, 0), (2, 1, 2, 1), (3, 0, 0, 0), (3, 1, 2, 0), (3, 3, 1, 0),
                                (2, 2, 2, 2), (4, 0, 1, 1)])
def test_prim_block_vs_brute_force(ls):
    rng = np.random.default_rng(sum((i + 3) * l for i, l in enumerate(ls)) + 17)
    cen = [rng.normal(size=3) * 0.9 for _ in range(4)]
    ex = list(np.exp(rng.uniform(np.log(0.15), np.log(6.0), size=4)))
    ref = brute.prim_block(ls, cen, ex)
    got = oracle.prim_block(ls, cen, ex)
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def _norm_numeric(a, l):
    """1 / sqrt(<x^l e^{-a r^2} | x^l e^{-a r^2}>) by 1-D Gauss-Hermite quadrature."""
    x, w = np.polynomial.hermite.hermgauss(30)
    s = math.sqrt(2 * a)
    ix = np.sum(w * (x / s) ** (2 * l)) / s      # int x^2l e^{-2a x^2}
    i0 = np.sum(w) / s                            # int e^{-2a x^2}
    return 1.0 / math.sqrt(ix * i0 * i0)


def test_contracted_quartet_vs_brute_force():
    mol, _ = synth.config("small_f")
    rng = np.random.default_rng(3)
    # pick shells with few primitives (brute force cost) and mixed l
    cand = [i for i, s in enumerate(mol.shells) if len(s[2]) <= 2]
    for _ in range(3):
        sh = [int(rng.choice(cand)) for _ in range(4)]
        got = oracle.shell_quartet(mol, *sh)
        ref = np.zeros_like(got)
        ls = [mol.shells[s][1] for s in sh]
        cen = [mol.atoms[mol.shells[s][0]] for s in sh]
        import itertools
        for idx in itertools.product(*[range(len(mol.shells[s][2])) for s in sh]):
            ex = [mol.shells[s][2][i] for s, i in zip(sh, idx)]
            w = 1.0
            for s, i, e, l in zip(sh, idx, ex, ls):
                w *= mol.shells[s][3][i] * _norm_numeric(e, l)
            ref += w * brute.prim_block(ls, cen, ex)
        assert np.max(np.abs(got - ref)) <= 1e-11 * max(np.max(np.abs(ref)), 1e-300)


# ---------------------------------------------------------------------------
# basis conventions


def _cart_metric(l):
    pw = oracle.cart_powers(l)

    def df(n):
        r = 1
        while n > 1:
            r *= n
            n -= 2
        return r

    G = np.zeros((len(pw), len(pw)))
    for i, a in enumerate(pw):
        for j, b in enumerate(pw):
            if all((a[k] + b[k]) % 2 == 0 for k in range(3)):
                G[i, j] = np.prod([df(a[k] + b[k] - 1) for k in range(3)]) / df(2 * l - 1)
    return G


@pytest.mark.parametrize("l", [0, 1, 2, 3, 4])
def test_solid_harmonics_orthonormal_and_harmonic(l):
    T = oracle.sph_matrix(l)
    assert T.shape == (2 * l + 1, (l + 1) * (l + 2) // 2)
    M = T @ _cart_metric(l) @ T.T
    assert np.max(np.abs(M - np.eye(2 * l + 1))) < 1e-13
    # harmonic: the Laplacian of each polynomial vanishes
    pw = oracle.cart_powers(l)
    for row in T:
        lap = {}
        for c, (px, py, pz) in zip(row, pw):
            for k, p in enumerate((px, py, pz)):
                if p >= 2:
                    key = [px, py, pz]
                    key[k] -= 2
                    lap[tuple(key)] = lap.get(tuple(key), 0.0) + c * p * (p - 1)
        assert all(abs(v) < 1e-12 for v in lap.values())


def test_solid_harmonics_convention():
    # d: m=0 is (2z^2 - x^2 - y^2)/2, m=-2 is sqrt(3) xy, m=2 is sqrt(3)/2 (x^2 - y^2)
    T = oracle.sph_matrix(2)
    pw = oracle.cart_powers(2)
    ix = {p: i for i, p in enumerate(pw)}
    assert T[2, ix[(0, 0, 2)]] == pytest.approx(1.0)
    assert T[2, ix[(2, 0, 0)]] == pytest.approx(-0.5)
    assert T[0, ix[(1, 1, 0)]] == pytest.approx(math.sqrt(3))
    assert T[4, ix[(2, 0, 0)]] == pytest.approx(math.sqrt(3) / 2)
    assert T[4, ix[(0, 2, 0)]] == pytest.approx(-math.sqrt(3) / 2)
    # the generator's explicit formula gives the same coefficients
    for l in range(5):
        assert np.allclose(oracle.sph_matrix(l), synth._sph_matrix(l), atol=1e-13)


@pytest.mark.parametrize("name", ["tiny", "small"])
def test_overlap_normalised_and_density_trace(name):
    mol, opt = synth.config(name)
    S = oracle.overlap(mol)
    assert np.allclose(np.diag(S), 1.0, atol=1e-12)
    nocc = synth.default_nocc(mol, opt["nocc"])
    D = synth.make_density(mol, nocc, opt["dseed"])
    assert np.trace(D @ S) == pytest.approx(2 * nocc, rel=1e-11)
    # the generator's quadrature overlap agrees with the oracle's Hermite one
    assert np.max(np.abs(S - synth.overlap_matrix(mol))) < 1e-12


# ---------------------------------------------------------------------------
# full tensor: symmetry, Schwarz, J/K consistency


@pytest.fixture(scope="module")
def tiny():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    g = oracle.eri_tensor(mol)
    return mol, opt, D, g


def test_eight_fold_symmetry(tiny):
    _, _, _, g = tiny
    s = np.max(np.abs(g))
    for perm in ["jikl", "ijlk", "jilk", "klij", "lkij", "klji", "lkji"]:
        assert np.max(np.abs(g - np.einsum("ijkl->" + perm, g))) <= 1e-14 * s * 10


def test_schwarz_inequality_elementwise(tiny):
    mol, _, _, _ = tiny
    mc = synth.Molecule(mol.atoms, mol.heavy, mol.shells, spherical=False)
    g = oracle.eri_tensor(mc)
    Qf = oracle.schwarz_full(mc)
    sl = oracle.shell_slices(mc)
    n = mc.nshell
    for a in range(n):
        for b in range(n):
            for c in range(n):
                for d in range(n):
                    blk = g[sl[a], sl[b], sl[c], sl[d]]
                    assert np.max(np.abs(blk)) <= Qf[a, b] * Qf[c, d] * (1 + 1e-12)
    # Q is the square root of the largest diagonal element
    for a in range(n):
        for b in range(n):
            diag = np.einsum("ijij->ij", g[sl[a], sl[b], sl[a], sl[b]])
            assert Qf[a, b] == pytest.approx(math.sqrt(np.max(np.abs(diag))), rel=1e-14)


def test_scatter_equals_tiny_mode(tiny):
    mol, opt, D, _ = tiny
    J, K = oracle.jk(mol, D, opt["thresh"])
    Jt, Kt = oracle.jk_tiny(mol, D, opt["thresh"])
    s = max(np.max(np.abs(Jt)), np.max(np.abs(Kt)))
    assert np.max(np.abs(J - Jt)) <= 1e-13 * s
    assert np.max(np.abs(K - Kt)) <= 1e-13 * s
    assert np.allclose(J, J.T, atol=1e-13 * s) and np.allclose(K, K.T, atol=1e-13 * s)


def test_screening_rule_matches_tiny_mode():
    # a loose threshold that drops part of the quartets on both paths
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    Q = oracle.schwarz(mol)
    thr = float(np.quantile(np.outer(Q, Q), 0.4))
    J, K, kept = oracle.jk(mol, D, thr, Q=Q, return_kept=True)
    npair = len(Q)
    assert 0 < kept < npair * (npair + 1) // 2
    Jt, Kt = oracle.jk_tiny(mol, D, thr, Q=Q)
    s = max(np.max(np.abs(Jt)), np.max(np.abs(Kt)))
    assert np.max(np.abs(J - Jt)) <= 1e-13 * s
    assert np.max(np.abs(K - Kt)) <= 1e-13 * s


def test_blocks_match_full_jk():
    mol, opt = synth.config("small")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    J, K = oracle.jk(mol, D, opt["thresh"])
    sl = oracle.shell_slices(mol)
    pairs = [(0, 0), (5, 2), (30, 7), (12, 31), (32, 32)]
    blocks = oracle.jk_blocks(mol, D, opt["thresh"], pairs)
    for (a, b), (Jb, Kb) in zip(pairs, blocks):
        assert np.max(np.abs(Jb - J[sl[a], sl[b]])) < 1e-12
        assert np.max(np.abs(Kb - K[sl[a], sl[b]])) < 1e-12


# ---------------------------------------------------------------------------
# physics invariants


def test_single_orbital_identity():
    # nocc = 1: tr(DJ) = tr(DK) = 4 (phi phi|phi phi), so E_JK = (phi phi|phi phi) > 0
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, 1, 77)
    J, K = oracle.jk(mol, D, 0.0)
    tj, tk = np.sum(D * J), np.sum(D * K)
    assert tj == pytest.approx(tk, rel=1e-12)
    assert oracle.energy(D, J, K) == pytest.approx(0.25 * tj, rel=1e-12) and tj > 0


def test_psd_density_traces_nonnegative():
    mol, opt = synth.config("small")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    J, K = oracle.jk(mol, D, 0.0)
    assert np.sum(D * J) > 0 and np.sum(D * K) > 0
    # the Coulomb energy exceeds the exchange energy for a closed-shell D
    assert 0.5 * np.sum(D * J) > 0.25 * np.sum(D * K)


def test_translation_invariance():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    J, K = oracle.jk(mol, D, opt["thresh"])
    m2 = mol.with_atoms(mol.atoms + np.array([0.7, -1.3, 2.9]))
    J2, K2 = oracle.jk(m2, D, opt["thresh"])
    assert np.max(np.abs(J - J2)) < 1e-12 and np.max(np.abs(K - K2)) < 1e-12
    assert oracle.energy(D, J, K) == pytest.approx(oracle.energy(D, J2, K2), abs=1e-11)


def _monomial_rotation(l, R):
    """U[(abc),(a'b'c')]: phi'_{abc}(R r) = sum U phi_{a'b'c'}(r) for Gaussians
    centred on rotated centres (expansion of (R v)^(a,b,c) in monomials of v)."""
    pw = oracle.cart_powers(l)
    ix = {p: i for i, p in enumerate(pw)}
    U = np.zeros((len(pw), len(pw)))
    for i, (a, b, c) in enumerate(pw):
        poly = {(0, 0, 0): 1.0}
        for row, pwr in ((0, a), (1, b), (2, c)):
            for _ in range(pwr):
                nxt = {}
                for key, v in poly.items():
                    for j in range(3):
                        k2 = list(key)
                        k2[j] += 1
                        nxt[tuple(k2)] = nxt.get(tuple(k2), 0.0) + v * R[row, j]
                poly = nxt
        for key, v in poly.items():
            U[i, ix[key]] += v
    return U


def test_rotation_invariance_cartesian():
    mol, opt = synth.config("tiny", spherical=False)
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    E = oracle.energy(D, *oracle.jk(mol, D, opt["thresh"]))
    rng = np.random.default_rng(9)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    mr = mol.with_atoms(mol.atoms @ R.T)
    blocks = [_monomial_rotation(l, R) for _, l, _, _ in mol.shells]
    n = sum(b.shape[0] for b in blocks)
    U = np.zeros((n, n))
    o = 0
    for b in blocks:
        U[o:o + b.shape[0], o:o + b.shape[0]] = b
        o += b.shape[0]
    Ui = np.linalg.inv(U)
    Dr = Ui.T @ D @ Ui
    Er = oracle.energy(Dr, *oracle.jk(mr, Dr, opt["thresh"]))
    assert Er == pytest.approx(E, abs=1e-10)


# ---------------------------------------------------------------------------
# gradient


def test_gradient_vs_finite_differences_and_net_force():
    mol, opt = synth.config("tiny")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    g = oracle.grad(mol, D, opt["thresh"])
    fd = oracle.energy_fd_grad(mol, D, opt["thresh"], h=1e-4).reshape(mol.natom, 3)
    assert np.max(np.abs(g - fd)) < 1e-6
    assert np.max(np.abs(g.sum(axis=0))) < 1e-11 * max(1.0, np.max(np.abs(g)))
    assert np.max(np.abs(g)) > 1e-3


def test_gradient_vs_fd_f_shells():
    # f shells (derivatives reach g): a subset of coordinates
    mol, opt = synth.config("tiny_f")
    D = synth.make_density(mol, opt["nocc"], opt["dseed"])
    g = oracle.grad(mol, D, opt["thresh"])
    coords = [(0, 0), (1, 2)]
    fd = oracle.energy_fd_grad(mol, D, opt["thresh"], h=1e-4, coords=coords)
    for (a, k), v in zip(coords, fd):
        assert abs(g[a, k] - v) < 1e-6
    assert np.max(np.abs(g.sum(axis=0))) < 1e-11 * max(1.0, np.max(np.abs(g)))
