"""Seeded synthetic molecules, contracted Gaussian basis sets and densities.

This module is the only code shared by the CPU oracle and the CUDA library's
tests and benchmark.  It produces *inputs* only: atom positions, shells
(exponents and contraction coefficients) and a closed-shell density matrix D.
It contains no electron-repulsion, Boys-function or J/K arithmetic.  To make D
idempotent in the overlap metric it evaluates one-electron overlap integrals,
which it does by Gauss-Hermite quadrature (a method that neither the oracle nor
the CUDA path uses); the overlap is not part of the J/K build.

Conventions shared by every consumer (they are conventions, not arithmetic):

* bohr; shells are (atom, l, exponents, coefficients).  The coefficients
  multiply *normalised* primitive Cartesian Gaussians
  N(a,l) x^l exp(-a r^2), N(a,l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!);
  every Cartesian component of a shell uses the same N(a,l) (the x^l one).
  The generator scales each shell so that its x^l component has unit norm.
* Cartesian components of a shell are ordered by descending x power, then
  descending y power (xx, xy, xz, yy, yz, zz).
* Spherical components: p is (x, y, z); l >= 2 is m = -l..l real solid
  harmonics with unit norm.

The molecular recipes follow the workloads the paper benchmarks (Sec. 4:
compact organic-like clusters, heavy:H about 0.4:0.6, contracted shells up to
d or f, exponents from diffuse to core, Schwarz tolerance 1e-12/1e-10): the
paper's own molecules and def2 basis sets are not used.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

L_CHAR = "spdfg"


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def nsph(l: int) -> int:
    return 2 * l + 1


def cart_powers(l: int):
    """Cartesian exponent triples of a shell, in the library's order."""
    out = []
    for i in range(l, -1, -1):
        for j in range(l - i, -1, -1):
            out.append((i, j, l - i - j))
    return out


@dataclass
class Molecule:
    """A synthetic molecule with its basis.

    atoms: float64 [natom, 3] (bohr); heavy: bool [natom]
    shells: list of (atom, l, exps float64[nprim], coefs float64[nprim])
    """
    atoms: np.ndarray
    heavy: np.ndarray
    shells: list
    spherical: bool = True
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def natom(self) -> int:
        return int(self.atoms.shape[0])

    @property
    def nshell(self) -> int:
        return len(self.shells)

    def nbf(self, spherical: bool | None = None) -> int:
        sph = self.spherical if spherical is None else spherical
        return sum((nsph(l) if sph else ncart(l)) for _, l, _, _ in self.shells)

    def flat(self):
        """Flattened arrays: shell_atom, shell_l, shell_nprim, shell_ptr, exps, coefs."""
        atom = np.array([s[0] for s in self.shells], dtype=np.int32)
        l = np.array([s[1] for s in self.shells], dtype=np.int32)
        nprim = np.array([len(s[2]) for s in self.shells], dtype=np.int32)
        ptr = np.zeros(len(self.shells), dtype=np.int32)
        if len(self.shells) > 1:
            ptr[1:] = np.cumsum(nprim)[:-1]
        exps = np.concatenate([s[2] for s in self.shells]).astype(np.float64)
        coefs = np.concatenate([s[3] for s in self.shells]).astype(np.float64)
        return atom, l, nprim, ptr, exps, coefs

    def with_atoms(self, atoms: np.ndarray) -> "Molecule":
        return Molecule(np.ascontiguousarray(atoms, dtype=np.float64), self.heavy.copy(),
                        list(self.shells), self.spherical, self.name, dict(self.meta))


# ----------------------------------------------------------------------------
# geometry


def _random_unit(rng) -> np.ndarray:
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def pack_cluster(rng, n_heavy: int, n_h: int, dmin: float, dmax: float,
                 max_tries: int = 100000) -> tuple[np.ndarray, np.ndarray]:
    """Random compact packing: each new atom sits U[dmin,dmax] from a random
    earlier heavy atom and at least dmin from every atom placed so far."""
    pos = [np.zeros(3)]
    heavy_idx = [0]
    tries = 0

    def place(anchor_pool):
        nonlocal tries
        while True:
            tries += 1
            if tries > max_tries:
                raise RuntimeError("packing failed")
            a = pos[anchor_pool[rng.integers(len(anchor_pool))]]
            p = a + rng.uniform(dmin, dmax) * _random_unit(rng)
            if all(np.linalg.norm(p - q) >= dmin for q in pos):
                return p

    for _ in range(n_heavy - 1):
        pos.append(place(heavy_idx))
        heavy_idx.append(len(pos) - 1)
    for _ in range(n_h):
        pos.append(place(heavy_idx))
    heavy = np.zeros(len(pos), dtype=bool)
    heavy[:n_heavy] = True
    return np.array(pos, dtype=np.float64), heavy


# ----------------------------------------------------------------------------
# basis


def _dfact(n: int) -> float:
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


def _shell_x_norm2(l: int, exps: np.ndarray, coefs: np.ndarray) -> float:
    """<x^l|x^l> of a contraction over normalised primitives (closed form of
    the product of two normalised Gaussians sharing a centre)."""
    a = exps[:, None]
    b = exps[None, :]
    s = (2.0 * np.sqrt(a * b) / (a + b)) ** (l + 1.5)
    return float(coefs @ s @ coefs)


def random_shell(rng, l: int, nprim_range: tuple[int, int], exp_range: tuple[float, float]):
    lo, hi = math.log(exp_range[0]), math.log(exp_range[1])
    nprim = int(rng.integers(nprim_range[0], nprim_range[1] + 1))
    while True:
        e = np.sort(np.exp(rng.uniform(lo, hi, size=nprim)))[::-1]
        if nprim == 1 or np.all(e[:-1] / e[1:] >= 1.2):
            break
    c = rng.uniform(0.1, 1.0, size=nprim)
    c = c / math.sqrt(_shell_x_norm2(l, e, c))
    return e.astype(np.float64), c.astype(np.float64)


def parse_recipe(s: str) -> list[int]:
    """'3s2p1d' -> [0,0,0,1,1,2]."""
    out = []
    i = 0
    while i < len(s):
        j = i
        while s[j].isdigit():
            j += 1
        out += [L_CHAR.index(s[j])] * int(s[i:j])
        i = j + 1
    return out


def make_molecule(seed: int, n_heavy: int, n_h: int, heavy_shells: str, h_shells: str,
                  nprim_range=(1, 6), exp_range=(0.1, 5e3), dist=(1.9, 2.9),
                  spherical: bool = True, name: str = "") -> Molecule:
    rng = np.random.default_rng(seed)
    atoms, heavy = pack_cluster(rng, n_heavy, n_h, dist[0], dist[1])
    shells = []
    for ia in range(len(atoms)):
        for l in parse_recipe(heavy_shells if heavy[ia] else h_shells):
            e, c = random_shell(rng, l, nprim_range, exp_range)
            shells.append((ia, l, e, c))
    return Molecule(atoms, heavy, shells, spherical, name,
                    dict(seed=seed, n_heavy=n_heavy, n_h=n_h, heavy_shells=heavy_shells,
                         h_shells=h_shells, nprim_range=nprim_range, exp_range=exp_range,
                         dist=dist))


# ----------------------------------------------------------------------------
# overlap by Gauss-Hermite quadrature (input preparation only)


def _sph_matrix(l: int) -> np.ndarray:
    """Cartesian -> real solid harmonic coefficients [2l+1, ncart(l)] from the
    explicit expansion of the real solid harmonics (Helgaker, Jorgensen and
    Olsen, eqs. 6.4.47-6.4.49); p is kept as (x, y, z)."""
    if l == 0:
        return np.ones((1, 1))
    if l == 1:
        return np.eye(3)
    pw = cart_powers(l)
    index = {p: k for k, p in enumerate(pw)}
    T = np.zeros((2 * l + 1, len(pw)))
    for row, m in enumerate(range(-l, l + 1)):
        am = abs(m)
        vm = 0.0 if m >= 0 else 0.5
        nlm = math.sqrt(2.0 * math.factorial(l + am) * math.factorial(l - am)
                        / (2.0 if m == 0 else 1.0)) / (2 ** am * math.factorial(l))
        for t in range((l - am) // 2 + 1):
            for u in range(t + 1):
                v = vm
                while v <= am / 2.0 + 1e-9:
                    two_v = int(round(2 * v))
                    if two_v <= am:
                        c = ((-1) ** int(round(t + v - vm)) * 0.25 ** t * math.comb(l, t)
                             * math.comb(l - t, am + t) * math.comb(t, u) * math.comb(am, two_v))
                        px = 2 * t + am - 2 * u - two_v
                        py = 2 * u + two_v
                        pz = l - 2 * t - am
                        T[row, index[(px, py, pz)]] += nlm * c
                    v += 1.0
    return T


def overlap_matrix(mol: Molecule, spherical: bool | None = None) -> np.ndarray:
    """AO overlap matrix by Gauss-Hermite quadrature of each 1-D factor,
    vectorised over all shell pairs with the same (l_a, l_b, nprim_a, nprim_b)."""
    sph = mol.spherical if spherical is None else spherical
    gh_x, gh_w = np.polynomial.hermite.hermgauss(8)  # exact to degree 15
    offs, o = [], 0
    for _, l, _, _ in mol.shells:
        offs.append(o)
        o += nsph(l) if sph else ncart(l)
    S = np.zeros((o, o))
    groups: dict = {}
    for ia, (_, la, ea, _) in enumerate(mol.shells):
        for ib in range(ia + 1):
            lb, eb = mol.shells[ib][1], mol.shells[ib][2]
            groups.setdefault((la, lb, len(ea), len(eb)), []).append((ia, ib))
    sphm = {l: _sph_matrix(l) for l in range(5)}
    for (la, lb, na, nb), pairs in groups.items():
        pairs = np.array(pairs)
        for c0 in range(0, len(pairs), 4096):
            pr = pairs[c0:c0 + 4096]
            A = mol.atoms[[mol.shells[i][0] for i in pr[:, 0]]][:, None, None, :]
            B = mol.atoms[[mol.shells[i][0] for i in pr[:, 1]]][:, None, None, :]
            a = np.array([mol.shells[i][2] for i in pr[:, 0]])[:, :, None]
            b = np.array([mol.shells[i][2] for i in pr[:, 1]])[:, None, :]
            ca = np.array([mol.shells[i][3] for i in pr[:, 0]])[:, :, None]
            cb = np.array([mol.shells[i][3] for i in pr[:, 1]])[:, None, :]
            p = a + b
            P = (a[..., None] * A + b[..., None] * B) / p[..., None]
            pref = np.exp(-(a * b / p) * np.sum((A - B) ** 2, axis=-1))
            norm_a = (2 * a / np.pi) ** 0.75 * (4 * a) ** (la / 2) / math.sqrt(_dfact(2 * la - 1))
            norm_b = (2 * b / np.pi) ** 0.75 * (4 * b) ** (lb / 2) / math.sqrt(_dfact(2 * lb - 1))
            w = ca * cb * norm_a * norm_b * pref * (np.pi / p) ** 1.5
            x = gh_x / np.sqrt(p)[..., None]
            M = np.zeros((3, la + 1, lb + 1) + p.shape)
            for d in range(3):
                xa = x + (P[..., d] - A[..., d])[..., None]
                xb = x + (P[..., d] - B[..., d])[..., None]
                for i in range(la + 1):
                    for j in range(lb + 1):
                        M[d, i, j] = np.sum(gh_w * xa ** i * xb ** j, axis=-1) / math.sqrt(math.pi)
            blk = np.zeros((len(pr), ncart(la), ncart(lb)))
            for ka, (ax, ay, az) in enumerate(cart_powers(la)):
                for kb, (bx, by, bz) in enumerate(cart_powers(lb)):
                    blk[:, ka, kb] = np.sum(w * M[0, ax, bx] * M[1, ay, by] * M[2, az, bz], axis=(1, 2))
            if sph:
                blk = np.einsum("mi,pij,nj->pmn", sphm[la], blk, sphm[lb])
            for (ia, ib), bl in zip(pr, blk):
                S[offs[ia]:offs[ia] + bl.shape[0], offs[ib]:offs[ib] + bl.shape[1]] = bl
                S[offs[ib]:offs[ib] + bl.shape[1], offs[ia]:offs[ia] + bl.shape[0]] = bl.T
    return S


def make_density(mol: Molecule, nocc: int, seed: int, spherical: bool | None = None,
                 S: np.ndarray | None = None) -> np.ndarray:
    """D = 2 C C^T with C ~ N(0,1) [n, nocc] orthonormalised in the overlap
    metric (Cholesky of C^T S C)."""
    if S is None:
        S = overlap_matrix(mol, spherical)
    n = S.shape[0]
    rng = np.random.default_rng(seed)
    C = rng.normal(size=(n, nocc))
    M = C.T @ S @ C
    Lc = np.linalg.cholesky(M)
    C = np.linalg.solve(Lc, C.T).T
    D = 2.0 * C @ C.T
    return 0.5 * (D + D.T)


# ----------------------------------------------------------------------------
# named workloads


def config(name: str, spherical: bool = True) -> tuple[Molecule, dict]:
    """Named synthetic workloads.  Returns (molecule, options) where options
    holds thresh, split, nocc and the density seed."""
    if name == "tiny":  # 1 heavy + 2 H, 1.4-2.0 bohr, thresh 1e-12, FP64
        m = make_molecule(1001, 1, 2, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3), (1.4, 2.0), spherical, name)
        return m, dict(thresh=1e-12, split=0.0, nocc=5, dseed=11001)
    if name == "small":  # 3 heavy + 5 H: spans many tiles but the oracle takes seconds
        m = make_molecule(1501, 3, 5, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3), (1.9, 2.9), spherical, name)
        return m, dict(thresh=1e-10, split=0.0, nocc=12, dseed=11501)
    if name == "small_f":  # 2 heavy + 3 H with the f recipe
        m = make_molecule(1601, 2, 3, "4s3p2d1f", "3s2p1d", (1, 8), (0.05, 1e4), (1.9, 2.9), spherical, name)
        return m, dict(thresh=1e-12, split=1e-5, nocc=12, dseed=11601)
    if name == "small_f3":  # 2 heavy + 3 H with the f recipe, 1-3 primitives (multi-centre f parity)
        m = make_molecule(1602, 2, 3, "4s3p2d1f", "3s2p1d", (1, 3), (0.05, 1e4), (1.9, 2.9), spherical, name)
        return m, dict(thresh=1e-12, split=1e-5, nocc=12, dseed=11602)
    if name == "tiny_f":  # 1 heavy + 1 H with the f recipe, 1-3 primitives (gradient pins)
        m = make_molecule(1701, 1, 1, "4s3p2d1f", "3s2p1d", (1, 3), (0.05, 1e4), (1.4, 2.0), spherical, name)
        return m, dict(thresh=1e-12, split=1e-5, nocc=6, dseed=11701)
    if name == "c60":  # 24 heavy + 36 H, ~516 bf, thresh 1e-10, FP64
        m = make_molecule(2001, 24, 36, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3), (1.9, 2.9), spherical, name)
        return m, dict(thresh=1e-10, split=1e-5, nocc=120, dseed=12001)
    if name == "c240":  # 96 heavy + 144 H, the 60-atom recipe, 2064 bf: the ~2k-function point
        m = make_molecule(2401, 96, 144, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3), (1.9, 2.9), spherical, name)
        # split 3e-3: the largest split whose mixed energy stays within 1e-6 Eh of the
        # plain FP64 build of this molecule with a margin (6.0e-7 Eh measured)
        return m, dict(thresh=1e-10, split=3e-3, nocc=None, dseed=12401)
    if name == "c200":  # 80 heavy + 120 H, f recipe, 4080 bf, mixed
        m = make_molecule(3001, 80, 120, "4s3p2d1f", "3s2p1d", (1, 8), (0.05, 1e4), (1.9, 2.9), spherical, name)
        return m, dict(thresh=1e-12, split=1e-5, nocc=None, dseed=13001)
    if name == "c120":  # 48 heavy + 72 H, f recipe, 2448 bf, mixed (the ~2k-function point)
        m = make_molecule(3002, 48, 72, "4s3p2d1f", "3s2p1d", (1, 8), (0.05, 1e4), (1.9, 2.9), spherical, name)
        return m, dict(thresh=1e-12, split=1e-5, nocc=None, dseed=13002)
    raise KeyError(name)


def batch_molecules(count: int = 256, base_seed: int = 5000, spherical: bool = True):
    """Molecules of 10-40 atoms (uniform), 40 % heavy, heavy 3s2p1d / H 2s1p."""
    mols = []
    for i in range(count):
        rng = np.random.default_rng(base_seed + i)
        natom = int(rng.integers(10, 41))
        nh = int(round(0.4 * natom))
        m = make_molecule(base_seed + i, nh, natom - nh, "3s2p1d", "2s1p", (1, 6), (0.1, 5e3),
                          (1.9, 2.9), spherical, f"batch{i}")
        mols.append(m)
    return mols


def nuclear_charges(mol: Molecule) -> np.ndarray:
    """Nuclear charges of the synthetic atoms (a convention of the inputs):
    heavy atoms are carbon-like (Z = 6), the others hydrogen (Z = 1)."""
    return np.where(mol.heavy, 6.0, 1.0)


def default_nocc(mol: Molecule, nocc) -> int:
    if nocc is not None:
        return int(nocc)
    return max(1, int(round(0.2 * mol.nbf())))
