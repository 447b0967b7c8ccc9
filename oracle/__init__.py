"""Plain FP64 CPU oracle for the direct-SCF J/K build (arXiv 2406.11185).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the CUDA library and its
Python binding never do.  It shares no code with the CUDA path: the integrals
are evaluated by ``oracle.c`` (McMurchie-Davidson, long-double Boys function);
this module only marshals arrays, converts between the spherical and Cartesian
bases, and provides the "tiny mode" full-tensor J/K by ``einsum``.

Every function cites what it follows:
* J, K: the Coulomb and exchange terms of Eq. 1 (Sec. 1.2.1), K without c_x;
* the ERI: the integral in the ERI paragraph of Sec. 1.2.2;
* screening: the Cauchy-Schwarz bound of the mixed-precision bullet of
  Sec. 1.2.2 (skip a shell quartet iff Q_ab Q_cd < thresh);
* energy E = 1/2 tr(DJ) - 1/4 tr(DK), its nuclear gradient and its second
  derivatives at fixed D (the gradient and Hessian tasks of Sec. 3);
* optionally the long-range ERI over erf(omega r)/r, the operator of the
  range-separated hybrid (omegaB97X) of the comparative benchmark, Sec. 4.1.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _oracle.so with the host C compiler."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        basis = [dp, ctypes.c_int, ip, ip, ip, ip, dp, dp]
        L.orc_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.orc_prim_block.argtypes = [ctypes.c_int] * 4 + [dp, ctypes.c_double] * 4 + [ctypes.c_double, dp]
        L.orc_prim_block_omega.argtypes = [ctypes.c_int] * 4 + [dp, ctypes.c_double] * 4 + [ctypes.c_double] * 2 + \
            [dp]
        L.orc_shell_quartet.argtypes = basis + [ctypes.c_int] * 4 + [dp]
        L.orc_schwarz.argtypes = basis + [dp, ctypes.c_int]
        L.orc_jk.argtypes = basis + [dp, ctypes.c_double, dp, dp, dp, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_long)]
        L.orc_jk_omega.argtypes = basis + [dp, ctypes.c_double, dp, dp, dp, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_long), ctypes.c_double]
        L.orc_jk_range.argtypes = basis + [dp, ctypes.c_double, dp, dp, dp, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_long), ctypes.c_long, ctypes.c_long]
        L.orc_jk_blocks.argtypes = basis + [dp, ctypes.c_double, dp, ctypes.c_int, ip, dp, dp, ctypes.c_int]
        L.orc_eri_tensor.argtypes = basis + [dp]
        L.orc_overlap.argtypes = basis + [dp]
        L.orc_one_electron.argtypes = basis + [ctypes.c_int, dp, dp, dp, dp]
        L.orc_grad.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, dp, dp, dp, ctypes.c_double, dp,
                               dp, ctypes.c_int]
        L.orc_one_electron_grad.argtypes = basis + [ctypes.c_int, dp, dp, dp, dp]
        L.orc_jk_hessian.argtypes = [dp, ctypes.c_int, ctypes.c_int, ip, ip, ip, ip, dp, dp, dp, ctypes.c_double,
                                     dp, dp, ctypes.c_int]
        _lib = L
    return _lib


def _p(a, t=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _nthreads(n):
    return int(n) if n else (os.cpu_count() or 1)


def ncart(l):
    return (l + 1) * (l + 2) // 2


# ----------------------------------------------------------------------------
# Boys function and primitive integrals


def boys(mmax: int, T: float) -> np.ndarray:
    """F_m(T), m = 0..mmax (long double inside, rounded to double)."""
    out = np.zeros(mmax + 1)
    lib().orc_boys(mmax, float(T), _p(out))
    return out


def prim_block(ls, centres, exps, scale=1.0, omega=0.0) -> np.ndarray:
    """Unnormalised primitive Cartesian [ab|cd] for total powers ls=(la,lb,lc,ld);
    with omega > 0 over the long-range operator erf(omega r)/r."""
    out = np.zeros([ncart(l) for l in ls])
    cs = [np.ascontiguousarray(c, dtype=np.float64) for c in centres]
    args = []
    for c, e in zip(cs, exps):
        args += [_p(c), float(e)]
    if omega > 0.0:
        lib().orc_prim_block_omega(*[int(l) for l in ls], *args, float(scale), float(omega), _p(out))
    else:
        lib().orc_prim_block(*[int(l) for l in ls], *args, float(scale), _p(out))
    return out


# ----------------------------------------------------------------------------
# real solid harmonics by the Helgaker recurrences (eqs. 6.4.70-6.4.73)


def _poly_mul_xyz(poly, k):
    out = {}
    for (px, py, pz), c in poly.items():
        key = (px + (k == 0), py + (k == 1), pz + (k == 2))
        out[key] = out.get(key, 0.0) + c
    return out


def _poly_add(p, q, a=1.0, b=1.0):
    out = {k: a * v for k, v in p.items()}
    for k, v in q.items():
        out[k] = out.get(k, 0.0) + b * v
    return out


def _poly_r2(p):
    return _poly_add(_poly_add(_poly_mul_xyz(_poly_mul_xyz(p, 0), 0), _poly_mul_xyz(_poly_mul_xyz(p, 1), 1)),
                     _poly_mul_xyz(_poly_mul_xyz(p, 2), 2))


def solid_harmonics(lmax: int):
    """S[l][m] as monomial dictionaries, m = -l..l."""
    S = [{0: {(0, 0, 0): 1.0}}]
    for l in range(lmax):
        nxt = {}
        d0 = 1.0 if l == 0 else 0.0
        f = math.sqrt((2.0 ** d0) * (2 * l + 1) / (2 * l + 2))
        sll, slml = S[l][l], S[l][-l]
        nxt[l + 1] = {k: f * v for k, v in _poly_add(_poly_mul_xyz(sll, 0), _poly_mul_xyz(slml, 1),
                                                     1.0, -(1.0 - d0)).items()}
        nxt[-l - 1] = {k: f * v for k, v in _poly_add(_poly_mul_xyz(sll, 1), _poly_mul_xyz(slml, 0),
                                                      1.0, (1.0 - d0)).items()}
        for m in range(-l, l + 1):
            zt = _poly_mul_xyz(S[l][m], 2)
            if l >= 1 and abs(m) <= l - 1:
                r2 = _poly_r2(S[l - 1][m])
                pm = _poly_add(zt, r2, (2 * l + 1), -math.sqrt((l + m) * (l - m)))
            else:
                pm = {k: (2 * l + 1) * v for k, v in zt.items()}
            nrm = math.sqrt((l + m + 1) * (l - m + 1))
            nxt[m] = {k: v / nrm for k, v in pm.items()}
        S.append(nxt)
    return S


def cart_powers(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


def sph_matrix(l: int) -> np.ndarray:
    """[2l+1, ncart(l)]: rows are m = -l..l (p: x, y, z)."""
    if l == 0:
        return np.ones((1, 1))
    if l == 1:
        return np.eye(3)
    S = solid_harmonics(l)
    pw = cart_powers(l)
    T = np.zeros((2 * l + 1, len(pw)))
    for r, m in enumerate(range(-l, l + 1)):
        for k, p in enumerate(pw):
            T[r, k] = S[l][m].get(p, 0.0)
    return T


# ----------------------------------------------------------------------------
# basis marshalling


class _Basis:
    def __init__(self, mol):
        self.mol = mol
        self.xyz = np.ascontiguousarray(mol.atoms, dtype=np.float64)
        atom, l, nprim, ptr, exps, coefs = mol.flat()
        self.atom, self.l, self.nprim, self.ptr = (np.ascontiguousarray(a, dtype=np.int32)
                                                  for a in (atom, l, nprim, ptr))
        self.exps = np.ascontiguousarray(exps, dtype=np.float64)
        self.coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        self.nshell = len(self.l)
        self.nc = int(sum(ncart(int(x)) for x in self.l))

    def args(self):
        ip = ctypes.c_int
        return [_p(self.xyz), self.nshell, _p(self.atom, ip), _p(self.l, ip), _p(self.nprim, ip),
                _p(self.ptr, ip), _p(self.exps), _p(self.coefs)]


def cart2sph(mol) -> np.ndarray:
    """Block-diagonal T [n_sph, n_cart] with phi_sph = T phi_cart."""
    blocks = [sph_matrix(l) for _, l, _, _ in mol.shells]
    n = sum(b.shape[0] for b in blocks)
    m = sum(b.shape[1] for b in blocks)
    T = np.zeros((n, m))
    i = j = 0
    for b in blocks:
        T[i:i + b.shape[0], j:j + b.shape[1]] = b
        i += b.shape[0]
        j += b.shape[1]
    return T


def _to_cart(mol, D):
    if not mol.spherical:
        return np.ascontiguousarray(D, dtype=np.float64)
    T = cart2sph(mol)
    return np.ascontiguousarray(T.T @ D @ T)


def _from_cart(mol, M):
    if not mol.spherical:
        return M
    T = cart2sph(mol)
    return T @ M @ T.T


def shell_quartet(mol, a, b, c, d) -> np.ndarray:
    """Contracted Cartesian block (ab|cd)."""
    B = _Basis(mol)
    out = np.zeros([ncart(mol.shells[s][1]) for s in (a, b, c, d)])
    lib().orc_shell_quartet(*B.args(), a, b, c, d, _p(out))
    return out


def schwarz(mol, nthreads=None) -> np.ndarray:
    """Q[a(a+1)/2+b] = sqrt(max |(mu nu|mu nu)|) over Cartesian mu in a, nu in b."""
    B = _Basis(mol)
    Q = np.zeros(B.nshell * (B.nshell + 1) // 2)
    lib().orc_schwarz(*B.args(), _p(Q), _nthreads(nthreads))
    return Q


def schwarz_full(mol, Q=None) -> np.ndarray:
    n = mol.nshell
    if Q is None:
        Q = schwarz(mol)
    M = np.zeros((n, n))
    a, b = np.tril_indices(n)
    M[a, b] = Q[a * (a + 1) // 2 + b]
    M[b, a] = M[a, b]
    return M


def jk(mol, D, thresh, Q=None, nthreads=None, return_kept=False, omega=0.0):
    """J, K in the basis of D (spherical iff mol.spherical), scatter mode.
    omega > 0: J and K of the long-range operator erf(omega r)/r (the
    quartets screened with the Coulomb bounds Q)."""
    B = _Basis(mol)
    if Q is None:
        Q = schwarz(mol, nthreads)
    Dc = _to_cart(mol, np.asarray(D, dtype=np.float64))
    J = np.zeros((B.nc, B.nc))
    K = np.zeros((B.nc, B.nc))
    kept = ctypes.c_long(0)
    if omega > 0.0:
        lib().orc_jk_omega(*B.args(), _p(np.ascontiguousarray(Q)), float(thresh), _p(Dc), _p(J), _p(K),
                           _nthreads(nthreads), ctypes.byref(kept), float(omega))
    else:
        lib().orc_jk(*B.args(), _p(np.ascontiguousarray(Q)), float(thresh), _p(Dc), _p(J), _p(K),
                     _nthreads(nthreads), ctypes.byref(kept))
    J, K = _from_cart(mol, J), _from_cart(mol, K)
    return (J, K, kept.value) if return_kept else (J, K)


def jk_range_count(mol, D, thresh, ab_lo, ab_hi, Q=None, nthreads=None) -> int:
    """Run the scatter-mode J/K sum over bra pairs [ab_lo, ab_hi) only (pair
    index a(a+1)/2+b in creation order) and return the number of kept shell
    quartets; used to time a bounded sample of the oracle."""
    B = _Basis(mol)
    if Q is None:
        Q = schwarz(mol, nthreads)
    Dc = _to_cart(mol, np.asarray(D, dtype=np.float64))
    J = np.zeros((B.nc, B.nc))
    K = np.zeros((B.nc, B.nc))
    kept = ctypes.c_long(0)
    lib().orc_jk_range(*B.args(), _p(np.ascontiguousarray(Q)), float(thresh), _p(Dc), _p(J), _p(K),
                       _nthreads(nthreads), ctypes.byref(kept), int(ab_lo), int(ab_hi))
    return kept.value


def energy(D, J, K) -> float:
    """E_JK = 1/2 tr(DJ) - 1/4 tr(DK)."""
    return float(0.5 * np.sum(D * J) - 0.25 * np.sum(D * K))


def eri_tensor(mol) -> np.ndarray:
    """Full (mu nu|la si) tensor in the molecule's basis (tiny molecules)."""
    B = _Basis(mol)
    g = np.zeros((B.nc,) * 4)
    lib().orc_eri_tensor(*B.args(), _p(g))
    if mol.spherical:
        T = cart2sph(mol)
        g = np.einsum("ai,bj,ck,dl,ijkl->abcd", T, T, T, T, g, optimize=True)
    return g


def shell_slices(mol, spherical=None):
    sph = mol.spherical if spherical is None else spherical
    out, o = [], 0
    for _, l, _, _ in mol.shells:
        n = 2 * l + 1 if sph else ncart(l)
        out.append(slice(o, o + n))
        o += n
    return out


def jk_tiny(mol, D, thresh, Q=None):
    """Tiny mode: J = einsum(g, D), K = einsum(g, D) over the full tensor, with
    every shell quartet whose Q_ab Q_cd < thresh set to zero."""
    g = eri_tensor(mol)
    Qf = schwarz_full(mol, Q)
    sl = shell_slices(mol)
    n = mol.nshell
    for a in range(n):
        for b in range(n):
            for c in range(n):
                for d in range(n):
                    if Qf[a, b] * Qf[c, d] < thresh:
                        g[sl[a], sl[b], sl[c], sl[d]] = 0.0
    J = np.einsum("ijkl,kl->ij", g, D)
    K = np.einsum("ikjl,kl->ij", g, D)
    return J, K


def jk_blocks(mol, D, thresh, pairs, Q=None, nthreads=None):
    """Blocks J[a,b], K[a,b] (molecule basis) for the shell pairs requested,
    each computed straight from the definition over all c, d."""
    B = _Basis(mol)
    Qf = np.ascontiguousarray(schwarz_full(mol, Q))
    Dc = _to_cart(mol, np.asarray(D, dtype=np.float64))
    req = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1, 2))
    sizes = [ncart(mol.shells[a][1]) * ncart(mol.shells[b][1]) for a, b in req]
    Jo = np.zeros(sum(sizes))
    Ko = np.zeros(sum(sizes))
    lib().orc_jk_blocks(*B.args(), _p(Qf), float(thresh), _p(Dc), len(req), _p(req, ctypes.c_int), _p(Jo),
                        _p(Ko), _nthreads(nthreads))
    out, o = [], 0
    for (a, b), s in zip(req, sizes):
        la, lb = mol.shells[a][1], mol.shells[b][1]
        Jb = Jo[o:o + s].reshape(ncart(la), ncart(lb))
        Kb = Ko[o:o + s].reshape(ncart(la), ncart(lb))
        if mol.spherical:
            Ta, Tb = sph_matrix(la), sph_matrix(lb)
            Jb, Kb = Ta @ Jb @ Tb.T, Ta @ Kb @ Tb.T
        out.append((Jb, Kb))
        o += s
    return out


def overlap(mol) -> np.ndarray:
    """Overlap matrix in the molecule's basis (input checks only)."""
    B = _Basis(mol)
    S = np.zeros((B.nc, B.nc))
    lib().orc_overlap(*B.args(), _p(S))
    return _from_cart(mol, S)


def grad(mol, D, thresh, Q=None, nthreads=None) -> np.ndarray:
    """dE_JK/dR [natom, 3] at fixed D (analytic derivative integrals)."""
    B = _Basis(mol)
    if Q is None:
        Q = schwarz(mol, nthreads)
    Dc = _to_cart(mol, np.asarray(D, dtype=np.float64))
    g = np.zeros((mol.natom, 3))
    ip = ctypes.c_int
    lib().orc_grad(_p(B.xyz), mol.natom, B.nshell, _p(B.atom, ip), _p(B.l, ip), _p(B.nprim, ip), _p(B.ptr, ip),
                   _p(B.exps), _p(B.coefs), _p(np.ascontiguousarray(Q)), float(thresh), _p(Dc), _p(g),
                   _nthreads(nthreads))
    return g


def jk_hessian(mol, D, thresh, Q=None, nthreads=None) -> np.ndarray:
    """d2E_JK / dR dR [3 natom, 3 natom] at fixed D (analytic second-derivative
    integrals; the two-electron part of the Hessian task of Sec. 3)."""
    B = _Basis(mol)
    if Q is None:
        Q = schwarz(mol, nthreads)
    Dc = _to_cart(mol, np.asarray(D, dtype=np.float64))
    H = np.zeros((3 * mol.natom, 3 * mol.natom))
    ip = ctypes.c_int
    lib().orc_jk_hessian(_p(B.xyz), mol.natom, B.nshell, _p(B.atom, ip), _p(B.l, ip), _p(B.nprim, ip),
                         _p(B.ptr, ip), _p(B.exps), _p(B.coefs), _p(np.ascontiguousarray(Q)), float(thresh),
                         _p(Dc), _p(H), _nthreads(nthreads))
    return H


def energy_fd_grad(mol, D, thresh, h=1e-4, coords=None, nthreads=None):
    """Central finite differences of E_JK(R) at fixed D (Q recomputed at each
    displaced geometry), for the listed (atom, xyz) coordinates."""
    if coords is None:
        coords = [(a, k) for a in range(mol.natom) for k in range(3)]
    out = []
    for a, k in coords:
        es = []
        for s in (+1, -1):
            x = mol.atoms.copy()
            x[a, k] += s * h
            m2 = mol.with_atoms(x)
            J, K = jk(m2, D, thresh, nthreads=nthreads)
            es.append(energy(D, J, K))
        out.append((es[0] - es[1]) / (2 * h))
    return np.array(out)


# ----------------------------------------------------------------------------
# SCF driver around the J/K build (the restricted closed-shell Fock iteration
# of Eq. 1 with c_x = 1 and no exchange-correlation term, i.e. Hartree-Fock)


def one_electron(mol, charges):
    """Overlap S, kinetic T and nuclear attraction V in the molecule's basis
    (the core Hamiltonian H = T + V of the Fock matrix of Eq. 1)."""
    B = _Basis(mol)
    q = np.ascontiguousarray(np.asarray(charges, dtype=np.float64))
    S = np.zeros((B.nc, B.nc))
    T = np.zeros((B.nc, B.nc))
    V = np.zeros((B.nc, B.nc))
    lib().orc_one_electron(*B.args(), mol.natom, _p(q), _p(S), _p(T), _p(V))
    return _from_cart(mol, S), _from_cart(mol, T), _from_cart(mol, V)


def nuclear_repulsion(mol, charges) -> float:
    """sum_{A<B} Z_A Z_B / |R_A - R_B|."""
    X = np.asarray(mol.atoms, dtype=np.float64)
    Z = np.asarray(charges, dtype=np.float64)
    e = 0.0
    for a in range(len(Z)):
        for b in range(a):
            e += Z[a] * Z[b] / np.linalg.norm(X[a] - X[b])
    return float(e)


def scf(mol, charges, nocc, thresh, max_iter=100, e_tol=1e-10, g_tol=1e-8, diis_size=8):
    """Restricted closed-shell SCF with the oracle's J and K, rebuilt in full
    from the current density every iteration (no incremental builds):
      F = H + J - 1/2 K,  E = 1/2 tr(D (H + F)) + E_nuc,  D = 2 C_occ C_occ^T,
    C from the generalised eigenproblem F C = S C e (by S^(-1/2)), starting
    from the core Hamiltonian, with Pulay DIIS on the error F D S - S D F.
    Returns dict(energy, D, iterations, converged, F, S, H, e_nuc)."""
    S, T, V = one_electron(mol, charges)
    H = T + V
    e_nuc = nuclear_repulsion(mol, charges)
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T

    def density(F):
        _, C = np.linalg.eigh(X.T @ F @ X)
        C = X @ C[:, :nocc]
        return 2.0 * C @ C.T

    D = density(H)
    Q = schwarz(mol)
    focks, errs = [], []
    E_old = None
    for it in range(1, max_iter + 1):
        J, K = jk(mol, D, thresh, Q=Q)
        F = H + J - 0.5 * K
        E = 0.5 * float(np.sum(D * (H + F))) + e_nuc
        err = F @ D @ S - S @ D @ F
        gnorm = float(np.max(np.abs(err)))
        if E_old is not None and abs(E - E_old) < e_tol and gnorm < g_tol:
            return dict(energy=E, D=D, iterations=it, converged=True, F=F, S=S, H=H, e_nuc=e_nuc)
        E_old = E
        focks.append(F)
        errs.append(err)
        focks, errs = focks[-diis_size:], errs[-diis_size:]
        n = len(focks)
        if n >= 2:
            Bm = -np.ones((n + 1, n + 1))
            Bm[n, n] = 0.0
            for i in range(n):
                for j in range(n):
                    Bm[i, j] = float(np.sum(errs[i] * errs[j]))
            rhs = np.zeros(n + 1)
            rhs[n] = -1.0
            c = np.linalg.solve(Bm, rhs)[:n]
            F = sum(ci * Fi for ci, Fi in zip(c, focks))
        D = density(F)
    return dict(energy=E, D=D, iterations=max_iter, converged=False, F=F, S=S, H=H, e_nuc=e_nuc)


def one_electron_grad(mol, charges, D, W) -> np.ndarray:
    """sum D dH/dR - sum W dS/dR [natom, 3] for D and W in the molecule's
    output basis (the one-electron part of the closed-shell SCF gradient)."""
    B = _Basis(mol)
    q = np.ascontiguousarray(np.asarray(charges, dtype=np.float64))
    g = np.zeros((mol.natom, 3))
    lib().orc_one_electron_grad(*B.args(), mol.natom, _p(q), _p(_to_cart(mol, np.asarray(D, dtype=np.float64))),
                                _p(_to_cart(mol, np.asarray(W, dtype=np.float64))), _p(g))
    return g


def scf_gradient(mol, charges, nocc, thresh, Q=None, nthreads=None, **scf_kw):
    """Nuclear gradient [natom, 3] of the converged closed-shell SCF energy
    (the single-point force task of Sec. 3, around the J/K gradient):

        dE/dR = sum D dH/dR - sum W dS/dR + dE_JK/dR|_D + dE_nuc/dR,
        W = 1/2 D F D (the energy-weighted density of the converged orbitals).

    Returns (energy, gradient, the scf() result)."""
    r = scf(mol, charges, nocc, thresh, **scf_kw)
    D, F = r["D"], r["F"]
    W = 0.5 * D @ F @ D
    q = np.ascontiguousarray(np.asarray(charges, dtype=np.float64))
    g = one_electron_grad(mol, q, D, W)
    g += grad(mol, D, thresh, Q=Q, nthreads=nthreads)
    X = np.asarray(mol.atoms, dtype=np.float64)
    for a in range(mol.natom):
        for b in range(mol.natom):
            if a != b:
                d = X[a] - X[b]
                g[a] -= q[a] * q[b] * d / np.linalg.norm(d) ** 3
    return r["energy"], g, r
