"""Closed-shell SCF driver around the GPU J/K build.

The iteration of Sec. 1.2.1 (Eq. 1) with the exact-exchange fraction c_x = 1
and no exchange-correlation term, i.e. restricted Hartree-Fock:

    F = H + J - 1/2 K,   H = T + V (adft_one_electron),
    E = 1/2 tr(D (H + F)) + E_nuc,   D = 2 C_occ C_occ^T,

with C from the generalised eigenproblem F C = S C e (orthogonalised by
S^(-1/2), torch.linalg.eigh on the GPU), the core Hamiltonian as the starting
guess and Pulay DIIS on the error F D S - S D F.

J and K come from adft_jk_build.  With incremental builds (the SCF-iteration
practice of Sec. 1.2.2), iteration n builds only the change of the density,
J(D_n) = J(D_m) + J(D_n - D_m), and screens it by the density-weighted bound:
a quartet is skipped iff Q_ab Q_cd max|dD| < thresh (and runs in FP64 iff
Q_ab Q_cd max|dD| >= split), i.e. the library is called with thresh and split
divided by max|dD|.  Every rebuild_every-th iteration is a full build, which
keeps the accumulated screening error bounded.
"""
from __future__ import annotations

import time

import numpy as np

from . import adft, synth


def nuclear_repulsion(atoms, charges) -> float:
    X = np.asarray(atoms, dtype=np.float64)
    Z = np.asarray(charges, dtype=np.float64)
    d = np.linalg.norm(X[:, None, :] - X[None, :, :], axis=-1)
    iu = np.triu_indices(len(Z), 1)
    return float(np.sum(Z[iu[0]] * Z[iu[1]] / d[iu]))


class RHF:
    """Restricted closed-shell SCF of one molecule on the current CUDA device."""

    def __init__(self, mol, charges=None, nocc=None, thresh=1e-10, precision="fp64", split=1e-5,
                 incremental=True, rebuild_every=8, stream=None):
        import torch
        self.torch = torch
        self.mol = mol
        self.charges = synth.nuclear_charges(mol) if charges is None else np.asarray(charges, dtype=np.float64)
        nel = int(round(float(np.sum(self.charges))))
        self.nocc = nel // 2 if nocc is None else int(nocc)
        self.thresh, self.precision, self.split = thresh, precision, split
        self.incremental, self.rebuild_every = incremental, max(1, int(rebuild_every))
        self.stream = stream
        self.basis = adft.Basis.from_molecule(mol)
        self.S, T, V = adft.adft_one_electron(self.basis, self.charges, stream=stream)
        self.H = T + V
        self.e_nuc = nuclear_repulsion(mol.atoms, self.charges)
        s, U = torch.linalg.eigh(self.S)
        self.X = (U * s.rsqrt()) @ U.T

    def _density(self, F):
        torch = self.torch
        _, C = torch.linalg.eigh(self.X.T @ F @ self.X)
        C = self.X @ C[:, :self.nocc]
        D = 2.0 * C @ C.T
        return 0.5 * (D + D.T)

    def _jk(self, D, thresh, split):
        return adft.adft_jk_build(self.basis, D, thresh=thresh, split=split, precision=self.precision, check=False,
                                  stream=self.stream)

    def run(self, max_iter=100, e_tol=1e-10, g_tol=1e-8, diis_size=8):
        """Iterate to |dE| < e_tol and max|FDS - SDF| < g_tol.  Returns a dict
        with the energy, density, iteration count, convergence flag and the
        J/K build times (ms, CUDA events on the current stream) and kinds."""
        torch = self.torch
        H, S = self.H, self.S
        D = self._density(H)
        J = K = D_ref = None
        focks, errs = [], []
        E_old = None
        builds = []
        for it in range(1, max_iter + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            full = J is None or not self.incremental or (it - 1) % self.rebuild_every == 0
            if full:
                J, K = self._jk(D, self.thresh, self.split)
                kind = "full"
            else:
                dD = D - D_ref
                m = float(dD.abs().max().item())
                if m > 0.0:
                    Jd, Kd = self._jk(dD, self.thresh / m, self.split / m)
                    J, K = J + Jd, K + Kd
                kind = "incremental"
            D_ref = D
            b.record()
            b.synchronize()
            builds.append((kind, a.elapsed_time(b)))
            F = H + J - 0.5 * K
            E = 0.5 * float(torch.sum(D * (H + F)).item()) + self.e_nuc
            err = F @ D @ S - S @ D @ F
            gnorm = float(err.abs().max().item())
            if E_old is not None and abs(E - E_old) < e_tol and gnorm < g_tol:
                return dict(energy=E, D=D, iterations=it, converged=True, builds=builds, gradient_norm=gnorm)
            E_old = E
            focks.append(F)
            errs.append(err)
            focks, errs = focks[-diis_size:], errs[-diis_size:]
            n = len(focks)
            if n >= 2:
                B = -torch.ones((n + 1, n + 1), dtype=torch.float64, device=F.device)
                B[n, n] = 0.0
                for i in range(n):
                    for j in range(n):
                        B[i, j] = torch.sum(errs[i] * errs[j])
                rhs = torch.zeros(n + 1, dtype=torch.float64, device=F.device)
                rhs[n] = -1.0
                c = torch.linalg.solve(B, rhs)[:n]
                F = sum(c[i] * focks[i] for i in range(n))
            D = self._density(F)
        return dict(energy=E, D=D, iterations=max_iter, converged=False, builds=builds, gradient_norm=gnorm)


def nuclear_repulsion_gradient(atoms, charges) -> np.ndarray:
    """d/dR_A sum_{A<B} Z_A Z_B / |R_A - R_B|, [natom, 3]."""
    X = np.asarray(atoms, dtype=np.float64)
    Z = np.asarray(charges, dtype=np.float64)
    d = X[:, None, :] - X[None, :, :]
    r = np.linalg.norm(d, axis=-1)
    np.fill_diagonal(r, np.inf)
    return -np.sum((Z[:, None] * Z[None, :] / r ** 3)[..., None] * d, axis=1)


def scf_gradient(rhf: RHF, result: dict):
    """Nuclear gradient [natom, 3] (CUDA float64) of a converged RHF energy,
    the single-point force task: sum D dH/dR - sum W dS/dR with
    W = 1/2 D F D (adft_one_electron_grad), plus dE_JK/dR at fixed D
    (adft_jk_grad, F = H + J - 1/2 K so E_JK = 1/2 tr(DJ) - 1/4 tr(DK)), plus
    the nuclear repulsion gradient."""
    torch = rhf.torch
    D = result["D"]
    J, K = rhf._jk(D, rhf.thresh, rhf.split)
    F = rhf.H + J - 0.5 * K
    W = 0.5 * (D @ F @ D)
    W = 0.5 * (W + W.T)
    g = adft.adft_one_electron_grad(rhf.basis, rhf.charges, D, W, stream=rhf.stream)
    g = g + adft.adft_jk_grad(rhf.basis, D, thresh=rhf.thresh, split=rhf.split, precision=rhf.precision, check=False,
                              stream=rhf.stream)
    return g + torch.as_tensor(nuclear_repulsion_gradient(rhf.mol.atoms, rhf.charges), device=g.device)


def run_scf(mol, **kw) -> dict:
    """RHF(mol, **options).run() with a wall-clock time added."""
    t = time.time()
    opts = {k: kw.pop(k) for k in ("max_iter", "e_tol", "g_tol", "diis_size") if k in kw}
    r = RHF(mol, **kw).run(**opts)
    r["wall_s"] = time.time() - t
    return r
