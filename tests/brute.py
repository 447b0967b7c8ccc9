"""Independent brute-force evaluation of primitive Cartesian ERIs for pins.

Uses 1/r12 = (2/sqrt(pi)) int_0^inf exp(-t^2 r12^2) dt.  For fixed t the
six-dimensional integral factorises into three two-dimensional integrals of a
polynomial times a Gaussian, which tensor Gauss-Hermite quadrature evaluates
exactly after the quadratic form is diagonalised by a Cholesky factor; the
t-integral is done by adaptive quadrature after t = u / (1 - u).  Nothing here
uses Hermite expansions, recurrences or the Boys function.
"""
import math

import numpy as np
from scipy.integrate import quad_vec


def cart_powers(l):
    return [(i, j, l - i - j) for i in range(l, -1, -1) for j in range(l - i, -1, -1)]


_GX, _GW = np.polynomial.hermite.hermgauss(12)


def _pair_integrals(t, la, lb, lc, ld, A, B, C, D, a, b, c, d):
    """I[k][i][j][m][n] for the three directions k at parameter t."""
    out = []
    for k in range(3):
        M = np.array([[a + b + t * t, -t * t], [-t * t, c + d + t * t]])
        h = np.array([a * A[k] + b * B[k], c * C[k] + d * D[k]])
        s0 = a * A[k] ** 2 + b * B[k] ** 2 + c * C[k] ** 2 + d * D[k] ** 2
        m = np.linalg.solve(M, h)
        const = s0 - h @ m
        L = np.linalg.cholesky(M)
        Linv_T = np.linalg.inv(L).T
        y1, y2 = np.meshgrid(_GX, _GX, indexing="ij")
        w = np.outer(_GW, _GW)
        x1 = m[0] + Linv_T[0, 0] * y1 + Linv_T[0, 1] * y2
        x2 = m[1] + Linv_T[1, 0] * y1 + Linv_T[1, 1] * y2
        pa = np.stack([(x1 - A[k]) ** i for i in range(la + 1)])
        pb = np.stack([(x1 - B[k]) ** i for i in range(lb + 1)])
        pc = np.stack([(x2 - C[k]) ** i for i in range(lc + 1)])
        pd = np.stack([(x2 - D[k]) ** i for i in range(ld + 1)])
        I = np.einsum("ixy,jxy,kxy,lxy,xy->ijkl", pa, pb, pc, pd, w) * math.exp(-const) / np.prod(np.diag(L))
        out.append(I)
    return out


def prim_block(ls, centres, exps, omega=None):
    """Unnormalised primitive [ab|cd] for all Cartesian components; with
    omega, over erf(omega r12)/r12 = (2/sqrt(pi)) int_0^omega exp(-t^2 r12^2) dt
    (the same t-integral stopped at t = omega)."""
    la, lb, lc, ld = ls
    A, B, C, D = (np.asarray(x, dtype=float) for x in centres)
    a, b, c, d = exps
    ca, cb, cc, cd = (cart_powers(l) for l in ls)

    def f(u):
        if u >= 1.0:
            return np.zeros(len(ca) * len(cb) * len(cc) * len(cd))
        t = u / (1.0 - u)
        I = _pair_integrals(t, la, lb, lc, ld, A, B, C, D, a, b, c, d)
        vals = np.empty((len(ca), len(cb), len(cc), len(cd)))
        for i, pa in enumerate(ca):
            for j, pb in enumerate(cb):
                for k, pc in enumerate(cc):
                    for m, pd in enumerate(cd):
                        v = 1.0
                        for x in range(3):
                            v *= I[x][pa[x], pb[x], pc[x], pd[x]]
                        vals[i, j, k, m] = v
        return vals.ravel() * (2.0 / math.sqrt(math.pi)) / (1.0 - u) ** 2

    u_max = 1.0 if omega is None else omega / (1.0 + omega)
    res, err = quad_vec(f, 0.0, u_max, epsabs=1e-16, epsrel=1e-13, limit=400)
    return res.reshape(len(ca), len(cb), len(cc), len(cd))


# ----------------------------------------------------------------------------
# One-electron integrals by quadrature (no Hermite expansions, no Boys
# function): every one-dimensional factor is a polynomial times one Gaussian,
# which Gauss-Hermite quadrature integrates exactly.

def _gauss_1d(polys, expo, centre):
    """int prod(polys)(x) exp(-expo (x - centre)^2) dx for callables of x."""
    x = centre + _GX / math.sqrt(expo)
    v = np.ones_like(x)
    for f in polys:
        v = v * f(x)
    return float(np.sum(_GW * v)) / math.sqrt(expo)


def _prim_norm(a, l):
    df = 1.0
    for k in range(2 * l - 1, 1, -2):
        df *= k
    return (2 * a / math.pi) ** 0.75 * (4 * a) ** (l / 2) / math.sqrt(df)


def one_electron_cartesian(mol, charges, what="T"):
    """Cartesian kinetic (what="T", as 1/2 sum_k <d_k a|d_k b>) or nuclear
    attraction (what="V", with 1/|r-C| = (2/sqrt(pi)) int_0^inf exp(-t^2 |r-C|^2) dt
    and the t-integral by adaptive quadrature after t = sqrt(p) u / (1 - u)) matrix
    of a small molecule."""
    shells = mol.shells
    offs, o = [], 0
    for _, l, _, _ in shells:
        offs.append(o)
        o += (l + 1) * (l + 2) // 2
    M = np.zeros((o, o))
    atoms = np.asarray(mol.atoms, dtype=float)
    for sa, (ia_, la, ea, ca) in enumerate(shells):
        for sb, (ib_, lb, eb, cb) in enumerate(shells):
            A, B = atoms[ia_], atoms[ib_]
            for a, c1 in zip(ea, ca):
                for b, c2 in zip(eb, cb):
                    w = c1 * c2 * _prim_norm(a, la) * _prim_norm(b, lb)
                    p = a + b
                    P = (a * A + b * B) / p
                    kab = math.exp(-a * b / p * float(np.sum((A - B) ** 2)))
                    for i, pa in enumerate(cart_powers(la)):
                        for j, pb in enumerate(cart_powers(lb)):
                            if what == "T":
                                S1, D1 = [], []
                                for k in range(3):
                                    fa = lambda x, k=k, e=pa[k]: (x - A[k]) ** e
                                    fb = lambda x, k=k, e=pb[k]: (x - B[k]) ** e
                                    da = lambda x, k=k, e=pa[k]: (e * (x - A[k]) ** (e - 1) if e else 0.0) - 2 * a * (x - A[k]) ** (e + 1)
                                    db = lambda x, k=k, e=pb[k]: (e * (x - B[k]) ** (e - 1) if e else 0.0) - 2 * b * (x - B[k]) ** (e + 1)
                                    S1.append(_gauss_1d([fa, fb], p, P[k]))
                                    D1.append(_gauss_1d([da, db], p, P[k]))
                                v = 0.5 * (D1[0] * S1[1] * S1[2] + S1[0] * D1[1] * S1[2] + S1[0] * S1[1] * D1[2])
                                M[offs[sa] + i, offs[sb] + j] += w * kab * v
                            else:
                                tot = 0.0
                                for C, Z in zip(atoms, charges):
                                    sc = math.sqrt(p)  # the integrand's scale in t

                                    def f(u):
                                        if u >= 1.0:
                                            return 0.0
                                        t = sc * u / (1.0 - u)
                                        q = p + t * t
                                        Rq = (p * P + t * t * C) / q
                                        g = math.exp(-p * t * t / q * float(np.sum((P - C) ** 2)))
                                        v = g
                                        for k in range(3):
                                            fa = lambda x, k=k, e=pa[k]: (x - A[k]) ** e
                                            fb = lambda x, k=k, e=pb[k]: (x - B[k]) ** e
                                            v *= _gauss_1d([fa, fb], q, Rq[k])
                                        return v * (2.0 / math.sqrt(math.pi)) * sc / (1.0 - u) ** 2
                                    val, _ = quad_vec(f, 0.0, 1.0, epsabs=1e-15, epsrel=1e-12, limit=400)
                                    tot += -Z * float(val)
                                M[offs[sa] + i, offs[sb] + j] += w * kab * tot
    return M
