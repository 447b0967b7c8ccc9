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


def prim_block(ls, centres, exps):
    """Unnormalised primitive [ab|cd] for all Cartesian components."""
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

    res, err = quad_vec(f, 0.0, 1.0, epsabs=1e-16, epsrel=1e-13, limit=400)
    return res.reshape(len(ca), len(cb), len(cc), len(cd))
