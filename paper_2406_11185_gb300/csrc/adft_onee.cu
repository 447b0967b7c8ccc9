// One-electron integrals of the core Hamiltonian (overlap S, kinetic energy T,
// nuclear attraction V) for the SCF driver around the J/K build: the Fock
// matrix of Eq. 1 (Sec. 1.2.1) is F = H + J - 1/2 c_x K with H = T + V.
// McMurchie-Davidson (Helgaker, Jorgensen and Olsen, Sec. 9.3 and 9.9):
//   S_ij = E^{ij}_0 sqrt(pi/p) per direction,
//   T_ij = -1/2 [ j(j-1) S_{i,j-2} - 2b(2j+1) S_ij + 4b^2 S_{i,j+2} ] per direction
//          (the second derivative of the ket Gaussian), T = Tx Sy Sz + ...,
//   V = -sum_C Z_C (2 pi / p) sum_tuv E^{ij}_t E^{kl}_u E^{mn}_v R_tuv(p, P - C).
// One thread per ordered shell pair; the blocks are written to full Cartesian
// matrices and transformed to the output basis like J and K.  Called once per
// geometry, so it favours simplicity over speed.
#include "adft_eri.cuh"

namespace adft {

struct OneElecArgs {
  BasisView bv;
  const int* shell_nprim;
  const int* shell_poff;
  const double* exps;
  const double* ncoefs;  // c_i N(a_i, l)
  const double* charges; // [natom]
  double* S;             // Cartesian [ncart][ncart]
  double* T;
  double* V;
};

__global__ void __launch_bounds__(128) k_one_electron(OneElecArgs g) {
  const BasisView& bv = g.bv;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)bv.nshell * bv.nshell) return;
  const int sa = (int)(idx / bv.nshell), sb = (int)(idx % bv.nshell);
  const int la = bv.shell_l[sa], lb = bv.shell_l[sb];
  const int na = ncart(la), nb = ncart(lb);
  const double* A = bv.xyz + 3 * bv.shell_atom[sa];
  const double* B = bv.xyz + 3 * bv.shell_atom[sb];
  const int oa = bv.shell_coff[sa], ob = bv.shell_coff[sb], nc = bv.ncart;
  constexpr int NCMAX = ncart(LMAX);
  constexpr int EMAX = (LMAX + 1) * (LMAX + 3) * (2 * LMAX + 3);  // E up to (la, lb + 2)
  double sblk[NCMAX * NCMAX], tblk[NCMAX * NCMAX], vblk[NCMAX * NCMAX];
  for (int x = 0; x < na * nb; ++x) sblk[x] = tblk[x] = vblk[x] = 0.0;
  const int jm = lb + 2, nt = la + jm + 1;  // kinetic needs j + 2
  const int se = (la + 1) * (jm + 1) * nt;
  double E[3 * EMAX];
  double R[nherm(2 * LMAX)];
  const double ABx = A[0] - B[0], ABy = A[1] - B[1], ABz = A[2] - B[2];
  const double rab2 = ABx * ABx + ABy * ABy + ABz * ABz;
  for (int i = 0; i < g.shell_nprim[sa]; ++i)
    for (int j = 0; j < g.shell_nprim[sb]; ++j) {
      const double a = g.exps[g.shell_poff[sa] + i], b = g.exps[g.shell_poff[sb] + j];
      const double p = a + b, o2p = 0.5 / p;
      const double cc = g.ncoefs[g.shell_poff[sa] + i] * g.ncoefs[g.shell_poff[sb] + j] * exp(-a * b / p * rab2);
      double P[3];
      for (int k = 0; k < 3; ++k) {
        P[k] = (a * A[k] + b * B[k]) / p;
        hermite_E_rt<double>(la, jm, P[k] - A[k], P[k] - B[k], o2p, E + k * se);
      }
      const double sq = sqrt(3.14159265358979323846 / p);
#define EE(k, ii, jj, t) E[(k) * se + ((ii) * (jm + 1) + (jj)) * nt + (t)]
      for (int ia = 0; ia < na; ++ia) {
        int ax[3];
        cart_pows_rt(la, ia, ax[0], ax[1], ax[2]);
        for (int ib = 0; ib < nb; ++ib) {
          int bx[3];
          cart_pows_rt(lb, ib, bx[0], bx[1], bx[2]);
          double s1[3], t1[3];
          for (int k = 0; k < 3; ++k) {
            const int ii = ax[k], jj = bx[k];
            s1[k] = EE(k, ii, jj, 0) * sq;
            const double sm2 = jj >= 2 ? EE(k, ii, jj - 2, 0) * sq : 0.0;
            const double sp2 = EE(k, ii, jj + 2, 0) * sq;
            t1[k] = -0.5 * (jj * (jj - 1) * sm2 - 2.0 * b * (2 * jj + 1) * s1[k] + 4.0 * b * b * sp2);
          }
          sblk[ia * nb + ib] += cc * s1[0] * s1[1] * s1[2];
          tblk[ia * nb + ib] += cc * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2]);
        }
      }
      const int L = la + lb;
      for (int c = 0; c < bv.natom; ++c) {
        const double* C = bv.xyz + 3 * c;
        prim_R_rt<double>(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], bv, R);
        const double pref = -g.charges[c] * 2.0 * 3.14159265358979323846 / p * cc;
        for (int ia = 0; ia < na; ++ia) {
          int ax[3];
          cart_pows_rt(la, ia, ax[0], ax[1], ax[2]);
          for (int ib = 0; ib < nb; ++ib) {
            int bx[3];
            cart_pows_rt(lb, ib, bx[0], bx[1], bx[2]);
            double s = 0.0;
            for (int t = 0; t <= ax[0] + bx[0]; ++t)
              for (int u = 0; u <= ax[1] + bx[1]; ++u)
                for (int v = 0; v <= ax[2] + bx[2]; ++v)
                  s += EE(0, ax[0], bx[0], t) * EE(1, ax[1], bx[1], u) * EE(2, ax[2], bx[2], v) * R[hidx_rt(t, u, v)];
            vblk[ia * nb + ib] += pref * s;
          }
        }
      }
#undef EE
    }
  for (int ia = 0; ia < na; ++ia)
    for (int ib = 0; ib < nb; ++ib) {
      const long long o = (long long)(oa + ia) * nc + ob + ib;
      g.S[o] = sblk[ia * nb + ib];
      g.T[o] = tblk[ia * nb + ib];
      g.V[o] = vblk[ia * nb + ib];
    }
}

cudaError_t launch_one_electron(const BasisView& bv, const int* shell_nprim, const int* shell_poff,
                                const double* exps, const double* ncoefs, const double* charges, double* S,
                                double* T, double* V, cudaStream_t s) {
  OneElecArgs g{bv, shell_nprim, shell_poff, exps, ncoefs, charges, S, T, V};
  const long long n = (long long)bv.nshell * bv.nshell;
  if (n == 0) return cudaSuccess;
  k_one_electron<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Nuclear gradient of the one-electron part of the closed-shell SCF energy
// (the single-point force task around the J/K gradient):
//   grad_R += sum_{mu nu} D_mu,nu dH_mu,nu/dR - sum_{mu nu} W_mu,nu dS_mu,nu/dR,
// W the energy-weighted density.  A primitive's derivative with respect to its
// centre, d/dA_k [x^i exp(-a x^2)] = 2a x^(i+1) exp(..) - i x^(i-1) exp(..)
// (x = the k coordinate relative to A), turns every derivative into raised
// and lowered integrals of the same McMurchie-Davidson tables; a nuclear
// attraction term moves with its nucleus C as -(d/dA + d/dB) (translational
// invariance).  One thread per ordered shell pair; contributions go to the
// gradient by FP64 atomics.  Dc and Wc are Cartesian [ncart][ncart].

struct OneElecGradArgs {
  BasisView bv;
  const int* shell_nprim;
  const int* shell_poff;
  const double* exps;
  const double* ncoefs;
  const double* charges;  // [natom]
  const double* Dc;
  const double* Wc;
  double* grad;           // [natom][3], accumulated
};

__global__ void __launch_bounds__(128) k_one_electron_grad(OneElecGradArgs g) {
  const BasisView& bv = g.bv;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)bv.nshell * bv.nshell) return;
  const int sa = (int)(idx / bv.nshell), sb = (int)(idx % bv.nshell);
  const int la = bv.shell_l[sa], lb = bv.shell_l[sb];
  const int na = ncart(la), nb = ncart(lb);
  const int atA = bv.shell_atom[sa], atB = bv.shell_atom[sb];
  const double* A = bv.xyz + 3 * atA;
  const double* B = bv.xyz + 3 * atB;
  const int oa = bv.shell_coff[sa], ob = bv.shell_coff[sb], nc = bv.ncart;
  // E up to (la + 1, lb + 3): raised bra, raised ket plus the kinetic j + 2
  constexpr int EMAX = (LMAX + 2) * (LMAX + 4) * (2 * LMAX + 6);
  const int im = la + 1, jm = lb + 3, nt = im + jm + 1;
  const int se = (im + 1) * (jm + 1) * nt;
  double E[3 * EMAX];
  double R[nherm(2 * LMAX + 1)];
  const double ABx = A[0] - B[0], ABy = A[1] - B[1], ABz = A[2] - B[2];
  const double rab2 = ABx * ABx + ABy * ABy + ABz * ABz;
  double gA[3] = {0.0, 0.0, 0.0}, gB[3] = {0.0, 0.0, 0.0};
#define EE(k, ii, jj, t) E[(k) * se + ((ii) * (jm + 1) + (jj)) * nt + (t)]
  for (int i = 0; i < g.shell_nprim[sa]; ++i)
    for (int j = 0; j < g.shell_nprim[sb]; ++j) {
      const double a = g.exps[g.shell_poff[sa] + i], b = g.exps[g.shell_poff[sb] + j];
      const double p = a + b, o2p = 0.5 / p;
      const double cc = g.ncoefs[g.shell_poff[sa] + i] * g.ncoefs[g.shell_poff[sb] + j] * exp(-a * b / p * rab2);
      double P[3];
      for (int k = 0; k < 3; ++k) {
        P[k] = (a * A[k] + b * B[k]) / p;
        hermite_E_rt<double>(im, jm, P[k] - A[k], P[k] - B[k], o2p, E + k * se);
      }
      const double sq = sqrt(3.14159265358979323846 / p);
      // overlap and kinetic parts
      for (int ia = 0; ia < na; ++ia) {
        int ax[3];
        cart_pows_rt(la, ia, ax[0], ax[1], ax[2]);
        for (int ib = 0; ib < nb; ++ib) {
          int bx[3];
          cart_pows_rt(lb, ib, bx[0], bx[1], bx[2]);
          const long long o = (long long)(oa + ia) * nc + ob + ib;
          const double dw = g.Dc[o], ww = g.Wc[o];
          for (int side = 0; side < 2; ++side)
            for (int k = 0; k < 3; ++k) {
              const double ex = side == 0 ? a : b;
              const int p0 = side == 0 ? ax[k] : bx[k];
              double ds = 0.0, dt = 0.0;
              for (int term = 0; term < 2; ++term) {
                if (term == 1 && p0 == 0) break;
                const double f = term == 0 ? 2.0 * ex : -(double)p0;
                int pa[3] = {ax[0], ax[1], ax[2]}, pb[3] = {bx[0], bx[1], bx[2]};
                if (side == 0) pa[k] = term == 0 ? p0 + 1 : p0 - 1;
                else pb[k] = term == 0 ? p0 + 1 : p0 - 1;
                double s1[3], t1[3];
                for (int d = 0; d < 3; ++d) {
                  const int ii = pa[d], jj = pb[d];
                  s1[d] = EE(d, ii, jj, 0) * sq;
                  const double sm2 = jj >= 2 ? EE(d, ii, jj - 2, 0) * sq : 0.0;
                  const double sp2 = EE(d, ii, jj + 2, 0) * sq;
                  t1[d] = -0.5 * (jj * (jj - 1) * sm2 - 2.0 * b * (2 * jj + 1) * s1[d] + 4.0 * b * b * sp2);
                }
                ds += f * s1[0] * s1[1] * s1[2];
                dt += f * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2]);
              }
              const double v = cc * (dw * dt - ww * ds);
              if (side == 0) gA[k] += v; else gB[k] += v;
            }
        }
      }
      // nuclear attraction: each nucleus's term moves with A, B and C
      const int L1 = la + lb + 1;
      for (int c = 0; c < bv.natom; ++c) {
        const double* C = bv.xyz + 3 * c;
        prim_R_rt<double>(L1, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], bv, R);
        const double pref = -g.charges[c] * 2.0 * 3.14159265358979323846 / p * cc;
        double gc[3] = {0.0, 0.0, 0.0};
        for (int ia = 0; ia < na; ++ia) {
          int ax[3];
          cart_pows_rt(la, ia, ax[0], ax[1], ax[2]);
          for (int ib = 0; ib < nb; ++ib) {
            int bx[3];
            cart_pows_rt(lb, ib, bx[0], bx[1], bx[2]);
            const double dw = g.Dc[(long long)(oa + ia) * nc + ob + ib];
            if (dw == 0.0) continue;
            for (int side = 0; side < 2; ++side)
              for (int k = 0; k < 3; ++k) {
                const double ex = side == 0 ? a : b;
                const int p0 = side == 0 ? ax[k] : bx[k];
                double dv = 0.0;
                for (int term = 0; term < 2; ++term) {
                  if (term == 1 && p0 == 0) break;
                  const double f = term == 0 ? 2.0 * ex : -(double)p0;
                  int pa[3] = {ax[0], ax[1], ax[2]}, pb[3] = {bx[0], bx[1], bx[2]};
                  if (side == 0) pa[k] = term == 0 ? p0 + 1 : p0 - 1;
                  else pb[k] = term == 0 ? p0 + 1 : p0 - 1;
                  double s = 0.0;
                  for (int t = 0; t <= pa[0] + pb[0]; ++t)
                    for (int u = 0; u <= pa[1] + pb[1]; ++u)
                      for (int w = 0; w <= pa[2] + pb[2]; ++w)
                        s += EE(0, pa[0], pb[0], t) * EE(1, pa[1], pb[1], u) * EE(2, pa[2], pb[2], w) *
                             R[hidx_rt(t, u, w)];
                  dv += f * s;
                }
                const double v = pref * dw * dv;
                if (side == 0) gA[k] += v; else gB[k] += v;
                gc[k] -= v;
              }
          }
        }
        for (int k = 0; k < 3; ++k)
          if (gc[k] != 0.0) atomicAdd(g.grad + 3 * c + k, gc[k]);
      }
    }
#undef EE
  for (int k = 0; k < 3; ++k) {
    atomicAdd(g.grad + 3 * atA + k, gA[k]);
    atomicAdd(g.grad + 3 * atB + k, gB[k]);
  }
}

cudaError_t launch_one_electron_grad(const BasisView& bv, const int* shell_nprim, const int* shell_poff,
                                     const double* exps, const double* ncoefs, const double* charges,
                                     const double* Dc, const double* Wc, double* grad, cudaStream_t s) {
  OneElecGradArgs g{bv, shell_nprim, shell_poff, exps, ncoefs, charges, Dc, Wc, grad};
  const long long n = (long long)bv.nshell * bv.nshell;
  if (n == 0) return cudaSuccess;
  k_one_electron_grad<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g);
  return cudaGetLastError();
}

}  // namespace adft
