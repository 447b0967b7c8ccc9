/*
 * oracle.c -- plain, slow FP64 CPU oracle for the direct-SCF Coulomb/exchange
 * (J/K) build of the Accelerated DFT paper (arXiv 2406.11185).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * What it computes (the plain definitions, evaluated with no shortcut other
 * than the 8-fold permutational symmetry of the integrals):
 *
 *   (mu nu|la si) = int int phi_mu(r) phi_nu(r) phi_la(r') phi_si(r') / |r-r'|
 *                                                   (Sec. 1.2.2, ERI paragraph)
 *   J_mu,nu = sum_{la,si} D_la,si (mu nu|la si)        (Eq. 1, Coulomb term)
 *   K_mu,nu = sum_{la,si} D_la,si (mu la|nu si)        (Eq. 1, exchange term,
 *                                                       c_x applied by caller)
 *   Schwarz screening: a shell quartet (ab|cd) is dropped iff
 *   Q_ab * Q_cd < thresh, Q_ab = sqrt(max_{mu in a, nu in b} |(mu nu|mu nu)|)
 *                                      (Sec. 1.2.2, mixed-precision bullet)
 *   dE/dR_A with E = 1/2 tr(DJ) - 1/4 tr(DK) at fixed D, and its second
 *   derivatives d2E/dR_A dR_B at fixed D; the one-electron part of the
 *   closed-shell SCF force.
 *   Optionally the long-range (erf-attenuated) operator erf(omega r)/r in
 *   place of 1/r in the ERIs and J, K (range-separated hybrids; omega > 0).
 *
 * Primitive integrals follow the McMurchie-Davidson scheme as written in
 * Helgaker, Jorgensen and Olsen, "Molecular Electronic-Structure Theory",
 * Sec. 9.5 (Hermite expansion coefficients), 9.8 (Boys function) and 9.9
 * (Hermite Coulomb integrals, two-electron integrals, eq. 9.9.33).  The Boys
 * function is evaluated in long double.  Everything is done in the Cartesian
 * basis; the Python wrapper transforms D to Cartesian and J, K back.
 *
 * Basis convention: contracted shells sum_i c_i N(a_i,l) x^ax y^ay z^az
 * exp(-a_i r^2) with N(a,l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!) for
 * every Cartesian component; components ordered by descending x then y power.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 5                 /* shell l up to 4, +1 for derivatives */
#define ORC_LT (4 * ORC_LMAX + 1)  /* largest total L handled by R tables */
#define ORC_NC(l) (((l) + 1) * ((l) + 2) / 2)

static const long double ORC_PI = 3.141592653589793238462643383279502884L;

/* ------------------------------------------------------------------------ */
/* Boys function F_m(T) = int_0^1 t^(2m) exp(-T t^2) dt  (Helgaker Sec. 9.8) */

static void boys_ld(int mmax, long double T, long double *F) {
  if (T < 30.0L) {
    /* series F_m = e^-T sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)), then
       downward recursion F_m = (2T F_{m+1} + e^-T) / (2m+1) */
    long double term = 1.0L / (2 * mmax + 1), sum = term;
    for (int k = 1; k < 100000; ++k) {
      term *= 2.0L * T / (2 * mmax + 2 * k + 1);
      sum += term;
      if (term < 1e-24L * sum) break;
    }
    long double e = expl(-T);
    F[mmax] = e * sum;
    for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0L * T * F[m + 1] + e) / (2 * m + 1);
  } else {
    /* F_0 = 1/2 sqrt(pi/T) erf(sqrt T), upward recursion (stable for T > m) */
    long double e = expl(-T);
    F[0] = 0.5L * sqrtl(ORC_PI / T) * erfl(sqrtl(T));
    for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) / (2.0L * T);
  }
}

void orc_boys(int mmax, double T, double *F) {
  long double Fl[64];
  boys_ld(mmax, (long double)T, Fl);
  for (int m = 0; m <= mmax; ++m) F[m] = (double)Fl[m];
}

/* ------------------------------------------------------------------------ */
/* Hermite expansion coefficients E^{ij}_t of one Cartesian direction
   (Helgaker eqs. 9.5.6, 9.5.7): x_A^i x_B^j exp(-a x_A^2 - b x_B^2)
   = sum_t E^{ij}_t Lambda_t(x; p, P_x). Layout E[(i*(jmax+1)+j)*(imax+jmax+1)+t]. */

static void hermite_e(int imax, int jmax, double a, double b, double Ax, double Bx, double *E) {
  const int nt = imax + jmax + 1;
  const double p = a + b, mu = a * b / p;
  const double Px = (a * Ax + b * Bx) / p;
  const double XAB = Ax - Bx, XPA = Px - Ax, XPB = Px - Bx, o2p = 0.5 / p;
#define EIDX(i, j, t) ((((i) * (jmax + 1)) + (j)) * nt + (t))
  memset(E, 0, sizeof(double) * (size_t)(imax + 1) * (jmax + 1) * nt);
  E[EIDX(0, 0, 0)] = exp(-mu * XAB * XAB);
  for (int i = 0; i <= imax; ++i) {
    for (int j = 0; j <= jmax; ++j) {
      if (i == 0 && j == 0) continue;
      for (int t = 0; t <= i + j; ++t) {
        double v;
        if (j == 0) { /* raise i from (i-1, 0) */
          double em = (t > 0) ? E[EIDX(i - 1, 0, t - 1)] : 0.0;
          double e0 = (t <= i - 1) ? E[EIDX(i - 1, 0, t)] : 0.0;
          double ep = (t + 1 <= i - 1) ? E[EIDX(i - 1, 0, t + 1)] : 0.0;
          v = o2p * em + XPA * e0 + (t + 1) * ep;
        } else { /* raise j from (i, j-1) */
          double em = (t > 0) ? E[EIDX(i, j - 1, t - 1)] : 0.0;
          double e0 = (t <= i + j - 1) ? E[EIDX(i, j - 1, t)] : 0.0;
          double ep = (t + 1 <= i + j - 1) ? E[EIDX(i, j - 1, t + 1)] : 0.0;
          v = o2p * em + XPB * e0 + (t + 1) * ep;
        }
        E[EIDX(i, j, t)] = v;
      }
    }
  }
#undef EIDX
}

/* ------------------------------------------------------------------------ */
/* Hermite Coulomb integrals R_{tuv} = R^0_{tuv} (Helgaker eqs. 9.9.18-9.9.20):
   R^n_{000} = (-2 alpha)^n F_n(alpha |PQ|^2), raised in t, u or v from R^{n+1}. */

/* R is stored as R[(t*(L+1)+u)*(L+1)+v]. */
#define RIDX(t, u, v) ((((t) * (L + 1)) + (u)) * (L + 1) + (v))

static void hermite_r(int L, double alpha, double X, double Y, double Z, double *R) {
  long double F[ORC_LT + 1];
  boys_ld(L, (long double)alpha * ((long double)X * X + (long double)Y * Y + (long double)Z * Z), F);
  const int sz = (L + 1) * (L + 1) * (L + 1);
  double bufa[sz], bufb[sz];
  double *cur = bufa, *nxt = bufb;
  for (int n = L; n >= 0; --n) {
    /* cur = R^n from nxt = R^{n+1} */
    long double pw = 1.0L;
    for (int k = 0; k < n; ++k) pw *= -2.0L * alpha;
    for (int t = 0; t <= L - n; ++t)
      for (int u = 0; u <= L - n - t; ++u)
        for (int v = 0; v <= L - n - t - u; ++v) {
          double val;
          if (t == 0 && u == 0 && v == 0) {
            val = (double)(pw * F[n]);
          } else if (t > 0) {
            val = X * nxt[RIDX(t - 1, u, v)];
            if (t > 1) val += (t - 1) * nxt[RIDX(t - 2, u, v)];
          } else if (u > 0) {
            val = Y * nxt[RIDX(t, u - 1, v)];
            if (u > 1) val += (u - 1) * nxt[RIDX(t, u - 2, v)];
          } else {
            val = Z * nxt[RIDX(t, u, v - 1)];
            if (v > 1) val += (v - 1) * nxt[RIDX(t, u, v - 2)];
          }
          cur[RIDX(t, u, v)] = val;
        }
    double *tmp = cur; cur = nxt; nxt = tmp;
  }
  /* after the loop the last computed layer (n = 0) sits in nxt */
  for (int t = 0; t <= L; ++t)
    for (int u = 0; u <= L - t; ++u)
      for (int v = 0; v <= L - t - u; ++v) R[RIDX(t, u, v)] = nxt[RIDX(t, u, v)];
}

/* ------------------------------------------------------------------------ */
/* Cartesian component lists */

static void cart_list(int l, int *pw /* [ncart][3] */) {
  int k = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j) {
      pw[3 * k + 0] = i; pw[3 * k + 1] = j; pw[3 * k + 2] = l - i - j; ++k;
    }
}

static int cart_index(int l, int ax, int ay) {
  /* position of (ax, ay, l-ax-ay) in cart_list(l) */
  int k = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j) {
      if (i == ax && j == ay) return k;
      ++k;
    }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Primitive block: out[ia][ib][ic][id] += scale * [ab|cd] for all Cartesian
   components of total powers la, lb, lc, ld (unnormalised primitives), by
   Helgaker eq. 9.9.33:
   [ab|cd] = 2 pi^(5/2) / (p q sqrt(p+q)) sum_{tuv} E^ab_{tuv}
             sum_{tau nu phi} (-1)^(tau+nu+phi) E^cd_{tau nu phi} R_{t+tau,u+nu,v+phi} */

/* With omega > 0 the operator is erf(omega r12)/r12.  Its Fourier transform
   is that of 1/r12 times exp(-k^2/(4 omega^2)), and the two charge
   distributions contribute exp(-k^2/(4p)) exp(-k^2/(4q)) = exp(-k^2/(4 alpha)),
   so the integral is the Coulomb one with 1/alpha replaced by
   1/alpha + 1/omega^2: alpha_w = alpha w / (alpha + w), w = omega^2, in the
   Boys argument and in the (-2 alpha)^n of the Hermite integrals, and the
   prefactor 2 pi^(5/2) / (p q sqrt(p+q)) times sqrt(alpha_w / alpha). */
static void prim_block_w(int la, int lb, int lc, int ld,
                         const double *A, double a, const double *B, double b,
                         const double *C, double c, const double *D, double d,
                         double scale, double omega, double *out) {
  if (la < 0 || lb < 0 || lc < 0 || ld < 0) return;
  const int L = la + lb + lc + ld;
  const double p = a + b, q = c + d, alpha_c = p * q / (p + q);
  const double w = omega * omega;
  const double alpha = omega > 0.0 ? alpha_c * w / (alpha_c + w) : alpha_c;
  double P[3], Q[3];
  for (int k = 0; k < 3; ++k) {
    P[k] = (a * A[k] + b * B[k]) / p;
    Q[k] = (c * C[k] + d * D[k]) / q;
  }
  const int ntab = la + lb + 1, ntcd = lc + ld + 1;
  double Eab[3 * (la + 1) * (lb + 1) * ntab];
  double Ecd[3 * (lc + 1) * (ld + 1) * ntcd];
  const int sab = (la + 1) * (lb + 1) * ntab, scd = (lc + 1) * (ld + 1) * ntcd;
  for (int k = 0; k < 3; ++k) {
    hermite_e(la, lb, a, b, A[k], B[k], Eab + k * sab);
    hermite_e(lc, ld, c, d, C[k], D[k], Ecd + k * scd);
  }
  double R[(L + 1) * (L + 1) * (L + 1)];
  hermite_r(L, alpha, P[0] - Q[0], P[1] - Q[1], P[2] - Q[2], R);
  const double pref = scale * 2.0 * pow((double)ORC_PI, 2.5) / (p * q * sqrt(p + q)) * sqrt(alpha / alpha_c);

  int pa[3 * ORC_NC(ORC_LMAX)], pb[3 * ORC_NC(ORC_LMAX)], pc[3 * ORC_NC(ORC_LMAX)], pd[3 * ORC_NC(ORC_LMAX)];
  cart_list(la, pa); cart_list(lb, pb); cart_list(lc, pc); cart_list(ld, pd);
  const int na = ORC_NC(la), nb = ORC_NC(lb), nc = ORC_NC(lc), nd = ORC_NC(ld);
#define EAB(k, i, j, t) Eab[(k) * sab + ((i) * (lb + 1) + (j)) * ntab + (t)]
#define ECD(k, i, j, t) Ecd[(k) * scd + ((i) * (ld + 1) + (j)) * ntcd + (t)]
  for (int ia = 0; ia < na; ++ia)
    for (int ib = 0; ib < nb; ++ib)
      for (int ic = 0; ic < nc; ++ic)
        for (int id = 0; id < nd; ++id) {
          const int *xa = pa + 3 * ia, *xb = pb + 3 * ib, *xc = pc + 3 * ic, *xd = pd + 3 * id;
          double s = 0.0;
          for (int t = 0; t <= xa[0] + xb[0]; ++t)
            for (int u = 0; u <= xa[1] + xb[1]; ++u)
              for (int v = 0; v <= xa[2] + xb[2]; ++v) {
                const double e1 = EAB(0, xa[0], xb[0], t) * EAB(1, xa[1], xb[1], u) * EAB(2, xa[2], xb[2], v);
                for (int tau = 0; tau <= xc[0] + xd[0]; ++tau)
                  for (int nu = 0; nu <= xc[1] + xd[1]; ++nu)
                    for (int phi = 0; phi <= xc[2] + xd[2]; ++phi) {
                      const double e2 = ECD(0, xc[0], xd[0], tau) * ECD(1, xc[1], xd[1], nu) *
                                        ECD(2, xc[2], xd[2], phi);
                      const double sg = ((tau + nu + phi) & 1) ? -1.0 : 1.0;
                      s += e1 * sg * e2 * R[RIDX(t + tau, u + nu, v + phi)];
                    }
              }
          out[((ia * nb + ib) * nc + ic) * nd + id] += pref * s;
        }
#undef EAB
#undef ECD
}

void orc_prim_block(int la, int lb, int lc, int ld,
                    const double *A, double a, const double *B, double b,
                    const double *C, double c, const double *D, double d,
                    double scale, double *out) {
  prim_block_w(la, lb, lc, ld, A, a, B, b, C, c, D, d, scale, 0.0, out);
}

void orc_prim_block_omega(int la, int lb, int lc, int ld,
                          const double *A, double a, const double *B, double b,
                          const double *C, double c, const double *D, double d,
                          double scale, double omega, double *out) {
  prim_block_w(la, lb, lc, ld, A, a, B, b, C, c, D, d, scale, omega, out);
}

/* ------------------------------------------------------------------------ */
/* Basis description passed by the wrapper */

typedef struct {
  const double *xyz;                      /* [natom][3] */
  int nshell;
  const int *atom, *l, *nprim, *ptr;      /* per shell */
  const double *exps, *coefs;             /* primitives */
  double omega;                           /* > 0: erf(omega r)/r operator */
} orc_basis;

static double dfact(int n) {
  double r = 1.0;
  while (n > 1) { r *= n; n -= 2; }
  return r;
}

static double prim_norm(double a, int l) {
  return pow(2.0 * a / (double)ORC_PI, 0.75) * pow(4.0 * a, 0.5 * l) / sqrt(dfact(2 * l - 1));
}

/* Contracted Cartesian block (ab|cd) of shells sa, sb, sc, sd. */
static void shell_quartet(const orc_basis *bs, int sa, int sb, int sc, int sd, double *out) {
  const int la = bs->l[sa], lb = bs->l[sb], lc = bs->l[sc], ld = bs->l[sd];
  const int n = ORC_NC(la) * ORC_NC(lb) * ORC_NC(lc) * ORC_NC(ld);
  memset(out, 0, sizeof(double) * n);
  const double *A = bs->xyz + 3 * bs->atom[sa], *B = bs->xyz + 3 * bs->atom[sb];
  const double *C = bs->xyz + 3 * bs->atom[sc], *D = bs->xyz + 3 * bs->atom[sd];
  for (int i = 0; i < bs->nprim[sa]; ++i)
    for (int j = 0; j < bs->nprim[sb]; ++j)
      for (int k = 0; k < bs->nprim[sc]; ++k)
        for (int m = 0; m < bs->nprim[sd]; ++m) {
          const double a = bs->exps[bs->ptr[sa] + i], b = bs->exps[bs->ptr[sb] + j];
          const double c = bs->exps[bs->ptr[sc] + k], d = bs->exps[bs->ptr[sd] + m];
          const double s = bs->coefs[bs->ptr[sa] + i] * prim_norm(a, la) *
                           bs->coefs[bs->ptr[sb] + j] * prim_norm(b, lb) *
                           bs->coefs[bs->ptr[sc] + k] * prim_norm(c, lc) *
                           bs->coefs[bs->ptr[sd] + m] * prim_norm(d, ld);
          prim_block_w(la, lb, lc, ld, A, a, B, b, C, c, D, d, s, bs->omega, out);
        }
}

void orc_shell_quartet(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                       const int *ptr, const double *exps, const double *coefs,
                       int sa, int sb, int sc, int sd, double *out) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  shell_quartet(&bs, sa, sb, sc, sd, out);
}

/* ------------------------------------------------------------------------ */
/* Schwarz bounds Q[ab] for a >= b, pair index a(a+1)/2 + b. */

static double schwarz_one(const orc_basis *bs, int a, int b, double *work) {
  const int na = ORC_NC(bs->l[a]), nb = ORC_NC(bs->l[b]);
  shell_quartet(bs, a, b, a, b, work);
  double mx = 0.0;
  for (int i = 0; i < na; ++i)
    for (int j = 0; j < nb; ++j) {
      const double v = fabs(work[((i * nb + j) * na + i) * nb + j]);
      if (v > mx) mx = v;
    }
  return sqrt(mx);
}

void orc_schwarz(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                 const int *ptr, const double *exps, const double *coefs, double *Q, int nthreads) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  const long npair = (long)nshell * (nshell + 1) / 2;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double *work = (double *)malloc(sizeof(double) * 15 * 15 * 15 * 15);
#pragma omp for schedule(dynamic, 16)
    for (long ab = 0; ab < npair; ++ab) {
      int a = (int)((sqrt(8.0 * ab + 1.0) - 1.0) / 2.0);
      while ((long)a * (a + 1) / 2 > ab) --a;
      while ((long)(a + 1) * (a + 2) / 2 <= ab) ++a;
      const int b = (int)(ab - (long)a * (a + 1) / 2);
      Q[ab] = schwarz_one(&bs, a, b, work);
    }
    free(work);
  }
}

/* ------------------------------------------------------------------------ */
/* J and K from all unique shell quartets (a>=b, c>=d, ab>=cd) kept by the
   Schwarz rule.  Each quartet's block is added once for every *distinct*
   image of the shell tuple under the 8 permutational symmetries; this sums
   every element of the full n^4 tensor exactly once.  D, J, K are Cartesian
   [nc][nc] row-major. */

static void shell_offsets(const orc_basis *bs, int *off) {
  int o = 0;
  for (int s = 0; s < bs->nshell; ++s) { off[s] = o; o += ORC_NC(bs->l[s]); }
  off[bs->nshell] = o;
}

/* the 8 images of (a,b,c,d); perm[k] gives which original slot lands in
   position 0..3 */
static const int PERM8[8][4] = {{0, 1, 2, 3}, {1, 0, 2, 3}, {0, 1, 3, 2}, {1, 0, 3, 2},
                                {2, 3, 0, 1}, {3, 2, 0, 1}, {2, 3, 1, 0}, {3, 2, 1, 0}};

static int distinct_images(const int *sh, int *keep) {
  int n = 0;
  for (int k = 0; k < 8; ++k) {
    int img[4];
    for (int s = 0; s < 4; ++s) img[s] = sh[PERM8[k][s]];
    int dup = 0;
    for (int j = 0; j < k && !dup; ++j) {
      if (!keep[j]) continue;
      int same = 1;
      for (int s = 0; s < 4; ++s) same &= (img[s] == sh[PERM8[j][s]]);
      dup = same;
    }
    keep[k] = !dup;
    n += keep[k];
  }
  return n;
}

static void scatter_jk(const int *sh, const int *off, const int *nsz, const double *blk, int nc,
                       const double *D, double *J, double *K) {
  int keep[8];
  distinct_images(sh, keep);
  const int n0 = nsz[0], n1 = nsz[1], n2 = nsz[2], n3 = nsz[3];
  for (int k = 0; k < 8; ++k) {
    if (!keep[k]) continue;
    for (int i0 = 0; i0 < n0; ++i0)
      for (int i1 = 0; i1 < n1; ++i1)
        for (int i2 = 0; i2 < n2; ++i2)
          for (int i3 = 0; i3 < n3; ++i3) {
            const double g = blk[((i0 * n1 + i1) * n2 + i2) * n3 + i3];
            const int f[4] = {off[0] + i0, off[1] + i1, off[2] + i2, off[3] + i3};
            const int w = f[PERM8[k][0]], x = f[PERM8[k][1]], y = f[PERM8[k][2]], z = f[PERM8[k][3]];
            J[(long)w * nc + x] += g * D[(long)y * nc + z];
            K[(long)w * nc + y] += g * D[(long)x * nc + z];
          }
  }
}

static void jk_range(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                     const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
                     const double *D, double *J, double *K, int nthreads, long *nkept, long ab_lo, long ab_hi,
                     double omega);

void orc_jk(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
            const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
            const double *D, double *J, double *K, int nthreads, long *nkept) {
  jk_range(xyz, nshell, atom, l, nprim, ptr, exps, coefs, Q, thresh, D, J, K, nthreads, nkept, 0,
           (long)nshell * (nshell + 1) / 2, 0.0);
}

/* The same with the long-range operator erf(omega r)/r (omega > 0); the
   quartets are screened with the Coulomb bounds Q, which bound the
   attenuated integrals too. */
void orc_jk_omega(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                  const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
                  const double *D, double *J, double *K, int nthreads, long *nkept, double omega) {
  jk_range(xyz, nshell, atom, l, nprim, ptr, exps, coefs, Q, thresh, D, J, K, nthreads, nkept, 0,
           (long)nshell * (nshell + 1) / 2, omega);
}

/* The same sum restricted to bra pairs ab in [ab_lo, ab_hi) (each with all
   its kets cd <= ab): a bounded sample of the work for timing. */
void orc_jk_range(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                  const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
                  const double *D, double *J, double *K, int nthreads, long *nkept, long ab_lo, long ab_hi) {
  jk_range(xyz, nshell, atom, l, nprim, ptr, exps, coefs, Q, thresh, D, J, K, nthreads, nkept, ab_lo, ab_hi, 0.0);
}

static void jk_range(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                     const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
                     const double *D, double *J, double *K, int nthreads, long *nkept, long ab_lo, long ab_hi,
                     double omega) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs, omega};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell];
  memset(J, 0, sizeof(double) * nc * nc);
  memset(K, 0, sizeof(double) * nc * nc);
  long kept = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel reduction(+ : kept)
  {
    double *Jt = (double *)calloc((size_t)nc * nc, sizeof(double));
    double *Kt = (double *)calloc((size_t)nc * nc, sizeof(double));
    double *blk = (double *)malloc(sizeof(double) * 15 * 15 * 15 * 15);
#pragma omp for schedule(dynamic, 1)
    for (long ab = ab_hi - 1; ab >= ab_lo; --ab) {
      int a = 0;
      while ((long)(a + 1) * (a + 2) / 2 <= ab) ++a;
      const int b = (int)(ab - (long)a * (a + 1) / 2);
      for (long cd = 0; cd <= ab; ++cd) {
        if (Q[ab] * Q[cd] < thresh) continue;
        int c = 0;
        while ((long)(c + 1) * (c + 2) / 2 <= cd) ++c;
        const int d = (int)(cd - (long)c * (c + 1) / 2);
        shell_quartet(&bs, a, b, c, d, blk);
        const int sh[4] = {a, b, c, d};
        const int of[4] = {off[a], off[b], off[c], off[d]};
        const int ns[4] = {ORC_NC(l[a]), ORC_NC(l[b]), ORC_NC(l[c]), ORC_NC(l[d])};
        scatter_jk(sh, of, ns, blk, nc, D, Jt, Kt);
        ++kept;
      }
    }
#pragma omp critical
    {
      for (long i = 0; i < (long)nc * nc; ++i) { J[i] += Jt[i]; K[i] += Kt[i]; }
    }
    free(Jt); free(Kt); free(blk);
  }
  if (nkept) *nkept = kept;
  free(off);
}

/* Sampled blocks for large molecules: for each requested shell pair (a, b)
   compute the full Cartesian blocks
     J_ab = sum_{c,d} (ab|cd) D_cd,   K_ab = sum_{c,d} (ac|bd) D_cd
   straight from the definition (no symmetry), each quartet subject to the
   Schwarz rule on its own bound Q_{bra} Q_{ket}.  Q is the full symmetric
   shell-pair matrix [nshell][nshell]. */
void orc_jk_blocks(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                   const int *ptr, const double *exps, const double *coefs, const double *Qfull,
                   double thresh, const double *D, int nreq, const int *req, double *Jout,
                   double *Kout, int nthreads) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell];
  long *roff = (long *)malloc(sizeof(long) * (nreq + 1));
  roff[0] = 0;
  for (int r = 0; r < nreq; ++r) roff[r + 1] = roff[r] + ORC_NC(l[req[2 * r]]) * ORC_NC(l[req[2 * r + 1]]);
  memset(Jout, 0, sizeof(double) * roff[nreq]);
  memset(Kout, 0, sizeof(double) * roff[nreq]);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  for (int r = 0; r < nreq; ++r) {
    const int a = req[2 * r], b = req[2 * r + 1];
    const int na = ORC_NC(l[a]), nb = ORC_NC(l[b]);
#pragma omp parallel
    {
      double *blk = (double *)malloc(sizeof(double) * 15 * 15 * 15 * 15);
      double *Jt = (double *)calloc(na * nb, sizeof(double));
      double *Kt = (double *)calloc(na * nb, sizeof(double));
#pragma omp for schedule(dynamic, 1)
      for (int c = 0; c < nshell; ++c) {
        const int ncc = ORC_NC(l[c]);
        for (int d = 0; d < nshell; ++d) {
          const int nd = ORC_NC(l[d]);
          if (Qfull[(long)a * nshell + b] * Qfull[(long)c * nshell + d] >= thresh) {
            shell_quartet(&bs, a, b, c, d, blk);
            for (int i = 0; i < na; ++i)
              for (int j = 0; j < nb; ++j) {
                double s = 0.0;
                for (int k = 0; k < ncc; ++k)
                  for (int m = 0; m < nd; ++m)
                    s += blk[((i * nb + j) * ncc + k) * nd + m] * D[(long)(off[c] + k) * nc + off[d] + m];
                Jt[i * nb + j] += s;
              }
          }
          if (Qfull[(long)a * nshell + c] * Qfull[(long)b * nshell + d] >= thresh) {
            shell_quartet(&bs, a, c, b, d, blk);
            for (int i = 0; i < na; ++i)
              for (int j = 0; j < nb; ++j) {
                double s = 0.0;
                for (int k = 0; k < ncc; ++k)
                  for (int m = 0; m < nd; ++m)
                    s += blk[((i * ncc + k) * nb + j) * nd + m] * D[(long)(off[c] + k) * nc + off[d] + m];
                Kt[i * nb + j] += s;
              }
          }
        }
      }
#pragma omp critical
      {
        for (int i = 0; i < na * nb; ++i) { Jout[roff[r] + i] += Jt[i]; Kout[roff[r] + i] += Kt[i]; }
      }
      free(blk); free(Jt); free(Kt);
    }
  }
  free(roff);
  free(off);
}

/* Full Cartesian ERI tensor [nc]^4 (tiny molecules only), no screening. */
void orc_eri_tensor(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                    const int *ptr, const double *exps, const double *coefs, double *out) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const long nc = off[nshell];
#pragma omp parallel
  {
    double *blk = (double *)malloc(sizeof(double) * 15 * 15 * 15 * 15);
#pragma omp for collapse(2) schedule(dynamic, 1)
    for (int a = 0; a < nshell; ++a)
      for (int b = 0; b < nshell; ++b)
        for (int c = 0; c < nshell; ++c)
          for (int d = 0; d < nshell; ++d) {
            shell_quartet(&bs, a, b, c, d, blk);
            const int na = ORC_NC(l[a]), nb = ORC_NC(l[b]), ncc = ORC_NC(l[c]), nd = ORC_NC(l[d]);
            for (int i = 0; i < na; ++i)
              for (int j = 0; j < nb; ++j)
                for (int k = 0; k < ncc; ++k)
                  for (int m = 0; m < nd; ++m)
                    out[(((off[a] + i) * nc + off[b] + j) * nc + off[c] + k) * nc + off[d] + m] =
                        blk[((i * nb + j) * ncc + k) * nd + m];
          }
    free(blk);
  }
  free(off);
}

/* ------------------------------------------------------------------------ */
/* Overlap matrix (Cartesian) S_ab = E^{ij}_0 E^{kl}_0 E^{mn}_0 (pi/p)^(3/2)
   (Helgaker eq. 9.5.41), used only to check input densities. */
void orc_overlap(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                 const int *ptr, const double *exps, const double *coefs, double *S) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell];
  memset(S, 0, sizeof(double) * nc * nc);
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb < nshell; ++sb) {
      const int la = l[sa], lb = l[sb];
      int pa[3 * ORC_NC(ORC_LMAX)], pb[3 * ORC_NC(ORC_LMAX)];
      cart_list(la, pa); cart_list(lb, pb);
      const double *A = xyz + 3 * atom[sa], *B = xyz + 3 * atom[sb];
      const int nt = la + lb + 1, st = (la + 1) * (lb + 1) * nt;
      double E[3 * 6 * 6 * 11];
      for (int i = 0; i < nprim[sa]; ++i)
        for (int j = 0; j < nprim[sb]; ++j) {
          const double a = exps[ptr[sa] + i], b = exps[ptr[sb] + j];
          for (int k = 0; k < 3; ++k) hermite_e(la, lb, a, b, A[k], B[k], E + k * st);
          const double w = coefs[ptr[sa] + i] * prim_norm(a, la) * coefs[ptr[sb] + j] * prim_norm(b, lb) *
                           pow((double)ORC_PI / (a + b), 1.5);
          for (int ia = 0; ia < ORC_NC(la); ++ia)
            for (int ib = 0; ib < ORC_NC(lb); ++ib) {
              double v = w;
              for (int k = 0; k < 3; ++k) v *= E[k * st + (pa[3 * ia + k] * (lb + 1) + pb[3 * ib + k]) * nt + 0];
              S[(long)(off[sa] + ia) * nc + off[sb] + ib] += v;
            }
        }
    }
  free(off);
}

/* ------------------------------------------------------------------------ */
/* Nuclear gradient of E = 1/2 tr(DJ) - 1/4 tr(DK) at fixed (Cartesian) D:
   dE/dR = sum_{mu nu la si} G_{mu nu la si} d(mu nu|la si)/dR,
   G = 1/2 D_mn D_ls - 1/8 (D_ml D_ns + D_ms D_nl), which has the 8-fold
   symmetry of the integrals, so every unique quartet enters with the number
   of its distinct images.  The derivative of a primitive with respect to its
   centre is d/dA_x [x_A^i e^{-a x_A^2}] = 2a x_A^(i+1) e^.. - i x_A^(i-1) e^..
   (Helgaker eq. 9.2.11 applied to a Cartesian factor); all four centres are
   differentiated explicitly. */

static void deriv_blocks(const orc_basis *bs, const int *sh, double *dblk /* [4][3][n] */, int n,
                         double *tmp_p, double *tmp_m) {
  memset(dblk, 0, sizeof(double) * 12 * n);
  const int lv[4] = {bs->l[sh[0]], bs->l[sh[1]], bs->l[sh[2]], bs->l[sh[3]]};
  int nv[4];
  for (int s = 0; s < 4; ++s) nv[s] = ORC_NC(lv[s]);
  const double *X[4];
  for (int s = 0; s < 4; ++s) X[s] = bs->xyz + 3 * bs->atom[sh[s]];
  int pw[4][3 * ORC_NC(ORC_LMAX)];
  for (int s = 0; s < 4; ++s) cart_list(lv[s], pw[s]);

  for (int i0 = 0; i0 < bs->nprim[sh[0]]; ++i0)
    for (int i1 = 0; i1 < bs->nprim[sh[1]]; ++i1)
      for (int i2 = 0; i2 < bs->nprim[sh[2]]; ++i2)
        for (int i3 = 0; i3 < bs->nprim[sh[3]]; ++i3) {
          const int ip[4] = {i0, i1, i2, i3};
          double ex[4], sc = 1.0;
          for (int s = 0; s < 4; ++s) {
            ex[s] = bs->exps[bs->ptr[sh[s]] + ip[s]];
            sc *= bs->coefs[bs->ptr[sh[s]] + ip[s]] * prim_norm(ex[s], lv[s]);
          }
          for (int s = 0; s < 4; ++s) { /* differentiate centre s */
            int lp[4] = {lv[0], lv[1], lv[2], lv[3]}, lm[4] = {lv[0], lv[1], lv[2], lv[3]};
            lp[s] += 1; lm[s] -= 1;
            const int np_ = ORC_NC(lp[0]) * ORC_NC(lp[1]) * ORC_NC(lp[2]) * ORC_NC(lp[3]);
            memset(tmp_p, 0, sizeof(double) * np_);
            orc_prim_block(lp[0], lp[1], lp[2], lp[3], X[0], ex[0], X[1], ex[1], X[2], ex[2], X[3], ex[3], sc, tmp_p);
            int nm_ = 0;
            if (lm[s] >= 0) {
              nm_ = ORC_NC(lm[0]) * ORC_NC(lm[1]) * ORC_NC(lm[2]) * ORC_NC(lm[3]);
              memset(tmp_m, 0, sizeof(double) * nm_);
              orc_prim_block(lm[0], lm[1], lm[2], lm[3], X[0], ex[0], X[1], ex[1], X[2], ex[2], X[3], ex[3], sc, tmp_m);
            }
            int npl[4], nmi[4];
            for (int t = 0; t < 4; ++t) { npl[t] = ORC_NC(lp[t]); nmi[t] = (lm[t] >= 0) ? ORC_NC(lm[t]) : 0; }
            for (int c0 = 0; c0 < nv[0]; ++c0)
              for (int c1 = 0; c1 < nv[1]; ++c1)
                for (int c2 = 0; c2 < nv[2]; ++c2)
                  for (int c3 = 0; c3 < nv[3]; ++c3) {
                    const int cc[4] = {c0, c1, c2, c3};
                    const int e = ((c0 * nv[1] + c1) * nv[2] + c2) * nv[3] + c3;
                    for (int k = 0; k < 3; ++k) {
                      int up[4], dn[4];
                      int pwk[3];
                      for (int t = 0; t < 3; ++t) pwk[t] = pw[s][3 * cc[s] + t];
                      /* index of component raised by 1 in direction k */
                      int ux = pwk[0] + (k == 0), uy = pwk[1] + (k == 1);
                      for (int t = 0; t < 4; ++t) up[t] = cc[t];
                      up[s] = cart_index(lp[s], ux, uy);
                      const double vp = tmp_p[((up[0] * npl[1] + up[1]) * npl[2] + up[2]) * npl[3] + up[3]];
                      double v = 2.0 * ex[s] * vp;
                      if (pwk[k] > 0) {
                        int dx = pwk[0] - (k == 0), dy = pwk[1] - (k == 1);
                        for (int t = 0; t < 4; ++t) dn[t] = cc[t];
                        dn[s] = cart_index(lm[s], dx, dy);
                        const double vm = tmp_m[((dn[0] * nmi[1] + dn[1]) * nmi[2] + dn[2]) * nmi[3] + dn[3]];
                        v -= pwk[k] * vm;
                      }
                      dblk[(s * 3 + k) * n + e] += v;
                    }
                  }
          }
        }
}

void orc_grad(const double *xyz, int natom, int nshell, const int *atom, const int *l, const int *nprim,
              const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
              const double *D, double *grad, int nthreads) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell];
  const long npair = (long)nshell * (nshell + 1) / 2;
  memset(grad, 0, sizeof(double) * 3 * natom);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double *gt = (double *)calloc(3 * natom, sizeof(double));
    const int big = 21 * 21 * 21 * 21;
    double *dblk = (double *)malloc(sizeof(double) * 12 * 15 * 15 * 15 * 15);
    double *tp = (double *)malloc(sizeof(double) * big);
    double *tm = (double *)malloc(sizeof(double) * big);
#pragma omp for schedule(dynamic, 1)
    for (long ab = npair - 1; ab >= 0; --ab) {
      int a = 0;
      while ((long)(a + 1) * (a + 2) / 2 <= ab) ++a;
      const int b = (int)(ab - (long)a * (a + 1) / 2);
      for (long cd = 0; cd <= ab; ++cd) {
        if (Q[ab] * Q[cd] < thresh) continue;
        int c = 0;
        while ((long)(c + 1) * (c + 2) / 2 <= cd) ++c;
        const int d = (int)(cd - (long)c * (c + 1) / 2);
        const int sh[4] = {a, b, c, d};
        int keep[8];
        const int nimg = distinct_images(sh, keep);
        const int ns[4] = {ORC_NC(l[a]), ORC_NC(l[b]), ORC_NC(l[c]), ORC_NC(l[d])};
        const int n = ns[0] * ns[1] * ns[2] * ns[3];
        deriv_blocks(&bs, sh, dblk, n, tp, tm);
        for (int i0 = 0; i0 < ns[0]; ++i0)
          for (int i1 = 0; i1 < ns[1]; ++i1)
            for (int i2 = 0; i2 < ns[2]; ++i2)
              for (int i3 = 0; i3 < ns[3]; ++i3) {
                const long m = off[a] + i0, nu = off[b] + i1, la_ = off[c] + i2, si = off[d] + i3;
                const double G = 0.5 * D[m * nc + nu] * D[la_ * nc + si] -
                                 0.125 * (D[m * nc + la_] * D[nu * nc + si] + D[m * nc + si] * D[nu * nc + la_]);
                const int e = ((i0 * ns[1] + i1) * ns[2] + i2) * ns[3] + i3;
                for (int s = 0; s < 4; ++s)
                  for (int k = 0; k < 3; ++k) gt[3 * atom[sh[s]] + k] += nimg * G * dblk[(s * 3 + k) * n + e];
              }
      }
    }
#pragma omp critical
    {
      for (int i = 0; i < 3 * natom; ++i) grad[i] += gt[i];
    }
    free(gt); free(dblk); free(tp); free(tm);
  }
  free(off);
}

/* ------------------------------------------------------------------------ */
/* One-electron integrals of the core Hamiltonian H = T + V used by the SCF
   driver around the J/K build (Eq. 1: F = H + J - 1/2 c_x K, with H the
   kinetic and nuclear-attraction terms).  Plain McMurchie-Davidson as in
   Helgaker, Jorgensen and Olsen:
     overlap, per direction      S_ij = E^{ij}_0 sqrt(pi/p)          (eq. 9.3.12)
     kinetic, per direction      T_ij = -1/2 [ j(j-1) S_{i,j-2} - 2b(2j+1) S_{ij}
                                              + 4 b^2 S_{i,j+2} ]     (from eq. 9.3.23:
                                 the second derivative of the ket Gaussian)
     T = Tx Sy Sz + Sx Ty Sz + Sx Sy Tz
     nuclear attraction          V = - sum_C Z_C (2 pi / p)
                                     sum_tuv E^{ij}_t E^{kl}_u E^{mn}_v R_tuv(p, P - C)   (eq. 9.9.32)
   Outputs are full Cartesian [nc][nc] matrices (row-major). */
void orc_one_electron(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                      const int *ptr, const double *exps, const double *coefs, int natom, const double *charges,
                      double *S, double *T, double *V) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell];
  memset(S, 0, sizeof(double) * nc * nc);
  memset(T, 0, sizeof(double) * nc * nc);
  memset(V, 0, sizeof(double) * nc * nc);
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb < nshell; ++sb) {
      const int la = l[sa], lb = l[sb], na = ORC_NC(la), nb = ORC_NC(lb);
      const double *A = xyz + 3 * atom[sa], *B = xyz + 3 * atom[sb];
      int pa[3 * ORC_NC(ORC_LMAX)], pb[3 * ORC_NC(ORC_LMAX)];
      cart_list(la, pa);
      cart_list(lb, pb);
      const int jm = lb + 2, nt = la + jm + 1;  /* E tables up to j = lb + 2 (kinetic) */
      const int se = (la + 1) * (jm + 1) * nt;
      for (int i = 0; i < nprim[sa]; ++i)
        for (int j = 0; j < nprim[sb]; ++j) {
          const double a = exps[ptr[sa] + i], b = exps[ptr[sb] + j], p = a + b;
          const double cc = coefs[ptr[sa] + i] * prim_norm(a, la) * coefs[ptr[sb] + j] * prim_norm(b, lb);
          double E[3 * (ORC_LMAX + 1) * (ORC_LMAX + 3) * (2 * ORC_LMAX + 3)];
          for (int k = 0; k < 3; ++k) hermite_e(la, jm, a, b, A[k], B[k], E + k * se);
#define EE(k, ii, jj, t) E[(k) * se + ((ii) * (jm + 1) + (jj)) * nt + (t)]
          double P[3];
          for (int k = 0; k < 3; ++k) P[k] = (a * A[k] + b * B[k]) / p;
          const double sq = sqrt((double)ORC_PI / p);
          const int L = la + lb;
          double R[(2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1) * (2 * ORC_LMAX + 1)];
          for (int ia = 0; ia < na; ++ia)
            for (int ib = 0; ib < nb; ++ib) {
              const int *xa = pa + 3 * ia, *xb = pb + 3 * ib;
              double s1[3], t1[3];
              for (int k = 0; k < 3; ++k) {
                const int ii = xa[k], jj = xb[k];
                s1[k] = EE(k, ii, jj, 0) * sq;
                const double sm2 = jj >= 2 ? EE(k, ii, jj - 2, 0) * sq : 0.0;
                const double sp2 = EE(k, ii, jj + 2, 0) * sq;
                t1[k] = -0.5 * (jj * (jj - 1) * sm2 - 2.0 * b * (2 * jj + 1) * s1[k] + 4.0 * b * b * sp2);
              }
              const long o = (long)(off[sa] + ia) * nc + off[sb] + ib;
              S[o] += cc * s1[0] * s1[1] * s1[2];
              T[o] += cc * (t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2]);
            }
          for (int c = 0; c < natom; ++c) {
            const double *C = xyz + 3 * c;
            hermite_r(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
            const double pref = -charges[c] * 2.0 * (double)ORC_PI / p;
            for (int ia = 0; ia < na; ++ia)
              for (int ib = 0; ib < nb; ++ib) {
                const int *xa = pa + 3 * ia, *xb = pb + 3 * ib;
                double s = 0.0;
                for (int t = 0; t <= xa[0] + xb[0]; ++t)
                  for (int u = 0; u <= xa[1] + xb[1]; ++u)
                    for (int v = 0; v <= xa[2] + xb[2]; ++v)
                      s += EE(0, xa[0], xb[0], t) * EE(1, xa[1], xb[1], u) * EE(2, xa[2], xb[2], v) *
                           R[RIDX(t, u, v)];
                V[(long)(off[sa] + ia) * nc + off[sb] + ib] += cc * pref * s;
              }
          }
#undef EE
        }
    }
  free(off);
}

/* ------------------------------------------------------------------------ */
/* Second derivatives of E_JK = 1/2 tr(DJ) - 1/4 tr(DK) at fixed D with respect
   to the nuclear coordinates (the analytic Hessian task of Sec. 3, first
   step: the two-electron part at fixed density).

   A primitive Gaussian's derivative with respect to its centre A_k is
     d/dA_k [x^i exp(-a (x-A)^2)] = 2a (x-A)^(i+1) exp(...) - i (x-A)^(i-1) exp(...),
   so every derivative of a primitive integral is a combination of primitive
   integrals with raised and lowered powers.  Second derivatives apply that
   rule twice (on the same centre or on two centres).  Per primitive quartet,
   the blocks of every needed power combination are evaluated once (with the
   contraction and normalisation factors) and the rule is applied recursively
   to the powers of each Cartesian component. */

#define HESS_MAXBLK 64

typedef struct {
  int n;
  int key[HESS_MAXBLK][4];
  double *blk[HESS_MAXBLK];
  const double *X[4];
  double ex[4], sc;
} blk_cache;

static const double *cache_block(blk_cache *c, const int l[4]) {
  for (int i = 0; i < c->n; ++i)
    if (c->key[i][0] == l[0] && c->key[i][1] == l[1] && c->key[i][2] == l[2] && c->key[i][3] == l[3])
      return c->blk[i];
  if (c->n == HESS_MAXBLK) return NULL;
  const size_t n = (size_t)ORC_NC(l[0]) * ORC_NC(l[1]) * ORC_NC(l[2]) * ORC_NC(l[3]);
  double *b = (double *)calloc(n, sizeof(double));
  orc_prim_block(l[0], l[1], l[2], l[3], c->X[0], c->ex[0], c->X[1], c->ex[1], c->X[2], c->ex[2], c->X[3],
                 c->ex[3], c->sc, b);
  for (int s = 0; s < 4; ++s) c->key[c->n][s] = l[s];
  c->blk[c->n] = b;
  return c->blk[c->n++];
}

static void cache_clear(blk_cache *c) {
  for (int i = 0; i < c->n; ++i) free(c->blk[i]);
  c->n = 0;
}

/* the primitive integral with powers pw[s][0..2] on the four centres,
   differentiated by the operators ops[2i] = centre, ops[2i+1] = direction */
static double dval(blk_cache *c, int pw[4][3], const int *ops, int nops) {
  if (nops == 0) {
    int l[4];
    for (int s = 0; s < 4; ++s) l[s] = pw[s][0] + pw[s][1] + pw[s][2];
    const double *b = cache_block(c, l);
    if (!b) return NAN;
    int idx = 0;
    for (int s = 0; s < 4; ++s) idx = idx * ORC_NC(l[s]) + cart_index(l[s], pw[s][0], pw[s][1]);
    return b[idx];
  }
  const int s = ops[0], k = ops[1];
  const int p = pw[s][k];
  pw[s][k] = p + 1;
  double v = 2.0 * c->ex[s] * dval(c, pw, ops + 2, nops - 1);
  if (p > 0) {
    pw[s][k] = p - 1;
    v -= p * dval(c, pw, ops + 2, nops - 1);
  }
  pw[s][k] = p;
  return v;
}

/* Hessian [3 natom][3 natom] of E_JK at fixed D (Cartesian D, row-major),
   over the quartets kept by the Schwarz rule with the given Q. */
void orc_jk_hessian(const double *xyz, int natom, int nshell, const int *atom, const int *l, const int *nprim,
                    const int *ptr, const double *exps, const double *coefs, const double *Q, double thresh,
                    const double *D, double *H, int nthreads) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell], n3 = 3 * natom;
  const long npair = (long)nshell * (nshell + 1) / 2;
  memset(H, 0, sizeof(double) * n3 * n3);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel
  {
    double *Ht = (double *)calloc((size_t)n3 * n3, sizeof(double));
    blk_cache cache;
    cache.n = 0;
#pragma omp for schedule(dynamic, 1)
    for (long ab = npair - 1; ab >= 0; --ab) {
      int a = 0;
      while ((long)(a + 1) * (a + 2) / 2 <= ab) ++a;
      const int b = (int)(ab - (long)a * (a + 1) / 2);
      for (long cd = 0; cd <= ab; ++cd) {
        if (Q[ab] * Q[cd] < thresh) continue;
        int c = 0;
        while ((long)(c + 1) * (c + 2) / 2 <= cd) ++c;
        const int d = (int)(cd - (long)c * (c + 1) / 2);
        const int sh[4] = {a, b, c, d};
        int keep[8];
        const int nimg = distinct_images(sh, keep);
        const int lv[4] = {l[a], l[b], l[c], l[d]};
        int pwl[4][3 * ORC_NC(ORC_LMAX)];
        for (int s = 0; s < 4; ++s) cart_list(lv[s], pwl[s]);
        for (int s = 0; s < 4; ++s) cache.X[s] = xyz + 3 * atom[sh[s]];
        for (int i0 = 0; i0 < nprim[a]; ++i0)
          for (int i1 = 0; i1 < nprim[b]; ++i1)
            for (int i2 = 0; i2 < nprim[c]; ++i2)
              for (int i3 = 0; i3 < nprim[d]; ++i3) {
                const int ip[4] = {i0, i1, i2, i3};
                cache.sc = 1.0;
                for (int s = 0; s < 4; ++s) {
                  cache.ex[s] = exps[ptr[sh[s]] + ip[s]];
                  cache.sc *= coefs[ptr[sh[s]] + ip[s]] * prim_norm(cache.ex[s], lv[s]);
                }
                for (int c0 = 0; c0 < ORC_NC(lv[0]); ++c0)
                  for (int c1 = 0; c1 < ORC_NC(lv[1]); ++c1)
                    for (int c2 = 0; c2 < ORC_NC(lv[2]); ++c2)
                      for (int c3 = 0; c3 < ORC_NC(lv[3]); ++c3) {
                        const int cc[4] = {c0, c1, c2, c3};
                        const long m = off[a] + c0, nu = off[b] + c1, la_ = off[c] + c2, si = off[d] + c3;
                        const double G = nimg * (0.5 * D[m * nc + nu] * D[la_ * nc + si] -
                                                 0.125 * (D[m * nc + la_] * D[nu * nc + si] +
                                                          D[m * nc + si] * D[nu * nc + la_]));
                        if (G == 0.0) continue;
                        int pw[4][3];
                        for (int s = 0; s < 4; ++s)
                          for (int t = 0; t < 3; ++t) pw[s][t] = pwl[s][3 * cc[s] + t];
                        for (int s = 0; s < 4; ++s)
                          for (int k = 0; k < 3; ++k)
                            for (int t = 0; t < 4; ++t)
                              for (int q = 0; q < 3; ++q) {
                                if (t * 3 + q < s * 3 + k) continue;  /* symmetric: upper triangle */
                                const int ops[4] = {s, k, t, q};
                                const double v = G * dval(&cache, pw, ops, 2);
                                const int r0 = 3 * atom[sh[s]] + k, r1 = 3 * atom[sh[t]] + q;
                                Ht[r0 * n3 + r1] += v;
                                if (t * 3 + q != s * 3 + k) Ht[r1 * n3 + r0] += v;
                              }
                      }
                cache_clear(&cache);
              }
      }
    }
#pragma omp critical
    {
      for (long i = 0; i < (long)n3 * n3; ++i) H[i] += Ht[i];
    }
    free(Ht);
  }
  free(off);
}

/* ------------------------------------------------------------------------ */
/* Nuclear gradient of the one-electron part of the closed-shell SCF energy
   (the single-point force task of Sec. 3 around the J/K gradient):
     sum_{mu nu} D_mu,nu dH_mu,nu/dR - sum_{mu nu} W_mu,nu dS_mu,nu/dR,
   W the energy-weighted density.  Derivatives with respect to the centres of
   the two functions by the raise/lower rule of the Hessian section; the
   derivative of a nuclear-attraction integral with respect to its nucleus C
   by translational invariance, d/dC = -(d/dA + d/dB) for that nucleus's term.
   Matrices are Cartesian [nc][nc] row-major; grad is [natom][3] (added to). */

/* S, T and the attraction to a unit positive charge at C (V = -2pi/p sum E E E R)
   of two unnormalised primitive Cartesian Gaussians with powers ia at A
   (exponent a) and ib at B (exponent b) */
static void prim_one_elem(const int ia[3], const double *A, double a, const int ib[3], const double *B, double b,
                          const double *C, double *s, double *t, double *v) {
  const double p = a + b;
  double E[3][(ORC_LMAX + 3) * (ORC_LMAX + 5) * (2 * ORC_LMAX + 8)];
  int jm[3], nt[3];
  for (int k = 0; k < 3; ++k) {
    jm[k] = ib[k] + 2;
    nt[k] = ia[k] + jm[k] + 1;
    hermite_e(ia[k], jm[k], a, b, A[k], B[k], E[k]);
  }
#define EO(k, ii, jj, tt) E[k][((ii) * (jm[k] + 1) + (jj)) * nt[k] + (tt)]
  const double sq = sqrt((double)ORC_PI / p);
  double s1[3], t1[3];
  for (int k = 0; k < 3; ++k) {
    const int ii = ia[k], jj = ib[k];
    s1[k] = EO(k, ii, jj, 0) * sq;
    const double sm2 = jj >= 2 ? EO(k, ii, jj - 2, 0) * sq : 0.0;
    const double sp2 = EO(k, ii, jj + 2, 0) * sq;
    t1[k] = -0.5 * (jj * (jj - 1) * sm2 - 2.0 * b * (2 * jj + 1) * s1[k] + 4.0 * b * b * sp2);
  }
  *s = s1[0] * s1[1] * s1[2];
  *t = t1[0] * s1[1] * s1[2] + s1[0] * t1[1] * s1[2] + s1[0] * s1[1] * t1[2];
  const int L = ia[0] + ib[0] + ia[1] + ib[1] + ia[2] + ib[2];
  double R[(2 * ORC_LMAX + 3) * (2 * ORC_LMAX + 3) * (2 * ORC_LMAX + 3)];
  double P[3];
  for (int k = 0; k < 3; ++k) P[k] = (a * A[k] + b * B[k]) / p;
  hermite_r(L, p, P[0] - C[0], P[1] - C[1], P[2] - C[2], R);
  double acc = 0.0;
  for (int tt = 0; tt <= ia[0] + ib[0]; ++tt)
    for (int u = 0; u <= ia[1] + ib[1]; ++u)
      for (int w = 0; w <= ia[2] + ib[2]; ++w) acc += EO(0, ia[0], ib[0], tt) * EO(1, ia[1], ib[1], u) *
                                                          EO(2, ia[2], ib[2], w) * R[RIDX(tt, u, w)];
  *v = -2.0 * (double)ORC_PI / p * acc;
#undef EO
}

void orc_one_electron_grad(const double *xyz, int nshell, const int *atom, const int *l, const int *nprim,
                           const int *ptr, const double *exps, const double *coefs, int natom,
                           const double *charges, const double *D, const double *W, double *grad) {
  orc_basis bs = {xyz, nshell, atom, l, nprim, ptr, exps, coefs};
  int *off = (int *)malloc(sizeof(int) * (nshell + 1));
  double *dvc = (double *)malloc(sizeof(double) * (natom > 0 ? natom : 1));
  shell_offsets(&bs, off);
  const int nc = off[nshell];
  for (int sa = 0; sa < nshell; ++sa)
    for (int sb = 0; sb < nshell; ++sb) {
      const int la = l[sa], lb = l[sb];
      const double *A = xyz + 3 * atom[sa], *B = xyz + 3 * atom[sb];
      int pa[3 * ORC_NC(ORC_LMAX)], pb[3 * ORC_NC(ORC_LMAX)];
      cart_list(la, pa);
      cart_list(lb, pb);
      for (int i = 0; i < nprim[sa]; ++i)
        for (int j = 0; j < nprim[sb]; ++j) {
          const double a = exps[ptr[sa] + i], b = exps[ptr[sb] + j];
          const double cc = coefs[ptr[sa] + i] * prim_norm(a, la) * coefs[ptr[sb] + j] * prim_norm(b, lb);
          for (int ia = 0; ia < ORC_NC(la); ++ia)
            for (int ib = 0; ib < ORC_NC(lb); ++ib) {
              const long o = (long)(off[sa] + ia) * nc + off[sb] + ib;
              const double dw = D[o], ww = W[o];
              for (int side = 0; side < 2; ++side)  /* 0: centre A (bra), 1: centre B (ket) */
                for (int k = 0; k < 3; ++k) {
                  int pw_a[3], pw_b[3];
                  for (int q = 0; q < 3; ++q) { pw_a[q] = pa[3 * ia + q]; pw_b[q] = pb[3 * ib + q]; }
                  int *pw = side == 0 ? pw_a : pw_b;
                  const double ex = side == 0 ? a : b;
                  const int p0 = pw[k];
                  double ds = 0.0, dt = 0.0;
                  for (int c = 0; c < natom; ++c) dvc[c] = 0.0;
                  for (int term = 0; term < 2; ++term) {
                    double f;
                    if (term == 0) { pw[k] = p0 + 1; f = 2.0 * ex; }
                    else { if (p0 == 0) break; pw[k] = p0 - 1; f = -(double)p0; }
                    double s, t, v;
                    for (int c = 0; c < natom; ++c) {
                      prim_one_elem(pw_a, A, a, pw_b, B, b, xyz + 3 * c, &s, &t, &v);
                      dvc[c] += f * charges[c] * v;
                    }
                    ds += f * s;
                    dt += f * t;
                    pw[k] = p0;
                  }
                  double dv = 0.0;
                  for (int c = 0; c < natom; ++c) dv += dvc[c];
                  const int ca = side == 0 ? atom[sa] : atom[sb];
                  grad[3 * ca + k] += cc * (dw * (dt + dv) - ww * ds);
                  /* the nucleus of each attraction term moves against both centres */
                  for (int c = 0; c < natom; ++c) grad[3 * c + k] -= cc * dw * dvc[c];
                }
            }
        }
    }
  free(dvc);
  free(off);
}
