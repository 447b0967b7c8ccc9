// Nuclear gradient of E_JK = 1/2 tr(DJ) - 1/4 tr(DK) at fixed D: the launcher
// tables, and the runtime-L kernel used for the class pairs that the
// cooperative two-pass kernels of adft_gradk.cuh do not cover (f shells).
//
//   dE/dR = sum over unique shell quartets of n_img sum_block G_mnls d(mn|ls)/dR,
//   G_mnls = 1/2 D_mn D_ls - 1/8 (D_ml D_ns + D_ms D_nl)
// (G has the 8-fold symmetry of the integrals, so each unique quartet enters
// with the number n_img = 8 s_ab s_cd s_(ab,cd) of its distinct images).
// The derivative of a primitive with respect to its centre raises or lowers
// one Cartesian power: d/dA_x [x_A^i e^{-a x_A^2}] = 2a x_A^(i+1) e^.. - i x_A^(i-1) e^..,
// so each centre derivative is the difference of two integral blocks with
// l + 1 (weighted by 2a per primitive) and l - 1.  Centres A and B are
// differentiated on the quartet (ab|cd), centre C on the swapped quartet
// (cd|ab), and centre D follows from translational invariance
// dD = -(dA + dB + dC).  Quartets are recomputed, none is stored.
#define ADFT_ERI_DECLARE_ONLY
#include "adft_eri.cuh"
#include "adft_gradk.cuh"

namespace adft {

// Contract the shifted blocks of one bra centre with G and return the three
// Cartesian components of the derivative (bra pair P = (a,b), ket pair Q).
// which = 0: differentiate a (l_a +/- 1); which = 1: differentiate b.
template <typename T>
__device__ __noinline__ void centre_derivative(const BasisView& bv, int P, int Qk, int la, int lb, int lc, int ld,
                                               int which, const T* __restrict__ D, long n, int oa, int ob, int oc,
                                               int od, T* out3, T* Gp, T* Gm, T eps) {
  const int lup_a = la + (which == 0), lup_b = lb + (which == 1);
  const int ldn_a = la - (which == 0), ldn_b = lb - (which == 1);
  const RtClass Cu = make_rt_class(lup_a, lup_b, lc, ld);
  const bool has_dn = (ldn_a >= 0 && ldn_b >= 0);
  RtClass Cd = Cu;
  if (has_dn) { Cd.la = ldn_a; Cd.lb = ldn_b; }
  const int NA = ncart(la), NB = ncart(lb), ND = ncart(ld), NCD = ncart(lc) * ND;
  const int NBu = ncart(lup_b), NBd = has_dn ? ncart(ldn_b) : 1;
  const T* wts = nullptr;
  if constexpr (sizeof(T) == 8) wts = (const T*)bv.pp_w64 + (which == 0 ? 0 : bv.npp);
  else wts = (const T*)bv.pp_w32 + (which == 0 ? 0 : bv.npp);
  T s0 = 0, s1 = 0, s2 = 0;
  for (int chunk = 0; chunk < Cu.nchunk; ++chunk) {
    quartet_block_rt<T>(Cu, bv, P, Qk, chunk, Gp, wts, -1, -1, eps);
    if (has_dn) quartet_block_rt<T>(Cd, bv, P, Qk, chunk, Gm, nullptr, -1, -1, eps);
    const int CK = Cu.ck, kc0 = chunk * CK, nk = min(CK, NCD - kc0);
    for (int ia = 0; ia < NA; ++ia) {
      int ax, ay, az;
      cart_pows_rt(la, ia, ax, ay, az);
      for (int ib = 0; ib < NB; ++ib) {
        int bx, by, bz;
        cart_pows_rt(lb, ib, bx, by, bz);
        const int mu = oa + ia, nu = ob + ib;
        const T Dmn = D[mu * n + nu];
        for (int k = 0; k < nk; ++k) {
          const int kc = kc0 + k, la_ = oc + kc / ND, si = od + kc % ND;
          const T G = T(0.5) * Dmn * D[la_ * n + si] -
                      T(0.125) * (D[mu * n + la_] * D[nu * n + si] + D[mu * n + si] * D[nu * n + la_]);
          // component index of the raised / lowered function on the shifted centre
          int p[3] = {which == 0 ? ax : bx, which == 0 ? ay : by, which == 0 ? az : bz};
          const int lsh = which == 0 ? la : lb;
          T d[3];
          for (int dir = 0; dir < 3; ++dir) {
            int q[3] = {p[0], p[1], p[2]};
            q[dir] += 1;
            const int iu = cart_index_dev(lsh + 1, q[0], q[1]);
            const int eu = (which == 0) ? (iu * NBu + ib) : (ia * NBu + iu);
            T v = Gp[eu * CK + k];
            if (p[dir] > 0 && has_dn) {
              q[dir] -= 2;
              const int idn = cart_index_dev(lsh - 1, q[0], q[1]);
              const int ed = (which == 0) ? (idn * NBd + ib) : (ia * NBd + idn);
              v -= T(p[dir]) * Gm[ed * CK + k];
            }
            d[dir] = v;
          }
          s0 += G * d[0]; s1 += G * d[1]; s2 += G * d[2];
        }
      }
    }
  }
  out3[0] = s0; out3[1] = s1; out3[2] = s2;
}

template <typename T>
__global__ void __launch_bounds__(JK_THREADS) k_grad_generic(GradLaunch g, int la, int lb, int lc, int ld) {
  const JKLaunch& a = g.jk;
  const long long total = (long long)__ldg(a.prefix + a.nseg);
  const int lane = threadIdx.x & 31;
  T Gp[GEN_BUDGET], Gm[GEN_BUDGET];
  const T* D = nullptr;
  if constexpr (sizeof(T) == 8) D = (const T*)a.D64; else D = (const T*)a.D32;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.counter, 32ULL);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total) break;
    if (*(volatile const int*)a.abort_flag) {
      if (lane == 0) atomicCAS(a.status, 0, ADFT_ERR_ABORTED);
      break;
    }
    const long long qi = (long long)base + lane;
    if (qi < total) {
      int bra, ket;
      decode_quartet(a, qi, bra, ket);
      const BasisView& bv = a.bv;
      const int sa = bv.pair_a[bra], sb = bv.pair_b[bra], sc = bv.pair_a[ket], sd = bv.pair_b[ket];
      const int oa = bv.shell_coff[sa], ob = bv.shell_coff[sb], oc = bv.shell_coff[sc], od = bv.shell_coff[sd];
      long long base;
      long nrow;
      mol_block(bv, bra, base, nrow);
      const T* Dm = D + base;
      T w = T(8);
      if (sa == sb) w *= T(0.5);
      if (sc == sd) w *= T(0.5);
      if (a.same_class && bra == ket) w *= T(0.5);
      T dA[3], dB[3], dC[3];
      const T eps = (T)a.prim_eps;
      centre_derivative<T>(bv, bra, ket, la, lb, lc, ld, 0, Dm, nrow, oa, ob, oc, od, dA, Gp, Gm, eps);
      centre_derivative<T>(bv, bra, ket, la, lb, lc, ld, 1, Dm, nrow, oa, ob, oc, od, dB, Gp, Gm, eps);
      centre_derivative<T>(bv, ket, bra, lc, ld, la, lb, 0, Dm, nrow, oc, od, oa, ob, dC, Gp, Gm, eps);
      const int ta = bv.shell_atom[sa], tb = bv.shell_atom[sb], tc = bv.shell_atom[sc], td = bv.shell_atom[sd];
      for (int k = 0; k < 3; ++k) {
        atomicAdd(g.grad + 3 * ta + k, (double)(w * dA[k]));
        atomicAdd(g.grad + 3 * tb + k, (double)(w * dB[k]));
        atomicAdd(g.grad + 3 * tc + k, (double)(w * dC[k]));
        atomicAdd(g.grad + 3 * td + k, -(double)(w * (dA[k] + dB[k] + dC[k])));
      }
    }
  }
}

cudaError_t launch_grad_generic(bool fp64, int X, int Y, const GradLaunch& g, int sms, cudaStream_t s) {
  if (X < 0 || Y < 0 || X >= NCLS || Y > X) return cudaErrorInvalidValue;
  const int grid = sms * 4;
  if (fp64)
    k_grad_generic<double><<<grid, JK_THREADS, 0, s>>>(g, cls_la(X), cls_lb(X), cls_la(Y), cls_lb(Y));
  else
    k_grad_generic<float><<<grid, JK_THREADS, 0, s>>>(g, cls_la(X), cls_lb(X), cls_la(Y), cls_lb(Y));
  return cudaGetLastError();
}

template <typename T, int... I>
static cudaError_t grad_dispatch(int X, int Y, const GradLaunch& g, int sms, cudaStream_t s,
                                 std::integer_sequence<int, I...>) {
  using Fn = cudaError_t (*)(const GradLaunch&, int, cudaStream_t);
  // entries with Y > X are never called (guarded below); they point at a valid launcher
  static constexpr Fn table[] = {&launch_grad_one<T, I / NCLS, (I % NCLS <= I / NCLS ? I % NCLS : 0)>...};
  if (X < 0 || Y < 0 || X >= NCLS || Y > X) return cudaErrorInvalidValue;
  return table[X * NCLS + Y](g, sms, s);
}

cudaError_t launch_grad_fp64(int X, int Y, const GradLaunch& g, int sms, cudaStream_t s) {
  return grad_dispatch<double>(X, Y, g, sms, s, std::make_integer_sequence<int, NCLS * NCLS>{});
}

cudaError_t launch_grad_fp32(int X, int Y, const GradLaunch& g, int sms, cudaStream_t s) {
  return grad_dispatch<float>(X, Y, g, sms, s, std::make_integer_sequence<int, NCLS * NCLS>{});
}

}  // namespace adft
