// Group-cooperative nuclear-gradient kernel for classes up to d shells.
//
// The derivative of a Cartesian Gaussian with respect to its centre raises or
// lowers one power, d/dA_x G_i(a) = 2a G_{i+1}(a) - i G_{i-1}(a), and the
// product of the raised (lowered) function with G_j(b) expands in the same
// Hermite Gaussians Lambda_t(P) as G_i G_j (Helgaker eq. 9.5.1).  So
//   d/dA_x Omega_ab = sum_t (2a E^{i+1,j}_t - i E^{i-1,j}_t) Lambda_t   (x part),
//   d/dB_x Omega_ab = sum_t (2b E^{i,j+1}_t - j E^{i,j-1}_t) Lambda_t,
// with the y and z factors unchanged, and both bra-centre derivatives of a
// primitive quartet follow from the same ket-transformed Hermite integrals
//   W_p[tuv][cd] = sum_q sum_{tau nu phi} (+-) E^cd_{tau nu phi} R_{t+tau,u+nu,v+phi},
// taken one Hermite level higher (t+u+v <= l_a+l_b+1) than for J and K.  The
// pass with SWAP = false differentiates the bra centres A and B of every
// kept quartet (ab|cd); the pass with SWAP = true runs the same kernel on
// (cd|ab) and differentiates C and D.  No centre is obtained by
// translational invariance, so zero net force is a property of the result.
//
// Each derivative block is contracted at once with
//   Gamma_abcd = n_img (1/2 D_ab D_cd - 1/8 (D_ac D_bd + D_ad D_bc)),
// n_img = 8 s_ab s_cd s_(ab,cd) images of the unique quartet, and the six
// sums of a quartet are kept by the group leader while consecutive quartets
// differentiate the same pair of atoms (bra-major work order), so the atomic
// additions into the gradient happen once per change of atom pair.
#pragma once
#include "adft_eri.cuh"

namespace adft {

__host__ __device__ constexpr int cmax(int x, int y) { return x > y ? x : y; }

template <typename T, int LA, int LB, int LC, int LD>
struct GradPlan {
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND;
  static constexpr int LAB = LA + LB, LCD = LC + LD, L1 = LAB + LCD + 1;
  static constexpr int NHAB1 = nherm(LAB + 1), NH1 = nherm(L1);
  static constexpr int NT1 = LAB + 3;                           // t range of the raised bra E table
  static constexpr int EA1 = (LA + 2) * (LB + 2) * NT1;         // bra E with l_a + 1, l_b + 1
  static constexpr int EC = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int WMAX = (sizeof(T) == 8 ? 112 : 128);
  static constexpr CoopShape SHAPE = coop_shape(NCD, NHAB1, WMAX, NH1, EC, NAB, EA1, (int)sizeof(T));
  static constexpr int GS = SHAPE.gs;
  static constexpr int CK = (NCD + GS - 1) / GS;
  static constexpr int NGW = 32 / GS;
  static constexpr int SLOTS = SHAPE.slots;
  static constexpr int SLOT = NH1 + 3 * EC;
  static constexpr int RED = 6 * GS;                             // group reduction scratch
  // slot region: R and ket E tables of the ket primitives, then W of a bra
  // primitive, then the reduction scratch
  static constexpr int REGION = cmax(cmax(SLOTS * SLOT, NHAB1 * NCD), RED);
  static constexpr int GROUP = REGION + NAB * NCD + 3 * EA1;
  static constexpr int WARP_BYTES = NGW * GROUP * (int)sizeof(T);
  static constexpr int WFIT = COOP_SMEM_BUDGET / WARP_BYTES;
  static constexpr int WARPS = WFIT > COOP_MAX_WARPS ? COOP_MAX_WARPS : WFIT;
  static constexpr int WREG = NHAB1 * CK;
  static constexpr bool fits = WARPS >= 1 && WREG <= WMAX && LA <= 2 && LB <= 2 && LC <= 2 && LD <= 2;
  static constexpr int SMEM = WARPS * WARP_BYTES;
};

// Atomic flush of one atom pair's accumulated derivatives.
__device__ __forceinline__ void grad_flush(double* grad, int ta, int tb, const double* acc) {
  if (ta < 0) return;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    atomicAdd(grad + 3 * ta + k, acc[k]);
    atomicAdd(grad + 3 * tb + k, acc[3 + k]);
  }
}

template <typename T, int LA, int LB, int LC, int LD, bool SWAP>
__global__ void __launch_bounds__(32 * COOP_MAX_WARPS) k_grad_coop(GradLaunch gl_) {
  using P = GradPlan<T, LA, LB, LC, LD>;
  constexpr int NB = P::NB, ND = P::ND, NAB = P::NAB, NCD = P::NCD, GS = P::GS, CK = P::CK;
  constexpr int NHAB1 = P::NHAB1, NH1 = P::NH1, EA1 = P::EA1, EC = P::EC, LAB = P::LAB;
  constexpr int NT1 = P::NT1, NTC = P::LCD + 1, LB2 = LB + 2;
  const JKLaunch& a = gl_.jk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ KetTermTable<LC, LD> ktab;
  build_ket_terms<LC, LD>(ktab);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / GS, gl = lane - g * GS;
  const bool in_group = g < P::NGW;
  T* gbase = reinterpret_cast<T*>(smem_raw) + (size_t)(warp * P::NGW + (in_group ? g : 0)) * P::GROUP;
  T* slots = gbase;                                                   // R + ket E tables; reduction scratch
  T* Gam = gbase + P::REGION;                                         // [NAB][NCD]
  T* Eab = Gam + NAB * NCD;                                           // [3][EA1] raised bra E
  const unsigned gmask = (GS == 32) ? 0xffffffffu : (((1u << GS) - 1u) << (g * GS));
  const long long total = (long long)__ldg(a.prefix + a.nseg);
  const BasisView& bv = a.bv;
  const PrimPair<T>* __restrict__ pp = Prec<T>::pp(bv);
  const T* __restrict__ o2pa = Prec<T>::o2p(bv);
  const float* __restrict__ qa = bv.pp_q32;
  const float eps = (float)a.prim_eps;
  const T* __restrict__ wts = nullptr;  // 2a of every primitive pair, then 2b
  if constexpr (sizeof(T) == 8) wts = (const T*)bv.pp_w64; else wts = (const T*)bv.pp_w32;
  int cur_ta = -1, cur_tb = -1;
  double acc[6] = {0, 0, 0, 0, 0, 0};

  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.counter, (unsigned long long)P::NGW);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total) break;
    if (*(volatile const int*)a.abort_flag) {
      if (lane == 0) atomicCAS(a.status, 0, ADFT_ERR_ABORTED);
      break;
    }
    const long long qi = (long long)base + g;
    if (!in_group || qi >= total) continue;
    int bra, ket;
    decode_quartet(a, qi, bra, ket);
    if constexpr (SWAP) { const int t = bra; bra = ket; ket = t; }
    const int sa = __ldg(bv.pair_a + bra), sb = __ldg(bv.pair_b + bra);
    const int sc = __ldg(bv.pair_a + ket), sd = __ldg(bv.pair_b + ket);
    const int oa = __ldg(bv.shell_coff + sa), ob = __ldg(bv.shell_coff + sb);
    const int oc = __ldg(bv.shell_coff + sc), od = __ldg(bv.shell_coff + sd);
    long long mbase;
    long n;
    mol_block(bv, bra, mbase, n);
    const T* __restrict__ Dm = dmat<T>(a) + mbase;
    T w = T(8);
    if (sa == sb) w *= cst<T>(0.5);
    if (sc == sd) w *= cst<T>(0.5);
    if (a.same_class && bra == ket) w *= cst<T>(0.5);
    // Gamma of this lane's ket components (read back only by the same lane)
    for (int kc = gl; kc < NCD; kc += GS) {
      const int c = oc + kc / ND, d = od + kc % ND;
      const T Dcd = __ldg(Dm + (long)c * n + d);
      for (int ab = 0; ab < NAB; ++ab) {
        const int ia = oa + ab / NB, ib = ob + ab % NB;
        const T v = cst<T>(0.5) * __ldg(Dm + (long)ia * n + ib) * Dcd -
                    cst<T>(0.125) * (__ldg(Dm + (long)ia * n + c) * __ldg(Dm + (long)ib * n + d) +
                                     __ldg(Dm + (long)ia * n + d) * __ldg(Dm + (long)ib * n + c));
        Gam[ab * NCD + kc] = w * v;
      }
    }
    const int off0 = __ldg(bv.pair_pp_off + bra), n0 = __ldg(bv.pair_pp_n + bra);
    const int off1 = __ldg(bv.pair_pp_off + ket), n1 = __ldg(bv.pair_pp_n + ket);
    const T AB[3] = {from_f64<T>(__ldg(bv.pair_AB + 3 * bra)), from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 1)),
                     from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 2))};
    const T CDx = from_f64<T>(__ldg(bv.pair_AB + 3 * ket)), CDy = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 1)),
            CDz = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 2));
    T sA[3] = {T(0), T(0), T(0)}, sB[3] = {T(0), T(0), T(0)};

    int n1e = n1;
    for (int ip = 0; ip < n0; ++ip) {
      n1e = shrink_kept(qa + off1, __ldg(qa + off0 + ip), eps, n1e);  // same in every lane
      if (n1e == 0) break;
      const PrimPair<T> bp = pp[off0 + ip];
      const T o2p = __ldg(o2pa + off0 + ip);
      const T ta2 = __ldg(wts + off0 + ip), tb2 = __ldg(wts + bv.npp + off0 + ip);
      for (int d = gl; d < 3; d += GS) {
        const T PA = d == 0 ? bp.PAx : d == 1 ? bp.PAy : bp.PAz;
        hermite_E<T, LA + 1, LB + 1>(PA, PA + AB[d], o2p, Eab + d * EA1);
      }
      T W[NHAB1 * CK];
#pragma unroll
      for (int x = 0; x < NHAB1 * CK; ++x) W[x] = T(0);
      __syncwarp(gmask);
      for (int q0 = 0; q0 < n1e; q0 += P::SLOTS) {
        const int nv = min(P::SLOTS, n1e - q0);
        if (gl < nv) {
          const int iq = off1 + q0 + gl;
          const PrimPair<T> kq = pp[iq];
          const T o2q = __ldg(o2pa + iq);
          T* sl = slots + gl * P::SLOT;
          hermite_E<T, LC, LD>(kq.PAx, kq.PAx + CDx, o2q, sl + NH1);
          hermite_E<T, LC, LD>(kq.PAy, kq.PAy + CDy, o2q, sl + NH1 + EC);
          hermite_E<T, LC, LD>(kq.PAz, kq.PAz + CDz, o2q, sl + NH1 + 2 * EC);
          const T r = Prec<T>::rsq(bp.p + kq.p);
          const T alpha = bp.p * kq.p * r * r;
          const T pref = cst<T>(4.0 * 34.98683665524972) * kq.K * r * o2p * o2q;
          prim_R_scaled<T, P::L1>(alpha, bp.Px - kq.Px, bp.Py - kq.Py, bp.Pz - kq.Pz, pref, bv, sl);
        }
        __syncwarp(gmask);
        for (int s = 0; s < nv; ++s) {
          const T* Rs = slots + s * P::SLOT;
          const T* Es = Rs + NH1;
#pragma unroll
          for (int k = 0; k < CK; ++k) {
            const int kc = gl + k * GS;
            if (kc < NCD) {
              int cx, cy, cz, dx, dy, dz;
              cart_pows_rt(LC, kc / ND, cx, cy, cz);
              cart_pows_rt(LD, kc % ND, dx, dy, dz);
              const T* Ex = Es + (cx * (LD + 1) + dx) * NTC;
              const T* Ey = Es + EC + (cy * (LD + 1) + dy) * NTC;
              const T* Ez = Es + 2 * EC + (cz * (LD + 1) + dz) * NTC;
              const int j1 = ktab.first[kc + 1];
              for (int j = ktab.first[kc]; j < j1; ++j) {
                const int pk = ktab.terms[j];
                const int tau = pk & 15, nu = (pk >> 4) & 15, phi = pk >> 8;
                T e2 = Ex[tau] * Ey[nu] * Ez[phi];
                if ((tau + nu + phi) & 1) e2 = -e2;
                const int sig = tau + nu + phi, mu = nu + phi;
                int t3[LAB + 2], t2[LAB + 2];
#pragma unroll
                for (int x = 0; x <= LAB + 1; ++x) {
                  const int nn = x + sig, mm = x + mu;
                  t3[x] = nn * (nn + 1) * (nn + 2) / 6;
                  t2[x] = mm * (mm + 1) / 2 + phi;
                }
#pragma unroll
                for (int nn = 0; nn <= LAB + 1; ++nn)
#pragma unroll
                  for (int m = 0; m <= nn; ++m)
#pragma unroll
                    for (int v = 0; v <= m; ++v)
                      W[hidx(nn - m, m - v, v) * CK + k] += e2 * Rs[t3[nn] + t2[m] + v];
              }
            }
          }
        }
        __syncwarp(gmask);
      }
      // W to shared memory (the slots are free after the last sync): lane gl
      // writes and reads only its own ket components
      T* Wsm = slots;  // [NHAB1][NCD]
#pragma unroll
      for (int k = 0; k < CK; ++k) {
        const int kc = gl + k * GS;
        if (kc < NCD) {
#pragma unroll
          for (int x = 0; x < NHAB1; ++x) Wsm[x * NCD + kc] = W[x * CK + k];
        }
      }
      // bra-centre derivatives of this bra primitive, contracted with Gamma;
      // E^{i,j}_t of direction d is Eab[d * EA1 + (i * LB2 + j) * NT1 + t]
      for (int kc = gl; kc < NCD; kc += GS) {
        for (int ab = 0; ab < NAB; ++ab) {
          int pa[3], pb[3];
          cart_pows_rt(LA, ab / NB, pa[0], pa[1], pa[2]);
          cart_pows_rt(LB, ab % NB, pb[0], pb[1], pb[2]);
          const T gm = Gam[ab * NCD + kc] * bp.K;
#pragma unroll
          for (int dir = 0; dir < 3; ++dir) {
            const int d1 = dir == 0 ? 1 : 0, d2 = dir == 2 ? 1 : 2;  // the two other directions
            const int i0 = pa[dir], j0 = pb[dir], i1 = pa[d1], j1 = pb[d1], i2 = pa[d2], j2 = pb[d2];
            const T* E0 = Eab + dir * EA1;
            const T* E1 = Eab + d1 * EA1 + (i1 * LB2 + j1) * NT1;
            const T* E2 = Eab + d2 * EA1 + (i2 * LB2 + j2) * NT1;
            T da = T(0), db = T(0);
            for (int t0 = 0; t0 <= i0 + j0 + 1; ++t0) {
              T vs = T(0);
              for (int t1 = 0; t1 <= i1 + j1; ++t1)
                for (int t2 = 0; t2 <= i2 + j2; ++t2) {
                  const int tx = dir == 0 ? t0 : t1;
                  const int ty = dir == 0 ? t1 : dir == 1 ? t0 : t2;
                  const int tz = dir == 2 ? t0 : t2;
                  vs += E1[t1] * E2[t2] * Wsm[hidx(tx, ty, tz) * NCD + kc];
                }
              T ca = ta2 * E0[((i0 + 1) * LB2 + j0) * NT1 + t0];
              if (i0 > 0) ca -= T(i0) * E0[((i0 - 1) * LB2 + j0) * NT1 + t0];
              T cb = tb2 * E0[(i0 * LB2 + j0 + 1) * NT1 + t0];
              if (j0 > 0) cb -= T(j0) * E0[(i0 * LB2 + j0 - 1) * NT1 + t0];
              da += ca * vs;
              db += cb * vs;
            }
            sA[dir] += gm * da;
            sB[dir] += gm * db;
          }
        }
      }
      __syncwarp(gmask);
    }
    // reduce the group's partial sums (the slots are free after the last sync)
#pragma unroll
    for (int dir = 0; dir < 3; ++dir) {
      slots[gl * 6 + dir] = sA[dir];
      slots[gl * 6 + 3 + dir] = sB[dir];
    }
    __syncwarp(gmask);
    if (gl == 0) {
      double v[6] = {0, 0, 0, 0, 0, 0};
      for (int x = 0; x < GS; ++x)
#pragma unroll
        for (int i = 0; i < 6; ++i) v[i] += (double)slots[x * 6 + i];
      const int ta = __ldg(bv.shell_atom + sa), tb = __ldg(bv.shell_atom + sb);
      if (ta != cur_ta || tb != cur_tb) {
        grad_flush(gl_.grad, cur_ta, cur_tb, acc);
        cur_ta = ta; cur_tb = tb;
#pragma unroll
        for (int i = 0; i < 6; ++i) acc[i] = 0.0;
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) acc[i] += v[i];
    }
    __syncwarp(gmask);
  }
  if (in_group && gl == 0) grad_flush(gl_.grad, cur_ta, cur_tb, acc);
}

// ---------------------------------------------------------------------------
// Gradient launcher of one class pair (X, Y), X >= Y: the two cooperative
// passes where both fit, else the runtime-L kernel of adft_grad.cu (all four
// centres in one pass).  sms: the device's SM count.
cudaError_t launch_grad_generic(bool fp64, int X, int Y, const GradLaunch& g, int sms, cudaStream_t s);

template <typename T, int X, int Y>
cudaError_t launch_grad_one(const GradLaunch& g, int sms, cudaStream_t s);

#ifndef ADFT_ERI_DECLARE_ONLY
template <typename T, int LA, int LB, int LC, int LD, bool SWAP>
static cudaError_t start_grad(const GradLaunch& g, int sms, cudaStream_t s) {
  using P = GradPlan<T, LA, LB, LC, LD>;
  static int per_sm_dev[PerDeviceFlag::MAXDEV] = {};  // resident blocks per SM, per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= PerDeviceFlag::MAXDEV) dev = 0;
  int& per_sm = per_sm_dev[dev];
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_grad_coop<T, LA, LB, LC, LD, SWAP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_grad_coop<T, LA, LB, LC, LD, SWAP>, 32 * P::WARPS,
                                                      P::SMEM);
    if (e != cudaSuccess) return e;
    per_sm = n > 0 ? n : 1;
  }
  k_grad_coop<T, LA, LB, LC, LD, SWAP><<<sms * per_sm, 32 * P::WARPS, P::SMEM, s>>>(g);
  return cudaGetLastError();
}

template <typename T, int X, int Y>
cudaError_t launch_grad_one(const GradLaunch& g, int sms, cudaStream_t s) {
  constexpr int LA = cls_la(X), LB = cls_lb(X), LC = cls_la(Y), LD = cls_lb(Y);
  if constexpr (X < Y) {
    return cudaErrorInvalidValue;
  } else if constexpr (GradPlan<T, LA, LB, LC, LD>::fits && GradPlan<T, LC, LD, LA, LB>::fits) {
    cudaError_t e = start_grad<T, LA, LB, LC, LD, false>(g, sms, s);
    if (e != cudaSuccess) return e;
    GradLaunch g2 = g;
    g2.jk.counter = g.counter2;
    return start_grad<T, LC, LD, LA, LB, true>(g2, sms, s);
  } else {
    return launch_grad_generic(sizeof(T) == 8, X, Y, g, sms, s);
  }
}
#endif

}  // namespace adft
