// Warp-uniform J/K kernel for the larger angular-momentum classes.
//
// One warp owns one shell quartet, and every instruction of the integral
// loops is executed by all lanes with the same control flow:
//   * ket transform: lane l owns bra Hermite index (t,u,v) = l (and l+32 if
//     the bra has more than 32); for every ket primitive in shared memory it
//     accumulates W[tuv][cd] = sum_{tau nu phi} e2_q[cd][tau nu phi]
//     R_q[t+tau, u+nu, v+phi] over all ket components cd, with the component
//     and (tau, nu, phi) loops unrolled at compile time, so the only
//     lane-dependent quantity is the R address;
//   * bra transform and digestion: lane l owns ket component l (and l+32):
//     G[ab][cd] += K_p sum_tuv Eprod_p[ab][tuv] W[tuv][cd], the (ab, tuv)
//     loops again unrolled and identical for every lane.
// The lane-invariant products e2_q = (+-) E^cd_x E^cd_y E^cd_z of a ket
// primitive and Eprod_p = E^ab_x E^ab_y E^ab_z of a bra primitive are
// formed once into shared memory.  Up to SL ket primitives are evaluated at
// once, one per lane (R in place, prefactor folded in).
#pragma once
// (included by adft_eri.cuh inside namespace adft)

// (ia, ib, t, u, v) of the k-th bra term in the order of the bra transform
// (integer work only, done once per entry and bra primitive)
template <int LA, int LB>
__device__ __forceinline__ void bra_term(int k, int& ia, int& ib, int& t, int& u, int& v) {
  constexpr int NB = ncart(LB);
  for (int ab = 0; ab < ncart(LA) * NB; ++ab) {
    ia = ab / NB; ib = ab % NB;
    const int sx = cart_x(LA, ia) + cart_x(LB, ib) + 1, sy = cart_y(LA, ia) + cart_y(LB, ib) + 1,
              sz = cart_z(LA, ia) + cart_z(LB, ib) + 1;
    const int n = sx * sy * sz;
    if (k < n) {
      t = k / (sy * sz);
      u = (k / sz) % sy;
      v = k % sz;
      return;
    }
    k -= n;
  }
  ia = ib = t = u = v = 0;
}

template <typename T, int LA, int LB, int LC, int LD>
struct WarpPlan {
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND;
  static constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  static constexpr int NHAB = nherm(LAB), NH = nherm(L);
  static constexpr int EA = (LA + 1) * (LB + 1) * (LAB + 1), EC = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int KT = ket_terms<LC, LD>();  // e2 entries per ket primitive
  static constexpr int BT = ket_terms<LA, LB>();  // Eprod entries per bra primitive
  static constexpr int HP = (NHAB + 31) / 32;     // bra Hermite indices per lane
  static constexpr int CP = (NCD + 31) / 32;      // ket components per lane
  static constexpr int SLOT = NH + 3 * EC + KT;   // R, ket E tables, e2
  static constexpr int FIXED = NHAB * NCD + NAB * NCD + 3 * EA + BT;  // W, G, bra E, Eprod
  static constexpr int warp_values(int sl) { return sl * SLOT + FIXED; }
  static constexpr int pick_sl() {
    const int opts[4] = {16, 8, 4, 2};
    for (int i = 0; i < 4; ++i)
      if (COOP_SMEM_BUDGET / (warp_values(opts[i]) * (int)sizeof(T)) >= 4) return opts[i];
    return 1;
  }
  static constexpr int SL = pick_sl();
  static constexpr int WARP_BYTES = warp_values(SL) * (int)sizeof(T);
  static constexpr int WFIT = COOP_SMEM_BUDGET / WARP_BYTES;
  static constexpr int WARPS = WFIT > COOP_MAX_WARPS ? COOP_MAX_WARPS : WFIT;
  static constexpr int SMEM = WARPS * WARP_BYTES;
  // bra with at most 32 Hermite functions (one per lane) and at most 18 ket
  // components.  Larger unrolled bodies spill and compile too slowly, and for
  // d/d bras (two Hermite passes per lane, 35 of 64 lane slots busy) the
  // cooperative kernel was faster on every class measured; those classes use
  // k_jk_coop only.
  static constexpr bool fits = WARPS >= 2 && HP == 1 && NCD <= 18 && LA <= 2 && LC <= 2;
};

template <typename T, int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(32 * COOP_MAX_WARPS) k_jk_warp(JKLaunch a) {
  using P = WarpPlan<T, LA, LB, LC, LD>;
  constexpr int NB = P::NB, ND = P::ND, NAB = P::NAB, NCD = P::NCD, NHAB = P::NHAB, NH = P::NH;
  constexpr int EA = P::EA, EC = P::EC, KT = P::KT, BT = P::BT, SL = P::SL, HP = P::HP, CP = P::CP;
  constexpr int LAB = P::LAB, LCD = P::LCD, NTA = LAB + 1, NTC = LCD + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* base = reinterpret_cast<T*>(smem_raw) + (size_t)warp * (P::WARP_BYTES / sizeof(T));
  T* slots = base;                      // [SL][SLOT]: R, E^cd (3 x EC), e2 (KT)
  T* Wsm = base + SL * P::SLOT;         // [NHAB][NCD]
  T* Gsm = Wsm + NHAB * NCD;            // [NAB][NCD]
  T* Eab = Gsm + NAB * NCD;             // [3][EA]
  T* Eprod = Eab + 3 * EA;              // [BT]
  const long long total = (long long)__ldg(a.prefix + a.nseg);
  const BasisView& bv = a.bv;
  const PrimPair<T>* __restrict__ pp = Prec<T>::pp(bv);
  const T* __restrict__ o2pa = Prec<T>::o2p(bv);
  const float* __restrict__ qa = bv.pp_q32;
  const float eps = (float)a.prim_eps;
  unsigned cpq = 0, cbp = 0;  // evaluated work (lane 0)

  // this lane's bra Hermite indices: offsets of R(t+tau, u+nu, v+phi) as
  // T3(n + sigma) + T2(m + mu) + v + phi, sigma = tau+nu+phi, mu = nu+phi
  int my_v[HP], t3[HP][LCD + 1], t2[HP][LCD + 1];
  bool my_ok[HP];
#pragma unroll
  for (int h = 0; h < HP; ++h) {
    const int idx = lane + 32 * h;
    my_ok[h] = idx < NHAB;
    int n = 0, m = 0, v = 0;
    if (my_ok[h]) {  // invert hidx: n = t+u+v, m = u+v
      while ((n + 1) * (n + 2) * (n + 3) / 6 <= idx) ++n;
      const int r = idx - n * (n + 1) * (n + 2) / 6;
      while ((m + 1) * (m + 2) / 2 <= r) ++m;
      v = r - m * (m + 1) / 2;
    }
    my_v[h] = v;
#pragma unroll
    for (int s = 0; s <= LCD; ++s) {
      const int nn = n + s, mm = m + s;
      t3[h][s] = nn * (nn + 1) * (nn + 2) / 6;
      t2[h][s] = mm * (mm + 1) / 2;
    }
  }

  for (;;) {
    unsigned long long qb = 0;
    if (lane == 0) qb = atomicAdd(a.counter, 1ULL);
    qb = __shfl_sync(0xffffffffu, qb, 0);
    if ((long long)qb >= total) break;
    if (*(volatile const int*)a.abort_flag) {
      if (lane == 0) atomicCAS(a.status, 0, ADFT_ERR_ABORTED);
      break;
    }
    int bra, ket;
    decode_quartet(a, (long long)qb, bra, ket);
    const int off0 = __ldg(bv.pair_pp_off + bra), n0 = __ldg(bv.pair_pp_n + bra);
    const int off1 = __ldg(bv.pair_pp_off + ket), n1 = __ldg(bv.pair_pp_n + ket);
    const T AB[3] = {from_f64<T>(__ldg(bv.pair_AB + 3 * bra)), from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 1)),
                     from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 2))};
    const T CD[3] = {from_f64<T>(__ldg(bv.pair_AB + 3 * ket)), from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 1)),
                     from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 2))};
    for (int x = lane; x < NAB * NCD; x += 32) Gsm[x] = T(0);

    int n1e = n1;
    for (int ip = 0; ip < n0; ++ip) {
      n1e = shrink_kept(qa + off1, __ldg(qa + off0 + ip), eps, n1e);  // same in every lane
      if (n1e == 0) break;
      if (lane == 0) { cpq += n1e; ++cbp; }
      const PrimPair<T> bp = pp[off0 + ip];
      const T o2p = __ldg(o2pa + off0 + ip);
      if (lane < 3) {
        const T PA = lane == 0 ? bp.PAx : lane == 1 ? bp.PAy : bp.PAz;
        hermite_E<T, LA, LB>(PA, PA + AB[lane], o2p, Eab + lane * EA);
      }
      T W[HP][NCD];
#pragma unroll
      for (int h = 0; h < HP; ++h)
#pragma unroll
        for (int c = 0; c < NCD; ++c) W[h][c] = T(0);
      __syncwarp();
      // Eprod[ab][tuv] of this bra primitive (lane-invariant products), the
      // entries split over the lanes through the compile-time index table
      for (int k = lane; k < BT; k += 32) {
        int ia, ib, t, u, v;
        bra_term<LA, LB>(k, ia, ib, t, u, v);
        const int ax = cart_x(LA, ia), ay = cart_y(LA, ia), az = cart_z(LA, ia);
        const int bx = cart_x(LB, ib), by = cart_y(LB, ib), bz = cart_z(LB, ib);
        Eprod[k] = bp.K * Eab[(ax * (LB + 1) + bx) * NTA + t] * Eab[EA + (ay * (LB + 1) + by) * NTA + u] *
                   Eab[2 * EA + (az * (LB + 1) + bz) * NTA + v];
      }
      __syncwarp();
      for (int q0 = 0; q0 < n1e; q0 += SL) {
        const int nv = min(SL, n1e - q0);
        if (lane < nv) {
          const int iq = off1 + q0 + lane;
          const PrimPair<T> kq = pp[iq];
          const T o2q = __ldg(o2pa + iq);
          T* sl = slots + lane * P::SLOT;
          T* Ec = sl + NH;
          hermite_E<T, LC, LD>(kq.PAx, kq.PAx + CD[0], o2q, Ec);
          hermite_E<T, LC, LD>(kq.PAy, kq.PAy + CD[1], o2q, Ec + EC);
          hermite_E<T, LC, LD>(kq.PAz, kq.PAz + CD[2], o2q, Ec + 2 * EC);
          const T r = Prec<T>::rsq(bp.p + kq.p);
          T alpha = bp.p * kq.p * r * r;
          T pref = cst<T>(4.0 * 34.98683665524972) * kq.K * r * o2p * o2q;
          attenuate((T)a.omega2, alpha, pref);
          prim_R_scaled<T, P::L>(alpha, bp.Px - kq.Px, bp.Py - kq.Py, bp.Pz - kq.Pz, pref, bv, sl);
          // e2[cd][tau nu phi] = (-1)^(tau+nu+phi) E_x E_y E_z
          T* e2 = Ec + 3 * EC;
          int k = 0;
#pragma unroll
          for (int kc = 0; kc < NCD; ++kc) {
            const int ic = kc / ND, id = kc % ND;
            const int cx = cart_pow(LC, ic, 0), cy = cart_pow(LC, ic, 1), cz = cart_pow(LC, ic, 2);
            const int dx = cart_pow(LD, id, 0), dy = cart_pow(LD, id, 1), dz = cart_pow(LD, id, 2);
#pragma unroll
            for (int tau = 0; tau <= cx + dx; ++tau)
#pragma unroll
              for (int nu = 0; nu <= cy + dy; ++nu) {
                const T exy = Ec[(cx * (LD + 1) + dx) * NTC + tau] * Ec[EC + (cy * (LD + 1) + dy) * NTC + nu];
#pragma unroll
                for (int phi = 0; phi <= cz + dz; ++phi, ++k) {
                  const T e = exy * Ec[2 * EC + (cz * (LD + 1) + dz) * NTC + phi];
                  e2[k] = ((tau + nu + phi) & 1) ? -e : e;
                }
              }
          }
        }
        __syncwarp();
        for (int s = 0; s < nv; ++s) {
          const T* Rs = slots + s * P::SLOT;
          const T* e2 = Rs + NH + 3 * EC;
#pragma unroll
          for (int h = 0; h < HP; ++h) {
            if (!my_ok[h]) continue;
            const T* Rv = Rs + my_v[h];
            int k = 0;
#pragma unroll
            for (int kc = 0; kc < NCD; ++kc) {
              const int ic = kc / ND, id = kc % ND;
              const int cx = cart_pow(LC, ic, 0), cy = cart_pow(LC, ic, 1), cz = cart_pow(LC, ic, 2);
              const int dx = cart_pow(LD, id, 0), dy = cart_pow(LD, id, 1), dz = cart_pow(LD, id, 2);
              T acc = T(0);
#pragma unroll
              for (int tau = 0; tau <= cx + dx; ++tau)
#pragma unroll
                for (int nu = 0; nu <= cy + dy; ++nu)
#pragma unroll
                  for (int phi = 0; phi <= cz + dz; ++phi, ++k)
                    acc += e2[k] * Rv[t3[h][tau + nu + phi] + t2[h][nu + phi] + phi];
              W[h][kc] += acc;
            }
          }
        }
        __syncwarp();
      }
      // bra transform: lane = ket component
#pragma unroll
      for (int h = 0; h < HP; ++h)
        if (my_ok[h])
#pragma unroll
          for (int c = 0; c < NCD; ++c) Wsm[(lane + 32 * h) * NCD + c] = W[h][c];
      __syncwarp();
#pragma unroll
      for (int cc = 0; cc < CP; ++cc) {
        const int kc = lane + 32 * cc;
        if (kc < NCD) {
          int k = 0;
#pragma unroll
          for (int ab = 0; ab < NAB; ++ab) {
            const int ia = ab / NB, ib = ab % NB;
            const int ax = cart_pow(LA, ia, 0), ay = cart_pow(LA, ia, 1), az = cart_pow(LA, ia, 2);
            const int bx = cart_pow(LB, ib, 0), by = cart_pow(LB, ib, 1), bz = cart_pow(LB, ib, 2);
            T acc = T(0);
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
              for (int u = 0; u <= ay + by; ++u)
#pragma unroll
                for (int v = 0; v <= az + bz; ++v, ++k) acc += Eprod[k] * Wsm[hidx(t, u, v) * NCD + kc];
            Gsm[ab * NCD + kc] += acc;
          }
        }
      }
      __syncwarp();
    }
    __syncwarp();  // the digestion reads the whole warp's block
    digest_coop<T, LA, LB, LC, LD>(a, bra, ket, lane, 32, Gsm);
    __syncwarp();
  }
  flush_work(a.work, cpq, cbp);
}
