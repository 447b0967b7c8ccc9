// Group-cooperative J/K kernel for the larger angular-momentum classes.
//
// A group of GS lanes owns one shell quartet (GS and SLOTS are chosen together
// by coop_shape below).  Lane gl owns ket components gl, gl+GS, ...; for
// every bra primitive p the group evaluates the Hermite integrals R of up to
// SLOTS ket primitives at once (one ket primitive per lane, written to shared
// memory together with that primitive's ket Hermite expansion coefficients),
// then every lane applies the ket transform of its own components to all of
// them:  W_p[tuv][cd] += sum_{tau nu phi} (+-) E^cd_{tau nu phi} R_{t+tau,u+nu,v+phi},
// one flat loop over each component's (tau, nu, phi) terms (KetTermTable).
// The bra transform of W_p is accumulated into the contracted block in
// shared memory, and the J/K digestion reads that block.  Compared with one
// thread per quartet this computes R once per primitive quartet instead of
// once per component chunk, and keeps every array out of local memory.
#pragma once
// (included by adft_eri.cuh inside namespace adft)

constexpr int COOP_SLOT_CAP = 8;
constexpr int COOP_SMEM_BUDGET = 200 * 1024;
constexpr int COOP_MAX_WARPS = 8;

// number of (tau, nu, phi) terms of the ket transform, summed over ket components
template <int LC, int LD>
__host__ __device__ constexpr int ket_terms() {
  int n = 0;
  for (int kc = 0; kc < ncart(LC) * ncart(LD); ++kc) {
    const int ic = kc / ncart(LD), id = kc % ncart(LD);
    n += (cart_pow(LC, ic, 0) + cart_pow(LD, id, 0) + 1) * (cart_pow(LC, ic, 1) + cart_pow(LD, id, 1) + 1) *
         (cart_pow(LC, ic, 2) + cart_pow(LD, id, 2) + 1);
  }
  return n;
}

// Flat term list of the ket transform of class (LC, LD): the (tau, nu, phi)
// triples of ket component kc, packed as tau | nu << 4 | phi << 8, are
// terms[first[kc] .. first[kc + 1]).  A lane then runs one loop over its
// component's terms, so the lanes of a group differ only in trip count (not
// in the shape of three nested loops).  Built by thread 0 of the block.
template <int LC, int LD>
struct KetTermTable {
  static constexpr int NCD = ncart(LC) * ncart(LD);
  static constexpr int KT = ket_terms<LC, LD>();
  unsigned short terms[KT];
  unsigned short first[NCD + 1];
};

template <int LC, int LD>
__device__ __forceinline__ void build_ket_terms(KetTermTable<LC, LD>& tab) {
  constexpr int ND = ncart(LD), NCD = ncart(LC) * ND;
  if (threadIdx.x == 0) {
    int k = 0;
    for (int kc = 0; kc < NCD; ++kc) {
      tab.first[kc] = (unsigned short)k;
      const int ic = kc / ND, id = kc % ND;
      const int sx = cart_x(LC, ic) + cart_x(LD, id), sy = cart_y(LC, ic) + cart_y(LD, id),
                sz = cart_z(LC, ic) + cart_z(LD, id);
      for (int tau = 0; tau <= sx; ++tau)
        for (int nu = 0; nu <= sy; ++nu)
          for (int phi = 0; phi <= sz; ++phi) tab.terms[k++] = (unsigned short)(tau | (nu << 4) | (phi << 8));
    }
    tab.first[NCD] = (unsigned short)k;
  }
  __syncthreads();
}

// pref * R_tuv of one primitive quartet into R (any memory space)
template <typename T, int L>
__device__ __forceinline__ void prim_R_scaled(T alpha, T X, T Y, T Z, T pref, const BasisView& bv, T* R) {
  T B[L + 1];
  const T Tb = alpha * (X * X + Y * Y + Z * Z);
  if constexpr (is_f64<T>) {
    boys_fp64<L>(Tb, bv.boys64, B);
    const T f = -2.0 * alpha;
    T pw = pref;
#pragma unroll
    for (int n = 0; n <= L; ++n) { B[n] *= pw; pw *= f; }
    hermite_R<T, L>(B, X, Y, Z, R);
  } else {
    boys_fp32_scaled<L>(Tb, bv.boys32, B);
#pragma unroll
    for (int n = 0; n <= L; ++n) B[n] *= (n & 1) ? -pref : pref;
    const float c = fmaxf(1.0f, 2.0f * Tb);
    const float s = sqrtf(2.0f * alpha / c);
    hermite_R<T, L>(B, X * s, Y * s, Z * s, R);
    float sp = s;
#pragma unroll
    for (int n = 1; n <= L; ++n) {
#pragma unroll
      for (int x = nherm(n - 1); x < nherm(n); ++x) R[x] *= sp;
      sp *= s;
    }
  }
}

// J/K digestion from the contracted block Gs[ab * GSTRIDE + cd] in shared memory (same
// weights and targets as digest_range): the GS lanes of the group split the
// distinct output elements, so every J and K element a quartet touches gets
// exactly one atomic, NAB + NCD + (NA + NB)(NC + ND) per quartet.
template <typename T, int LA, int LB, int LC, int LD, int GSTRIDE = ncart(LC) * ncart(LD)>
__device__ __forceinline__ void digest_coop(const JKLaunch& a, int bra, int ket, int gl, int GS, const T* Gs) {
  constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  constexpr int NAB = NA * NB, NCD = NC * ND;
  const BasisView& bv = a.bv;
  const int sa = __ldg(bv.pair_a + bra), sb = __ldg(bv.pair_b + bra);
  const int sc = __ldg(bv.pair_a + ket), sd = __ldg(bv.pair_b + ket);
  const int oa = __ldg(bv.shell_coff + sa), ob = __ldg(bv.shell_coff + sb);
  const int oc = __ldg(bv.shell_coff + sc), od = __ldg(bv.shell_coff + sd);
  long long base;
  long n;
  mol_block(bv, bra, base, n);
  T w = T(1);
  if (sa == sb) w *= cst<T>(0.5);
  if (sc == sd) w *= cst<T>(0.5);
  if (a.same_class && bra == ket) w *= cst<T>(0.5);
  const T w4 = T(4) * w, w2 = T(2) * w;
  const T* __restrict__ D = dmat<T>(a) + base;
  double* __restrict__ Jm = a.J + base;
  double* __restrict__ Km = a.K + base;
  for (int ab = gl; ab < NAB; ab += GS) {  // J_ab = sum_cd g D_cd
    T s = T(0);
    for (int cd = 0; cd < NCD; ++cd) s += Gs[ab * GSTRIDE + cd] * __ldg(D + (oc + cd / ND) * n + od + cd % ND);
    atomicAdd(Jm + (oa + ab / NB) * n + ob + ab % NB, (double)(w4 * s));
  }
  for (int cd = gl; cd < NCD; cd += GS) {  // J_cd = sum_ab g D_ab
    T s = T(0);
    for (int ab = 0; ab < NAB; ++ab) s += Gs[ab * GSTRIDE + cd] * __ldg(D + (oa + ab / NB) * n + ob + ab % NB);
    atomicAdd(Jm + (oc + cd / ND) * n + od + cd % ND, (double)(w4 * s));
  }
  for (int o = gl; o < NA * NC; o += GS) {  // K_ac = sum_bd g D_bd
    const int x = o / NC, c = o % NC;
    T s = T(0);
    for (int y = 0; y < NB; ++y)
      for (int d = 0; d < ND; ++d) s += Gs[(x * NB + y) * GSTRIDE + c * ND + d] * __ldg(D + (ob + y) * n + od + d);
    atomicAdd(Km + (oa + x) * n + oc + c, (double)(w2 * s));
  }
  for (int o = gl; o < NA * ND; o += GS) {  // K_ad = sum_bc g D_bc
    const int x = o / ND, d = o % ND;
    T s = T(0);
    for (int y = 0; y < NB; ++y)
      for (int c = 0; c < NC; ++c) s += Gs[(x * NB + y) * GSTRIDE + c * ND + d] * __ldg(D + (ob + y) * n + oc + c);
    atomicAdd(Km + (oa + x) * n + od + d, (double)(w2 * s));
  }
  for (int o = gl; o < NB * NC; o += GS) {  // K_bc = sum_ad g D_ad
    const int y = o / NC, c = o % NC;
    T s = T(0);
    for (int x = 0; x < NA; ++x)
      for (int d = 0; d < ND; ++d) s += Gs[(x * NB + y) * GSTRIDE + c * ND + d] * __ldg(D + (oa + x) * n + od + d);
    atomicAdd(Km + (ob + y) * n + oc + c, (double)(w2 * s));
  }
  for (int o = gl; o < NB * ND; o += GS) {  // K_bd = sum_ac g D_ac
    const int y = o / ND, d = o % ND;
    T s = T(0);
    for (int x = 0; x < NA; ++x)
      for (int c = 0; c < NC; ++c) s += Gs[(x * NB + y) * GSTRIDE + c * ND + d] * __ldg(D + (oa + x) * n + oc + c);
    atomicAdd(Km + (ob + y) * n + od + d, (double)(w2 * s));
  }
}

// Group shape: GS lanes share one quartet and stage SLOTS ket primitives at a
// time (SLOTS <= GS, one primitive per lane).  The shape maximises the useful
// fraction of the warp, (lanes in whole groups / 32) * (NCD / (GS * CK)) with
// CK = ceil(NCD / GS) ket components per lane, under the register budget
// NHAB * CK <= wmax for the per-lane W block and the shared-memory budget of at
// least 4 warps per block (one per SM sub-partition); for each GS the largest
// SLOTS in {min(GS, 8), 4, 2, 1} that fits is taken, and between equally
// useful shapes the one with more slots wins.
struct CoopShape {
  int gs, slots;
};
__host__ __device__ constexpr CoopShape coop_shape(int ncd, int nhab, int wmax, int nh, int ec, int nab, int ea,
                                                   int tsize) {
  CoopShape best{32 < ncd ? 32 : ncd, 1};
  double best_u = -1.0;
  for (int gs = 1; gs <= 32 && gs <= ncd; ++gs) {
    const int ck = (ncd + gs - 1) / gs;
    if (nhab * ck > wmax) continue;
    int slots = gs < COOP_SLOT_CAP ? gs : COOP_SLOT_CAP;
    bool ok = false;
    for (; slots >= 1; slots = (slots > 4 ? 4 : slots / 2)) {
      const int group = slots * (nh + 3 * ec) + nab * ncd + 3 * ea;
      const int warp_bytes = (32 / gs) * group * tsize;
      if (COOP_SMEM_BUDGET / warp_bytes >= 4) { ok = true; break; }
    }
    if (!ok) continue;
    const double u = (double)((32 / gs) * gs) / 32.0 * (double)ncd / (double)(gs * ck);
    if (u > best_u + 1e-9 || (u > best_u - 1e-9 && slots > best.slots)) {
      best_u = u;
      best = CoopShape{gs, slots};
    }
  }
  return best;
}

template <typename T, int LA, int LB, int LC, int LD>
struct CoopPlan {
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND;
  static constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  static constexpr int NHAB = nherm(LAB), NH = nherm(L);
  static constexpr int EA = (LA + 1) * (LB + 1) * (LAB + 1), EC = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int WMAX = (sizeof(T) == 8 ? 80 : 100);
  static constexpr CoopShape SHAPE = coop_shape(NCD, NHAB, WMAX, NH, EC, NAB, EA, (int)sizeof(T));
  static constexpr int GS = SHAPE.gs;
  static constexpr int CK = (NCD + GS - 1) / GS;
  static constexpr int NGW = 32 / GS;
  static constexpr int SLOTS = SHAPE.slots;
  static constexpr int SLOT = NH + 3 * EC;
  static constexpr int GROUP = SLOTS * SLOT + NAB * NCD + 3 * EA;
  static constexpr int WARP_BYTES = NGW * GROUP * (int)sizeof(T);
  static constexpr int WFIT = COOP_SMEM_BUDGET / WARP_BYTES;
  static constexpr int WARPS = WFIT > COOP_MAX_WARPS ? COOP_MAX_WARPS : WFIT;
  static constexpr int WREG = NHAB * CK;  // W values per lane (registers)
  // classes up to d shells (f classes keep the runtime-L kernel, which
  // compiles far faster)
  static constexpr bool fits = WARPS >= 1 && WREG <= WMAX && LA <= 2 && LC <= 2;
  static constexpr int SMEM = WARPS * WARP_BYTES;
};

template <typename T, int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(32 * COOP_MAX_WARPS, 1) k_jk_coop(JKLaunch a) {
  using P = CoopPlan<T, LA, LB, LC, LD>;
  constexpr int NB = P::NB, ND = P::ND, NAB = P::NAB, NCD = P::NCD, GS = P::GS, CK = P::CK;
  constexpr int NHAB = P::NHAB, NH = P::NH, EA = P::EA, EC = P::EC, LAB = P::LAB;
  constexpr int NTA = LAB + 1, NTC = P::LCD + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ KetTermTable<LC, LD> ktab;
  build_ket_terms<LC, LD>(ktab);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / GS, gl = lane - g * GS;
  const bool in_group = g < P::NGW;
  T* gbase = reinterpret_cast<T*>(smem_raw) + (size_t)(warp * P::NGW + (in_group ? g : 0)) * P::GROUP;
  T* slots = gbase;                     // [SLOTS][SLOT]: R then 3 x EC ket E tables
  T* Gs = gbase + P::SLOTS * P::SLOT;   // [NAB][NCD] contracted block
  T* Eab = Gs + NAB * NCD;              // [3][EA] bra E of the current bra primitive
  const unsigned gmask = (GS == 32) ? 0xffffffffu : (((1u << GS) - 1u) << (g * GS));
  const long long total = (long long)__ldg(a.prefix + a.nseg);
  const BasisView& bv = a.bv;
  const PrimPair<T>* __restrict__ pp = Prec<T>::pp(bv);
  const T* __restrict__ o2pa = Prec<T>::o2p(bv);
  const float* __restrict__ qa = bv.pp_q32;
  const float eps = (float)a.prim_eps;
  unsigned cpq = 0, cbp = 0;  // evaluated work (group leaders)

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
    const int off0 = __ldg(bv.pair_pp_off + bra), n0 = __ldg(bv.pair_pp_n + bra);
    const int off1 = __ldg(bv.pair_pp_off + ket), n1 = __ldg(bv.pair_pp_n + ket);
    const T AB[3] = {from_f64<T>(__ldg(bv.pair_AB + 3 * bra)), from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 1)),
                     from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 2))};
    const T CDx = from_f64<T>(__ldg(bv.pair_AB + 3 * ket)), CDy = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 1)),
            CDz = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 2));
    for (int kc = gl; kc < NCD; kc += GS)
      for (int ab = 0; ab < NAB; ++ab) Gs[ab * NCD + kc] = T(0);

    int n1e = n1;
    for (int ip = 0; ip < n0; ++ip) {
      n1e = shrink_kept(qa + off1, __ldg(qa + off0 + ip), eps, n1e);  // same in every lane
      if (n1e == 0) break;
      if (gl == 0) { cpq += n1e; ++cbp; }
      const PrimPair<T> bp = pp[off0 + ip];
      const T o2p = __ldg(o2pa + off0 + ip);
      for (int d = gl; d < 3; d += GS) {  // groups may have fewer than 3 lanes
        const T PA = d == 0 ? bp.PAx : d == 1 ? bp.PAy : bp.PAz;
        const T ABd = d == 0 ? AB[0] : d == 1 ? AB[1] : AB[2];  // (no dynamic register index)
        hermite_E<T, LA, LB>(PA, PA + ABd, o2p, Eab + d * EA);
      }
      T W[NHAB * CK];
#pragma unroll
      for (int x = 0; x < NHAB * CK; ++x) W[x] = T(0);
      __syncwarp(gmask);
      for (int q0 = 0; q0 < n1e; q0 += P::SLOTS) {
        const int nv = min(P::SLOTS, n1e - q0);
        if (gl < nv) {
          const int iq = off1 + q0 + gl;
          const PrimPair<T> kq = pp[iq];
          const T o2q = __ldg(o2pa + iq);
          T* sl = slots + gl * P::SLOT;
          hermite_E<T, LC, LD>(kq.PAx, kq.PAx + CDx, o2q, sl + NH);
          hermite_E<T, LC, LD>(kq.PAy, kq.PAy + CDy, o2q, sl + NH + EC);
          hermite_E<T, LC, LD>(kq.PAz, kq.PAz + CDz, o2q, sl + NH + 2 * EC);
          const T r = Prec<T>::rsq(bp.p + kq.p);
          T alpha = bp.p * kq.p * r * r;
          T pref = cst<T>(4.0 * 34.98683665524972) * kq.K * r * o2p * o2q;
          attenuate((T)a.omega2, alpha, pref);
          prim_R_scaled<T, P::L>(alpha, bp.Px - kq.Px, bp.Py - kq.Py, bp.Pz - kq.Pz, pref, bv, sl);
        }
        __syncwarp(gmask);
        for (int s = 0; s < nv; ++s) {
          const T* Rs = slots + s * P::SLOT;
          const T* Es = Rs + NH;
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
                // R index of (t+tau, u+nu, v+phi) = T3(n0 + sig) + T2(m0 + mu) + v + phi
                const int sig = tau + nu + phi, mu = nu + phi;
                int t3[LAB + 1], t2[LAB + 1];
#pragma unroll
                for (int x = 0; x <= LAB; ++x) {
                  const int nn = x + sig, mm = x + mu;
                  t3[x] = nn * (nn + 1) * (nn + 2) / 6;
                  t2[x] = mm * (mm + 1) / 2 + phi;
                }
#pragma unroll
                for (int n = 0; n <= LAB; ++n)
#pragma unroll
                  for (int m = 0; m <= n; ++m)
#pragma unroll
                    for (int v = 0; v <= m; ++v)
                      W[hidx(n - m, m - v, v) * CK + k] += e2 * Rs[t3[n] + t2[m] + v];
              }
            }
          }
        }
        __syncwarp(gmask);
      }
      // bra transform of this bra primitive into the contracted block
#pragma unroll
      for (int k = 0; k < CK; ++k) {
        const int kc = gl + k * GS;
        if (kc < NCD) {
#pragma unroll
          for (int ab = 0; ab < NAB; ++ab) {
            const int ia = ab / NB, ib = ab % NB;
            const int ax = cart_pow(LA, ia, 0), ay = cart_pow(LA, ia, 1), az = cart_pow(LA, ia, 2);
            const int bx = cart_pow(LB, ib, 0), by = cart_pow(LB, ib, 1), bz = cart_pow(LB, ib, 2);
            T acc = T(0);
#pragma unroll
            for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
              for (int u = 0; u <= ay + by; ++u) {
                const T exy = Eab[(ax * (LB + 1) + bx) * NTA + t] * Eab[EA + (ay * (LB + 1) + by) * NTA + u];
#pragma unroll
                for (int v = 0; v <= az + bz; ++v)
                  acc += exy * Eab[2 * EA + (az * (LB + 1) + bz) * NTA + v] * W[hidx(t, u, v) * CK + k];
              }
            Gs[ab * NCD + kc] += bp.K * acc;
          }
        }
      }
      __syncwarp(gmask);
    }
    __syncwarp(gmask);  // the digestion reads the whole group's block
    digest_coop<T, LA, LB, LC, LD>(a, bra, ket, gl, GS, Gs);
    __syncwarp(gmask);
  }
  flush_work(a.work, cpq, cbp);
}
