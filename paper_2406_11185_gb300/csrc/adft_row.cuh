// Row-blocked J/K kernel for the larger angular-momentum classes.
//
// A group of GS lanes owns one shell quartet; lane gl owns the bra Hermite
// functions h = gl, gl + GS, ... (RPL of them, "rows") and keeps the rows of
// W[h][cd] for all ket components cd in registers.  The ket transform
//   W[h][cd] += sum_j e2_q[cd][j] R_q[h + j],   j = (tau, nu, phi),
// runs term-major: for every ket Hermite function j (compile time) the lane
// loads R_q[h + j] once per row and applies it to every ket component whose
// expansion contains j, with the lane-invariant coefficients e2_q[cd][j] read
// as VW-wide broadcast vectors.  Per primitive quartet a lane issues
// RPL * nherm(LC+LD) scalar and ~KT / VW vector shared-memory loads for
// RPL * KT FMAs (KT = ket terms of the class), against one load per FMA when
// a lane owns ket components instead.
//
// e2_q = (-1)^(tau+nu+phi) E^cd_x E^cd_y E^cd_z depends on the ket primitive
// only; when all kept ket primitives of the quartet fit in the group's SL
// slots it is built once per quartet and reused for every bra primitive (only
// R is recomputed).  The bra transform G[ab][cd] += K_p sum_h Eprod_p[ab][h]
// W[h][cd] goes through shared memory once per bra primitive, VW ket
// components per lane and step, and the digestion is the cooperative one.
#pragma once
// (included by adft_eri.cuh inside namespace adft)

// Hermite index j -> (n, m, v) with n = t+u+v, m = u+v (inverse of hidx)
__host__ __device__ constexpr int herm_n(int j) {
  int n = 0;
  while ((n + 1) * (n + 2) * (n + 3) / 6 <= j) ++n;
  return n;
}
__host__ __device__ constexpr int herm_m(int j) {
  const int r = j - herm_n(j) * (herm_n(j) + 1) * (herm_n(j) + 2) / 6;
  int m = 0;
  while ((m + 1) * (m + 2) / 2 <= r) ++m;
  return m;
}
__host__ __device__ constexpr int herm_v(int j) {
  return j - herm_n(j) * (herm_n(j) + 1) * (herm_n(j) + 2) / 6 - herm_m(j) * (herm_m(j) + 1) / 2;
}

// ket component kc of class (LC, LD) has Hermite term j in its expansion
template <int LC, int LD>
__host__ __device__ constexpr bool ket_has(int kc, int j) {
  const int ic = kc / ncart(LD), id = kc % ncart(LD);
  const int n = herm_n(j), m = herm_m(j), v = herm_v(j);
  return n - m <= cart_x(LC, ic) + cart_x(LD, id) && m - v <= cart_y(LC, ic) + cart_y(LD, id) &&
         v <= cart_z(LC, ic) + cart_z(LD, id);
}
template <int LC, int LD>
__host__ __device__ constexpr int ket_count(int j) {
  int c = 0;
  for (int kc = 0; kc < ncart(LC) * ncart(LD); ++kc) c += ket_has<LC, LD>(kc, j) ? 1 : 0;
  return c;
}
// i-th ket component containing term j (-1 past the last)
template <int LC, int LD>
__host__ __device__ constexpr int ket_col(int j, int i) {
  for (int kc = 0; kc < ncart(LC) * ncart(LD); ++kc)
    if (ket_has<LC, LD>(kc, j)) {
      if (i == 0) return kc;
      --i;
    }
  return -1;
}
// e2 layout: term-major, the entries of term j at [ket_start(j), +ket_count(j))
// padded to a multiple of VW so that every term starts on a vector boundary
template <int LC, int LD, int VW>
__host__ __device__ constexpr int ket_start(int j) {
  int s = 0;
  for (int i = 0; i < j; ++i) s += (ket_count<LC, LD>(i) + VW - 1) / VW * VW;
  return s;
}

// Runtime copies of the index tables (built by thread 0 of the block):
//   kcode[p]: E-table offsets of e2 entry p, x | y << 8 | z << 16, the sign
//             (-1)^(tau+nu+phi) in bit 24 and bit 25 set for a real entry;
//   first/h/bcode: the bra terms of bra component ab are k in
//             [first[ab], first[ab+1]), bra Hermite function h[k], E^ab
//             offsets bcode[k] (x | y << 8 | z << 16).
template <int LA, int LB, int LC, int LD, int VW>
struct RowTables {
  static constexpr int NAB = ncart(LA) * ncart(LB);
  static constexpr int BT = ket_terms<LA, LB>();
  static constexpr int KSIZE = ket_start<LC, LD, VW>(nherm(LC + LD));
  unsigned kcode[KSIZE];
  unsigned bcode[BT];
  unsigned short first[NAB + 1];
  unsigned char h[BT];
};

template <int LA, int LB, int LC, int LD, int VW>
__device__ __forceinline__ void build_row_tables(RowTables<LA, LB, LC, LD, VW>& tb) {
  constexpr int NB = ncart(LB), ND = ncart(LD), NCD = ncart(LC) * ND;
  constexpr int NTA = LA + LB + 1, NTC = LC + LD + 1;
  if (threadIdx.x == 0) {
    int p = 0;
    for (int j = 0; j < nherm(LC + LD); ++j) {
      const int n = herm_n(j), m = herm_m(j), v = herm_v(j), t = n - m, u = m - v;
      for (int kc = 0; kc < NCD; ++kc) {
        if (!ket_has<LC, LD>(kc, j)) continue;
        const int ic = kc / ND, id = kc % ND;
        const unsigned ex = (cart_x(LC, ic) * (LD + 1) + cart_x(LD, id)) * NTC + t;
        const unsigned ey = (cart_y(LC, ic) * (LD + 1) + cart_y(LD, id)) * NTC + u;
        const unsigned ez = (cart_z(LC, ic) * (LD + 1) + cart_z(LD, id)) * NTC + v;
        tb.kcode[p++] = ex | (ey << 8) | (ez << 16) | ((unsigned)(n & 1) << 24) | (1u << 25);
      }
      while (p % VW) tb.kcode[p++] = 0u;
    }
    int k = 0;
    for (int ab = 0; ab < ncart(LA) * NB; ++ab) {
      tb.first[ab] = (unsigned short)k;
      const int ia = ab / NB, ib = ab % NB;
      const int ax = cart_x(LA, ia), ay = cart_y(LA, ia), az = cart_z(LA, ia);
      const int bx = cart_x(LB, ib), by = cart_y(LB, ib), bz = cart_z(LB, ib);
      for (int t = 0; t <= ax + bx; ++t)
        for (int u = 0; u <= ay + by; ++u)
          for (int v = 0; v <= az + bz; ++v) {
            tb.h[k] = (unsigned char)hidx(t, u, v);
            tb.bcode[k++] = (unsigned)((ax * (LB + 1) + bx) * NTA + t) |
                            ((unsigned)((ay * (LB + 1) + by) * NTA + u) << 8) |
                            ((unsigned)((az * (LB + 1) + bz) * NTA + v) << 16);
          }
    }
    tb.first[ncart(LA) * NB] = (unsigned short)k;
  }
  __syncthreads();
}

// row[I] for a compile-time I, zero past the end
template <int I, int N, typename T>
__device__ __forceinline__ T row_at(const T (&row)[N]) {
  if constexpr (I < N) return row[I];
  else return T(0);
}

// VW-wide vectors of T for the broadcast e2 loads and the bra transform
template <typename T> struct RowVec;
template <> struct RowVec<float> {
  using V = float4;
  static constexpr int W = 4;
  template <int I> static __device__ __forceinline__ float get(const float4& v) {
    return I == 0 ? v.x : I == 1 ? v.y : I == 2 ? v.z : v.w;
  }
  static __device__ __forceinline__ void fma(float4& acc, float e, const float4& w) {
    acc.x += e * w.x; acc.y += e * w.y; acc.z += e * w.z; acc.w += e * w.w;
  }
  static __device__ __forceinline__ void add(float4& a, const float4& b) {
    a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
  }
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  // row[C0 .. C0 + 4), zero past N
  template <int C0, int N> static __device__ __forceinline__ float4 pack(const float (&row)[N]) {
    return make_float4(row_at<C0, N>(row), row_at<C0 + 1, N>(row), row_at<C0 + 2, N>(row), row_at<C0 + 3, N>(row));
  }
};
template <> struct RowVec<double> {
  using V = double2;
  static constexpr int W = 2;
  template <int I> static __device__ __forceinline__ double get(const double2& v) { return I == 0 ? v.x : v.y; }
  static __device__ __forceinline__ void fma(double2& acc, double e, const double2& w) {
    acc.x += e * w.x; acc.y += e * w.y;
  }
  static __device__ __forceinline__ void add(double2& a, const double2& b) { a.x += b.x; a.y += b.y; }
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  template <int C0, int N> static __device__ __forceinline__ double2 pack(const double (&row)[N]) {
    return make_double2(row_at<C0, N>(row), row_at<C0 + 1, N>(row));
  }
};

// Group shape: GS lanes per quartet, RPL = ceil(NHAB / GS) rows per lane,
// under a register cap RPL * row_regs <= cap, row_regs = the 32-bit registers
// of one row (its W values and its 2 (LC+LD+1) R offsets).  The shape
// maximises the busy fraction (lanes in whole groups / 32) * NHAB / (GS RPL);
// between equally busy shapes the one with more rows per lane (more reuse of
// every e2 vector) wins.
struct RowShape {
  int gs, rpl;
};
__host__ __device__ constexpr RowShape row_shape(int nhab, int row_regs, int cap) {
  RowShape best{32, (nhab + 31) / 32};
  double best_u = -1.0;
  for (int gs = 1; gs <= 32; ++gs) {
    const int rpl = (nhab + gs - 1) / gs;
    if (rpl * row_regs > cap) continue;
    const double u = (double)((32 / gs) * gs) / 32.0 * (double)nhab / (double)(gs * rpl);
    if (u > best_u + 1e-9 || (u > best_u - 1e-9 && rpl > best.rpl)) {
      best_u = u;
      best = RowShape{gs, rpl};
    }
  }
  return best;
}
__host__ __device__ constexpr int row_pad(int x, int vw) { return (x + vw - 1) / vw * vw; }
// values of one group: e2 [SL][KSIZE], W / ket E [max(NHAB NCDP, SL 3 EC)],
// G [NAB][NCDP], R [SL][NH], bra E [3][EA], Eprod [BT] (each vector aligned)
__host__ __device__ constexpr int row_we(int sl, int nhab, int ncdp, int ec, int vw) {
  return nhab * ncdp > sl * 3 * ec ? nhab * ncdp : row_pad(sl * 3 * ec, vw);
}
__host__ __device__ constexpr int row_group(int sl, int ksize, int nhab, int ncdp, int ec, int nab, int nh, int ea,
                                            int bt, int vw) {
  return sl * ksize + row_we(sl, nhab, ncdp, ec, vw) + nab * ncdp + row_pad(sl * nh, vw) + row_pad(3 * ea, vw) +
         row_pad(bt, vw);
}
// slots per group: the largest of min(GS, 8), 4, 2, 1 that leaves room for
// at least 4 warps per block
__host__ __device__ constexpr int row_slots(int gs, int ksize, int nhab, int ncdp, int ec, int nab, int nh, int ea,
                                            int bt, int vw, int tsize) {
  int sl = gs < COOP_SLOT_CAP ? gs : COOP_SLOT_CAP;
  for (; sl > 1; sl = (sl > 4 ? 4 : sl / 2))
    if (COOP_SMEM_BUDGET / ((32 / gs) * row_group(sl, ksize, nhab, ncdp, ec, nab, nh, ea, bt, vw) * tsize) >= 4)
      return sl;
  return 1;
}

// Occupancy-aware shape (policy 1): the d-class kernels are latency-bound at
// a few warps per SM, so this policy scores a shape by busy fraction x the
// warps per SM that its shared memory (228 KB per SM, the slots taken as
// large as 4 resident warps allow) and an estimate of its registers (rows +
// 120 per thread) let reside, up to 8.
struct RowShape3 {
  int gs, rpl, sl;
};
__host__ __device__ constexpr RowShape3 row_shape_occ(int nhab, int row_regs, int cap, int ksize, int ncdp, int ec,
                                                      int nab, int nh, int ea, int bt, int vw, int tsize) {
  RowShape3 best{32, (nhab + 31) / 32, 1};
  double best_s = -1.0;
  for (int gs = 1; gs <= 32; ++gs) {
    const int rpl = (nhab + gs - 1) / gs;
    if (rpl * row_regs > cap) continue;
    const int ngw = 32 / gs;
    const double u = (double)(ngw * gs) / 32.0 * (double)nhab / (double)(gs * rpl);
    const int opts[4] = {COOP_SLOT_CAP, 4, 2, 1};
    int sl = 1, wsm = 0;
    for (int i = 0; i < 4; ++i) {
      if (opts[i] > gs) continue;
      sl = opts[i];
      wsm = (228 * 1024) / (ngw * row_group(sl, ksize, nhab, ncdp, ec, nab, nh, ea, bt, vw) * tsize);
      if (wsm >= 4) break;
    }
    const int regs = rpl * row_regs + 120 > 255 ? 255 : rpl * row_regs + 120;
    const int wreg = 65536 / (32 * regs);
    int occ = wsm < wreg ? wsm : wreg;
    if (occ > 8) occ = 8;
    const double score = u * (double)occ;
    if (score > best_s + 1e-9 || (score > best_s - 1e-9 && rpl > best.rpl)) {
      best_s = score;
      best = RowShape3{gs, rpl, sl};
    }
  }
  return best;
}

// POLICY 0: the busiest shape (row_shape, row_slots); POLICY 1: the
// occupancy-aware one (row_shape_occ).  A policy-1 plan that equals the
// policy-0 plan does not fit, so no kernel is compiled twice.
template <typename T, int LA, int LB, int LC, int LD, int POLICY = 0>
struct RowPlan {
  static constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  static constexpr int NAB = NA * NB, NCD = NC * ND;
  static constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  static constexpr int NHAB = nherm(LAB), NHCD = nherm(LCD), NH = nherm(L);
  static constexpr int EA = (LA + 1) * (LB + 1) * (LAB + 1), EC = (LC + 1) * (LD + 1) * (LCD + 1);
  static constexpr int BT = ket_terms<LA, LB>();
  static constexpr int VW = RowVec<T>::W;
  static constexpr int KSIZE = ket_start<LC, LD, VW>(NHCD);
  static constexpr int NCDP = (NCD + VW - 1) / VW * VW;
  static constexpr int ROW_REGS = NCD * (int)(sizeof(T) / 4) + 2 * (LCD + 1);
  static constexpr int REG_CAP = 104;  // registers of the rows of one lane
  static constexpr RowShape SHAPE0 = row_shape(NHAB, ROW_REGS, REG_CAP);
  static constexpr int SL0 = row_slots(SHAPE0.gs, KSIZE, NHAB, NCDP, EC, NAB, NH, EA, BT, VW, (int)sizeof(T));
  static constexpr RowShape3 SHAPE1 =
      row_shape_occ(NHAB, ROW_REGS, REG_CAP, KSIZE, NCDP, EC, NAB, NH, EA, BT, VW, (int)sizeof(T));
  static constexpr int GS = POLICY == 0 ? SHAPE0.gs : SHAPE1.gs;
  static constexpr int RPL = POLICY == 0 ? SHAPE0.rpl : SHAPE1.rpl;
  static constexpr int SL = POLICY == 0 ? SL0 : SHAPE1.sl;
  static constexpr int NGW = 32 / GS;
  static constexpr int WE = row_we(SL, NHAB, NCDP, EC, VW);
  static constexpr int RSZ = row_pad(SL * NH, VW), EASZ = row_pad(3 * EA, VW);
  static constexpr int GROUP = row_group(SL, KSIZE, NHAB, NCDP, EC, NAB, NH, EA, BT, VW);
  static constexpr int WARP_BYTES = NGW * GROUP * (int)sizeof(T);
  static constexpr int WFIT = COOP_SMEM_BUDGET / WARP_BYTES;
  static constexpr int WARPS = WFIT > COOP_MAX_WARPS ? COOP_MAX_WARPS : WFIT;
  static constexpr int SMEM = WARPS * WARP_BYTES;
  static constexpr bool distinct =
      POLICY == 0 || !(SHAPE1.gs == SHAPE0.gs && SHAPE1.rpl == SHAPE0.rpl && SHAPE1.sl == SL0);
  // the classes of the cooperative kernel (up to d shells) with at least two
  // warps per block and rows within the register cap
  static constexpr bool fits = WARPS >= 2 && RPL * ROW_REGS <= REG_CAP && LA <= 2 && LC <= 2 && distinct;
};

template <typename T, int LA, int LB, int LC, int LD, int POLICY>
__global__ void __launch_bounds__(32 * COOP_MAX_WARPS, 1) k_jk_row(JKLaunch a) {
  using P = RowPlan<T, LA, LB, LC, LD, POLICY>;
  using RV = RowVec<T>;
  using V = typename RV::V;
  constexpr int NAB = P::NAB, NCD = P::NCD, NCDP = P::NCDP, NHAB = P::NHAB, NHCD = P::NHCD, NH = P::NH;
  constexpr int EA = P::EA, EC = P::EC, BT = P::BT, VW = P::VW, KSIZE = P::KSIZE;
  constexpr int GS = P::GS, RPL = P::RPL, SL = P::SL, LCD = P::LCD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RowTables<LA, LB, LC, LD, VW> tb;
  // zero the staging memory once: padded slots (see below) then only ever
  // hold finite values
  for (int i = threadIdx.x; i < P::WARPS * P::WARP_BYTES / 16; i += blockDim.x)
    reinterpret_cast<uint4*>(smem_raw)[i] = make_uint4(0u, 0u, 0u, 0u);
  build_row_tables<LA, LB, LC, LD, VW>(tb);  // ends with __syncthreads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane / GS, gl = lane - g * GS;
  const bool in_group = g < P::NGW;
  T* e2g = reinterpret_cast<T*>(smem_raw) + (size_t)(warp * P::NGW + (in_group ? g : 0)) * P::GROUP;
  T* WE = e2g + SL * KSIZE;   // W rows [NHAB][NCDP]; ket E tables [SL][3 EC] while e2 is built
  T* Gs = WE + P::WE;         // contracted block [NAB][NCDP]
  T* Rg = Gs + NAB * NCDP;    // R of the staged ket primitives [SL][NH]
  T* Eab = Rg + P::RSZ;       // bra E of the current bra primitive [3][EA]
  T* Eprod = Eab + P::EASZ;   // K_p E^ab_x E^ab_y E^ab_z [BT]
  const long long total = (long long)__ldg(a.prefix + a.nseg);
  const BasisView& bv = a.bv;
  const PrimPair<T>* __restrict__ pp = Prec<T>::pp(bv);
  const T* __restrict__ o2pa = Prec<T>::o2p(bv);
  const float* __restrict__ qa = bv.pp_q32;
  const float eps = (float)a.prim_eps;
  unsigned cpq = 0, cbp = 0;  // evaluated work (group leaders)

  // this lane's rows h = gl + GS i: R(t+tau, u+nu, v+phi) sits at
  // T3(n + sigma) + T2(m + mu) + v + phi (n = t+u+v, m = u+v,
  // sigma = tau+nu+phi, mu = nu+phi); rows past NHAB use h = 0 (in bounds,
  // never stored)
  int t3[RPL][LCD + 1], t2[RPL][LCD + 1];
#pragma unroll
  for (int i = 0; i < RPL; ++i) {
    const int h = gl + GS * i;
    int n = 0, m = 0, v = 0;
    if (h < NHAB) {
      n = herm_n(h);
      m = herm_m(h);
      v = herm_v(h);
    }
#pragma unroll
    for (int s = 0; s <= LCD; ++s) {
      t3[i][s] = (n + s) * (n + s + 1) * (n + s + 2) / 6;
      t2[i][s] = (m + s) * (m + s + 1) / 2 + v;
    }
  }

  // Every lane of a warp runs the same trip counts (the warp maxima), so the
  // groups of a warp stay converged and every phase ends in a full-warp
  // __syncwarp.  A group with less work (or none: lanes outside every group,
  // or a group past the end of the work list) runs padded steps that write
  // nothing and add zeros: its extra R slots are zeroed, and every slot holds
  // finite values from the start.
  constexpr unsigned FULL = 0xffffffffu;
  for (;;) {
    unsigned long long base = 0;
    int stop = 0;
    if (lane == 0) {
      base = atomicAdd(a.counter, (unsigned long long)P::NGW);
      stop = *(volatile const int*)a.abort_flag;
    }
    base = __shfl_sync(FULL, base, 0);
    stop = __shfl_sync(FULL, stop, 0);
    if ((long long)base >= total) break;
    if (stop) {
      if (lane == 0) atomicCAS(a.status, 0, ADFT_ERR_ABORTED);
      break;
    }
    const long long qi = (long long)base + g;
    const bool valid = in_group && qi < total;
    int bra = 0, ket = 0, off0 = 0, n0 = 0, off1 = 0, n1 = 0;
    T AB[3] = {T(0), T(0), T(0)};
    T CDx = T(0), CDy = T(0), CDz = T(0);
    if (valid) {
      decode_quartet(a, qi, bra, ket);
      off0 = __ldg(bv.pair_pp_off + bra);
      n0 = __ldg(bv.pair_pp_n + bra);
      off1 = __ldg(bv.pair_pp_off + ket);
      n1 = __ldg(bv.pair_pp_n + ket);
      AB[0] = from_f64<T>(__ldg(bv.pair_AB + 3 * bra));
      AB[1] = from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 1));
      AB[2] = from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 2));
      CDx = from_f64<T>(__ldg(bv.pair_AB + 3 * ket));
      CDy = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 1));
      CDz = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 2));
      for (int x = gl; x < NAB * NCDP; x += GS) Gs[x] = T(0);
    }
    const int n0max = __reduce_max_sync(FULL, n0);
    // all kept ket primitives in one batch: their e2 is built once and kept
    const bool keep_e2 = n1 <= SL;
    bool have_e2 = false;

    int n1e = n1;
    for (int ip = 0; ip < n0max; ++ip) {
      n1e = ip < n0 ? shrink_kept(qa + off1, __ldg(qa + off0 + ip), eps, n1e) : 0;  // same in a group
      if (__all_sync(FULL, n1e == 0)) break;
      const bool act = n1e > 0;  // this group evaluates bra primitive ip
      if (gl == 0 && act) { cpq += n1e; ++cbp; }
      PrimPair<T> bp = {};
      T o2p = T(0);
      if (act) {
        bp = pp[off0 + ip];
        o2p = __ldg(o2pa + off0 + ip);
        for (int d = gl; d < 3; d += GS) {  // groups may have fewer than 3 lanes
          const T PA = d == 0 ? bp.PAx : d == 1 ? bp.PAy : bp.PAz;
          const T ABd = d == 0 ? AB[0] : d == 1 ? AB[1] : AB[2];  // (no dynamic register index)
          hermite_E<T, LA, LB>(PA, PA + ABd, o2p, Eab + d * EA);
        }
      }
      T W[RPL][NCD];
#pragma unroll
      for (int i = 0; i < RPL; ++i)
#pragma unroll
        for (int c = 0; c < NCD; ++c) W[i][c] = T(0);
      __syncwarp();
      if (act)
        for (int k = gl; k < BT; k += GS) {
          const unsigned c = tb.bcode[k];
          Eprod[k] = bp.K * Eab[c & 255u] * Eab[EA + ((c >> 8) & 255u)] * Eab[2 * EA + (c >> 16)];
        }
      const int nbmax = __reduce_max_sync(FULL, n1e);
      for (int q0 = 0; q0 < nbmax; q0 += SL) {
        const int nvmax = min(SL, nbmax - q0);          // warp-uniform slot count
        const int nv = max(0, min(SL, n1e - q0));       // this group's slots
        const bool build = act && !have_e2;
        if (in_group && gl < nvmax) {
          T* Rs = Rg + gl * NH;
          if (gl < nv) {
            const int iq = off1 + q0 + gl;
            const PrimPair<T> kq = pp[iq];
            const T o2q = __ldg(o2pa + iq);
            if (build) {
              T* Ec = WE + gl * 3 * EC;
              hermite_E<T, LC, LD>(kq.PAx, kq.PAx + CDx, o2q, Ec);
              hermite_E<T, LC, LD>(kq.PAy, kq.PAy + CDy, o2q, Ec + EC);
              hermite_E<T, LC, LD>(kq.PAz, kq.PAz + CDz, o2q, Ec + 2 * EC);
            }
            const T r = Prec<T>::rsq(bp.p + kq.p);
            T alpha = bp.p * kq.p * r * r;
            T pref = cst<T>(4.0 * 34.98683665524972) * kq.K * r * o2p * o2q;
            attenuate((T)a.omega2, alpha, pref);
            prim_R_scaled<T, P::L>(alpha, bp.Px - kq.Px, bp.Py - kq.Py, bp.Pz - kq.Pz, pref, bv, Rs);
          } else {
            for (int x = 0; x < NH; ++x) Rs[x] = T(0);  // padded slot: adds zero
          }
        }
        __syncwarp();
        if (build) {
          for (int e = gl; e < nv * KSIZE; e += GS) {
            const int s = e / KSIZE;
            const unsigned c = tb.kcode[e - s * KSIZE];
            const T* Ec = WE + s * 3 * EC;
            T val = T(0);
            if (c >> 25) {
              val = Ec[c & 255u] * Ec[EC + ((c >> 8) & 255u)] * Ec[2 * EC + ((c >> 16) & 255u)];
              if ((c >> 24) & 1u) val = -val;
            }
            e2g[e] = val;
          }
          have_e2 = keep_e2;
        }
        __syncwarp();
        // ket transform, term-major (see the top of the file)
        for (int s = 0; s < nvmax; ++s) {
          const T* Rs = Rg + s * NH;
          const T* es = e2g + s * KSIZE;
          static_for<NHCD>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            constexpr int sg = herm_n(j), mu = herm_m(j), phi = herm_v(j);
            constexpr int p0 = ket_start<LC, LD, VW>(j);
            constexpr int nvec = (ket_count<LC, LD>(j) + VW - 1) / VW;
            T r[RPL];
#pragma unroll
            for (int i = 0; i < RPL; ++i) r[i] = Rs[t3[i][sg] + t2[i][mu] + phi];
            static_for<nvec>([&](auto bb) {
              constexpr int b = decltype(bb)::value;
              const V ev = *reinterpret_cast<const V*>(es + p0 + b * VW);
              static_for<VW>([&](auto ww) {
                constexpr int w = decltype(ww)::value;
                constexpr int kc = ket_col<LC, LD>(j, b * VW + w);
                if constexpr (kc >= 0) {
                  const T e = RV::template get<w>(ev);
#pragma unroll
                  for (int i = 0; i < RPL; ++i) W[i][kc] += e * r[i];
                }
              });
            });
          });
        }
        __syncwarp();
      }
      // W rows to shared memory (padding columns zero), then the bra
      // transform: lane unit (ab, VW ket components)
      if (act) {
#pragma unroll
        for (int i = 0; i < RPL; ++i) {
          const int h = gl + GS * i;
          if (h < NHAB) {
            static_for<NCDP / VW>([&](auto cc) {
              constexpr int c0 = decltype(cc)::value * VW;
              *reinterpret_cast<V*>(WE + h * NCDP + c0) = RV::template pack<c0, NCD>(W[i]);
            });
          }
        }
      }
      __syncwarp();
      if (act) {
        constexpr int NV = NCDP / VW;
        for (int u = gl; u < NAB * NV; u += GS) {
          const int ab = u / NV, c0 = (u - ab * NV) * VW;
          V acc = RV::zero();
          const int k1 = tb.first[ab + 1];
          for (int k = tb.first[ab]; k < k1; ++k)
            RV::fma(acc, Eprod[k], *reinterpret_cast<const V*>(WE + tb.h[k] * NCDP + c0));
          V* gp = reinterpret_cast<V*>(Gs + ab * NCDP + c0);
          V gv = *gp;
          RV::add(gv, acc);
          *gp = gv;
        }
      }
      __syncwarp();
    }
    if (valid) digest_coop<T, LA, LB, LC, LD, NCDP>(a, bra, ket, gl, GS, Gs);
    __syncwarp();
  }
  flush_work(a.work, cpq, cbp);
}
