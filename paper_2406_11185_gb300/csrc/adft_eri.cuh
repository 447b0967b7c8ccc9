// Device templates of the per-class ERI kernels (McMurchie-Davidson) with the
// J/K digestion fused in.  Included by the per-precision translation units,
// which instantiate one kernel per angular-momentum class pair
// (la lb | lc ld), la >= lb, lc >= ld, (la,lb) >= (lc,ld).  Sec. 1.2.2 gives
// every angular-momentum combination its own generated code path, since their
// recurrence graphs differ; here the C++ compiler generates those paths from
// one template instead of a separate code generator.
//
// Integral scheme (Helgaker, Jorgensen, Olsen, "Molecular Electronic-Structure
// Theory", Sec. 9.5 and 9.9): for primitive pairs p (bra) and q (ket)
//   [ab|cd] = 2 pi^(5/2) / (p q sqrt(p+q)) K_p K_q
//             sum_{tuv} E^ab_tuv sum_{tau nu phi} (-1)^(tau+nu+phi)
//             E^cd_{tau nu phi} R_{t+tau, u+nu, v+phi}(alpha, P-Q)
// evaluated as W_p[tuv][cd] = sum_q (ket transform) followed by one bra
// transform per bra primitive, so the bra transform is amortised over the ket
// primitives.  A thread owns one shell quartet and a chunk of CK ket
// Cartesian components (all bra components), which bounds its state.
#pragma once
#include <type_traits>
#include <utility>

#include "adft_internal.cuh"

namespace adft {

// ---------------------------------------------------------------------------
// small index helpers (all constexpr so that unrolled loops fold them)

// Cartesian component k of a shell of angular momentum l -> powers (x, y, z),
// ordered by descending x, then descending y.
__host__ __device__ constexpr int cart_x(int l, int k) {
  int i = l, off = 0;
  while (k >= off + (l - i + 1)) { off += l - i + 1; --i; }
  return i;
}
__host__ __device__ constexpr int cart_z(int l, int k) {
  int i = l, off = 0;
  while (k >= off + (l - i + 1)) { off += l - i + 1; --i; }
  return k - off;
}
__host__ __device__ constexpr int cart_y(int l, int k) { return l - cart_x(l, k) - cart_z(l, k); }
__host__ __device__ constexpr int cart_pow(int l, int k, int d) {
  return d == 0 ? cart_x(l, k) : d == 1 ? cart_y(l, k) : cart_z(l, k);
}

// Hermite index (t, u, v), t + u + v <= L, ordered by n = t+u+v, then by
// m = u+v, then by v: position = n(n+1)(n+2)/6 + m(m+1)/2 + v.
__host__ __device__ constexpr int hidx(int t, int u, int v) {
  return (t + u + v) * (t + u + v + 1) * (t + u + v + 2) / 6 + (u + v) * (u + v + 1) / 2 + v;
}

template <typename T> __device__ __forceinline__ T dload(const T* p) { return __ldg(p); }

// constants and matrices of the three arithmetic types (double, float,
// double-float)
template <typename T> __device__ __forceinline__ constexpr T cst(double x) { return T(x); }
template <typename T> __device__ __forceinline__ const T* dmat(const JKLaunch& a);
template <> __device__ __forceinline__ const double* dmat<double>(const JKLaunch& a) { return a.D64; }
template <> __device__ __forceinline__ const float* dmat<float>(const JKLaunch& a) { return a.D32; }
template <typename T> __device__ __forceinline__ T from_f64(double x) { return (T)x; }
template <typename T> constexpr bool is_f64 = std::is_same<T, double>::value;
template <typename T> constexpr bool is_f32 = std::is_same<T, float>::value;


template <typename T> struct Prec;
template <> struct Prec<double> {
  static __device__ __forceinline__ const PrimPair<double>* pp(const BasisView& b) { return b.pp64; }
  static __device__ __forceinline__ const double* o2p(const BasisView& b) { return b.pp_o2p64; }
  static __device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
  static constexpr int BUDGET = 640;
};
template <> struct Prec<float> {
  static __device__ __forceinline__ const PrimPair<float>* pp(const BasisView& b) { return b.pp32; }
  static __device__ __forceinline__ const float* o2p(const BasisView& b) { return b.pp_o2p32; }
  static __device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
  static constexpr int BUDGET = 640;
};

// Long-range operator erf(omega r)/r (range-separated hybrids, the omegaB97X
// functional of Sec. 4.1).  Its Fourier transform is that of 1/r times
// exp(-k^2 / (4 w2)), w2 = omega^2, so a primitive quartet's integral is the
// Coulomb one with 1/alpha -> 1/alpha + 1/w2: alpha -> alpha w2 / (alpha + w2)
// in the Boys argument and in the Hermite recursion, and the prefactor times
// sqrt(w2 / (alpha + w2)).  w2 = 0 leaves both untouched (the 1/r operator).
template <typename T>
__device__ __forceinline__ void attenuate(T w2, T& alpha, T& pref) {
  if (w2 > T(0)) {
    const T s = w2 / (alpha + w2);
    alpha *= s;
    pref *= sqrt(s);
  }
}

// Primitive-quartet screening inside a kept shell quartet: the primitive
// pairs of a pair are stored by descending bound Q_p, so the ket primitives q
// kept for bra primitive p (Q_p Q_q >= eps) are a prefix of the ket's list,
// and its length n can only shrink from one bra primitive to the next.
// shrink_kept(qk, qp, eps, n) shortens n for bra primitive bound qp (FP32
// compares: a bound test needs no more); over all bra primitives of a
// quartet it reads at most n0 + n1 bounds.  Once n is 0 it stays 0.
__device__ __forceinline__ int shrink_kept(const float* __restrict__ qk, float qp, float eps, int n) {
  while (n > 0 && qp * __ldg(qk + n - 1) < eps) --n;
  return n;
}

// Warp-sum of the evaluated-work counters of the calling lanes, added once per
// warp into work[0] (primitive quartets) and work[1] (bra primitives).  All
// 32 lanes must call it.  (A lane's own counts stay far below 2^32: a launch
// evaluates at most a few 1e10 primitive quartets over >= 1e4 lanes.)
__device__ __forceinline__ void flush_work(unsigned long long* work, unsigned pq, unsigned bp) {
  unsigned long long p = pq, b = bp;
  for (int o = 16; o > 0; o >>= 1) {
    p += __shfl_down_sync(0xffffffffu, p, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if (work && (threadIdx.x & 31) == 0 && (p | b)) {
    atomicAdd(work, p);
    atomicAdd(work + 1, b);
  }
}

// reciprocals 1/(2m+1), m < 32
__constant__ static const double c_inv_odd64[32] = {
    1.0 / 1, 1.0 / 3, 1.0 / 5, 1.0 / 7, 1.0 / 9, 1.0 / 11, 1.0 / 13, 1.0 / 15, 1.0 / 17, 1.0 / 19, 1.0 / 21,
    1.0 / 23, 1.0 / 25, 1.0 / 27, 1.0 / 29, 1.0 / 31, 1.0 / 33, 1.0 / 35, 1.0 / 37, 1.0 / 39, 1.0 / 41,
    1.0 / 43, 1.0 / 45, 1.0 / 47, 1.0 / 49, 1.0 / 51, 1.0 / 53, 1.0 / 55, 1.0 / 57, 1.0 / 59, 1.0 / 61, 1.0 / 63};
__constant__ static const float c_inv_odd32[32] = {
    1.f / 1, 1.f / 3, 1.f / 5, 1.f / 7, 1.f / 9, 1.f / 11, 1.f / 13, 1.f / 15, 1.f / 17, 1.f / 19, 1.f / 21,
    1.f / 23, 1.f / 25, 1.f / 27, 1.f / 29, 1.f / 31, 1.f / 33, 1.f / 35, 1.f / 37, 1.f / 39, 1.f / 41,
    1.f / 43, 1.f / 45, 1.f / 47, 1.f / 49, 1.f / 51, 1.f / 53, 1.f / 55, 1.f / 57, 1.f / 59, 1.f / 61, 1.f / 63};

// ---------------------------------------------------------------------------
// Boys function F_m(T) = int_0^1 t^2m exp(-T t^2) dt  (Helgaker Sec. 9.8.1).
// FP64: 7-term Taylor expansion of F_L about the nearest tabulated point
// (spacing 0.1, table built by the library's own series code), then downward
// recursion F_m = (2T F_{m+1} + e^-T)/(2m+1); for T >= 60 the closed form
// F_0 = sqrt(pi/T)/2 (erf(sqrt T) = 1 to double precision) and upward
// recursion F_{m+1} = ((2m+1) F_m - e^-T)/(2T).
template <int L>
__device__ __forceinline__ void boys_fp64(double T, const double* __restrict__ tab, double* F) {
  if (T < BOYS_TMAX) {
    const int i = __double2int_rn(T * (1.0 / BOYS_H));
    const double y = i * BOYS_H - T;
    const double* row = tab + i * (BOYS_MMAX + 1) + L;
    double acc = __ldg(row + 6);
#pragma unroll
    for (int k = 6; k >= 1; --k) acc = __ldg(row + k - 1) + acc * (y * (1.0 / k));
    const double e = exp(-T);
    F[L] = acc;
#pragma unroll
    for (int m = L - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) * (1.0 / (2 * m + 1));
  } else {
    // T >= 60: F_0 = sqrt(pi/T)/2 and F_{m+1} = (2m+1) F_m / (2T); the
    // neglected e^-T terms are below 1e-13 of F_m for m <= 13.
    const double rt = rsqrt(T);
    const double h = 0.5 * rt * rt;
    F[0] = 0.88622692545275801365 * rt;
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = (2 * m + 1) * F[m] * h;
  }
}

// FP32, scaled: G_m = c^m F_m(T) with c = max(1, 2T), so that G_m stays in
// range for any T (the caller rescales the Hermite integrals accordingly).
// 5-term Taylor expansion below T = 60; above, the asymptotic recursion
// G_{m+1} = (2m+1) G_m whose neglected e^-T term is below 1e-10 relative.
template <int L>
__device__ __forceinline__ void boys_fp32_scaled(float T, const float* __restrict__ tab, float* G) {
  if (T < (float)BOYS_TMAX) {
    const int i = __float2int_rn(T * (float)(1.0 / BOYS_H));
    const float y = i * (float)BOYS_H - T;
    const float* row = tab + i * (BOYS_MMAX + 1) + L;
    float acc = __ldg(row + 4);
#pragma unroll
    for (int k = 4; k >= 1; --k) acc = __ldg(row + k - 1) + acc * (y * (1.0f / k));
    const float e = __expf(-T);
    float F[L + 1];
    F[L] = acc;
#pragma unroll
    for (int m = L - 1; m >= 0; --m) F[m] = (2.0f * T * F[m + 1] + e) * (1.0f / (2 * m + 1));
    const float c = fmaxf(1.0f, 2.0f * T);
    float cn = 1.0f;
#pragma unroll
    for (int m = 0; m <= L; ++m) { G[m] = F[m] * cn; cn *= c; }
  } else {
    G[0] = 0.88622692545f * rsqrtf(T);
#pragma unroll
    for (int m = 0; m < L; ++m) G[m + 1] = (2 * m + 1) * G[m];
  }
}

// ---------------------------------------------------------------------------
// Hermite expansion coefficients of one direction (Helgaker eqs. 9.5.6-9.5.7),
// without the exp(-mu X_AB^2) factor (it lives in the pair prefactor K):
// E[(i*(LB+1)+j)*(LA+LB+1)+t], i <= LA, j <= LB, t <= i+j.
template <typename T, int LA, int LB>
__device__ __forceinline__ void hermite_E(T PA, T PB, T o2p, T* E) {
  constexpr int NT = LA + LB + 1;
#pragma unroll
  for (int x = 0; x < (LA + 1) * (LB + 1) * NT; ++x) E[x] = T(0);
  E[0] = T(1);
#pragma unroll
  for (int i = 1; i <= LA; ++i)
#pragma unroll
    for (int t = 0; t <= i; ++t) {
      T v = PA * ((t <= i - 1) ? E[((i - 1) * (LB + 1)) * NT + t] : T(0));
      if (t > 0) v += o2p * E[((i - 1) * (LB + 1)) * NT + t - 1];
      if (t + 1 <= i - 1) v += T(t + 1) * E[((i - 1) * (LB + 1)) * NT + t + 1];
      E[(i * (LB + 1)) * NT + t] = v;
    }
#pragma unroll
  for (int i = 0; i <= LA; ++i)
#pragma unroll
    for (int j = 1; j <= LB; ++j)
#pragma unroll
      for (int t = 0; t <= i + j; ++t) {
        const int src = (i * (LB + 1) + j - 1) * NT;
        T v = PB * ((t <= i + j - 1) ? E[src + t] : T(0));
        if (t > 0) v += o2p * E[src + t - 1];
        if (t + 1 <= i + j - 1) v += T(t + 1) * E[src + t + 1];
        E[(i * (LB + 1) + j) * NT + t] = v;
      }
}

// Hermite Coulomb integrals R_tuv, t+u+v <= L (Helgaker eqs. 9.9.18-9.9.20),
// from the base values B_n = R^n_000, raised in t, u or v from layer n+1, in
// place: layer n overwrites layer n+1, and inside a layer the entries are
// produced by decreasing t+u+v, so an entry is overwritten only after every
// entry of the new layer that reads it has been computed.
template <typename T, int L>
__device__ __forceinline__ void hermite_R(const T* B, T X, T Y, T Z, T* R) {
#pragma unroll
  for (int n = L; n >= 0; --n)
#pragma unroll
    for (int s = L - n; s >= 0; --s)
#pragma unroll
      for (int t = s; t >= 0; --t)
#pragma unroll
        for (int u = s - t; u >= 0; --u) {
          const int v = s - t - u;
          T val;
          if (s == 0) {
            val = B[n];
          } else if (t > 0) {
            val = X * R[hidx(t - 1, u, v)];
            if (t > 1) val += T(t - 1) * R[hidx(t - 2, u, v)];
          } else if (u > 0) {
            val = Y * R[hidx(t, u - 1, v)];
            if (u > 1) val += T(u - 1) * R[hidx(t, u - 2, v)];
          } else {
            val = Z * R[hidx(t, u, v - 1)];
            if (v > 1) val += T(v - 1) * R[hidx(t, u, v - 2)];
          }
          R[hidx(t, u, v)] = val;
        }
}

// Base values R^n_000 and the Hermite integrals of one primitive quartet.
// FP64: B_n = (-2 alpha)^n F_n(T), R as defined.
// FP32: with c = max(1, 2T), s^2 = 2 alpha / c: B_n = (-c)^n F_n c^0... i.e.
// B_n = (-1)^n G_n, coordinates scaled by s, and R_tuv = s^(t+u+v) Rs_tuv,
// which keeps every intermediate in single-precision range.
template <typename T, int L>
__device__ __forceinline__ void prim_R(T alpha, T X, T Y, T Z, const BasisView& bv, T* R) {
  T B[L + 1];
  const T Tb = alpha * (X * X + Y * Y + Z * Z);
  if constexpr (is_f64<T>) {
    boys_fp64<L>(Tb, bv.boys64, B);
    T f = -2.0 * alpha, pw = f;
#pragma unroll
    for (int n = 1; n <= L; ++n) { B[n] *= pw; pw *= f; }
    hermite_R<T, L>(B, X, Y, Z, R);
  } else {
    boys_fp32_scaled<L>(Tb, bv.boys32, B);
#pragma unroll
    for (int n = 1; n <= L; n += 2) B[n] = -B[n];
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

// ---------------------------------------------------------------------------
// Compile-time loop: f(std::integral_constant<int, i>{}) for i = 0 .. N-1.
// Component indices handed out this way are constants, so every loop bound
// and array index derived from them folds at compile time and the thread's
// arrays stay in registers.
template <typename F, int... I>
__device__ __forceinline__ void static_for_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_seq(f, std::make_integer_sequence<int, N>{});
}

// Contracted Cartesian block of one shell quartet for the ket components
// [C0, C0 + NK) in one thread, G[ab*NK + k] = (ab|cd)_{C0+k}, with every
// intermediate in registers.  Primitive quartets with Q_p Q_q < eps are
// skipped; npq and nbp are increased by the primitive quartets and bra
// primitives evaluated.
template <typename T, int LA, int LB, int LC, int LD, int C0, int NK>
__device__ __forceinline__ void quartet_block_range(const BasisView& bv, int bra, int ket, T* G, T eps, int& npq,
                                                    int& nbp, T w2) {
  constexpr int NB = ncart(LB), ND = ncart(LD);
  constexpr int NAB = ncart(LA) * NB, NCD = ncart(LC) * ND;
  constexpr int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  constexpr int NHAB = nherm(LAB);
  constexpr int EA = (LA + 1) * (LB + 1) * (LAB + 1), EC = (LC + 1) * (LD + 1) * (LCD + 1);
  constexpr int NTA = LAB + 1, NTC = LCD + 1;
  const PrimPair<T>* __restrict__ pp = Prec<T>::pp(bv);

  const int off0 = __ldg(bv.pair_pp_off + bra), n0 = __ldg(bv.pair_pp_n + bra);
  const int off1 = __ldg(bv.pair_pp_off + ket), n1 = __ldg(bv.pair_pp_n + ket);
  const T ABx = from_f64<T>(__ldg(bv.pair_AB + 3 * bra)), ABy = from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 1)),
          ABz = from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 2));
  const T CDx = from_f64<T>(__ldg(bv.pair_AB + 3 * ket)), CDy = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 1)),
          CDz = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 2));

  static_assert(C0 >= 0 && NK >= 1 && C0 + NK <= NCD, "component range");
#pragma unroll
  for (int x = 0; x < NAB * NK; ++x) G[x] = T(0);

  const float* __restrict__ qa = bv.pp_q32;
  const float epsf = (float)eps;
  int n1e = n1;
  for (int ip = 0; ip < n0; ++ip) {
    n1e = shrink_kept(qa + off1, __ldg(qa + off0 + ip), epsf, n1e);
    if (n1e == 0) break;
    npq += n1e;
    ++nbp;
    const PrimPair<T> bp = pp[off0 + ip];
    const T o2p = __ldg(Prec<T>::o2p(bv) + off0 + ip);

    T W[NHAB * NK];
#pragma unroll
    for (int x = 0; x < NHAB * NK; ++x) W[x] = T(0);

    for (int iq = 0; iq < n1e; ++iq) {
      const PrimPair<T> kq = pp[off1 + iq];
      const T o2q = __ldg(Prec<T>::o2p(bv) + off1 + iq);
      T Ecd[3][EC];
      hermite_E<T, LC, LD>(kq.PAx, kq.PAx + CDx, o2q, Ecd[0]);
      hermite_E<T, LC, LD>(kq.PAy, kq.PAy + CDy, o2q, Ecd[1]);
      hermite_E<T, LC, LD>(kq.PAz, kq.PAz + CDz, o2q, Ecd[2]);
      // 1/(p+q) = r^2, alpha = p q r^2, 2 pi^(5/2) K_q / (p q sqrt(p+q)) = 4 (2 pi^(5/2)) K_q r o2p o2q
      const T r = Prec<T>::rsq(bp.p + kq.p);
      T alpha = bp.p * kq.p * r * r;
      T pref = cst<T>(4.0 * 34.98683665524972) * kq.K * r * o2p * o2q;
      attenuate(w2, alpha, pref);
      T R[nherm(L)];
      prim_R<T, L>(alpha, bp.Px - kq.Px, bp.Py - kq.Py, bp.Pz - kq.Pz, bv, R);
      // ket transform W[tuv][cd] += sum_{tau nu phi} (+-) E^cd R_{t+tau, u+nu, v+phi}
      static_for<NK>([&](auto kk) {
        constexpr int k = decltype(kk)::value, kc = C0 + k;
        constexpr int cx = cart_x(LC, kc / ND), cy = cart_y(LC, kc / ND), cz = cart_z(LC, kc / ND);
        constexpr int dx = cart_x(LD, kc % ND), dy = cart_y(LD, kc % ND), dz = cart_z(LD, kc % ND);
#pragma unroll
        for (int tau = 0; tau <= cx + dx; ++tau) {
          const T ex = pref * Ecd[0][(cx * (LD + 1) + dx) * NTC + tau];
#pragma unroll
          for (int nu = 0; nu <= cy + dy; ++nu) {
            const T exy = ex * Ecd[1][(cy * (LD + 1) + dy) * NTC + nu];
#pragma unroll
            for (int phi = 0; phi <= cz + dz; ++phi) {
              T e2 = exy * Ecd[2][(cz * (LD + 1) + dz) * NTC + phi];
              if ((tau + nu + phi) & 1) e2 = -e2;
              // all bra Hermite functions (t,u,v), t+u+v <= LAB
#pragma unroll
              for (int n = 0; n <= LAB; ++n)
#pragma unroll
                for (int m = 0; m <= n; ++m)
#pragma unroll
                  for (int v = 0; v <= m; ++v) {
                    const int t = n - m, u = m - v;
                    W[hidx(t, u, v) * NK + k] += e2 * R[hidx(t + tau, u + nu, v + phi)];
                  }
            }
          }
        }
      });
    }
    // bra transform of this bra primitive (its E tables are formed only now,
    // when R is dead, which keeps the register footprint of the ket loop down)
    T Eab[3][EA];
    hermite_E<T, LA, LB>(bp.PAx, bp.PAx + ABx, o2p, Eab[0]);
    hermite_E<T, LA, LB>(bp.PAy, bp.PAy + ABy, o2p, Eab[1]);
    hermite_E<T, LA, LB>(bp.PAz, bp.PAz + ABz, o2p, Eab[2]);
    static_for<NAB>([&](auto abk) {
      constexpr int ab = decltype(abk)::value;
      constexpr int ax = cart_x(LA, ab / NB), ay = cart_y(LA, ab / NB), az = cart_z(LA, ab / NB);
      constexpr int bx = cart_x(LB, ab % NB), by = cart_y(LB, ab % NB), bz = cart_z(LB, ab % NB);
#pragma unroll
      for (int t = 0; t <= ax + bx; ++t)
#pragma unroll
        for (int u = 0; u <= ay + by; ++u) {
          const T exy = bp.K * Eab[0][(ax * (LB + 1) + bx) * NTA + t] * Eab[1][(ay * (LB + 1) + by) * NTA + u];
#pragma unroll
          for (int v = 0; v <= az + bz; ++v) {
            const T e1 = exy * Eab[2][(az * (LB + 1) + bz) * NTA + v];
#pragma unroll
            for (int k = 0; k < NK; ++k) G[ab * NK + k] += e1 * W[hidx(t, u, v) * NK + k];
          }
        }
    });
  }
}

// ---------------------------------------------------------------------------
// Runtime-L versions for the larger classes: one compiled kernel per
// precision serves every class with L > 4, with state in thread-local arrays
// sized for f shells (plus one derivative order).

constexpr int GEN_LMAX = LMAX + 1;                       // shells incl. derivative
constexpr int GEN_L = 4 * LMAX + 1;                      // largest total L
constexpr int GEN_NH = nherm(GEN_L);
constexpr int GEN_E = (GEN_LMAX + 1) * (LMAX + 1) * (GEN_LMAX + LMAX + 1);
constexpr int GEN_BUDGET = 640;

__device__ __forceinline__ int hidx_rt(int t, int u, int v) {
  const int n = t + u + v, m = u + v;
  return n * (n + 1) * (n + 2) / 6 + m * (m + 1) / 2 + v;
}
// position of the component (x, y, l-x-y) in the Cartesian order of shell l
__device__ __forceinline__ int cart_index_dev(int l, int x, int y) {
  const int d = l - x;  // components with larger x come first
  return d * (d + 1) / 2 + (d - y);
}
__device__ __forceinline__ void cart_pows_rt(int l, int k, int& x, int& y, int& z) {
  int i = l, off = 0;
  while (k >= off + (l - i + 1)) { off += l - i + 1; --i; }
  x = i; z = k - off; y = l - x - z;
}

template <typename T>
__device__ __forceinline__ void hermite_E_rt(int LA, int LB, T PA, T PB, T o2p, T* E) {
  const int NT = LA + LB + 1;
  for (int x = 0; x < (LA + 1) * (LB + 1) * NT; ++x) E[x] = T(0);
  E[0] = T(1);
#pragma unroll 1
  for (int i = 1; i <= LA; ++i)
#pragma unroll 1
    for (int t = 0; t <= i; ++t) {
      const int src = ((i - 1) * (LB + 1)) * NT;
      T v = (t <= i - 1) ? PA * E[src + t] : T(0);
      if (t > 0) v += o2p * E[src + t - 1];
      if (t + 1 <= i - 1) v += T(t + 1) * E[src + t + 1];
      E[(i * (LB + 1)) * NT + t] = v;
    }
#pragma unroll 1
  for (int i = 0; i <= LA; ++i)
#pragma unroll 1
    for (int j = 1; j <= LB; ++j)
#pragma unroll 1
      for (int t = 0; t <= i + j; ++t) {
        const int src = (i * (LB + 1) + j - 1) * NT;
        T v = (t <= i + j - 1) ? PB * E[src + t] : T(0);
        if (t > 0) v += o2p * E[src + t - 1];
        if (t + 1 <= i + j - 1) v += T(t + 1) * E[src + t + 1];
        E[(i * (LB + 1) + j) * NT + t] = v;
      }
}

__device__ __forceinline__ void boys_fp64_rt(int L, double T, const double* __restrict__ tab, double* F) {
  if (T < BOYS_TMAX) {
    const int i = __double2int_rn(T * (1.0 / BOYS_H));
    const double y = i * BOYS_H - T;
    const double* row = tab + i * (BOYS_MMAX + 1) + L;
    double acc = __ldg(row + 6);
#pragma unroll
    for (int k = 6; k >= 1; --k) acc = __ldg(row + k - 1) + acc * (y * (1.0 / k));
    const double e = exp(-T);
    F[L] = acc;
#pragma unroll 1
    for (int m = L - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + e) * c_inv_odd64[m];
  } else {
    const double rt = rsqrt(T);
    const double h = 0.5 * rt * rt;
    F[0] = 0.88622692545275801365 * rt;
#pragma unroll 1
    for (int m = 0; m < L; ++m) F[m + 1] = (2 * m + 1) * F[m] * h;
  }
}

__device__ __forceinline__ void boys_fp32_scaled_rt(int L, float T, const float* __restrict__ tab, float* G) {
  if (T < (float)BOYS_TMAX) {
    const int i = __float2int_rn(T * (float)(1.0 / BOYS_H));
    const float y = i * (float)BOYS_H - T;
    const float* row = tab + i * (BOYS_MMAX + 1) + L;
    float acc = __ldg(row + 4);
#pragma unroll
    for (int k = 4; k >= 1; --k) acc = __ldg(row + k - 1) + acc * (y * (1.0f / k));
    const float e = __expf(-T);
    G[L] = acc;
#pragma unroll 1
    for (int m = L - 1; m >= 0; --m) G[m] = (2.0f * T * G[m + 1] + e) * c_inv_odd32[m];
    const float c = fmaxf(1.0f, 2.0f * T);
    float cn = c;
#pragma unroll 1
    for (int m = 1; m <= L; ++m) { G[m] *= cn; cn *= c; }
  } else {
    G[0] = 0.88622692545f * rsqrtf(T);
#pragma unroll 1
    for (int m = 0; m < L; ++m) G[m + 1] = (2 * m + 1) * G[m];
  }
}

// In place: layer n overwrites layer n+1.  Inside a layer the entries are
// produced by decreasing t+u+v, so an entry is overwritten only after every
// entry of the new layer that reads it has been computed.
template <typename T>
__device__ __forceinline__ void hermite_R_rt(int L, const T* B, T X, T Y, T Z, T* R) {
#pragma unroll 1
  for (int n = L; n >= 0; --n) {
#pragma unroll 1
    for (int s = L - n; s >= 0; --s) {
#pragma unroll 1
      for (int t = s; t >= 0; --t) {
#pragma unroll 1
        for (int u = s - t; u >= 0; --u) {
          const int v = s - t - u;
          T val;
          if (s == 0) {
            val = B[n];
          } else if (t > 0) {
            val = X * R[hidx_rt(t - 1, u, v)];
            if (t > 1) val += T(t - 1) * R[hidx_rt(t - 2, u, v)];
          } else if (u > 0) {
            val = Y * R[hidx_rt(t, u - 1, v)];
            if (u > 1) val += T(u - 1) * R[hidx_rt(t, u - 2, v)];
          } else {
            val = Z * R[hidx_rt(t, u, v - 1)];
            if (v > 1) val += T(v - 1) * R[hidx_rt(t, u, v - 2)];
          }
          R[hidx_rt(t, u, v)] = val;
        }
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ void prim_R_rt(int L, T alpha, T X, T Y, T Z, const BasisView& bv, T* R) {
  T B[GEN_L + 1];
  const T Tb = alpha * (X * X + Y * Y + Z * Z);
  if constexpr (is_f64<T>) {
    boys_fp64_rt(L, Tb, bv.boys64, B);
    const T f = -2.0 * alpha;
    T pw = f;
#pragma unroll 1
    for (int n = 1; n <= L; ++n) { B[n] *= pw; pw *= f; }
    hermite_R_rt<T>(L, B, X, Y, Z, R);
  } else {
    boys_fp32_scaled_rt(L, Tb, bv.boys32, B);
#pragma unroll 1
    for (int n = 1; n <= L; n += 2) B[n] = -B[n];
    const float c = fmaxf(1.0f, 2.0f * Tb);
    const float s = sqrtf(2.0f * alpha / c);
    hermite_R_rt<T>(L, B, X * s, Y * s, Z * s, R);
    float sp = s;
#pragma unroll 1
    for (int n = 1; n <= L; ++n) {
      const int lo = n * (n + 1) * (n + 2) / 6, hi = (n + 1) * (n + 2) * (n + 3) / 6;
      for (int x = lo; x < hi; ++x) R[x] *= sp;
      sp *= s;
    }
  }
}

// Runtime class description.
struct RtClass {
  int la, lb, lc, ld, ck, nchunk;
};

__host__ __device__ constexpr RtClass make_rt_class(int la, int lb, int lc, int ld) {
  RtClass c{la, lb, lc, ld, 1, 1};
  const int nab = ncart(la) * ncart(lb), ncd = ncart(lc) * ncart(ld);
  const int raw = GEN_BUDGET / (nab + nherm(la + lb));
  c.ck = raw < 1 ? 1 : (raw > ncd ? ncd : raw);
  c.nchunk = (ncd + c.ck - 1) / c.ck;
  return c;
}

// Array capacities of one instantiation: E tables, R, W.
template <int NE_, int NH_, int NW_>
struct RtSizes {
  static constexpr int NE = NE_, NH = NH_, NW = NW_;
};
using GenSizes = RtSizes<GEN_E, GEN_NH, GEN_BUDGET>;

// eps > 0 skips the primitive quartets with Q_p Q_q < eps; work (if not NULL)
// is increased by the primitive quartets and bra primitives evaluated.
template <typename T, typename S = GenSizes>
__device__ __noinline__ void quartet_block_rt(const RtClass& C, const BasisView& bv, int bra, int ket, int chunk,
                                              T* G, const T* __restrict__ bra_w = nullptr, int pp_bra = -1,
                                              int pp_ket = -1, T eps = T(0), int* work = nullptr,
                                              T w2 = T(0)) {
  const int LA = C.la, LB = C.lb, LC = C.lc, LD = C.ld, CK = C.ck;
  const int NB = ncart(LB), ND = ncart(LD);
  const int NAB = ncart(LA) * NB, NCD = ncart(LC) * ND;
  const int LAB = LA + LB, LCD = LC + LD, L = LAB + LCD;
  const int NTA = LAB + 1, NTC = LCD + 1;
  const int EA = (LA + 1) * (LB + 1) * NTA, EC = (LC + 1) * (LD + 1) * NTC;
  const PrimPair<T>* __restrict__ pp = Prec<T>::pp(bv);
  // pp_bra / pp_ket >= 0 restrict the bra / ket to that single primitive pair
  const int off0 = pp_bra >= 0 ? pp_bra : __ldg(bv.pair_pp_off + bra);
  const int n0 = pp_bra >= 0 ? 1 : __ldg(bv.pair_pp_n + bra);
  const int off1 = pp_ket >= 0 ? pp_ket : __ldg(bv.pair_pp_off + ket);
  const int n1 = pp_ket >= 0 ? 1 : __ldg(bv.pair_pp_n + ket);
  const T ABx = from_f64<T>(__ldg(bv.pair_AB + 3 * bra)), ABy = from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 1)),
          ABz = from_f64<T>(__ldg(bv.pair_AB + 3 * bra + 2));
  const T CDx = from_f64<T>(__ldg(bv.pair_AB + 3 * ket)), CDy = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 1)),
          CDz = from_f64<T>(__ldg(bv.pair_AB + 3 * ket + 2));
  const int nhab = nherm(LAB);
  const int kc0 = chunk * CK;
  const int nk = min(CK, NCD - kc0);

  T Eab[3 * S::NE], Ecd[3 * S::NE];
  T R[S::NH];
  T W[S::NW];
  for (int x = 0; x < NAB * CK; ++x) G[x] = T(0);

  int n1e = n1;
#pragma unroll 1
  for (int ip = 0; ip < n0; ++ip) {
    if (eps > T(0)) {
      n1e = shrink_kept(bv.pp_q32 + off1, __ldg(bv.pp_q32 + off0 + ip), (float)eps, n1e);
      if (n1e == 0) break;
    }
    if (work) { work[0] += n1e; ++work[1]; }
    const PrimPair<T> bp = pp[off0 + ip];
    const T o2p = __ldg(Prec<T>::o2p(bv) + off0 + ip);
    hermite_E_rt<T>(LA, LB, bp.PAx, bp.PAx + ABx, o2p, Eab);
    hermite_E_rt<T>(LA, LB, bp.PAy, bp.PAy + ABy, o2p, Eab + EA);
    hermite_E_rt<T>(LA, LB, bp.PAz, bp.PAz + ABz, o2p, Eab + 2 * EA);
    for (int x = 0; x < nhab * CK; ++x) W[x] = T(0);
#pragma unroll 1
    for (int iq = 0; iq < n1e; ++iq) {
      const PrimPair<T> kq = pp[off1 + iq];
      const T o2q = __ldg(Prec<T>::o2p(bv) + off1 + iq);
      hermite_E_rt<T>(LC, LD, kq.PAx, kq.PAx + CDx, o2q, Ecd);
      hermite_E_rt<T>(LC, LD, kq.PAy, kq.PAy + CDy, o2q, Ecd + EC);
      hermite_E_rt<T>(LC, LD, kq.PAz, kq.PAz + CDz, o2q, Ecd + 2 * EC);
      const T r = Prec<T>::rsq(bp.p + kq.p);
      T alpha = bp.p * kq.p * r * r;
      T pref = cst<T>(4.0 * 34.98683665524972) * kq.K * r * o2p * o2q;
      attenuate(w2, alpha, pref);
      prim_R_rt<T>(L, alpha, bp.Px - kq.Px, bp.Py - kq.Py, bp.Pz - kq.Pz, bv, R);
#pragma unroll 1
      for (int k = 0; k < nk; ++k) {
        const int kc = kc0 + k;
        int cx, cy, cz, dx, dy, dz;
        cart_pows_rt(LC, kc / ND, cx, cy, cz);
        cart_pows_rt(LD, kc % ND, dx, dy, dz);
#pragma unroll 1
        for (int tau = 0; tau <= cx + dx; ++tau) {
          const T ex = Ecd[(cx * (LD + 1) + dx) * NTC + tau];
#pragma unroll 1
          for (int nu = 0; nu <= cy + dy; ++nu) {
            const T exy = ex * Ecd[EC + (cy * (LD + 1) + dy) * NTC + nu];
#pragma unroll 1
            for (int phi = 0; phi <= cz + dz; ++phi) {
              T e2 = pref * exy * Ecd[2 * EC + (cz * (LD + 1) + dz) * NTC + phi];
              if ((tau + nu + phi) & 1) e2 = -e2;
              int h = 0;
#pragma unroll 1
              for (int n = 0; n <= LAB; ++n)
#pragma unroll 1
                for (int m = 0; m <= n; ++m)
#pragma unroll 4
                  for (int v = 0; v <= m; ++v, ++h) {
                    const int t = n - m, u = m - v;
                    W[h * CK + k] += e2 * R[hidx_rt(t + tau, u + nu, v + phi)];
                  }
            }
          }
        }
      }
    }
    const T Kw = bra_w ? bp.K * bra_w[off0 + ip] : bp.K;
#pragma unroll 1
    for (int ab = 0; ab < NAB; ++ab) {
      int ax, ay, az, bx, by, bz;
      cart_pows_rt(LA, ab / NB, ax, ay, az);
      cart_pows_rt(LB, ab % NB, bx, by, bz);
#pragma unroll 1
      for (int t = 0; t <= ax + bx; ++t)
#pragma unroll 1
        for (int u = 0; u <= ay + by; ++u)
#pragma unroll 1
          for (int v = 0; v <= az + bz; ++v) {
            const T e1 = Kw * Eab[(ax * (LB + 1) + bx) * NTA + t] * Eab[EA + (ay * (LB + 1) + by) * NTA + u] *
                         Eab[2 * EA + (az * (LB + 1) + bz) * NTA + v];
            const int h = hidx_rt(t, u, v);
            for (int k = 0; k < nk; ++k) G[ab * CK + k] += e1 * W[h * CK + k];
          }
    }
  }
}

template <typename T>
__device__ __noinline__ void digest_rt(const RtClass& C, const JKLaunch& a, int bra, int ket, int chunk,
                                       const T* G) {
  const int NA = ncart(C.la), NB = ncart(C.lb), ND = ncart(C.ld);
  const int NCD = ncart(C.lc) * ND, CK = C.ck;
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
  const T* __restrict__ D = nullptr;
  D = dmat<T>(a) + base;
  double* __restrict__ Jm = a.J + base;
  double* __restrict__ Km = a.K + base;
  const int kc0 = chunk * CK, nk = min(CK, NCD - kc0);
#pragma unroll 1
  for (int ab = 0; ab < NA * NB; ++ab) {
    T s = T(0);
    for (int k = 0; k < nk; ++k) {
      const int kc = kc0 + k;
      s += G[ab * CK + k] * dload(D + (oc + kc / ND) * n + od + kc % ND);
    }
    atomicAdd(Jm + (oa + ab / NB) * n + ob + ab % NB, (double)(w4 * s));
  }
#pragma unroll 1
  for (int k = 0; k < nk; ++k) {
    const int kc = kc0 + k, ic = kc / ND, id = kc % ND;
    T s = T(0);
    for (int ab = 0; ab < NA * NB; ++ab) s += G[ab * CK + k] * dload(D + (oa + ab / NB) * n + ob + ab % NB);
    atomicAdd(Jm + (oc + ic) * n + od + id, (double)(w4 * s));
#pragma unroll 1
    for (int ia = 0; ia < NA; ++ia) {
      T s_ac = T(0), s_ad = T(0);
      for (int ib = 0; ib < NB; ++ib) {
        const T g = G[(ia * NB + ib) * CK + k];
        s_ac += g * dload(D + (ob + ib) * n + od + id);
        s_ad += g * dload(D + (ob + ib) * n + oc + ic);
      }
      atomicAdd(Km + (oa + ia) * n + oc + ic, (double)(w2 * s_ac));
      atomicAdd(Km + (oa + ia) * n + od + id, (double)(w2 * s_ad));
    }
#pragma unroll 1
    for (int ib = 0; ib < NB; ++ib) {
      T s_bc = T(0), s_bd = T(0);
      for (int ia = 0; ia < NA; ++ia) {
        const T g = G[(ia * NB + ib) * CK + k];
        s_bc += g * dload(D + (oa + ia) * n + od + id);
        s_bd += g * dload(D + (oa + ia) * n + oc + ic);
      }
      atomicAdd(Km + (ob + ib) * n + oc + ic, (double)(w2 * s_bc));
      atomicAdd(Km + (ob + ib) * n + od + id, (double)(w2 * s_bd));
    }
  }
}

// ---------------------------------------------------------------------------
// work decoding: quartet index -> (bra, ket) by binary search over the
// prefix of kept kets per (bra, bucket) segment (the implicit class-sorted
// work list).  The segment found is the last one starting at or before qi,
// which is never an empty one.
__device__ __forceinline__ void decode_quartet(const JKLaunch& a, long long qi, int& bra, int& ket) {
  int lo = 0, hi = a.nseg;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a.prefix + mid) <= qi) lo = mid; else hi = mid;
  }
  const long long j = qi - __ldg(a.prefix + lo) + __ldg(a.ket_start + lo);
  bra = a.bra_first + lo / NBK;
  ket = a.ket_first + (int)j;
}

// The same for the items base + d of a warp (0 <= d < 32, every lane of the
// warp calls it): a 32-ary search by the whole warp for the segment of base,
// then each lane finds its own segment among the next 32 segment starts by a
// binary search over the lanes' registers (segments beyond those 32, e.g.
// after a run of empty ones, fall back to decode_quartet).
__device__ __forceinline__ void decode_warp(const JKLaunch& a, long long base, int d, int& bra, int& ket) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = a.nseg;  // prefix[lo] <= base < prefix[hi]
  while (hi - lo > 32) {
    const long long span = hi - lo;
    const int p = lo + (int)((span * lane) >> 5);
    const unsigned le = __ballot_sync(0xffffffffu, __ldg(a.prefix + p) <= base);
    const int k = 31 - __clz(le);  // lane 0 probes lo, so k >= 0
    const int nlo = lo + (int)((span * k) >> 5);
    hi = k == 31 ? hi : lo + (int)((span * (k + 1)) >> 5);
    lo = nlo;
  }
  // r_j: start of segment lo + 1 + j relative to base (33 = beyond the list)
  const int idx = lo + 1 + lane;
  const long long pj = idx <= a.nseg ? __ldg(a.prefix + idx) : base + 33;
  const int rj = (int)min(max(pj - base, 0LL), 33LL);
  int c = 0;  // number of j with r_j <= d (r is non-decreasing in j)
#pragma unroll
  for (int st = 16; st > 0; st >>= 1) {
    const int r = __shfl_sync(0xffffffffu, rj, c + st - 1);
    if (r <= d) c += st;
  }
  if (__shfl_sync(0xffffffffu, rj, c & 31) <= d && c < 32) ++c;
  const long long pstart = __shfl_sync(0xffffffffu, pj, (c + 31) & 31);
  if (c == 32) {  // past the 32 segment starts held by the warp
    decode_quartet(a, base + d, bra, ket);
    return;
  }
  const int seg = lo + c;
  const long long start = c == 0 ? __ldg(a.prefix + lo) : pstart;
  const long long j = base + d - start + __ldg(a.ket_start + seg);
  bra = a.bra_first + seg / NBK;
  ket = a.ket_first + (int)j;
}

// J/K digestion of one quartet block (Cartesian, unsymmetrised accumulators):
// with w = s_ab s_cd s_(ab,cd) (1/2 for each coincidence)
//   J_ab += 4w sum_cd g D_cd,        J_cd += 4w sum_ab g D_ab,
//   K_ac += 2w sum_bd g D_bd,        K_ad += 2w sum_bc g D_bc,
//   K_bc += 2w sum_ad g D_ad,        K_bd += 2w sum_ac g D_ac,
// which after X <- (X + X^T)/2 equals the sum over all 8 index permutations.
// G holds the ket components [C0, C0 + NK) of the block (G[ab*NK + k]).
// Each thread reads every D element it needs once and sums over both inner
// indices before its atomic (one atomic per touched J and K element).  All 32
// lanes call it (valid = 0 for a lane without a quartet); when every valid
// lane of the warp holds the same bra pair, the J_ab sums are reduced across
// the warp first and one lane adds them.
template <typename T, int LA, int LB, int LC, int LD, int C0, int NK>
__device__ __forceinline__ void digest_range(const JKLaunch& a, int bra, int ket, bool valid, const T* G) {
  constexpr int NA = ncart(LA), NB = ncart(LB), NC = ncart(LC), ND = ncart(LD);
  constexpr int NAB = NA * NB;
  constexpr int CLO = C0 / ND, CHI = (C0 + NK - 1) / ND;  // ket c shells touched: [CLO, CHI]
  const BasisView& bv = a.bv;
  const int lane = threadIdx.x & 31;
  const int bra0 = __shfl_sync(0xffffffffu, valid ? bra : -1, __ffs(__ballot_sync(0xffffffffu, valid)) - 1);
  const bool warp_bra = __all_sync(0xffffffffu, !valid || bra == bra0);
  T jab[NAB];
  int oa = 0, ob = 0;
  long long base = 0;
  long n = 0;
  T w4 = T(0);
  if (valid) {
    const int sa = __ldg(bv.pair_a + bra), sb = __ldg(bv.pair_b + bra);
    const int sc = __ldg(bv.pair_a + ket), sd = __ldg(bv.pair_b + ket);
    oa = __ldg(bv.shell_coff + sa); ob = __ldg(bv.shell_coff + sb);
    const int oc = __ldg(bv.shell_coff + sc), od = __ldg(bv.shell_coff + sd);
    mol_block(bv, bra, base, n);
    T w = T(1);
    if (sa == sb) w *= cst<T>(0.5);
    if (sc == sd) w *= cst<T>(0.5);
    if (a.same_class && bra == ket) w *= cst<T>(0.5);
    w4 = T(4) * w;
    const T w2 = T(2) * w;
    const T* __restrict__ D = dmat<T>(a) + base;
    double* __restrict__ Jm = a.J + base;
    double* __restrict__ Km = a.K + base;
    T Dk[NK], Dab[NAB], Dbd[NB * ND], Dbc[NB * NC], Dad[NA * ND], Dac[NA * NC];
#pragma unroll
    for (int k = 0; k < NK; ++k) Dk[k] = dload(D + (oc + (C0 + k) / ND) * n + od + (C0 + k) % ND);
#pragma unroll
    for (int x = 0; x < NA; ++x)
#pragma unroll
      for (int y = 0; y < NB; ++y) Dab[x * NB + y] = dload(D + (oa + x) * n + ob + y);
#pragma unroll
    for (int y = 0; y < NB; ++y) {
#pragma unroll
      for (int d = 0; d < ND; ++d) Dbd[y * ND + d] = dload(D + (ob + y) * n + od + d);
#pragma unroll
      for (int c = CLO; c <= CHI; ++c) Dbc[y * NC + c] = dload(D + (ob + y) * n + oc + c);
    }
#pragma unroll
    for (int x = 0; x < NA; ++x) {
#pragma unroll
      for (int d = 0; d < ND; ++d) Dad[x * ND + d] = dload(D + (oa + x) * n + od + d);
#pragma unroll
      for (int c = CLO; c <= CHI; ++c) Dac[x * NC + c] = dload(D + (oa + x) * n + oc + c);
    }
    // J_ab (added below, possibly after a warp reduction)
#pragma unroll
    for (int ab = 0; ab < NAB; ++ab) {
      T s = T(0);
#pragma unroll
      for (int k = 0; k < NK; ++k) s += G[ab * NK + k] * Dk[k];
      jab[ab] = s;
    }
    // J_cd
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      T s = T(0);
#pragma unroll
      for (int ab = 0; ab < NAB; ++ab) s += G[ab * NK + k] * Dab[ab];
      atomicAdd(Jm + (oc + (C0 + k) / ND) * n + od + (C0 + k) % ND, (double)(w4 * s));
    }
    // K_ac, K_ad (c and d of the range's components)
#pragma unroll
    for (int x = 0; x < NA; ++x) {
#pragma unroll
      for (int c = CLO; c <= CHI; ++c) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NK; ++k)
          if ((C0 + k) / ND == c)
#pragma unroll
            for (int y = 0; y < NB; ++y) s += G[(x * NB + y) * NK + k] * Dbd[y * ND + (C0 + k) % ND];
        atomicAdd(Km + (oa + x) * n + oc + c, (double)(w2 * s));
      }
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        bool touched = false;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NK; ++k)
          if ((C0 + k) % ND == d) {
            touched = true;
#pragma unroll
            for (int y = 0; y < NB; ++y) s += G[(x * NB + y) * NK + k] * Dbc[y * NC + (C0 + k) / ND];
          }
        if (touched) atomicAdd(Km + (oa + x) * n + od + d, (double)(w2 * s));
      }
    }
    // K_bc, K_bd
#pragma unroll
    for (int y = 0; y < NB; ++y) {
#pragma unroll
      for (int c = CLO; c <= CHI; ++c) {
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NK; ++k)
          if ((C0 + k) / ND == c)
#pragma unroll
            for (int x = 0; x < NA; ++x) s += G[(x * NB + y) * NK + k] * Dad[x * ND + (C0 + k) % ND];
        atomicAdd(Km + (ob + y) * n + oc + c, (double)(w2 * s));
      }
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        bool touched = false;
        T s = T(0);
#pragma unroll
        for (int k = 0; k < NK; ++k)
          if ((C0 + k) % ND == d) {
            touched = true;
#pragma unroll
            for (int x = 0; x < NA; ++x) s += G[(x * NB + y) * NK + k] * Dac[x * NC + (C0 + k) / ND];
          }
        if (touched) atomicAdd(Km + (ob + y) * n + od + d, (double)(w2 * s));
      }
    }
  }
  // J_ab: one atomic per element per warp when the whole warp shares the bra
  // (the work list is bra-major, so this is the common case)
  if (warp_bra) {
#pragma unroll
    for (int ab = 0; ab < NAB; ++ab) {
      double v = valid ? (double)(w4 * jab[ab]) : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == __ffs(__ballot_sync(0xffffffffu, valid)) - 1)
        atomicAdd(a.J + base + (oa + ab / NB) * n + ob + ab % NB, v);
    }
  } else if (valid) {
#pragma unroll
    for (int ab = 0; ab < NAB; ++ab) atomicAdd(a.J + base + (oa + ab / NB) * n + ob + ab % NB, (double)(w4 * jab[ab]));
  }
}

// ---------------------------------------------------------------------------
// Persistent J/K kernel of one class pair and one precision band.  Warps take
// 32 work items at a time from a device atomic counter (the single-GPU form of
// the dynamically scheduled global task counter of Sec. 1.2.2); an item is a
// (quartet, ket chunk).  No thread ever waits on another.
constexpr int JK_THREADS = 128;

// Classes small enough to keep every intermediate in registers get a fully
// unrolled instantiation; the rest use the runtime-L kernel.
__host__ __device__ constexpr bool is_small_class(int la, int lb, int lc, int ld) {
  return la + lb + lc + ld <= 4 && ncart(la) * ncart(lb) * ncart(lc) * ncart(ld) <= 81;
}

// Small classes: one thread per quartet with the whole block in registers.
template <typename T, int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(JK_THREADS) k_jk(JKLaunch a) {
  constexpr int NAB = ncart(LA) * ncart(LB), NCD = ncart(LC) * ncart(LD);
  const long long total = (long long)__ldg(a.prefix + a.nseg);
  const int lane = threadIdx.x & 31;
  unsigned cpq = 0, cbp = 0;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.counter, 32ULL);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total) break;
    if (*(volatile const int*)a.abort_flag) {
      if (lane == 0) atomicCAS(a.status, 0, ADFT_ERR_ABORTED);
      break;
    }
    const long long item = (long long)base + lane;
    const bool valid = item < total;
    int bra = 0, ket = 0;
    T G[NAB * NCD];
    decode_warp(a, (long long)base, valid ? lane : 0, bra, ket);
    if (valid) {
      int npq = 0, nbp = 0;
      quartet_block_range<T, LA, LB, LC, LD, 0, NCD>(a.bv, bra, ket, G, (T)a.prim_eps, npq, nbp, (T)a.omega2);
      cpq += npq;
      cbp += nbp;
    }
    digest_range<T, LA, LB, LC, LD, 0, NCD>(a, bra, ket, valid, G);
  }
  flush_work(a.work, cpq, cbp);
}

template <typename T, int LA, int LB, int LC, int LD>
__global__ void __launch_bounds__(JK_THREADS) k_jk_generic(JKLaunch a) {
  constexpr RtClass C = make_rt_class(LA, LB, LC, LD);
  constexpr int LAB = LA + LB, LCD = LC + LD;
  constexpr int EA = (LA + 1) * (LB + 1) * (LAB + 1), EC = (LC + 1) * (LD + 1) * (LCD + 1);
  using S = RtSizes<(EA > EC ? EA : EC), nherm(LAB + LCD), nherm(LAB) * C.ck>;
  constexpr int NG = ncart(LA) * ncart(LB) * C.ck;
  const long long total = (long long)__ldg(a.prefix + a.nseg) * C.nchunk;
  const int lane = threadIdx.x & 31;
  T G[NG];
  unsigned cpq = 0, cbp = 0;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.counter, 32ULL);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((long long)base >= total) break;
    if (*(volatile const int*)a.abort_flag) {
      if (lane == 0) atomicCAS(a.status, 0, ADFT_ERR_ABORTED);
      break;
    }
    const long long item = (long long)base + lane;
    if (item < total) {
      // chunk-major order: the lanes of a warp share one ket chunk (uniform
      // component loops) and take consecutive quartets
      const long long nq = total / C.nchunk;
      const int chunk = (int)(item / nq);
      const long long qi = item - (long long)chunk * nq;
      int bra, ket;
      decode_quartet(a, qi, bra, ket);
      int wk[2] = {0, 0};
      quartet_block_rt<T, S>(C, a.bv, bra, ket, chunk, G, nullptr, -1, -1, (T)a.prim_eps, wk, (T)a.omega2);
      if (chunk == 0) { cpq += wk[0]; cbp += wk[1]; }  // count each quartet once
      digest_rt<T>(C, a, bra, ket, chunk, G);
    }
  }
  flush_work(a.work, cpq, cbp);
}

#ifdef ADFT_ERI_SCHWARZ
// Schwarz bounds of the pairs of one class, first step: one thread per
// (pair i, chunk of components, bra primitive pair p) evaluates the diagonal
// elements (mn|mn) of its chunk with the bra restricted to p and every ket
// primitive, into part[(i * NAB + mn) * maxp + p].  Splitting over p keeps
// each thread's serial work to one row of primitive quartets.
static __global__ void __launch_bounds__(JK_THREADS) k_schwarz_part(BasisView bv, RtClass C, int first, int n,
                                                                    int maxp, double* part) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long per = (long long)C.nchunk * maxp;
  if (t >= (long long)n * per) return;
  const int i = (int)(t / per), r = (int)(t % per);
  const int chunk = r / maxp, ip = r % maxp;
  const int pr = first + i;
  if (ip >= bv.pair_pp_n[pr]) return;
  const int NAB = ncart(C.la) * ncart(C.lb);
  double G[GEN_BUDGET];
  quartet_block_rt<double>(C, bv, pr, pr, chunk, G, nullptr, bv.pair_pp_off[pr] + ip, -1);
  for (int k = 0; k < C.ck; ++k) {
    const int kc = chunk * C.ck + k;
    if (kc < NAB) part[((long long)i * NAB + kc) * maxp + ip] = G[kc * C.ck + k];
  }
}

// Second step: (mn|mn) = sum over p in order (the same every run), and
// Qmax[pr] = max over mn of |(mn|mn)| by an integer atomicMax on the bits of
// the non-negative double (its ordering matches; the maximum does not depend
// on the order).  Qmax must be zero on entry; the caller takes the root.
static __global__ void k_schwarz_reduce(BasisView bv, int first, int n, int nab, int maxp, const double* part,
                                        unsigned long long* Qmax) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * nab) return;
  const int i = (int)(t / nab);
  const int np = bv.pair_pp_n[first + i];
  const double* src = part + t * maxp;
  double s = 0.0;
  for (int p = 0; p < np; ++p) s += src[p];
  atomicMax(Qmax + first + i, (unsigned long long)__double_as_longlong(fabs(s)));
}

// Primitive-pair bounds of the pairs of one class: Qp = sqrt(max |[mn|mn]_p|)
// with only primitive pair p on both sides (one thread per primitive pair).
static __global__ void __launch_bounds__(JK_THREADS) k_prim_schwarz(BasisView bv, RtClass C, int first, int n,
                                                                    const int* __restrict__ pp_pair, double* Qp) {
  const int pp_first = bv.pair_pp_off[first];
  const int pp_end = bv.pair_pp_off[first + n - 1] + bv.pair_pp_n[first + n - 1];
  const int g = pp_first + blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= pp_end) return;
  const int pr = pp_pair[g];
  const int NAB = ncart(C.la) * ncart(C.lb);
  double mx = 0.0;
  double G[GEN_BUDGET];
  for (int chunk = 0; chunk < C.nchunk; ++chunk) {
    quartet_block_rt<double>(C, bv, pr, pr, chunk, G, nullptr, g, g);
    for (int k = 0; k < C.ck; ++k) {
      const int kc = chunk * C.ck + k;
      if (kc < NAB) mx = fmax(mx, fabs(G[kc * C.ck + k]));
    }
  }
  Qp[g] = sqrt(mx);
}

#endif  // ADFT_ERI_SCHWARZ

#include "adft_coop.cuh"
#include "adft_warp.cuh"
#include "adft_row.cuh"

// ---------------------------------------------------------------------------
// dispatch: one launcher per (X, Y) class pair, X >= Y.  The launchers are
// explicitly instantiated in several translation units (adft_eri_*.cu) so
// that they compile in parallel; adft_dispatch.cu holds the tables.
template <typename T, int X, int Y>
cudaError_t launch_one(const JKLaunch& a, int grid, int variant, cudaStream_t s, KernelInfo* info);

#ifndef ADFT_ERI_DECLARE_ONLY
// A flag per CUDA device: a kernel's dynamic shared-memory attribute is set
// once per device (it does not carry over to another device).  Concurrent
// first calls may both set it, which is harmless.
struct PerDeviceFlag {
  static constexpr int MAXDEV = 64;
  bool set[MAXDEV] = {};
  bool& current() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= MAXDEV) d = 0;
    return set[d];
  }
};

// Launch kern with smem bytes of dynamic shared memory, or, with info, report
// how many blocks of it fit on one SM.  configured: the instantiation's
// one-time flag (for the current device) for the shared-memory attribute.
template <typename Kern>
static cudaError_t start(Kern kern, const JKLaunch& a, int grid, int threads, int smem, bool& configured,
                         int variants, cudaStream_t s, KernelInfo* info) {
  if (smem > 0 && !configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (info) {
    info->variants = variants;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&info->max_blocks_per_sm, kern, threads, smem);
  }
  kern<<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int X, int Y>
cudaError_t launch_one(const JKLaunch& a, int grid, int variant, cudaStream_t s, KernelInfo* info) {
  constexpr int LA = cls_la(X), LB = cls_lb(X), LC = cls_la(Y), LD = cls_lb(Y);
  if constexpr (X < Y) {
    return cudaErrorInvalidValue;
  } else if constexpr (is_small_class(LA, LB, LC, LD)) {
    static PerDeviceFlag configured;
    return start(k_jk<T, LA, LB, LC, LD>, a, grid, JK_THREADS, 0, configured.current(), 1, s, info);
  } else if constexpr (CoopPlan<T, LA, LB, LC, LD>::fits) {
    // Up to four kernels serve these classes and the autotuner picks one.
    // Variant 0 is the warp kernel in FP64 where it exists and the
    // cooperative one otherwise; variant 1 the other of the two where both
    // exist; then the row-blocked kernel with the busiest shape (policy 0) and
    // with the occupancy-aware shape (policy 1), where their plans fit.
    using W = WarpPlan<T, LA, LB, LC, LD>;
    using C = CoopPlan<T, LA, LB, LC, LD>;
    using R0 = RowPlan<T, LA, LB, LC, LD, 0>;
    using R1 = RowPlan<T, LA, LB, LC, LD, 1>;
    constexpr bool hw = W::fits, h0 = R0::fits, h1 = R1::fits;
    constexpr int nvar = 1 + (hw ? 1 : 0) + (h0 ? 1 : 0) + (h1 ? 1 : 0);
    constexpr bool warp_first = hw && sizeof(T) == 8;
    int v = variant;
    if constexpr (hw) {
      if (v == 0 || v == 1) {
        if ((v == 0) == warp_first) {
          static PerDeviceFlag configured;
          return start(k_jk_warp<T, LA, LB, LC, LD>, a, grid, 32 * W::WARPS, W::SMEM, configured.current(), nvar,
                       s, info);
        }
        static PerDeviceFlag configured;
        return start(k_jk_coop<T, LA, LB, LC, LD>, a, grid, 32 * C::WARPS, C::SMEM, configured.current(), nvar, s,
                     info);
      }
      v -= 2;
    } else {
      if (v == 0) {
        static PerDeviceFlag configured;
        return start(k_jk_coop<T, LA, LB, LC, LD>, a, grid, 32 * C::WARPS, C::SMEM, configured.current(), nvar, s,
                     info);
      }
      v -= 1;
    }
    if constexpr (h0) {
      if (v == 0) {
        static PerDeviceFlag configured;
        return start(k_jk_row<T, LA, LB, LC, LD, 0>, a, grid, 32 * R0::WARPS, R0::SMEM, configured.current(), nvar,
                     s, info);
      }
      --v;
    }
    if constexpr (h1) {
      if (v == 0) {
        static PerDeviceFlag configured;
        return start(k_jk_row<T, LA, LB, LC, LD, 1>, a, grid, 32 * R1::WARPS, R1::SMEM, configured.current(), nvar,
                     s, info);
      }
    }
    return cudaErrorInvalidValue;  // variant past the count (adft_set_tuning rejects it)
  } else {
    static_assert(!WarpPlan<T, LA, LB, LC, LD>::fits, "warp-kernel classes also need the cooperative kernel");
    static PerDeviceFlag configured;
    return start(k_jk_generic<T, LA, LB, LC, LD>, a, grid, JK_THREADS, 0, configured.current(), 1, s, info);
  }
}
#endif

}  // namespace adft
