// Host orchestration and the data-parallel setup / screening / transform
// kernels of the GB300 J/K library.  Public entry points: include/adft.h.
//
// A basis holds one molecule; a batch is a basis holding several molecules:
// shells and atoms are concatenated, shell pairs are formed only inside a
// molecule and grouped by angular-momentum class, then by molecule, then by
// descending Schwarz bound.  Every per-call array (Cartesian D, J, K) is
// packed molecule after molecule, so one persistent kernel per class pair
// serves all molecules of a batch.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "adft_internal.cuh"

namespace adft {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

#define ADFT_CUDA(call)                                                                 \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                   \
      return e_ == cudaErrorMemoryAllocation ? ADFT_ERR_OOM : ADFT_ERR_CUDA;            \
    }                                                                                  \
  } while (0)

// ---------------------------------------------------------------------------
// Boys table: F_m(i h) for i < BOYS_NT, m <= BOYS_MMAX, from the series
// F_m(T) = e^-T sum_k (2T)^k / ((2m+1)(2m+3)...(2m+2k+1)) summed in long
// double for the largest m, then downward recursion (Helgaker Sec. 9.8).

static void boys_row(double T, double* F) {
  const int M = BOYS_MMAX;
  long double term = 1.0L / (2 * M + 1), sum = term;
  for (int k = 1; k < 200000; ++k) {
    term *= 2.0L * T / (2 * M + 2 * k + 1);
    sum += term;
    if (term < 1e-25L * sum) break;
  }
  const long double e = expl(-(long double)T);
  long double f = e * sum;
  F[M] = (double)f;
  for (int m = M - 1; m >= 0; --m) {
    f = (2.0L * T * f + e) / (2 * m + 1);
    F[m] = (double)f;
  }
}

struct DeviceTables {
  double* boys64 = nullptr;
  float* boys32 = nullptr;
};
static std::mutex g_tab_mu;
static DeviceTables g_tab[64];

cudaError_t boys_tables(const double** t64, const float** t32) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (!g_tab[dev].boys64) {
    const int W = BOYS_MMAX + 1;
    std::vector<double> h(BOYS_NT * W);
    std::vector<float> hf(BOYS_NT * W);
    for (int i = 0; i < BOYS_NT; ++i) boys_row(i * BOYS_H, &h[i * W]);
    for (size_t i = 0; i < h.size(); ++i) hf[i] = (float)h[i];
    double* d64 = nullptr;
    float* d32 = nullptr;
    if ((e = cudaMalloc(&d64, h.size() * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d32, hf.size() * sizeof(float))) != cudaSuccess) { cudaFree(d64); return e; }
    cudaMemcpy(d64, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(d32, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice);
    g_tab[dev].boys64 = d64;
    g_tab[dev].boys32 = d32;
  }
  *t64 = g_tab[dev].boys64;
  *t32 = g_tab[dev].boys32;
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Cartesian -> real solid harmonic coefficients, from the explicit expansion
// of the real solid harmonics (Helgaker, Jorgensen, Olsen eqs. 6.4.47-6.4.49);
// rows m = -l..l (p: x, y, z), columns in the Cartesian order of the library.
constexpr int SPH_MAXC = 10;  // ncart(3)
__constant__ double c_sph[LMAX + 1][2 * LMAX + 1][SPH_MAXC];

static double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
static double binom(int n, int k) { return (k < 0 || k > n) ? 0.0 : fact(n) / (fact(k) * fact(n - k)); }
static int cart_index_host(int l, int x, int y) {
  int k = 0;
  for (int i = l; i >= 0; --i)
    for (int j = l - i; j >= 0; --j) {
      if (i == x && j == y) return k;
      ++k;
    }
  return -1;
}

static void sph_coefficients(double out[LMAX + 1][2 * LMAX + 1][SPH_MAXC]) {
  memset(out, 0, sizeof(double) * (LMAX + 1) * (2 * LMAX + 1) * SPH_MAXC);
  out[0][0][0] = 1.0;
  for (int k = 0; k < 3; ++k) out[1][k][k] = 1.0;
  for (int l = 2; l <= LMAX; ++l) {
    for (int m = -l; m <= l; ++m) {
      const int am = abs(m);
      const double nlm = sqrt(2.0 * fact(l + am) * fact(l - am) / (m == 0 ? 2.0 : 1.0)) / (pow(2.0, am) * fact(l));
      // v runs over integers (m >= 0) or half-integers (m < 0): use w = 2v
      for (int t = 0; t <= (l - am) / 2; ++t)
        for (int u = 0; u <= t; ++u)
          for (int w = (m < 0 ? 1 : 0); w <= am; w += 2) {
            const int sgn_exp = t + (w - (m < 0 ? 1 : 0)) / 2;
            const double c = ((sgn_exp & 1) ? -1.0 : 1.0) * pow(0.25, t) * binom(l, t) * binom(l - t, am + t) *
                             binom(t, u) * binom(am, w);
            const int px = 2 * t + am - 2 * u - w, py = 2 * u + w;
            out[l][m + l][cart_index_host(l, px, py)] += nlm * c;
          }
    }
  }
}

static inline bool is_mixed(int prec) { return prec == ADFT_PREC_MIXED; }

// ---------------------------------------------------------------------------
// basis handle

struct Workspace {
  double* Dc = nullptr;     // Cartesian D, packed per molecule
  float* Dc32 = nullptr;
  double* Jc = nullptr;     // Cartesian accumulators (unsymmetrised)
  double* Kc = nullptr;
  double* Jw = nullptr;     // J, K in the output basis (energy calls)
  double* Kw = nullptr;
  int* cnt64 = nullptr;     // per (class pair, bra): kept FP64 kets
  int* cnt32 = nullptr;     //                        kept FP32 kets
  int* kst64 = nullptr;     //                        first FP64 ket - class start
  int* kst32 = nullptr;     //                        first FP32 ket - class start
  long long* pre64 = nullptr;  // per class pair: prefix sums over its bras
  long long* pre32 = nullptr;
  unsigned long long* counters = nullptr;  // [3 sets][2 * NCP] work counters
  int* status = nullptr;    // [4]: status word, abort flag
  double* scal = nullptr;   // [4]: energy, max|D|, max|D-D^T|
  double* Emol = nullptr;   // [nmol] energies
  double* charges = nullptr;  // [natom] nuclear charges of a one-electron call
  unsigned long long* stats = nullptr;     // [10], see ScreenArgs::stats
  unsigned long long* work = nullptr;      // [2 bands][NCP][2] evaluated primitive quartets, bra primitives
};

}  // namespace adft

struct adft_basis {
  int device = 0;
  int nmol = 1;
  int natom = 0, nshell = 0, ncart = 0, nbf = 0, spherical = 1;  // totals
  std::vector<int> mol_atom_off, mol_shell_off, mol_cf_off, mol_f_off;  // [nmol+1]
  std::vector<int> mol_nc, mol_nbf;                                     // [nmol]
  std::vector<long long> mol_cbase, mol_obase;                          // [nmol+1] packed n^2 offsets
  std::vector<int> shell_l, shell_atom, shell_nprim, shell_poff, shell_coff, shell_soff, shell_mol;
  std::vector<double> xyz, exps, ncoefs;  // ncoefs: c_i N(a_i, l)
  // pairs: class-major, then molecule, then descending Q
  int npair = 0;
  int cls_first[adft::NCLS + 1];
  std::vector<int> seg_first;  // [NCLS][nmol+1]: first pair of class X of molecule m
  // [(X * nmol + m) * NBK + k] (+1 end): first pair of contraction bucket k of
  // class X, molecule m (pairs ordered by bucket, then descending Q)
  std::vector<int> bseg_first;
  std::vector<int> pair_a, pair_b;
  std::vector<double> pair_Q;
  long long npp = 0, npp_dense = 0;
  long long cnt_off[adft::NCP];
  long long pre_off[adft::NCP];
  // device arrays
  int *d_shell_l = nullptr, *d_shell_atom = nullptr, *d_shell_coff = nullptr, *d_shell_soff = nullptr;
  int *d_shell_nprim = nullptr, *d_shell_poff = nullptr;
  double *d_xyz = nullptr, *d_exps = nullptr, *d_ncoefs = nullptr;
  int *d_pair_a = nullptr, *d_pair_b = nullptr, *d_pair_ppoff = nullptr, *d_pair_ppn = nullptr, *d_pair_mol = nullptr;
  double *d_pair_Q = nullptr, *d_pair_AB = nullptr;
  long long* d_cumppn = nullptr;
  int* d_bseg_first = nullptr;
  int *d_mol_nc = nullptr, *d_mol_nbf = nullptr, *d_mol_cf_off = nullptr, *d_mol_f_off = nullptr;
  long long *d_mol_cbase = nullptr, *d_mol_obase = nullptr;
  adft::PrimPair<double>* d_pp64 = nullptr;
  adft::PrimPair<float>* d_pp32 = nullptr;
  int* d_pp_src = nullptr;    // [npp] (ia << 8) | ib
  double* d_ppw64 = nullptr;  // [2][npp] 2a, 2b
  double* d_o2p64 = nullptr;  // [npp] 1/(2p)
  float* d_o2p32 = nullptr;
  float* d_ppq32 = nullptr;   // [npp] primitive-pair bound Q_p, descending within each pair
  bool work_valid = false;    // the last call ran the J/K kernels (evaluated-work counters filled)
  float* d_ppw32 = nullptr;
  int *d_func_shell = nullptr, *d_func_comp = nullptr;    // output function -> (shell, component)
  int *d_cfunc_shell = nullptr, *d_cfunc_comp = nullptr;  // Cartesian function -> (shell, component)
  const double* boys64 = nullptr;
  const float* boys32 = nullptr;
  adft::Workspace ws;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int ev_valid = 0;
  int tune_blocks[2][adft::NCP];   // blocks per SM of every class-pair kernel and band (autotuner)
  int tune_variant[2][adft::NCP];  // kernel variant of every class pair and band (autotuner)
  int sms = 152;
  std::vector<void*> allocations;
};

struct adft_batch {
  adft_basis* b = nullptr;  // the concatenated basis (owned)
  // CUDA graph of the last captured call
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::tuple<const void*, const void*, const void*, const void*, const void*, double, double, int, void*> key;
  bool has_graph = false;
};

namespace adft {

template <typename T>
static int dalloc(adft_basis* b, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    return ADFT_ERR_OOM;
  }
  b->allocations.push_back((void*)*p);
  return ADFT_OK;
}

template <typename T>
static int upload(adft_basis* b, T** p, const std::vector<T>& h) {
  int st = dalloc(b, p, h.size());
  if (st) return st;
  if (!h.empty()) ADFT_CUDA(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return ADFT_OK;
}

static BasisView view(const adft_basis* b) {
  BasisView v;
  v.nshell = b->nshell; v.natom = b->natom; v.ncart = b->ncart; v.nbf = b->nbf; v.spherical = b->spherical;
  v.shell_l = b->d_shell_l; v.shell_atom = b->d_shell_atom; v.shell_coff = b->d_shell_coff; v.xyz = b->d_xyz;
  v.npair = b->npair; v.pair_a = b->d_pair_a; v.pair_b = b->d_pair_b; v.pair_Q = b->d_pair_Q;
  v.pair_pp_off = b->d_pair_ppoff; v.pair_pp_n = b->d_pair_ppn; v.pair_AB = b->d_pair_AB;
  v.pp64 = b->d_pp64; v.pp32 = b->d_pp32; v.boys64 = b->boys64; v.boys32 = b->boys32;
  v.pp_w64 = b->d_ppw64; v.pp_w32 = b->d_ppw32; v.npp = b->npp;
  v.pp_o2p64 = b->d_o2p64; v.pp_o2p32 = b->d_o2p32;
  v.pp_q32 = b->d_ppq32;
  v.pair_mol = (b->nmol > 1) ? b->d_pair_mol : nullptr;
  v.mol_cbase = b->d_mol_cbase; v.mol_nc = b->d_mol_nc;
  return v;
}

// ---------------------------------------------------------------------------
// a1: primitive-pair construction, one thread per primitive pair.
__global__ void k_build_pairs(int npair, const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                              const int* __restrict__ ppoff, const int* __restrict__ pp_src,
                              const int* __restrict__ shell_atom, const int* __restrict__ shell_poff,
                              const double* __restrict__ xyz, const double* __restrict__ exps,
                              const double* __restrict__ ncoefs, long long npp, PrimPair<double>* pp64,
                              PrimPair<float>* pp32, double* w64, float* w32, double* o2p64, float* o2p32,
                              int* pp_pair) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npp) return;
  // pair owning primitive pair g (ppoff is ascending)
  int lo = 0, hi = npair;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ppoff[mid] <= g) lo = mid; else hi = mid;
  }
  const int pr = lo, sa = pair_a[pr], sb = pair_b[pr];
  const int ia = pp_src[g] >> 8, ib = pp_src[g] & 255;  // primitive indices in shells a and b
  const double a = exps[shell_poff[sa] + ia], b = exps[shell_poff[sb] + ib];
  const double* A = xyz + 3 * shell_atom[sa];
  const double* B = xyz + 3 * shell_atom[sb];
  const double p = a + b, mu = a * b / p;
  const double ABx = A[0] - B[0], ABy = A[1] - B[1], ABz = A[2] - B[2];
  const double Px = (a * A[0] + b * B[0]) / p, Py = (a * A[1] + b * B[1]) / p, Pz = (a * A[2] + b * B[2]) / p;
  const double K = ncoefs[shell_poff[sa] + ia] * ncoefs[shell_poff[sb] + ib] *
                   exp(-mu * (ABx * ABx + ABy * ABy + ABz * ABz));
  pp64[g] = PrimPair<double>{Px, Py, Pz, p, Px - A[0], Py - A[1], Pz - A[2], K};
  pp32[g] = PrimPair<float>{(float)Px, (float)Py, (float)Pz, (float)p, (float)(Px - A[0]), (float)(Py - A[1]),
                            (float)(Pz - A[2]), (float)K};
  w64[g] = 2.0 * a; w64[npp + g] = 2.0 * b;
  o2p64[g] = 0.5 / p;
  o2p32[g] = (float)(0.5 / p);
  w32[g] = (float)(2.0 * a); w32[npp + g] = (float)(2.0 * b);
  if (pp_pair) pp_pair[g] = pr;
}

// ---------------------------------------------------------------------------
// a3: screening.  For every bra pair i (class X, molecule m) and ket class
// Y <= X, the kept kets are a prefix of molecule m's segment of class Y
// (sorted by descending Q): those with Q_i Q_k >= thresh; of them the FP64
// ones are those with Q_i Q_k >= split.
struct ScreenArgs {
  int cls_first[NCLS + 1];
  long long cnt_off[NCP];
  int nmol;
  const int* bseg_first;    // [(NCLS * nmol) * NBK + 1] bucketed segment starts
  const int* pair_mol;      // [npair] or NULL (one molecule)
  const double* Q;
  const int* ppn;
  const long long* cumppn;  // [npair + 1] running sum of ppn in pair order
  double thresh, split;
  int mixed;
  int* cnt64;
  int* cnt32;
  int* kst64;
  int* kst32;
  // [0] q64 [1] q32 [2] total unique [3] prim64 [4] prim32 [5] flop64 [6] flop32 (primitive
  // counts and flops before primitive-quartet screening) [7] flop64 [8] flop32 of the
  // per-quartet part only (the kernels count the primitive-level part)
  unsigned long long* stats;
  float f_pq[NCP], f_bra[NCP], f_q[NCP];
};

__device__ __forceinline__ int count_prefix(const double* Q, int first, int n, double Qi, double thr) {
  // number of leading k in [first, first+n) with Qi * Q[k] >= thr
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (Qi * Q[first + mid] >= thr) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_screen(ScreenArgs a, int npair) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long q64 = 0, q32 = 0, tot = 0, p64 = 0, p32 = 0;
  double f64 = 0.0, f32 = 0.0, g64 = 0.0, g32 = 0.0;
  if (i < npair) {
    int X = 0;
    while (a.cls_first[X + 1] <= i) ++X;
    const int m = a.pair_mol ? a.pair_mol[i] : 0;
    const double Qi = a.Q[i];
    const int nppi = a.ppn[i];
    for (int Y = 0; Y <= X; ++Y) {
      const int cp = cp_index(X, Y);
      for (int k = 0; k < NBK; ++k) {
        const int g = (Y * a.nmol + m) * NBK + k;
        const int f = a.bseg_first[g];
        int n = a.bseg_first[g + 1] - f;
        // same class: kets at or before the bra in pair order (ab >= cd once)
        if (Y == X) n = max(0, min(n, i - f + 1));
        const int keep = count_prefix(a.Q, f, n, Qi, a.thresh);
        int n64 = keep;
        if (a.mixed) n64 = min(keep, count_prefix(a.Q, f, n, Qi, a.split));
        const long long o = a.cnt_off[cp] + (long long)(i - a.cls_first[X]) * NBK + k;
        a.cnt64[o] = n64;
        a.cnt32[o] = keep - n64;
        a.kst64[o] = f - a.cls_first[Y];
        a.kst32[o] = f - a.cls_first[Y] + n64;
        q64 += n64; q32 += keep - n64; tot += n;
        const unsigned long long s64 = a.cumppn[f + n64] - a.cumppn[f];
        const unsigned long long s32 = a.cumppn[f + keep] - a.cumppn[f + n64];
        p64 += s64 * nppi; p32 += s32 * nppi;
        f64 += (double)a.f_pq[cp] * nppi * s64 + ((double)a.f_bra[cp] * nppi + a.f_q[cp]) * n64;
        f32 += (double)a.f_pq[cp] * nppi * s32 + ((double)a.f_bra[cp] * nppi + a.f_q[cp]) * (keep - n64);
        g64 += (double)a.f_q[cp] * n64;
        g32 += (double)a.f_q[cp] * (keep - n64);
      }
    }
  }
  // warp-reduce the statistics, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    q64 += __shfl_down_sync(0xffffffffu, q64, o);
    q32 += __shfl_down_sync(0xffffffffu, q32, o);
    tot += __shfl_down_sync(0xffffffffu, tot, o);
    p64 += __shfl_down_sync(0xffffffffu, p64, o);
    p32 += __shfl_down_sync(0xffffffffu, p32, o);
    f64 += __shfl_down_sync(0xffffffffu, f64, o);
    f32 += __shfl_down_sync(0xffffffffu, f32, o);
    g64 += __shfl_down_sync(0xffffffffu, g64, o);
    g32 += __shfl_down_sync(0xffffffffu, g32, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(a.stats + 0, q64); atomicAdd(a.stats + 1, q32); atomicAdd(a.stats + 2, tot);
    atomicAdd(a.stats + 3, p64); atomicAdd(a.stats + 4, p32);
    atomicAdd(a.stats + 5, (unsigned long long)f64); atomicAdd(a.stats + 6, (unsigned long long)f32);
    atomicAdd(a.stats + 7, (unsigned long long)g64); atomicAdd(a.stats + 8, (unsigned long long)g32);
  }
}

// ---------------------------------------------------------------------------
// Algorithmic arithmetic of one class's ERI + digestion work (FMA = 2 flops),
// used only for the reported FLOP/s.  It counts the sparse McMurchie-Davidson
// formulation the kernels evaluate:
//   per primitive quartet: the ket transform, 2 NHAB flops per (tau, nu, phi)
//     term of every ket component, plus 2.39 per term for its E products;
//     the Hermite integrals, 1.42 per entry of the layers 1..L; the Boys
//     function, prefactors and ket E tables, 35.5 + 9.6 L;
//   per bra primitive: the bra transform, 2 NCD flops per (t, u, v) term of
//     every bra component, plus 2.08 per term for its E products;
//   per contracted quartet: the digestion, 12 flops per Cartesian integral.
// The fractional coefficients were fitted to the FP64 instruction counts
// (DFMA x 2 + DMUL + DADD, ncu) of the small-class kernel, which executes
// exactly this formulation, on the 60-atom molecule (every class within
// 4.5 %); the cooperative and warp kernels execute 10-25 % more than this
// count (lane-local recomputation), so FLOP/s from it is conservative there.
struct ClassFlops { double per_pq, per_bra, per_q; };

static int herm_count(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }

static ClassFlops class_flops(int la, int lb, int lc, int ld) {
  const int NB = ncart(lb), ND = ncart(ld);
  const int NAB = ncart(la) * NB, NCD = ncart(lc) * ND;
  const int L = la + lb + lc + ld, NHAB = herm_count(la + lb);
  auto pows = [](int l, int k, int* p) {
    int i = l, off = 0;
    while (k >= off + (l - i + 1)) { off += l - i + 1; --i; }
    p[0] = i; p[2] = k - off; p[1] = l - p[0] - p[2];
  };
  double kterms = 0, bterms = 0, rr = 0;
  for (int kc = 0; kc < NCD; ++kc) {
    int c[3], d[3];
    pows(lc, kc / ND, c); pows(ld, kc % ND, d);
    kterms += (double)(c[0] + d[0] + 1) * (c[1] + d[1] + 1) * (c[2] + d[2] + 1);
  }
  for (int ab = 0; ab < NAB; ++ab) {
    int a[3], b[3];
    pows(la, ab / NB, a); pows(lb, ab % NB, b);
    bterms += (double)(a[0] + b[0] + 1) * (a[1] + b[1] + 1) * (a[2] + b[2] + 1);
  }
  for (int k = 1; k <= L; ++k) rr += herm_count(k);
  ClassFlops f;
  f.per_pq = 35.5 + 9.6 * L + 1.42 * rr + (2.39 + 2.0 * NHAB) * kterms;
  f.per_bra = (2.08 + 2.0 * NCD) * bterms;
  f.per_q = 12.0 * NAB * NCD;
  return f;
}

// Exclusive prefix sums of the per-bra counts of every (class pair, band):
// one block per segment, 1024-element tiles with a block scan.
struct ScanArgs {
  long long cnt_off[NCP];
  long long pre_off[NCP];
  int nseg[NCP];            // NBK x bras of the class pair
  const int* cnt64;
  const int* cnt32;
  long long* pre64;
  long long* pre32;
};

__global__ void __launch_bounds__(1024) k_scan(ScanArgs a) {
  const int seg = blockIdx.x >> 1, band = blockIdx.x & 1;
  const int n = a.nseg[seg];
  const int* cnt = (band ? a.cnt32 : a.cnt64) + a.cnt_off[seg];
  long long* pre = (band ? a.pre32 : a.pre64) + a.pre_off[seg];
  __shared__ long long warp_sums[32];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int base = 0; base < n; base += blockDim.x) {
    const int i = base + threadIdx.x;
    long long v = (i < n) ? cnt[i] : 0;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
      long long s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      warp_sums[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    const long long before = carry + (wid > 0 ? warp_sums[wid - 1] : 0);
    if (i < n) pre[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) pre[n] = carry;
}

// ---------------------------------------------------------------------------
// a7: spherical <-> Cartesian transforms (block-diagonal T, rows m, columns
// Cartesian components), on packed per-molecule blocks:
//   D_cart = T^T D T,   X_out = T sym(X_cart) T^T,   sym(X) = (X + X^T) / 2.
struct XformArgs {
  int nmol, spherical;
  const long long* cbase;   // [nmol+1] packed Cartesian offsets
  const long long* obase;   // [nmol+1] packed output offsets
  const int* nc;            // [nmol]
  const int* nbf;           // [nmol]
  const int* cf_off;        // [nmol+1] Cartesian function offsets
  const int* f_off;         // [nmol+1] output function offsets
  const int* cshell;        // Cartesian function -> shell
  const int* ccomp;
  const int* fshell;        // output function -> shell
  const int* fcomp;
  const int* shell_l;
  const int* shell_coff;    // local Cartesian offset of a shell inside its molecule
  const int* shell_soff;    // local output offset
};

__device__ __forceinline__ int find_mol(const long long* base, int nmol, long long g) {
  int lo = 0, hi = nmol;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_d_to_cart(XformArgs x, long long total, const double* __restrict__ D, double* Dc, float* Dc32) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int m = find_mol(x.cbase, x.nmol, g);
  const long long loc = g - x.cbase[m];
  const int nc = x.nc[m], nb = x.nbf[m];
  const int i = (int)(loc / nc), j = (int)(loc % nc);
  const double* Dm = D + x.obase[m];
  double v;
  if (!x.spherical) {
    v = Dm[(long long)i * nb + j];
  } else {
    const int gi = x.cf_off[m] + i, gj = x.cf_off[m] + j;
    const int sa = x.cshell[gi], sb = x.cshell[gj], ka = x.ccomp[gi], kb = x.ccomp[gj];
    const int la = x.shell_l[sa], lb = x.shell_l[sb];
    const int oa = x.shell_soff[sa], ob = x.shell_soff[sb];
    v = 0.0;
    for (int mm = 0; mm < 2 * la + 1; ++mm) {
      const double ta = c_sph[la][mm][ka];
      if (ta == 0.0) continue;
      double s = 0.0;
      for (int mn = 0; mn < 2 * lb + 1; ++mn) s += c_sph[lb][mn][kb] * Dm[(long long)(oa + mm) * nb + ob + mn];
      v += ta * s;
    }
  }
  Dc[g] = v;
  Dc32[g] = (float)v;
}

__global__ void k_from_cart(XformArgs x, long long total, const double* __restrict__ Jc,
                            const double* __restrict__ Kc, double* J, double* K) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int m = find_mol(x.obase, x.nmol, g);
  const long long loc = g - x.obase[m];
  const int nc = x.nc[m], nb = x.nbf[m];
  const int I = (int)(loc / nb), Jn = (int)(loc % nb);
  const double* Jm = Jc + x.cbase[m];
  const double* Km = Kc + x.cbase[m];
  if (!x.spherical) {
    J[g] = 0.5 * (Jm[(long long)I * nc + Jn] + Jm[(long long)Jn * nc + I]);
    K[g] = 0.5 * (Km[(long long)I * nc + Jn] + Km[(long long)Jn * nc + I]);
    return;
  }
  const int gi = x.f_off[m] + I, gj = x.f_off[m] + Jn;
  const int sa = x.fshell[gi], sb = x.fshell[gj], ma = x.fcomp[gi], mb = x.fcomp[gj];
  const int la = x.shell_l[sa], lb = x.shell_l[sb];
  const int oa = x.shell_coff[sa], ob = x.shell_coff[sb];
  double vj = 0.0, vk = 0.0;
  for (int ka = 0; ka < ncart(la); ++ka) {
    const double ta = c_sph[la][ma][ka];
    if (ta == 0.0) continue;
    double sj = 0.0, sk = 0.0;
    for (int kb = 0; kb < ncart(lb); ++kb) {
      const double tb = c_sph[lb][mb][kb];
      const long long p = (long long)(oa + ka) * nc + ob + kb, q = (long long)(ob + kb) * nc + oa + ka;
      sj += tb * (Jm[p] + Jm[q]);
      sk += tb * (Km[p] + Km[q]);
    }
    vj += ta * sj;
    vk += ta * sk;
  }
  J[g] = 0.5 * vj;
  K[g] = 0.5 * vk;
}

// a8: E = 1/2 sum D J - 1/4 sum D K over one molecule's block (one block of
// threads per molecule, grid-stride inside the block).
__global__ void k_energy(const long long* __restrict__ obase, const double* __restrict__ D,
                         const double* __restrict__ J, const double* __restrict__ K, double* E) {
  const int m = blockIdx.y;
  const long long lo = obase[m], hi = obase[m + 1];
  double s = 0.0;
  for (long long g = lo + (long long)blockIdx.x * blockDim.x + threadIdx.x; g < hi;
       g += (long long)gridDim.x * blockDim.x)
    s += D[g] * (0.5 * J[g] - 0.25 * K[g]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(E + m, s);
  }
}

// D validation over the packed blocks: max|D|, max|D - D^T|, non-finite flag.
__global__ void k_check_d(XformArgs x, long long total, const double* __restrict__ D, double* scal, int* status) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, d = 0.0;
  int bad = 0;
  if (g < total) {
    const int m = find_mol(x.obase, x.nmol, g);
    const long long loc = g - x.obase[m];
    const int nb = x.nbf[m];
    const int i = (int)(loc / nb), j = (int)(loc % nb);
    const double v = D[g], w = D[x.obase[m] + (long long)j * nb + i];
    if (!isfinite(v)) bad = 1;
    a = fabs(v);
    d = fabs(v - w);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_down_sync(0xffffffffu, a, o));
    d = fmax(d, __shfl_down_sync(0xffffffffu, d, o));
    bad |= __shfl_down_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long*)&scal[1], (unsigned long long)__double_as_longlong(a));
    atomicMax((unsigned long long*)&scal[2], (unsigned long long)__double_as_longlong(d));
    if (bad) atomicCAS(status, 0, ADFT_ERR_NONFINITE);
  }
}

static int num_sms() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static XformArgs xform_args(const adft_basis* b) {
  XformArgs x;
  x.nmol = b->nmol; x.spherical = b->spherical;
  x.cbase = b->d_mol_cbase; x.obase = b->d_mol_obase; x.nc = b->d_mol_nc; x.nbf = b->d_mol_nbf;
  x.cf_off = b->d_mol_cf_off; x.f_off = b->d_mol_f_off;
  x.cshell = b->d_cfunc_shell; x.ccomp = b->d_cfunc_comp; x.fshell = b->d_func_shell; x.fcomp = b->d_func_comp;
  x.shell_l = b->d_shell_l; x.shell_coff = b->d_shell_coff; x.shell_soff = b->d_shell_soff;
  return x;
}

// ---------------------------------------------------------------------------
// one call: validation, D -> Cartesian, screening and work lists

static int prepare(adft_basis* b, const double* D, const adft_opts* o, cudaStream_t s) {
  Workspace& w = b->ws;
  b->ev_valid = 0;
  ADFT_CUDA(cudaEventRecord(b->ev[0], s));
  const long long nc2 = b->mol_cbase[b->nmol], nb2 = b->mol_obase[b->nmol];
  const int T256 = 256;
  const XformArgs x = xform_args(b);
  ADFT_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), s));
  ADFT_CUDA(cudaMemsetAsync(w.scal, 0, 4 * sizeof(double), s));
  if (o->check) {
    k_check_d<<<(unsigned)((nb2 + T256 - 1) / T256), T256, 0, s>>>(x, nb2, D, w.scal, w.status);
    ADFT_CUDA(cudaGetLastError());
  }
  k_d_to_cart<<<(unsigned)((nc2 + T256 - 1) / T256), T256, 0, s>>>(x, nc2, D, w.Dc, w.Dc32);
  ADFT_CUDA(cudaGetLastError());
  ADFT_CUDA(cudaMemsetAsync(w.Jc, 0, nc2 * sizeof(double), s));
  ADFT_CUDA(cudaMemsetAsync(w.Kc, 0, nc2 * sizeof(double), s));
  ADFT_CUDA(cudaMemsetAsync(w.counters, 0, 6 * NCP * sizeof(unsigned long long), s));
  ADFT_CUDA(cudaMemsetAsync(w.stats, 0, 10 * sizeof(unsigned long long), s));
  ADFT_CUDA(cudaMemsetAsync(w.work, 0, 4 * NCP * sizeof(unsigned long long), s));
  b->work_valid = false;

  ScreenArgs sa;
  memcpy(sa.cls_first, b->cls_first, sizeof(sa.cls_first));
  memcpy(sa.cnt_off, b->cnt_off, sizeof(sa.cnt_off));
  sa.nmol = b->nmol;
  sa.bseg_first = b->d_bseg_first;
  sa.pair_mol = b->nmol > 1 ? b->d_pair_mol : nullptr;
  sa.Q = b->d_pair_Q; sa.ppn = b->d_pair_ppn; sa.cumppn = b->d_cumppn;
  sa.thresh = o->thresh;
  sa.mixed = is_mixed(o->precision);
  sa.split = sa.mixed ? o->split : 0.0;
  sa.cnt64 = w.cnt64; sa.cnt32 = w.cnt32; sa.kst64 = w.kst64; sa.kst32 = w.kst32; sa.stats = w.stats;
  for (int X = 0; X < NCLS; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      const ClassFlops f = class_flops(cls_la(X), cls_lb(X), cls_la(Y), cls_lb(Y));
      const int cp = cp_index(X, Y);
      sa.f_pq[cp] = (float)f.per_pq; sa.f_bra[cp] = (float)f.per_bra; sa.f_q[cp] = (float)f.per_q;
    }
  if (b->npair > 0) {
    k_screen<<<(b->npair + T256 - 1) / T256, T256, 0, s>>>(sa, b->npair);
    ADFT_CUDA(cudaGetLastError());
  }
  ScanArgs sc;
  for (int X = 0; X < NCLS; ++X)
    for (int Y = 0; Y <= X; ++Y) {
      const int cp = cp_index(X, Y);
      sc.cnt_off[cp] = b->cnt_off[cp];
      sc.pre_off[cp] = b->pre_off[cp];
      sc.nseg[cp] = NBK * (b->cls_first[X + 1] - b->cls_first[X]);
    }
  sc.cnt64 = w.cnt64; sc.cnt32 = w.cnt32; sc.pre64 = w.pre64; sc.pre32 = w.pre32;
  k_scan<<<2 * NCP, 1024, 0, s>>>(sc);
  ADFT_CUDA(cudaGetLastError());
  ADFT_CUDA(cudaEventRecord(b->ev[1], s));
  b->last_stream = s;
  return ADFT_OK;
}

static JKLaunch base_launch(adft_basis* b) {
  Workspace& w = b->ws;
  JKLaunch L;
  L.bv = view(b);
  L.D64 = w.Dc; L.D32 = w.Dc32; L.J = w.Jc; L.K = w.Kc;
  L.abort_flag = w.status + 1;
  L.status = w.status;
  L.prim_eps = 0.0;
  L.work = nullptr;
  L.omega2 = 0.0;
  return L;
}

// Launch one kernel per class pair and band, all FP64 kernels first, then the
// FP32 ones; events ev[2], ev[3] close the two groups.  pass selects the work
// counters (0: J/K, 1: gradient after J/K in the same call).
template <typename Fn>
static int for_each_class_pair(adft_basis* b, const adft_opts* o, JKLaunch L, cudaStream_t s, int pass, Fn fn) {
  Workspace& w = b->ws;
  for (int band = 0; band < (is_mixed(o->precision) ? 2 : 1); ++band) {
    for (int X = NCLS - 1; X >= 0; --X)
      for (int Y = X; Y >= 0; --Y) {
        const int nX = b->cls_first[X + 1] - b->cls_first[X];
        const int nY = b->cls_first[Y + 1] - b->cls_first[Y];
        if (nX == 0 || nY == 0) continue;
        const int cp = cp_index(X, Y);
        if (o->pair_mask && !o->pair_mask[band * NCP + cp]) continue;  // another rank's share
        L.bra_first = b->cls_first[X]; L.nseg = NBK * nX; L.ket_first = b->cls_first[Y];
        L.same_class = (X == Y);
        L.prefix = (band ? w.pre32 : w.pre64) + b->pre_off[cp];
        L.ket_start = (band ? w.kst32 : w.kst64) + b->cnt_off[cp];
        L.counter = w.counters + 2 * NCP * pass + 2 * cp + band;
        L.prim_eps = PRIM_QUARTET_FRAC * o->thresh;
        L.omega2 = o->omega * o->omega;
        L.work = w.work + 2 * (band * NCP + cp);
        const int grid = b->sms * b->tune_blocks[band][cp];
        cudaError_t e = fn(X, Y, L, band, grid, b->tune_variant[band][cp]);
        if (e != cudaSuccess) {
          set_error(std::string(band ? "fp32" : "fp64") + " launch: " + cudaGetErrorString(e));
          return ADFT_ERR_CUDA;
        }
      }
    ADFT_CUDA(cudaEventRecord(b->ev[2 + band], s));
  }
  if (!is_mixed(o->precision)) ADFT_CUDA(cudaEventRecord(b->ev[3], s));
  return ADFT_OK;
}

static int run_jk(adft_basis* b, const double* D, const adft_opts* o, cudaStream_t s) {
  int st = prepare(b, D, o, s);
  if (st) return st;
  b->work_valid = true;
  return for_each_class_pair(b, o, base_launch(b), s, 0,
                             [&](int X, int Y, const JKLaunch& L, int band, int grid, int variant) {
    return band == 1 ? launch_jk_fp32(X, Y, L, grid, variant, s) : launch_jk_fp64(X, Y, L, grid, variant, s);
  });
}

static int run_grad(adft_basis* b, const adft_opts* o, cudaStream_t s, double* grad, int pass) {
  ADFT_CUDA(cudaMemsetAsync(grad, 0, 3 * sizeof(double) * b->natom, s));
  // counter sets: 0 J/K, 1 the first gradient pass after J/K in the same call
  // (or the autotuner), 2 the second (swapped) gradient pass
  return for_each_class_pair(b, o, base_launch(b), s, pass, [&](int X, int Y, const JKLaunch& L, int band, int, int) {
    GradLaunch g;
    g.jk = L;
    g.grad = grad;
    g.counter2 = b->ws.counters + 4 * NCP + 2 * cp_index(X, Y) + band;
    return band == 0 ? launch_grad_fp64(X, Y, g, b->sms, s) : launch_grad_fp32(X, Y, g, b->sms, s);
  });
}

static int output_jk(adft_basis* b, cudaStream_t s, double* J, double* K) {
  const long long nb2 = b->mol_obase[b->nmol];
  k_from_cart<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(xform_args(b), nb2, b->ws.Jc, b->ws.Kc, J, K);
  ADFT_CUDA(cudaGetLastError());
  return ADFT_OK;
}

static int output_energy(adft_basis* b, cudaStream_t s, const double* D, const double* J, const double* K,
                         double* E) {
  ADFT_CUDA(cudaMemsetAsync(E, 0, sizeof(double) * b->nmol, s));
  const long long per = b->mol_obase[b->nmol] / b->nmol;
  const int bx = (int)std::min<long long>(std::max<long long>(1, per / (256 * 64)), (long long)b->sms * 4);
  k_energy<<<dim3(bx, b->nmol), 256, 0, s>>>(b->d_mol_obase, D, J, K, E);
  ADFT_CUDA(cudaGetLastError());
  return ADFT_OK;
}

static int finish_check(adft_basis* b, const adft_opts* o, cudaStream_t s) {
  if (!o->check) return ADFT_OK;
  int st = 0;
  double scal[4];
  ADFT_CUDA(cudaMemcpyAsync(&st, b->ws.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  ADFT_CUDA(cudaMemcpyAsync(scal, b->ws.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ADFT_CUDA(cudaStreamSynchronize(s));
  if (st != 0) {
    set_error(st == ADFT_ERR_NONFINITE ? "D holds NaN or Inf" : st == ADFT_ERR_ABORTED ? "aborted" : "device status set");
    return st;
  }
  if (scal[2] > 1e-12 * scal[1]) {
    char buf[160];
    snprintf(buf, sizeof buf, "D is not symmetric: max|D-D^T| = %.3e, max|D| = %.3e", scal[2], scal[1]);
    set_error(buf);
    return ADFT_ERR_ASYM_D;
  }
  return ADFT_OK;
}

static int check_opts(const adft_opts* o) {
  if (!o) { set_error("opts is NULL"); return ADFT_ERR_ARG; }
  if (!(o->thresh >= 0.0) || !isfinite(o->thresh)) { set_error("thresh must be finite and >= 0"); return ADFT_ERR_ARG; }
  // Basis creation drops primitive pairs whose bound product is at most
  // PRIM_EPS = 1e-15; that stays within 1e-3 of the threshold only for
  // thresh >= 1e-12, so smaller thresholds (including 0) cannot be honoured.
  if (o->thresh < 1e-12) {
    set_error("thresh must be >= 1e-12 (primitive pairs with bound products <= 1e-15 are dropped at basis creation)");
    return ADFT_ERR_ARG;
  }
  if (o->precision != ADFT_PREC_FP64 && o->precision != ADFT_PREC_MIXED) {
    set_error("precision must be ADFT_PREC_FP64 or ADFT_PREC_MIXED");
    return ADFT_ERR_ARG;
  }
  if (is_mixed(o->precision) && (!(o->split >= 0.0) || !isfinite(o->split))) {
    set_error("split must be finite and >= 0");
    return ADFT_ERR_ARG;
  }
  if (o->check != 0 && o->check != 1) { set_error("check must be 0 or 1"); return ADFT_ERR_ARG; }
  if (!(o->omega >= 0.0) || !isfinite(o->omega)) { set_error("omega must be finite and >= 0"); return ADFT_ERR_ARG; }
  return ADFT_OK;
}

static int set_device(adft_basis* b) {
  int cur = 0;
  ADFT_CUDA(cudaGetDevice(&cur));
  if (cur != b->device) { set_error("the basis was created on another CUDA device"); return ADFT_ERR_ARG; }
  return ADFT_OK;
}

// ---------------------------------------------------------------------------
// basis construction (one molecule or a batch of molecules)

struct HostMol {
  const double* xyz;
  int natom;
  std::vector<int> l, atom, nprim;        // per shell, atom local to the molecule
  std::vector<double> exps, ncoefs;       // per primitive, ncoefs = c_i N(a_i, l)
};

static int build_basis(adft_basis* b, const std::vector<HostMol>& mols, int spherical) {
  int st = ADFT_OK;
  b->nmol = (int)mols.size();
  b->spherical = spherical;
  b->sms = 0;
  if (cudaGetDevice(&b->device) != cudaSuccess) { set_error("no CUDA device"); return ADFT_ERR_CUDA; }
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
  if (b->sms <= 0) b->sms = 152;
  // ---- shells and per-molecule offsets
  b->mol_atom_off.assign(1, 0); b->mol_shell_off.assign(1, 0); b->mol_cf_off.assign(1, 0); b->mol_f_off.assign(1, 0);
  b->mol_cbase.assign(1, 0); b->mol_obase.assign(1, 0);
  int poff = 0;
  for (int m = 0; m < b->nmol; ++m) {
    const HostMol& M = mols[m];
    b->xyz.insert(b->xyz.end(), M.xyz, M.xyz + 3 * M.natom);
    int coff = 0, soff = 0, q = 0;
    for (size_t s = 0; s < M.l.size(); ++s) {
      const int l = M.l[s];
      b->shell_l.push_back(l);
      b->shell_atom.push_back(b->mol_atom_off[m] + M.atom[s]);
      b->shell_nprim.push_back(M.nprim[s]);
      b->shell_poff.push_back(poff);
      b->shell_coff.push_back(coff);
      b->shell_soff.push_back(spherical ? soff : coff);
      b->shell_mol.push_back(m);
      for (int i = 0; i < M.nprim[s]; ++i) {
        b->exps.push_back(M.exps[q + i]);
        b->ncoefs.push_back(M.ncoefs[q + i]);
      }
      q += M.nprim[s];
      poff += M.nprim[s];
      coff += ncart(l);
      soff += 2 * l + 1;
    }
    const int nbf = spherical ? soff : coff;
    b->mol_nc.push_back(coff);
    b->mol_nbf.push_back(nbf);
    b->mol_atom_off.push_back(b->mol_atom_off[m] + M.natom);
    b->mol_shell_off.push_back(b->mol_shell_off[m] + (int)M.l.size());
    b->mol_cf_off.push_back(b->mol_cf_off[m] + coff);
    b->mol_f_off.push_back(b->mol_f_off[m] + nbf);
    b->mol_cbase.push_back(b->mol_cbase[m] + (long long)coff * coff);
    b->mol_obase.push_back(b->mol_obase[m] + (long long)nbf * nbf);
  }
  b->natom = b->mol_atom_off[b->nmol];
  b->nshell = b->mol_shell_off[b->nmol];
  b->ncart = b->mol_cf_off[b->nmol];
  b->nbf = b->mol_f_off[b->nmol];

  // ---- pairs inside each molecule: class-major, molecule-minor (l_a >= l_b; ties: larger index first)
  std::vector<std::vector<std::vector<std::pair<int, int>>>> by(NCLS, std::vector<std::vector<std::pair<int, int>>>(b->nmol));
  for (int m = 0; m < b->nmol; ++m)
    for (int a = b->mol_shell_off[m]; a < b->mol_shell_off[m + 1]; ++a)
      for (int c = b->mol_shell_off[m]; c <= a; ++c) {
        int x = a, y = c;
        if (b->shell_l[y] > b->shell_l[x]) std::swap(x, y);
        by[cls_of(b->shell_l[x], b->shell_l[y])][m].push_back({x, y});
      }
  std::vector<int> pa, pb, pmol;
  b->seg_first.assign(NCLS * (b->nmol + 1), 0);
  for (int X = 0; X < NCLS; ++X) {
    b->cls_first[X] = (int)pa.size();
    for (int m = 0; m < b->nmol; ++m) {
      b->seg_first[X * (b->nmol + 1) + m] = (int)pa.size();
      for (auto& pr : by[X][m]) { pa.push_back(pr.first); pb.push_back(pr.second); pmol.push_back(m); }
    }
    b->seg_first[X * (b->nmol + 1) + b->nmol] = (int)pa.size();
  }
  b->cls_first[NCLS] = (int)pa.size();
  b->npair = (int)pa.size();

  st = boys_tables(&b->boys64, &b->boys32);
  if (st != cudaSuccess) { set_error("Boys table upload failed"); return ADFT_ERR_CUDA; }
  {
    double h_sph[LMAX + 1][2 * LMAX + 1][SPH_MAXC];
    sph_coefficients(h_sph);
    if (cudaMemcpyToSymbol(c_sph, h_sph, sizeof(h_sph)) != cudaSuccess) {
      set_error("spherical coefficient upload failed");
      return ADFT_ERR_CUDA;
    }
  }
  if ((st = upload(b, &b->d_shell_l, b->shell_l)) || (st = upload(b, &b->d_shell_atom, b->shell_atom)) ||
      (st = upload(b, &b->d_shell_coff, b->shell_coff)) || (st = upload(b, &b->d_shell_soff, b->shell_soff)) ||
      (st = upload(b, &b->d_shell_nprim, b->shell_nprim)) || (st = upload(b, &b->d_shell_poff, b->shell_poff)) ||
      (st = upload(b, &b->d_xyz, b->xyz)) || (st = upload(b, &b->d_exps, b->exps)) ||
      (st = upload(b, &b->d_ncoefs, b->ncoefs)) || (st = upload(b, &b->d_mol_nc, b->mol_nc)) ||
      (st = upload(b, &b->d_mol_nbf, b->mol_nbf)) || (st = upload(b, &b->d_mol_cf_off, b->mol_cf_off)) ||
      (st = upload(b, &b->d_mol_f_off, b->mol_f_off)) || (st = upload(b, &b->d_mol_cbase, b->mol_cbase)) ||
      (st = upload(b, &b->d_mol_obase, b->mol_obase)))
    return st;
  {
    std::vector<int> fs, fc, cs, cc;
    for (int s = 0; s < b->nshell; ++s) {
      const int l = b->shell_l[s];
      for (int k = 0; k < ncart(l); ++k) { cs.push_back(s); cc.push_back(k); }
      const int nf = spherical ? 2 * l + 1 : ncart(l);
      for (int k = 0; k < nf; ++k) { fs.push_back(s); fc.push_back(k); }
    }
    if ((st = upload(b, &b->d_func_shell, fs)) || (st = upload(b, &b->d_func_comp, fc)) ||
        (st = upload(b, &b->d_cfunc_shell, cs)) || (st = upload(b, &b->d_cfunc_comp, cc)))
      return st;
  }

  // ---- a1/a2: pair data with every primitive pair, bounds Q_ab and Q_p;
  // then sort each (class, molecule) segment by Q descending, drop primitive
  // pairs with Q_p * max(Q_p) <= PRIM_EPS and rebuild in that order.
  auto build = [&](const std::vector<int>& A, const std::vector<int>& B, const std::vector<int>& src,
                   const std::vector<int>& ppoff, const std::vector<int>& ppn, bool first, int* pp_pair_dev) -> int {
    const long long tot = (long long)src.size();
    b->npp = tot;
    int r;
    if (first) {
      if ((r = dalloc(b, &b->d_pair_a, A.size())) || (r = dalloc(b, &b->d_pair_b, A.size())) ||
          (r = dalloc(b, &b->d_pair_ppoff, A.size())) || (r = dalloc(b, &b->d_pair_ppn, A.size())) ||
          (r = dalloc(b, &b->d_pair_Q, A.size())) || (r = dalloc(b, &b->d_pair_AB, 3 * A.size())) ||
          (r = dalloc(b, &b->d_pp64, (size_t)tot)) || (r = dalloc(b, &b->d_pp32, (size_t)tot)) ||
          (r = dalloc(b, &b->d_ppw64, 2 * (size_t)tot)) || (r = dalloc(b, &b->d_ppw32, 2 * (size_t)tot)) ||
          (r = dalloc(b, &b->d_pp_src, (size_t)tot)) || (r = dalloc(b, &b->d_o2p64, (size_t)tot)) ||
          (r = dalloc(b, &b->d_o2p32, (size_t)tot)))
        return r;
    }
    ADFT_CUDA(cudaMemcpy(b->d_pair_a, A.data(), A.size() * sizeof(int), cudaMemcpyHostToDevice));
    ADFT_CUDA(cudaMemcpy(b->d_pair_b, B.data(), B.size() * sizeof(int), cudaMemcpyHostToDevice));
    ADFT_CUDA(cudaMemcpy(b->d_pair_ppoff, ppoff.data(), ppoff.size() * sizeof(int), cudaMemcpyHostToDevice));
    ADFT_CUDA(cudaMemcpy(b->d_pair_ppn, ppn.data(), ppn.size() * sizeof(int), cudaMemcpyHostToDevice));
    if (tot > 0) ADFT_CUDA(cudaMemcpy(b->d_pp_src, src.data(), src.size() * sizeof(int), cudaMemcpyHostToDevice));
    std::vector<double> ab(3 * A.size());
    for (size_t i = 0; i < A.size(); ++i)
      for (int k = 0; k < 3; ++k)
        ab[3 * i + k] = b->xyz[3 * b->shell_atom[A[i]] + k] - b->xyz[3 * b->shell_atom[B[i]] + k];
    ADFT_CUDA(cudaMemcpy(b->d_pair_AB, ab.data(), ab.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (tot > 0) {
      const int T = 256;
      k_build_pairs<<<(unsigned)((tot + T - 1) / T), T>>>((int)A.size(), b->d_pair_a, b->d_pair_b, b->d_pair_ppoff,
                                                         b->d_pp_src, b->d_shell_atom, b->d_shell_poff, b->d_xyz,
                                                         b->d_exps, b->d_ncoefs, tot, b->d_pp64, b->d_pp32,
                                                         b->d_ppw64, b->d_ppw32, b->d_o2p64, b->d_o2p32,
                                                         pp_pair_dev);
      ADFT_CUDA(cudaGetLastError());
    }
    return ADFT_OK;
  };
  std::vector<int> src, ppoff(pa.size()), ppn(pa.size());
  for (size_t i = 0; i < pa.size(); ++i) {
    ppoff[i] = (int)src.size();
    for (int x = 0; x < b->shell_nprim[pa[i]]; ++x)
      for (int y = 0; y < b->shell_nprim[pb[i]]; ++y) src.push_back((x << 8) | y);
    ppn[i] = (int)src.size() - ppoff[i];
    if (src.size() > 0x7fffffffULL) { set_error("too many primitive pairs"); return ADFT_ERR_UNSUPPORTED; }
  }
  int* d_pp_pair = nullptr;
  double* d_Qp = nullptr;
  if ((st = dalloc(b, &d_pp_pair, src.size())) || (st = dalloc(b, &d_Qp, src.size()))) return st;
  if ((st = build(pa, pb, src, ppoff, ppn, true, d_pp_pair))) return st;
  {
    BasisView v = view(b);
    v.pair_mol = nullptr;  // bounds need no packed offsets
    ADFT_CUDA(cudaMemset(b->d_pair_Q, 0, (size_t)b->npair * sizeof(double)));
    // scratch of the partial diagonals: the largest class's n * NAB * maxp
    std::vector<int> maxp(NCLS, 0);
    size_t part_n = 0;
    for (int X = 0; X < NCLS; ++X) {
      for (int i = b->cls_first[X]; i < b->cls_first[X + 1]; ++i) maxp[X] = std::max(maxp[X], ppn[i]);
      const size_t nab = (size_t)ncart(cls_la(X)) * ncart(cls_lb(X));
      part_n = std::max(part_n, (size_t)(b->cls_first[X + 1] - b->cls_first[X]) * nab * (size_t)maxp[X]);
    }
    // (freed once the bounds are read back: it is the largest temporary here)
    double* d_part = nullptr;
    if (cudaMalloc((void**)&d_part, std::max<size_t>(part_n, 1) * sizeof(double)) != cudaSuccess) {
      set_error("cudaMalloc of the Schwarz scratch failed");
      return ADFT_ERR_OOM;
    }
    struct PartFree {
      double* p;
      ~PartFree() { cudaFree(p); }
    } part_guard{d_part};
    for (int X = 0; X < NCLS; ++X) {
      const int n = b->cls_first[X + 1] - b->cls_first[X];
      if (n == 0) continue;
      cudaError_t e = launch_schwarz(X, v, b->cls_first[X], n, maxp[X], d_part, b->d_pair_Q, 0);
      if (e != cudaSuccess) { set_error(std::string("schwarz: ") + cudaGetErrorString(e)); return ADFT_ERR_CUDA; }
      const int last = b->cls_first[X + 1] - 1;
      const int npp_cls = ppoff[last] + ppn[last] - ppoff[b->cls_first[X]];
      e = launch_prim_schwarz(X, v, b->cls_first[X], n, d_pp_pair, npp_cls, d_Qp, 0);
      if (e != cudaSuccess) { set_error(std::string("prim schwarz: ") + cudaGetErrorString(e)); return ADFT_ERR_CUDA; }
    }
    std::vector<double> Q(b->npair), Qp(src.size());
    if (cudaMemcpy(Q.data(), b->d_pair_Q, Q.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (!Qp.empty() && cudaMemcpy(Qp.data(), d_Qp, Qp.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)) {
      set_error(std::string("schwarz readback: ") + cudaGetErrorString(cudaGetLastError()));
      return ADFT_ERR_CUDA;
    }
    for (double& q : Q) q = sqrt(q);  // the kernel leaves max |(mn|mn)|
    const double qpmax = Qp.empty() ? 0.0 : *std::max_element(Qp.begin(), Qp.end());
    // kept primitive pairs of every pair, then the order inside each (class,
    // molecule) segment: contraction bucket of that count, then descending Q
    std::vector<int> kept(b->npair, 0);
    for (int o = 0; o < b->npair; ++o)
      for (int k = ppoff[o]; k < ppoff[o] + ppn[o]; ++k) kept[o] += (Qp[k] * qpmax > PRIM_EPS);
    std::vector<int> idx(b->npair);
    std::iota(idx.begin(), idx.end(), 0);
    b->bseg_first.assign((size_t)NCLS * b->nmol * NBK + 1, 0);
    for (int X = 0; X < NCLS; ++X)
      for (int m = 0; m < b->nmol; ++m) {
        const int s0 = b->seg_first[X * (b->nmol + 1) + m], s1 = b->seg_first[X * (b->nmol + 1) + m + 1];
        std::stable_sort(idx.begin() + s0, idx.begin() + s1, [&](int i, int j) {
          const int bi = pp_bucket(kept[i]), bj = pp_bucket(kept[j]);
          return bi != bj ? bi < bj : Q[i] > Q[j];
        });
        int pos = s0;
        for (int k = 0; k < NBK; ++k) {
          b->bseg_first[((size_t)X * b->nmol + m) * NBK + k] = pos;
          while (pos < s1 && pp_bucket(kept[idx[pos]]) == k) ++pos;
        }
      }
    b->bseg_first[(size_t)NCLS * b->nmol * NBK] = b->npair;
    if ((st = upload(b, &b->d_bseg_first, b->bseg_first))) return st;
    std::vector<int> sa(b->npair), sb(b->npair), nsrc, nppoff(b->npair), nppn(b->npair);
    std::vector<double> nqp;  // bound of every kept primitive pair, in the new order
    b->pair_Q.resize(b->npair);
    b->npp_dense = (long long)src.size();
    for (int i = 0; i < b->npair; ++i) {
      const int o = idx[i];
      sa[i] = pa[o]; sb[i] = pb[o]; b->pair_Q[i] = Q[o];
      nppoff[i] = (int)nsrc.size();
      // kept primitive pairs by descending bound, so that the primitive
      // quartets kept by the kernels' screening are a prefix of the ket's
      std::vector<std::pair<double, int>> kp;
      for (int k = ppoff[o]; k < ppoff[o] + ppn[o]; ++k)
        if (Qp[k] * qpmax > PRIM_EPS) kp.emplace_back(Qp[k], src[k]);
      std::stable_sort(kp.begin(), kp.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
        return x.first > y.first;
      });
      for (const auto& e : kp) { nsrc.push_back(e.second); nqp.push_back(e.first); }
      nppn[i] = (int)nsrc.size() - nppoff[i];
    }
    b->pair_a = sa; b->pair_b = sb;
    if ((st = build(sa, sb, nsrc, nppoff, nppn, false, nullptr))) return st;
    {
      std::vector<float> nqp32(nqp.begin(), nqp.end());
      if ((st = upload(b, &b->d_ppq32, nqp32))) return st;
    }
    ADFT_CUDA(cudaMemcpy(b->d_pair_Q, b->pair_Q.data(), b->npair * sizeof(double), cudaMemcpyHostToDevice));
    std::vector<long long> cum(b->npair + 1, 0);
    for (int i = 0; i < b->npair; ++i) cum[i + 1] = cum[i] + nppn[i];
    if ((st = upload(b, &b->d_cumppn, cum))) return st;
    if ((st = upload(b, &b->d_pair_mol, pmol))) return st;  // pmol is unchanged by the in-segment sort
  }
  // ---- workspace
  {
    long long co = 0, po = 0;
    for (int X = 0; X < NCLS; ++X)
      for (int Y = 0; Y <= X; ++Y) {
        const int cp = cp_index(X, Y);
        const long long nseg = (long long)NBK * (b->cls_first[X + 1] - b->cls_first[X]);
        b->cnt_off[cp] = co; b->pre_off[cp] = po;
        co += nseg; po += nseg + 1;
        b->tune_blocks[0][cp] = 4;
        b->tune_blocks[1][cp] = 8;
        b->tune_variant[0][cp] = b->tune_variant[1][cp] = 0;
      }
    Workspace& w = b->ws;
    const size_t nc2 = (size_t)b->mol_cbase[b->nmol], nb2 = (size_t)b->mol_obase[b->nmol];
    if ((st = dalloc(b, &w.Dc, nc2)) || (st = dalloc(b, &w.Dc32, nc2)) || (st = dalloc(b, &w.Jc, nc2)) ||
        (st = dalloc(b, &w.Kc, nc2)) || (st = dalloc(b, &w.Jw, nb2)) || (st = dalloc(b, &w.Kw, nb2)) ||
        (st = dalloc(b, &w.cnt64, (size_t)co)) || (st = dalloc(b, &w.cnt32, (size_t)co)) ||
        (st = dalloc(b, &w.kst64, (size_t)co)) || (st = dalloc(b, &w.kst32, (size_t)co)) ||
        (st = dalloc(b, &w.pre64, (size_t)po)) || (st = dalloc(b, &w.pre32, (size_t)po)) ||
        (st = dalloc(b, &w.counters, 6 * NCP)) || (st = dalloc(b, &w.status, 4)) ||
        (st = dalloc(b, &w.scal, 4)) || (st = dalloc(b, &w.Emol, (size_t)b->nmol)) || (st = dalloc(b, &w.stats, 10)) ||
        (st = dalloc(b, &w.charges, (size_t)b->natom)) ||
        (st = dalloc(b, &w.work, 4 * NCP)))
      return st;
    ADFT_CUDA(cudaMemset(w.status, 0, 4 * sizeof(int)));
  }
  for (auto& e : b->ev) ADFT_CUDA(cudaEventCreate(&e));
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error(std::string("basis setup: ") + cudaGetErrorString(cudaGetLastError()));
    return ADFT_ERR_CUDA;
  }
  return ADFT_OK;
}

}  // namespace adft

using namespace adft;

// ===========================================================================
// C ABI

extern "C" {

const char* adft_version(void) { return "adft-gb300 0.2"; }

const char* adft_status_string(int st) {
  switch (st) {
    case ADFT_OK: return "ok";
    case ADFT_ERR_ARG: return "invalid argument";
    case ADFT_ERR_UNSUPPORTED: return "unsupported request";
    case ADFT_ERR_ASYM_D: return "density matrix is not symmetric";
    case ADFT_ERR_NONFINITE: return "density matrix holds NaN or Inf";
    case ADFT_ERR_OOM: return "out of memory";
    case ADFT_ERR_CUDA: return "CUDA runtime error";
    case ADFT_ERR_TIMEOUT: return "device wait timed out";
    case ADFT_ERR_ABORTED: return "aborted";
    default: return "unknown status";
  }
}

const char* adft_last_error_message(void) { return g_last_error.c_str(); }

void adft_basis_destroy(adft_basis* b) {
  if (!b) return;
  for (auto& e : b->ev)
    if (e) cudaEventDestroy(e);
  for (void* p : b->allocations) cudaFree(p);
  delete b;
}

int adft_basis_create(const double* atom_xyz, int natom, const adft_shell* shells, int nshell, int spherical,
                      adft_basis** out) {
  if (!out) { set_error("out is NULL"); return ADFT_ERR_ARG; }
  *out = nullptr;
  if (!atom_xyz || natom <= 0 || !shells || nshell <= 0) {
    set_error("atom_xyz/shells must be non-NULL and natom, nshell > 0");
    return ADFT_ERR_ARG;
  }
  if (spherical != 0 && spherical != 1) { set_error("spherical must be 0 or 1"); return ADFT_ERR_ARG; }
  for (int i = 0; i < 3 * natom; ++i)
    if (!isfinite(atom_xyz[i])) { set_error("atom_xyz holds a non-finite value"); return ADFT_ERR_ARG; }
  HostMol M;
  M.xyz = atom_xyz;
  M.natom = natom;
  for (int s = 0; s < nshell; ++s) {
    const adft_shell& sh = shells[s];
    if (sh.atom < 0 || sh.atom >= natom || sh.l < 0 || sh.l > ADFT_LMAX || sh.nprim < 1 ||
        sh.nprim > ADFT_MAX_NPRIM || !sh.exps || !sh.coefs) {
      char buf[128];
      snprintf(buf, sizeof buf, "shell %d: atom, l (<= %d), nprim (1..%d) or pointers invalid", s, ADFT_LMAX,
               ADFT_MAX_NPRIM);
      set_error(buf);
      return ADFT_ERR_ARG;
    }
    double df = 1.0;
    for (int k = 2 * sh.l - 1; k > 1; k -= 2) df *= k;
    for (int i = 0; i < sh.nprim; ++i) {
      if (!(sh.exps[i] > 0.0) || !isfinite(sh.exps[i]) || !isfinite(sh.coefs[i])) {
        set_error("shell exponents must be finite and > 0, coefficients finite");
        return ADFT_ERR_ARG;
      }
      const double a = sh.exps[i];
      M.exps.push_back(a);
      M.ncoefs.push_back(sh.coefs[i] * pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * sh.l) / sqrt(df));
    }
    M.l.push_back(sh.l); M.atom.push_back(sh.atom); M.nprim.push_back(sh.nprim);
  }
  adft_basis* b = new (std::nothrow) adft_basis();
  if (!b) { set_error("host allocation failed"); return ADFT_ERR_OOM; }
  const int st = build_basis(b, std::vector<HostMol>{M}, spherical);
  if (st) { adft_basis_destroy(b); return st; }
  *out = b;
  return ADFT_OK;
}

int adft_basis_nbf(const adft_basis* b, int* nbf) {
  if (!b || !nbf) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  *nbf = b->nbf;
  return ADFT_OK;
}

int adft_basis_dims(const adft_basis* b, int* natom, int* nshell, int* nc) {
  if (!b) { set_error("NULL basis"); return ADFT_ERR_ARG; }
  if (natom) *natom = b->natom;
  if (nshell) *nshell = b->nshell;
  if (nc) *nc = b->ncart;
  return ADFT_OK;
}

int adft_basis_schwarz(const adft_basis* b, double* Q) {
  if (!b || !Q) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  if (b->nmol != 1) { set_error("Schwarz bounds are reported for single-molecule bases"); return ADFT_ERR_ARG; }
  for (int i = 0; i < b->npair; ++i) {
    int x = b->pair_a[i], y = b->pair_b[i];
    if (y > x) std::swap(x, y);
    Q[(long long)x * (x + 1) / 2 + y] = b->pair_Q[i];
  }
  return ADFT_OK;
}

static int call_begin(adft_basis* b, const void* D, const adft_opts* o) {
  if (!b || !D) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  int st = check_opts(o);
  if (st) return st;
  return set_device(b);
}

int adft_jk_build(adft_basis* b, const double* D, const adft_opts* o, double* J, double* K) {
  int st = call_begin(b, D, o);
  if (st) return st;
  if (!J || !K) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = run_jk(b, D, o, s))) return st;
  if ((st = output_jk(b, s, J, K))) return st;
  ADFT_CUDA(cudaEventRecord(b->ev[4], s));
  b->ev_valid = 1;
  return finish_check(b, o, s);
}

int adft_jk_energy(adft_basis* b, const double* D, const adft_opts* o, double* E, int E_on_device) {
  int st = call_begin(b, D, o);
  if (st) return st;
  if (!E) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = run_jk(b, D, o, s))) return st;
  if ((st = output_jk(b, s, b->ws.Jw, b->ws.Kw))) return st;
  if ((st = output_energy(b, s, D, b->ws.Jw, b->ws.Kw, b->ws.Emol))) return st;
  ADFT_CUDA(cudaEventRecord(b->ev[4], s));
  b->ev_valid = 1;
  if (E_on_device) {
    ADFT_CUDA(cudaMemcpyAsync(E, b->ws.Emol, sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    ADFT_CUDA(cudaMemcpyAsync(E, b->ws.Emol, sizeof(double), cudaMemcpyDeviceToHost, s));
    ADFT_CUDA(cudaStreamSynchronize(s));
  }
  return finish_check(b, o, s);
}

int adft_jk_grad(adft_basis* b, const double* D, const adft_opts* o, double* grad) {
  int st = call_begin(b, D, o);
  if (st) return st;
  if (!grad) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  if (o->omega > 0.0) { set_error("adft_jk_grad: omega > 0 is not supported"); return ADFT_ERR_UNSUPPORTED; }
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = prepare(b, D, o, s))) return st;
  if ((st = run_grad(b, o, s, grad, 0))) return st;
  ADFT_CUDA(cudaEventRecord(b->ev[4], s));
  b->ev_valid = 1;
  return finish_check(b, o, s);
}

int adft_jk_last_stats(adft_basis* b, adft_stats* out) {
  if (!b || !out) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  unsigned long long h[10];
  ADFT_CUDA(cudaStreamSynchronize(b->last_stream));
  ADFT_CUDA(cudaMemcpy(h, b->ws.stats, sizeof(h), cudaMemcpyDeviceToHost));
  out->quartets_fp64 = (int64_t)h[0];
  out->quartets_fp32 = (int64_t)h[1];
  out->quartets_total = (int64_t)h[2];
  out->prim_quartets_fp64 = (int64_t)h[3];
  out->prim_quartets_fp32 = (int64_t)h[4];
  out->flops_fp64 = (double)h[5];
  out->flops_fp32 = (double)h[6];
  if (b->work_valid) {  // what the kernels evaluated after primitive-quartet screening
    std::vector<unsigned long long> wk(4 * NCP);
    ADFT_CUDA(cudaMemcpy(wk.data(), b->ws.work, wk.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    double fl[2] = {(double)h[7], (double)h[8]};
    unsigned long long pq[2] = {0, 0};
    for (int band = 0; band < 2; ++band)
      for (int X = 0; X < NCLS; ++X)
        for (int Y = 0; Y <= X; ++Y) {
          const int cp = cp_index(X, Y);
          const ClassFlops f = class_flops(cls_la(X), cls_lb(X), cls_la(Y), cls_lb(Y));
          const unsigned long long* c = wk.data() + 2 * (band * NCP + cp);
          pq[band] += c[0];
          fl[band] += f.per_pq * (double)c[0] + f.per_bra * (double)c[1];
        }
    out->prim_quartets_fp64 = (int64_t)pq[0];
    out->prim_quartets_fp32 = (int64_t)pq[1];
    out->flops_fp64 = fl[0];
    out->flops_fp32 = fl[1];
  }
  return ADFT_OK;
}

int adft_one_electron(adft_basis* b, const double* charges, void* stream, double* S, double* T, double* V) {
  if (!b || !charges || !S || !T || !V) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  if (b->nmol != 1) { set_error("one-electron integrals are computed for single-molecule bases"); return ADFT_ERR_ARG; }
  for (int i = 0; i < b->natom; ++i)
    if (!isfinite(charges[i])) { set_error("charges must be finite"); return ADFT_ERR_ARG; }
  int st = set_device(b);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = b->ws;
  ADFT_CUDA(cudaMemcpyAsync(w.charges, charges, sizeof(double) * b->natom, cudaMemcpyHostToDevice, s));
  BasisView v = view(b);
  ADFT_CUDA(launch_one_electron(v, b->d_shell_nprim, b->d_shell_poff, b->d_exps, b->d_ncoefs, w.charges, w.Jc, w.Kc,
                                w.Dc, s));
  if ((st = output_jk(b, s, S, T))) return st;
  const long long nb2 = b->mol_obase[b->nmol];
  k_from_cart<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(xform_args(b), nb2, w.Dc, w.Dc, V, w.Kw);
  ADFT_CUDA(cudaGetLastError());
  b->last_stream = s;
  return ADFT_OK;
}

int adft_one_electron_grad(adft_basis* b, const double* charges, const double* D, const double* W, void* stream,
                           double* grad) {
  if (!b || !charges || !D || !W || !grad) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  if (b->nmol != 1) { set_error("one-electron gradients are computed for single-molecule bases"); return ADFT_ERR_ARG; }
  for (int i = 0; i < b->natom; ++i)
    if (!isfinite(charges[i])) { set_error("charges must be finite"); return ADFT_ERR_ARG; }
  int st = set_device(b);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)stream;
  Workspace& w = b->ws;
  const long long nc2 = b->mol_cbase[b->nmol];
  const XformArgs x = xform_args(b);
  ADFT_CUDA(cudaMemcpyAsync(w.charges, charges, sizeof(double) * b->natom, cudaMemcpyHostToDevice, s));
  // D and W to Cartesian (the FP32 copy is scratch here; every build rewrites it)
  k_d_to_cart<<<(unsigned)((nc2 + 255) / 256), 256, 0, s>>>(x, nc2, D, w.Dc, w.Dc32);
  ADFT_CUDA(cudaGetLastError());
  k_d_to_cart<<<(unsigned)((nc2 + 255) / 256), 256, 0, s>>>(x, nc2, W, w.Jc, w.Dc32);
  ADFT_CUDA(cudaGetLastError());
  ADFT_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * 3 * b->natom, s));
  ADFT_CUDA(launch_one_electron_grad(view(b), b->d_shell_nprim, b->d_shell_poff, b->d_exps, b->d_ncoefs, w.charges,
                                     w.Dc, w.Jc, grad, s));
  b->last_stream = s;
  return ADFT_OK;
}

int adft_jk_last_class_stats(adft_basis* b, int64_t* quartets, int64_t* prim_quartets, int64_t* bra_prims,
                             double* flops) {
  if (!b) { set_error("NULL basis"); return ADFT_ERR_ARG; }
  ADFT_CUDA(cudaStreamSynchronize(b->last_stream));
  std::vector<unsigned long long> wk(4 * NCP, 0);
  if (b->work_valid)
    ADFT_CUDA(cudaMemcpy(wk.data(), b->ws.work, wk.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  for (int band = 0; band < 2; ++band)
    for (int X = 0; X < NCLS; ++X)
      for (int Y = 0; Y <= X; ++Y) {
        const int cp = cp_index(X, Y), o = band * NCP + cp;
        const long long nseg = (long long)NBK * (b->cls_first[X + 1] - b->cls_first[X]);
        long long q = 0;
        if (quartets && nseg > 0)
          ADFT_CUDA(cudaMemcpy(&q, (band ? b->ws.pre32 : b->ws.pre64) + b->pre_off[cp] + nseg, sizeof(q),
                               cudaMemcpyDeviceToHost));
        const unsigned long long* c = wk.data() + 2 * o;
        const ClassFlops f = class_flops(cls_la(X), cls_lb(X), cls_la(Y), cls_lb(Y));
        if (quartets) quartets[o] = q;
        if (prim_quartets) prim_quartets[o] = (int64_t)c[0];
        if (bra_prims) bra_prims[o] = (int64_t)c[1];
        if (flops) {
          long long qq = q;
          if (!quartets && nseg > 0)
            ADFT_CUDA(cudaMemcpy(&qq, (band ? b->ws.pre32 : b->ws.pre64) + b->pre_off[cp] + nseg, sizeof(qq),
                                 cudaMemcpyDeviceToHost));
          flops[o] = f.per_pq * (double)c[0] + f.per_bra * (double)c[1] + f.per_q * (double)qq;
        }
      }
  return ADFT_OK;
}

int adft_jk_last_timings(adft_basis* b, double* ms) {
  if (!b || !ms) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  if (!b->ev_valid) { set_error("no completed call to time"); return ADFT_ERR_ARG; }
  ADFT_CUDA(cudaEventSynchronize(b->ev[4]));
  for (int i = 0; i < 4; ++i) {
    float t = 0.0f;
    ADFT_CUDA(cudaEventElapsedTime(&t, b->ev[i], b->ev[i + 1]));
    ms[i] = t;
  }
  return ADFT_OK;
}

int adft_basis_set_abort(adft_basis* b, int flag) {
  if (!b) { set_error("NULL basis"); return ADFT_ERR_ARG; }
  int v = flag ? 1 : 0;
  ADFT_CUDA(cudaMemcpy(b->ws.status + 1, &v, sizeof(int), cudaMemcpyHostToDevice));
  return ADFT_OK;
}

int adft_jk_status(adft_basis* b) {
  if (!b) { set_error("NULL basis"); return ADFT_ERR_ARG; }
  int st = 0;
  ADFT_CUDA(cudaStreamSynchronize(b->last_stream));
  ADFT_CUDA(cudaMemcpy(&st, b->ws.status, sizeof(int), cudaMemcpyDeviceToHost));
  return st;
}

// ---- autotuner: kernel variant and blocks per SM of every class-pair kernel and band

// table entry of the public tuning table: blocks per SM + TUNE_VARIANT_STRIDE * variant
constexpr int TUNE_VARIANT_STRIDE = 256;

static cudaError_t launch_band(int band, int X, int Y, const JKLaunch& L, int grid, int variant, cudaStream_t s,
                               KernelInfo* info = nullptr) {
  return band == 1 ? launch_jk_fp32(X, Y, L, grid, variant, s, info)
                   : launch_jk_fp64(X, Y, L, grid, variant, s, info);
}

static void export_tuning(const adft_basis* b, int* table) {
  for (int band = 0; band < 2; ++band)
    for (int cp = 0; cp < NCP; ++cp)
      table[band * NCP + cp] = b->tune_blocks[band][cp] + TUNE_VARIANT_STRIDE * b->tune_variant[band][cp];
}

int adft_autotune(adft_basis* b, const double* D, const adft_opts* o, int* table, double* ms_out) {
  int st = call_begin(b, D, o);
  if (st) return st;
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = prepare(b, D, o, s))) return st;
  static const int cand[] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  ADFT_CUDA(cudaEventCreate(&e0));
  ADFT_CUDA(cudaEventCreate(&e1));
  if (ms_out)
    for (int i = 0; i < 2 * NCP; ++i) ms_out[i] = 0.0;
  for (int band = 0; band < (is_mixed(o->precision) ? 2 : 1); ++band)
    for (int X = NCLS - 1; X >= 0; --X)
      for (int Y = X; Y >= 0; --Y) {
        const int cp = cp_index(X, Y);
        if (b->cls_first[X + 1] == b->cls_first[X] || b->cls_first[Y + 1] == b->cls_first[Y]) continue;
        JKLaunch L = base_launch(b);
        L.bra_first = b->cls_first[X]; L.nseg = NBK * (b->cls_first[X + 1] - b->cls_first[X]);
        L.ket_first = b->cls_first[Y]; L.same_class = (X == Y);
        L.prefix = (band ? b->ws.pre32 : b->ws.pre64) + b->pre_off[cp];
        L.ket_start = (band ? b->ws.kst32 : b->ws.kst64) + b->cnt_off[cp];
        L.counter = b->ws.counters + 2 * NCP + 2 * cp + band;
        L.prim_eps = PRIM_QUARTET_FRAC * o->thresh;
        L.omega2 = o->omega * o->omega;
        KernelInfo ki{1, 1};
        ADFT_CUDA(launch_band(band, X, Y, L, 0, 0, s, &ki));
        float best = 1e30f;
        int best_c = b->tune_blocks[band][cp], best_v = b->tune_variant[band][cp];
        for (int v = 0; v < ki.variants; ++v) {
          KernelInfo kv{1, 1};
          ADFT_CUDA(launch_band(band, X, Y, L, 0, v, s, &kv));
          for (int c : cand) {
            if (c > 1 && c > kv.max_blocks_per_sm) continue;  // would not be resident at once
            ADFT_CUDA(cudaMemsetAsync(L.counter, 0, sizeof(unsigned long long), s));
            ADFT_CUDA(cudaEventRecord(e0, s));
            cudaError_t e = launch_band(band, X, Y, L, b->sms * c, v, s);
            if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return ADFT_ERR_CUDA; }
            ADFT_CUDA(cudaEventRecord(e1, s));
            ADFT_CUDA(cudaEventSynchronize(e1));
            float ms = 0.0f;
            ADFT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best * 0.97f) { best = ms; best_c = c; best_v = v; }
          }
        }
        b->tune_blocks[band][cp] = best_c;
        b->tune_variant[band][cp] = best_v;
        if (ms_out) ms_out[band * NCP + cp] = best;
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (table) export_tuning(b, table);
  return ADFT_OK;
}

int adft_jk_plan(adft_basis* b, const double* D, const adft_opts* o, adft_stats* st, int64_t* quartets) {
  int r = call_begin(b, D, o);
  if (r) return r;
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((r = prepare(b, D, o, s))) return r;
  ADFT_CUDA(cudaStreamSynchronize(s));
  if (quartets) {
    for (int band = 0; band < 2; ++band)
      for (int X = 0; X < NCLS; ++X)
        for (int Y = 0; Y <= X; ++Y) {
          const int cp = cp_index(X, Y);
          const int nX = b->cls_first[X + 1] - b->cls_first[X];
          long long v = 0;
          ADFT_CUDA(cudaMemcpy(&v, (band ? b->ws.pre32 : b->ws.pre64) + b->pre_off[cp] + (long long)NBK * nX, sizeof(v),
                               cudaMemcpyDeviceToHost));
          quartets[band * NCP + cp] = v;
        }
  }
  return st ? adft_jk_last_stats(b, st) : ADFT_OK;
}

int adft_set_tuning(adft_basis* b, const int* table) {
  if (!b || !table) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  for (int band = 0; band < 2; ++band)
    for (int X = 0; X < NCLS; ++X)
      for (int Y = 0; Y <= X; ++Y) {
        const int cp = cp_index(X, Y), t = table[band * NCP + cp];
        const int c = t % TUNE_VARIANT_STRIDE, v = t / TUNE_VARIANT_STRIDE;
        KernelInfo ki{1, 1};
        ADFT_CUDA(launch_band(band, X, Y, JKLaunch{}, 0, 0, nullptr, &ki));
        if (t < 0 || c < 1 || c > 64 || v >= ki.variants) {
          set_error("tuning entry " + std::to_string(band * NCP + cp) + ": blocks per SM must be in 1..64 and the "
                    "variant below the class pair's variant count");
          return ADFT_ERR_ARG;
        }
      }
  for (int band = 0; band < 2; ++band)
    for (int cp = 0; cp < NCP; ++cp) {
      b->tune_blocks[band][cp] = table[band * NCP + cp] % TUNE_VARIANT_STRIDE;
      b->tune_variant[band][cp] = table[band * NCP + cp] / TUNE_VARIANT_STRIDE;
    }
  return ADFT_OK;
}

// ---- batched form

int adft_batch_create(adft_basis* const* mols, int nmol, adft_batch** out) {
  if (!out || !mols || nmol <= 0) { set_error("mols/out must be non-NULL and nmol > 0"); return ADFT_ERR_ARG; }
  *out = nullptr;
  std::vector<HostMol> H(nmol);
  int spherical = -1, dev = -1;
  for (int m = 0; m < nmol; ++m) {
    const adft_basis* s = mols[m];
    if (!s || s->nmol != 1) { set_error("every batch member must be a single-molecule basis"); return ADFT_ERR_ARG; }
    if (spherical >= 0 && s->spherical != spherical) { set_error("mixed spherical/Cartesian bases"); return ADFT_ERR_ARG; }
    if (dev >= 0 && s->device != dev) { set_error("bases on different devices"); return ADFT_ERR_ARG; }
    spherical = s->spherical; dev = s->device;
    HostMol& M = H[m];
    M.xyz = s->xyz.data();
    M.natom = s->natom;
    M.l = s->shell_l; M.atom = s->shell_atom; M.nprim = s->shell_nprim;
    M.exps = s->exps; M.ncoefs = s->ncoefs;
  }
  adft_batch* bt = new (std::nothrow) adft_batch();
  if (!bt) { set_error("host allocation failed"); return ADFT_ERR_OOM; }
  bt->b = new (std::nothrow) adft_basis();
  if (!bt->b) { delete bt; set_error("host allocation failed"); return ADFT_ERR_OOM; }
  const int st = build_basis(bt->b, H, spherical);
  if (st) { adft_batch_destroy(bt); return st; }
  *out = bt;
  return ADFT_OK;
}

int adft_batch_offsets(const adft_batch* bt, int64_t* offsets) {
  if (!bt || !offsets) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  for (int m = 0; m <= bt->b->nmol; ++m) offsets[m] = bt->b->mol_obase[m];
  return ADFT_OK;
}

int adft_batch_grad_offsets(const adft_batch* bt, int64_t* offsets) {
  if (!bt || !offsets) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  for (int m = 0; m <= bt->b->nmol; ++m) offsets[m] = 3LL * bt->b->mol_atom_off[m];
  return ADFT_OK;
}



static int batch_sequence(adft_basis* b, const double* D, const adft_opts* o, cudaStream_t s, double* J, double* K,
                          double* E, double* grad) {
  int st = run_jk(b, D, o, s);
  if (st) return st;
  if ((st = output_jk(b, s, J, K))) return st;
  if (E && (st = output_energy(b, s, D, J, K, E))) return st;
  if (grad && (st = run_grad(b, o, s, grad, 1))) return st;
  ADFT_CUDA(cudaEventRecord(b->ev[4], s));
  return ADFT_OK;
}

int adft_batch_jk(adft_batch* bt, const double* D, const adft_opts* o, double* J, double* K, double* E,
                  double* grad) {
  if (!bt) { set_error("NULL batch"); return ADFT_ERR_ARG; }
  adft_basis* b = bt->b;
  int st = call_begin(b, D, o);
  if (st) return st;
  if (!J || !K) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  if (o->pair_mask) { set_error("pair_mask is for single-molecule calls; shard a batch by molecules"); return ADFT_ERR_ARG; }
  if (o->omega > 0.0) { set_error("adft_batch_jk: omega > 0 is not supported"); return ADFT_ERR_UNSUPPORTED; }
  cudaStream_t s = (cudaStream_t)o->stream;
  if (o->check || s == nullptr) {
    // direct launches (validation needs a synchronisation; the legacy
    // default stream cannot be captured)
    if ((st = batch_sequence(b, D, o, s, J, K, E, grad))) return st;
    b->ev_valid = 1;
    return finish_check(b, o, s);
  }
  // one CUDA graph per (buffers, options): captured on first use, replayed after
  auto key = std::make_tuple((const void*)D, (const void*)J, (const void*)K, (const void*)E, (const void*)grad,
                             o->thresh, o->split, o->precision, (void*)s);
  if (!bt->has_graph || bt->key != key) {
    if (bt->exec) { cudaGraphExecDestroy(bt->exec); bt->exec = nullptr; }
    if (bt->graph) { cudaGraphDestroy(bt->graph); bt->graph = nullptr; }
    bt->has_graph = false;
    ADFT_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    st = batch_sequence(b, D, o, s, J, K, E, grad);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st) { if (g) cudaGraphDestroy(g); return st; }
    if (ec != cudaSuccess) { set_error(std::string("graph capture: ") + cudaGetErrorString(ec)); return ADFT_ERR_CUDA; }
    bt->graph = g;
    ADFT_CUDA(cudaGraphInstantiate(&bt->exec, bt->graph, 0));
    bt->key = key;
    bt->has_graph = true;
  }
  ADFT_CUDA(cudaGraphLaunch(bt->exec, s));
  b->last_stream = s;
  b->ev_valid = 1;
  return ADFT_OK;
}

int adft_batch_last_stats(adft_batch* bt, adft_stats* st) {
  if (!bt) { set_error("NULL batch"); return ADFT_ERR_ARG; }
  return adft_jk_last_stats(bt->b, st);
}

int adft_batch_last_timings(adft_batch* bt, double* ms) {
  if (!bt) { set_error("NULL batch"); return ADFT_ERR_ARG; }
  return adft_jk_last_timings(bt->b, ms);
}

int adft_batch_autotune(adft_batch* bt, const double* D, const adft_opts* o, int* table, double* ms) {
  if (!bt) { set_error("NULL batch"); return ADFT_ERR_ARG; }
  if (o && o->omega > 0.0) { set_error("adft_batch_autotune: omega > 0 is not supported"); return ADFT_ERR_UNSUPPORTED; }
  if (bt->has_graph) {  // the captured graph holds the old launch shapes
    cudaGraphExecDestroy(bt->exec); cudaGraphDestroy(bt->graph);
    bt->exec = nullptr; bt->graph = nullptr; bt->has_graph = false;
  }
  return adft_autotune(bt->b, D, o, table, ms);
}

int adft_batch_set_tuning(adft_batch* bt, const int* table) {
  if (!bt) { set_error("NULL batch"); return ADFT_ERR_ARG; }
  const int st = adft_set_tuning(bt->b, table);
  if (st) return st;
  if (bt->has_graph) {  // the captured graph holds the old launch shapes
    cudaGraphExecDestroy(bt->exec); cudaGraphDestroy(bt->graph);
    bt->exec = nullptr; bt->graph = nullptr; bt->has_graph = false;
  }
  return ADFT_OK;
}

void adft_batch_destroy(adft_batch* bt) {
  if (!bt) return;
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  adft_basis_destroy(bt->b);
  delete bt;
}

}  // extern "C"
