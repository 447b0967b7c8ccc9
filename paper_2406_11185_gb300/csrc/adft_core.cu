// Host orchestration and the data-parallel setup / screening / transform
// kernels of the GB300 J/K library.  Public entry points: include/adft.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <string>
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

// ---------------------------------------------------------------------------
// basis handle

struct Workspace {
  double* Dc = nullptr;     // Cartesian D
  float* Dc32 = nullptr;
  double* Jc = nullptr;     // Cartesian accumulators
  double* Kc = nullptr;
  double* Jw = nullptr;     // J, K in the output basis (energy / gradient calls)
  double* Kw = nullptr;
  int* cnt64 = nullptr;     // per (class pair, bra) kept FP64 kets
  int* cnt32 = nullptr;     // per (class pair, bra) kept FP32 kets
  long long* pre64 = nullptr;  // per (class pair) prefix arrays
  long long* pre32 = nullptr;
  unsigned long long* counters = nullptr;  // [2 * NCP]
  int* status = nullptr;    // [4]: status, abort flag
  double* scal = nullptr;   // [4]: energy, max|D|, max|D-D^T|
  unsigned long long* stats = nullptr;     // [8]
};

}  // namespace adft

struct adft_basis {
  int device = 0;
  int natom = 0, nshell = 0, ncart = 0, nbf = 0, spherical = 1;
  std::vector<int> shell_l, shell_atom, shell_nprim, shell_poff, shell_coff, shell_soff;
  std::vector<double> xyz, exps, ncoefs;  // ncoefs: c_i N(a_i, l)
  // pairs in class order (sorted by Q descending inside each class)
  int npair = 0;
  int cls_first[adft::NCLS + 1];
  std::vector<int> pair_a, pair_b;
  std::vector<double> pair_Q;
  long long npp = 0;
  // per class pair: offset of its per-bra count arrays and its prefix array
  long long cnt_off[adft::NCP];
  long long pre_off[adft::NCP];
  long long cnt_total = 0, pre_total = 0;
  // device arrays
  int *d_shell_l = nullptr, *d_shell_atom = nullptr, *d_shell_coff = nullptr, *d_shell_soff = nullptr;
  int *d_shell_nprim = nullptr, *d_shell_poff = nullptr;
  double *d_xyz = nullptr, *d_exps = nullptr, *d_ncoefs = nullptr;
  int *d_pair_a = nullptr, *d_pair_b = nullptr, *d_pair_ppoff = nullptr, *d_pair_ppn = nullptr;
  double *d_pair_Q = nullptr, *d_pair_AB = nullptr;
  long long* d_cumppn = nullptr;
  adft::PrimPair<double>* d_pp64 = nullptr;
  adft::PrimPair<float>* d_pp32 = nullptr;
  double* d_ppw64 = nullptr;  // [2][npp] 2a, 2b
  float* d_ppw32 = nullptr;
  int *d_func_shell = nullptr, *d_func_comp = nullptr;  // output-basis function -> (shell, component)
  int *d_cfunc_shell = nullptr, *d_cfunc_comp = nullptr;  // Cartesian function -> (shell, component)
  const double* boys64 = nullptr;
  const float* boys32 = nullptr;
  adft::Workspace ws;
  cudaStream_t last_stream = nullptr;
  int last_prec = 0;
  std::vector<void*> allocations;
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
  return v;
}

// ---------------------------------------------------------------------------
// a1: primitive-pair construction, one thread per primitive pair.
__global__ void k_build_pairs(int npair, const int* __restrict__ pair_a, const int* __restrict__ pair_b,
                              const int* __restrict__ ppoff, const int* __restrict__ shell_atom,
                              const int* __restrict__ shell_nprim, const int* __restrict__ shell_poff,
                              const double* __restrict__ xyz, const double* __restrict__ exps,
                              const double* __restrict__ ncoefs, long long npp, PrimPair<double>* pp64,
                              PrimPair<float>* pp32, double* pairAB, double* w64, float* w32) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= npp) return;
  // pair owning primitive pair g (ppoff is ascending)
  int lo = 0, hi = npair;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (ppoff[mid] <= g) lo = mid; else hi = mid;
  }
  const int pr = lo, sa = pair_a[pr], sb = pair_b[pr];
  const int local = (int)(g - ppoff[pr]);
  const int nb = shell_nprim[sb];
  const int ia = local / nb, ib = local % nb;
  const double a = exps[shell_poff[sa] + ia], b = exps[shell_poff[sb] + ib];
  const double* A = xyz + 3 * shell_atom[sa];
  const double* B = xyz + 3 * shell_atom[sb];
  const double p = a + b, mu = a * b / p;
  const double ABx = A[0] - B[0], ABy = A[1] - B[1], ABz = A[2] - B[2];
  const double Px = (a * A[0] + b * B[0]) / p, Py = (a * A[1] + b * B[1]) / p, Pz = (a * A[2] + b * B[2]) / p;
  const double K = ncoefs[shell_poff[sa] + ia] * ncoefs[shell_poff[sb] + ib] *
                   exp(-mu * (ABx * ABx + ABy * ABy + ABz * ABz));
  PrimPair<double> r{Px, Py, Pz, p, Px - A[0], Py - A[1], Pz - A[2], K};
  pp64[g] = r;
  PrimPair<float> f{(float)Px, (float)Py, (float)Pz, (float)p, (float)(Px - A[0]), (float)(Py - A[1]),
                    (float)(Pz - A[2]), (float)K};
  pp32[g] = f;
  w64[g] = 2.0 * a; w64[npp + g] = 2.0 * b;
  w32[g] = (float)(2.0 * a); w32[npp + g] = (float)(2.0 * b);
  if (local == 0) {
    pairAB[3 * pr] = ABx; pairAB[3 * pr + 1] = ABy; pairAB[3 * pr + 2] = ABz;
  }
}

// ---------------------------------------------------------------------------
// a3: screening.  For every bra pair i (class X) and ket class Y <= X, the
// kept kets are a prefix of Y's list (sorted by Q descending): count those
// with Q_i Q_k >= thresh and, of them, those with Q_i Q_k >= split (FP64).
struct ScreenArgs {
  int cls_first[NCLS + 1];
  long long cnt_off[NCP];
  const double* Q;
  const int* ppn;
  const long long* cumppn;  // [npair + 1] running sum of ppn in pair order
  double thresh, split;
  int mixed;
  int* cnt64;
  int* cnt32;
  unsigned long long* stats;  // [0] q64 [1] q32 [2] total unique [3] prim64 [4] prim32
};

__device__ __forceinline__ int count_prefix(const double* Q, int first, int n, double Qi, double thr) {
  // number of leading k in [first, first+n) with Qi * Q[k] >= thr
  int lo = 0, hi = n;  // answer in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (Qi * Q[first + mid] >= thr) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_screen(ScreenArgs a, int npair) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long q64 = 0, q32 = 0, tot = 0, p64 = 0, p32 = 0;
  if (i < npair) {
    int X = 0;
    while (a.cls_first[X + 1] <= i) ++X;
    const int li = i - a.cls_first[X];
    const double Qi = a.Q[i];
    const int nppi = a.ppn[i];
    for (int Y = 0; Y <= X; ++Y) {
      const int f = a.cls_first[Y];
      int n = a.cls_first[Y + 1] - f;
      if (Y == X) n = li + 1;
      const int keep = count_prefix(a.Q, f, n, Qi, a.thresh);
      int n64 = keep;
      if (a.mixed) n64 = min(keep, count_prefix(a.Q, f, n, Qi, a.split));
      const long long o = a.cnt_off[cp_index(X, Y)] + li;
      a.cnt64[o] = n64;
      a.cnt32[o] = keep - n64;
      q64 += n64; q32 += keep - n64; tot += n;
      const unsigned long long s64 = a.cumppn[f + n64] - a.cumppn[f];
      const unsigned long long s32 = a.cumppn[f + keep] - a.cumppn[f + n64];
      p64 += s64 * nppi; p32 += s32 * nppi;
    }
  }
  // warp-reduce the statistics, one atomic per warp
  for (int o = 16; o > 0; o >>= 1) {
    q64 += __shfl_down_sync(0xffffffffu, q64, o);
    q32 += __shfl_down_sync(0xffffffffu, q32, o);
    tot += __shfl_down_sync(0xffffffffu, tot, o);
    p64 += __shfl_down_sync(0xffffffffu, p64, o);
    p32 += __shfl_down_sync(0xffffffffu, p32, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(a.stats + 0, q64); atomicAdd(a.stats + 1, q32); atomicAdd(a.stats + 2, tot);
    atomicAdd(a.stats + 3, p64); atomicAdd(a.stats + 4, p32);
  }
}

// Exclusive prefix sums of the per-bra counts of every (class pair, band):
// one block per segment, 1024-element tiles with a block scan.
struct ScanArgs {
  long long cnt_off[NCP];
  long long pre_off[NCP];
  int nbra[NCP];
  const int* cnt64;
  const int* cnt32;
  long long* pre64;
  long long* pre32;
};

__global__ void __launch_bounds__(1024) k_scan(ScanArgs a) {
  const int seg = blockIdx.x >> 1, band = blockIdx.x & 1;
  const int n = a.nbra[seg];
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
// Cartesian components): D_cart = T^T D T and X_out = T sym(X_cart) T^T.
__global__ void k_d_to_cart(int nc, int nbf, int spherical, const int* __restrict__ cshell,
                            const int* __restrict__ ccomp, const int* __restrict__ shell_l,
                            const int* __restrict__ shell_soff, const double* __restrict__ D, double* Dc,
                            float* Dc32) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)nc * nc) return;
  const int i = (int)(g / nc), j = (int)(g % nc);
  double v;
  if (!spherical) {
    v = D[(long long)i * nbf + j];
  } else {
    const int sa = cshell[i], sb = cshell[j], ka = ccomp[i], kb = ccomp[j];
    const int la = shell_l[sa], lb = shell_l[sb];
    const int oa = shell_soff[sa], ob = shell_soff[sb];
    v = 0.0;
    for (int m = 0; m < 2 * la + 1; ++m) {
      const double ta = c_sph[la][m][ka];
      if (ta == 0.0) continue;
      double s = 0.0;
      for (int mm = 0; mm < 2 * lb + 1; ++mm) s += c_sph[lb][mm][kb] * D[(long long)(oa + m) * nbf + ob + mm];
      v += ta * s;
    }
  }
  Dc[g] = v;
  Dc32[g] = (float)v;
}

__global__ void k_from_cart(int nc, int nbf, int spherical, const int* __restrict__ fshell,
                            const int* __restrict__ fcomp, const int* __restrict__ shell_l,
                            const int* __restrict__ shell_coff, const double* __restrict__ Jc,
                            const double* __restrict__ Kc, double* J, double* K) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= (long long)nbf * nbf) return;
  const int I = (int)(g / nbf), Jn = (int)(g % nbf);
  if (!spherical) {
    J[g] = 0.5 * (Jc[(long long)I * nc + Jn] + Jc[(long long)Jn * nc + I]);
    K[g] = 0.5 * (Kc[(long long)I * nc + Jn] + Kc[(long long)Jn * nc + I]);
    return;
  }
  const int sa = fshell[I], sb = fshell[Jn], ma = fcomp[I], mb = fcomp[Jn];
  const int la = shell_l[sa], lb = shell_l[sb];
  const int oa = shell_coff[sa], ob = shell_coff[sb];
  double vj = 0.0, vk = 0.0;
  for (int ka = 0; ka < ncart(la); ++ka) {
    const double ta = c_sph[la][ma][ka];
    if (ta == 0.0) continue;
    double sj = 0.0, sk = 0.0;
    for (int kb = 0; kb < ncart(lb); ++kb) {
      const double tb = c_sph[lb][mb][kb];
      const long long x = (long long)(oa + ka) * nc + ob + kb, y = (long long)(ob + kb) * nc + oa + ka;
      sj += tb * (Jc[x] + Jc[y]);
      sk += tb * (Kc[x] + Kc[y]);
    }
    vj += ta * sj;
    vk += ta * sk;
  }
  J[g] = 0.5 * vj;
  K[g] = 0.5 * vk;
}

// a8: E = 1/2 sum D J - 1/4 sum D K (block reduction, one atomic per block)
__global__ void k_energy(long long n, const double* __restrict__ D, const double* __restrict__ J,
                         const double* __restrict__ K, double* E) {
  double s = 0.0;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x)
    s += D[g] * (0.5 * J[g] - 0.25 * K[g]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(E, s);
  }
}

// D validation: max|D|, max|D - D^T| and a non-finite flag (no trap).
__global__ void k_check_d(int n, const double* __restrict__ D, double* scal, int* status) {
  const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, d = 0.0;
  int bad = 0;
  if (g < (long long)n * n) {
    const int i = (int)(g / n), j = (int)(g % n);
    const double x = D[g], y = D[(long long)j * n + i];
    if (!isfinite(x)) bad = 1;
    a = fabs(x);
    d = fabs(x - y);
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

static int grid_for(int threads_per_block, int blocks_per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  (void)threads_per_block;
  return sms * blocks_per_sm;
}

// ---------------------------------------------------------------------------
// one J/K build into the handle's Cartesian accumulators

static int prepare(adft_basis* b, const double* D, const adft_opts* o, cudaStream_t s) {
  Workspace& w = b->ws;
  const long long nc2 = (long long)b->ncart * b->ncart;
  const int T256 = 256;
  ADFT_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), s));
  ADFT_CUDA(cudaMemsetAsync(w.scal, 0, 4 * sizeof(double), s));
  if (o->check) {
    const long long nb2 = (long long)b->nbf * b->nbf;
    k_check_d<<<(unsigned)((nb2 + T256 - 1) / T256), T256, 0, s>>>(b->nbf, D, w.scal, w.status);
    ADFT_CUDA(cudaGetLastError());
  }
  k_d_to_cart<<<(unsigned)((nc2 + T256 - 1) / T256), T256, 0, s>>>(b->ncart, b->nbf, b->spherical, b->d_cfunc_shell,
                                                                  b->d_cfunc_comp, b->d_shell_l, b->d_shell_soff, D,
                                                                  w.Dc, w.Dc32);
  ADFT_CUDA(cudaGetLastError());
  ADFT_CUDA(cudaMemsetAsync(w.Jc, 0, nc2 * sizeof(double), s));
  ADFT_CUDA(cudaMemsetAsync(w.Kc, 0, nc2 * sizeof(double), s));
  ADFT_CUDA(cudaMemsetAsync(w.counters, 0, 2 * NCP * sizeof(unsigned long long), s));
  ADFT_CUDA(cudaMemsetAsync(w.stats, 0, 8 * sizeof(unsigned long long), s));

  ScreenArgs sa;
  memcpy(sa.cls_first, b->cls_first, sizeof(sa.cls_first));
  memcpy(sa.cnt_off, b->cnt_off, sizeof(sa.cnt_off));
  sa.Q = b->d_pair_Q; sa.ppn = b->d_pair_ppn; sa.cumppn = b->d_cumppn;
  sa.thresh = o->thresh;
  sa.mixed = (o->precision == ADFT_PREC_MIXED);
  sa.split = sa.mixed ? o->split : 0.0;
  sa.cnt64 = w.cnt64; sa.cnt32 = w.cnt32; sa.stats = w.stats;
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
      sc.nbra[cp] = b->cls_first[X + 1] - b->cls_first[X];
    }
  sc.cnt64 = w.cnt64; sc.cnt32 = w.cnt32; sc.pre64 = w.pre64; sc.pre32 = w.pre32;
  k_scan<<<2 * NCP, 1024, 0, s>>>(sc);
  ADFT_CUDA(cudaGetLastError());
  b->last_stream = s;
  b->last_prec = o->precision;
  return ADFT_OK;
}

static JKLaunch base_launch(adft_basis* b) {
  Workspace& w = b->ws;
  JKLaunch L;
  L.bv = view(b);
  L.D64 = w.Dc; L.D32 = w.Dc32; L.J = w.Jc; L.K = w.Kc;
  L.abort_flag = w.status + 1;
  L.status = w.status;
  return L;
}

// Launch one kernel per class pair and band; fn(X, Y, launch, band) issues it.
template <typename Fn>
static int for_each_class_pair(adft_basis* b, const adft_opts* o, JKLaunch L, Fn fn) {
  Workspace& w = b->ws;
  for (int X = NCLS - 1; X >= 0; --X)
    for (int Y = X; Y >= 0; --Y) {
      const int nX = b->cls_first[X + 1] - b->cls_first[X];
      const int nY = b->cls_first[Y + 1] - b->cls_first[Y];
      if (nX == 0 || nY == 0) continue;
      const int cp = cp_index(X, Y);
      L.bra_first = b->cls_first[X]; L.nbra = nX; L.ket_first = b->cls_first[Y];
      L.same_class = (X == Y);
      L.prefix = w.pre64 + b->pre_off[cp];
      L.ket_start = nullptr;
      L.counter = w.counters + 2 * cp;
      cudaError_t e = fn(X, Y, L, 0);
      if (e != cudaSuccess) { set_error(std::string("fp64 launch: ") + cudaGetErrorString(e)); return ADFT_ERR_CUDA; }
      if (o->precision == ADFT_PREC_MIXED) {
        L.prefix = w.pre32 + b->pre_off[cp];
        L.ket_start = w.cnt64 + b->cnt_off[cp];
        L.counter = w.counters + 2 * cp + 1;
        e = fn(X, Y, L, 1);
        if (e != cudaSuccess) { set_error(std::string("fp32 launch: ") + cudaGetErrorString(e)); return ADFT_ERR_CUDA; }
      }
    }
  return ADFT_OK;
}

static int run_jk(adft_basis* b, const double* D, const adft_opts* o, cudaStream_t s) {
  int st = prepare(b, D, o, s);
  if (st) return st;
  const int grid64 = grid_for(128, 4), grid32 = grid_for(128, 8);
  return for_each_class_pair(b, o, base_launch(b), [&](int X, int Y, const JKLaunch& L, int band) {
    return band == 0 ? launch_jk_fp64(X, Y, L, grid64, s) : launch_jk_fp32(X, Y, L, grid32, s);
  });
}

static int finish_check(adft_basis* b, const adft_opts* o, cudaStream_t s) {
  if (!o->check) return ADFT_OK;
  int st = 0;
  double scal[4];
  ADFT_CUDA(cudaMemcpyAsync(&st, b->ws.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  ADFT_CUDA(cudaMemcpyAsync(scal, b->ws.scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ADFT_CUDA(cudaStreamSynchronize(s));
  if (st != 0) {
    set_error(st == ADFT_ERR_NONFINITE ? "D holds NaN or Inf" : "device status set");
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
  if (o->precision != ADFT_PREC_FP64 && o->precision != ADFT_PREC_MIXED) {
    set_error("precision must be ADFT_PREC_FP64 or ADFT_PREC_MIXED");
    return ADFT_ERR_ARG;
  }
  if (o->precision == ADFT_PREC_MIXED && (!(o->split >= 0.0) || !isfinite(o->split))) {
    set_error("split must be finite and >= 0");
    return ADFT_ERR_ARG;
  }
  if (o->check != 0 && o->check != 1) { set_error("check must be 0 or 1"); return ADFT_ERR_ARG; }
  return ADFT_OK;
}

static int set_device(adft_basis* b) {
  int cur = 0;
  ADFT_CUDA(cudaGetDevice(&cur));
  if (cur != b->device) { set_error("the basis was created on another CUDA device"); return ADFT_ERR_ARG; }
  return ADFT_OK;
}

}  // namespace adft

using namespace adft;

// ===========================================================================
// C ABI

extern "C" {

const char* adft_version(void) { return "adft-gb300 0.1"; }

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
    for (int i = 0; i < sh.nprim; ++i)
      if (!(sh.exps[i] > 0.0) || !isfinite(sh.exps[i]) || !isfinite(sh.coefs[i])) {
        set_error("shell exponents must be finite and > 0, coefficients finite");
        return ADFT_ERR_ARG;
      }
  }
  adft_basis* b = new (std::nothrow) adft_basis();
  if (!b) { set_error("host allocation failed"); return ADFT_ERR_OOM; }
  int st = ADFT_OK;
  auto fail = [&](int code) { adft_basis_destroy(b); return code; };
  if (cudaGetDevice(&b->device) != cudaSuccess) { set_error("no CUDA device"); return fail(ADFT_ERR_CUDA); }
  b->natom = natom; b->nshell = nshell; b->spherical = spherical;
  b->xyz.assign(atom_xyz, atom_xyz + 3 * natom);
  int coff = 0, soff = 0, poff = 0;
  for (int s = 0; s < nshell; ++s) {
    const adft_shell& sh = shells[s];
    b->shell_l.push_back(sh.l); b->shell_atom.push_back(sh.atom); b->shell_nprim.push_back(sh.nprim);
    b->shell_poff.push_back(poff); b->shell_coff.push_back(coff); b->shell_soff.push_back(spherical ? soff : coff);
    coff += ncart(sh.l); soff += 2 * sh.l + 1; poff += sh.nprim;
    double df = 1.0;
    for (int k = 2 * sh.l - 1; k > 1; k -= 2) df *= k;
    for (int i = 0; i < sh.nprim; ++i) {
      const double a = sh.exps[i];
      const double N = pow(2.0 * a / M_PI, 0.75) * pow(4.0 * a, 0.5 * sh.l) / sqrt(df);
      b->exps.push_back(a);
      b->ncoefs.push_back(sh.coefs[i] * N);
    }
  }
  b->ncart = coff;
  b->nbf = spherical ? soff : coff;

  // pairs grouped by class (la >= lb; ties in l: larger shell index first)
  std::vector<std::vector<std::pair<int, int>>> by_cls(NCLS);
  for (int a = 0; a < nshell; ++a)
    for (int c = 0; c <= a; ++c) {
      int x = a, y = c;
      if (b->shell_l[y] > b->shell_l[x]) std::swap(x, y);
      by_cls[cls_of(b->shell_l[x], b->shell_l[y])].push_back({x, y});
    }
  b->npair = nshell * (nshell + 1) / 2;
  std::vector<int> pa, pb;
  b->cls_first[0] = 0;
  for (int X = 0; X < NCLS; ++X) {
    for (auto& pr : by_cls[X]) { pa.push_back(pr.first); pb.push_back(pr.second); }
    b->cls_first[X + 1] = (int)pa.size();
  }

  st = boys_tables(&b->boys64, &b->boys32);
  if (st != cudaSuccess) { set_error("Boys table upload failed"); return fail(ADFT_ERR_CUDA); }
  {
    double h_sph[LMAX + 1][2 * LMAX + 1][SPH_MAXC];
    sph_coefficients(h_sph);
    if (cudaMemcpyToSymbol(c_sph, h_sph, sizeof(h_sph)) != cudaSuccess) {
      set_error("spherical coefficient upload failed");
      return fail(ADFT_ERR_CUDA);
    }
  }
  if ((st = upload(b, &b->d_shell_l, b->shell_l)) || (st = upload(b, &b->d_shell_atom, b->shell_atom)) ||
      (st = upload(b, &b->d_shell_coff, b->shell_coff)) || (st = upload(b, &b->d_shell_soff, b->shell_soff)) ||
      (st = upload(b, &b->d_shell_nprim, b->shell_nprim)) || (st = upload(b, &b->d_shell_poff, b->shell_poff)) ||
      (st = upload(b, &b->d_xyz, b->xyz)) || (st = upload(b, &b->d_exps, b->exps)) ||
      (st = upload(b, &b->d_ncoefs, b->ncoefs)))
    return fail(st);
  // function maps
  {
    std::vector<int> fs, fc, cs, cc;
    for (int s = 0; s < nshell; ++s) {
      const int l = b->shell_l[s];
      for (int k = 0; k < ncart(l); ++k) { cs.push_back(s); cc.push_back(k); }
      const int nf = spherical ? 2 * l + 1 : ncart(l);
      for (int k = 0; k < nf; ++k) { fs.push_back(s); fc.push_back(k); }
    }
    if ((st = upload(b, &b->d_func_shell, fs)) || (st = upload(b, &b->d_func_comp, fc)) ||
        (st = upload(b, &b->d_cfunc_shell, cs)) || (st = upload(b, &b->d_cfunc_comp, cc)))
      return fail(st);
  }

  // build pair data twice: once in class order to get Q, then in Q order
  auto build = [&](const std::vector<int>& A, const std::vector<int>& B, bool first) -> int {
    std::vector<int> ppoff(A.size()), ppn(A.size());
    long long tot = 0;
    for (size_t i = 0; i < A.size(); ++i) {
      ppoff[i] = (int)tot;
      ppn[i] = b->shell_nprim[A[i]] * b->shell_nprim[B[i]];
      tot += ppn[i];
    }
    if (tot > 0x7fffffffLL) { set_error("too many primitive pairs"); return ADFT_ERR_UNSUPPORTED; }
    b->npp = tot;
    int r;
    if (first) {
      if ((r = dalloc(b, &b->d_pair_a, A.size())) || (r = dalloc(b, &b->d_pair_b, A.size())) ||
          (r = dalloc(b, &b->d_pair_ppoff, A.size())) || (r = dalloc(b, &b->d_pair_ppn, A.size())) ||
          (r = dalloc(b, &b->d_pair_Q, A.size())) || (r = dalloc(b, &b->d_pair_AB, 3 * A.size())) ||
          (r = dalloc(b, &b->d_pp64, (size_t)tot)) || (r = dalloc(b, &b->d_pp32, (size_t)tot)) ||
          (r = dalloc(b, &b->d_ppw64, 2 * (size_t)tot)) || (r = dalloc(b, &b->d_ppw32, 2 * (size_t)tot)))
        return r;
    }
    ADFT_CUDA(cudaMemcpy(b->d_pair_a, A.data(), A.size() * sizeof(int), cudaMemcpyHostToDevice));
    ADFT_CUDA(cudaMemcpy(b->d_pair_b, B.data(), B.size() * sizeof(int), cudaMemcpyHostToDevice));
    ADFT_CUDA(cudaMemcpy(b->d_pair_ppoff, ppoff.data(), ppoff.size() * sizeof(int), cudaMemcpyHostToDevice));
    ADFT_CUDA(cudaMemcpy(b->d_pair_ppn, ppn.data(), ppn.size() * sizeof(int), cudaMemcpyHostToDevice));
    const int T = 256;
    k_build_pairs<<<(unsigned)((tot + T - 1) / T), T>>>((int)A.size(), b->d_pair_a, b->d_pair_b, b->d_pair_ppoff,
                                                       b->d_shell_atom, b->d_shell_nprim, b->d_shell_poff,
                                                       b->d_xyz, b->d_exps, b->d_ncoefs, tot, b->d_pp64,
                                                       b->d_pp32, b->d_pair_AB, b->d_ppw64, b->d_ppw32);
    ADFT_CUDA(cudaGetLastError());
    return ADFT_OK;
  };
  if ((st = build(pa, pb, true))) return fail(st);
  // a2: Schwarz bounds on the device
  {
    BasisView v = view(b);
    for (int X = 0; X < NCLS; ++X) {
      const int n = b->cls_first[X + 1] - b->cls_first[X];
      if (n == 0) continue;
      cudaError_t e = launch_schwarz(X, v, b->cls_first[X], n, b->d_pair_Q, 0);
      if (e != cudaSuccess) { set_error(std::string("schwarz: ") + cudaGetErrorString(e)); return fail(ADFT_ERR_CUDA); }
    }
    std::vector<double> Q(b->npair);
    if (cudaMemcpy(Q.data(), b->d_pair_Q, Q.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
      set_error(std::string("schwarz readback: ") + cudaGetErrorString(cudaGetLastError()));
      return fail(ADFT_ERR_CUDA);
    }
    // sort each class by Q descending (stable), rebuild in that order
    std::vector<int> idx(b->npair);
    std::iota(idx.begin(), idx.end(), 0);
    for (int X = 0; X < NCLS; ++X)
      std::stable_sort(idx.begin() + b->cls_first[X], idx.begin() + b->cls_first[X + 1],
                       [&](int i, int j) { return Q[i] > Q[j]; });
    std::vector<int> sa(b->npair), sb(b->npair);
    b->pair_Q.resize(b->npair);
    for (int i = 0; i < b->npair; ++i) { sa[i] = pa[idx[i]]; sb[i] = pb[idx[i]]; b->pair_Q[i] = Q[idx[i]]; }
    b->pair_a = sa; b->pair_b = sb;
    if ((st = build(sa, sb, false))) return fail(st);
    if (cudaMemcpy(b->d_pair_Q, b->pair_Q.data(), b->npair * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
      set_error("Q upload failed");
      return fail(ADFT_ERR_CUDA);
    }
    std::vector<long long> cum(b->npair + 1, 0);
    for (int i = 0; i < b->npair; ++i) cum[i + 1] = cum[i] + (long long)b->shell_nprim[sa[i]] * b->shell_nprim[sb[i]];
    if ((st = upload(b, &b->d_cumppn, cum))) return fail(st);
  }
  // workspace
  {
    long long co = 0, po = 0;
    for (int X = 0; X < NCLS; ++X)
      for (int Y = 0; Y <= X; ++Y) {
        const int cp = cp_index(X, Y);
        const int nX = b->cls_first[X + 1] - b->cls_first[X];
        b->cnt_off[cp] = co; b->pre_off[cp] = po;
        co += nX; po += nX + 1;
      }
    b->cnt_total = co; b->pre_total = po;
    Workspace& w = b->ws;
    const size_t nc2 = (size_t)b->ncart * b->ncart, nb2 = (size_t)b->nbf * b->nbf;
    if ((st = dalloc(b, &w.Dc, nc2)) || (st = dalloc(b, &w.Dc32, nc2)) || (st = dalloc(b, &w.Jc, nc2)) ||
        (st = dalloc(b, &w.Kc, nc2)) || (st = dalloc(b, &w.Jw, nb2)) || (st = dalloc(b, &w.Kw, nb2)) ||
        (st = dalloc(b, &w.cnt64, (size_t)co)) || (st = dalloc(b, &w.cnt32, (size_t)co)) ||
        (st = dalloc(b, &w.pre64, (size_t)po)) || (st = dalloc(b, &w.pre32, (size_t)po)) ||
        (st = dalloc(b, &w.counters, 2 * NCP)) || (st = dalloc(b, &w.status, 4)) ||
        (st = dalloc(b, &w.scal, 4)) || (st = dalloc(b, &w.stats, 8)))
      return fail(st);
    if (cudaMemset(w.status, 0, 4 * sizeof(int)) != cudaSuccess) { set_error("memset"); return fail(ADFT_ERR_CUDA); }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    set_error(std::string("basis setup: ") + cudaGetErrorString(cudaGetLastError()));
    return fail(ADFT_ERR_CUDA);
  }
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
  for (int i = 0; i < b->npair; ++i) {
    int x = b->pair_a[i], y = b->pair_b[i];
    if (y > x) std::swap(x, y);
    Q[(long long)x * (x + 1) / 2 + y] = b->pair_Q[i];
  }
  return ADFT_OK;
}

int adft_jk_build(adft_basis* b, const double* D, const adft_opts* o, double* J, double* K) {
  if (!b || !D || !J || !K) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  int st = check_opts(o);
  if (st) return st;
  if ((st = set_device(b))) return st;
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = run_jk(b, D, o, s))) return st;
  const long long nb2 = (long long)b->nbf * b->nbf;
  k_from_cart<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(b->ncart, b->nbf, b->spherical, b->d_func_shell,
                                                            b->d_func_comp, b->d_shell_l, b->d_shell_coff, b->ws.Jc,
                                                            b->ws.Kc, J, K);
  ADFT_CUDA(cudaGetLastError());
  return finish_check(b, o, s);
}

int adft_jk_energy(adft_basis* b, const double* D, const adft_opts* o, double* E, int E_on_device) {
  if (!b || !D || !E) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  int st = check_opts(o);
  if (st) return st;
  if ((st = set_device(b))) return st;
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = run_jk(b, D, o, s))) return st;
  const long long nb2 = (long long)b->nbf * b->nbf;
  k_from_cart<<<(unsigned)((nb2 + 255) / 256), 256, 0, s>>>(b->ncart, b->nbf, b->spherical, b->d_func_shell,
                                                            b->d_func_comp, b->d_shell_l, b->d_shell_coff, b->ws.Jc,
                                                            b->ws.Kc, b->ws.Jw, b->ws.Kw);
  ADFT_CUDA(cudaGetLastError());
  double* Ed = b->ws.scal;  // scal[0] holds the energy
  ADFT_CUDA(cudaMemsetAsync(Ed, 0, sizeof(double), s));
  k_energy<<<grid_for(256, 2), 256, 0, s>>>(nb2, D, b->ws.Jw, b->ws.Kw, Ed);
  ADFT_CUDA(cudaGetLastError());
  if (E_on_device) {
    ADFT_CUDA(cudaMemcpyAsync(E, Ed, sizeof(double), cudaMemcpyDeviceToDevice, s));
  } else {
    ADFT_CUDA(cudaMemcpyAsync(E, Ed, sizeof(double), cudaMemcpyDeviceToHost, s));
    ADFT_CUDA(cudaStreamSynchronize(s));
  }
  return finish_check(b, o, s);
}

int adft_jk_last_stats(adft_basis* b, adft_stats* out) {
  if (!b || !out) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  unsigned long long h[8];
  ADFT_CUDA(cudaStreamSynchronize(b->last_stream));
  ADFT_CUDA(cudaMemcpy(h, b->ws.stats, sizeof(h), cudaMemcpyDeviceToHost));
  out->quartets_fp64 = (int64_t)h[0];
  out->quartets_fp32 = (int64_t)h[1];
  out->quartets_total = (int64_t)h[2];
  out->prim_quartets_fp64 = (int64_t)h[3];
  out->prim_quartets_fp32 = (int64_t)h[4];
  out->flops_fp64 = 0.0;
  out->flops_fp32 = 0.0;
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

int adft_jk_grad(adft_basis* b, const double* D, const adft_opts* o, double* grad) {
  if (!b || !D || !grad) { set_error("NULL argument"); return ADFT_ERR_ARG; }
  int st = check_opts(o);
  if (st) return st;
  if ((st = set_device(b))) return st;
  cudaStream_t s = (cudaStream_t)o->stream;
  if ((st = prepare(b, D, o, s))) return st;
  ADFT_CUDA(cudaMemsetAsync(grad, 0, 3 * sizeof(double) * b->natom, s));
  const int grid = grid_for(128, 4);
  st = for_each_class_pair(b, o, base_launch(b), [&](int X, int Y, const JKLaunch& L, int band) {
    GradLaunch g;
    g.jk = L;
    g.grad = grad;
    return band == 0 ? launch_grad_fp64(X, Y, g, grid, s) : launch_grad_fp32(X, Y, g, grid, s);
  });
  if (st) return st;
  return finish_check(b, o, s);
}

int adft_batch_create(adft_basis* const* mols, int nmol, adft_batch** out) {
  (void)mols; (void)nmol; (void)out;
  set_error("batched form not built yet");
  return ADFT_ERR_UNSUPPORTED;
}
int adft_batch_offsets(const adft_batch*, int64_t*) { return ADFT_ERR_UNSUPPORTED; }
int adft_batch_grad_offsets(const adft_batch*, int64_t*) { return ADFT_ERR_UNSUPPORTED; }
int adft_batch_jk(adft_batch*, const double*, const adft_opts*, double*, double*, double*, double*) {
  return ADFT_ERR_UNSUPPORTED;
}
void adft_batch_destroy(adft_batch*) {}

}  // extern "C"
