// Internal declarations shared by the translation units of the GB300 J/K
// library.  Nothing here is part of the public C ABI (include/adft.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "adft.h"

namespace adft {

constexpr int LMAX = ADFT_LMAX;               // shells up to f
constexpr int NCLS = (LMAX + 1) * (LMAX + 2) / 2;  // pair classes (la >= lb)
constexpr int NCP = NCLS * (NCLS + 1) / 2;    // class pairs (X >= Y)
constexpr int LTOT = 4 * LMAX + 1;            // largest L incl. one derivative
constexpr int BOYS_MMAX = LTOT + 8;           // table columns
constexpr double BOYS_H = 0.1;                // table spacing in T
constexpr int BOYS_NT = 601;                  // T = 0 .. 60
constexpr double BOYS_TMAX = 60.0;            // beyond: asymptotic / upward

__host__ __device__ constexpr int ncart(int l) { return (l + 1) * (l + 2) / 2; }
__host__ __device__ constexpr int nherm(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int cls_of(int la, int lb) { return la * (la + 1) / 2 + lb; }
__host__ __device__ constexpr int cls_la(int X) {
  return X < 1 ? 0 : X < 3 ? 1 : X < 6 ? 2 : X < 10 ? 3 : 4;
}
__host__ __device__ constexpr int cls_lb(int X) { return X - cls_la(X) * (cls_la(X) + 1) / 2; }
__host__ __device__ constexpr int cp_index(int X, int Y) { return X * (X + 1) / 2 + Y; }

// Primitive-pair record (8 values): Gaussian product centre P, exponent sum p,
// P - A, and K = c_a c_b exp(-a b / p |A-B|^2) (normalised-primitive
// coefficients included).  P - B = (P - A) + (A - B).
template <typename T>
struct alignas(sizeof(T) * 8) PrimPair {
  T Px, Py, Pz, p, PAx, PAy, PAz, K;
};

// Device view of one basis (all arrays on the device).
struct BasisView {
  int nshell, natom, ncart, nbf, spherical;
  const int* shell_l;
  const int* shell_atom;
  const int* shell_coff;   // first Cartesian function of each shell
  const double* xyz;       // [natom][3]
  int npair;
  const int* pair_a;       // shell with the larger l (ties: larger index)
  const int* pair_b;
  const double* pair_Q;    // Schwarz bound
  const int* pair_pp_off;  // first primitive pair
  const int* pair_pp_n;    // number of primitive pairs
  const double* pair_AB;   // [npair][3] A - B
  const PrimPair<double>* pp64;
  const PrimPair<float>* pp32;
  const double* boys64;    // [BOYS_NT][BOYS_MMAX+1] F_m(i h)
  const float* boys32;
  const double* pp_o2p64;  // [npp]: 1 / (2p) of every primitive pair
  const float* pp_o2p32;
  const double* pp_w64;    // [2][npp]: 2 a and 2 b of every primitive pair
  const float* pp_w32;
  const float* pp_q32;     // [npp] primitive-pair bound Q_p; descending within each pair
  long long npp;
  // several molecules (a batch): molecule of each pair, offset and row length
  // of the molecule's block in the packed Cartesian matrices; NULL = one
  // molecule whose block starts at 0 with row length ncart.
  const int* pair_mol;
  const long long* mol_cbase;
  const int* mol_nc;
};

// offset and row length of the packed Cartesian block of a pair's molecule
__device__ __forceinline__ void mol_block(const BasisView& bv, int pair, long long& base, long& n) {
  if (bv.pair_mol) {
    const int m = __ldg(bv.pair_mol + pair);
    base = __ldg(bv.mol_cbase + m);
    n = __ldg(bv.mol_nc + m);
  } else {
    base = 0;
    n = bv.ncart;
  }
}

// Contraction buckets.  Inside each (class, molecule) segment the pairs are
// ordered by bucket of their primitive-pair count, then by descending Schwarz
// bound, so the kets a bra keeps are a Q-prefix of every bucket, and a warp's
// consecutive quartets (same bra, neighbouring kets of one bucket) run
// primitive loops of similar length.  Upper bounds of the buckets:
constexpr int NBK = 10;
__host__ __device__ constexpr int pp_bucket(int npp) {
  return npp <= 1 ? 0 : npp <= 2 ? 1 : npp <= 4 ? 2 : npp <= 6 ? 3 : npp <= 9 ? 4 : npp <= 13 ? 5
       : npp <= 18 ? 6 : npp <= 25 ? 7 : npp <= 36 ? 8 : 9;
}

// One class-pair launch of the J/K kernel.  The work list is implicit: one
// segment per (bra, ket bucket), bra-major; segment s holds the kept kets of
// bra bra_first + s / NBK in bucket s % NBK.
struct JKLaunch {
  BasisView bv;
  int bra_first, nseg;      // bras of class X start at bra_first; nseg = NBK x bras
  int ket_first;            // pairs of class Y start here
  int same_class;           // X == Y
  const long long* prefix;  // [nseg + 1] quartets before each segment
  const int* ket_start;     // [nseg] first ket of the segment (band), relative to ket_first
  unsigned long long* counter;  // dynamic work counter (zeroed)
  const double* D64;        // Cartesian D [ncart][ncart]
  const float* D32;
  double* J;                // Cartesian accumulators (unsymmetrised)
  double* K;
  const int* abort_flag;    // device flag polled between work chunks
  int* status;              // device status word
  double prim_eps;          // primitive quartets with Q_p Q_q below this are skipped
  unsigned long long* work; // [2]: primitive quartets and bra primitives evaluated, or NULL
  double omega2;            // omega^2 of the operator erf(omega r)/r; 0 = 1/r
};

struct GradLaunch {
  JKLaunch jk;
  double* grad;                    // [natom][3]
  unsigned long long* counter2;    // work counter of the second (swapped) pass
};

// What a class-pair launcher reports instead of launching when asked: how many
// kernel variants serve the class pair and how many blocks of the selected
// variant fit on one SM.
struct KernelInfo {
  int variants;
  int max_blocks_per_sm;
};

// Launchers implemented in the per-precision translation units.  variant
// selects among the kernels that serve the class pair (0 = default); with
// info != nullptr nothing is launched and *info is filled in.
cudaError_t launch_jk_fp64(int X, int Y, const JKLaunch& a, int grid, int variant, cudaStream_t s,
                           KernelInfo* info = nullptr);
cudaError_t launch_jk_fp32(int X, int Y, const JKLaunch& a, int grid, int variant, cudaStream_t s,
                           KernelInfo* info = nullptr);
// Gradient launchers: the grid follows from the SM count and the kernel's occupancy.
cudaError_t launch_grad_fp64(int X, int Y, const GradLaunch& a, int sms, cudaStream_t s);
cudaError_t launch_grad_fp32(int X, int Y, const GradLaunch& a, int sms, cudaStream_t s);
// Qmax[pr] = max |(mn|mn)| of the pairs [first, first + n) of class X (zeroed
// by the caller; Q = sqrt(Qmax)).  maxp: the largest primitive-pair count of
// those pairs; part: scratch of n * ncart(la) ncart(lb) * maxp doubles.
cudaError_t launch_schwarz(int X, const BasisView& bv, int first, int n, int maxp, double* part, double* Qmax,
                           cudaStream_t s);
cudaError_t launch_prim_schwarz(int X, const BasisView& bv, int first, int n, const int* pp_pair, int npp_class,
                                double* Qp, cudaStream_t s);
// Cartesian one-electron matrices S, T, V (full [ncart][ncart]) of a
// single-molecule basis; charges: device [natom].
cudaError_t launch_one_electron(const BasisView& bv, const int* shell_nprim, const int* shell_poff,
                                const double* exps, const double* ncoefs, const double* charges, double* S,
                                double* T, double* V, cudaStream_t s);
cudaError_t launch_one_electron_grad(const BasisView& bv, const int* shell_nprim, const int* shell_poff,
                                     const double* exps, const double* ncoefs, const double* charges,
                                     const double* Dc, const double* Wc, double* grad, cudaStream_t s);
// Primitive pairs whose bound Qp * max(Qp) is at or below this are dropped at
// basis creation (1e-3 of the paper's default tolerance 1e-12).
constexpr double PRIM_EPS = 1e-15;
// Inside a kept shell quartet, primitive quartets with Q_p Q_q below
// PRIM_QUARTET_FRAC * thresh are skipped (each is bounded by that value).
constexpr double PRIM_QUARTET_FRAC = 1e-4;
// Boys tables in device memory of the current device (built once).
cudaError_t boys_tables(const double** t64, const float** t32);

void set_error(const std::string& msg);

}  // namespace adft
