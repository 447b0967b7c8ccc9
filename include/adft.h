/*
 * adft.h -- C ABI of the GB300 direct-SCF Coulomb/exchange (J/K) library.
 *
 * The library evaluates the Coulomb and exact-exchange matrices of Eq. 1
 * (Sec. 1.2.1 of "Acceleration without Disruption: DFT Software as a
 * Service", arXiv 2406.11185)
 *
 *     J_mn = sum_ls D_ls (mn|ls),        K_mn = sum_ls D_ls (ml|ns)
 *
 * (K without the hybrid factor c_x, which the caller applies) from
 * four-centre electron-repulsion integrals over contracted Gaussian shells
 * (the integral of the ERI paragraph of Sec. 1.2.2), computed directly on
 * one GPU without density fitting.  Shell quartets are screened with the
 * Cauchy-Schwarz bound S = Q_ab Q_cd and, in mixed precision, dispatched to
 * FP32 or FP64 kernels by that bound (the mixed-precision bullet of Sec.
 * 1.2.2).  The energy E_JK = 1/2 tr(DJ) - 1/4 tr(DK) and its nuclear gradient
 * at fixed D are also provided.
 *
 * Conventions
 *   - Units: bohr, hartree.
 *   - A shell is (atom, l, exponents a_i, coefficients c_i).  The c_i multiply
 *     normalised primitive Cartesian Gaussians
 *        N(a,l) x^ax y^ay z^az exp(-a r^2),
 *        N(a,l) = (2a/pi)^(3/4) (4a)^(l/2) / sqrt((2l-1)!!),
 *     the same N for every Cartesian component of the shell.  The library does
 *     not renormalise contractions.
 *   - Cartesian components are ordered by descending x power, then descending
 *     y power (xx, xy, xz, yy, yz, zz).  Spherical components: p is (x, y, z);
 *     l >= 2 is m = -l..l of the unit-norm real solid harmonics.
 *   - Basis functions are ordered shell by shell in the order given to
 *     adft_basis_create.  All matrices are row-major nbf x nbf float64.
 *   - Schwarz bound: Q_ab = sqrt(max over Cartesian components mu in a,
 *     nu in b of |(mu nu|mu nu)|).  A shell quartet is skipped iff
 *     Q_ab Q_cd < thresh.  In mixed precision it runs in FP64 iff
 *     Q_ab Q_cd >= split, else in FP32 with its contributions added into
 *     FP64 accumulators.
 *
 * Memory and threads
 *   - "dev" pointers are CUDA device pointers on the current device; "host"
 *     pointers are ordinary host memory.  The caller owns every buffer it
 *     passes.  The library owns the basis handle and the device workspace it
 *     allocates at creation; nothing is allocated per J/K call.
 *   - Every call that takes an adft_opts enqueues its work on opts->stream
 *     (NULL = the legacy default stream) and returns without synchronising,
 *     unless opts->check is 1 (see below) or a host output is requested.
 *   - A handle may be used by one stream at a time.
 *
 * Errors: every function returns ADFT_OK (0) or a negative status; nothing
 * aborts or traps.  adft_status_string() gives a description, and
 * adft_last_error_message() the detail of the last failing call on this
 * thread.
 */
#ifndef ADFT_H
#define ADFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ADFT_LMAX 3        /* highest shell angular momentum supported (f) */
#define ADFT_MAX_NPRIM 16  /* highest number of primitives in one shell */

enum {
  ADFT_OK = 0,
  ADFT_ERR_ARG = -1,          /* null pointer, bad size, l > ADFT_LMAX, nprim out of range, ... */
  ADFT_ERR_UNSUPPORTED = -2,  /* valid request the library does not implement */
  ADFT_ERR_ASYM_D = -3,       /* max|D - D^T| > 1e-12 max|D| (only with opts->check) */
  ADFT_ERR_NONFINITE = -4,    /* D holds NaN or Inf (only with opts->check) */
  ADFT_ERR_OOM = -5,          /* device or host allocation failed */
  ADFT_ERR_CUDA = -6,         /* a CUDA runtime call failed */
  ADFT_ERR_TIMEOUT = -7,      /* a bounded device-side wait ran out */
  ADFT_ERR_ABORTED = -8       /* the abort flag of the handle was raised */
};

/* Precision modes.  FP64: every kept quartet in FP64.  MIXED: the
 * Schwarz-bound dispatch of Sec. 1.2.2, FP64 iff Q_ab Q_cd >= split, else
 * FP32 with its contributions added into FP64 accumulators. */
enum { ADFT_PREC_FP64 = 0, ADFT_PREC_MIXED = 1 };

typedef struct adft_basis adft_basis; /* opaque, library-owned */
typedef struct adft_batch adft_batch; /* opaque, library-owned */

typedef struct {
  int atom;             /* index into the atom array, 0 <= atom < natom */
  int l;                /* angular momentum, 0 <= l <= ADFT_LMAX */
  int nprim;            /* 1 <= nprim <= ADFT_MAX_NPRIM */
  const double* exps;   /* host [nprim], > 0 */
  const double* coefs;  /* host [nprim], coefficients of normalised primitives */
} adft_shell;

typedef struct {
  double thresh;   /* Schwarz threshold: skip iff Q_ab Q_cd < thresh.  Must be >= 1e-12
                      (ADFT_ERR_ARG otherwise): basis creation drops primitive pairs
                      whose bound product is <= 1e-15, i.e. at most 1e-3 thresh. */
  double split;    /* mixed modes only: FP64 band iff Q_ab Q_cd >= split */
  int precision;   /* ADFT_PREC_FP64 or ADFT_PREC_MIXED */
  int check;       /* 1: validate D on the device, synchronise the stream and
                      return ADFT_ERR_ASYM_D / ADFT_ERR_NONFINITE; 0: no check,
                      fully asynchronous */
  void* stream;    /* cudaStream_t, NULL = legacy default stream */
  const unsigned char* pair_mask; /* host [2][55] or NULL (all): 1 = evaluate this
                      (band, class pair) in this call, band-major (FP64, FP32),
                      class pair X(X+1)/2 + Y.  With a mask, J, K, E and the
                      gradient are partial sums: over calls (ranks) whose masks
                      partition the class pairs they add up to the full result,
                      so one sum all-reduce of J and K (or E, or the gradient) is
                      the only exchange.  Single-molecule calls only (a batch is
                      sharded by molecules). */
  double omega;    /* range separation: 0 = the Coulomb operator 1/r12; > 0 = the
                      long-range operator erf(omega r12)/r12 of range-separated
                      hybrids (the omegaB97X functional of Sec. 4.1) in every ERI of J
                      and K (adft_jk_build, adft_jk_energy, adft_autotune).  Quartets
                      are still screened with the Coulomb bounds Q, which bound the
                      attenuated integrals too.  Must be finite and >= 0
                      (ADFT_ERR_ARG); adft_jk_grad and the batched calls return
                      ADFT_ERR_UNSUPPORTED for omega > 0. */
} adft_opts;

/* Per-call statistics of the last J/K build (host copies).  After a build
 * the primitive counts and flops are what the kernels evaluated: inside a
 * kept shell quartet, primitive quartets with Q_p Q_q < 1e-4 * thresh are
 * skipped.  After adft_jk_plan (no kernels run) they are the counts before
 * that primitive screening. */
typedef struct {
  int64_t quartets_fp64;     /* shell quartets evaluated in FP64 */
  int64_t quartets_fp32;     /* shell quartets evaluated in FP32 */
  int64_t quartets_total;    /* unique shell quartets before screening */
  int64_t prim_quartets_fp64; /* primitive quartets evaluated inside the FP64 ones */
  int64_t prim_quartets_fp32; /* primitive quartets evaluated inside the FP32 ones */
  double flops_fp64;         /* counted FP64 flops of the ERI + digestion kernels */
  double flops_fp32;         /* counted FP32 flops of the ERI + digestion kernels */
} adft_stats;

/* Create a basis on the current CUDA device: copies the geometry and shells,
 * builds the shell-pair data (Gaussian product centres, exponents and
 * prefactors of every primitive pair; as in Sec. 1.2.2, each contraction of a
 * given angular momentum is its own shell, i.e. a segmented contraction), evaluates the
 * Schwarz bounds Q_ab on the GPU and sorts the pairs of each
 * angular-momentum class (l_a >= l_b) by descending Q (the angular-momentum
 * reordering of Sec. 1.2.2).  Primitive pairs whose bound Q_p times the
 * largest Q_p is at most 1e-15 are dropped; the others are kept in order of
 * descending Q_p.  Synchronous.
 *   atom_xyz: host [natom*3] bohr.  shells: host [nshell].
 *   spherical: 1 = spherical functions, 0 = Cartesian functions.
 *   out: receives the handle; release it with adft_basis_destroy. */
int adft_basis_create(const double* atom_xyz, int natom, const adft_shell* shells, int nshell,
                      int spherical, adft_basis** out);

/* Number of basis functions (spherical or Cartesian as created). */
int adft_basis_nbf(const adft_basis* b, int* nbf);

/* Number of atoms and shells. */
int adft_basis_dims(const adft_basis* b, int* natom, int* nshell, int* ncart);

/* Copy the Schwarz bounds to host memory: Q[a*(a+1)/2 + b] for shells
 * a >= b in creation order.  Q: host [nshell*(nshell+1)/2]. */
int adft_basis_schwarz(const adft_basis* b, double* Q);

/* J and K of Eq. 1 for a symmetric density D.
 *   D, J, K: dev [nbf*nbf] row-major float64; J and K are overwritten.
 *   K is sum_ls D_ls (ml|ns) without c_x.  The result is symmetric to
 *   round-off.  Statistics of the call are kept for adft_jk_last_stats. */
int adft_jk_build(adft_basis* b, const double* D, const adft_opts* opts, double* J, double* K);

/* E_JK = 1/2 tr(DJ) - 1/4 tr(DK).  Builds J and K internally (into the
 * handle's workspace) and writes the energy.
 *   E: dev pointer to one float64 if E_on_device = 1, else a host pointer
 *   (then the call synchronises the stream). */
int adft_jk_energy(adft_basis* b, const double* D, const adft_opts* opts, double* E, int E_on_device);

/* Nuclear gradient dE_JK/dR at fixed D (derivative integrals contracted with
 * G = 1/2 D(x)D - 1/8 (D(x)D exchange-permuted); quartets recomputed, none
 * stored).  Screening and the precision bands use the undifferentiated
 * bounds S = Q_ab Q_cd.
 *   grad: dev [natom*3] float64, overwritten. */
int adft_jk_grad(adft_basis* b, const double* D, const adft_opts* opts, double* grad);

/* One-electron matrices of the core Hamiltonian H = T + V that the Fock
 * matrix of Eq. 1 adds to J and K (the SCF driver around the J/K build):
 * overlap S, kinetic energy T and nuclear attraction
 * V_mn = -sum_C Z_C <m| 1/|r - R_C| |n>, in the basis's functions (spherical
 * or Cartesian as created).  Single-molecule bases only.
 *   charges: host [natom] nuclear charges Z_C (finite).
 *   S, T, V: dev [nbf*nbf] row-major float64, overwritten.
 *   stream: cudaStream_t or NULL.  Asynchronous (the charges are copied before
 *   the call returns). */
int adft_one_electron(adft_basis* b, const double* charges, void* stream, double* S, double* T, double* V);

/* Nuclear gradient of the one-electron part of the closed-shell SCF energy
 * (the single-point force task, Sec. 3, around adft_jk_grad):
 *   grad = sum D dH/dR - sum W dS/dR,  H = T + V as in adft_one_electron,
 * W the energy-weighted density (1/2 D F D at convergence).  The caller adds
 * adft_jk_grad (at the same D) and the nuclear repulsion gradient.
 *   charges: host [natom].  D, W: dev [nbf][nbf] in the basis's output
 *   functions, symmetric.  grad: dev [natom][3], overwritten.
 * Enqueued on stream (NULL = legacy default stream); no synchronisation.
 * Uses the handle's Cartesian D and J workspaces (do not overlap with a
 * build of the same handle on another stream).  Single-molecule bases only
 * (ADFT_ERR_ARG otherwise). */
int adft_one_electron_grad(adft_basis* b, const double* charges, const double* D, const double* W, void* stream,
                           double* grad);

/* Statistics of the last adft_jk_build / adft_jk_energy / adft_jk_grad on
 * this handle (synchronises the handle's last stream). */
int adft_jk_last_stats(adft_basis* b, adft_stats* st);

/* Per class pair and band of the last adft_jk_build / adft_jk_energy (or
 * adft_jk_plan: then only quartets): kept shell quartets, evaluated primitive
 * quartets and bra primitives, and counted flops of the ERI + digestion kernel
 * (the class's flop model applied to those counts).  Each output is host
 * [2][55] (band-major: FP64 then FP32; class pair X(X+1)/2 + Y) or NULL.
 * Synchronises the handle's last stream. */
int adft_jk_last_class_stats(adft_basis* b, int64_t* quartets, int64_t* prim_quartets, int64_t* bra_prims,
                             double* flops);

/* Device time of the phases of the last adft_jk_build / adft_jk_energy /
 * adft_jk_grad on this handle, from CUDA events recorded on its stream
 * (synchronises on the last event).  ms: host [4] milliseconds:
 *   [0] D check, D -> Cartesian, screening and work-list scan,
 *   [1] the FP64 ERI (or derivative) kernels, [2] the FP32 ones (0 unless
 *   mixed), [3] Cartesian -> output transform and energy. */
int adft_jk_last_timings(adft_basis* b, double* ms);

/* Autotuner (per angular-momentum class pair and precision band): times
 * every class-pair kernel of one build of D in each kernel variant that
 * serves the class pair and with 1, 2, 4 and 8 resident blocks per SM.  The
 * d-class pairs up to (dd|dp) have two to four variants: the cooperative
 * group kernel, a warp-per-quartet kernel for (dp|pp), (dp|ds), (dp|dp), and
 * the row-blocked kernel in one or two launch shapes; the other pairs have
 * one.  Block counts that cannot be resident at once are skipped.  The
 * fastest choice is kept in the handle for later calls.  The J/K accumulators of the
 * handle are left undefined.
 *   table: host [2][55] ints (band-major: FP64 then FP32; class pair
 *   X(X+1)/2 + Y with class X = l_a(l_a+1)/2 + l_b) or NULL; each entry is
 *   blocks_per_SM + 256 * variant.
 *   ms: host [2][55] doubles, the best time of every class-pair kernel
 *   (0 for empty ones), or NULL.
 * Synchronous. */
int adft_autotune(adft_basis* b, const double* D, const adft_opts* opts, int* table, double* ms);

/* Plan only: run the screening and work-list pass for D (no integrals) and
 * report what a build would evaluate.  st: the counts of adft_jk_last_stats
 * (flops are the counted estimate); quartets: host [2][55] int64 shell
 * quartets per band and class pair, or NULL.  Synchronous. */
int adft_jk_plan(adft_basis* b, const double* D, const adft_opts* opts, adft_stats* st, int64_t* quartets);

/* Install a launch-shape table (same layout and encoding as adft_autotune's).
 * ADFT_ERR_ARG if an entry's blocks per SM is outside 1..64 or its variant is
 * not below the class pair's number of variants; the handle is unchanged then. */
int adft_set_tuning(adft_basis* b, const int* table);

/* Raise (1) or clear (0) the handle's abort flag.  A running or later build
 * sees it on the device and returns ADFT_ERR_ABORTED (with opts->check = 1)
 * or leaves a status readable by adft_jk_status. */
int adft_basis_set_abort(adft_basis* b, int flag);

/* Read the device status word of the handle (ADFT_OK or an error of the last
 * asynchronous call); synchronises the handle's last stream. */
int adft_jk_status(adft_basis* b);

void adft_basis_destroy(adft_basis* b);

/* ---- batched form: many molecules, one persistent launch per class ----- */

/* Group existing bases (not copied; they must outlive the batch).
 *   mols: host [nmol] handles, all created with the same `spherical`. */
int adft_batch_create(adft_basis* const* mols, int nmol, adft_batch** out);

/* Offsets (in float64 elements) of each molecule's nbf x nbf block in the
 * packed matrices: offsets host [nmol+1], offsets[i+1]-offsets[i] = nbf_i^2. */
int adft_batch_offsets(const adft_batch* bt, int64_t* offsets);

/* Offsets of each molecule's natom x 3 gradient block: host [nmol+1]. */
int adft_batch_grad_offsets(const adft_batch* bt, int64_t* offsets);

/* J, K (and optionally E and the gradient) of every molecule with one
 * persistent launch per angular-momentum class pair and band over a global
 * quartet work list spanning all molecules (the batch is built as one basis
 * whose shell pairs never mix molecules).
 *   D_packed, J_packed, K_packed: dev, packed per adft_batch_offsets.
 *   E: dev [nmol] or NULL.  grad_packed: dev per adft_batch_grad_offsets or
 *   NULL.
 * With opts->check = 0 and a non-NULL stream the whole call is captured into
 * a CUDA graph on first use and replayed by later calls with the same
 * buffers and options; the first call must not itself run inside a stream
 * capture.  With opts->check = 1 the launches are issued directly and the
 * stream is synchronised to report the validation result. */
int adft_batch_jk(adft_batch* bt, const double* D_packed, const adft_opts* opts, double* J_packed,
                  double* K_packed, double* E, double* grad_packed);

/* Statistics and phase times of the last adft_batch_jk (see
 * adft_jk_last_stats / adft_jk_last_timings). */
int adft_batch_last_stats(adft_batch* bt, adft_stats* st);
int adft_batch_last_timings(adft_batch* bt, double* ms);

/* The autotuner of the batch's class-pair kernels (see adft_autotune). */
int adft_batch_autotune(adft_batch* bt, const double* D_packed, const adft_opts* opts, int* table, double* ms);

/* Install a launch-shape table (adft_autotune's layout and encoding) in the
 * batch, e.g. one tuned on a smaller batch of the same kind of molecules.
 * The batch's captured CUDA graph is dropped and re-captured on the next
 * call.  ADFT_ERR_ARG as for adft_set_tuning. */
int adft_batch_set_tuning(adft_batch* bt, const int* table);

void adft_batch_destroy(adft_batch* bt);

/* ---- energy without allocation ------------------------------------------ */

/* Largest nbf accepted by adft_energy_static: the size, in doubles, of the
 * library's built-in device scratch array (128 KiB on every device that
 * loads the library, held until the process exits). */
#define ADFT_STATIC_MAX_NBF 16384

/* E = 1/2 tr(DJ) - 1/4 tr(DK) from caller-owned D, J, K, for callers that
 * cannot allocate device memory at the point of the call (a memory pool that
 * forbids growth, a region where cudaMalloc would synchronise the device, an
 * allocator owned by another framework).  The paper has no counterpart; it is
 * a convenience of this library.  It allocates nothing: its scratch (one
 * partial sum per row) is a fixed array inside the library, so every call
 * shares it and keeps the last call's contents, and calls that overlap on the
 * GPU race on it (serialise them, e.g. on one stream).
 *   D, J, K: dev [nbf*nbf] row-major float64.  E: dev pointer to one float64.
 *   All four must live on the current device, and the stream must belong to
 *   it: the kernels run on the current device and dereference these pointers.
 *   nbf: 1..ADFT_STATIC_MAX_NBF, else ADFT_ERR_ARG.  stream: cudaStream_t or
 *   NULL.  Asynchronous.  The first call on each device looks up the device
 *   address of the scratch array (with that device current); make that first
 *   call before any stream capture.  With lazy module loading (the CUDA
 *   default) that first lookup may load the library's device code, which
 *   reserves device memory for the code and the array once per device; later
 *   calls allocate nothing.  ADFT_ERR_CUDA reports a failed launch of this
 *   call only (an error left by earlier work is not reported or cleared). */
int adft_energy_static(const double* D, const double* J, const double* K, int nbf, double* E, void* stream);

/* ---- measurement --------------------------------------------------------- */

/* ALU peak of the current device for the roofline of the ERI kernels (which
 * are bound by plain FP64 / FP32 arithmetic): a kernel of independent fused
 * multiply-add chains on every SM, timed with CUDA events on the legacy
 * default stream after one warm-up launch.  The paper has no counterpart; it
 * is measurement support.
 *   fp64: 1 = FP64 FMAs, 0 = FP32 FMAs.  iters: loop trips (each trip is 128
 *   FMAs per thread; 2048 blocks of 256 threads on 152 SMs).
 *   tflops: receives 2 x FMAs / time in TFLOP/s.  ms: the kernel time or NULL.
 * Synchronous. */
int adft_alu_peak(int fp64, int iters, double* tflops, double* ms);

/* ---- utilities ---------------------------------------------------------- */

const char* adft_status_string(int status);
const char* adft_last_error_message(void);

/* Library version string. */
const char* adft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ADFT_H */
