/*
 * mt_oracle.h -- CPU FP64 oracle for the particle mass-transfer step of
 * Engdahl, Schmidt & Benson, "Accelerating and parallelizing Lagrangian
 * simulations of mixing-limited reactive transport" (arXiv 1811.05474).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) includes, links or calls this code; only the tests, the
 * package smoke check and the benchmark's CPU-baseline leg do.  It shares no
 * header, helper, table or constant with the CUDA path.
 *
 * What it computes, in the paper's notation:
 *   move      Eq. 2 with alpha_L = 0 and the random-walk share of diffusion
 *             (Sec. 3): x <- x + v dt + sqrt(2 D_rw dt) xi, reflecting walls.
 *   weights   Eq. 3: nu_ij proportional to exp(-s_ij^2 / (8 D_mt dt)); the
 *             prefactor (8 pi D_mt dt)^(-1/2) ds cancels in the normalisation.
 *   normalise Sec. 1.1: P_ij = nu_ij / sum_j nu_ij (ROW, the literal text), or
 *             its symmetric part (P + P^T)/2 (SYM, the mass-conserving reading).
 *   exchange  Eq. 4 and Eq. 7: dM_i = 1/2 sum_j P_ij (M_j - M_i); M += dM, per
 *             species, from start-of-step masses and positions (Sec. 1.1,
 *             "matrix explicit").
 *   matrix    Eq. 5-6 with the sign that agrees with Eq. 4:
 *             dM = 1/2 [P - diag(P 1)] M  (a second, independent formulation).
 *   react     Sec. 3 and Sec. 7: A + B -> E, irreversible and at equilibrium,
 *             per particle after the transfer: m = min(A, B); A -= m; B -= m.
 *   search    Sec. 2.1: fixed-radius neighbour search within s_max.
 *
 * Positions are fixed point: x = X * 2^-k with X a signed 64-bit integer and k
 * the number of fractional bits.  The cutoff is s_max rounded down to that
 * grid, Smax = floor(s_max * 2^k) ticks; a pair is in range iff
 * |dX| <= Smax (1-d) or dX^2 + dY^2 <= Smax^2 (2-d), evaluated exactly in
 * integers.  Every function is plain loops in FP64, single-threaded except
 * the sorted-window transfer's per-particle loops (see mto_set_threads).
 */
#ifndef MT_ORACLE_H
#define MT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { MTO_SEARCH_CUTOFF = 0, MTO_SEARCH_FULL = 2 };
enum { MTO_NORM_SYM = 0, MTO_NORM_ROW = 1 };
enum { MTO_WALLS_REFLECT = 0, MTO_WALLS_PERIODIC = 1 };

typedef struct {
  int32_t dim;        /* 1 or 2 */
  int32_t frac_bits;  /* k in x = X * 2^-k */
  double  L[2];       /* domain [0, L0] (x [0, L1]) */
  double  v[2];       /* constant advection velocity */
  double  D_mt;       /* diffusion coefficient carried by mass transfer, Eq. 3 */
  double  D_rw;       /* diffusion coefficient carried by the random walk, Eq. 2 */
  double  dt;         /* time step */
  double  smax;       /* cutoff distance s_max (Sec. 2.1) */
  int32_t search;     /* MTO_SEARCH_CUTOFF or MTO_SEARCH_FULL (no cutoff) */
  int32_t norm;       /* MTO_NORM_SYM or MTO_NORM_ROW */
  int32_t react;      /* 1: apply A + B -> E after the transfer */
  int32_t walls;      /* MTO_WALLS_REFLECT (Sec. 3) or MTO_WALLS_PERIODIC: the
                         domain wraps, positions live in [0, L) and pairs
                         take the minimum-image separation (needs s_max < L/2) */
} mto_params;

/* x -> nearest grid point X = rint(x * 2^k) (ties to even). */
int64_t mto_quantize(double x, int32_t k);
/* X -> x = X * 2^-k (rounded to double if |X| >= 2^53). */
double mto_dequantize(int64_t X, int32_t k);
/* Element-wise forms of the two conversions over n values. */
void mto_quantize_n(int64_t n, const double* x, int32_t k, int64_t* X);
void mto_dequantize_n(int64_t n, const int64_t* X, int32_t k, double* x);
/* Smax = floor(s_max * 2^k). */
int64_t mto_cutoff_ticks(const mto_params* p);

/* Move every particle once (Eq. 2; Sec. 3).  X holds dim*n ticks, axis-major
 * (all x, then all y).  xi holds dim*n standard normals (float, same layout).
 * The displacement in ticks is rint(b * xi), b = sqrt(2 D_rw dt) * 2^k, the
 * product formed in binary64 and rounded once; the drift is rint(v dt 2^k).  A
 * position outside [0, L] is mirrored at the wall it crossed, repeatedly,
 * until it lies inside (at most 64 mirrors, then clamped). */
void mto_move(const mto_params* p, int64_t n, int64_t* X, const float* xi);

/* Weight row sums r_i = sum_j nu_ij (self included, nu_ii = 1); Eq. 3. */
void mto_row_sums(const mto_params* p, int64_t n, const int64_t* X, double* r);

/* One mass-transfer step for nspec species (Eq. 3, 4, 7 with the chosen
 * normalisation), plain O(n^2) loops over all pairs.  M is nspec arrays of n
 * masses, read; Mout receives the new masses (must not alias M).  Returns 0,
 * or -1 on invalid parameters. */
int mto_mass_transfer(const mto_params* p, int64_t n, const int64_t* X,
                      int32_t nspec, const double* const* M, double* const* Mout);

/* The same step via the dense matrix form (Eq. 5-6, sign as in Eq. 4):
 * builds P (n x n), then Pcal = 1/2 [P - diag(P 1)], then dM = Pcal M by a
 * naive matrix-vector product.  For n <= 4096. */
int mto_mass_transfer_matrix(const mto_params* p, int64_t n, const int64_t* X,
                             int32_t nspec, const double* const* M,
                             double* const* Mout);

/* The same step for a subset of particles only, each computed from its plain
 * definition over all n particles (for sampled checks at large n): out[s] is
 * the new mass of particle idx[s] for each species.  out is nspec arrays of
 * nsample entries. */
int mto_mass_transfer_sample(const mto_params* p, int64_t n, const int64_t* X,
                             int32_t nspec, const double* const* M,
                             int64_t nsample, const int64_t* idx,
                             double* const* out);

/* 1-d only: the same step with the fixed-radius search done by sorting the
 * particles by position and scanning windows (Sec. 2.1's sparse search, no
 * tree).  Visits exactly the pairs the cutoff admits.  Its per-particle
 * loops run on mto_set_threads() threads (1 by default); each particle's
 * sums are the same whatever the thread count. */
int mto_mass_transfer_sorted_1d(const mto_params* p, int64_t n,
                                const int64_t* X, int32_t nspec,
                                const double* const* M, double* const* Mout);

/* Threads for the sorted-window transfer's per-particle loops when the
 * oracle is built with OpenMP (for the all-cores CPU baseline); returns the
 * count in effect (1 without OpenMP). */
int mto_set_threads(int32_t threads);

/* Irreversible equilibrium reaction per particle (Sec. 3, Sec. 7). */
void mto_react(int64_t n, double* A, double* B);

/* Unordered pairs {i, j}, i < j, within the cutoff, by testing all pairs.
 * Writes at most cap pairs in (i ascending, j ascending) order; returns the
 * total count. */
int64_t mto_pairs_brute(const mto_params* p, int64_t n, const int64_t* X,
                        int64_t cap, int32_t* pi, int32_t* pj);

/* 1-d only: the same pair set via sort and window scan.  Pairs are written as
 * (min, max) in no particular order; returns the total count. */
int64_t mto_pairs_sorted_1d(const mto_params* p, int64_t n, const int64_t* X,
                            int64_t cap, int32_t* pi, int32_t* pj);

/* One full time step in the paper's order (Sec. 1.1, Sec. 7): move, mass
 * transfer of A and B (sorted-window search in 1-d with a cutoff, else the
 * plain all-pairs loop), then the reaction.  A and B are updated in place
 * (a scratch copy is allocated internally).  Returns 0 or -1. */
int mto_step(const mto_params* p, int64_t n, int64_t* X, const float* xi,
             double* A, double* B);

/* Sum A, sum B, sum (A - B), mean A, in index order. */
void mto_observables(int64_t n, const double* A, const double* B, double out[4]);

#ifdef __cplusplus
}
#endif
#endif
