/*
 * mt_oracle.c -- plain, slow CPU FP64 oracle for the mass-transfer particle
 * tracking step (arXiv 1811.05474).  TEST INFRASTRUCTURE ONLY: see
 * mt_oracle.h for what each function computes and which passage of the paper
 * it follows.  Built with -O2 -ffp-contract=off so that no multiply-add is
 * fused; every loop runs in index order on one thread.
 */
#include "mt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-particle loops of the sorted-window transfer (1 unless
 * set; each particle's sums are computed alone, in the same order, whatever
 * the thread count, so results do not depend on it). */
static int g_threads = 1;

int mto_set_threads(int32_t threads) {
#ifdef _OPENMP
  g_threads = threads >= 1 ? threads : 1;
  return g_threads;
#else
  (void)threads;
  g_threads = 1;
  return 1;
#endif
}

int64_t mto_quantize(double x, int32_t k) { return llrint(ldexp(x, k)); }

double mto_dequantize(int64_t X, int32_t k) { return ldexp((double)X, -k); }

void mto_quantize_n(int64_t n, const double* x, int32_t k, int64_t* X) {
  for (int64_t i = 0; i < n; ++i) X[i] = mto_quantize(x[i], k);
}

void mto_dequantize_n(int64_t n, const int64_t* X, int32_t k, double* x) {
  for (int64_t i = 0; i < n; ++i) x[i] = mto_dequantize(X[i], k);
}

int64_t mto_cutoff_ticks(const mto_params* p) {
  return (int64_t)floor(ldexp(p->smax, p->frac_bits));
}

static int valid(const mto_params* p) {
  if (p->dim != 1 && p->dim != 2) return 0;
  if (p->frac_bits < 0 || p->frac_bits > 62) return 0;
  if (!(p->D_mt > 0.0) || !(p->dt > 0.0) || !(p->D_rw >= 0.0)) return 0;
  if (p->norm != MTO_NORM_SYM && p->norm != MTO_NORM_ROW) return 0;
  if (p->search != MTO_SEARCH_CUTOFF && p->search != MTO_SEARCH_FULL) return 0;
  if (p->walls != MTO_WALLS_REFLECT && p->walls != MTO_WALLS_PERIODIC) return 0;
  if (p->walls == MTO_WALLS_PERIODIC && p->search == MTO_SEARCH_CUTOFF)
    for (int32_t d = 0; d < p->dim; ++d) /* one image per pair: 2 Smax < L */
      if (2 * (int64_t)floor(ldexp(p->smax, p->frac_bits)) >= llrint(ldexp(p->L[d], p->frac_bits)))
        return 0;
  if (p->search == MTO_SEARCH_CUTOFF) {
    if (!(p->smax >= 0.0)) return 0;
    /* |dX|, |dY| <= Smax < 2^31 keeps dX^2 + dY^2 inside 63 bits. */
    if (ldexp(p->smax, p->frac_bits) >= 2147483648.0) return 0;
  }
  return 1;
}

/* ---------------------------------------------------------------- move --- */

/* Mirror y back into [0, Lq] at whichever wall it crossed (Sec. 3: particles
 * that leave the domain are reflected back into it). */
static int64_t reflect(int64_t y, int64_t Lq) {
  for (int it = 0; it < 64; ++it) {
    if (y < 0)
      y = -y;
    else if (y > Lq)
      y = 2 * Lq - y;
    else
      return y;
  }
  return y < 0 ? 0 : (y > Lq ? Lq : y);
}

/* Periodic walls: y taken modulo Lq into [0, Lq). */
static int64_t wrap(int64_t y, int64_t Lq) {
  const int64_t m = y % Lq;
  return m < 0 ? m + Lq : m;
}

void mto_move(const mto_params* p, int64_t n, int64_t* X, const float* xi) {
  const int32_t k = p->frac_bits;
  /* Eq. 2 with alpha_L = 0: the random walk carries D_rw (Sec. 3).  The
   * displacement sqrt(2 D_rw dt) xi is a binary64 product (in grid units,
   * b = sqrt(2 D_rw dt) 2^k), rounded once to the nearest tick. */
  const double b = ldexp(sqrt(2.0 * p->D_rw * p->dt), k);
  for (int32_t d = 0; d < p->dim; ++d) {
    const int64_t drift = llrint(ldexp(p->v[d] * p->dt, k));
    const int64_t Lq = llrint(ldexp(p->L[d], k));
    for (int64_t i = 0; i < n; ++i) {
      const double step = b * (double)xi[(int64_t)d * n + i];
      const int64_t y = X[(int64_t)d * n + i] + drift + (int64_t)llrint(step);
      X[(int64_t)d * n + i] = p->walls == MTO_WALLS_PERIODIC ? wrap(y, Lq) : reflect(y, Lq);
    }
  }
}

/* ------------------------------------------------------- pair relation --- */

/* Is the pair (i, j) inside the cutoff?  Exact integer test on tick
 * differences (Sec. 2.1: all pairs within s_max). */
static int in_range(const mto_params* p, int64_t S, int64_t dx, int64_t dy) {
  if (p->search == MTO_SEARCH_FULL) return 1;
  const uint64_t ax = (uint64_t)(dx < 0 ? -dx : dx);
  if (ax > (uint64_t)S) return 0;
  if (p->dim == 1) return 1;
  const uint64_t ay = (uint64_t)(dy < 0 ? -dy : dy);
  if (ay > (uint64_t)S) return 0;
  return ax * ax + ay * ay <= (uint64_t)S * (uint64_t)S;
}

/* Eq. 3 without its prefactor: exp(-s^2 / (8 D_mt dt)). */
static double weight(const mto_params* p, double inv8, int64_t dx, int64_t dy) {
  const double sx = ldexp((double)dx, -p->frac_bits);
  double s2 = sx * sx;
  if (p->dim == 2) {
    const double sy = ldexp((double)dy, -p->frac_bits);
    s2 = s2 + sy * sy;
  }
  return exp(-(s2 * inv8));
}

static double inv8(const mto_params* p) { return 1.0 / (8.0 * p->D_mt * p->dt); }

/* Separation X_j - X_i along axis d; with periodic walls the minimum image,
 * in (-Lq/2, Lq/2]. */
static int64_t sep(const mto_params* p, int32_t d, int64_t xi_, int64_t xj) {
  int64_t s = xj - xi_;
  if (p->walls == MTO_WALLS_PERIODIC) {
    const int64_t Lq = llrint(ldexp(p->L[d], p->frac_bits));
    if (2 * s > Lq) s -= Lq;
    else if (2 * s <= -Lq) s += Lq;
  }
  return s;
}

static int64_t dX(const mto_params* p, int64_t n, const int64_t* X, int64_t i,
                  int64_t j) {
  (void)n;
  return sep(p, 0, X[i], X[j]);
}

static int64_t dY(const mto_params* p, int64_t n, const int64_t* X, int64_t i,
                  int64_t j) {
  return p->dim == 2 ? sep(p, 1, X[n + i], X[n + j]) : 0;
}

/* ------------------------------------------------------------- weights --- */

void mto_row_sums(const mto_params* p, int64_t n, const int64_t* X, double* r) {
  const int64_t S = mto_cutoff_ticks(p);
  const double c = inv8(p);
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      const int64_t dx = dX(p, n, X, i, j), dy = dY(p, n, X, i, j);
      if (in_range(p, S, dx, dy)) s += weight(p, c, dx, dy);
    }
    r[i] = s;
  }
}

/* Normalised weight of the ordered pair (i, j) given w = nu_ij and the row
 * sums: the paper's row normalisation P_ij = nu_ij / sum_j nu_ij, or the
 * symmetric (P_ij + P_ji) / 2. */
static double normalised(const mto_params* p, double w, double ri, double rj) {
  if (p->norm == MTO_NORM_ROW) return w / ri;
  return 0.5 * (w / ri + w / rj);
}

/* ------------------------------------------------------- mass transfer --- */

int mto_mass_transfer(const mto_params* p, int64_t n, const int64_t* X,
                      int32_t nspec, const double* const* M,
                      double* const* Mout) {
  if (!valid(p) || n < 0 || nspec < 1) return -1;
  const int64_t S = mto_cutoff_ticks(p);
  const double c = inv8(p);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  if (!r) return -1;
  mto_row_sums(p, n, X, r);
  for (int32_t s = 0; s < nspec; ++s) {
    for (int64_t i = 0; i < n; ++i) {
      double acc = 0.0; /* sum_j P_ij (M_j - M_i), Eq. 4 */
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const int64_t dx = dX(p, n, X, i, j), dy = dY(p, n, X, i, j);
        if (!in_range(p, S, dx, dy)) continue;
        const double w = weight(p, c, dx, dy);
        acc += normalised(p, w, r[i], r[j]) * (M[s][j] - M[s][i]);
      }
      Mout[s][i] = M[s][i] + 0.5 * acc; /* Eq. 7 */
    }
  }
  free(r);
  return 0;
}

int mto_mass_transfer_matrix(const mto_params* p, int64_t n, const int64_t* X,
                             int32_t nspec, const double* const* M,
                             double* const* Mout) {
  if (!valid(p) || n < 0 || n > 4096 || nspec < 1) return -1;
  const int64_t S = mto_cutoff_ticks(p);
  const double c = inv8(p);
  const size_t nn = (size_t)(n > 0 ? n : 1);
  double* nu = (double*)calloc(nn * nn, sizeof(double));
  double* P = (double*)calloc(nn * nn, sizeof(double));
  double* r = (double*)calloc(nn, sizeof(double));
  if (!nu || !P || !r) {
    free(nu); free(P); free(r);
    return -1;
  }
  /* nu_ij (Eq. 3) as a dense matrix, zero outside the cutoff. */
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      const int64_t dx = dX(p, n, X, i, j), dy = dY(p, n, X, i, j);
      if (in_range(p, S, dx, dy)) nu[i * n + j] = weight(p, c, dx, dy);
    }
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += nu[i * n + j];
    r[i] = s;
  }
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j)
      P[i * n + j] = normalised(p, nu[i * n + j], r[i], r[j]);
  /* Pcal = 1/2 [P - diag(P 1)] (Eq. 6 with the sign of Eq. 4), then
   * dM = Pcal M (Eq. 5) and M + dM (Eq. 7). */
  for (int64_t i = 0; i < n; ++i) {
    double rowP = 0.0;
    for (int64_t j = 0; j < n; ++j) rowP += P[i * n + j];
    for (int64_t j = 0; j < n; ++j) P[i * n + j] *= 0.5;
    P[i * n + i] -= 0.5 * rowP;
  }
  for (int32_t s = 0; s < nspec; ++s)
    for (int64_t i = 0; i < n; ++i) {
      double dm = 0.0;
      for (int64_t j = 0; j < n; ++j) dm += P[i * n + j] * M[s][j];
      Mout[s][i] = M[s][i] + dm;
    }
  free(nu); free(P); free(r);
  return 0;
}

static double row_sum_one(const mto_params* p, int64_t n, const int64_t* X,
                          int64_t i, int64_t S, double c) {
  double s = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    const int64_t dx = dX(p, n, X, i, j), dy = dY(p, n, X, i, j);
    if (in_range(p, S, dx, dy)) s += weight(p, c, dx, dy);
  }
  return s;
}

int mto_mass_transfer_sample(const mto_params* p, int64_t n, const int64_t* X,
                             int32_t nspec, const double* const* M,
                             int64_t nsample, const int64_t* idx,
                             double* const* out) {
  if (!valid(p) || n < 0 || nspec < 1) return -1;
  const int64_t S = mto_cutoff_ticks(p);
  const double c = inv8(p);
  for (int64_t t = 0; t < nsample; ++t) {
    const int64_t i = idx[t];
    if (i < 0 || i >= n) return -1;
    const double ri = row_sum_one(p, n, X, i, S, c);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (nspec > 8) return -1;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const int64_t dx = dX(p, n, X, i, j), dy = dY(p, n, X, i, j);
      if (!in_range(p, S, dx, dy)) continue;
      const double w = weight(p, c, dx, dy);
      const double rj = p->norm == MTO_NORM_SYM ? row_sum_one(p, n, X, j, S, c) : ri;
      const double P = normalised(p, w, ri, rj);
      for (int32_t s = 0; s < nspec; ++s) acc[s] += P * (M[s][j] - M[s][i]);
    }
    for (int32_t s = 0; s < nspec; ++s) out[s][t] = M[s][i] + 0.5 * acc[s];
  }
  return 0;
}

/* -------------------------------------------------- sorted 1-d search --- */

static const int64_t* g_sort_keys; /* qsort has no context argument */

static int by_position(const void* a, const void* b) {
  const int64_t i = *(const int64_t*)a, j = *(const int64_t*)b;
  if (g_sort_keys[i] < g_sort_keys[j]) return -1;
  if (g_sort_keys[i] > g_sort_keys[j]) return 1;
  return i < j ? -1 : (i > j ? 1 : 0);
}

static int64_t* sorted_order(int64_t n, const int64_t* X) {
  int64_t* ord = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!ord) return NULL;
  for (int64_t i = 0; i < n; ++i) ord[i] = i;
  g_sort_keys = X;
  qsort(ord, (size_t)n, sizeof(int64_t), by_position);
  return ord;
}

int mto_mass_transfer_sorted_1d(const mto_params* p, int64_t n,
                                const int64_t* X, int32_t nspec,
                                const double* const* M, double* const* Mout) {
  if (!valid(p) || p->dim != 1 || p->search != MTO_SEARCH_CUTOFF || n < 0 ||
      nspec < 1 || p->walls != MTO_WALLS_REFLECT)
    return -1;
  const int64_t S = mto_cutoff_ticks(p);
  const double c = inv8(p);
  int64_t* ord = sorted_order(n, X);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  int64_t* lo = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  int64_t* hi = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!ord || !r || !lo || !hi) {
    free(ord); free(r); free(lo); free(hi);
    return -1;
  }
  /* Window [lo[a], hi[a]] of sorted positions within Smax of position a. */
  int64_t b = 0, e = 0;
  for (int64_t a = 0; a < n; ++a) {
    const int64_t xa = X[ord[a]];
    while (xa - X[ord[b]] > S) ++b;
    if (e < a) e = a;
    while (e + 1 < n && X[ord[e + 1]] - xa <= S) ++e;
    lo[a] = b;
    hi[a] = e;
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
  for (int64_t a = 0; a < n; ++a) {
    const int64_t i = ord[a];
    double s = 0.0;
    for (int64_t q = lo[a]; q <= hi[a]; ++q) s += weight(p, c, X[ord[q]] - X[i], 0);
    r[a] = s;
  }
  for (int32_t s = 0; s < nspec; ++s)
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads)
#endif
    for (int64_t a = 0; a < n; ++a) {
      const int64_t i = ord[a];
      double acc = 0.0;
      for (int64_t q = lo[a]; q <= hi[a]; ++q) {
        if (q == a) continue;
        const int64_t j = ord[q];
        const double w = weight(p, c, X[j] - X[i], 0);
        acc += normalised(p, w, r[a], r[q]) * (M[s][j] - M[s][i]);
      }
      Mout[s][i] = M[s][i] + 0.5 * acc;
    }
  free(ord); free(r); free(lo); free(hi);
  return 0;
}

/* -------------------------------------------------------------- react --- */

void mto_react(int64_t n, double* A, double* B) {
  for (int64_t i = 0; i < n; ++i) {
    const double m = A[i] < B[i] ? A[i] : B[i];
    A[i] = A[i] - m;
    B[i] = B[i] - m;
  }
}

/* -------------------------------------------------------------- pairs --- */

int64_t mto_pairs_brute(const mto_params* p, int64_t n, const int64_t* X,
                        int64_t cap, int32_t* pi, int32_t* pj) {
  if (!valid(p)) return -1;
  const int64_t S = mto_cutoff_ticks(p);
  int64_t cnt = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j) {
      const int64_t dx = dX(p, n, X, i, j), dy = dY(p, n, X, i, j);
      if (!in_range(p, S, dx, dy)) continue;
      if (cnt < cap) {
        pi[cnt] = (int32_t)i;
        pj[cnt] = (int32_t)j;
      }
      ++cnt;
    }
  return cnt;
}

int64_t mto_pairs_sorted_1d(const mto_params* p, int64_t n, const int64_t* X,
                            int64_t cap, int32_t* pi, int32_t* pj) {
  if (!valid(p) || p->dim != 1 || p->search != MTO_SEARCH_CUTOFF ||
      p->walls != MTO_WALLS_REFLECT)
    return -1;
  const int64_t S = mto_cutoff_ticks(p);
  int64_t* ord = sorted_order(n, X);
  if (!ord) return -1;
  int64_t cnt = 0;
  for (int64_t a = 0; a < n; ++a)
    for (int64_t q = a + 1; q < n && X[ord[q]] - X[ord[a]] <= S; ++q) {
      if (cnt < cap) {
        const int64_t i = ord[a], j = ord[q];
        pi[cnt] = (int32_t)(i < j ? i : j);
        pj[cnt] = (int32_t)(i < j ? j : i);
      }
      ++cnt;
    }
  free(ord);
  return cnt;
}

/* --------------------------------------------------------------- step --- */

int mto_step(const mto_params* p, int64_t n, int64_t* X, const float* xi,
             double* A, double* B) {
  if (!valid(p) || n < 0) return -1;
  mto_move(p, n, X, xi);
  const size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
  double* A2 = (double*)malloc(sz);
  double* B2 = (double*)malloc(sz);
  if (!A2 || !B2) {
    free(A2); free(B2);
    return -1;
  }
  const double* M[2] = {A, B};
  double* Mo[2] = {A2, B2};
  int rc;
  if (p->dim == 1 && p->search == MTO_SEARCH_CUTOFF && p->walls == MTO_WALLS_REFLECT)
    rc = mto_mass_transfer_sorted_1d(p, n, X, 2, M, Mo);
  else
    rc = mto_mass_transfer(p, n, X, 2, M, Mo);
  if (rc == 0) {
    memcpy(A, A2, sz > 0 && n > 0 ? sz : 0);
    memcpy(B, B2, sz > 0 && n > 0 ? sz : 0);
    if (p->react) mto_react(n, A, B);
  }
  free(A2); free(B2);
  return rc;
}

void mto_observables(int64_t n, const double* A, const double* B, double out[4]) {
  double sa = 0.0, sb = 0.0, sd = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    sa += A[i];
    sb += B[i];
    sd += A[i] - B[i];
  }
  out[0] = sa;
  out[1] = sb;
  out[2] = sd;
  out[3] = n > 0 ? sa / (double)n : 0.0;
}
