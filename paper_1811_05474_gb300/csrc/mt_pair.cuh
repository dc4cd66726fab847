// mt_pair.cuh -- per-pair arithmetic shared by the transfer kernels: the
// exact cutoff test, the co-location weight (Eq. 3), the normalisation
// (Sec. 1.1), and mass access / accumulation / update / reaction in each
// precision (Eq. 4, Eq. 7; Sec. 3 reaction).
#pragma once

#include "mt_internal.cuh"

namespace mt {

// ---------------------------------------------------------- pair weights --

__device__ __forceinline__ bool in_range2(long long dx, long long dy, long long S) {
  const unsigned long long ax = (unsigned long long)(dx < 0 ? -dx : dx);
  const unsigned long long ay = (unsigned long long)(dy < 0 ? -dy : dy);
  if (ax > (unsigned long long)S || ay > (unsigned long long)S) return false;
  return ax * ax + ay * ay <= (unsigned long long)S * (unsigned long long)S;
}

// nu_ij without its prefactor (it cancels in the normalisation):
// exp(-s^2 / (8 D_mt dt)) with s = |dX| 2^-k (Eq. 3).
template <bool MIX, int DIM>
struct Weight;

// ------------------------------------------------- binary64 exponential --
// exp(-t) for t >= 0 in binary64 (the weights of Eq. 3 in MT_FP64), by
// Tang's table-driven method (P. T. P. Tang, ACM TOMS 15(2), 1989): with
// k = rint(-t 32/ln2) = 32 m + j (0 <= j < 32) and r = -t - k ln2/32
// (|r| <= ln2/64; ln2/32 split into a 37-bit head, so that k times it is
// exact for |k| < 2^16, and a tail), exp(-t) = 2^m 2^(j/32) e^r, where
// 2^(j/32) comes from a table of its correctly rounded values and e^r - 1
// = r + r^2 q(r) from the Taylor polynomial of degree 6 (truncation below
// 2^-57 relative for |r| <= ln2/64).  The result is 2^(j/32) + 2^(j/32)
// (e^r - 1) with one rounding, then scaled by 2^m in its exponent field.
// Error about 1 ulp; 11 binary64 operations.
__constant__ double kExp2j32[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0,
};
__device__ __forceinline__ double exp_neg(double t) {
  if (!(t <= 745.5)) return t > 745.5 ? 0.0 : t + t;  // underflow; a NaN stays one
  const double x = -t;
  const double kMagic = 0x1.8p52;  // rint by addition: ulp 1 at 1.5 * 2^52
  const double kd = __fma_rn(x, 0x1.71547652b82fep+5, kMagic);  // x 32 / ln2
  const int k = (int)(unsigned int)(unsigned long long)__double_as_longlong(kd);
  const double kf = kd - kMagic;
  double r = __fma_rn(-kf, 0x1.62e42fefa0000p-6, x);  // head of ln2 / 32
  r = __fma_rn(-kf, 0x1.cf79abc9e3b3ap-45, r);        // tail
  double q = __fma_rn(r, 0x1.6c16c16c16c17p-10, 0x1.1111111111111p-7);  // 1/720, 1/120
  q = __fma_rn(r, q, 0x1.5555555555555p-5);                               // 1/24
  q = __fma_rn(r, q, 0x1.5555555555555p-3);                               // 1/6
  q = __fma_rn(r, q, 0.5);
  const double em1 = __fma_rn(__dmul_rn(r, r), q, r);
  const double T = kExp2j32[k & 31];
  const double res = __fma_rn(T, em1, T);
  const int m = k >> 5;
  if (m >= -1021)
    return __longlong_as_double(__double_as_longlong(res) + ((long long)m << 52));
  return scalbn(res, m);  // a subnormal result
}

template <int DIM>
struct Weight<false, DIM> {
  using T = double;
  static __device__ __forceinline__ double eval(const Dev& d, long long dx, long long dy) {
    const double sx = __dmul_rn((double)dx, d.scale);
    double s2 = __dmul_rn(sx, sx);
    if (DIM == 2) {
      const double sy = __dmul_rn((double)dy, d.scale);
      s2 = __dadd_rn(s2, __dmul_rn(sy, sy));
    }
    return exp_neg(__dmul_rn(s2, d.inv8));
  }
  // 1-d, |D| <= Smax < 2^30: the same value as eval(d, D, 0), since
  // (D 2^-k)^2 rounds to fl(D^2) 2^-2k and inv8 2^-2k is exact
  static __device__ __forceinline__ double near(const Dev& d, long long D) {
    const double dd = i2d_exact((int)D);  // (the binary64 pipe is kept for arithmetic)
    return exp_neg(__dmul_rn(__dmul_rn(dd, dd), d.inv8s));
  }
};

template <int DIM>
struct Weight<true, DIM> {
  using T = float;
  static __device__ __forceinline__ float eval(const Dev& d, long long dx, long long dy) {
    const float fx = ll_to_float(dx);
    float s2 = __fmul_rn(fx, fx);
    if (DIM == 2) {
      const float fy = ll_to_float(dy);
      s2 = __fadd_rn(s2, __fmul_rn(fy, fy));
    }
    return __expf(-__fmul_rn(s2, d.inv8f));
  }
  // 1-d, |D| <= Smax < 2^30 (the same value as eval(d, D, 0))
  static __device__ __forceinline__ float near(const Dev& d, long long D) {
    const float f = __int2float_rn((int)D);
    return __expf(-__fmul_rn(__fmul_rn(f, f), d.inv8f));
  }
};

// Binary32 weights, normalised weights and 1 / r_i: both mixed precisions.
constexpr bool mixw(int precision) { return precision != MT_FP64; }

// ------------------------------------------------------------ mass access --

template <int PR>
struct Mass;

// Per-particle accumulation of sum_j P_ij (M_j - M_i): binary64 in MT_FP64
// and MT_MIXED; in MT_MIXED_DF32 the binary32 terms are summed by cascaded
// compensated summation (Ogita, Rump & Oishi's Sum2): each addition's exact rounding error, from
// Knuth's two-sum, is added into a second sum, and the pair (s, c) is used
// unrounded.  The flux P_ij (M_j - M_i) is bitwise antisymmetric between i
// and j, so the transfer conserves mass to the pair's precision.
struct kahan {
  float s, c;
};
template <>
struct Mass<MT_FP64> {
  using V = double;
  using Acc = double;
  // the product and the accumulation as one fused multiply-add
  static __device__ __forceinline__ void acc(double& a, double P, double d) {
    a = __fma_rn(P, d, a);
  }
  static __device__ __forceinline__ double load(const unsigned long long* M, long long i) {
    return f64_load(M, i);
  }
  static __device__ __forceinline__ void store(unsigned long long* M, long long i, double v) {
    f64_store(M, i, v);
  }
  static __device__ __forceinline__ double diff(double a, double b) { return a - b; }
  // M + dM/2 (Eq. 7 with the 1/2 of Eq. 4), then the reaction.
  static __device__ __forceinline__ void update(double& A, double& B, double dA, double dB,
                                                int react) {
    A = __fma_rn(0.5, dA, A);  // 0.5 dA is exact: the same as A + 0.5 dA
    B = __fma_rn(0.5, dB, B);
    if (react) {  // min(A, B) off both: the smaller becomes exactly 0
      if (A < B) {
        B = B - A;
        A = 0.0;
      } else {
        A = A - B;
        B = 0.0;
      }
    }
  }
  static __device__ __forceinline__ double to_double(double v) { return v; }
};

// MT_MIXED: the normalised weight P is binary32; the masses, the
// difference M_j - M_i, the flux term P (M_j - M_i) (P widened exactly), its
// sum, the update and the reaction are binary64.
template <>
struct Mass<MT_MIXED> {
  using V = double;
  using Acc = double;
  static __device__ __forceinline__ void acc(double& a, float P, double d) {
    a = __fma_rn(widen_exact(P), d, a);
  }
  static __device__ __forceinline__ double load(const unsigned long long* M, long long i) {
    return f64_load(M, i);
  }
  static __device__ __forceinline__ void store(unsigned long long* M, long long i, double v) {
    f64_store(M, i, v);
  }
  static __device__ __forceinline__ double diff(double a, double b) { return a - b; }
  static __device__ __forceinline__ void update(double& A, double& B, double dA, double dB,
                                                int react) {
    Mass<MT_FP64>::update(A, B, dA, dB, react);
  }
  static __device__ __forceinline__ double to_double(double v) { return v; }
};

// MT_MIXED_DF32: masses as unevaluated sums of two binary32 numbers, flux
// terms in binary32 summed with compensation, compensated update and
// reaction (binary32 arithmetic only).
template <>
struct Mass<MT_MIXED_DF32> {
  using V = df;
  using Acc = kahan;
  static __device__ __forceinline__ void acc(kahan& a, float P, float d) {
    const df e = two_sum(a.s, __fmul_rn(P, d));
    a.s = e.hi;
    a.c = __fadd_rn(a.c, e.lo);
  }
  static __device__ __forceinline__ df load(const unsigned long long* M, long long i) {
    return df_load(M, i);
  }
  static __device__ __forceinline__ void store(unsigned long long* M, long long i, df v) {
    df_store(M, i, v);
  }
  static __device__ __forceinline__ float diff(df a, df b) {
    return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
  }
  static __device__ __forceinline__ void update(df& A, df& B, kahan dA, kahan dB, int react) {
    A = df_add(A, {0.5f * dA.s, 0.5f * dA.c});
    B = df_add(B, {0.5f * dB.s, 0.5f * dB.c});
    if (react) {
      if (df_le(A, B)) {
        B = df_sub(B, A);
        A = {0.0f, 0.0f};
      } else {
        A = df_sub(A, B);
        B = {0.0f, 0.0f};
      }
    }
  }
  static __device__ __forceinline__ double to_double(df v) { return (double)v.hi + (double)v.lo; }
};

// The two mass arrays one exchange pass works on (word offsets into a mass
// buffer of nspec * n words): A and B, or the extra species sp and sp + 1;
// when sp is the last species the second array repeats it and is not
// stored.
struct SpeciesPair {
  long long oa, ob;
  bool store_b;
};
template <bool TR>
__device__ __forceinline__ SpeciesPair species_pair(const Dev& d, int sp) {
  if (!TR) return {0, d.n, true};
  const bool two = sp + 1 < d.nspec;
  return {(long long)sp * d.n, (long long)(two ? sp + 1 : sp) * d.n, two};
}

// Row sum r_i over a dense neighbourhood (hundreds to thousands of terms):
// binary64, or with binary32 weights a binary32 sum with each addition's rounding error
// (Knuth's two-sum) collected in a second term, so the sum keeps about twice
// binary32's precision however many weights it adds.
template <bool MIX>
struct RowSum;
template <>
struct RowSum<false> {
  double r;
  __device__ __forceinline__ explicit RowSum(double v) : r(v) {}
  __device__ __forceinline__ void add(double w) { r += w; }
  __device__ __forceinline__ double value() const { return r; }
};
template <>
struct RowSum<true> {
  float s, c;
  __device__ __forceinline__ explicit RowSum(float v) : s(v), c(0.0f) {}
  __device__ __forceinline__ void add(float w) {
    const df e = two_sum(s, w);
    s = e.hi;
    c = __fadd_rn(c, e.lo);
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, c); }
};

template <bool MIX>
__device__ __forceinline__ void store_rinv(const Dev& d, long long p, typename Weight<MIX, 1>::T r) {
  if (MIX)
    static_cast<float*>(d.rinv)[p] = __frcp_rn((float)r);
  else
    static_cast<double*>(d.rinv)[p] = rcp_ge1((double)r);
}

template <bool MIX>
__device__ __forceinline__ typename Weight<MIX, 1>::T load_rinv(const Dev& d, long long p) {
  if (MIX)
    return static_cast<const float*>(d.rinv)[p];
  else
    return static_cast<const double*>(d.rinv)[p];
}

// Normalised weight of the ordered pair (p, q) (Sec. 1.1): ROW w / r_p, or
// SYM (w / r_p + w / r_q) / 2.
template <typename T>
__device__ __forceinline__ T normalised(int norm, T w, T ip, T iq) {
  return norm == MT_NORM_ROW ? w * ip : T(0.5) * w * (ip + iq);
}

// Combining per-lane partial sums in a fixed shuffle tree (warp-cooperative
// sums over a dense neighbourhood): row sums in T, flux accumulators in Acc.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double acc_warp_sum(double v) { return warp_sum(v); }
__device__ __forceinline__ double acc_merge(double a, double b) { return a + b; }
__device__ __forceinline__ kahan acc_merge(kahan a, kahan b) {
  const df e = two_sum(a.s, b.s);
  return {e.hi, __fadd_rn(__fadd_rn(a.c, b.c), e.lo)};
}
// Exact halving of a flux sum (a power-of-two scaling of both terms).
__device__ __forceinline__ double acc_half(double a) { return 0.5 * a; }
__device__ __forceinline__ kahan acc_half(kahan a) { return {0.5f * a.s, 0.5f * a.c}; }
__device__ __forceinline__ kahan acc_warp_sum(kahan v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_down_sync(0xffffffffu, v.s, o);
    const float c2 = __shfl_down_sync(0xffffffffu, v.c, o);
    const df e = two_sum(v.s, s2);
    v.s = e.hi;
    v.c = __fadd_rn(__fadd_rn(v.c, c2), e.lo);
  }
  return v;
}

// Observables arithmetic: sums in the precision's own format (binary64 or
// double-binary32), converted to binary64 per CTA.
__device__ __forceinline__ double obs_add(double a, double b) { return a + b; }
__device__ __forceinline__ df obs_add(df a, df b) { return df_add(a, b); }
__device__ __forceinline__ double obs_shfl(double v, int o) {
  return __shfl_down_sync(0xffffffffu, v, o);
}
__device__ __forceinline__ df obs_shfl(df v, int o) {
  return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ double obs_double(double v) { return v; }
__device__ __forceinline__ double obs_double(df v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ double obs_diff(double a, double b) { return a - b; }
__device__ __forceinline__ df obs_diff(df a, df b) { return df_sub(a, b); }

// Fixed-order reductions of the observables sums (three values).
template <typename MV>
struct Obs3 {
  MV a, b, d;
};
template <typename MV>
__device__ __forceinline__ Obs3<MV> obs3_add(Obs3<MV> x, Obs3<MV> y) {
  return {obs_add(x.a, y.a), obs_add(x.b, y.b), obs_add(x.d, y.d)};
}
template <typename MV>
__device__ __forceinline__ Obs3<MV> obs3_warp(Obs3<MV> v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = obs3_add(v, Obs3<MV>{obs_shfl(v.a, o), obs_shfl(v.b, o), obs_shfl(v.d, o)});
  return v;
}
// Block-wide (NT threads): warp trees, then warp 0 over the warp totals;
// the result is valid in thread 0.  Called by every thread.
template <typename MV, int NT>
__device__ __forceinline__ Obs3<MV> obs3_block(Obs3<MV> v, Obs3<MV>* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = obs3_warp(v);
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  Obs3<MV> t{};
  if (warp == 0) {
    if (lane < NT / 32) t = s_w[lane];
    t = obs3_warp(t);
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ double ldcg_obs(const double* p) { return __ldcg(p); }
__device__ __forceinline__ df ldcg_obs(const df* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return {v.x, v.y};
}

template <typename MV>
__device__ __forceinline__ void obs_row(const Dev& d, long long row, int r, long long n,
                                        Obs3<MV> t) {
  double* o = d.obs + 4 * (row * d.nreal + r);
  const double a = obs_double(t.a);
  o[0] = a;
  o[1] = obs_double(t.b);
  o[2] = obs_double(t.d);
  o[3] = a / (double)n;
}


}  // namespace mt
