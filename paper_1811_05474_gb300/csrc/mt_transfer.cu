// mt_transfer.cu -- weights (Eq. 3), normalisation (Sec. 1.1), exchange
// (Eq. 4, Eq. 7) and the A + B -> E reaction (Sec. 3, Sec. 7), in two
// passes: pass 1 forms the row sums r_i = sum_j nu_ij (self included) and
// stores 1 / r_i; pass 2 forms dM_i = 1/2 sum_j P_ij (M_j - M_i) for A and B,
// updates, reacts and reduces the per-step observables.
//
// Neighbour search variants:
//   walk  (1-d cell list) particles are sorted by position, so the pairs of
//         particle p are the contiguous slots around p whose tick distance is
//         <= Smax; each thread walks left and right until it leaves range.
//   cell2 (2-d cell list) candidates are the 3 x 3 block of cells around the
//         particle's cell (cell width > Smax), contiguous per row.
//   brute all n particles in shared-memory tiles, with (BRUTE) or without
//         (FULL, the paper's full-matrix reference) the cutoff test.
// Precision: mixw(PR) = false is IEEE binary64 throughout; mixw(PR) = true forms
// weights and normalised weights in binary32 and updates the double-binary32
// masses with compensated additions.
#include "mt_pair.cuh"

namespace mt {

// ------------------------------------------- step epilogue (last CTA) --
// The last CTA of a step's final pass advances the step counter and flips
// the buffer selectors.  Called by every thread.
__device__ void finish_step(const Dev& d, int flip_x, int flip_m) {
  __shared__ bool s_last;
  Ctrl* c = d.ctrl;
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&c->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  c->step += 1;
  c->xcur ^= flip_x;
  c->mcur ^= flip_m;
  c->done = 0;
}

// ------------------------------------------------------------ observables --
// After every step (every path): sum A, sum B, sum (A - B) and mean A of each
// realisation, one ring row per step (sum A and sum B are conserved by the
// symmetric transfer, sum (A - B) by the reaction too: the conservative
// components of Sec. 3).  Each realisation's slot range is cut
// into fixed chunks of kObsChunk slots (the state keeps a realisation's
// particles in its own range); a CTA sums one chunk -- each thread its
// strided slots in order, then fixed shuffle trees -- in the precision's
// own arithmetic (binary64, or double-binary32 in MIXED), and the CTA that
// completes a realisation's last chunk adds its chunk sums (thread-strided
// in order, then the block tree).  The result depends on
// the state only, not on how the step was scheduled.

// A thread's sums over its slots, in slot order: binary64, or in MIXED
// Sum2-style compensated sums of the double-binary32 masses (each high part
// added with Knuth's two-sum, the rounding errors and the low parts collected
// in a second term; as accurate here as double-binary32 additions, at a third
// of the operations).
template <int PR>
struct ThreadObs;
template <>
struct ThreadObs<false> {  // binary64 masses
  Obs3<double> v{};
  __device__ __forceinline__ void add(double a, double b) {
    v = obs3_add(v, Obs3<double>{a, b, a - b});
  }
  __device__ __forceinline__ Obs3<double> value() const { return v; }
};
template <>
struct ThreadObs<true> {  // double-binary32 masses
  kahan a{0.f, 0.f}, b{0.f, 0.f}, d{0.f, 0.f};
  static __device__ __forceinline__ void put(kahan& k, float hi, float lo) {
    const df e = two_sum(k.s, hi);
    k.s = e.hi;
    k.c = __fadd_rn(k.c, __fadd_rn(e.lo, lo));
  }
  __device__ __forceinline__ void add(df A, df B) {
    put(a, A.hi, A.lo);
    put(b, B.hi, B.lo);
    put(d, A.hi, A.lo);
    put(d, -B.hi, -B.lo);
  }
  __device__ __forceinline__ Obs3<df> value() const {
    return {fast_two_sum(a.s, a.c), fast_two_sum(b.s, b.c), fast_two_sum(d.s, d.c)};
  }
};

// PREV: the state at the step's start (obs_snapshot, by k_obs_snapshot or
// the predicted-segment kernel), while
// the step runs beside it (it writes the other mass buffer); otherwise the
// current state.  Either writes the row of the step the state follows.
template <int PR, bool PREV>
__global__ void __launch_bounds__(kThreads) k_obs(Dev d) {
  using MS = Mass<PR>;
  using MV = typename MS::V;
  constexpr int kPer = kObsChunk / kThreads;  // slots per thread
  __shared__ Obs3<MV> s_w[kThreads / 32];
  __shared__ bool s_last;
  Ctrl* c = d.ctrl;
  if (PREV && !c->obs_prev_todo) return;  // fixed before the launch: every CTA agrees
  const unsigned long long step = PREV ? c->obs_step : c->step;
  const int ch = blockIdx.x;
  const unsigned long long* M = d.M[PREV ? c->obs_mc : c->mcur];
  // this thread's slots: loaded together, then added in slot order
  const long long a0 = d.ochunk[ch], a1 = d.ochunk[ch + 1];
  MV va[kPer], vb[kPer];
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    const long long p = a0 + threadIdx.x + (long long)k * kThreads;
    va[k] = p < a1 ? MS::load(M, p) : MV{};
    vb[k] = p < a1 ? MS::load(M, d.n + p) : MV{};
  }
  ThreadObs<PR == MT_MIXED_DF32> acc;
#pragma unroll
  for (int k = 0; k < kPer; ++k) acc.add(va[k], vb[k]);
  const Obs3<MV> t = obs3_block<MV, kThreads>(acc.value(), s_w);
  MV* part = reinterpret_cast<MV*>(d.opart);  // 8-byte words, 4 per chunk
  const int r = d.ochr[ch];
  const Real R = d.rt[r];
  if (threadIdx.x == 0) {
    part[4 * ch + 0] = t.a;
    part[4 * ch + 1] = t.b;
    part[4 * ch + 2] = t.d;
    __threadfence();
    s_last = atomicAdd(&d.ocnt[r], 1) + 1 == R.nch;
  }
  __syncthreads();
  if (!s_last) return;
  // the realisation's last chunk: thread t adds its chunks t, t + 256, ...
  // in order (four in flight), then the block tree
  __threadfence();
  auto get = [&](int k) {
    return Obs3<MV>{ldcg_obs(&part[4 * k + 0]), ldcg_obs(&part[4 * k + 1]),
                    ldcg_obs(&part[4 * k + 2])};
  };
  const int k1 = R.ch0 + R.nch;
  Obs3<MV> u{};
  int k = R.ch0 + threadIdx.x;
  for (; k + 3 * kThreads < k1; k += 4 * kThreads) {
    const Obs3<MV> p0 = get(k), p1 = get(k + kThreads), p2 = get(k + 2 * kThreads),
                   p3 = get(k + 3 * kThreads);
    u = obs3_add(obs3_add(obs3_add(obs3_add(u, p0), p1), p2), p3);
  }
  for (; k < k1; k += kThreads) u = obs3_add(u, get(k));
  u = obs3_block<MV, kThreads>(u, s_w);
  if (threadIdx.x == 0) {
    const long long row = (long long)((step - 1) % (unsigned long long)d.observe_cap);
    obs_row(d, row, r, R.n, u);
    d.ocnt[r] = 0;
    c->obs_done_step = step;
  }
}

__global__ void k_obs_snapshot(Dev d) { obs_snapshot(d.ctrl); }

cudaError_t launch_obs_snapshot(const Dev& d, cudaStream_t s) {
  if (d.observe_cap <= 0 || d.nochunk <= 0) return cudaSuccess;
  k_obs_snapshot<<<1, 1, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_obs_prev(const Dev& d, int precision, cudaStream_t s) {
  if (d.observe_cap <= 0 || d.nochunk <= 0) return cudaSuccess;
  if (precision == MT_MIXED_DF32)
    k_obs<MT_MIXED_DF32, true><<<d.nochunk, kThreads, 0, s>>>(d);
  else
    k_obs<MT_FP64, true><<<d.nochunk, kThreads, 0, s>>>(d);  // binary64 masses
  return cudaGetLastError();
}

cudaError_t launch_obs(const Dev& d, int precision, cudaStream_t s) {
  if (d.observe_cap <= 0 || d.nochunk <= 0) return cudaSuccess;
  if (precision == MT_MIXED_DF32)
    k_obs<MT_MIXED_DF32, false><<<d.nochunk, kThreads, 0, s>>>(d);
  else
    k_obs<MT_FP64, false><<<d.nochunk, kThreads, 0, s>>>(d);  // binary64 masses
  return cudaGetLastError();
}

// ================================================================ 1-d walk ==

template <int PR>
__global__ void __launch_bounds__(kThreads) k_rowsum_walk(Dev d) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const long long* Xs = d.X[xc ^ 1];
  const long long x = Xs[p];
  T r = T(1);  // self: nu_pp = 1
  if (!d.periodic) {
    for (long long q = p - 1; q >= 0; --q) {
      const long long D = x - Xs[q];
      if (D > d.S) break;
      r += W::eval(d, D, 0);
    }
    for (long long q = p + 1; q < d.n; ++q) {
      const long long D = Xs[q] - x;
      if (D > d.S) break;
      r += W::eval(d, D, 0);
    }
  } else {
    // periodic: the walks continue around the realisation's ring (2 Smax <
    // L, so no slot is reached from both sides)
    const Ring g = ring_of(d, d.id[xc][d.src[p]]);
    for (long long k = 1; k < g.n; ++k) {
      const long long D = wrap(x - Xs[ring_step(g, p, -k)], g.Lq);
      if (D > d.S) break;
      r += W::eval(d, D, 0);
    }
    for (long long k = 1; k < g.n; ++k) {
      const long long D = wrap(Xs[ring_step(g, p, k)] - x, g.Lq);
      if (D > d.S) break;
      r += W::eval(d, D, 0);
    }
  }
  store_rinv<mixw(PR)>(d, p, r);
  // gather id and masses into the sorted slots (stage buffer)
  const int s = d.src[p];
  d.id[xc ^ 1][p] = d.id[xc][s];
  gather_masses(d, mc, p, s);
}

// TR = false: species A and B (species 0, 1), then the reaction, the
// observables and the end of the step.  TR = true: the extra species sp and
// sp + 1 (sp alone when it is the last), conservative, run before the A/B
// pass of the same step.
template <int PR, bool TR>
__global__ void __launch_bounds__(kThreads) k_exchange_walk(Dev d, int sp) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  const bool valid = p < d.n;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const SpeciesPair sq = species_pair<TR>(d, sp);
  MV A{}, B{};
  if (valid) {
    const long long* Xs = d.X[xc ^ 1];
    const unsigned long long* MA = d.M[mc ^ 1] + sq.oa;
    const unsigned long long* MB = d.M[mc ^ 1] + sq.ob;
    const long long x = Xs[p];
    const T ip = load_rinv<mixw(PR)>(d, p);
    A = MS::load(MA, p);
    B = MS::load(MB, p);
    typename MS::Acc dA{}, dB{};
    auto pair = [&](long long q, long long D) {
      const T P = normalised<T>(d.norm, W::eval(d, D, 0), ip, load_rinv<mixw(PR)>(d, q));
      MS::acc(dA, P, MS::diff(MS::load(MA, q), A));
      MS::acc(dB, P, MS::diff(MS::load(MB, q), B));
    };
    if (!d.periodic) {
      for (long long q = p - 1; q >= 0; --q) {
        const long long D = x - Xs[q];
        if (D > d.S) break;
        pair(q, D);
      }
      for (long long q = p + 1; q < d.n; ++q) {
        const long long D = Xs[q] - x;
        if (D > d.S) break;
        pair(q, D);
      }
    } else {
      const Ring g = ring_of(d, d.id[xc ^ 1][p]);
      for (long long k = 1; k < g.n; ++k) {
        const long long q = ring_step(g, p, -k);
        const long long D = wrap(x - Xs[q], g.Lq);
        if (D > d.S) break;
        pair(q, D);
      }
      for (long long k = 1; k < g.n; ++k) {
        const long long q = ring_step(g, p, k);
        const long long D = wrap(Xs[q] - x, g.Lq);
        if (D > d.S) break;
        pair(q, D);
      }
    }
    MS::update(A, B, dA, dB, TR ? 0 : d.react);
    MS::store(d.M[mc] + sq.oa, p, A);
    if (sq.store_b) MS::store(d.M[mc] + sq.ob, p, B);
  }
  if (!TR) finish_step(d, 1, 0);
}

// |dx| <= S in one unsigned comparison (1-d)
__device__ __forceinline__ bool within1(long long dx, long long S) {
  return (unsigned long long)(dx + S) <= (unsigned long long)(2 * S);
}

// ======================================================= 1-d dense tiles ==
// Dense neighbourhoods (tens to thousands of neighbours per particle): a CTA
// takes 256 consecutive sorted slots.  Each particle first finds its exact
// neighbour slots [jl, jr) (itself included) from the cell starts; the
// union over the CTA is one contiguous range, staged through shared memory
// in chunks of kTileChunk.  Each warp walks the union of its lanes' ranges
// with every lane reading the same slot (a shared-memory broadcast) and
// keeping the pair when the slot lies in its own range: an index test, no
// branch, and no data-dependent exit.  Inside the cutoff |dX| < 2^30, so the
// separation is the difference of the positions' low 32-bit words.  The
// particle itself adds nu_pp = 1 to r_p and an exact zero flux.

constexpr int kTileChunk = 512;
constexpr int kTileGroup = 16;  // row-sum terms added plainly before compensation

// Exact neighbour slots [jl, jr) of the particle at x: every sorted slot q
// with |X_q - x| <= Smax.  The bounds lie in the cells of x -/+ Smax.
__device__ __forceinline__ void exact_range(const Dev& d, const long long* Xs, long long x,
                                            long long& jl, long long& jr) {
  long long c = cell_of(d, x - d.S, 0);
  long long q = d.start[c], e = d.start[c + 1];
  while (q < e && Xs[q] < x - d.S) ++q;
  jl = q;
  c = cell_of(d, x + d.S, 0);
  q = d.start[c];
  e = d.start[c + 1];
  while (q < e && Xs[q] <= x + d.S) ++q;
  jr = q;
}

// The CTA's and the warp's candidate ranges from the lanes' exact ranges.
struct TileRanges {
  long long lo, hi;    // CTA: union of its particles' ranges
  long long wlo, whi;  // warp: union of its lanes' ranges (empty if no lane is valid)
};
__device__ __forceinline__ TileRanges tile_ranges(long long jl, long long jr, long long b0,
                                                  long long b1, long long* s_lohi) {
  const long long p = b0 + threadIdx.x;
  const long long w0 = b0 + (threadIdx.x & ~31);
  const int last = w0 < b1 ? (int)min(31LL, b1 - 1 - w0) : 0;
  TileRanges t;
  t.wlo = __shfl_sync(0xffffffffu, jl, 0);
  t.whi = __shfl_sync(0xffffffffu, jr, last);
  if (w0 >= b1) t.wlo = t.whi = 0;
  if (p == b0) s_lohi[0] = jl;
  if (p == b1 - 1) s_lohi[1] = jr;
  __syncthreads();
  t.lo = s_lohi[0];
  t.hi = s_lohi[1];
  return t;
}

template <int PR>
__global__ void __launch_bounds__(kThreads) k_rowsum_tile(Dev d) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  __shared__ unsigned int s_x[kTileChunk];
  __shared__ long long s_lohi[2];
  const long long b0 = (long long)blockIdx.x * kThreads;
  const long long b1 = min(b0 + (long long)kThreads, d.n);
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const long long* Xs = d.X[xc ^ 1];
  const long long p = b0 + threadIdx.x;
  const bool valid = p < b1;
  const long long x = valid ? Xs[p] : 0;
  long long jl = 0, jr = 0;
  if (valid) exact_range(d, Xs, x, jl, jr);
  const TileRanges t = tile_ranges(jl, jr, b0, b1, s_lohi);
  const unsigned int x32 = (unsigned int)x;
  // The weights are summed plainly in groups of kTileGroup candidates (two
  // chains) and each group's sum enters a compensated sum: the group sums'
  // rounding (at most kTileGroup terms of at most 1) stays near binary32's
  // precision relative to r_p, at a plain addition per weight.
  RowSum<mixw(PR)> r(T(0));
  for (long long c0 = t.lo; c0 < t.hi; c0 += kTileChunk) {
    const int nc = (int)min((long long)kTileChunk, t.hi - c0);
    for (int i = threadIdx.x; i < nc; i += kThreads) s_x[i] = (unsigned int)Xs[c0 + i];
    __syncthreads();
    const int j0 = (int)(max(t.wlo, c0) - c0), j1 = (int)(min(t.whi, c0 + nc) - c0);
    const int ql = (int)(jl - c0);
    const unsigned int qn = (unsigned int)(jr - jl);
    auto term = [&](int j) {
      const T w = W::near(d, (int)(s_x[j] - x32));
      return (unsigned int)(j - ql) < qn ? w : T(0);
    };
    int j = j0;
    for (; j + kTileGroup <= j1; j += kTileGroup) {
      T g0 = T(0), g1 = T(0);
#pragma unroll
      for (int k = 0; k < kTileGroup; k += 2) {
        g0 += term(j + k);
        g1 += term(j + k + 1);
      }
      r.add(g0 + g1);
    }
    T g = T(0);
    for (; j < j1; ++j) g += term(j);
    r.add(g);
    __syncthreads();
  }
  if (!valid) return;
  store_rinv<mixw(PR)>(d, p, r.value());
  const int s = d.src[p];
  d.id[xc ^ 1][p] = d.id[xc][s];
  gather_masses(d, mc, p, s);
}

template <int PR, bool TR>
__global__ void __launch_bounds__(kThreads) k_exchange_tile(Dev d, int sp) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  __shared__ unsigned int s_x[kTileChunk];
  __shared__ T s_r[kTileChunk];
  __shared__ MV s_a[kTileChunk];
  __shared__ MV s_b[kTileChunk];
  __shared__ long long s_lohi[2];
  const long long b0 = (long long)blockIdx.x * kThreads;
  const long long b1 = min(b0 + (long long)kThreads, d.n);
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const SpeciesPair sq = species_pair<TR>(d, sp);
  const long long* Xs = d.X[xc ^ 1];
  const unsigned long long* MA = d.M[mc ^ 1] + sq.oa;
  const unsigned long long* MB = d.M[mc ^ 1] + sq.ob;
  const long long p = b0 + threadIdx.x;
  const bool valid = p < b1;
  const long long x = valid ? Xs[p] : 0;
  long long jl = 0, jr = 0;
  if (valid) exact_range(d, Xs, x, jl, jr);
  const TileRanges t = tile_ranges(jl, jr, b0, b1, s_lohi);
  const unsigned int x32 = (unsigned int)x;
  // SYM: P = w (1/r_p + 1/r_q) / 2 is formed as 2P = w (1/r_p + 1/r_q) and
  // the sums are halved at the end; ROW: P = w / r_p (the staged 1/r_q is
  // 0).  Halving is exact, so the result is the same as with P.
  const bool sym = d.norm != MT_NORM_ROW;
  MV A{}, B{};
  T ip = T(0);
  if (valid) {
    A = MS::load(MA, p);
    B = MS::load(MB, p);
    ip = load_rinv<mixw(PR)>(d, p);
  }
  // two accumulator sets (even and odd candidates) halve the dependent
  // chain of compensated additions
  typename MS::Acc dA{}, dB{}, dA1{}, dB1{};
  for (long long c0 = t.lo; c0 < t.hi; c0 += kTileChunk) {
    const int nc = (int)min((long long)kTileChunk, t.hi - c0);
    for (int i = threadIdx.x; i < nc; i += kThreads) {
      s_x[i] = (unsigned int)Xs[c0 + i];
      s_r[i] = sym ? load_rinv<mixw(PR)>(d, c0 + i) : T(0);
      s_a[i] = MS::load(MA, c0 + i);
      s_b[i] = MS::load(MB, c0 + i);
    }
    __syncthreads();
    const int j0 = (int)(max(t.wlo, c0) - c0), j1 = (int)(min(t.whi, c0 + nc) - c0);
    const int ql = (int)(jl - c0);
    const unsigned int qn = (unsigned int)(jr - jl);
    auto pair = [&](int j, typename MS::Acc& a, typename MS::Acc& b) {
      const T w = W::near(d, (int)(s_x[j] - x32));
      const T P2 = (unsigned int)(j - ql) < qn ? w * (ip + s_r[j]) : T(0);
      MS::acc(a, P2, MS::diff(s_a[j], A));
      MS::acc(b, P2, MS::diff(s_b[j], B));
    };
    int j = j0;
    for (; j + 1 < j1; j += 2) {
      pair(j, dA, dB);
      pair(j + 1, dA1, dB1);
    }
    if (j < j1) pair(j, dA, dB);
    __syncthreads();
  }
  dA = acc_merge(dA, dA1);
  dB = acc_merge(dB, dB1);
  if (sym) {
    dA = acc_half(dA);
    dB = acc_half(dB);
  }
  if (valid) {
    MS::update(A, B, dA, dB, TR ? 0 : d.react);
    MS::store(d.M[mc] + sq.oa, p, A);
    if (sq.store_b) MS::store(d.M[mc] + sq.ob, p, B);
  }
  if (!TR) finish_step(d, 1, 0);
}

// ================================================== 1-d SPaM (stored P) ==
// The SPaM form of Sec. 6: the nonzero weights of the step's transfer
// matrix are stored and both passes read them, so each unordered pair's
// exponential is evaluated once.  In sorted order the nonzeros of row p are
// the contiguous slots around p: cnt_l(p) to the left and cnt_r(p) to the
// right.  The band keeps nu(p, p + k), k = 1 .. min(cnt_r(p), band_cap), in
// tiles of 32 slots: entry (p, k) is at ((p / 32) band_cap + k - 1) 32 +
// p % 32, so a warp reading its right neighbours streams one contiguous
// block, and reading its left neighbours (entries (p - k, k)) streams two
// adjacent ones.  Weights past the band are recomputed from the positions.
//   band_build     right neighbours: nu stored, right part of r_p, cnt_r;
//                  left count cnt_l; ids and masses into the sorted slots
//   band_rowsum    left part of r_p from the band -> 1 / r_p
//   band_exchange  Eq. 4 / 7 with the stored weights

__device__ __forceinline__ long long band_at(const Dev& d, long long q, long long k) {
  return (((q >> 5) * d.band_cap) + (k - 1)) * 32 + (q & 31);
}

// The slots a particle's walks cover: with periodic walls its realisation's
// ring; else the whole sorted range (realisations are separated by more than
// Smax, so the cutoff ends every walk inside its own realisation).
__device__ __forceinline__ Ring walk_ring(const Dev& d, int id) {
  return d.periodic ? ring_of(d, id) : Ring{0, d.n, 0};
}

// Slot k steps to the right (left for k < 0) of p.
__device__ __forceinline__ long long ring(const Dev& d, const Ring& g, long long p, long long k) {
  return d.periodic ? ring_step(g, p, k) : p + k;
}

// The longest right and left walks from slot p.
__device__ __forceinline__ long long walk_right(const Dev& d, const Ring& g, long long p) {
  return d.periodic ? g.n - 1 : d.n - 1 - p;
}
__device__ __forceinline__ long long walk_left(const Dev& d, const Ring& g, long long p) {
  return d.periodic ? g.n - 1 : p;
}

// Tick distance from slot q up to slot p (p to the right of q).
__device__ __forceinline__ long long gap(const Dev& d, const Ring& g, const long long* Xs,
                                         long long q, long long p) {
  return d.periodic ? wrap(Xs[p] - Xs[q], g.Lq) : Xs[p] - Xs[q];
}

template <int PR>
__global__ void __launch_bounds__(kThreads) k_band_build(Dev d) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const long long* Xs = d.X[xc ^ 1];
  T* band = static_cast<T*>(d.band);
  const int s = d.src[p];
  const Ring g = walk_ring(d, d.id[xc][s]);
  RowSum<mixw(PR)> r(T(0));
  long long k = 1;
  const long long kr = walk_right(d, g, p);
  for (; k <= kr; ++k) {
    const long long D = gap(d, g, Xs, p, ring(d, g, p, k));
    if (D > d.S) break;
    const T w = W::eval(d, D, 0);
    if (k <= d.band_cap) band[band_at(d, p, k)] = w;
    r.add(w);
  }
  d.cnt[p] = (int)(k - 1);
  const long long kl = walk_left(d, g, p);
  for (k = 1; k <= kl; ++k)
    if (gap(d, g, Xs, ring(d, g, p, -k), p) > d.S) break;
  d.cnt[d.n + p] = (int)(k - 1);
  static_cast<T*>(d.rinv)[p] = r.value();  // right part of r_p, completed by band_rowsum
  d.id[xc ^ 1][p] = d.id[xc][s];
  gather_masses(d, mc, p, s);
}

template <int PR>
__global__ void __launch_bounds__(kThreads) k_band_rowsum(Dev d) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const T* band = static_cast<const T*>(d.band);
  const int xc = d.ctrl->xcur;
  const Ring g = walk_ring(d, d.id[xc ^ 1][p]);
  RowSum<mixw(PR)> r(T(1));  // self
  r.add(static_cast<const T*>(d.rinv)[p]);  // right part
  const int kl = d.cnt[d.n + p];
  const int kb = kl < d.band_cap ? kl : d.band_cap;
#pragma unroll 4
  for (int k = 1; k <= kb; ++k) r.add(band[band_at(d, ring(d, g, p, -k), k)]);
  if (kl > kb) {
    const long long* Xs = d.X[xc ^ 1];
    for (int k = kb + 1; k <= kl; ++k) r.add(W::eval(d, gap(d, g, Xs, ring(d, g, p, -k), p), 0));
  }
  store_rinv<mixw(PR)>(d, p, r.value());
}

template <int PR, bool TR>
__global__ void __launch_bounds__(kThreads) k_band_exchange(Dev d, int sp) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  const bool valid = p < d.n;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const SpeciesPair sq = species_pair<TR>(d, sp);
  MV A{}, B{};
  if (valid) {
    const long long* Xs = d.X[xc ^ 1];
    const Ring g = walk_ring(d, d.id[xc ^ 1][p]);
    const unsigned long long* MA = d.M[mc ^ 1] + sq.oa;
    const unsigned long long* MB = d.M[mc ^ 1] + sq.ob;
    const T* band = static_cast<const T*>(d.band);
    const T ip = load_rinv<mixw(PR)>(d, p);
    A = MS::load(MA, p);
    B = MS::load(MB, p);
    typename MS::Acc dA{}, dB{};
    auto pair = [&](long long q, T w) {
      const T P = normalised<T>(d.norm, w, ip, load_rinv<mixw(PR)>(d, q));
      MS::acc(dA, P, MS::diff(MS::load(MA, q), A));
      MS::acc(dB, P, MS::diff(MS::load(MB, q), B));
    };
    const int kl = d.cnt[d.n + p], kr = d.cnt[p];
    const int bl = kl < d.band_cap ? kl : d.band_cap;
    const int br = kr < d.band_cap ? kr : d.band_cap;
#pragma unroll 2
    for (int k = 1; k <= bl; ++k) {
      const long long q = ring(d, g, p, -k);
      pair(q, band[band_at(d, q, k)]);
    }
    for (int k = bl + 1; k <= kl; ++k) {
      const long long q = ring(d, g, p, -k);
      pair(q, W::eval(d, gap(d, g, Xs, q, p), 0));
    }
#pragma unroll 2
    for (int k = 1; k <= br; ++k) pair(ring(d, g, p, k), band[band_at(d, p, k)]);
    for (int k = br + 1; k <= kr; ++k) {
      const long long q = ring(d, g, p, k);
      pair(q, W::eval(d, gap(d, g, Xs, p, q), 0));
    }
    MS::update(A, B, dA, dB, TR ? 0 : d.react);
    MS::store(d.M[mc] + sq.oa, p, A);
    if (sq.store_b) MS::store(d.M[mc] + sq.ob, p, B);
  }
  if (!TR) finish_step(d, 1, 0);
}

// =============================================================== 2-d cells ==

// One run [q0, q1) of candidate slots for the particle in slot p at (x, y).
template <int PR, bool EXCHANGE, bool PER>
__device__ __forceinline__ void cell2_run(const Dev& d, const long long* Xs, long long p,
                                          long long x, long long y, int q0, int q1,
                                          typename Weight<mixw(PR), 2>::T& r,
                                          const unsigned long long* M,
                                          typename Weight<mixw(PR), 2>::T ip,
                                          typename Mass<PR>::V A, typename Mass<PR>::V B,
                                          typename Mass<PR>::Acc& dA,
                                          typename Mass<PR>::Acc& dB, long long ob) {
  using W = Weight<mixw(PR), 2>;
  using T = typename W::T;
  using MS = Mass<PR>;
  for (int q = q0; q < q1; ++q) {
    long long dx = Xs[q] - x, dy = Xs[d.n + q] - y;
    if (PER) {
      dx = min_image(dx, d.Lq[0]);
      dy = min_image(dy, d.Lq[1]);
    }
    if (!in_range2(dx, dy, d.S)) continue;
    const T w = W::eval(d, dx, dy);
    if (!EXCHANGE) {
      r += w;
    } else if (q != p) {
      const T P = normalised<T>(d.norm, w, ip, load_rinv<mixw(PR)>(d, q));
      MS::acc(dA, P, MS::diff(MS::load(M, q), A));
      MS::acc(dB, P, MS::diff(MS::load(M, ob + q), B));
    }
  }
}

// All candidates of the particle in slot p: the 3 x 3 block of cells around
// its cell (reflecting walls), or the wrapped cell spans (periodic).  M:
// the first species' masses; the second's are ob words further.
template <int PR, bool EXCHANGE, bool PER>
__device__ __forceinline__ void cell2_loop(const Dev& d, const long long* Xs, long long p,
                                           long long x, long long y,
                                           typename Weight<mixw(PR), 2>::T& r,
                                           const unsigned long long* M,
                                           typename Weight<mixw(PR), 2>::T ip,
                                           typename Mass<PR>::V A, typename Mass<PR>::V B,
                                           typename Mass<PR>::Acc& dA,
                                           typename Mass<PR>::Acc& dB, long long ob) {
  if (PER) {
    cells2_visit(d, x, y, [&](int q0, int q1) {
      cell2_run<PR, EXCHANGE, true>(d, Xs, p, x, y, q0, q1, r, M, ip, A, B, dA, dB, ob);
    });
    return;
  }
  long long kx = x >> d.cshift, ky = y >> d.cshift;
  kx = kx >= d.ncx ? d.ncx - 1 : kx;
  ky = ky >= d.ncy ? d.ncy - 1 : ky;
  const long long kx0 = kx > 0 ? kx - 1 : 0;
  const long long kx1 = kx + 1 < d.ncx ? kx + 1 : d.ncx - 1;
  for (long long row = ky - 1; row <= ky + 1; ++row) {
    if (row < 0 || row >= d.ncy) continue;
    cell2_run<PR, EXCHANGE, false>(d, Xs, p, x, y, d.start[row * d.ncx + kx0],
                                    d.start[row * d.ncx + kx1 + 1], r, M, ip, A, B, dA, dB, ob);
  }
}

// PER: periodic walls (wrapped cell spans, minimum-image separations), a
// separate instantiation so the reflecting kernels keep their registers.
template <int PR, bool PER>
__global__ void __launch_bounds__(kThreads) k_rowsum_cell2(Dev d) {
  using T = typename Weight<mixw(PR), 2>::T;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const long long* Xs = d.X[xc ^ 1];
  T r = T(0);
  typename Mass<PR>::Acc dummy{};
  typename Mass<PR>::V z{};
  cell2_loop<PR, false, PER>(d, Xs, p, Xs[p], Xs[d.n + p], r, nullptr, T(0), z, z, dummy,
                              dummy, 0);
  store_rinv<mixw(PR)>(d, p, r);
  const int s = d.src[p];
  d.id[xc ^ 1][p] = d.id[xc][s];
  gather_masses(d, mc, p, s);
}

template <int PR, bool TR, bool PER>
__global__ void __launch_bounds__(kThreads) k_exchange_cell2(Dev d, int sp) {
  using T = typename Weight<mixw(PR), 2>::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  const bool valid = p < d.n;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const SpeciesPair sq = species_pair<TR>(d, sp);
  MV A{}, B{};
  if (valid) {
    const long long* Xs = d.X[xc ^ 1];
    const unsigned long long* MA = d.M[mc ^ 1] + sq.oa;
    const unsigned long long* MB = d.M[mc ^ 1] + sq.ob;
    A = MS::load(MA, p);
    B = MS::load(MB, p);
    T r = T(0);
    typename MS::Acc dA{}, dB{};
    cell2_loop<PR, true, PER>(d, Xs, p, Xs[p], Xs[d.n + p], r, MA, load_rinv<mixw(PR)>(d, p), A, B,
                               dA, dB, sq.ob - sq.oa);
    MS::update(A, B, dA, dB, TR ? 0 : d.react);
    MS::store(d.M[mc] + sq.oa, p, A);
    if (sq.store_b) MS::store(d.M[mc] + sq.ob, p, B);
  }
  if (!TR) finish_step(d, 1, 0);
}

// ============================================================ brute force ==
// All pairs, j-particles staged through shared memory in tiles.  Particles
// keep their caller order (no sort); masses ping-pong between buffers.

template <int PR, bool CUT, int DIM>
__global__ void __launch_bounds__(kThreads) k_rowsum_brute(Dev d) {
  using W = Weight<mixw(PR), DIM>;
  using T = typename W::T;
  __shared__ long long s_x[kBruteTile];
  __shared__ long long s_y[DIM == 2 ? kBruteTile : 1];
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  const bool valid = p < d.n;
  const long long* X = d.X[d.ctrl->xcur];
  const long long x = valid ? X[p] : 0;
  const long long y = (valid && DIM == 2) ? X[d.n + p] : 0;
  T r = T(0);
  for (long long j0 = 0; j0 < d.n; j0 += kBruteTile) {
    const long long j = j0 + threadIdx.x;
    if (j < d.n) {
      s_x[threadIdx.x] = X[j];
      if (DIM == 2) s_y[threadIdx.x] = X[d.n + j];
    }
    __syncthreads();
    const int jn = (int)min((long long)kBruteTile, d.n - j0);
    if (valid) {
      for (int jj = 0; jj < jn; ++jj) {
        long long dx = s_x[jj] - x;
        long long dy = DIM == 2 ? s_y[jj] - y : 0;
        if (d.periodic) {
          dx = min_image(dx, d.Lq[0]);
          if (DIM == 2) dy = min_image(dy, d.Lq[1]);
        }
        if (CUT) {
          if (DIM == 1 ? !within1(dx, d.S) : !in_range2(dx, dy, d.S)) continue;
        }
        r += W::eval(d, dx, dy);
      }
    }
    __syncthreads();
  }
  if (valid) store_rinv<mixw(PR)>(d, p, r);
}

template <int PR, bool CUT, int DIM, bool TR>
__global__ void __launch_bounds__(kThreads) k_exchange_brute(Dev d, int sp) {
  using W = Weight<mixw(PR), DIM>;
  using T = typename W::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  __shared__ long long s_x[kBruteTile];
  __shared__ long long s_y[DIM == 2 ? kBruteTile : 1];
  __shared__ T s_ri[kBruteTile];
  __shared__ MV s_a[kBruteTile];
  __shared__ MV s_b[kBruteTile];
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  const bool valid = p < d.n;
  const int mc = d.ctrl->mcur;
  const long long* X = d.X[d.ctrl->xcur];
  const SpeciesPair sq = species_pair<TR>(d, sp);
  const unsigned long long* MA = d.M[mc] + sq.oa;
  const unsigned long long* MB = d.M[mc] + sq.ob;
  const long long x = valid ? X[p] : 0;
  const long long y = (valid && DIM == 2) ? X[d.n + p] : 0;
  MV A{}, B{};
  T ip = T(0);
  if (valid) {
    A = MS::load(MA, p);
    B = MS::load(MB, p);
    ip = load_rinv<mixw(PR)>(d, p);
  }
  typename MS::Acc dA{}, dB{};
  for (long long j0 = 0; j0 < d.n; j0 += kBruteTile) {
    const long long j = j0 + threadIdx.x;
    if (j < d.n) {
      s_x[threadIdx.x] = X[j];
      if (DIM == 2) s_y[threadIdx.x] = X[d.n + j];
      s_ri[threadIdx.x] = load_rinv<mixw(PR)>(d, j);
      s_a[threadIdx.x] = MS::load(MA, j);
      s_b[threadIdx.x] = MS::load(MB, j);
    }
    __syncthreads();
    const int jn = (int)min((long long)kBruteTile, d.n - j0);
    if (valid) {
      for (int jj = 0; jj < jn; ++jj) {
        if (j0 + jj == p) continue;
        long long dx = s_x[jj] - x;
        long long dy = DIM == 2 ? s_y[jj] - y : 0;
        if (d.periodic) {
          dx = min_image(dx, d.Lq[0]);
          if (DIM == 2) dy = min_image(dy, d.Lq[1]);
        }
        if (CUT) {
          if (DIM == 1 ? !within1(dx, d.S) : !in_range2(dx, dy, d.S)) continue;
        }
        const T w = W::eval(d, dx, dy);
        // a weight that underflowed to zero adds exact zeros: skip the
        // flux arithmetic (the full matrix still evaluates every weight)
        if (w == T(0)) continue;
        const T P = normalised<T>(d.norm, w, ip, s_ri[jj]);
        MS::acc(dA, P, MS::diff(s_a[jj], A));
        MS::acc(dB, P, MS::diff(s_b[jj], B));
      }
    }
    __syncthreads();
  }
  if (valid) {
    MS::update(A, B, dA, dB, TR ? 0 : d.react);
    MS::store(d.M[mc ^ 1] + sq.oa, p, A);
    if (sq.store_b) MS::store(d.M[mc ^ 1] + sq.ob, p, B);
  }
  if (!TR) finish_step(d, 0, 1);
}

// Species 2 and up into the sorted slots (the row-sum pass moved A and B).
__global__ void __launch_bounds__(kThreads) k_gather_species(Dev d) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  gather_species(d, d.ctrl->mcur, p, d.src[p]);
}

// --------------------------------------------------------------- launch --

template <int PR, bool PER>
static void cell2_passes(const Dev& d, unsigned int g, cudaStream_t s, Marker& mk) {
  mk("rowsum_cell2", s);
  k_rowsum_cell2<PR, PER><<<g, kThreads, 0, s>>>(d);
  if (d.nspec > 2) {
    mk("gather_species", s);
    k_gather_species<<<g, kThreads, 0, s>>>(d);
  }
  for (int sp = 2; sp < d.nspec; sp += 2) {
    mk("exchange_cell2_species", s);
    k_exchange_cell2<PR, true, PER><<<g, kThreads, 0, s>>>(d, sp);
  }
  mk("exchange_cell2", s);
  k_exchange_cell2<PR, false, PER><<<g, kThreads, 0, s>>>(d, 0);
}

template <int PR, bool TR>
static void launch_exchange_brute(const Dev& d, bool cut, unsigned int g, cudaStream_t s,
                                  int sp) {
  if (cut) {
    if (d.dim == 1)
      k_exchange_brute<PR, true, 1, TR><<<g, kThreads, 0, s>>>(d, sp);
    else
      k_exchange_brute<PR, true, 2, TR><<<g, kThreads, 0, s>>>(d, sp);
  } else {
    if (d.dim == 1)
      k_exchange_brute<PR, false, 1, TR><<<g, kThreads, 0, s>>>(d, sp);
    else
      k_exchange_brute<PR, false, 2, TR><<<g, kThreads, 0, s>>>(d, sp);
  }
}

// The extra species' passes (pairs 2-3, 4-5, ...) run between the row sums
// and the A/B pass, which ends the step.
template <int PR>
static void transfer_t(const Dev& d, int search, cudaStream_t s, Marker& mk) {
  const unsigned int g = (unsigned int)((d.n + kThreads - 1) / kThreads);
  if (search == MT_SEARCH_CELL) {
    if (d.dim == 1 && d.band_cap > 0) {
      mk("band_build", s);
      k_band_build<PR><<<g, kThreads, 0, s>>>(d);
      mk("band_rowsum", s);
      k_band_rowsum<PR><<<g, kThreads, 0, s>>>(d);
      if (d.nspec > 2) {
        mk("gather_species", s);
        k_gather_species<<<g, kThreads, 0, s>>>(d);
      }
      for (int sp = 2; sp < d.nspec; sp += 2) {
        mk("band_exchange_species", s);
        k_band_exchange<PR, true><<<g, kThreads, 0, s>>>(d, sp);
      }
      mk("band_exchange", s);
      k_band_exchange<PR, false><<<g, kThreads, 0, s>>>(d, 0);
    } else if (d.dim == 1 && d.tile) {
      mk("rowsum_tile", s);
      k_rowsum_tile<PR><<<g, kThreads, 0, s>>>(d);
      if (d.nspec > 2) {
        mk("gather_species", s);
        k_gather_species<<<g, kThreads, 0, s>>>(d);
      }
      for (int sp = 2; sp < d.nspec; sp += 2) {
        mk("exchange_tile_species", s);
        k_exchange_tile<PR, true><<<g, kThreads, 0, s>>>(d, sp);
      }
      mk("exchange_tile", s);
      k_exchange_tile<PR, false><<<g, kThreads, 0, s>>>(d, 0);
    } else if (d.dim == 1) {
      mk("rowsum_walk", s);
      k_rowsum_walk<PR><<<g, kThreads, 0, s>>>(d);
      if (d.nspec > 2) {
        mk("gather_species", s);
        k_gather_species<<<g, kThreads, 0, s>>>(d);
      }
      for (int sp = 2; sp < d.nspec; sp += 2) {
        mk("exchange_walk_species", s);
        k_exchange_walk<PR, true><<<g, kThreads, 0, s>>>(d, sp);
      }
      mk("exchange_walk", s);
      k_exchange_walk<PR, false><<<g, kThreads, 0, s>>>(d, 0);
    } else if (d.periodic) {
      cell2_passes<PR, true>(d, g, s, mk);
    } else {
      cell2_passes<PR, false>(d, g, s, mk);
    }
  } else {
    const bool cut = search == MT_SEARCH_BRUTE;
    mk(cut ? "rowsum_brute" : "rowsum_full", s);
    if (cut) {
      if (d.dim == 1)
        k_rowsum_brute<PR, true, 1><<<g, kThreads, 0, s>>>(d);
      else
        k_rowsum_brute<PR, true, 2><<<g, kThreads, 0, s>>>(d);
    } else {
      if (d.dim == 1)
        k_rowsum_brute<PR, false, 1><<<g, kThreads, 0, s>>>(d);
      else
        k_rowsum_brute<PR, false, 2><<<g, kThreads, 0, s>>>(d);
    }
    for (int sp = 2; sp < d.nspec; sp += 2) {
      mk(cut ? "exchange_brute_species" : "exchange_full_species", s);
      launch_exchange_brute<PR, true>(d, cut, g, s, sp);
    }
    mk(cut ? "exchange_brute" : "exchange_full", s);
    launch_exchange_brute<PR, false>(d, cut, g, s, 0);
  }
}

cudaError_t launch_transfer(const Dev& d, int search, int precision, cudaStream_t s,
                            Marker& mk) {
  if (precision == MT_MIXED)
    transfer_t<MT_MIXED>(d, search, s, mk);
  else if (precision == MT_MIXED_DF32)
    transfer_t<MT_MIXED_DF32>(d, search, s, mk);
  else
    transfer_t<MT_FP64>(d, search, s, mk);
  return cudaGetLastError();
}

}  // namespace mt
