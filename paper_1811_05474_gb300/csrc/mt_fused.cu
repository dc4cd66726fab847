// mt_fused.cu -- the whole 1-d time step (move, cell-list sort, weights,
// normalisation, exchange, reaction, observables) in one kernel launch.
//
// The particles are kept sorted by (x, id).  fstart[c] is the first sorted
// slot of cell c (cells 2^cshift ticks wide) and cb[s] the first cell of
// segment s; segments hold about seg_target particles each.  A CTA that
// processes segment s = [c0, c1):
//   1. loads the old slots of its cells widened by a halo (hc cells, which
//      covers 2 Smax) and by the displacement bound (Dc cells), coalesced,
//      into registers;
//   2. moves them (Eq. 2 on the grid, Sec. 3 walls) -- a particle near a
//      segment edge is moved by more than one CTA, with the same result;
//   3. keeps those whose new cell lies in [c0 - hc, c1 + hc), counting-sorts
//      them into shared-memory bins and sorts each bin by (x, id) (bins of
//      more than kBinMax particles, e.g. particles piled against a wall, are
//      sorted by the whole CTA);
//   4. finds its output offset without a global scan: every particle whose
//      old cell is below c0 - Dc ends below c0, every particle whose old cell
//      is at or above c0 + Dc ends at or above c0, so the offset is fstart
//      [c0 - Dc] plus the particles of the old cells in between that moved
//      below c0;
//   5. forms r_i = sum_j nu_ij for every staged particle within Smax of its
//      cells and dM_i = 1/2 sum_j P_ij (M_j - M_i) for its own particles
//      (Eq. 3, 4, 7), walking the sorted shared-memory array, then reacts;
//   6. writes its own particles, the next step's fstart for its cells and
//      the next step's segment boundaries that fall in its output range.
//
// Two tiers.  k_step1d stages up to 1024 particles per CTA (256 threads, a
// persistent grid of 4 CTAs per SM).  A segment that does not fit, or whose
// pair work is heavy (a dense cluster), is queued; a CUDA-graph conditional
// node then runs k_step1d_big over the queue: a cluster of 8 CTAs (512
// threads, up to 4096 staged particles each) per segment, splitting its row
// sums and exchange across 8 SMs.  Only if a segment does not fit there
// either does a second conditional node redo the step with the general
// pipeline (scan, scatter, cell sort, two transfer passes).  Whichever tier
// completes the step advances it.
//
// Batches.  Independent realisations share the kernel: each has its own
// stretch of the tick axis and its own segments (segment starts sslot[] are
// fixed slots, since a realisation's particles stay in its slot range, and a
// realisation's first segment starts at its first cell, which no other
// realisation's particle can reach).  The CTA that finishes the last segment
// of a realisation reduces that realisation's observables.
#include <cooperative_groups.h>
#include <cuda_pipeline.h>

#include "mt_pair.cuh"

namespace cg = cooperative_groups;

namespace mt {

constexpr int kBinMax = 32;  // bins up to this size sort in one thread
constexpr int kBigMax = 64;  // larger bins a CTA sorts cooperatively

template <int NT, int PER>
struct Tier {
  static constexpr int kT = NT;
  static constexpr int kPer = PER;
  static constexpr int kCap = NT * PER;
  static constexpr int kBins = NT * 4;
  static constexpr int kBinsPerThread = 4;
};
using Fast = Tier<256, 4>;
using Big = Tier<512, 8>;
static_assert(Fast::kCap == kFusedCap, "staging capacity");
static_assert(Fast::kCap <= kFusedPairCap, "left counts share the pair list's weights");

template <typename TR>
size_t tier_smem(int precision) {
  const size_t r = precision == MT_FP64 ? 8 : 4;  // 1 / r_i
  return (size_t)TR::kCap * (8 + 8 + 8 + 4 + r) + (size_t)(2 * TR::kBins + 1) * 4;
}


__device__ __forceinline__ long long lmin(long long a, long long b) { return a < b ? a : b; }
__device__ __forceinline__ long long lmax(long long a, long long b) { return a > b ? a : b; }

enum : int { kSegOk = 0, kSegCapacity = 1, kSegDense = 2, kSegHeavy = 3 };

// A segment whose sum over bins of (particles per bin)^2 exceeds this is
// pair-heavy (a dense cluster, e.g. particles piled against a wall): the
// first tier hands it to the second, which splits its exchange across
// the CTAs of a thread-block cluster so that its O(n^2) work does not sit
// on one SM.
constexpr int kHeavyWork = 16384;
constexpr int kWalk = 32;  // neighbours per side a thread walks before a warp takes over

// First index q in [0, m) with a[q] >= key (a sorted ascending).
__device__ __forceinline__ int lower_at_least(const long long* a, int m, long long key) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// More than kWalk neighbours on a side of sorted slot j: the (kWalk + 1)-th
// slot to the left or right is within S.
__device__ __forceinline__ bool dense_at(const long long* sx, int m, int j, long long x,
                                         long long S) {
  return (j > kWalk && x - sx[j - kWalk - 1] <= S) || (j + kWalk + 1 < m && sx[j + kWalk + 1] - x <= S);
}

// The per-segment scalars read from the previous step's boundaries and cell
// starts (loaded one segment ahead by the persistent loop).
struct SegScalars {
  int c0, c1;          // own cells [c0, c1)
  int a0, L, o0, o1;   // staged old slots [a0, a0 + L); old slots of cells c0 -+ Dc
};

__device__ __forceinline__ SegScalars load_seg(const Dev& d, int sc, long long Dc, int seg) {
  const int* So = d.fstart[sc];
  SegScalars s;
  s.c0 = d.cb[sc][seg];
  s.c1 = d.cb[sc][seg + 1];
  const long long Hc = d.hc, ncell = d.ncell;
  s.a0 = So[lmax(s.c0 - Hc - Dc, 0)];
  s.L = So[lmin(s.c1 + Hc + Dc, ncell)] - s.a0;
  s.o0 = So[lmax(s.c0 - Dc, 0)];
  s.o1 = So[lmin(s.c0 + Dc, ncell)];
  return s;
}

// Asynchronous load of the next segment's scalars into shared memory while
// the current segment is processed (the first tier), so that no global
// round trip sits between two segments: stage 1 (thread 0, at the segment
// start) copies c0, c1 and the aligned word holding its prediction flag;
// stage 2 (thread 0, part-way through the segment) copies the four cell
// starts that c0 and c1 select.  The words land in w[0 .. 6]: c0, c1, a0,
// start of cell c1 + Hc + Dc, o0, o1, prediction word.
struct SegPrefetch {
  int* w;     // shared words
  int seg;    // the segment (>= nseg: none)
  int sc;
  long long Dc;
};

__device__ __forceinline__ void prefetch_stage1(const Dev& d, const SegPrefetch& pf) {
  if (pf.seg >= d.nseg) return;
  __pipeline_memcpy_async(&pf.w[0], &d.cb[pf.sc][pf.seg], 4);
  __pipeline_memcpy_async(&pf.w[1], &d.cb[pf.sc][pf.seg + 1], 4);
  if (d.use_pred)
    __pipeline_memcpy_async(&pf.w[6], d.pred[pf.sc] + (pf.seg & ~3), 4);  // 4-aligned in the buffer
  __pipeline_commit();
}

__device__ __forceinline__ void prefetch_stage2(const Dev& d, const SegPrefetch& pf) {
  if (pf.seg >= d.nseg) return;
  __pipeline_wait_prior(0);
  const int* So = d.fstart[pf.sc];
  const long long c0 = pf.w[0], c1 = pf.w[1], Hc = d.hc, ncell = d.ncell, Dc = pf.Dc;
  __pipeline_memcpy_async(&pf.w[2], &So[lmax(c0 - Hc - Dc, 0)], 4);
  __pipeline_memcpy_async(&pf.w[3], &So[lmin(c1 + Hc + Dc, ncell)], 4);
  __pipeline_memcpy_async(&pf.w[4], &So[lmax(c0 - Dc, 0)], 4);
  __pipeline_memcpy_async(&pf.w[5], &So[lmin(c0 + Dc, ncell)], 4);
  __pipeline_commit();
}

// A bulk prefetch into L2 of bytes [lo, hi) of a workspace array (arrays
// start on 256-byte boundaries and their regions are multiples of 256
// bytes, so rounding the range out to 16 bytes stays inside the region).
// Nothing waits for it: it only turns later loads into L2 hits.
__device__ __forceinline__ void l2_prefetch(const void* base, long long lo, long long hi) {
  const long long b0 = lo & ~15LL, b1 = (hi + 15) & ~15LL;
  if (b1 > b0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                     static_cast<const char*>(base) + b0),
                 "r"((unsigned int)(b1 - b0))
                 : "memory");
}

// The step's control words, read once per kernel launch (they change only
// when the step ends).
struct StepState {
  int xc, mc, sc;             // current X / id, mass and segment buffers
  unsigned long long step;    // steps completed
  const float* noise;         // injected normals or null
};

__device__ __forceinline__ StepState step_state(const Dev& d) {
  const Ctrl* c = d.ctrl;
  return {c->xcur, c->mcur, c->scur, c->step, c->noise};
}

// The next segment's staged slots [a0, a0 + L) (positions, ids, both mass
// arrays) asked into L2 while the current segment runs its transfer, once
// its cell starts have arrived (thread 0, after prefetch_stage2), so that
// its staging loads do not wait on HBM.
__device__ __forceinline__ void prefetch_next_l2(const Dev& d, const SegPrefetch& pf,
                                                 const StepState& st) {
  if (pf.seg >= d.nseg) return;
  __pipeline_wait_prior(0);
  const long long a0 = pf.w[2], e = pf.w[3];
  if (e <= a0 || e - a0 > 2 * (long long)kFusedCap) return;  // nothing, or not staged
  l2_prefetch(d.X[st.xc], a0 * 8, e * 8);
  l2_prefetch(d.id[st.xc], a0 * 4, e * 4);
  l2_prefetch(d.M[st.mc], a0 * 8, e * 8);
  l2_prefetch(d.M[st.mc], (d.n + a0) * 8, (d.n + e) * 8);
}

// ------------------------------------------------ first tier: pair list --
// The first tier's transfer (row sums, exchange, reaction) over a list of
// the unordered pairs of its staged, sorted particles.  Owners are the
// staged slots j with x_j in [xlo - 2 Smax, xhi + Smax); each owns its pairs
// (j, k), k > j, x_k - x_j <= Smax -- R_j consecutive slots, since the slots
// are sorted -- and pair q of owner j sits at pfx[j] + (k - j - 1) in the
// list.  The weight nu (Eq. 3) of every listed pair is evaluated once, by
// one thread per pair (no divergent walks), and stored; the row sums
// r_j = 1 + sum of its left pairs' weights + sum of its right pairs' (in
// that order, the order of the cluster tiers' walks) and the exchange of
// own particles then read the stored weights.  A slot's left pairs are
// (j - t, j) for t = 1, 2, ... while R_{j-t} >= t.
constexpr int kPairCap = kFusedPairCap;

template <typename TR, typename T>
__host__ __device__ constexpr size_t pair_region_offset() {
  return ((size_t)TR::kCap * (8 + 8 + 8 + 4 + sizeof(T)) + (size_t)(2 * TR::kBins + 1) * 4 + 7) &
         ~(size_t)7;
}
template <typename TR, typename T>
__host__ __device__ constexpr size_t pair_region_bytes() {
  return (size_t)kPairCap * sizeof(T) + (size_t)(TR::kCap + 1) * 2 + (size_t)kPairCap * 2;
}

// Dynamic shared memory of the first tier: staging, bins and the pair list.
size_t fused_smem_bytes(int precision) {
  return precision == MT_FP64 ? pair_region_offset<Fast, double>() + pair_region_bytes<Fast, double>()
                              : pair_region_offset<Fast, float>() + pair_region_bytes<Fast, float>();
}

// First index q in [0, m) with a[q] >= key (a sorted ascending), by one
// warp: each round the 32 lanes probe evenly spaced slots and the ballot
// narrows the range 32-fold (two rounds for m <= 1024).  Called by all 32
// lanes; every lane gets the result.
__device__ __forceinline__ int warp_lower_at_least(const long long* a, int m, long long key) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = m;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const int step = (hi - lo + 31) >> 5;
    const int p = lo + lane * step;
    const unsigned int below = __ballot_sync(0xffffffffu, p < hi && a[p] < key);
    const int cnt = __popc(below);  // probes below key form a prefix
    if (cnt == 0) return lo;
    const int last = lo + (cnt - 1) * step;
    hi = min(hi, last + step);
    lo = last + 1;
  }
  const int p = lo + lane;
  return lo + __popc(__ballot_sync(0xffffffffu, p < hi && a[p] < key));
}

template <int PR, typename TR>
__device__ bool pair_transfer(const Dev& d, const StepState& st, unsigned char* smem, bool active,
                              int m, int w0, int w1, long long out0, long long xlo, long long xhi) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  constexpr int NT = TR::kT, CAP = TR::kCap;
  constexpr int kCnt = 64;  // pair-count bins of the lane assignment
  long long* sx = reinterpret_cast<long long*>(smem);
  unsigned long long* sA = reinterpret_cast<unsigned long long*>(sx + CAP);
  unsigned long long* sB = sA + CAP;
  int* sid = reinterpret_cast<int*>(sB + CAP);
  T* sr = reinterpret_cast<T*>(sid + CAP);
  int* perm = reinterpret_cast<int*>(sr + CAP) + TR::kBins + 1;  // the bins' scatter cursors
  T* sw = reinterpret_cast<T*>(smem + pair_region_offset<TR, T>());  // [kPairCap]
  unsigned short* pfx = reinterpret_cast<unsigned short*>(sw + kPairCap);  // [CAP + 1]
  unsigned short* own = pfx + CAP + 1;                                    // [kPairCap]
  __shared__ int s_idx[3];
  __shared__ int s_part[NT / 32];
  __shared__ int s_hist[kCnt];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long S = d.S;
  // (A) owners [olo, rhi) and row-sum slots [rlo, rhi), one search per warp
  if (warp < 3) {
    const long long key = warp == 0 ? xlo - 2 * S : warp == 1 ? xlo - S : xhi + S;
    const int v = active ? warp_lower_at_least(sx, m, key) : 0;
    if (lane == 0) s_idx[warp] = v;
  } else if (warp == 3) {
    for (int b = lane; b < kCnt; b += 32) s_hist[b] = 0;
  }
  __syncthreads();
  const int olo = s_idx[0], rlo = s_idx[1], rhi = s_idx[2];
  const int no = rhi - olo, nrs = rhi - rlo;
  // Left and right pair counts of slot j: R_j = slots k > j with
  // x_k - x_j <= Smax, L_j = slots i < j with x_j - x_i <= Smax.
  auto right_count = [&](int j) {
    const long long x = sx[j];
    int c = 0;
    for (int k = j + 1; k < m && sx[k] - x <= S; ++k) ++c;
    return c;
  };
  auto left_count = [&](int j) {
    const long long x = sx[j];
    int c = 0;
    for (int i = j - 1; i >= 0 && x - sx[i] <= S; --i) ++c;
    return c;
  };
  // (B) R_j of every owner; L_j and the count c = L + R of every row-sum
  // slot (L_j kept in the weights' array, free until (E))
  int* lcount = reinterpret_cast<int*>(sw);  // [no] (no <= CAP <= kPairCap words)
  for (int jj = tid; jj < no; jj += NT) {
    const int j = olo + jj;
    const int R = right_count(j);
    pfx[jj] = (unsigned short)R;
    if (j >= rlo) {
      const int Lc = left_count(j), c = R + Lc;
      lcount[jj] = Lc;
      atomicAdd(&s_hist[c < kCnt ? c : kCnt - 1], 1);
    }
  }
  __syncthreads();
  // (C) exclusive prefix sums: pair offsets pfx[0 .. no] (each thread its
  // four consecutive owners) and, by warp 0, the count bins
  int np;
  {
    constexpr int E = CAP / NT;
    int loc[E];
    int sum = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = tid * E + e;
      loc[e] = i < no ? pfx[i] : 0;
      sum += loc[e];
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_part[warp] = inc;
    __syncthreads();
    int run = inc - sum;
    np = 0;
    for (int w = 0; w < NT / 32; ++w) {
      const int t = s_part[w];
      if (w < warp) run += t;
      np += t;
    }
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int i = tid * E + e;
      if (i < no) pfx[i] = (unsigned short)run;
      run += loc[e];
    }
    if (tid == 0) pfx[no] = (unsigned short)np;
    if (warp == 0) {
      const int h0 = s_hist[2 * lane], h1 = s_hist[2 * lane + 1];
      int hin = h0 + h1;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, hin, o);
        if (lane >= o) hin += t;
      }
      s_hist[2 * lane] = hin - h0 - h1;
      s_hist[2 * lane + 1] = hin - h1;
    }
    __syncthreads();
  }
  if (np > kPairCap) return false;  // uniform across the CTA
  // (D) the pair list's owners, and the row-sum slots in order of their
  // pair count (counting sort; the order within a count does not matter):
  // a warp's lanes then take slots with equal counts and run the same
  // number of iterations of the loops below, each over the slot's left
  // pairs then its right pairs in one sequence.  Each slot's sums are the
  // same whatever lane forms them.
  for (int jj = tid; jj < no; jj += NT) {
    const int q1 = pfx[jj + 1];
    for (int q = pfx[jj]; q < q1; ++q) own[q] = (unsigned short)jj;
    const int j = olo + jj;
    if (j >= rlo) {
      const int L = lcount[jj], c = L + (q1 - pfx[jj]);
      perm[atomicAdd(&s_hist[c < kCnt ? c : kCnt - 1], 1)] = j | (L << 16);
    }
  }
  __syncthreads();
  // (E) one weight per unordered pair
  for (int q = tid; q < np; q += NT) {
    const int jj = own[q];
    const int j = olo + jj, k = j + 1 + (q - pfx[jj]);
    sw[q] = W::near(d, sx[k] - sx[j]);
  }
  __syncthreads();
  // Pair u of slot j (u < c): u < L is the left pair (j - u - 1, j), else
  // the right pair (j, j + 1 + u - L); its list index and its partner slot.
  auto pair_of = [&](int j, int jj, int left, int u, int& q, int& partner) {
    if (u < left) {
      const int t = u + 1;
      q = pfx[jj - t] + t - 1;
      partner = j - t;
    } else {
      q = pfx[jj] + (u - left);
      partner = j + 1 + (u - left);
    }
  };
  // (F) row sums: 1 + left pairs' weights + right pairs' weights, in that order
  for (int p = tid; p < nrs; p += NT) {
    const int v = perm[p], j = v & 0xffff, left = v >> 16, jj = j - olo;
    const int c = left + (pfx[jj + 1] - pfx[jj]);
    T r = T(1);
    for (int u = 0; u < c; ++u) {
      int q, partner;
      pair_of(j, jj, left, u, q, partner);
      r += sw[q];
    }
    sr[j] = mixw(PR) ? T(__frcp_rn((float)r)) : T(rcp_ge1((double)r));
  }
  __syncthreads();
  // (G) binary64 weights under the symmetric normalisation: each listed
  // pair's P = nu (1/r_j + 1/r_k) / 2 once, in place of nu (pairs with an
  // end outside the row-sum range are never read); binary32 weights form P
  // where they are used (three binary32 operations)
  const bool sym = d.norm != MT_NORM_ROW;
  constexpr bool kPairP = !mixw(PR);
  if (kPairP && sym) {
    for (int q = tid; q < np; q += NT) {
      const int jj = own[q];
      const int j = olo + jj, k = j + 1 + (q - pfx[jj]);
      if (j >= rlo && k < rhi) sw[q] = normalised<T>(MT_NORM_SYM, sw[q], sr[j], sr[k]);
    }
    __syncthreads();
  }
  // (H) exchange and reaction of own particles
  if (active) {
    long long* Xn = d.X[st.xc ^ 1];
    int* In = d.id[st.xc ^ 1];
    unsigned long long* Mn = d.M[st.mc ^ 1];
    if (out0 + (w1 - w0) > d.n) raise_error(d.ctrl, kErrIndex, out0);
    for (int p = tid; p < nrs; p += NT) {
      const int v = perm[p], j = v & 0xffff, left = v >> 16, jj = j - olo;
      if (j < w0 || j >= w1) continue;  // a neighbour of own particles only
      const int cnt = left + (pfx[jj + 1] - pfx[jj]);
      const T ip = sr[j];
      MV A = MS::load(sA, j), B = MS::load(sB, j);
      typename MS::Acc dA{}, dB{};
      for (int u = 0; u < cnt; ++u) {
        int q, i;
        pair_of(j, jj, left, u, q, i);
        const T P = kPairP && sym ? sw[q] : normalised<T>(d.norm, sw[q], ip, sr[i]);
        MS::acc(dA, P, MS::diff(MS::load(sA, i), A));
        MS::acc(dB, P, MS::diff(MS::load(sB, i), B));
      }
      MS::update(A, B, dA, dB, d.react);
      const long long o = out0 + (j - w0);
      if (o < d.n) {
        MS::store(Mn, o, A);
        MS::store(Mn, d.n + o, B);
      }
    }
    for (int j = w0 + tid; j < w1; j += NT) {  // positions and ids, coalesced
      const long long o = out0 + (j - w0);
      if (o < d.n) {
        Xn[o] = sx[j];
        In[o] = sid[j];
      }
    }
  }
  __syncthreads();
  return true;
}

// Process one segment with the CTA (all NT threads call it).  The CTA
// computes the exchange for the own particles j with (j - first own) %
// nslice == slice, and the cell starts / segment boundaries only for slice
// 0; each thread adds the particles it updates to its observables
// accumulators (obs_sum, in shared memory).  Returns kSegOk, or why the
// segment does not fit this tier (then nothing of it has been written).
template <int PR, typename TR, int CL>
__device__ int fused_segment(const Dev& d, const StepState& st, int seg, unsigned char* smem,
                             const SegScalars& g, int slice, int nslice, bool route_heavy,
                             bool* heavy_out = nullptr, const SegPrefetch* pf = nullptr,
                             bool cache_w = false) {
  using W = Weight<mixw(PR), 1>;
  using T = typename W::T;
  using MS = Mass<PR>;
  using MV = typename MS::V;
  constexpr int NT = TR::kT, PER = TR::kPer, CAP = TR::kCap, NB = TR::kBins;
  long long* sx = reinterpret_cast<long long*>(smem);
  unsigned long long* sA = reinterpret_cast<unsigned long long*>(sx + CAP);
  unsigned long long* sB = sA + CAP;
  int* sid = reinterpret_cast<int*>(sB + CAP);
  T* sr = reinterpret_cast<T*>(sid + CAP);
  int* bstart = reinterpret_cast<int*>(sr + CAP);  // [NB + 1]
  int* bcur = bstart + NB + 1;                     // [NB]
  __shared__ int s_lt, s_w0, s_w1, s_bad, s_nbig, s_work, s_nd, s_nd2, s_wcbad, s_wcok;
  __shared__ int s_big[kBigMax];
  __shared__ int s_scan[NT / 32];

  Ctrl* c = d.ctrl;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int xc = st.xc, mc = st.mc, sc = st.sc;
  const long long* Xo = d.X[xc];
  const int* Io = d.id[xc];
  const unsigned long long* Mo = d.M[mc];
  const long long c0 = g.c0, c1 = g.c1, a0 = g.a0, L = g.L, o0 = g.o0, o1 = g.o1;
  const int wsh = d.cshift;
  const long long ncell = d.ncell;
  const long long Hc = d.hc;
  const long long wlo = lmax(c0 - Hc, 0) << wsh;
  const long long whi = lmin(c1 + Hc, ncell) << wsh;
  const long long xlo = c0 << wsh, xhi = c1 << wsh;  // own cells in ticks
  int sh2 = wsh;
  while (sh2 < 62 && ((whi - wlo) >> sh2) >= NB) ++sh2;
  // bins the window spans (bins are cells unless the window has >= NB cells)
  const int nb = whi > wlo ? (int)(((whi - 1 - wlo) >> sh2) + 1) : 1;
  int status = kSegOk;
  bool active = c0 < c1;
  if (active && L > CAP) {
    status = kSegCapacity;
    active = false;
  }
  if (tid == 0) {
    s_lt = 0;
    s_w0 = 0;
    s_w1 = 0;
    s_bad = 0;
    s_nbig = 0;
    s_work = 0;
    s_nd = 0;
    s_nd2 = 0;
  }
  for (int b = tid; b <= nb; b += NT) bstart[b] = 0;
  __syncthreads();

  // ---- 1-2: stage and move ------------------------------------------------
  // Registers keep only the new position and bin of each staged particle;
  // its id and masses are read again (cache hits) when it is scattered.
  const long long* Xs = Xo + a0;
  const int* Is = Io + a0;
  long long rx[PER];
  int rbin[PER];
  if (active) {
    const unsigned long long step = st.step;
    const float* noise = st.noise;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const long long e = tid + (long long)k * NT;
      rbin[k] = -1;
      bool lt = false, in0 = false, in1 = false;
      if (e < L) {
        const long long slot = a0 + e;
        const int id = Is[e];
        const Real* R = d.rt + (id >> d.lbits);
        const int loc = id & d.lmask;
        const long long base = R->base;
        float z;
        if (noise) {
          z = noise[R->off + loc];
        } else {
          const uint4 u = philox4x32_10(
              make_uint4((unsigned int)loc, (unsigned int)step, (unsigned int)(step >> 32), R->real),
              d.key0, d.key1);
          z = box_muller(u.x, u.y).x;
        }
        const long long x =
            base + reflect(Xs[e] - base + d.drift[0] + walk_ticks(d.bq, z), R->Lq);
        rx[k] = x;
        lt = slot >= o0 && slot < o1 && x < xlo;
        if (x >= wlo && x < whi) {
          const int b = (int)((x - wlo) >> sh2);
          rbin[k] = b;
          atomicAdd(&bstart[b + 1], 1);
          in0 = x < xlo;
          in1 = x < xhi;
        }
      }
      // warp-aggregated counts (one shared atomic per warp, not per particle)
      const int n_lt = __popc(__ballot_sync(0xffffffffu, lt));
      const int n_0 = __popc(__ballot_sync(0xffffffffu, in0));
      const int n_1 = __popc(__ballot_sync(0xffffffffu, in1));
      if (lane == 0) {
        if (n_lt) atomicAdd(&s_lt, n_lt);
        if (n_0) atomicAdd(&s_w0, n_0);
        if (n_1) atomicAdd(&s_w1, n_1);
      }
    }
  }
  if (pf && tid == 0) prefetch_stage2(d, *pf);  // the next segment's cell starts
  __syncthreads();

  // ---- 3: counting sort into bins, then (x, id) order inside each bin -----
  if (active) {
    constexpr int BPT = TR::kBinsPerThread;
    int v[BPT];
    int sum = 0, work = 0;
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      v[j] = tid * BPT + j < nb ? bstart[1 + tid * BPT + j] : 0;
      sum += v[j];
      work += v[j] * v[j];
      if (v[j] > kBinMax) {
        const int at = atomicAdd(&s_nbig, 1);
        if (at < kBigMax)
          s_big[at] = tid * BPT + j;
        else
          s_bad = 1;
      }
    }
    int inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) s_scan[warp] = inc;
    if (work > 0) atomicAdd(&s_work, work < kHeavyWork ? work : kHeavyWork);
    __syncthreads();
    int run = inc - sum;
    for (int w = 0; w < warp; ++w) run += s_scan[w];
#pragma unroll
    for (int j = 0; j < BPT; ++j) {
      const int b = tid * BPT + j;
      if (b < nb) {
        bcur[b] = run;  // scatter cursor: the bin's first slot
        run += v[j];
        bstart[1 + b] = run;
      }
    }
  } else {
    __syncthreads();
  }
  __syncthreads();
  if (tid == 0 && s_nbig > 1) {
    // dense bins in ascending order (atomics filled the list in any order;
    // the CTAs of a cluster must visit them in the same order)
    const int nb = s_nbig < kBigMax ? s_nbig : kBigMax;
    for (int a = 1; a < nb; ++a) {
      const int v = s_big[a];
      int b = a - 1;
      while (b >= 0 && s_big[b] > v) {
        s_big[b + 1] = s_big[b];
        --b;
      }
      s_big[b + 1] = v;
    }
  }
  if (active && s_bad) {
    status = kSegDense;
    active = false;
  }
  if (heavy_out) *heavy_out = s_work >= kHeavyWork || L > Fast::kCap;
  if (active && route_heavy && s_work >= kHeavyWork) {
    status = kSegHeavy;
    active = false;
  }
  if (active) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      if (rbin[k] >= 0) {
        const int slot = atomicAdd(&bcur[rbin[k]], 1);
        const long long e = tid + (long long)k * NT;
        sx[slot] = rx[k];
        sid[slot] = Is[e];
        sA[slot] = Mo[a0 + e];
        sB[slot] = Mo[d.n + a0 + e];
      }
    }
  }
  __syncthreads();
  if (active) {
    for (int b = tid; b < nb; b += NT) {
      const int lo = bstart[b], hi = bstart[b + 1];
      if (hi - lo > kBinMax) continue;  // dense bin: sorted below by the whole CTA
      for (int i = lo + 1; i < hi; ++i) {
        const long long xi = sx[i];
        const int ii = sid[i];
        const unsigned long long ai = sA[i], bi = sB[i];
        int j = i - 1;
        while (j >= lo && (sx[j] > xi || (sx[j] == xi && sid[j] > ii))) {
          sx[j + 1] = sx[j];
          sid[j + 1] = sid[j];
          sA[j + 1] = sA[j];
          sB[j + 1] = sB[j];
          --j;
        }
        sx[j + 1] = xi;
        sid[j + 1] = ii;
        sA[j + 1] = ai;
        sB[j + 1] = bi;
      }
    }
  }
  __syncthreads();
  // Dense bins, sorted by the whole CTA.  Up to kRankMax records (256 in
  // the first tier, 1023 in the second): each record's rank is the number of
  // smaller (x, id) keys in the bin, packed into 64 bits as (x - bin start)
  // << 31 | id (bins are at most 2^32 ticks wide here), then every record
  // moves to its rank.  Larger bins: in-place
  // bitonic sort, every comparator ascending (partner i ^ (2j - 1) first in
  // each merge) so any length sorts.
  if (active) {
    const int nbig = s_nbig < kBigMax ? s_nbig : kBigMax;
    // the scatter cursors are free now: they hold the packed keys
    unsigned long long* key = reinterpret_cast<unsigned long long*>(
        (reinterpret_cast<uintptr_t>(bcur) + 7) & ~static_cast<uintptr_t>(7));
    // first tier: one record per thread (registers); second tier: up to 2
    constexpr int kRankMax = (NB / 2 - 1) < (NT > 256 ? 2 * NT : NT) ? (NB / 2 - 1)
                                                                      : (NT > 256 ? 2 * NT : NT);
    constexpr int E = (kRankMax + NT - 1) / NT;  // records per thread
    for (int t = 0; t < nbig; ++t) {
      const int lo = bstart[s_big[t]], len = bstart[s_big[t] + 1] - lo;
      if (len <= kRankMax && sh2 <= 32) {
        if constexpr (CL > 1) {
          // a bin's records sit in scatter order, which differs between the
          // cluster's CTAs: all take the first CTA's arrangement
          cg::cluster_group cl = cg::this_cluster();
          cl.sync();
          if (slice != 0) {
            for (int i = tid; i < len; i += NT) {
              sx[lo + i] = *cl.map_shared_rank(&sx[lo + i], 0u);
              sid[lo + i] = *cl.map_shared_rank(&sid[lo + i], 0u);
              sA[lo + i] = *cl.map_shared_rank(&sA[lo + i], 0u);
              sB[lo + i] = *cl.map_shared_rank(&sB[lo + i], 0u);
            }
          }
          __syncthreads();
        }
        const long long blo = wlo + ((long long)s_big[t] << sh2);
        for (int i = tid; i < len; i += NT)
          key[i] = ((unsigned long long)(sx[lo + i] - blo) << 31) | (unsigned int)sid[lo + i];
        __syncthreads();
        int rk[E];
        long long vx[E];
        int vid[E];
        unsigned long long va[E], vb[E];
        if constexpr (CL > 1) {
          // second tier: the cluster's CTAs rank every CL-th record each (a
          // warp per record, lanes striding the keys) and read the other
          // ranks from their peers' shared memory (same arrangement, same
          // dense-bin order in every CTA)
          int* srank = reinterpret_cast<int*>(sr);  // free until the row sums
          cg::cluster_group cl = cg::this_cluster();
          const int nmine = (len - slice + CL - 1) / CL;
          for (int k = warp; k < nmine; k += NT / 32) {
            const int i = slice + k * CL;
            const unsigned long long mki = key[i];
            int cnt = 0;
            for (int q = lane; q < len; q += 32) cnt += key[q] < mki ? 1 : 0;
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0) srank[i] = cnt;
          }
          cl.sync();
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int i = tid + e * NT;
            if (i < len) {
              const unsigned int owner = (unsigned int)(i % CL);
              rk[e] = *cl.map_shared_rank(&srank[i], owner);
              vx[e] = sx[lo + i];
              vid[e] = sid[lo + i];
              va[e] = sA[lo + i];
              vb[e] = sB[lo + i];
            }
          }
          cl.sync();  // every peer has read this CTA's ranks
        } else {
          unsigned long long mk[E];
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int i = tid + e * NT;
            mk[e] = i < len ? key[i] : ~0ULL;
            rk[e] = 0;
          }
#pragma unroll 4
          for (int q = 0; q < len; ++q) {
            const unsigned long long kq = key[q];
#pragma unroll
            for (int e = 0; e < E; ++e) rk[e] += kq < mk[e] ? 1 : 0;
          }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            const int i = lo + tid + e * NT;
            if (tid + e * NT < len) {
              vx[e] = sx[i];
              vid[e] = sid[i];
              va[e] = sA[i];
              vb[e] = sB[i];
            }
          }
          __syncthreads();
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
          if (tid + e * NT < len) {
            const int to = lo + rk[e];
            sx[to] = vx[e];
            sid[to] = vid[e];
            sA[to] = va[e];
            sB[to] = vb[e];
          }
        }
        __syncthreads();
        continue;
      }
      int np2 = 1;
      while (np2 < len) np2 <<= 1;
      for (int mm = 2; mm <= np2; mm <<= 1) {
        for (int jj = mm >> 1; jj > 0; jj >>= 1) {
          for (int i = tid; i < np2; i += NT) {
            const int l = (jj == (mm >> 1)) ? (i ^ (mm - 1)) : (i ^ jj);
            if (l > i && l < len) {
              const int a = lo + i, b = lo + l;
              if (sx[b] < sx[a] || (sx[b] == sx[a] && sid[b] < sid[a])) {
                const long long tx = sx[a];
                sx[a] = sx[b];
                sx[b] = tx;
                const int ti = sid[a];
                sid[a] = sid[b];
                sid[b] = ti;
                const unsigned long long ta = sA[a];
                sA[a] = sA[b];
                sA[b] = ta;
                const unsigned long long tb = sB[a];
                sB[a] = sB[b];
                sB[b] = tb;
              }
            }
          }
          __syncthreads();
        }
      }
    }
  }

  // ---- 5: row sums, then exchange and reaction for own particles ----------
  const int m = bstart[nb];
  const int w0 = s_w0, w1 = s_w1;
  const long long out0 = o0 + s_lt;
  const long long S = d.S;
  if constexpr (CL == 1) {
    if (pf && tid == 0) prefetch_next_l2(d, *pf, st);
    if (!pair_transfer<PR, TR>(d, st, smem, active, m, w0, w1, out0, xlo, xhi)) {
      status = kSegHeavy;  // more pairs than the list holds: the second tier takes it
      active = false;
    }
  } else {
    // Row sums.  A particle with more than kWalk neighbours on a side is
    // dense: it is queued (in bcur, free by now) and summed by a whole warp,
    // lanes striding over its neighbour range, combined in a fixed tree.  The
    // choice and the order depend only on the neighbourhood, so every CTA that
    // forms r_j forms the same value.
    int* dlist = bcur;
    if (active) {
      for (int t = tid;; t += NT) {
        const int j = CL > 1 ? t * CL + slice : t;  // with a cluster: every CL-th
        if (j >= m) break;
        const long long x = sx[j];
        if (x < xlo - S || x >= xhi + S) continue;  // not a neighbour of an own particle
        if (dense_at(sx, m, j, x, S)) {
          const int at = atomicAdd(&s_nd, 1);
          if (at < NB) {
            dlist[at] = j;
            continue;
          }
        }
        // at most kWalk neighbours a side (or the dense list is full)
        T r = T(1);
        for (int q = j - 1; q >= 0 && x - sx[q] <= S; --q) r += W::near(d, x - sx[q]);
        for (int q = j + 1; q < m && sx[q] - x <= S; ++q) r += W::near(d, sx[q] - x);
        sr[j] = mixw(PR) ? T(__frcp_rn((float)r)) : T(rcp_ge1((double)r));
      }
    }
    __syncthreads();
    // Binary64 weights of dense rows are dear (an exponential each): the
    // predicted-segment kernel keeps them, row j of the staged slots at
    // wc[j m + q], between the row sums and the exchange (read through L2:
    // the rows are written by other CTAs of the cluster)
    constexpr bool kCache = PR == MT_FP64 && CL > 1;
    const bool cw = kCache && cache_w && (long long)m * m <= d.wc_cap;
    if (active) {
      const int nd = s_nd < NB ? s_nd : NB;
      for (int k = warp; k < nd; k += NT / 32) {
        const int j = dlist[k];
        const long long x = sx[j];
        const int lo = lower_at_least(sx, m, x - S), hi = lower_at_least(sx, m, x + S + 1);
        T* wrow = kCache ? reinterpret_cast<T*>(d.wc) + (size_t)j * m : nullptr;
        auto nu = [&](int qq) {
          const T w = W::near(d, x > sx[qq] ? x - sx[qq] : sx[qq] - x);
          if (kCache && cw) wrow[qq] = w;
          return w;
        };
        // second tier: four chains per lane (dense particles are its work);
        // first tier: one (registers are scarce there)
        T r0 = T(0), r1 = T(0), r2 = T(0), r3 = T(0);
        int q = lo + lane;
        if constexpr (CL > 1) {
          for (; q + 96 < hi; q += 128) {
            r0 += nu(q);
            r1 += nu(q + 32);
            r2 += nu(q + 64);
            r3 += nu(q + 96);
          }
        }
        for (; q < hi; q += 32) r0 += nu(q);
        const T r = warp_sum((r0 + r1) + (r2 + r3));
        if (lane == 0) sr[j] = mixw(PR) ? T(__frcp_rn((float)r)) : T(rcp_ge1((double)r));
      }
    }
    if constexpr (CL > 1) {
      // Every CTA of the cluster staged and sorted the same particles; each
      // formed the row sums of every CL-th one.  Gather the rest from the
      // peers' shared memory (distributed shared memory), between two cluster
      // barriers so no CTA reads a peer that has moved on.
      cg::cluster_group cl = cg::this_cluster();
      if (tid == 0) s_wcbad = s_nd > NB ? 1 : 0;  // a dense row summed without the cache
      cl.sync();
      if (tid == 0) {
        int bad = 0;
        for (int r = 0; r < CL; ++r) bad |= *cl.map_shared_rank(&s_wcbad, r);
        s_wcok = bad ? 0 : 1;
      }
      if (active) {
        for (int j = tid; j < m; j += NT) {
          const int owner = j % CL;
          if (owner == slice) continue;
          const long long x = sx[j];
          if (x < xlo - S || x >= xhi + S) continue;
          sr[j] = *cl.map_shared_rank(&sr[j], owner);
        }
      }
      cl.sync();
    } else {
      __syncthreads();
    }
    if (active) {
      long long* Xn = d.X[xc ^ 1];
      int* In = d.id[xc ^ 1];
      unsigned long long* Mn = d.M[mc ^ 1];
      if (out0 + (w1 - w0) > d.n) raise_error(c, kErrIndex, out0);
      for (int j = w0 + slice + tid * nslice; j < w1; j += NT * nslice) {
        const long long x = sx[j];
        const T ip = sr[j];
        if (dense_at(sx, m, j, x, S)) {
          const int at = atomicAdd(&s_nd2, 1);
          if (at < NB) {
            dlist[at] = j;  // a warp does it below
            continue;
          }
        }
        MV A = MS::load(sA, j), B = MS::load(sB, j);
        typename MS::Acc dA{}, dB{};
        for (int q = j - 1; q >= 0 && x - sx[q] <= S; --q) {
          const T P = normalised<T>(d.norm, W::near(d, x - sx[q]), ip, sr[q]);
          MS::acc(dA, P, MS::diff(MS::load(sA, q), A));
          MS::acc(dB, P, MS::diff(MS::load(sB, q), B));
        }
        for (int q = j + 1; q < m && sx[q] - x <= S; ++q) {
          const T P = normalised<T>(d.norm, W::near(d, sx[q] - x), ip, sr[q]);
          MS::acc(dA, P, MS::diff(MS::load(sA, q), A));
          MS::acc(dB, P, MS::diff(MS::load(sB, q), B));
        }
        MS::update(A, B, dA, dB, d.react);
        const long long o = out0 + (j - w0);
        if (o < d.n) {
          Xn[o] = x;
          In[o] = sid[j];
          MS::store(Mn, o, A);
          MS::store(Mn, d.n + o, B);
        }
      }
    }
    __syncthreads();
    if (active) {
      // dense own particles: one warp each, lanes striding the neighbourhood
      long long* Xn = d.X[xc ^ 1];
      int* In = d.id[xc ^ 1];
      unsigned long long* Mn = d.M[mc ^ 1];
      const int nd = s_nd2 < NB ? s_nd2 : NB;
      for (int k = warp; k < nd; k += NT / 32) {
        const int j = dlist[k];
        const long long x = sx[j];
        const T ip = sr[j];
        MV A = MS::load(sA, j), B = MS::load(sB, j);
        typename MS::Acc dA{}, dB{};
        const int lo = lower_at_least(sx, m, x - S), hi = lower_at_least(sx, m, x + S + 1);
        // second tier: four chains per lane (q, q + 32, q + 64, q + 96),
        // merged at the end; first tier: one
        typename MS::Acc cA[4] = {}, cB[4] = {};
        // the row's weights from the cache where every dense row went in
        const bool from_c = kCache && cw && s_wcok;
        const T* wrow = reinterpret_cast<const T*>(d.wc) + (size_t)j * m;
        auto pair = [&](int qq, int ch) {
          if (qq == j) return;
          const T w =
              from_c ? __ldcg(&wrow[qq]) : W::near(d, x > sx[qq] ? x - sx[qq] : sx[qq] - x);
          const T P = normalised<T>(d.norm, w, ip, sr[qq]);
          MS::acc(cA[ch], P, MS::diff(MS::load(sA, qq), A));
          MS::acc(cB[ch], P, MS::diff(MS::load(sB, qq), B));
        };
        int q = lo + lane;
        if constexpr (CL > 1) {
          for (; q + 96 < hi; q += 128) {
            pair(q, 0);
            pair(q + 32, 1);
            pair(q + 64, 2);
            pair(q + 96, 3);
          }
          for (; q < hi; q += 32) pair(q, 0);
          dA = acc_warp_sum(acc_merge(acc_merge(cA[0], cA[1]), acc_merge(cA[2], cA[3])));
          dB = acc_warp_sum(acc_merge(acc_merge(cB[0], cB[1]), acc_merge(cB[2], cB[3])));
        } else {
          for (; q < hi; q += 32) pair(q, 0);
          dA = acc_warp_sum(cA[0]);
          dB = acc_warp_sum(cB[0]);
        }
        if (lane == 0) {
          MS::update(A, B, dA, dB, d.react);
          const long long o = out0 + (j - w0);
          if (o < d.n) {
            Xn[o] = x;
            In[o] = sid[j];
            MS::store(Mn, o, A);
            MS::store(Mn, d.n + o, B);
          }
        }
      }
    }
    // no CTA of the cluster writes the next segment's cached rows before
    // every CTA has read this segment's (cw is the same in all of them)
    if (kCache && cw) cg::this_cluster().sync();
  }
  if (active && slice == 0) {
    // ---- 6: next step's cell starts and segment boundaries ----------------
    int* Sn = d.fstart[sc ^ 1];
    for (long long cc = c0 + tid; cc < c1; cc += NT) {
      const long long key = cc << wsh;
      int lo;
      if (sh2 == wsh) {
        lo = bstart[(key - wlo) >> sh2];  // bins are the cells
      } else {
        lo = w0;  // first own slot with x >= key
        int hi = w1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (sx[mid] < key)
            lo = mid + 1;
          else
            hi = mid;
        }
      }
      Sn[cc] = (int)(out0 + (lo - w0));
    }
    // Segment s2 >= 1 starts after the cell that holds slot sslot[s2] - 1;
    // this CTA sets the boundaries whose slot it wrote.  The first such s2
    // is found by a short walk from seg + 1 (out0 is near sslot[seg]).
    int* CBn = d.cb[sc ^ 1];
    const long long own = w1 - w0;
    int s2 = seg + 1;
    if (d.sslot[seg] > out0) {
      while (s2 > 1 && d.sslot[s2 - 1] > out0) --s2;
    } else if (d.sslot[seg + 1] <= out0) {
      while (s2 < d.nseg && d.sslot[s2] <= out0) ++s2;
    }
    for (s2 += tid; s2 < d.nseg; s2 += NT) {
      const long long q = d.sslot[s2] - 1;  // last slot before segment s2's first
      if (q >= out0 + own) break;
      // a realisation's first segment starts at its first cell, fixed
      if (q >= out0 && d.sreal[s2] == d.sreal[s2 - 1])
        CBn[s2] = (int)((sx[w0 + (q - out0)] >> wsh) + 1);
    }
  }
  __syncthreads();
  return status;
}

// End of a fused step (one thread, after every segment is done).
__device__ __forceinline__ void fused_advance(const Dev& d) {
  Ctrl* c = d.ctrl;
  c->step += 1;
  c->xcur ^= 1;
  c->mcur ^= 1;
  c->scur ^= 1;
  c->fallback = 0;
  c->npred = c->npred_next;
  c->npred_next = 0;
}

// The first tier and the predicted-segment kernel run side by side; the
// last CTA of each joins.  join_decide (one thread): 0 for the first of the
// two to arrive; for the second (or the first tier alone, without the
// predicted-segment kernel) 1 if the step is complete, 2 if segments were
// newly queued or a predicted segment did not fit (the second tier runs).
__device__ __forceinline__ int join_decide(const Dev& d) {
  Ctrl* c = d.ctrl;
  __threadfence();
  if (d.use_pred && atomicAdd(&c->kjoin, 1u) != 1u) return 0;  // the first of two
  __threadfence();
  const int nov = atomicAdd(&c->nov, 0);
  const int ov = atomicAdd(&c->overflow, 0);
  return nov > 0 || ov != 0 ? 2 : 1;
}

// The deciding thread: advance the step or raise the graph condition.
__device__ __forceinline__ void join_finish(const Dev& d, int role,
                                            cudaGraphConditionalHandle cond, int use_cond) {
  Ctrl* c = d.ctrl;
  const bool more = role == 2;
  if (!more) fused_advance(d);
  if (more) c->big_steps += 1;
  if (c->nov > c->ov_value) c->ov_value = c->nov;  // largest queue seen (diagnostic)
  c->kjoin = 0;
  c->seg_ctr = 0;
  if (use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
}

// The end of the first tier or the predicted-segment kernel (thread 0 of
// its last CTA).
__device__ __forceinline__ void end_of_tier(const Dev& d, cudaGraphConditionalHandle cond,
                                            int use_cond) {
  const int role = join_decide(d);
  if (role != 0) join_finish(d, role, cond, use_cond);
}

// First tier: a persistent grid (a few CTAs per SM) looping over the
// segments; each segment's boundary scalars are loaded while the previous
// segment is processed.  MT_FP64's shared memory admits three CTAs per SM,
// so it is compiled for three (more registers, none spilled).
template <int PR>
__global__ void __launch_bounds__(Fast::kT, PR == MT_FP64 ? 3 : kFusedCtasPerSm)
    k_step1d(Dev d, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ bool s_last;
  Ctrl* c = d.ctrl;
  const StepState st = step_state(d);
  const int sc = st.sc;
  const long long Dc = (c->dmax >> d.cshift) + 2;
  const unsigned char* pcur = d.pred[sc];
  unsigned char* pnext = d.pred[sc ^ 1];
  // Segments: the first wave by CTA index, then tickets.  Two segments
  // ahead: while segment `seg` is processed, the next one's scalars and
  // prediction flag load and the ticket after it is drawn, so no global
  // round trip sits between two segments.  Segments predicted pair-heavy
  // belong to the predicted-segment kernel.  (two ticket words: a skipped
  // segment has no barrier of its own before the next ticket is written)
  __shared__ int s_ticket[2];
  __shared__ int s_pre[2][8];
  if (threadIdx.x == 0) s_ticket[1] = (int)gridDim.x + atomicAdd(&c->seg_ctr, 1);
  __syncthreads();
  int par = 0;
  int seg = blockIdx.x, s1 = s_ticket[1];
  SegScalars cur = {};
  unsigned char pc = 0;
  if (seg < d.nseg) {
    cur = load_seg(d, sc, Dc, seg);
    pc = d.use_pred ? pcur[seg] : 0;
  }
  while (seg < d.nseg) {
    const SegPrefetch pf{s_pre[par], s1, sc, Dc};
    int tk = d.nseg;
    if (threadIdx.x == 0) {
      if (s1 < d.nseg) tk = (int)gridDim.x + atomicAdd(&c->seg_ctr, 1);
      prefetch_stage1(d, pf);
    }
    if (!pc) {
      const int rc = fused_segment<PR, Fast, 1>(d, st, seg, smem, cur, 0, 1, true, nullptr, &pf);
      if (rc != kSegOk && threadIdx.x == 0) d.ovlist[atomicAdd(&c->nov, 1)] = seg;
      if (threadIdx.x == 0) {
        pnext[seg] = rc == kSegOk ? 0 : 1;
        if (rc != kSegOk) atomicAdd(&c->npred_next, 1);
      }
    } else if (threadIdx.x == 0) {
      prefetch_stage2(d, pf);
    }
    if (threadIdx.x == 0) {
      __pipeline_wait_prior(0);
      s_ticket[par] = tk;
    }
    __syncthreads();
    const int s2 = s_ticket[par];
    if (s1 < d.nseg) {
      const int* w = s_pre[par];
      cur = {w[0], w[1], w[2], w[3] - w[2], w[4], w[5]};
      pc = d.use_pred ? (unsigned char)((unsigned int)w[6] >> (8 * (s1 & 3))) : 0;
    }
    par ^= 1;
    seg = s1;
    s1 = s2;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&c->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  if (threadIdx.x == 0) {
    c->done = 0;
    end_of_tier(d, cond, use_cond);
  }
}

// The predicted-segment kernel: one thread-block cluster takes the segments
// that were pair-heavy last step (the layer piled against a wall stays in
// the same segment from step to step), at the same time as the first tier
// works on the rest.  All CTAs of the cluster list the predicted segments
// in index order (an ordered compaction per chunk of indices) and process
// them one after another like the second tier; each records whether its
// segment is still heavy for the next step's prediction.
template <int PR, int CL>
__global__ void __launch_bounds__(Big::kT, 1)
    k_step1d_pred(Dev d, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ bool s_last;
  __shared__ int s_warp[Big::kT / 32];
  __shared__ int s_list[Big::kT];
  __shared__ int s_nlist;
  Ctrl* c = d.ctrl;
  const StepState st = step_state(d);
  const int sc = st.sc;
  const long long Dc = (c->dmax >> d.cshift) + 2;
  const int rank = blockIdx.x % CL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned char* pcur = d.pred[sc];
  unsigned char* pnext = d.pred[sc ^ 1];
  if (d.obs_snap && blockIdx.x == 0 && tid == 0) obs_snapshot(c);  // read behind this kernel
  if (blockIdx.x < CL && c->npred > 0) {  // the first cluster does the work
    for (int base = 0; base < d.nseg; base += Big::kT) {
      const int sidx = base + tid;
      const bool f = sidx < d.nseg && pcur[sidx] != 0;
      const unsigned int bal = __ballot_sync(0xffffffffu, f);
      if (lane == 0) s_warp[warp] = __popc(bal);
      __syncthreads();
      if (tid == 0) {
        int run = 0;
        for (int w = 0; w < Big::kT / 32; ++w) {
          const int v = s_warp[w];
          s_warp[w] = run;
          run += v;
        }
        s_nlist = run;
      }
      __syncthreads();
      if (f) s_list[s_warp[warp] + __popc(bal & ((1u << lane) - 1u))] = sidx;
      __syncthreads();
      const int nl = s_nlist;
      for (int k = 0; k < nl; ++k) {
        const int seg = s_list[k];
        bool heavy = true;
        const int rc = fused_segment<PR, Big, CL>(d, st, seg, smem, load_seg(d, sc, Dc, seg),
                                                   rank, CL, false, &heavy, nullptr, true);
        if (rc != kSegOk && tid == 0 && atomicExch(&c->overflow, 1) == 0) {
          c->ov_reason = rc;
          c->ov_seg = seg;
        }
        if (tid == 0 && rank == 0) {
          pnext[seg] = heavy ? 1 : 0;
          if (heavy) atomicAdd(&c->npred_next, 1);
        }
      }
      __syncthreads();  // s_list is rewritten for the next chunk
    }
  }
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(&c->gdone, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  if (tid == 0) {
    c->gdone = 0;
    end_of_tier(d, cond, use_cond);
  }
}

// Second tier: the queued segments with larger staging.  Each segment is
// taken by one thread-block cluster of CL CTAs (on CL SMs; 16 where the
// device can co-schedule a cluster that large, else 8): all stage and sort
// it, each forms the row sums of every CL-th particle (shared through
// distributed shared memory) and the exchange of every CL-th own particle.
// Clusters loop over the queue.
template <int PR, int CL>
__global__ void __launch_bounds__(Big::kT, 1)
    k_step1d_big(Dev d, cudaGraphConditionalHandle cond, int use_cond) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ bool s_last;
  Ctrl* c = d.ctrl;
  const int nov = c->nov;
  const StepState st = step_state(d);
  const int sc = st.sc;
  const long long Dc = (c->dmax >> d.cshift) + 2;
  const int rank = blockIdx.x % CL, cid = blockIdx.x / CL;
  const int ncl = gridDim.x / CL;
  for (int q = cid; q < nov; q += ncl) {
    const int seg = d.ovlist[q];
    const int rc =
        fused_segment<PR, Big, CL>(d, st, seg, smem, load_seg(d, sc, Dc, seg), rank, CL, false);
    if (rc != kSegOk && threadIdx.x == 0 && atomicExch(&c->overflow, 1) == 0) {
      c->ov_reason = rc;
      c->ov_seg = seg;
    }
  }
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&c->done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int ov = atomicAdd(&c->overflow, 0);
  if (threadIdx.x == 0) {
    if (!ov) fused_advance(d);
    if (ov) {
      c->fallback = 1;
      c->fallbacks += 1;
      c->overflow = 0;
    }
    c->nov = 0;
    if (use_cond) cudaGraphSetConditional(cond, ov ? 1u : 0u);
    c->done = 0;
  }
}

// fstart[target] := start (the general pipeline's cell starts), and the
// segment boundaries cb[target][s] = first cell c with start[c] >= sslot[s]
// (a realisation's first segment: the realisation's first cell).
__global__ void k_fused_prep(Dev d, int flip) {
  const int target = d.ctrl->scur ^ flip;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= d.ncell) {
    d.fstart[target][i] = d.start[i];
    if (i == d.ncell) {
      d.fstart[0][i] = (int)d.n;
      d.fstart[1][i] = (int)d.n;
    }
  }
  if (i <= d.nseg) {
    int* cb = d.cb[target];
    if (i == 0) {
      cb[0] = 0;
    } else if (i == d.nseg) {
      cb[i] = (int)d.ncell;
      d.cb[target ^ 1][i] = (int)d.ncell;
      d.cb[target ^ 1][0] = 0;
    } else if (d.sreal[i] != d.sreal[i - 1]) {
      // the first segment of a realisation starts at its first cell in both
      // buffers: no particle of another realisation ever enters it, so every
      // segment's own particles belong to one realisation
      const int first = (int)(d.rt[d.sreal[i]].base >> d.cshift);
      cb[i] = first;
      d.cb[target ^ 1][i] = first;
    } else {
      const long long want = d.sslot[i];
      long long lo = 0, hi = d.ncell;
      while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (d.start[mid] < want)
          lo = mid + 1;
        else
          hi = mid;
      }
      cb[i] = (int)lo;
    }
  }
}

__global__ void k_fused_flip(Dev d, int flip) {
  if (flip) d.ctrl->scur ^= 1;
  d.ctrl->fallback = 0;
  d.ctrl->nov = 0;
  d.ctrl->npred = d.ctrl->npred_next;
  d.ctrl->npred_next = 0;
}

// Largest |rint(b xi)| over an injected noise buffer -> Ctrl::dmax.
__global__ void k_noise_bound(Dev d, const float* xi, long long count) {
  __shared__ unsigned long long s_max;
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  unsigned long long mine = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const long long v = walk_ticks(d.bq, xi[i]);
    const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
    mine = a > mine ? a : mine;
  }
  atomicMax(&s_max, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    long long dr = d.drift[0] < 0 ? -d.drift[0] : d.drift[0];
    if (d.dim == 2) {
      const long long d2 = d.drift[1] < 0 ? -d.drift[1] : d.drift[1];
      dr = d2 > dr ? d2 : dr;
    }
    atomicMax(reinterpret_cast<unsigned long long*>(&d.ctrl->dmax),
              s_max + (unsigned long long)dr + 2ULL);
  }
}

__global__ void k_set_dmax(Dev d, long long v) { d.ctrl->dmax = v; }

// Cluster size of the second tier: 16 if a 16-CTA cluster of it can be
// resident (non-portable size), else 8.
static int g_big_cluster = 8;

// Highest launch priority of the device (the predicted-segment kernel's
// CTAs should take their SMs before the first tier fills them).
static int g_top_priority = 0;
// The first tier's launch priority: just below the predicted-segment kernel,
// above the default (lowest) priority of the work that runs beside the step
// (the previous step's observables), whose CTAs then fill the SMs the first
// tier leaves at its tail instead of taking them at its start.
static int g_fast_priority = 0;

template <int PR, int CL>
static cudaError_t configure_big(int precision) {
  auto k = k_step1d_big<PR, CL>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tier_smem<Big>(precision));
  if (e == cudaSuccess && CL > 8)
    e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  auto kp = k_step1d_pred<PR, CL>;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tier_smem<Big>(precision));
  if (e == cudaSuccess && CL > 8)
    e = cudaFuncSetAttribute(kp, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  return e;
}

template <int PR, int CL>
static int max_active_clusters(int precision) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(CL * 8);
  cfg.blockDim = dim3(Big::kT);
  cfg.dynamicSmemBytes = tier_smem<Big>(precision);
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_step1d_big<PR, CL>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Resident first-tier CTAs per SM for each precision (the persistent grid
// is that many per SM), from the occupancy calculator at configuration.
static int g_fast_ctas_per_sm[3] = {kFusedCtasPerSm, kFusedCtasPerSm, kFusedCtasPerSm};

template <int PR>
static cudaError_t configure_tiers(int cl) {
  cudaError_t e = cudaFuncSetAttribute(k_step1d<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)fused_smem_bytes(PR));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step1d<PR>, Fast::kT,
                                                    fused_smem_bytes(PR));
  if (e != cudaSuccess) return e;
  const int slot = PR == MT_FP64 ? 0 : PR == MT_MIXED ? 1 : 2;
  g_fast_ctas_per_sm[slot] = per_sm < 1 ? 1 : (per_sm > kFusedCtasPerSm ? kFusedCtasPerSm : per_sm);
  return cl == 16 ? configure_big<PR, 16>(PR) : configure_big<PR, 8>(PR);
}

int fused_ctas_per_sm(int precision) {
  const int slot = precision == MT_FP64 ? 0 : precision == MT_MIXED ? 1 : 2;
  static bool known[3] = {false, false, false};
  if (!known[slot]) {
    const cudaError_t e = precision == MT_FP64   ? configure_tiers<MT_FP64>(8)
                          : precision == MT_MIXED ? configure_tiers<MT_MIXED>(8)
                                                  : configure_tiers<MT_MIXED_DF32>(8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return kFusedCtasPerSm;
    }
    known[slot] = true;
  }
  return g_fast_ctas_per_sm[slot];
}

cudaError_t fused_configure() {
  cudaError_t e;
  if ((e = configure_tiers<MT_FP64>(8)) != cudaSuccess) return e;
  if ((e = configure_tiers<MT_MIXED>(8)) != cudaSuccess) return e;
  if ((e = configure_tiers<MT_MIXED_DF32>(8)) != cudaSuccess) return e;
  g_big_cluster = 8;
  if (configure_tiers<MT_FP64>(16) == cudaSuccess && configure_tiers<MT_MIXED>(16) == cudaSuccess &&
      configure_tiers<MT_MIXED_DF32>(16) == cudaSuccess &&
      max_active_clusters<MT_FP64, 16>(MT_FP64) >= 1 &&
      max_active_clusters<MT_MIXED, 16>(MT_MIXED) >= 1 &&
      max_active_clusters<MT_MIXED_DF32, 16>(MT_MIXED_DF32) >= 1)
    g_big_cluster = 16;
  cudaGetLastError();  // a refused non-portable size leaves the 8-CTA choice
  int lo = 0, hi = 0;
  if (cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess) {
    g_top_priority = hi;
    g_fast_priority = hi < lo ? hi + 1 : hi;  // numerically smaller is higher
  }
  cudaGetLastError();
  return cudaSuccess;
}

cudaError_t launch_fused_step(const Dev& d, int precision, cudaGraphConditionalHandle cond,
                              int use_cond, cudaStream_t s) {
  const size_t sm = fused_smem_bytes(precision);
  const int per_sm = g_fast_ctas_per_sm[precision == MT_FP64 ? 0 : precision == MT_MIXED ? 1 : 2];
  const int g = d.nseg < per_sm * d.nsm ? d.nseg : per_sm * d.nsm;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributePriority;
  at[0].val.priority = g_fast_priority;
  cfg.gridDim = dim3((unsigned int)g);
  cfg.blockDim = dim3(Fast::kT);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (precision == MT_MIXED) return cudaLaunchKernelEx(&cfg, k_step1d<MT_MIXED>, d, cond, use_cond);
  if (precision == MT_MIXED_DF32)
    return cudaLaunchKernelEx(&cfg, k_step1d<MT_MIXED_DF32>, d, cond, use_cond);
  return cudaLaunchKernelEx(&cfg, k_step1d<MT_FP64>, d, cond, use_cond);
}

template <int PR, int CL>
static cudaError_t launch_big(const Dev& d, cudaGraphConditionalHandle cond, int use_cond,
                              cudaStream_t s) {
  // up to 8 clusters, fewer if there are fewer segments
  const int clusters = d.nseg < 8 ? d.nseg : 8;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned int)(clusters * CL));
  cfg.blockDim = dim3(Big::kT);
  cfg.dynamicSmemBytes = tier_smem<Big>(PR);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_step1d_big<PR, CL>, d, cond, use_cond);
}

template <int PR, int CL>
static cudaError_t launch_pred(const Dev& d, cudaGraphConditionalHandle cond, int use_cond,
                               cudaStream_t s, cudaEvent_t started) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[3];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributePriority;
  at[1].val.priority = g_top_priority;
  cfg.gridDim = dim3((unsigned int)CL);  // one cluster
  cfg.blockDim = dim3(Big::kT);
  cfg.dynamicSmemBytes = tier_smem<Big>(PR);
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  if (started) {  // fires once every CTA of the cluster has begun
    at[2].id = cudaLaunchAttributeLaunchCompletionEvent;
    at[2].val.launchCompletionEvent.event = started;
    at[2].val.launchCompletionEvent.flags = 0;
    cfg.numAttrs = 3;
  }
  return cudaLaunchKernelEx(&cfg, k_step1d_pred<PR, CL>, d, cond, use_cond);
}

template <int PR>
static cudaError_t launch_cluster_tier(const Dev& d, bool pred, cudaGraphConditionalHandle cond,
                                       int use_cond, cudaStream_t s, cudaEvent_t started) {
  if (g_big_cluster == 16)
    return pred ? launch_pred<PR, 16>(d, cond, use_cond, s, started)
                : launch_big<PR, 16>(d, cond, use_cond, s);
  return pred ? launch_pred<PR, 8>(d, cond, use_cond, s, started)
              : launch_big<PR, 8>(d, cond, use_cond, s);
}

static cudaError_t launch_cluster(const Dev& d, int precision, bool pred,
                                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s,
                                  cudaEvent_t started = nullptr) {
  if (precision == MT_MIXED)
    return launch_cluster_tier<MT_MIXED>(d, pred, cond, use_cond, s, started);
  if (precision == MT_MIXED_DF32)
    return launch_cluster_tier<MT_MIXED_DF32>(d, pred, cond, use_cond, s, started);
  return launch_cluster_tier<MT_FP64>(d, pred, cond, use_cond, s, started);
}

cudaError_t launch_fused_big(const Dev& d, int precision, cudaGraphConditionalHandle cond,
                             int use_cond, cudaStream_t s) {
  return launch_cluster(d, precision, false, cond, use_cond, s);
}

cudaError_t launch_fused_pred(const Dev& d, int precision, cudaGraphConditionalHandle cond,
                              int use_cond, cudaStream_t s, cudaEvent_t started) {
  return launch_cluster(d, precision, true, cond, use_cond, s, started);
}

// Direct launches without a predicted segment: the first tier's partner in
// the join (launched before the first tier, so it arrives first).
__global__ void k_join_stub(Dev d) { end_of_tier(d, 0, 0); }

cudaError_t launch_join_stub(const Dev& d, cudaStream_t s) {
  k_join_stub<<<1, 1, 0, s>>>(d);
  return cudaGetLastError();
}

cudaError_t launch_fused_prep(const Dev& d, int flip, cudaStream_t s) {
  long long cnt = (d.ncell > d.nseg ? d.ncell : d.nseg) + 1;
  cnt = cnt > d.nreal ? cnt : d.nreal;
  k_fused_prep<<<(unsigned int)((cnt + 255) / 256), 256, 0, s>>>(d, flip);
  k_fused_flip<<<1, 1, 0, s>>>(d, flip);
  return cudaGetLastError();
}

cudaError_t launch_noise_bound(const Dev& d, const float* xi, cudaStream_t s) {
  if (!xi) {
    // built-in generator: |z| <= sqrt(-2 ln 2^-24) < 5.78
    long long dr = d.drift[0] < 0 ? -d.drift[0] : d.drift[0];
    if (d.dim == 2) {
      const long long d2 = d.drift[1] < 0 ? -d.drift[1] : d.drift[1];
      dr = d2 > dr ? d2 : dr;
    }
    k_set_dmax<<<1, 1, 0, s>>>(d, dr + (long long)ceil(d.bq * 5.78) + 2);
    return cudaGetLastError();
  }
  k_set_dmax<<<1, 1, 0, s>>>(d, 0);
  const long long cnt = (long long)d.dim * d.n;
  if (cnt > 0) {
    const unsigned int g = (unsigned int)((cnt + 255) / 256 < 1024 ? (cnt + 255) / 256 : 1024);
    k_noise_bound<<<g, 256, 0, s>>>(d, xi, cnt);
  }
  return cudaGetLastError();
}

}  // namespace mt
