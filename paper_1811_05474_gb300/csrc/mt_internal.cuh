// mt_internal.cuh -- device-side state, shared device helpers and kernel
// launchers of libmt.  See include/mt.h for the public contract.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mt.h"

namespace mt {

constexpr int kThreads = 256;          // threads per CTA for per-particle kernels
constexpr int kScanItems = 16;         // cell counts per thread in the scan
constexpr int kScanTile = kThreads * kScanItems;
constexpr int kSmallCell = 32;         // cells up to this size sort in one thread
constexpr int kBigSortCap = 2048;      // cells up to this size sort in shared memory
constexpr int kBruteTile = 256;        // j-particles staged per tile, brute force
constexpr long long kSpinLimit = 1LL << 22;  // bounded waits (scan look-back)
constexpr int kObsChunk = 4096;  // slots per observables chunk (16 per thread)
constexpr double kTileMinNeighbours = 32.0;  // mean neighbours a side for tiled passes
constexpr int kFusedCap = 1024;        // particles one fused-step CTA stages
constexpr int kFusedCtasPerSm = 4;     // resident CTAs per SM of the fused step (at most)
constexpr int kFusedPairCap = 2048;    // unordered pairs one fused-step CTA lists

// Device error codes (Ctrl::err); the first one raised is kept.
enum : int { kErrNone = 0, kErrIndex = 1, kErrTimeout = 2, kErrInput = 3 };

// Per-handle control block in device memory.  Kernels read the ping-pong
// selectors and the step counter from here, so a captured graph replays
// correctly step after step.
struct Ctrl {
  unsigned long long step;      // completed steps since upload
  unsigned long long epoch;     // scan epoch (tags look-back status words)
  unsigned long long npairs;    // pair export counter
  int xcur;                     // which X / id buffer holds the current state
  int mcur;                     // which mass buffer holds the current masses
  int err;                      // first device error code
  int nbig;                     // cells too large for the per-thread sort
  unsigned int done;            // CTAs finished (last-CTA reductions)
  unsigned int tile_ctr;        // scan tile ticket
  long long err_info;           // detail for err (an index)
  const float* noise;           // injected normals [dim][n] by caller index, or null
  long long dmax;               // bound on one step's displacement, in ticks
  int scur;                     // which fused start / segment array is current
  int overflow;                 // a fused-step segment did not fit (this step)
  int fallback;                 // the general pipeline must redo this step
  int ov_reason;                // first second-tier overflow: 1 capacity, 2 dense bins
  long long ov_seg;             // ... its segment
  long long ov_value;           // ... (reserved)
  unsigned long long fallbacks; // steps the general pipeline redid since upload
  unsigned long long big_steps; // steps that needed the second fused tier
  int nov;                      // segments queued for the second tier this step
  int seg_ctr;                  // first-tier segments handed out beyond the first wave
  unsigned int gdone;           // CTAs of the predicted-segment kernel finished
  unsigned int kjoin;           // of the two concurrent fused kernels, how many are done
  int npred;                    // segments predicted pair-heavy for this step
  int npred_next;               // ... counted during this step for the next
  int scan_hold;                // test hook: the scan's first tile withholds its status
  long long spin_limit;         // bound of each look-back wait (0: kSpinLimit)
  // Observables of the previous step, computed beside a step (the fused
  // path's graph): the state's mass buffer and step at the step's start,
  // whether that step's rows are still to be written, and the last step
  // whose rows were written.
  int obs_mc;
  int obs_prev_todo;
  unsigned long long obs_step;
  unsigned long long obs_done_step;
};

// The snapshot the previous step's observables read (one thread, at the
// start of a step, before the step advances the control block).
__device__ __forceinline__ void obs_snapshot(Ctrl* c) {
  c->obs_mc = c->mcur;
  c->obs_step = c->step;
  c->obs_prev_todo = c->step > 0 && c->obs_done_step != c->step ? 1 : 0;
}

// One realisation of a batch (a single system is a batch of one).  Batched
// realisations are 1-d and sit side by side on one tick axis: realisation r
// owns [base, base + Lq], and consecutive domains are more than Smax apart,
// so no pair crosses two realisations.  A particle's id is (r << lbits) |
// its index within r, and its caller index is off + that index.
struct Real {
  long long base;      // first tick of its domain on the shared axis
  long long Lq;        // its domain length in ticks
  long long off;       // its first particle in the caller's order
  long long n;         // its particles
  unsigned int real;   // Philox counter word of its random walk
  int seg0;            // its first fused segment
  int nseg;            // its fused segments
  int ch0;             // its first observables chunk
  int nch;             // its observables chunks
  int pad;
};

// Everything a kernel needs, passed by value.
struct Dev {
  Ctrl* ctrl;
  long long* X[2];          // [dim][n] grid ticks, ping-pong
  int* id[2];               // caller's index of each slot, ping-pong
  unsigned long long* M[2]; // [2][n] 8-byte mass words (A then B), ping-pong
  int* src;                 // slot -> slot before the sort
  void* rinv;               // 1 / r_i (double in FP64, float in MIXED)
  int* count;               // [ncell] particles per cell
  int* start;               // [ncell + 1] first slot of each cell
  int* cursor;              // [ncell] scatter cursor
  unsigned long long* scan_status;  // [ntiles] look-back words
  int* big;                 // [nbig_cap] cells for the large-cell sort
  int* ochunk;              // [nochunk + 1] first slot of each observables chunk
  int nochunk;
  unsigned long long* opart;  // [nochunk][4] chunk sums (8-byte words)
  int* ochr;                // [nochunk] realisation of each chunk
  int* ocnt;                // [nreal] chunks summed this step
  double* obs;              // [observe_cap][4] observables ring
  int* fstart[2];           // [ncell + 1] cell starts of the sorted state (fused path)
  int* cb[2];               // [nseg + 1] first cell of each fused segment
  int* ovlist;              // [nseg] segments queued for the second fused tier
  unsigned char* pred[2];   // [nseg] segments predicted pair-heavy (by scur parity)
  int use_pred;             // 1: the predicted-segment kernel runs beside the first tier
  int obs_snap;             // 1: the predicted-segment kernel takes the observables' snapshot
  double* wc;               // [wc_cap] the cluster kernel's cache of dense rows' binary64 weights
  long long wc_cap;         // doubles (0: none)
  int periodic;             // 1: periodic walls (wrap, minimum-image separations)
  int nspec;                // species per particle (masses hold nspec * n words)
  int band_cap;             // SPaM form: stored weights per particle (0: off)
  int tile;                 // 1: dense 1-d transfer passes over shared-memory tiles
  int* cnt;                 // [2][n] SPaM: right, then left neighbours of each slot
  void* band;               // SPaM: nu(p, p + k), k <= band_cap, in tiles of 32 slots
  long long n;
  int dim;
  int norm;                 // MT_NORM_*
  int react;
  int observe_cap;
  int cshift;               // cell width 2^cshift ticks
  long long ncx, ncy, ncell;
  long long S;              // cutoff in ticks
  long long Lq[2];          // domain length in ticks
  long long drift[2];       // v dt in ticks
  double bq;                // sqrt(2 D_rw dt) 2^k
  float inv8f;              // 1 / (8 D_mt dt) 2^-2k, float
  double inv8;              // 1 / (8 D_mt dt), double
  double scale;             // 2^-k
  double inv8s;             // inv8 scale^2 (exact): the weights' exponent from D^2 in ticks
  unsigned int key0, key1;  // Philox key (seed)
  unsigned int real;        // realisation counter word
  int nbig_cap;
  int nseg;                 // fused segments (CTAs of the fused step)
  int seg_target;           // particles a fused segment aims for
  int nsm;                  // multiprocessors of the device
  long long hc;             // fused halo in cells (covers 2 Smax)
  const Real* rt;           // [nreal] realisations
  int nreal;
  int lbits;                // id = (realisation << lbits) | index within it
  int lmask;                // (1 << lbits) - 1
  const int* sslot;         // [nseg + 1] first slot each fused segment aims for
  const int* sreal;         // [nseg] realisation of each fused segment
};

// Caller index of a particle id.
__device__ __forceinline__ long long caller_index(const Dev& d, int id) {
  return d.rt[id >> d.lbits].off + (id & d.lmask);
}

// ---------------------------------------------------------------- helpers --

__device__ __forceinline__ void raise_error(Ctrl* c, int code, long long info) {
  if (atomicCAS(&c->err, 0, code) == 0) c->err_info = info;
}

// Mirror y back into [0, Lq] (Sec. 3 reflecting walls), at most 64 times.
__device__ __forceinline__ long long reflect(long long y, long long Lq) {
#pragma unroll 1
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

// A and B of the particle in slot s of buffer mc move to slot p of the
// other buffer (species 2 and up: gather_species, in a pass of their own so
// the transfer kernels keep their registers).
__device__ __forceinline__ void gather_masses(const Dev& d, int mc, long long p, long long s) {
  const unsigned long long* in = d.M[mc];
  unsigned long long* out = d.M[mc ^ 1];
  out[p] = in[s];
  out[d.n + p] = in[d.n + s];
}
__device__ __forceinline__ void gather_species(const Dev& d, int mc, long long p, long long s) {
  const unsigned long long* in = d.M[mc];
  unsigned long long* out = d.M[mc ^ 1];
  for (int k = 2; k < d.nspec; ++k) out[k * d.n + p] = in[k * d.n + s];
}

// Periodic walls: y modulo Lq into [0, Lq).
__device__ __forceinline__ long long wrap(long long y, long long Lq) {
  const long long m = y % Lq;
  return m < 0 ? m + Lq : m;
}

// Periodic walls in 1-d: the ring of sorted slots a particle's walks go
// around -- its realisation's slot range [off, off + n) -- and the domain
// length the separations wrap at (a single system is realisation 0).
struct Ring {
  long long off, n, Lq;
};
__device__ __forceinline__ Ring ring_of(const Dev& d, int id) {
  const Real& R = d.rt[id >> d.lbits];
  return {R.off, R.n, R.Lq};
}
// Slot k steps to the right (left for k < 0, |k| < n) of slot p on ring g.
__device__ __forceinline__ long long ring_step(const Ring& g, long long p, long long k) {
  long long q = p + k;
  if (q < g.off) q += g.n;
  else if (q >= g.off + g.n) q -= g.n;
  return q;
}

// Periodic walls: the minimum-image separation of two positions in [0, Lq),
// in (-Lq/2, Lq/2].
__device__ __forceinline__ long long min_image(long long s, long long Lq) {
  if (2 * s > Lq) return s - Lq;
  if (2 * s <= -Lq) return s + Lq;
  return s;
}

__device__ __forceinline__ long long cell_of(const Dev& d, long long x, long long y) {
  long long kx = x >> d.cshift;
  kx = kx < 0 ? 0 : (kx >= d.ncx ? d.ncx - 1 : kx);
  if (d.dim == 1) return kx;
  long long ky = y >> d.cshift;
  ky = ky < 0 ? 0 : (ky >= d.ncy ? d.ncy - 1 : ky);
  return ky * d.ncx + kx;
}

// 2-d cell list (cells wider than Smax): the cells of one axis that can hold
// a neighbour of coordinate v.  Reflecting walls: the cell of v and the two
// beside it.  Periodic walls: the cells covering [v - Smax, v + Smax], in two
// pieces when the interval wraps (merged into every cell when they meet, so
// no cell is visited twice).  [a0, a1] and [b0, b1] (b0 > b1: no second).
struct CellSpan {
  long long a0, a1, b0, b1;
};
__device__ __forceinline__ CellSpan axis_cells(const Dev& d, long long v, long long Lq,
                                               long long nc) {
  auto cell = [&](long long u) {
    const long long k = u >> d.cshift;
    return k < 0 ? 0 : (k >= nc ? nc - 1 : k);
  };
  CellSpan s{0, -1, 0, -1};
  if (!d.periodic) {
    const long long k = cell(v);
    s.a0 = k > 0 ? k - 1 : 0;
    s.a1 = k + 1 < nc ? k + 1 : nc - 1;
    return s;
  }
  const long long lo = v - d.S, hi = v + d.S;
  if (lo < 0) {
    s = {0, cell(hi), cell(lo + Lq), nc - 1};
  } else if (hi >= Lq) {
    s = {0, cell(hi - Lq), cell(lo), nc - 1};
  } else {
    s.a0 = cell(lo);
    s.a1 = cell(hi);
  }
  if (s.b0 <= s.b1 && s.a1 >= s.b0 - 1) s = {0, nc - 1, 0, -1};
  return s;
}

// Calls f(q0, q1) for each run [q0, q1) of sorted slots (one per cell row
// and x piece) that can hold a neighbour of (x, y).
template <class F>
__device__ __forceinline__ void cells2_visit(const Dev& d, long long x, long long y, F&& f) {
  const CellSpan cx = axis_cells(d, x, d.Lq[0], d.ncx);
  const CellSpan cy = axis_cells(d, y, d.Lq[1], d.ncy);
  for (int iy = 0; iy < 2; ++iy) {
    const long long r0 = iy ? cy.b0 : cy.a0, r1 = iy ? cy.b1 : cy.a1;
    for (long long row = r0; row <= r1; ++row)
      for (int ix = 0; ix < 2; ++ix) {
        const long long k0 = ix ? cx.b0 : cx.a0, k1 = ix ? cx.b1 : cx.a1;
        if (k0 <= k1) f((int)d.start[row * d.ncx + k0], (int)d.start[row * d.ncx + k1 + 1]);
      }
  }
}

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of the
// 2x(32x32->64) multiply / xor network with Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, unsigned int k0, unsigned int k1) {
  const unsigned int M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const unsigned int W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned int lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const unsigned int lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += W0;
    k1 += W1;
  }
  return c;
}

// 64-bit integer -> binary32 conversion through 32-bit instructions
// (conversions with a 64-bit integer operand run on the binary64 pipe, which
// is narrow on this GPU).  Rounds to nearest even, like the 64-bit form.
__device__ __forceinline__ float ll_to_float(long long v) {
  if (v >= -2147483647LL && v <= 2147483647LL) return __int2float_rn((int)v);
  // |v| >= 2^31: the high word carries every bit binary32 can keep except
  // a possible sticky tail, which the low word's contribution rounds in.
  const float hi = __int2float_rn((int)(v >> 32)) * 4294967296.0f;
  const float lo = __uint2float_rn((unsigned int)(v & 0xffffffffLL));
  return __fadd_rn(hi, lo);
}

// Exact binary32 -> binary64 widening from the bits, with integer
// operations only (the binary64 pipe is kept for arithmetic): the sign,
// the exponent re-biased (subnormals normalised), the fraction moved to the
// top of 52 bits; infinities and NaNs keep their class and payload.
__device__ __forceinline__ double widen_exact(float f) {
  const unsigned int u = __float_as_uint(f);
  const unsigned int ex = u & 0x7f800000u;
  if (ex != 0u && ex != 0x7f800000u) {  // a normal number: the high word is the sign, the
    // exponent + 896 and the fraction's top 20 bits; the low word its last 3 bits
    const unsigned int hi = (u & 0x80000000u) | (((u & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hi, (int)(u << 29));
  }
  const unsigned int e = (u >> 23) & 0xffu, m = u & 0x7fffffu;
  unsigned long long E, F;
  if (e == 0xffu) {
    E = 0x7ff;
    F = (unsigned long long)m << 29;
  } else if (e != 0u) {
    E = e + 896u;
    F = (unsigned long long)m << 29;
  } else if (m != 0u) {  // m * 2^-149 with its leading bit at p
    const int p = 31 - __clz(m);
    E = (unsigned long long)(p + 874);
    F = ((unsigned long long)m << (52 - p)) & ((1ULL << 52) - 1);
  } else {
    E = 0;
    F = 0;
  }
  return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | (E << 52) | F));
}

// An int as binary64 from its bits with integer operations only (exact:
// every int is a binary64 number).
__device__ __forceinline__ double i2d_exact(int v) {
  if (v == 0) return 0.0;
  const unsigned int a = v < 0 ? 0u - (unsigned int)v : (unsigned int)v;
  const int p = 31 - __clz(a);  // leading bit
  const unsigned long long m = ((unsigned long long)a << (52 - p)) & ((1ULL << 52) - 1);
  return __longlong_as_double((long long)(((unsigned long long)(v < 0) << 63) |
                                          ((unsigned long long)(p + 1023) << 52) | m));
}

// 1 / r for a row sum r >= 1 (finite) in binary64 without a division: a
// binary32 reciprocal of r's leading 24 bits (read from its bits), widened,
// then two Newton steps y <- y + y (1 - r y) with fused multiply-adds
// (relative error 2^-22 -> 2^-44 -> below 2^-88 before the last rounding):
// within one unit in the last place of 1 / r.
__device__ __forceinline__ double rcp_ge1(double r) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(r);
  const unsigned int e = (unsigned int)((u >> 52) & 0x7ff);
  const float rf = __uint_as_float(((e - 1023u + 127u) << 23) | (unsigned int)((u >> 29) & 0x7fffffu));
  double y = widen_exact(__frcp_rn(rf));
  y = __fma_rn(y, __fma_rn(-r, y, 1.0), y);
  return __fma_rn(y, __fma_rn(-r, y, 1.0), y);
}

// Eq. 2's random-walk displacement on the grid: the nearest tick to b xi,
// b = sqrt(2 D_rw dt) 2^k, with the product formed in binary64.
__device__ __forceinline__ long long walk_ticks(double b, float xi) {
  return __double2ll_rn(__dmul_rn(b, (double)xi));
}

// Two standard normals from two 32-bit words (Box-Muller, binary32, with
// the hardware logarithm and sine/cosine): u1 in (0, 1], angle uniform on
// [-pi, pi).  |z| <= sqrt(-2 ln 2^-24) < 5.78.
__device__ __forceinline__ float2 box_muller(unsigned int a, unsigned int b) {
  const float u1 = ((a >> 8) + 1u) * (1.0f / 16777216.0f);
  const float u2 = (b >> 8) * (1.0f / 16777216.0f);
  const float rad = sqrtf(-2.0f * __logf(u1));
  float s, c;
  __sincosf(__fmaf_rn(6.28318530717958648f, u2, -3.14159265358979324f), &s, &c);
  return make_float2(rad * c, rad * s);
}

// ------------------------------------------ double-binary32 mass arithmetic --
// A mass in MIXED precision is hi + lo with |lo| <= ulp(hi)/2.  The additions
// are error-free transformations (Knuth two-sum, Dekker fast-two-sum).

struct df {
  float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  const df s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.hi, b.hi);
  const df t = two_sum(a.lo, b.lo);
  df u = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }

__device__ __forceinline__ bool df_le(df a, df b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo);
}

__device__ __forceinline__ df df_load(const unsigned long long* M, long long i) {
  const float2 v = reinterpret_cast<const float2*>(M)[i];
  return {v.x, v.y};
}

__device__ __forceinline__ void df_store(unsigned long long* M, long long i, df v) {
  reinterpret_cast<float2*>(M)[i] = make_float2(v.hi, v.lo);
}

__device__ __forceinline__ double f64_load(const unsigned long long* M, long long i) {
  return __longlong_as_double((long long)M[i]);
}

__device__ __forceinline__ void f64_store(unsigned long long* M, long long i, double v) {
  M[i] = (unsigned long long)__double_as_longlong(v);
}

// ---------------------------------------------------------------- launchers --
// Each returns the cudaError_t of its launch.  grid sizes are computed from d.
// A Marker, when enabled, records a CUDA event on the stream before each
// kernel so that a step's kernels can be timed one by one.

constexpr int kMaxMarks = 16;

struct Marker {
  cudaEvent_t* ev = nullptr;  // null: disabled
  const char** names = nullptr;
  int count = 0;
  // Mark the start of kernel `name`; a null name marks the start of a gap
  // (the stream idles while the host reads device state), not a kernel.
  void operator()(const char* name, cudaStream_t s) {
    if (!ev || count >= kMaxMarks) return;
    names[count] = name;
    record(ev[count], s);
    ++count;
  }
  // Inside stream capture the record must become an external event node
  // so that every graph replay records it.
  static cudaError_t record(cudaEvent_t e, cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    return st == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal)
               : cudaEventRecord(e, s);
  }
};

cudaError_t launch_move(const Dev& d, bool move, bool hist, cudaStream_t s);
cudaError_t launch_sort(const Dev& d, cudaStream_t s, Marker& mk);  // scan, scatter, cell sort
cudaError_t launch_permute(const Dev& d, cudaStream_t s);  // gather id/masses after sort, flip
cudaError_t launch_transfer(const Dev& d, int search, int precision, cudaStream_t s, Marker& mk);
// after a step: the observables row of every realisation
cudaError_t launch_obs(const Dev& d, int precision, cudaStream_t s);
// the fused path's graph: snapshot the state's buffer and step, then (beside
// the step's kernels) the observables of the state at the snapshot
cudaError_t launch_obs_snapshot(const Dev& d, cudaStream_t s);
cudaError_t launch_obs_prev(const Dev& d, int precision, cudaStream_t s);
cudaError_t launch_upload(const Dev& d, const double* x, const double* A,
                          const double* B, int precision, cudaStream_t s);
cudaError_t launch_read_masses(const Dev& d, double* A, double* B, int precision,
                               cudaStream_t s);
// in != NULL: species sp <- in[n] (caller's order); else out[n] <- species sp
cudaError_t launch_species_io(const Dev& d, int sp, double* out, const double* in, int precision,
                              cudaStream_t s);
cudaError_t launch_read_positions(const Dev& d, double* x, long long* X, cudaStream_t s);
cudaError_t launch_pairs(const Dev& d, int search, int* pi, int* pj, long long cap,
                         cudaStream_t s);
// Fused 1-d step (mt_fused.cu).
size_t fused_smem_bytes(int precision);
cudaError_t fused_configure();  // opt in to the large dynamic shared memory
int fused_ctas_per_sm(int precision);  // resident first-tier CTAs per SM
cudaError_t launch_fused_step(const Dev& d, int precision, cudaGraphConditionalHandle cond,
                              int use_cond, cudaStream_t s);
// started (optional): an event that fires once every CTA of the kernel has
// begun (a launch-completion event)
cudaError_t launch_fused_pred(const Dev& d, int precision, cudaGraphConditionalHandle cond,
                              int use_cond, cudaStream_t s, cudaEvent_t started = nullptr);  // predicted heavy segments
cudaError_t launch_join_stub(const Dev& d, cudaStream_t s);
cudaError_t launch_fused_big(const Dev& d, int precision, cudaGraphConditionalHandle cond,
                             int use_cond, cudaStream_t s);
cudaError_t launch_fused_prep(const Dev& d, int flip, cudaStream_t s);  // start/cb from d.start
cudaError_t launch_noise_bound(const Dev& d, const float* xi, cudaStream_t s);

cudaError_t launch_philox(uint4 c, unsigned int k0, unsigned int k1, long long n,
                          unsigned int* out, cudaStream_t s);
cudaError_t launch_walk_normals(const long long* gid, long long n, unsigned long long step,
                                unsigned int real, unsigned int k0, unsigned int k1, int dim,
                                float* out, cudaStream_t s);

}  // namespace mt
