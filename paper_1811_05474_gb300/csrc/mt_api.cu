// mt_api.cu -- the C ABI of libmt (include/mt.h): parameter resolution and
// validation, workspace layout, step sequencing on the handle's stream, CUDA
// graph replay for mt_run, read-back and error reporting.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mt_internal.cuh"

using namespace mt;

namespace {

thread_local std::string g_err;

mt_status fail(mt_status s, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
mt_status fail(mt_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(MT_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                           \
  } while (0)

constexpr double kTwo30 = 1073741824.0;            // 2^30
constexpr double kTwo61 = 2305843009213693952.0;   // 2^61
constexpr size_t kAlign = 256;
constexpr long long kWcCap = 1LL << 22;  // 32 MiB of cached weights (rows of up to 2048 slots)
constexpr long long kWcMinN = 1LL << 17;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Everything derived from mt_params that the kernels need.
struct Derived {
  mt_params p;  // resolved
  long long S = 0, Lq[2] = {0, 0}, drift[2] = {0, 0};
  double bq = 0.0;
  int cshift = 0;
  long long ncx = 1, ncy = 1, ncell = 0;
  long long nbig_cap = 0, ntiles = 0;
  long long wc_cap = 0;  // doubles of the dense-row weight cache
  // fused 1-d step (one kernel per step) and its tiling
  bool fused = false;
  long long seg_target = 0, nseg = 0, hc = 0;
  // realisations (one for a single system) and the fused segments' targets
  int nreal = 1, lbits = 31;
  std::vector<Real> rt;
  std::vector<int> sslot, sreal;
  std::vector<int> ochunk;  // first slot of each observables chunk (+ n)
  std::vector<int> ochr;    // realisation of each chunk
  // workspace offsets
  size_t o_ctrl, o_X[2], o_id[2], o_M[2], o_src, o_rinv, o_count, o_start, o_cursor,
      o_status, o_big, o_obs, o_fstart[2], o_cb[2], o_ovlist, o_pred[2], o_rt, o_sslot,
      o_sreal, o_ochunk, o_opart, o_ochr, o_ocnt, o_cnt, o_band, o_wc, total;
  long long band = 0;  // SPaM band entries per particle (0: off)
  bool tile = false;   // dense 1-d: tiled transfer passes
};

int default_frac_bits(const mt_params& p) {
  double Lmax = p.L[0];
  if (p.dim == 2 && p.L[1] > Lmax) Lmax = p.L[1];
  int k = 62;
  while (k > 0 && (std::ldexp(p.cutoff, k) >= kTwo30 || std::ldexp(Lmax, k) >= kTwo61)) --k;
  return k;
}

// Multiprocessors of the current device (0 without one), read once.
int device_sms() {
  static int cached = -1;
  if (cached < 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      n = 0;
    cudaGetLastError();
    cached = n;
  }
  return cached;
}

int ceil_log2(long long v) {  // smallest c with 2^c >= v (v >= 1)
  int c = 0;
  while (c < 62 && (1LL << c) < v) ++c;
  return c;
}

int floor_log2(double v) {  // v >= 1
  int c = 0;
  while (c < 62 && std::ldexp(1.0, c + 1) <= v) ++c;
  return c;
}

// b: a batch of independent 1-d realisations, or NULL for one system.
mt_status resolve(const mt_params* in, const mt_batch* b, Derived* out) {
  if (!in) return fail(MT_ERR_INVALID, "params is NULL");
  Derived D;
  mt_params p = *in;
  if (p.dim != 1 && p.dim != 2) return fail(MT_ERR_INVALID, "dim must be 1 or 2 (got %d)", p.dim);
  long long nmax = 0;
  if (b) {
    if (b->count < 1) return fail(MT_ERR_INVALID, "a batch needs >= 1 realisation");
    if (!b->n || !b->L) return fail(MT_ERR_INVALID, "batch n and L arrays are required");
    if (p.dim != 1) return fail(MT_ERR_INVALID, "batches are 1-d");
    if (p.search != MT_SEARCH_CELL) return fail(MT_ERR_INVALID, "batches use MT_SEARCH_CELL");
    long long tot = 0;
    double Lmax = 0.0;
    for (int r = 0; r < b->count; ++r) {
      if (b->n[r] < 1 || b->n[r] >= (1LL << 31))
        return fail(MT_ERR_INVALID, "realisation %d: n must be in [1, 2^31)", r);
      if (!finite_pos(b->L[r]))
        return fail(MT_ERR_INVALID, "realisation %d: L must be finite and > 0", r);
      tot += b->n[r];
      if (tot >= (1LL << 31) - 1) return fail(MT_ERR_INVALID, "batch has >= 2^31 - 1 particles");
      nmax = b->n[r] > nmax ? b->n[r] : nmax;
      Lmax = b->L[r] > Lmax ? b->L[r] : Lmax;
    }
    const int lb = ceil_log2(nmax);
    if (lb > 30 || ((long long)b->count << lb) > (1LL << 31))
      return fail(MT_ERR_INVALID, "batch: count * 2^ceil(log2(max n)) must be <= 2^31");
    D.nreal = b->count;
    D.lbits = lb;
    p.n = tot;
    p.L[0] = Lmax;  // for the grid rule; replaced by the shared axis below
  }
  if (p.n < 0 || p.n >= (1LL << 31) - 1)
    return fail(MT_ERR_INVALID, "n must be in [0, 2^31 - 1) (got %lld)", (long long)p.n);
  for (int a = 0; a < p.dim; ++a)
    if (!finite_pos(p.L[a])) return fail(MT_ERR_INVALID, "L[%d] must be finite and > 0", a);
  if (p.dim == 1) p.L[1] = 0.0, p.v[1] = 0.0;
  if (!finite_pos(p.D_mt)) return fail(MT_ERR_INVALID, "D_mt must be finite and > 0");
  if (!(std::isfinite(p.D_rw) && p.D_rw >= 0.0))
    return fail(MT_ERR_INVALID, "D_rw must be finite and >= 0");
  if (!finite_pos(p.dt)) return fail(MT_ERR_INVALID, "dt must be finite and > 0");
  for (int a = 0; a < p.dim; ++a)
    if (!std::isfinite(p.v[a])) return fail(MT_ERR_INVALID, "v[%d] must be finite", a);
  if (!std::isfinite(p.cutoff)) return fail(MT_ERR_INVALID, "cutoff must be finite");
  if (p.cutoff <= 0.0) p.cutoff = 3.0 * std::sqrt(4.0 * p.D_mt * p.dt);
  if (p.search < MT_SEARCH_CELL || p.search > MT_SEARCH_FULL)
    return fail(MT_ERR_INVALID, "unknown search %d", p.search);
  if (p.precision != MT_FP64 && p.precision != MT_MIXED && p.precision != MT_MIXED_DF32)
    return fail(MT_ERR_INVALID, "unknown precision %d", p.precision);
  if (p.norm != MT_NORM_SYM && p.norm != MT_NORM_ROW)
    return fail(MT_ERR_INVALID, "unknown norm %d", p.norm);
  if (p.react != 0 && p.react != 1) return fail(MT_ERR_INVALID, "react must be 0 or 1");
  if (p.observe_cap < 0) return fail(MT_ERR_INVALID, "observe_cap must be >= 0");
  if (p.walls != MT_WALLS_REFLECT && p.walls != MT_WALLS_PERIODIC)
    return fail(MT_ERR_INVALID, "unknown walls %d", p.walls);
  if (p.species == 0) p.species = 2;
  if (p.species < 2 || p.species > MT_MAX_SPECIES)
    return fail(MT_ERR_INVALID, "species must be 0 or in [2, %d] (got %d)", MT_MAX_SPECIES,
                p.species);
  if (p.stored_p < 0) return fail(MT_ERR_INVALID, "stored_p must be >= 0");
  if (p.stored_p > 0 && (p.dim != 1 || p.search != MT_SEARCH_CELL))
    return fail(MT_ERR_INVALID, "stored_p needs 1-d MT_SEARCH_CELL");
  const bool periodic = p.walls == MT_WALLS_PERIODIC;
  if (p.frac_bits == 0) p.frac_bits = default_frac_bits(p);
  const int k = p.frac_bits;
  if (k < 1 || k > 62) return fail(MT_ERR_INVALID, "frac_bits must be in [1, 62] (got %d)", k);
  if (std::ldexp(p.cutoff, k) >= kTwo30)
    return fail(MT_ERR_INVALID, "cutoff * 2^frac_bits must be < 2^30");
  for (int a = 0; a < p.dim; ++a) {
    if (std::ldexp(p.L[a], k) >= kTwo61)
      return fail(MT_ERR_INVALID, "L[%d] * 2^frac_bits must be < 2^61", a);
    const double drift = std::ldexp(p.v[a] * p.dt, k);
    if (std::fabs(drift) >= kTwo61 / 4)
      return fail(MT_ERR_INVALID, "|v[%d] dt| 2^frac_bits must be < 2^59", a);
    D.Lq[a] = std::llrint(std::ldexp(p.L[a], k));
    D.drift[a] = std::llrint(drift);
  }
  const double bw = std::ldexp(std::sqrt(2.0 * p.D_rw * p.dt), k);
  if (bw * 64.0 >= kTwo61 / 4)
    return fail(MT_ERR_INVALID, "sqrt(2 D_rw dt) 2^frac_bits is too large for the grid");
  D.bq = bw;
  D.S = (long long)std::floor(std::ldexp(p.cutoff, k));
  if (periodic && p.search != MT_SEARCH_FULL) {
    for (int a = 0; a < p.dim; ++a)
      if (!b && 2 * D.S >= D.Lq[a])
        return fail(MT_ERR_INVALID, "periodic walls need the cutoff below L[%d]/2", a);
    if (b)
      for (int r = 0; r < b->count; ++r)
        if (2 * D.S >= std::llrint(std::ldexp(b->L[r], k)))
          return fail(MT_ERR_INVALID, "realisation %d: periodic walls need the cutoff below L/2", r);
  }
  // cell grid
  std::vector<long long> lq;  // batch: each realisation's length in ticks
  double lq_sum = (double)D.Lq[0];
  if (b) {
    lq_sum = 0.0;
    for (int r = 0; r < b->count; ++r) {
      lq.push_back(std::llrint(std::ldexp(b->L[r], k)));
      lq_sum += (double)lq.back();
    }
  }
  if (p.search == MT_SEARCH_CELL) {
    const long long n1 = p.n > 0 ? p.n : 1;
    int c = p.cell_shift;
    if (c == 0) {
      if (p.dim == 1) {
        const double per = lq_sum / (double)n1;  // ticks per particle
        c = per >= 2.0 ? floor_log2(per) + 1 : 1;
      } else {
        const int cmin = ceil_log2(D.S + 1);
        const double side = std::sqrt((double)D.Lq[0] * (double)D.Lq[1] / (double)n1);
        const int ct = side >= 2.0 ? floor_log2(side) : 1;
        c = ct > cmin ? ct : cmin;
      }
    }
    if (c < 1 || c > 62) return fail(MT_ERR_INVALID, "cell_shift must be in [1, 62]");
    if (p.dim == 2 && (1LL << c) <= D.S)
      return fail(MT_ERR_INVALID, "2-d cells must be wider than the cutoff (2^cell_shift > Smax)");
    // keep the cell array modest
    for (;;) {
      if (b) {
        // realisations side by side, gaps of more than Smax between them
        const long long w = 1LL << c, gapc = (D.S + w - 1) / w + 1;
        double cells = 0.0;
        for (int r = 0; r < b->count; ++r) cells += (double)((lq[r] >> c) + 1 + gapc);
        cells -= (double)gapc;
        if (std::ldexp(cells, c) >= kTwo61)
          return fail(MT_ERR_INVALID, "batch too long for the grid: lower frac_bits");
        D.ncx = (long long)cells;
        D.Lq[0] = (D.ncx << c) - 1;  // the shared axis
      } else {
        D.ncx = (D.Lq[0] >> c) + 1;
      }
      D.ncy = p.dim == 2 ? (D.Lq[1] >> c) + 1 : 1;
      if ((double)D.ncx * (double)D.ncy <= (double)(1LL << 28)) break;
      ++c;
    }
    D.cshift = c;
    p.cell_shift = c;
    D.ncell = D.ncx * D.ncy;
  } else {
    D.ncell = 0;
    p.cell_shift = 0;
  }
  D.nbig_cap = p.n / (kSmallCell + 1) + 1;
  // Fused 1-d step: segments of seg_target particles staged with a halo of
  // hc cells (2 Smax) and the displacement bound; pick the largest target
  // (<= 1024) whose expected staging, with 50% headroom, fits kFusedCap.
  if (p.search == MT_SEARCH_CELL && p.dim == 1 && p.n > 0 && !periodic && p.species == 2 &&
      p.stored_p == 0) {
    const long long w = 1LL << D.cshift;
    D.hc = (2 * D.S + w - 1) / w + 1;
    double dr = std::fabs((double)D.drift[0]);
    const long long dc = (long long)((dr + std::ceil(D.bq * 5.78) + 2.0) / (double)w) + 2;
    const double per_cell = (double)p.n / (double)D.ncell;
    // right neighbours per particle (mean density x Smax): the first tier
    // lists the pairs of owners within about T + 3 Smax of density
    const double rn = (double)D.S * (double)p.n / lq_sum;
    // As many particles per segment as the staging and the pair list hold
    // with 50 % headroom, at most kSegMax: larger segments spread the
    // segment's fixed cost (barriers, bins, halo) over more particles, and
    // the tickets balance the CTAs (measured at N = 10^6: 412 particles per
    // segment 184 us per step, 600-700 about 167 us, MIXED).
    constexpr double kSegMax = 640.0;
    const double t_stage = (double)kFusedCap - 64.0 - 2.0 * (double)(D.hc + dc + 1) * per_cell * 1.5;
    const double t_pairs = rn > 0.0 ? ((double)kFusedPairCap - 64.0) / (1.5 * rn) - 3.0 * rn : 1e9;
    long long T = (long long)std::floor(std::min(std::min(t_stage, t_pairs), kSegMax));
    if (p.seg_target != 0) {
      if (p.seg_target < 16 || p.seg_target > kFusedCap)
        return fail(MT_ERR_INVALID, "seg_target must be 0 or in [16, %d]", kFusedCap);
      T = p.seg_target;
    } else if (T >= 64) {
      // a system smaller than one wave of such segments: one segment per
      // resident first-tier CTA of the current device, so all SMs work
      const long long slots = (long long)fused_ctas_per_sm(p.precision) * device_sms();
      if (slots > 0 && p.n < T * slots) {
        T = (p.n + slots - 1) / slots;
        if (T < 64) T = 64;
      }
    }
    if (T >= 16 && (T >= 64 || p.seg_target != 0)) {
      D.fused = true;
      D.seg_target = T;
      p.seg_target = (int32_t)T;
    }
  }
  if (!D.fused) p.seg_target = 0;
  // SPaM band: right neighbours kept per particle; the mean count with
  // headroom for the Poisson spread of a uniform density
  if (p.stored_p == 1) {
    const double mean = (double)D.S * (double)p.n / (double)D.Lq[0];
    const double b = std::ceil(1.25 * mean + 4.0 * std::sqrt(mean) + 8.0);
    p.stored_p = (int32_t)std::min(b, 1.0e6);
  }
  if (p.stored_p > 0 && p.stored_p > p.n) p.stored_p = (int32_t)std::max<long long>(p.n, 2);
  D.band = p.stored_p;
  // dense 1-d neighbourhoods (>= kTileMinNeighbours a side on average) walk
  // shared-memory tiles instead of per-particle global-memory walks
  if (p.search == MT_SEARCH_CELL && p.dim == 1 && !periodic && D.band == 0 && p.n > 0)
    D.tile = (double)D.S * (double)p.n / lq_sum >= kTileMinNeighbours;
  // realisation table and fused segments (each realisation's own, so its
  // particles' slot range [off, off + n) is split at off + j T)
  {
    const long long T = D.fused ? D.seg_target : 0;
    long long off = 0, cb = 0;
    const long long w = p.search == MT_SEARCH_CELL ? (1LL << D.cshift) : 1;
    const long long gapc = (D.S + w - 1) / w + 1;
    for (int r = 0; r < D.nreal; ++r) {
      Real R = {};
      R.n = b ? b->n[r] : p.n;
      R.Lq = b ? lq[r] : D.Lq[0];
      R.base = b ? (cb << D.cshift) : 0;
      R.off = off;
      R.real = (unsigned int)(b && b->realisation ? b->realisation[r] : p.realisation + r);
      R.seg0 = (int)D.sslot.size();
      R.nseg = T > 0 ? (int)((R.n + T - 1) / T) : 0;
      for (int j = 0; j < R.nseg; ++j) {
        D.sslot.push_back((int)(off + j * T));
        D.sreal.push_back(r);
      }
      R.ch0 = (int)D.ochunk.size();
      for (long long j = 0; j < R.n; j += kObsChunk) {
        D.ochunk.push_back((int)(off + j));
        D.ochr.push_back(r);
      }
      R.nch = (int)D.ochunk.size() - R.ch0;
      if (b) cb += (lq[r] >> D.cshift) + 1 + gapc;
      off += R.n;
      D.rt.push_back(R);
    }
    D.nseg = (long long)D.sslot.size();
    D.sslot.push_back((int)p.n);
    if (D.sreal.empty()) D.sreal.push_back(0);
    D.ochunk.push_back((int)p.n);
  }
  if (b) p.L[0] = std::ldexp((double)D.Lq[0], -k);
  D.ntiles = (D.ncell + kScanTile - 1) / kScanTile;
  // workspace layout
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes);
    return at;
  };
  const size_t n = (size_t)p.n;
  D.o_ctrl = take(sizeof(Ctrl));
  for (int b2 = 0; b2 < 2; ++b2) D.o_X[b2] = take((size_t)p.dim * n * 8);
  for (int b2 = 0; b2 < 2; ++b2) D.o_id[b2] = take(n * 4);
  for (int b2 = 0; b2 < 2; ++b2) D.o_M[b2] = take((size_t)p.species * n * 8);
  D.o_src = take(n * 4);
  D.o_rinv = take(n * 8);
  D.o_count = take((size_t)D.ncell * 4);
  D.o_start = take((size_t)(D.ncell + 1) * 4);
  D.o_cursor = take((size_t)D.ncell * 4);
  D.o_status = take((size_t)D.ntiles * 8);
  D.o_big = take((size_t)D.nbig_cap * 4);
  D.o_obs = take((size_t)p.observe_cap * D.nreal * 4 * 8);
  for (int b2 = 0; b2 < 2; ++b2) D.o_fstart[b2] = take(D.fused ? (size_t)(D.ncell + 1) * 4 : 0);
  for (int b2 = 0; b2 < 2; ++b2) D.o_cb[b2] = take(D.fused ? (size_t)(D.nseg + 1) * 4 : 0);
  D.o_ovlist = take(D.fused ? (size_t)D.nseg * 4 : 0);
  // binary64 weights of the wall layer's dense rows, kept between the
  // predicted-segment kernel's row sums and its exchange (large systems)
  D.wc_cap = D.fused && p.precision == MT_FP64 && p.n >= kWcMinN ? kWcCap : 0;
  D.o_wc = take((size_t)D.wc_cap * 8);
  for (int b2 = 0; b2 < 2; ++b2) D.o_pred[b2] = take(D.fused ? (size_t)D.nseg : 0);
  D.o_rt = take(D.rt.size() * sizeof(Real));
  D.o_sslot = take(D.sslot.size() * 4);
  D.o_sreal = take(D.sreal.size() * 4);
  D.o_cnt = take(D.band > 0 ? 2 * n * 4 : 0);
  D.o_band = take(D.band > 0 ? (size_t)D.band * ((n + 31) / 32 * 32) *
                                   (p.precision == MT_FP64 ? 8 : 4)
                             : 0);
  D.o_ochunk = take(D.ochunk.size() * 4);
  D.o_opart = take((D.ochunk.size() - 1) * 4 * 8);
  D.o_ochr = take(D.ochr.size() * 4);
  D.o_ocnt = take((size_t)D.nreal * 4);
  D.total = o;
  D.p = p;
  *out = D;
  return MT_OK;
}

}  // namespace

namespace mt {
// Lets other translation units report through mt_last_error().
mt_status set_last_error(mt_status s, const char* msg) {
  g_err = msg;
  return s;
}
}  // namespace mt

struct mt_handle {
  Derived D;
  Dev dev;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // fused path: the predicted-segment kernel runs on a second stream beside
  // the first tier (fork / join events around it in the captured graph)
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  // fires once the predicted-segment kernel's CTAs have all begun: the first
  // tier waits for it in the graph, so that its persistent CTAs, which fill
  // every SM, never take the SMs the cluster needs before the cluster is
  // placed (otherwise the cluster waits for the first tier to drain)
  cudaEvent_t pstart = nullptr;
  // fused path with observables: the previous step's observables run
  // beside the step in the graph (obs_defer), behind the predicted segments
  // where those run, else on this third stream when the first tier is
  // bound by the binary64 pipe (MT_FP64, MT_MIXED; with MT_MIXED_DF32 and
  // no predicted segments they follow the step in its graph); the last
  // step's are pending until a call that reads them (flush_obs).
  bool obs_defer = false;
  cudaStream_t side2 = nullptr;
  cudaEvent_t join2 = nullptr;
  bool obs_pending = false;
  bool uploaded = false;
  long long steps = 0;     // host mirror of the step counter
  const float* noise = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool profile = false;
  cudaEvent_t ev[kMaxMarks + 1] = {};
  const char* ev_names[kMaxMarks] = {};
  int ev_count = 0;  // kernels marked in the last profiled step
};

namespace {

bool capturable(cudaStream_t s) {
  return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}

mt_status read_ctrl(mt_handle* h, Ctrl* c) {
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaMemcpy(c, h->ws + h->D.o_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
  return MT_OK;
}

mt_status check_device(mt_handle* h) {
  Ctrl c;
  const mt_status s = read_ctrl(h, &c);
  if (s != MT_OK) return s;
  if (c.err == kErrTimeout)
    return fail(MT_ERR_TIMEOUT, "device wait gave up (scan tile %lld)", c.err_info);
  if (c.err == kErrInput)
    return fail(MT_ERR_INVALID, "uploaded position %lld outside [0, L] or NaN", c.err_info);
  if (c.err != kErrNone)
    return fail(MT_ERR_DEVICE, "device index check failed (code %d, at %lld)", c.err, c.err_info);
  return MT_OK;
}

// The observables of the last graph step on the fused path, which the next
// step's graph would have computed beside itself: enqueue them now (a call
// is about to read the ring, the state, or to leave the graph).
mt_status flush_obs(mt_handle* h) {
  if (!h->obs_pending) return MT_OK;
  h->obs_pending = false;
  CU(launch_obs(h->dev, h->D.p.precision, h->stream));
  return MT_OK;
}

// The general pipeline: move + histogram, scan, scatter, cell sort, two
// transfer passes; on the 1-d cell path it also refreshes the fused path's
// cell starts and segment boundaries.
mt_status enqueue_general(mt_handle* h, const Dev& d, Marker& mk) {
  const mt_params& p = h->D.p;
  mk("move", h->stream);
  if (p.search == MT_SEARCH_CELL) {
    CU(launch_move(d, true, true, h->stream));
    CU(launch_sort(d, h->stream, mk));
  } else {
    CU(launch_move(d, true, false, h->stream));
  }
  CU(launch_transfer(d, p.search, p.precision, h->stream, mk));
  if (h->D.fused) {
    mk("fused_prep", h->stream);
    CU(launch_fused_prep(d, 1, h->stream));
  }
  return MT_OK;
}

// Enqueue one step's kernels directly (no graph), with an event before each
// kernel and one after the last when profiling is on.  On the fused path the
// host reads whether a segment overflowed and, if so, runs the general
// pipeline for the step.
mt_status enqueue_step(mt_handle* h, const Dev& d) {
  const mt_params& p = h->D.p;
  if (p.n == 0) return MT_OK;
  {
    const mt_status s = flush_obs(h);
    if (s != MT_OK) return s;
  }
  Marker mk;
  if (h->profile) {
    mk.ev = h->ev;
    mk.names = h->ev_names;
  }
  if (h->D.fused) {
    // the step's prediction (segments pair-heavy last step) decides whether
    // the predicted-segment kernel runs; here it runs before the first tier
    // (in the captured graph, beside it)
    Ctrl c;
    mt_status s = MT_OK;
    if (d.use_pred) {
      s = read_ctrl(h, &c);
      if (s != MT_OK) return s;
      if (c.npred > 0) {
        mk("fused_pred", h->stream);
        CU(launch_fused_pred(d, p.precision, 0, 0, h->stream));
      } else {
        mk("join_stub", h->stream);  // (the graph launches the predicted-segment kernel here)
        CU(launch_join_stub(d, h->stream));  // the first tier's partner in the join
      }
    }
    mk("fused_step", h->stream);
    CU(launch_fused_step(d, p.precision, 0, 0, h->stream));
    // a gap mark: the idle time while the host reads the control block is
    // not counted in the kernel before it
    mk(nullptr, h->stream);
    s = read_ctrl(h, &c);
    if (s != MT_OK) return s;
    if (c.nov > 0 || c.overflow) {
      mk("fused_big", h->stream);
      CU(launch_fused_big(d, p.precision, 0, 0, h->stream));
      mk(nullptr, h->stream);
      s = read_ctrl(h, &c);
      if (s != MT_OK) return s;
      if (c.fallback) {
        const mt_status s2 = enqueue_general(h, d, mk);
        if (s2 != MT_OK) return s2;
      }
    }
  } else {
    const mt_status s = enqueue_general(h, d, mk);
    if (s != MT_OK) return s;
  }
  if (p.observe_cap > 0) {
    mk("observables", h->stream);
    CU(launch_obs(d, p.precision, h->stream));
  }
  if (h->profile) {
    CU(Marker::record(h->ev[mk.count], h->stream));
    h->ev_count = mk.count;
  }
  return MT_OK;
}

// Capture one step into an executable graph.  On the fused path the graph
// is [fused step] -> IF(overflow) {general pipeline}.
mt_status build_graph(mt_handle* h) {
  const Dev& d = h->dev;
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  cudaGraph_t g = nullptr;
  CU(cudaGraphCreate(&g, 0));
  mt_status s = MT_OK;
  Marker none;
  if (h->D.fused) {
    // g: { [predicted segments, taking the observables' snapshot] ->
    //   [previous step's observables] | [fast tier] } -> IF(queued)
    //   { [second tier] -> IF(overflow) { general } }
    cudaGraphConditionalHandle cond1, cond2;
    CU(cudaGraphConditionalHandleCreate(&cond1, g, 0, 0));
    // large systems fork: the predicted-segment kernel on the side stream,
    // the first tier on the handle's stream; with observables, the previous
    // step's follow the predicted segments on the side stream (on the SMs
    // those leave while the first tier still runs), or, without the fork,
    // run on a third stream beside the first tier (they read the mass
    // buffer the step only reads); all join before the conditional
    const bool fork = d.use_pred != 0;
    const bool obs = h->obs_defer;
    CU(cudaStreamBeginCaptureToGraph(h->stream, g, nullptr, nullptr, 0, mode));
    cudaError_t e1 = cudaSuccess;
    // the observables' snapshot: by the predicted-segment kernel where it
    // runs (the observables follow it), else a kernel of its own
    if (obs && !fork) e1 = launch_obs_snapshot(d, h->stream);
    if ((fork || obs) && e1 == cudaSuccess) e1 = cudaEventRecord(h->fork, h->stream);
    if (fork) {
      if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(h->side, h->fork, 0);
      Dev dp = d;
      dp.obs_snap = obs ? 1 : 0;
      if (e1 == cudaSuccess)
        e1 = launch_fused_pred(dp, h->D.p.precision, cond1, 1, h->side, h->pstart);
      if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(h->stream, h->pstart, 0);
    }
    if (obs && fork) {  // behind the predicted segments, on their SMs
      if (e1 == cudaSuccess) e1 = launch_obs_prev(d, h->D.p.precision, h->side);
    } else if (obs) {
      if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(h->side2, h->fork, 0);
      if (e1 == cudaSuccess) e1 = launch_obs_prev(d, h->D.p.precision, h->side2);
    }
    if (e1 == cudaSuccess) e1 = launch_fused_step(d, h->D.p.precision, cond1, 1, h->stream);
    if (fork && e1 == cudaSuccess) e1 = cudaEventRecord(h->join, h->side);
    if (fork && e1 == cudaSuccess) e1 = cudaStreamWaitEvent(h->stream, h->join, 0);
    if (obs && !fork && e1 == cudaSuccess) e1 = cudaEventRecord(h->join2, h->side2);
    if (obs && !fork && e1 == cudaSuccess) e1 = cudaStreamWaitEvent(h->stream, h->join2, 0);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(MT_ERR_CUDA, "graph capture of the fused step failed");
    }
    cudaGraph_t body1 = nullptr;
    cudaGraphNode_t cnode = nullptr;  // the IF node
    {
      // the IF node follows every kernel node without a dependent
      const size_t want = 1 + (fork ? 1 : 0) + (obs ? (fork ? 1 : 2) : 0);
      cudaGraphNode_t knodes[4] = {nullptr, nullptr, nullptr, nullptr};
      size_t nn = 4;
      CU(cudaGraphGetNodes(g, knodes, &nn));
      if (nn != want) {
        cudaGraphDestroy(g);
        return fail(MT_ERR_CUDA, "fused step graph: expected %zu kernel nodes, got %zu", want, nn);
      }
      cudaGraphNode_t leaves[4];
      size_t nleaf = 0;
      for (size_t i = 0; i < nn; ++i) {
        size_t ndep = 0;
        CU(cudaGraphNodeGetDependentNodes(knodes[i], nullptr, nullptr, &ndep));
        if (ndep == 0) leaves[nleaf++] = knodes[i];
      }
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond1;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      CU(cudaGraphAddNode(&cnode, g, leaves, nullptr, nleaf, &cp));
      body1 = cp.conditional.phGraph_out[0];
    }
    CU(cudaGraphConditionalHandleCreate(&cond2, body1, 0, 0));
    CU(cudaStreamBeginCaptureToGraph(h->stream, body1, nullptr, nullptr, 0, mode));
    e1 = launch_fused_big(d, h->D.p.precision, cond2, 1, h->stream);
    e2 = cudaStreamEndCapture(h->stream, &body1);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      cudaGraphDestroy(g);
      return fail(MT_ERR_CUDA, "graph capture of the second fused tier failed");
    }
    cudaGraph_t body2 = nullptr;
    {
      cudaGraphNode_t bnode = nullptr;
      size_t nn = 1;
      CU(cudaGraphGetNodes(body1, &bnode, &nn));
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = cond2;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      cudaGraphNode_t cnode = nullptr;
      CU(cudaGraphAddNode(&cnode, body1, &bnode, nullptr, 1, &cp));
      body2 = cp.conditional.phGraph_out[0];
    }
    CU(cudaStreamBeginCaptureToGraph(h->stream, body2, nullptr, nullptr, 0, mode));
    s = enqueue_general(h, d, none);
    const cudaError_t e3 = cudaStreamEndCapture(h->stream, &body2);
    if (s == MT_OK && e3 != cudaSuccess) s = fail(MT_ERR_CUDA, "graph capture of the fallback failed");
    // the step's own observables: the next step's graph (or flush_obs)
    // where they are deferred, else after the IF node
    if (s == MT_OK && !obs && h->D.p.observe_cap > 0) {
      CU(cudaStreamBeginCaptureToGraph(h->stream, g, &cnode, nullptr, 1, mode));
      const cudaError_t e4 = launch_obs(d, h->D.p.precision, h->stream);
      const cudaError_t e5 = cudaStreamEndCapture(h->stream, &g);
      if (e4 != cudaSuccess || e5 != cudaSuccess)
        s = fail(MT_ERR_CUDA, "graph capture of the observables failed");
    }
  } else {
    CU(cudaStreamBeginCaptureToGraph(h->stream, g, nullptr, nullptr, 0, mode));
    s = enqueue_general(h, d, none);
    if (s == MT_OK && launch_obs(d, h->D.p.precision, h->stream) != cudaSuccess)
      s = fail(MT_ERR_CUDA, "observables launch failed");
    const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (s == MT_OK && e != cudaSuccess) s = fail(MT_ERR_CUDA, "graph capture failed");
  }
  if (s != MT_OK) {
    cudaGraphDestroy(g);
    return s;
  }
  const cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return fail(MT_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return MT_OK;
}

}  // namespace

extern "C" {

mt_status mt_params_init(mt_params* p) {
  if (!p) return fail(MT_ERR_INVALID, "params is NULL");
  std::memset(p, 0, sizeof *p);
  p->dim = 1;
  p->L[0] = 1000.0;
  p->L[1] = 1000.0;
  p->D_mt = 0.1;
  p->D_rw = 0.1;
  p->dt = 1.0;
  p->cutoff = 0.0;
  p->search = MT_SEARCH_CELL;
  p->precision = MT_FP64;
  p->norm = MT_NORM_SYM;
  p->react = 1;
  return MT_OK;
}

mt_status mt_resolve(const mt_params* p, mt_params* out) { return mt_batch_resolve(p, nullptr, out); }

mt_status mt_batch_resolve(const mt_params* p, const mt_batch* b, mt_params* out) {
  Derived D;
  const mt_status s = resolve(p, b, &D);
  if (s != MT_OK) return s;
  if (!out) return fail(MT_ERR_INVALID, "out is NULL");
  *out = D.p;
  return MT_OK;
}

mt_status mt_workspace_bytes(const mt_params* p, size_t* bytes) {
  return mt_batch_workspace_bytes(p, nullptr, bytes);
}

mt_status mt_batch_workspace_bytes(const mt_params* p, const mt_batch* b, size_t* bytes) {
  Derived D;
  const mt_status s = resolve(p, b, &D);
  if (s != MT_OK) return s;
  if (!bytes) return fail(MT_ERR_INVALID, "bytes is NULL");
  *bytes = D.total;
  return MT_OK;
}

mt_status mt_create(const mt_params* p, void* workspace, size_t workspace_bytes, void* stream,
                    mt_handle** out) {
  return mt_batch_create(p, nullptr, workspace, workspace_bytes, stream, out);
}

mt_status mt_batch_create(const mt_params* p, const mt_batch* b, void* workspace,
                          size_t workspace_bytes, void* stream, mt_handle** out) {
  if (!out) return fail(MT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  Derived D;
  mt_status s = resolve(p, b, &D);
  if (s != MT_OK) return s;
  if (!workspace) return fail(MT_ERR_WORKSPACE, "workspace is NULL");
  if ((uintptr_t)workspace % kAlign != 0)
    return fail(MT_ERR_WORKSPACE, "workspace must be %zu-byte aligned", kAlign);
  if (workspace_bytes < D.total)
    return fail(MT_ERR_WORKSPACE, "workspace has %zu bytes, needs %zu", workspace_bytes, D.total);
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, workspace) != cudaSuccess ||
      attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(MT_ERR_WORKSPACE, "workspace is not device memory");
  }
  mt_handle* h = new mt_handle();
  h->D = D;
  h->ws = static_cast<char*>(workspace);
  if (stream) {
    h->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return fail(MT_ERR_CUDA, "cudaStreamCreateWithFlags failed");
    }
    h->own_stream = true;
  }
  Dev& d = h->dev;
  std::memset(&d, 0, sizeof d);
  char* w = h->ws;
  d.ctrl = reinterpret_cast<Ctrl*>(w + D.o_ctrl);
  for (int b = 0; b < 2; ++b) {
    d.X[b] = reinterpret_cast<long long*>(w + D.o_X[b]);
    d.id[b] = reinterpret_cast<int*>(w + D.o_id[b]);
    d.M[b] = reinterpret_cast<unsigned long long*>(w + D.o_M[b]);
  }
  d.src = reinterpret_cast<int*>(w + D.o_src);
  d.rinv = w + D.o_rinv;
  d.count = reinterpret_cast<int*>(w + D.o_count);
  d.start = reinterpret_cast<int*>(w + D.o_start);
  d.cursor = reinterpret_cast<int*>(w + D.o_cursor);
  d.scan_status = reinterpret_cast<unsigned long long*>(w + D.o_status);
  d.big = reinterpret_cast<int*>(w + D.o_big);
  d.obs = reinterpret_cast<double*>(w + D.o_obs);
  for (int b = 0; b < 2; ++b) {
    d.fstart[b] = reinterpret_cast<int*>(w + D.o_fstart[b]);
    d.cb[b] = reinterpret_cast<int*>(w + D.o_cb[b]);
  }
  d.ovlist = reinterpret_cast<int*>(w + D.o_ovlist);
  for (int b = 0; b < 2; ++b) d.pred[b] = reinterpret_cast<unsigned char*>(w + D.o_pred[b]);
  d.nseg = (int)D.nseg;
  d.seg_target = (int)D.seg_target;
  d.hc = D.hc;
  {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 1;
    d.nsm = nsm;
  }
  // the predicted-segment kernel pays off when the first tier has more than
  // one wave of segments (large systems); small ones keep the plain chain
  d.use_pred =
      D.fused && D.nseg > (long long)fused_ctas_per_sm(D.p.precision) * d.nsm ? 1 : 0;
  d.periodic = D.p.walls == MT_WALLS_PERIODIC ? 1 : 0;
  d.nspec = D.p.species;
  d.band_cap = (int)D.band;
  d.tile = D.tile ? 1 : 0;
  d.cnt = reinterpret_cast<int*>(w + D.o_cnt);
  d.band = w + D.o_band;
  d.n = D.p.n;
  d.dim = D.p.dim;
  d.norm = D.p.norm;
  d.react = D.p.react;
  d.observe_cap = D.p.observe_cap;
  d.cshift = D.cshift;
  d.ncx = D.ncx;
  d.ncy = D.ncy;
  d.ncell = D.ncell;
  d.S = D.S;
  for (int a = 0; a < 2; ++a) {
    d.Lq[a] = D.Lq[a];
    d.drift[a] = D.drift[a];
  }
  d.bq = D.bq;
  d.inv8 = 1.0 / (8.0 * D.p.D_mt * D.p.dt);
  d.scale = std::ldexp(1.0, -D.p.frac_bits);
  d.inv8f = (float)(d.inv8 * d.scale * d.scale);
  d.inv8s = std::ldexp(d.inv8, -2 * D.p.frac_bits);
  d.key0 = (unsigned int)(D.p.seed & 0xffffffffu);
  d.key1 = (unsigned int)(D.p.seed >> 32);
  d.real = (unsigned int)D.p.realisation;
  d.nbig_cap = (int)D.nbig_cap;
  d.wc = reinterpret_cast<double*>(w + D.o_wc);
  d.wc_cap = D.wc_cap;
  d.rt = reinterpret_cast<const Real*>(w + D.o_rt);
  d.nreal = D.nreal;
  d.lbits = D.lbits;
  d.lmask = (int)((1LL << D.lbits) - 1);
  d.sslot = reinterpret_cast<const int*>(w + D.o_sslot);
  d.sreal = reinterpret_cast<const int*>(w + D.o_sreal);
  d.ochunk = reinterpret_cast<int*>(w + D.o_ochunk);
  d.nochunk = (int)D.ochunk.size() - 1;
  d.opart = reinterpret_cast<unsigned long long*>(w + D.o_opart);
  d.ochr = reinterpret_cast<int*>(w + D.o_ochr);
  d.ocnt = reinterpret_cast<int*>(w + D.o_ocnt);
  const Derived& hd = h->D;  // the tables live as long as the handle
  cudaError_t e = D.fused ? fused_configure() : cudaSuccess;
  if (e == cudaSuccess && d.use_pred) {
    e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->pstart, cudaEventDisableTiming);
  }
  h->obs_defer = D.fused && D.p.observe_cap > 0 && d.nochunk > 0 &&
                 (d.use_pred || D.p.precision != MT_MIXED_DF32);
  if (e == cudaSuccess && h->obs_defer && !d.use_pred) {
    e = cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->join2, cudaEventDisableTiming);
  }
  if (e == cudaSuccess && (h->side || h->side2))
    e = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws, 0, D.total, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + D.o_rt, hd.rt.data(), hd.rt.size() * sizeof(Real),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + D.o_sslot, hd.sslot.data(), hd.sslot.size() * 4,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + D.o_sreal, hd.sreal.data(), hd.sreal.size() * 4,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(w + D.o_ochunk, hd.ochunk.data(), hd.ochunk.size() * 4,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && !hd.ochr.empty())
    e = cudaMemcpyAsync(w + D.o_ochr, hd.ochr.data(), hd.ochr.size() * 4, cudaMemcpyHostToDevice,
                        h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    if (h->side) cudaStreamDestroy(h->side);
    if (h->side2) cudaStreamDestroy(h->side2);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->join) cudaEventDestroy(h->join);
    if (h->join2) cudaEventDestroy(h->join2);
    if (h->pstart) cudaEventDestroy(h->pstart);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return fail(MT_ERR_CUDA, "handle setup: %s", cudaGetErrorString(e));
  }
  *out = h;
  return MT_OK;
}

mt_status mt_upload(mt_handle* h, const double* x, const double* A, const double* B,
                    int32_t mem) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (mem != MT_MEM_HOST && mem != MT_MEM_DEVICE) return fail(MT_ERR_INVALID, "bad mem kind");
  const mt_params& p = h->D.p;
  const size_t n = (size_t)p.n;
  if (n > 0 && (!x || !A || !B)) return fail(MT_ERR_INVALID, "x, A and B are required");
  CU(cudaMemsetAsync(h->ws + h->D.o_ctrl, 0, sizeof(Ctrl), h->stream));
  CU(cudaMemsetAsync(h->ws + h->D.o_ocnt, 0, (size_t)h->D.nreal * 4, h->stream));
  if (h->D.fused)
    for (int b = 0; b < 2; ++b) CU(cudaMemsetAsync(h->ws + h->D.o_pred[b], 0, h->D.nseg, h->stream));
  // the scan epoch restarts with the control block: clear old status words
  if (h->D.ntiles > 0) CU(cudaMemsetAsync(h->ws + h->D.o_status, 0, h->D.ntiles * 8, h->stream));
  h->steps = 0;
  h->uploaded = true;
  h->obs_pending = false;
  if (n == 0) return MT_OK;
  const Dev& d = h->dev;
  // the control block was cleared: restore the noise source and its bound
  CU(cudaMemcpyAsync(&d.ctrl->noise, &h->noise, sizeof(h->noise), cudaMemcpyHostToDevice,
                     h->stream));
  CU(launch_noise_bound(d, h->noise, h->stream));
  double* xs = reinterpret_cast<double*>(d.X[1]);
  double* ms = reinterpret_cast<double*>(d.M[1]);
  const cudaMemcpyKind kind = mem == MT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CU(cudaMemcpyAsync(xs, x, (size_t)p.dim * n * 8, kind, h->stream));
  CU(cudaMemcpyAsync(ms, A, n * 8, kind, h->stream));
  CU(cudaMemcpyAsync(ms + n, B, n * 8, kind, h->stream));
  CU(launch_upload(d, xs, ms, ms + n, p.precision, h->stream));
  if (p.search == MT_SEARCH_CELL) {
    // sort once so the state is in cell order between steps
    Marker none;
    CU(launch_move(d, false, true, h->stream));
    CU(launch_sort(d, h->stream, none));
    CU(launch_permute(d, h->stream));
    if (h->D.fused) CU(launch_fused_prep(d, 0, h->stream));
  }
  if (mem == MT_MEM_HOST) CU(cudaStreamSynchronize(h->stream));
  return MT_OK;
}

mt_status mt_set_noise(mt_handle* h, const float* xi) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  h->noise = xi;
  if (!h->uploaded) return MT_OK;  // mt_upload installs it
  CU(cudaMemcpyAsync(&h->dev.ctrl->noise, &h->noise, sizeof(h->noise), cudaMemcpyHostToDevice,
                     h->stream));
  CU(launch_noise_bound(h->dev, xi, h->stream));
  return MT_OK;
}

mt_status mt_test_hold_scan(mt_handle* h, int32_t hold, int64_t spin_limit) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "mt_test_hold_scan before mt_upload");
  if ((hold != 0 && hold != 1) || spin_limit < 0)
    return fail(MT_ERR_INVALID, "hold must be 0 or 1 and spin_limit >= 0");
  const int hv = hold;
  const long long lv = spin_limit;
  CU(cudaMemcpyAsync(&h->dev.ctrl->scan_hold, &hv, sizeof(hv), cudaMemcpyHostToDevice, h->stream));
  CU(cudaMemcpyAsync(&h->dev.ctrl->spin_limit, &lv, sizeof(lv), cudaMemcpyHostToDevice,
                     h->stream));
  CU(cudaStreamSynchronize(h->stream));  // the sources live on this stack frame
  return MT_OK;
}

mt_status mt_run(mt_handle* h, int64_t nsteps) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "mt_run before mt_upload");
  if (nsteps < 0) return fail(MT_ERR_INVALID, "nsteps must be >= 0");
  if (h->profile || !capturable(h->stream) || h->D.p.n == 0) {
    for (int64_t i = 0; i < nsteps; ++i) {
      const mt_status s = enqueue_step(h, h->dev);
      if (s != MT_OK) return s;
      ++h->steps;
    }
    return MT_OK;
  }
  if (!h->graph) {
    const mt_status s = build_graph(h);
    if (s != MT_OK) return s;
  }
  for (int64_t i = 0; i < nsteps; ++i) {
    CU(cudaGraphLaunch(h->graph, h->stream));
    ++h->steps;
  }
  if (nsteps > 0 && h->obs_defer) h->obs_pending = true;
  return MT_OK;
}

mt_status mt_step(mt_handle* h) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "mt_step before mt_upload");
  return mt_run(h, 1);
}

mt_status mt_sync(mt_handle* h) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  const mt_status s = flush_obs(h);
  if (s != MT_OK) return s;
  return check_device(h);
}

mt_status mt_read_masses(mt_handle* h, double* A, double* B, int32_t mem) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "no state uploaded");
  if (mem != MT_MEM_HOST && mem != MT_MEM_DEVICE) return fail(MT_ERR_INVALID, "bad mem kind");
  const size_t n = (size_t)h->D.p.n;
  if (n == 0) return check_device(h);
  if (!A || !B) return fail(MT_ERR_INVALID, "A and B are required");
  if (mem == MT_MEM_DEVICE) {
    CU(launch_read_masses(h->dev, A, B, h->D.p.precision, h->stream));
  } else {
    Ctrl c;
    const mt_status s = read_ctrl(h, &c);
    if (s != MT_OK) return s;
    double* stage = reinterpret_cast<double*>(h->dev.M[c.mcur ^ 1]);
    CU(launch_read_masses(h->dev, stage, stage + n, h->D.p.precision, h->stream));
    CU(cudaMemcpyAsync(A, stage, n * 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(B, stage + n, n * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  return check_device(h);
}

static mt_status species_io(mt_handle* h, int32_t sp, double* out, const double* in,
                            int32_t mem) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "no state uploaded");
  if (mem != MT_MEM_HOST && mem != MT_MEM_DEVICE) return fail(MT_ERR_INVALID, "bad mem kind");
  if (sp < 0 || sp >= h->D.p.species)
    return fail(MT_ERR_INVALID, "species %d out of range [0, %d)", sp, h->D.p.species);
  const size_t n = (size_t)h->D.p.n;
  if (n == 0) return check_device(h);
  if (!out && !in) return fail(MT_ERR_INVALID, "species array is NULL");
  if (mem == MT_MEM_DEVICE) {
    CU(launch_species_io(h->dev, sp, out, in, h->D.p.precision, h->stream));
    return MT_OK;
  }
  Ctrl c;
  const mt_status s = read_ctrl(h, &c);
  if (s != MT_OK) return s;
  double* stage = reinterpret_cast<double*>(h->dev.M[c.mcur ^ 1]);
  if (in) {
    CU(cudaMemcpyAsync(stage, in, n * 8, cudaMemcpyHostToDevice, h->stream));
    CU(launch_species_io(h->dev, sp, nullptr, stage, h->D.p.precision, h->stream));
  } else {
    CU(launch_species_io(h->dev, sp, stage, nullptr, h->D.p.precision, h->stream));
    CU(cudaMemcpyAsync(out, stage, n * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  return check_device(h);
}

mt_status mt_set_species(mt_handle* h, int32_t s, const double* M, int32_t mem) {
  return species_io(h, s, nullptr, M, mem);
}

mt_status mt_read_species(mt_handle* h, int32_t s, double* M, int32_t mem) {
  return species_io(h, s, M, nullptr, mem);
}

static mt_status read_pos(mt_handle* h, double* x, long long* X, int32_t mem) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "no state uploaded");
  if (mem != MT_MEM_HOST && mem != MT_MEM_DEVICE) return fail(MT_ERR_INVALID, "bad mem kind");
  const size_t n = (size_t)h->D.p.n, m = (size_t)h->D.p.dim * n;
  if (n == 0) return check_device(h);
  if (!x && !X) return fail(MT_ERR_INVALID, "output is NULL");
  if (mem == MT_MEM_DEVICE) {
    CU(launch_read_positions(h->dev, x, X, h->stream));
  } else {
    Ctrl c;
    const mt_status s = read_ctrl(h, &c);
    if (s != MT_OK) return s;
    void* stage = h->dev.X[c.xcur ^ 1];
    CU(launch_read_positions(h->dev, x ? static_cast<double*>(stage) : nullptr,
                             X ? static_cast<long long*>(stage) : nullptr, h->stream));
    CU(cudaMemcpyAsync(x ? static_cast<void*>(x) : static_cast<void*>(X), stage, m * 8,
                       cudaMemcpyDeviceToHost, h->stream));
  }
  return check_device(h);
}

mt_status mt_read_positions(mt_handle* h, double* x, int32_t mem) {
  return read_pos(h, x, nullptr, mem);
}

mt_status mt_read_ticks(mt_handle* h, int64_t* X, int32_t mem) {
  return read_pos(h, nullptr, reinterpret_cast<long long*>(X), mem);
}

mt_status mt_read_observables(mt_handle* h, double* out, int64_t cap, int64_t* count) {
  if (!h || !count) return fail(MT_ERR_INVALID, "handle or count is NULL");
  {
    const mt_status fs = flush_obs(h);
    if (fs != MT_OK) return fs;
  }
  const long long ocap = h->D.p.observe_cap;
  long long have = h->steps < ocap ? h->steps : ocap;
  if (cap < have) have = cap < 0 ? 0 : cap;
  *count = 0;
  const mt_status s = check_device(h);
  if (s != MT_OK) return s;
  if (have == 0) return MT_OK;
  if (!out) return fail(MT_ERR_INVALID, "out is NULL");
  const size_t width = (size_t)h->D.nreal * 4;  // doubles per row
  std::vector<double> ring((size_t)ocap * width);
  const cudaError_t e =
      cudaMemcpy(ring.data(), h->dev.obs, ring.size() * 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(MT_ERR_CUDA, "reading observables: %s", cudaGetErrorString(e));
  const long long first = h->steps - have;  // step index of the oldest row returned
  for (long long i = 0; i < have; ++i) {
    const long long row = (first + i) % ocap;
    std::memcpy(out + width * i, ring.data() + width * row, width * 8);
  }
  *count = have;
  return MT_OK;
}

mt_status mt_copy_observables_async(mt_handle* h, double* out, int64_t rows) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  {
    const mt_status fs = flush_obs(h);
    if (fs != MT_OK) return fs;
  }
  const long long ocap = h->D.p.observe_cap;
  const long long have = h->steps < ocap ? h->steps : ocap;
  if (rows < 1 || rows > have)
    return fail(MT_ERR_INVALID, "rows must be in [1, %lld] (steps enqueued, observe_cap)", have);
  if (!out) return fail(MT_ERR_INVALID, "out is NULL");
  const size_t width = (size_t)h->D.nreal * 4;  // doubles per row
  const long long r0 = (h->steps - rows) % ocap;  // ring row of the oldest step copied
  const long long n1 = r0 + rows <= ocap ? rows : ocap - r0;
  CU(cudaMemcpyAsync(out, h->dev.obs + width * r0, width * 8 * n1, cudaMemcpyDefault, h->stream));
  if (n1 < rows)
    CU(cudaMemcpyAsync(out + width * n1, h->dev.obs, width * 8 * (rows - n1), cudaMemcpyDefault,
                       h->stream));
  return MT_OK;
}

mt_status mt_copy_observables_row_async(mt_handle* h, double* out, int64_t step) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  const long long ocap = h->D.p.observe_cap;
  if (ocap <= 0 || step < 1 || step > h->steps || step <= h->steps - ocap)
    return fail(MT_ERR_INVALID, "step must be in [max(1, %lld), %lld] (steps enqueued, observe_cap)",
                h->steps - ocap + 1, h->steps);
  if (!out) return fail(MT_ERR_INVALID, "out is NULL");
  // the last step's row is still to be computed where the observables run
  // beside the next step: enqueue it now; earlier rows are already behind
  // the steps enqueued
  if (step == h->steps) {
    const mt_status fs = flush_obs(h);
    if (fs != MT_OK) return fs;
  }
  const size_t width = (size_t)h->D.nreal * 4;
  const long long r = (step - 1) % ocap;
  CU(cudaMemcpyAsync(out, h->dev.obs + width * r, width * 8, cudaMemcpyDefault, h->stream));
  return MT_OK;
}

mt_status mt_read_pairs(mt_handle* h, int32_t* pi, int32_t* pj, int64_t cap, int64_t* count) {
  if (!h || !count) return fail(MT_ERR_INVALID, "handle or count is NULL");
  if (!h->uploaded) return fail(MT_ERR_STATE, "no state uploaded");
  if (h->D.p.search == MT_SEARCH_FULL)
    return fail(MT_ERR_INVALID, "no cutoff pair set for MT_SEARCH_FULL");
  if (cap < 0 || (cap > 0 && (!pi || !pj))) return fail(MT_ERR_INVALID, "bad pair buffers");
  CU(launch_pairs(h->dev, h->D.p.search, pi, pj, cap, h->stream));
  const mt_status s = check_device(h);
  if (s != MT_OK) return s;
  unsigned long long np = 0;
  CU(cudaMemcpy(&np, &h->dev.ctrl->npairs, 8, cudaMemcpyDeviceToHost));
  *count = (int64_t)np;
  return MT_OK;
}

mt_status mt_steps_done(const mt_handle* h, int64_t* steps) {
  if (!h || !steps) return fail(MT_ERR_INVALID, "handle or steps is NULL");
  *steps = h->steps;
  return MT_OK;
}

mt_status mt_philox(mt_handle* h, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                    uint32_t k1, int64_t n, uint32_t* out) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  if (n < 0 || (n > 0 && !out)) return fail(MT_ERR_INVALID, "bad output");
  CU(launch_philox(make_uint4(c0, c1, c2, c3), k0, k1, n, out, h->stream));
  return MT_OK;
}

mt_status mt_walk_normals(const mt_params* p, const int64_t* gid, int64_t n, uint64_t step,
                          float* out, void* stream) {
  if (!p) return fail(MT_ERR_INVALID, "params is NULL");
  if (p->dim != 1 && p->dim != 2) return fail(MT_ERR_INVALID, "dim must be 1 or 2");
  if (n < 0 || (n > 0 && (!gid || !out))) return fail(MT_ERR_INVALID, "bad arrays");
  CU(launch_walk_normals(reinterpret_cast<const long long*>(gid), n, step,
                         (unsigned int)p->realisation, (unsigned int)(p->seed & 0xffffffffu),
                         (unsigned int)(p->seed >> 32), p->dim, out,
                         static_cast<cudaStream_t>(stream)));
  return MT_OK;
}

mt_status mt_set_profiling(mt_handle* h, int32_t on) {
  if (!h) return fail(MT_ERR_INVALID, "handle is NULL");
  const bool want = on != 0;
  if (want == h->profile) return MT_OK;
  if (want && !h->ev[0]) {
    for (int i = 0; i <= kMaxMarks; ++i) CU(cudaEventCreate(&h->ev[i]));
  }
  h->profile = want;
  h->ev_count = 0;
  if (h->graph) {  // the captured graph must (not) contain the event records
    CU(cudaStreamSynchronize(h->stream));
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  return MT_OK;
}

mt_status mt_read_profile(mt_handle* h, float* ms, int32_t cap, int32_t* count) {
  if (!h || !count) return fail(MT_ERR_INVALID, "handle or count is NULL");
  *count = 0;
  if (!h->profile || h->ev_count == 0) return MT_OK;
  CU(cudaEventSynchronize(h->ev[h->ev_count]));
  int k = 0;  // marks with a null name are gaps, not kernels
  for (int i = 0; i < h->ev_count; ++i) {
    if (!h->ev_names[i]) continue;
    if (k < cap) {
      if (!ms) return fail(MT_ERR_INVALID, "ms is NULL");
      CU(cudaEventElapsedTime(&ms[k], h->ev[i], h->ev[i + 1]));
    }
    ++k;
  }
  *count = k;
  return MT_OK;
}

const char* mt_profile_name(const mt_handle* h, int32_t idx) {
  if (!h || idx < 0) return "";
  int k = 0;
  for (int i = 0; i < h->ev_count; ++i) {
    if (!h->ev_names[i]) continue;
    if (k++ == idx) return h->ev_names[i];
  }
  return "";
}

// ------------------------------------------------------------ checkpoint --
// File: kCkptMagic, format version, sizeof(mt_params), the resolved
// parameters, the host step count, the realisation table's size and bytes,
// the workspace's size and bytes (little-endian, as on both host
// architectures).  The workspace holds the whole device state (positions,
// ids, masses, cell starts, segment tables, the step counter, the
// observables ring and the tiers' scheduling flags), so a handle that takes
// it back continues exactly as the saved one would have.  The only pointer
// in it, the noise source, is replaced by the loading handle's own.

namespace {
constexpr char kCkptMagic[8] = {'M', 'T', 'C', 'K', 'P', 'T', '0', '1'};
constexpr uint32_t kCkptVersion = 1;

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t params_bytes;
  mt_params p;
  int64_t steps;
  uint64_t rt_bytes;
  uint64_t ws_bytes;
};

bool same_params(const mt_params& a, const mt_params& b) {
  return std::memcmp(&a, &b, sizeof(mt_params)) == 0;
}

mt_status read_header(FILE* f, CkptHeader* hd) {
  if (std::fread(hd, sizeof(CkptHeader), 1, f) != 1)
    return fail(MT_ERR_INVALID, "checkpoint: short header");
  if (std::memcmp(hd->magic, kCkptMagic, sizeof kCkptMagic) != 0)
    return fail(MT_ERR_INVALID, "checkpoint: not a checkpoint file");
  if (hd->version != kCkptVersion || hd->params_bytes != sizeof(mt_params))
    return fail(MT_ERR_INVALID, "checkpoint: format version %u not supported", hd->version);
  return MT_OK;
}
}  // namespace

mt_status mt_save(mt_handle* h, const char* path) {
  if (!h || !path) return fail(MT_ERR_INVALID, "mt_save: NULL argument");
  {
    const mt_status fs = flush_obs(h);
    if (fs != MT_OK) return fs;
  }
  if (!h->uploaded) return fail(MT_ERR_STATE, "mt_save before mt_upload");
  mt_status s = check_device(h);  // waits for the stream
  if (s != MT_OK) return s;
  if (h->side) CU(cudaStreamSynchronize(h->side));
  if (h->side2) CU(cudaStreamSynchronize(h->side2));
  std::vector<char> ws(h->D.total);
  if (!ws.empty()) CU(cudaMemcpy(ws.data(), h->ws, ws.size(), cudaMemcpyDeviceToHost));
  CkptHeader hd;
  std::memset(&hd, 0, sizeof hd);
  std::memcpy(hd.magic, kCkptMagic, sizeof kCkptMagic);
  hd.version = kCkptVersion;
  hd.params_bytes = sizeof(mt_params);
  hd.p = h->D.p;
  hd.steps = h->steps;
  hd.rt_bytes = h->D.rt.size() * sizeof(Real);
  hd.ws_bytes = ws.size();
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(MT_ERR_INVALID, "mt_save: cannot open %s", path);
  bool ok = std::fwrite(&hd, sizeof hd, 1, f) == 1;
  if (ok && hd.rt_bytes) ok = std::fwrite(h->D.rt.data(), hd.rt_bytes, 1, f) == 1;
  if (ok && hd.ws_bytes) ok = std::fwrite(ws.data(), hd.ws_bytes, 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(MT_ERR_INVALID, "mt_save: write to %s failed", path);
  return MT_OK;
}

mt_status mt_checkpoint_params(const char* path, mt_params* p) {
  if (!path || !p) return fail(MT_ERR_INVALID, "mt_checkpoint_params: NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MT_ERR_INVALID, "checkpoint: cannot open %s", path);
  CkptHeader hd;
  const mt_status s = read_header(f, &hd);
  std::fclose(f);
  if (s != MT_OK) return s;
  *p = hd.p;
  return MT_OK;
}

mt_status mt_load(mt_handle* h, const char* path) {
  if (!h || !path) return fail(MT_ERR_INVALID, "mt_load: NULL argument");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MT_ERR_INVALID, "checkpoint: cannot open %s", path);
  CkptHeader hd;
  mt_status s = read_header(f, &hd);
  std::vector<char> rt, ws;
  if (s == MT_OK) {
    if (!same_params(hd.p, h->D.p) || hd.ws_bytes != h->D.total ||
        hd.rt_bytes != h->D.rt.size() * sizeof(Real))
      s = fail(MT_ERR_INVALID, "mt_load: the checkpoint was saved by a handle with other parameters");
  }
  if (s == MT_OK) {
    rt.resize(hd.rt_bytes);
    ws.resize(hd.ws_bytes);
    if ((hd.rt_bytes && std::fread(rt.data(), hd.rt_bytes, 1, f) != 1) ||
        (hd.ws_bytes && std::fread(ws.data(), hd.ws_bytes, 1, f) != 1))
      s = fail(MT_ERR_INVALID, "mt_load: truncated checkpoint");
    else if (hd.rt_bytes && std::memcmp(rt.data(), h->D.rt.data(), hd.rt_bytes) != 0)
      s = fail(MT_ERR_INVALID, "mt_load: the checkpoint holds other realisations");
  }
  std::fclose(f);
  if (s != MT_OK) return s;
  CU(cudaStreamSynchronize(h->stream));
  if (h->side) CU(cudaStreamSynchronize(h->side));
  if (h->side2) CU(cudaStreamSynchronize(h->side2));
  if (!ws.empty()) CU(cudaMemcpy(h->ws, ws.data(), ws.size(), cudaMemcpyHostToDevice));
  h->steps = hd.steps;
  h->obs_pending = false;  // the saved state's rows were written before it was saved
  h->uploaded = true;
  // the saved noise pointer belongs to the saving process: use this handle's
  CU(cudaMemcpyAsync(&h->dev.ctrl->noise, &h->noise, sizeof(h->noise), cudaMemcpyHostToDevice,
                     h->stream));
  if (h->D.p.n > 0) CU(launch_noise_bound(h->dev, h->noise, h->stream));
  return check_device(h);
}

const char* mt_last_error(void) { return g_err.c_str(); }

void mt_destroy(mt_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (int i = 0; i <= kMaxMarks; ++i)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  if (h->side) {
    cudaStreamSynchronize(h->side);
    cudaStreamDestroy(h->side);
  }
  if (h->side2) {
    cudaStreamSynchronize(h->side2);
    cudaStreamDestroy(h->side2);
  }
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->join) cudaEventDestroy(h->join);
  if (h->join2) cudaEventDestroy(h->join2);
  if (h->pstart) cudaEventDestroy(h->pstart);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
