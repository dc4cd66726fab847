// mt_move_sort.cu -- the random-walk move (Eq. 2, Sec. 3 walls) and the
// cell-list build: a counting sort of particles by cell key (histogram,
// single-pass look-back scan, atomic scatter, then a sort inside each cell
// that makes the order unique).  The uniform grid replaces the paper's
// KD-tree fixed-radius search (Sec. 2.1).
#include "mt_internal.cuh"

namespace mt {

// ------------------------------------------------------------------ move --
// Moves every particle once (unless !MOVE) and histograms its cell key
// (if HIST).  Thread 0 also resets the per-step counters of the sort.
template <int DIM, bool MOVE, bool HIST>
__global__ void __launch_bounds__(kThreads) k_move(Dev d) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  Ctrl* c = d.ctrl;
  if (p == 0) {
    c->tile_ctr = 0;
    c->nbig = 0;
    c->epoch += 1;
  }
  if (p >= d.n) return;
  const int xc = c->xcur;
  long long* X = d.X[xc];
  long long pos[2] = {X[p], DIM == 2 ? X[d.n + p] : 0};
  if (MOVE) {
    const int id = d.id[xc][p];
    // realisation of the particle (always 0 in 2-d, where base = 0)
    const Real* R = d.rt + (id >> d.lbits);
    const int loc = id & d.lmask;
    const long long base = R->base;
    float z[2];
    const float* noise = c->noise;
    if (noise) {
      z[0] = noise[R->off + loc];
      if (DIM == 2) z[1] = noise[d.n + loc];
    } else {
      const unsigned long long st = c->step;
      const uint4 u = philox4x32_10(
          make_uint4((unsigned int)loc, (unsigned int)st, (unsigned int)(st >> 32), R->real),
          d.key0, d.key1);
      const float2 g = box_muller(u.x, u.y);
      z[0] = g.x;
      z[1] = g.y;
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      // Eq. 2 on the grid: drift + rint(b * xi), then the wall mirror.
      const long long step = walk_ticks(d.bq, z[a]);
      if (d.periodic && a == 0)
        pos[0] = base + wrap(pos[0] - base + d.drift[0] + step, R->Lq);
      else if (d.periodic)
        pos[a] = wrap(pos[a] + d.drift[a] + step, d.Lq[a]);
      else if (a == 0)
        pos[0] = base + reflect(pos[0] - base + d.drift[0] + step, R->Lq);
      else
        pos[a] = reflect(pos[a] + d.drift[a] + step, d.Lq[a]);
      X[(long long)a * d.n + p] = pos[a];
    }
  }
  if (HIST) atomicAdd(&d.count[cell_of(d, pos[0], pos[1])], 1);
}

// ------------------------------------------------------------------ scan --
// Exclusive scan of count[] into start[] and cursor[] (and count[] := 0),
// one pass with decoupled look-back.  Tiles are handed out in launch order
// by a ticket, so a tile only waits on tiles already running; the wait is
// bounded anyway and raises kErrTimeout instead of hanging.
// Status word: [63:48] epoch tag, [47:46] flag (1 aggregate, 2 prefix),
// [45:0] value.
__device__ __forceinline__ unsigned long long pack(unsigned long long tag, unsigned long long flag,
                                                   long long v) {
  return (tag << 48) | (flag << 46) | ((unsigned long long)v & ((1ULL << 46) - 1));
}

__global__ void __launch_bounds__(kThreads) k_scan(Dev d) {
  __shared__ int s_tile;
  __shared__ long long s_warp[kThreads / 32];
  __shared__ long long s_excl;
  Ctrl* c = d.ctrl;
  if (threadIdx.x == 0) s_tile = (int)atomicAdd(&c->tile_ctr, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const long long base = tile * kScanTile + (long long)threadIdx.x * kScanItems;
  int v[kScanItems];
  long long mine = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long k = base + i;
    v[i] = k < d.ncell ? d.count[k] : 0;
    mine += v[i];
  }
  // block-wide exclusive scan of the per-thread sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long inc = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    long long w = lane < kThreads / 32 ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < kThreads / 32) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const long long block_total = s_warp[kThreads / 32 - 1];
  const long long thread_excl = inc - mine + (warp > 0 ? s_warp[warp - 1] : 0);
  if (threadIdx.x == 0) {
    const unsigned long long tag = (c->epoch % 65535ULL) + 1ULL;
    volatile unsigned long long* st = d.scan_status;
    long long excl = 0;
    if (tile == 0) {
      // (the test hook withholds this word: every later tile's wait then
      // runs out and raises kErrTimeout)
      if (!c->scan_hold) atomicExch(&d.scan_status[0], pack(tag, 2, block_total));
    } else {
      atomicExch(&d.scan_status[tile], pack(tag, 1, block_total));
      const long long limit = c->spin_limit > 0 ? c->spin_limit : kSpinLimit;
      long long t = tile - 1, spins = 0;
      while (t >= 0) {
        const unsigned long long w = st[t];
        const unsigned long long flag = (w >> 46) & 3ULL;
        if ((w >> 48) != tag || flag == 0) {
          if (++spins > limit) {
            raise_error(c, kErrTimeout, tile);
            break;
          }
          continue;
        }
        excl += (long long)(w & ((1ULL << 46) - 1));
        if (flag == 2) break;
        --t;
      }
      atomicExch(&d.scan_status[tile], pack(tag, 2, excl + block_total));
    }
    s_excl = excl;
  }
  __syncthreads();
  long long run = s_excl + thread_excl;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const long long k = base + i;
    if (k < d.ncell) {
      d.start[k] = (int)run;
      d.cursor[k] = (int)run;
      d.count[k] = 0;
      run += v[i];
      if (k == d.ncell - 1) d.start[d.ncell] = (int)run;
    }
  }
}

// --------------------------------------------------------------- scatter --
template <int DIM>
__global__ void __launch_bounds__(kThreads) k_scatter(Dev d) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur;
  const long long* X = d.X[xc];
  long long* Y = d.X[xc ^ 1];
  const long long x = X[p], y = DIM == 2 ? X[d.n + p] : 0;
  const long long slot = atomicAdd(&d.cursor[cell_of(d, x, y)], 1);
  if (slot < 0 || slot >= d.n) {
    raise_error(d.ctrl, kErrIndex, slot);
    return;
  }
  Y[slot] = x;
  if (DIM == 2) Y[d.n + slot] = y;
  d.src[slot] = (int)p;
}

// ------------------------------------------------------------- cell sort --
// Order inside a cell: by (x, src) in 1-d, which makes the whole array
// sorted by position; by src in 2-d.  src is the slot before the sort, so
// the result does not depend on the order the atomics handed out slots.
template <int DIM>
__device__ __forceinline__ bool before(long long xa, int sa, long long xb, int sb) {
  if (DIM == 1) return xa < xb || (xa == xb && sa < sb);
  return sa < sb;
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_cellsort(Dev d) {
  const long long k = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (k >= d.ncell) return;
  const int a = d.start[k], b = d.start[k + 1];
  const int len = b - a;
  if (len < 2) return;
  if (len > kSmallCell) {
    const int slot = atomicAdd(&d.ctrl->nbig, 1);
    if (slot < d.nbig_cap)
      d.big[slot] = (int)k;
    else
      raise_error(d.ctrl, kErrIndex, k);
    return;
  }
  long long* X = d.X[d.ctrl->xcur ^ 1];
  int* src = d.src;
  for (int i = a + 1; i < b; ++i) {
    const long long xi = X[i];
    const long long yi = DIM == 2 ? X[d.n + i] : 0;
    const int si = src[i];
    int j = i - 1;
    while (j >= a && before<DIM>(xi, si, X[j], src[j])) {
      X[j + 1] = X[j];
      if (DIM == 2) X[d.n + j + 1] = X[d.n + j];
      src[j + 1] = src[j];
      --j;
    }
    X[j + 1] = xi;
    if (DIM == 2) X[d.n + j + 1] = yi;
    src[j + 1] = si;
  }
}

// Large cells: one CTA per cell, bitonic sort with every comparator
// ascending (partner i ^ (2j - 1) in the first stage of each merge), which
// sorts any length when positions >= len are treated as +infinity.
template <int DIM>
__global__ void __launch_bounds__(1024) k_bigsort(Dev d) {
  __shared__ long long s_key[kBigSortCap];
  __shared__ int s_src[kBigSortCap];
  __shared__ int s_idx[kBigSortCap];
  Ctrl* c = d.ctrl;
  const int nbig = min(c->nbig, d.nbig_cap);
  long long* X = d.X[c->xcur ^ 1];
  int* src = d.src;
  for (int b = blockIdx.x; b < nbig; b += gridDim.x) {
    const long long k = d.big[b];
    const int a = d.start[k];
    const int len = d.start[k + 1] - a;
    if (len <= kBigSortCap) {
      int np2 = 1;
      while (np2 < len) np2 <<= 1;
      for (int i = threadIdx.x; i < len; i += blockDim.x) {
        s_key[i] = DIM == 1 ? X[a + i] : 0;
        s_src[i] = src[a + i];
        s_idx[i] = i;
      }
      __syncthreads();
      for (int m = 2; m <= np2; m <<= 1) {
        for (int j = m >> 1; j > 0; j >>= 1) {
          for (int i = threadIdx.x; i < np2; i += blockDim.x) {
            const int l = (j == (m >> 1)) ? (i ^ (m - 1)) : (i ^ j);
            if (l > i && l < len) {
              if (before<DIM>(s_key[l], s_src[l], s_key[i], s_src[i])) {
                const long long tk = s_key[i]; s_key[i] = s_key[l]; s_key[l] = tk;
                const int ts = s_src[i]; s_src[i] = s_src[l]; s_src[l] = ts;
                const int ti = s_idx[i]; s_idx[i] = s_idx[l]; s_idx[l] = ti;
              }
            }
          }
          __syncthreads();
        }
      }
      // apply the permutation: gather into registers, then write
      long long ry[kBigSortCap / 1024 + 1];
      long long rx[kBigSortCap / 1024 + 1];
      int t = 0;
      for (int i = threadIdx.x; i < len; i += blockDim.x, ++t) {
        rx[t] = X[a + s_idx[i]];
        if (DIM == 2) ry[t] = X[d.n + a + s_idx[i]];
      }
      __syncthreads();
      t = 0;
      for (int i = threadIdx.x; i < len; i += blockDim.x, ++t) {
        X[a + i] = rx[t];
        if (DIM == 2) X[d.n + a + i] = ry[t];
        src[a + i] = s_src[i];
      }
      __syncthreads();
    } else {
      // same network directly on global memory (very large cells only)
      long long np2l = 1;
      while (np2l < len) np2l <<= 1;
      for (long long m = 2; m <= np2l; m <<= 1) {
        for (long long j = m >> 1; j > 0; j >>= 1) {
          for (long long i = threadIdx.x; i < np2l; i += blockDim.x) {
            const long long l = (j == (m >> 1)) ? (i ^ (m - 1)) : (i ^ j);
            if (l > i && l < len) {
              const long long xi = X[a + i], xl = X[a + l];
              if (before<DIM>(xl, src[a + l], xi, src[a + i])) {
                X[a + i] = xl;
                X[a + l] = xi;
                if (DIM == 2) {
                  const long long yi = X[d.n + a + i];
                  X[d.n + a + i] = X[d.n + a + l];
                  X[d.n + a + l] = yi;
                }
                const int ts = src[a + i];
                src[a + i] = src[a + l];
                src[a + l] = ts;
              }
            }
          }
          __syncthreads();
        }
      }
    }
  }
}

// ------------------------------------------------------------- permute --
// After a sort without a transfer (upload): gather id and masses into the
// sorted slots, then the next kernel flips the selectors.
__global__ void __launch_bounds__(kThreads) k_permute(Dev d) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const int s = d.src[p];
  d.id[xc ^ 1][p] = d.id[xc][s];
  gather_masses(d, mc, p, s);
  gather_species(d, mc, p, s);
}

__global__ void k_flip(Dev d, int fx, int fm) {
  d.ctrl->xcur ^= fx;
  d.ctrl->mcur ^= fm;
}

// -------------------------------------------------------------- philox --
__global__ void k_philox(uint4 c, unsigned int k0, unsigned int k1, long long n,
                         unsigned int* out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 r = philox4x32_10(make_uint4(c.x + (unsigned int)i, c.y, c.z, c.w), k0, k1);
  out[4 * i + 0] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

// ------------------------------------------------------------ launchers --
static unsigned int blocks_for(long long n, int t) { return (unsigned int)((n + t - 1) / t); }

cudaError_t launch_move(const Dev& d, bool move, bool hist, cudaStream_t s) {
  const unsigned int g = blocks_for(d.n, kThreads);
  if (d.dim == 1) {
    if (move && hist) k_move<1, true, true><<<g, kThreads, 0, s>>>(d);
    else if (move) k_move<1, true, false><<<g, kThreads, 0, s>>>(d);
    else k_move<1, false, true><<<g, kThreads, 0, s>>>(d);
  } else {
    if (move && hist) k_move<2, true, true><<<g, kThreads, 0, s>>>(d);
    else if (move) k_move<2, true, false><<<g, kThreads, 0, s>>>(d);
    else k_move<2, false, true><<<g, kThreads, 0, s>>>(d);
  }
  return cudaGetLastError();
}

cudaError_t launch_sort(const Dev& d, cudaStream_t s, Marker& mk) {
  const unsigned int gs = blocks_for(d.ncell, kScanTile);
  mk("scan", s);
  k_scan<<<gs, kThreads, 0, s>>>(d);
  const unsigned int gp = blocks_for(d.n, kThreads);
  const unsigned int gc = blocks_for(d.ncell, kThreads);
  const unsigned int gb = (unsigned int)(d.nbig_cap < 304 ? d.nbig_cap : 304);
  if (d.dim == 1) {
    mk("scatter", s);
    k_scatter<1><<<gp, kThreads, 0, s>>>(d);
    mk("cellsort", s);
    k_cellsort<1><<<gc, kThreads, 0, s>>>(d);
    mk("bigsort", s);
    k_bigsort<1><<<gb, 1024, 0, s>>>(d);
  } else {
    mk("scatter", s);
    k_scatter<2><<<gp, kThreads, 0, s>>>(d);
    mk("cellsort", s);
    k_cellsort<2><<<gc, kThreads, 0, s>>>(d);
    mk("bigsort", s);
    k_bigsort<2><<<gb, 1024, 0, s>>>(d);
  }
  return cudaGetLastError();
}

cudaError_t launch_permute(const Dev& d, cudaStream_t s) {
  k_permute<<<blocks_for(d.n, kThreads), kThreads, 0, s>>>(d);
  k_flip<<<1, 1, 0, s>>>(d, 1, 1);
  return cudaGetLastError();
}

// The built-in random walk's normals of particles given by their indices in
// a system (the counter a single handle uses for caller index gid): one per
// axis, axis-major.
__global__ void k_walk_normals(const long long* gid, long long n, unsigned long long step,
                               unsigned int real, unsigned int k0, unsigned int k1, int dim,
                               float* out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const long long id = gid[p];
  const uint4 u = philox4x32_10(
      make_uint4((unsigned int)id, (unsigned int)step, (unsigned int)(step >> 32), real), k0, k1);
  const float2 g = box_muller(u.x, u.y);
  out[p] = g.x;
  if (dim == 2) out[n + p] = g.y;
}

cudaError_t launch_walk_normals(const long long* gid, long long n, unsigned long long step,
                                unsigned int real, unsigned int k0, unsigned int k1, int dim,
                                float* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_walk_normals<<<blocks_for(n, 256), 256, 0, s>>>(gid, n, step, real, k0, k1, dim, out);
  return cudaGetLastError();
}

cudaError_t launch_philox(uint4 c, unsigned int k0, unsigned int k1, long long n,
                          unsigned int* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_philox<<<blocks_for(n, 256), 256, 0, s>>>(c, k0, k1, n, out);
  return cudaGetLastError();
}

}  // namespace mt
