// mt_io.cu -- state upload, read-back in the caller's particle order, and
// the pair export used to compare the search with the oracle's pair set.
#include "mt_internal.cuh"

namespace mt {

static unsigned int blocks_for(long long n, int t) { return (unsigned int)((n + t - 1) / t); }

// x (dim*n doubles), A, B (n doubles), all device memory in the caller's
// order -> grid ticks X = rint(x 2^k) (plus the realisation's base on the
// shared axis), id = (realisation << lbits) | index within it, masses in the
// precision's format.  Positions outside [0, L] or NaN raise kErrInput.
__global__ void k_upload(Dev d, const double* x, const double* A, const double* B, double pow2k,
                         int mixed) {
  const long long i = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (i >= d.n) return;
  Ctrl* c = d.ctrl;
  const int xc = c->xcur, mc = c->mcur;
  int lo = 0, hi = d.nreal - 1;  // last realisation with off <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (d.rt[mid].off <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int r = lo;
  const Real R = d.rt[r];
  for (int a = 0; a < d.dim; ++a) {
    const long long Lq = a == 0 ? R.Lq : d.Lq[a];
    const double v = x[(long long)a * d.n + i];
    long long X = 0;
    if (!(v >= 0.0)) {
      raise_error(c, kErrInput, i);
    } else {
      X = __double2ll_rn(v * pow2k);
      if (d.periodic && X == Lq) {
        X = 0;  // L is the same point as 0
      } else if (X > Lq) {
        raise_error(c, kErrInput, i);
        X = Lq;
      }
    }
    d.X[xc][(long long)a * d.n + i] = a == 0 ? R.base + X : X;
  }
  d.id[xc][i] = (r << d.lbits) | (int)(i - R.off);
  if (mixed) {
    const double a = A[i], b = B[i];
    const float ah = __double2float_rn(a), bh = __double2float_rn(b);
    df_store(d.M[mc], i, {ah, __double2float_rn(a - (double)ah)});
    df_store(d.M[mc], d.n + i, {bh, __double2float_rn(b - (double)bh)});
  } else {
    f64_store(d.M[mc], i, A[i]);
    f64_store(d.M[mc], d.n + i, B[i]);
  }
  for (int k = 2; k < d.nspec; ++k) d.M[mc][k * d.n + i] = 0ULL;  // +0 in both formats
}

cudaError_t launch_upload(const Dev& d, const double* x, const double* A, const double* B,
                          int precision, cudaStream_t s) {
  const double pow2k = 1.0 / d.scale;
  k_upload<<<blocks_for(d.n, kThreads), kThreads, 0, s>>>(d, x, A, B, pow2k,
                                                          precision == MT_MIXED_DF32);
  return cudaGetLastError();
}

__global__ void k_read_masses(Dev d, double* A, double* B, int mixed) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const int idp = d.id[xc][p];
  const long long id = idp < 0 || (idp >> d.lbits) >= d.nreal ? -1 : caller_index(d, idp);
  if (id < 0 || id >= d.n) {
    raise_error(d.ctrl, kErrIndex, p);
    return;
  }
  const unsigned long long* M = d.M[mc];
  if (mixed) {
    const df a = df_load(M, p), b = df_load(M, d.n + p);
    A[id] = (double)a.hi + (double)a.lo;
    B[id] = (double)b.hi + (double)b.lo;
  } else {
    A[id] = f64_load(M, p);
    B[id] = f64_load(M, d.n + p);
  }
}

cudaError_t launch_read_masses(const Dev& d, double* A, double* B, int precision,
                               cudaStream_t s) {
  k_read_masses<<<blocks_for(d.n, kThreads), kThreads, 0, s>>>(d, A, B,
                                                               precision == MT_MIXED_DF32);
  return cudaGetLastError();
}

// One species in the caller's order: v[caller index] <-> slot p of the
// current mass buffer.
__global__ void k_species_io(Dev d, int sp, double* out, const double* in, int mixed) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur, mc = d.ctrl->mcur;
  const int idp = d.id[xc][p];
  const long long id = idp < 0 || (idp >> d.lbits) >= d.nreal ? -1 : caller_index(d, idp);
  if (id < 0 || id >= d.n) {
    raise_error(d.ctrl, kErrIndex, p);
    return;
  }
  unsigned long long* M = d.M[mc] + (long long)sp * d.n;
  if (in) {
    const double v = in[id];
    if (mixed) {
      const float h = __double2float_rn(v);
      df_store(M, p, {h, __double2float_rn(v - (double)h)});
    } else {
      f64_store(M, p, v);
    }
  } else if (mixed) {
    const df v = df_load(M, p);
    out[id] = (double)v.hi + (double)v.lo;
  } else {
    out[id] = f64_load(M, p);
  }
}

cudaError_t launch_species_io(const Dev& d, int sp, double* out, const double* in, int precision,
                              cudaStream_t s) {
  k_species_io<<<blocks_for(d.n, kThreads), kThreads, 0, s>>>(d, sp, out, in,
                                                              precision == MT_MIXED_DF32);
  return cudaGetLastError();
}

__global__ void k_read_positions(Dev d, double* x, long long* X) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur;
  const int idp = d.id[xc][p];
  const long long id = idp < 0 || (idp >> d.lbits) >= d.nreal ? -1 : caller_index(d, idp);
  if (id < 0 || id >= d.n) {
    raise_error(d.ctrl, kErrIndex, p);
    return;
  }
  const long long base = d.rt[idp >> d.lbits].base;
  for (int a = 0; a < d.dim; ++a) {
    const long long v = d.X[xc][(long long)a * d.n + p] - (a == 0 ? base : 0);
    if (x) x[(long long)a * d.n + id] = (double)v * d.scale;
    if (X) X[(long long)a * d.n + id] = v;
  }
}

cudaError_t launch_read_positions(const Dev& d, double* x, long long* X, cudaStream_t s) {
  k_read_positions<<<blocks_for(d.n, kThreads), kThreads, 0, s>>>(d, x, X);
  return cudaGetLastError();
}

// ------------------------------------------------------------- pairs --

__device__ __forceinline__ void emit(const Dev& d, int a, int b, int* pi, int* pj,
                                     long long cap) {
  const unsigned long long slot = atomicAdd(&d.ctrl->npairs, 1ULL);
  a = (int)caller_index(d, a);
  b = (int)caller_index(d, b);
  if ((long long)slot < cap) {
    pi[slot] = a < b ? a : b;
    pj[slot] = a < b ? b : a;
  }
}

__global__ void k_pairs_walk(Dev d, int* pi, int* pj, long long cap) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur;
  const long long* X = d.X[xc];
  const int* id = d.id[xc];
  const long long x = X[p];
  if (!d.periodic) {
    for (long long q = p + 1; q < d.n; ++q) {
      if (X[q] - x > d.S) break;
      emit(d, id[p], id[q], pi, pj, cap);
    }
    return;
  }
  // periodic: walk right around the realisation's ring (each pair is found
  // from the particle that has the other on its right within Smax)
  const Ring g = ring_of(d, id[p]);
  for (long long k = 1; k < g.n; ++k) {
    const long long q = ring_step(g, p, k);
    const long long D = wrap(X[q] - x, g.Lq);
    if (D > d.S) break;
    emit(d, id[p], id[q], pi, pj, cap);
  }
}

__device__ __forceinline__ bool in_range2_io(long long dx, long long dy, long long S) {
  const unsigned long long ax = (unsigned long long)(dx < 0 ? -dx : dx);
  const unsigned long long ay = (unsigned long long)(dy < 0 ? -dy : dy);
  if (ax > (unsigned long long)S || ay > (unsigned long long)S) return false;
  return ax * ax + ay * ay <= (unsigned long long)S * (unsigned long long)S;
}

__global__ void k_pairs_cell2(Dev d, int* pi, int* pj, long long cap) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur;
  const long long* X = d.X[xc];
  const int* id = d.id[xc];
  const long long x = X[p], y = X[d.n + p];
  cells2_visit(d, x, y, [&](int q0, int q1) {
    for (int q = q0; q < q1; ++q) {
      if (q <= p) continue;
      long long dx = X[q] - x, dy = X[d.n + q] - y;
      if (d.periodic) {
        dx = min_image(dx, d.Lq[0]);
        dy = min_image(dy, d.Lq[1]);
      }
      if (in_range2_io(dx, dy, d.S)) emit(d, id[p], id[q], pi, pj, cap);
    }
  });
}

__global__ void k_pairs_brute(Dev d, int* pi, int* pj, long long cap) {
  const long long p = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (p >= d.n) return;
  const int xc = d.ctrl->xcur;
  const long long* X = d.X[xc];
  const int* id = d.id[xc];
  const long long x = X[p], y = d.dim == 2 ? X[d.n + p] : 0;
  for (long long q = p + 1; q < d.n; ++q) {
    long long dx = X[q] - x;
    if (d.periodic) dx = min_image(dx, d.Lq[0]);
    bool ok;
    if (d.dim == 1)
      ok = dx <= d.S && -dx <= d.S;
    else
      ok = in_range2_io(dx, d.periodic ? min_image(X[d.n + q] - y, d.Lq[1]) : X[d.n + q] - y, d.S);
    if (ok) emit(d, id[p], id[q], pi, pj, cap);
  }
}

__global__ void k_zero_pairs(Dev d) { d.ctrl->npairs = 0; }

cudaError_t launch_pairs(const Dev& d, int search, int* pi, int* pj, long long cap,
                         cudaStream_t s) {
  k_zero_pairs<<<1, 1, 0, s>>>(d);
  const unsigned int g = blocks_for(d.n, kThreads);
  if (d.n > 0) {
    if (search == MT_SEARCH_CELL && d.dim == 1)
      k_pairs_walk<<<g, kThreads, 0, s>>>(d, pi, pj, cap);
    else if (search == MT_SEARCH_CELL)
      k_pairs_cell2<<<g, kThreads, 0, s>>>(d, pi, pj, cap);
    else
      k_pairs_brute<<<g, kThreads, 0, s>>>(d, pi, pj, cap);
  }
  return cudaGetLastError();
}

}  // namespace mt
