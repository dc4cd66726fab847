// mt_noalloc.cu -- mt_transfer_1d_noalloc: one mass-transfer step (Eq. 3,
// 4, 7) and, optionally, the A + B -> E reaction for particles on a line,
// computed in binary64 without any device allocation by this library or the
// caller.
//
// Some callers cannot call cudaMalloc: code running where the allocator is
// owned by someone else (a host application that hands out only its own
// buffers, a plug-in inside another runtime, a pipeline that forbids
// allocation while it runs).  They still pass their own input and output
// arrays; the per-particle intermediates (positions on the tick grid and
// 1 / r_i) live in the fixed array g_noalloc_scratch below.  The call waits
// for its stream before it returns (it reads back the input check).
//
// The scratch array is a file-scope __device__ variable: every GPU that loads
// libmt holds its 16 MiB + 256 bytes until the process exits, whether or not
// this entry point is called.  It bounds n to kNoAllocMax = 2^20 particles.
// All calls share it and it keeps the last call's contents; calls that
// overlap on the GPU (different streams, or different host threads without
// ordering) race on it and give wrong results.
#include <cmath>
#include <mutex>

#include "mt_internal.cuh"

namespace mt {
mt_status set_last_error(mt_status s, const char* msg);
}

namespace {

constexpr long long kNoAllocMax = 1LL << 20;
constexpr size_t kTicksBytes = (size_t)kNoAllocMax * 8;
constexpr size_t kRinvBytes = (size_t)kNoAllocMax * 8;
constexpr size_t kScratchBytes = kTicksBytes + kRinvBytes + 256;

// [ticks: int64 x kNoAllocMax][1/r: double x kNoAllocMax][error word + pad]
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Error word at the end of the scratch: 0 ok, 1 position outside [0, L] or
// NaN, 2 positions not sorted ascending.  Cleared at the start of every call.
__global__ void k_na_quantize(const double* x, long long n, double pow2k, long long Lq,
                              long long* ticks, int* err) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  long long X = 0;
  if (!(v >= 0.0)) {
    atomicCAS(err, 0, 1);
  } else {
    X = __double2ll_rn(v * pow2k);
    if (X > Lq) atomicCAS(err, 0, 1);
  }
  if (i > 0 && !(x[i - 1] <= v)) atomicCAS(err, 0, 2);
  ticks[i] = X;
}

// exp(-s^2 / (8 D_mt dt)), s = |dX| 2^-k (Eq. 3 without its prefactor).
__device__ __forceinline__ double na_weight(long long D, double scale, double inv8) {
  const double s = __dmul_rn((double)D, scale);
  return exp(-__dmul_rn(__dmul_rn(s, s), inv8));
}

__global__ void k_na_rowsum(const long long* ticks, long long n, long long S, double scale,
                            double inv8, double* rinv) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const long long x = ticks[p];
  // Each walk stops at the first neighbour out of range, or out of order: on
  // unsorted input (rejected after the call) the work stays O(n k).
  double r = 1.0;
  for (long long q = p - 1; q >= 0; --q) {
    const long long D = x - ticks[q];
    if (D < 0 || D > S) break;
    r += na_weight(D, scale, inv8);
  }
  for (long long q = p + 1; q < n; ++q) {
    const long long D = ticks[q] - x;
    if (D < 0 || D > S) break;
    r += na_weight(D, scale, inv8);
  }
  rinv[p] = 1.0 / r;
}

__global__ void k_na_exchange(const long long* ticks, const double* rinv, const double* A,
                              const double* B, double* Ao, double* Bo, long long n, long long S,
                              double scale, double inv8, int norm, int react) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const long long x = ticks[p];
  const double ip = rinv[p], a = A[p], b = B[p];
  double dA = 0.0, dB = 0.0;
  for (int side = 0; side < 2; ++side) {
    for (long long q = side ? p + 1 : p - 1; q >= 0 && q < n; q += side ? 1 : -1) {
      const long long D = side ? ticks[q] - x : x - ticks[q];
      if (D < 0 || D > S) break;
      const double w = na_weight(D, scale, inv8);
      const double P = norm == MT_NORM_ROW ? w * ip : 0.5 * w * (ip + rinv[q]);
      dA += P * (A[q] - a);
      dB += P * (B[q] - b);
    }
  }
  double a2 = a + 0.5 * dA, b2 = b + 0.5 * dB;
  if (react) {
    const double m = a2 < b2 ? a2 : b2;
    a2 = a2 - m;
    b2 = b2 - m;
  }
  Ao[p] = a2;
  Bo[p] = b2;
}

mt_status err(mt_status s, const char* msg) { return mt::set_last_error(s, msg); }

// The scratch array's device address on the current device, looked up once
// per device (cudaGetSymbolAddress, with that device current).
mt_status scratch_on_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return err(MT_ERR_CUDA, "mt_transfer_1d_noalloc: no usable current device");
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return err(MT_ERR_CUDA, "mt_transfer_1d_noalloc: cudaGetSymbolAddress failed");
    g_scratch_ptr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
  return MT_OK;
}

}  // namespace

extern "C" mt_status mt_transfer_1d_noalloc(const double* x, const double* A, const double* B,
                                            double* A_out, double* B_out, int64_t n, double L,
                                            double D_mt, double dt, double cutoff, int32_t norm,
                                            int32_t react, void* stream) {
  if (n < 0 || n > kNoAllocMax)
    return err(MT_ERR_INVALID,
               "mt_transfer_1d_noalloc: n must be in [0, 1048576] (the fixed scratch size)");
  if (!(std::isfinite(L) && L > 0.0) || !(std::isfinite(D_mt) && D_mt > 0.0) ||
      !(std::isfinite(dt) && dt > 0.0) || !std::isfinite(cutoff))
    return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: L, D_mt, dt must be finite and > 0");
  if (norm != MT_NORM_SYM && norm != MT_NORM_ROW)
    return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: unknown norm");
  if (react != 0 && react != 1) return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: react is 0/1");
  if (n > 0 && (!x || !A || !B || !A_out || !B_out))
    return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: NULL array");
  if (n > 0 && (A_out == A || A_out == B || B_out == A || B_out == B))
    return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: outputs must not alias inputs");
  const double smax = cutoff > 0.0 ? cutoff : 3.0 * std::sqrt(4.0 * D_mt * dt);
  // the grid rule of mt_resolve: largest k with s_max 2^k < 2^30, L 2^k < 2^61
  int k = 62;
  while (k > 0 && (std::ldexp(smax, k) >= 1073741824.0 || std::ldexp(L, k) >= 2305843009213693952.0))
    --k;
  if (k < 1) return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: cutoff or L too large");
  unsigned char* base = nullptr;
  const mt_status s = scratch_on_current_device(&base);
  if (s != MT_OK) return s;
  if (n == 0) return MT_OK;
  long long* ticks = reinterpret_cast<long long*>(base);
  double* rinv = reinterpret_cast<double*>(base + kTicksBytes);
  int* errw = reinterpret_cast<int*>(base + kTicksBytes + kRinvBytes);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long S = (long long)std::floor(std::ldexp(smax, k));
  const long long Lq = std::llrint(std::ldexp(L, k));
  const double scale = std::ldexp(1.0, -k), inv8 = 1.0 / (8.0 * D_mt * dt);
  const unsigned int g = (unsigned int)((n + 255) / 256);
  if (cudaMemsetAsync(errw, 0, sizeof(int), st) != cudaSuccess)
    return err(MT_ERR_CUDA, "mt_transfer_1d_noalloc: clearing the error word failed");
  k_na_quantize<<<g, 256, 0, st>>>(x, n, std::ldexp(1.0, k), Lq, ticks, errw);
  k_na_rowsum<<<g, 256, 0, st>>>(ticks, n, S, scale, inv8, rinv);
  k_na_exchange<<<g, 256, 0, st>>>(ticks, rinv, A, B, A_out, B_out, n, S, scale, inv8, norm,
                                   react);
  if (cudaGetLastError() != cudaSuccess)
    return err(MT_ERR_CUDA, "mt_transfer_1d_noalloc: kernel launch failed");
  int hflag = 0;
  if (cudaMemcpyAsync(&hflag, errw, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return err(MT_ERR_CUDA, "mt_transfer_1d_noalloc: stream failed");
  if (hflag == 1) return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: position outside [0, L]");
  if (hflag == 2) return err(MT_ERR_INVALID, "mt_transfer_1d_noalloc: positions not sorted");
  return MT_OK;
}
