// mt_probe.cu -- throughput probes for the non-HBM rooflines of the
// transfer kernels: binary64 fused multiply-add, binary32 fused
// multiply-add, the binary32 fast exponential (__expf), the library's
// binary64 exponential (exp) and the weights' own binary64 exponential
// (exp_neg).  Not part of the paper: they measure the device peaks the FP64
// and brute-force passes are compared against.  Also the test hook that
// evaluates exp_neg on a device array.
//
// Each thread runs kChains independent dependency chains for `iters`
// rounds (enough independent work per warp to keep the pipe busy), on a
// grid of kBlocksPerSm CTAs per multiprocessor; the chains' final values
// are summed into one word per CTA so nothing is dead code.  Rate =
// operations / event-timed kernel duration (one warm-up launch first).
#include <cmath>

#include "mt_pair.cuh"

namespace mt {
mt_status set_last_error(mt_status s, const char* msg);
}

namespace {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;
constexpr int kBlocksPerSm = 8;

template <int WHICH>
__global__ void __launch_bounds__(kProbeThreads) k_probe(double* out, int iters, double seed) {
  const double t = seed + 1e-7 * (double)(threadIdx.x + blockIdx.x * blockDim.x);
  double a[kChains];
  float f[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    a[k] = t + 0.01 * k;
    f[k] = (float)a[k];
  }
  const double m = 0.999999, c = 1e-9;
  const float mf = 0.999999f, cf = 1e-9f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) {
      if (WHICH == 0) a[k] = __fma_rn(a[k], m, c);              // binary64 FMA
      if (WHICH == 1) f[k] = __fmaf_rn(f[k], mf, cf);           // binary32 FMA
      if (WHICH == 2) f[k] = __expf(-f[k]);                     // binary32 fast exp
      if (WHICH == 3) a[k] = exp(-a[k]);                        // binary64 exp
      if (WHICH == 4) a[k] = mt::exp_neg(a[k]);                 // the weights' exp(-t)
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += (WHICH == 0 || WHICH >= 3) ? a[k] : (double)f[k];
  __shared__ double red[kProbeThreads / 32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < kProbeThreads / 32; ++w) v += red[w];
    out[blockIdx.x] = v;
  }
}

template <int WHICH>
cudaError_t launch_probe(double* out, int blocks, int iters, cudaStream_t s) {
  k_probe<WHICH><<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.5);
  return cudaGetLastError();
}

cudaError_t launch_which(int which, double* out, int blocks, int iters, cudaStream_t s) {
  switch (which) {
    case 0: return launch_probe<0>(out, blocks, iters, s);
    case 1: return launch_probe<1>(out, blocks, iters, s);
    case 2: return launch_probe<2>(out, blocks, iters, s);
    case 3: return launch_probe<3>(out, blocks, iters, s);
    default: return launch_probe<4>(out, blocks, iters, s);
  }
}

__global__ void k_exp_neg(const double* t, double* out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = mt::exp_neg(t[i]);
}

}  // namespace

extern "C" mt_status mt_test_exp_neg(const double* t, double* out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!t || !out)))
    return mt::set_last_error(MT_ERR_INVALID, "mt_test_exp_neg: n < 0 or NULL array");
  if (n == 0) return MT_OK;
  const long long blocks = (n + 255) / 256;
  k_exp_neg<<<(unsigned int)blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(t, out, n);
  if (cudaGetLastError() != cudaSuccess)
    return mt::set_last_error(MT_ERR_CUDA, "mt_test_exp_neg: launch failed");
  return MT_OK;
}

extern "C" mt_status mt_probe_rate(int32_t which, void* scratch, size_t scratch_bytes,
                                   void* stream, double* ops_per_s) {
  if (which < 0 || which > 4 || !ops_per_s)
    return mt::set_last_error(MT_ERR_INVALID, "mt_probe_rate: which must be 0..4");
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return mt::set_last_error(MT_ERR_CUDA, "mt_probe_rate: no device");
  const int blocks = nsm * kBlocksPerSm;
  if (!scratch || scratch_bytes < (size_t)blocks * sizeof(double))
    return mt::set_last_error(MT_ERR_WORKSPACE, "mt_probe_rate: scratch too small");
  // rounds per thread: about 2^31 operations per launch for the fast pipes,
  // 2^28 for the binary64 ones
  const int iters = which == 0 ? 2048 : which >= 3 ? 256 : 16384;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* out = static_cast<double*>(scratch);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return mt::set_last_error(MT_ERR_CUDA, "mt_probe_rate: event");
  cudaError_t e = launch_which(which, out, blocks, iters / 8, s);  // warm-up
  float best = 0.f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) e = launch_which(which, out, blocks, iters, s);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || best <= 0.f)
    return mt::set_last_error(MT_ERR_CUDA, "mt_probe_rate: launch failed");
  const double ops = (double)blocks * kProbeThreads * (double)iters * kChains;
  *ops_per_s = ops / (best * 1e-3);
  return MT_OK;
}
