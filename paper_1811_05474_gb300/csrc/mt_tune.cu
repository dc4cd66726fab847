// mt_tune.cu -- mt_autotune: pick the cell width and the segment size of the
// one-kernel 1-d step by timing short runs of candidate configurations on
// the caller's inputs and workspace.  Host code over the public API only.
//
// Candidates: cell_shift in {c - 1, c, c + 1, c + 2} around the width the
// resolver chooses (about two particles per cell) and seg_target in {the
// resolver's choice, 256, 512, 1024}.  Each candidate runs `warmup` steps
// (the first builds its CUDA graph) and is then timed over `steps` steps
// with CUDA events on the stream.  The state the candidates advance is a
// scratch copy in the workspace; the caller's arrays are only read.
#include <cstring>
#include <vector>

#include "mt_internal.cuh"

namespace mt {
mt_status set_last_error(mt_status s, const char* msg);
}

namespace {

struct Candidate {
  int cell_shift, seg_target;
};

// The candidate set for p (resolved values of the resolver's own choice
// first; duplicates removed).
mt_status candidates(const mt_params* p, const mt_batch* b, std::vector<Candidate>* out) {
  mt_params r;
  mt_status s = mt_batch_resolve(p, b, &r);
  if (s != MT_OK) return s;
  out->clear();
  out->push_back({r.cell_shift, r.seg_target});
  if (r.dim != 1 || r.search != MT_SEARCH_CELL) return MT_OK;  // nothing to tune
  const int c0 = r.cell_shift;
  const int segs[4] = {0, 256, 512, 1024};
  for (int dc = -1; dc <= 2; ++dc) {
    const int c = c0 + dc;
    if (c < 1 || c > 62) continue;
    for (int t : segs) {
      mt_params q = *p;
      q.cell_shift = c;
      q.seg_target = t;
      mt_params rq;
      if (mt_batch_resolve(&q, b, &rq) != MT_OK || rq.seg_target == 0) continue;
      bool dup = false;
      for (const Candidate& e : *out)
        dup |= e.cell_shift == rq.cell_shift && e.seg_target == rq.seg_target;
      if (!dup) out->push_back({rq.cell_shift, rq.seg_target});
    }
  }
  return MT_OK;
}

mt_params with(const mt_params* p, const Candidate& c) {
  mt_params q = *p;
  q.cell_shift = c.cell_shift;
  q.seg_target = c.seg_target;
  return q;
}

}  // namespace

extern "C" {

mt_status mt_autotune_workspace_bytes(const mt_params* p, const mt_batch* b, size_t* bytes) {
  if (!bytes) return mt::set_last_error(MT_ERR_INVALID, "bytes is NULL");
  std::vector<Candidate> cs;
  mt_status s = candidates(p, b, &cs);
  if (s != MT_OK) return s;
  size_t most = 0;
  for (const Candidate& c : cs) {
    const mt_params q = with(p, c);
    size_t n = 0;
    s = mt_batch_workspace_bytes(&q, b, &n);
    if (s != MT_OK) return s;
    most = n > most ? n : most;
  }
  *bytes = most;
  return MT_OK;
}

mt_status mt_autotune(const mt_params* p, const mt_batch* b, const double* x, const double* A,
                      const double* B, int32_t mem, void* workspace, size_t workspace_bytes,
                      void* stream, int32_t warmup, int32_t steps, mt_params* best,
                      float* best_ms) {
  if (!best) return mt::set_last_error(MT_ERR_INVALID, "best is NULL");
  if (warmup < 1 || steps < 1)
    return mt::set_last_error(MT_ERR_INVALID, "warmup and steps must be >= 1");
  std::vector<Candidate> cs;
  mt_status s = candidates(p, b, &cs);
  if (s != MT_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStream_t own = nullptr;  // the events must be on the handles' stream
  if (!st) {
    if (cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) != cudaSuccess)
      return mt::set_last_error(MT_ERR_CUDA, "mt_autotune: cudaStreamCreateWithFlags failed");
    st = own;
    stream = own;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (own) cudaStreamDestroy(own);
    return mt::set_last_error(MT_ERR_CUDA, "mt_autotune: cudaEventCreate failed");
  }
  float top = -1.0f;
  Candidate pick = cs[0];
  int tried = 0;
  for (const Candidate& c : cs) {
    const mt_params q = with(p, c);
    size_t need = 0;
    if (mt_batch_workspace_bytes(&q, b, &need) != MT_OK || need > workspace_bytes) continue;
    mt_handle* h = nullptr;
    s = mt_batch_create(&q, b, workspace, workspace_bytes, stream, &h);
    if (s == MT_OK) s = mt_upload(h, x, A, B, mem);
    if (s == MT_OK) s = mt_run(h, warmup);
    if (s == MT_OK) s = mt_sync(h);
    float ms = 0.0f;
    if (s == MT_OK) {
      cudaEventRecord(e0, st);
      s = mt_run(h, steps);
      cudaEventRecord(e1, st);
      if (s == MT_OK) s = mt_sync(h);
      if (s == MT_OK && (cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        s = mt::set_last_error(MT_ERR_CUDA, "mt_autotune: event timing failed");
    }
    if (h) mt_destroy(h);
    if (s != MT_OK) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (own) cudaStreamDestroy(own);
      return s;
    }
    ++tried;
    ms /= (float)steps;
    if (top < 0.0f || ms < top) {
      top = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (own) cudaStreamDestroy(own);
  if (tried == 0) return mt::set_last_error(MT_ERR_WORKSPACE, "mt_autotune: workspace too small");
  mt_params q = *p;
  q.cell_shift = pick.cell_shift;
  q.seg_target = pick.seg_target;
  s = mt_batch_resolve(&q, b, best);
  if (s != MT_OK) return s;
  if (best_ms) *best_ms = top;
  return MT_OK;
}

}  // extern "C"
