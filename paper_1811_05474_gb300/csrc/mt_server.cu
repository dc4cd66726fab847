// mt_server.cu -- a request server for simulations of the paper's method:
// requests of different sizes and dimensions arrive over time; each is
// admitted when a slot (a CUDA stream) and room in the device pool are
// free, keeps its particle state resident in its own workspace, and is
// advanced in chunks of graph-replayed steps interleaved with the other
// resident requests, whose work overlaps on the device.  Host code over the
// public API (mt_create / mt_upload / mt_run / mt_read_*).
//
// Scheduling (mt_server_poll, never blocks on running work):
//   1. retire: a request whose chunk has finished (its event has completed)
//      records the chunk's time, then either gets its next chunk or, after
//      its last step, has its results read back, its handle destroyed and
//      its pool block freed;
//   2. admit: while a slot is free, the oldest queued request whose
//      footprint fits the pool (first fit) is created, uploaded and given its
//      first chunk; with backfill on, a later request may be admitted when
//      the oldest does not fit yet.
// Each request runs exactly the steps it would run alone, on its own state:
// its results do not depend on what else is resident.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "mt_internal.cuh"

namespace mt {
mt_status set_last_error(mt_status s, const char* msg);
}

namespace {

constexpr size_t kPoolAlign = 256;

// First-fit allocator over [0, size) of the caller's pool.
class Pool {
 public:
  explicit Pool(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* at) {
    bytes = (bytes + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *at = it->first;
      const size_t rest = it->second - bytes, next = it->first + bytes;
      free_.erase(it);
      if (rest) free_[next] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return true;
    }
    return false;
  }
  void release(size_t at, size_t bytes) {
    bytes = (bytes + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
    used_ -= bytes;
    auto it = free_.emplace(at, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;  // offset -> length
  size_t used_ = 0, peak_ = 0;
};

struct Request {
  int64_t id = 0;
  mt_params p{};
  int64_t steps = 0, done = 0;
  std::vector<double> x;             // positions until admitted
  std::vector<double> M;             // species masses [species][n]: inputs, then results
  std::vector<double> obs;           // observables rows after the last step
  int state = MT_REQ_QUEUED;
  mt_status status = MT_OK;
  size_t footprint = 0, at = 0;
  bool held = false;                 // owns [at, at + footprint) of the pool
  int slot = -1;
  mt_handle* h = nullptr;
  int64_t chunk = 0;                 // steps of the chunk in flight
  double t_submit = 0, t_admit = 0, t_done = 0, gpu_ms = 0;
};

// Species a request carries (its parameters' 0 means 2).
int species_of(const mt_params& p) { return p.species > 2 ? p.species : 2; }

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  Request* req = nullptr;
};

}  // namespace

struct mt_server {
  mt_server_config cfg{};
  char* pool_base = nullptr;
  size_t pool_bytes = 0;
  std::unique_ptr<Pool> pool;
  std::vector<Slot> slots;
  std::deque<Request*> queue;                        // submitted, not admitted
  std::map<int64_t, std::unique_ptr<Request>> reqs;  // every request not released
  std::vector<float> step_ms;                        // one sample per finished chunk
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

mt_status err(mt_status s, const char* msg) { return mt::set_last_error(s, msg); }

size_t footprint_of(const mt_params& p) {
  size_t b = 0;
  if (mt_workspace_bytes(&p, &b) != MT_OK) return 0;
  return (b + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
}

void fail_request(mt_server* s, Request* r, mt_status st) {
  r->state = MT_REQ_FAILED;
  r->status = st;
  r->t_done = s->now();
  if (r->h) {
    mt_destroy(r->h);
    r->h = nullptr;
  }
  if (r->slot >= 0) {
    s->slots[r->slot].req = nullptr;
    r->slot = -1;
  }
  if (r->held) s->pool->release(r->at, r->footprint);
  r->held = false;
}

mt_status enqueue_chunk(mt_server* s, Request* r) {
  Slot& sl = s->slots[r->slot];
  r->chunk = std::min<int64_t>(s->cfg.chunk_steps, r->steps - r->done);
  if (cudaEventRecord(sl.e0, sl.stream) != cudaSuccess) return err(MT_ERR_CUDA, "event record");
  const mt_status st = mt_run(r->h, r->chunk);
  if (st != MT_OK) return st;
  if (cudaEventRecord(sl.e1, sl.stream) != cudaSuccess) return err(MT_ERR_CUDA, "event record");
  return MT_OK;
}

mt_status finish(mt_server* s, Request* r) {
  const size_t n = (size_t)r->p.n;
  const int S = species_of(r->p);
  r->M.assign((size_t)S * n, 0.0);
  mt_status st = MT_OK;
  for (int k = 0; k < S && st == MT_OK && n > 0; ++k)
    st = mt_read_species(r->h, k, r->M.data() + (size_t)k * n, MT_MEM_HOST);
  if (st == MT_OK && r->p.observe_cap > 0) {
    const int64_t rows = std::min<int64_t>(r->p.observe_cap, r->steps);
    r->obs.assign((size_t)rows * 4, 0.0);
    int64_t got = 0;
    st = mt_read_observables(r->h, r->obs.data(), rows, &got);
    r->obs.resize((size_t)got * 4);
  }
  r->x.clear();
  r->x.shrink_to_fit();
  mt_destroy(r->h);
  r->h = nullptr;
  s->slots[r->slot].req = nullptr;
  r->slot = -1;
  s->pool->release(r->at, r->footprint);
  r->held = false;
  r->t_done = s->now();
  if (st != MT_OK) {
    r->state = MT_REQ_FAILED;
    r->status = st;
    return MT_OK;
  }
  r->state = MT_REQ_DONE;
  return MT_OK;
}

// Admit r into free slot k at pool offset `at`.
void admit(mt_server* s, Request* r, int k, size_t at) {
  Slot& sl = s->slots[k];
  r->at = at;
  r->held = true;
  r->slot = k;
  sl.req = r;
  r->state = MT_REQ_RUNNING;
  r->t_admit = s->now();
  mt_status st = mt_create(&r->p, s->pool_base + at, r->footprint, sl.stream, &r->h);
  const size_t n = (size_t)r->p.n;
  if (st == MT_OK)
    st = mt_upload(r->h, r->x.data(), r->M.data(), r->M.data() + n, MT_MEM_HOST);
  for (int k = 2; k < species_of(r->p) && st == MT_OK && n > 0; ++k)
    st = mt_set_species(r->h, k, r->M.data() + (size_t)k * n, MT_MEM_HOST);
  if (st == MT_OK) {
    r->M.clear();
    st = r->steps > 0 ? enqueue_chunk(s, r) : MT_OK;
  }
  if (st != MT_OK) fail_request(s, r, st);
}

}  // namespace

extern "C" {

mt_status mt_server_footprint(const mt_params* p, size_t* bytes) {
  if (!p || !bytes) return err(MT_ERR_INVALID, "mt_server_footprint: NULL argument");
  size_t b = 0;
  const mt_status st = mt_workspace_bytes(p, &b);
  if (st != MT_OK) return st;
  *bytes = (b + kPoolAlign - 1) / kPoolAlign * kPoolAlign;
  return MT_OK;
}

mt_status mt_server_create(const mt_server_config* cfg, void* pool, size_t pool_bytes,
                           mt_server** out) {
  if (!cfg || !out) return err(MT_ERR_INVALID, "mt_server_create: NULL argument");
  *out = nullptr;
  if (cfg->max_active < 1 || cfg->max_active > 1024 || cfg->chunk_steps < 1)
    return err(MT_ERR_INVALID, "mt_server_create: max_active in [1, 1024], chunk_steps >= 1");
  if (!pool || (uintptr_t)pool % kPoolAlign != 0)
    return err(MT_ERR_WORKSPACE, "mt_server_create: pool must be 256-byte aligned device memory");
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, pool) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return err(MT_ERR_WORKSPACE, "mt_server_create: pool is not device memory");
  }
  mt_server* s = new (std::nothrow) mt_server();
  if (!s) return err(MT_ERR_INVALID, "mt_server_create: out of host memory");
  s->cfg = *cfg;
  s->pool_base = static_cast<char*>(pool);
  s->pool_bytes = pool_bytes;
  s->pool.reset(new Pool(pool_bytes));
  s->t0 = std::chrono::steady_clock::now();
  s->slots.resize((size_t)cfg->max_active);
  for (Slot& sl : s->slots) {
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sl.e0) != cudaSuccess || cudaEventCreate(&sl.e1) != cudaSuccess) {
      mt_server_destroy(s);
      return err(MT_ERR_CUDA, "mt_server_create: stream or event creation failed");
    }
  }
  *out = s;
  return MT_OK;
}

mt_status mt_server_submit(mt_server* s, const mt_params* p, const double* x, const double* A,
                           const double* B, int64_t steps, int64_t* id) {
  if (!p) return err(MT_ERR_INVALID, "mt_server_submit: NULL argument");
  mt_params r;
  mt_status st = mt_resolve(p, &r);
  if (st != MT_OK) return st;
  if (r.species != 2)
    return err(MT_ERR_INVALID, "mt_server_submit: more than two species need mt_server_submit_species");
  const size_t n = (size_t)r.n;
  if (n > 0 && (!A || !B)) return err(MT_ERR_INVALID, "mt_server_submit: x, A, B required");
  std::vector<double> M;
  M.reserve(2 * n);
  if (n > 0) {
    M.assign(A, A + n);
    M.insert(M.end(), B, B + n);
  }
  return mt_server_submit_species(s, p, x, M.data(), steps, id);
}

mt_status mt_server_submit_species(mt_server* s, const mt_params* p, const double* x,
                                   const double* M, int64_t steps, int64_t* id) {
  if (!s || !p || !id) return err(MT_ERR_INVALID, "mt_server_submit: NULL argument");
  if (steps < 0) return err(MT_ERR_INVALID, "mt_server_submit: steps must be >= 0");
  mt_params r;
  mt_status st = mt_resolve(p, &r);
  if (st != MT_OK) return st;
  const size_t n = (size_t)r.n, m = (size_t)r.dim * n;
  if (n > 0 && (!x || !M)) return err(MT_ERR_INVALID, "mt_server_submit: x and masses required");
  const size_t fp = footprint_of(*p);
  if (fp == 0) return err(MT_ERR_INVALID, "mt_server_submit: no workspace size for these params");
  if (fp > s->pool_bytes)
    return err(MT_ERR_WORKSPACE, "mt_server_submit: the request's footprint exceeds the pool");
  std::unique_ptr<Request> q(new (std::nothrow) Request());
  if (!q) return err(MT_ERR_INVALID, "mt_server_submit: out of host memory");
  q->id = s->next_id++;
  q->p = *p;
  q->steps = steps;
  q->footprint = fp;
  q->x.assign(x, x + m);
  q->M.assign(M, M + (size_t)r.species * n);
  q->t_submit = s->now();
  *id = q->id;
  s->queue.push_back(q.get());
  s->reqs[q->id] = std::move(q);
  return MT_OK;
}

mt_status mt_server_poll(mt_server* s, int32_t* queued, int32_t* running) {
  if (!s) return err(MT_ERR_INVALID, "mt_server_poll: server is NULL");
  // 1. retire finished chunks
  for (Slot& sl : s->slots) {
    Request* r = sl.req;
    if (!r) continue;
    const cudaError_t q = r->steps > 0 ? cudaEventQuery(sl.e1) : cudaSuccess;
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) {
      fail_request(s, r, err(MT_ERR_CUDA, "mt_server_poll: a request's stream failed"));
      continue;
    }
    if (r->steps > 0) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, sl.e0, sl.e1);
      r->gpu_ms += ms;
      s->step_ms.push_back(ms / (float)r->chunk);
      r->done += r->chunk;
      r->chunk = 0;
    }
    if (r->done >= r->steps) {
      finish(s, r);
    } else {
      const mt_status st = enqueue_chunk(s, r);
      if (st != MT_OK) fail_request(s, r, st);
    }
  }
  // 2. admit: oldest first; later ones too if backfill is on
  for (auto it = s->queue.begin(); it != s->queue.end();) {
    int k = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
      if (!s->slots[i].req) {
        k = (int)i;
        break;
      }
    if (k < 0) break;
    Request* r = *it;
    size_t at = 0;
    if (s->pool->alloc(r->footprint, &at)) {
      it = s->queue.erase(it);
      admit(s, r, k, at);
    } else if (s->cfg.backfill) {
      ++it;
    } else {
      break;
    }
  }
  int32_t run = 0;
  for (const Slot& sl : s->slots) run += sl.req ? 1 : 0;
  if (queued) *queued = (int32_t)s->queue.size();
  if (running) *running = run;
  return MT_OK;
}

mt_status mt_server_info(const mt_server* s, int64_t id, mt_request_info* info) {
  if (!s || !info) return err(MT_ERR_INVALID, "mt_server_info: NULL argument");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return err(MT_ERR_INVALID, "mt_server_info: unknown request");
  const Request& r = *it->second;
  std::memset(info, 0, sizeof *info);
  info->state = r.state;
  info->status = r.status;
  info->steps_done = r.done;
  info->t_submit = r.t_submit;
  info->t_admit = r.t_admit;
  info->t_done = r.t_done;
  info->gpu_ms = r.gpu_ms;
  info->footprint = r.footprint;
  return MT_OK;
}

mt_status mt_server_result(const mt_server* s, int64_t id, double* A, double* B,
                           double* observables, int64_t cap, int64_t* rows) {
  if (!s) return err(MT_ERR_INVALID, "mt_server_result: server is NULL");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return err(MT_ERR_INVALID, "mt_server_result: unknown request");
  const Request& r = *it->second;
  if (r.state == MT_REQ_FAILED) return err(r.status, "mt_server_result: the request failed");
  if (r.state != MT_REQ_DONE) return err(MT_ERR_STATE, "mt_server_result: request not finished");
  const size_t n = (size_t)r.p.n;
  if (n > 0 && (!A || !B)) return err(MT_ERR_INVALID, "mt_server_result: A and B required");
  if (n > 0) {
    std::memcpy(A, r.M.data(), n * 8);
    std::memcpy(B, r.M.data() + n, n * 8);
  }
  const int64_t have = (int64_t)(r.obs.size() / 4);
  const int64_t give = std::min<int64_t>(have, cap > 0 ? cap : 0);
  if (give > 0 && !observables) return err(MT_ERR_INVALID, "mt_server_result: observables NULL");
  if (give > 0) std::memcpy(observables, r.obs.data() + (size_t)(have - give) * 4, (size_t)give * 32);
  if (rows) *rows = give;
  return MT_OK;
}

mt_status mt_server_result_species(const mt_server* s, int64_t id, int32_t sp, double* out) {
  if (!s) return err(MT_ERR_INVALID, "mt_server_result_species: server is NULL");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return err(MT_ERR_INVALID, "mt_server_result_species: unknown request");
  const Request& r = *it->second;
  if (r.state == MT_REQ_FAILED) return err(r.status, "mt_server_result_species: the request failed");
  if (r.state != MT_REQ_DONE)
    return err(MT_ERR_STATE, "mt_server_result_species: request not finished");
  const size_t n = (size_t)r.p.n;
  if (sp < 0 || sp >= species_of(r.p))
    return err(MT_ERR_INVALID, "mt_server_result_species: species out of range");
  if (n > 0 && !out) return err(MT_ERR_INVALID, "mt_server_result_species: out is NULL");
  if (n > 0) std::memcpy(out, r.M.data() + (size_t)sp * n, n * 8);
  return MT_OK;
}

mt_status mt_server_release(mt_server* s, int64_t id) {
  if (!s) return err(MT_ERR_INVALID, "mt_server_release: server is NULL");
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return err(MT_ERR_INVALID, "mt_server_release: unknown request");
  if (it->second->state != MT_REQ_DONE && it->second->state != MT_REQ_FAILED)
    return err(MT_ERR_STATE, "mt_server_release: request still queued or running");
  s->reqs.erase(it);
  return MT_OK;
}

mt_status mt_server_stats(const mt_server* s, mt_server_summary* out, float* step_ms,
                          int64_t cap) {
  if (!s || !out) return err(MT_ERR_INVALID, "mt_server_stats: NULL argument");
  std::memset(out, 0, sizeof *out);
  out->pool_used = s->pool->used();
  out->pool_peak = s->pool->peak();
  out->step_samples = (int64_t)s->step_ms.size();
  for (const auto& kv : s->reqs) {
    const int st = kv.second->state;
    out->queued += st == MT_REQ_QUEUED;
    out->running += st == MT_REQ_RUNNING;
    out->done += st == MT_REQ_DONE;
    out->failed += st == MT_REQ_FAILED;
  }
  const int64_t give = std::min<int64_t>(cap > 0 ? cap : 0, out->step_samples);
  if (give > 0 && !step_ms) return err(MT_ERR_INVALID, "mt_server_stats: step_ms NULL");
  if (give > 0) std::memcpy(step_ms, s->step_ms.data(), (size_t)give * sizeof(float));
  return MT_OK;
}

void mt_server_destroy(mt_server* s) {
  if (!s) return;
  for (Slot& sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.req && sl.req->h) mt_destroy(sl.req->h);
    if (sl.e0) cudaEventDestroy(sl.e0);
    if (sl.e1) cudaEventDestroy(sl.e1);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

}  // extern "C"
