// Serving (declarations and contracts in include/nbldpc.h): the continuous-
// batching scheduler and the CUDA executor behind nbldpc_server_*.
//
// The scheduler is host logic only: queues, a resident-bytes budget, a fixed
// set of streams.  nbldpc_server_poll runs one round: retire launches whose
// executor reports completion, admit waiting requests in arrival order while
// they fit the budget, and start one launch per free stream with up to
// max_jobs admitted requests.  The CUDA executor works through the library's
// public calls (nbldpc_decode_batch / nbldpc_decode and their workspace
// sizes), the stream-ordered allocator and one event per launch; nothing on
// the device ever waits for the host.
#include "nbldpc.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// ---------------------------------------------------------------- CUDA executor
struct CudaExec {
  int device = 0;
  std::vector<cudaStream_t> streams;
  // the server's own stream-ordered pool: it keeps up to the budget mapped
  // between launches (the default pool returns freed memory to the system at
  // synchronizations, and mapping it again stalled the next launches)
  cudaMemPool_t pool = nullptr;
  struct Launch {
    cudaEvent_t ev = nullptr;
  };
  std::unordered_map<uint64_t, Launch> launches;
  uint64_t next = 1;

  ~CudaExec() {
    for (auto& kv : launches) {
      cudaEventSynchronize(kv.second.ev);
      cudaEventDestroy(kv.second.ev);
    }
    for (cudaStream_t s : streams) cudaStreamDestroy(s);
    if (pool) cudaMemPoolDestroy(pool);
  }

  static int shape(const nbldpc_request* r, int* n, int* q) {
    return nbldpc_code_info(r->code, q, n, nullptr, nullptr);
  }

  // device bytes of one request: reliabilities and outputs, 256-byte sections
  static size_t request_bytes(void*, const nbldpc_request* r) {
    int n = 0, q = 0;
    if (shape(r, &n, &q) != NBLDPC_OK) return 0;
    const size_t f = (size_t)r->frames;
    return round_up(f * n * q, 256) + round_up(f * n, 256) + round_up(f * 4, 256) + round_up(f, 256);
  }

  static size_t launch_bytes(void*, const nbldpc_request* const* reqs, int n, int plain) {
    size_t b = 0;
    if (plain) {
      for (int i = 0; i < n; ++i) {
        size_t w = 0;
        if (nbldpc_decode_workspace_size(reqs[i]->code, reqs[i]->frames, &w) != NBLDPC_OK) return 0;
        b += round_up(w, 256);
      }
      return b;
    }
    nbldpc_job jobs[NBLDPC_MAX_BATCH_JOBS];
    for (int i = 0; i < n; ++i) {
      jobs[i] = nbldpc_job{reqs[i]->code, nullptr, reqs[i]->frames, reqs[i]->max_iters, reqs[i]->early_stop,
                           nullptr, nullptr, nullptr};
    }
    if (nbldpc_decode_batch_workspace_size(jobs, n, &b) != NBLDPC_OK) return 0;
    return round_up(b, 256);
  }

  static int start(void* ctx, const nbldpc_request* const* reqs, int n, int stream, int plain, uint64_t* token) {
    CudaExec* ex = static_cast<CudaExec*>(ctx);
    cudaStream_t st = ex->streams[(size_t)stream % ex->streams.size()];
    if (cudaSetDevice(ex->device) != cudaSuccess) return NBLDPC_ERR_CUDA;
    // one allocation per launch: per request reliabilities + outputs, then the workspace(s)
    std::vector<size_t> off(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
      off[i] = total;
      total += request_bytes(nullptr, reqs[i]);
    }
    const size_t ws_off = total;
    const size_t wsb = launch_bytes(nullptr, reqs, n, plain);
    total += wsb;
    unsigned char* buf = nullptr;
    if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&buf), total, ex->pool, st) != cudaSuccess)
      return NBLDPC_ERR_NOMEM;
    nbldpc_job jobs[NBLDPC_MAX_BATCH_JOBS];
    size_t ws_cur = ws_off;
    int status = NBLDPC_OK;
    for (int i = 0; i < n && status == NBLDPC_OK; ++i) {
      const nbldpc_request* r = reqs[i];
      int nc = 0, q = 0;
      shape(r, &nc, &q);
      const size_t f = (size_t)r->frames;
      unsigned char* g = buf + off[i];
      uint8_t* sym = g + round_up(f * nc * q, 256);
      int32_t* its = reinterpret_cast<int32_t*>(sym + round_up(f * nc, 256));
      uint8_t* ok = reinterpret_cast<uint8_t*>(its) + round_up(f * 4, 256);
      if (cudaMemcpyAsync(g, r->gamma_host, f * nc * q, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        status = NBLDPC_ERR_CUDA;
        break;
      }
      if (plain) {
        size_t w = 0;
        nbldpc_decode_workspace_size(r->code, r->frames, &w);
        status = nbldpc_decode(r->code, g, r->frames, r->max_iters, 0, sym, its, ok, buf + ws_cur, w, st);
        ws_cur += round_up(w, 256);
      }
      jobs[i] = nbldpc_job{r->code, g, r->frames, r->max_iters, r->early_stop, sym, its, ok};
    }
    if (status == NBLDPC_OK && !plain) status = nbldpc_decode_batch(jobs, n, buf + ws_off, wsb, st);
    for (int i = 0; i < n && status == NBLDPC_OK; ++i) {
      const nbldpc_request* r = reqs[i];
      int nc = 0, q = 0;
      shape(r, &nc, &q);
      const size_t f = (size_t)r->frames;
      if (cudaMemcpyAsync(r->out_sym_host, jobs[i].out_sym_dev, f * nc, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
          cudaMemcpyAsync(r->out_iters_host, jobs[i].out_iters_dev, f * 4, cudaMemcpyDeviceToHost, st) !=
              cudaSuccess ||
          cudaMemcpyAsync(r->out_ok_host, jobs[i].out_ok_dev, f, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        status = NBLDPC_ERR_CUDA;
    }
    // the buffer returns to the pool once the stream has passed the copies out
    if (cudaFreeAsync(buf, st) != cudaSuccess && status == NBLDPC_OK) status = NBLDPC_ERR_CUDA;
    if (status != NBLDPC_OK) return status;
    Launch l;
    if (cudaEventCreateWithFlags(&l.ev, cudaEventDisableTiming) != cudaSuccess) return NBLDPC_ERR_CUDA;
    if (cudaEventRecord(l.ev, st) != cudaSuccess) {
      cudaEventDestroy(l.ev);
      return NBLDPC_ERR_CUDA;
    }
    *token = ex->next++;
    ex->launches[*token] = l;
    return NBLDPC_OK;
  }

  static int done(void* ctx, uint64_t token) {
    CudaExec* ex = static_cast<CudaExec*>(ctx);
    auto it = ex->launches.find(token);
    if (it == ex->launches.end()) return NBLDPC_ERR_ARG;
    const cudaError_t e = cudaEventQuery(it->second.ev);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return NBLDPC_ERR_CUDA;
  }

  static int finish(void* ctx, uint64_t token) {
    CudaExec* ex = static_cast<CudaExec*>(ctx);
    auto it = ex->launches.find(token);
    if (it == ex->launches.end()) return NBLDPC_ERR_ARG;
    const cudaError_t e = cudaEventSynchronize(it->second.ev);
    cudaEventDestroy(it->second.ev);
    ex->launches.erase(it);
    return e == cudaSuccess ? NBLDPC_OK : NBLDPC_ERR_CUDA;
  }
};

struct InFlight {
  std::vector<uint64_t> ids;
  uint64_t token;
  size_t reserved;   // workspace + the requests' bytes
  int stream;
};

}  // namespace

struct nbldpc_server {
  nbldpc_server_executor ex{};
  CudaExec* cuda = nullptr;           // owned when created by nbldpc_server_create
  size_t budget = 0;
  int streams = 1, max_jobs = 1, plain = 0;
  std::unordered_map<uint64_t, nbldpc_request> reqs;   // submitted, not yet returned by poll
  std::unordered_map<uint64_t, size_t> req_bytes;
  std::deque<uint64_t> waiting, admitted, done;
  std::vector<InFlight> inflight;
  size_t used = 0, peak = 0;
  uint64_t launches = 0, submitted = 0, completed = 0, next_id = 1;
};

namespace {

int make_server(const nbldpc_server_executor& ex, size_t budget, int streams, int max_jobs, int plain,
                nbldpc_server** out) {
  if (!out) return NBLDPC_ERR_ARG;
  *out = nullptr;
  if (streams < 1 || max_jobs < 1 || max_jobs > NBLDPC_MAX_BATCH_JOBS || budget == 0) return NBLDPC_ERR_ARG;
  if (!ex.request_bytes || !ex.launch_bytes || !ex.start || !ex.done || !ex.finish) return NBLDPC_ERR_ARG;
  nbldpc_server* s = new (std::nothrow) nbldpc_server();
  if (!s) return NBLDPC_ERR_NOMEM;
  s->ex = ex;
  s->budget = budget;
  s->plain = plain ? 1 : 0;
  s->streams = s->plain ? 1 : streams;        // plain: one stream, one request per launch
  s->max_jobs = s->plain ? 1 : max_jobs;
  *out = s;
  return NBLDPC_OK;
}

}  // namespace

extern "C" {

int nbldpc_server_create_custom(const nbldpc_server_executor* executor, size_t budget_bytes, int streams,
                                int max_jobs, int plain, nbldpc_server** out) {
  if (!executor) return NBLDPC_ERR_ARG;
  return make_server(*executor, budget_bytes, streams, max_jobs, plain, out);
}

int nbldpc_server_create(size_t budget_bytes, int streams, int max_jobs, int plain, nbldpc_server** out) {
  if (!out) return NBLDPC_ERR_ARG;
  *out = nullptr;
  if (streams < 1) return NBLDPC_ERR_ARG;
  CudaExec* cx = new (std::nothrow) CudaExec();
  if (!cx) return NBLDPC_ERR_NOMEM;
  if (cudaGetDevice(&cx->device) != cudaSuccess) {
    delete cx;
    return NBLDPC_ERR_CUDA;
  }
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = cx->device;
  uint64_t keep = budget_bytes;
  if (cudaMemPoolCreate(&cx->pool, &props) != cudaSuccess ||
      cudaMemPoolSetAttribute(cx->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    delete cx;
    return NBLDPC_ERR_CUDA;
  }
  const int ns = plain ? 1 : streams;
  for (int i = 0; i < ns; ++i) {
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      delete cx;
      return NBLDPC_ERR_CUDA;
    }
    cx->streams.push_back(st);
  }
  nbldpc_server_executor ex{cx, &CudaExec::request_bytes, &CudaExec::launch_bytes, &CudaExec::start,
                            &CudaExec::done, &CudaExec::finish};
  const int st = make_server(ex, budget_bytes, streams, max_jobs, plain, out);
  if (st != NBLDPC_OK) {
    delete cx;
    return st;
  }
  (*out)->cuda = cx;
  return NBLDPC_OK;
}

int nbldpc_server_submit(nbldpc_server* s, const nbldpc_request* req, uint64_t* id) {
  if (!s || !req || !id || req->frames < 1 || req->max_iters < 0) return NBLDPC_ERR_ARG;
  // the CUDA executor reads the code and the host buffers; a custom executor keeps its own
  if (s->cuda && (!req->code || !req->gamma_host || !req->out_sym_host || !req->out_iters_host || !req->out_ok_host))
    return NBLDPC_ERR_ARG;
  nbldpc_request r = *req;
  r.id = s->next_id++;
  s->reqs[r.id] = r;
  s->req_bytes[r.id] = s->ex.request_bytes(s->ex.ctx, &s->reqs[r.id]);
  s->waiting.push_back(r.id);
  ++s->submitted;
  *id = r.id;
  return NBLDPC_OK;
}

int nbldpc_server_poll(nbldpc_server* s, uint64_t* done_ids, int capacity, int* n_done) {
  if (!s || capacity < 0 || (capacity > 0 && !done_ids)) return NBLDPC_ERR_ARG;
  // retire launches whose copies out have completed
  for (size_t i = 0; i < s->inflight.size();) {
    InFlight& l = s->inflight[i];
    const int d = s->ex.done(s->ex.ctx, l.token);
    if (d < 0) return d;
    if (d == 0) {
      ++i;
      continue;
    }
    const int f = s->ex.finish(s->ex.ctx, l.token);
    if (f != NBLDPC_OK) return f;
    s->used -= l.reserved;
    for (uint64_t id : l.ids) s->done.push_back(id);
    s->inflight.erase(s->inflight.begin() + (long)i);
  }
  // admission in arrival order against the budget (a request larger than the
  // whole budget goes alone once nothing else is resident)
  while (!s->waiting.empty()) {
    const uint64_t id = s->waiting.front();
    const size_t b = s->req_bytes[id];
    if (s->used + b > s->budget && (s->used > 0 || !s->admitted.empty())) break;
    s->waiting.pop_front();
    s->used += b;
    s->admitted.push_back(id);
  }
  s->peak = std::max(s->peak, s->used);
  // one launch per free stream
  std::vector<char> busy((size_t)s->streams, 0);
  for (const InFlight& l : s->inflight) busy[(size_t)l.stream] = 1;
  for (int st = 0; st < s->streams && !s->admitted.empty(); ++st) {
    if (busy[(size_t)st]) continue;
    std::vector<uint64_t> group;
    std::vector<const nbldpc_request*> rp;
    while (!s->admitted.empty() && (int)group.size() < s->max_jobs) {
      group.push_back(s->admitted.front());
      s->admitted.pop_front();
      rp.push_back(&s->reqs[group.back()]);
    }
    const size_t wb = s->ex.launch_bytes(s->ex.ctx, rp.data(), (int)rp.size(), s->plain);
    if (s->used + wb > s->budget && !s->inflight.empty()) {
      for (auto it = group.rbegin(); it != group.rend(); ++it) s->admitted.push_front(*it);
      break;
    }
    uint64_t token = 0;
    const int rc = s->ex.start(s->ex.ctx, rp.data(), (int)rp.size(), st, s->plain, &token);
    if (rc != NBLDPC_OK) {
      for (auto it = group.rbegin(); it != group.rend(); ++it) s->admitted.push_front(*it);
      return rc;
    }
    size_t rb = 0;
    for (uint64_t id : group) rb += s->req_bytes[id];
    // the requests' bytes were counted at admission and now belong to the launch
    s->used += wb;
    s->peak = std::max(s->peak, s->used);
    s->inflight.push_back(InFlight{group, token, wb + rb, st});
    ++s->launches;
    busy[(size_t)st] = 1;
  }
  int n = 0;
  while (n < capacity && !s->done.empty()) {
    const uint64_t id = s->done.front();
    s->done.pop_front();
    done_ids[n++] = id;
    s->reqs.erase(id);
    s->req_bytes.erase(id);
    ++s->completed;
  }
  if (n_done) *n_done = n;
  return NBLDPC_OK;
}

int nbldpc_server_stats_get(const nbldpc_server* s, nbldpc_server_stats* out) {
  if (!s || !out) return NBLDPC_ERR_ARG;
  out->used_bytes = s->used;
  out->peak_bytes = s->peak;
  out->launches = s->launches;
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->waiting = (int)s->waiting.size();
  out->admitted = (int)s->admitted.size();
  out->in_flight = (int)s->inflight.size();
  return NBLDPC_OK;
}

void nbldpc_server_destroy(nbldpc_server* s) {
  if (!s) return;
  for (InFlight& l : s->inflight) s->ex.finish(s->ex.ctx, l.token);
  delete s->cuda;
  delete s;
}

}  // extern "C"
