// Continuous-batching server of libmsrcg.
//
// Requests (one linear system each: grid, cell permeability, boundary types,
// right-hand side, tolerance) are admitted while their estimated device
// memory fits a budget; an admitted request gets its own level hierarchy
// (built stream ordered, so building never waits for solves in flight) and
// stays resident until its result is copied back.  Every call to progress()
// launches the requests admitted since the last launch as one batched wave
// (one CTA per request, the single-CTA recursive solver), on a stream of its
// own: waves overlap on the device, so a request that arrives while others
// run starts as soon as it is built instead of waiting for them.  Finished
// waves release their requests' memory, which admits waiting requests.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <vector>

#include "msrcg_internal.cuh"

using namespace msrcg;

namespace {

struct Request {
  int64_t id = 0;
  int state = 0;  // 0 waiting, 1 built, 2 launched, 3 done
  int status = MSRCG_OK;
  msrcg_grid grid{};
  int ncomp = 1;
  long long N = 0;
  const double* K_host = nullptr;
  const uint8_t* bc_host = nullptr;
  const double* b_host = nullptr;
  double* x_host = nullptr;
  double tol = 1e-8;
  size_t bytes = 0;
  msrcg_hier* h = nullptr;
  double* d_b = nullptr;
  double* d_x = nullptr;
  msrcg_stats stats{};
};

constexpr int kWaveCap = 1024;  // requests per wave

struct Wave {
  cudaStream_t s = nullptr;
  cudaEvent_t ev = nullptr;
  std::vector<int64_t> ids;
  SolveState* states = nullptr;  // pinned, kWaveCap entries
  bool busy = false;
};

int boundary_faces(const msrcg_grid& g) {
  const long long nx = g.n[0], ny = g.n[1], nz = g.dim == 3 ? g.n[2] : 1;
  return (int)(2 * (ny * nz + nx * nz) + (g.dim == 3 ? 2 * nx * ny : 0));
}

// Device bytes a request will hold: its hierarchy (the build's own
// allocation plan) plus its right-hand side and solution.
size_t estimate_bytes(const msrcg_grid& g, const msrcg_opts& o) {
  const size_t N = (size_t)g.n[0] * g.n[1] * (g.dim == 3 ? g.n[2] : 1);
  return msrcg_build_bytes(&g, &o) + 16 * N;
}

}  // namespace

struct msrcg_server {
  size_t budget = 0, used = 0;
  msrcg_opts opts{};
  int device = 0;
  int64_t next_id = 1;
  std::deque<int64_t> waiting;
  std::map<int64_t, Request> reqs;
  std::vector<Wave> waves;
  cudaStream_t build_stream = nullptr;
};

namespace {

// Release a finished or failed request's device memory (stream ordered).
void drop_device(msrcg_server* sv, Request& r, cudaStream_t s) {
  if (r.d_b) cudaFreeAsync(r.d_b, s);
  if (r.d_x) cudaFreeAsync(r.d_x, s);
  r.d_b = r.d_x = nullptr;
  if (r.h) {
    r.h->alloc_stream = s;
    msrcg_free(r.h);
    r.h = nullptr;
  }
  sv->used -= std::min(sv->used, r.bytes);
}

// Stage a request's inputs on the device (K and the boundary mask into the
// caller's temporaries *dK, *dbc; b and the solution buffer into the
// request) and build its hierarchy.
int stage_and_build(msrcg_server* sv, Request& r, void** dK, void** dbc) {
  cudaStream_t s = sv->build_stream;
  const int nbf = boundary_faces(r.grid);
  MSRCG_CUDA_TRY(cudaMallocAsync(dK, sizeof(double) * r.N * r.ncomp, s));
  MSRCG_CUDA_TRY(cudaMallocAsync(dbc, (size_t)nbf, s));
  MSRCG_CUDA_TRY(cudaMallocAsync((void**)&r.d_b, sizeof(double) * r.N, s));
  MSRCG_CUDA_TRY(cudaMallocAsync((void**)&r.d_x, sizeof(double) * r.N, s));
  MSRCG_CUDA_TRY(cudaMemcpyAsync(*dK, r.K_host, sizeof(double) * r.N * r.ncomp, cudaMemcpyHostToDevice, s));
  MSRCG_CUDA_TRY(cudaMemcpyAsync(*dbc, r.bc_host, (size_t)nbf, cudaMemcpyHostToDevice, s));
  MSRCG_CUDA_TRY(cudaMemcpyAsync(r.d_b, r.b_host, sizeof(double) * r.N, cudaMemcpyHostToDevice, s));
  return msrcg_build_ex(&r.grid, (const double*)*dK, r.ncomp, (const uint8_t*)*dbc, &sv->opts, s, s, &r.h);
}

// Build the hierarchy of a waiting request and stage its right-hand side.
// The temporaries are freed on every path; on failure the caller releases
// the request's own buffers (drop_device).
int admit(msrcg_server* sv, Request& r) {
  void *dK = nullptr, *dbc = nullptr;
  const int rc = stage_and_build(sv, r, &dK, &dbc);
  if (dK) cudaFreeAsync(dK, sv->build_stream);
  if (dbc) cudaFreeAsync(dbc, sv->build_stream);
  if (rc) {
    r.h = nullptr;
    return rc;
  }
  // the builder synchronised the build stream: the hierarchy and the staged
  // right-hand side are ready for any other stream.  The request was charged
  // its estimate; when the measured size is larger, charge the difference
  // too, so that releasing r.bytes later returns exactly what was charged.
  const size_t measured = r.h->bytes + (size_t)(16 * r.N);
  if (measured > r.bytes) {
    sv->used += measured - r.bytes;
    r.bytes = measured;
  }
  return MSRCG_OK;
}

int retire(msrcg_server* sv) {
  for (Wave& w : sv->waves) {
    if (!w.busy) continue;
    cudaError_t q = cudaEventQuery(w.ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return msrcg_cuda_fail(q, "cudaEventQuery", __FILE__, __LINE__);
    std::vector<msrcg_hier*> hs;
    for (int64_t id : w.ids) hs.push_back(sv->reqs[id].h);
    std::vector<msrcg_stats> st(hs.size());
    msrcg_batch_finish((int)hs.size(), hs.data(), w.states, st.data());
    for (size_t i = 0; i < w.ids.size(); ++i) {
      Request& r = sv->reqs[w.ids[i]];
      r.stats = st[i];
      r.status = st[i].status;
      if (r.status == MSRCG_ENOCONV && r.h->o.precision == 1 && r.h->o.escalate) {
        // the FP32 preconditioner did not get there: solve this request again
        // with the FP64 one (the host waits for it; rare by design)
        msrcg_hier* tw = nullptr;
        if (msrcg_twin(r.h, w.s, &tw) == MSRCG_OK) {
          const int flexible = r.stats.flexible;
          msrcg_solve(tw, r.d_b, r.tol, r.d_x, &r.stats, w.s);
          r.stats.flexible = flexible;
          r.stats.escalated = 1;
          r.status = r.stats.status;
        }
      }
      // the wave has finished: copy the solution into the caller's buffer
      cudaError_t e = cudaMemcpy(r.x_host, r.d_x, sizeof(double) * r.N, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess && r.status == MSRCG_OK) r.status = msrcg_cuda_fail(e, "cudaMemcpy", __FILE__, __LINE__);
      r.state = 3;
      drop_device(sv, r, w.s);
    }
    w.ids.clear();
    w.busy = false;
  }
  return MSRCG_OK;
}

// Launch every built request of one dimension as one wave.
int launch(msrcg_server* sv, int dim) {
  // built requests of this dimension (and the first one's tolerance), in order
  std::vector<int64_t> ids;
  double tol = 0.0;
  for (auto& kv : sv->reqs) {
    const Request& r = kv.second;
    if (r.state != 1 || r.grid.dim != dim) continue;
    if (ids.empty()) tol = r.tol;
    if (r.tol != tol || (int)ids.size() >= kWaveCap) continue;
    ids.push_back(kv.first);
  }
  if (ids.empty()) return MSRCG_OK;
  Wave* w = nullptr;
  for (Wave& c : sv->waves)
    if (!c.busy) {
      w = &c;
      break;
    }
  if (!w) return MSRCG_OK;  // every stream busy: the requests go with a later wave
  std::vector<msrcg_hier*> hs;
  std::vector<const double*> bs;
  std::vector<double*> xs;
  for (int64_t id : ids) {
    Request& r = sv->reqs[id];
    hs.push_back(r.h);
    bs.push_back(r.d_b);
    xs.push_back(r.d_x);
  }
  int rc = msrcg_batch_enqueue((int)ids.size(), hs.data(), bs.data(), tol, xs.data(), w->s, w->states);
  if (rc) return rc;
  for (int64_t id : ids) sv->reqs[id].state = 2;
  MSRCG_CUDA_TRY(cudaEventRecord(w->ev, w->s));
  w->ids = ids;
  w->busy = true;
  return MSRCG_OK;
}

}  // namespace

extern "C" int msrcg_server_create(size_t budget_bytes, int max_waves, const msrcg_opts* opts, msrcg_server** out) {
  if (!out || budget_bytes == 0) return MSRCG_EINVAL;
  *out = nullptr;
  msrcg_server* sv = new msrcg_server();
  sv->budget = budget_bytes;
  if (opts) sv->opts = *opts;
  else msrcg_default_opts(&sv->opts);
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    delete sv;
    return MSRCG_ECUDA;
  }
  const int nw = max_waves > 0 ? max_waves : 8;
  sv->waves.resize(nw);
  bool ok = cudaStreamCreateWithFlags(&sv->build_stream, cudaStreamNonBlocking) == cudaSuccess;
  for (Wave& w : sv->waves) {
    ok = ok && cudaStreamCreateWithFlags(&w.s, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&w.ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMallocHost((void**)&w.states, sizeof(SolveState) * kWaveCap) == cudaSuccess;
  }
  if (!ok) {
    msrcg_server_destroy(sv);
    return MSRCG_ECUDA;
  }
  *out = sv;
  return MSRCG_OK;
}

extern "C" int msrcg_server_submit(msrcg_server* sv, const msrcg_grid* grid, const double* K, int ncomp,
                                   const uint8_t* bc, const double* b, double tol, double* x, int64_t* id) {
  if (!sv || !grid || !K || !bc || !b || !x || !id || !(tol > 0.0) || !isfinite(tol)) return MSRCG_EINVAL;
  if (grid->dim != 2 && grid->dim != 3) return MSRCG_EINVAL;
  for (int a = 0; a < grid->dim; ++a)
    if (grid->n[a] < 1) return MSRCG_EINVAL;
  if (ncomp != 1 && ncomp != grid->dim) return MSRCG_EINVAL;
  Request r;
  r.id = sv->next_id++;
  r.grid = *grid;
  if (r.grid.dim == 2) {
    r.grid.n[2] = 1;
    r.grid.h[2] = 1.0;
  }
  r.ncomp = ncomp;
  r.N = (long long)r.grid.n[0] * r.grid.n[1] * r.grid.n[2];
  r.K_host = K;
  r.bc_host = bc;
  r.b_host = b;
  r.x_host = x;
  r.tol = tol;
  r.bytes = estimate_bytes(r.grid, sv->opts);
  if (r.bytes == 0) return MSRCG_EINVAL;
  if (r.bytes > sv->budget) return MSRCG_ENOMEM;
  sv->reqs[r.id] = r;
  sv->waiting.push_back(r.id);
  *id = r.id;
  return msrcg_server_progress(sv) < 0 ? MSRCG_ECUDA : MSRCG_OK;
}

extern "C" int msrcg_server_progress(msrcg_server* sv) {
  if (!sv) return MSRCG_EINVAL;
  int rc = retire(sv);
  if (rc) return rc;
  // admit in arrival order while the budget allows
  while (!sv->waiting.empty()) {
    Request& r = sv->reqs[sv->waiting.front()];
    if (sv->used + r.bytes > sv->budget) break;
    sv->used += r.bytes;
    sv->waiting.pop_front();
    rc = admit(sv, r);
    if (rc) {
      r.status = rc;
      r.state = 3;
      drop_device(sv, r, sv->build_stream);
      continue;
    }
    r.state = 1;
  }
  rc = launch(sv, 2);
  if (!rc) rc = launch(sv, 3);
  if (rc) return rc;
  int inflight = 0;
  for (auto& kv : sv->reqs) inflight += kv.second.state < 3;
  return inflight;
}

extern "C" int msrcg_server_poll(msrcg_server* sv, int64_t id, msrcg_stats* stats) {
  if (!sv) return MSRCG_EINVAL;
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return MSRCG_EINVAL;
  if (it->second.state != 3) {
    int rc = msrcg_server_progress(sv);
    if (rc < 0) return rc;
    it = sv->reqs.find(id);
  }
  if (it->second.state != 3) return 0;
  if (stats) *stats = it->second.stats;
  const int status = it->second.status;
  sv->reqs.erase(it);
  return status == MSRCG_OK ? 1 : status;
}

extern "C" int msrcg_server_drain(msrcg_server* sv) {
  if (!sv) return MSRCG_EINVAL;
  for (;;) {
    int n = msrcg_server_progress(sv);
    if (n < 0) return n;
    bool busy = false;
    for (Wave& w : sv->waves) busy = busy || w.busy;
    bool pending = false;
    for (auto& kv : sv->reqs) pending = pending || kv.second.state < 3;
    if (!pending) return MSRCG_OK;
    if (busy) {
      for (Wave& w : sv->waves)
        if (w.busy) {
          cudaEventSynchronize(w.ev);
          break;
        }
    }
  }
}

extern "C" size_t msrcg_server_bytes_in_use(const msrcg_server* sv) { return sv ? sv->used : 0; }

extern "C" void msrcg_server_destroy(msrcg_server* sv) {
  if (!sv) return;
  cudaDeviceSynchronize();
  retire(sv);
  for (auto& kv : sv->reqs) drop_device(sv, kv.second, sv->build_stream);
  cudaStreamSynchronize(sv->build_stream);
  for (Wave& w : sv->waves) {
    if (w.states) cudaFreeHost(w.states);
    if (w.ev) cudaEventDestroy(w.ev);
    if (w.s) cudaStreamDestroy(w.s);
  }
  if (sv->build_stream) cudaStreamDestroy(sv->build_stream);
  (void)cudaGetLastError();
  delete sv;
}
