// ibm_serve.cu -- the serving layer: many independent cases resident on one
// GPU at once (continuous batching).  Host code on top of the lattice ABI.
//
// A case waits in a FIFO until the device-memory budget, a free slot and the
// correction-kernel CTA budget admit it.  An admitted case owns a lattice
// handle and a stream, and is advanced in chunks of steps (CUDA-graph
// replays of one step each), so the kernels of different cases run side by
// side.  Completion of a chunk is seen through an event, never by blocking.
// The CTA budget matters because a correction kernel with more than one CTA
// keeps all its CTAs resident while it waits at its grid barrier: with the
// sum of such CTAs held below the device's capacity, every launched
// correction kernel can become fully resident.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "ibm_internal.h"

using ibm::kBandCap;
using ibm::kForceChunk;
using ibm::kGCap;
using ibm::kSmallIbMarkers;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { CASE_PENDING = 0, CASE_ACTIVE = 1, CASE_DONE = 2, CASE_FAILED = 3 };

struct CaseRec {
  long long id = 0;
  ibm_lattice_desc desc{};
  std::vector<ibm_body_desc> bodies;
  std::vector<int> nmark;
  std::vector<double> xy, ds;
  bool has_ds = false;
  int nsteps = 0, remaining = 0;
  unsigned outputs = 0;
  double bytes = 0.0;
  int ib_ctas = 1;
  int ib_budget = 0;          // CTAs counted against the budget (grid-barrier launches only)
  ibm_handle h = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};   // ring of chunk-completion events
  int head = 0, inflight = 0;
  double t_submit = 0.0, t_done = 0.0;
  int state = CASE_PENDING;
  ibm_status status = IBM_OK;
  std::string err;
  std::vector<double> rho, ux, uy, bodies_out, resid;
};

// Device bytes one case needs (the allocations of ibm_create_lattice,
// ibm_add_markers and the first field read).
double case_bytes(const ibm_lattice_desc& d, int M, int nb) {
  const double s = d.prec == IBM_FP64 ? 8 : (d.prec == IBM_FP32 ? 4 : 2);
  const double r = d.prec == IBM_FP64 ? 8 : 4;
  const double nxp = (double)((d.nx + 31) / 32 * 32);
  const double nodes = (double)d.nx * d.ny;
  const double ent = d.prec == IBM_FP64 ? 16 : 8;
  const double bcap = 16.0 * M;
  double b = 9.0 * d.ny * nxp * s + 3.0 * nodes * r + 4.0 * nodes + 4.0 * (nxp / 32) * d.ny;
  b += 24.0 * nodes;                                        // staging of rho, ux, uy reads
  b += M * (5 * 8.0 + 4 + 2 * r + 16 * (r + 12) + 4 * r + 3 * r + kGCap * ent + 4);
  b += M * 2.0 * r * (d.n_corr + 1);
  b += bcap * (8 + kBandCap * ent + 8 * r + 4);
  b += nb * (sizeof(ibm::BodyDev) + 24.0 * (M / kForceChunk + 1));
  return b + (1 << 20);
}

// Correction-loop CTAs of a served case: one CTA per `per_cta` markers, at
// most ibm::kMaxIbCluster, so that every multi-CTA correction kernel can run
// as one thread-block cluster (CTAs scheduled together, hardware barrier)
// and many cases' correction kernels are resident at once.
constexpr int kServeMarkersPerCta = 512;
int server_ib_ctas(int M, int per_cta) {
  if (M == 0) return 0;
  if (per_cta <= 0) per_cta = kServeMarkersPerCta;
  return std::max(1, std::min(ibm::kMaxIbCluster, (M + per_cta - 1) / per_cta));
}

}  // namespace

struct ibm_server_s {
  ibm_server_desc desc{};
  int sms = 0;
  double budget = 0.0;
  int cta_budget = 0;
  std::deque<long long> pending;
  std::map<long long, CaseRec*> cases;
  std::vector<long long> active;
  std::vector<cudaStream_t> streams;       // idle streams for reuse
  std::vector<cudaEvent_t> events;
  cudaMemPool_t pool = nullptr;
  int max_cluster[4] = {-1, -1, -1, -1};     // per precision, from ibm::ib_max_cluster
  double bytes_in_use = 0.0;
  int ctas_in_use = 0;
  long long next_id = 1;
  long long submitted = 0, completed = 0, failed = 0;
  std::vector<double> tts_ms;
  double t_first = -1.0, t_last = 0.0;
  double lattice_updates = 0.0;
  double t_admit = 0.0, t_launch = 0.0, t_harvest = 0.0;   // host seconds
  std::string err;
};

namespace {

ibm_status sfail(ibm_server s, ibm_status st, const std::string& m) {
  if (s) s->err = m;
  ibm::set_thread_error(m.c_str());
  return st;
}

void case_fail(ibm_server s, CaseRec* c, ibm_status st, const char* where) {
  c->state = CASE_FAILED;
  c->status = st;
  c->err = std::string(where) + ": " + (c->h ? ibm_last_error(c->h) : ibm_last_error(nullptr));
  s->failed++;
}

void release_device(ibm_server s, CaseRec* c) {
  if (c->h) { ibm_destroy(c->h); c->h = nullptr; }
  if (c->stream) { s->streams.push_back(c->stream); c->stream = nullptr; }
  for (auto& e : c->ev)
    if (e) { s->events.push_back(e); e = nullptr; }
  s->bytes_in_use -= c->bytes;
  s->ctas_in_use -= c->ib_budget;
  s->active.erase(std::remove(s->active.begin(), s->active.end(), c->id), s->active.end());
}

ibm_status launch_chunk(ibm_server s, CaseRec* c) {
  const int n = std::min(c->remaining, s->desc.steps_per_launch);
  const bool last = n == c->remaining;
  const unsigned flags = (last && (c->outputs & IBM_OUT_MACRO)) ? IBM_STEP_DEFAULT : IBM_STEP_NO_MACRO;
  ibm_status st = ibm_step(c->h, n, flags);
  if (st != IBM_OK) return st;
  c->remaining -= n;
  if (cudaEventRecord(c->ev[(c->head + c->inflight) & 1], c->stream) != cudaSuccess) {
    cudaGetLastError();
    return IBM_ERR_CUDA;
  }
  c->inflight++;
  return IBM_OK;
}

// Keep up to two chunks of the case queued on its stream.
ibm_status top_up(ibm_server s, CaseRec* c) {
  while (c->remaining > 0 && c->inflight < 2) {
    ibm_status st = launch_chunk(s, c);
    if (st != IBM_OK) return st;
  }
  return IBM_OK;
}

ibm_status admit(ibm_server s, CaseRec* c) {
  if (!s->streams.empty()) { c->stream = s->streams.back(); s->streams.pop_back(); }
  else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    c->stream = nullptr;
    return IBM_ERR_CUDA;
  }
  for (auto& e : c->ev) {
    if (!s->events.empty()) { e = s->events.back(); s->events.pop_back(); }
    else if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      e = nullptr;
      return IBM_ERR_CUDA;
    }
  }
  c->head = 0;
  c->inflight = 0;
  ibm_lattice_desc d = c->desc;
  d.cuda_stream = c->stream;
  d.device = s->desc.device;
  ibm_status st = ibm::create_lattice(&d, &c->h, s->pool);
  if (st != IBM_OK) return st;
  if (c->ib_ctas > 0 && (st = ibm_set_option(c->h, IBM_OPT_IB_CTAS, c->ib_ctas)) != IBM_OK) return st;
  size_t off = 0;
  for (size_t b = 0; b < c->bodies.size(); ++b) {
    st = ibm_add_markers(c->h, c->xy.data() + 2 * off, c->has_ds ? c->ds.data() + off : nullptr,
                         c->nmark[b], &c->bodies[b], nullptr);
    if (st != IBM_OK) return st;
    off += c->nmark[b];
  }
  return top_up(s, c);
}

ibm_status harvest(ibm_server s, CaseRec* c) {
  const size_t n = (size_t)c->desc.nx * c->desc.ny;
  ibm_status st = IBM_OK;
  if (c->outputs & IBM_OUT_MACRO) {
    c->rho.resize(n); c->ux.resize(n); c->uy.resize(n);
    if ((st = ibm_read_fields(c->h, IBM_FIELD_RHO, c->rho.data(), n)) != IBM_OK) return st;
    if ((st = ibm_read_fields(c->h, IBM_FIELD_UX, c->ux.data(), n)) != IBM_OK) return st;
    if ((st = ibm_read_fields(c->h, IBM_FIELD_UY, c->uy.data(), n)) != IBM_OK) return st;
  }
  if (c->outputs & IBM_OUT_BODIES) {
    c->bodies_out.resize(9 * c->bodies.size());
    if ((st = ibm_read_fields(c->h, IBM_FIELD_BODIES, c->bodies_out.data(), c->bodies_out.size())) != IBM_OK)
      return st;
  }
  if (c->outputs & IBM_OUT_RESIDUAL) {
    c->resid.resize(c->desc.n_corr + 1);
    st = ibm_read_fields(c->h, IBM_FIELD_RESIDUAL, c->resid.data(), c->resid.size());
    if (st != IBM_OK && st != IBM_WARN_NOT_CONVERGED) return st;
  }
  return IBM_OK;
}

}  // namespace

extern "C" {

ibm_status ibm_server_create(const ibm_server_desc* desc, ibm_server* out) {
  if (!out) return sfail(nullptr, IBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!desc) return sfail(nullptr, IBM_ERR_INVALID, "desc is NULL");
  if (desc->max_active < 1 || desc->steps_per_launch < 1)
    return sfail(nullptr, IBM_ERR_INVALID, "max_active and steps_per_launch must be >= 1");
  ibm_server s = nullptr;
  try {
    s = new ibm_server_s();
  } catch (...) {
    return sfail(nullptr, IBM_ERR_NOMEM, "host allocation failed");
  }
  s->desc = *desc;
  int prev = 0;
  cudaGetDevice(&prev);
  if (cudaSetDevice(desc->device) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return sfail(nullptr, IBM_ERR_CUDA, "cannot select the CUDA device");
  }
  cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, desc->device);
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  cudaGetLastError();
  s->budget = desc->max_device_bytes > 0 ? desc->max_device_bytes : 0.8 * (double)free_b;
  s->cta_budget = desc->ib_cta_budget > 0 ? desc->ib_cta_budget : 2 * s->sms;
  {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = desc->device;
    if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
      cudaGetLastError();
      cudaSetDevice(prev);
      delete s;
      return sfail(nullptr, IBM_ERR_CUDA, "cannot create the server's memory pool");
    }
    // keep freed memory cached up to the budget: retiring a case returns
    // nothing to the driver
    unsigned long long keep = (unsigned long long)s->budget;
    cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    cudaGetLastError();
  }
  cudaSetDevice(prev);
  *out = s;
  return IBM_OK;
}

ibm_status ibm_server_submit(ibm_server s, const ibm_case_desc* c, long long* case_id) {
  if (!s) return sfail(nullptr, IBM_ERR_INVALID, "server is NULL");
  if (!c || c->nsteps < 0 || c->nbodies < 0 || (c->nbodies > 0 && (!c->bodies || !c->nmarkers || !c->xy)))
    return sfail(s, IBM_ERR_INVALID, "invalid case description");
  if (c->lattice.prec < IBM_FP64 || c->lattice.prec > IBM_BF16_DEV)
    return sfail(s, IBM_ERR_INVALID, "unknown precision");
  try {
    CaseRec* r = new CaseRec();
    r->id = s->next_id++;
    r->desc = c->lattice;
    r->nsteps = r->remaining = c->nsteps;
    r->outputs = c->outputs;
    int M = 0;
    for (int b = 0; b < c->nbodies; ++b) {
      if (c->nmarkers[b] <= 0) { delete r; return sfail(s, IBM_ERR_INVALID, "a body needs markers"); }
      r->bodies.push_back(c->bodies[b]);
      r->nmark.push_back(c->nmarkers[b]);
      M += c->nmarkers[b];
    }
    r->xy.assign(c->xy ? c->xy : nullptr, c->xy ? c->xy + 2 * (size_t)M : nullptr);
    if (c->ds) { r->ds.assign(c->ds, c->ds + M); r->has_ds = true; }
    r->bytes = case_bytes(c->lattice, M, c->nbodies);
    r->ib_ctas = server_ib_ctas(M, s->desc.ib_markers_per_cta);
    if (r->ib_ctas >= 2) {
      // a grid that cannot be scheduled as one cluster falls back to the
      // grid barrier, whose CTAs must all be resident: count those
      const int p = c->lattice.prec;
      if (s->max_cluster[p] < 0) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(s->desc.device);
        s->max_cluster[p] = ibm::ib_max_cluster(p, ibm::kIbThreads);
        cudaSetDevice(prev);
      }
      r->ib_budget = r->ib_ctas <= s->max_cluster[p] ? 0 : r->ib_ctas;
    }
    r->t_submit = now_s();
    if (s->t_first < 0) s->t_first = r->t_submit;
    s->cases[r->id] = r;
    s->pending.push_back(r->id);
    s->submitted++;
    if (case_id) *case_id = r->id;
  } catch (const std::bad_alloc&) {
    return sfail(s, IBM_ERR_NOMEM, "host allocation failed");
  }
  return IBM_OK;
}

ibm_status ibm_server_progress(ibm_server s, int* completed) {
  if (!s) return sfail(nullptr, IBM_ERR_INVALID, "server is NULL");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->desc.device);
  int done_now = 0;
  // finished chunks: launch the next one, or harvest the case
  std::vector<long long> act = s->active;
  for (long long id : act) {
    CaseRec* c = s->cases[id];
    cudaError_t q = cudaSuccess;
    while (c->inflight > 0) {
      q = cudaEventQuery(c->ev[c->head]);
      if (q != cudaSuccess) break;
      c->head ^= 1;
      c->inflight--;
    }
    if (q != cudaSuccess && q != cudaErrorNotReady) {
      cudaGetLastError();
      case_fail(s, c, IBM_ERR_CUDA, "chunk");
      release_device(s, c);
      continue;
    }
    if (c->remaining > 0) {
      const double t0 = now_s();
      ibm_status st = top_up(s, c);
      s->t_launch += now_s() - t0;
      if (st != IBM_OK) { case_fail(s, c, st, "ibm_step"); release_device(s, c); }
      continue;
    }
    if (c->inflight > 0) continue;
    const double t0 = now_s();
    ibm_status st = harvest(s, c);
    s->t_harvest += now_s() - t0;
    if (st != IBM_OK) {
      case_fail(s, c, st, "ibm_read_fields");
    } else {
      c->state = CASE_DONE;
      c->t_done = now_s();
      s->t_last = c->t_done;
      s->tts_ms.push_back(1e3 * (c->t_done - c->t_submit));
      s->lattice_updates += (double)c->desc.nx * c->desc.ny * c->nsteps;
      s->completed++;
      done_now++;
    }
    release_device(s, c);
  }
  // admit waiting cases in submission order
  while (!s->pending.empty()) {
    CaseRec* c = s->cases[s->pending.front()];
    const bool empty = s->active.empty();
    if ((int)s->active.size() >= s->desc.max_active) break;
    if (!empty && s->bytes_in_use + c->bytes > s->budget) break;
    if (!empty && s->ctas_in_use + c->ib_budget > s->cta_budget) break;
    s->pending.pop_front();
    c->state = CASE_ACTIVE;
    s->active.push_back(c->id);
    s->bytes_in_use += c->bytes;
    s->ctas_in_use += c->ib_budget;
    const double t0 = now_s();
    ibm_status st = admit(s, c);
    s->t_admit += now_s() - t0;
    if (st != IBM_OK) { case_fail(s, c, st, "admission"); release_device(s, c); }
  }
  cudaSetDevice(prev);
  if (completed) *completed = done_now;
  return IBM_OK;
}

ibm_status ibm_server_wait(ibm_server s, long long case_id) {
  if (!s) return sfail(nullptr, IBM_ERR_INVALID, "server is NULL");
  if (case_id >= 0 && !s->cases.count(case_id)) return sfail(s, IBM_ERR_INVALID, "unknown case");
  for (;;) {
    ibm_server_progress(s, nullptr);
    if (case_id >= 0) {
      const int st = s->cases[case_id]->state;
      if (st == CASE_DONE || st == CASE_FAILED) return IBM_OK;
    } else if (s->active.empty() && s->pending.empty()) {
      return IBM_OK;
    }
  }
}

ibm_status ibm_server_result(ibm_server s, long long case_id, int field, double* host_dst, size_t n_elems) {
  if (!s) return sfail(nullptr, IBM_ERR_INVALID, "server is NULL");
  auto it = s->cases.find(case_id);
  if (it == s->cases.end()) return sfail(s, IBM_ERR_INVALID, "unknown case");
  CaseRec* c = it->second;
  if (c->state == CASE_FAILED) return sfail(s, c->status, c->err);
  if (c->state != CASE_DONE) return sfail(s, IBM_ERR_INVALID, "case not finished");
  const std::vector<double>* v = nullptr;
  switch (field) {
    case IBM_FIELD_RHO: v = &c->rho; break;
    case IBM_FIELD_UX: v = &c->ux; break;
    case IBM_FIELD_UY: v = &c->uy; break;
    case IBM_FIELD_BODIES: v = &c->bodies_out; break;
    case IBM_FIELD_RESIDUAL: v = &c->resid; break;
    default: return sfail(s, IBM_ERR_INVALID, "unknown field");
  }
  if (v->empty()) return sfail(s, IBM_ERR_INVALID, "field not requested for this case");
  if (!host_dst || n_elems != v->size()) return sfail(s, IBM_ERR_INVALID, "n_elems does not match the field");
  std::copy(v->begin(), v->end(), host_dst);
  return IBM_OK;
}

ibm_status ibm_server_release(ibm_server s, long long case_id) {
  if (!s) return sfail(nullptr, IBM_ERR_INVALID, "server is NULL");
  auto it = s->cases.find(case_id);
  if (it == s->cases.end()) return sfail(s, IBM_ERR_INVALID, "unknown case");
  if (it->second->state != CASE_DONE && it->second->state != CASE_FAILED)
    return sfail(s, IBM_ERR_INVALID, "case not finished");
  delete it->second;
  s->cases.erase(it);
  return IBM_OK;
}

ibm_status ibm_server_get_stats(ibm_server s, ibm_server_stats* out) {
  if (!s || !out) return sfail(s, IBM_ERR_INVALID, "server and out are required");
  ibm_server_stats r{};
  r.submitted = s->submitted;
  r.completed = s->completed;
  r.failed = s->failed;
  r.active = (long long)s->active.size();
  r.pending = (long long)s->pending.size();
  r.device_bytes = s->bytes_in_use;
  r.host_admit_s = s->t_admit;
  r.host_launch_s = s->t_launch;
  r.host_harvest_s = s->t_harvest;
  if (!s->tts_ms.empty()) {
    std::vector<double> t = s->tts_ms;
    std::sort(t.begin(), t.end());
    auto pct = [&](double p) {
      const double k = p * (t.size() - 1);
      const size_t i = (size_t)k;
      const double f = k - i;
      return i + 1 < t.size() ? t[i] * (1 - f) + t[i + 1] * f : t[i];
    };
    r.p50_ms = pct(0.50);
    r.p95_ms = pct(0.95);
    r.p99_ms = pct(0.99);
    double sum = 0.0;
    for (double v : t) sum += v;
    r.mean_ms = sum / t.size();
    const double span = s->t_last - s->t_first;
    if (span > 0) {
      r.solves_per_s = s->completed / span;
      r.mlups = s->lattice_updates / span / 1e6;
    }
  }
  *out = r;
  return IBM_OK;
}

ibm_status ibm_server_destroy(ibm_server s) {
  if (!s) return IBM_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->desc.device);
  for (auto& kv : s->cases) {
    CaseRec* c = kv.second;
    if (c->h) ibm_destroy(c->h);      // frees are ordered on the case's stream
    if (c->stream) { cudaStreamSynchronize(c->stream); cudaStreamDestroy(c->stream); }
    for (cudaEvent_t e : c->ev)
      if (e) cudaEventDestroy(e);
    delete c;
  }
  for (cudaStream_t st : s->streams) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
  for (cudaEvent_t e : s->events) cudaEventDestroy(e);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  cudaGetLastError();
  cudaSetDevice(prev);
  delete s;
  return IBM_OK;
}

const char* ibm_server_last_error(ibm_server s) { return s ? s->err.c_str() : ibm_last_error(nullptr); }

}  // extern "C"
