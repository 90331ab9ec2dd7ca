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
//
// Batched mode (desc.batched): admitted cases keep their own lattices, but
// one persistent kernel per round (ibm_batch.cuh) advances all resident
// cases of a storage precision by steps_per_launch steps, taking their
// correction tasks and collide+stream tiles from one work queue.  A round is
// a captured CUDA graph -- upload of the round's table, the kernel, read-back
// of its error word -- replayed from two alternating table buffers, so the
// host prepares one round while the device runs the other.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
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
  // batched mode
  int enq_remaining = 0;      // steps not yet placed in a round
  int done_steps = 0;         // steps of rounds that have completed
  int corr = 0, tiles = 0, rows = 0;   // correction tasks, tiles and rows per tile of a step
  bool ready_pending = false; // its set-up event has not yet been waited for by the lane
  double ns_per_step = 0.0;   // measured device time per step in its rounds (0: not yet)
};

// Batched execution of one storage precision: a stream, two table buffers
// (pinned host and device) with their captured graphs, and the rounds in
// flight, oldest first.
struct BatchRound {
  int buf = 0;
  std::vector<std::pair<long long, int>> members;   // case id, steps in this round
};
struct BatchLane {
  bool on = false;
  int prec = -1;
  cudaStream_t stream = nullptr;
  int grid = 0, cap = 0, task_cap = 0;
  size_t rec_bytes = 0, table_bytes = 0;
  unsigned char* host[2] = {nullptr, nullptr};
  void* dev[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  std::deque<BatchRound> rounds;
  int next_buf = 0;
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
  return b + (1 << 20) + 2.0 * (16 << 20);                  // + the unused part of two 16 MiB chunks
}

// Correction-loop CTAs of a served case: one CTA per `per_cta` markers, at
// most ibm::kMaxIbCluster, so that every multi-CTA correction kernel can run
// as one thread-block cluster (CTAs scheduled together, hardware barrier)
// and many cases' correction kernels are resident at once.
constexpr int kServeMarkersPerCta = 512;
// SMs the batched kernel leaves to the set-up and read-back kernels.
constexpr int kBatchReservedSms = 8;
// A fast case takes at most this many times steps_per_launch steps a round.
constexpr int kMaxStepScale = 8;
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
  BatchLane lanes[4];                        // batched mode, per storage precision
  long long wait_ns = 1000000000LL;          // batched kernel's wait limit
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
  st = ibm::add_bodies(c->h, (int)c->bodies.size(), c->bodies.data(), c->nmark.data(), c->xy.data(),
                       c->has_ds ? c->ds.data() : nullptr);
  if (st != IBM_OK) return st;
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
  if ((c->outputs & IBM_OUT_BODIES) && !c->bodies.empty()) {
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

// ------------------------------------------------------------------ batched mode
bool batch_prec_ok(int prec) { return prec == IBM_FP32 || prec == IBM_FP16_DEV || prec == IBM_BF16_DEV; }

int b_grid(int prec) {
  switch (prec) {
    case IBM_FP32: return ibm::BatchOps<ibm::PREC_FP32>::grid();
    case IBM_FP16_DEV: return ibm::BatchOps<ibm::PREC_FP16_DEV>::grid();
    default: return ibm::BatchOps<ibm::PREC_BF16_DEV>::grid();
  }
}
size_t b_rec_bytes(int prec) {
  switch (prec) {
    case IBM_FP32: return ibm::BatchOps<ibm::PREC_FP32>::case_bytes();
    case IBM_FP16_DEV: return ibm::BatchOps<ibm::PREC_FP16_DEV>::case_bytes();
    default: return ibm::BatchOps<ibm::PREC_BF16_DEV>::case_bytes();
  }
}
void b_record(const ibm::Ctx& h, void* dst, int steps, int macro_last, int corr, int tiles, int rows,
              long long wait_ns) {
  switch (h.prec) {
    case IBM_FP32:
      ibm::BatchOps<ibm::PREC_FP32>::record(h, dst, steps, macro_last, corr, tiles, rows, wait_ns);
      break;
    case IBM_FP16_DEV:
      ibm::BatchOps<ibm::PREC_FP16_DEV>::record(h, dst, steps, macro_last, corr, tiles, rows, wait_ns);
      break;
    default:
      ibm::BatchOps<ibm::PREC_BF16_DEV>::record(h, dst, steps, macro_last, corr, tiles, rows, wait_ns);
  }
}
unsigned long long b_end_time(int prec, const void* rec) {
  switch (prec) {
    case IBM_FP32: return ibm::BatchOps<ibm::PREC_FP32>::end_time(rec);
    case IBM_FP16_DEV: return ibm::BatchOps<ibm::PREC_FP16_DEV>::end_time(rec);
    default: return ibm::BatchOps<ibm::PREC_BF16_DEV>::end_time(rec);
  }
}
void b_launch(int prec, void* table, int cap, int grid, cudaStream_t st) {
  switch (prec) {
    case IBM_FP32: ibm::BatchOps<ibm::PREC_FP32>::launch(table, cap, grid, st); break;
    case IBM_FP16_DEV: ibm::BatchOps<ibm::PREC_FP16_DEV>::launch(table, cap, grid, st); break;
    default: ibm::BatchOps<ibm::PREC_BF16_DEV>::launch(table, cap, grid, st);
  }
}

void lane_free(BatchLane& L) {
  if (L.stream) cudaStreamSynchronize(L.stream);
  for (int b = 0; b < 2; ++b) {
    if (L.graph[b]) cudaGraphExecDestroy(L.graph[b]);
    if (L.host[b]) cudaFreeHost(L.host[b]);
    if (L.dev[b]) cudaFree(L.dev[b]);
    if (L.done[b]) cudaEventDestroy(L.done[b]);
    L.graph[b] = nullptr; L.host[b] = nullptr; L.dev[b] = nullptr; L.done[b] = nullptr;
  }
  if (L.stream) cudaStreamDestroy(L.stream);
  L.stream = nullptr;
  L.rounds.clear();
  L.on = false;
  cudaGetLastError();
}

// Stream, table buffers and the two graphs of a round (upload the table,
// run the kernel, read back the head with its error word and the case
// records with their end times).
ibm_status lane_init(ibm_server s, int prec) {
  BatchLane& L = s->lanes[prec];
  if (L.on) return IBM_OK;
  L.prec = prec;
  // the persistent kernel leaves some SMs' worth of CTA slots free: admission
  // (lattice set-up, band build) and harvest (field read-back) run their
  // small kernels beside it instead of waiting for a round to end
  {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->desc.device);
    const int full = b_grid(prec), per_sm = sms > 0 ? full / sms : 0;
    L.grid = per_sm > 0 ? per_sm * std::max(1, sms - kBatchReservedSms) : 0;
  }
  if (L.grid <= 0) return sfail(s, IBM_ERR_CUDA, "the batched kernel cannot be resident on this device");
  L.cap = s->desc.max_active;
  L.task_cap = 16384;
  L.rec_bytes = b_rec_bytes(prec);
  L.table_bytes = ibm::kBatchHeadBytes + (size_t)L.cap * L.rec_bytes + (size_t)L.task_cap * sizeof(int2);
  bool ok = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess;
  for (int b = 0; ok && b < 2; ++b) {
    ok = cudaMallocHost((void**)&L.host[b], L.table_bytes) == cudaSuccess &&
         cudaMalloc(&L.dev[b], L.table_bytes) == cudaSuccess &&
         cudaEventCreateWithFlags(&L.done[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) break;
    std::memset(L.host[b], 0, L.table_bytes);
    cudaGraph_t g = nullptr;
    ok = cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (!ok) break;
    cudaMemcpyAsync(L.dev[b], L.host[b], L.table_bytes, cudaMemcpyHostToDevice, L.stream);
    b_launch(prec, L.dev[b], L.cap, L.grid, L.stream);
    cudaMemcpyAsync(L.host[b], L.dev[b], ibm::kBatchHeadBytes + (size_t)L.cap * L.rec_bytes,
                    cudaMemcpyDeviceToHost, L.stream);
    ok = cudaStreamEndCapture(L.stream, &g) == cudaSuccess &&
         cudaGraphInstantiate(&L.graph[b], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
  }
  if (!ok) {
    lane_free(L);
    return sfail(s, IBM_ERR_CUDA, "setting up the batched kernel's stream, tables or graphs failed");
  }
  L.on = true;
  L.rounds.clear();
  L.next_buf = 0;
  return IBM_OK;
}

// Admission in batched mode: the case's lattice, markers and band are set
// up on its own stream; the lane waits for that before the case's first
// round.
ibm_status admit_batched(ibm_server s, CaseRec* c) {
  ibm_status st = lane_init(s, c->desc.prec);
  if (st != IBM_OK) return st;
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
  ibm_lattice_desc d = c->desc;
  d.cuda_stream = c->stream;
  d.device = s->desc.device;
  if ((st = ibm::create_lattice(&d, &c->h, s->pool)) != IBM_OK) return st;
  st = ibm::add_bodies(c->h, (int)c->bodies.size(), c->bodies.data(), c->nmark.data(), c->xy.data(),
                       c->has_ds ? c->ds.data() : nullptr);
  if (st != IBM_OK) return st;
  ibm::Ctx& h = *c->h;
  if (h.nm > 0) {
    ibm::launch_band_build(h, c->stream);
    h.band_valid = true;
  }
  const int tile_nodes = s->desc.tile_nodes > 0 ? s->desc.tile_nodes : 32768;
  c->corr = h.nm == 0 ? 0 : (h.any_moving ? 1 : server_ib_ctas(h.nm, s->desc.ib_markers_per_cta));
  c->rows = std::max(1, std::min(h.geom.ny, tile_nodes / std::max(1, h.geom.nx)));
  c->tiles = (h.geom.ny + c->rows - 1) / c->rows;
  c->enq_remaining = c->nsteps;
  c->done_steps = 0;
  if (cudaEventRecord(c->ev[0], c->stream) != cudaSuccess) { cudaGetLastError(); return IBM_ERR_CUDA; }
  c->ready_pending = true;
  if (cudaGetLastError() != cudaSuccess) return IBM_ERR_CUDA;
  return IBM_OK;
}

// Builds and launches one round of lane L from the resident cases that have
// steps left to place.  Returns false when there was nothing to launch.
bool lane_round(ibm_server s, BatchLane& L, ibm_status* st_out) {
  *st_out = IBM_OK;
  if (!L.on || L.rounds.size() >= 2) return false;
  const int S = s->desc.steps_per_launch;
  std::vector<CaseRec*> members;
  int ntask = 0;
  for (long long id : s->active) {
    CaseRec* c = s->cases[id];
    if (c->state != CASE_ACTIVE || !c->h || c->desc.prec != L.prec || c->enq_remaining <= 0) continue;
    if ((int)members.size() >= L.cap || ntask + c->corr + c->tiles > L.task_cap) break;
    members.push_back(c);
    ntask += c->corr + c->tiles;
  }
  if (members.empty()) return false;
  // Steps per case: a case whose steps have been timed gets as many as fit
  // the time the slowest timed member needs for steps_per_launch steps (at
  // most kMaxStepScale times that), so that no case idles while the slowest
  // one finishes its round.
  double t_round = 0.0;
  for (CaseRec* c : members) t_round = std::max(t_round, S * c->ns_per_step);
  auto steps_of = [&](CaseRec* c) {
    int n = S;
    if (t_round > 0.0 && c->ns_per_step > 0.0)
      n = (int)std::max(1.0, std::min((double)kMaxStepScale * S, std::floor(t_round / c->ns_per_step)));
    return std::min(c->enq_remaining, n);
  };
  const int b = L.next_buf;
  unsigned char* tab = L.host[b];
  int2* tasks = reinterpret_cast<int2*>(tab + ibm::kBatchHeadBytes + (size_t)L.cap * L.rec_bytes);
  int rounds = 0, k = 0;
  BatchRound R;
  R.buf = b;
  for (size_t slot = 0; slot < members.size(); ++slot) {
    CaseRec* c = members[slot];
    ibm::Ctx& h = *c->h;
    const int steps = steps_of(c);
    const int macro_last = (steps == c->enq_remaining && (c->outputs & IBM_OUT_MACRO)) ? 1 : 0;
    b_record(h, tab + ibm::kBatchHeadBytes + slot * L.rec_bytes, steps, macro_last, c->corr, c->tiles, c->rows,
             s->wait_ns);
    h.parity ^= steps & 1;
    h.steps += steps;
    h.launches += steps;               // one batched launch covers every step of the round
    c->enq_remaining -= steps;
    rounds = std::max(rounds, steps);
    R.members.push_back({c->id, steps});
    if (c->ready_pending) {
      if (cudaStreamWaitEvent(L.stream, c->ev[0], 0) != cudaSuccess) { cudaGetLastError(); *st_out = IBM_ERR_CUDA; }
      c->ready_pending = false;
    }
  }
  // task order of one step: every case's correction tasks, then all tiles
  // (corr_first 1), or case by case (2)
  const bool by_case = s->desc.corr_first == 2;
  for (int pass = 0; pass < (by_case ? 1 : 2); ++pass)
    for (size_t slot = 0; slot < members.size(); ++slot) {
      CaseRec* c = members[slot];
      if (by_case || pass == 0)
        for (int q = 0; q < c->corr; ++q) tasks[k++] = make_int2((int)slot, q);
      if (by_case || pass == 1)
        for (int q = 0; q < c->tiles; ++q) tasks[k++] = make_int2((int)slot, c->corr + q);
    }
  ibm::BatchHead* head = reinterpret_cast<ibm::BatchHead*>(tab);
  head->next = 0;
  head->err = 0;
  head->per_round = k;
  head->rounds = rounds;
  head->wait_ns = s->wait_ns;
  if (cudaGraphLaunch(L.graph[b], L.stream) != cudaSuccess ||
      cudaEventRecord(L.done[b], L.stream) != cudaSuccess) {
    cudaGetLastError();
    *st_out = IBM_ERR_CUDA;
  }
  L.rounds.push_back(std::move(R));
  L.next_buf ^= 1;
  return true;
}

// Completed rounds of lane L: count the members' steps, harvest finished
// cases.  A round whose wait ran out fails every case still in flight on the
// lane (after the lane's stream has drained, so no round still uses them).
void lane_poll(ibm_server s, BatchLane& L, int* done_now) {
  while (!L.rounds.empty()) {
    BatchRound& R = L.rounds.front();
    const cudaError_t q = cudaEventQuery(L.done[R.buf]);
    if (q == cudaErrorNotReady) return;
    const ibm::BatchHead* head = reinterpret_cast<const ibm::BatchHead*>(L.host[R.buf]);
    if (q != cudaSuccess || head->err) {
      cudaGetLastError();
      cudaStreamSynchronize(L.stream);
      cudaGetLastError();
      const ibm_status st = q != cudaSuccess ? IBM_ERR_CUDA : IBM_ERR_TIMEOUT;
      for (auto& r : L.rounds)
        for (auto& m : r.members) {
          CaseRec* c = s->cases[m.first];
          if (c->state != CASE_ACTIVE) continue;
          c->state = CASE_FAILED;
          c->status = st;
          c->err = st == IBM_ERR_TIMEOUT ? "batched kernel: a dependency wait ran out"
                                         : "batched kernel: CUDA error";
          s->failed++;
          release_device(s, c);
        }
      L.rounds.clear();
      return;
    }
    for (size_t slot = 0; slot < R.members.size(); ++slot) {
      const auto& m = R.members[slot];
      CaseRec* c = s->cases[m.first];
      if (c->state != CASE_ACTIVE) continue;
      const unsigned long long t1 =
          b_end_time(L.prec, L.host[R.buf] + ibm::kBatchHeadBytes + slot * L.rec_bytes);
      if (t1 > head->t_start && m.second > 0) {
        const double per = (double)(t1 - head->t_start) / m.second;
        c->ns_per_step = c->ns_per_step > 0.0 ? 0.5 * (c->ns_per_step + per) : per;
      }
      c->done_steps += m.second;
      if (c->done_steps < c->nsteps) continue;
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
        if (done_now) (*done_now)++;
      }
      release_device(s, c);
    }
    L.rounds.pop_front();
  }
}

}  // namespace

extern "C" {

ibm_status ibm_server_create(const ibm_server_desc* desc, ibm_server* out) {
  if (!out) return sfail(nullptr, IBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!desc) return sfail(nullptr, IBM_ERR_INVALID, "desc is NULL");
  if (desc->max_active < 1 || desc->steps_per_launch < 1)
    return sfail(nullptr, IBM_ERR_INVALID, "max_active and steps_per_launch must be >= 1");
  if (desc->batched != 0 && desc->batched != 1) return sfail(nullptr, IBM_ERR_INVALID, "batched must be 0 or 1");
  if (desc->batched && desc->max_active > 1024)
    return sfail(nullptr, IBM_ERR_INVALID, "a batched server holds at most 1024 cases");
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
  if (s->desc.batched && !batch_prec_ok(c->lattice.prec))
    return sfail(s, IBM_ERR_INVALID, "the batched server runs FP32 and 16-bit storage only");
  if (s->desc.batched && c->nbodies > ibm::kBatchThreads)
    return sfail(s, IBM_ERR_INVALID, "the batched server takes at most 256 bodies per case");
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
    if (r->ib_ctas >= 2 && !s->desc.batched) {
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
  if (s->desc.batched) {
    // completed rounds: count steps, harvest finished cases
    for (auto& L : s->lanes)
      if (L.on) lane_poll(s, L, &done_now);
  } else {
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
    ibm_status st = s->desc.batched ? admit_batched(s, c) : admit(s, c);
    s->t_admit += now_s() - t0;
    if (st != IBM_OK) { case_fail(s, c, st, "admission"); release_device(s, c); }
  }
  ibm_status rst = IBM_OK;
  if (s->desc.batched) {
    // keep two rounds in flight on every lane
    const double t0 = now_s();
    for (auto& L : s->lanes) {
      ibm_status st = IBM_OK;
      while (st == IBM_OK && lane_round(s, L, &st)) {
      }
      if (st != IBM_OK) rst = sfail(s, st, "launching a batched round failed");
    }
    s->t_launch += now_s() - t0;
  }
  cudaSetDevice(prev);
  if (completed) *completed = done_now;
  return rst;
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
  const unsigned need = field == IBM_FIELD_BODIES ? IBM_OUT_BODIES
                        : (field == IBM_FIELD_RESIDUAL ? IBM_OUT_RESIDUAL : IBM_OUT_MACRO);
  if (!(c->outputs & need)) return sfail(s, IBM_ERR_INVALID, "field not requested for this case");
  if (n_elems != v->size()) return sfail(s, IBM_ERR_INVALID, "n_elems does not match the field");
  if (n_elems == 0) return IBM_OK;                 // a case without bodies
  if (!host_dst) return sfail(s, IBM_ERR_INVALID, "host_dst is NULL");
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
  for (auto& L : s->lanes) lane_free(L);   // waits for rounds still in flight
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

ibm_status ibm_server_autotune(ibm_server s, const ibm_case_desc* samples, int n, const int* tile_nodes,
                               int n_tiles, const int* markers_per_cta, int n_mpc, int* best_tile_nodes,
                               int* best_markers_per_cta, int* best_corr_first, double* best_seconds) {
  if (!s) return sfail(nullptr, IBM_ERR_INVALID, "server is NULL");
  if (!s->desc.batched) return sfail(s, IBM_ERR_INVALID, "the autotuner tunes the batched mode");
  if (!s->active.empty() || !s->pending.empty()) return sfail(s, IBM_ERR_INVALID, "the server must be idle");
  if (n < 1 || !samples) return sfail(s, IBM_ERR_INVALID, "at least one sample case is required");
  if (n_tiles < 0 || n_mpc < 0 || (n_tiles > 0 && !tile_nodes) || (n_mpc > 0 && !markers_per_cta))
    return sfail(s, IBM_ERR_INVALID, "invalid candidate lists");
  std::vector<int> tiles, mpcs;
  for (int k = 0; k < n_tiles; ++k)
    if (tile_nodes[k] > 0) tiles.push_back(tile_nodes[k]);
  for (int k = 0; k < n_mpc; ++k)
    if (markers_per_cta[k] > 0) mpcs.push_back(markers_per_cta[k]);
  if (tiles.empty()) tiles = {8192, 16384, 32768, 65536};
  if (mpcs.empty()) mpcs = {256, 512, 1024};
  try {
    // the sample runs stay out of the server's statistics
    const long long sub0 = s->submitted, comp0 = s->completed, fail0 = s->failed;
    const std::vector<double> tts0 = s->tts_ms;
    const double tf0 = s->t_first, tl0 = s->t_last, lu0 = s->lattice_updates;
    const double ta0 = s->t_admit, tla0 = s->t_launch, th0 = s->t_harvest;
    const ibm_server_desc keep = s->desc;
    auto run = [&](int tile, int mpc, int order, double* sec) -> ibm_status {
      s->desc.tile_nodes = tile;
      s->desc.ib_markers_per_cta = mpc;
      s->desc.corr_first = order;
      std::vector<long long> ids;
      const double t0 = now_s();
      for (int k = 0; k < n; ++k) {
        long long id = 0;
        ibm_status st = ibm_server_submit(s, &samples[k], &id);
        if (st != IBM_OK) return st;
        ids.push_back(id);
      }
      ibm_server_wait(s, -1);
      *sec = now_s() - t0;
      ibm_status worst = IBM_OK;
      for (long long id : ids) {
        if (s->cases[id]->state == CASE_FAILED) worst = s->cases[id]->status;
        ibm_server_release(s, id);
      }
      return worst;
    };
    double sec = 0.0;
    // untimed first run: lane set-up, graph upload, memory-pool growth
    ibm_status st = run(tiles[0], mpcs[0], 1, &sec);
    int bt = tiles[0], bm = mpcs[0], bo = 1;
    double best = 1e300;
    for (int t : tiles)
      for (int m : mpcs)
        for (int o = 1; o <= 2 && st == IBM_OK; ++o) {
          st = run(t, m, o, &sec);
          if (st == IBM_OK && sec < best) { best = sec; bt = t; bm = m; bo = o; }
        }
    s->desc = keep;
    s->submitted = sub0; s->completed = comp0; s->failed = fail0;
    s->tts_ms = tts0;
    s->t_first = tf0; s->t_last = tl0; s->lattice_updates = lu0;
    s->t_admit = ta0; s->t_launch = tla0; s->t_harvest = th0;
    if (st != IBM_OK) return sfail(s, st, "a sample run of the autotuner failed");
    s->desc.tile_nodes = bt;
    s->desc.ib_markers_per_cta = bm;
    s->desc.corr_first = bo;
    if (best_tile_nodes) *best_tile_nodes = bt;
    if (best_markers_per_cta) *best_markers_per_cta = bm;
    if (best_corr_first) *best_corr_first = bo;
    if (best_seconds) *best_seconds = best;
    return IBM_OK;
  } catch (const std::bad_alloc&) {
    return sfail(s, IBM_ERR_NOMEM, "host allocation failed");
  }
}

const char* ibm_server_last_error(ibm_server s) { return s ? s->err.c_str() : ibm_last_error(nullptr); }

}  // extern "C"
