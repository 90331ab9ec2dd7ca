// ibm_api.cu -- the C ABI of include/ibm.h: argument checks, device
// allocation, the per-step launch sequence and its CUDA-graph replay, and
// field transfers.  Every entry point catches C++ exceptions and returns a
// status; none lets one cross the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "ibm_internal.h"

using namespace ibm;


namespace {

ibm_alloc_fn g_alloc = nullptr;
ibm_free_fn g_free = nullptr;
void* g_actx = nullptr;
thread_local std::string t_err;

constexpr int kEventPairs = 4096;     // timed steps held before folding
constexpr int kEventsPerStep = 2;     // around the main collide+stream launch

ibm_status fail(Ctx* h, ibm_status st, const std::string& msg) {
  if (h) h->err = msg; else t_err = msg;
  return st;
}

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; prev = -1; return; }
    if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

// In pool mode every allocation of at most kPoolCarveMax bytes is carved from
// a kPoolChunk chunk of the pool, released with the lattice.  Each call to the
// pool's allocator costs host time (about 0.4 ms per call was measured once
// an earlier pool had served a few hundred lattices in the process), and a
// lattice holds about thirty buffers, most of them small.
constexpr size_t kPoolChunk = 16u << 20, kPoolCarveMax = 4u << 20;

void* dev_alloc(Ctx& h, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (h.pool && bytes <= kPoolCarveMax) {
    const size_t a = (bytes + 255) & ~(size_t)255;
    if (h.chunk_left < a) {
      void* c = nullptr;
      if (cudaMallocFromPoolAsync(&c, kPoolChunk, h.pool, h.stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      h.chunks.push_back(c);
      h.chunk_ptr = static_cast<char*>(c);
      h.chunk_left = kPoolChunk;
    }
    p = h.chunk_ptr;
    h.chunk_ptr += a;
    h.chunk_left -= a;
    return p;                     // released with its chunk
  }
  if (h.pool) {
    if (cudaMallocFromPoolAsync(&p, bytes, h.pool, h.stream) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  } else if (g_alloc) {
    p = g_alloc(bytes, h.device, (void*)h.stream, g_actx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h.allocs.push_back(p);
  return p;
}

void dev_free(Ctx& h, void* p) {
  if (!p) return;
  bool own = false;
  for (size_t k = 0; k < h.allocs.size(); ++k)
    if (h.allocs[k] == p) { h.allocs.erase(h.allocs.begin() + k); own = true; break; }
  if (h.pool && !own) return;     // carved from a chunk: released with the chunk
  if (h.pool) cudaFreeAsync(p, h.stream);
  else if (g_free) g_free(p, h.device, (void*)h.stream, g_actx);
  else cudaFree(p);
}

#define IBM_CK(h, call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      cudaGetLastError();                                                            \
      return fail(h, IBM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                                \
  } while (0)

#define IBM_ALLOC(h, ptr, type, count)                                               \
  do {                                                                               \
    (ptr) = (type)dev_alloc(*(h), sizeof(*(ptr)) * (size_t)(count));                  \
    if (!(ptr)) return fail(h, IBM_ERR_NOMEM, "device allocation of " #ptr " failed"); \
  } while (0)

bool is_finite(double v) { return std::isfinite(v); }

void destroy_graphs(Ctx& h) {
  for (int p = 0; p < 2; ++p)
    for (int m = 0; m < 2; ++m)
      if (h.graph[p][m]) { cudaGraphExecDestroy(h.graph[p][m]); h.graph[p][m] = nullptr; }
  for (int p = 0; p < 2; ++p)
    if (h.graph_block[p]) { cudaGraphExecDestroy(h.graph_block[p]); h.graph_block[p] = nullptr; }
}

void enqueue_step(Ctx& h, int parity, bool macro, bool timing);

// Capture `count` consecutive steps starting at `parity` into one graph.
cudaError_t capture_steps(Ctx& c, int parity, int count, bool macro_last, cudaGraphExec_t* out) {
  cudaGraph_t graph;
  cudaError_t e = cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int j = 0; j < count; ++j)
    enqueue_step(c, parity ^ (j & 1), macro_last && j == count - 1, false);
  e = cudaStreamEndCapture(c.stream, &graph);
  if (e != cudaSuccess) return e;
  // per-node priorities: the correction chain keeps its high priority inside
  // the graph (by default a graph runs at the priority of its stream)
  e = cudaGraphInstantiateWithFlags(out, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) *out = nullptr;
  return e;
}

ibm_status check_device_flags(Ctx* h) {
  if (!h->dctr) return IBM_OK;
  int ctr[CTR_COUNT] = {0, 0, 0, 0};
  IBM_CK(h, cudaMemcpyAsync(ctr, h->dctr, sizeof(ctr), cudaMemcpyDeviceToHost, h->stream));
  IBM_CK(h, cudaStreamSynchronize(h->stream));
  if (ctr[CTR_ERR] & ERR_BAND_CAP) return fail(h, IBM_ERR_BOUNDS, "band node capacity exceeded");
  if (ctr[CTR_ERR] & ERR_LIST_CAP)
    return fail(h, IBM_ERR_BOUNDS, "more than 32 markers cover one node (markers too dense)");
  if (ctr[CTR_ERR] & ERR_SEG_CAP) return fail(h, IBM_ERR_BOUNDS, "band segment capacity exceeded");
  if (ctr[CTR_ERR] & ERR_G_CAP)
    return fail(h, IBM_ERR_BOUNDS, "a marker couples to more than 64 markers (markers too dense)");
  if (ctr[CTR_ERR] & ERR_BARRIER)
    return fail(h, IBM_ERR_TIMEOUT, "the correction-loop grid barrier timed out");
  if (ctr[CTR_ERR] & ERR_DIVERGED)
    return fail(h, IBM_ERR_DIVERGED, "non-finite population or residual (the state has diverged)");
  if (ctr[CTR_ERR] & WARN_NOT_CONV) {
    // a warning: reported once, then cleared on the device
    const int rest = ctr[CTR_ERR] & ~WARN_NOT_CONV;
    IBM_CK(h, cudaMemcpyAsync(h->dctr + CTR_ERR, &rest, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    IBM_CK(h, cudaStreamSynchronize(h->stream));
    return fail(h, IBM_WARN_NOT_CONVERGED, "no-slip residual above corr_tol after n_corr iterations");
  }
  return IBM_OK;
}

ibm_status sync_stream(Ctx* h) {
  IBM_CK(h, cudaStreamSynchronize(h->stream));
  IBM_CK(h, cudaGetLastError());
  return check_device_flags(h);
}

ibm_status ensure_io(Ctx* h, size_t doubles) {
  if (h->io_cap >= doubles) return IBM_OK;
  if (h->dio) { IBM_CK(h, cudaStreamSynchronize(h->stream)); dev_free(*h, h->dio); h->dio = nullptr; }
  IBM_ALLOC(h, h->dio, double*, doubles);
  h->io_cap = doubles;
  return IBM_OK;
}

// The launch sequence of one time step.  Without markers: one collide+stream
// launch.  With markers the step forks: the correction-loop kernel (which
// ends with collide+stream of the band row segments) runs on the
// high-priority stream while collide+stream covers every band-free row
// segment on the main stream; after the join, moving bodies are advanced
// and re-binned.
void enqueue_step(Ctx& h, int parity, bool macro, bool timing) {
  const bool t = timing && h.ev_used < kEventPairs;
  cudaEvent_t* e = t ? &h.ev[kEventsPerStep * h.ev_used] : nullptr;
  if (h.nm == 0) {
    if (t) cudaEventRecord(e[0], h.stream);
    launch_collide_stream(h, parity, macro, K1_ALL, h.stream);
    if (t) cudaEventRecord(e[1], h.stream);
  } else {
    cudaEventRecord(h.ev_fork, h.stream);
    cudaStreamWaitEvent(h.ib_stream, h.ev_fork, 0);
    launch_ib_loop(h, parity, macro, h.ib_stream);
    cudaEventRecord(h.ev_join, h.ib_stream);
    if (t) cudaEventRecord(e[0], h.stream);
    launch_collide_stream(h, parity, macro, K1_MAIN, h.stream);
    if (t) cudaEventRecord(e[1], h.stream);
    cudaStreamWaitEvent(h.stream, h.ev_join, 0);
    launch_body_update(h, h.stream);
  }
  if (t) h.ev_used++;
}

ibm_status fold_events(Ctx* h) {
  if (h->ev_used == 0) return IBM_OK;
  IBM_CK(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < h->ev_used; ++k) {
    float a = 0.f;
    cudaEvent_t* e = &h->ev[kEventsPerStep * k];
    IBM_CK(h, cudaEventElapsedTime(&a, e[0], e[1]));
    h->acc_ms += a;
  }
  h->acc_n += h->ev_used;
  h->ev_used = 0;
  return IBM_OK;
}

// Band nodes of the current band (sizes the grids of the phase kernels;
// synchronises the stream).
ibm_status count_band(Ctx* h) {
  int ctr[CTR_COUNT] = {0, 0, 0, 0};
  IBM_CK(h, cudaMemcpyAsync(ctr, h->dctr, sizeof(ctr), cudaMemcpyDeviceToHost, h->stream));
  IBM_CK(h, cudaStreamSynchronize(h->stream));
  h->nband_host = std::min(ctr[CTR_NBAND], h->bcap);
  return IBM_OK;
}

// The NaN/Inf scan of the whole lattice after every watchdog_steps steps
// (checked between graph replays, so with blocks of steps it runs at the
// first block boundary at or after the due step).
void watchdog_if_due(Ctx& c) {
  if (c.watchdog_steps <= 0 || c.watch_due < c.watchdog_steps) return;
  launch_watchdog(c, c.stream);
  c.launches += 1;
  c.watch_due = 0;
}

// CTAs of the correction kernel: one for small boundaries, 3/4 of the SMs
// above kSmallIbMarkers markers, or the count set by IBM_OPT_IB_CTAS.  A
// grid of 2..16 CTAs that fits the device as one cluster is launched as a
// cluster (hardware barrier, CTAs scheduled together).
void choose_ib_grid(Ctx& c) {
  const int M = c.nm;
  // Large boundaries: three CTAs per four SMs.  The correction kernel runs
  // beside collide+stream and holds its SMs' registers while it runs; on the
  // 4096^2 Couette step (14052 markers) 3/4 of the SMs gave the shortest step
  // (the correction chain still ends before collide+stream).
  const int wide = (3 * c.ib_grid_max + 3) / 4;
  c.ib_grid = c.ib_grid_opt > 0 ? (c.ib_grid_opt < c.ib_grid_max ? c.ib_grid_opt : c.ib_grid_max)
                                : (M <= kSmallIbMarkers ? 1 : wide);
  c.ib_cluster = false;
  // The grid barrier's arrival counter only grows and each barrier waits for
  // the next multiple of the grid size: a new grid size must start from a
  // counter that is a multiple of it, so it restarts at zero (every caller
  // has the stream's earlier work ordered before this memset).
  if (c.ib_grid != c.ib_grid_last && c.dbar) {
    cudaMemsetAsync(c.dbar, 0, sizeof(unsigned long long), c.stream);
    c.ib_grid_last = c.ib_grid;
  }
  if (c.ib_grid >= 2 && c.ib_grid <= kMaxIbCluster) {
    if (c.ib_cluster_max < 0) c.ib_cluster_max = ib_max_cluster(c.prec, c.ib_threads);
    c.ib_cluster = c.ib_grid <= c.ib_cluster_max;
  }
  // the Jacobi cluster of IBM_OPT_IB_PHASES = 2 (none: the persistent kernel)
  c.ib_jc_cluster = c.ib_phases == 2 && M > kSmallIbMarkers ? jacobi_cluster_size(c.prec, M) : 0;
}

ibm_status upload_markers(Ctx* h) {
  Ctx& c = *h;
  const int M = c.nm;
  // release the previous marker-sized buffers
  void* olds[] = {c.dX, c.dY, c.dds, c.ddX, c.ddY, c.dmbody, c.dUx, c.dUy, c.dW, c.dnode_of,
                  c.dband_of, c.dclaim, c.dbnode, c.dbcnt, c.dent, c.dbq, c.dmq, c.dAh,
                  c.dCm, c.dG, c.dgcnt, c.dbodies, c.dfpart};
  IBM_CK(h, cudaStreamSynchronize(c.stream));
  // clear the node -> band map and segment flags of the old band
  IBM_CK(h, cudaMemsetAsync(c.dnode2band, 0xFF, sizeof(int) * (size_t)c.geom.nx * c.geom.ny, c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dsegflag, 0, sizeof(int) * (size_t)c.nseg_x * c.geom.ny, c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dctr, 0, CTR_COUNT * sizeof(int), c.stream));
  IBM_CK(h, cudaStreamSynchronize(c.stream));
  dev_free(c, c.dseglist);
  c.dseglist = nullptr;
  for (void* p : olds) dev_free(c, p);
  c.mcap = M;
  c.bcap = M * kStencil;
  const size_t R = c.r_bytes;
  IBM_ALLOC(h, c.dX, double*, M);
  IBM_ALLOC(h, c.dY, double*, M);
  IBM_ALLOC(h, c.dds, double*, M);
  IBM_ALLOC(h, c.ddX, double*, M);
  IBM_ALLOC(h, c.ddY, double*, M);
  IBM_ALLOC(h, c.dmbody, int*, M);
  c.dUx = dev_alloc(c, R * M);
  c.dUy = dev_alloc(c, R * M);
  c.dW = dev_alloc(c, R * M * kStencil);
  IBM_ALLOC(h, c.dnode_of, int*, M * kStencil);
  IBM_ALLOC(h, c.dband_of, int*, M * kStencil);
  IBM_ALLOC(h, c.dclaim, int*, M * kStencil);
  IBM_ALLOC(h, c.dbnode, int*, c.bcap);
  IBM_ALLOC(h, c.dbcnt, int*, c.bcap);
  c.dent = dev_alloc(c, (R == 8 ? sizeof(Ent<double>) : sizeof(Ent<float>)) * (size_t)c.bcap * kBandCap);
  IBM_ALLOC(h, c.dfpart, double*, (size_t)((M + kForceChunk - 1) / kForceChunk) * c.nb * 3);
  // correction-kernel CTAs: one for small boundaries (its grid barrier is a
  // block barrier, so such kernels of several lattices may run side by
  // side), one per SM otherwise
  choose_ib_grid(c);
  c.dbq = dev_alloc(c, R * 8 * (size_t)c.bcap);
  c.dmq = dev_alloc(c, R * 4 * (size_t)M);
  c.dAh = dev_alloc(c, R * 2 * (size_t)M * (c.desc.n_corr + 1));
  c.dCm = dev_alloc(c, R * 3 * (size_t)M);
  c.dG = dev_alloc(c, (R == 8 ? sizeof(Ent<double>) : sizeof(Ent<float>)) * (size_t)M * kGCap);
  IBM_ALLOC(h, c.dgcnt, int*, M);
  IBM_ALLOC(h, c.dbodies, BodyDev*, c.nb);
  {
    const long long nseg = (long long)c.nseg_x * c.geom.ny;
    c.segcap = (int)(c.bcap < nseg ? c.bcap : nseg);
    IBM_ALLOC(h, c.dseglist, int*, c.segcap);
  }
  if (!c.dUx || !c.dUy || !c.dW || !c.dent || !c.dbq || !c.dmq || !c.dAh || !c.dCm || !c.dG)
    return fail(h, IBM_ERR_NOMEM, "device allocation of marker arrays failed");
  IBM_CK(h, cudaMemcpyAsync(c.dX, c.hX.data(), 8 * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.dY, c.hY.data(), 8 * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.dds, c.hds.data(), 8 * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.ddX, c.hdX.data(), 8 * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.ddY, c.hdY.data(), 8 * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.dmbody, c.hmbody.data(), 4 * M, cudaMemcpyHostToDevice, c.stream));
  std::vector<char> ux(R * M), uy(R * M);
  for (int l = 0; l < M; ++l) {
    if (R == 8) { ((double*)ux.data())[l] = c.hUx[l]; ((double*)uy.data())[l] = c.hUy[l]; }
    else { ((float*)ux.data())[l] = (float)c.hUx[l]; ((float*)uy.data())[l] = (float)c.hUy[l]; }
  }
  IBM_CK(h, cudaMemcpyAsync(c.dUx, ux.data(), R * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.dUy, uy.data(), R * M, cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.dbodies, c.hbodies.data(), sizeof(BodyDev) * c.nb,
                            cudaMemcpyHostToDevice, c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dAh, 0, R * 2 * (size_t)M * (c.desc.n_corr + 1), c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dCm, 0, R * 3 * (size_t)M, c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dG, 0, (R == 8 ? sizeof(Ent<double>) : sizeof(Ent<float>)) * (size_t)M * kGCap,
                            c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dent, 0, (R == 8 ? sizeof(Ent<double>) : sizeof(Ent<float>)) *
                                           (size_t)c.bcap * kBandCap, c.stream));
  IBM_CK(h, cudaMemsetAsync(c.dbcnt, 0, sizeof(int) * c.bcap, c.stream));
  IBM_CK(h, cudaStreamSynchronize(c.stream));   // host vectors are temporaries
  c.dev_nm = c.nm;
  c.dev_nb = c.nb;
  c.band_valid = false;
  destroy_graphs(c);
  return IBM_OK;
}

// Device -> host copy of the moving state before markers are re-uploaded.
ibm_status download_moving_state(Ctx* h) {
  Ctx& c = *h;
  // the markers and bodies the device holds (appended ones not yet uploaded
  // have only their host copy)
  const int M = c.dev_nm, B = c.dev_nb;
  if (M == 0 || !c.any_moving) return IBM_OK;
  std::vector<char> ux(c.r_bytes * M), uy(c.r_bytes * M);
  IBM_CK(h, cudaMemcpyAsync(c.hX.data(), c.dX, 8 * M, cudaMemcpyDeviceToHost, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.hY.data(), c.dY, 8 * M, cudaMemcpyDeviceToHost, c.stream));
  IBM_CK(h, cudaMemcpyAsync(ux.data(), c.dUx, c.r_bytes * M, cudaMemcpyDeviceToHost, c.stream));
  IBM_CK(h, cudaMemcpyAsync(uy.data(), c.dUy, c.r_bytes * M, cudaMemcpyDeviceToHost, c.stream));
  IBM_CK(h, cudaMemcpyAsync(c.hbodies.data(), c.dbodies, sizeof(BodyDev) * B, cudaMemcpyDeviceToHost,
                            c.stream));
  IBM_CK(h, cudaStreamSynchronize(c.stream));
  for (int l = 0; l < M; ++l) {
    c.hUx[l] = c.r_bytes == 8 ? ((double*)ux.data())[l] : ((float*)ux.data())[l];
    c.hUy[l] = c.r_bytes == 8 ? ((double*)uy.data())[l] : ((float*)uy.data())[l];
  }
  return IBM_OK;
}

}  // namespace

namespace ibm {
// Message for ibm_last_error(NULL), for entry points that take no handle.
void set_thread_error(const char* msg) { t_err = msg; }
}  // namespace ibm

extern "C" {

int ibm_abi_version(void) { return IBM_ABI_VERSION; }

ibm_status ibm_set_allocator(ibm_alloc_fn alloc, ibm_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr))
    return fail(nullptr, IBM_ERR_INVALID, "ibm_set_allocator: give both functions or neither");
  g_alloc = alloc;
  g_free = release;
  g_actx = ctx;
  return IBM_OK;
}

const char* ibm_last_error(ibm_handle h) { return h ? h->err.c_str() : t_err.c_str(); }

}  // extern "C"

ibm_status ibm::create_lattice(const ibm_lattice_desc* desc, ibm_handle* out, cudaMemPool_t pool) {
  if (!out) return fail(nullptr, IBM_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(nullptr, IBM_ERR_INVALID, "desc is NULL");
  ibm_lattice_desc d = *desc;
  if (d.collision != IBM_COLL_BGK && d.collision != IBM_COLL_MRT)
    return fail(nullptr, IBM_ERR_INVALID, "unknown collision operator");
  {
    const double paper_rates[3] = {1.1, 1.25, 1.8};   // section 3: s_e, s_eps, s_q
    for (int k = 0; k < 3; ++k) {
      if (d.mrt_s[k] == 0.0) d.mrt_s[k] = paper_rates[k];
      if (!is_finite(d.mrt_s[k]) || d.mrt_s[k] <= 0.0 || d.mrt_s[k] >= 2.0)
        return fail(nullptr, IBM_ERR_INVALID, "MRT rates must lie in (0, 2)");
    }
  }
  if (d.nx < 4 || d.ny < 4) return fail(nullptr, IBM_ERR_INVALID, "nx and ny must be >= 4");
  if ((long long)d.nx * d.ny >= (1LL << 31) || d.ny > 65535)
    return fail(nullptr, IBM_ERR_INVALID, "lattice too large (nx*ny < 2^31, ny <= 65535)");
  if (!is_finite(d.tau) || d.tau <= 0.5) return fail(nullptr, IBM_ERR_INVALID, "tau must be finite and > 0.5");
  if (!is_finite(d.rho0) || d.rho0 <= 0.0) return fail(nullptr, IBM_ERR_INVALID, "rho0 must be finite and > 0");
  if (d.prec < 0 || d.prec > 3) return fail(nullptr, IBM_ERR_INVALID, "unknown precision");
  for (int s = 0; s < 4; ++s) {
    if (d.bc[s] < 0 || d.bc[s] > 6) return fail(nullptr, IBM_ERR_INVALID, "unknown boundary rule");
    if (!is_finite(d.wall_u[s][0]) || !is_finite(d.wall_u[s][1]))
      return fail(nullptr, IBM_ERR_INVALID, "wall velocity not finite");
  }
  if ((d.bc[0] == IBM_BC_PERIODIC) != (d.bc[1] == IBM_BC_PERIODIC) ||
      (d.bc[2] == IBM_BC_PERIODIC) != (d.bc[3] == IBM_BC_PERIODIC))
    return fail(nullptr, IBM_ERR_INVALID, "periodic sides must be paired");
  for (int s = 1; s < 4; ++s)
    if (d.bc[s] == IBM_BC_INLET_EQ || d.bc[s] == IBM_BC_INLET_NEE)
      return fail(nullptr, IBM_ERR_INVALID, "inlet supported on the -x side only");
  for (int s = 0; s < 4; ++s)
    if (s != 1 && d.bc[s] == IBM_BC_OUTLET_NEE)
      return fail(nullptr, IBM_ERR_INVALID, "outlet supported on the +x side only");
  if (d.bc[0] == IBM_BC_OUTLET_ZEROGRAD || d.bc[2] == IBM_BC_OUTLET_ZEROGRAD ||
      d.bc[3] == IBM_BC_OUTLET_ZEROGRAD)
    return fail(nullptr, IBM_ERR_INVALID, "outlet supported on the +x side only");
  if (!is_finite(d.inlet_u[0]) || !is_finite(d.inlet_u[1]))
    return fail(nullptr, IBM_ERR_INVALID, "inlet velocity not finite");
  if (d.n_corr < 0 || d.n_corr > 1000) return fail(nullptr, IBM_ERR_INVALID, "n_corr must be in [0, 1000]");
  if (!is_finite(d.corr_tol) || d.corr_tol < 0) return fail(nullptr, IBM_ERR_INVALID, "corr_tol must be >= 0");
  if (d.delta_points == 0) d.delta_points = 4;
  if (d.delta_points < 2 || d.delta_points > 4)
    return fail(nullptr, IBM_ERR_INVALID, "delta_points must be 2, 3 or 4 (Eq. 15a-c)");

  ibm_ctx* h = nullptr;
  try {
    h = new ibm_ctx();
  } catch (...) {
    return fail(nullptr, IBM_ERR_NOMEM, "host allocation failed");
  }
  DeviceGuard guard(d.device);
  if (!guard.ok) { delete h; return fail(nullptr, IBM_ERR_CUDA, "cannot select the CUDA device"); }
  Ctx& c = *h;
  c.pool = pool;
  c.desc = d;
  c.device = d.device;
  c.prec = d.prec;
  c.s_bytes = d.prec == IBM_FP64 ? 8 : (d.prec == IBM_FP32 ? 4 : 2);
  c.r_bytes = d.prec == IBM_FP64 ? 8 : 4;
  c.geom.nx = d.nx;
  c.geom.ny = d.ny;
  c.geom.nxp = (d.nx + 31) / 32 * 32;
  c.geom.plane = (long long)d.ny * c.geom.nxp;
  c.nseg_x = c.geom.nxp / kSegW;
  for (int s = 0; s < 4; ++s) c.geom.bc[s] = d.bc[s];
  auto bail = [&](ibm_status st) {
    t_err = c.err;
    ibm_destroy(h);
    return st;
  };
  if (d.cuda_stream) {
    c.stream = (cudaStream_t)d.cuda_stream;
  } else {
    if (cudaStreamCreate(&c.stream) != cudaSuccess) {
      cudaGetLastError();
      c.err = "cudaStreamCreate failed";
      c.stream = nullptr;
      return bail(IBM_ERR_CUDA);
    }
    c.own_stream = true;
  }
  {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    c.ib_prio = hi;   // numerically lowest = highest priority
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d.device);
    const int per_sm = ib_blocks_per_sm(d.prec);
    if (sms <= 0 || per_sm < 1) {
      cudaGetLastError();
      c.err = "the correction-loop kernel cannot be resident on this device";
      return bail(IBM_ERR_CUDA);
    }
    c.ib_grid = sms;
    c.ib_grid_max = sms;
    if (cudaStreamCreateWithPriority(&c.ib_stream, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      c.err = "creating the correction-loop stream or its events failed";
      return bail(IBM_ERR_CUDA);
    }
  }
  ibm_status st = IBM_OK;
  do {
    c.f = dev_alloc(c, c.s_bytes * 9 * (size_t)c.geom.plane);
    c.macro = dev_alloc(c, c.r_bytes * 3 * (size_t)d.nx * d.ny);
    c.dnode2band = (int*)dev_alloc(c, sizeof(int) * (size_t)d.nx * d.ny);
    c.dctr = (int*)dev_alloc(c, CTR_COUNT * sizeof(int));
    c.dbar = (unsigned long long*)dev_alloc(c, sizeof(unsigned long long));
    c.dsegflag = (int*)dev_alloc(c, sizeof(int) * (size_t)c.nseg_x * d.ny);
    c.dresid = dev_alloc(c, c.r_bytes * (d.n_corr + 1));
    if (!c.f || !c.macro || !c.dnode2band || !c.dctr || !c.dresid || !c.dsegflag || !c.dbar) {
      c.err = "device allocation of the lattice failed";
      st = IBM_ERR_NOMEM;
      break;
    }
    if (cudaMemsetAsync(c.f, 0, c.s_bytes * 9 * (size_t)c.geom.plane, c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.dnode2band, 0xFF, sizeof(int) * (size_t)d.nx * d.ny, c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.dctr, 0, CTR_COUNT * sizeof(int), c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.dbar, 0, sizeof(unsigned long long), c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.dsegflag, 0, sizeof(int) * (size_t)c.nseg_x * d.ny, c.stream) != cudaSuccess ||
        cudaMemsetAsync(c.dresid, 0, c.r_bytes * (d.n_corr + 1), c.stream) != cudaSuccess) {
      c.err = std::string("device memset failed: ") + cudaGetErrorString(cudaGetLastError());
      st = IBM_ERR_CUDA;
      break;
    }
    launch_fields(c, FIELD_OP_REST, nullptr, nullptr, c.stream);
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      c.err = std::string("initialisation failed: ") + cudaGetErrorString(e);
      st = IBM_ERR_CUDA;
      break;
    }
  } while (0);
  if (st != IBM_OK) return bail(st);
  *out = h;
  return IBM_OK;
}

// One body and its markers appended to the host copy; with `upload` the
// marker arrays are then re-uploaded (as ibm_add_markers does).
static ibm_status add_body(ibm_handle h, const double* xy, const double* ds, int n, const ibm_body_desc* body,
                           int* body_id_out, bool upload) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (!xy || n <= 0 || !body) return fail(h, IBM_ERR_INVALID, "xy, n > 0 and body are required");
  try {
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(h, IBM_ERR_CUDA, "cannot select the CUDA device");
    Ctx& c = *h;
    const ibm_body_desc& b = *body;
    if (b.kind < 0 || b.kind > 2) return fail(h, IBM_ERR_INVALID, "unknown body kind");
    const double vals[] = {b.xc[0], b.xc[1], b.u[0], b.u[1], b.omega, b.theta, b.rho_s, b.rho_f,
                           b.volume, b.inertia, b.radius, b.gravity[0], b.gravity[1]};
    for (double v : vals)
      if (!is_finite(v)) return fail(h, IBM_ERR_INVALID, "body description has a non-finite value");
    if (b.kind == IBM_BODY_FREE &&
        (b.rho_s <= 0 || b.rho_f <= 0 || b.volume <= 0 || b.inertia <= 0 || b.radius <= 0))
      return fail(h, IBM_ERR_INVALID, "a free body needs rho_s, rho_f, volume, inertia, radius > 0");
    std::vector<double> mds(n);
    for (int k = 0; k < n; ++k)
      if (!is_finite(xy[2 * k]) || !is_finite(xy[2 * k + 1]))
        return fail(h, IBM_ERR_INVALID, "marker position not finite");
    if (ds) {
      for (int k = 0; k < n; ++k) {
        if (!is_finite(ds[k]) || ds[k] <= 0) return fail(h, IBM_ERR_INVALID, "ds must be finite and > 0");
        mds[k] = ds[k];
      }
    } else {
      double per = 0.0;
      for (int k = 0; k < n; ++k) {
        const int k2 = (k + 1) % n;
        per += std::hypot(xy[2 * k2] - xy[2 * k], xy[2 * k2 + 1] - xy[2 * k + 1]);
      }
      if (!(per > 0)) return fail(h, IBM_ERR_INVALID, "cannot derive ds from a zero perimeter");
      for (int k = 0; k < n; ++k) mds[k] = per / n;
    }
    // The 4 x 4 support of every marker must stay inside closed axes and off
    // the inlet / outlet columns (and off the inner neighbour of an
    // extrapolation side, which rebuilds the boundary column).
    const Geom& g = c.geom;
    for (int k = 0; k < n; ++k) {
      const long long bx = (long long)std::floor(xy[2 * k]) - 1, by = (long long)std::floor(xy[2 * k + 1]) - 1;
      if (g.bc[0] != BC_PERIODIC) {
        const long long lo = g.bc[0] == BC_INLET ? 1 : (g.bc[0] == BC_INLET_NEE ? 2 : 0);
        const long long hi = g.bc[1] == BC_OUTLET ? g.nx - 3 : (g.bc[1] == BC_OUTLET_NEE ? g.nx - 3 : g.nx - 1);
        if (bx < lo || bx + 3 > hi)
          return fail(h, IBM_ERR_INVALID, "a marker support leaves the domain or touches an inlet/outlet column");
      }
      if (g.bc[2] != BC_PERIODIC && (by < 0 || by + 3 > g.ny - 1))
        return fail(h, IBM_ERR_INVALID, "a marker support leaves the domain in y");
    }
    {
      ibm_status st = download_moving_state(h);
      if (st != IBM_OK) return st;
    }
    BodyDev B{};
    B.kind = b.kind;
    B.m0 = c.nm;
    B.m1 = c.nm + n;
    B.xc[0] = b.xc[0]; B.xc[1] = b.xc[1];
    B.u[0] = b.u[0]; B.u[1] = b.u[1];
    B.omega = b.omega; B.theta = b.theta;
    B.u_prev[0] = b.u[0]; B.u_prev[1] = b.u[1];
    B.omega_prev = b.omega; B.theta0 = b.theta;
    B.rho_s = b.rho_s; B.rho_f = b.rho_f; B.volume = b.volume; B.inertia = b.inertia;
    B.radius = b.radius; B.mass = b.rho_s * b.volume;
    B.gravity[0] = b.gravity[0]; B.gravity[1] = b.gravity[1];
    for (int k = 0; k < n; ++k) {
      const double X = xy[2 * k], Y = xy[2 * k + 1];
      c.hX.push_back(X);
      c.hY.push_back(Y);
      c.hds.push_back(mds[k]);
      c.hdX.push_back(X - b.xc[0]);
      c.hdY.push_back(Y - b.xc[1]);
      c.hUx.push_back(b.u[0] - b.omega * (Y - b.xc[1]));
      c.hUy.push_back(b.u[1] + b.omega * (X - b.xc[0]));
      c.hmbody.push_back(c.nb);
    }
    c.hbodies.push_back(B);
    c.nm += n;
    const int id = c.nb++;
    if (b.kind != IBM_BODY_FIXED) c.any_moving = true;
    if (upload) {
      ibm_status st = upload_markers(h);
      if (st != IBM_OK) {
        c.broken = true;                 // marker arrays are partly released
        return st;
      }
    }
    if (body_id_out) *body_id_out = id;
    return IBM_OK;
  } catch (const std::bad_alloc&) {
    return fail(h, IBM_ERR_NOMEM, "host allocation failed");
  } catch (...) {
    return fail(h, IBM_ERR_INVALID, "unexpected error in ibm_add_markers");
  }
}

// Every body of a case, then one upload of the marker arrays (the serving
// layer's admission: one round trip instead of one per body).
ibm_status ibm::add_bodies(ibm_handle h, int nbodies, const ibm_body_desc* bodies, const int* nmark,
                           const double* xy, const double* ds) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  size_t off = 0;
  for (int b = 0; b < nbodies; ++b) {
    ibm_status st = add_body(h, xy + 2 * off, ds ? ds + off : nullptr, nmark[b], &bodies[b], nullptr, false);
    if (st != IBM_OK) {
      h->broken = true;                  // the host copy holds bodies the device has not seen
      return st;
    }
    off += nmark[b];
  }
  if (nbodies == 0) return IBM_OK;
  try {
    DeviceGuard guard(h->device);
    ibm_status st = upload_markers(h);
    if (st != IBM_OK) h->broken = true;
    return st;
  } catch (const std::bad_alloc&) {
    h->broken = true;
    return fail(h, IBM_ERR_NOMEM, "host allocation failed");
  }
}

extern "C" {

ibm_status ibm_create_lattice(const ibm_lattice_desc* desc, ibm_handle* out) {
  return ibm::create_lattice(desc, out, nullptr);
}

ibm_status ibm_add_markers(ibm_handle h, const double* xy, const double* ds, int n,
                           const ibm_body_desc* body, int* body_id_out) {
  return add_body(h, xy, ds, n, body, body_id_out, true);
}

ibm_status ibm_step(ibm_handle h, int nsteps, unsigned flags) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (nsteps < 0) return fail(h, IBM_ERR_INVALID, "nsteps must be >= 0");
  if (nsteps == 0) return IBM_OK;
  try {
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(h, IBM_ERR_CUDA, "cannot select the CUDA device");
    Ctx& c = *h;
    if (c.broken)
      return fail(h, IBM_ERR_INVALID, "a failed marker upload left this lattice unusable; destroy it");
    const bool timing = (flags & IBM_STEP_TIME_KERNELS) != 0;
    const bool use_graph = !(flags & (IBM_STEP_NO_GRAPH | IBM_STEP_TIME_KERNELS));
    if (timing && c.ev.empty()) {
      c.ev.resize(kEventsPerStep * kEventPairs);
      for (auto& e : c.ev) IBM_CK(h, cudaEventCreate(&e));
    }
    if (c.nm > 0 && !c.band_valid) {
      launch_band_build(c, c.stream);
      c.band_valid = true;
      if (c.ib_phases == 1) {
        ibm_status st = count_band(h);
        if (st != IBM_OK) return st;
      }
    }
    const bool want_macro = !(flags & IBM_STEP_NO_MACRO);
    for (int k = 0; k < nsteps;) {
      const int parity = c.parity;
      // whole blocks of steps that write no output fields go as one graph
      const int plain = nsteps - k - (want_macro ? 1 : 0);
      if (use_graph && plain >= kBlockSteps) {
        if (!c.graph_block[parity]) {
          cudaError_t e = capture_steps(c, parity, kBlockSteps, false, &c.graph_block[parity]);
          if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, IBM_ERR_CUDA, std::string("capturing a block of steps: ") + cudaGetErrorString(e));
          }
        }
        IBM_CK(h, cudaGraphLaunch(c.graph_block[parity], c.stream));
        c.launches += (long long)kBlockSteps * kernels_per_step(c);
        c.steps += kBlockSteps;
        c.watch_due += kBlockSteps;
        watchdog_if_due(c);
        k += kBlockSteps;
        continue;
      }
      const int macro = (k == nsteps - 1 && want_macro) ? 1 : 0;
      ++k;
      if (use_graph) {
        if (!c.graph[parity][macro]) {
          cudaError_t e = capture_steps(c, parity, 1, macro != 0, &c.graph[parity][macro]);
          if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(h, IBM_ERR_CUDA, std::string("capturing a step: ") + cudaGetErrorString(e));
          }
        }
        IBM_CK(h, cudaGraphLaunch(c.graph[parity][macro], c.stream));
      } else {
        if (timing && c.ev_used >= kEventPairs) {
          ibm_status st = fold_events(h);
          if (st != IBM_OK) return st;
        }
        enqueue_step(c, parity, macro != 0, timing);
        IBM_CK(h, cudaGetLastError());
      }
      c.parity ^= 1;
      c.launches += kernels_per_step(c);
      c.steps += 1;
      c.watch_due += 1;
      watchdog_if_due(c);
    }
    IBM_CK(h, cudaGetLastError());
    // with a tolerance, the call waits for its steps and reports a residual
    // above it (or any device error) at once
    if (c.desc.corr_tol > 0 && c.nm > 0) return sync_stream(h);
    return IBM_OK;
  } catch (...) {
    return fail(h, IBM_ERR_INVALID, "unexpected error in ibm_step");
  }
}

ibm_status ibm_set_marker_velocities(ibm_handle h, const double* uv, int n) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (!uv || n != h->nm) return fail(h, IBM_ERR_INVALID, "uv must hold one (u_x, u_y) pair per marker");
  for (int k = 0; k < 2 * n; ++k)
    if (!is_finite(uv[k])) return fail(h, IBM_ERR_INVALID, "marker velocity not finite");
  if (n == 0) return IBM_OK;
  try {
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(h, IBM_ERR_CUDA, "cannot select the CUDA device");
    Ctx& c = *h;
    const int R = c.r_bytes;
    std::vector<char> ux((size_t)R * n), uy((size_t)R * n);
    for (int l = 0; l < n; ++l) {
      if (c.hbodies[c.hmbody[l]].kind != IBM_BODY_FIXED) continue;
      c.hUx[l] = uv[2 * l];
      c.hUy[l] = uv[2 * l + 1];
    }
    for (int l = 0; l < n; ++l) {
      if (R == 8) { ((double*)ux.data())[l] = c.hUx[l]; ((double*)uy.data())[l] = c.hUy[l]; }
      else { ((float*)ux.data())[l] = (float)c.hUx[l]; ((float*)uy.data())[l] = (float)c.hUy[l]; }
    }
    // Pageable sources are staged before cudaMemcpyAsync returns, so the
    // temporaries may go; the copies are ordered before the next step.
    if (c.any_moving) {
      // moving markers' device velocities are newer than hUx: copy only
      // the fixed bodies' marker ranges
      int l = 0;
      while (l < n) {
        if (c.hbodies[c.hmbody[l]].kind != IBM_BODY_FIXED) { ++l; continue; }
        int e = l;
        while (e < n && c.hmbody[e] == c.hmbody[l]) ++e;
        IBM_CK(h, cudaMemcpyAsync((char*)c.dUx + (size_t)R * l, ux.data() + (size_t)R * l, (size_t)R * (e - l),
                                  cudaMemcpyHostToDevice, c.stream));
        IBM_CK(h, cudaMemcpyAsync((char*)c.dUy + (size_t)R * l, uy.data() + (size_t)R * l, (size_t)R * (e - l),
                                  cudaMemcpyHostToDevice, c.stream));
        l = e;
      }
    } else {
      IBM_CK(h, cudaMemcpyAsync(c.dUx, ux.data(), (size_t)R * n, cudaMemcpyHostToDevice, c.stream));
      IBM_CK(h, cudaMemcpyAsync(c.dUy, uy.data(), (size_t)R * n, cudaMemcpyHostToDevice, c.stream));
    }
    return IBM_OK;
  } catch (...) {
    return fail(h, IBM_ERR_NOMEM, "host allocation failed");
  }
}

ibm_status ibm_sync(ibm_handle h) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  DeviceGuard guard(h->device);
  return sync_stream(h);
}

ibm_status ibm_read_fields(ibm_handle h, int field, double* host_dst, size_t n_elems) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (!host_dst) return fail(h, IBM_ERR_INVALID, "host_dst is NULL");
  try {
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(h, IBM_ERR_CUDA, "cannot select the CUDA device");
    Ctx& c = *h;
    const size_t n = (size_t)c.geom.nx * c.geom.ny;
    ibm_status st = sync_stream(h);
    if (st != IBM_OK) return st;
    switch (field) {
      case IBM_FIELD_RHO:
      case IBM_FIELD_UX:
      case IBM_FIELD_UY: {
        if (n_elems != n) return fail(h, IBM_ERR_INVALID, "n_elems must be nx*ny");
        if ((st = ensure_io(h, 3 * n)) != IBM_OK) return st;
        launch_fields(c, FIELD_OP_MACRO_OUT, nullptr, c.dio, c.stream);
        const size_t off = (size_t)(field - IBM_FIELD_RHO) * n;
        IBM_CK(h, cudaMemcpyAsync(host_dst, c.dio + off, 8 * n, cudaMemcpyDeviceToHost, c.stream));
        break;
      }
      case IBM_FIELD_F: {
        if (n_elems != 9 * n) return fail(h, IBM_ERR_INVALID, "n_elems must be 9*nx*ny");
        if ((st = ensure_io(h, 9 * n)) != IBM_OK) return st;
        launch_fields(c, FIELD_OP_READ_F, nullptr, c.dio, c.stream);
        IBM_CK(h, cudaMemcpyAsync(host_dst, c.dio, 8 * 9 * n, cudaMemcpyDeviceToHost, c.stream));
        break;
      }
      case IBM_FIELD_BODIES: {
        if (n_elems != (size_t)9 * c.nb) return fail(h, IBM_ERR_INVALID, "n_elems must be 9*nbodies");
        std::vector<BodyDev> bd(c.nb);
        if (c.nb)
          IBM_CK(h, cudaMemcpyAsync(bd.data(), c.dbodies, sizeof(BodyDev) * c.nb, cudaMemcpyDeviceToHost,
                                    c.stream));
        IBM_CK(h, cudaStreamSynchronize(c.stream));
        for (int b = 0; b < c.nb; ++b) {
          double* o = host_dst + 9 * b;
          o[0] = bd[b].xc[0]; o[1] = bd[b].xc[1]; o[2] = bd[b].u[0]; o[3] = bd[b].u[1];
          o[4] = bd[b].omega; o[5] = bd[b].theta; o[6] = bd[b].F_ib[0]; o[7] = bd[b].F_ib[1];
          o[8] = bd[b].T_ib;
        }
        return IBM_OK;
      }
      case IBM_FIELD_BODY_STATE: {
        if (n_elems != (size_t)9 * c.nb) return fail(h, IBM_ERR_INVALID, "n_elems must be 9*nbodies");
        std::vector<BodyDev> bd(c.nb);
        if (c.nb)
          IBM_CK(h, cudaMemcpyAsync(bd.data(), c.dbodies, sizeof(BodyDev) * c.nb, cudaMemcpyDeviceToHost,
                                    c.stream));
        IBM_CK(h, cudaStreamSynchronize(c.stream));
        for (int b = 0; b < c.nb; ++b) {
          double* o = host_dst + 9 * b;
          o[0] = bd[b].xc[0]; o[1] = bd[b].xc[1]; o[2] = bd[b].u[0]; o[3] = bd[b].u[1];
          o[4] = bd[b].omega; o[5] = bd[b].theta; o[6] = bd[b].u_prev[0]; o[7] = bd[b].u_prev[1];
          o[8] = bd[b].omega_prev;
        }
        return IBM_OK;
      }
      case IBM_FIELD_RESIDUAL: {
        const int N = c.desc.n_corr;
        if (n_elems != (size_t)N + 1) return fail(h, IBM_ERR_INVALID, "n_elems must be n_corr+1");
        std::vector<char> raw(c.r_bytes * (N + 1));
        IBM_CK(h, cudaMemcpyAsync(raw.data(), c.dresid, raw.size(), cudaMemcpyDeviceToHost, c.stream));
        IBM_CK(h, cudaStreamSynchronize(c.stream));
        for (int k = 0; k <= N; ++k)
          host_dst[k] = c.r_bytes == 8 ? ((double*)raw.data())[k] : (double)((float*)raw.data())[k];
        if (c.desc.corr_tol > 0 && !(host_dst[N] <= c.desc.corr_tol))
          return fail(h, IBM_WARN_NOT_CONVERGED, "no-slip residual above corr_tol after n_corr iterations");
        return IBM_OK;
      }
      case IBM_FIELD_MARKERS: {
        if (n_elems != (size_t)2 * c.nm) return fail(h, IBM_ERR_INVALID, "n_elems must be 2*nmarkers");
        std::vector<double> X(c.nm), Y(c.nm);
        if (c.nm) {
          IBM_CK(h, cudaMemcpyAsync(X.data(), c.dX, 8 * c.nm, cudaMemcpyDeviceToHost, c.stream));
          IBM_CK(h, cudaMemcpyAsync(Y.data(), c.dY, 8 * c.nm, cudaMemcpyDeviceToHost, c.stream));
        }
        IBM_CK(h, cudaStreamSynchronize(c.stream));
        for (int l = 0; l < c.nm; ++l) { host_dst[2 * l] = X[l]; host_dst[2 * l + 1] = Y[l]; }
        return IBM_OK;
      }
      default:
        return fail(h, IBM_ERR_INVALID, "unknown field");
    }
    IBM_CK(h, cudaStreamSynchronize(c.stream));
    IBM_CK(h, cudaGetLastError());
    return IBM_OK;
  } catch (...) {
    return fail(h, IBM_ERR_INVALID, "unexpected error in ibm_read_fields");
  }
}

ibm_status ibm_write_fields(ibm_handle h, int field, const double* host_src, size_t n_elems) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (!host_src) return fail(h, IBM_ERR_INVALID, "host_src is NULL");
  try {
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(h, IBM_ERR_CUDA, "cannot select the CUDA device");
    Ctx& c = *h;
    const size_t n = (size_t)c.geom.nx * c.geom.ny;
    ibm_status st = IBM_OK;
    if (field == IBM_FIELD_F) {
      if (n_elems != 9 * n) return fail(h, IBM_ERR_INVALID, "n_elems must be 9*nx*ny");
      for (size_t k = 0; k < 9 * n; ++k)
        if (!is_finite(host_src[k])) return fail(h, IBM_ERR_INVALID, "populations must be finite");
      if ((st = ensure_io(h, 9 * n)) != IBM_OK) return st;
      IBM_CK(h, cudaMemcpyAsync(c.dio, host_src, 8 * 9 * n, cudaMemcpyHostToDevice, c.stream));
      launch_fields(c, FIELD_OP_WRITE_F, c.dio, nullptr, c.stream);
      c.parity = 0;
      launch_fields(c, FIELD_OP_MACROS, nullptr, nullptr, c.stream);
    } else if (field == IBM_FIELD_MACRO_INIT) {
      if (n_elems != 3 * n) return fail(h, IBM_ERR_INVALID, "n_elems must be 3*nx*ny");
      for (size_t k = 0; k < 3 * n; ++k)
        if (!is_finite(host_src[k])) return fail(h, IBM_ERR_INVALID, "fields must be finite");
      for (size_t k = 0; k < n; ++k)
        if (!(host_src[k] > 0)) return fail(h, IBM_ERR_INVALID, "density must be > 0");
      if ((st = ensure_io(h, 3 * n)) != IBM_OK) return st;
      IBM_CK(h, cudaMemcpyAsync(c.dio, host_src, 8 * 3 * n, cudaMemcpyHostToDevice, c.stream));
      launch_fields(c, FIELD_OP_INIT_EQ, c.dio, nullptr, c.stream);
      c.parity = 0;
    } else if (field == IBM_FIELD_BODY_STATE) {
      if (n_elems != (size_t)9 * c.nb) return fail(h, IBM_ERR_INVALID, "n_elems must be 9*nbodies");
      for (size_t k = 0; k < n_elems; ++k)
        if (!is_finite(host_src[k])) return fail(h, IBM_ERR_INVALID, "body state must be finite");
      if (c.nb == 0) return IBM_OK;
      // the rest of each record (kind, marker range, mass properties,
      // reference angle, last forces) stays as it is on the device
      std::vector<BodyDev> bd(c.nb);
      IBM_CK(h, cudaMemcpyAsync(bd.data(), c.dbodies, sizeof(BodyDev) * c.nb, cudaMemcpyDeviceToHost, c.stream));
      IBM_CK(h, cudaStreamSynchronize(c.stream));
      for (int b = 0; b < c.nb; ++b) {
        const double* v = host_src + 9 * b;
        bd[b].xc[0] = v[0]; bd[b].xc[1] = v[1]; bd[b].u[0] = v[2]; bd[b].u[1] = v[3];
        bd[b].omega = v[4]; bd[b].theta = v[5]; bd[b].u_prev[0] = v[6]; bd[b].u_prev[1] = v[7];
        bd[b].omega_prev = v[8];
      }
      IBM_CK(h, cudaMemcpyAsync(c.dbodies, bd.data(), sizeof(BodyDev) * c.nb, cudaMemcpyHostToDevice, c.stream));
      IBM_CK(h, cudaStreamSynchronize(c.stream));
      // markers to the new pose; the band follows them before the next step
      if (c.any_moving && c.nm > 0) {
        launch_marker_move(c, c.stream);
        c.band_valid = false;
      }
    } else {
      return fail(h, IBM_ERR_INVALID, "field is not writable");
    }
    return sync_stream(h);
  } catch (...) {
    return fail(h, IBM_ERR_INVALID, "unexpected error in ibm_write_fields");
  }
}

ibm_status ibm_kernel_times(ibm_handle h, double* ms_total, int* launches) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  DeviceGuard guard(h->device);
  ibm_status st = fold_events(h);
  if (st != IBM_OK) return st;
  if (ms_total) *ms_total = h->acc_ms;
  if (launches) *launches = h->acc_n;
  h->acc_ms = 0.0;
  h->acc_n = 0;
  return IBM_OK;
}

ibm_status ibm_get_sizes(ibm_handle h, long long* nodes, int* markers, int* bodies, int* band_nodes,
                         int* band_segments) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  DeviceGuard guard(h->device);
  if (nodes) *nodes = (long long)h->geom.nx * h->geom.ny;
  if (markers) *markers = h->nm;
  if (bodies) *bodies = h->nb;
  if (band_nodes || band_segments) {
    int ctr[CTR_COUNT] = {0, 0, 0, 0};
    if (h->nm > 0 && !h->band_valid) {
      launch_band_build(*h, h->stream);
      h->band_valid = true;
    }
    IBM_CK(h, cudaMemcpyAsync(ctr, h->dctr, sizeof(ctr), cudaMemcpyDeviceToHost, h->stream));
    IBM_CK(h, cudaStreamSynchronize(h->stream));
    if (band_nodes) *band_nodes = h->nm > 0 ? ctr[CTR_NBAND] : 0;
    if (band_segments) *band_segments = h->nm > 0 ? ctr[CTR_NSEG] : 0;
  }
  return IBM_OK;
}

ibm_status ibm_autotune_ib(ibm_handle h, const int* candidates, int n, int steps_each, int* best,
                           double* best_us) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (steps_each < 2) return fail(h, IBM_ERR_INVALID, "steps_each must be >= 2");
  if (n < 0 || (n > 0 && !candidates)) return fail(h, IBM_ERR_INVALID, "invalid candidate list");
  for (int k = 0; k < n; ++k)
    if (candidates[k] < 0) return fail(h, IBM_ERR_INVALID, "negative candidate");
  std::vector<int> cand(candidates, candidates + n);
  if (cand.empty()) {
    // one CTA, a cluster, and 1/2, 3/4 and all of the SMs
    const int sms = h->ib_grid_max;
    for (int v : {1, 8, 16, sms / 2, (3 * sms + 3) / 4, sms})
      if (v >= 1 && std::find(cand.begin(), cand.end(), v) == cand.end()) cand.push_back(v);
  }
  if (h->nm == 0) {                      // nothing to tune: no correction kernel
    if (best) *best = 0;
    if (best_us) *best_us = 0.0;
    return IBM_OK;
  }
  try {
    DeviceGuard guard(h->device);
    if (!guard.ok) return fail(h, IBM_ERR_CUDA, "cannot select the CUDA device");
    cudaEvent_t e0, e1;
    IBM_CK(h, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaGetLastError();
      return fail(h, IBM_ERR_CUDA, "cudaEventCreate failed");
    }
    int pick = cand[0];
    float pick_ms = -1.0f;
    ibm_status st = IBM_OK;
    for (int v : cand) {
      if ((st = ibm_set_option(h, IBM_OPT_IB_CTAS, v)) != IBM_OK) break;
      // two untimed steps build both step kinds' graphs for this setting
      if ((st = ibm_step(h, 2, IBM_STEP_NO_MACRO)) != IBM_OK) break;
      cudaEventRecord(e0, h->stream);
      if ((st = ibm_step(h, steps_each, IBM_STEP_NO_MACRO)) != IBM_OK) break;
      cudaEventRecord(e1, h->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = IBM_ERR_CUDA; break; }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (pick_ms < 0.0f || ms < pick_ms) { pick_ms = ms; pick = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != IBM_OK) {
      if (st == IBM_ERR_CUDA) { cudaGetLastError(); return fail(h, st, "timing the candidates failed"); }
      return st;
    }
    if ((st = ibm_set_option(h, IBM_OPT_IB_CTAS, pick)) != IBM_OK) return st;
    if (best) *best = pick;
    if (best_us) *best_us = 1e3 * (double)pick_ms / steps_each;
    return check_device_flags(h);
  } catch (...) {
    return fail(h, IBM_ERR_NOMEM, "host allocation failed");
  }
}

ibm_status ibm_set_option(ibm_handle h, int option, long long value) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (option == IBM_OPT_IB_THREADS) {
    if (value != 256 && value != 512 && value != 1024)
      return fail(h, IBM_ERR_INVALID, "IBM_OPT_IB_THREADS must be 256, 512 or 1024");
    DeviceGuard guard(h->device);
    if (ib_blocks_per_sm(h->prec, (int)value) < 1)
      return fail(h, IBM_ERR_INVALID, "the correction kernel cannot be resident with that many threads");
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->ib_threads = (int)value;
    h->ib_cluster_max = -1;
    choose_ib_grid(*h);
    destroy_graphs(*h);
    return IBM_OK;
  }
  if (option == IBM_OPT_IB_PHASES) {
    if (value < 0 || value > 2) return fail(h, IBM_ERR_INVALID, "IBM_OPT_IB_PHASES must be 0, 1 or 2");
    DeviceGuard guard(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->ib_phases = (int)value;
    choose_ib_grid(*h);
    destroy_graphs(*h);
    if (h->ib_phases == 1 && h->band_valid) return count_band(h);
    return IBM_OK;
  }
  if (option == IBM_OPT_WATCHDOG_STEPS) {
    if (value < 0 || value > (1LL << 40)) return fail(h, IBM_ERR_INVALID, "IBM_OPT_WATCHDOG_STEPS out of range");
    h->watchdog_steps = (int)std::min<long long>(value, 1 << 30);
    h->watch_due = 0;
    return IBM_OK;
  }
  if (option == IBM_OPT_BARRIER_LIMIT_US || option == IBM_OPT_TEST_DROP_ARRIVAL) {
    if (option == IBM_OPT_BARRIER_LIMIT_US && (value < 100 || value > 60000000))
      return fail(h, IBM_ERR_INVALID, "IBM_OPT_BARRIER_LIMIT_US must be in [100, 6e7]");
    if (option == IBM_OPT_TEST_DROP_ARRIVAL && value != 0 && value != 1)
      return fail(h, IBM_ERR_INVALID, "IBM_OPT_TEST_DROP_ARRIVAL must be 0 or 1");
    DeviceGuard guard(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (option == IBM_OPT_BARRIER_LIMIT_US) h->bar_limit_ns = value * 1000LL;
    else h->test_drop_arrival = (int)value;
    destroy_graphs(*h);                  // the kernels take both as arguments
    return IBM_OK;
  }
  if (option != IBM_OPT_IB_CTAS) return fail(h, IBM_ERR_INVALID, "unknown option");
  if (value < 0 || value > (1 << 20)) return fail(h, IBM_ERR_INVALID, "IBM_OPT_IB_CTAS out of range");
  h->ib_grid_opt = (int)value;
  DeviceGuard guard(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  choose_ib_grid(*h);
  destroy_graphs(*h);
  return IBM_OK;
}

ibm_status ibm_get_counters(ibm_handle h, long long* kernel_launches, long long* steps) {
  if (!h) return fail(nullptr, IBM_ERR_INVALID, "handle is NULL");
  if (kernel_launches) *kernel_launches = h->launches;
  if (steps) *steps = h->steps;
  return IBM_OK;
}

ibm_status ibm_destroy(ibm_handle h) {
  if (!h) return IBM_OK;
  ibm_status st = IBM_OK;
  {
    DeviceGuard guard(h->device);
    if (h->stream && cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaGetLastError();
      st = IBM_ERR_CUDA;
    }
    destroy_graphs(*h);
    for (auto& e : h->ev) cudaEventDestroy(e);
    std::vector<void*> all = h->allocs;
    for (void* p : all) dev_free(*h, p);
    for (void* c : h->chunks) cudaFreeAsync(c, h->stream);
    h->chunks.clear();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (h->ib_stream) cudaStreamDestroy(h->ib_stream);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
  }
  delete h;
  return st;
}

}  // extern "C"
