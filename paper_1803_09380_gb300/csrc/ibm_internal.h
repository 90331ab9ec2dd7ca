// ibm_internal.h -- the library-side state behind an ibm_handle and the
// launchers each translation unit provides.  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ibm.h"
#include "ibm_device.cuh"

namespace ibm {

// FP64 record of one rigid body on the device (Eqs. 37-42 state).
struct BodyDev {
  int kind, m0, m1, pad;
  double xc[2], u[2], omega, theta;
  double u_prev[2], omega_prev, theta0;
  double rho_s, rho_f, volume, inertia, radius, mass;
  double gravity[2];
  double F_ib[2], T_ib;     // Eq. 29 sums of the last step (no internal-mass terms)
};

enum { ERR_BAND_CAP = 1, ERR_LIST_CAP = 2, ERR_SEG_CAP = 4, ERR_BARRIER = 8, ERR_G_CAP = 16,
       ERR_DIVERGED = 32,      // a non-finite residual or population (the watchdog)
       WARN_NOT_CONV = 64 };   // r^N above corr_tol (a warning, cleared once reported)

// One entry of a band node's list of covering markers: marker id and its
// spreading weight W_l(x) ds_l.
template <class R>
struct alignas(2 * sizeof(R) > 8 ? 16 : 8) Ent {
  int m;
  R w;
};

constexpr int kIbThreads = 256;                  // threads per correction-loop CTA
constexpr int kGCap = 64;                        // coupled markers per marker (G row)
constexpr int kBlockSteps = 8;       // steps per multi-step graph (even: parity returns)
constexpr int kForceChunk = 128;                 // markers per partial force sum
constexpr int kSmallIbMarkers = 512;             // up to this many markers: one correction CTA
constexpr long long kBarrierNs = 2000000000LL;   // grid-barrier wait limit: 2 s

// Device counters: band nodes, band row segments, error bits.
enum { CTR_NBAND = 0, CTR_NSEG = 1, CTR_ERR = 2, CTR_COUNT = 4 };

// Collide+stream launch modes: every node; every 32-node row segment
// without a band node (runs while the correction loop runs); the band
// segments only (after the correction).
enum { K1_ALL = 0, K1_MAIN = 1 };
constexpr int kSegW = 32;

enum {
  FIELD_OP_READ_F = 0,
  FIELD_OP_WRITE_F = 1,
  FIELD_OP_INIT_EQ = 2,
  FIELD_OP_MACROS = 3,
  FIELD_OP_MACRO_OUT = 4,
  FIELD_OP_REST = 5
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaMemPool_t pool = nullptr;  // set: stream-ordered allocations from this pool
  char* chunk_ptr = nullptr;      // pool mode: free part of the current small-allocation chunk
  size_t chunk_left = 0;
  std::vector<void*> chunks;      // pool mode: the chunks, released with the lattice
  cudaStream_t ib_stream = nullptr;   // high-priority stream of the correction loop
  int ib_prio = 0;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  ibm_lattice_desc desc{};
  Geom geom{};
  int prec = PREC_FP32;
  size_t s_bytes = 4;       // bytes per stored population
  size_t r_bytes = 4;       // bytes per arithmetic value
  void* f = nullptr;        // [9][ny][nxp] populations, AA layout
  void* macro = nullptr;    // [3][ny][nx] rho, ux, uy (arithmetic type)
  int parity = 0;           // 0: natural layout, next step even; 1: swapped, next odd

  // markers (host master copy, FP64)
  std::vector<double> hX, hY, hds, hdX, hdY, hUx, hUy;
  std::vector<int> hmbody;
  std::vector<BodyDev> hbodies;
  int nm = 0, nb = 0;
  int dev_nm = 0, dev_nb = 0;   // markers and bodies of the last upload
  bool any_moving = false;

  // marker / band device arrays (sized for nm markers, 16 nm band nodes)
  int mcap = 0, bcap = 0;
  double *dX = nullptr, *dY = nullptr, *dds = nullptr, *ddX = nullptr, *ddY = nullptr;
  int* dmbody = nullptr;
  void *dUx = nullptr, *dUy = nullptr;       // marker velocity (R)
  void* dW = nullptr;                        // [16 nm] stencil weights (R)
  int* dnode_of = nullptr;                   // [16 nm] stencil node or -1
  int* dband_of = nullptr;                   // [16 nm] band index or -1
  int* dclaim = nullptr;                     // [16 nm]
  int* dnode2band = nullptr;                 // [ny nx] band index or -1
  int* dbnode = nullptr;                     // [bcap] node of band entry
  int* dbcnt = nullptr;                      // [bcap] covering markers
  void* dent = nullptr;                      // [bcap * kBandCap] Ent<R>, ascending marker id
  void* dbq = nullptr;                       // [bcap][8] band-node quantities (R)
  void* dmq = nullptr;                       // [nm][4] rho*, b (R)
  void* dAh = nullptr;                       // [n_corr+1][nm][2] momentum deviations A^n (R)
  void* dCm = nullptr;                       // [nm][3] summed second-moment deviation (R)
  void* dG = nullptr;                        // [nm][kGCap] Ent<R> marker coupling rows
  int* dgcnt = nullptr;                      // [nm]
  void* dresid = nullptr;                    // [n_corr + 1] (R)
  int* dctr = nullptr;                       // CTR_* counters
  int nseg_x = 0;                            // 32-node segments per row
  int segcap = 0;
  int* dsegflag = nullptr;                   // [ny][nseg_x] 1 if the segment has a band node
  int* dseglist = nullptr;                   // [segcap] band segments
  BodyDev* dbodies = nullptr;
  double* dfpart = nullptr;                  // [chunks][nb][3] force partial sums
  unsigned long long* dbar = nullptr;        // grid-barrier arrivals of the correction kernel
  int ib_grid = 0;                           // CTAs of the correction kernel
  int ib_grid_max = 0;                       // one per SM
  int ib_threads = kIbThreads;               // threads per correction-loop CTA: 256, 512, 1024
  bool ib_cluster = false;                   // launch the correction kernel as one cluster
  int ib_cluster_max = -1;                   // largest schedulable cluster (-1: not yet asked)
  int ib_grid_last = 0;                      // grid size the barrier counter is aligned to
  int ib_grid_opt = 0;                       // caller's choice (IBM_OPT_IB_CTAS), 0 = by size
  bool band_collide = true;                  // stream the band segments after the correction
  bool band_valid = false;
  bool broken = false;                       // a failed marker upload left arrays unset
  long long bar_limit_ns = kBarrierNs;       // grid-barrier wait limit (IBM_OPT_BARRIER_LIMIT_US)
  int test_drop_arrival = 0;                 // IBM_OPT_TEST_DROP_ARRIVAL
  int watchdog_steps = 0;                    // IBM_OPT_WATCHDOG_STEPS (0: off)
  int ib_phases = 0;                         // IBM_OPT_IB_PHASES: 0 one persistent kernel, 1 phase
                                             // kernels, 2 Jacobi iterations in one cluster
  int ib_jc_cluster = 0;                     // CTAs of that cluster (0: not available)
  long long nband_host = 0;                  // band nodes at the last count (sizes the phase grids)
  long long watch_due = 0;                   // steps since the last watchdog scan

  // CUDA graphs of one step, per parity and macro flag
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  cudaGraphExec_t graph_block[2] = {nullptr, nullptr};   // kBlockSteps steps from parity p

  // kernel timing: kEventsPerStep events per timed step
  std::vector<cudaEvent_t> ev;
  int ev_used = 0;                           // timed steps recorded
  double acc_ms = 0.0;
  int acc_n = 0;

  // staging for field transfers
  double* dio = nullptr;
  size_t io_cap = 0;

  // counters
  long long launches = 0;   // kernels enqueued by ibm_step
  long long steps = 0;

  std::vector<void*> allocs;
  std::string err;
};

}  // namespace ibm

// The object behind an ibm_handle.
struct ibm_ctx : public ibm::Ctx {};

namespace ibm {

// Number of CUDA kernels one time step launches (matches enqueue_step).
inline int kernels_per_step(const Ctx& h) {
  int k = 1;                                       // collide + stream
  if (has_nee(h.geom)) k += 1;                     // extrapolation columns
  if (h.nm > 0) {
    const int N = h.desc.n_corr;
    (void)N;
    // correction loop (one kernel; one per phase; or pre, cluster, post),
    // band collide+stream
    k += h.ib_phases == 1 ? h.desc.n_corr + 4
         : (h.ib_phases == 2 && h.ib_jc_cluster >= 2 ? (h.desc.n_corr > 1 ? 4 : 3) : 2);
    if (h.nb > 0 && h.any_moving) k += 2 + 6;      // body update, marker move, band rebuild
  }
  return k;
}

template <class R>
StepConsts<R> make_consts(const Ctx& h) {
  StepConsts<R> c;
  const ibm_lattice_desc& d = h.desc;
  c.omega = (R)(1.0 / d.tau);
  c.mrt = d.collision == IBM_COLL_MRT;
  c.mrt_k[0] = (R)((d.mrt_s[0] - 1.0 / d.tau) / 36.0);
  c.mrt_k[1] = (R)((d.mrt_s[1] - 1.0 / d.tau) / 36.0);
  c.mrt_k[2] = (R)((d.mrt_s[2] - 1.0 / d.tau) / 12.0);
  c.rho0 = (R)d.rho0;
  c.inlet_u[0] = (R)d.inlet_u[0];
  c.inlet_u[1] = (R)d.inlet_u[1];
  const double uu = d.inlet_u[0] * d.inlet_u[0] + d.inlet_u[1] * d.inlet_u[1];
  for (int i = 0; i < 9; ++i) {
    const double w = wgt<double>(i);
    for (int s = 0; s < 4; ++s)
      c.wall[s][i] = (R)(6.0 * w * d.rho0 * (cx(i) * d.wall_u[s][0] + cy(i) * d.wall_u[s][1]));
    const double eu = cx(i) * d.inlet_u[0] + cy(i) * d.inlet_u[1];
    c.feq_in[i] = (R)(w * d.rho0 * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu));
  }
  return c;
}

// Kernel launch with a scheduling priority attribute (kept by stream capture,
// so the correction loop's small kernels are dispatched ahead of the waiting
// blocks of the concurrent collide+stream launch).
template <typename... KArgs, typename... Args>
inline void launch_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, int prio,
                        Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// The same launch as one thread-block cluster of grid.x CTAs: the hardware
// schedules the cluster's CTAs together, so a barrier across them can never
// wait for a CTA that is not resident.
template <typename... KArgs, typename... Args>
inline void launch_prio_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t s, int prio,
                                Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = grid.x;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ibm_api.cu
void set_thread_error(const char* msg);
// ibm_create_lattice with an optional memory pool: when pool is not NULL
// every device allocation of the handle is stream-ordered on its stream
// (no device-wide synchronisation when the handle is destroyed).
ibm_status create_lattice(const ibm_lattice_desc* desc, ibm_handle* out, cudaMemPool_t pool);
// ibm_add_markers for every body of a case (nmark[b] markers each, xy and ds
// concatenated body after body, ds may be NULL) with one upload at the end.
ibm_status add_bodies(ibm_handle h, int nbodies, const ibm_body_desc* bodies, const int* nmark, const double* xy,
                      const double* ds);

// ibm_lbm.cu
void launch_collide_stream(const Ctx& h, int parity, bool macro, int mode, cudaStream_t s);
void launch_fields(const Ctx& h, int op, const double* dev_in, double* dev_out, cudaStream_t s);
// Scan of every stored population for NaN/Inf; sets ERR_DIVERGED.
void launch_watchdog(const Ctx& h, cudaStream_t s);

// ibm_batch.cu: the batched serving kernel (one persistent kernel over a
// task queue advancing many lattices).  The table a launch reads is
// [BatchHead, padded to kBatchHeadBytes][cap case records][tasks of one
// round as (case slot, task) int2].
constexpr int kBatchThreads = 256;
constexpr int kBatchHeadBytes = 256;
struct BatchHead {
  unsigned int next;         // next task index to hand out
  unsigned int err;          // nonzero: a wait ran out (the launch's results are void)
  int per_round;             // tasks of one round (one time step of every case)
  int rounds;                // rounds of this launch
  long long wait_ns;         // limit of every wait
  unsigned long long t_start;  // %globaltimer when the first task was taken
};
// One storage precision's batched kernel (instantiated for FP32, FP16 and
// BF16 storage in ibm_batch_f32.cu, ibm_batch_f16.cu, ibm_batch_bf16.cu).
template <int P>
struct BatchOps {
  static size_t case_bytes();
  // CTAs of the batched kernel the device holds at once (0: cannot run).
  static int grid();
  // The case record of lattice h for one launch, written to host memory dst.
  static void record(const Ctx& h, void* dst, int steps, int macro_last, int corr, int tiles, int rows,
                     long long wait_ns);
  static void launch(void* dev_table, int cap, int grid, cudaStream_t s);
  // %globaltimer at which the case of record rec finished its last task
  static unsigned long long end_time(const void* rec);
};

// ibm_ib.cu
void launch_band_build(const Ctx& h, cudaStream_t s);
void launch_ib_loop(const Ctx& h, int parity, bool macro, cudaStream_t s);
int ib_blocks_per_sm(int prec, int threads = kIbThreads);
// Largest number of correction-kernel CTAs (at most kMaxIbCluster) that the
// device can schedule as one cluster; 0 when cluster launches are not
// available.
int ib_max_cluster(int prec, int threads);
constexpr int kMaxIbCluster = 16;
// CTAs of the cluster that runs the Jacobi iterations of M markers (0: none).
int jacobi_cluster_size(int prec, int M);
void launch_body_update(const Ctx& h, cudaStream_t s);
// Rigid motion of every moving body's markers to its current pose (Eqs. 41-42).
void launch_marker_move(const Ctx& h, cudaStream_t s);

}  // namespace ibm
