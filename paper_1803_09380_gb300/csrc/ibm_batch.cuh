// ibm_batch.cuh -- one persistent kernel that advances many resident lattices
// at once: the batched mode of the serving layer (the paper has no
// counterpart; each case is one lattice of the method, stepped exactly as
// ibm_step steps it).
//
// Work queue.  A launch advances every case of a table by up to `rounds`
// time steps.  One round holds, for every case, its correction tasks (the
// nranks CTAs that share its correction loop: Eqs. 22-29, then for moving
// bodies the update of Eqs. 37-42, the marker motion and the band rebuild)
// and its tile tasks (collide+stream of a range of rows, Eqs. 1, 3, 7).  The
// tasks of all rounds form one sequence; resident CTAs take them in order
// from an atomic counter.  Dependencies:
//   correction of round r  after every tile of round r - 1 of the case,
//   tile of round r        after every correction task of round r (a case
//                          without markers: after every tile of round r - 1).
// Each dependency points to tasks earlier in the sequence, which were taken
// by CTAs that are running; so a CTA never waits for a task nobody holds.
// The one exception is the barrier among a case's correction tasks, which
// needs its nranks CTAs resident together (nranks <= 16, far below the
// grid).  Every wait is bounded: when one runs out the launch records an
// error and every later wait gives up at once, so the kernel always drains.
//
// The correction applies its summed correction to the band nodes itself
// (apply = 1), so the tiles collide and stream every node with the vector
// paths of ibm_k1.cuh; results are bitwise those of ibm_step in FP32 and
// FP64 (the 16-bit forms differ from ibm_step's scalar band path in the
// rounding of f - w_i).
//
// Each storage precision is compiled in its own translation unit
// (ibm_batch_f32.cu, ibm_batch_f16.cu, ibm_batch_bf16.cu), which
// instantiates BatchOps<P> from this header.
#pragma once

#include <algorithm>
#include <cstring>

#include "ibm_ib.cuh"

namespace ibm {
namespace {

// The case of one table slot: the correction loop's arguments, what the band
// rebuild of moving bodies writes, and this launch's schedule.  The
// counters start at zero with every upload of the table.
template <int P>
struct alignas(16) BatchCase {
  typedef typename Prec<P>::R R;
  IbArgs<P> ib;
  // band rebuild and marker motion (moving bodies only)
  double *X, *Y;
  const double *dX, *dY;
  R *W, *Ux, *Uy;
  int *node_of, *claim, *band_of, *bcnt, *gcnt, *node2band, *bnode, *segflag;
  Ent<R> *ent, *G;
  int points;
  // schedule of this launch
  int parity;        // AA parity before the launch's first step
  int steps;         // time steps of this case in this launch
  int macro_last;    // write rho, u on the last of them
  int mrt;           // collision operator
  int corr;          // correction tasks per step (0: no markers)
  int tiles;         // tile tasks per step
  int rows;          // rows per tile
  int moving;        // bodies move: update, marker motion, band rebuild
  unsigned int corr_done;    // correction tasks finished
  unsigned int tiles_done;   // tile tasks finished
  unsigned long long t_end;  // %globaltimer when the case's last task of the launch ended
};

// Thread 0 waits until *ctr >= target (acquire), then the CTA continues;
// false when the launch has failed or the wait ran out.
__device__ bool wait_at_least(unsigned int* ctr, unsigned int target, BatchHead* head, int* s_ok) {
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned long long t0 = global_ns();
    for (;;) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(ctr) : "memory");
      if (cur >= target) break;
      unsigned int e;
      asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(e) : "l"(&head->err) : "memory");
      if (e) { ok = 0; break; }
      if ((long long)(global_ns() - t0) > head->wait_ns) {
        atomicOr(&head->err, 1u);
        ok = 0;
        break;
      }
    }
    __threadfence();
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0;
}

// Every thread's writes of the task are done (block barrier); thread 0 then
// publishes them (release) by counting the task as finished.
__device__ __forceinline__ void signal_done(unsigned int* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(ctr) : "memory");
  }
}

// Collide+stream of rows [y0, y1) of one case: warps take the row spans in
// turn; threads then take the extrapolation columns of those rows.
template <int P, int PAR, bool MACRO, bool MRT>
__device__ __noinline__ void batch_tile(const IbArgs<P>& a, int y0, int y1) {
  constexpr int VEC = PAR ? VecTraits<P>::VEC_ODD : VecTraits<P>::VEC;
  const Geom& g = a.g;
  const int wpr = (g.nx + 32 * VEC - 1) / (32 * VEC);
  const int nspan = (y1 - y0) * wpr;
  const int lane = threadIdx.x & 31;
  for (int sp = threadIdx.x >> 5; sp < nspan; sp += kBatchThreads / 32)
    k1_span<P, PAR, MACRO, K1_ALL, MRT>(g, a.c, a.A, a.mac, nullptr, 0, y0 + sp / wpr, sp % wpr, lane);
  if (has_nee(g)) {
    const int rows = y1 - y0;
    for (int q = threadIdx.x; q < 2 * rows; q += kBatchThreads)
      open_column<P, PAR, MACRO, MRT>(g, a.c, a.A, a.mac, q / rows, y0 + q % rows);
  }
}

// The correction loop of one case as a function of its own (its register
// allocation stays separate from the tiles').
template <int P, int PAR>
__device__ __noinline__ void batch_correct(const IbArgs<P>& a, int rank, int nranks) {
  ib_step_body<P, PAR, kBatchThreads>(a, rank, nranks);
}

template <int P>
__device__ void batch_tile_dispatch(const IbArgs<P>& a, int par, bool macro, bool mrt, int y0, int y1) {
  if (par == 0) {
    if (macro) { if (mrt) batch_tile<P, 0, true, true>(a, y0, y1); else batch_tile<P, 0, true, false>(a, y0, y1); }
    else { if (mrt) batch_tile<P, 0, false, true>(a, y0, y1); else batch_tile<P, 0, false, false>(a, y0, y1); }
  } else {
    if (macro) { if (mrt) batch_tile<P, 1, true, true>(a, y0, y1); else batch_tile<P, 1, true, false>(a, y0, y1); }
    else { if (mrt) batch_tile<P, 1, false, true>(a, y0, y1); else batch_tile<P, 1, false, false>(a, y0, y1); }
  }
}

// Bodies of a moving case after its correction, by one CTA: Newton-Euler
// update (Eqs. 37-42), rigid marker motion, and the band rebuild for the next
// step (the phases of the band build separated by block barriers).
template <int P>
__device__ __noinline__ void batch_move(const BatchCase<P>& c) {
  typedef typename Prec<P>::R R;
  const IbArgs<P>& a = c.ib;
  const int M = a.M, T = M * kStencil, NT = kBatchThreads;
  __syncthreads();
  body_update_cta(a.g, a.bodies, a.nb);
  __syncthreads();
  for (int l = threadIdx.x; l < M; l += NT)
    marker_move_item<R>(a.bodies, a.mbody, c.dX, c.dY, c.X, c.Y, c.Ux, c.Uy, l);
  __syncthreads();
  const int nold = min(a.ctr[CTR_NBAND], a.bcap);
  for (int b = threadIdx.x; b < nold; b += NT) band_clear_item(a.g, c.bnode, c.node2band, c.segflag, a.nseg_x, b);
  __syncthreads();
  if (threadIdx.x == 0) { a.ctr[CTR_NBAND] = 0; a.ctr[CTR_NSEG] = 0; }
  for (int t = threadIdx.x; t < T; t += NT)
    band_claim_item<R>(a.g, c.X, c.Y, c.W, c.node_of, c.node2band, c.claim, c.points, t);
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += NT)
    band_alloc_item(c.node_of, c.claim, c.node2band, c.bnode, c.bcnt, a.ctr, a.bcap, t);
  __syncthreads();
  for (int t = threadIdx.x; t < T; t += NT)
    band_fill_item<R>(c.node_of, c.W, a.ds, c.node2band, c.band_of, c.bcnt, c.ent, a.ctr, t);
  __syncthreads();
  const int nnew = min(a.ctr[CTR_NBAND], a.bcap);
  for (int b = threadIdx.x; b < nnew; b += NT) band_sort_item<R>(c.bcnt, c.ent, b);
  __syncthreads();
  for (int l = threadIdx.x; l < M; l += NT) build_g_item<R>(c.band_of, c.W, c.bcnt, c.ent, c.G, c.gcnt, a.ctr, l);
}

template <int P>
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch(unsigned char* table, int cap) {
  BatchHead* head = reinterpret_cast<BatchHead*>(table);
  BatchCase<P>* cases = reinterpret_cast<BatchCase<P>*>(table + kBatchHeadBytes);
  const int2* tasks = reinterpret_cast<const int2*>(table + kBatchHeadBytes + (size_t)cap * sizeof(BatchCase<P>));
  __shared__ BatchCase<P> sc;
  __shared__ unsigned int s_t;
  __shared__ int s_ok;
  const unsigned int per_round = (unsigned int)head->per_round;
  const unsigned int total = per_round * (unsigned int)head->rounds;
  constexpr int kWords = sizeof(BatchCase<P>) / 8;
  static_assert(sizeof(BatchCase<P>) % 8 == 0, "case record copied in 8-byte words");
  for (;;) {
    __syncthreads();                                   // the previous task is done with sc, s_t
    if (threadIdx.x == 0) s_t = atomicAdd(&head->next, 1u);
    __syncthreads();
    const unsigned int t = s_t;
    if (t >= total) break;
    const int r = (int)(t / per_round);
    const int2 tk = tasks[t % per_round];
    BatchCase<P>* gc = cases + tk.x;
    if (t == 0 && threadIdx.x == 0) head->t_start = global_ns();
    if (r >= gc->steps) continue;                      // the case takes fewer steps this launch
    {
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(gc);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(&sc);
      for (int k = threadIdx.x; k < kWords; k += kBatchThreads) dst[k] = src[k];
    }
    __syncthreads();
    if (r >= sc.steps) continue;
    const int par = sc.parity ^ (r & 1);
    if (tk.y < sc.corr) {
      if (!wait_at_least(&gc->tiles_done, (unsigned int)(r * sc.tiles), head, &s_ok)) continue;
      if (par == 0) batch_correct<P, 0>(sc.ib, tk.y, sc.corr);
      else batch_correct<P, 1>(sc.ib, tk.y, sc.corr);
      if (sc.moving) batch_move<P>(sc);
      signal_done(&gc->corr_done);
    } else {
      // after the case's correction of this round -- or, without markers,
      // after every tile of the previous round (the odd step reads the
      // neighbouring rows' slots)
      const bool ok = sc.corr > 0
                          ? wait_at_least(&gc->corr_done, (unsigned int)((r + 1) * sc.corr), head, &s_ok)
                          : wait_at_least(&gc->tiles_done, (unsigned int)(r * sc.tiles), head, &s_ok);
      if (!ok) continue;
      const int k = tk.y - sc.corr;
      const int y0 = k * sc.rows, y1 = min(sc.ib.g.ny, y0 + sc.rows);
      batch_tile_dispatch<P>(sc.ib, par, sc.macro_last && r == sc.steps - 1, sc.mrt != 0, y0, y1);
      signal_done(&gc->tiles_done);
      if (r == sc.steps - 1 && threadIdx.x == 0) atomicMax(&gc->t_end, global_ns());
    }
  }
}

template <int P>
void case_record_t(const Ctx& h, void* dst, int steps, int macro_last, int corr, int tiles, int rows,
                   long long wait_ns) {
  typedef typename Prec<P>::R R;
  BatchCase<P> c;
  std::memset(&c, 0, sizeof(c));
  c.ib = make_ib_args<P>(h);
  c.ib.apply = 1;
  c.ib.cluster = 0;
  c.ib.bar_limit_ns = wait_ns;
  c.ib.drop_arrival = 0;
  c.X = h.dX;
  c.Y = h.dY;
  c.dX = h.ddX;
  c.dY = h.ddY;
  c.W = (R*)h.dW;
  c.Ux = (R*)h.dUx;
  c.Uy = (R*)h.dUy;
  c.node_of = h.dnode_of;
  c.claim = h.dclaim;
  c.band_of = h.dband_of;
  c.bcnt = h.dbcnt;
  c.gcnt = h.dgcnt;
  c.node2band = h.dnode2band;
  c.bnode = h.dbnode;
  c.segflag = h.dsegflag;
  c.ent = (Ent<R>*)h.dent;
  c.G = (Ent<R>*)h.dG;
  c.points = h.desc.delta_points;
  c.parity = h.parity;
  c.steps = steps;
  c.macro_last = macro_last;
  c.mrt = h.desc.collision == IBM_COLL_MRT ? 1 : 0;
  c.corr = corr;
  c.tiles = tiles;
  c.rows = rows;
  c.moving = (h.nb > 0 && h.any_moving) ? 1 : 0;
  std::memcpy(dst, &c, sizeof(c));
}

}  // namespace

template <int P>
size_t BatchOps<P>::case_bytes() {
  return sizeof(BatchCase<P>);
}

template <int P>
void BatchOps<P>::record(const Ctx& h, void* dst, int steps, int macro_last, int corr, int tiles, int rows,
                         long long wait_ns) {
  case_record_t<P>(h, dst, steps, macro_last, corr, tiles, rows, wait_ns);
}

template <int P>
int BatchOps<P>::grid() {
  int n = 0, sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch<P>, kBatchThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n * sms;
}

template <int P>
unsigned long long BatchOps<P>::end_time(const void* rec) {
  return reinterpret_cast<const BatchCase<P>*>(rec)->t_end;
}

template <int P>
void BatchOps<P>::launch(void* dev_table, int cap, int grid, cudaStream_t s) {
  k_batch<P><<<grid, kBatchThreads, 0, s>>>((unsigned char*)dev_table, cap);
}

}  // namespace ibm
