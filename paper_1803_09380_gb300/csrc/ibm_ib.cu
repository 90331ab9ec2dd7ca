// ibm_ib.cu -- the per-lattice kernels of the immersed-boundary side of a
// step (the correction loop, the band build, the band collide+stream, the
// body update) and their launchers.  The device code they run is in
// ibm_ib.cuh.
#include <algorithm>

#include "ibm_ib.cuh"

namespace ibm {

// ------------------------------------------------------------------ band build
// One launch per phase: kernel boundaries are the only ordering used, so no
// thread ever waits on another.
__global__ void k_band_clear(Geom g, const int* __restrict__ ctr, const int* __restrict__ bnode,
                             int* __restrict__ node2band, int* __restrict__ segflag, int nseg_x,
                             int bcap) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < min(ctr[CTR_NBAND], bcap)) band_clear_item(g, bnode, node2band, segflag, nseg_x, b);
}

template <class R>
__global__ void k_band_claim(Geom g, int M, const double* __restrict__ X, const double* __restrict__ Y,
                             R* __restrict__ W, int* __restrict__ node_of, int* __restrict__ node2band,
                             int* __restrict__ claim, int points, int* __restrict__ ctr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  // reset the band and segment counts (k_band_clear, the previous launch,
  // has read them; k_band_alloc, the next, counts from zero)
  if (t == 0) { ctr[CTR_NBAND] = 0; ctr[CTR_NSEG] = 0; }
  if (t < M * kStencil) band_claim_item<R>(g, X, Y, W, node_of, node2band, claim, points, t);
}

__global__ void k_band_alloc(int M, const int* __restrict__ node_of, const int* __restrict__ claim,
                             int* __restrict__ node2band, int* __restrict__ bnode,
                             int* __restrict__ bcnt, int* __restrict__ ctr, int bcap) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < M * kStencil) band_alloc_item(node_of, claim, node2band, bnode, bcnt, ctr, bcap, t);
}

__global__ void k_band_segments(Geom g, const int* __restrict__ bnode, int* __restrict__ segflag,
                                int* __restrict__ seglist, int* __restrict__ ctr, int nseg_x, int bcap,
                                int segcap) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < min(ctr[CTR_NBAND], bcap)) band_segment_item(g, bnode, segflag, seglist, ctr, nseg_x, segcap, b);
}

template <class R>
__global__ void k_band_fill(int M, const int* __restrict__ node_of, const R* __restrict__ W,
                            const double* __restrict__ ds, const int* __restrict__ node2band,
                            int* __restrict__ band_of, int* __restrict__ bcnt,
                            Ent<R>* __restrict__ ent, int* __restrict__ ctr) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < M * kStencil) band_fill_item<R>(node_of, W, ds, node2band, band_of, bcnt, ent, ctr, t);
}

template <class R>
__global__ void k_band_sort(const int* __restrict__ ctr, int* __restrict__ bcnt,
                            Ent<R>* __restrict__ ent, int bcap) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < min(ctr[CTR_NBAND], bcap)) band_sort_item<R>(bcnt, ent, b);
}

template <class R>
__global__ void k_build_g(int M, const int* __restrict__ band_of, const R* __restrict__ W,
                          const int* __restrict__ bcnt, const Ent<R>* __restrict__ ent,
                          Ent<R>* __restrict__ G, int* __restrict__ gcnt, int* __restrict__ ctr) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < M) build_g_item<R>(band_of, W, bcnt, ent, G, gcnt, ctr, l);
}

// ------------------------------------------------------------------ IB loop
template <int P, int PAR, int NT>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 1) k_ib_step(IbArgs<P> a) {
  ib_step_body<P, PAR, NT>(a, blockIdx.x, gridDim.x);
}

// The correction loop as a chain of short kernels on the high-priority
// stream (IBM_OPT_IB_PHASES): the CTAs of each phase leave their SMs as soon
// as their share is done, instead of holding registers at grid barriers
// while the band-free collide+stream needs the SMs; kernel boundaries order
// the phases.  Each phase folds its CTA's residual maximum into the history
// with an integer maximum of the bit pattern (order-independent).
template <int P, int PAR>
__global__ void __launch_bounds__(kIbThreads) k_ib_gather(IbArgs<P> a) {
  typedef typename Prec<P>::R R;
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k <= a.N; k += kIbThreads) a.resid[k] = R(0);
  ib_phase_gather<P, PAR, kIbThreads>(a, blockIdx.x * kIbThreads + threadIdx.x, gridDim.x * kIbThreads,
                                      min(a.ctr[CTR_NBAND], a.bcap));
}

template <int P>
__global__ void __launch_bounds__(kIbThreads) k_ib_interp(IbArgs<P> a) {
  __shared__ typename Prec<P>::R red[kIbThreads / 32];
  ib_phase_interp<P, kIbThreads>(a, blockIdx.x * kIbThreads + threadIdx.x, gridDim.x * kIbThreads, red);
  fold_max<P, kIbThreads>(red, a.resid);
}

template <int P>
__global__ void __launch_bounds__(kIbThreads) k_ib_jacobi(IbArgs<P> a, int n) {
  __shared__ typename Prec<P>::R red[kIbThreads / 32];
  ib_phase_jacobi<P, kIbThreads>(a, n, blockIdx.x * kIbThreads + threadIdx.x, gridDim.x * kIbThreads, red);
  fold_max<P, kIbThreads>(red, a.resid + n);
}

template <int P>
__global__ void __launch_bounds__(kIbThreads) k_ib_final(IbArgs<P> a) {
  __shared__ typename Prec<P>::R red[kIbThreads / 32];
  __shared__ double sh[96];
  const int tid = blockIdx.x * kIbThreads + threadIdx.x, nth = gridDim.x * kIbThreads;
  ib_phase_final<P, kIbThreads>(a, tid, nth, nth - 1 - tid, min(a.ctr[CTR_NBAND], a.bcap), blockIdx.x,
                                gridDim.x, red, sh);
  fold_max<P, kIbThreads>(red, a.resid + a.N);
}

template <int P>
__global__ void __launch_bounds__(kIbThreads) k_ib_moments(IbArgs<P> a) {
  __shared__ double sh[96];
  if (blockIdx.x == 0 && threadIdx.x == 0) ib_check_resid<P>(a);
  ib_phase_moments<P, kIbThreads>(a, blockIdx.x * kIbThreads + threadIdx.x, gridDim.x * kIbThreads,
                                  blockIdx.x, gridDim.x, sh);
}

// The correction loop with its Jacobi iterations in one thread-block
// cluster (IBM_OPT_IB_PHASES = 2): a persistent kernel gathers the band and
// interpolates (one grid barrier); the cluster iterates with the markers'
// momentum deviations A^n in shared memory -- each CTA holds a contiguous
// slice of the markers, reads its neighbours' values from the other CTAs'
// shared memory and meets them at the hardware cluster barrier -- and
// writes every level A^n to the history; a second persistent kernel does the
// history pass, the forces and the second moments (one grid barrier).
template <int P, int PAR, int NT>
__global__ void __launch_bounds__(NT, 3) k_ib_pre(IbArgs<P> a) {
  typedef typename Prec<P>::R R;
  __shared__ R red[NT / 32];
  const int tid = blockIdx.x * NT + threadIdx.x, nth = gridDim.x * NT;
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k <= a.N; k += NT) a.resid[k] = R(0);
  ib_phase_gather<P, PAR, NT>(a, tid, nth, min(a.ctr[CTR_NBAND], a.bcap));
  grid_barrier<R>(a.bar, a.ctr, (const R*)nullptr, (R*)nullptr, a.cluster, a.bar_limit_ns, gridDim.x);
  ib_phase_interp<P, NT>(a, tid, nth, red);
  fold_max<P, NT>(red, a.resid);
}

template <int P, int NT>
__global__ void __launch_bounds__(NT, 3) k_ib_post(IbArgs<P> a) {
  typedef typename Prec<P>::R R;
  __shared__ R red[NT / 32];
  __shared__ double sh[96];
  const int tid = blockIdx.x * NT + threadIdx.x, nth = gridDim.x * NT;
  ib_phase_final<P, NT>(a, tid, nth, nth - 1 - tid, min(a.ctr[CTR_NBAND], a.bcap), blockIdx.x, gridDim.x,
                        red, sh);
  grid_barrier<R>(a.bar, a.ctr, red, a.resid + a.N, a.cluster, a.bar_limit_ns, gridDim.x);
  if (blockIdx.x == 0 && threadIdx.x == 0) ib_check_resid<P>(a);
  ib_phase_moments<P, NT>(a, tid, nth, blockIdx.x, gridDim.x, sh);
}

__device__ __forceinline__ unsigned int cluster_rank() {
  unsigned int r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Shared-memory address `addr` of this CTA mapped to cluster CTA `rank`.
__device__ __forceinline__ unsigned int dsmem_map(unsigned int addr, unsigned int rank) {
  unsigned int r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void dsmem_ld(unsigned int addr, float2& v) {
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
}
__device__ __forceinline__ void dsmem_ld(unsigned int addr, double2& v) {
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(addr) : "memory");
}

// Threads per CTA of the Jacobi cluster.
constexpr int kJcThreads = 1024;

// Shared memory of one CTA of the Jacobi cluster for a slice of `per`
// markers: A^n and A^{n+1} (pairs); when a slice is larger than the CTA
// (REG false) also b, the first kRowHead entries of each G row as weights
// and cluster addresses of the coupled markers' A slots, the row lengths
// and the interpolated densities.
template <class R>
__host__ __device__ constexpr size_t jacobi_smem_bytes(int per, bool reg) {
  return (size_t)per * (2 * 2 * sizeof(R) +
                        (reg ? 0 : 2 * sizeof(R) + (kRowHead + 1) * sizeof(R) + kRowHead * sizeof(unsigned int) +
                                       sizeof(int)));
}

// One Jacobi update of marker l (A^{n+1} = A^n + b - G A^n): the first
// kRowHead entries of its G row come as weights w[] and peer addresses ad[]
// of A^n's slots (offset `off` selects the buffer), the rest from G itself;
// the row is summed in its stored (ascending marker) order, as deviation()
// sums it.
template <class R, class V, class Args>
__device__ __forceinline__ void jacobi_row(const Args& a, int l, int k1, const R* w, const unsigned int* ad,
                                           unsigned int off, unsigned int base, int per, R& djx, R& djy,
                                           V b) {
  V v[kRowHead];
#pragma unroll
  for (int j = 0; j < kRowHead; ++j)
    if (j < k1) dsmem_ld(ad[j] + off, v[j]);
  R sx = R(0), sy = R(0);
#pragma unroll
  for (int j = 0; j < kRowHead; ++j)
    if (j < k1) {
      sx += w[j] * v[j].x;
      sy += w[j] * v[j].y;
    }
  for (int k = kRowHead; k < k1; ++k) {                      // rare long rows: the rest from G
    const Ent<R> q = a.G[(long long)l * kGCap + k];
    const int owner = q.m / per;
    V u;
    dsmem_ld(dsmem_map(base + off + (unsigned int)((q.m - owner * per) * sizeof(V)), (unsigned int)owner), u);
    sx += q.w * u.x;
    sy += q.w * u.y;
  }
  djx = b.x - sx;
  djy = b.y - sy;
}

// Jacobi iterations n = 1 .. N-1 by the `per`-marker slices of the
// cluster's CTAs (the residual of A^N is the history pass's).  The G rows
// are constant through the iterations: their first kRowHead entries are
// taken once as weights and peer addresses -- in registers when a slice
// fits the CTA (REG: one marker per thread), else staged in shared memory --
// so an iteration is kRowHead independent distributed-shared-memory loads
// per marker and one hardware cluster barrier, split so that the store of
// A^{n+1} to the history overlaps the wait.
template <int P, bool REG>
__global__ void __launch_bounds__(kJcThreads, 1) k_ib_jacobi_cluster(IbArgs<P> a, int per) {
  typedef typename Prec<P>::R R;
  typedef typename Vec2<R>::T V;
  constexpr int NTC = kJcThreads;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* As = reinterpret_cast<V*>(smem_raw);                    // [2][per]: A^n and A^{n+1} of the slice
  V* bs = As + 2 * per;                                      // [per]: b                    (!REG)
  R* wt = reinterpret_cast<R*>(bs + per);                    // [kRowHead][per]             (!REG)
  R* rs = wt + kRowHead * per;                               // [per]: interpolated density (!REG)
  unsigned int* ad = reinterpret_cast<unsigned int*>(rs + per);   // [kRowHead][per]        (!REG)
  int* nc = reinterpret_cast<int*>(ad + kRowHead * per);     // [per]: row length           (!REG)
  __shared__ R red[2 * (NTC / 32)];
  const unsigned int crank = cluster_rank();
  const int M = a.M, N = a.N;
  const int m0 = (int)crank * per, cnt = max(0, min(M, m0 + per) - m0);
  V* Ah = reinterpret_cast<V*>(a.Ah);
  const unsigned int base = (unsigned int)__cvta_generic_to_shared(As);
  // the row heads (REG: this thread's marker i = threadIdx.x)
  R w_r[REG ? kRowHead : 1];
  unsigned int ad_r[REG ? kRowHead : 1];
  V b_r, a_r;
  R rs_r = R(1);
  int k1_r = 0;
  for (int i = threadIdx.x; i < cnt; i += NTC) {
    const int l = m0 + i;
    const V a1 = Ah[M + l];                                  // A^1 = b
    As[i] = a1;
    V b;
    b.x = a.mq[4 * l + 1];
    b.y = a.mq[4 * l + 2];
    const int k1 = a.gcnt[l];
    const Ent<R>* row = a.G + (long long)l * kGCap;
#pragma unroll
    for (int j = 0; j < kRowHead; ++j) {
      unsigned int addr = base + (unsigned int)(i * sizeof(V));
      R w = R(0);
      if (j < k1) {
        const Ent<R> q = row[j];
        const int owner = q.m / per;
        addr = dsmem_map(base + (unsigned int)((q.m - owner * per) * sizeof(V)), (unsigned int)owner);
        w = q.w;
      }
      if (REG) {
        ad_r[j] = addr;
        w_r[j] = w;
      } else {
        ad[j * per + i] = addr;
        wt[j * per + i] = w;
      }
    }
    if (REG) {
      b_r = b;
      a_r = a1;
      rs_r = a.mq[4 * l];
      k1_r = k1;
    } else {
      bs[i] = b;
      rs[i] = a.mq[4 * l];
      nc[i] = k1;
    }
  }
  cluster_sync_all();
  const unsigned int half = (unsigned int)(per * sizeof(V));
  const bool mine = REG && (int)threadIdx.x < cnt;
  int cur = 0;
  for (int n = 1; n < N; ++n) {
    const V* Acur = As + cur * per;
    V* Anxt = As + (cur ^ 1) * per;
    const unsigned int off = cur ? half : 0u;
    R rmax = R(0);
    if (REG) {
      if (mine) {
        R djx, djy;
        jacobi_row<R, V>(a, m0 + threadIdx.x, k1_r, w_r, ad_r, off, base, per, djx, djy, b_r);
        a_r.x = a_r.x + djx;
        a_r.y = a_r.y + djy;
        Anxt[threadIdx.x] = a_r;
        rmax = (R)(sqrt(djx * djx + djy * djy) / rs_r);
      }
    } else {
      for (int i = threadIdx.x; i < cnt; i += NTC) {
        R w[kRowHead];
        unsigned int adl[kRowHead];
#pragma unroll
        for (int j = 0; j < kRowHead; ++j) {
          w[j] = wt[j * per + i];
          adl[j] = ad[j * per + i];
        }
        R djx, djy;
        jacobi_row<R, V>(a, m0 + i, nc[i], w, adl, off, base, per, djx, djy, bs[i]);
        V an;
        an.x = Acur[i].x + djx;
        an.y = Acur[i].y + djy;
        Anxt[i] = an;
        Ah[(long long)(n + 1) * M + m0 + i] = an;
        rmax = nanmax(rmax, (R)(sqrt(djx * djx + djy * djy) / rs[i]));
      }
    }
    R* rd = red + (n & 1) * (NTC / 32);                      // two buffers: no block barrier
    warp_max_to<R>(rmax, rd);
    cluster_arrive();                                         // A^{n+1} written, A^n read
    if (mine) Ah[(long long)(n + 1) * M + m0 + threadIdx.x] = a_r;
    cluster_wait();
    if (threadIdx.x == 0) {
      R m = rd[0];
      for (int k = 1; k < NTC / 32; ++k) m = nanmax(m, rd[k]);
      if (m > R(0) || m != m) AtomicBits<R>::max(a.resid + n, m);
    }
    cur ^= 1;
  }
}

constexpr int kJacobiSmemMax = 192 * 1024;                  // dynamic shared memory of one CTA

// Collide+stream of the 32-node row segments that hold band nodes, after
// the correction kernel has corrected them: one warp per segment.
template <int P, int PAR, bool MACRO, bool MRT>
__global__ void __launch_bounds__(256) k_band_collide(IbArgs<P> a) {
  const Geom& g = a.g;
  const StepConsts<typename Prec<P>::R>& c = a.c;
  typename Prec<P>::S* __restrict__ A = a.A;
  typename Prec<P>::R* __restrict__ mac = a.mac;
  const int nseg_x = a.nseg_x;
  const int nseg = a.ctr[CTR_NSEG];
  const int lane = threadIdx.x & (kSegW - 1);
  const int nw = (gridDim.x * blockDim.x) / kSegW;
  for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / kSegW; k < nseg; k += nw) {
    const int seg = a.seglist[k];
    const int y = seg / nseg_x, x = (seg % nseg_x) * kSegW + lane;
    if (x >= g.nx || nee_column(g, x)) continue;          // k_open_columns streams those
    // Eq. 27 at a band node first (the same thread then reads the node's
    // corrected populations; they are its own slots)
    if (!a.apply && a.N > 0) {
      const int b = a.node2band[y * g.nx + x];
      if (b >= 0) apply_band_correction<P>(g, c, A, PAR, a.bq, a.bcnt, a.ent, a.Cm, b, x, y);
    }
    if (PAR == 0) even_node<P, MACRO, MRT>(g, c, A, mac, x, y);
    else odd_node<P, MACRO, MRT>(g, c, A, mac, x, y);
  }
}


// ------------------------------------------------------------------ bodies
__global__ void k_body_update(Geom g, BodyDev* __restrict__ bodies, int nb) {
  body_update_cta(g, bodies, nb);
}

template <class R>
__global__ void k_marker_move(int M, const BodyDev* __restrict__ bodies, const int* __restrict__ mbody,
                              const double* __restrict__ dX, const double* __restrict__ dY,
                              double* __restrict__ X, double* __restrict__ Y, R* __restrict__ Ux,
                              R* __restrict__ Uy) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l < M) marker_move_item<R>(bodies, mbody, dX, dY, X, Y, Ux, Uy, l);
}

// ------------------------------------------------------------------ launchers
static unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

template <class R>
static void band_build_t(const Ctx& h, cudaStream_t s) {
  const int T = h.nm * kStencil;
  if (T == 0) return;
  k_band_clear<<<blocks_for(h.bcap, 256), 256, 0, s>>>(h.geom, h.dctr, h.dbnode, h.dnode2band,
                                                        h.dsegflag, h.nseg_x, h.bcap);
  k_band_claim<R><<<blocks_for(T, 256), 256, 0, s>>>(h.geom, h.nm, h.dX, h.dY, (R*)h.dW, h.dnode_of,
                                                      h.dnode2band, h.dclaim, h.desc.delta_points, h.dctr);
  k_band_alloc<<<blocks_for(T, 256), 256, 0, s>>>(h.nm, h.dnode_of, h.dclaim, h.dnode2band, h.dbnode,
                                                  h.dbcnt, h.dctr, h.bcap);
  k_band_fill<R><<<blocks_for(T, 256), 256, 0, s>>>(h.nm, h.dnode_of, (const R*)h.dW, h.dds, h.dnode2band,
                                                     h.dband_of, h.dbcnt, (Ent<R>*)h.dent, h.dctr);
  k_band_sort<R><<<blocks_for(h.bcap, 128), 128, 0, s>>>(h.dctr, h.dbcnt, (Ent<R>*)h.dent, h.bcap);
  k_band_segments<<<blocks_for(h.bcap, 256), 256, 0, s>>>(h.geom, h.dbnode, h.dsegflag, h.dseglist, h.dctr,
                                                          h.nseg_x, h.bcap, h.segcap);
  k_build_g<R><<<blocks_for(h.nm, 64), 64, 0, s>>>(h.nm, h.dband_of, (const R*)h.dW, h.dbcnt,
                                                    (const Ent<R>*)h.dent, (Ent<R>*)h.dG, h.dgcnt, h.dctr);
}

void launch_band_build(const Ctx& h, cudaStream_t s) {
  if (h.r_bytes == 8) band_build_t<double>(h, s);
  else band_build_t<float>(h, s);
}

template <int P, int NT>
static void launch_ib(int parity, bool cluster, dim3 grid, dim3 block, cudaStream_t s, int prio,
                      const IbArgs<P>& a) {
  if (cluster) {
    if (parity == 0) launch_prio_cluster(k_ib_step<P, 0, NT>, grid, block, s, prio, a);
    else launch_prio_cluster(k_ib_step<P, 1, NT>, grid, block, s, prio, a);
  } else {
    if (parity == 0) launch_prio(k_ib_step<P, 0, NT>, grid, block, s, prio, a);
    else launch_prio(k_ib_step<P, 1, NT>, grid, block, s, prio, a);
  }
}

template <int P, bool MRT>
static void launch_band_collide(dim3 g2, dim3 b2, cudaStream_t s, int prio, const IbArgs<P>& a,
                                int parity, bool macro) {
  if (parity == 0) {
    if (macro) launch_prio(k_band_collide<P, 0, true, MRT>, g2, b2, s, prio, a);
    else launch_prio(k_band_collide<P, 0, false, MRT>, g2, b2, s, prio, a);
  } else {
    if (macro) launch_prio(k_band_collide<P, 1, true, MRT>, g2, b2, s, prio, a);
    else launch_prio(k_band_collide<P, 1, false, MRT>, g2, b2, s, prio, a);
  }
}


// One cluster of h.ib_jc_cluster CTAs runs the Jacobi iterations
// (IBM_OPT_IB_PHASES = 2).
template <int P>
static void launch_jacobi_cluster(const Ctx& h, cudaStream_t s, const IbArgs<P>& a) {
  const int C = h.ib_jc_cluster, per = (h.nm + C - 1) / C;
  const bool reg = per <= kJcThreads;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kJcThreads);
  cfg.dynamicSmemBytes = jacobi_smem_bytes<typename Prec<P>::R>(per, reg);
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = h.ib_prio;
  attr[1].id = cudaLaunchAttributeClusterDimension;
  attr[1].val.clusterDim.x = C;
  attr[1].val.clusterDim.y = 1;
  attr[1].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 2;
  if (reg) cudaLaunchKernelEx(&cfg, k_ib_jacobi_cluster<P, true>, a, per);
  else cudaLaunchKernelEx(&cfg, k_ib_jacobi_cluster<P, false>, a, per);
}

template <int P>
static void ib_loop_t(const Ctx& h, int parity, bool macro, cudaStream_t s) {
  if (h.nm == 0) return;
  IbArgs<P> a = make_ib_args<P>(h);
  if (h.ib_phases == 2 && h.ib_jc_cluster >= 2) {
    // gather + interpolation | Jacobi in one cluster | history, forces, moments
    a.apply = 0;
    const dim3 grid(h.ib_grid), block(kIbThreads);
    auto go = [&](auto kern) {
      if (a.cluster) launch_prio_cluster(kern, grid, block, s, h.ib_prio, a);
      else launch_prio(kern, grid, block, s, h.ib_prio, a);
    };
    if (parity == 0) go(k_ib_pre<P, 0, kIbThreads>);
    else go(k_ib_pre<P, 1, kIbThreads>);
    if (h.desc.n_corr > 1) launch_jacobi_cluster<P>(h, s, a);
    go(k_ib_post<P, kIbThreads>);
  } else if (h.ib_phases == 1) {
    // one kernel per phase; grids sized by the work (every loop strides, so
    // any size is correct): markers, and band nodes as last counted
    auto ctas = [](long long items) { return dim3((unsigned)std::max(1LL, (items + kIbThreads - 1) / kIbThreads)); };
    const long long band = std::max<long long>(h.nband_host + h.nband_host / 4, 1);
    const dim3 gm = ctas(h.nm), gb = ctas(band), gf = ctas(std::max<long long>(h.nm, band)), bt(kIbThreads);
    a.apply = 0;
    if (parity == 0) launch_prio(k_ib_gather<P, 0>, gb, bt, s, h.ib_prio, a);
    else launch_prio(k_ib_gather<P, 1>, gb, bt, s, h.ib_prio, a);
    launch_prio(k_ib_interp<P>, gm, bt, s, h.ib_prio, a);
    for (int n = 1; n < h.desc.n_corr; ++n) launch_prio(k_ib_jacobi<P>, gm, bt, s, h.ib_prio, a, n);
    launch_prio(k_ib_final<P>, gf, bt, s, h.ib_prio, a);
    launch_prio(k_ib_moments<P>, gm, bt, s, h.ib_prio, a);
  } else {
  const dim3 grid(h.ib_grid), block(h.ib_threads);
  switch (h.ib_threads) {
    case 512:
      launch_ib<P, 512>(parity, a.cluster != 0, grid, block, s, h.ib_prio, a);
      break;
    case 1024:
      launch_ib<P, 1024>(parity, a.cluster != 0, grid, block, s, h.ib_prio, a);
      break;
    default:
      launch_ib<P, kIbThreads>(parity, a.cluster != 0, grid, block, s, h.ib_prio, a);
  }
  }
  // the band segments, once corrected
  if (h.band_collide) {
    const int need = (h.segcap * kSegW + 255) / 256;
    const dim3 g2(need < 8 * h.ib_grid_max ? (need > 0 ? need : 1) : 8 * h.ib_grid_max), b2(256);
    if (a.c.mrt) launch_band_collide<P, true>(g2, b2, s, h.ib_prio, a, parity, macro);
    else launch_band_collide<P, false>(g2, b2, s, h.ib_prio, a, parity, macro);
  }
}

void launch_ib_loop(const Ctx& h, int parity, bool macro, cudaStream_t s) {
  switch (h.prec) {
    case PREC_FP64: ib_loop_t<PREC_FP64>(h, parity, macro, s); break;
    case PREC_FP32: ib_loop_t<PREC_FP32>(h, parity, macro, s); break;
    case PREC_FP16_DEV: ib_loop_t<PREC_FP16_DEV>(h, parity, macro, s); break;
    default: ib_loop_t<PREC_BF16_DEV>(h, parity, macro, s); break;
  }
}

// Largest co-resident CTA count of the correction-loop kernel (1 per SM is
// used; the kernel's grid barrier needs every CTA resident).
template <int P>
static int ib_blocks_per_sm_t(int threads) {
  int n0 = 0, n1 = 0;
  switch (threads) {
    case 512:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_ib_step<P, 0, 512>, 512, 0);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_ib_step<P, 1, 512>, 512, 0);
      break;
    case 1024:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_ib_step<P, 0, 1024>, 1024, 0);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_ib_step<P, 1, 1024>, 1024, 0);
      break;
    default:
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n0, k_ib_step<P, 0, kIbThreads>, kIbThreads, 0);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n1, k_ib_step<P, 1, kIbThreads>, kIbThreads, 0);
  }
  return n0 < n1 ? n0 : n1;
}

int ib_blocks_per_sm(int prec, int threads) {
  switch (prec) {
    case PREC_FP64: return ib_blocks_per_sm_t<PREC_FP64>(threads);
    case PREC_FP32: return ib_blocks_per_sm_t<PREC_FP32>(threads);
    case PREC_FP16_DEV: return ib_blocks_per_sm_t<PREC_FP16_DEV>(threads);
    default: return ib_blocks_per_sm_t<PREC_BF16_DEV>(threads);
  }
}

template <int P, int NT>
static int max_cluster_nt() {
  int best = 0;
  for (int k = 0; k < 2; ++k) {
    void (*kern)(IbArgs<P>) = k == 0 ? k_ib_step<P, 0, NT> : k_ib_step<P, 1, NT>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  }
  for (int c = kMaxIbCluster; c >= 2; --c) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(NT);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n0 = 0, n1 = 0;
    if (cudaOccupancyMaxActiveClusters(&n0, k_ib_step<P, 0, NT>, &cfg) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&n1, k_ib_step<P, 1, NT>, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (n0 > 0 && n1 > 0) { best = c; break; }
  }
  return best;
}

template <int P>
static int max_cluster_t(int threads) {
  switch (threads) {
    case 512: return max_cluster_nt<P, 512>();
    case 1024: return max_cluster_nt<P, 1024>();
    default: return max_cluster_nt<P, kIbThreads>();
  }
}

int ib_max_cluster(int prec, int threads) {
  int dev = 0, ok = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !ok) {
    cudaGetLastError();
    return 0;
  }
  switch (prec) {
    case PREC_FP64: return max_cluster_t<PREC_FP64>(threads);
    case PREC_FP32: return max_cluster_t<PREC_FP32>(threads);
    case PREC_FP16_DEV: return max_cluster_t<PREC_FP16_DEV>(threads);
    default: return max_cluster_t<PREC_BF16_DEV>(threads);
  }
}

template <class R>
static void body_update_t(const Ctx& h, cudaStream_t s) {
  k_body_update<<<1, ((h.nb + 31) / 32) * 32, 0, s>>>(h.geom, h.dbodies, h.nb);
  k_marker_move<R><<<blocks_for(h.nm, 128), 128, 0, s>>>(h.nm, h.dbodies, h.dmbody, h.ddX, h.ddY, h.dX, h.dY,
                                                         (R*)h.dUx, (R*)h.dUy);
  band_build_t<R>(h, s);
}

void launch_body_update(const Ctx& h, cudaStream_t s) {
  if (h.nb == 0 || !h.any_moving) return;
  if (h.r_bytes == 8) body_update_t<double>(h, s);
  else body_update_t<float>(h, s);
}

void launch_marker_move(const Ctx& h, cudaStream_t s) {
  if (h.nm == 0 || !h.any_moving) return;
  if (h.r_bytes == 8)
    k_marker_move<double><<<blocks_for(h.nm, 128), 128, 0, s>>>(h.nm, h.dbodies, h.dmbody, h.ddX, h.ddY, h.dX,
                                                                 h.dY, (double*)h.dUx, (double*)h.dUy);
  else
    k_marker_move<float><<<blocks_for(h.nm, 128), 128, 0, s>>>(h.nm, h.dbodies, h.dmbody, h.ddX, h.ddY, h.dX,
                                                                h.dY, (float*)h.dUx, (float*)h.dUy);
}


// Largest cluster (at most 16 CTAs) that can run the Jacobi iterations of
// M markers with the slices in shared memory; 0 when none can.
template <int P>
static int jacobi_cluster_t(int M) {
  void (*kr)(IbArgs<P>, int) = k_ib_jacobi_cluster<P, true>;
  void (*ks)(IbArgs<P>, int) = k_ib_jacobi_cluster<P, false>;
  // the attributes allow any slice size up to kJacobiSmemMax, so that
  // lattices with different marker counts can share the kernels
  for (auto kern : {kr, ks})
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kJacobiSmemMax) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
  for (int c = kMaxIbCluster; c >= 2; --c) {
    const int per = (M + c - 1) / c;
    const bool reg = per <= kJcThreads;
    const size_t smem = jacobi_smem_bytes<typename Prec<P>::R>(per, reg);
    if (smem > (size_t)kJacobiSmemMax) break;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c);
    cfg.blockDim = dim3(kJcThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, reg ? kr : ks, &cfg) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (n > 0) return c;
  }
  return 0;
}

int jacobi_cluster_size(int prec, int M) {
  int dev = 0, ok = 0;
  if (M < 2 || cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&ok, cudaDevAttrClusterLaunch, dev) != cudaSuccess || !ok) {
    cudaGetLastError();
    return 0;
  }
  switch (prec) {
    case PREC_FP64: return jacobi_cluster_t<PREC_FP64>(M);
    case PREC_FP32: return jacobi_cluster_t<PREC_FP32>(M);
    case PREC_FP16_DEV: return jacobi_cluster_t<PREC_FP16_DEV>(M);
    default: return jacobi_cluster_t<PREC_BF16_DEV>(M);
  }
}

}  // namespace ibm
