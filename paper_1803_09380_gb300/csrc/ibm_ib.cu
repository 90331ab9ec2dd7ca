// ibm_ib.cu -- the per-lattice kernels of the immersed-boundary side of a
// step (the correction loop, the band build, the band collide+stream, the
// body update) and their launchers.  The device code they run is in
// ibm_ib.cuh.
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

template <int P>
static void ib_loop_t(const Ctx& h, int parity, bool macro, cudaStream_t s) {
  if (h.nm == 0) return;
  IbArgs<P> a = make_ib_args<P>(h);
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

}  // namespace ibm
