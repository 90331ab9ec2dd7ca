// ibm_lbm.cu -- the fused BGK collide + AA-pattern stream kernel (arXiv
// 1803.09380, Eq. 1 with the single-relaxation operator of section 2.1, the
// equilibrium of Eq. 3 and the moments of Eq. 7) and the kernels that move
// populations between the in-place AA layout and plain [9][ny][nx] arrays.
//
// Collide+stream is HBM-bound: every node reads its nine populations once and
// writes them once (18 s bytes per node update, s = bytes per stored
// population).  One thread per node, warps on 32 consecutive x of a row.  The
// even step touches only the thread's own node.  The odd step reads each
// population from the neighbour it streams from and writes it to the
// neighbour it streams to.  Nodes on a non-periodic side, and the two
// columns before an outlet, take a per-node path through the location rules
// of ibm_device.cuh.
//
// In the AA pattern every slot read or written during a step belongs to
// exactly one node, so the nodes of a step can be split in any way.  A step
// with immersed markers is split into the row segments without band nodes
// (launched while the correction loop runs on another stream: the loop only
// touches band-node slots) and the band segments (launched after it).
#include "ibm_internal.h"

namespace ibm {

template <class R>
__device__ __forceinline__ void bgk(const R* p, R* ps, R& rho, R& jx, R& jy, R omega) {
  moments9(p, rho, jx, jy);
  R inv = R(1) / rho;
  R ux = jx * inv, uy = jy * inv;
  R pxx = jx * ux, pxy = jx * uy, pyy = jy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    R fe = feq_i<R>(i, rho, jx, jy, pxx, pxy, pyy);
    ps[i] = p[i] - omega * (p[i] - fe);
  }
}

template <class R>
__device__ __forceinline__ void write_macro(R* mac, long long n, long long k, R rho, R jx, R jy) {
  R inv = R(1) / rho;
  mac[k] = rho;
  mac[n + k] = jx * inv;
  mac[2 * n + k] = jy * inv;
}

// ------------------------------------------------------------------ even step
// Reads A[i][x], writes f*_i to A[opp(i)][x]: purely node-local.
template <int P, bool MACRO>
__device__ __forceinline__ void even_node(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                          typename Prec<P>::S* __restrict__ A,
                                          typename Prec<P>::R* __restrict__ mac, int x, int y) {
  typedef typename Prec<P>::R R;
  const long long base = (long long)y * g.nxp + x;
  R p[9], ps[9], rho, jx, jy;
#pragma unroll
  for (int i = 0; i < 9; ++i) p[i] = Prec<P>::ld(A[i * g.plane + base], i);
  if (x == 0 && g.bc[0] == BC_INLET) {
#pragma unroll
    for (int i = 0; i < 9; ++i) ps[i] = c.feq_in[i];
    rho = c.rho0; jx = c.rho0 * c.inlet_u[0]; jy = c.rho0 * c.inlet_u[1];
  } else {
    bgk<R>(p, ps, rho, jx, jy, c.omega);
  }
  if (MACRO) write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + x, rho, jx, jy);
#pragma unroll
  for (int i = 0; i < 9; ++i) A[opp(i) * g.plane + base] = Prec<P>::st(ps[i], opp(i));
}

// ------------------------------------------------------------------ odd step
// Boundary path for one or two nodes (two when x = nx-2 before an outlet:
// those columns share slots, so one thread reads both before writing).
template <int P, bool MACRO>
__device__ void odd_boundary(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                             typename Prec<P>::S* A, typename Prec<P>::R* mac, int x, int y) {
  typedef typename Prec<P>::R R;
  if (g.bc[1] == BC_OUTLET && x == g.nx - 1) return;   // done by the x = nx-2 thread
  const int nn = (g.bc[1] == BC_OUTLET && x == g.nx - 2) ? 2 : 1;
  R ps[2][9];
  for (int q = 0; q < nn; ++q) {
    const int xq = x + q;
    R p[9], rho, jx, jy;
    long long where;
#pragma unroll
    for (int i = 0; i < 9; ++i) p[i] = post_stream<P>(g, c, A, 1, xq, y, i, where);
    if (xq == 0 && g.bc[0] == BC_INLET) {
#pragma unroll
      for (int i = 0; i < 9; ++i) ps[q][i] = c.feq_in[i];
      rho = c.rho0; jx = c.rho0 * c.inlet_u[0]; jy = c.rho0 * c.inlet_u[1];
    } else {
      bgk<R>(p, ps[q], rho, jx, jy, c.omega);
    }
    if (MACRO) write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + xq, rho, jx, jy);
  }
  for (int q = 0; q < nn; ++q) {
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      OddTargets t = oddTargets(g, x + q, y, j);
      R v = ps[q][j];
      if (t.wside >= 0) v -= c.wall[t.wside][j];
      for (int k = 0; k < t.n; ++k)
        A[slot_index(g, t.slot[k], t.tx[k], t.ty[k])] = Prec<P>::st(v, t.slot[k]);
    }
  }
}

template <int P, bool MACRO>
__device__ __forceinline__ void odd_node(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                         typename Prec<P>::S* __restrict__ A,
                                         typename Prec<P>::R* __restrict__ mac, int x, int y) {
  typedef typename Prec<P>::R R;
  if (needs_boundary_path(g, x, y)) {
    odd_boundary<P, MACRO>(g, c, A, mac, x, y);
    return;
  }
  // Interior or periodic node: neighbours by wrap-around (a no-op unless the
  // axis is periodic, since interior nodes of closed axes never wrap).
  const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
  const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
  R p[9], ps[9], rho, jx, jy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int sx = cx(i) > 0 ? xm : (cx(i) < 0 ? xp : x);
    const int sy = cy(i) > 0 ? ym : (cy(i) < 0 ? yp : y);
    p[i] = Prec<P>::ld(A[opp(i) * g.plane + (long long)sy * g.nxp + sx], opp(i));
  }
  bgk<R>(p, ps, rho, jx, jy, c.omega);
  if (MACRO) write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + x, rho, jx, jy);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int tx = cx(i) > 0 ? xp : (cx(i) < 0 ? xm : x);
    const int ty = cy(i) > 0 ? yp : (cy(i) < 0 ? ym : y);
    A[i * g.plane + (long long)ty * g.nxp + tx] = Prec<P>::st(ps[i], i);
  }
}

// One time step of collide+stream.  PAR 0: even step, 1: odd step.
// MODE K1_ALL: one thread per node of the grid (nx/256 blocks, ny rows).
// MODE K1_MAIN: the same grid, but every warp whose 32-node segment holds a
//   band node returns at once (those nodes wait for the correction loop).
// MODE K1_BAND: persistent warps walk the list of band segments.
template <int P, int PAR, bool MACRO, int MODE>
__global__ void __launch_bounds__(256) k_collide_stream(Geom g, StepConsts<typename Prec<P>::R> c,
                                                        typename Prec<P>::S* __restrict__ A,
                                                        typename Prec<P>::R* __restrict__ mac,
                                                        const int* __restrict__ segflag,
                                                        const int* __restrict__ seglist,
                                                        const int* __restrict__ ctr, int nseg_x) {
  if (MODE == K1_BAND) {
    const int nseg = ctr[CTR_NSEG];
    const int lane = threadIdx.x & (kSegW - 1);
    const int nw = (gridDim.x * blockDim.x) / kSegW;
    for (int k = (blockIdx.x * blockDim.x + threadIdx.x) / kSegW; k < nseg; k += nw) {
      const int seg = seglist[k];
      const int y = seg / nseg_x, x = (seg % nseg_x) * kSegW + lane;
      if (x >= g.nx) continue;
      if (PAR == 0) even_node<P, MACRO>(g, c, A, mac, x, y);
      else odd_node<P, MACRO>(g, c, A, mac, x, y);
    }
    return;
  }
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx) return;
  if (MODE == K1_MAIN && segflag[y * nseg_x + x / kSegW]) return;
  if (PAR == 0) even_node<P, MACRO>(g, c, A, mac, x, y);
  else odd_node<P, MACRO>(g, c, A, mac, x, y);
}

// ------------------------------------------------------------------ fields
template <int P>
__global__ void k_read_f(Geom g, StepConsts<typename Prec<P>::R> c,
                         const typename Prec<P>::S* __restrict__ A, int parity,
                         double* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx) return;
  const long long n = (long long)g.nx * g.ny, k = (long long)y * g.nx + x;
  long long where;
#pragma unroll
  for (int i = 0; i < 9; ++i) out[i * n + k] = (double)post_stream<P>(g, c, A, parity, x, y, i, where);
}

template <int P>
__global__ void k_write_f(Geom g, typename Prec<P>::S* __restrict__ A, const double* __restrict__ in) {
  typedef typename Prec<P>::R R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx) return;
  const long long n = (long long)g.nx * g.ny, k = (long long)y * g.nx + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) A[slot_index(g, i, x, y)] = Prec<P>::st((R)in[i * n + k], i);
}

// f := f^eq(rho, u) in the natural (parity 0) layout; also records the
// moments as the current macroscopic fields.
template <int P>
__global__ void k_init_eq(Geom g, typename Prec<P>::S* __restrict__ A, const double* __restrict__ in,
                          typename Prec<P>::R* __restrict__ mac) {
  typedef typename Prec<P>::R R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx) return;
  const long long n = (long long)g.nx * g.ny, k = (long long)y * g.nx + x;
  const R rho = (R)in[k], ux = (R)in[n + k], uy = (R)in[2 * n + k];
  const R jx = rho * ux, jy = rho * uy;
  const R pxx = jx * ux, pxy = jx * uy, pyy = jy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    A[slot_index(g, i, x, y)] = Prec<P>::st(feq_i<R>(i, rho, jx, jy, pxx, pxy, pyy), i);
  mac[k] = rho; mac[n + k] = ux; mac[2 * n + k] = uy;
}

// Moments of the current (uncorrected) post-stream state into the
// macroscopic fields.
template <int P>
__global__ void k_macros(Geom g, StepConsts<typename Prec<P>::R> c,
                         const typename Prec<P>::S* __restrict__ A, int parity,
                         typename Prec<P>::R* __restrict__ mac) {
  typedef typename Prec<P>::R R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx) return;
  R p[9], rho, jx, jy;
  long long where;
#pragma unroll
  for (int i = 0; i < 9; ++i) p[i] = post_stream<P>(g, c, A, parity, x, y, i, where);
  moments9<R>(p, rho, jx, jy);
  write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + x, rho, jx, jy);
}

// Rest equilibrium f_i = w_i rho0 (Eq. 3 with u = 0), natural layout.
template <int P>
__global__ void k_fill_rest(Geom g, StepConsts<typename Prec<P>::R> c, typename Prec<P>::S* __restrict__ A,
                            typename Prec<P>::R* __restrict__ mac) {
  typedef typename Prec<P>::R R;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= g.nx) return;
  const long long n = (long long)g.nx * g.ny, k = (long long)y * g.nx + x;
#pragma unroll
  for (int i = 0; i < 9; ++i) A[slot_index(g, i, x, y)] = Prec<P>::st(wgt<R>(i) * c.rho0, i);
  mac[k] = c.rho0; mac[n + k] = R(0); mac[2 * n + k] = R(0);
}

template <class R>
__global__ void k_macro_to_double(long long n, const R* __restrict__ mac, double* __restrict__ out) {
  long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = (double)mac[k];
}

// ------------------------------------------------------------------ launchers
static dim3 row_grid(const Geom& g, int bs) { return dim3((g.nx + bs - 1) / bs, g.ny); }

template <int P, int PAR, bool MACRO>
static void launch_k1(const Ctx& h, const StepConsts<typename Prec<P>::R>& c, int mode, cudaStream_t s) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  S* A = (S*)h.f;
  R* mac = (R*)h.macro;
  if (mode == K1_BAND) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int need = (h.segcap * kSegW + 255) / 256;
    const int blocks = need < 4 * sms ? (need > 0 ? need : 1) : 4 * sms;
    k_collide_stream<P, PAR, MACRO, K1_BAND><<<blocks, 256, 0, s>>>(h.geom, c, A, mac, h.dsegflag,
                                                                    h.dseglist, h.dctr, h.nseg_x);
  } else if (mode == K1_MAIN) {
    k_collide_stream<P, PAR, MACRO, K1_MAIN><<<row_grid(h.geom, 256), 256, 0, s>>>(
        h.geom, c, A, mac, h.dsegflag, h.dseglist, h.dctr, h.nseg_x);
  } else {
    k_collide_stream<P, PAR, MACRO, K1_ALL><<<row_grid(h.geom, 256), 256, 0, s>>>(
        h.geom, c, A, mac, h.dsegflag, h.dseglist, h.dctr, h.nseg_x);
  }
}

template <int P>
static void launch_collide_stream_t(const Ctx& h, int parity, bool macro, int mode, cudaStream_t s) {
  typedef typename Prec<P>::R R;
  StepConsts<R> c = make_consts<R>(h);
  if (parity == 0) {
    if (macro) launch_k1<P, 0, true>(h, c, mode, s);
    else launch_k1<P, 0, false>(h, c, mode, s);
  } else {
    if (macro) launch_k1<P, 1, true>(h, c, mode, s);
    else launch_k1<P, 1, false>(h, c, mode, s);
  }
}

void launch_collide_stream(const Ctx& h, int parity, bool macro, int mode, cudaStream_t s) {
  switch (h.prec) {
    case PREC_FP64: launch_collide_stream_t<PREC_FP64>(h, parity, macro, mode, s); break;
    case PREC_FP32: launch_collide_stream_t<PREC_FP32>(h, parity, macro, mode, s); break;
    case PREC_FP16_DEV: launch_collide_stream_t<PREC_FP16_DEV>(h, parity, macro, mode, s); break;
    default: launch_collide_stream_t<PREC_BF16_DEV>(h, parity, macro, mode, s); break;
  }
}

template <int P>
static void launch_fields_t(const Ctx& h, int op, const double* dev_in, double* dev_out,
                            cudaStream_t s) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  StepConsts<R> c = make_consts<R>(h);
  dim3 grid = row_grid(h.geom, 128);
  S* A = (S*)h.f;
  R* mac = (R*)h.macro;
  const long long n = (long long)h.geom.nx * h.geom.ny;
  switch (op) {
    case FIELD_OP_READ_F: k_read_f<P><<<grid, 128, 0, s>>>(h.geom, c, A, h.parity, dev_out); break;
    case FIELD_OP_WRITE_F: k_write_f<P><<<grid, 128, 0, s>>>(h.geom, A, dev_in); break;
    case FIELD_OP_INIT_EQ: k_init_eq<P><<<grid, 128, 0, s>>>(h.geom, A, dev_in, mac); break;
    case FIELD_OP_MACROS: k_macros<P><<<grid, 128, 0, s>>>(h.geom, c, A, h.parity, mac); break;
    case FIELD_OP_REST: k_fill_rest<P><<<grid, 128, 0, s>>>(h.geom, c, A, mac); break;
    case FIELD_OP_MACRO_OUT:
      k_macro_to_double<R><<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(3 * n, mac, dev_out);
      break;
  }
}

void launch_fields(const Ctx& h, int op, const double* dev_in, double* dev_out, cudaStream_t s) {
  switch (h.prec) {
    case PREC_FP64: launch_fields_t<PREC_FP64>(h, op, dev_in, dev_out, s); break;
    case PREC_FP32: launch_fields_t<PREC_FP32>(h, op, dev_in, dev_out, s); break;
    case PREC_FP16_DEV: launch_fields_t<PREC_FP16_DEV>(h, op, dev_in, dev_out, s); break;
    default: launch_fields_t<PREC_BF16_DEV>(h, op, dev_in, dev_out, s); break;
  }
}

}  // namespace ibm
