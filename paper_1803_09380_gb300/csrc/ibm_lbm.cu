// ibm_lbm.cu -- the fused BGK collide + AA-pattern stream kernel (arXiv
// 1803.09380, Eq. 1 with the single-relaxation operator of section 2.1, the
// equilibrium of Eq. 3 and the moments of Eq. 7) and the kernels that move
// populations between the in-place AA layout and plain [9][ny][nx] arrays.
//
// Collide+stream is HBM-bound: every node reads its nine populations once and
// writes them once (18 s bytes per node update, s = bytes per stored
// population).  Each thread owns 4 consecutive nodes of a row (2 in FP64), so
// every access is one aligned 8- or 16-byte vector.  The even step touches
// only the thread's own nodes.  The odd step reads each population from the
// neighbour it streams from and writes it to the neighbour it streams to:
// the one-element shift is done with warp shuffles (see odd_vec).  Nodes on
// a non-periodic side, and the two columns before an outlet, take a
// per-node path through the location rules of ibm_device.cuh.
//
// In the AA pattern every slot read or written during a step belongs to
// exactly one node, so the nodes of a step can be split in any way.  A step
// with immersed markers is split into the row segments without band nodes
// (launched while the correction loop runs on another stream: the loop only
// touches band-node slots) and the band segments (launched after it).
#include <algorithm>

#include "ibm_internal.h"
#include "ibm_k1.cuh"

namespace ibm {

// One time step of collide+stream.  PAR 0: even step, 1: odd step.  A warp
// covers one span of 32 * VEC consecutive nodes of a row, each lane VEC
// nodes.
// MODE K1_ALL: every node.
// MODE K1_MAIN: every node outside the 32-node segments that hold band nodes
//   (the correction-loop kernel streams those segments after correcting
//   them).
// Even step: per lane, aligned vectors (ragged row ends node by node).  Odd
// step: spans without boundary or ragged nodes take the vector path (lanes
// whose nodes lie in band segments sit out); the others go node by node
// through the boundary-aware path.
// Threads per collide+stream block (whole warps per row span).  Two warps:
// a correction-kernel CTA resident beside collide+stream then displaces
// only the registers it needs, not whole 256-thread blocks (on the 4096^2
// FP32 Couette step 64 beat 128 and 256 by 0.3 % and 2.4 %; FP16 storage
// gained 5.6 %; alone the kernel is unchanged).
constexpr int kK1Threads = 64;

// Resident blocks asked of the register allocator: 1024 threads (64
// registers) for the node-local even step, 768 (80) for the odd step with
// its shuffles; FP64 needs 256 threads fewer.  Without it the allocator's
// own choice varied with unrelated edits, once spilling the odd step's hot
// loop.
constexpr int k1_min_blocks(int P, int PAR) {
  return ((PAR ? 3 : 4) - (P == PREC_FP64 ? 1 : 0)) * (256 / kK1Threads);
}

template <int P, int PAR, bool MACRO, int MODE, bool MRT>
__global__ void __launch_bounds__(kK1Threads, k1_min_blocks(P, PAR)) k_collide_stream(Geom g, StepConsts<typename Prec<P>::R> c,
                                                        typename Prec<P>::S* __restrict__ A,
                                                        typename Prec<P>::R* __restrict__ mac,
                                                        const int* __restrict__ segflag, int nseg_x) {
  k1_span<P, PAR, MACRO, MODE, MRT>(g, c, A, mac, segflag, nseg_x, blockIdx.y,
                                    (blockIdx.x * blockDim.x + threadIdx.x) >> 5, threadIdx.x & 31);
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

// NaN/Inf watchdog: every stored population of the lattice (padding columns
// excluded) is checked; one bit in the error word records a non-finite value.
template <int P>
__global__ void k_watchdog(Geom g, const typename Prec<P>::S* __restrict__ A, int* __restrict__ ctr) {
  typedef typename Prec<P>::R R;
  const long long n = (long long)g.ny * g.nx;
  bool bad = false;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const long long y = k / g.nx, x = k - y * g.nx;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const R v = Prec<P>::ld(A[i * g.plane + y * g.nxp + x], i);
      bad |= !isfinite(v);
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&ctr[CTR_ERR], ERR_DIVERGED);
}

// ------------------------------------------------------------------ launchers
static dim3 row_grid(const Geom& g, int bs) { return dim3((g.nx + bs - 1) / bs, g.ny); }

template <int P, int PAR, bool MACRO, bool MRT>
static void launch_k1(const Ctx& h, const StepConsts<typename Prec<P>::R>& c, int mode, cudaStream_t s) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  S* A = (S*)h.f;
  R* mac = (R*)h.macro;
  constexpr int VEC = PAR ? VecTraits<P>::VEC_ODD : VecTraits<P>::VEC;
  const int warps_per_row = (h.geom.nx + 32 * VEC - 1) / (32 * VEC);
  constexpr int wpb = kK1Threads / 32;
  const dim3 grid((warps_per_row + wpb - 1) / wpb, h.geom.ny);
  if (mode == K1_MAIN) {
    k_collide_stream<P, PAR, MACRO, K1_MAIN, MRT><<<grid, kK1Threads, 0, s>>>(
        h.geom, c, A, mac, h.dsegflag, h.nseg_x);
  } else {
    k_collide_stream<P, PAR, MACRO, K1_ALL, MRT><<<grid, kK1Threads, 0, s>>>(
        h.geom, c, A, mac, h.dsegflag, h.nseg_x);
  }
}

// Extrapolation sides (IBM_BC_INLET_NEE / IBM_BC_OUTLET_NEE): one thread per
// row and side streams the boundary node x_b and its inner neighbour x_f.
// It reads x_f's post-stream populations, rebuilds the whole state of x_b as
//   f_i(x_b) = f_i^eq(rho_b, u_b) + [f_i(x_f) - f_i^eq(rho(x_f), u(x_f))]
// (inlet: u_b = U_in, rho_b = rho(x_f); outlet: rho_b = rho0, u_b = u(x_f)),
// collides both nodes and stores their post-collision populations where
// this step kind keeps them.  In the AA pattern the pair's slots belong to
// the pair, so the other kernels of the step never touch them.
template <int P, int PAR, bool MACRO, bool MRT>
__global__ void k_open_columns(Geom g, StepConsts<typename Prec<P>::R> c, typename Prec<P>::S* __restrict__ A,
                               typename Prec<P>::R* __restrict__ mac) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * g.ny) return;
  const int side = t / g.ny;
  open_column<P, PAR, MACRO, MRT>(g, c, A, mac, side, t - side * g.ny);
}

template <int P, int PAR, bool MACRO>
static void launch_open_columns(const Ctx& h, const StepConsts<typename Prec<P>::R>& c, cudaStream_t s) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  const int n = 2 * h.geom.ny;
  if (c.mrt)
    k_open_columns<P, PAR, MACRO, true><<<(n + 127) / 128, 128, 0, s>>>(h.geom, c, (S*)h.f, (R*)h.macro);
  else
    k_open_columns<P, PAR, MACRO, false><<<(n + 127) / 128, 128, 0, s>>>(h.geom, c, (S*)h.f, (R*)h.macro);
}

template <int P>
static void launch_collide_stream_t(const Ctx& h, int parity, bool macro, int mode, cudaStream_t s) {
  typedef typename Prec<P>::R R;
  StepConsts<R> c = make_consts<R>(h);
  if (c.mrt) {
    if (parity == 0) {
      if (macro) launch_k1<P, 0, true, true>(h, c, mode, s);
      else launch_k1<P, 0, false, true>(h, c, mode, s);
    } else {
      if (macro) launch_k1<P, 1, true, true>(h, c, mode, s);
      else launch_k1<P, 1, false, true>(h, c, mode, s);
    }
  } else {
    if (parity == 0) {
      if (macro) launch_k1<P, 0, true, false>(h, c, mode, s);
      else launch_k1<P, 0, false, false>(h, c, mode, s);
    } else {
      if (macro) launch_k1<P, 1, true, false>(h, c, mode, s);
      else launch_k1<P, 1, false, false>(h, c, mode, s);
    }
  }
  if (has_nee(h.geom)) {
    if (parity == 0) {
      if (macro) launch_open_columns<P, 0, true>(h, c, s);
      else launch_open_columns<P, 0, false>(h, c, s);
    } else {
      if (macro) launch_open_columns<P, 1, true>(h, c, s);
      else launch_open_columns<P, 1, false>(h, c, s);
    }
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

void launch_watchdog(const Ctx& h, cudaStream_t s) {
  const long long n = (long long)h.geom.nx * h.geom.ny;
  const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 4LL * h.ib_grid_max);
  switch (h.prec) {
    case PREC_FP64: k_watchdog<PREC_FP64><<<blocks, 256, 0, s>>>(h.geom, (const double*)h.f, h.dctr); break;
    case PREC_FP32: k_watchdog<PREC_FP32><<<blocks, 256, 0, s>>>(h.geom, (const float*)h.f, h.dctr); break;
    case PREC_FP16_DEV:
      k_watchdog<PREC_FP16_DEV><<<blocks, 256, 0, s>>>(h.geom, (const __half*)h.f, h.dctr);
      break;
    default:
      k_watchdog<PREC_BF16_DEV><<<blocks, 256, 0, s>>>(h.geom, (const __nv_bfloat16*)h.f, h.dctr);
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
