// ibm_ib.cuh -- device code of the immersed-boundary side of a step (arXiv
// 1803.09380, section 2.3): the distribution-function correction loop, the
// band build it runs on, body force and torque, and the rigid-body update.
// Shared by the per-lattice kernels (ibm_ib.cu) and the batched serving
// kernel (ibm_batch.cu).
//
// Moment form of the correction.  The nodal equilibrium of Eq. 3 is linear in
// (rho, j = rho u, Pi = rho u u):  f_i^eq = w_i [rho + 3 e.j + 9/2 ee:Pi -
// 3/2 tr Pi].  So the interpolated equilibria of Eq. 28 are the equilibria of
// the interpolated moments (rho*, j*, Pi*), and with the boundary density
// rho_b = rho* the deviation of Eq. 28 is
//     delta f_i = w_i [3 e.dj + 9/2 ee:dPi - 3/2 tr dPi],
//     dj = rho* U - j*,   dPi = rho* U U - Pi*.
// Spreading (Eq. 26) and correction (Eq. 27) are linear too: node x gains
// momentum sum_l W_l(x) ds_l dj_l and keeps its density, while the spread dPi
// changes only the second moment of f, which no later interpolation reads
// (interpolation uses the nodal equilibrium, i.e. rho and j).  Hence the N
// iterations run entirely on small per-band-node and per-marker arrays:
//     j^n(x) = j^0(x) + sum_{l covers x} W_l(x) ds_l A^n_l,   A^n_l = sum_{k<n} dj^k_l,
// and f is touched twice per step: a gather of (rho, j^0) on the band nodes
// and one final application of the summed correction.  The same identity
// gives the force of Eq. 29: F_body = -sum_l ds_l A^N_l.
//
// Determinism: each band node sums its covering markers in ascending marker
// order (lists sorted after the parallel build), and every reduction has a
// fixed tree shape; no floating-point atomics.
#pragma once

#include "ibm_internal.h"
#include "ibm_k1.cuh"

namespace ibm {

// Eq. 15c in double precision: 1/4 (1 + cos(pi |r| / 2)), zero for |r| >= 2.
__device__ __forceinline__ double delta4(double r) {
  const double a = fabs(r);
  return a >= 2.0 ? 0.0 : 0.25 * (1.0 + cospi(0.5 * a));
}

// Eq. 15a (2 points, the linear hat) and Eq. 15b (3 points).  Both supports
// lie inside the 4 x 4 window floor(X)-1 .. floor(X)+2 that the band uses, so
// the other kernels only change the weights (some become zero).
__device__ __forceinline__ double delta_w(int points, double r) {
  const double a = fabs(r);
  if (points == 2) return a >= 1.0 ? 0.0 : 1.0 - a;
  if (points == 3) {
    if (a < 0.5) return (1.0 + sqrt(1.0 - 3.0 * a * a)) / 3.0;
    if (a < 1.5) return (5.0 - 3.0 * a - sqrt(1.0 - 3.0 * (1.0 - a) * (1.0 - a))) / 6.0;
    return 0.0;
  }
  return delta4(r);
}

__device__ __forceinline__ int wrap_axis(int c, int n, bool periodic) {
  if (periodic) { c %= n; return c < 0 ? c + n : c; }
  return (c < 0 || c >= n) ? -1 : c;
}

// Maximum that keeps a NaN (a diverged residual must not be hidden).
template <class R>
__device__ __forceinline__ R nanmax(R a, R b) { return (a > b || a != a) ? a : b; }

template <class R> struct AtomicBits;
template <> struct AtomicBits<float> {
  static __device__ void max(float* a, float v) { atomicMax((unsigned int*)a, __float_as_uint(v)); }
};
template <> struct AtomicBits<double> {
  static __device__ void max(double* a, double v) {
    atomicMax((unsigned long long*)a, (unsigned long long)__double_as_longlong(v));
  }
};
// ------------------------------------------------------------------ band build
// One item per (marker, stencil slot) or per band node.  The build runs in
// phases -- clear the previous band, claim nodes, allocate band entries, fill
// and sort the covering lists, build the coupling rows -- each phase reading
// only what earlier phases wrote: as separate kernel launches (ibm_step) or
// as block-stride loops separated by block barriers inside one CTA (the
// batched kernel).  Atomics assign band slots; every list is sorted by
// marker id afterwards, so results do not depend on their order.
__device__ __forceinline__ void band_clear_item(const Geom& g, const int* __restrict__ bnode,
                                                int* __restrict__ node2band, int* __restrict__ segflag,
                                                int nseg_x, int b) {
  const int n = bnode[b];
  node2band[n] = -1;
  segflag[(n / g.nx) * nseg_x + (n % g.nx) / kSegW] = 0;
}

template <class R>
__device__ __forceinline__ void band_claim_item(const Geom& g, const double* __restrict__ X,
                                                const double* __restrict__ Y, R* __restrict__ W,
                                                int* __restrict__ node_of, int* __restrict__ node2band,
                                                int* __restrict__ claim, int points, int t) {
  const int l = t / kStencil, s = t % kStencil;
  const double Xl = X[l], Yl = Y[l];
  const int bx = (int)floor(Xl) - 1 + (s & 3), by = (int)floor(Yl) - 1 + (s >> 2);
  const int x = wrap_axis(bx, g.nx, g.bc[0] == BC_PERIODIC);
  const int y = wrap_axis(by, g.ny, g.bc[2] == BC_PERIODIC);
  int n = -1;
  double w = 0.0;
  if (x >= 0 && y >= 0) {
    n = y * g.nx + x;
    w = delta_w(points, Xl - (double)bx) * delta_w(points, Yl - (double)by);
  }
  W[t] = (R)w;
  node_of[t] = n;
  claim[t] = (n >= 0) ? (atomicCAS(&node2band[n], -1, -2) == -1) : 0;
}

__device__ __forceinline__ void band_alloc_item(const int* __restrict__ node_of, const int* __restrict__ claim,
                                                int* __restrict__ node2band, int* __restrict__ bnode,
                                                int* __restrict__ bcnt, int* __restrict__ ctr, int bcap,
                                                int t) {
  if (!claim[t]) return;
  const int n = node_of[t];
  const int b = atomicAdd(&ctr[CTR_NBAND], 1);
  if (b < bcap) {
    bnode[b] = n;
    bcnt[b] = 0;
    node2band[n] = b;
  } else {
    atomicOr(&ctr[CTR_ERR], ERR_BAND_CAP);
  }
}

// Row segments (32 nodes) holding a band node: flagged once, listed once.
__device__ __forceinline__ void band_segment_item(const Geom& g, const int* __restrict__ bnode,
                                                  int* __restrict__ segflag, int* __restrict__ seglist,
                                                  int* __restrict__ ctr, int nseg_x, int segcap, int b) {
  const int n = bnode[b];
  const int seg = (n / g.nx) * nseg_x + (n % g.nx) / kSegW;
  if (atomicCAS(&segflag[seg], 0, 1) != 0) return;
  const int k = atomicAdd(&ctr[CTR_NSEG], 1);
  if (k < segcap) seglist[k] = seg;
  else atomicOr(&ctr[CTR_ERR], ERR_SEG_CAP);
}

template <class R>
__device__ __forceinline__ void band_fill_item(const int* __restrict__ node_of, const R* __restrict__ W,
                                               const double* __restrict__ ds, const int* __restrict__ node2band,
                                               int* __restrict__ band_of, int* __restrict__ bcnt,
                                               Ent<R>* __restrict__ ent, int* __restrict__ ctr, int t) {
  const int n = node_of[t];
  const int b = n >= 0 ? node2band[n] : -1;
  band_of[t] = b;
  if (b < 0) return;
  const int l = t / kStencil;
  const int pos = atomicAdd(&bcnt[b], 1);
  if (pos < kBandCap) {
    Ent<R> e;
    e.m = l;
    e.w = (R)((double)W[t] * ds[l]);
    ent[(long long)b * kBandCap + pos] = e;
  } else {
    atomicOr(&ctr[CTR_ERR], ERR_LIST_CAP);
  }
}

template <class R>
__device__ __forceinline__ void band_sort_item(int* __restrict__ bcnt, Ent<R>* __restrict__ ent, int b) {
  const int n = min(bcnt[b], kBandCap);
  bcnt[b] = n;
  Ent<R>* e = ent + (long long)b * kBandCap;
  for (int i = 1; i < n; ++i) {          // insertion sort by marker id
    const Ent<R> k = e[i];
    int j = i - 1;
    while (j >= 0 && e[j].m > k.m) { e[j + 1] = e[j]; --j; }
    e[j + 1] = k;
  }
}

// ------------------------------------------------------------------ G matrix
// Marker coupling of one spread followed by one interpolation:
//   G_lm = sum_x W_l(x) W_m(x) ds_m,
// summed over the shared stencil nodes x in stencil order, then stored by
// ascending m.  One item per marker.
template <class R>
__device__ void build_g_item(const int* __restrict__ band_of, const R* __restrict__ W,
                             const int* __restrict__ bcnt, const Ent<R>* __restrict__ ent,
                             Ent<R>* __restrict__ G, int* __restrict__ gcnt, int* __restrict__ ctr, int l) {
  int nm[kGCap];
  R gv[kGCap];
  int n = 0;
  bool overflow = false;
  for (int s = 0; s < kStencil; ++s) {
    const int b = band_of[l * kStencil + s];
    if (b < 0) continue;
    const R wl = W[l * kStencil + s];
    const Ent<R>* e = ent + (long long)b * kBandCap;
    const int c = bcnt[b];
    for (int k = 0; k < c; ++k) {
      const Ent<R> q = e[k];
      const R v = wl * q.w;
      int j = 0;
      while (j < n && nm[j] != q.m) ++j;
      if (j < n) gv[j] += v;
      else if (n < kGCap) { nm[n] = q.m; gv[n] = v; ++n; }
      else overflow = true;
    }
  }
  for (int i = 1; i < n; ++i) {          // ascending marker id
    const int km = nm[i];
    const R kv = gv[i];
    int j = i - 1;
    while (j >= 0 && nm[j] > km) { nm[j + 1] = nm[j]; gv[j + 1] = gv[j]; --j; }
    nm[j + 1] = km; gv[j + 1] = kv;
  }
  for (int j = 0; j < n; ++j) {
    Ent<R> q;
    q.m = nm[j];
    q.w = gv[j];
    G[(long long)l * kGCap + j] = q;
  }
  gcnt[l] = n;
  if (overflow) atomicOr(&ctr[CTR_ERR], ERR_G_CAP);
}

// ------------------------------------------------------------------ IB loop
// One persistent kernel runs the whole correction loop of a step, one CTA
// per SM, with a bounded grid barrier between phases that read other CTAs'
// results.  With J*^0_l the interpolated momentum of the uncorrected state,
// b_l = rho*_l U_l - J*^0_l and A^0 = 0, the Jacobi iteration of Eqs. 22-27
// on the momentum is
//     dj^n = b - G A^n,   A^{n+1} = A^n + dj^n,   r^n = max_l |dj^n_l| / rho*_l,
// because spreading and interpolating are linear (node momentum
// j^n(x) = j^0(x) + sum_m W_m(x) ds_m A^n_m).  The second moments do not feed
// back, so their deviations are formed once every A^n is known:
//     C_l = sum_n (rho*_l U U - Pi*^n_l),  sum_n Pi*^n_l =
//           sum_x W_l(x) / rho(x) sum_n j^n(x) j^n(x).
// Phases (| = grid barrier):
//   gather rho, j^0 of every band node | interpolate rho*, J*^0 and do
//   iteration 0 | iterations 1..N-1, each | residual r^N; per band node the
//   spread D^N and sum_n j^n j^n | per marker C_l | apply the summed
//   correction to f on every band node (Eq. 27 summed over n), FP64 partial
//   force sums | collide+stream of the band row segments, force totals.
template <int P>
struct IbArgs {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  Geom g;
  StepConsts<R> c;
  S* A;
  R* mac;
  int* ctr;
  int bcap, M, N, nb, nseg_x;
  const int* bnode;
  R* bq;                      // [bcap][8]: rho, j0x, j0y, S2xx, S2xy, S2yy, dJx, dJy
  const int* bcnt;
  const Ent<R>* ent;
  const int* band_of;
  const R* W;
  const Ent<R>* G;
  const int* gcnt;
  R* mq;                      // [M][4]: rho*, b_x, b_y, pad
  R* Ah;                      // [N+1][M][2] accumulated momentum deviations
  R* Cm;                      // [M][3]
  const R* Ux;
  const R* Uy;
  R* resid;
  const int* seglist;
  BodyDev* bodies;
  const int* mbody;
  const double* X;
  const double* Y;
  const double* ds;
  double* fpart;              // [chunks][nb][3]
  unsigned long long* bar;    // grid-barrier arrivals (monotonic)
  const int* node2band;       // [ny][nx] band index of a node, -1 outside the band
  int apply;                  // 1: apply the correction here; 0: k_band_collide applies it
  int cluster;                // 1: launched as one thread-block cluster
  R corr_tol;                 // > 0: flag WARN_NOT_CONV when r^N exceeds it
  long long bar_limit_ns;     // global-memory grid-barrier wait limit
  int drop_arrival;           // testing: the last CTA skips its first arrival of the step
};

// The correction kernel's arguments for lattice h (host side).
template <int P>
inline IbArgs<P> make_ib_args(const Ctx& h) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  IbArgs<P> a;
  a.g = h.geom;
  a.c = make_consts<R>(h);
  a.A = (S*)h.f;
  a.mac = (R*)h.macro;
  a.ctr = h.dctr;
  a.bcap = h.bcap;
  a.M = h.nm;
  a.N = h.desc.n_corr;
  a.nb = h.nb;
  a.nseg_x = h.nseg_x;
  a.bnode = h.dbnode;
  a.bq = (R*)h.dbq;
  a.bcnt = h.dbcnt;
  a.ent = (const Ent<R>*)h.dent;
  a.band_of = h.dband_of;
  a.W = (const R*)h.dW;
  a.G = (const Ent<R>*)h.dG;
  a.gcnt = h.dgcnt;
  a.mq = (R*)h.dmq;
  a.Ah = (R*)h.dAh;
  a.Cm = (R*)h.dCm;
  a.Ux = (const R*)h.dUx;
  a.Uy = (const R*)h.dUy;
  a.resid = (R*)h.dresid;
  a.seglist = h.dseglist;
  a.bodies = h.dbodies;
  a.mbody = h.dmbody;
  a.X = h.dX;
  a.Y = h.dY;
  a.ds = h.dds;
  a.fpart = h.dfpart;
  a.bar = h.dbar;
  a.node2band = h.dnode2band;
  a.apply = h.band_collide ? 0 : 1;
  a.cluster = (h.ib_cluster && h.ib_grid > 1) ? 1 : 0;
  a.corr_tol = (R)h.desc.corr_tol;
  a.bar_limit_ns = h.bar_limit_ns;
  a.drop_arrival = h.test_drop_arrival;
  return a;
}

// Eq. 27 summed over the iterations at band node b = node (x, y):
// f_i += w_i [3 e.dJ + 9/2 ee:dPi - 3/2 tr dPi], with dJ the final spread
// D^N (bq[6..7]) and dPi = sum over the covering markers of W ds C_l.
// Where the nine post-stream populations of (x, y) live: flat index (-1 for
// an inlet node or an open side, whose value is the inlet equilibrium), the
// slot, and the bounce-back side whose wall term is added on reading (or
// -1) -- the rules of post_stream below, for all nine at once, so that a
// caller can put the nine loads in flight together.
__device__ __forceinline__ void post_stream_locs(const Geom& g, int parity, int x, int y, long long (&where)[9],
                                                 int (&slot)[9], int (&wside)[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    wside[i] = -1;
    slot[i] = i;
    if (x == 0 && g.bc[0] == BC_INLET) { where[i] = -1; continue; }
    if (parity == 0) { where[i] = slot_index(g, i, x, y); continue; }
    int sx, sy;
    if (!locE(g, x, y, i, sx, sy, slot[i], wside[i])) { where[i] = -1; continue; }
    where[i] = slot_index(g, slot[i], sx, sy);
  }
}

// Read-modify-write of the nine post-stream populations, by one thread.
template <int P>
__device__ __forceinline__ void apply_band_correction(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                                      typename Prec<P>::S* __restrict__ A, int parity,
                                                      const typename Prec<P>::R* __restrict__ bq,
                                                      const int* __restrict__ bcnt,
                                                      const Ent<typename Prec<P>::R>* __restrict__ ent,
                                                      const typename Prec<P>::R* __restrict__ Cm,
                                                      int b, int x, int y) {
  typedef typename Prec<P>::R R;
  R pxx = R(0), pxy = R(0), pyy = R(0);
  const int cnt = bcnt[b];
  const Ent<R>* e = ent + (long long)b * kBandCap;
  for (int k0 = 0; k0 < cnt; k0 += 8) {
    Ent<R> q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (k0 + j < cnt) q[j] = e[k0 + j];
      else { q[j].m = 0; q[j].w = R(0); }
    }
    R c0[8], c1[8], c2[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      c0[j] = Cm[3 * q[j].m];
      c1[j] = Cm[3 * q[j].m + 1];
      c2[j] = Cm[3 * q[j].m + 2];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      pxx += q[j].w * c0[j];
      pxy += q[j].w * c1[j];
      pyy += q[j].w * c2[j];
    }
  }
  const R jx = bq[8 * b + 6], jy = bq[8 * b + 7];
  // the nine locations are distinct: all nine loads first, then the stores
  long long where[9];
  int slot[9], ws[9];
  post_stream_locs(g, parity, x, y, where, slot, ws);
  typename Prec<P>::S v[9];
#pragma unroll
  for (int i = 0; i < 9; ++i)
    if (where[i] >= 0) v[i] = A[where[i]];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if (where[i] < 0) continue;
    const R df = feq_i<R>(i, R(0), jx, jy, pxx, pxy, pyy);
    A[where[i]] = Prec<P>::st(Prec<P>::ld(v[i], slot[i]) + df, slot[i]);
  }
  (void)c;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier of the nranks CTAs that run one correction loop together (a whole
// launch, or the CTAs of the batched kernel that took one case's correction
// tasks), all resident.  A 64-bit arrival counter only grows: the k-th
// barrier of all loops of the case is complete when it reaches k * nranks.  The wait is bounded: after
// limit_ns nanoseconds the CTA records ERR_BARRIER and goes on, so a broken
// launch ends with an error status instead of hanging.  When dst is given,
// the per-warp maxima in red[] are combined first and folded into *dst.
// drop (testing only) makes this CTA skip its arrival, so that the others'
// waits run out.
template <class R>
__device__ __forceinline__ void grid_barrier(unsigned long long* bar, int* ctr, const R* red, R* dst,
                                             int cluster, long long limit_ns, int nranks, bool drop = false) {
  __syncthreads();
  if (threadIdx.x == 0 && dst) {
    R m = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = nanmax(m, red[k]);
    if (m > R(0) || m != m) AtomicBits<R>::max(dst, m);
  }
  if (nranks == 1) {                              // one CTA: a block barrier suffices
    __syncthreads();
    return;
  }
  if (cluster) {                                  // one cluster: the hardware cluster barrier
    // release orders this CTA's global writes before the arrival; acquire
    // makes the other CTAs' writes visible after the wait
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
    return;
  }
  if (threadIdx.x == 0 && !drop) {
    // The arrival is a release at GPU scope (it carries the CTA's writes,
    // ordered before it by the block barrier above); the polling loads are
    // acquires, so the other CTAs' writes are visible once the count is
    // reached (the block barrier below hands them to the CTA's threads).
    const unsigned long long g = (unsigned long long)nranks;
    unsigned long long t;
    asm volatile("atom.add.release.gpu.global.u64 %0, [%1], 1;" : "=l"(t) : "l"(bar) : "memory");
    t += 1ull;
    const unsigned long long target = ((t + g - 1) / g) * g;
    const unsigned long long t0 = global_ns();
    unsigned long long cur;
    for (;;) {
      asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(cur) : "l"(bar) : "memory");
      if (cur >= target) break;
      if ((long long)(global_ns() - t0) > limit_ns) { atomicOr(&ctr[CTR_ERR], ERR_BARRIER); break; }
    }
  }
  __syncthreads();
}

// Warp maximum of v into red[warp] (read by grid_barrier).
template <class R>
__device__ __forceinline__ void warp_max_to(R v, R* red) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
}

// Block sums of three doubles with a fixed-shape reduction (warp butterfly,
// then the warp totals in warp order).
__device__ __forceinline__ void block_sum3(double& a, double& b, double& c, double* sh) {
#pragma unroll
  for (int off = 16; off >= 1; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
    c += __shfl_xor_sync(0xffffffffu, c, off);
  }
  const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) { sh[w] = a; sh[32 + w] = b; sh[64 + w] = c; }
  __syncthreads();
  a = sh[0]; b = sh[32]; c = sh[64];
  for (int k = 1; k < nw; ++k) { a += sh[k]; b += sh[32 + k]; c += sh[64 + k]; }
  __syncthreads();
}

template <class R> struct Vec2;
template <> struct Vec2<float> { typedef float2 T; };
template <> struct Vec2<double> { typedef double2 T; };

// sum over a sparse list (marker, weight) of weight * A[marker] (two
// components), in list order; entries are gathered eight at a time so their
// loads, and then the eight A loads, are in flight together.
template <class R>
__device__ __forceinline__ void sparse_dot(const Ent<R>* __restrict__ e, int n, const R* __restrict__ A,
                                           int pad_m, R& sx, R& sy) {
  typedef typename Vec2<R>::T V;
  const V* Av = reinterpret_cast<const V*>(A);
  for (int k0 = 0; k0 < n; k0 += 8) {
    Ent<R> q[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (k0 + j < n) q[j] = e[k0 + j];
      else { q[j].m = pad_m; q[j].w = R(0); }
    }
    V v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = Av[q[j].m];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      sx += q[j].w * v[j].x;
      sy += q[j].w * v[j].y;
    }
  }
}

// Same sum for a stored row of at least kRowHead slots whose length is read
// from cntp: the first kRowHead entries are loaded together with the length,
// so a row of up to kRowHead entries (every row of a ring of markers one
// lattice unit apart: 7 to 10) costs two dependent memory trips.
constexpr int kRowHead = 10;
template <class R>
__device__ __forceinline__ void row_dot(const Ent<R>* __restrict__ e, const int* __restrict__ cntp,
                                        const R* __restrict__ A, int pad_m, R& sx, R& sy) {
  typedef typename Vec2<R>::T V;
  const V* Av = reinterpret_cast<const V*>(A);
  Ent<R> q[kRowHead];
#pragma unroll
  for (int j = 0; j < kRowHead; ++j) q[j] = e[j];
  const int n = *cntp;
#pragma unroll
  for (int j = 0; j < kRowHead; ++j)
    if (j >= n) { q[j].m = pad_m; q[j].w = R(0); }
  V v[kRowHead];
#pragma unroll
  for (int j = 0; j < kRowHead; ++j) v[j] = Av[q[j].m];
#pragma unroll
  for (int j = 0; j < kRowHead; ++j) {
    sx += q[j].w * v[j].x;
    sy += q[j].w * v[j].y;
  }
  if (n > kRowHead) sparse_dot<R>(e + kRowHead, n - kRowHead, A, pad_m, sx, sy);
}

// dj = b_l - sum_m G_lm A_m for marker l (row in ascending m).
template <class R, class Args>
__device__ __forceinline__ void deviation(const Args& a, int l, const R* __restrict__ An, R& djx, R& djy) {
  R sx = R(0), sy = R(0);
  row_dot<R>(a.G + (long long)l * kGCap, a.gcnt + l, An, l, sx, sy);
  djx = a.mq[4 * l + 1] - sx;
  djy = a.mq[4 * l + 2] - sy;
}
// The correction loop of one step in phases.  Each phase runs on nth
// threads numbered tid (band-node work from the other end, rtid = nth - 1 -
// tid), grouped in CTAs of NT threads numbered rank of nranks; a phase reads
// only what earlier phases wrote.  ib_step_body separates them with grid
// barriers inside one persistent kernel; the phase kernels of ibm_ib.cu
// separate them with kernel boundaries.  Phases that contribute to the
// residual history leave their warps' maxima in red[].
template <int P, int PAR, int NT>
__device__ __forceinline__ void ib_phase_gather(const IbArgs<P>& a, int tid, int nth, int nband) {
  typedef typename Prec<P>::R R;
  // gather rho and j^0 at every band node
  for (int b = tid; b < nband; b += nth) {
    const int n = a.bnode[b];
    const int x = n % a.g.nx, y = n / a.g.nx;
    R p[9], rho, jx, jy;
    long long w[9];
    int sl[9], ws[9];
    post_stream_locs(a.g, PAR, x, y, w, sl, ws);         // nine loads in flight together
    typename Prec<P>::S v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i)
      if (w[i] >= 0) v[i] = a.A[w[i]];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      if (w[i] < 0) { p[i] = a.c.feq_in[i]; continue; }
      p[i] = Prec<P>::ld(v[i], sl[i]);
      if (ws[i] >= 0) p[i] += a.c.wall[ws[i]][i];
    }
    moments9<R>(p, rho, jx, jy);
    a.bq[8 * b] = rho;
    a.bq[8 * b + 1] = jx;
    a.bq[8 * b + 2] = jy;
  }
}

template <int P, int NT>
__device__ __forceinline__ void ib_phase_interp(const IbArgs<P>& a, int tid, int nth,
                                                typename Prec<P>::R* red) {
  typedef typename Prec<P>::R R;
  const int M = a.M, N = a.N;
  // phase 0: interpolate rho*, J*^0 (Eq. 22b with Eq. 28 in moment form),
  // b_l = rho* U_l - J*^0 and A^1 = b (A^0 = 0); band nodes: S2 = j^0 j^0
  {
    R rmax = R(0);
    for (int l = tid; l < M; l += nth) {
      R rs = R(0), jx = R(0), jy = R(0);
      int bb[kStencil];
      R ww[kStencil];
#pragma unroll
      for (int s = 0; s < kStencil; ++s) {
        const int b = a.band_of[l * kStencil + s];
        bb[s] = b < 0 ? 0 : b;
        ww[s] = b < 0 ? R(0) : a.W[l * kStencil + s];
      }
#pragma unroll
      for (int s = 0; s < kStencil; ++s) {
        rs += ww[s] * a.bq[8 * bb[s]];
        jx += ww[s] * a.bq[8 * bb[s] + 1];
        jy += ww[s] * a.bq[8 * bb[s] + 2];
      }
      const R bx = rs * a.Ux[l] - jx, by = rs * a.Uy[l] - jy;
      a.mq[4 * l] = rs;
      a.mq[4 * l + 1] = bx;
      a.mq[4 * l + 2] = by;
      a.Ah[2 * l] = R(0);
      a.Ah[2 * l + 1] = R(0);
      if (N > 0) {
        a.Ah[2 * M + 2 * l] = bx;
        a.Ah[2 * M + 2 * l + 1] = by;
      }
      rmax = nanmax(rmax, (R)(sqrt(bx * bx + by * by) / rs));
    }
    warp_max_to<R>(rmax, red);
  }
}

// Jacobi iteration n (1 <= n < N): A^{n+1} = A^n + b - G A^n.
template <int P, int NT>
__device__ __forceinline__ void ib_phase_jacobi(const IbArgs<P>& a, int n, int tid, int nth,
                                                typename Prec<P>::R* red) {
  typedef typename Prec<P>::R R;
  const int M = a.M;
  const R* An = a.Ah + (long long)n * 2 * M;
  R* An1 = a.Ah + (long long)(n + 1) * 2 * M;
  R rmax = R(0);
  for (int l = tid; l < M; l += nth) {
    R djx, djy;
    deviation<R>(a, l, An, djx, djy);
    An1[2 * l] = An[2 * l] + djx;
    An1[2 * l + 1] = An[2 * l + 1] + djy;
    rmax = nanmax(rmax, (R)(sqrt(djx * djx + djy * djy) / a.mq[4 * l]));
  }
  warp_max_to<R>(rmax, red);
}

template <int P, int NT>
__device__ __forceinline__ void ib_phase_final(const IbArgs<P>& a, int tid, int nth, int rtid, int nband, int rank,
                                               int nranks, typename Prec<P>::R* red, double* sh) {
  typedef typename Prec<P>::R R;
  const int M = a.M, N = a.N;
  // final phase: residual r^N; per band node the final spread D^N and
  // sum_n j^n j^n over the iterations (entries gathered once, then every
  // A^n read eight at a time)
  const R* AN = a.Ah + (long long)N * 2 * M;
  {
    R rmax = R(0);
    for (int l = tid; l < M; l += nth) {
      R djx, djy;
      deviation<R>(a, l, AN, djx, djy);
      rmax = nanmax(rmax, (R)(sqrt(djx * djx + djy * djy) / a.mq[4 * l]));
    }
    warp_max_to<R>(rmax, red);
  }
  if (N > 0) {
    typedef typename Vec2<R>::T V;
    for (int b = rtid; b < nband; b += nth) {
      const R j0x = a.bq[8 * b + 1], j0y = a.bq[8 * b + 2];
      const Ent<R>* e = a.ent + (long long)b * kBandCap;
      Ent<R> q[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) q[j] = e[j];
      const int cnt = a.bcnt[b];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (j >= cnt) { q[j].m = 0; q[j].w = R(0); }
      R sxx = R(0), sxy = R(0), syy = R(0), dx = R(0), dy = R(0);
      // two levels per trip: the sixteen A loads of n and n + 1 are in
      // flight together (sums per level in list order, as one level alone)
      for (int n = 0; n <= N; n += 2) {
        const bool two = n + 1 <= N;
        const R* An = a.Ah + (long long)n * 2 * M;
        const R* Bn = two ? An + 2 * M : An;
        const V* Av = reinterpret_cast<const V*>(An);
        const V* Bv = reinterpret_cast<const V*>(Bn);
        V v[8], u[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          v[j] = Av[q[j].m];
          u[j] = Bv[q[j].m];
        }
        R px = R(0), py = R(0), ox = R(0), oy = R(0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          px += q[j].w * v[j].x;
          py += q[j].w * v[j].y;
          ox += q[j].w * u[j].x;
          oy += q[j].w * u[j].y;
        }
        if (cnt > 8) {
          sparse_dot<R>(e + 8, cnt - 8, An, 0, px, py);
          if (two) sparse_dot<R>(e + 8, cnt - 8, Bn, 0, ox, oy);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
          const int lv = n + t;
          if (lv > N) break;
          const R qx = t == 0 ? px : ox, qy = t == 0 ? py : oy;
          if (lv < N) {
            const R jx = j0x + qx, jy = j0y + qy;
            sxx += jx * jx; sxy += jx * jy; syy += jy * jy;
          } else {
            dx = qx; dy = qy;
          }
        }
      }
      a.bq[8 * b + 3] = sxx;
      a.bq[8 * b + 4] = sxy;
      a.bq[8 * b + 5] = syy;
      a.bq[8 * b + 6] = dx;
      a.bq[8 * b + 7] = dy;
    }
  }
  // Eq. 29: partial force and torque of each body over fixed chunks of
  // kForceChunk markers (CTAs take chunks in turn), F_l = -ds_l A^N_l,
  // T_l = (X_l - x_c) x F_l, FP64; the chunking does not depend on the grid,
  // so neither do the sums.
  const int nchunk = (M + kForceChunk - 1) / kForceChunk;
  if (a.nb > 0) {
    for (int k = rank; k < nchunk; k += nranks) {
      const int lo = k * kForceChunk, hi = min(M, lo + kForceChunk);
      const int b0 = a.mbody[lo], b1 = a.mbody[hi - 1];
      for (int bd = b0; bd <= b1; ++bd) {
        const BodyDev& B = a.bodies[bd];
        const int l0 = max(lo, B.m0), l1 = min(hi, B.m1);
        double fx = 0.0, fy = 0.0, tq = 0.0;
        for (int l = l0 + (int)threadIdx.x; l < l1; l += NT) {
          const double Fx = -a.ds[l] * (double)AN[2 * l], Fy = -a.ds[l] * (double)AN[2 * l + 1];
          fx += Fx;
          fy += Fy;
          tq += (a.X[l] - B.xc[0]) * Fy - (a.Y[l] - B.xc[1]) * Fx;
        }
        block_sum3(fx, fy, tq, sh);
        if (threadIdx.x == 0) {
          double* o = a.fpart + ((long long)k * a.nb + bd) * 3;
          o[0] = fx; o[1] = fy; o[2] = tq;
        }
      }
    }
  }
}

// r^N is complete: a non-finite residual means the state has diverged; one
// above corr_tol is reported as a warning (one thread).
template <int P>
__device__ __forceinline__ void ib_check_resid(const IbArgs<P>& a) {
  typedef typename Prec<P>::R R;
  const R rN = a.resid[a.N];
  if (!isfinite(rN)) atomicOr(&a.ctr[CTR_ERR], ERR_DIVERGED);
  else if (a.corr_tol > R(0) && rN > a.corr_tol) atomicOr(&a.ctr[CTR_ERR], WARN_NOT_CONV);
}

template <int P, int NT>
__device__ __forceinline__ void ib_phase_moments(const IbArgs<P>& a, int tid, int nth, int rank, int nranks,
                                                 double* sh) {
  typedef typename Prec<P>::R R;
  const int M = a.M, N = a.N;
  // second-moment deviations summed over the iterations:
  // C_l = N rho* U U - sum_x W_l(x) / rho(x) sum_n j^n j^n
  if (N > 0) {
    for (int l = tid; l < M; l += nth) {
      R pxx = R(0), pxy = R(0), pyy = R(0);
      int bb[kStencil];
      R ww[kStencil];
#pragma unroll
      for (int s = 0; s < kStencil; ++s) {
        const int b = a.band_of[l * kStencil + s];
        bb[s] = b < 0 ? 0 : b;
        ww[s] = b < 0 ? R(0) : a.W[l * kStencil + s];
      }
#pragma unroll
      for (int s = 0; s < kStencil; ++s) {
        const R w = ww[s] / a.bq[8 * bb[s]];
        pxx += w * a.bq[8 * bb[s] + 3];
        pxy += w * a.bq[8 * bb[s] + 4];
        pyy += w * a.bq[8 * bb[s] + 5];
      }
      const R rs = a.mq[4 * l], ux = a.Ux[l], uy = a.Uy[l];
      a.Cm[3 * l] = R(N) * rs * ux * ux - pxx;
      a.Cm[3 * l + 1] = R(N) * rs * ux * uy - pxy;
      a.Cm[3 * l + 2] = R(N) * rs * uy * uy - pyy;
    }
  }

  // body totals: one body per CTA, fixed-shape reduction over the chunks
  for (int bd = rank; bd < a.nb; bd += nranks) {
    BodyDev& B = a.bodies[bd];
    const int k0 = B.m0 / kForceChunk, k1 = (B.m1 - 1) / kForceChunk;
    double f0 = 0.0, f1 = 0.0, f2 = 0.0;
    for (int k = k0 + (int)threadIdx.x; k <= k1; k += NT) {
      const double* o = a.fpart + ((long long)k * a.nb + bd) * 3;
      f0 += o[0]; f1 += o[1]; f2 += o[2];
    }
    block_sum3(f0, f1, f2, sh);
    if (threadIdx.x == 0) {
      B.F_ib[0] = f0;
      B.F_ib[1] = f1;
      B.T_ib = f2;
    }
  }

}

// Folds the CTA's warp maxima in red[] into *dst (integer maximum of the
// bit pattern: order-independent).
template <int P, int NT>
__device__ __forceinline__ void fold_max(const typename Prec<P>::R* red, typename Prec<P>::R* dst) {
  typedef typename Prec<P>::R R;
  __syncthreads();
  if (threadIdx.x == 0) {
    R m = red[0];
    for (int k = 1; k < NT / 32; ++k) m = nanmax(m, red[k]);
    if (m > R(0) || m != m) AtomicBits<R>::max(dst, m);
  }
}

// Eq. 27 summed over the iterations at every band node (when the correction
// kernel applies it itself).
template <int P, int PAR>
__device__ __forceinline__ void ib_phase_apply(const IbArgs<P>& a, int tid, int nth, int nband) {
  for (int b = tid; b < nband; b += nth) {
    const int n = a.bnode[b];
    apply_band_correction<P>(a.g, a.c, a.A, PAR, a.bq, a.bcnt, a.ent, a.Cm, b, n % a.g.nx, n / a.g.nx);
  }
}

// The whole correction loop of one step, run by CTA `rank` of the nranks
// CTAs (NT threads each) that share it.
template <int P, int PAR, int NT>
__device__ void ib_step_body(const IbArgs<P>& a, int rank, int nranks) {
  typedef typename Prec<P>::R R;
  __shared__ R red[NT / 32];
  __shared__ double sh[96];
  const int tid = rank * NT + threadIdx.x;
  const int nth = nranks * NT;
  const int rtid = nth - 1 - tid;                  // band work starts from the other end
  const int nband = min(a.ctr[CTR_NBAND], a.bcap);
  const int N = a.N;
  // residual history of this step starts at zero (first read-modify-write
  // after the next barrier)
  if (rank == 0)
    for (int k = threadIdx.x; k <= N; k += NT) a.resid[k] = R(0);
  ib_phase_gather<P, PAR, NT>(a, tid, nth, nband);
  grid_barrier<R>(a.bar, a.ctr, (const R*)nullptr, (R*)nullptr, a.cluster, a.bar_limit_ns, nranks,
                  a.drop_arrival && rank == nranks - 1);
  ib_phase_interp<P, NT>(a, tid, nth, red);
  grid_barrier<R>(a.bar, a.ctr, red, a.resid, a.cluster, a.bar_limit_ns, nranks);
  for (int n = 1; n < N; ++n) {
    ib_phase_jacobi<P, NT>(a, n, tid, nth, red);
    grid_barrier<R>(a.bar, a.ctr, red, a.resid + n, a.cluster, a.bar_limit_ns, nranks);
  }
  ib_phase_final<P, NT>(a, tid, nth, rtid, nband, rank, nranks, red, sh);
  grid_barrier<R>(a.bar, a.ctr, red, a.resid + N, a.cluster, a.bar_limit_ns, nranks);
  if (rank == 0 && threadIdx.x == 0) ib_check_resid<P>(a);
  ib_phase_moments<P, NT>(a, tid, nth, rank, nranks, sh);
  if (a.apply) {
    grid_barrier<R>(a.bar, a.ctr, (const R*)nullptr, (R*)nullptr, a.cluster, a.bar_limit_ns, nranks);
    if (N > 0) ib_phase_apply<P, PAR>(a, tid, nth, nband);   // the apply reads every C_l
  }
}

// ------------------------------------------------------------------ bodies
// Eq. 39 on body i from a partner at offset d = x_i - x_j.
__device__ inline void collision_force(const BodyDev& Bi, double Rj, double dx, double dy, double* F) {
  const double eps_c = 0.01, xi = 0.05 * 2.0 * Bi.radius;
  const double gmag = sqrt(Bi.gravity[0] * Bi.gravity[0] + Bi.gravity[1] * Bi.gravity[1]);
  const double cij = Bi.mass * (1.0 - Bi.rho_f / Bi.rho_s) * gmag;
  const double d = sqrt(dx * dx + dy * dy);
  if (d > Bi.radius + Rj + xi || d <= 0.0) return;
  const double s = (d - Bi.radius - Rj - xi) / xi;
  F[0] += cij / eps_c * s * s * dx / d;
  F[1] += cij / eps_c * s * s * dy / d;
}

// Newton-Euler update of every body (one CTA, one thread per body, nb <=
// blockDim.x, FP64): Eqs. 37-38 (internal-mass terms, lagged), 39
// (collisions with other free bodies and with mirror images across closed
// walls), 40-42.  Every thread of the CTA calls it (it holds a block barrier).
__device__ inline void body_update_cta(const Geom& g, BodyDev* __restrict__ bodies, int nb) {
  const int b = threadIdx.x;
  double Fc[2] = {0.0, 0.0};
  BodyDev B;
  if (b < nb) {
    B = bodies[b];
    if (B.kind == IBM_BODY_FREE) {
      for (int o = 0; o < nb; ++o) {
        if (o == b || bodies[o].kind != IBM_BODY_FREE) continue;
        collision_force(B, bodies[o].radius, B.xc[0] - bodies[o].xc[0], B.xc[1] - bodies[o].xc[1], Fc);
      }
      for (int s = 0; s < 4; ++s) {
        if (g.bc[s] != BC_BOUNCEBACK && g.bc[s] != BC_FREESLIP) continue;
        const double w = s == 0 ? -0.5 : (s == 1 ? g.nx - 0.5 : (s == 2 ? -0.5 : g.ny - 0.5));
        if (s < 2) collision_force(B, B.radius, B.xc[0] - (2.0 * w - B.xc[0]), 0.0, Fc);
        else collision_force(B, B.radius, 0.0, B.xc[1] - (2.0 * w - B.xc[1]), Fc);
      }
    }
  }
  __syncthreads();   // every body read the old positions before any update
  if (b >= nb) return;
  if (B.kind == IBM_BODY_FREE) {
    double Ft[2];
    for (int d = 0; d < 2; ++d)
      Ft[d] = B.F_ib[d] + B.rho_f * B.volume * (B.u[d] - B.u_prev[d]) + Fc[d] +
              B.mass * (1.0 - B.rho_f / B.rho_s) * B.gravity[d];
    const double Tt = B.T_ib + B.rho_f / B.rho_s * B.inertia * (B.omega - B.omega_prev);
    const double un0 = B.u[0], un1 = B.u[1], wn = B.omega;
    B.xc[0] += un0 + 0.5 * Ft[0] / B.mass;
    B.xc[1] += un1 + 0.5 * Ft[1] / B.mass;
    B.theta += wn + 0.5 * Tt / B.inertia;
    B.u_prev[0] = un0; B.u_prev[1] = un1;
    B.u[0] = un0 + Ft[0] / B.mass;
    B.u[1] = un1 + Ft[1] / B.mass;
    B.omega_prev = wn;
    B.omega = wn + Tt / B.inertia;
  } else if (B.kind == IBM_BODY_PRESCRIBED) {
    B.xc[0] += B.u[0];
    B.xc[1] += B.u[1];
    B.theta += B.omega;
  }
  bodies[b] = B;
}

// Rigid motion of marker l of a moving body and its new velocity
// U + omega x (X - x_c).
template <class R>
__device__ __forceinline__ void marker_move_item(const BodyDev* __restrict__ bodies, const int* __restrict__ mbody,
                                                 const double* __restrict__ dX, const double* __restrict__ dY,
                                                 double* __restrict__ X, double* __restrict__ Y,
                                                 R* __restrict__ Ux, R* __restrict__ Uy, int l) {
  const BodyDev& B = bodies[mbody[l]];
  if (B.kind == IBM_BODY_FIXED) return;
  double sn, cs;
  sincos(B.theta - B.theta0, &sn, &cs);
  const double x = B.xc[0] + cs * dX[l] - sn * dY[l];
  const double y = B.xc[1] + sn * dX[l] + cs * dY[l];
  X[l] = x;
  Y[l] = y;
  Ux[l] = (R)(B.u[0] - B.omega * (y - B.xc[1]));
  Uy[l] = (R)(B.u[1] + B.omega * (x - B.xc[0]));
}


}  // namespace ibm
