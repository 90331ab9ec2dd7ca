// ibm_k1.cuh -- one node of the fused BGK collide + AA-pattern stream
// (arXiv 1803.09380, Eq. 1 with the single-relaxation operator of section
// 2.1, equilibrium of Eq. 3, moments of Eq. 7), shared by the collide+stream
// kernels and by the correction-loop kernel, which runs the band segments.
#pragma once

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

}  // namespace ibm
