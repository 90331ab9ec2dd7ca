// ibm_k1.cuh -- one node of the fused collide + AA-pattern stream
// (arXiv 1803.09380, Eq. 1 with either the single-relaxation operator of
// section 2.1 or the MRT operator of Eqs. 2, 5, 6; equilibrium of Eq. 3,
// moments of Eq. 7), shared by the collide+stream kernels and by the
// band collide kernel.
#pragma once

#include "ibm_internal.h"

namespace ibm {

// The nine equilibria of Eq. 3 in the moment form of feq_i, evaluated by
// opposite pairs: f_i and f_opp(i) share w_i [lead - 1.5 tr Pi + 4.5 ee:Pi]
// and differ in the sign of 3 w_i e.j, so a pair costs a few operations
// instead of two full evaluations.
template <class R>
__device__ __forceinline__ void feq_all(R lead, R jx, R jy, R pxx, R pxy, R pyy, R* fe) {
  const R tr = pxx + pyy;
  const R base = lead - R(1.5) * tr;
  const R w0 = R(4) / R(9), w1 = R(1) / R(9), w5 = R(1) / R(36);
  fe[0] = w0 * base;
  const R ax = w1 * (base + R(4.5) * pxx), bx = (R(3) * w1) * jx;
  fe[1] = ax + bx;
  fe[3] = ax - bx;
  const R ay = w1 * (base + R(4.5) * pyy), by = (R(3) * w1) * jy;
  fe[2] = ay + by;
  fe[4] = ay - by;
  const R q = R(4.5) * tr, c = R(9) * pxy;      // ee:Pi = tr +- 2 pxy on the diagonals
  const R ad = w5 * (base + q + c), bd = (R(3) * w5) * (jx + jy);
  fe[5] = ad + bd;
  fe[7] = ad - bd;
  const R ae = w5 * (base + q - c), be = (R(3) * w5) * (jy - jx);
  fe[6] = ae + be;
  fe[8] = ae - be;
}

// DEV: p holds deviations d_i = f_i - w_i (the 16-bit storage form) and so
// does ps.  Since sum_i w_i = 1 and sum_i e_i w_i = 0, the deviations' sums
// are rho - 1 and j, and f_i^eq - w_i is the equilibrium of Eq. 3 with rho
// replaced by rho - 1 in its leading term (u = j / rho keeps the full rho):
// the collision runs on the deviations directly, without adding and
// removing the weights.
template <class R, bool DEV = false>
__device__ __forceinline__ void bgk(const R* p, R* ps, R& rho, R& jx, R& jy, R omega) {
  moments9(p, rho, jx, jy);
  const R lead = rho;                      // leading term of f^eq (rho, or rho - 1)
  if (DEV) rho = R(1) + rho;
  R inv = R(1) / rho;
  R ux = jx * inv, uy = jy * inv;
  R pxx = jx * ux, pxy = jx * uy, pyy = jy * uy;
  R fe[9];
  feq_all<R>(lead, jx, jy, pxx, pxy, pyy, fe);
#pragma unroll
  for (int i = 0; i < 9; ++i) ps[i] = p[i] - omega * (p[i] - fe[i]);
}

// MRT (Eq. 2) written as BGK at the stress rate s_nu = 1/tau plus the
// difference on the energy (e), energy-square (eps) and energy-flux (q_x,
// q_y) moments, rows 1, 2, 4, 6 of Eq. 5:
//   f_i' = f_i - s_nu d_i - sum_k (s_k - s_nu) / |M_k|^2  M_ki (M_k . d),
// d = f - f^eq.  The conserved moments of d vanish, so their rates (taken
// as s_nu) do not enter.  c.mrt_k holds (s_e - s_nu)/36, (s_eps - s_nu)/36
// and (s_q - s_nu)/12.
template <class R, bool DEV = false>
__device__ __forceinline__ void mrt(const R* p, R* ps, R& rho, R& jx, R& jy,
                                    const StepConsts<R>& c) {
  moments9(p, rho, jx, jy);
  const R lead = rho;                      // as in bgk: rho, or rho - 1 for deviations
  if (DEV) rho = R(1) + rho;
  R inv = R(1) / rho;
  R ux = jx * inv, uy = jy * inv;
  R pxx = jx * ux, pxy = jx * uy, pyy = jy * uy;
  R d[9];
  feq_all<R>(lead, jx, jy, pxx, pxy, pyy, d);
#pragma unroll
  for (int i = 0; i < 9; ++i) d[i] = p[i] - d[i];
  const R s14 = (d[1] + d[3]) + (d[2] + d[4]);
  const R s58 = (d[5] + d[7]) + (d[6] + d[8]);
  const R me = c.mrt_k[0] * ((s58 + s58) - s14 - R(4) * d[0]);
  const R mp = c.mrt_k[1] * (R(4) * d[0] - (s14 + s14) + s58);
  const R a57 = d[5] - d[7];
  const R qx = c.mrt_k[2] * (R(2) * (d[3] - d[1]) + a57 + (d[8] - d[6]));
  const R qy = c.mrt_k[2] * (R(2) * (d[4] - d[2]) + a57 + (d[6] - d[8]));
  const R cax = -me - (mp + mp);          // axis directions share e, eps parts
  const R cdg = (me + me) + mp;           // diagonal directions
  const R w = c.omega;
  ps[0] = p[0] - (w * d[0] + R(4) * (mp - me));
  ps[1] = p[1] - (w * d[1] + (cax - (qx + qx)));
  ps[2] = p[2] - (w * d[2] + (cax - (qy + qy)));
  ps[3] = p[3] - (w * d[3] + (cax + (qx + qx)));
  ps[4] = p[4] - (w * d[4] + (cax + (qy + qy)));
  ps[5] = p[5] - (w * d[5] + (cdg + qx + qy));
  ps[6] = p[6] - (w * d[6] + (cdg - qx + qy));
  ps[7] = p[7] - (w * d[7] + (cdg - qx - qy));
  ps[8] = p[8] - (w * d[8] + (cdg + qx - qy));
}

// The collision of the lattice: the operator is a template parameter of
// the kernels, so the BGK kernels carry no trace of the MRT arithmetic.
template <class R, bool MRT, bool DEV = false>
__device__ __forceinline__ void collide(const R* p, R* ps, R& rho, R& jx, R& jy,
                                        const StepConsts<R>& c) {
  if constexpr (MRT)
    mrt<R, DEV>(p, ps, rho, jx, jy, c);
  else
    bgk<R, DEV>(p, ps, rho, jx, jy, c.omega);
}

// Collision of full populations p (the scalar paths).  Where the storage
// precision collides deviations (Prec<P>::kDev), p - w_i is formed first
// (exact in FP32 while f_i stays within a factor two of w_i) and the weights
// are added back once: the velocity terms are then added to rho - 1, not to
// rho ~ 1, which keeps their low bits in single precision.
template <int P, bool MRT>
__device__ __forceinline__ void collide_full(const typename Prec<P>::R* p, typename Prec<P>::R* ps,
                                             typename Prec<P>::R& rho, typename Prec<P>::R& jx,
                                             typename Prec<P>::R& jy,
                                             const StepConsts<typename Prec<P>::R>& c) {
  typedef typename Prec<P>::R R;
  if constexpr (Prec<P>::kDev) {
    R d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = p[i] - wgt<R>(i);
    collide<R, MRT, true>(d, ps, rho, jx, jy, c);
#pragma unroll
    for (int i = 0; i < 9; ++i) ps[i] += wgt<R>(i);
  } else {
    collide<R, MRT, false>(p, ps, rho, jx, jy, c);
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
template <int P, bool MACRO, bool MRT>
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
    collide_full<P, MRT>(p, ps, rho, jx, jy, c);
  }
  if (MACRO) write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + x, rho, jx, jy);
#pragma unroll
  for (int i = 0; i < 9; ++i) A[opp(i) * g.plane + base] = Prec<P>::st(ps[i], opp(i));
}

// ------------------------------------------------------------------ odd step
// Boundary path for one or two nodes (two when x = nx-2 before an outlet:
// those columns share slots, so one thread reads both before writing).
template <int P, bool MACRO, bool MRT>
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
      collide_full<P, MRT>(p, ps[q], rho, jx, jy, c);
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

template <int P, bool MACRO, bool MRT>
__device__ __forceinline__ void odd_node(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                         typename Prec<P>::S* __restrict__ A,
                                         typename Prec<P>::R* __restrict__ mac, int x, int y) {
  typedef typename Prec<P>::R R;
  if (needs_boundary_path(g, x, y)) {
    odd_boundary<P, MACRO, MRT>(g, c, A, mac, x, y);
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
  collide_full<P, MRT>(p, ps, rho, jx, jy, c);
  if (MACRO) write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + x, rho, jx, jy);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int tx = cx(i) > 0 ? xp : (cx(i) < 0 ? xm : x);
    const int ty = cy(i) > 0 ? yp : (cy(i) < 0 ? ym : y);
    A[i * g.plane + (long long)ty * g.nxp + tx] = Prec<P>::st(ps[i], i);
  }
}

// ------------------------------------------------------------------ vectors
// VEC consecutive nodes per thread, moved as one vector access per slot:
// four nodes (16 bytes in FP32, 8 bytes in 16-bit storage) or two FP64
// nodes (16 bytes).
template <int P>
struct VecTraits {
  typedef typename Prec<P>::S S;
  static constexpr int VEC = sizeof(S) == 8 ? 2 : 4;
  // nodes per lane in the odd step; half as many (fewer live registers,
  // more resident warps) measured 5 % slower on the 4096^2 FP32 step
  static constexpr int VEC_ODD = VEC;
};

template <int BYTES> struct VecWord;
template <> struct VecWord<2> { typedef unsigned short T; };
template <> struct VecWord<4> { typedef unsigned int T; };
template <> struct VecWord<8> { typedef uint2 T; };
template <> struct VecWord<16> { typedef uint4 T; };

template <class S, int VEC>
struct alignas(sizeof(S) * VEC) SVec {
  S v[VEC];
};

template <class S, int VEC>
__device__ __forceinline__ SVec<S, VEC> vload(const S* p) {
  typedef typename VecWord<sizeof(S) * VEC>::T T;
  SVec<S, VEC> r;
  *reinterpret_cast<T*>(&r) = *reinterpret_cast<const T*>(p);
  return r;
}
template <class S, int VEC>
__device__ __forceinline__ void vstore(S* p, const SVec<S, VEC>& r) {
  typedef typename VecWord<sizeof(S) * VEC>::T T;
  *reinterpret_cast<T*>(p) = *reinterpret_cast<const T*>(&r);
}

template <class S>
__device__ __forceinline__ S shfl_up1(S v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <class S>
__device__ __forceinline__ S shfl_down1(S v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Collide VEC nodes whose pre-collision populations are p[i][k]
// (arithmetic type), in place, writing macros if asked.
template <int P, bool MACRO, bool MRT, int VEC>
__device__ __forceinline__ void collide_vec(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                            typename Prec<P>::R (&p)[9][VEC],
                                            typename Prec<P>::R* __restrict__ mac, int x0, int y,
                                            bool active = true) {
  typedef typename Prec<P>::R R;
  constexpr bool DEV = Prec<P>::kDev;     // p holds deviations f_i - w_i
#pragma unroll
  for (int k = 0; k < VEC; ++k) {
    R q[9], qs[9], rho, jx, jy;
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i] = p[i][k];
    if (x0 + k == 0 && g.bc[0] == BC_INLET) {
#pragma unroll
      for (int i = 0; i < 9; ++i) qs[i] = DEV ? c.feq_in[i] - wgt<R>(i) : c.feq_in[i];
      rho = c.rho0; jx = c.rho0 * c.inlet_u[0]; jy = c.rho0 * c.inlet_u[1];
    } else {
      collide<R, MRT, DEV>(q, qs, rho, jx, jy, c);
    }
    if (MACRO && active)
      write_macro<R>(mac, (long long)g.nx * g.ny, (long long)y * g.nx + x0 + k, rho, jx, jy);
#pragma unroll
    for (int i = 0; i < 9; ++i) p[i][k] = qs[i];
  }
}

// Even step for the VEC nodes x0.. of row y (all inside the lattice):
// aligned vector loads of A[i], vector stores to A[opp(i)].  A lane with
// `skip` set (its nodes lie in a band segment, which another kernel streams)
// loads but neither computes nor stores: its loads are issued before the
// flag has arrived and their values are dropped.
template <int P, bool MACRO, bool MRT>
__device__ __forceinline__ void even_vec(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                         typename Prec<P>::S* __restrict__ A,
                                         typename Prec<P>::R* __restrict__ mac, int x0, int y,
                                         bool skip = false) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  constexpr int VEC = VecTraits<P>::VEC;
  const long long base = (long long)y * g.nxp + x0;
  R p[9][VEC];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const SVec<S, VEC> v = vload<S, VEC>(A + i * g.plane + base);
#pragma unroll
    for (int k = 0; k < VEC; ++k) p[i][k] = Prec<P>::ldv(v.v[k], i);
  }
  if (skip) return;
  collide_vec<P, MACRO, MRT, VEC>(g, c, p, mac, x0, y);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    SVec<S, VEC> v;
#pragma unroll
    for (int k = 0; k < VEC; ++k) v.v[k] = Prec<P>::stv(p[i][k], opp(i));
    vstore<S, VEC>(A + opp(i) * g.plane + base, v);
  }
}

// Odd step for one warp span of 32 * VEC consecutive nodes of row y that
// holds no boundary node (periodic wrap only across the row ends).  Each
// lane owns nodes x0 .. x0+VEC-1.  Loads and stores are aligned vectors; the
// one-element shift of the directions with an x component is done with warp
// shuffles.  A lane with `skip` set (its nodes lie in a band segment, which
// another kernel streams) loads and stores nothing.  Elements that cross to
// the neighbouring span or to a skipped lane are read or written with
// scalar accesses by the thread whose node owns the slot (the lanes at the
// ends of each run of active lanes), so no slot of another node is written.
template <int P, bool MACRO, bool MRT>
__device__ __forceinline__ void odd_vec(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                        typename Prec<P>::S* __restrict__ A,
                                        typename Prec<P>::R* __restrict__ mac, int x0, int y, int lane,
                                        bool skip) {
  typedef typename Prec<P>::S S;
  typedef typename Prec<P>::R R;
  constexpr int VEC = VecTraits<P>::VEC_ODD;
  const int xl = x0 == 0 ? g.nx - 1 : x0 - 1;              // left of the lane's nodes
  const int xr = x0 + VEC == g.nx ? 0 : x0 + VEC;           // right of the lane's nodes
  const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
  const bool skip_l = __shfl_up_sync(0xffffffffu, skip, 1);
  const bool skip_r = __shfl_down_sync(0xffffffffu, skip, 1);
  const bool lo = lane == 0 || skip_l;                      // left end of an active run
  const bool hi = lane == 31 || skip_r;                     // right end of an active run
  R p[9][VEC];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int sy = cy(i) > 0 ? ym : (cy(i) < 0 ? yp : y);
    const int sl = opp(i);
    const S* row = A + sl * g.plane + (long long)sy * g.nxp;
    SVec<S, VEC> v;
    if (!skip) {
      v = vload<S, VEC>(row + x0);
    } else {
#pragma unroll
      for (int k = 0; k < VEC; ++k) v.v[k] = S(0);
    }
    if (cx(i) == 0) {
#pragma unroll
      for (int k = 0; k < VEC; ++k) p[i][k] = Prec<P>::ldv(v.v[k], sl);
    } else if (cx(i) > 0) {                                  // f_i(x) sits at x - 1
      S left = shfl_up1<S>(v.v[VEC - 1]);
      if (lo && !skip) left = row[xl];
      p[i][0] = Prec<P>::ldv(left, sl);
#pragma unroll
      for (int k = 1; k < VEC; ++k) p[i][k] = Prec<P>::ldv(v.v[k - 1], sl);
    } else {                                                 // f_i(x) sits at x + 1
      S right = shfl_down1<S>(v.v[0]);
      if (hi && !skip) right = row[xr];
#pragma unroll
      for (int k = 0; k < VEC - 1; ++k) p[i][k] = Prec<P>::ldv(v.v[k + 1], sl);
      p[i][VEC - 1] = Prec<P>::ldv(right, sl);
    }
  }
  collide_vec<P, MACRO, MRT, VEC>(g, c, p, mac, x0, y, !skip);
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int ty = cy(i) > 0 ? yp : (cy(i) < 0 ? ym : y);
    S* row = A + i * g.plane + (long long)ty * g.nxp;
    S o[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) o[k] = Prec<P>::stv(p[i][k], i);
    if (cx(i) == 0) {
      SVec<S, VEC> v;
#pragma unroll
      for (int k = 0; k < VEC; ++k) v.v[k] = o[k];
      if (!skip) vstore<S, VEC>(row + x0, v);
    } else if (cx(i) > 0) {                                  // node x writes slot x + 1
      const S from_left = shfl_up1<S>(o[VEC - 1]);
      if (!skip) {
        if (lo) {
#pragma unroll
          for (int k = 0; k < VEC - 1; ++k) row[x0 + 1 + k] = o[k];
        } else {
          SVec<S, VEC> v;
          v.v[0] = from_left;
#pragma unroll
          for (int k = 1; k < VEC; ++k) v.v[k] = o[k - 1];
          vstore<S, VEC>(row + x0, v);
        }
        if (hi) row[xr] = o[VEC - 1];
      }
    } else {                                                 // node x writes slot x - 1
      const S from_right = shfl_down1<S>(o[0]);
      if (!skip) {
        if (hi) {
#pragma unroll
          for (int k = 1; k < VEC; ++k) row[x0 + k - 1] = o[k];
        } else {
          SVec<S, VEC> v;
#pragma unroll
          for (int k = 0; k < VEC - 1; ++k) v.v[k] = o[k + 1];
          v.v[VEC - 1] = from_right;
          vstore<S, VEC>(row + x0, v);
        }
        if (lo) row[xl] = o[0];
      }
    }
  }
}

// ------------------------------------------------------------------ spans
// One warp's share of a collide+stream step: the span of 32 * VEC
// consecutive nodes of row y that starts at node wrow * 32 * VEC (all 32
// lanes of the warp call it together).  PAR 0: even step, 1: odd step.
// MODE K1_ALL: every node.  MODE K1_MAIN: every node outside the 32-node
// segments that hold band nodes (segflag).  Even step: per lane, aligned
// vectors (ragged row ends node by node).  Odd step: spans without boundary
// or ragged nodes take the vector path (lanes whose nodes lie in band
// segments sit out); the others go node by node through the boundary-aware
// path.  Extrapolation columns are left to open_column.
template <int P, int PAR, bool MACRO, int MODE, bool MRT>
__device__ __forceinline__ void k1_span(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                        typename Prec<P>::S* __restrict__ A,
                                        typename Prec<P>::R* __restrict__ mac,
                                        const int* __restrict__ segflag, int nseg_x, int y, int wrow,
                                        int lane) {
  constexpr int VEC = PAR ? VecTraits<P>::VEC_ODD : VecTraits<P>::VEC;
  const int xw = wrow * (32 * VEC);
  if (xw >= g.nx) return;                               // whole warp
  const int x0 = xw + lane * VEC;
  const bool flagged = MODE == K1_MAIN && x0 < g.nx && segflag[y * nseg_x + x0 / kSegW] != 0;
  if (PAR == 0) {
    if (x0 >= g.nx) return;
    const bool nee = has_nee(g) && (nee_column(g, x0) || nee_column(g, min(x0 + VEC, g.nx) - 1));
    if (x0 + VEC <= g.nx && !nee) {
      even_vec<P, MACRO, MRT>(g, c, A, mac, x0, y, flagged);   // loads before the flag is needed
    } else {
      if (flagged) return;
      for (int x = x0; x < g.nx && x < x0 + VEC; ++x)
        if (!nee_column(g, x)) even_node<P, MACRO, MRT>(g, c, A, mac, x, y);
    }
    return;
  }
  const bool closed_x = g.bc[0] != BC_PERIODIC;
  const int x_special =
      closed_x ? ((g.bc[1] == BC_OUTLET || g.bc[1] == BC_OUTLET_NEE) ? g.nx - 2 : g.nx - 1) : g.nx;
  const bool edge = (g.bc[2] != BC_PERIODIC && (y == 0 || y == g.ny - 1)) ||
                    (closed_x && xw == 0) || (xw + 32 * VEC > x_special) || (xw + 32 * VEC > g.nx);
  if (edge) {
    for (int k = 0; k < VEC; ++k) {
      const int x = x0 + k;
      if (x >= g.nx) break;
      if (MODE == K1_MAIN && segflag[y * nseg_x + x / kSegW]) continue;
      if (nee_column(g, x)) continue;                          // k_open_columns
      odd_node<P, MACRO, MRT>(g, c, A, mac, x, y);
    }
    return;
  }
  if (__all_sync(0xffffffffu, flagged)) return;               // the whole span is band segments
  odd_vec<P, MACRO, MRT>(g, c, A, mac, x0, y, lane, flagged);
}

// ------------------------------------------------------------------ open sides
// Extrapolation sides (IBM_BC_INLET_NEE / IBM_BC_OUTLET_NEE): one thread
// streams row y of side `side` (0: -x inlet, 1: +x outlet), the boundary
// node x_b and its inner neighbour x_f.  It reads x_f's post-stream
// populations, rebuilds the whole state of x_b as
//   f_i(x_b) = f_i^eq(rho_b, u_b) + [f_i(x_f) - f_i^eq(rho(x_f), u(x_f))]
// (inlet: u_b = U_in, rho_b = rho(x_f); outlet: rho_b = rho0, u_b = u(x_f)),
// collides both nodes and stores their post-collision populations where
// this step kind keeps them.  In the AA pattern the pair's slots belong to
// the pair, so the other work of the step never touches them.
template <int P, int PAR, bool MACRO, bool MRT>
__device__ __forceinline__ void open_column(const Geom& g, const StepConsts<typename Prec<P>::R>& c,
                                            typename Prec<P>::S* __restrict__ A,
                                            typename Prec<P>::R* __restrict__ mac, int side, int y) {
  typedef typename Prec<P>::R R;
  if (g.bc[side] != (side == 0 ? BC_INLET_NEE : BC_OUTLET_NEE)) return;
  const int xb = side == 0 ? 0 : g.nx - 1, xf = side == 0 ? 1 : g.nx - 2;
  R pf[9], pb[9], ps[2][9];
  long long where;
#pragma unroll
  for (int i = 0; i < 9; ++i) pf[i] = post_stream<P>(g, c, A, PAR, xf, y, i, where);
  R rf, jxf, jyf;
  moments9<R>(pf, rf, jxf, jyf);
  const R inv = R(1) / rf;
  const R uxf = jxf * inv, uyf = jyf * inv;
  const R rb = side == 0 ? rf : c.rho0;
  const R uxb = side == 0 ? c.inlet_u[0] : uxf, uyb = side == 0 ? c.inlet_u[1] : uyf;
  const R jxb = rb * uxb, jyb = rb * uyb;
#pragma unroll
  for (int i = 0; i < 9; ++i)
    pb[i] = feq_i<R>(i, rb, jxb, jyb, jxb * uxb, jxb * uyb, jyb * uyb) +
            (pf[i] - feq_i<R>(i, rf, jxf, jyf, jxf * uxf, jxf * uyf, jyf * uyf));
  const long long nn = (long long)g.nx * g.ny;
  {
    R rho, jx, jy;
    collide_full<P, MRT>(pb, ps[0], rho, jx, jy, c);
    if (MACRO) write_macro<R>(mac, nn, (long long)y * g.nx + xb, rho, jx, jy);
    collide_full<P, MRT>(pf, ps[1], rho, jx, jy, c);
    if (MACRO) write_macro<R>(mac, nn, (long long)y * g.nx + xf, rho, jx, jy);
  }
  for (int q = 0; q < 2; ++q) {
    const int x = q == 0 ? xb : xf;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      if (PAR == 0) {                                      // even step: node-local
        A[slot_index(g, opp(j), x, y)] = Prec<P>::st(ps[q][j], opp(j));
      } else {
        OddTargets o = oddTargets(g, x, y, j);
        R v = ps[q][j];
        if (o.wside >= 0) v -= c.wall[o.wside][j];
        for (int k = 0; k < o.n; ++k) A[slot_index(g, o.slot[k], o.tx[k], o.ty[k])] = Prec<P>::st(v, o.slot[k]);
      }
    }
  }
}

}  // namespace ibm
