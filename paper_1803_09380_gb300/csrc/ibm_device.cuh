// ibm_device.cuh -- device-side building blocks of the IB-LBM library:
// the D2Q9 lattice (arXiv 1803.09380, Eq. 4, ordering from the rows of
// Eq. 5), the storage precisions, the equilibrium (Eq. 3) and moments
// (Eq. 7), and the AA-pattern location rules that say where a post-stream
// population lives in the single in-place population buffer.
//
// AA pattern.  One buffer A[k][y][x] (k = slot, x fastest, rows padded to
// nxp).  Two kinds of step alternate:
//   even step: node x reads f_i(x) = A[i][x], collides, writes the
//              post-collision f*_i(x) to A[opp(i)][x] (its own node);
//   odd step:  node x reads f_i(x) from the slot where the even step left
//              the population that streams into x (locE below), collides,
//              and writes f*_i(x) where the next even step reads it: slot
//              i of the node it streams to (oddTargets below).
// After an odd step (parity 0) the post-stream f_i(x) sits in A[i][x].
// After an even step (parity 1) it sits at locE(x, i): normally
// A[opp(i)][x - e_i].  Every boundary rule is expressed in those two maps,
// so the even step never needs a boundary branch.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace ibm {

enum { PREC_FP64 = 0, PREC_FP32 = 1, PREC_FP16_DEV = 2, PREC_BF16_DEV = 3 };
enum { BC_PERIODIC = 0, BC_BOUNCEBACK = 1, BC_FREESLIP = 2, BC_INLET = 3, BC_OUTLET = 4,
       BC_INLET_NEE = 5, BC_OUTLET_NEE = 6 };

// Stencil slots per marker (4 x 4 support of the delta function, Eq. 15c)
// and capacity of the per-band-node list of covering markers.
constexpr int kStencil = 16;
constexpr int kBandCap = 32;

// ----------------------------------------------------------------- D2Q9
__host__ __device__ constexpr int cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) & 3) + 1 : ((i - 3) & 3) + 5);
}
// Direction index of lattice vector (a, b), a, b in {-1, 0, 1}.
__host__ __device__ constexpr int dir_of(int a, int b) {
  return (a == 0 && b == 0) ? 0
       : (b == 0) ? (a > 0 ? 1 : 3)
       : (a == 0) ? (b > 0 ? 2 : 4)
       : (a > 0) ? (b > 0 ? 5 : 8)
       : (b > 0 ? 6 : 7);
}
template <class R>
__host__ __device__ constexpr R wgt(int i) {
  return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}

// ----------------------------------------------------------------- storage
// S is the stored type of one population, R the arithmetic type.  The
// 16-bit forms keep f_i - w_i (the deviation from the rest weight).
template <int P> struct Prec;
// ld/st convert between storage and the full population f_i; ldv/stv are
// the vector kernels' forms, which hand the collision the deviation
// f_i - w_i where kDev is set (16-bit storage keeps the deviation itself;
// FP32 stores f_i and converts, which keeps the velocity terms' low bits)
// and f_i otherwise.
template <> struct Prec<PREC_FP64> {
  typedef double S; typedef double R;
  static constexpr bool kDev = false;
  static __device__ __forceinline__ R ld(S v, int) { return v; }
  static __device__ __forceinline__ S st(R v, int) { return v; }
  static __device__ __forceinline__ R ldv(S v, int) { return v; }
  static __device__ __forceinline__ S stv(R v, int) { return v; }
};
template <> struct Prec<PREC_FP32> {
  typedef float S; typedef float R;
  static constexpr bool kDev = true;      // collide deviations, store full f
  static __device__ __forceinline__ R ld(S v, int) { return v; }
  static __device__ __forceinline__ S st(R v, int) { return v; }
  static __device__ __forceinline__ R ldv(S v, int i) { return v - wgt<float>(i); }
  static __device__ __forceinline__ S stv(R v, int i) { return v + wgt<float>(i); }
};
template <> struct Prec<PREC_FP16_DEV> {
  typedef __half S; typedef float R;
  static constexpr bool kDev = true;
  static __device__ __forceinline__ R ld(S v, int i) { return wgt<float>(i) + __half2float(v); }
  static __device__ __forceinline__ S st(R v, int i) { return __float2half_rn(v - wgt<float>(i)); }
  static __device__ __forceinline__ R ldv(S v, int) { return __half2float(v); }
  static __device__ __forceinline__ S stv(R v, int) { return __float2half_rn(v); }
};
template <> struct Prec<PREC_BF16_DEV> {
  typedef __nv_bfloat16 S; typedef float R;
  static constexpr bool kDev = true;
  static __device__ __forceinline__ R ld(S v, int i) { return wgt<float>(i) + __bfloat162float(v); }
  static __device__ __forceinline__ S st(R v, int i) { return __float2bfloat16_rn(v - wgt<float>(i)); }
  static __device__ __forceinline__ R ldv(S v, int) { return __bfloat162float(v); }
  static __device__ __forceinline__ S stv(R v, int) { return __float2bfloat16_rn(v); }
};

// ----------------------------------------------------------------- geometry
struct Geom {
  int nx, ny, nxp;          // size and padded row stride (elements)
  long long plane;          // ny * nxp: distance between slots
  int bc[4];                // -x, +x, -y, +y
};

template <class R>
struct StepConsts {
  R omega;                  // 1 / tau
  int mrt;                  // 0: BGK, 1: MRT (Eqs. 2, 5, 6)
  R mrt_k[3];               // (s_e - 1/tau)/36, (s_eps - 1/tau)/36, (s_q - 1/tau)/12
  R wall[4][9];             // 6 w_i rho0 (e_i . U_wall[side])
  R feq_in[9];              // inlet equilibrium f^eq(rho0, U_in)
  R rho0;
  R inlet_u[2];
};

__device__ __forceinline__ bool is_open(int b) {
  return b == BC_INLET || b == BC_OUTLET || b == BC_INLET_NEE || b == BC_OUTLET_NEE;
}

// Columns of an extrapolation side and their inner neighbours: streamed by
// k_open_columns, one thread per row and side, never by the other kernels.
__host__ __device__ __forceinline__ bool nee_column(const Geom& g, int x) {
  return (g.bc[0] == BC_INLET_NEE && x <= 1) || (g.bc[1] == BC_OUTLET_NEE && x >= g.nx - 2);
}
__host__ __device__ __forceinline__ bool has_nee(const Geom& g) {
  return g.bc[0] == BC_INLET_NEE || g.bc[1] == BC_OUTLET_NEE;
}

__device__ __forceinline__ long long slot_index(const Geom& g, int k, int x, int y) {
  return (long long)k * g.plane + (long long)y * g.nxp + x;
}

// Where the post-stream population f_i(x, y) lives after an EVEN step.
// Returns false for an inlet node (its state is the inlet equilibrium).
// Otherwise (sx, sy, slot) is the stored location and wside >= 0 names a
// bounce-back side whose wall term must be added when reading.
__device__ __forceinline__ bool locE(const Geom& g, int x, int y, int i, int& sx, int& sy,
                                     int& slot, int& wside) {
#pragma unroll 1
  for (int depth = 0; depth < 2; ++depth) {
    if (x == 0 && g.bc[0] == BC_INLET) return false;
    int tx = x - cx(i), ty = y - cy(i);
    int crx = -1, cry = -1;
    if (tx < 0) { if (g.bc[0] == BC_PERIODIC) tx += g.nx; else crx = 0; }
    else if (tx >= g.nx) { if (g.bc[1] == BC_PERIODIC) tx -= g.nx; else crx = 1; }
    if (ty < 0) { if (g.bc[2] == BC_PERIODIC) ty += g.ny; else cry = 2; }
    else if (ty >= g.ny) { if (g.bc[3] == BC_PERIODIC) ty -= g.ny; else cry = 3; }
    wside = -1;
    if (crx < 0 && cry < 0) { sx = tx; sy = ty; slot = opp(i); return true; }
    bool open = (crx >= 0 && is_open(g.bc[crx])) || (cry >= 0 && is_open(g.bc[cry]));
    if (open) {
      if (crx == 1 && g.bc[1] == BC_OUTLET) { x = g.nx - 2; continue; }  // zero gradient
      return false;
    }
    if (crx < 0 && g.bc[cry] == BC_FREESLIP) {       // specular off a y wall
      sx = tx; sy = y; slot = opp(dir_of(cx(i), -cy(i))); return true;
    }
    if (cry < 0 && g.bc[crx] == BC_FREESLIP) {       // specular off an x wall
      sx = x; sy = ty; slot = opp(dir_of(-cx(i), cy(i))); return true;
    }
    sx = x; sy = y; slot = i; wside = cry >= 0 ? cry : crx;   // bounce-back
    return true;
  }
  return false;
}

// Where the ODD step stores the post-collision f*_j(x, y): up to two
// (node, slot) targets (the second is the zero-gradient outlet copy), and
// the bounce-back side whose wall term is subtracted (or -1).
struct OddTargets {
  int n;
  int tx[2], ty[2], slot[2];
  int wside;
};
__device__ __forceinline__ OddTargets oddTargets(const Geom& g, int x, int y, int j) {
  OddTargets o;
  o.n = 0; o.wside = -1;
  int tx = x + cx(j), ty = y + cy(j);
  int crx = -1, cry = -1;
  if (tx < 0) { if (g.bc[0] == BC_PERIODIC) tx += g.nx; else crx = 0; }
  else if (tx >= g.nx) { if (g.bc[1] == BC_PERIODIC) tx -= g.nx; else crx = 1; }
  if (ty < 0) { if (g.bc[2] == BC_PERIODIC) ty += g.ny; else cry = 2; }
  else if (ty >= g.ny) { if (g.bc[3] == BC_PERIODIC) ty -= g.ny; else cry = 3; }
  int nx_ = 0, ny_ = 0, k = 0;
  if (crx < 0 && cry < 0) { nx_ = tx; ny_ = ty; k = j; }
  else if ((crx >= 0 && is_open(g.bc[crx])) || (cry >= 0 && is_open(g.bc[cry]))) { return o; }
  else if (crx < 0 && g.bc[cry] == BC_FREESLIP) { nx_ = tx; ny_ = y; k = dir_of(cx(j), -cy(j)); }
  else if (cry < 0 && g.bc[crx] == BC_FREESLIP) { nx_ = x; ny_ = ty; k = dir_of(-cx(j), cy(j)); }
  else { nx_ = x; ny_ = y; k = opp(j); o.wside = cry >= 0 ? cry : crx; }
  o.tx[0] = nx_; o.ty[0] = ny_; o.slot[0] = k; o.n = 1;
  if (g.bc[1] == BC_OUTLET && nx_ == g.nx - 2 && cx(k) < 0) {
    o.tx[1] = g.nx - 1; o.ty[1] = ny_; o.slot[1] = k; o.n = 2;
  }
  return o;
}

// Node needs the generic (boundary-aware) path of the odd step: it sits on
// a non-periodic side, or in the last two columns before an outlet (those
// two share slots and must be handled by one thread, reads before writes).
__device__ __forceinline__ bool needs_boundary_path(const Geom& g, int x, int y) {
  return (g.bc[0] != BC_PERIODIC && x == 0) ||
         (g.bc[1] != BC_PERIODIC && x >= g.nx - ((g.bc[1] == BC_OUTLET || g.bc[1] == BC_OUTLET_NEE) ? 2 : 1)) ||
         (g.bc[2] != BC_PERIODIC && y == 0) ||
         (g.bc[3] != BC_PERIODIC && y == g.ny - 1);
}

// ----------------------------------------------------------------- physics
// Eq. 7 in a fixed order, mirror pairs first.
template <class R>
__device__ __forceinline__ void moments9(const R* p, R& rho, R& jx, R& jy) {
  rho = ((p[0] + (p[1] + p[3])) + (p[2] + p[4])) + ((p[5] + p[7]) + (p[6] + p[8]));
  jx = ((p[1] - p[3]) + (p[5] - p[7])) + (p[8] - p[6]);
  jy = ((p[2] - p[4]) + (p[5] - p[7])) + (p[6] - p[8]);
}

// Eq. 3 with c_s^2 = 1/3, written through the moments (rho, j = rho u,
// Pi = rho u u): f_i^eq = w_i [rho + 3 e.j + 4.5 e e : Pi - 1.5 tr Pi].
template <class R>
__device__ __forceinline__ R feq_i(int i, R rho, R jx, R jy, R pxx, R pxy, R pyy) {
  const R ex = R(cx(i)), ey = R(cy(i));
  R ej = ex * jx + ey * jy;
  R eep = ex * ex * pxx + R(2) * ex * ey * pxy + ey * ey * pyy;
  return wgt<R>(i) * (rho + R(3) * ej + R(4.5) * eep - R(1.5) * (pxx + pyy));
}

// Post-stream population f_i(x, y) of the current state (parity 0: after an
// odd step, parity 1: after an even step), and the flat slot it lives in
// (-1 for an inlet node, whose state is the inlet equilibrium).
template <int P>
__device__ __forceinline__ typename Prec<P>::R post_stream(
    const Geom& g, const StepConsts<typename Prec<P>::R>& c, const typename Prec<P>::S* A,
    int parity, int x, int y, int i, long long& where) {
  typedef typename Prec<P>::R R;
  if (x == 0 && g.bc[0] == BC_INLET) { where = -1; return c.feq_in[i]; }
  if (parity == 0) {
    where = slot_index(g, i, x, y);
    return Prec<P>::ld(A[where], i);
  }
  int sx, sy, slot, ws;
  if (!locE(g, x, y, i, sx, sy, slot, ws)) { where = -1; return c.feq_in[i]; }
  where = slot_index(g, slot, sx, sy);
  R v = Prec<P>::ld(A[where], slot);
  if (ws >= 0) v += c.wall[ws][i];
  return v;
}

}  // namespace ibm
