// ibm_noalloc.cu -- the immersed-boundary correction loop for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or a host process with a fixed device-memory
// budget, plug-ins that may only touch buffers handed to them, or code paths
// where an allocation could block or fail at an unrecoverable moment.  For
// them, ibm_ib_correct_noalloc runs the same band-build and correction
// kernels as ibm_step on buffers the caller owns, and keeps every
// intermediate array in one file-scope device array of fixed size instead of
// allocating.  That array is reserved when the library is loaded and is held
// on every GPU the library touches until the process exits.
#include <mutex>
#include <string>

#include "ibm_internal.h"

namespace ibm {
namespace {

// Limits of the no-allocation path and the scratch they need (FP64 worst
// case, each array rounded up to 256 bytes): about 7.5 MB.
constexpr long long kNaMaxNodes = 262144;    // nx * ny
constexpr int kNaMaxMarkers = 512;
constexpr int kNaMaxCorr = 64;
constexpr size_t kNaScratchBytes = 8u << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
void* g_na_base[kNaMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (the name is only a host-side stand-in for it).
cudaError_t scratch_base(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_base[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_na_base[dev] = p;
  }
  *out = g_na_base[dev];
  return cudaSuccess;
}

// Bump allocator over the scratch array (256-byte aligned pieces).  A piece
// that does not fit fails every later take as well (ok stays false), so one
// check after the last take covers them all.
struct Carve {
  unsigned char* base;
  size_t used;
  size_t cap;
  bool ok = true;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    if (!ok || used + bytes > cap) {
      ok = false;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
};

template <class R>
__global__ void k_na_prepare(int M, const double* __restrict__ xy, const double* __restrict__ ds,
                             const double* __restrict__ uv, double* __restrict__ X, double* __restrict__ Y,
                             double* __restrict__ dsm, double* __restrict__ dX, double* __restrict__ dY,
                             int* __restrict__ mbody, R* __restrict__ Ux, R* __restrict__ Uy,
                             BodyDev* __restrict__ body) {
  const int l = blockIdx.x * blockDim.x + threadIdx.x;
  if (l == 0) {
    BodyDev b = {};
    b.kind = IBM_BODY_FIXED;
    b.m0 = 0;
    b.m1 = M;
    *body = b;
  }
  if (l >= M) return;
  X[l] = xy[2 * l];
  Y[l] = xy[2 * l + 1];
  dsm[l] = ds[l];
  dX[l] = xy[2 * l];
  dY[l] = xy[2 * l + 1];
  mbody[l] = 0;
  Ux[l] = (R)uv[2 * l];
  Uy[l] = (R)uv[2 * l + 1];
}

template <class R>
__global__ void k_na_finish(int n, const R* __restrict__ resid, const BodyDev* __restrict__ body,
                            double* __restrict__ resid_out, double* __restrict__ force_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n && resid_out) resid_out[k] = (double)resid[k];
  if (k == 0 && force_out) {
    force_out[0] = body->F_ib[0];
    force_out[1] = body->F_ib[1];
  }
}

ibm_status na_fail(ibm_status st, const std::string& msg) {
  set_thread_error(msg.c_str());
  return st;
}

}  // namespace
}  // namespace ibm

using namespace ibm;

extern "C" ibm_status ibm_ib_correct_noalloc(int nx, int ny, int prec, void* f, int n_markers,
                                             const double* xy, const double* ds, const double* uvel,
                                             int n_corr, double* resid_out, double* force_out,
                                             void* cuda_stream) {
  if (nx < 4 || ny < 4) return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: nx and ny must be >= 4");
  if ((long long)nx * ny > kNaMaxNodes)
    return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: nx*ny exceeds the limit of 262144 nodes");
  if (n_markers < 1 || n_markers > kNaMaxMarkers)
    return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: n_markers must be in [1, 512]");
  if (n_corr < 0 || n_corr > kNaMaxCorr)
    return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: n_corr must be in [0, 64]");
  if (prec != IBM_FP64 && prec != IBM_FP32)
    return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: prec must be IBM_FP64 or IBM_FP32");
  if (!f || !xy || !ds || !uvel)
    return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: f, xy, ds and uvel are required");
  // CUDA keeps one pending launch error per host thread: clear what earlier
  // work left there, so that the checks below see only this call's work.
  cudaGetLastError();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    cudaGetLastError();
    return na_fail(IBM_ERR_CUDA, "ibm_ib_correct_noalloc: no usable current CUDA device");
  }
  void* base = nullptr;
  cudaError_t e = scratch_base(dev, &base);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return na_fail(IBM_ERR_CUDA, std::string("ibm_ib_correct_noalloc: cudaGetSymbolAddress: ") +
                                     cudaGetErrorString(e));
  }
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0 || ib_blocks_per_sm(prec) < 1) {
    cudaGetLastError();
    return na_fail(IBM_ERR_CUDA, "ibm_ib_correct_noalloc: the correction kernel cannot be resident");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;

  // A stack context whose device arrays are all pieces of the scratch array.
  Ctx c;
  c.device = dev;
  c.stream = s;
  c.prec = prec;
  c.s_bytes = prec == IBM_FP64 ? 8 : 4;
  c.r_bytes = c.s_bytes;
  c.desc.nx = nx;
  c.desc.ny = ny;
  c.desc.tau = 1.0;
  c.desc.rho0 = 1.0;
  c.desc.prec = prec;
  c.desc.n_corr = n_corr;
  c.desc.delta_points = 4;
  c.geom.nx = nx;
  c.geom.ny = ny;
  c.geom.nxp = nx;                          // caller's layout: [9][ny][nx]
  c.geom.plane = (long long)nx * ny;
  for (int k = 0; k < 4; ++k) c.geom.bc[k] = BC_PERIODIC;
  c.f = f;
  c.nm = n_markers;
  c.nb = 1;
  c.mcap = n_markers;
  c.bcap = n_markers * kStencil;
  c.nseg_x = (nx + kSegW - 1) / kSegW;
  c.segcap = c.bcap;
  // At most 512 markers: the correction kernel runs as one CTA with block
  // barriers (as ibm_step does for boundaries this small), so it never waits
  // for CTAs that other work on the device keeps from being scheduled.
  c.ib_grid = 1;
  c.ib_grid_last = 1;
  c.ib_grid_max = sms;
  c.ib_prio = 0;
  c.band_collide = false;                   // correction only
  const size_t R = c.r_bytes;
  const size_t ent_bytes = prec == IBM_FP64 ? sizeof(Ent<double>) : sizeof(Ent<float>);
  const long long nodes = (long long)nx * ny;
  Carve cv{reinterpret_cast<unsigned char*>(base), 0, kNaScratchBytes};
  c.dnode2band = cv.take<int>(nodes);
  c.dsegflag = cv.take<int>((size_t)c.nseg_x * ny);
  c.dseglist = cv.take<int>(c.segcap);
  c.dctr = cv.take<int>(CTR_COUNT);
  c.dbar = cv.take<unsigned long long>(1);
  c.dX = cv.take<double>(n_markers);
  c.dY = cv.take<double>(n_markers);
  c.dds = cv.take<double>(n_markers);
  c.ddX = cv.take<double>(n_markers);
  c.ddY = cv.take<double>(n_markers);
  c.dmbody = cv.take<int>(n_markers);
  c.dUx = cv.take<unsigned char>(R * n_markers);
  c.dUy = cv.take<unsigned char>(R * n_markers);
  c.dW = cv.take<unsigned char>(R * c.bcap);
  c.dnode_of = cv.take<int>(c.bcap);
  c.dband_of = cv.take<int>(c.bcap);
  c.dclaim = cv.take<int>(c.bcap);
  c.dbnode = cv.take<int>(c.bcap);
  c.dbcnt = cv.take<int>(c.bcap);
  c.dent = cv.take<unsigned char>(ent_bytes * (size_t)c.bcap * kBandCap);
  c.dbq = cv.take<unsigned char>(R * 8 * (size_t)c.bcap);
  c.dmq = cv.take<unsigned char>(R * 4 * (size_t)n_markers);
  c.dAh = cv.take<unsigned char>(R * 2 * (size_t)n_markers * (n_corr + 1));
  c.dCm = cv.take<unsigned char>(R * 3 * (size_t)n_markers);
  c.dG = cv.take<unsigned char>(ent_bytes * (size_t)n_markers * kGCap);
  c.dgcnt = cv.take<int>(n_markers);
  c.dresid = cv.take<unsigned char>(R * (n_corr + 1));
  c.dbodies = cv.take<BodyDev>(1);
  c.dfpart = cv.take<double>((size_t)((n_markers + kForceChunk - 1) / kForceChunk) * 3);
  if (!cv.ok)
    return na_fail(IBM_ERR_INVALID, "ibm_ib_correct_noalloc: the scratch array is too small for this call");

  // The scratch array keeps the previous call's contents: reset what the
  // kernels expect to start empty.
  e = cudaMemsetAsync(c.dnode2band, 0xFF, sizeof(int) * (size_t)nodes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.dsegflag, 0, sizeof(int) * (size_t)c.nseg_x * ny, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.dctr, 0, sizeof(int) * CTR_COUNT, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.dbar, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.dbcnt, 0, sizeof(int) * (size_t)c.bcap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.dent, 0, ent_bytes * (size_t)c.bcap * kBandCap, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.dG, 0, ent_bytes * (size_t)n_markers * kGCap, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return na_fail(IBM_ERR_CUDA, std::string("ibm_ib_correct_noalloc: ") + cudaGetErrorString(e));
  }
  if (prec == IBM_FP64)
    k_na_prepare<double><<<(n_markers + 127) / 128, 128, 0, s>>>(n_markers, xy, ds, uvel, c.dX, c.dY, c.dds,
        c.ddX, c.ddY, c.dmbody, (double*)c.dUx, (double*)c.dUy, c.dbodies);
  else
    k_na_prepare<float><<<(n_markers + 127) / 128, 128, 0, s>>>(n_markers, xy, ds, uvel, c.dX, c.dY, c.dds,
        c.ddX, c.ddY, c.dmbody, (float*)c.dUx, (float*)c.dUy, c.dbodies);
  launch_band_build(c, s);
  launch_ib_loop(c, 0, false, s);
  if (prec == IBM_FP64)
    k_na_finish<double><<<1, 128, 0, s>>>(n_corr + 1, (const double*)c.dresid, c.dbodies, resid_out, force_out);
  else
    k_na_finish<float><<<1, 128, 0, s>>>(n_corr + 1, (const float*)c.dresid, c.dbodies, resid_out, force_out);
  e = cudaGetLastError();                   // launch errors of this call's kernels
  int ctr[CTR_COUNT] = {0, 0, 0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(ctr, c.dctr, sizeof(ctr), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return na_fail(IBM_ERR_CUDA, std::string("ibm_ib_correct_noalloc: ") + cudaGetErrorString(e));
  }
  if (ctr[CTR_ERR] & ERR_DIVERGED)
    return na_fail(IBM_ERR_DIVERGED, "ibm_ib_correct_noalloc: non-finite no-slip residual");
  if (ctr[CTR_ERR] & (ERR_BAND_CAP | ERR_LIST_CAP | ERR_SEG_CAP | ERR_G_CAP))
    return na_fail(IBM_ERR_BOUNDS, "ibm_ib_correct_noalloc: markers too dense for the band capacity");
  return IBM_OK;
}
