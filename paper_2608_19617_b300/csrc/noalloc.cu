// lbm_step_window_noalloc: one forward window without any device allocation.
//
// Some callers cannot call cudaMalloc: a host process that hands this library
// only buffers it registered up front (a serving runtime with a fixed memory
// pool, a plug-in inside another application's allocator), or a sandbox that
// does not expose the CUDA allocator at all.  For them this entry point runs
// the sampled forward window of lbm_step_window on buffers the caller already
// owns, and keeps its only scratch -- the per-block window sums, the
// window-end results and two flags -- in a file-scope device array that is
// part of the library image.  The call waits for its stream before it
// returns, since it reads the window means back to the host.
//
// The scratch array lives on every GPU that loads the library until the
// process exits.  It is shared by every call on a device and keeps the last
// call's contents; each call clears what has to start at zero.  Calls that
// overlap on the GPU (two streams at once) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lattice.cuh"
#include "lbmadj.h"

namespace {
#include "kernels.cuh"
}  // namespace

namespace {

// Largest grid the scratch array holds: kNoallocMaxBlocks blocks of 128
// nodes (2,097,152 lattice nodes), 32 bytes of window sums per block.
constexpr int kNoallocMaxBlocks = 16384;
constexpr size_t kHeaderBytes = 256;   // WindowAcc, then the non-finite flag (byte 128) and the bad-class flag (132)
constexpr size_t kScratchBytes = kHeaderBytes + size_t(kNoallocMaxBlocks) * 32;

static_assert(sizeof(lbm::WindowAcc) <= 128, "the window results must fit before the flags");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The array's
// name is a host-side stand-in in host code, so the address is looked up once
// per device with that device current.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Does node (x, y, z) of class cls obey the rules lbm_create checks on the
// host: interior nodes FLUID; a face node with links from outside the domain
// not FLUID; an inlet on the x = 0 face with exactly the unknowns of that
// face (D2Q9: c1, c5, c8); a pressure outlet (D2Q9) likewise on x = nx-1; a
// zero-gradient outlet on a bounded x face whose unknowns are exactly the
// directions entering through that face.  A map that breaks them would make
// the boundary rules read outside the lattice or leave populations unset.
template <class L>
__device__ bool class_ok(const lbm::Geo& g, int x, int y, int z, bool face, uint8_t cls) {
  using namespace lbm;
  if (cls > OUTLET_ZG) return false;
  if (!face) return cls == FLUID;
  unsigned unk = 0, in_x0 = 0, in_x1 = 0;
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    unsigned j;
    if (!neighbour(g, x, y, z, -L::cx(a), -L::cy(a), -L::cz(a), j)) unk |= 1u << a;
    if (L::cx(a) == 1) in_x0 |= 1u << a;
    if (L::cx(a) == -1) in_x1 |= 1u << a;
  }
  switch (cls) {
    case FLUID: return unk == 0;
    case WALL: return true;
    case INLET: return x == 0 && unk == (L::Q == 9 ? ((1u << 1) | (1u << 5) | (1u << 8)) : in_x0);
    case OUTLET_P: return L::Q == 9 && x == g.nx - 1 && unk == ((1u << 3) | (1u << 6) | (1u << 7));
    default:
      return !g.px && ((x == 0 && unk == in_x0) || (x == g.nx - 1 && unk == in_x1));
  }
}

// The fused forward step of lbm_step_window with three differences: g(phi)
// is evaluated from gamma on the fly (as the design kernel does, in FP64,
// then rounded), the pressure objective samples cs^2 rho directly instead of
// cs^2 (rho - 1) plus a precomputed constant, and every node checks its class
// (bad_class) since the map never passed the host checks of lbm_create.
template <class L>
__global__ void __launch_bounds__(lbm::kBlock) fwd_step_noalloc_kernel(lbm::FwdArgs<float> A, const float* gamma,
                                                                      double q, double g_max, int* bad_class) {
  using namespace lbm;
  const Geo& g = A.geo;
  const int x = blockIdx.x * kBlock + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  const bool alive = x < g.nx;
  float bj = 0, bm = 0;
  if (alive) {
    const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
    const bool face = on_face<L>(g, x, y, z);
    uint8_t cls = A.cls[i];
    if (!class_ok<L>(g, x, y, z, face, cls)) {
      *bad_class = 1;
      cls = face ? uint8_t(WALL) : uint8_t(FLUID);   // keep every access inside the lattice; the call fails
    }
    const float u0 = (face && cls == INLET) ? A.uin[y + g.ny * z] : 0.f;
    float f[L::Q];
    gather<L, float>(A.src, g, x, y, z, i, face, cls, u0, A.ph.rho_out, f);
    Mom<L, float> M;
    moments<L, float>(f, A.ph, M);
    if (!(M.rho > 0.f) || !isfinite(M.pn) || !isfinite(M.m[0] + M.m[1] + M.m[2])) *A.nonfinite = 1;
    const double phi = 1.0 - double(gamma[i]);
    const float gi = float(g_max * (1.0 - phi * (1.0 + q) / (phi + q)));
    Blend<float> C;
    blend_coefs<L, float>(M, gi, C);
    blend_store<L, float>(A.dst, g.n, i, C);
    if (A.sample) {
      const int* b = A.obj.box;
      if (x >= b[0] && x < b[1] && y >= b[2] && y < b[3] && z >= b[4] && z < b[5]) {
        const float w = A.wobj[i];
        if (w != 0.f) {
          const float psi = A.obj.kind == OBJ_PRES ? cs2<float>() * M.rho : local_objective<L, float>(M, A.obj, gi);
          bj = w * psi;
        }
      }
      if (A.obj.mon == MON_DRAG) bm = -2.f * gi * M.m[0];
    }
  }
  if (A.sample) {
    block_sum2<float>(bj, bm);
    sample_commit(double(bj), double(bm), A.blk);
  }
}

}  // namespace

// Records the reason returned by lbm_last_error (defined with the other entry points).
void lbm_set_last_error(const char* msg);

namespace {
lbm_status fail_with(lbm_status st, const char* msg) {
  lbm_set_last_error(msg);
  return st;
}

lbm_status fail_cuda(const char* what, cudaError_t e) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  lbm_set_last_error(m.c_str());
  return LBM_ERR_CUDA;
}

template <class L>
cudaError_t launch_step(dim3 grid, cudaStream_t s, const lbm::FwdArgs<float>& A, const float* gamma, double q,
                        double g_max, int* bad_class) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(lbm::kBlock);
  cfg.stream = s;
  return cudaLaunchKernelEx(&cfg, fwd_step_noalloc_kernel<L>, A, gamma, q, g_max, bad_class);
}
}  // namespace

extern "C" lbm_status lbm_step_window_noalloc(const lbm_config* cfg, const uint8_t* node_class,
                                              const float* design_gamma, const float* objective_weights,
                                              const float* inlet_u, float* pop, float* pop_tmp, void* stream,
                                              double* J_window, double* monitor_window) {
  if (!cfg || !node_class || !design_gamma || !objective_weights || !inlet_u || !pop || !pop_tmp)
    return fail_with(LBM_ERR_ARG, "null argument (every pointer except J_window and monitor_window is required)");
  // Configuration checks shared with lbm_create (no allocation involved).
  size_t bytes = 0;
  const lbm_status vs = lbm_workspace_size(cfg, &bytes);
  if (vs != LBM_OK) return vs;
  const lbm_config& c = *cfg;
  if (c.precision != LBM_FP32) return fail_with(LBM_ERR_ARG, "the no-allocation window runs the FP32 solver only");
  const int gx = (c.nx + lbm::kBlock - 1) / lbm::kBlock;
  const long long nblocks = (long long)gx * c.ny * c.nz;
  if (nblocks > kNoallocMaxBlocks)
    return fail_with(LBM_ERR_ARG,
                     "lattice too large for the no-allocation scratch (at most 16384 blocks of 128 nodes)");
  if (pop == pop_tmp) return fail_with(LBM_ERR_ARG, "pop and pop_tmp must be different buffers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // The call ends with a read-back and a wait on the stream, which a stream
  // in capture mode cannot take: refuse it before enqueuing anything.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return fail_cuda("cudaStreamIsCapturing", e);
  if (cap != cudaStreamCaptureStatusNone)
    return fail_with(LBM_ERR_ARG, "the stream is capturing a CUDA graph; this call reads its results back and waits "
                                  "for the stream, so it must be called outside a capture");

  void* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess) return fail_cuda("cudaGetSymbolAddress of the no-allocation scratch", e);
  unsigned char* base = static_cast<unsigned char*>(scratch);
  lbm::WindowAcc* acc = reinterpret_cast<lbm::WindowAcc*>(base);
  int* nonfinite = reinterpret_cast<int*>(base + 128);
  int* bad_class = reinterpret_cast<int*>(base + 132);
  double* blk = reinterpret_cast<double*>(base + kHeaderBytes);
  // Start from zero: window sums, results and flags (has_prev too: a call does
  // not compare against an earlier call's window).
  e = cudaMemsetAsync(base, 0, kHeaderBytes + size_t(nblocks) * 32, s);
  if (e != cudaSuccess) return fail_cuda("cudaMemsetAsync of the scratch", e);

  const size_t n = size_t(c.nx) * c.ny * c.nz;
  lbm::FwdArgs<float> A{};
  A.gfield = nullptr;
  A.cls = node_class;
  A.uin = inlet_u;
  A.wobj = objective_weights;
  A.geo = lbm::Geo{c.nx, c.ny, c.nz, c.periodic[0], c.periodic[1], c.periodic[2], unsigned(n), unsigned(c.nx),
                   unsigned(c.nx) * unsigned(c.ny)};
  A.ph = lbm::Phys<float>{float(c.tau), float(c.cs_smag * c.cs_smag), float(c.rho_out)};
  A.obj.kind = c.objective_kind;
  A.obj.mon = c.monitor_kind;
  for (int k = 0; k < 3; ++k) A.obj.uref[k] = float(c.objective_uref[k]);
  for (int k = 0; k < 6; ++k) A.obj.box[k] = c.obj_box[k];
  A.obj.ws = float(double(c.sample_every) / double(c.window_len));
  A.blk = blk;
  A.nonfinite = nonfinite;
  const dim3 grid(gx, c.ny, c.nz);
  float* buf[2] = {pop, pop_tmp};
  int cur = 0;
  for (int k = 0; k < c.window_len; ++k) {
    A.src = buf[cur];
    A.dst = buf[cur ^ 1];
    A.sample = k % c.sample_every == 0;
    e = c.lattice == LBM_D2Q9 ? launch_step<D2Q9>(grid, s, A, design_gamma, c.q_interp, c.g_max, bad_class)
                              : launch_step<D3Q19>(grid, s, A, design_gamma, c.q_interp, c.g_max, bad_class);
    if (e != cudaSuccess) return fail_cuda("launch of the no-allocation step kernel", e);
    cur ^= 1;
  }
  const double mon_scale =
      c.monitor_kind == LBM_MON_DRAG ? 1.0 / (0.5 * c.rho_out * c.monitor_u * c.monitor_u * c.monitor_l) : 0.0;
  {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(1);
    lc.blockDim = dim3(lbm::kEndThreads);
    lc.stream = s;
    e = cudaLaunchKernelEx(&lc, lbm::window_end_kernel, blk, int(nblocks), acc, c.conv_tol,
                           static_cast<const int*>(nonfinite), double(c.window_len / c.sample_every), 0.0,
                           mon_scale, int(c.monitor_kind));
    if (e != cudaSuccess) return fail_cuda("launch of the window-end kernel", e);
  }
  if (cur == 1) {
    e = cudaMemcpyAsync(pop, pop_tmp, n * c.lattice * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return fail_cuda("cudaMemcpyAsync of the last field into pop", e);
  }
  // Window results and the two flags, read back through a stack copy of the
  // scratch header.
  unsigned char h[kHeaderBytes];
  e = cudaMemcpyAsync(h, base, kHeaderBytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return fail_cuda("cudaMemcpyAsync of the window results", e);
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail_cuda("cudaStreamSynchronize", e);
  lbm::WindowAcc res;
  int flag_nonfinite = 0, flag_class = 0;
  std::memcpy(&res, h, sizeof res);
  std::memcpy(&flag_nonfinite, h + 128, sizeof(int));
  std::memcpy(&flag_class, h + 132, sizeof(int));
  if (flag_class)
    return fail_with(LBM_ERR_ARG, "node_class breaks the rules lbm_create checks (a class out of range, a non-FLUID "
                                  "interior node, or a boundary class on the wrong face); pop holds no valid window");
  if (flag_nonfinite || res.nonfinite)
    return fail_with(LBM_ERR_NONFINITE, "the window produced a non-positive density or a non-finite value");
  if (J_window) *J_window = res.jmean;
  if (monitor_window) *monitor_window = res.mmean;
  return LBM_OK;
}
