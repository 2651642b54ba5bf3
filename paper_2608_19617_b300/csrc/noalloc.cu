// lbm_step_window_noalloc: one forward window without any device allocation.
//
// Some callers cannot call cudaMalloc: code running inside a CUDA graph that
// is being captured, a host that hands out only pre-registered buffers, or a
// sandbox whose allocator is not reachable from this library.  For them this
// entry point runs the sampled forward window of lbm_step_window on buffers
// the caller already owns, and keeps its only scratch -- the per-block window
// sums, the window-end results and the non-finite flag -- in a file-scope
// device array that is part of the library image.
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
constexpr size_t kHeaderBytes = 256;   // WindowAcc + non-finite flag
constexpr size_t kScratchBytes = kHeaderBytes + size_t(kNoallocMaxBlocks) * 32;

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

// The fused forward step of lbm_step_window with two differences: g(phi) is
// evaluated from gamma on the fly (as the design kernel does, in FP64, then
// rounded), and the pressure objective samples cs^2 rho directly instead of
// cs^2 (rho - 1) plus a precomputed constant.
template <class L>
__global__ void __launch_bounds__(lbm::kBlock) fwd_step_noalloc_kernel(lbm::FwdArgs<float> A, const float* gamma,
                                                                      double q, double g_max) {
  using namespace lbm;
  const Geo& g = A.geo;
  const int x = blockIdx.x * kBlock + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  const bool alive = x < g.nx;
  float bj = 0, bm = 0;
  if (alive) {
    const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
    const bool face = on_face<L>(g, x, y, z);
    const uint8_t cls = face ? A.cls[i] : uint8_t(FLUID);
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
#pragma unroll
    for (int a = 0; a < L::Q; ++a) A.dst[a * g.n + i] = mul_rn(float(L::w(a)), blend_value<L, float>(a, C));
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
lbm_status fail_arg(const char* msg) {
  lbm_set_last_error(msg);
  return LBM_ERR_ARG;
}
}  // namespace

extern "C" lbm_status lbm_step_window_noalloc(const lbm_config* cfg, const uint8_t* node_class,
                                              const float* design_gamma, const float* objective_weights,
                                              const float* inlet_u, float* pop, float* pop_tmp, void* stream,
                                              double* J_window, double* monitor_window) {
  if (!cfg || !node_class || !design_gamma || !objective_weights || !inlet_u || !pop || !pop_tmp)
    return LBM_ERR_ARG;
  // Configuration checks shared with lbm_create (no allocation involved).
  size_t bytes = 0;
  const lbm_status vs = lbm_workspace_size(cfg, &bytes);
  if (vs != LBM_OK) return vs;
  const lbm_config& c = *cfg;
  if (c.precision != LBM_FP32) return fail_arg("the no-allocation window runs the FP32 solver only");
  const int gx = (c.nx + lbm::kBlock - 1) / lbm::kBlock;
  const long long nblocks = (long long)gx * c.ny * c.nz;
  if (nblocks > kNoallocMaxBlocks)
    return fail_arg("lattice too large for the no-allocation scratch (at most 16384 blocks of 128 nodes)");
  if (pop == pop_tmp) return fail_arg("pop and pop_tmp must be different buffers");

  void* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) {
    lbm_set_last_error("cudaGetSymbolAddress of the no-allocation scratch failed");
    return LBM_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* base = static_cast<unsigned char*>(scratch);
  lbm::WindowAcc* acc = reinterpret_cast<lbm::WindowAcc*>(base);
  int* nonfinite = reinterpret_cast<int*>(base + 128);
  double* blk = reinterpret_cast<double*>(base + kHeaderBytes);
  // Start from zero: window sums, results and flag (has_prev too: a call does
  // not compare against an earlier call's window).
  if (cudaMemsetAsync(base, 0, kHeaderBytes + size_t(nblocks) * 32, s) != cudaSuccess) return LBM_ERR_CUDA;

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
    if (c.lattice == LBM_D2Q9)
      fwd_step_noalloc_kernel<D2Q9><<<grid, lbm::kBlock, 0, s>>>(A, design_gamma, c.q_interp, c.g_max);
    else
      fwd_step_noalloc_kernel<D3Q19><<<grid, lbm::kBlock, 0, s>>>(A, design_gamma, c.q_interp, c.g_max);
    cur ^= 1;
  }
  const double mon_scale =
      c.monitor_kind == LBM_MON_DRAG ? 1.0 / (0.5 * c.rho_out * c.monitor_u * c.monitor_u * c.monitor_l) : 0.0;
  lbm::window_end_kernel<<<1, lbm::kEndThreads, 0, s>>>(blk, int(nblocks), acc, c.conv_tol, nonfinite,
                                                         double(c.window_len / c.sample_every), 0.0, mon_scale,
                                                         c.monitor_kind);
  if (cur == 1 &&
      cudaMemcpyAsync(pop, pop_tmp, n * c.lattice * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return LBM_ERR_CUDA;
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  lbm::WindowAcc h;
  if (cudaMemcpyAsync(&h, acc, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;
  if (h.nonfinite) return LBM_ERR_NONFINITE;
  if (J_window) *J_window = h.jmean;
  if (monitor_window) *monitor_window = h.mmean;
  return LBM_OK;
}
