// TMA-staged interior step kernels.
//
// The interior kernels of kernels.cuh load each pulled population straight
// from global memory into registers, so the bytes a streaming SM keeps in
// flight are bounded by its resident threads.  Here persistent blocks walk the
// interior row segments (tiles of kBlock nodes) and one thread per block
// stages the source rows of later tiles in shared memory with tensor-memory
// -accelerator copies (cp.async.bulk.tensor), kTmaStages tiles deep, while the
// block computes the current tile from shared memory.
//
// The population field [Q][nz][ny][nx] is described to the TMA unit as a 3D
// tensor {nx, ny, nz Q}: direction a of node (x, y, z) is element
// (x, y, z + nz a).  A forward tile at (x0 .. x0+127, y, z) pulls, for each a,
// the row (y - c_ya, z - c_za) shifted by -c_xa; one box of kTmaBox elements
// starting at x0 - 5 (a multiple of 4, as the TMA unit requires of the
// innermost coordinate of a 4-byte type) covers every shift.  The box may
// start left of x = 0 or end right of nx; those elements are filled with zero
// and never used.  The node arithmetic is forward_core(), the same explicitly
// rounded function the per-step kernels use, and the block sums go to the
// same per-tile slots.
//
// Every wait on a copy is bounded: a wait that runs out raises status[0],
// waits (bounded) for the block's other copies in flight and leaves.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace lbm {

constexpr int kTmaStages = 3;
constexpr int kTmaBox = kBlock + 8;   // nodes x0-5 .. x0+130
constexpr int kTmaLead = 5;           // x0 - box start
constexpr unsigned kTmaWaitPolls = 1u << 24;

// Shared-memory row of one staged box, padded to a multiple of 128 bytes so
// that every copy lands on a 128-byte boundary.
template <class R>
__host__ __device__ constexpr int tma_row() { return int(((kTmaBox * sizeof(R) + 127) / 128) * 128 / sizeof(R)); }

template <class L, class R>
__host__ __device__ constexpr size_t fwd_tma_smem() { return size_t(kTmaStages) * L::Q * tma_row<R>() * sizeof(R); }

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// One bounded wait for the phase of the given parity; true once it completed.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  for (unsigned it = 0; it < kTmaWaitPolls; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z),
        "r"(smem_addr(bar))
      : "memory");
}

// Interior tile t -> its first node (x0, y, z).
template <class L>
__device__ __forceinline__ void tile_origin(unsigned t, unsigned igx, unsigned igy, int& x0, int& y, int& z) {
  const unsigned bx = t % igx, r = t / igx, by = r % igy, bz = r / igy;
  x0 = 1 + int(bx) * kBlock;
  y = 1 + int(by);
  z = L::D == 3 ? 1 + int(bz) : int(bz);   // D2Q9: z is the slice of a batch
}

// Interior forward step, TMA-staged.  Dynamic shared memory: kTmaStages x Q
// rows of tma_row<R>() elements (fwd_tma_smem).
template <class L, class R, bool MOM = false>
__global__ void __launch_bounds__(kBlock) fwd_tma_kernel(const __grid_constant__ CUtensorMap src_map, FwdArgs<R> A,
                                                         unsigned ntiles, unsigned igx, unsigned igy, int* status) {
  extern __shared__ __align__(128) unsigned char tma_smem[];
  __shared__ __align__(8) unsigned long long full[kTmaStages];
  R* buf = reinterpret_cast<R*>(tma_smem);
  pdl_enter();
  const Geo& g = A.geo;
  const FwdStep<R> P{A.src, A.dst, A.sample, A.mom};
  const unsigned tid = threadIdx.x;
  if (tid == 0) {
    for (int s = 0; s < kTmaStages; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // Thread 0: stage the source rows of the block's j-th tile.
  auto issue = [&](unsigned j) {
    const unsigned t = blockIdx.x + j * gridDim.x;
    if (t >= ntiles) return;
    int x0, y, z;
    tile_origin<L>(t, igx, igy, x0, y, z);
    const int st = int(j % kTmaStages);
    mbar_expect_tx(&full[st], unsigned(L::Q * kTmaBox * sizeof(R)));
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
      tma_load_3d(buf + (st * L::Q + a) * tma_row<R>(), &src_map, x0 - kTmaLead, y - L::cy(a),
                  z - L::cz(a) + g.nz * a, &full[st]);
  };
  if (tid == 0)
    for (unsigned j = 0; j + 1 < unsigned(kTmaStages); ++j) issue(j);
  for (unsigned j = 0; blockIdx.x + j * gridDim.x < ntiles; ++j) {
    if (tid == 0) issue(j + kTmaStages - 1);   // into the stage the previous tile released
    const int st = int(j % kTmaStages);
    int ok = 1;
    if (tid == 0) ok = mbar_wait(&full[st], (j / kTmaStages) & 1u);
    if (__syncthreads_or(!ok)) {
      // A copy never arrived: report, let the block's other copies land, leave.
      if (tid == 0) {
        atomicExch(status, 1);
        for (unsigned k = j; k < j + kTmaStages; ++k)
          if (blockIdx.x + k * gridDim.x < ntiles) mbar_wait(&full[k % kTmaStages], (k / kTmaStages) & 1u);
      }
      return;
    }
    const unsigned t = blockIdx.x + j * gridDim.x;
    int x0, y, z;
    tile_origin<L>(t, igx, igy, x0, y, z);
    const int x = x0 + int(tid);
    R bj = 0, bm = 0;
    if (x < g.nx - 1) {
      const R* row = buf + st * L::Q * tma_row<R>() + kTmaLead + int(tid);
      R f[L::Q];
#pragma unroll
      for (int a = 0; a < L::Q; ++a) f[a] = row[a * tma_row<R>() - L::cx(a)];
      forward_core<L, R, MOM>(A, P, x, y, z, unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz, f, bj, bm);
    }
    if (A.sample) {   // uniform across the grid
      block_sum2<R>(bj, bm);
      sample_commit(double(bj), double(bm), A.blk, t);
    }
    __syncthreads();   // every thread is done with stage st before it is refilled
  }
}

}  // namespace lbm
