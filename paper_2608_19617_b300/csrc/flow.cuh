// Persistent step kernels: one cooperative launch runs a whole run of time
// steps (a checkpoint segment of the forward window, of the recompute, or of
// the adjoint sweep) instead of one launch per step.
//
// The lattice is cut into P bands, contiguous ranges of node indices (face
// nodes weighted heavier so that the bands cost about the same).  Block b owns
// band b for every step of the launch: its interior nodes in index order and
// its face nodes through the face table rows that fall in the band.  A step of
// band b reads only the bands its nodes pull from (forward) or push to
// (adjoint) and overwrites a buffer that those same bands read one step
// earlier, so block b may start step k as soon as every band in its wait set
// W(b) = deps(b) u rdeps(b) has finished step k-1.  W(b) is built on the host
// from the exact index sets (periodic wrap and boundary tables included).
//
// Progress is published per band: done[b] = steps finished in this launch
// (zeroed before the launch).  Thread 0 publishes with a release store after
// the block barrier, which orders every store of the block before the counter;
// waiters read the counters with acquire loads, and the fields written inside
// the launch are loaded through L2 (ldf<true>).  Every wait is bounded by the
// global timer: a wait that runs out raises status[0], every other waiter sees
// it and leaves, and the host reports the launch as failed.  The grid is
// launched cooperatively with no more blocks than can be resident at once.
#pragma once

#include "kernels.cuh"

namespace lbm {

constexpr int kFlowBlock = 256;      // threads per band
constexpr int kFlowMinBlocks = 4;    // FP32 register budget: 4 bands per SM (64 registers)
constexpr int kFlowMaxBands = 4096;  // upper bound on P (workspace sizing)
constexpr int kFlowMaxWait = 64;     // upper bound on |W(b)|

struct Flow {
  const unsigned* band;   // [P+1] node-index bounds of the bands
  const unsigned* fband;  // [P+1] face-table row bounds of the bands
  const int* wptr;        // [P+1] offsets of the wait sets in widx
  const int* widx;        // concatenated wait sets
  int* done;              // [P] steps finished in this launch
  int* status;            // [0] != 0: a wait timed out, every block leaves
  double* blk;            // [P][4] compensated window sums of the bands
  unsigned long long wait_ns;   // longest wait without progress
  int silent;             // test hook: this band never publishes (-1: none)
};

// Per-step field addresses.  Ping-pong (stride == 0): step k reads a and
// writes b on even k, the reverse on odd k.  Chain: step k writes
// b + k stride and reads a (k = 0) or the previous step's output.
template <class R>
struct Chain {
  R* a;
  R* b;
  long long stride;   // elements
  __device__ __forceinline__ const R* src(int k) const {
    if (stride == 0) return (k & 1) ? b : a;
    return k == 0 ? a : b + (long long)(k - 1) * stride;
  }
  __device__ __forceinline__ R* dst(int k) const {
    if (stride == 0) return (k & 1) ? a : b;
    return b + (long long)k * stride;
  }
};

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Block-wide: wait until every band of W(b) has done >= target steps.  Warp 0
// polls, one lane per band.  Returns false (for the whole block) when a wait
// ran out or another block raised the status.
__device__ __forceinline__ bool flow_wait(const Flow& fl, unsigned b, int target) {
  __shared__ int s_ok;
  if (threadIdx.x < 32) {
    const int w0 = fl.wptr[b], w1 = fl.wptr[b + 1];
    bool ok = true;
    const unsigned long long t0 = global_ns();
    for (int w = w0 + int(threadIdx.x); ok && w < w1; w += 32) {
      const int* p = fl.done + fl.widx[w];
      unsigned it = 0;
      while (ld_acquire_gpu(p) < target) {
        if ((++it & 31u) == 0) {
          if (ld_acquire_gpu(fl.status) != 0) { ok = false; break; }
          if (global_ns() - t0 > fl.wait_ns) { atomicExch(fl.status, 1); ok = false; break; }
        }
      }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (threadIdx.x == 0) s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Block-wide: publish that band b has finished `value` steps.
__device__ __forceinline__ void flow_publish(const Flow& fl, unsigned b, int value) {
  __syncthreads();
  if (threadIdx.x == 0 && int(b) != fl.silent) st_release_gpu(fl.done + b, value);
}

// Sampling instants of a window (Eq. 42): every dW-th step from the first
// sampled step s0 on; s0 = 0 for a window of the consecutive-window scheme,
// s0 = T - |W| for a full-time run of T steps (Sec. 4.2.3).  dW = 0: never.
__host__ __device__ __forceinline__ bool sampled_step(int step, int s0, int dW) {
  return dW > 0 && step >= s0 && (step - s0) % dW == 0;
}

// Step the coordinates of a node forward by kFlowBlock indices.
__device__ __forceinline__ void flow_advance(const Geo& g, int& x, int& y, int& z) {
  x += kFlowBlock;
  while (x >= g.nx) {
    x -= g.nx;
    if (++y == g.ny) { y = 0; ++z; }
  }
}

template <class L>
__device__ __forceinline__ bool flow_is_face(const Geo& g, int x, int y, int z) {
  return x == 0 || x == g.nx - 1 || y == 0 || y == g.ny - 1 || (L::D == 3 && (z == 0 || z == g.nz - 1));
}

__device__ __forceinline__ void flow_coords(const Geo& g, unsigned i, int& x, int& y, int& z) {
  x = int(i % unsigned(g.nx));
  y = int((i / unsigned(g.nx)) % unsigned(g.ny));
  z = int(i / g.sz);
}

// Face nodes go through out-of-line calls: inlined, their table gathers add
// some 20 registers to the whole loop nest, which then holds fewer bands per
// SM; only a handful of threads per band take them.
template <class L, class R>
__device__ __noinline__ void fwd_face_node(const FwdArgs<R>& A, const FwdStep<R>& P, unsigned kf, R& bj, R& bm) {
  const unsigned i = A.ft.idx[kf];
  int x, y, z;
  flow_coords(A.geo, i, x, y, z);
  if (P.mom) forward_node<L, R, true, true, true>(A, P, x, y, z, i, kf, bj, bm);
  else forward_node<L, R, true, true, false>(A, P, x, y, z, i, kf, bj, bm);
}

template <class L, class R>
__device__ __noinline__ void adj_face_node(const AdjArgs<R>& A, const AdjStep<R>& P, unsigned kf) {
  const unsigned i = A.ft.idx[kf];
  int x, y, z;
  flow_coords(A.geo, i, x, y, z);
  adjoint_node<L, R, true, true>(A, P, x, y, z, i, kf);
}

// Forward steps step0 .. step0+nsteps-1 of a window (or of a recompute when
// sample_every == 0: nothing is sampled).
template <class L, class R>
__global__ void __launch_bounds__(kFlowBlock, sizeof(R) == 4 ? kFlowMinBlocks : 1)
    fwd_flow_kernel(FwdArgs<R> A, Chain<R> ch, Flow fl, int nsteps, int step0, int sample_every, int sample_from) {
  const Geo& g = A.geo;
  const unsigned b = blockIdx.x;
  const unsigned i0 = fl.band[b], i1 = fl.band[b + 1], f0 = fl.fband[b], f1 = fl.fband[b + 1];
  int x0 = 0, y0 = 0, z0 = 0;
  if (i0 + threadIdx.x < i1) flow_coords(g, i0 + threadIdx.x, x0, y0, z0);
#pragma unroll 1
  for (int k = 0; k < nsteps; ++k) {
    if (k > 0 && !flow_wait(fl, b, k)) break;
    // A.mom: moment checkpoint of the launch's last output
    const FwdStep<R> P{ch.src(k), ch.dst(k), sampled_step(step0 + k, sample_from, sample_every),
                       k == nsteps - 1 ? A.mom : nullptr};
    R bj = 0, bm = 0;
    int x = x0, y = y0, z = z0;
#pragma unroll 1
    for (unsigned i = i0 + threadIdx.x; i < i1; i += kFlowBlock) {
      if (!flow_is_face<L>(g, x, y, z)) {
        if (P.mom) forward_node<L, R, false, true, true>(A, P, x, y, z, i, 0u, bj, bm);
        else forward_node<L, R, false, true, false>(A, P, x, y, z, i, 0u, bj, bm);
      }
      flow_advance(g, x, y, z);
    }
#pragma unroll 1
    for (unsigned kf = f0 + threadIdx.x; kf < f1; kf += kFlowBlock) fwd_face_node<L, R>(A, P, kf, bj, bm);
    if (P.sample) {   // uniform across the block
      block_sum2<R, kFlowBlock>(bj, bm);
      sample_commit(double(bj), double(bm), fl.blk, b);
    }
    flow_publish(fl, b, k + 1);
  }
}

// Adjoint steps of one segment, from its last step back to its first.
// Step k of the launch is window step step0 + j with j = nsteps-1-k: it reads
// p^{n-1} from pprev.src-style addressing of the segment (slot j), b^{n+1}
// from the previous step's output (k = 0: bnext0, or nothing when terminal),
// and writes ping-pong between o0 and o1.
template <class R>
struct AdjChain {
  const R* p0;          // segment slot 0
  const R* p1;          // segment slot 1; slot j >= 1 at p1 + (j-1) stride
  long long stride;
  const R* bnext0;      // b^{n+1} of the launch's first step (nullptr: terminal)
  R* o0;
  R* o1;
};

template <class L, class R>
__global__ void __launch_bounds__(kFlowBlock, sizeof(R) == 4 ? kFlowMinBlocks : 1)
    adj_flow_kernel(AdjArgs<R> A, AdjChain<R> ch, Flow fl, int nsteps, int step0, int sample_every, int sample_from) {
  const Geo& g = A.geo;
  const unsigned b = blockIdx.x;
  const unsigned i0 = fl.band[b], i1 = fl.band[b + 1], f0 = fl.fband[b], f1 = fl.fband[b + 1];
  int x0 = 0, y0 = 0, z0 = 0;
  if (i0 + threadIdx.x < i1) flow_coords(g, i0 + threadIdx.x, x0, y0, z0);
#pragma unroll 1
  for (int k = 0; k < nsteps; ++k) {
    if (k > 0 && !flow_wait(fl, b, k)) break;
    const int j = nsteps - 1 - k;
    const AdjStep<R> P{k == 0 ? ch.bnext0 : ((k & 1) ? ch.o0 : ch.o1),
                       j == 0 ? ch.p0 : ch.p1 + (long long)(j - 1) * ch.stride,
                       (k & 1) ? ch.o1 : ch.o0,
                       sampled_step(step0 + j, sample_from, sample_every),
                       k == 0 && ch.bnext0 == nullptr};
    int x = x0, y = y0, z = z0;
#pragma unroll 1
    for (unsigned i = i0 + threadIdx.x; i < i1; i += kFlowBlock) {
      if (!flow_is_face<L>(g, x, y, z)) adjoint_node<L, R, false, true>(A, P, x, y, z, i, 0u);
      flow_advance(g, x, y, z);
    }
#pragma unroll 1
    for (unsigned kf = f0 + threadIdx.x; kf < f1; kf += kFlowBlock) adj_face_node<L, R>(A, P, kf);
    flow_publish(fl, b, k + 1);
  }
}

}  // namespace lbm
