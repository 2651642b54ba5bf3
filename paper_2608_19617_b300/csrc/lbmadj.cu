// Host side of the C ABI declared in include/lbmadj.h: configuration checks,
// workspace carving, the window / adjoint drivers and their launches.
//
// The forward window runs |W| fused collide-stream launches, copying (or
// 16-bit encoding) the carried field into checkpoint slot s before step
// n0 + s K.  The adjoint walks the segments backward: it restores segment s
// from its checkpoint, recomputes its K-1 later states into the segment
// buffer with the same forward kernel (bitwise the same trajectory for
// native checkpoints), then runs K adjoint launches from the last state to
// the first.  The design sensitivity of every adjoint step is added into a
// per-node FP64 (sum, compensation) pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "lbmadj.h"
#include "filter.cuh"
#include "kernels.cuh"

namespace {

thread_local std::string g_last_error;

lbm_status fail(lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess) return fail(LBM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

#define LBM_TRY(expr)              \
  do {                             \
    lbm_status s_ = (expr);        \
    if (s_ != LBM_OK) return s_;   \
  } while (0)

constexpr size_t kAlign = 256;
// Sampled steps whose block partials wait in the ring before a fold into the
// FP64 window sums.
constexpr int kRingSlots = 32;
size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

template <class L>
unsigned unknown_mask(const lbm_config& c, int x, int y, int z) {
  unsigned m = 0;
  for (int a = 0; a < L::Q; ++a) {
    const int X = x - L::cx(a), Y = y - L::cy(a), Z = z - L::cz(a);
    bool out = false;
    if (!c.periodic[0] && (X < 0 || X >= c.nx)) out = true;
    if (!c.periodic[1] && (Y < 0 || Y >= c.ny)) out = true;
    if (!c.periodic[2] && (Z < 0 || Z >= c.nz)) out = true;
    if (out) m |= 1u << a;
  }
  return m;
}

template <class L>
unsigned mask_with_cx(int sx) {
  unsigned m = 0;
  for (int a = 0; a < L::Q; ++a)
    if (L::cx(a) == sx) m |= 1u << a;
  return m;
}

// Layout of the caller's workspace.
struct Layout {
  size_t f[2], b[2], g, gamma, wobj, cls, uin, gacc, gpart, gout, stage, ckpt, ckpt_slot, seg, seg_slots,
      partials, ring, acc, flags, xraw, xfilt, wfilt, slice_j, slice_c,
      total;
  int nblocks_fwd, nblocks_1d, nslots;
  int rgx;                    // blocks of kBlock along a row (x = 0 .. nx-1)
  int iy, iz;                 // inner rows along y and z (forward row kernel's grid)
  int nfr;                    // face rows (forward face-row kernel's grid)
  size_t seg_sets;            // 2 when recompute and adjoint are pipelined
  bool stage_in_seg;
};

lbm_status validate_config(const lbm_config& c) {
  if (c.lattice != LBM_D2Q9 && c.lattice != LBM_D3Q19) return fail(LBM_ERR_ARG, "lattice must be 9 or 19");
  if (c.nx < 1 || c.ny < 1 || c.nz < 1) return fail(LBM_ERR_ARG, "lattice sizes must be >= 1");
  // D2Q9 with nz > 1 is a batch of nz independent 2D lattices (c_z = 0).
  if (c.ny > 65535 || c.nz > 65535) return fail(LBM_ERR_ARG, "ny and nz must be <= 65535");
  if (double(c.nx) * c.ny * c.nz * c.lattice >= 2147483647.0)
    return fail(LBM_ERR_ARG, "Q * nx * ny * nz must stay below 2^31 (32-bit element indices)");
  const int dims[3] = {c.nx, c.ny, c.nz};
  for (int k = 0; k < 3; ++k) {
    if (c.periodic[k] != 0 && c.periodic[k] != 1) return fail(LBM_ERR_ARG, "periodic flags must be 0 or 1");
    const bool used = k < 2 || c.lattice == LBM_D3Q19;
    if (used && !c.periodic[k] && dims[k] < 3) return fail(LBM_ERR_ARG, "a bounded axis needs >= 3 nodes");
  }
  if (c.precision != LBM_FP32 && c.precision != LBM_FP64) return fail(LBM_ERR_ARG, "precision must be FP32 or FP64");
  if (!(c.tau > 0.5) || !std::isfinite(c.tau)) return fail(LBM_ERR_ARG, "tau must be > 0.5");
  if (!(c.cs_smag >= 0.0) || !std::isfinite(c.cs_smag)) return fail(LBM_ERR_ARG, "cs_smag must be >= 0");
  if (!(c.q_interp > 0.0) || !std::isfinite(c.q_interp)) return fail(LBM_ERR_ARG, "q_interp must be > 0");
  if (!(c.g_max >= 0.0 && c.g_max <= 1.0)) return fail(LBM_ERR_ARG, "g_max must be in [0, 1]");
  if (!(c.rho_out > 0.0) || !std::isfinite(c.rho_out)) return fail(LBM_ERR_ARG, "rho_out must be > 0");
  if (c.objective_kind < 0 || c.objective_kind > 3) return fail(LBM_ERR_ARG, "objective_kind out of range");
  if (c.monitor_kind < 0 || c.monitor_kind > 1) return fail(LBM_ERR_ARG, "monitor_kind out of range");
  if (c.monitor_kind == LBM_MON_DRAG && !(c.monitor_u > 0.0 && c.monitor_l > 0.0))
    return fail(LBM_ERR_ARG, "monitor_u and monitor_l must be > 0 for the drag monitor");
  if (c.window_len < 1) return fail(LBM_ERR_ARG, "window_len must be >= 1");
  if (c.sample_every < 1 || c.window_len % c.sample_every) return fail(LBM_ERR_ARG, "sample_every must divide window_len");
  if (c.ckpt_every < 1 || c.window_len % c.ckpt_every) return fail(LBM_ERR_ARG, "ckpt_every must divide window_len");
  if (c.ckpt_format < 0 || c.ckpt_format > 3) return fail(LBM_ERR_ARG, "ckpt_format out of range");
  if ((c.ckpt_format == LBM_CKPT_FP16 || c.ckpt_format == LBM_CKPT_BF16) && c.precision != LBM_FP32)
    return fail(LBM_ERR_ARG, "16-bit checkpoints need the FP32 solver");
  if (!(c.conv_tol >= 0.0)) return fail(LBM_ERR_ARG, "conv_tol must be >= 0");
  if (c.pipeline != 0 && c.pipeline != 1) return fail(LBM_ERR_ARG, "pipeline must be 0 or 1");
  for (const int32_t* bx : {c.obj_box, c.design_box})
    for (int k = 0; k < 3; ++k)
      if (bx[2 * k] < 0 || bx[2 * k] > bx[2 * k + 1] || bx[2 * k + 1] > dims[k])
        return fail(LBM_ERR_ARG, "box bounds must satisfy 0 <= lo <= hi <= size");
  return LBM_OK;
}

Layout make_layout(const lbm_config& c) {
  Layout L{};
  const size_t n = size_t(c.nx) * c.ny * c.nz;
  const int q = c.lattice;
  const int d = c.lattice == LBM_D2Q9 ? 2 : 3;
  const size_t rs = c.precision == LBM_FP64 ? 8 : 4;
  const size_t lat = align_up(size_t(q) * n * rs);
  // Whole rows along x (kernels.cuh, row geometry): the forward step runs the
  // inner rows and the face rows in two kernels, the adjoint step all rows in
  // one; one sample slot per block of a row.
  const bool d2 = c.lattice == LBM_D2Q9;
  L.rgx = (c.nx + lbm::kBlock - 1) / lbm::kBlock;
  L.iy = c.ny > 2 ? c.ny - 2 : 0;
  L.iz = d2 ? c.nz : (c.nz > 2 ? c.nz - 2 : 0);
  L.nfr = (c.ny >= 2 ? 2 : 1) * c.nz + (d2 ? 0 : (c.nz >= 2 ? 2 : 1) * L.iy);
  L.nblocks_fwd = L.rgx * c.ny * c.nz;
  L.nblocks_1d = int((n + lbm::kBlock - 1) / lbm::kBlock);
  L.nslots = c.window_len / c.ckpt_every;
  const bool native = c.ckpt_format == LBM_CKPT_NATIVE;
  const bool moment = c.ckpt_format == LBM_CKPT_MOMENT;
  // moment checkpoints: slot 0 (the window's start field) native, slots 1.. the coefficient planes
  L.ckpt_slot = native   ? lat
                : moment ? align_up(size_t(d == 2 ? 7 : 11) * n * rs)
                         : align_up(size_t(q) * n * 2) + align_up(size_t(d + 1) * n * 4) +
                               align_up(size_t(L.nblocks_1d) * 4);
  L.seg_slots = native ? size_t(c.ckpt_every - 1) : size_t(c.ckpt_every);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += align_up(bytes); return o; };
  L.f[0] = take(lat);
  L.f[1] = take(lat);
  L.b[0] = take(lat);
  L.b[1] = take(lat);
  L.g = take(n * rs);
  L.gamma = take(n * 4);
  L.wobj = take(n * 4);
  L.cls = take(n);
  L.uin = take(size_t(c.ny) * c.nz * 4);
  L.gacc = take(n * 16);
  L.gpart = take(n * rs);
  L.gout = take(n * 8);
  L.partials = take(size_t(L.nblocks_fwd) * 32);
  L.ring = take(size_t(kRingSlots) * L.nblocks_fwd * 2 * rs);
  L.xraw = take(n * 4);       // raw design variables (filtered designs)
  L.slice_j = take(size_t(c.nz) * 16);   // per-slice window means (J, M) of a D2Q9 batch
  L.slice_c = take(size_t(c.nz) * 8);    // per-slice constant of a pressure objective
  L.xfilt = take(n * 8);      // filtered field x~
  L.wfilt = take(n * 8);      // filter normalisation W_i
  L.acc = take(sizeof(lbm::WindowAcc));
  L.flags = take(16);
  L.ckpt = take(moment ? lat + L.ckpt_slot * size_t(L.nslots - 1) : L.ckpt_slot * L.nslots);
  L.seg_sets = c.pipeline ? 2 : 1;
  L.seg = take(lat * L.seg_slots * L.seg_sets);
  const size_t stage_bytes = size_t(q) * n * 8;
  L.stage_in_seg = lat * L.seg_slots * L.seg_sets >= stage_bytes;
  L.stage = L.stage_in_seg ? L.seg : take(stage_bytes);
  L.total = off;
  return L;
}

struct Pending {
  int phase;
  cudaEvent_t a, b;
  int64_t launches, lus;
};

}  // namespace

// Polymorphic per-(lattice, precision) implementation.
struct Impl {
  virtual ~Impl() = default;
  // sample: 0, or 1 + the ring slot that takes the step's block partials
  virtual void fwd(const void* src, void* dst, int sample, void* mom = nullptr) = 0;
  virtual void fold(int count) = 0;   // add count ring slots into the FP64 window sums
  virtual void adj(const void* bnext, const void* pprev, void* bout, int sample) = 0;
  virtual void pull(const void* b, void* out) = 0;
  virtual void set_design() = 0;
  virtual void grad() = 0;
  virtual void fold() = 0;
  virtual void unshift(const void* src) = 0;
  virtual void shift(void* dst) = 0;
  virtual void to_double(const void* src) = 0;
  virtual void encode(const void* p, int slot) = 0;
  virtual void decode(int slot, void* p) = 0;
  // Field of checkpoint s of the last window (decoded if need be), in this context's precision.
  virtual const void* checkpoint_field(int s) = 0;
  // dst (this context's precision) <- src field in precision rs_src.
  virtual void import_field(const void* src, size_t rs_src, void* dst) = 0;
};

// A captured CUDA graph with the timing events its replays record.
struct GraphRec {
  cudaGraphExec_t exec = nullptr;
  std::vector<Pending> events;
};

struct lbm_ctx {
  lbm_config cfg;
  Layout lay;
  char* ws;
  cudaStream_t stream;        // the caller's stream: everything runs in its order
  cudaStream_t ls = nullptr;  // stream launches go to (the capture stream while capturing)
  cudaStream_t cap = nullptr; // private stream used only to capture graphs
  cudaStream_t side = nullptr;            // forward face-row kernels run here, forked from ls and joined back
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  // Pipelined adjoint: the recompute of the next segment runs on rec (with its
  // own side stream) while the adjoint of the current segment runs on ls.
  cudaStream_t rec = nullptr, rec_side = nullptr;
  cudaEvent_t rec_fork = nullptr, rec_join = nullptr, start_ev = nullptr, rec_done[2] = {}, adj_done[2] = {};
  cudaStream_t side_cur = nullptr;        // side stream / events of the stream now in ls
  cudaEvent_t fork_cur = nullptr, join_cur = nullptr;
  bool use_graphs = true;
  bool use_pdl = true;        // programmatic dependent launch of the step kernels
  lbm::ZgRows zg{};           // x-face rows next to zero-gradient outlet nodes
  int64_t kernels = 0;        // kernel launches enqueued so far
  int64_t kernels_window = 0, kernels_adjoint = 0;   // per window / per adjoint sweep, as last enqueued
  lbm_ctx* along = nullptr;   // lbm_step_window_along: the context whose checkpoints start each segment
  bool capturing = false;
  std::vector<Pending>* sink = nullptr;   // where end() files events while capturing
  GraphRec gwin[2][2];        // forward window graphs by [start parity][timing]
  GraphRec gadj[2];           // adjoint sweep graphs by [timing]
  lbm::Geo geo;
  size_t n, q, rs;
  int cur;                    // index of the buffer holding the carried field
  int64_t steps = 0, windows = 0;
  bool window_valid = false, grad_valid = false;
  double last_j = 0, last_m = 0, ratio = INFINITY;
  int converged = 0, nwin_for_ratio = 0;
  int bout_last = 0;          // adjoint buffer holding b^{n0}
  double jconst = 0;
  int sample_from = 0;        // first sampled step of a window (lbm_set_sample_start)
  bool timing = false;
  int64_t timing_failures = 0;
  bool filtered = false;      // design set through lbm_set_design_filtered
  lbm::FilterGeo fgeo{};
  lbm_timing tm{};
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  std::unique_ptr<Impl> impl;

  template <class T = void>
  T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  void* lattice(int k) const { return ws + lay.f[k]; }
  void* adjbuf(int k) const { return ws + lay.b[k]; }
  void* seg_slot(int s, int j) const {   // state p^{n0 + sK - 1 + j}
    const size_t lat = align_up(q * n * rs);
    const size_t set = lay.seg_sets == 2 ? size_t(s & 1) : 0;   // pipelined: segments alternate buffers
    char* base = ws + lay.seg + set * lat * lay.seg_slots;
    if (cfg.ckpt_format == LBM_CKPT_NATIVE) {
      if (j == 0) return ws + lay.ckpt + lay.ckpt_slot * s;
      return base + lat * (j - 1);
    }
    if (cfg.ckpt_format == LBM_CKPT_MOMENT && s == 0 && j == 0) return ws + lay.ckpt;   // native slot 0
    return base + lat * j;
  }
  void* ckpt_mom(int s) const {   // moment checkpoint s >= 1
    return ws + lay.ckpt + align_up(q * n * rs) + lay.ckpt_slot * size_t(s - 1);
  }

  cudaEvent_t event() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  // Record a timing event; inside a capture it becomes an external event
  // record node, which stays readable by cudaEventElapsedTime after replays.
  void record(cudaEvent_t e) {
    if (capturing) cudaEventRecordWithFlags(e, ls, cudaEventRecordExternal);
    else cudaEventRecord(e, ls);
  }
  // Phase bracket: call begin() before and end() after a run of launches.
  cudaEvent_t begin() {
    if (!timing) return nullptr;
    cudaEvent_t e = event();
    if (e) record(e);
    return e;
  }
  void end(cudaEvent_t a, int phase, int64_t launches, int64_t lus) {
    if (!timing || !a) return;
    cudaEvent_t b = event();
    if (!b) return;
    record(b);
    (capturing ? *sink : pending).push_back({phase, a, b, launches, lus});
  }
  // Add the elapsed times of a replayed graph's events (after a sync).
  void harvest_graph(const GraphRec& g) {
    for (const auto& p : g.events) add_pair(p);
  }
  void drop_graph(GraphRec& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    for (auto& p : g.events) { pool.push_back(p.a); pool.push_back(p.b); }
    g.events.clear();
  }
  // Add one event pair's elapsed time; a pair that cannot be read is
  // counted in timing_failures and its error is cleared so that it does not
  // surface as a later call's cudaGetLastError.
  void add_pair(const Pending& p) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      tm.ms[p.phase] += ms;
      tm.launches[p.phase] += p.launches;
      tm.lattice_updates[p.phase] += p.lus;
    } else {
      cudaGetLastError();
      timing_failures += 1;
    }
  }
  void harvest() {   // after a stream synchronisation
    for (auto& p : pending) {
      add_pair(p);
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  ~lbm_ctx() {
    for (auto& row : gwin) for (auto& g : row) drop_graph(g);
    for (auto& g : gadj) drop_graph(g);
    for (auto& p : pending) { pool.push_back(p.a); pool.push_back(p.b); }
    for (auto e : pool) cudaEventDestroy(e);
    if (cap) cudaStreamDestroy(cap);
    if (rec) cudaStreamDestroy(rec);
    if (side) cudaStreamDestroy(side);
    if (rec_side) cudaStreamDestroy(rec_side);
    for (cudaEvent_t e : {fork_ev, join_ev, rec_fork, rec_join, start_ev, rec_done[0], rec_done[1], adj_done[0], adj_done[1]})
      if (e) cudaEventDestroy(e);
  }
};

namespace {

template <class L, class R>
struct ImplT final : Impl {
  lbm_ctx* c;
  explicit ImplT(lbm_ctx* ctx) : c(ctx) {}

  dim3 grid() const { return dim3((c->cfg.nx + lbm::kBlock - 1) / lbm::kBlock, c->cfg.ny, c->cfg.nz); }
  int flat_blocks() const {
    long long b = (long long)(c->n * c->q + 255) / 256;
    return int(b < 148 * 32 ? b : 148 * 32);
  }
  dim3 sgrid() const { return dim3(c->lay.rgx, c->cfg.ny, c->cfg.nz); }
  dim3 rgrid() const { return dim3(c->lay.rgx, c->lay.iy, c->lay.iz); }
  dim3 fgrid() const { return dim3(c->lay.rgx, c->lay.nfr); }
  // Inner-row kernel on the launch stream, face-row kernel on the side
  // stream, forked and joined with events so that both run concurrently (and
  // become parallel branches when captured into a graph).
  template <class IK, class FK>
  void fork_join(IK inner, FK face) {
    cudaEventRecord(c->fork_cur, c->ls);
    cudaStreamWaitEvent(c->side_cur, c->fork_cur, 0);
    face(c->side_cur);
    c->kernels += 1;
    if (c->lay.iy > 0 && c->lay.iz > 0) {
      inner(c->ls);
      c->kernels += 1;
    }
    cudaEventRecord(c->join_cur, c->side_cur);
    cudaStreamWaitEvent(c->ls, c->join_cur, 0);
  }
  // Step kernels: optionally with programmatic stream serialization, so that a
  // launch overlaps the tail of its predecessor (the kernel waits in
  // pdl_enter before touching data).
  template <class... Args>
  void launch(void (*kernel)(Args...), dim3 grid, cudaStream_t st, Args... args) {
    launch_b(kernel, grid, lbm::kBlock, st, args...);
  }
  template <class... Args>
  void launch_b(void (*kernel)(Args...), dim3 grid, int block, cudaStream_t st, Args... args) {
    if (c->use_pdl) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = grid;
      cfg.blockDim = dim3(block);
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, kernel, args...);
    } else {
      kernel<<<grid, block, 0, st>>>(args...);
    }
  }
  lbm::Phys<R> phys() const { return {R(c->cfg.tau), R(c->cfg.cs_smag * c->cfg.cs_smag), R(c->cfg.rho_out)}; }
  lbm::Obj<R> obj() const {
    lbm::Obj<R> o{};
    const lbm_config& k = c->cfg;
    o.kind = k.objective_kind;
    o.mon = k.monitor_kind;
    for (int i = 0; i < 3; ++i) o.uref[i] = R(k.objective_uref[i]);
    for (int i = 0; i < 6; ++i) o.box[i] = k.obj_box[i];
    o.ws = R(double(k.sample_every) / double(k.window_len - c->sample_from));   // 1 / samples
    return o;
  }

  lbm::FwdArgs<R> fwd_args(const void* src, void* dst, int sample, void* mom = nullptr) const {
    lbm::FwdArgs<R> A;
    A.mom = static_cast<R*>(mom);
    A.src = static_cast<const R*>(src);
    A.dst = static_cast<R*>(dst);
    A.gfield = c->template at<R>(c->lay.g);
    A.cls = c->template at<uint8_t>(c->lay.cls);
    A.uin = c->template at<float>(c->lay.uin);
    A.wobj = c->template at<float>(c->lay.wobj);
    A.geo = c->geo;
    A.ph = phys();
    A.obj = obj();
    A.sample = sample;
    A.ring = c->template at<R>(c->lay.ring);
    A.nblk = unsigned(c->lay.nblocks_fwd);
    A.blk = nullptr;
    A.nonfinite = c->template at<int>(c->lay.flags);
    return A;
  }
  lbm::AdjArgs<R> adj_args(const void* bnext, const void* pprev, void* bout, int sample) const {
    lbm::AdjArgs<R> A;
    A.bnext = static_cast<const R*>(bnext);
    A.pprev = static_cast<const R*>(pprev);
    A.bout = static_cast<R*>(bout);
    A.gfield = c->template at<R>(c->lay.g);
    A.cls = c->template at<uint8_t>(c->lay.cls);
    A.uin = c->template at<float>(c->lay.uin);
    A.wobj = c->template at<float>(c->lay.wobj);
    A.gpart = c->template at<R>(c->lay.gpart);
    A.geo = c->geo;
    A.ph = phys();
    A.obj = obj();
    A.sample = sample;
    A.terminal = bnext == nullptr;
    for (int i = 0; i < 6; ++i) A.dbox[i] = c->cfg.design_box[i];
    A.zg = c->zg;
    return A;
  }
  // One forward step: the inner rows and the face rows concurrently (a
  // moment-checkpoint step runs its own instantiation, MOM).
  void fwd(const void* src, void* dst, int sample, void* mom) override {
    const lbm::FwdArgs<R> A = fwd_args(src, dst, sample, mom);
    fork_join(
        [&](cudaStream_t st) {
          if (mom) launch(lbm::fwd_row_kernel<L, R, true>, rgrid(), st, A);
          else launch(lbm::fwd_row_kernel<L, R, false>, rgrid(), st, A);
        },
        [&](cudaStream_t st) {
          if (mom) launch(lbm::fwd_facerow_kernel<L, R, true>, fgrid(), st, A);
          else launch(lbm::fwd_facerow_kernel<L, R, false>, fgrid(), st, A);
        });
  }

  // One adjoint step: one kernel over every row; a lattice without periodic
  // axes runs the instantiation whose link selects carry no wrap arithmetic.
  void adj(const void* bnext, const void* pprev, void* bout, int sample) override {
    const lbm::AdjArgs<R> A = adj_args(bnext, pprev, bout, sample);
    const bool per = c->cfg.periodic[0] || c->cfg.periodic[1] || c->cfg.periodic[2];
    if (per) launch(lbm::adj_step_kernel<L, R, true>, sgrid(), c->ls, A);
    else launch(lbm::adj_step_kernel<L, R, false>, sgrid(), c->ls, A);
    c->kernels += 1;
  }

  const void* checkpoint_field(int s) override {
    const int fmt = c->cfg.ckpt_format;
    if (fmt == LBM_CKPT_NATIVE || (fmt == LBM_CKPT_MOMENT && s == 0)) return c->seg_slot(s, 0);
    decode(s, c->seg_slot(s, 0));
    return c->seg_slot(s, 0);
  }
  void import_field(const void* src, size_t rs_src, void* dst) override {
    const long long total = (long long)(c->n * c->q);
    c->kernels += 1;
    if (rs_src == 4)
      lbm::convert_kernel<float, R><<<flat_blocks(), 256, 0, c->ls>>>(static_cast<const float*>(src),
                                                                       static_cast<R*>(dst), total);
    else
      lbm::convert_kernel<double, R><<<flat_blocks(), 256, 0, c->ls>>>(static_cast<const double*>(src),
                                                                        static_cast<R*>(dst), total);
  }

  void fold(int count) override {
    const int nb = int(std::min<long long>((2LL * c->lay.nblocks_fwd + 255) / 256, 148 * 8));
    c->kernels += 1;
    lbm::sample_fold_kernel<R><<<nb, 256, 0, c->ls>>>(c->template at<R>(c->lay.ring), count,
                                                      unsigned(c->lay.nblocks_fwd), c->template at<double>(c->lay.partials));
  }
  void pull(const void* b, void* out) override {
    lbm::adj_pull_kernel<L, R><<<grid(), lbm::kBlock, 0, c->ls>>>(
        static_cast<const R*>(b), c->template at<uint8_t>(c->lay.cls), static_cast<R*>(out), c->geo);
  }
  void set_design() override {
    lbm::design_kernel<R><<<flat_blocks(), 256, 0, c->ls>>>(
        c->template at<float>(c->lay.gamma), c->template at<R>(c->lay.g), (long long)c->n, c->cfg.q_interp, c->cfg.g_max, c->template at<int>(c->lay.flags) + 1);
  }
  void fold() override {
    const int* d = c->cfg.design_box;
    const long long cells = (long long)(d[1] - d[0]) * (d[3] - d[2]) * (d[5] - d[4]);
    if (cells == 0) return;
    const long long blocks = (cells + 255) / 256;
    c->kernels += 1;
    lbm::grad_fold_kernel<R><<<int(blocks < 148 * 32 ? blocks : 148 * 32), 256, 0, c->ls>>>(
        c->template at<R>(c->lay.gpart), c->template at<double2>(c->lay.gacc), c->geo, d[0], d[1], d[2], d[3],
        d[4], d[5]);
  }
  void grad() override {
    const int* d = c->cfg.design_box;
    lbm::gradient_kernel<<<flat_blocks(), 256, 0, c->ls>>>(
        c->template at<double2>(c->lay.gacc), c->template at<float>(c->lay.gamma), c->template at<double>(c->lay.gout),
        c->geo, d[0], d[1], d[2], d[3], d[4], d[5], c->cfg.q_interp, c->cfg.g_max);
  }
  void unshift(const void* src) override {
    lbm::unshift_kernel<L, R><<<flat_blocks(), 256, 0, c->ls>>>(static_cast<const R*>(src),
                                                                      c->template at<double>(c->lay.stage),
                                                                      (long long)c->n);
  }
  void shift(void* dst) override {
    lbm::shift_kernel<L, R><<<flat_blocks(), 256, 0, c->ls>>>(c->template at<double>(c->lay.stage),
                                                                    static_cast<R*>(dst), (long long)c->n,
                                                                    c->template at<int>(c->lay.flags) + 1);
  }
  void to_double(const void* src) override {
    lbm::copy_double_kernel<R><<<flat_blocks(), 256, 0, c->ls>>>(
        static_cast<const R*>(src), c->template at<double>(c->lay.stage), (long long)(c->n * c->q));
  }
  template <class T>
  void encode_t(const void* p, int slot) {
    char* base = c->ws + c->lay.ckpt + c->lay.ckpt_slot * slot;
    T* dev = reinterpret_cast<T*>(base);
    float* mom = reinterpret_cast<float*>(base + align_up(c->q * c->n * 2));
    int* ex = reinterpret_cast<int*>(base + align_up(c->q * c->n * 2) + align_up((L::D + 1) * c->n * 4));
    c->kernels += 1;
    lbm::ckpt_encode_kernel<L, T><<<c->lay.nblocks_1d, lbm::kBlock, 0, c->ls>>>(
        static_cast<const float*>(p), dev, mom, ex, (long long)c->n);
  }
  template <class T>
  void decode_t(int slot, void* p) {
    char* base = c->ws + c->lay.ckpt + c->lay.ckpt_slot * slot;
    T* dev = reinterpret_cast<T*>(base);
    float* mom = reinterpret_cast<float*>(base + align_up(c->q * c->n * 2));
    int* ex = reinterpret_cast<int*>(base + align_up(c->q * c->n * 2) + align_up((L::D + 1) * c->n * 4));
    c->kernels += 1;
    lbm::ckpt_decode_kernel<L, T><<<c->lay.nblocks_1d, lbm::kBlock, 0, c->ls>>>(
        dev, mom, ex, static_cast<float*>(p), (long long)c->n);
  }
  void encode(const void* p, int slot) override {
    if constexpr (sizeof(R) == 4) {
      if (c->cfg.ckpt_format == LBM_CKPT_FP16) encode_t<__half>(p, slot); else encode_t<__nv_bfloat16>(p, slot);
    }
  }
  void decode(int slot, void* p) override {
    if (c->cfg.ckpt_format == LBM_CKPT_MOMENT) {
      c->kernels += 1;
      lbm::mom_decode_kernel<L, R><<<c->lay.nblocks_1d, lbm::kBlock, 0, c->ls>>>(
          static_cast<const R*>(c->ckpt_mom(slot)), static_cast<R*>(p), unsigned(c->n));
      return;
    }
    if constexpr (sizeof(R) == 4) {
      if (c->cfg.ckpt_format == LBM_CKPT_FP16) decode_t<__half>(slot, p); else decode_t<__nv_bfloat16>(slot, p);
    }
  }
};

template <class L>
lbm_status validate_classes(const lbm_config& c, const uint8_t* cls) {
  const unsigned in_mask = mask_with_cx<L>(1);
  for (int z = 0; z < c.nz; ++z)
    for (int y = 0; y < c.ny; ++y)
      for (int x = 0; x < c.nx; ++x) {
        const size_t i = size_t(x) + size_t(c.nx) * (size_t(y) + size_t(c.ny) * z);
        const uint8_t k = cls[i];
        if (k > LBM_OUTLET_ZEROGRAD) return fail(LBM_ERR_ARG, "node %zu: class %d out of range", i, int(k));
        const bool face = x == 0 || x == c.nx - 1 || y == 0 || y == c.ny - 1 ||
                          (L::D == 3 && (z == 0 || z == c.nz - 1));
        if (!face) {
          if (k != LBM_FLUID) return fail(LBM_ERR_ARG, "node %zu: interior nodes must be FLUID", i);
          continue;
        }
        const unsigned unk = unknown_mask<L>(c, x, y, z);
        switch (k) {
          case LBM_FLUID:
            if (unk) return fail(LBM_ERR_ARG, "node %zu: boundary node with unknown populations is FLUID", i);
            break;
          case LBM_WALL: break;
          case LBM_INLET: {
            const unsigned want = L::Q == 9 ? ((1u << 1) | (1u << 5) | (1u << 8)) : in_mask;
            if (x != 0 || unk != want)
              return fail(LBM_ERR_ARG, "node %zu: inlet nodes must lie on the x=0 face away from other faces", i);
            break;
          }
          case LBM_OUTLET_PRESSURE:
            if (L::Q != 9 || x != c.nx - 1 || unk != ((1u << 3) | (1u << 6) | (1u << 7)))
              return fail(LBM_ERR_ARG, "node %zu: pressure outlets are D2Q9 nodes on the x=nx-1 face away from walls", i);
            break;
          case LBM_OUTLET_ZEROGRAD: {
            if (c.periodic[0] || !(x == 0 || x == c.nx - 1))
              return fail(LBM_ERR_ARG, "node %zu: zero-gradient outlets lie on a bounded x face", i);
            const unsigned want = mask_with_cx<L>(x == 0 ? 1 : -1);
            if (unk != want)
              return fail(LBM_ERR_ARG, "node %zu: zero-gradient outlet must not touch another face", i);
            break;
          }
        }
      }
  return LBM_OK;
}

lbm_status check_flags(lbm_ctx* c, int which, lbm_status st, const char* what) {
  int h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c->at<int>(c->lay.flags) + which, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (h) {
    CUDA_TRY(cudaMemsetAsync(c->at<int>(c->lay.flags) + which, 0, sizeof(int), c->stream));
    return fail(st, "%s", what);
  }
  return LBM_OK;
}

// Work of one forward window (Alg. 1 inner loop): checkpoint s before step
// n0 + sK, K fused steps per segment, window-end reduction.  Enqueued on c->ls.
lbm_status enqueue_window(lbm_ctx* c) {
  const lbm_config& k = c->cfg;
  const int K = k.ckpt_every, S = c->lay.nslots;
  const bool native = k.ckpt_format == LBM_CKPT_NATIVE;
  const bool moment = k.ckpt_format == LBM_CKPT_MOMENT;
  const size_t lat_bytes = c->q * c->n * c->rs;
  const int64_t k0 = c->kernels;
  int pending = 0;   // sampled steps waiting in the ring
  for (int s = 0; s < S; ++s) {
    if (c->along) {   // start the segment from the reference context's checkpoint s
      lbm_ctx* r = c->along;
      cudaStream_t rls = r->ls;
      r->ls = c->ls;
      const void* src = r->impl->checkpoint_field(s);
      r->ls = rls;
      c->impl->import_field(src, r->rs, c->lattice(c->cur));
    }
    cudaEvent_t e = c->begin();
    if (native || (moment && s == 0))
      CUDA_TRY(cudaMemcpyAsync(c->seg_slot(s, 0), c->lattice(c->cur), lat_bytes, cudaMemcpyDeviceToDevice, c->ls));
    else if (!moment) c->impl->encode(c->lattice(c->cur), s);
    c->end(e, 3, moment && s > 0 ? 0 : 1, 0);
    // moment checkpoints: the segment's last step also stores checkpoint s + 1
    void* mom = moment && s + 1 < S ? c->ckpt_mom(s + 1) : nullptr;
    e = c->begin();
    for (int j = 0; j < K; ++j) {
      const int step = s * K + j;
      const bool sampled = lbm::sampled_step(step, c->sample_from, k.sample_every);
      c->impl->fwd(c->lattice(c->cur), c->lattice(c->cur ^ 1), sampled ? 1 + pending : 0, j == K - 1 ? mom : nullptr);
      c->cur ^= 1;
      if (sampled && ++pending == kRingSlots) {
        c->impl->fold(pending);
        pending = 0;
      }
    }
    c->end(e, 0, K, int64_t(K) * int64_t(c->n));
  }
  if (pending) c->impl->fold(pending);
  const double mon_scale =
      k.monitor_kind == LBM_MON_DRAG ? 1.0 / (0.5 * k.rho_out * k.monitor_u * k.monitor_u * k.monitor_l) : 0.0;
  const double nsamples = double((k.window_len - c->sample_from) / k.sample_every);
  if (k.lattice == LBM_D2Q9) {
    lbm::slice_end_kernel<<<k.nz, lbm::kEndThreads, 0, c->ls>>>(
        c->at<double>(c->lay.partials), c->lay.rgx * k.ny,
        nsamples, c->at<double>(c->lay.slice_c), mon_scale, k.monitor_kind,
        c->at<double>(c->lay.slice_j));
    c->kernels += 1;
  }
  lbm::window_end_kernel<<<1, lbm::kEndThreads, 0, c->ls>>>(
      c->at<double>(c->lay.partials), c->lay.nblocks_fwd, c->at<lbm::WindowAcc>(c->lay.acc), k.conv_tol,
      c->at<int>(c->lay.flags), nsamples, c->jconst, mon_scale, k.monitor_kind);
  c->kernels += 1;
  c->kernels_window = c->kernels - k0;
  return LBM_OK;
}

// Work of one adjoint sweep (Alg. 2 reverse loop): per segment, restore,
// recompute K-1 states, then K adjoint steps from the last state back.
// Pipelined (cfg.pipeline): segment s-1 is restored and recomputed on the
// rec stream into the other segment buffer while the adjoint of segment s
// runs on ls; events order each recompute after the adjoint that last used
// its buffer and each adjoint after its segment's recompute.
lbm_status enqueue_adjoint(lbm_ctx* c) {
  const lbm_config& k = c->cfg;
  const int K = k.ckpt_every, S = c->lay.nslots;
  const bool native = k.ckpt_format == LBM_CKPT_NATIVE;
  const bool pipe = c->lay.seg_sets == 2;
  const size_t lat = align_up(c->q * c->n * c->rs);
  const int64_t k0 = c->kernels;
  CUDA_TRY(cudaMemsetAsync(c->at(c->lay.gacc), 0, c->n * 16, c->ls));
  CUDA_TRY(cudaMemsetAsync(c->at(c->lay.gpart), 0, c->n * c->rs, c->ls));
  cudaStream_t main = c->ls;
  auto on_rec = [&](bool rec) {   // route launches (and their face-row kernels) to one pipeline stream
    c->ls = rec ? c->rec : main;
    c->side_cur = rec ? c->rec_side : c->side;
    c->fork_cur = rec ? c->rec_fork : c->fork_ev;
    c->join_cur = rec ? c->rec_join : c->join_ev;
  };
  const bool moment = k.ckpt_format == LBM_CKPT_MOMENT;
  auto recompute = [&](int s) {
    cudaEvent_t e = c->begin();
    const bool restore = !native && !(moment && s == 0);   // native slots are read in place
    if (restore) c->impl->decode(s, c->seg_slot(s, 0));
    c->end(e, 3, restore ? 1 : 0, 0);
    e = c->begin();
    for (int j = 1; j < K; ++j) c->impl->fwd(c->seg_slot(s, j - 1), c->seg_slot(s, j), 0);
    c->end(e, 1, K - 1, int64_t(K - 1) * int64_t(c->n));
  };
  if (pipe) {
    cudaEventRecord(c->start_ev, main);
    cudaStreamWaitEvent(c->rec, c->start_ev, 0);
    on_rec(true);
    recompute(S - 1);
    cudaEventRecord(c->rec_done[(S - 1) & 1], c->rec);
    on_rec(false);
  }
  int bo = 0;
  const void* bnext = nullptr;
  for (int s = S - 1; s >= 0; --s) {
    if (!pipe) {
      recompute(s);
    } else {
      if (s >= 1) {
        on_rec(true);
        if (s + 1 <= S - 1) cudaStreamWaitEvent(c->rec, c->adj_done[(s + 1) & 1], 0);
        recompute(s - 1);
        cudaEventRecord(c->rec_done[(s - 1) & 1], c->rec);
        on_rec(false);
      }
      cudaStreamWaitEvent(main, c->rec_done[s & 1], 0);
    }
    cudaEvent_t e = c->begin();
    for (int j = K - 1; j >= 0; --j) {
      const int step = s * K + j;
      c->impl->adj(bnext, c->seg_slot(s, j), c->adjbuf(bo), lbm::sampled_step(step, c->sample_from, k.sample_every));
      bnext = c->adjbuf(bo);
      bo ^= 1;
    }
    c->end(e, 2, K, int64_t(K) * int64_t(c->n));
    c->impl->fold();
    if (pipe) cudaEventRecord(c->adj_done[s & 1], main);
  }
  c->kernels_adjoint = c->kernels - k0;
  return LBM_OK;
}

// Record body() into a CUDA graph on the private capture stream and
// instantiate it.  The caller's stream may be the legacy default stream,
// which cannot be captured; the graph is launched into it afterwards.
lbm_status capture(lbm_ctx* c, GraphRec& G, lbm_status (*body)(lbm_ctx*)) {
  if (!c->cap) CUDA_TRY(cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  const int cur0 = c->cur;
  c->ls = c->cap;
  c->capturing = true;
  c->sink = &G.events;
  cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
  lbm_status st = e == cudaSuccess ? body(c) : LBM_ERR_CUDA;
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(c->cap, &graph);
  c->ls = c->stream;
  c->capturing = false;
  c->sink = nullptr;
  c->cur = cur0;
  if (e != cudaSuccess) return fail(LBM_ERR_CUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
  if (st != LBM_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (e2 != cudaSuccess) return fail(LBM_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e2));
  e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) { G.exec = nullptr; return fail(LBM_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e)); }
  return LBM_OK;
}

}  // namespace

void lbm_set_last_error(const char* msg) { g_last_error = msg; }

extern "C" {

const char* lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_ERR_ARG: return "invalid argument";
    case LBM_ERR_WORKSPACE: return "workspace too small or misaligned";
    case LBM_ERR_CUDA: return "CUDA error";
    case LBM_ERR_STATE: return "call out of order";
    case LBM_ERR_NONFINITE: return "non-finite or non-positive density";
    case LBM_NOT_CONVERGED: return "not converged";
  }
  return "unknown status";
}

const char* lbm_last_error(void) { return g_last_error.c_str(); }

lbm_status lbm_workspace_size(const lbm_config* cfg, size_t* bytes) {
  if (!cfg || !bytes) return fail(LBM_ERR_ARG, "null argument");
  LBM_TRY(validate_config(*cfg));
  *bytes = make_layout(*cfg).total;
  return LBM_OK;
}

lbm_status lbm_create(const lbm_config* cfg, const uint8_t* node_class, const float* design_gamma,
                      const float* objective_weights, const float* inlet_u, void* workspace,
                      size_t workspace_bytes, void* stream, lbm_ctx** out) {
  if (!cfg || !node_class || !design_gamma || !out) return fail(LBM_ERR_ARG, "null argument");
  *out = nullptr;
  LBM_TRY(validate_config(*cfg));
  const lbm_config& c = *cfg;
  LBM_TRY(c.lattice == LBM_D2Q9 ? validate_classes<D2Q9>(c, node_class) : validate_classes<D3Q19>(c, node_class));
  const Layout lay = make_layout(c);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign))
    return fail(LBM_ERR_WORKSPACE, "workspace must be a 256-byte aligned device pointer");
  if (workspace_bytes < lay.total)
    return fail(LBM_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, lay.total);
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, workspace) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(LBM_ERR_WORKSPACE, "workspace is not device memory");
  }

  auto ctx = std::make_unique<lbm_ctx>();
  ctx->cfg = c;
  ctx->lay = lay;
  ctx->ws = static_cast<char*>(workspace);
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->ls = ctx->stream;
  ctx->n = size_t(c.nx) * c.ny * c.nz;
  ctx->q = c.lattice;
  ctx->rs = c.precision == LBM_FP64 ? 8 : 4;
  ctx->geo = lbm::Geo{c.nx, c.ny, c.nz, c.periodic[0], c.periodic[1], c.periodic[2], unsigned(ctx->n),
                      unsigned(c.nx), unsigned(c.nx) * unsigned(c.ny)};
  ctx->cur = 0;
  lbm_ctx* x = ctx.get();
  CUDA_TRY(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
  ctx->side_cur = ctx->side;
  ctx->fork_cur = ctx->fork_ev;
  ctx->join_cur = ctx->join_ev;
  if (c.pipeline) {
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->rec, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->rec_side, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&ctx->rec_fork, &ctx->rec_join, &ctx->start_ev, &ctx->rec_done[0], &ctx->rec_done[1],
                           &ctx->adj_done[0], &ctx->adj_done[1]})
      CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  if (c.lattice == LBM_D2Q9) {
    if (c.precision == LBM_FP32) ctx->impl.reset(new ImplT<D2Q9, float>(x));
    else ctx->impl.reset(new ImplT<D2Q9, double>(x));
  } else {
    if (c.precision == LBM_FP32) ctx->impl.reset(new ImplT<D3Q19, float>(x));
    else ctx->impl.reset(new ImplT<D3Q19, double>(x));
  }
  const size_t n = ctx->n;
  cudaStream_t s = ctx->stream;
  CUDA_TRY(cudaMemsetAsync(x->at(lay.f[0]), 0, align_up(ctx->q * n * ctx->rs), s));   // rest equilibrium
  CUDA_TRY(cudaMemsetAsync(x->at(lay.partials), 0, size_t(lay.nblocks_fwd) * 32, s));
  CUDA_TRY(cudaMemsetAsync(x->at(lay.acc), 0, sizeof(lbm::WindowAcc), s));
  CUDA_TRY(cudaMemsetAsync(x->at(lay.flags), 0, 16, s));
  CUDA_TRY(cudaMemcpyAsync(x->at(lay.cls), node_class, n, cudaMemcpyDefault, s));
  x->zg = lbm::zg_rows(node_class, x->geo);
  CUDA_TRY(cudaMemcpyAsync(x->at(lay.gamma), design_gamma, n * 4, cudaMemcpyDefault, s));
  if (objective_weights) CUDA_TRY(cudaMemcpyAsync(x->at(lay.wobj), objective_weights, n * 4, cudaMemcpyDefault, s));
  else CUDA_TRY(cudaMemsetAsync(x->at(lay.wobj), 0, n * 4, s));
  if (inlet_u) CUDA_TRY(cudaMemcpyAsync(x->at(lay.uin), inlet_u, size_t(c.ny) * c.nz * 4, cudaMemcpyDefault, s));
  else CUDA_TRY(cudaMemsetAsync(x->at(lay.uin), 0, size_t(c.ny) * c.nz * 4, s));
  CUDA_TRY(cudaMemsetAsync(x->at(lay.gacc), 0, n * 16, s));
  // Constant part of a pressure objective: cs^2 * sum of weights (FP64, host).
  if (c.objective_kind == LBM_OBJ_PRESSURE) {
    std::vector<float> w(n, 0.f);
    if (objective_weights) {
      CUDA_TRY(cudaMemcpyAsync(w.data(), objective_weights, n * 4, cudaMemcpyDefault, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    }
    double sw = 0, cw = 0;
    const int* b = c.obj_box;
    for (int z = b[4]; z < b[5]; ++z)
      for (int y = b[2]; y < b[3]; ++y)
        for (int xx = b[0]; xx < b[1]; ++xx) {
          const double v = w[size_t(xx) + size_t(c.nx) * (size_t(y) + size_t(c.ny) * z)];
          const double t = sw + v;
          cw += std::fabs(sw) >= std::fabs(v) ? (sw - t) + v : (v - t) + sw;
          sw = t;
        }
    ctx->jconst = (sw + cw) / 3.0;
  }
  {
    // per-slice constants (D2Q9 batches); zero unless the objective is a pressure
    std::vector<double> sc(size_t(c.nz), 0.0);
    if (c.objective_kind == LBM_OBJ_PRESSURE && objective_weights) {
      std::vector<float> w(n);
      CUDA_TRY(cudaMemcpy(w.data(), objective_weights, n * 4, cudaMemcpyDefault));
      const int* b = c.obj_box;
      for (int z = b[4]; z < b[5]; ++z) {
        double sw = 0, cw = 0;
        for (int y = b[2]; y < b[3]; ++y)
          for (int xx = b[0]; xx < b[1]; ++xx) {
            const double v = w[size_t(xx) + size_t(c.nx) * (size_t(y) + size_t(c.ny) * z)];
            const double t = sw + v;
            cw += std::fabs(sw) >= std::fabs(v) ? (sw - t) + v : (v - t) + sw;
            sw = t;
          }
        sc[size_t(z)] = (sw + cw) / 3.0;
      }
    }
    CUDA_TRY(cudaMemcpyAsync(x->at(lay.slice_c), sc.data(), sc.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  {
    std::vector<float> u(size_t(c.ny) * c.nz, 0.f);
    if (inlet_u) {
      CUDA_TRY(cudaMemcpyAsync(u.data(), inlet_u, u.size() * 4, cudaMemcpyDefault, s));
      CUDA_TRY(cudaStreamSynchronize(s));
    }
    for (float v : u)
      if (!(std::fabs(v) < 0.5f)) return fail(LBM_ERR_ARG, "inlet velocities must satisfy |u| < 0.5");
  }
  x->impl->set_design();
  CUDA_TRY(cudaGetLastError());
  LBM_TRY(check_flags(x, 1, LBM_ERR_ARG, "design values must lie in [0, 1]"));
  *out = ctx.release();
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* ctx) { delete ctx; }

lbm_status lbm_step_window(lbm_ctx* c, double* J_window, double* monitor_window) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  const lbm_config& k = c->cfg;
  const int cur0 = c->cur;
  if (c->use_graphs) {
    GraphRec& G = c->gwin[cur0][c->timing ? 1 : 0];
    if (!G.exec) LBM_TRY(capture(c, G, enqueue_window));
    CUDA_TRY(cudaGraphLaunch(G.exec, c->stream));
    c->cur = cur0 ^ (k.window_len & 1);
  } else {
    LBM_TRY(enqueue_window(c));
  }
  CUDA_TRY(cudaGetLastError());
  lbm::WindowAcc acc;
  CUDA_TRY(cudaMemcpyAsync(&acc, c->at(c->lay.acc), sizeof acc, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (c->use_graphs) c->harvest_graph(c->gwin[cur0][c->timing ? 1 : 0]);
  c->harvest();
  c->steps += k.window_len;
  if (acc.nonfinite) {
    c->window_valid = false;
    c->grad_valid = false;
    return fail(LBM_ERR_NONFINITE, "window %lld produced a non-positive density or a non-finite value",
                (long long)c->windows);
  }
  c->windows += 1;
  c->window_valid = true;
  c->grad_valid = false;
  c->last_j = acc.jmean;
  c->last_m = acc.mmean;
  c->nwin_for_ratio += 1;
  c->ratio = c->nwin_for_ratio >= 2 ? acc.ratio : INFINITY;
  c->converged = c->nwin_for_ratio >= 2 ? acc.converged : 0;
  if (J_window) *J_window = acc.jmean;
  if (monitor_window) *monitor_window = acc.mmean;
  return LBM_OK;
}

lbm_status lbm_run_until_converged(lbm_ctx* c, int32_t max_windows, int32_t* windows, double* J_window,
                                   double* monitor_window, double* ratio) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  if (max_windows < 1) return fail(LBM_ERR_ARG, "max_windows must be >= 1");
  double J = 0, M = 0;
  int32_t w = 0;
  while (w < max_windows) {
    LBM_TRY(lbm_step_window(c, &J, &M));
    w += 1;
    if (c->converged) break;
  }
  if (windows) *windows = w;
  if (J_window) *J_window = J;
  if (monitor_window) *monitor_window = M;
  if (ratio) *ratio = c->ratio;
  if (!c->converged)
    return fail(LBM_NOT_CONVERGED, "Eq. 26 did not hold within %d windows (last ratio %.3e)", max_windows, c->ratio);
  return LBM_OK;
}

lbm_status lbm_step_window_along(lbm_ctx* c, lbm_ctx* ref, double* J_window, double* monitor_window) {
  if (!c || !ref) return fail(LBM_ERR_ARG, "null context");
  if (c == ref) return fail(LBM_ERR_ARG, "the reference must be another context");
  const lbm_config &k = c->cfg, &r = ref->cfg;
  if (k.lattice != r.lattice || k.nx != r.nx || k.ny != r.ny || k.nz != r.nz || k.window_len != r.window_len ||
      k.ckpt_every != r.ckpt_every)
    return fail(LBM_ERR_ARG, "the reference must have the same lattice, window length and checkpoint interval");
  if (k.ckpt_format == LBM_CKPT_MOMENT)
    return fail(LBM_ERR_ARG, "a window along a reference cannot store moment checkpoints (its segments restart)");
  if (!ref->window_valid) return fail(LBM_ERR_STATE, "the reference has no completed window");
  CUDA_TRY(cudaStreamSynchronize(ref->stream));
  // one direct enqueue: no graph holds the reference's buffers
  c->along = ref;
  const lbm_status st = enqueue_window(c);
  c->along = nullptr;
  LBM_TRY(st);
  CUDA_TRY(cudaGetLastError());
  lbm::WindowAcc acc;
  CUDA_TRY(cudaMemcpyAsync(&acc, c->at(c->lay.acc), sizeof acc, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->harvest();
  c->steps += k.window_len;
  if (acc.nonfinite) {
    c->window_valid = false;
    c->grad_valid = false;
    return fail(LBM_ERR_NONFINITE, "the window along the reference produced a non-positive density or a non-finite value");
  }
  c->windows += 1;
  c->window_valid = true;
  c->grad_valid = false;
  c->last_j = acc.jmean;
  c->last_m = acc.mmean;
  c->nwin_for_ratio += 1;
  c->ratio = c->nwin_for_ratio >= 2 ? acc.ratio : INFINITY;
  c->converged = c->nwin_for_ratio >= 2 ? acc.converged : 0;
  if (J_window) *J_window = acc.jmean;
  if (monitor_window) *monitor_window = acc.mmean;
  return LBM_OK;
}

lbm_status lbm_window_objectives(lbm_ctx* c, double* J, double* monitor, size_t nslices) {
  if (!c || !J) return fail(LBM_ERR_ARG, "null argument");
  if (c->cfg.lattice != LBM_D2Q9) return fail(LBM_ERR_ARG, "per-slice objectives exist for D2Q9 batches only");
  if (nslices != size_t(c->cfg.nz)) return fail(LBM_ERR_ARG, "nslices %zu, expected nz = %d", nslices, c->cfg.nz);
  if (!c->window_valid) return fail(LBM_ERR_STATE, "no completed window");
  std::vector<double> h(2 * nslices);
  CUDA_TRY(cudaMemcpyAsync(h.data(), c->at(c->lay.slice_j), h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  for (size_t s = 0; s < nslices; ++s) {
    J[s] = h[2 * s];
    if (monitor) monitor[s] = h[2 * s + 1];
  }
  return LBM_OK;
}

lbm_status lbm_window_converged(lbm_ctx* c, int* converged, double* ratio) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  if (converged) *converged = c->converged;
  if (ratio) *ratio = c->ratio;
  return LBM_OK;
}

lbm_status lbm_adjoint_window(lbm_ctx* c, double* J_eff) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  if (!c->window_valid) return fail(LBM_ERR_STATE, "no completed window to differentiate");
  GraphRec* G = nullptr;
  if (c->use_graphs) {
    G = &c->gadj[c->timing ? 1 : 0];
    if (!G->exec) LBM_TRY(capture(c, *G, enqueue_adjoint));
    CUDA_TRY(cudaGraphLaunch(G->exec, c->stream));
  } else {
    LBM_TRY(enqueue_adjoint(c));
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  if (G) c->harvest_graph(*G);
  c->harvest();
  // The sweep runs an even or odd number of adjoint steps: b^{n0} is in buffer (W-1) & 1.
  c->bout_last = (c->cfg.window_len - 1) & 1;
  c->grad_valid = true;
  if (J_eff) *J_eff = c->last_j;
  return LBM_OK;
}

lbm_status lbm_design_gradient(lbm_ctx* c, double* grad, size_t n) {
  if (!c || !grad) return fail(LBM_ERR_ARG, "null argument");
  if (!c->grad_valid) return fail(LBM_ERR_STATE, "no adjoint window computed");
  if (n != c->n) return fail(LBM_ERR_ARG, "gradient length %zu, expected %zu", n, c->n);
  c->impl->grad();
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(grad, c->at(c->lay.gout), n * 8, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_set_design(lbm_ctx* c, const float* gamma) {
  if (!c || !gamma) return fail(LBM_ERR_ARG, "null argument");
  CUDA_TRY(cudaMemcpyAsync(c->at(c->lay.gamma), gamma, c->n * 4, cudaMemcpyDefault, c->stream));
  c->filtered = false;
  c->impl->set_design();
  CUDA_TRY(cudaGetLastError());
  c->window_valid = false;
  c->grad_valid = false;
  c->nwin_for_ratio = 0;
  return check_flags(c, 1, LBM_ERR_ARG, "design values must lie in [0, 1]");
}

lbm_status lbm_get_design(lbm_ctx* c, float* gamma, size_t n) {
  if (!c || !gamma) return fail(LBM_ERR_ARG, "null argument");
  if (n != c->n) return fail(LBM_ERR_ARG, "design length %zu, expected %zu", n, c->n);
  CUDA_TRY(cudaMemcpyAsync(gamma, c->at(c->lay.gamma), n * 4, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_set_design_filtered(lbm_ctx* c, const float* x_raw, const lbm_filter* f) {
  if (!c || !x_raw || !f) return fail(LBM_ERR_ARG, "null argument");
  if (!(f->radius > 0.0 && f->radius < 64.0)) return fail(LBM_ERR_ARG, "filter radius must be in (0, 64)");
  if (!(f->beta > 0.0) || !(f->eta > 0.0 && f->eta < 1.0))
    return fail(LBM_ERR_ARG, "projection needs beta > 0 and 0 < eta < 1");
  lbm::FilterGeo g{};
  g.nx = c->cfg.nx;
  g.ny = c->cfg.ny;
  g.nz = c->cfg.nz;
  for (int k = 0; k < 6; ++k) g.box[k] = c->cfg.design_box[k];
  g.R = int(std::ceil(f->radius));
  g.radius = f->radius;
  g.beta = f->beta;
  g.eta = f->eta;
  g.d3 = c->cfg.lattice == LBM_D3Q19;
  CUDA_TRY(cudaMemcpyAsync(c->at(c->lay.xraw), x_raw, c->n * 4, cudaMemcpyDefault, c->stream));
  const long long blocks = (long long)(c->n + 255) / 256;
  lbm::filter_project_kernel<<<int(blocks < 148 * 32 ? blocks : 148 * 32), 256, 0, c->stream>>>(
      c->at<float>(c->lay.xraw), c->at<float>(c->lay.gamma), c->at<double>(c->lay.xfilt), c->at<double>(c->lay.wfilt), g);
  c->impl->set_design();
  CUDA_TRY(cudaGetLastError());
  c->window_valid = false;
  c->grad_valid = false;
  c->nwin_for_ratio = 0;
  c->filtered = true;
  c->fgeo = g;
  return check_flags(c, 1, LBM_ERR_ARG, "raw design values must lie in [0, 1]");
}

lbm_status lbm_design_gradient_filtered(lbm_ctx* c, double* grad, size_t n) {
  if (!c || !grad) return fail(LBM_ERR_ARG, "null argument");
  if (!c->grad_valid) return fail(LBM_ERR_STATE, "no adjoint window computed");
  if (!c->filtered) return fail(LBM_ERR_STATE, "the design was not set through lbm_set_design_filtered");
  if (n != c->n) return fail(LBM_ERR_ARG, "gradient length %zu, expected %zu", n, c->n);
  c->impl->grad();
  double* t = c->at<double>(c->lay.stage);
  double* out = t + c->n;
  const long long blocks = (long long)(c->n + 255) / 256;
  const int nb = int(blocks < 148 * 32 ? blocks : 148 * 32);
  lbm::filter_adjoint_scale_kernel<<<nb, 256, 0, c->stream>>>(c->at<double>(c->lay.gout), c->at<double>(c->lay.xfilt),
                                                               c->at<double>(c->lay.wfilt), t, c->fgeo);
  lbm::filter_adjoint_gather_kernel<<<nb, 256, 0, c->stream>>>(c->at<double>(c->lay.gout), t, out, c->fgeo);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(grad, out, n * 8, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_filter_chain_rule(lbm_ctx* c, const double* dgamma, double* dx, size_t n) {
  if (!c || !dgamma || !dx) return fail(LBM_ERR_ARG, "null argument");
  if (!c->filtered) return fail(LBM_ERR_STATE, "the design was not set through lbm_set_design_filtered");
  if (n != c->n) return fail(LBM_ERR_ARG, "sensitivity length %zu, expected %zu", n, c->n);
  double* t = c->at<double>(c->lay.stage);   // the stage holds Q N >= 3 N doubles
  double* out = t + c->n;
  double* g = t + 2 * c->n;
  CUDA_TRY(cudaMemcpyAsync(g, dgamma, n * 8, cudaMemcpyDefault, c->stream));
  const long long blocks = (long long)(c->n + 255) / 256;
  const int nb = int(blocks < 148 * 32 ? blocks : 148 * 32);
  lbm::filter_adjoint_scale_kernel<<<nb, 256, 0, c->stream>>>(g, c->at<double>(c->lay.xfilt),
                                                               c->at<double>(c->lay.wfilt), t, c->fgeo);
  lbm::filter_adjoint_gather_kernel<<<nb, 256, 0, c->stream>>>(g, t, out, c->fgeo);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(dx, out, n * 8, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_design_volume(lbm_ctx* c, double* volume) {
  if (!c || !volume) return fail(LBM_ERR_ARG, "null argument");
  const int* d = c->cfg.design_box;
  const long long cells = (long long)(d[1] - d[0]) * (d[3] - d[2]) * (d[5] - d[4]);
  if (cells <= 0) return fail(LBM_ERR_ARG, "the design box is empty");
  const long long want = (cells + lbm::kVolThreads - 1) / lbm::kVolThreads;
  const int nb = int(want < 148 * 4 ? want : 148 * 4);
  double* part = c->at<double>(c->lay.stage);
  lbm::design_volume_kernel<<<nb, lbm::kVolThreads, 0, c->stream>>>(
      c->at<float>(c->lay.gamma), c->cfg.nx, c->cfg.ny, d[0], d[1], d[2], d[3], d[4], d[5], part);
  CUDA_TRY(cudaGetLastError());
  std::vector<double> h(nb);
  CUDA_TRY(cudaMemcpyAsync(h.data(), part, size_t(nb) * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += h[b];
  *volume = s / double(cells);
  return LBM_OK;
}

lbm_status lbm_get_state(lbm_ctx* c, double* f, size_t n) {
  if (!c || !f) return fail(LBM_ERR_ARG, "null argument");
  if (n != c->n * c->q) return fail(LBM_ERR_ARG, "state length %zu, expected %zu", n, c->n * c->q);
  c->impl->unshift(c->lattice(c->cur));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(f, c->at(c->lay.stage), n * 8, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx* c, const double* f, size_t n) {
  if (!c || !f) return fail(LBM_ERR_ARG, "null argument");
  if (n != c->n * c->q) return fail(LBM_ERR_ARG, "state length %zu, expected %zu", n, c->n * c->q);
  CUDA_TRY(cudaMemcpyAsync(c->at(c->lay.stage), f, n * 8, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaMemsetAsync(c->at<int>(c->lay.flags), 0, sizeof(int), c->stream));   // clear the sticky non-finite flag
  c->impl->shift(c->lattice(c->cur));
  CUDA_TRY(cudaGetLastError());
  c->window_valid = false;
  c->grad_valid = false;
  c->nwin_for_ratio = 0;
  return check_flags(c, 1, LBM_ERR_ARG, "state holds non-finite values");
}

lbm_status lbm_get_adjoint_state(lbm_ctx* c, double* a, size_t n) {
  if (!c || !a) return fail(LBM_ERR_ARG, "null argument");
  if (!c->grad_valid) return fail(LBM_ERR_STATE, "no adjoint window computed");
  if (n != c->n * c->q) return fail(LBM_ERR_ARG, "state length %zu, expected %zu", n, c->n * c->q);
  // a^{n0-1} = S^T b^{n0}: pull into the other adjoint buffer, widen to FP64.
  c->impl->pull(c->adjbuf(c->bout_last), c->adjbuf(c->bout_last ^ 1));
  c->impl->to_double(c->adjbuf(c->bout_last ^ 1));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(a, c->at(c->lay.stage), n * 8, cudaMemcpyDefault, c->stream));
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_advance(lbm_ctx* c, int32_t nsteps) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  if (nsteps < 0) return fail(LBM_ERR_ARG, "nsteps must be >= 0");
  cudaEvent_t e = c->begin();
  for (int j = 0; j < nsteps; ++j) {
    c->impl->fwd(c->lattice(c->cur), c->lattice(c->cur ^ 1), 0);
    c->cur ^= 1;
  }
  c->end(e, 0, nsteps, int64_t(nsteps) * int64_t(c->n));
  CUDA_TRY(cudaGetLastError());
  c->steps += nsteps;
  c->window_valid = false;
  c->grad_valid = false;
  LBM_TRY(check_flags(c, 0, LBM_ERR_NONFINITE, "a non-positive density or non-finite value appeared"));
  c->harvest();
  return LBM_OK;
}

lbm_status lbm_set_timing(lbm_ctx* c, int32_t enable) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  c->timing = enable != 0;
  return LBM_OK;
}

lbm_status lbm_get_timing(lbm_ctx* c, lbm_timing* out) {
  if (!c || !out) return fail(LBM_ERR_ARG, "null argument");
  CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->harvest();
  *out = c->tm;
  c->tm = lbm_timing{};
  return LBM_OK;
}

lbm_status lbm_set_graphs(lbm_ctx* c, int32_t enable) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  c->use_graphs = enable != 0;
  return LBM_OK;
}

lbm_status lbm_set_pdl(lbm_ctx* c, int32_t enable) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  if ((enable != 0) != c->use_pdl) {
    // captured graphs hold the old launch attributes: capture again on next use
    for (auto& row : c->gwin) for (auto& g : row) c->drop_graph(g);
    for (auto& g : c->gadj) c->drop_graph(g);
  }
  c->use_pdl = enable != 0;
  return LBM_OK;
}

lbm_status lbm_set_sample_start(lbm_ctx* c, int32_t first) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  const lbm_config& k = c->cfg;
  if (first < 0 || first >= k.window_len || (k.window_len - first) % k.sample_every)
    return fail(LBM_ERR_ARG, "the first sampled step must lie in [0, window_len) with window_len - first a multiple of sample_every");
  if (first != c->sample_from) {
    // captured graphs hold the old sampling flags and weight: capture again on next use
    for (auto& row : c->gwin) for (auto& g : row) c->drop_graph(g);
    for (auto& g : c->gadj) c->drop_graph(g);
  }
  c->sample_from = first;
  c->window_valid = false;
  c->grad_valid = false;
  return LBM_OK;
}

lbm_status lbm_get_schedule(lbm_ctx* c, lbm_schedule* out) {
  if (!c || !out) return fail(LBM_ERR_ARG, "null argument");
  out->graphs = c->use_graphs ? 1 : 0;
  out->pdl = c->use_pdl ? 1 : 0;
  out->kernels_window = c->kernels_window;
  out->kernels_adjoint = c->kernels_adjoint;
  return LBM_OK;
}

lbm_status lbm_get_counters(lbm_ctx* c, int64_t* steps, int64_t* windows) {
  if (!c) return fail(LBM_ERR_ARG, "null context");
  if (steps) *steps = c->steps;
  if (windows) *windows = c->windows;
  return LBM_OK;
}

}  // extern "C"
