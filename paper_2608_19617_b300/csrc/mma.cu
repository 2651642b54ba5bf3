// The Method of Moving Asymptotes (Svanberg 1987): the design update of the
// optimization loop (Sec. 3.3, topology optimization procedure).
//
// One iteration from a point x with objective f_0, constraints f_i <= 0
// (i = 1..m) and their gradients:
//   1. asymptotes L_j < x_j < U_j: x_j -/+ 0.5 (xmax_j - xmin_j) at the first
//      two iterations, then contracted by 0.7 where the last two changes of
//      x_j alternate in sign, widened by 1.2 where they agree, each kept
//      within [0.01, 10] (xmax_j - xmin_j) of x_j;
//   2. move limits alpha_j = max(xmin_j, L_j + 0.1 (x_j - L_j)),
//      beta_j = min(xmax_j, U_j - 0.1 (U_j - x_j));
//   3. the convex separable approximations
//      f~_i(z) = r_i + sum_j p_ij / (U_j - z_j) + q_ij / (z_j - L_j),
//      p_ij = (U_j - x_j)^2 max(0, df_i/dx_j), q_ij = (x_j - L_j)^2 max(0, -df_i/dx_j),
//      r_i chosen so that f~_i(x) = f_i(x);
//   4. the subproblem min f~_0 + sum_i (c y_i + y_i^2 / 2) subject to
//      f~_i(z) - y_i <= 0, y >= 0, alpha <= z <= beta (c = 1000; the y_i keep it
//      feasible), solved by the dual method: for multipliers lam >= 0 every
//      z_j has the closed form (sqrt(P_j) L_j + sqrt(Q_j) U_j) / (sqrt(P_j) +
//      sqrt(Q_j)), P = p_0 + lam.p, Q = q_0 + lam.q, clipped to [alpha_j, beta_j].
//
// The per-variable work (steps 1-3, each evaluation of the dual, the final
// update) runs in the kernels below, one grid-stride pass over the n
// variables each, with per-block FP64 partial sums that the host adds in a
// fixed order.  The dual W(lam) is concave in the m multipliers; the host
// maximises it by a projected Newton iteration with a backtracking line
// search, from the dual's gradient (the constraint values at z(lam)) and its
// Hessian (-sum over free z_j of a_i a_k / h_j, a_ij = df~_i/dz_j,
// h_j = d^2 L / dz_j^2).  Everything is FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbmadj.h"

// Records the reason returned by lbm_last_error (defined with the other entry points).
void lbm_set_last_error(const char* msg);

namespace {

constexpr int kMmaThreads = 256;
constexpr int kMmaMaxBlocks = 296;          // 2 x 148 SMs
constexpr int kMmaSums = 1 + LBM_MMA_MAX_M + LBM_MMA_MAX_M * (LBM_MMA_MAX_M + 1) / 2;
constexpr double kSInit = 0.5, kSSlow = 0.7, kSFast = 1.2, kAlbefa = 0.1, kCArt = 1000.0;

lbm_status mma_fail(lbm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  lbm_set_last_error(buf);
  return s;
}

#define MMA_CUDA(expr)                                                                               \
  do {                                                                                               \
    cudaError_t e_ = (expr);                                                                         \
    if (e_ != cudaSuccess) return mma_fail(LBM_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

// Device arrays of one MMA run (all FP64, [n] unless noted).
struct MmaDev {
  size_t n;
  int m;
  const double* xmin;
  const double* xmax;
  double* xold1;
  double* xold2;
  double* low;
  double* upp;
  double* alpha;
  double* beta;
  double* p;        // [m+1][n]
  double* q;        // [m+1][n]
  double* part;     // [blocks][kMmaSums]
};

struct Lam {
  double v[LBM_MMA_MAX_M];
};

// Block sum of one value per thread into part[blockIdx.x * kMmaSums + s].
__device__ void block_sum(double v, double* part, int s) {
  __shared__ double w[kMmaThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int k = 0; k < kMmaThreads / 32; ++k) t += w[k];
    part[size_t(blockIdx.x) * kMmaSums + s] = t;
  }
  __syncthreads();
}

// Steps 1-3: asymptotes, move limits, p and q; partial sums of
// sum_j p_ij / (U_j - x_j) + q_ij / (x_j - L_j) for r_i.
__global__ void __launch_bounds__(kMmaThreads) mma_prepare_kernel(MmaDev D, const double* __restrict__ x,
                                                                  const double* __restrict__ dfdx, int iter) {
  const size_t n = D.n;
  double acc[LBM_MMA_MAX_M + 1];
  for (int i = 0; i <= D.m; ++i) acc[i] = 0;
  for (size_t j = size_t(blockIdx.x) * kMmaThreads + threadIdx.x; j < n; j += size_t(gridDim.x) * kMmaThreads) {
    const double xj = x[j], span = D.xmax[j] - D.xmin[j];
    double L, U;
    if (iter <= 2) {
      L = xj - kSInit * span;
      U = xj + kSInit * span;
    } else {
      const double o1 = D.xold1[j], o2 = D.xold2[j];
      const double sg = (xj - o1) * (o1 - o2);
      const double fac = sg < 0 ? kSSlow : (sg > 0 ? kSFast : 1.0);
      L = xj - fac * (o1 - D.low[j]);
      U = xj + fac * (D.upp[j] - o1);
      L = fmin(fmax(L, xj - 10.0 * span), xj - 0.01 * span);
      U = fmin(fmax(U, xj + 0.01 * span), xj + 10.0 * span);
    }
    D.low[j] = L;
    D.upp[j] = U;
    D.alpha[j] = fmax(D.xmin[j], L + kAlbefa * (xj - L));
    D.beta[j] = fmin(D.xmax[j], U - kAlbefa * (U - xj));
    const double ux = U - xj, xl = xj - L;
    for (int i = 0; i <= D.m; ++i) {
      const double g = dfdx[size_t(i) * n + j];
      const double pi = ux * ux * fmax(g, 0.0), qi = xl * xl * fmax(-g, 0.0);
      D.p[size_t(i) * n + j] = pi;
      D.q[size_t(i) * n + j] = qi;
      acc[i] += pi / ux + qi / xl;
    }
  }
  for (int i = 0; i <= D.m; ++i) block_sum(acc[i], D.part, i);
}

// z_j(lam) and whether it is strictly inside [alpha_j, beta_j].
__device__ __forceinline__ double z_of(const MmaDev& D, const Lam& lam, size_t j, double xj, double& P, double& Q,
                                       bool& free_var) {
  const size_t n = D.n;
  P = D.p[j];
  Q = D.q[j];
  for (int i = 1; i <= D.m; ++i) {
    P += lam.v[i - 1] * D.p[size_t(i) * n + j];
    Q += lam.v[i - 1] * D.q[size_t(i) * n + j];
  }
  const double sp = sqrt(P), sq = sqrt(Q);
  const double a = D.alpha[j], b = D.beta[j];
  if (!(sp + sq > 0)) {   // no term depends on z_j: it stays at x_j
    free_var = false;
    return fmin(fmax(xj, a), b);
  }
  const double z = (sp * D.low[j] + sq * D.upp[j]) / (sp + sq);
  free_var = z > a && z < b;
  return fmin(fmax(z, a), b);
}

// One evaluation of the dual: per-block sums of
//   s_i = sum_j p_ij / (U_j - z_j) + q_ij / (z_j - L_j)         (i = 0..m)
//   H_ik = -sum_{free j} a_ij a_kj / h_j                         (1 <= i <= k <= m)
__global__ void __launch_bounds__(kMmaThreads) mma_dual_kernel(MmaDev D, const double* __restrict__ x, Lam lam) {
  const size_t n = D.n;
  const int m = D.m;
  double s[LBM_MMA_MAX_M + 1];
  double h[LBM_MMA_MAX_M * (LBM_MMA_MAX_M + 1) / 2];
  for (int i = 0; i <= m; ++i) s[i] = 0;
  for (int i = 0; i < m * (m + 1) / 2; ++i) h[i] = 0;
  for (size_t j = size_t(blockIdx.x) * kMmaThreads + threadIdx.x; j < n; j += size_t(gridDim.x) * kMmaThreads) {
    double P, Q;
    bool fr;
    const double z = z_of(D, lam, j, x[j], P, Q, fr);
    const double du = D.upp[j] - z, dl = z - D.low[j];
    double a[LBM_MMA_MAX_M];
    for (int i = 0; i <= m; ++i) {
      const double pi = D.p[size_t(i) * n + j], qi = D.q[size_t(i) * n + j];
      s[i] += pi / du + qi / dl;
      if (i > 0) a[i - 1] = pi / (du * du) - qi / (dl * dl);
    }
    if (fr) {
      const double hj = 2.0 * P / (du * du * du) + 2.0 * Q / (dl * dl * dl);
      int t = 0;
      for (int i = 0; i < m; ++i)
        for (int k = i; k < m; ++k) h[t++] -= a[i] * a[k] / hj;
    }
  }
  for (int i = 0; i <= m; ++i) block_sum(s[i], D.part, i);
  for (int i = 0; i < m * (m + 1) / 2; ++i) block_sum(h[i], D.part, m + 1 + i);
}

// The new point z(lam*), and the history of the iterates.
__global__ void __launch_bounds__(kMmaThreads) mma_finish_kernel(MmaDev D, double* __restrict__ x, Lam lam) {
  for (size_t j = size_t(blockIdx.x) * kMmaThreads + threadIdx.x; j < D.n; j += size_t(gridDim.x) * kMmaThreads) {
    double P, Q;
    bool fr;
    const double xj = x[j];
    const double z = z_of(D, lam, j, xj, P, Q, fr);
    D.xold2[j] = D.xold1[j];
    D.xold1[j] = xj;
    x[j] = z;
  }
}

}  // namespace

struct lbm_mma {
  MmaDev dev;
  int iter = 0;
  int blocks = 0;
  cudaStream_t stream = nullptr;
  std::vector<double> part;   // host copy of the block sums
  double last_lam[LBM_MMA_MAX_M] = {};
  int last_newton = 0;
};

namespace {

struct MmaLayout {
  size_t xmin, xmax, xold1, xold2, low, upp, alpha, beta, p, q, part, total;
};

MmaLayout mma_layout(size_t n, int m) {
  MmaLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += up256(bytes); return o; };
  const size_t v = n * sizeof(double);
  L.xmin = take(v);
  L.xmax = take(v);
  L.xold1 = take(v);
  L.xold2 = take(v);
  L.low = take(v);
  L.upp = take(v);
  L.alpha = take(v);
  L.beta = take(v);
  L.p = take(v * size_t(m + 1));
  L.q = take(v * size_t(m + 1));
  L.part = take(size_t(kMmaMaxBlocks) * kMmaSums * sizeof(double));
  L.total = off;
  return L;
}

// Sums of the block partials, in block order.
lbm_status gather(lbm_mma* o, int count, double* out) {
  MMA_CUDA(cudaMemcpyAsync(o->part.data(), o->dev.part, size_t(o->blocks) * kMmaSums * sizeof(double),
                           cudaMemcpyDeviceToHost, o->stream));
  MMA_CUDA(cudaStreamSynchronize(o->stream));
  for (int s = 0; s < count; ++s) {
    double t = 0;
    for (int b = 0; b < o->blocks; ++b) t += o->part[size_t(b) * kMmaSums + s];
    out[s] = t;
  }
  return LBM_OK;
}

struct DualEval {
  double W;
  double g[LBM_MMA_MAX_M];
  double H[LBM_MMA_MAX_M][LBM_MMA_MAX_M];
  double scale;   // magnitude of the terms behind g (for the stopping test)
};

lbm_status eval_dual(lbm_mma* o, const double* x, const double* r, const double* lam, DualEval& e) {
  const int m = o->dev.m;
  Lam L{};
  for (int i = 0; i < m; ++i) L.v[i] = lam[i];
  mma_dual_kernel<<<o->blocks, kMmaThreads, 0, o->stream>>>(o->dev, x, L);
  MMA_CUDA(cudaGetLastError());
  double s[kMmaSums];
  {
    const lbm_status st = gather(o, 1 + m + m * (m + 1) / 2, s);
    if (st != LBM_OK) return st;
  }
  const double f0 = r[0] + s[0];
  e.W = f0;
  e.scale = 1.0;
  for (int i = 0; i < m; ++i) {
    const double fi = r[i + 1] + s[i + 1];
    const double y = fmax(0.0, lam[i] - kCArt);
    e.g[i] = fi - y;
    e.W += lam[i] * (fi - y) + kCArt * y + 0.5 * y * y;
    e.scale = fmax(e.scale, fabs(r[i + 1]) + fabs(s[i + 1]));
  }
  int t = 1 + m;
  for (int i = 0; i < m; ++i)
    for (int k = i; k < m; ++k) {
      e.H[i][k] = e.H[k][i] = s[t++];
    }
  for (int i = 0; i < m; ++i)
    if (lam[i] > kCArt) e.H[i][i] -= 1.0;
  return LBM_OK;
}

// Newton step on the free block: solve (-A) d = b for the symmetric negative
// definite A (the dual Hessian) by Cholesky of -A; false when it is not
// numerically definite.
bool solve_neg_def(int k, double A[LBM_MMA_MAX_M][LBM_MMA_MAX_M], const double* b, double* d) {
  double Lc[LBM_MMA_MAX_M][LBM_MMA_MAX_M] = {};
  double diag = 0;
  for (int i = 0; i < k; ++i) diag = fmax(diag, -A[i][i]);
  const double eps = 1e-14 * (diag > 0 ? diag : 1.0);
  for (int i = 0; i < k; ++i) {
    for (int j = 0; j <= i; ++j) {
      double v = -A[i][j] + (i == j ? eps : 0.0);
      for (int t = 0; t < j; ++t) v -= Lc[i][t] * Lc[j][t];
      if (i == j) {
        if (!(v > 0)) return false;
        Lc[i][i] = sqrt(v);
      } else {
        Lc[i][j] = v / Lc[j][j];
      }
    }
  }
  // (-A) d = b: the Newton ascent step d = -A^{-1} b of the concave dual
  double y[LBM_MMA_MAX_M];
  for (int i = 0; i < k; ++i) {
    double v = b[i];
    for (int t = 0; t < i; ++t) v -= Lc[i][t] * y[t];
    y[i] = v / Lc[i][i];
  }
  for (int i = k - 1; i >= 0; --i) {
    double v = y[i];
    for (int t = i + 1; t < k; ++t) v -= Lc[t][i] * d[t];
    d[i] = v / Lc[i][i];
  }
  return true;
}

// The kernels read x and dfdx directly: accept device (or managed) memory only,
// so that a host pointer is an argument error rather than a device fault.
bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" {

lbm_status lbm_mma_workspace_size(size_t n, int32_t m, size_t* bytes) {
  if (!bytes) return mma_fail(LBM_ERR_ARG, "null argument");
  if (n == 0 || m < 1 || m > LBM_MMA_MAX_M)
    return mma_fail(LBM_ERR_ARG, "need n >= 1 and 1 <= m <= %d", LBM_MMA_MAX_M);
  *bytes = mma_layout(n, m).total;
  return LBM_OK;
}

lbm_status lbm_mma_create(size_t n, int32_t m, const double* xmin, const double* xmax, void* workspace,
                          size_t workspace_bytes, void* stream, lbm_mma** out) {
  if (!out || !xmin || !xmax || !workspace) return mma_fail(LBM_ERR_ARG, "null argument");
  *out = nullptr;
  size_t need = 0;
  const lbm_status st = lbm_mma_workspace_size(n, m, &need);
  if (st != LBM_OK) return st;
  if (reinterpret_cast<uintptr_t>(workspace) % 256 || workspace_bytes < need)
    return mma_fail(LBM_ERR_WORKSPACE, "workspace must be 256-byte aligned and at least %zu bytes", need);
  std::vector<double> lo(n), hi(n);
  MMA_CUDA(cudaMemcpy(lo.data(), xmin, n * sizeof(double), cudaMemcpyDefault));
  MMA_CUDA(cudaMemcpy(hi.data(), xmax, n * sizeof(double), cudaMemcpyDefault));
  for (size_t j = 0; j < n; ++j)
    if (!(lo[j] < hi[j]) || !std::isfinite(lo[j]) || !std::isfinite(hi[j]))
      return mma_fail(LBM_ERR_ARG, "variable %zu: need finite xmin < xmax", j);
  const MmaLayout L = mma_layout(n, m);
  char* ws = static_cast<char*>(workspace);
  auto* o = new lbm_mma;
  o->dev = MmaDev{n, m,
                  reinterpret_cast<const double*>(ws + L.xmin), reinterpret_cast<const double*>(ws + L.xmax),
                  reinterpret_cast<double*>(ws + L.xold1), reinterpret_cast<double*>(ws + L.xold2),
                  reinterpret_cast<double*>(ws + L.low), reinterpret_cast<double*>(ws + L.upp),
                  reinterpret_cast<double*>(ws + L.alpha), reinterpret_cast<double*>(ws + L.beta),
                  reinterpret_cast<double*>(ws + L.p), reinterpret_cast<double*>(ws + L.q),
                  reinterpret_cast<double*>(ws + L.part)};
  o->stream = static_cast<cudaStream_t>(stream);
  const size_t want = (n + kMmaThreads - 1) / kMmaThreads;
  o->blocks = int(want < size_t(kMmaMaxBlocks) ? want : size_t(kMmaMaxBlocks));
  o->part.assign(size_t(o->blocks) * kMmaSums, 0.0);
  cudaError_t e = cudaMemcpyAsync(ws + L.xmin, lo.data(), n * sizeof(double), cudaMemcpyHostToDevice, o->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + L.xmax, hi.data(), n * sizeof(double), cudaMemcpyHostToDevice, o->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(o->stream);
  if (e != cudaSuccess) {
    delete o;
    return mma_fail(LBM_ERR_CUDA, "copying the bounds: %s", cudaGetErrorString(e));
  }
  *out = o;
  return LBM_OK;
}

lbm_status lbm_mma_update(lbm_mma* o, double* x, const double* fval, const double* dfdx, double* lam_out) {
  if (!o || !x || !fval || !dfdx) return mma_fail(LBM_ERR_ARG, "null argument");
  if (!on_device(x) || !on_device(dfdx)) return mma_fail(LBM_ERR_ARG, "x and dfdx must be device memory");
  const int m = o->dev.m;
  for (int i = 0; i <= m; ++i)
    if (!std::isfinite(fval[i])) return mma_fail(LBM_ERR_ARG, "fval[%d] is not finite", i);
  o->iter += 1;
  mma_prepare_kernel<<<o->blocks, kMmaThreads, 0, o->stream>>>(o->dev, x, dfdx, o->iter);
  MMA_CUDA(cudaGetLastError());
  double s[LBM_MMA_MAX_M + 1];
  {
    const lbm_status st = gather(o, m + 1, s);
    if (st != LBM_OK) return st;
  }
  double r[LBM_MMA_MAX_M + 1];
  for (int i = 0; i <= m; ++i) r[i] = fval[i] - s[i];

  // Projected Newton ascent on the concave dual over lam >= 0.
  double lam[LBM_MMA_MAX_M] = {};
  DualEval e{};
  {
    const lbm_status st = eval_dual(o, x, r, lam, e);
    if (st != LBM_OK) return st;
  }
  int it = 0;
  for (; it < 200; ++it) {
    bool fr[LBM_MMA_MAX_M];
    double pg = 0;
    for (int i = 0; i < m; ++i) {
      fr[i] = lam[i] > 0 || e.g[i] > 0;
      if (fr[i]) pg = fmax(pg, fabs(e.g[i]));
    }
    if (pg <= 1e-13 * e.scale) break;
    int idx[LBM_MMA_MAX_M], k = 0;
    for (int i = 0; i < m; ++i)
      if (fr[i]) idx[k++] = i;
    double A[LBM_MMA_MAX_M][LBM_MMA_MAX_M], b[LBM_MMA_MAX_M], dk[LBM_MMA_MAX_M];
    for (int a = 0; a < k; ++a) {
      b[a] = e.g[idx[a]];
      for (int c = 0; c < k; ++c) A[a][c] = e.H[idx[a]][idx[c]];
    }
    double d[LBM_MMA_MAX_M] = {};
    if (solve_neg_def(k, A, b, dk)) {
      for (int a = 0; a < k; ++a) d[idx[a]] = dk[a];
    } else {
      for (int a = 0; a < k; ++a) d[idx[a]] = b[a];   // gradient ascent when the block is singular
    }
    // Backtracking along the projected path (Armijo); stop once no step
    // ascends or the multipliers no longer change at working precision.
    double t = 1.0, step = 0.0;
    bool moved = false;
    for (int ls = 0; ls < 80; ++ls, t *= 0.5) {
      double trial[LBM_MMA_MAX_M], inc = 0;
      for (int i = 0; i < m; ++i) {
        trial[i] = fmax(0.0, lam[i] + t * d[i]);
        inc += e.g[i] * (trial[i] - lam[i]);
      }
      DualEval et{};
      const lbm_status st = eval_dual(o, x, r, trial, et);
      if (st != LBM_OK) return st;
      if (inc > 0 && et.W >= e.W + 1e-4 * inc) {
        for (int i = 0; i < m; ++i) {
          step = fmax(step, fabs(trial[i] - lam[i]));
          lam[i] = trial[i];
        }
        e = et;
        moved = true;
        break;
      }
    }
    double lmax = 0;
    for (int i = 0; i < m; ++i) lmax = fmax(lmax, fabs(lam[i]));
    if (!moved || step <= 1e-15 * (1.0 + lmax)) break;
  }
  o->last_newton = it;
  Lam L{};
  for (int i = 0; i < m; ++i) {
    L.v[i] = lam[i];
    o->last_lam[i] = lam[i];
    if (lam_out) lam_out[i] = lam[i];
  }
  mma_finish_kernel<<<o->blocks, kMmaThreads, 0, o->stream>>>(o->dev, x, L);
  MMA_CUDA(cudaGetLastError());
  MMA_CUDA(cudaStreamSynchronize(o->stream));
  return LBM_OK;
}

lbm_status lbm_mma_destroy(lbm_mma* o) {
  delete o;
  return LBM_OK;
}

}  // extern "C"
