// Design pre-processing of Sec. 3.3: a linear density filter of radius r over
// the design box and the Heaviside projection of Wang et al. (2011), plus the
// chain rule that carries dJ/dgamma back to the raw design variables.
//
//   x~_i  = sum_j w_ij x_j / W_i,  w_ij = max(0, r - |x_i - x_j|),  W_i = sum_j w_ij
//           (i, j inside the design box; outside it x~ = x)
//   gamma = H(x~) = (tanh(b eta) + tanh(b (x~ - eta))) / (tanh(b eta) + tanh(b (1 - eta)))
//   dJ/dx_j = sum_i w_ij H'(x~_i) dJ/dgamma_i / W_i      (j inside the box)
//
// These run once per design update, not per time step, so they are written
// plainly in FP64: one thread per node gathers its window.
#pragma once

#include <cstdint>

namespace lbm {

struct FilterGeo {
  int nx, ny, nz;
  int box[6];          // x0, x1, y0, y1, z0, z1 (half-open)
  int R;               // ceil(radius)
  double radius, beta, eta;
  int d3;              // 1: the window extends in z
};

__device__ __forceinline__ bool in_box(const FilterGeo& f, int x, int y, int z) {
  return x >= f.box[0] && x < f.box[1] && y >= f.box[2] && y < f.box[3] && z >= f.box[4] && z < f.box[5];
}

__device__ __forceinline__ double proj_den(const FilterGeo& f) {
  return tanh(f.beta * f.eta) + tanh(f.beta * (1.0 - f.eta));
}

// gamma = H(filter(x)) inside the box, x outside; also stores x~ and W_i.
__global__ void filter_project_kernel(const float* __restrict__ x, float* __restrict__ gamma, double* __restrict__ xf,
                                      double* __restrict__ wsum, FilterGeo f) {
  const long long n = (long long)f.nx * f.ny * f.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int X = int(i % f.nx), Y = int((i / f.nx) % f.ny), Z = int(i / ((long long)f.nx * f.ny));
    if (!in_box(f, X, Y, Z)) {
      gamma[i] = x[i];
      xf[i] = double(x[i]);
      wsum[i] = 1.0;
      continue;
    }
    double s = 0.0, w = 0.0;
    const int rz = f.d3 ? f.R : 0;
    for (int dz = -rz; dz <= rz; ++dz)
      for (int dy = -f.R; dy <= f.R; ++dy)
        for (int dx = -f.R; dx <= f.R; ++dx) {
          const int x2 = X + dx, y2 = Y + dy, z2 = Z + dz;
          if (!in_box(f, x2, y2, z2)) continue;
          const double wij = f.radius - sqrt(double(dx * dx + dy * dy + dz * dz));
          if (wij <= 0.0) continue;
          s += wij * double(x[x2 + (long long)f.nx * (y2 + (long long)f.ny * z2)]);
          w += wij;
        }
    const double v = s / w;
    xf[i] = v;
    wsum[i] = w;
    gamma[i] = float((tanh(f.beta * f.eta) + tanh(f.beta * (v - f.eta))) / proj_den(f));
  }
}

// t_i = H'(x~_i) g_i / W_i inside the box (the first half of the chain rule).
__global__ void filter_adjoint_scale_kernel(const double* __restrict__ g, const double* __restrict__ xf,
                                            const double* __restrict__ wsum, double* __restrict__ t, FilterGeo f) {
  const long long n = (long long)f.nx * f.ny * f.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int X = int(i % f.nx), Y = int((i / f.nx) % f.ny), Z = int(i / ((long long)f.nx * f.ny));
    if (!in_box(f, X, Y, Z)) {
      t[i] = 0.0;
      continue;
    }
    const double th = tanh(f.beta * (xf[i] - f.eta));
    t[i] = f.beta * (1.0 - th * th) / proj_den(f) * g[i] / wsum[i];
  }
}

// dJ/dx_j = sum_i w_ij t_i inside the box, g_j outside (the filter is symmetric in w_ij).
__global__ void filter_adjoint_gather_kernel(const double* __restrict__ g, const double* __restrict__ t,
                                             double* __restrict__ out, FilterGeo f) {
  const long long n = (long long)f.nx * f.ny * f.nz;
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
    const int X = int(j % f.nx), Y = int((j / f.nx) % f.ny), Z = int(j / ((long long)f.nx * f.ny));
    if (!in_box(f, X, Y, Z)) {
      out[j] = g[j];
      continue;
    }
    double s = 0.0;
    const int rz = f.d3 ? f.R : 0;
    for (int dz = -rz; dz <= rz; ++dz)
      for (int dy = -f.R; dy <= f.R; ++dy)
        for (int dx = -f.R; dx <= f.R; ++dx) {
          const int x2 = X + dx, y2 = Y + dy, z2 = Z + dz;
          if (!in_box(f, x2, y2, z2)) continue;
          const double wij = f.radius - sqrt(double(dx * dx + dy * dy + dz * dz));
          if (wij <= 0.0) continue;
          s += wij * t[x2 + (long long)f.nx * (y2 + (long long)f.ny * z2)];
        }
    out[j] = s;
  }
}

// Volume fraction of Sec. 3.3, V = (1/n_D) sum_{i in D} (1 - phi_i) = mean gamma
// over the design box: per-block sums of gamma (FP64) over the box nodes,
// added by the host in block order.
constexpr int kVolThreads = 256;
__global__ void __launch_bounds__(kVolThreads) design_volume_kernel(const float* __restrict__ gamma, int nx, int ny,
                                                                    int x0, int x1, int y0, int y1, int z0, int z1,
                                                                    double* __restrict__ part) {
  const long long bx = x1 - x0, by = y1 - y0, cells = bx * by * (long long)(z1 - z0);
  double s = 0.0;
  for (long long k = blockIdx.x * (long long)kVolThreads + threadIdx.x; k < cells;
       k += (long long)gridDim.x * kVolThreads) {
    const long long X = x0 + k % bx, Y = y0 + (k / bx) % by, Z = z0 + k / (bx * by);
    s += double(gamma[X + nx * (Y + (long long)ny * Z)]);
  }
  __shared__ double w[kVolThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kVolThreads / 32; ++k) t += w[k];
    part[blockIdx.x] = t;
  }
}

}  // namespace lbm
