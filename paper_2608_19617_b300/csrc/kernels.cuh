// Device code of the windowed regularized LBM-LES and its discrete adjoint.
//
// Storage: populations are kept shifted by their rest weights, p~_a = p_a - w_a,
// in structure-of-arrays layout [Q][N] (x fastest).  Near the rest state the
// shifted values are small, so FP32 keeps the non-equilibrium part (which
// drives the collision at tau ~ 0.5) to full relative precision.  All
// formulas below are the paper's, rewritten in the shifted variables; the
// shift cancels exactly wherever it enters (w_a = w_abar, sum w c = 0,
// sum w c c = cs^2 I).
//
// One thread owns one lattice node.  A forward step pulls p^{n-1} from the
// upstream neighbours (streaming, Eq. 7), completes the boundary populations
// (Eqs. 19-21), collides (Eqs. 12-16), blends (Eq. 23) and stores p^n at its
// own node: 4Q bytes read + 4Q bytes written + 4 bytes of g per node in FP32.
// An adjoint step pulls the adjoint of p^n from the downstream neighbours
// (Eq. 36), recomputes f^n from p^{n-1}, applies the transposed local
// Jacobian in moment space (Eq. 35) and the transposed boundary rule
// (Eqs. 37-39), and stores the result at its own node.
//
// Two identities keep the per-direction work small.  The regularized
// collision (Eq. 16) only carries Hermite moments up to second order, so
// h_a = w_a (H0 + H1.c_a + c_a.H2.c_a), and the partial bounce-back of Eq. 23,
// p = (1-g) h + g h_abar, keeps the even part and scales the odd part H1 by
// (1 - 2g).  Hence p~_a = w_a (a0 + b m.c_a + 4.5 c_a.X.c_a) with two scalars,
// one vector and one symmetric tensor per node; the adjoint of the blend scales
// the first adjoint moment by (1 - 2g); and the sensitivity term of Eq. 40,
// sum_a a_a (h_abar - h_a), equals -6 m . sum_a w_a c_a a_a.
//
// Boundary nodes take out-of-line slow paths so that the interior code stays
// small (instruction-cache pressure), and indices are 32-bit (Q N < 2^31 is
// checked on the host).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lattice.cuh"

namespace lbm {

enum : uint8_t { FLUID = 0, WALL = 1, INLET = 2, OUTLET_P = 3, OUTLET_ZG = 4 };
enum { OBJ_DISS = 0, OBJ_VEL = 1, OBJ_PRES = 2, OBJ_DRAG = 3 };
enum { MON_DRAG = 0, MON_OBJ = 1 };

constexpr int kBlock = 128;   // threads per block (one row segment of 128 nodes)

struct Geo {
  int nx, ny, nz;
  int px, py, pz;             // periodic flags
  unsigned n;                 // nx*ny*nz
  unsigned sy, sz;            // strides of y and z
};

template <class R>
struct Phys {
  R tau;       // molecular relaxation time
  R c2;        // (C_s * filter width)^2
  R rho_out;   // outlet density
};

// Objective description (sampling instants only).
template <class R>
struct Obj {
  int kind;
  int mon;               // monitored quantity
  R uref[3];
  int box[6];            // weights read only inside
  R ws;                  // sampling weight dW/|W| (adjoint source scale)
};

// Window-end results.
// One block's compensated window sums: (j sum, j compensation, monitor sum,
// monitor compensation); 32-byte aligned for one vector access.
struct alignas(32) Sums {
  double x, y, z, w;
};

struct WindowAcc {
  double jmean, mmean, mprev, ratio;
  int has_prev, converged, nonfinite;
};

template <class T>
__device__ __forceinline__ T cs2() { return T(1.0 / 3.0); }

// Programmatic dependent launch: a step kernel launched with programmatic
// stream serialization may start before its predecessor finishes; it waits
// here for the predecessor's completion (and memory) before touching any data,
// then lets its own successor begin launching.  Without the launch attribute
// both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// Is step `step` of a window a sampling instant: every dW-th step from the
// first sampled step s0 on (Eq. 42; s0 > 0 only for the full-time run).
__host__ __device__ __forceinline__ bool sampled_step(int step, int s0, int dW) {
  return dW > 0 && step >= s0 && (step - s0) % dW == 0;
}

__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x)) c += (s - t) + x; else c += (x - t) + s;
  s = t;
}

// Neighbour (x+dx, y+dy, z+dz) with periodic wrap; false if outside.  Host
// and device code, so that the host can check the face gathers' indices.
HD bool neighbour(const Geo& g, int x, int y, int z, int dx, int dy, int dz,
                                          unsigned& j) {
  int X = x + dx, Y = y + dy, Z = z + dz;
  if (X < 0 || X >= g.nx) { if (!g.px) return false; X = (X + g.nx) % g.nx; }
  if (Y < 0 || Y >= g.ny) { if (!g.py) return false; Y = (Y + g.ny) % g.ny; }
  if (Z < 0 || Z >= g.nz) { if (!g.pz) return false; Z = (Z + g.nz) % g.nz; }
  j = unsigned(X) + unsigned(Y) * g.sy + unsigned(Z) * g.sz;
  return true;
}

// Explicitly rounded products and fused multiply-adds.  The per-node forward
// arithmetic (boundary rules, moments, closure, blend,
// samples) is written with them, in a
// fixed order, wherever a product meets a sum: the compiler then has no
// contraction left to choose, and every kernel that inlines it (interior,
// face, the step that writes a moment checkpoint, the checkpoint decoder)
// computes the same bits.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class L>
__device__ __forceinline__ bool on_face(const Geo& g, int x, int y, int z) {
  bool f = (x == 0) | (x == g.nx - 1) | (y == 0) | (y == g.ny - 1);
  if (L::D == 3) f |= (z == 0) | (z == g.nz - 1);
  return f;
}

template <class L>
__device__ __forceinline__ int offset(const Geo& g, int a) {
  return L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz);
}

// ---------------------------------------------------------------------------
// Row geometry.  The step kernels run over whole lattice rows along x, in
// blocks of kBlock threads starting at x = 0, so that every warp's loads and
// stores cover whole, aligned 128-byte lines.  The block that covers nodes
// bx kBlock .. of row (y, z) keeps its sample partials in slot
// bx + ceil(nx / kBlock) (y + ny z), whichever kernel runs it, so the rows of
// one D2Q9 batch slice own consecutive slots.  Every node pulls with
// branch-free index arithmetic: a link from outside the domain reads the node
// itself (an in-row, don't-care value), a periodic axis wraps; the nodes with
// such links (on a bounded face) then replace them by their boundary rule.
// These functions are host and device code so that the host can check every
// index a launch forms.
// ---------------------------------------------------------------------------

// Sample slot of the block covering nodes bx kBlock .. of row (y, z).
HD unsigned row_slot(const Geo& g, int bx, int y, int z) {
  return unsigned(bx) + unsigned((g.nx + kBlock - 1) / kBlock) * (unsigned(y) + unsigned(g.ny) * unsigned(z));
}

// Index the pull of direction a reads for node i at (x, y, z) (Eq. 7):
// i - c_a with periodic wrap, or i itself for a link from outside the domain.
// PER = false: the lattice has no periodic axis (the wrap arithmetic compiles out).
template <class L, bool PER = true>
HD unsigned node_src(const Geo& g, int x, int y, int z, unsigned i, int a) {
  unsigned j = i - unsigned(L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz));
  bool out = false;
  if (L::cx(a) > 0 && x == 0) { if (PER && g.px) j += unsigned(g.nx); else out = true; }
  if (L::cx(a) < 0 && x == g.nx - 1) { if (PER && g.px) j -= unsigned(g.nx); else out = true; }
  if (L::cy(a) > 0 && y == 0) { if (PER && g.py) j += g.sz; else out = true; }
  if (L::cy(a) < 0 && y == g.ny - 1) { if (PER && g.py) j -= g.sz; else out = true; }
  if (L::cz(a) > 0 && z == 0) { if (PER && g.pz) j += g.n; else out = true; }
  if (L::cz(a) < 0 && z == g.nz - 1) { if (PER && g.pz) j -= g.n; else out = true; }
  return out ? i : j;
}

// Index the adjoint pull of direction a reads for node i (Eq. 36): i + c_a
// with periodic wrap; kNone for a link that leaves the domain (adjoint 0).
constexpr unsigned kNone = 0xffffffffu;
template <class L, bool PER = true>
HD unsigned node_dst(const Geo& g, int x, int y, int z, unsigned i, int a) {
  unsigned j = i + unsigned(L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz));
  bool out = false;
  if (L::cx(a) < 0 && x == 0) { if (PER && g.px) j += unsigned(g.nx); else out = true; }
  if (L::cx(a) > 0 && x == g.nx - 1) { if (PER && g.px) j -= unsigned(g.nx); else out = true; }
  if (L::cy(a) < 0 && y == 0) { if (PER && g.py) j += g.sz; else out = true; }
  if (L::cy(a) > 0 && y == g.ny - 1) { if (PER && g.py) j -= g.sz; else out = true; }
  if (L::cz(a) < 0 && z == 0) { if (PER && g.pz) j += g.n; else out = true; }
  if (L::cz(a) > 0 && z == g.nz - 1) { if (PER && g.pz) j -= g.n; else out = true; }
  return out ? kNone : j;
}

// Links of node (x, y, z) that come from outside the domain (bounded axes).
template <class L, bool PER = true>
HD unsigned node_unknowns(const Geo& g, int x, int y, int z) {
  unsigned m = 0;
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    const bool out = (!(PER && g.px) && ((L::cx(a) > 0 && x == 0) || (L::cx(a) < 0 && x == g.nx - 1))) ||
                     (!(PER && g.py) && ((L::cy(a) > 0 && y == 0) || (L::cy(a) < 0 && y == g.ny - 1))) ||
                     (!(PER && g.pz) && ((L::cz(a) > 0 && z == 0) || (L::cz(a) < 0 && z == g.nz - 1)));
    if (out) m |= 1u << a;
  }
  return m;
}

// Node (x, y + dy, z + dz) on the same x plane (periodic wrap), or kNone
// outside: where the adjoint looks for zero-gradient outlet nodes that
// copied one of this node's populations.
HD unsigned same_x_neighbour(const Geo& g, int y, int z, unsigned i, int dy, int dz) {
  int Y = y + dy, Z = z + dz;
  unsigned j = i + unsigned(dy * int(g.sy) + dz * int(g.sz));
  if (Y < 0) { if (!g.py) return kNone; j += g.sz; }
  if (Y >= g.ny) { if (!g.py) return kNone; j -= g.sz; }
  if (Z < 0) { if (!g.pz) return kNone; j += g.n; }
  if (Z >= g.nz) { if (!g.pz) return kNone; j -= g.n; }
  return j;
}

// Rows (y, z) of the x = 0 (face 0) and x = nx-1 (face 1) planes whose node
// may have lent a population to a zero-gradient outlet node on the same
// face (same_x_neighbour): the bounding box of that face's outlet nodes grown
// by one node, the whole axis where it is periodic; empty (y0 > y1) without
// outlets.  Only those rows run the adjoint's pull-back of the copies.
struct ZgRows {
  int f[2][4];   // per face: y0, y1, z0, z1 (inclusive)
};

inline ZgRows zg_rows(const uint8_t* cls, const Geo& g) {
  ZgRows r;
  for (int f = 0; f < 2; ++f) {
    r.f[f][0] = r.f[f][2] = 1 << 30;
    r.f[f][1] = r.f[f][3] = -(1 << 30);
    const int x = f == 0 ? 0 : g.nx - 1;
    if (f == 1 && g.nx == 1) continue;
    for (int z = 0; z < g.nz; ++z)
      for (int y = 0; y < g.ny; ++y) {
        if (cls[size_t(x) + size_t(g.nx) * (size_t(y) + size_t(g.ny) * size_t(z))] != OUTLET_ZG) continue;
        if (y < r.f[f][0]) r.f[f][0] = y;
        if (y > r.f[f][1]) r.f[f][1] = y;
        if (z < r.f[f][2]) r.f[f][2] = z;
        if (z > r.f[f][3]) r.f[f][3] = z;
      }
    if (r.f[f][0] > r.f[f][1]) continue;
    r.f[f][0] = g.py ? 0 : r.f[f][0] - 1;
    r.f[f][1] = g.py ? g.ny - 1 : r.f[f][1] + 1;
    r.f[f][2] = g.pz ? 0 : r.f[f][2] - 1;
    r.f[f][3] = g.pz ? g.nz - 1 : r.f[f][3] + 1;
  }
  return r;
}

// Node (x, y, z) lies on an x face within that face's ZgRows box.
HD bool zg_row(const ZgRows& r, const Geo& g, int x, int y, int z) {
  const int f = x == 0 ? 0 : (x == g.nx - 1 ? 1 : -1);
  return f >= 0 && y >= r.f[f][0] && y <= r.f[f][1] && z >= r.f[f][2] && z <= r.f[f][3];
}

// The forward step runs two kernels on disjoint rows: the inner rows
// (1 <= y <= ny-2 and, in 3D, 1 <= z <= nz-2; every slice of a D2Q9 batch),
// whose only links from outside the domain are those of the x = 0 and
// x = nx-1 nodes on a bounded x axis, and the face rows (on a y or z face).
// The inner-row kernel keeps the x-face completion to those links, which
// keeps its registers, and so its occupancy, at those of a plain pull.
// Inner rows per z (D3Q19: z interior; D2Q9: every slice) and z of inner row block rz.
template <class L>
HD int inner_rows_y(const Geo& g) { return g.ny > 2 ? g.ny - 2 : 0; }
template <class L>
HD int inner_rows_z(const Geo& g) { return L::D == 3 ? (g.nz > 2 ? g.nz - 2 : 0) : g.nz; }

// Face rows: per z (all z) the rows y = 0 and y = ny-1 (one if ny == 1), then
// in 3D for the inner y the rows z = 0 and z = nz-1 (one if nz == 1).  For a
// D2Q9 batch the face rows of slice z are rows fy z .. fy z + fy - 1.
template <class L>
HD int face_rows(const Geo& g) {
  const int fy = g.ny >= 2 ? 2 : 1, fz = g.nz >= 2 ? 2 : 1;
  return fy * g.nz + (L::D == 3 ? fz * inner_rows_y<L>(g) : 0);
}

template <class L>
HD void face_row_yz(const Geo& g, int r, int& y, int& z) {
  const int fy = g.ny >= 2 ? 2 : 1, fz = g.nz >= 2 ? 2 : 1;
  if (r < fy * g.nz) {
    z = r / fy;
    y = (r % fy) ? g.ny - 1 : 0;
  } else {
    r -= fy * g.nz;
    y = 1 + r / fz;
    z = (r % fz) ? g.nz - 1 : 0;
  }
}

// Index the pull of direction a reads for inner-row node i at x (Eq. 7):
// i - c_a, except for a link from outside the domain (the node itself) and
// across a periodic x axis (wrapped).
template <class L>
HD unsigned row_src(const Geo& g, int x, unsigned i, int a) {
  unsigned j = i - unsigned(L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz));
  if (L::cx(a) > 0 && x == 0) j = g.px ? j + unsigned(g.nx) : i;
  if (L::cx(a) < 0 && x == g.nx - 1) j = g.px ? j - unsigned(g.nx) : i;
  return j;
}

// Links of an inner-row node that come from outside a bounded x axis.
template <class L>
HD unsigned row_unknowns(const Geo& g, int x) {
  if (g.px) return 0u;
  unsigned m = 0;
  for (int a = 0; a < L::Q; ++a)
    if ((x == 0 && L::cx(a) > 0) || (x == g.nx - 1 && L::cx(a) < 0)) m |= 1u << a;
  return m;
}

// Boundary rules of Eqs. 19-21 (and the 3D velocity inlet) on the unknown
// populations flagged in mask, in shifted form.
template <class L, class R>
__device__ __forceinline__ void apply_rules(R (&f)[L::Q], unsigned mask, uint8_t cls, R u0, R rho_out) {
  if (!mask) return;
  if (cls == WALL) {
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
      if (mask & (1u << a)) f[a] = (mask & (1u << L::opp(a))) ? R(0) : f[L::opp(a)];
  } else if (cls == INLET) {
    if (L::Q == 9) {
      // Zou-He velocity inlet, Eq. 20, in shifted form (w1=w3, w5=w7, w2=w4).
      const R s = fma_rn(R(2), f[3] + f[6] + f[7], f[0] + f[2] + f[4]);
      const R rho = (R(1) + s) / (R(1) - u0);
      const R ru = mul_rn(rho, u0);
      f[1] = fma_rn(R(2.0 / 3.0), ru, f[3]);
      f[5] = fma_rn(R(1.0 / 6.0), ru, fma_rn(R(0.5), f[4] - f[2], f[7]));
      f[8] = fma_rn(R(1.0 / 6.0), ru, fma_rn(R(0.5), f[2] - f[4], f[6]));
    } else {
      // Moving-wall bounce-back with rho0 = 1: f_a = f_abar + 2 w_a c_a.u / cs^2.
#pragma unroll
      for (int a = 0; a < L::Q; ++a)
        if (mask & (1u << a)) f[a] = fma_rn(R(6.0 * L::w(a) * L::cx(a)), u0, f[L::opp(a)]);
    }
  } else if (cls == OUTLET_P) {
    // Zou-He pressure outlet, Eq. 21 (D2Q9): u = (1 + s)/rho0 - 1 in shifted form.
    const R s = fma_rn(R(2), f[1] + f[5] + f[8], f[0] + f[2] + f[4]);
    const R ux = (R(1) + s) / rho_out - R(1);
    const R ru = mul_rn(rho_out, ux);
    f[3] = fma_rn(R(-2.0 / 3.0), ru, f[1]);
    f[6] = fma_rn(R(-1.0 / 6.0), ru, fma_rn(R(0.5), f[4] - f[2], f[8]));
    f[7] = fma_rn(R(-1.0 / 6.0), ru, fma_rn(R(0.5), f[2] - f[4], f[5]));
  }
}

// ---------------------------------------------------------------------------
// Streaming with boundary completion on a domain face: f^n at node (x,y,z)
// from p^{n-1}, addresses from the geometry (no face table).  Returns the
// mask of links that came from outside the domain.
// ---------------------------------------------------------------------------
template <class L, class R>
__device__ __forceinline__ unsigned gather_geo(const R* __restrict__ P, const Geo& g, int x, int y, int z,
                                               uint8_t cls, R u0, R rho_out, R (&f)[L::Q]) {
  unsigned unk = 0;
#pragma unroll
  for (int a = 0; a < L::Q; ++a) {
    unsigned j;
    if (neighbour(g, x, y, z, -L::cx(a), -L::cy(a), -L::cz(a), j)) {
      f[a] = P[a * g.n + j];
    } else {
      f[a] = R(0);
      unk |= 1u << a;
    }
  }
  if (!unk) return 0;
  if (cls == OUTLET_ZG) {
    // Unknown f_a(i) = f_a(i + n_in) after streaming = p_a(i + n_in - c_a).
    const int xn = (x == g.nx - 1) ? x - 1 : x + 1;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      if (unk & (1u << a)) {
        unsigned j = 0;
        neighbour(g, xn, y, z, -L::cx(a), -L::cy(a), -L::cz(a), j);   // inside (validated on the host)
        f[a] = P[a * g.n + j];
      }
    }
  } else {
    apply_rules<L, R>(f, unk, cls, u0, rho_out);   // Eqs. 19-21
  }
  return unk;
}

// Out-of-line copy for kernels whose face nodes are rare (no-allocation path).
template <class L, class R>
__device__ __noinline__ unsigned gather_face(const R* __restrict__ P, const Geo& g, int x, int y, int z,
                                             uint8_t cls, R u0, R rho_out, R* f) {
  R t[L::Q];
  const unsigned unk = gather_geo<L, R>(P, g, x, y, z, cls, u0, rho_out, t);
#pragma unroll
  for (int a = 0; a < L::Q; ++a) f[a] = t[a];
  return unk;
}

template <class L, class R>
__device__ __forceinline__ unsigned gather(const R* __restrict__ P, const Geo& g, int x, int y, int z, unsigned i,
                                           bool face, uint8_t cls, R u0, R rho_out, R (&f)[L::Q]) {
  if (!face) {
#pragma unroll
    for (int a = 0; a < L::Q; ++a) f[a] = P[a * g.n + i - offset<L>(g, a)];
    return 0;
  }
  R t[L::Q];
  const unsigned unk = gather_face<L, R>(P, g, x, y, z, cls, u0, rho_out, t);
#pragma unroll
  for (int a = 0; a < L::Q; ++a) f[a] = t[a];
  return unk;
}

// ---------------------------------------------------------------------------
// Moments and the regularized LES collision (Eqs. 5, 12-16), shifted form.
// ---------------------------------------------------------------------------
template <class L, class R>
struct Mom {
  R rt, rho, inv;          // rho - 1, rho, 1/rho
  R m[3], u[3];            // momentum, velocity
  R pi[6];                 // Pi_xx, Pi_yy, Pi_zz, Pi_xy, Pi_xz, Pi_yz  (Eq. 13)
  R pp;                    // Pi:Pi
  R pn;                    // |Pi| = sqrt(2 Pi:Pi)
  R s;                     // sqrt(tau^2 + 2 C^2 |Pi| / (rho cs^4))
  R te, om;                // tau_eff (Eq. 14), 1 - 1/tau_eff
};

// Add v into an accumulator; the first contribution sets it (no addition to
// zero).  In the fully unrolled direction loops `set` is a compile-time
// constant, so the branch folds away.
template <class R>
__device__ __forceinline__ void acc_add(R& x, bool& set, R v) {
  if (set) x += v; else { x = v; set = true; }
}

// Zeroth, first and second moments of a population-shaped array, each
// weighted by wt(a) (1 for f, w_a for adjoints; entries of the second moment
// xx, yy, zz, xy, xz, yz).  Opposite directions a, abar (a < abar) enter as
// s = f_a + f_abar and d = f_a - f_abar (w_a = w_abar): the even moments are
// sums of s, the odd ones signed sums of d, added in a fixed order.
template <class L, class R, bool W>
__device__ __forceinline__ void raw_moments(const R (&f)[L::Q], R& m0, R (&m1)[3], R (&m2)[6]) {
  R rt = W ? mul_rn(R(L::w(0)), f[0]) : f[0];
  R m[3] = {R(0), R(0), R(0)}, q[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  bool ms[3] = {false, false, false}, qs[6] = {false, false, false, false, false, false};
#pragma unroll
  for (int a = 1; a < L::Q; ++a) {
    const int b = L::opp(a);
    if (b < a) continue;
    R s = f[a] + f[b], d = f[a] - f[b];
    if (W) {
      s = mul_rn(R(L::w(a)), s);
      d = mul_rn(R(L::w(a)), d);
    }
    const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
    rt += s;
    if (cx) acc_add(m[0], ms[0], cx > 0 ? d : -d);
    if (cy) acc_add(m[1], ms[1], cy > 0 ? d : -d);
    if (cz) acc_add(m[2], ms[2], cz > 0 ? d : -d);
    if (cx) acc_add(q[0], qs[0], s);
    if (cy) acc_add(q[1], qs[1], s);
    if (cz) acc_add(q[2], qs[2], s);
    if (cx * cy) acc_add(q[3], qs[3], cx * cy > 0 ? s : -s);
    if (cx * cz) acc_add(q[4], qs[4], cx * cz > 0 ? s : -s);
    if (cy * cz) acc_add(q[5], qs[5], cy * cz > 0 ? s : -s);
  }
  m0 = rt;
#pragma unroll
  for (int k = 0; k < 3; ++k) m1[k] = m[k];
#pragma unroll
  for (int k = 0; k < 6; ++k) m2[k] = q[k];
}

template <class L, class R>
__device__ __forceinline__ void moments_from_raw(R rt, const R (&m)[3], const R (&m2)[6], const Phys<R>& ph,
                                                 Mom<L, R>& M);

template <class L, class R>
__device__ __forceinline__ void moments(const R (&f)[L::Q], const Phys<R>& ph, Mom<L, R>& M) {
  R rt, m[3], m2[6];
  raw_moments<L, R, false>(f, rt, m, m2);
  moments_from_raw<L, R>(rt, m, m2, ph, M);
}

// Density, velocity, Pi (Eq. 13), |Pi| and tau_eff (Eq. 14) from the raw
// moments of the pulled populations.
template <class L, class R>
__device__ __forceinline__ void moments_from_raw(R rt, const R (&m)[3], const R (&m2)[6], const Phys<R>& ph,
                                                 Mom<L, R>& M) {
  M.rt = rt;
  M.rho = R(1) + rt;
  M.inv = R(1) / M.rho;
  M.m[0] = m[0]; M.m[1] = m[1]; M.m[2] = L::D == 3 ? m[2] : R(0);
  M.u[0] = mul_rn(m[0], M.inv); M.u[1] = mul_rn(m[1], M.inv); M.u[2] = mul_rn(M.m[2], M.inv);
  // Pi = M2 - rho cs^2 I - m m^T / rho; with shifted moments M2~ = M2 - cs^2 I.
  const R c = cs2<R>();
  M.pi[0] = fma_rn(-m[0], M.u[0], fma_rn(-rt, c, m2[0]));
  M.pi[1] = fma_rn(-m[1], M.u[1], fma_rn(-rt, c, m2[1]));
  M.pi[2] = (L::D == 3) ? fma_rn(-M.m[2], M.u[2], fma_rn(-rt, c, m2[2])) : R(0);
  M.pi[3] = fma_rn(-m[0], M.u[1], m2[3]);
  M.pi[4] = (L::D == 3) ? fma_rn(-m[0], M.u[2], m2[4]) : R(0);
  M.pi[5] = (L::D == 3) ? fma_rn(-m[1], M.u[2], m2[5]) : R(0);
  const R diag = fma_rn(M.pi[2], M.pi[2], fma_rn(M.pi[1], M.pi[1], mul_rn(M.pi[0], M.pi[0])));
  const R off = fma_rn(M.pi[5], M.pi[5], fma_rn(M.pi[4], M.pi[4], mul_rn(M.pi[3], M.pi[3])));
  M.pp = fma_rn(R(2), off, diag);
  M.pn = sqrt(mul_rn(R(2), M.pp));
  // Eq. 14: 2 C^2 |Pi| / (rho cs^4) = 18 C^2 |Pi| / rho.
  M.s = sqrt(fma_rn(mul_rn(mul_rn(R(18), ph.c2), M.pn), M.inv, mul_rn(ph.tau, ph.tau)));
  M.te = mul_rn(R(0.5), ph.tau + M.s);
  M.om = R(1) - R(1) / M.te;
}

// b_a = s0 + s1.c_a + c_a.S2.c_a for every direction a (S2 symmetric,
// entries xx, yy, zz, xy, xz, yz).  Opposite directions share the even part
// s0 + c.S2.c and take the odd part s1.c with opposite signs.
template <class L, class R>
__device__ __forceinline__ void quad_all(R s0, const R (&s1)[3], const R (&s2)[6], R (&out)[L::Q]) {
  out[0] = s0;
#pragma unroll
  for (int a = 1; a < L::Q; ++a) {
    const int b = L::opp(a);
    if (b < a) continue;
    const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
    R e = s0;
    if (cx) e += s2[0];
    if (cy) e += s2[1];
    if (cz) e += s2[2];
    if (cx * cy) e = fma_rn(cx * cy > 0 ? R(2) : R(-2), s2[3], e);
    if (cx * cz) e = fma_rn(cx * cz > 0 ? R(2) : R(-2), s2[4], e);
    if (cy * cz) e = fma_rn(cy * cz > 0 ? R(2) : R(-2), s2[5], e);
    R o = R(0);
    bool os = false;
    if (cx) acc_add(o, os, cx > 0 ? s1[0] : -s1[0]);
    if (cy) acc_add(o, os, cy > 0 ? s1[1] : -s1[1]);
    if (cz) acc_add(o, os, cz > 0 ? s1[2] : -s1[2]);
    out[a] = e + o;
    out[b] = e - o;
  }
}

// Blended post-collision field (Eqs. 16 and 23):
//   h~_a = f^eq_a - w_a + (1 - 1/tau_eff) w_a/(2 cs^4) (c_a c_a - cs^2 I) : Pi
//        = w_a (a0 + 3 m.c_a + 4.5 c_a.X.c_a),
//   a0 = rho - 1 - 1.5 m.u - 1.5 om tr(Pi),  X = m u^T + om Pi,
// and the blend scales the odd part: p~_a = w_a (a0 + b m.c_a + 4.5 c_a.X.c_a)
// with b = 3 (1 - 2g).  Two scalars a0, b, the vector m and the symmetric X
// per node give every direction.
template <class R>
struct Blend {
  R a0, b;
  R m[3];
  R X[6];   // xx, yy, zz, xy, xz, yz
};

template <class L, class R>
__device__ __forceinline__ void blend_coefs(const Mom<L, R>& M, R g, Blend<R>& C) {
  const R tr = M.pi[0] + M.pi[1] + M.pi[2];
  const R mu = fma_rn(M.m[2], M.u[2], fma_rn(M.m[1], M.u[1], mul_rn(M.m[0], M.u[0])));
  C.a0 = fma_rn(mul_rn(R(-1.5), M.om), tr, fma_rn(R(-1.5), mu, M.rt));
  C.b = mul_rn(R(3), fma_rn(R(-2), g, R(1)));
#pragma unroll
  for (int k = 0; k < 3; ++k) C.m[k] = M.m[k];
  C.X[0] = fma_rn(M.om, M.pi[0], mul_rn(M.m[0], M.u[0]));
  C.X[1] = fma_rn(M.om, M.pi[1], mul_rn(M.m[1], M.u[1]));
  C.X[2] = fma_rn(M.om, M.pi[2], mul_rn(M.m[2], M.u[2]));
  C.X[3] = fma_rn(M.om, M.pi[3], mul_rn(M.m[0], M.u[1]));
  C.X[4] = fma_rn(M.om, M.pi[4], mul_rn(M.m[0], M.u[2]));
  C.X[5] = fma_rn(M.om, M.pi[5], mul_rn(M.m[1], M.u[2]));
}

// p~_a = w_a (a0 + b m.c_a + 4.5 c_a.X.c_a) of every direction, stored at node
// i of dst ([Q][n]).  Opposite directions share the even part a0 + 4.5 c.X.c
// (fused multiply-adds in a fixed order) and take the odd part b m.c with
// opposite signs.  Every kernel that writes or rebuilds a carried field calls
// this, so they agree bit for bit.
template <class L, class R>
__device__ __forceinline__ void blend_store(R* __restrict__ dst, unsigned n, unsigned i, const Blend<R>& C) {
  dst[i] = mul_rn(R(L::w(0)), C.a0);
#pragma unroll
  for (int a = 1; a < L::Q; ++a) {
    const int b = L::opp(a);
    if (b < a) continue;
    const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
    R e = C.a0;
    if (cx) e = fma_rn(R(4.5), C.X[0], e);
    if (cy) e = fma_rn(R(4.5), C.X[1], e);
    if (cz) e = fma_rn(R(4.5), C.X[2], e);
    if (cx * cy) e = fma_rn(cx * cy > 0 ? R(9) : R(-9), C.X[3], e);
    if (cx * cz) e = fma_rn(cx * cz > 0 ? R(9) : R(-9), C.X[4], e);
    if (cy * cz) e = fma_rn(cy * cz > 0 ? R(9) : R(-9), C.X[5], e);
    R mc = R(0);
    bool ms = false;
    if (cx) acc_add(mc, ms, cx > 0 ? C.m[0] : -C.m[0]);
    if (cy) acc_add(mc, ms, cy > 0 ? C.m[1] : -C.m[1]);
    if (cz) acc_add(mc, ms, cz > 0 ? C.m[2] : -C.m[2]);
    const R o = mul_rn(C.b, mc);
    dst[unsigned(a) * n + i] = mul_rn(R(L::w(a)), e + o);
    dst[unsigned(b) * n + i] = mul_rn(R(L::w(a)), e - o);
  }
}

// ---------------------------------------------------------------------------
// Block reduction of two values in the working precision; result in thread 0.
// ---------------------------------------------------------------------------
template <class R, int NT = kBlock>
__device__ __forceinline__ void block_sum2(R& a, R& b) {
  __shared__ R sa[NT / 32], sb[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sa[warp] = a; sb[warp] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = sa[0];
    b = sb[0];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) { a += sa[k]; b += sb[k]; }
  }
}

// Each block keeps its own compensated FP64 window sums (j and the monitor) in
// blk[4 b .. 4 b + 3]; thread 0 adds the block's sample.  No atomics, no
// cross-block step: the window-end kernel reduces the blocks in a fixed order.
__device__ __forceinline__ void sample_commit(double bj, double bm, double* blk, unsigned bid) {
  if (threadIdx.x == 0) {
    Sums a = reinterpret_cast<Sums*>(blk)[bid];
    neumaier(a.x, a.y, bj);
    neumaier(a.z, a.w, bm);
    reinterpret_cast<Sums*>(blk)[bid] = a;
  }
}

__device__ __forceinline__ void sample_commit(double bj, double bm, double* blk) {
  sample_commit(bj, bm, blk, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// The per-step kernels leave each sampled step's block partials (j, monitor)
// in the working precision in a ring of slots, one store by thread 0 and no
// read, so a block's last warp retires as soon as its reduction is done.
// sample_fold_kernel then adds them into the blocks' FP64 (sum, compensation)
// window sums: one thread per block and quantity sums its slots in step order
// in FP64 (each partial converts exactly; 32 additions round at 2^-53
// relative) and adds that into the pair with one Neumaier step.  FP64
// arithmetic is scarce on B300 (about 1/64 of the FP32 rate), so the fold
// keeps it to one addition per slot.
template <class R>
__device__ __forceinline__ void ring_store(R bj, R bm, R* ring, size_t slot) {
  if (threadIdx.x == 0) {
    if constexpr (sizeof(R) == 4) reinterpret_cast<float2*>(ring)[slot] = make_float2(bj, bm);
    else reinterpret_cast<double2*>(ring)[slot] = make_double2(bj, bm);
  }
}

template <class R>
__global__ void sample_fold_kernel(const R* __restrict__ ring, int count, unsigned nblk, double* __restrict__ blk) {
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < 2u * nblk; t += gridDim.x * blockDim.x) {
    // t = 2 b + q: block b, quantity q (0: objective, 1: monitor); ring[2 (r nblk + b) + q]
    double s = 0.0;
    for (int r = 0; r < count; ++r) s += double(ring[2 * size_t(r) * nblk + t]);
    double* pair = blk + 2 * size_t(t);   // Sums: (j sum, j comp, monitor sum, monitor comp)
    neumaier(pair[0], pair[1], s);
  }
}

// ---------------------------------------------------------------------------
// Forward step.
// ---------------------------------------------------------------------------
template <class R>
struct FwdArgs {
  const R* __restrict__ src;     // p^{n-1}
  R* __restrict__ dst;           // p^n
  const R* __restrict__ gfield;  // g(phi) per node
  const uint8_t* __restrict__ cls;
  const float* __restrict__ uin; // [nz][ny]
  const float* __restrict__ wobj;
  Geo geo;
  Phys<R> ph;
  Obj<R> obj;
  int sample;                    // 0, or at a sampling instant 1 + the ring slot of its block partials
  R* ring;                       // [slots][nblk][2] block partials of the sampled steps
  unsigned nblk;                 // blocks of one step (interior + face kernel)
  double* blk;                   // per-block FP64 window sums (4 doubles per block; no-allocation kernel only)
  int* nonfinite;
  R* mom;                        // non-null: also store the step's collision coefficients (moment checkpoint)
};

template <class L, class R>
__device__ __forceinline__ R local_objective(const Mom<L, R>& M, const Obj<R>& ob, R gi) {
  switch (ob.kind) {
    case OBJ_DISS:
      return mul_rn(mul_rn(mul_rn(R(1.5), M.te - R(0.5)), M.pp), M.inv) / mul_rn(M.te, M.te);
    case OBJ_VEL: {
      const R dx = M.u[0] - ob.uref[0], dy = M.u[1] - ob.uref[1], dz = M.u[2] - ob.uref[2];
      const R v = fma_rn(dy, dy, mul_rn(dx, dx));
      return L::D == 3 ? fma_rn(dz, dz, v) : v;
    }
    case OBJ_PRES: return mul_rn(cs2<R>(), M.rt);   // constant cs^2 sum(w) added at the window end
    default: return mul_rn(mul_rn(R(-2), gi), M.m[0]);   // sum_a c_xa F_a = -2 g m_x
  }
}

// The per-step fields of a step.
template <class R>
struct FwdStep {
  const R* src;   // p^{n-1}
  R* dst;         // p^n
  int sample;
  R* mom;         // non-null: moment checkpoint of p^n (mom_coefs<L>() planes of n values)
};

// Moment checkpoints.  The carried field is p~ = blend_store(C) at
// every node (interior and face alike), so the coefficients C as the step
// computed them regenerate p~ exactly: a0, b, m (D values) and X (D(D+1)/2),
// 7 planes in 2D and 11 in 3D instead of Q.
template <class L>
__host__ __device__ constexpr int mom_coefs() { return L::D == 2 ? 7 : 11; }

template <class L, class R>
__device__ __forceinline__ void store_coefs(R* mom, unsigned n, unsigned i, const Blend<R>& C) {
  mom[i] = C.a0;
  mom[n + i] = C.b;
  if (L::D == 2) {
    mom[2 * n + i] = C.m[0];
    mom[3 * n + i] = C.m[1];
    mom[4 * n + i] = C.X[0];
    mom[5 * n + i] = C.X[1];
    mom[6 * n + i] = C.X[3];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) mom[(2 + k) * n + i] = C.m[k];
#pragma unroll
    for (int k = 0; k < 6; ++k) mom[(5 + k) * n + i] = C.X[k];
  }
}

template <class L, class R>
__device__ __forceinline__ void load_coefs(const R* __restrict__ mom, unsigned n, unsigned i, Blend<R>& C) {
  C.a0 = mom[i];
  C.b = mom[n + i];
  C.m[2] = R(0);
  C.X[2] = C.X[4] = C.X[5] = R(0);
  if (L::D == 2) {
    C.m[0] = mom[2 * n + i];
    C.m[1] = mom[3 * n + i];
    C.X[0] = mom[4 * n + i];
    C.X[1] = mom[5 * n + i];
    C.X[3] = mom[6 * n + i];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) C.m[k] = mom[(2 + k) * n + i];
#pragma unroll
    for (int k = 0; k < 6; ++k) C.X[k] = mom[(5 + k) * n + i];
  }
}

// Collision, blend, store and sample of one node whose pulled populations f
// are loaded (Eqs. 12-16, 23, 24-25); a sampled step adds the node's
// objective and monitor terms to bj, bm.  MOM: the step also stores its blend
// coefficients to P.mom (a moment checkpoint).  That step runs its own kernel
// instantiation, so the other steps carry no branch for it; the explicit
// arithmetic makes both instantiations compute the same bits.
template <class L, class R, bool MOM = false>
__device__ __forceinline__ void forward_core(const FwdArgs<R>& A, const FwdStep<R>& P, int x, int y, int z,
                                             unsigned i, const R (&f)[L::Q], R& bj, R& bm) {
  const Geo& g = A.geo;
  Mom<L, R> M;
  moments<L, R>(f, A.ph, M);
  if (!(M.rho > R(0)) || !isfinite(M.pn) || !isfinite(M.m[0] + M.m[1] + M.m[2])) *A.nonfinite = 1;
  const R gi = A.gfield[i];
  Blend<R> C;
  blend_coefs<L, R>(M, gi, C);
  if constexpr (MOM) store_coefs<L, R>(P.mom, g.n, i, C);
  blend_store<L, R>(P.dst, g.n, i, C);
  if (P.sample) {
    const int* b = A.obj.box;
    if (x >= b[0] && x < b[1] && y >= b[2] && y < b[3] && z >= b[4] && z < b[5]) {
      const R w = R(A.wobj[i]);
      if (w != R(0)) bj = fma_rn(w, local_objective<L, R>(M, A.obj, gi), bj);
    }
    if (A.obj.mon == MON_DRAG) bm = fma_rn(mul_rn(R(-2), gi), M.m[0], bm);
  }
}

// Pull of node i (Eq. 7) with its boundary completion (Eqs. 19-21, the 3D
// velocity inlet): the links from outside the domain take the node's rule,
// or for a zero-gradient outlet the post-streaming value of the neighbour
// along the inward normal, p_a(i + n_in - c_a).  Returns the links completed
// by a rule (0 off the bounded faces and for a zero-gradient outlet, whose
// links are copies), with the node's class and inlet velocity.
template <class L, class R, bool PER = true>
__device__ __forceinline__ unsigned node_gather(const R* __restrict__ P, const uint8_t* __restrict__ cls_arr,
                                                const float* __restrict__ uin, R rho_out, const Geo& g, int x, int y,
                                                int z, unsigned i, R (&f)[L::Q], uint8_t& cls, R& u0) {
#pragma unroll
  for (int a = 0; a < L::Q; ++a) f[a] = P[a * g.n + node_src<L, PER>(g, x, y, z, i, a)];
  cls = FLUID;
  u0 = R(0);
  const unsigned mask = node_unknowns<L, PER>(g, x, y, z);
  if (!mask) return 0u;
  cls = cls_arr[i];
  if (cls == INLET) u0 = R(uin[unsigned(y) + unsigned(g.ny) * unsigned(z)]);
  if (cls == OUTLET_ZG) {
    const int xn = x == 0 ? 1 : x - 1;
    const unsigned k = x == 0 ? i + 1u : i - 1u;
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
      if (mask & (1u << a)) f[a] = P[a * g.n + node_src<L, PER>(g, xn, y, z, k, a)];
    return 0u;
  }
  apply_rules<L, R>(f, mask, cls, u0, rho_out);
  return mask;
}

// Completion of an x-face node of an inner row (bounded x axis): the links in
// mask came from outside the domain and take the node's rule (Eqs. 19-21, the
// 3D velocity inlet), or for a zero-gradient outlet the post-streaming value
// of the neighbour along the inward normal, p_a(i + n_in - c_a).
template <class L, class R>
__device__ __forceinline__ void xface_complete(const R* __restrict__ P, const Geo& g, int x, unsigned i,
                                               unsigned mask, uint8_t cls, R u0, R rho_out, R (&f)[L::Q]) {
  if (cls == OUTLET_ZG) {
    const unsigned k = x == 0 ? i + 1u : i - 1u;
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
      if (mask & (1u << a)) f[a] = P[a * g.n + k - unsigned(L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz))];
  } else {
    apply_rules<L, R>(f, mask, cls, u0, rho_out);
  }
}

// Pull of an inner-row node (Eq. 7) with its x-face completion; returns the
// links completed by a rule (0 off the x faces and for a zero-gradient
// outlet, whose links are copies), with the node's class and inlet velocity.
template <class L, class R>
__device__ __forceinline__ unsigned row_gather(const R* __restrict__ P, const uint8_t* __restrict__ cls_arr,
                                               const float* __restrict__ uin, R rho_out, const Geo& g, int x, int y,
                                               int z, unsigned i, R (&f)[L::Q], uint8_t& cls, R& u0) {
#pragma unroll
  for (int a = 0; a < L::Q; ++a) f[a] = P[a * g.n + row_src<L>(g, x, i, a)];
  cls = FLUID;
  u0 = R(0);
  const unsigned mask = row_unknowns<L>(g, x);
  if (!mask) return 0u;
  cls = cls_arr[i];
  if (cls == INLET) u0 = R(uin[unsigned(y) + unsigned(g.ny) * unsigned(z)]);
  xface_complete<L, R>(P, g, x, i, mask, cls, u0, rho_out, f);
  return cls == OUTLET_ZG ? 0u : mask;
}

// Forward step over the inner rows (row geometry above): pull (Eq. 7), the
// x-face completion on the first and last node of a row, then forward_core.
template <class L, class R, bool MOM = false>
__global__ void __launch_bounds__(kBlock) fwd_row_kernel(FwdArgs<R> A) {
  pdl_enter();
  const Geo& g = A.geo;
  const int x = int(blockIdx.x) * kBlock + int(threadIdx.x), y = 1 + int(blockIdx.y);
  const int z = L::D == 3 ? 1 + int(blockIdx.z) : int(blockIdx.z);   // D2Q9: z is the slice of a batch
  R bj = 0, bm = 0;
  if (x < g.nx) {
    const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
    R f[L::Q];
    uint8_t cls;
    R u0;
    row_gather<L, R>(A.src, A.cls, A.uin, A.ph.rho_out, g, x, y, z, i, f, cls, u0);
    forward_core<L, R, MOM>(A, FwdStep<R>{A.src, A.dst, A.sample, A.mom}, x, y, z, i, f, bj, bm);
  }
  if (A.sample) {   // uniform across the grid
    block_sum2<R>(bj, bm);
    ring_store(bj, bm, A.ring, size_t(A.sample - 1) * A.nblk + row_slot(g, int(blockIdx.x), y, z));
  }
}

// One face-row node with its sources from the geometry: class and inlet
// velocity from the node arrays, populations through gather_geo().
template <class L, class R, bool MOM>
__device__ __forceinline__ void face_geo_node(const FwdArgs<R>& A, int x, int y, int z, R& bj, R& bm) {
  const Geo& g = A.geo;
  const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
  const uint8_t cls = A.cls[i];
  const R u0 = cls == INLET ? R(A.uin[unsigned(y) + unsigned(g.ny) * unsigned(z)]) : R(0);
  const FwdStep<R> P{A.src, A.dst, A.sample, A.mom};
  R f[L::Q];
  gather_geo<L, R>(P.src, g, x, y, z, cls, u0, A.ph.rho_out, f);
  forward_core<L, R, MOM>(A, P, x, y, z, i, f, bj, bm);
}

// Forward step over the face rows: one block row of the grid per face row
// (face_row_yz).
template <class L, class R, bool MOM = false>
__global__ void __launch_bounds__(kBlock) fwd_facerow_kernel(FwdArgs<R> A) {
  pdl_enter();
  const Geo& g = A.geo;
  const int x = int(blockIdx.x) * kBlock + int(threadIdx.x);
  int y, z;
  face_row_yz<L>(g, int(blockIdx.y), y, z);
  R bj = 0, bm = 0;
  if (x < g.nx) face_geo_node<L, R, MOM>(A, x, y, z, bj, bm);
  if (A.sample) {
    block_sum2<R>(bj, bm);
    ring_store(bj, bm, A.ring, size_t(A.sample - 1) * A.nblk + row_slot(g, int(blockIdx.x), y, z));
  }
}

// Window end (one block of kEndThreads): sum the per-block window sums in a
// fixed order with compensation, form the means of Eq. 42 and the ratio of
// Eq. 26, and clear the block sums for the next window.
constexpr int kEndThreads = 1024;
__global__ void __launch_bounds__(kEndThreads) window_end_kernel(double* blk, int nblocks, WindowAcc* acc,
                                                                 double tol, const int* nonfinite,
                                                                 double nsamples, double jconst,
                                                                 double mon_scale, int mon_kind) {
  __shared__ double sh[4][kEndThreads];
  double sj = 0, cj = 0, sm = 0, cm = 0;
  for (int b = threadIdx.x; b < nblocks; b += kEndThreads) {
    Sums a = reinterpret_cast<Sums*>(blk)[b];
    neumaier(sj, cj, a.x);
    neumaier(sj, cj, a.y);
    neumaier(sm, cm, a.z);
    neumaier(sm, cm, a.w);
    reinterpret_cast<Sums*>(blk)[b] = Sums{0.0, 0.0, 0.0, 0.0};
  }
  // Fixed-shape tree over the threads' (sum, compensation) pairs: deterministic.
  const int t = threadIdx.x;
  sh[0][t] = sj; sh[1][t] = cj; sh[2][t] = sm; sh[3][t] = cm;
  for (int stride = kEndThreads / 2; stride > 0; stride >>= 1) {
    __syncthreads();
    if (t < stride) {
      neumaier(sh[0][t], sh[1][t], sh[0][t + stride]);
      sh[1][t] += sh[1][t + stride];
      neumaier(sh[2][t], sh[3][t], sh[2][t + stride]);
      sh[3][t] += sh[3][t + stride];
    }
  }
  if (t != 0) return;
  const double tj = sh[0][0], tcj = sh[1][0], tm = sh[2][0], tcm = sh[3][0];
  const double jm = (tj + tcj) / nsamples + jconst;
  const double mm = mon_kind == MON_DRAG ? (tm + tcm) / nsamples * mon_scale : jm;
  if (acc->has_prev) {
    const double d = fabs(mm - acc->mprev);
    acc->ratio = fabs(mm) < 1e-30 ? d : d / fabs(mm);
    acc->converged = acc->ratio < tol;
  } else {
    acc->ratio = __longlong_as_double(0x7ff0000000000000LL);
    acc->converged = 0;
  }
  acc->jmean = jm;
  acc->mmean = mm;
  acc->mprev = mm;
  acc->has_prev = 1;
  acc->nonfinite = nonfinite[0];
}

// Per-slice window means of a batch of independent 2D lattices (D2Q9, nz > 1):
// one block per slice sums the block sums of that slice's rows (per_slice
// consecutive blocks of the step grid) in a fixed order.  Runs before
// window_end_kernel, which clears the block sums.
__global__ void __launch_bounds__(kEndThreads) slice_end_kernel(const double* blk, int per_slice, double nsamples,
                                                                const double* jconst, double mon_scale, int mon_kind,
                                                                double* out) {
  __shared__ double sh[4][kEndThreads];
  const int slice = blockIdx.x, t = threadIdx.x;
  double sj = 0, cj = 0, sm = 0, cm = 0;
  for (int b = t; b < per_slice; b += kEndThreads) {
    const Sums a = reinterpret_cast<const Sums*>(blk)[size_t(slice) * per_slice + b];
    neumaier(sj, cj, a.x);
    neumaier(sj, cj, a.y);
    neumaier(sm, cm, a.z);
    neumaier(sm, cm, a.w);
  }
  sh[0][t] = sj; sh[1][t] = cj; sh[2][t] = sm; sh[3][t] = cm;
  for (int stride = kEndThreads / 2; stride > 0; stride >>= 1) {
    __syncthreads();
    if (t < stride) {
      neumaier(sh[0][t], sh[1][t], sh[0][t + stride]);
      sh[1][t] += sh[1][t + stride];
      neumaier(sh[2][t], sh[3][t], sh[2][t + stride]);
      sh[3][t] += sh[3][t + stride];
    }
  }
  if (t != 0) return;
  const double jm = (sh[0][0] + sh[1][0]) / nsamples + jconst[slice];
  out[2 * slice] = jm;
  out[2 * slice + 1] = mon_kind == MON_DRAG ? (sh[2][0] + sh[3][0]) / nsamples * mon_scale : jm;
}

// ---------------------------------------------------------------------------
// Adjoint step (Eqs. 35-39), moment-space form of the transposed Jacobian.
//
// The collision h(f) depends on f only through rho, m and M2 = sum c c f, so
// (dh/df)^T v = d/drho + c_a . d/dm + c_a c_a : d/dM2 of psi = sum_b v_b h_b.
// The gradients of psi with respect to those moments are obtained by reverse
// differentiation of Eqs. 3, 13, 14, 16 (and of the objective), O(Q) work.
// ---------------------------------------------------------------------------
template <class R>
struct AdjArgs {
  const R* __restrict__ bnext;   // b^{n+1} after the boundary transpose
  const R* __restrict__ pprev;   // p^{n-1}
  R* __restrict__ bout;          // b^n after the boundary transpose
  const R* __restrict__ gfield;
  const uint8_t* __restrict__ cls;
  const float* __restrict__ uin;
  const float* __restrict__ wobj;
  R* __restrict__ gpart;         // per-node sensitivity partial of the current segment
  Geo geo;
  Phys<R> ph;
  Obj<R> obj;
  int sample;
  int terminal;                  // 1: b^{n+1} = 0 (last step of the window)
  int dbox[6];                   // design box
  ZgRows zg;                     // x-face rows next to zero-gradient outlet nodes
};

// Transposed boundary completion at a face node (in place on b).
template <class L, class R>
__device__ __forceinline__ void bc_transpose(R (&b)[L::Q], unsigned unk, uint8_t cls, R u0) {
  if (!unk) return;
  if (cls == WALL) {
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
      if ((unk & (1u << a)) && !(unk & (1u << L::opp(a)))) b[L::opp(a)] += b[a];
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
      if (unk & (1u << a)) b[a] = R(0);
  } else if (cls == INLET) {
    if (L::Q == 9) {
      // Transpose of Eq. 20: the coefficients of Eq. 38, chi = u0/(1-u0).
      const R chi = u0 / (R(1) - u0);
      const R t = chi * (R(2.0 / 3.0) * b[1] + R(1.0 / 6.0) * (b[5] + b[8]));
      const R b1 = b[1], b5 = b[5], b8 = b[8];
      b[0] += t;
      b[2] += t + R(0.5) * (b8 - b5);
      b[4] += t + R(0.5) * (b5 - b8);
      b[3] += R(2) * t + b1;
      b[6] += R(2) * t + b8;
      b[7] += R(2) * t + b5;
      b[1] = b[5] = b[8] = R(0);
    } else {
#pragma unroll
      for (int a = 0; a < L::Q; ++a)
        if (unk & (1u << a)) { b[L::opp(a)] += b[a]; b[a] = R(0); }
    }
  } else if (cls == OUTLET_P) {
    // Transpose of Eq. 21: the coefficients of Eq. 39.
    const R t = R(-2.0 / 3.0) * b[3] - R(1.0 / 6.0) * (b[6] + b[7]);
    const R b3 = b[3], b6 = b[6], b7 = b[7];
    b[0] += t;
    b[2] += t + R(0.5) * (b7 - b6);
    b[4] += t + R(0.5) * (b6 - b7);
    b[1] += R(2) * t + b3;
    b[8] += R(2) * t + b6;
    b[5] += R(2) * t + b7;
    b[3] = b[6] = b[7] = R(0);
  }
  // OUTLET_ZG: the unknown entries keep b_a(i); the node they were copied
  // from pulls them (see pull_face).
}

// Face part of the adjoint pull (out of line).
template <class L, class R>
__device__ __noinline__ void pull_face(const R* __restrict__ b, const uint8_t* __restrict__ cls, const Geo& g,
                                       int x, int y, int z, R* a) {
#pragma unroll
  for (int k = 0; k < L::Q; ++k) {
    unsigned j;
    a[k] = neighbour(g, x, y, z, L::cx(k), L::cy(k), L::cz(k), j) ? b[k * g.n + j] : R(0);
  }
  // A zero-gradient outlet node j copied p_k(i) into its unknown f_k(j),
  // j = i + c_k - n_in; pull those adjoints back.
  if (x == g.nx - 1 || x == 0) {
    const int sx = (x == g.nx - 1) ? -1 : 1;   // c_kx of the directions unknown on this face
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
      if (L::cx(k) != sx) continue;
      unsigned j;
      if (neighbour(g, x, y, z, 0, L::cy(k), L::cz(k), j) && cls[j] == OUTLET_ZG) a[k] += b[k * g.n + j];
    }
  }
}

// a_k(i) = b_k(i + c_k): adjoint streaming (Eq. 36), pulled from downstream,
// plus the transposed zero-gradient copies.  b == nullptr means b = 0.
template <class L, class R>
__device__ __forceinline__ void pull_adjoint(const R* __restrict__ b, const uint8_t* __restrict__ cls,
                                             const Geo& g, int x, int y, int z, unsigned i, bool face,
                                             R (&a)[L::Q]) {
  if (b == nullptr) {
#pragma unroll
    for (int k = 0; k < L::Q; ++k) a[k] = R(0);
  } else if (!face) {
#pragma unroll
    for (int k = 0; k < L::Q; ++k) a[k] = b[k * g.n + i + offset<L>(g, k)];
  } else {
    R t[L::Q];
    pull_face<L, R>(b, cls, g, x, y, z, t);
#pragma unroll
    for (int k = 0; k < L::Q; ++k) a[k] = t[k];
  }
}

// Adjoint of the window's start field: a = S^T b (no collision).
template <class L, class R>
__global__ void __launch_bounds__(kBlock) adj_pull_kernel(const R* __restrict__ b, const uint8_t* __restrict__ cls,
                                                          R* __restrict__ out, Geo g) {
  const int x = blockIdx.x * kBlock + threadIdx.x, y = blockIdx.y, z = blockIdx.z;
  if (x >= g.nx) return;
  const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
  R a[L::Q];
  pull_adjoint<L, R>(b, cls, g, x, y, z, i, on_face<L>(g, x, y, z), a);
#pragma unroll
  for (int k = 0; k < L::Q; ++k) out[k * g.n + i] = a[k];
}

template <class R>
struct AdjStep {
  const R* bnext;   // b^{n+1}
  const R* pprev;   // p^{n-1}
  R* bout;          // b^n
  int sample;
  int terminal;
};

// One node of an adjoint step (row geometry): the adjoint pull of Eq. 36
// (node_dst) plus the transposed zero-gradient copies, the transposed
// collision and blend (Eqs. 30-35) and the transposed boundary rule
// (Eqs. 37-39).
template <class L, class R, bool PER = true>
__device__ __forceinline__ void adjoint_node(const AdjArgs<R>& A, const AdjStep<R>& P, int x, int y, int z, unsigned i) {
  const Geo& g = A.geo;
  const R* bnext = P.bnext;
  const R* pprev = P.pprev;
  R* bout = P.bout;

  // Weighted moments of the pulled adjoint a^n: A0 = sum w a, A1 = sum w c a,
  // A2 = sum w c c a.  Everything below needs a only through them.
  R A0, A1[3], A2[6];
  {
    R a[L::Q];
    if (P.terminal) {
#pragma unroll
      for (int k = 0; k < L::Q; ++k) a[k] = R(0);
    } else {
#pragma unroll
      for (int k = 0; k < L::Q; ++k) {
        const unsigned j = node_dst<L, PER>(g, x, y, z, i, k);
        a[k] = j != kNone ? bnext[k * g.n + j] : R(0);
      }
      // A zero-gradient outlet node j on this x face copied p_k(i) into its
      // unknown f_k(j), j = i + c_k - n_in: pull those adjoints back.  Only
      // the rows next to outlet nodes look (an x-face thread on any other row
      // would hold its block for the class and adjoint loads).
      if (zg_row(A.zg, g, x, y, z)) {
        const int sx = x == 0 ? 1 : -1;
#pragma unroll
        for (int k = 0; k < L::Q; ++k) {
          if (L::cx(k) != sx) continue;
          const unsigned j = same_x_neighbour(g, y, z, i, L::cy(k), L::cz(k));
          if (j != kNone && A.cls[j] == OUTLET_ZG) a[k] += bnext[k * g.n + j];
        }
      }
    }
    raw_moments<L, R, true>(a, A0, A1, A2);
  }

  R f[L::Q];
  uint8_t cls;
  R u0;
  const unsigned mask = node_gather<L, R, PER>(pprev, A.cls, A.uin, A.ph.rho_out, g, x, y, z, i, f, cls, u0);
  Mom<L, R> M;
  moments<L, R>(f, A.ph, M);
  const R gi = A.gfield[i];

  // Sensitivity term of Eq. 40: sum_b a_b (h_bbar - h_b) = -6 m . A1 (times g'(phi) later).
  R gt = R(-6) * (M.m[0] * A1[0] + M.m[1] * A1[1] + M.m[2] * A1[2]);

  // Moments of v = (d p / d h)^T a: the blend scales the first moment by (1 - 2g).
  const R V0 = A0;
  const R sc = R(1) - R(2) * gi;
  const R V1[3] = {sc * A1[0], sc * A1[1], sc * A1[2]};
  const R* V2 = A2;
  const R* u = M.u;
  const R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  // V2 u (symmetric V2)
  const R V2u0 = V2[0] * u[0] + V2[3] * u[1] + V2[4] * u[2];
  const R V2u1 = V2[3] * u[0] + V2[1] * u[1] + V2[5] * u[2];
  const R V2u2 = V2[4] * u[0] + V2[5] * u[1] + V2[2] * u[2];
  const R uV2u = u[0] * V2u0 + u[1] * V2u1 + u[2] * V2u2;
  // psi_eq = rho E(u):  E = V0 + 3 V1.u + 4.5 u.V2.u - 1.5 V0 u.u   (Eq. 3)
  const R E = V0 + R(3) * (V1[0] * u[0] + V1[1] * u[1] + V1[2] * u[2]) + R(4.5) * uV2u - R(1.5) * V0 * uu;
  R cu[3];   // d psi / d u at fixed rho
  cu[0] = M.rho * (R(3) * V1[0] + R(9) * V2u0 - R(3) * V0 * u[0]);
  cu[1] = M.rho * (R(3) * V1[1] + R(9) * V2u1 - R(3) * V0 * u[1]);
  cu[2] = M.rho * (R(3) * V1[2] + R(9) * V2u2 - R(3) * V0 * u[2]);
  R crho = E;          // d psi / d rho at fixed u, Pi, tau_eff
  R cm0 = 0;           // d psi / d m_x directly (drag objective)
  // psi_neq = om * 4.5 R:Pi with R = V2 - cs^2 V0 I   (Eq. 16)
  const R c = cs2<R>();
  const R Rm[6] = {V2[0] - c * V0, V2[1] - c * V0, (L::D == 3 ? V2[2] - c * V0 : R(0)), V2[3], V2[4], V2[5]};
  const R RP = R(4.5) * (Rm[0] * M.pi[0] + Rm[1] * M.pi[1] + Rm[2] * M.pi[2] +
                         R(2) * (Rm[3] * M.pi[3] + Rm[4] * M.pi[4] + Rm[5] * M.pi[5]));
  R ctau = RP / (M.te * M.te);   // d psi / d tau_eff through om = 1 - 1/tau_eff
  R cpi[6];                      // d psi / d Pi_pq (full symmetric matrix entries)
#pragma unroll
  for (int k = 0; k < 6; ++k) cpi[k] = M.om * R(4.5) * Rm[k];

  if (P.sample) {
    const int* bx = A.obj.box;
    if (x >= bx[0] && x < bx[1] && y >= bx[2] && y < bx[3] && z >= bx[4] && z < bx[5]) {
      const R ws = R(A.wobj[i]) * A.obj.ws;
      if (ws != R(0)) {
        switch (A.obj.kind) {
          case OBJ_DISS: {
            // psi = 1.5 (te - 1/2) Pi:Pi / (rho te^2)
            const R k0 = R(1.5) * M.inv / (M.te * M.te);
            const R val = k0 * (M.te - R(0.5)) * M.pp;
#pragma unroll
            for (int k = 0; k < 6; ++k) cpi[k] += ws * R(2) * k0 * (M.te - R(0.5)) * M.pi[k];
            ctau += ws * R(1.5) * M.pp * M.inv * (R(1) - M.te) / (M.te * M.te * M.te);
            crho += -ws * val * M.inv;
            break;
          }
          case OBJ_VEL: {
            cu[0] += ws * R(2) * (u[0] - A.obj.uref[0]);
            cu[1] += ws * R(2) * (u[1] - A.obj.uref[1]);
            if (L::D == 3) cu[2] += ws * R(2) * (u[2] - A.obj.uref[2]);
            break;
          }
          case OBJ_PRES: crho += ws * c; break;
          default: {
            cm0 += ws * R(-2) * gi;
            gt += ws * R(-2) * M.m[0];   // direct d psi / d g, times g'(phi) later
          }
        }
      }
    }
  }
  // tau_eff(|Pi|, rho) of Eq. 14: d te/d|Pi| = 4.5 C^2/(s rho), d te/d rho = -4.5 C^2 |Pi|/(s rho^2) (Eq. 32)
  {
    const R k1 = R(4.5) * A.ph.c2 / (M.s * M.rho);      // d te / d|Pi|
    crho += ctau * (-k1 * M.pn * M.inv);
    if (M.pn > R(0)) {
      const R kp = ctau * k1 * R(2) / M.pn;            // times d|Pi|/dPi = 2 Pi / |Pi|
#pragma unroll
      for (int k = 0; k < 6; ++k) cpi[k] += kp * M.pi[k];
    }
  }
  // u = m / rho
  R gm[3], grho;
  gm[0] = cu[0] * M.inv + cm0;
  gm[1] = cu[1] * M.inv;
  gm[2] = cu[2] * M.inv;
  grho = crho - (u[0] * cu[0] + u[1] * cu[1] + u[2] * cu[2]) * M.inv;
  // Pi(rho, m, M2) = M2 - rho cs^2 I - m m^T / rho
  {
    const R* m = M.m;
    const R pm0 = cpi[0] * m[0] + cpi[3] * m[1] + cpi[4] * m[2];
    const R pm1 = cpi[3] * m[0] + cpi[1] * m[1] + cpi[5] * m[2];
    const R pm2 = cpi[4] * m[0] + cpi[5] * m[1] + cpi[2] * m[2];
    grho += -c * (cpi[0] + cpi[1] + cpi[2]) + (m[0] * pm0 + m[1] * pm1 + m[2] * pm2) * M.inv * M.inv;
    gm[0] -= R(2) * pm0 * M.inv;
    gm[1] -= R(2) * pm1 * M.inv;
    gm[2] -= R(2) * pm2 * M.inv;
  }
  // b_a = d psi / d f_a = grho + c_a . gm + c_a c_a : cpi
  R b[L::Q];
  quad_all<L, R>(grho, gm, cpi, b);
  if (mask) bc_transpose<L, R>(b, mask, cls, u0);
#pragma unroll
  for (int k = 0; k < L::Q; ++k) bout[k * g.n + i] = b[k];

  const int* d = A.dbox;
  if (x >= d[0] && x < d[1] && y >= d[2] && y < d[3] && z >= d[4] && z < d[5]) A.gpart[i] += gt;
}

// One adjoint step over every node: grid (ceil(nx / kBlock), ny, nz).  Unlike
// the forward step it needs no split into inner and face rows: its boundary
// completion costs no occupancy (measured: one kernel beats the pair).
// Resident blocks per SM the adjoint step is compiled for, i.e. its register
// budget (65536 / (128 blocks)): FP32 D2Q9 12 (42 registers; left alone the
// non-periodic instantiation takes 46), FP32 D3Q19 9 (56), FP64 5 (102).  A
// minimum of 1 block lets the compiler spend up to 93 registers on the FP32
// D3Q19 kernel, which then runs at 7 blocks per SM and about 25% slower.
template <class L, class R>
constexpr int adj_min_blocks() {
  return sizeof(R) == 4 ? (L::Q == 9 ? 12 : 9) : 5;
}

template <class L, class R, bool PER = true>
__global__ void __launch_bounds__(kBlock, adj_min_blocks<L, R>()) adj_step_kernel(AdjArgs<R> A) {
  pdl_enter();
  const Geo& g = A.geo;
  const int x = int(blockIdx.x) * kBlock + int(threadIdx.x), y = int(blockIdx.y), z = int(blockIdx.z);
  if (x >= g.nx) return;
  adjoint_node<L, R, PER>(A, AdjStep<R>{A.bnext, A.pprev, A.bout, A.sample, A.terminal}, x, y, z,
                     unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz);
}

// Fold a segment's sensitivity partials into the FP64 (sum, compensation)
// accumulator and clear them (once per segment of K steps).
template <class R>
__global__ void grad_fold_kernel(R* __restrict__ gpart, double2* __restrict__ gacc, Geo g, int x0, int x1,
                                 int y0, int y1, int z0, int z1) {
  const int bx = x1 - x0, by = y1 - y0;
  const long long total = (long long)bx * by * (z1 - z0);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int x = x0 + int(k % bx), y = y0 + int((k / bx) % by), z = z0 + int(k / ((long long)bx * by));
    const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
    double2 s = gacc[i];
    neumaier(s.x, s.y, double(gpart[i]));
    gacc[i] = s;
    gpart[i] = R(0);
  }
}

// ---------------------------------------------------------------------------
// Small kernels: design field, gradient, state conversion, checkpoints.
// ---------------------------------------------------------------------------

// g(phi) = g_max (1 - phi (1+q)/(phi+q)), phi = 1 - gamma  (Sec. 2.2)
template <class R>
__global__ void design_kernel(const float* __restrict__ gamma, R* __restrict__ gf, long long n, double q,
                              double g_max, int* bad) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gm = gamma[i];
    if (!(gm >= 0.f && gm <= 1.f)) *bad = 1;
    const double phi = 1.0 - double(gm);
    gf[i] = R(g_max * (1.0 - phi * (1.0 + q) / (phi + q)));
  }
}

// dJ/dgamma = -g'(phi) * G = g_max q (1+q) / (phi+q)^2 * G inside the design box.
__global__ void gradient_kernel(const double2* __restrict__ gacc, const float* __restrict__ gamma,
                                double* __restrict__ out, Geo g, int x0, int x1, int y0, int y1,
                                int z0, int z1, double q, double g_max) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n;
       i += (long long)gridDim.x * blockDim.x) {
    const int x = int(i % g.nx), y = int((i / g.nx) % g.ny), z = int(i / g.sz);
    double v = 0.0;
    if (x >= x0 && x < x1 && y >= y0 && y < y1 && z >= z0 && z < z1) {
      const double phi = 1.0 - double(gamma[i]);
      const double dgp = g_max * q * (1.0 + q) / ((phi + q) * (phi + q));
      const double2 s = gacc[i];
      v = dgp * (s.x + s.y);
    }
    out[i] = v;
  }
}

// Moment checkpoint -> p~ at every node through blend_store(), the step
// kernels' own arithmetic, so the field is bitwise the one the step stored.
template <class L, class R>
__global__ void __launch_bounds__(kBlock) mom_decode_kernel(const R* __restrict__ mom, R* __restrict__ p, unsigned n) {
  const unsigned i = blockIdx.x * kBlock + threadIdx.x;
  if (i >= n) return;
  Blend<R> C;
  load_coefs<L, R>(mom, n, i, C);
  blend_store<L, R>(p, n, i, C);
}

template <class L, class R>
__global__ void unshift_kernel(const R* __restrict__ src, double* __restrict__ dst, long long n) {
  const long long total = n * L::Q;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int a = int(k / n);
    double w = 0;
#pragma unroll
    for (int b = 0; b < L::Q; ++b) if (b == a) w = L::w(b);
    dst[k] = double(src[k]) + w;
  }
}

template <class L, class R>
__global__ void shift_kernel(const double* __restrict__ src, R* __restrict__ dst, long long n, int* bad) {
  const long long total = n * L::Q;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int a = int(k / n);
    double w = 0;
#pragma unroll
    for (int b = 0; b < L::Q; ++b) if (b == a) w = L::w(b);
    const double v = src[k];
    if (!isfinite(v)) *bad = 1;
    dst[k] = R(v - w);
  }
}

// Shifted field of one working precision into another (same [Q][N] layout).
template <class S, class D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, long long total) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x)
    dst[k] = D(src[k]);
}

template <class R>
__global__ void copy_double_kernel(const R* __restrict__ src, double* __restrict__ dst, long long total) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x)
    dst[k] = double(src[k]);
}

// 16-bit checkpoints: deviation from the equilibrium of the stored field's own
// moments, scaled per block of kBlock nodes by a power of two so that the
// block's largest deviation sits near 2^14, plus rho-1 and m in FP32.
template <class T> __device__ __forceinline__ T to16(float v);
template <> __device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
__device__ __forceinline__ float from16(__half v) { return __half2float(v); }
__device__ __forceinline__ float from16(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class L>
__device__ __forceinline__ float feq_shifted(float rt, float rho, const float (&u)[3], int a) {
  const float cu = L::cx(a) * u[0] + L::cy(a) * u[1] + L::cz(a) * u[2];
  const float uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return float(L::w(a)) * (rt + rho * (3.f * cu + 4.5f * cu * cu - 1.5f * uu));
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock) ckpt_encode_kernel(const float* __restrict__ p, T* __restrict__ dev,
                                                             float* __restrict__ mom, int* __restrict__ expo,
                                                             long long n) {
  __shared__ float smax[kBlock / 32];
  const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
  float f[L::Q], d[L::Q];
  float mx = 0.f;
  float rt = 0.f, u[3] = {0.f, 0.f, 0.f}, rho = 1.f;
  if (i < n) {
    float m[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      f[a] = p[a * n + i];
      rt += f[a];
      m[0] += L::cx(a) * f[a];
      m[1] += L::cy(a) * f[a];
      m[2] += L::cz(a) * f[a];
    }
    rho = 1.f + rt;
    u[0] = m[0] / rho; u[1] = m[1] / rho; u[2] = m[2] / rho;
    mom[i] = rt;
    mom[n + i] = m[0];
    mom[2 * n + i] = m[1];
    if (L::D == 3) mom[3 * n + i] = m[2];
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
      d[a] = f[a] - feq_shifted<L>(rt, rho, u, a);
      mx = fmaxf(mx, fabsf(d[a]));
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) smax[threadIdx.x >> 5] = mx;
  __syncthreads();
  float bmax = 0.f;
#pragma unroll
  for (int k = 0; k < kBlock / 32; ++k) bmax = fmaxf(bmax, smax[k]);
  int e = 0;
  if (bmax > 0.f) { frexpf(bmax, &e); e = 14 - e; }   // scale = 2^e puts bmax in [2^13, 2^14)
  if (threadIdx.x == 0) expo[blockIdx.x] = e;
  if (i < n) {
#pragma unroll
    for (int a = 0; a < L::Q; ++a) dev[a * n + i] = to16<T>(ldexpf(d[a], e));
  }
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock) ckpt_decode_kernel(const T* __restrict__ dev, const float* __restrict__ mom,
                                                             const int* __restrict__ expo, float* __restrict__ p,
                                                             long long n) {
  const long long i = blockIdx.x * (long long)kBlock + threadIdx.x;
  if (i >= n) return;
  const int e = expo[blockIdx.x];
  const float rt = mom[i];
  const float rho = 1.f + rt;
  float u[3] = {mom[n + i] / rho, mom[2 * n + i] / rho, L::D == 3 ? mom[3 * n + i] / rho : 0.f};
#pragma unroll
  for (int a = 0; a < L::Q; ++a) p[a * n + i] = feq_shifted<L>(rt, rho, u, a) + ldexpf(from16(dev[a * n + i]), -e);
}

}  // namespace lbm
