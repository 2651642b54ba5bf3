// Velocity sets of the two lattices as compile-time functions, so that fully
// unrolled loops over directions fold every c_a, w_a and opposite index into
// immediates (no constant-memory loads on the hot path).
//
// D2Q9 follows the paper's order (Sec. 2.1.1, Eqs. 2 and 4).  D3Q19 is the
// standard set (rest 1/3, axis 1/18, face diagonals 1/36) in the order
// documented in include/lbmadj.h.
#pragma once

#define HD __host__ __device__ __forceinline__

struct D2Q9 {
  static constexpr int Q = 9;
  static constexpr int D = 2;
  HD static constexpr int cx(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : (a == 3 || a == 6 || a == 7) ? -1 : 0;
  }
  HD static constexpr int cy(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : (a == 4 || a == 7 || a == 8) ? -1 : 0;
  }
  HD static constexpr int cz(int) { return 0; }
  HD static constexpr double w(int a) { return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
  HD static constexpr int opp(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 5 + 2) % 4) + 5);
  }
};

struct D3Q19 {
  static constexpr int Q = 19;
  static constexpr int D = 3;
  // c1..c6: +x,-x,+y,-y,+z,-z; c7..c18: (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),
  // (1,0,1),(-1,0,-1),(1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1)
  HD static constexpr int cx(int a) {
    return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
         : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
  }
  HD static constexpr int cy(int a) {
    return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
         : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
  }
  HD static constexpr int cz(int a) {
    return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
         : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
  }
  HD static constexpr double w(int a) { return a == 0 ? 1.0 / 3.0 : (a <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }
  HD static constexpr int opp(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }
};

// Compile-time self checks of the tables.
template <class L>
constexpr bool lattice_tables_consistent() {
  double sw = 0;
  for (int a = 0; a < L::Q; ++a) {
    const int b = L::opp(a);
    if (L::cx(b) != -L::cx(a) || L::cy(b) != -L::cy(a) || L::cz(b) != -L::cz(a)) return false;
    if (L::opp(b) != a) return false;
    sw += L::w(a);
  }
  return sw > 1.0 - 1e-12 && sw < 1.0 + 1e-12;
}
static_assert(lattice_tables_consistent<D2Q9>(), "D2Q9 tables");
static_assert(lattice_tables_consistent<D3Q19>(), "D3Q19 tables");
