// Host check of the step kernels' index arithmetic (compiled and run by
// test_row_geometry.py; no GPU).  For each lattice shape and periodicity it
// enumerates every thread of the row and face-row launches exactly as the
// kernels form them and checks that the rows cover every node once, that
// every population index the pulls, the x-face completion and the adjoint's
// zero-gradient term read lies in the lattice and is the node the geometry
// names, and that every block-sum slot lies in its range.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "kernels.cuh"

using namespace lbm;

static int failures = 0;
#define CHECK(cond, ...)                                 \
  do {                                                   \
    if (!(cond)) {                                       \
      if (failures < 20) { printf(__VA_ARGS__); printf("\n"); } \
      ++failures;                                        \
    }                                                    \
  } while (0)

// Node (x+dx, y+dy, z+dz) with periodic wrap, or -1 outside.
static long long nb(const Geo& g, int x, int y, int z, int dx, int dy, int dz) {
  int p[3] = {x + dx, y + dy, z + dz};
  const int d[3] = {g.nx, g.ny, g.nz}, per[3] = {g.px, g.py, g.pz};
  for (int k = 0; k < 3; ++k)
    if (p[k] < 0 || p[k] >= d[k]) {
      if (!per[k]) return -1;
      p[k] = (p[k] + d[k]) % d[k];
    }
  return p[0] + (long long)g.nx * (p[1] + (long long)g.ny * p[2]);
}

template <class L>
static void check(int nx, int ny, int nz, int px, int py, int pz) {
  const Geo g{nx, ny, nz, px, py, pz, unsigned(nx * ny * nz), unsigned(nx), unsigned(nx * ny)};
  const long long n = (long long)nx * ny * nz;
  std::vector<int> hit(size_t(n), 0);
  const int rgx = (nx + kBlock - 1) / kBlock;
  const int iy = inner_rows_y<L>(g), iz = inner_rows_z<L>(g), nfr = face_rows<L>(g);
  const long long row_blocks = (long long)rgx * iy * iz, nblk = row_blocks + (long long)rgx * nfr;
  // row kernels: grid (rgx, iy, iz) of kBlock threads
  for (int bz = 0; bz < iz; ++bz)
    for (int by = 0; by < iy; ++by)
      for (int bx = 0; bx < rgx; ++bx) {
        const long long bid = bx + (long long)rgx * (by + (long long)iy * bz);
        CHECK(bid >= 0 && bid < row_blocks, "row block id %lld", bid);
        for (int t = 0; t < kBlock; ++t) {
          const int x = bx * kBlock + t, y = 1 + by, z = L::D == 3 ? 1 + bz : bz;
          if (x >= nx) continue;
          const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
          CHECK((long long)i < n, "row node %u outside", i);
          hit[i] += 1;
          const unsigned mask = row_unknowns<L>(g, x);
          for (int a = 0; a < L::Q; ++a) {
            const long long up = nb(g, x, y, z, -L::cx(a), -L::cy(a), -L::cz(a));
            const unsigned j = row_src<L>(g, x, i, a);
            CHECK((long long)j < n, "src %u outside (x %d y %d z %d a %d)", j, x, y, z, a);
            if (mask & (1u << a)) CHECK(up < 0 && j == i, "unknown link a=%d at x=%d", a, x);
            else CHECK(up == (long long)j, "src of a=%d at (%d,%d,%d): %u, want %lld", a, x, y, z, j, up);
            const long long down = nb(g, x, y, z, L::cx(a), L::cy(a), L::cz(a));
            const unsigned d = row_dst<L>(g, x, i, a);
            CHECK(d == kNone ? down < 0 : down == (long long)d, "dst of a=%d at (%d,%d,%d)", a, x, y, z);
            if (mask & (1u << a)) {
              // zero-gradient copy: p_a(i + n_in - c_a)
              const unsigned k = x == 0 ? i + 1u : i - 1u;
              const unsigned zg = k - unsigned(L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz));
              const long long want = nb(g, x == 0 ? 1 : nx - 2, y, z, -L::cx(a), -L::cy(a), -L::cz(a));
              CHECK(want >= 0 && (long long)zg == want, "zero-gradient source of a=%d at (%d,%d,%d)", a, x, y, z);
            }
          }
          if (mask) {   // the adjoint's zero-gradient term reads the same-face neighbour (x, y + c_y, z + c_z)
            const int sx = x == 0 ? 1 : -1;
            for (int k = 0; k < L::Q; ++k) {
              if (L::cx(k) != sx) continue;
              const unsigned j = i + unsigned(L::cy(k) * int(g.sy) + L::cz(k) * int(g.sz));
              CHECK((long long)j == nb(g, x, y, z, 0, L::cy(k), L::cz(k)), "ext node of k=%d at (%d,%d,%d)", k, x, y, z);
            }
          }
        }
      }
  // face-row kernels: grid (rgx, nfr)
  for (int r = 0; r < nfr; ++r) {
    int y, z;
    face_row_yz<L>(g, r, y, z);
    CHECK(y >= 0 && y < ny && z >= 0 && z < nz, "face row %d -> (%d, %d)", r, y, z);
    const bool onface = y == 0 || y == ny - 1 || (L::D == 3 && (z == 0 || z == nz - 1));
    CHECK(onface, "face row %d is not on a face", r);
    if (L::D == 2) {
      const int fy = ny >= 2 ? 2 : 1;
      CHECK(z == r / fy, "D2Q9 face row %d belongs to slice %d", r, z);
    }
    for (int bx = 0; bx < rgx; ++bx) {
      const long long bid = row_blocks + bx + (long long)rgx * r;
      CHECK(bid >= row_blocks && bid < nblk, "face block id %lld", bid);
      for (int t = 0; t < kBlock; ++t) {
        const int x = bx * kBlock + t;
        if (x >= nx) continue;
        hit[size_t(x + (long long)nx * (y + (long long)ny * z))] += 1;
      }
    }
  }
  for (long long i = 0; i < n; ++i)
    CHECK(hit[size_t(i)] == 1, "node %lld covered %d times (shape %d %d %d)", i, hit[size_t(i)], nx, ny, nz);
}

int main() {
  const int per[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 1}};
  const int shapes3[][3] = {{3, 3, 3}, {5, 4, 3}, {130, 6, 5}, {128, 3, 4}, {129, 7, 6}, {256, 5, 3}, {7, 3, 130}};
  const int shapes2[][3] = {{3, 3, 1}, {10, 7, 1}, {131, 9, 3}, {128, 3, 1}, {300, 20, 2}, {257, 4, 5}};
  for (auto& p : per) {
    for (auto& s : shapes3) check<D3Q19>(s[0], s[1], s[2], p[0], p[1], p[2]);
    for (auto& s : shapes2) check<D2Q9>(s[0], s[1], s[2], p[0], p[1], 0);
  }
  // periodic axes may be short
  check<D3Q19>(1, 4, 4, 1, 0, 0);
  check<D3Q19>(6, 1, 4, 0, 1, 0);
  check<D3Q19>(6, 4, 1, 0, 0, 1);
  check<D3Q19>(2, 2, 2, 1, 1, 1);
  check<D2Q9>(1, 5, 1, 1, 0, 0);
  check<D2Q9>(6, 1, 3, 0, 1, 0);
  check<D2Q9>(2, 2, 2, 1, 1, 0);
  printf("%s (%d failures)\n", failures ? "FAILED" : "ok", failures);
  return failures ? 1 : 0;
}
