// Host check of the step kernels' index arithmetic (compiled and run by
// test_row_geometry.py; no GPU).  For each lattice shape and periodicity it
// enumerates every thread of the step launches exactly as the kernels form
// them and checks that the grid covers every node once, that the unknown
// links are those from outside the domain, that every population index the
// pulls, the zero-gradient copies and the adjoint's same-face lookups read
// lies in the lattice and is the node the geometry names, and that every
// block-sum slot lies in its range (a D2Q9 slice's blocks contiguous), and
// that the rows running the adjoint's zero-gradient pull-back cover every
// node an outlet copied from.
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
  const long long nblk = (long long)rgx * ny * nz;
  unsigned xface = 0;   // the directions entering through the x = 0 face (c_x = +1)
  for (int a = 0; a < L::Q; ++a)
    if (L::cx(a) > 0) xface |= 1u << a;
  // step kernels: grid (rgx, ny, nz) of kBlock threads, node (bx kBlock + t, by, bz)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int bx = 0; bx < rgx; ++bx) {
        const long long bid = bx + (long long)rgx * (y + (long long)ny * z);
        CHECK(bid >= 0 && bid < nblk, "block id %lld", bid);
        if (L::D == 2) CHECK(bid / ((long long)rgx * ny) == z, "block %lld outside slice %d", bid, z);
        for (int t = 0; t < kBlock; ++t) {
          const int x = bx * kBlock + t;
          if (x >= nx) continue;
          const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
          CHECK((long long)i < n, "node %u outside", i);
          hit[i] += 1;
          const unsigned mask = node_unknowns<L>(g, x, y, z);
          if (!px && !py && !pz) CHECK(mask == (node_unknowns<L, false>(g, x, y, z)), "unknowns without wrap");
          for (int a = 0; a < L::Q; ++a) {
            const long long up = nb(g, x, y, z, -L::cx(a), -L::cy(a), -L::cz(a));
            CHECK(((mask >> a) & 1u) == (up < 0 ? 1u : 0u), "unknown mask of a=%d at (%d,%d,%d)", a, x, y, z);
            const unsigned j = node_src<L>(g, x, y, z, i, a);
            if (!px && !py && !pz) CHECK(j == (node_src<L, false>(g, x, y, z, i, a)), "node_src without wrap");
            CHECK((long long)j < n, "src %u outside (x %d y %d z %d a %d)", j, x, y, z, a);
            if (up < 0) CHECK(j == i, "unknown link a=%d at (%d,%d,%d) reads %u", a, x, y, z, j);
            else CHECK(up == (long long)j, "src of a=%d at (%d,%d,%d): %u, want %lld", a, x, y, z, j, up);
            const long long down = nb(g, x, y, z, L::cx(a), L::cy(a), L::cz(a));
            const unsigned d = node_dst<L>(g, x, y, z, i, a);
            if (!px && !py && !pz) CHECK(d == (node_dst<L, false>(g, x, y, z, i, a)), "node_dst without wrap");
            CHECK(d == kNone ? down < 0 : down == (long long)d, "dst of a=%d at (%d,%d,%d)", a, x, y, z);
          }
          // a zero-gradient outlet may sit where the unknowns are exactly one x face's:
          // its copies read the pull of the inward neighbour
          const bool left = x == 0 && mask == xface, right = x == nx - 1 && nx > 1;
          unsigned xface1 = 0;
          for (int a = 0; a < L::Q; ++a)
            if (L::cx(a) < 0) xface1 |= 1u << a;
          if (left || (right && mask == xface1)) {
            const int xn = x == 0 ? 1 : x - 1;
            const unsigned k = x == 0 ? i + 1u : i - 1u;
            for (int a = 0; a < L::Q; ++a) {
              if (!((mask >> a) & 1u)) continue;
              const unsigned zg = node_src<L>(g, xn, y, z, k, a);
              const long long want = nb(g, xn, y, z, -L::cx(a), -L::cy(a), -L::cz(a));
              CHECK(want >= 0 && (long long)zg == want, "zero-gradient source of a=%d at (%d,%d,%d)", a, x, y, z);
            }
          }
          // the face gathers (gather_geo, pull_face): neighbour() for every link,
          // and the zero-gradient copy's upstream node where such an outlet may sit
          for (int a = 0; a < L::Q; ++a) {
            for (int sgn = -1; sgn <= 1; sgn += 2) {
              unsigned j = 0;
              const bool in = neighbour(g, x, y, z, sgn * L::cx(a), sgn * L::cy(a), sgn * L::cz(a), j);
              const long long want = nb(g, x, y, z, sgn * L::cx(a), sgn * L::cy(a), sgn * L::cz(a));
              CHECK(in == (want >= 0) && (!in || (long long)j == want), "neighbour of a=%d at (%d,%d,%d)", a, x, y, z);
            }
          }
          if (left || (right && mask == xface1)) {
            const int xn = x == 0 ? 1 : x - 1;
            for (int a = 0; a < L::Q; ++a) {
              if (!((mask >> a) & 1u)) continue;
              unsigned j = 0;
              const bool in = neighbour(g, xn, y, z, -L::cx(a), -L::cy(a), -L::cz(a), j);
              CHECK(in && (long long)j < n, "gather_geo zero-gradient source of a=%d at (%d,%d,%d)", a, x, y, z);
            }
          }
          if (!px && (x == 0 || x == nx - 1)) {   // the adjoint's same-face neighbours
            for (int k = 0; k < L::Q; ++k) {
              const unsigned j = same_x_neighbour(g, y, z, i, L::cy(k), L::cz(k));
              const long long want = nb(g, x, y, z, 0, L::cy(k), L::cz(k));
              CHECK(j == kNone ? want < 0 : want == (long long)j, "same-face neighbour of k=%d at (%d,%d,%d)", k, x, y, z);
            }
          }
        }
      }
  for (long long i = 0; i < n; ++i)
    CHECK(hit[size_t(i)] == 1, "node %lld covered %d times (shape %d %d %d)", i, hit[size_t(i)], nx, ny, nz);
}

// The forward step's split: the inner-row kernel (grid rgx x iy x iz) and the
// face-row kernel (grid rgx x nfr) cover every node once; every block's
// sample slot is distinct; the inner-row pulls (row_src), their unknown links
// (row_unknowns) and the zero-gradient copies of xface_complete read the
// nodes the geometry names.
template <class L>
static void check_split(int nx, int ny, int nz, int px, int py, int pz) {
  const Geo g{nx, ny, nz, px, py, pz, unsigned(nx * ny * nz), unsigned(nx), unsigned(nx * ny)};
  const long long n = (long long)nx * ny * nz;
  std::vector<int> hit(size_t(n), 0);
  const int rgx = (nx + kBlock - 1) / kBlock;
  const int iy = inner_rows_y<L>(g), iz = inner_rows_z<L>(g), nfr = face_rows<L>(g);
  const long long nslot = (long long)rgx * ny * nz;
  std::vector<int> slot(size_t(nslot), 0);
  for (int bz = 0; bz < iz; ++bz)
    for (int by = 0; by < iy; ++by)
      for (int bx = 0; bx < rgx; ++bx) {
        const int y = 1 + by, z = L::D == 3 ? 1 + bz : bz;
        const unsigned sl = row_slot(g, bx, y, z);
        CHECK((long long)sl < nslot, "row slot %u", sl);
        if ((long long)sl < nslot) slot[sl] += 1;
        for (int t = 0; t < kBlock; ++t) {
          const int x = bx * kBlock + t;
          if (x >= nx) continue;
          const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
          hit[i] += 1;
          const unsigned mask = row_unknowns<L>(g, x);
          CHECK(mask == node_unknowns<L>(g, x, y, z), "inner-row unknowns at (%d,%d,%d)", x, y, z);
          for (int a = 0; a < L::Q; ++a) {
            const long long up = nb(g, x, y, z, -L::cx(a), -L::cy(a), -L::cz(a));
            const unsigned j = row_src<L>(g, x, i, a);
            CHECK((long long)j < n, "row src %u outside", j);
            if (up < 0) CHECK(j == i, "row unknown a=%d at (%d,%d,%d)", a, x, y, z);
            else CHECK(up == (long long)j, "row src of a=%d at (%d,%d,%d)", a, x, y, z);
            if (mask & (1u << a)) {   // xface_complete's zero-gradient copy
              const unsigned k = x == 0 ? i + 1u : i - 1u;
              const unsigned zg = k - unsigned(L::cx(a) + L::cy(a) * int(g.sy) + L::cz(a) * int(g.sz));
              const long long want = nb(g, x == 0 ? 1 : nx - 2, y, z, -L::cx(a), -L::cy(a), -L::cz(a));
              CHECK(want >= 0 && (long long)zg == want, "row zero-gradient source of a=%d at (%d,%d,%d)", a, x, y, z);
            }
          }
        }
      }
  for (int r = 0; r < nfr; ++r) {
    int y, z;
    face_row_yz<L>(g, r, y, z);
    CHECK(y >= 0 && y < ny && z >= 0 && z < nz, "face row %d -> (%d, %d)", r, y, z);
    CHECK(y == 0 || y == ny - 1 || (L::D == 3 && (z == 0 || z == nz - 1)), "face row %d is not on a face", r);
    for (int bx = 0; bx < rgx; ++bx) {
      const unsigned sl = row_slot(g, bx, y, z);
      CHECK((long long)sl < nslot, "face slot %u", sl);
      if ((long long)sl < nslot) slot[sl] += 1;
      for (int t = 0; t < kBlock; ++t) {
        const int x = bx * kBlock + t;
        if (x < nx) hit[size_t(x + (long long)nx * (y + (long long)ny * z))] += 1;
      }
    }
  }
  for (long long i = 0; i < n; ++i)
    CHECK(hit[size_t(i)] == 1, "split: node %lld covered %d times (shape %d %d %d)", i, hit[size_t(i)], nx, ny, nz);
  for (long long k = 0; k < nslot; ++k) CHECK(slot[size_t(k)] == 1, "slot %lld used %d times", k, slot[size_t(k)]);
}

// The rows that run the adjoint's zero-gradient pull-back (zg_row over
// zg_rows of the class map) include every x-face node with a same-face
// neighbour that is a zero-gradient outlet, on class maps with outlet nodes
// at random places on both x faces (bounded x axis, as validated).
template <class L>
static void check_zg(int nx, int ny, int nz, int py, int pz, unsigned seed, int density) {
  const Geo g{nx, ny, nz, 0, py, pz, unsigned(nx * ny * nz), unsigned(nx), unsigned(nx * ny)};
  std::vector<uint8_t> cls(size_t(nx) * ny * nz, FLUID);
  unsigned h = seed;
  int nzg = 0;
  for (int f = 0; f < 2; ++f)
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y) {
        h = h * 1664525u + 1013904223u;
        if (int((h >> 16) % 100) < density) {
          cls[size_t(f ? nx - 1 : 0) + size_t(nx) * (size_t(y) + size_t(ny) * z)] = OUTLET_ZG;
          ++nzg;
        }
      }
  const ZgRows r = zg_rows(cls.data(), g);
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        const unsigned i = unsigned(x) + unsigned(y) * g.sy + unsigned(z) * g.sz;
        const bool row = zg_row(r, g, x, y, z);
        if (x != 0 && x != nx - 1) { CHECK(!row, "zg row off the x faces at (%d,%d,%d)", x, y, z); continue; }
        if (!nzg) CHECK(!row, "zg row without outlets at (%d,%d,%d)", x, y, z);
        const int sx = x == 0 ? 1 : -1;
        for (int k = 0; k < L::Q; ++k) {
          if (L::cx(k) != sx) continue;
          const unsigned j = same_x_neighbour(g, y, z, i, L::cy(k), L::cz(k));
          if (j == kNone) continue;
          if (cls[j] == OUTLET_ZG)
            CHECK(row, "node (%d,%d,%d) lends link %d to an outlet but is outside the zg rows (shape %d %d %d)",
                  x, y, z, k, nx, ny, nz);
        }
      }
}

int main() {
  const int per[4][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 1}};
  const int shapes3[][3] = {{3, 3, 3}, {5, 4, 3}, {130, 6, 5}, {128, 3, 4}, {129, 7, 6}, {256, 5, 3}, {7, 3, 130}};
  const int shapes2[][3] = {{3, 3, 1}, {10, 7, 1}, {131, 9, 3}, {128, 3, 1}, {300, 20, 2}, {257, 4, 5}};
  for (auto& p : per) {
    for (auto& s : shapes3) {
      check<D3Q19>(s[0], s[1], s[2], p[0], p[1], p[2]);
      check_split<D3Q19>(s[0], s[1], s[2], p[0], p[1], p[2]);
    }
    for (auto& s : shapes2) {
      check<D2Q9>(s[0], s[1], s[2], p[0], p[1], 0);
      check_split<D2Q9>(s[0], s[1], s[2], p[0], p[1], 0);
    }
  }
  // periodic axes may be short
  check<D3Q19>(1, 4, 4, 1, 0, 0);
  check<D3Q19>(6, 1, 4, 0, 1, 0);
  check<D3Q19>(6, 4, 1, 0, 0, 1);
  check<D3Q19>(2, 2, 2, 1, 1, 1);
  check<D2Q9>(1, 5, 1, 1, 0, 0);
  check<D2Q9>(6, 1, 3, 0, 1, 0);
  check<D2Q9>(2, 2, 2, 1, 1, 0);
  check_split<D3Q19>(1, 4, 4, 1, 0, 0);
  check_split<D3Q19>(6, 1, 4, 0, 1, 0);
  check_split<D3Q19>(6, 4, 1, 0, 0, 1);
  check_split<D3Q19>(2, 2, 2, 1, 1, 1);
  check_split<D2Q9>(1, 5, 1, 1, 0, 0);
  check_split<D2Q9>(6, 1, 3, 0, 1, 0);
  check_split<D2Q9>(2, 2, 2, 1, 1, 0);
  const int zgshape3[][3] = {{3, 3, 3}, {5, 9, 7}, {130, 12, 10}, {4, 40, 3}};
  const int zgshape2[][3] = {{3, 3, 1}, {10, 17, 1}, {131, 9, 3}};
  for (int py = 0; py < 2; ++py)
    for (int pz = 0; pz < 2; ++pz)
      for (int d : {0, 1, 5, 30, 100}) {
        for (auto& s : zgshape3) check_zg<D3Q19>(s[0], s[1], s[2], py, pz, 17u + unsigned(d), d);
        for (auto& s : zgshape2) check_zg<D2Q9>(s[0], s[1], s[2], py, 0, 29u + unsigned(d), d);
      }
  printf("%s (%d failures)\n", failures ? "FAILED" : "ok", failures);
  return failures ? 1 : 0;
}
