// Host-side checks of the tile-blocked numbering, the shell slots and the
// tail-node enumeration (the index logic shared by host and device code).
// Built and run by tests/test_host_logic.py; prints "ok" and exits 0 on success.
#include <cstdio>
#include <cstdlib>
#include <map>
#include <vector>

#include "../../paper_2205_08909_gb300/csrc/mfcg_internal.h"

using namespace mfcg;

#define REQUIRE(c)                                                              \
  do {                                                                          \
    if (!(c)) {                                                                 \
      std::printf("FAILED %s at line %d (p=%d N=%d,%d,%d T=%d,%d,%d)\n", #c, __LINE__, p, N[0], N[1], N[2], T[0], \
                  T[1], T[2]);                                                  \
      return 1;                                                                 \
    }                                                                           \
  } while (0)

static int check(int p, const int N[3], const int T[3]) {
  TileGeom g;
  int64_t fam[3];
  TailDiv td;
  init_tile_geom(p, N, T, g, fam, &td);
  const int64_t n = g.n_dofs;
  // 1. bijection onto [0, n)
  std::vector<int> hit(n, 0);
  for (int k = 0; k < g.nn[2]; ++k)
    for (int j = 0; j < g.nn[1]; ++j)
      for (int i = 0; i < g.nn[0]; ++i) {
        const int64_t id = node_index(g, i, j, k);
        REQUIRE(id >= 0 && id < n);
        hit[id]++;
      }
  for (int64_t t = 0; t < n; ++t) REQUIRE(hit[t] == 1);
  // 2. the owned nodes of every tile form one contiguous range, tiles in order
  int64_t expect_base = 0;
  for (int tz = 0; tz < g.nt[2]; ++tz)
    for (int ty = 0; ty < g.nt[1]; ++ty)
      for (int tx = 0; tx < g.nt[0]; ++tx) {
        const int ox = owned_count(g, 0, tx), oy = owned_count(g, 1, ty), oz = owned_count(g, 2, tz);
        int64_t lo = n, hi = -1;
        for (int lk = 0; lk < oz; ++lk)
          for (int lj = 0; lj < oy; ++lj)
            for (int li = 0; li < ox; ++li) {
              const int64_t id = node_index(g, p * g.T[0] * tx + li, p * g.T[1] * ty + lj, p * g.T[2] * tz + lk);
              lo = id < lo ? id : lo;
              hi = id > hi ? id : hi;
            }
        REQUIRE(lo == expect_base && hi - lo + 1 == (int64_t)ox * oy * oz);
        expect_base += (int64_t)ox * oy * oz;
        // the kernels' decoding of owned positions inverts owned_offset, and
        // the step visits the positions in order
        const OwnedShape sh = owned_shape(ox, oy, oz);
        int si = 0, sj = 0, sk = 0;
        for (int o = 0; o < ox * oy * oz; ++o) {
          int li, lj, lk;
          owned_coords(sh, o, li, lj, lk);
          REQUIRE(li >= 0 && li < ox && lj >= 0 && lj < oy && lk >= 0 && lk < oz);
          REQUIRE(owned_offset(li, lj, lk, ox, oy, oz) == o);
          if (o > 0) owned_next(sh, si, sj, sk);
          REQUIRE(si == li && sj == lj && sk == lk);
        }
      }
  // 3. shell writes of the tile kernel: unique slots
  std::map<int64_t, int64_t> slot_node;  // slot -> global node id written there
  for (int tz = 0; tz < g.nt[2]; ++tz)
    for (int ty = 0; ty < g.nt[1]; ++ty)
      for (int tx = 0; tx < g.nt[0]; ++tx) {
        const int64_t tile = tx + (int64_t)g.nt[0] * (ty + (int64_t)g.nt[1] * tz);
        const int bx = brick_extent(g, 0, tx), by = brick_extent(g, 1, ty), bz = brick_extent(g, 2, tz);
        const bool lastx = tx == g.nt[0] - 1, lasty = ty == g.nt[1] - 1, lastz = tz == g.nt[2] - 1;
        for (int lk = 0; lk < bz; ++lk)
          for (int lj = 0; lj < by; ++lj)
            for (int li = 0; li < bx; ++li) {
              const int i = p * g.T[0] * tx + li, j = p * g.T[1] * ty + lj, k = p * g.T[2] * tz + lk;
              const bool dir = is_dirichlet(g, i, j, k);
              const bool shared = !dir && ((li == 0 && tx > 0) || (li == bx - 1 && !lastx) || (lj == 0 && ty > 0) ||
                                           (lj == by - 1 && !lasty) || (lk == 0 && tz > 0) || (lk == bz - 1 && !lastz));
              if (!shared) continue;
              const int s = shell_slot(g, li, lj, lk, bx, by, bz);
              REQUIRE(s >= 0 && s < g.face_stride);
              const int64_t slot = tile * g.face_stride + s;
              REQUIRE(slot_node.count(slot) == 0);
              slot_node[slot] = i + (int64_t)g.nn[0] * (j + (int64_t)g.nn[1] * k);
            }
      }
  // 4. the tail enumerates exactly the shared non-Dirichlet nodes, once, and
  //    reads for each the slots its contributor tiles wrote for that node
  std::vector<int> seen(n, 0);
  int64_t reads = 0;
  for (int64_t t = 0; t < fam[0] + fam[1] + fam[2]; ++t) {
    int i, j, k;
    decode_tail_node(g, fam, td, t, i, j, k);
    REQUIRE(i > 0 && j > 0 && k > 0 && i < g.nn[0] - 1 && j < g.nn[1] - 1 && k < g.nn[2] - 1);
    const int64_t lex = i + (int64_t)g.nn[0] * (j + (int64_t)g.nn[1] * k);
    REQUIRE(seen[lex] == 0);
    seen[lex] = 1;
    int txs[2], lis[2], tys[2], ljs[2], tzs[2], lks[2];
    const int nx = contributors(g, 0, i, txs, lis), ny = contributors(g, 1, j, tys, ljs),
              nz = contributors(g, 2, k, tzs, lks);
    REQUIRE(nx * ny * nz >= 2);
    for (int cz = 0; cz < nz; ++cz)
      for (int cy = 0; cy < ny; ++cy)
        for (int cx = 0; cx < nx; ++cx) {
          const int64_t tl = txs[cx] + (int64_t)g.nt[0] * (tys[cy] + (int64_t)g.nt[1] * tzs[cz]);
          const int64_t slot = tl * g.face_stride + shell_slot(g, lis[cx], ljs[cy], lks[cz], brick_extent(g, 0, txs[cx]),
                                                               brick_extent(g, 1, tys[cy]), brick_extent(g, 2, tzs[cz]));
          REQUIRE(slot_node.count(slot) == 1 && slot_node[slot] == lex);
          ++reads;
        }
  }
  REQUIRE(reads == (int64_t)slot_node.size());  // every written partial is consumed exactly once
  for (int k = 1; k < g.nn[2] - 1; ++k)
    for (int j = 1; j < g.nn[1] - 1; ++j)
      for (int i = 1; i < g.nn[0] - 1; ++i) {
        auto plane = [&](int d, int x) { return x % (p * g.T[d]) == 0 && x > 0 && x < g.nn[d] - 1; };
        const bool shared = plane(0, i) || plane(1, j) || plane(2, k);
        REQUIRE(seen[i + (int64_t)g.nn[0] * (j + (int64_t)g.nn[1] * k)] == (shared ? 1 : 0));
      }
  return 0;
}

// multiply-shift division agrees with integer division
static int check_fastdiv() {
  const int p = 0, N[3] = {0, 0, 0}, T[3] = {0, 0, 0};
  for (uint32_t d = 1; d < 3000; ++d) {
    const FastDiv f = make_fastdiv(d);
    for (uint32_t n = 0; n < 5000; ++n) REQUIRE(fdiv(n, f) == n / d);
    for (uint32_t n = (1u << 31) - 5000; n < (1u << 31); n += 7) REQUIRE(fdiv(n, f) == n / d);
  }
  return 0;
}

int main() {
  int count = 0;
  if (check_fastdiv()) return 1;
  for (int p = 1; p <= 8; ++p) {
    const int meshes[][3] = {{1, 1, 1}, {2, 3, 4}, {5, 4, 3}, {7, 2, 9}, {8, 8, 8}, {9, 5, 6}};
    const int tiles[][3] = {{2, 2, 2}, {4, 4, 4}, {3, 2, 5}, {1, 1, 1}, {2, 3, 1}};
    for (auto& m : meshes)
      for (auto& t : tiles) {
        int T[3] = {t[0], t[1], t[2]};
        if (p == 1)
          for (int d = 0; d < 3; ++d) T[d] = T[d] < 2 ? 2 : T[d];
        if (check(p, m, T)) return 1;
        ++count;
      }
  }
  std::printf("ok %d layouts\n", count);
  return 0;
}
