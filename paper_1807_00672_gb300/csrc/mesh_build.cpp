// Host-side mesh construction (see mesh_build.h).
//
// Geometry of the cell-centred scheme (Sec. 2.2, Eq. 3): for each triangle its
// area Omega_i and perimeter; for each edge its length l_k and the unit normal
// n_k pointing out of its left cell. Computed in FP64 from the node
// coordinates and cast to the device precision at upload.
//
// Edge orientation: the left cell of an interior edge is the one with the
// lower caller index and the normal is taken along that cell's
// counter-clockwise traversal, so the library's faces are oriented the same
// way whatever internal numbering it uses.
//
// Compiled with -ffp-contract=off so each geometric quantity is the plainly
// rounded value of its formula.
#include "mesh_build.h"

#include "../../include/swe.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

namespace swe {

namespace {

// Spreads the low 32 bits of x to the even bit positions of a 64-bit word.
inline uint64_t spread_bits(uint64_t x) {
  x &= 0xffffffffull;
  x = (x | (x << 16)) & 0x0000ffff0000ffffull;
  x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
  x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
  x = (x | (x << 2)) & 0x3333333333333333ull;
  x = (x | (x << 1)) & 0x5555555555555555ull;
  return x;
}

}  // namespace

std::vector<int32_t> morton_order(const double* xy, int64_t V, const int32_t* tri, int64_t T) {
  double x0 = xy[0], x1 = xy[0], y0 = xy[1], y1 = xy[1];
  for (int64_t v = 0; v < V; ++v) {
    x0 = std::min(x0, xy[2 * v]); x1 = std::max(x1, xy[2 * v]);
    y0 = std::min(y0, xy[2 * v + 1]); y1 = std::max(y1, xy[2 * v + 1]);
  }
  double span = std::max(x1 - x0, y1 - y0);
  if (!(span > 0.0)) span = 1.0;
  const double q = 4194303.0;  // 22 bits per axis
  std::vector<uint64_t> key(T);
  for (int64_t i = 0; i < T; ++i) {
    int32_t a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
    double cx = (xy[2 * a] + xy[2 * b] + xy[2 * c]) / 3.0;
    double cy = (xy[2 * a + 1] + xy[2 * b + 1] + xy[2 * c + 1]) / 3.0;
    uint64_t ix = (uint64_t)std::min(q, std::max(0.0, (cx - x0) / span * q));
    uint64_t iy = (uint64_t)std::min(q, std::max(0.0, (cy - y0) / span * q));
    key[i] = spread_bits(ix) | (spread_bits(iy) << 1);
  }
  std::vector<int32_t> order(T);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t p, int32_t r) { return key[p] < key[r]; });
  return order;
}

std::vector<int32_t> rcm_order(int64_t T, const std::vector<int32_t>& nbr) {
  auto degree = [&](int64_t c) {
    int d = 0;
    for (int k = 0; k < 3; ++k) d += nbr[3 * c + k] >= 0;
    return d;
  };
  // Breadth-first levels from s over the unplaced cells of its component:
  // fills `seen` with stamp, returns the cells in visiting order and the
  // number of levels (the eccentricity of s plus one) in *levels.
  std::vector<int32_t> seen(T, -1), level(T, 0), queue;
  queue.reserve(T);
  auto bfs = [&](int32_t s, int32_t stamp, int* levels) {
    queue.clear();
    queue.push_back(s);
    seen[s] = stamp;
    level[s] = 0;
    for (size_t q = 0; q < queue.size(); ++q) {
      const int32_t c = queue[q];
      for (int k = 0; k < 3; ++k) {
        const int32_t d = nbr[3 * (int64_t)c + k];
        if (d < 0 || seen[d] == stamp) continue;
        seen[d] = stamp;
        level[d] = level[c] + 1;
        queue.push_back(d);
      }
    }
    *levels = level[queue.back()] + 1;
  };
  std::vector<uint8_t> placed(T, 0);
  std::vector<int32_t> order;
  order.reserve(T);
  int32_t stamp = 0;
  for (int64_t first = 0; first < T; ++first) {
    if (placed[first]) continue;
    // Start cell: lowest degree of the component (lowest index on ties),
    // then the pseudo-peripheral search of George and Liu: move to the
    // lowest-degree cell of the last level while that lengthens the levels.
    int levels = 0;
    bfs((int32_t)first, stamp, &levels);
    int32_t r = (int32_t)first;
    for (int32_t c : queue)
      if (degree(c) < degree(r) || (degree(c) == degree(r) && c < r)) r = c;
    ++stamp;
    bfs(r, stamp, &levels);
    for (int iter = 0; iter < 16; ++iter) {
      const int last = levels - 1;
      int32_t x = -1;
      for (int32_t c : queue)
        if (level[c] == last && (x < 0 || degree(c) < degree(x) || (degree(c) == degree(x) && c < x)))
          x = c;
      int lx = 0;
      ++stamp;
      bfs(x, stamp, &lx);
      if (lx <= levels) break;
      r = x;
      levels = lx;
    }
    // Cuthill-McKee from r: each cell's unplaced neighbours by increasing
    // degree, lower index first on ties.
    const size_t begin = order.size();
    order.push_back(r);
    placed[r] = 1;
    for (size_t q = begin; q < order.size(); ++q) {
      const int32_t c = order[q];
      int32_t next[3];
      int n = 0;
      for (int k = 0; k < 3; ++k) {
        const int32_t d = nbr[3 * (int64_t)c + k];
        if (d >= 0 && !placed[d]) {
          bool dup = false;
          for (int i = 0; i < n; ++i) dup = dup || next[i] == d;
          if (!dup) next[n++] = d;
        }
      }
      std::sort(next, next + n, [&](int32_t a, int32_t b) {
        const int da = degree(a), db = degree(b);
        return da != db ? da < db : a < b;
      });
      for (int i = 0; i < n; ++i) {
        placed[next[i]] = 1;
        order.push_back(next[i]);
      }
    }
    ++stamp;
  }
  std::reverse(order.begin(), order.end());
  return order;
}

namespace {

// Shared-memory accesses of one face record in the FP32 tiled step, in
// 16-byte units: the loads of its two cells (A, B) and the stores of its
// face slots on the sides that are tile cells. Wall and padding records
// (side B a wall) run another branch of the loop and are left out.
struct RecAccess {
  int32_t addr[4];
  bool on[4];
};

RecAccess rec_access(int32_t a, int32_t b, int tile) {
  RecAccess r{};
  const bool body = b != kWall;
  auto cell = [&](int32_t c) { return c < 0 ? ((-1 - c) & (tile - 1)) : c; };
  auto slot = [&](int32_t c) {
    const int s = -1 - c;
    return s + (s / tile) * kRecordSlotPad;
  };
  r.on[0] = r.on[1] = body;
  r.addr[0] = body ? cell(a) : 0;
  r.addr[1] = body ? cell(b) : 0;
  r.on[2] = body && a < 0;
  r.addr[2] = r.on[2] ? slot(a) : 0;
  r.on[3] = body && b < 0;
  r.addr[3] = r.on[3] ? slot(b) : 0;
  return r;
}

// The accesses of the records placed in one block of eight so far: per
// access and bank group (16-byte address mod 8) the distinct addresses. An
// access of the block takes as many shared-memory wavefronts as its fullest
// group holds addresses (one when all differ in group or coincide).
struct BlockBanks {
  int32_t seen[4][8][8];
  int8_t n[4][8];
  int8_t mx[4];
  void clear() {
    std::memset(n, 0, sizeof(n));
    std::memset(mx, 0, sizeof(mx));
  }
  bool has(int k, int g, int32_t addr) const {
    for (int i = 0; i < n[k][g]; ++i)
      if (seen[k][g][i] == addr) return true;
    return false;
  }
  // wavefronts the record would add to the block
  int cost(const RecAccess& r) const {
    int c = 0;
    for (int k = 0; k < 4; ++k) {
      if (!r.on[k]) continue;
      const int g = r.addr[k] & 7;
      if (!has(k, g, r.addr[k]) && n[k][g] + 1 > mx[k]) c += 1;
    }
    return c;
  }
  void add(const RecAccess& r) {
    for (int k = 0; k < 4; ++k) {
      if (!r.on[k]) continue;
      const int g = r.addr[k] & 7;
      if (has(k, g, r.addr[k])) continue;
      seen[k][g][n[k][g]++] = r.addr[k];
      if (n[k][g] > mx[k]) mx[k] = n[k][g];
    }
  }
};

// Record classes of the stored order: 0 both cells in the tile, 1 a halo
// side, 2 wall or padding.
int rec_class(int32_t a, int32_t b) { return b == kWall ? 2 : (a >= 0 || b >= 0) ? 1 : 0; }

// New order of records [r0, r1) of one tile: the kernel deals record r to
// the thread whose quarter warp takes the aligned block of eight r / 8, so
// each block is filled greedily, in order, with the first of the next
// kWindow unplaced records of the current class that adds no wavefront (or,
// if none, the one that adds the fewest). Classes stay contiguous and in
// their order; within a class the records stay close to their cell order.
void bank_order(const std::vector<int32_t>& tA, const std::vector<int32_t>& tB, int64_t r0,
                int64_t r1, int tile, std::vector<int32_t>& order) {
  constexpr size_t kWindow = 128;
  order.clear();
  BlockBanks bb;
  bb.clear();
  std::vector<char> used;
  int64_t i = r0;
  while (i < r1) {
    int64_t j = i;
    while (j < r1 && rec_class(tA[j], tB[j]) == rec_class(tA[i], tB[i])) ++j;
    used.assign((size_t)(j - i), 0);
    size_t head = 0;
    for (int64_t placed = 0; placed < j - i; ++placed) {
      if (order.size() % 8 == 0) bb.clear();
      while (used[head]) ++head;
      size_t best = head, seen = 0;
      int best_cost = 1 << 30;
      for (size_t k = head; k < used.size() && seen < kWindow; ++k) {
        if (used[k]) continue;
        ++seen;
        const int c = bb.cost(rec_access(tA[i + k], tB[i + k], tile));
        if (c < best_cost) {
          best_cost = c;
          best = k;
          if (c == 0) break;
        }
      }
      used[best] = 1;
      bb.add(rec_access(tA[i + best], tB[i + best], tile));
      order.push_back((int32_t)(i + best));
    }
    i = j;
  }
}

// Applies bank_order to every tile of m (host threads over tiles).
void order_records_for_banks(HostMesh& m) {
  const int64_t nt = m.ntiles;
  unsigned nth = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (m.T < 200000) nth = 1;
  auto work = [&](int64_t t0, int64_t t1) {
    std::vector<int32_t> order;
    std::vector<int32_t> a, b;
    std::vector<double> x, y, l;
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t r0 = m.toff[t], r1 = m.toff[t + 1];
      bank_order(m.tA, m.tB, r0, r1, m.tile, order);
      a.resize(order.size()); b.resize(order.size());
      x.resize(order.size()); y.resize(order.size()); l.resize(order.size());
      for (size_t q = 0; q < order.size(); ++q) {
        const int32_t r = order[q];
        a[q] = m.tA[r]; b[q] = m.tB[r]; x[q] = m.tnx[r]; y[q] = m.tny[r]; l[q] = m.tlen[r];
      }
      std::copy(a.begin(), a.end(), m.tA.begin() + r0);
      std::copy(b.begin(), b.end(), m.tB.begin() + r0);
      std::copy(x.begin(), x.end(), m.tnx.begin() + r0);
      std::copy(y.begin(), y.end(), m.tny.begin() + r0);
      std::copy(l.begin(), l.end(), m.tlen.begin() + r0);
    }
  };
  if (nth == 1) {
    work(0, nt);
    return;
  }
  // Ranges whose thread cannot be started are done on this thread.
  std::vector<std::thread> pool;
  unsigned started = 0;
  try {
    for (; started < nth; ++started)
      pool.emplace_back(work, nt * started / nth, nt * (started + 1) / nth);
  } catch (...) {
  }
  for (unsigned k = started; k < nth; ++k) work(nt * k / nth, nt * (k + 1) / nth);
  for (std::thread& th : pool) th.join();
}

}  // namespace

int build_host_mesh(const double* xy, int64_t V, const int32_t* tri_in, int64_t T, int order,
                    int32_t tile, bool with_edges, HostMesh& m, bool bank) {
  if (!xy || !tri_in || V <= 0 || T <= 0) return T == 0 ? -2 : -1;
  if (T >= (int64_t)INT32_MAX / 3 || V >= (int64_t)INT32_MAX) return -1;
  m = HostMesh();
  m.V = V;
  m.T = T;

  // 1. Validate, orient counter-clockwise, areas.
  std::vector<int32_t> tri(tri_in, tri_in + 3 * T);
  std::vector<double> area_c(T);
  for (int64_t i = 0; i < T; ++i) {
    int32_t a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
    if (a < 0 || b < 0 || c < 0 || a >= V || b >= V || c >= V) return -2;
    if (a == b || b == c || a == c) return -2;
    double ax = xy[2 * a], ay = xy[2 * a + 1];
    double s = 0.5 * ((xy[2 * b] - ax) * (xy[2 * c + 1] - ay) - (xy[2 * c] - ax) * (xy[2 * b + 1] - ay));
    if (!std::isfinite(s) || s == 0.0) return -2;
    if (s < 0.0) {
      tri[3 * i + 1] = c;
      tri[3 * i + 2] = b;
      s = -s;
    }
    area_c[i] = s;
  }

  // 2. Half-edges bucketed by their lower node (counting sort), then matched
  //    within each bucket by their upper node.
  std::vector<int64_t> start(V + 1, 0);
  for (int64_t i = 0; i < 3 * T; ++i) {
    int64_t cell = i / 3;
    int k = (int)(i % 3);
    int32_t a = tri[3 * cell + k], b = tri[3 * cell + (k + 1) % 3];
    start[std::min(a, b) + 1]++;
  }
  for (int64_t v = 0; v < V; ++v) start[v + 1] += start[v];
  std::vector<int64_t> fill(start.begin(), start.end() - 1);
  std::vector<int64_t> bucket(3 * T);  // half-edge id = 3 * cell + k
  for (int64_t i = 0; i < 3 * T; ++i) {
    int64_t cell = i / 3;
    int k = (int)(i % 3);
    int32_t a = tri[3 * cell + k], b = tri[3 * cell + (k + 1) % 3];
    bucket[fill[std::min(a, b)]++] = i;
  }
  // edge_of_half[h] = caller-side edge id; edges listed in bucket order.
  std::vector<int32_t> edge_of_half(3 * T, -1);
  std::vector<int32_t> cL, cR;  // caller cell ids; cR = -1 for walls
  std::vector<int8_t> kL;      // face index of the edge within its left cell
  cL.reserve(3 * T / 2 + 16);
  cR.reserve(3 * T / 2 + 16);
  kL.reserve(3 * T / 2 + 16);
  auto upper = [&](int64_t h) {
    int64_t cell = h / 3;
    int k = (int)(h % 3);
    return std::max(tri[3 * cell + k], tri[3 * cell + (k + 1) % 3]);
  };
  for (int64_t v = 0; v < V; ++v) {
    int64_t b0 = start[v], b1 = start[v + 1];
    // sort the (few) half-edges of this bucket by (upper node, cell)
    std::sort(bucket.begin() + b0, bucket.begin() + b1, [&](int64_t p, int64_t q) {
      int32_t up = upper(p), uq = upper(q);
      if (up != uq) return up < uq;
      return p < q;
    });
    int64_t j = b0;
    while (j < b1) {
      int64_t r = j + 1;
      while (r < b1 && upper(bucket[r]) == upper(bucket[j])) ++r;
      if (r - j > 2) return -2;  // non-manifold edge
      int32_t e = (int32_t)cL.size();
      int64_t h0 = bucket[j];
      if (r - j == 2) {
        int64_t h1 = bucket[j + 1];
        if (h0 / 3 == h1 / 3) return -2;
        // h0 < h1 and half-edge ids grow with the cell: h0 is the lower cell
        cL.push_back((int32_t)(h0 / 3));
        cR.push_back((int32_t)(h1 / 3));
        kL.push_back((int8_t)(h0 % 3));
        edge_of_half[h0] = e;
        edge_of_half[h1] = e;
      } else {
        cL.push_back((int32_t)(h0 / 3));
        cR.push_back(-1);
        kL.push_back((int8_t)(h0 % 3));
        edge_of_half[h0] = e;
        m.Eb++;
      }
      j = r;
    }
  }
  m.E = (int64_t)cL.size();

  // 3. Edge geometry from the left cell's traversal.
  std::vector<double> gnx(m.E), gny(m.E), glen(m.E);
  for (int64_t e = 0; e < m.E; ++e) {
    int32_t c = cL[e];
    int k = kL[e];
    int32_t a = tri[3 * (int64_t)c + k], b = tri[3 * (int64_t)c + (k + 1) % 3];
    double dx = xy[2 * b] - xy[2 * a];
    double dy = xy[2 * b + 1] - xy[2 * a + 1];
    double l = std::sqrt(dx * dx + dy * dy);
    gnx[e] = dy / l;
    gny[e] = -dx / l;
    glen[e] = l;
  }

  // 4. Cell order.
  m.perm.resize(T);
  std::iota(m.perm.begin(), m.perm.end(), 0);
  if (order == 1) {
    m.perm = morton_order(xy, V, tri.data(), T);
  } else if (order == 2) {
    std::vector<int32_t> nbr(3 * T, -1);  // edge neighbours, by face
    for (int64_t i = 0; i < T; ++i)
      for (int k = 0; k < 3; ++k) {
        const int32_t e = edge_of_half[3 * i + k];
        nbr[3 * i + k] = (cL[e] == i) ? cR[e] : cL[e];
      }
    m.perm = rcm_order(T, nbr);
  } else if (order != 0) {
    return -1;
  }
  m.iperm.resize(T);
  for (int64_t j = 0; j < T; ++j) m.iperm[m.perm[j]] = (int32_t)j;

  // 5. Internal-order cell data: area and perimeter (faces k = 0, 1, 2).
  m.area.resize(T);
  m.perim.resize(T);
  for (int64_t j = 0; j < T; ++j) {
    int64_t i = m.perm[j];
    double p = 0.0;
    for (int k = 0; k < 3; ++k) p = p + glen[edge_of_half[3 * i + k]];
    m.area[j] = area_c[i];
    m.perim[j] = p;
  }

  // 6. Two-launch layout: edges sorted by their lower internal cell.
  if (with_edges) {
    std::vector<int64_t> ekey(m.E);
    for (int64_t e = 0; e < m.E; ++e) {
      int64_t a = m.iperm[cL[e]];
      int64_t b = cR[e] >= 0 ? m.iperm[cR[e]] : a;
      ekey[e] = (std::min(a, b) << 32) | std::max(a, b);
    }
    std::vector<int32_t> eorder(m.E);
    std::iota(eorder.begin(), eorder.end(), 0);
    std::stable_sort(eorder.begin(), eorder.end(),
                     [&](int32_t p, int32_t r) { return ekey[p] < ekey[r]; });
    std::vector<int32_t> enew(m.E);
    m.eL.resize(m.E); m.eR.resize(m.E); m.nx.resize(m.E); m.ny.resize(m.E); m.len.resize(m.E);
    for (int64_t s = 0; s < m.E; ++s) {
      int32_t e = eorder[s];
      enew[e] = (int32_t)s;
      m.eL[s] = m.iperm[cL[e]];
      m.eR[s] = cR[e] >= 0 ? m.iperm[cR[e]] : -1;
      m.nx[s] = gnx[e]; m.ny[s] = gny[e]; m.len[s] = glen[e];
    }
    for (int k = 0; k < 3; ++k) m.cface[k].resize(T);
    for (int64_t j = 0; j < T; ++j) {
      int64_t i = m.perm[j];
      for (int k = 0; k < 3; ++k) {
        int32_t e = edge_of_half[3 * i + k];
        bool right = (cL[e] != i);
        m.cface[k][j] = enew[e] | (right ? (int32_t)0x80000000 : 0);
      }
    }
  }

  // 7. Tiled layout.
  if (tile > 0) {
    if (tile % 32 != 0 || tile > 4096) return -1;
    m.tile = tile;
    m.ntiles = (T + tile - 1) / tile;
    m.toff.assign(1, 0);
    m.hoff.assign(1, 0);
    m.tA.reserve((size_t)(1.75 * T) + 64);
    // Per tile: every face of every tile cell, an interior face whose cells
    // are both in the tile emitted once. Sides: a tile cell by its face slot
    // (face k of tile cell j is slot k * tile + j, encoded -1 - slot), a cell
    // of another tile as tile + its index in the tile's halo list (where the
    // kernels stage it, after the tile's cells), a wall as kWall. Records with both cells in the tile come first, then those with a
    // halo side, then walls (fewer divergent warps); within a class, in cell
    // order. Record and halo lists are padded to multiples of 4 entries
    // (null records: both sides kWall, zero length; halo padding repeats the
    // tile's first cell).
    struct Rec { int32_t a, b; int32_t e; int cls; };
    std::vector<Rec> recs;
    std::vector<int32_t> halo;
    std::vector<int32_t> halo_pos(T, -1);  // internal cell -> index in the current halo
    for (int64_t t = 0; t < m.ntiles; ++t) {
      recs.clear();
      halo.clear();
      const int64_t j0 = t * tile, j1 = std::min<int64_t>(T, j0 + tile);
      for (int64_t j = j0; j < j1; ++j) {
        int64_t i = m.perm[j];
        for (int k = 0; k < 3; ++k) {
          int32_t e = edge_of_half[3 * i + k];
          bool right = (cL[e] != i);
          int32_t other = right ? cL[e] : cR[e];
          int64_t jo = other >= 0 ? m.iperm[other] : -1;
          bool other_local = (jo >= j0 && jo < j1);
          if (right && other_local) continue;
          int32_t slot_self = -1 - (int32_t)(k * tile + (j - j0));
          int32_t enc_other;
          int cls;
          if (jo < 0) {
            enc_other = kWall;
            cls = 2;
          } else if (other_local) {
            int ko = -1;  // the other cell's face index for this edge
            for (int kk = 0; kk < 3; ++kk)
              if (edge_of_half[3 * (int64_t)other + kk] == e) ko = kk;
            enc_other = -1 - (int32_t)(ko * tile + (jo - j0));
            cls = 0;
          } else {
            if (halo_pos[jo] < 0) {
              halo_pos[jo] = (int32_t)halo.size();
              halo.push_back((int32_t)jo);
            }
            enc_other = tile + halo_pos[jo];  // the cell's place after the tile's cells
            cls = 1;
          }
          // side A is always the edge's left cell
          if (!right) recs.push_back({slot_self, enc_other, e, cls});
          else        recs.push_back({enc_other, slot_self, e, cls});
        }
      }
      for (int32_t c : halo) halo_pos[c] = -1;
      std::stable_sort(recs.begin(), recs.end(),
                       [](const Rec& p, const Rec& q) { return p.cls < q.cls; });
      const size_t nrec = (recs.size() + 3) / 4 * 4;
      for (const Rec& rc : recs) {
        m.tA.push_back(rc.a);
        m.tB.push_back(rc.b);
        m.tnx.push_back(gnx[rc.e]);
        m.tny.push_back(gny[rc.e]);
        m.tlen.push_back(glen[rc.e]);
      }
      for (size_t r = recs.size(); r < nrec; ++r) {
        m.tA.push_back(kWall);
        m.tB.push_back(kWall);
        m.tnx.push_back(0.0);
        m.tny.push_back(0.0);
        m.tlen.push_back(0.0);
        m.null_records++;
      }
      m.toff.push_back((int64_t)m.tA.size());
      const size_t nh = (halo.size() + 3) / 4 * 4;
      for (int32_t c : halo) m.hidx.push_back(c);
      for (size_t h = halo.size(); h < nh; ++h) m.hidx.push_back((int32_t)j0);
      m.hoff.push_back((int64_t)m.hidx.size());
      m.rec_cap = std::max<int64_t>(m.rec_cap, (int64_t)nrec);
      m.halo_cap = std::max<int64_t>(m.halo_cap, (int64_t)nh);
    }
    if (m.halo_cap == 0) m.halo_cap = 4;
    if (bank) order_records_for_banks(m);
  }
  return 0;
}

}  // namespace swe

extern "C" swe_status swe_cell_order(const double* xy, int64_t n_nodes, const int32_t* tri,
                                     int64_t n_tris, int32_t order, int32_t* perm) {
  if (!perm || order < SWE_ORDER_NONE || order > SWE_ORDER_RCM) return SWE_EINVAL;
  return swe::guarded([&] {
    swe::HostMesh hm;
    const int rc = swe::build_host_mesh(xy, n_nodes, tri, n_tris, order, 0, false, hm);
    if (rc == -2) return SWE_EMESH;
    if (rc != 0) return SWE_EINVAL;
    std::copy(hm.perm.begin(), hm.perm.end(), perm);
    return SWE_OK;
  });
}
