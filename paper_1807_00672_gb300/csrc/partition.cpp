// Domain decomposition of one mesh into sub-domains (the paper's stated
// future work, Sec. 5: several GPUs on one mesh), host side.
//
// Cells are ordered by the Morton code of their centroids and split into
// n_parts contiguous ranges of (nearly) equal size; part p owns its range.
// Each part's local mesh holds its own cells and one ring of ghost cells:
// the cells of other parts that share an edge with one of its cells. Local
// cells keep the global order (sorted by global index), and each local
// triangle keeps its global node order, so every face of an owned cell is
// oriented, and every cell's faces are ordered, exactly as in the whole mesh
// (the edge's left cell is its lower index): one step of the local mesh
// updates the owned cells bit for bit as one step of the whole mesh does,
// provided the ghosts hold their owners' current values and the step uses
// the global time step. The exchange plan lists, for each ordered pair of
// parts (from, to), the cells owned by `from` that `to` holds as ghosts, in
// global order, by their local indices on both sides.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <numeric>
#include <vector>

#include "../../include/swe.h"
#include "mesh_build.h"

struct swe_partition {
  int32_t nparts = 0;
  int64_t T = 0;
  std::vector<int32_t> owner;  // part owning each global cell
  struct Part {
    std::vector<int32_t> cells;  // global ids of the local cells, ascending
    std::vector<uint8_t> ghost;  // 1: a copy of another part's cell
    std::vector<int32_t> nodes;  // global ids of the local nodes, ascending
    std::vector<int32_t> tri;    // local triangles (local node ids, global node order)
    int64_t nghost = 0;
  };
  std::vector<Part> parts;
};

namespace {

// Local index of global cell c in a part (its cells are ascending), or -1.
int64_t local_index(const swe_partition::Part& p, int32_t c) {
  auto it = std::lower_bound(p.cells.begin(), p.cells.end(), c);
  if (it == p.cells.end() || *it != c) return -1;
  return it - p.cells.begin();
}

}  // namespace

extern "C" {

static swe_status partition_create(const double* xy, int64_t n_nodes, const int32_t* tri,
                                   int64_t n_tris, int32_t n_parts, swe_partition** out) {
  if (!out) return SWE_EINVAL;
  *out = nullptr;
  if (!xy || !tri || n_nodes <= 0 || n_tris < 0 || n_parts < 1) return SWE_EINVAL;
  if (n_tris == 0) return SWE_EMESH;
  if (n_parts > n_tris || n_tris >= (int64_t)INT32_MAX / 3 || n_nodes >= (int64_t)INT32_MAX)
    return SWE_EINVAL;
  const int64_t T = n_tris;
  for (int64_t i = 0; i < 3 * T; ++i)
    if (tri[i] < 0 || tri[i] >= n_nodes) return SWE_EMESH;

  // Edge neighbours: half-edges sorted by their (lower, upper) node pair.
  struct Half {
    uint64_t key;
    int32_t cell;
  };
  std::vector<Half> half(3 * T);
  for (int64_t i = 0; i < T; ++i)
    for (int k = 0; k < 3; ++k) {
      const uint64_t a = (uint32_t)tri[3 * i + k], b = (uint32_t)tri[3 * i + (k + 1) % 3];
      if (a == b) return SWE_EMESH;
      half[3 * i + k] = {(std::min(a, b) << 32) | std::max(a, b), (int32_t)i};
    }
  std::sort(half.begin(), half.end(), [](const Half& p, const Half& q) {
    return p.key != q.key ? p.key < q.key : p.cell < q.cell;
  });
  std::vector<int32_t> nbr(3 * T, -1);  // up to three neighbours per cell
  std::vector<uint8_t> nn(T, 0);
  for (size_t j = 0; j < half.size();) {
    size_t r = j + 1;
    while (r < half.size() && half[r].key == half[j].key) ++r;
    if (r - j > 2) return SWE_EMESH;  // an edge of more than two triangles
    if (r - j == 2) {
      const int32_t a = half[j].cell, b = half[j + 1].cell;
      if (a == b) return SWE_EMESH;
      nbr[3 * (int64_t)a + nn[a]++] = b;
      nbr[3 * (int64_t)b + nn[b]++] = a;
    }
    j = r;
  }

  // Morton order of the centroids (as the library's cell renumbering),
  // split into contiguous ranges.
  const std::vector<int32_t> order = swe::morton_order(xy, n_nodes, tri, T);

  swe_partition* P = new swe_partition();
  P->nparts = n_parts;
  P->T = T;
  P->owner.assign(T, 0);
  for (int32_t p = 0; p < n_parts; ++p) {
    const int64_t b = T * p / n_parts, e = T * (p + 1) / n_parts;
    for (int64_t j = b; j < e; ++j) P->owner[order[j]] = p;
  }
  P->parts.resize(n_parts);
  std::vector<uint8_t> mark(T, 0);
  std::vector<int32_t> node_local(n_nodes, -1);
  for (int32_t p = 0; p < n_parts; ++p) {
    swe_partition::Part& part = P->parts[p];
    const int64_t b = T * p / n_parts, e = T * (p + 1) / n_parts;
    for (int64_t j = b; j < e; ++j) {
      const int32_t c = order[j];
      if (!mark[c]) { mark[c] = 1; part.cells.push_back(c); }
      for (int k = 0; k < nn[c]; ++k) {
        const int32_t d = nbr[3 * (int64_t)c + k];
        if (!mark[d]) { mark[d] = 1; part.cells.push_back(d); }
      }
    }
    std::sort(part.cells.begin(), part.cells.end());
    part.ghost.resize(part.cells.size());
    part.nodes.reserve(3 * part.cells.size());
    for (size_t l = 0; l < part.cells.size(); ++l) {
      const int32_t c = part.cells[l];
      mark[c] = 0;
      part.ghost[l] = P->owner[c] != p ? 1 : 0;
      part.nghost += part.ghost[l];
      for (int k = 0; k < 3; ++k) part.nodes.push_back(tri[3 * (int64_t)c + k]);
    }
    std::sort(part.nodes.begin(), part.nodes.end());
    part.nodes.erase(std::unique(part.nodes.begin(), part.nodes.end()), part.nodes.end());
    for (size_t l = 0; l < part.nodes.size(); ++l) node_local[part.nodes[l]] = (int32_t)l;
    part.tri.resize(3 * part.cells.size());
    for (size_t l = 0; l < part.cells.size(); ++l)
      for (int k = 0; k < 3; ++k) part.tri[3 * l + k] = node_local[tri[3 * (int64_t)part.cells[l] + k]];
    for (int32_t v : part.nodes) node_local[v] = -1;
  }
  *out = P;
  return SWE_OK;
}

swe_status swe_partition_create(const double* xy, int64_t n_nodes, const int32_t* tri,
                                int64_t n_tris, int32_t n_parts, swe_partition** out) {
  if (out) *out = nullptr;
  return swe::guarded([&] { return partition_create(xy, n_nodes, tri, n_tris, n_parts, out); });
}

swe_status swe_partition_sizes(const swe_partition* P, int32_t part, int64_t* sizes) {
  if (!P || !sizes || part < 0 || part >= P->nparts) return SWE_EINVAL;
  const swe_partition::Part& p = P->parts[part];
  sizes[0] = (int64_t)p.cells.size();
  sizes[1] = p.nghost;
  sizes[2] = (int64_t)p.nodes.size();
  return SWE_OK;
}

swe_status swe_partition_local_mesh(const swe_partition* P, int32_t part, const double* xy,
                                    int32_t* cells, uint8_t* ghost, double* local_xy,
                                    int32_t* local_tri) {
  if (!P || part < 0 || part >= P->nparts || (local_xy && !xy)) return SWE_EINVAL;
  const swe_partition::Part& p = P->parts[part];
  if (cells) std::copy(p.cells.begin(), p.cells.end(), cells);
  if (ghost) std::copy(p.ghost.begin(), p.ghost.end(), ghost);
  if (local_xy)
    for (size_t l = 0; l < p.nodes.size(); ++l) {
      local_xy[2 * l] = xy[2 * (int64_t)p.nodes[l]];
      local_xy[2 * l + 1] = xy[2 * (int64_t)p.nodes[l] + 1];
    }
  if (local_tri) std::copy(p.tri.begin(), p.tri.end(), local_tri);
  return SWE_OK;
}

swe_status swe_partition_exchange(const swe_partition* P, int32_t from, int32_t to, int64_t* n,
                                  int32_t* from_cells, int32_t* to_cells) {
  if (!P || !n || from < 0 || to < 0 || from >= P->nparts || to >= P->nparts) return SWE_EINVAL;
  const swe_partition::Part& f = P->parts[from];
  const swe_partition::Part& t = P->parts[to];
  int64_t k = 0;
  if (from != to)
    for (size_t l = 0; l < t.cells.size(); ++l) {
      if (!t.ghost[l] || P->owner[t.cells[l]] != from) continue;
      if (from_cells) from_cells[k] = (int32_t)local_index(f, t.cells[l]);
      if (to_cells) to_cells[k] = (int32_t)l;
      ++k;
    }
  *n = k;
  return SWE_OK;
}

void swe_partition_destroy(swe_partition* P) { delete P; }

}  // extern "C"
