// Host-side mesh construction for the CUDA step: edges, FP64 geometry,
// locality renumbering and per-tile face lists. No CUDA in here.
#pragma once

#include <cstdint>
#include <new>
#include <vector>

namespace swe {

// Runs a C-ABI call's body so that no C++ exception crosses the boundary:
// std::bad_alloc becomes status -3 (SWE_ENOMEM), any other exception -1
// (SWE_EINVAL).
template <typename F>
int guarded(F&& body) noexcept {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return -3;
  } catch (...) {
    return -1;
  }
}

// Encoding of one side of a tile face record:
//   >= 0             tile + q for the cell of another tile at index q of the
//                    tile's halo list (its place after the tile's cells)
//   kWall            wall (mirror ghost)
//   < 0, != kWall    local face slot s = -1 - value: face s / tile of tile cell s % tile
constexpr int32_t kWall = INT32_MIN;

struct HostMesh {
  int64_t V = 0, T = 0, E = 0, Eb = 0;
  // perm[j] = caller index of internal cell j; iperm is its inverse.
  std::vector<int32_t> perm, iperm;
  // Internal-order cell data (FP64).
  std::vector<double> area, perim;
  // Two-launch layout: edges in internal order, and per cell the ids of its
  // three faces (face k joins the cell's oriented nodes k and k+1), with bit 31
  // set when the cell is the edge's right side.
  std::vector<int32_t> eL, eR;   // eR = -1 for a wall
  std::vector<double> nx, ny, len;
  std::vector<int32_t> cface[3];
  // Tiled layout: tiles of `tile` consecutive internal cells. Tile t owns
  // the face records [toff[t], toff[t+1]), each with two encoded sides and
  // the edge's geometry oriented from side A (the edge's left cell) to side
  // B, and the halo list hidx[hoff[t] .. hoff[t+1]) of the internal indices
  // of the other tiles' cells its records touch. rec_cap and halo_cap are
  // the largest padded record and halo counts of any tile.
  int32_t tile = 0;
  int64_t ntiles = 0;
  std::vector<int64_t> toff, hoff;
  std::vector<int32_t> tA, tB, hidx;
  std::vector<double> tnx, tny, tlen;
  int64_t rec_cap = 0, halo_cap = 0;
  int64_t null_records = 0;
};

// Cells ordered by the Z-order (Morton) code of their centroids, 22 bits per
// axis over the nodes' bounding square; ties keep the caller order. Node ids
// must be valid.
std::vector<int32_t> morton_order(const double* xy, int64_t V, const int32_t* tri, int64_t T);

// Reverse Cuthill-McKee order of the cells of a graph given as three
// neighbours per cell (-1: none): breadth-first from a pseudo-peripheral
// cell of each connected component (George and Liu's search), every visited
// cell's unvisited neighbours appended by increasing degree (lower index on
// ties), the whole sequence reversed. order[j] = the cell at position j.
std::vector<int32_t> rcm_order(int64_t T, const std::vector<int32_t>& nbr);

// Offset, in slots, between the face slots of consecutive faces k of the
// FP32 tiled step (face k of tile cell j at k (tile + pad) + j); the same
// value as the kernels' kSlotPad, which the record order below models.
constexpr int kRecordSlotPad = 3;

// Returns 0 or a negative status: -1 bad arguments, -2 invalid mesh.
// order: 0 = caller order, 1 = Morton order of centroids, 2 = reverse
// Cuthill-McKee order of the edge-neighbour graph.
// tile > 0 also builds the tiled layout; with_edges builds the two-launch one.
// bank_order (FP32 tiled step): within each class of a tile's records, the
// records are reordered so that the eight records one quarter warp handles
// at a time spread their shared-memory accesses over the banks (see
// order_records_for_banks); results do not depend on the order.
int build_host_mesh(const double* xy, int64_t V, const int32_t* tri, int64_t T, int order,
                    int32_t tile, bool with_edges, HostMesh& out, bool bank_order = false);

}  // namespace swe
