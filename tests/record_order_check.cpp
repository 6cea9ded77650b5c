// Host check of the FP32 tiled layout's record order (mesh_build.cpp,
// bank_order): for every tile the records built with the bank-aware order
// are a permutation of those built without it, each record keeping its
// geometry, and the three record classes (both cells in the tile, a halo
// side, walls and padding) stay contiguous and in that order. Reads a mesh
// (int64 V, int64 T, V x 2 doubles, T x 3 int32) from argv[1]; prints
// "ok <tiles> <records>" or the first failure, and exits non-zero on one.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <tuple>
#include <vector>

#include "../paper_1807_00672_gb300/csrc/mesh_build.h"

namespace {

int rec_class(int32_t a, int32_t b) {
  return b == swe::kWall ? 2 : (a >= 0 || b >= 0) ? 1 : 0;
}

using Rec = std::tuple<int32_t, int32_t, double, double, double>;

}  // namespace

int main(int argc, char** argv) {
  if (argc < 3) return 2;
  FILE* f = std::fopen(argv[1], "rb");
  if (!f) return 2;
  int64_t V = 0, T = 0;
  if (std::fread(&V, 8, 1, f) != 1 || std::fread(&T, 8, 1, f) != 1) return 2;
  std::vector<double> xy(2 * V);
  std::vector<int32_t> tri(3 * T);
  if (std::fread(xy.data(), 8, 2 * V, f) != (size_t)(2 * V) ||
      std::fread(tri.data(), 4, 3 * T, f) != (size_t)(3 * T))
    return 2;
  std::fclose(f);
  const int tile = std::atoi(argv[2]);
  swe::HostMesh plain, banked;
  if (swe::build_host_mesh(xy.data(), V, tri.data(), T, 1, tile, false, plain, false) != 0) return 3;
  if (swe::build_host_mesh(xy.data(), V, tri.data(), T, 1, tile, false, banked, true) != 0) return 3;
  if (plain.toff != banked.toff || plain.hidx != banked.hidx) {
    std::printf("tile offsets or halo lists differ\n");
    return 1;
  }
  int64_t nrec = 0;
  for (int64_t t = 0; t < plain.ntiles; ++t) {
    std::vector<Rec> p, b;
    int last_class = 0;
    for (int64_t r = plain.toff[t]; r < plain.toff[t + 1]; ++r) {
      p.emplace_back(plain.tA[r], plain.tB[r], plain.tnx[r], plain.tny[r], plain.tlen[r]);
      b.emplace_back(banked.tA[r], banked.tB[r], banked.tnx[r], banked.tny[r], banked.tlen[r]);
      const int c = rec_class(banked.tA[r], banked.tB[r]);
      if (c < last_class) {
        std::printf("tile %lld: record classes out of order at record %lld\n", (long long)t,
                    (long long)r);
        return 1;
      }
      last_class = c;
    }
    nrec += (int64_t)p.size();
    std::sort(p.begin(), p.end());
    std::sort(b.begin(), b.end());
    if (p != b) {
      std::printf("tile %lld: records are not a permutation of the stored ones\n", (long long)t);
      return 1;
    }
  }
  std::printf("ok %lld %lld\n", (long long)plain.ntiles, (long long)nrec);
  return 0;
}
