// Internal to libswe: the handle structures behind the C ABI and the helpers
// its translation units share. Not part of the public interface.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/swe.h"
#include "swe_kernels.cuh"

namespace swe_host {

// Message of the last failed CUDA call on this thread (swe_last_cuda_error).
extern thread_local std::string g_cuda_msg;

// Records the failure of a CUDA call (message, call text, file, line); true
// if e is an error.
bool cuda_failed_at(cudaError_t e, const char* what, const char* file, int line);

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Bump allocator over one cudaMalloc. take() returns nullptr (and sets
// overflow) instead of handing out memory past the allocation.
struct Arena {
  char* base = nullptr;
  size_t size = 0, used = 0;
  bool overflow = false;
  void* take(size_t bytes) {
    if (used + align_up(bytes) > size) {
      overflow = true;
      return nullptr;
    }
    void* p = base + used;
    used += align_up(bytes);
    return p;
  }
};

struct Layout {
  size_t total = 0;
  void add(size_t bytes) { total += align_up(bytes); }
};

// Where one scenario lives inside the mesh.
struct Scenario {
  int64_t caller0 = 0;  // first caller cell index (scenarios are concatenated)
  int64_t ncells = 0;
  int64_t cell0 = 0;    // first internal cell (tile-aligned in the tiled layout)
  int64_t tile0 = 0, ntiles = 0;
  int64_t chunk0 = 0, nchunks = 0;  // work chunks (= mass partial slots) of the tiled kernel
};

}  // namespace swe_host

struct swe_mesh {
  swe_params prm{};
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t V = 0, T = 0, E = 0, Eb = 0;
  int kernel = SWE_KERNEL_TILED;
  int tile = 256;
  int64_t ntiles = 0, records = 0, halos = 0;
  int stages = 2;
  int cpt = 2;  // cells per thread of the tiled kernel (threads = tile / cpt)
  swe::TileLayout layout{};
  int64_t Tp = 0;  // internal cell slots (tiled: scenarios padded to whole tiles)
  std::vector<swe_host::Scenario> scen;
  int64_t nchunks = 0;
  swe_host::Arena arena;
  int32_t* perm = nullptr;  // internal cell -> caller cell (-1 for padding)
  void* area = nullptr;
  void* irP = nullptr;
  void* rarea = nullptr;  // 1 / area, FP64 tiled meshes
  int32_t* iperm = nullptr;  // caller cell -> internal cell
  bool ghosts = false;       // swe_mesh_create_part: some cells are ghosts
  int32_t *eL = nullptr, *eR = nullptr, *cf[3] = {nullptr, nullptr, nullptr};
  void *nx = nullptr, *ny = nullptr, *len = nullptr;
  int64_t *toff = nullptr, *hoff = nullptr;
  int32_t *tS = nullptr, *hidx = nullptr;
  int32_t* hpad = nullptr;  // halo lists padded to halo_cap per tile (layout.hreg)
  void *tg0 = nullptr, *tg1 = nullptr, *tg2 = nullptr;
  void* trec = nullptr;  // FP32: interleaved records {packed sides, nx, ny, l}
  swe::Chunk* chunks = nullptr;  // work of each block of the tiled kernels
  swe::Chunk* chunks_back = nullptr;  // the same chunks, tiles last to first
  swe::Chunk* chunks_pool = nullptr;  // k_tiled_step's chunks with tile pools
  swe::Chunk* chunks_pool_back = nullptr;  // the same, walked backwards
  bool pooled = false;  // the step launches the pooled k_tiled_step on chunks_pool*
  int grid_edge = 1, grid_cell = 1, grid_cfl = 1, max_grid = 1;
  // Handles that use this mesh (states). swe_mesh_destroy while some are
  // alive only marks the mesh; the last of them to go frees it.
  int refs = 0;
  bool dead = false;
};

struct swe_state {
  swe_mesh* mesh = nullptr;
  swe_host::Arena arena;
  void *h[2] = {nullptr, nullptr}, *hu[2] = {nullptr, nullptr}, *hv[2] = {nullptr, nullptr};
  void *z = nullptr, *gn2 = nullptr;
  void* hlo = nullptr;  // FP32 depth residual per cell (compensated_depth), else null
  int stride = 1;  // 4: interleaved cells (h, hu, hv, z) for the tiled kernel
  void* fx[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  double* partial = nullptr;
  double* stage = nullptr;       // T doubles in caller order
  swe::Ctl* ctl = nullptr;       // one per scenario
  swe::Ctl* host_ctl = nullptr;  // pinned mirror
  cudaStream_t capture = nullptr;
  cudaGraphExec_t graph = nullptr;
  bool open_ended = true;  // the device t_end is +inf for every scenario
  bool walk_back = false;  // the next step walks the chunks backwards
};

namespace swe_host {

inline int nscen(const swe_mesh* m) { return (int)m->scen.size(); }

inline swe::Num num_of(const swe_mesh* m) {
  return swe::make_num(m->prm.g, m->prm.courant, m->prm.h_eps, m->prm.wait_rounds);
}

template <typename Real>
swe::DevMesh<Real> dev_mesh(const swe_mesh* m) {
  swe::DevMesh<Real> d{};
  d.T = m->T;
  d.E = m->E;
  d.area = (const Real*)m->area;
  d.irP = (const Real*)m->irP;
  d.rarea = (const Real*)m->rarea;
  d.eL = m->eL;
  d.eR = m->eR;
  d.nx = (const Real*)m->nx;
  d.ny = (const Real*)m->ny;
  d.len = (const Real*)m->len;
  d.cf0 = m->cf[0];
  d.cf1 = m->cf[1];
  d.cf2 = m->cf[2];
  d.chunks = m->chunks;
  d.ntiles = m->ntiles;
  d.toff = m->toff;
  d.hoff = m->hoff;
  d.hidx = m->hidx;
  d.hpad = m->hpad;
  d.tS = m->tS;
  d.tg0 = (const Real*)m->tg0;
  d.tg1 = (const Real*)m->tg1;
  d.tg2 = (const Real*)m->tg2;
  d.trec = (const int4*)m->trec;
  return d;
}

template <typename Real>
swe::DevState<Real> dev_state(const swe_state* s) {
  swe::DevState<Real> d{};
  for (int b = 0; b < 2; ++b) {
    d.h[b] = (Real*)s->h[b];
    d.hu[b] = (Real*)s->hu[b];
    d.hv[b] = (Real*)s->hv[b];
  }
  d.stride = s->stride;
  d.z = (const Real*)s->z;
  d.gn2 = (const Real*)s->gn2;
  d.hlo = (Real*)s->hlo;
  for (int k = 0; k < 5; ++k) d.fx[k] = (Real*)s->fx[k];
  d.partial = s->partial;
  d.ctl = s->ctl;
  return d;
}

// Largest dynamic shared memory a block may opt into on the current device
// (0 if the query fails).
int smem_optin_bytes();

// One forward step of the mesh's kernel on explicitly given state buffers;
// back: walk every chunk's tiles last to first (same results).
void launch_forward(const swe_mesh* m, const swe::DevState<float>& ds, cudaStream_t st,
                    bool back = false);
void launch_forward(const swe_mesh* m, const swe::DevState<double>& ds, cudaStream_t st,
                    bool back = false);
// Caller order (FP64) -> internal order in the mesh precision, and back;
// stride 4 for interleaved cells.
void gather_any(const swe_mesh* m, const double* src, void* dst, int stride);
void scatter_any(const swe_mesh* m, const void* src, double* dst, int stride);
// Makes every scenario's device end time +inf (steps take their CFL dt).
swe_status make_open_ended(swe_state* s);
// Copies every scenario's control word to the state's pinned mirror.
swe_status read_ctl(const swe_state* s);
// Other handles that use a mesh hold it: it is freed when the last goes.
void retain_mesh(swe_mesh* m);
void release_mesh(swe_mesh* m);

}  // namespace swe_host
