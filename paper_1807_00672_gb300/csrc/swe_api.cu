// C ABI of the shallow-water step library (declared in include/swe.h).
//
// A mesh handle holds one or more independent scenarios (an ensemble), each
// with its own triangles, state, time step and clock; a single mesh is an
// ensemble of one. Handles own one device arena each (mesh: geometry,
// connectivity and the tiled kernel's work chunks; state: two state buffers,
// friction coefficients, scratch and one control word per scenario). Steps
// are queued on the mesh's stream; repeated steps replay a captured CUDA
// graph of kStepsPerGraph launches. Kernels read each scenario's current
// buffer, dt and stop flag from its control word, so one graph serves any
// step count and end time (the host crosses to the device only at set-up and
// copy-out, Sec. 2.3).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <thread>
#include <vector>

#include "../../include/swe.h"
#include "mesh_build.h"
#include "swe_handles.cuh"
#include "swe_kernels.cuh"

namespace swe {

static_assert(kRecordSlotPad == kSlotPad, "the host record order models the kernels' face slots");

// Sets the end time of every scenario and re-clamps its next dt.
__global__ void k_set_end(Ctl* ctls, int n, double t_end) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    Ctl* ctl = ctls + i;
    ctl->t_end = t_end;
    if (ctl->err) { ctl->done = 1; continue; }
    const double rest = t_end - ctl->t;
    ctl->done = (ctl->t >= t_end) ? 1 : 0;
    if (ctl->dt_cfl >= rest) { ctl->dt = rest; ctl->clamped = 1; }
    else { ctl->dt = ctl->dt_cfl; ctl->clamped = 0; }
  }
}

// Caller-order Manning n (FP64, device) -> internal-order g n^2 in the mesh
// precision, formed in FP64 as the host path forms it: dst[j] = g (n n).
template <typename Real>
__global__ void k_gather_gn2(const double* __restrict__ n, const int32_t* __restrict__ perm,
                             Real* __restrict__ dst, int64_t cells, double g) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cells;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = perm[j];
    if (c >= 0) {
      const double nn = n[c];
      dst[j] = Real(__dmul_rn(g, __dmul_rn(nn, nn)));
    }
  }
}

// Caller-order fields (Host = double or float; any of f0, f1, f2 may be
// null) -> the state's cells: d_k[iperm[c] stride] = Real(f_k[c]) for the
// caller cells c in [0, n). The sources are read in caller order (coalesced,
// which suits page-locked host memory read across the host link) and
// converted by round to nearest (Real narrower than Host) or exactly.
template <typename Real, typename Host>
__global__ void k_put_fields(const Host* __restrict__ f0, const Host* __restrict__ f1,
                             const Host* __restrict__ f2, const int32_t* __restrict__ iperm,
                             int64_t n, Real* d0, Real* d1, Real* d2, int stride) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = (int64_t)iperm[c] * stride;
    if (f0) d0[j] = Real(f0[c]);
    if (f1) d1[j] = Real(f1[c]);
    if (f2) d2[j] = Real(f2[c]);
  }
}

// The reverse over caller cells [c0, c1): f_k[c] = Host(d_k[iperm[c] stride])
// (any f_k may be null), written in caller order. lo (FP32 states with a
// depth residual, else null): the depth is h + lo, summed in FP64 (exactly:
// |lo| is at most half an ulp of h) and rounded once to Host.
template <typename Real, typename Host>
__global__ void k_take_fields(const Real* s0, const Real* s1, const Real* s2, const Real* lo,
                              const int32_t* __restrict__ iperm, int64_t c0, int64_t c1, Host* f0,
                              Host* f1, Host* f2, int stride) {
  for (int64_t c = c0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < c1;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = iperm[c], j = i * stride;
    if (f0) f0[c] = lo ? Host((double)s0[j] + (double)lo[i]) : Host(s0[j]);
    if (f1) f1[c] = Host(s1[j]);
    if (f2) f2[c] = Host(s2[j]);
  }
}

}  // namespace swe

namespace swe_host {

thread_local std::string g_cuda_msg;

int smem_optin_bytes() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return v;
}

bool cuda_failed_at(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return false;
  const char* base = file;
  for (const char* c = file; *c; ++c)
    if (*c == '/') base = c + 1;
  g_cuda_msg = std::string(cudaGetErrorString(e)) + " in " + what + " (" + base + ":" +
               std::to_string(line) + ")";
  return true;
}

}  // namespace swe_host

using namespace swe_host;

namespace {

constexpr int kStepsPerGraph = 16;
// Default cells per tile: 512 for FP32 (fewer faces computed twice and less
// per-tile work than 256, one block of 256 threads), 256 for FP64 (whose
// tiles take twice the shared memory).
constexpr int kDefaultTileF32 = 512;
constexpr int kDefaultTileF64 = 256;
constexpr int64_t kEnsembleWaves = 3;  // waves of work chunks for several scenarios

#define cuda_failed(call) swe_host::cuda_failed_at((call), #call, __FILE__, __LINE__)

#define CK(call)                                  \
  do {                                            \
    if (cuda_failed(call)) return SWE_ECUDA;      \
  } while (0)

}  // namespace


namespace {

int grid_for(int64_t n, int threads, int cap) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// Opts the tiled kernel into its dynamic shared memory and returns its
// resident blocks per SM (0 if it cannot run with this layout).
template <typename Real, int NT, int NS, int TC, bool Early = false, bool CH = false,
          bool Pool = false>
int prepare_tiled(const swe::TileLayout& L) {
  constexpr bool comp = sizeof(Real) == 4;
  auto k = swe::k_tiled_step<Real, comp, NT, NS, TC, Early, CH, Pool>;
  // The limit is a property of the kernel, shared by every mesh that
  // launches it: set it to the device's largest opt-in size (not this
  // layout's), so that a later mesh with a smaller layout cannot lower it
  // below what an earlier one needs.
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int cap = swe_host::smem_optin_bytes() - (int)fa.sharedSizeBytes;  // less its static part
  if (cap <= 0 || (int)L.total > cap ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, L.total) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Opts the pipelined FP32 kernel (halo_schedule 2) into its dynamic shared
// memory; resident blocks per SM.
template <int NT, int TC>
int prepare_pipe(const swe::TileLayout& L) {
  auto k = swe::k_tiled_step_pipe<NT, TC>;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int cap = swe_host::smem_optin_bytes() - (int)fa.sharedSizeBytes;
  if (cap <= 0 || (int)L.total > cap ||
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, NT, L.total) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

template <typename Real, int NT, int CPT>
int blocks_per_sm_tiled_nt(const swe_mesh* m) {
  constexpr int TC = NT * CPT;
  // the Early kernel (halo_schedule 1) and the pipelined one (2) exist for
  // FP32 with 2 stages only
  if constexpr (sizeof(Real) == 4) {
    if (m->layout.pipe) return prepare_pipe<NT, TC>(m->layout);
    if (m->layout.early) return prepare_tiled<Real, NT, 2, TC, true>(m->layout);
    if (m->prm.compensated_depth) {
      prepare_tiled<Real, NT, 2, TC, false, true, true>(m->layout);  // its pooled variant
      return prepare_tiled<Real, NT, 2, TC, false, true>(m->layout);
    }
    // the pooled variant (FP32, halo schedule 0) shares the layout
    if (m->stages == 2) prepare_tiled<Real, NT, 2, TC, false, false, true>(m->layout);
    else prepare_tiled<Real, NT, 3, TC, false, false, true>(m->layout);
  }
  return m->stages == 3 ? prepare_tiled<Real, NT, 3, TC>(m->layout)
                        : prepare_tiled<Real, NT, 2, TC>(m->layout);
}

template <typename Real, int CPT>
int blocks_per_sm_tiled_cpt(const swe_mesh* m) {
  if constexpr (sizeof(Real) == 4 && CPT == 1) {
    if (m->tile == 512) return m->layout.pipe ? prepare_pipe<512, 512>(m->layout) : 0;
  }
  switch (m->tile / CPT) {
    case 32: return blocks_per_sm_tiled_nt<Real, 32, CPT>(m);
    case 64: return blocks_per_sm_tiled_nt<Real, 64, CPT>(m);
    case 128: return blocks_per_sm_tiled_nt<Real, 128, CPT>(m);
    default: return blocks_per_sm_tiled_nt<Real, 256, CPT>(m);
  }
}

template <typename Real>
int blocks_per_sm_tiled(const swe_mesh* m) {
  return m->cpt == 2 ? blocks_per_sm_tiled_cpt<Real, 2>(m) : blocks_per_sm_tiled_cpt<Real, 1>(m);
}

template <typename Real, bool Comp, int NT, int CPT>
void launch_tiled_nt(const swe_mesh* m, const swe::DevMesh<Real>& dm, const swe::DevState<Real>& ds,
                     const swe::Num& num, cudaStream_t st) {
  const swe::TileLayout& L = m->layout;
  const int g = (int)m->nchunks;
  constexpr int TC = NT * CPT;
  // Programmatic dependent launch: a step's blocks fetch their first tiles'
  // mesh data while the previous step's last blocks finish, and wait for it
  // (griddepcontrol.wait) before reading the state.
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)g);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = L.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if constexpr (sizeof(Real) == 4) {
    if (L.pipe) {
      cudaLaunchKernelEx(&cfg, swe::k_tiled_step_pipe<NT, TC>, dm, ds, num, L);
      return;
    }
  }
  if constexpr (NT <= 256) {  // 512 threads exist only for the pipelined kernel
    if constexpr (sizeof(Real) == 4) {
      if (ds.hlo) {  // compensated depth (2 stages, halo schedule 0)
        if (m->pooled)
          cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 2, TC, false, true, true>, dm, ds, num, L);
        else
          cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 2, TC, false, true>, dm, ds, num, L);
        return;
      }
      if (m->pooled && !L.early) {  // chunk tables with tile pools
        if (m->stages == 3)
          cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 3, TC, false, false, true>, dm, ds, num, L);
        else
          cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 2, TC, false, false, true>, dm, ds, num, L);
        return;
      }
      if (L.early) {
        cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 2, TC, true>, dm, ds, num, L);
        return;
      }
    }
    if (m->stages == 3)
      cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 3, TC>, dm, ds, num, L);
    else
      cudaLaunchKernelEx(&cfg, swe::k_tiled_step<Real, Comp, NT, 2, TC>, dm, ds, num, L);
  }
}

template <typename Real, bool Comp, int CPT>
void launch_tiled_cpt(const swe_mesh* m, const swe::DevMesh<Real>& dm, const swe::DevState<Real>& ds,
                      const swe::Num& num, cudaStream_t st) {
  if constexpr (sizeof(Real) == 4 && CPT == 1) {
    if (m->tile == 512) {  // 512 threads: the pipelined kernel only
      launch_tiled_nt<Real, Comp, 512, 1>(m, dm, ds, num, st);
      return;
    }
  }
  switch (m->tile / CPT) {
    case 32: launch_tiled_nt<Real, Comp, 32, CPT>(m, dm, ds, num, st); break;
    case 64: launch_tiled_nt<Real, Comp, 64, CPT>(m, dm, ds, num, st); break;
    case 128: launch_tiled_nt<Real, Comp, 128, CPT>(m, dm, ds, num, st); break;
    default: launch_tiled_nt<Real, Comp, 256, CPT>(m, dm, ds, num, st); break;
  }
}

template <typename Real>
void set_edge_grids(swe_mesh* m) {
  int occ_cell = 0, occ_edge = 0, occ_cfl = 0;
  constexpr bool comp = sizeof(Real) == 4;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cell, swe::k_cell_update<Real, comp>, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_edge, swe::k_edge_flux<Real>, 256, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_cfl, swe::k_cfl<Real>, 256, 0);
  occ_cell = occ_cell > 0 ? occ_cell : 1;
  occ_edge = occ_edge > 0 ? occ_edge : 1;
  occ_cfl = occ_cfl > 0 ? occ_cfl : 1;
  m->grid_edge = grid_for(m->E, 256, m->sms * occ_edge * 4);
  m->grid_cell = grid_for(m->T, 256, m->sms * occ_cell);
  m->grid_cfl = grid_for(m->T, 256, m->sms * occ_cfl);
}

void launch_one_step(swe_state* s, cudaStream_t st) {
  if (s->mesh->prm.precision == SWE_F64) launch_forward(s->mesh, dev_state<double>(s), st, s->walk_back);
  else launch_forward(s->mesh, dev_state<float>(s), st, s->walk_back);
  s->walk_back = !s->walk_back;
}

// CFL step (kind swe::kCflOnly) or mass only (swe::kMassOnly, tiled
// meshes) of the current state.
template <typename Real>
void launch_cfl(const swe_state* s, int kind = swe::kCflOnly) {
  const swe_mesh* m = s->mesh;
  if (m->kernel == SWE_KERNEL_EDGE)
    swe::k_cfl<Real><<<m->grid_cfl, 256, 0, m->stream>>>(dev_mesh<Real>(m), dev_state<Real>(s), num_of(m));
  else
    swe::k_cfl_tiled<Real><<<(int)m->nchunks, 256, 0, m->stream>>>(dev_mesh<Real>(m), dev_state<Real>(s),
                                                                  num_of(m), m->tile, kind);
}

template <typename Real>
void launch_gather(const swe_mesh* m, const double* src, void* dst, int stride) {
  swe::k_gather<Real><<<grid_for(m->Tp, 256, m->sms * 16), 256, 0, m->stream>>>(src, m->perm, (Real*)dst,
                                                                               m->Tp, stride);
}

template <typename Real>
void launch_scatter(const swe_mesh* m, const void* src, double* dst, int stride) {
  swe::k_scatter<Real><<<grid_for(m->Tp, 256, m->sms * 16), 256, 0, m->stream>>>((const Real*)src, m->perm,
                                                                                dst, m->Tp, stride);
}

size_t real_size(const swe_mesh* m) { return m->prm.precision == SWE_F64 ? 8 : 4; }

// Host FP64 vector -> device array of the mesh precision. Synchronous: the
// host vector may go out of scope on return.
swe_status upload_real(const swe_mesh* m, const std::vector<double>& v, void* dst) {
  if (v.empty()) return SWE_OK;
  if (m->prm.precision == SWE_F64) {
    CK(cudaMemcpyAsync(dst, v.data(), v.size() * 8, cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
  } else {
    std::vector<float> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = (float)v[i];
    CK(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, m->stream));
    CK(cudaStreamSynchronize(m->stream));
  }
  return SWE_OK;
}

template <typename T>
swe_status upload(const swe_mesh* m, const std::vector<T>& v, void* dst) {
  if (v.empty()) return SWE_OK;
  CK(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, m->stream));
  CK(cudaStreamSynchronize(m->stream));
  return SWE_OK;
}

swe_status status_from_err(int err) {
  if (err & swe::kErrTimeout) return SWE_ETIMEOUT;
  if (err & swe::kErrNan) return SWE_ENAN;
  if (err & swe::kErrDry) return SWE_EDRY;
  return SWE_OK;
}

// Status over every scenario (the most severe error any of them raised).
swe_status status_all(const swe_state* s) {
  int err = 0;
  for (int i = 0; i < nscen(s->mesh); ++i) err |= s->host_ctl[i].err;
  return status_from_err(err);
}

bool all_done(const swe_state* s) {
  for (int i = 0; i < nscen(s->mesh); ++i)
    if (!s->host_ctl[i].done) return false;
  return true;
}


swe_status ensure_graph(swe_state* s) {
  if (s->graph) return SWE_OK;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(s->capture, cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < kStepsPerGraph; ++k) launch_one_step(s, s->capture);
  cudaError_t e = cudaStreamEndCapture(s->capture, &g);
  if (cuda_failed(e)) return SWE_ECUDA;
  e = cudaGraphInstantiate(&s->graph, g, 0);
  cudaGraphDestroy(g);
  if (cuda_failed(e)) { s->graph = nullptr; return SWE_ECUDA; }
  // upload now, so that the first replay costs what every later one does
  CK(cudaGraphUpload(s->graph, s->mesh->stream));
  return SWE_OK;
}

// Queues n steps: whole graphs, then single launches for the remainder.
swe_status queue_steps(swe_state* s, int64_t n) {
  cudaStream_t st = s->mesh->stream;
  if (n >= kStepsPerGraph) {
    swe_status r = ensure_graph(s);
    if (r != SWE_OK) return r;
    for (int64_t k = 0; k < n / kStepsPerGraph; ++k) CK(cudaGraphLaunch(s->graph, st));
    n %= kStepsPerGraph;
  }
  for (int64_t k = 0; k < n; ++k) launch_one_step(s, st);
  CK(cudaGetLastError());
  return SWE_OK;
}

void set_end(swe_state* s, double t_end) {
  const int n = nscen(s->mesh);
  swe::k_set_end<<<(n + 127) / 128, 128, 0, s->mesh->stream>>>(s->ctl, n, t_end);
}

// Makes every device end time +inf (no clamp) unless it already is.
void open_end(swe_state* s) {
  if (s->open_ended) return;
  set_end(s, std::numeric_limits<double>::infinity());
  s->open_ended = true;
}

// Device address of a caller host array that kernels may read and write
// directly: page-locked host memory (cudaHostAlloc, cudaHostRegister) is
// mapped into the device's address space. Null for any other memory.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

template <typename Host>
void launch_put(const swe_mesh* m, const Host* const f[3], void* const d[3], int stride) {
  if (!f[0] && !f[1] && !f[2]) return;
  const int grid = grid_for(m->T, 256, m->sms * 16);
  if (m->prm.precision == SWE_F64)
    swe::k_put_fields<double, Host><<<grid, 256, 0, m->stream>>>(
        f[0], f[1], f[2], m->iperm, m->T, (double*)d[0], (double*)d[1], (double*)d[2], stride);
  else
    swe::k_put_fields<float, Host><<<grid, 256, 0, m->stream>>>(
        f[0], f[1], f[2], m->iperm, m->T, (float*)d[0], (float*)d[1], (float*)d[2], stride);
}

// Caller-order arrays (any may be null) -> the state's arrays dst[k] (cells
// `stride` apart). Device arrays (on_device) and page-locked host arrays are
// read by one kernel across the host link; other host arrays go through the
// staging buffer (T doubles), one at a time.
template <typename Host>
swe_status put_fields(const swe_state* s, const Host* const src[3], void* const dst[3], int stride,
                      bool on_device) {
  const swe_mesh* m = s->mesh;
  const Host* direct[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < 3; ++k)
    if (src[k]) direct[k] = on_device ? src[k] : (const Host*)mapped_host(src[k]);
  launch_put<Host>(m, direct, dst, stride);
  for (int k = 0; k < 3; ++k) {
    if (!src[k] || direct[k]) continue;
    CK(cudaMemcpyAsync(s->stage, src[k], m->T * sizeof(Host), cudaMemcpyHostToDevice, m->stream));
    const Host* one[3] = {nullptr, nullptr, nullptr};
    one[k] = (const Host*)s->stage;
    launch_put<Host>(m, one, dst, stride);
  }
  CK(cudaGetLastError());
  return SWE_OK;
}

// (h, hu, hv) in caller order -> buffer 0.
template <typename Host>
swe_status upload_state_fields(swe_state* s, const Host* h, const Host* hu, const Host* hv,
                               bool on_device = false) {
  const Host* src[3] = {h, hu, hv};
  void* dst[3] = {s->h[0], s->hu[0], s->hv[0]};
  if (s->hlo) CK(cudaMemsetAsync(s->hlo, 0, 4 * (size_t)s->mesh->Tp, s->mesh->stream));
  return put_fields<Host>(s, src, dst, s->stride, on_device);
}

// Orders the mesh stream after the work queued so far on the caller's
// stream (the device-pointer calls: the caller wrote its buffers there).
swe_status wait_for_caller(const swe_mesh* m, void* caller_stream) {
  cudaStream_t cs = (cudaStream_t)caller_stream;
  if (!cs || cs == m->stream) return SWE_OK;
  cudaEvent_t ev = nullptr;
  CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(ev, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(m->stream, ev, 0);
  cudaEventDestroy(ev);  // released once the recorded work completes
  if (cuda_failed(e)) return SWE_ECUDA;
  return SWE_OK;
}

// Resets every scenario's control word to t = 0 in buffer 0 and computes
// its dt and mass.
swe_status reset_and_cfl(swe_state* s) {
  const swe_mesh* m = s->mesh;
  for (int i = 0; i < nscen(m); ++i) {
    swe::Ctl c{};
    c.t = 0.0;
    c.t_end = std::numeric_limits<double>::infinity();
    c.part0 = m->scen[i].chunk0;
    c.nparts = m->scen[i].nchunks;
    c.subdomain = m->ghosts ? 1 : 0;
    s->host_ctl[i] = c;
  }
  s->open_ended = true;
  CK(cudaMemcpyAsync(s->ctl, s->host_ctl, sizeof(swe::Ctl) * nscen(m), cudaMemcpyHostToDevice,
                     m->stream));
  if (m->prm.precision == SWE_F64) launch_cfl<double>(s);
  else launch_cfl<float>(s);
  CK(cudaGetLastError());
  swe_status r = read_ctl(s);
  if (r != SWE_OK) return r;
  return status_all(s);
}

swe_status resolve_params(const swe_params* params, swe_params& p) {
  swe_params_default(&p);
  if (params) p = *params;
  if (p.precision != SWE_F64 && p.precision != SWE_F32) return SWE_EINVAL;
  if (p.order < SWE_ORDER_NONE || p.order > SWE_ORDER_RCM) return SWE_EINVAL;
  if (p.kernel < SWE_KERNEL_AUTO || p.kernel > SWE_KERNEL_TILED) return SWE_EINVAL;
  if (p.cells_per_thread == 0) p.cells_per_thread = 2;
  if (p.tile == 0)
    p.tile = (p.precision == SWE_F32 && p.cells_per_thread == 2) ? kDefaultTileF32 : kDefaultTileF64;
  if (p.cells_per_thread != 1 && p.cells_per_thread != 2) return SWE_EINVAL;
  const int nt = p.tile / p.cells_per_thread;
  if (p.stages == 0) p.stages = 2;
  // 512 threads per block: only the pipelined FP32 kernel, one cell per thread
  const bool nt512 = nt == 512 && p.halo_schedule == 2 && p.precision == SWE_F32 &&
                     p.cells_per_thread == 1 && p.stages == 2;
  if (p.tile % p.cells_per_thread != 0 || (nt != 32 && nt != 64 && nt != 128 && nt != 256 && !nt512))
    return SWE_EINVAL;
  if (p.stages != 2 && p.stages != 3) return SWE_EINVAL;
  if (p.halo_schedule < 0 || p.halo_schedule > 2) return SWE_EINVAL;
  if (p.wait_rounds < -1) return SWE_EINVAL;
  if (p.compensated_depth != 0 && p.compensated_depth != 1) return SWE_EINVAL;
  if (p.compensated_depth &&
      (p.precision != SWE_F32 || p.kernel == SWE_KERNEL_EDGE || p.stages != 2 || p.halo_schedule != 0))
    return SWE_EINVAL;
  if (!(p.g > 0.0) || !(p.courant > 0.0) || !(p.h_eps >= 0.0)) return SWE_EINVAL;
  if (p.kernel == SWE_KERNEL_AUTO) p.kernel = SWE_KERNEL_TILED;
  return SWE_OK;
}

// Builds a mesh of n scenarios (swe_mesh_create_batch).
swe_status create_batch(int32_t n, const double* const* xy, const int64_t* n_nodes,
                        const int32_t* const* tri, const int64_t* n_tris, const swe_params* params,
                        void* cuda_stream, swe_mesh** out, const uint8_t* ghost = nullptr) {
  if (!out) return SWE_EINVAL;
  *out = nullptr;
  if (n <= 0 || !xy || !n_nodes || !tri || !n_tris) return SWE_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (n_tris[i] == 0) return SWE_EMESH;
    if (!xy[i] || !tri[i] || n_nodes[i] <= 0 || n_tris[i] < 0) return SWE_EINVAL;
  }
  swe_params p;
  swe_status st = resolve_params(params, p);
  if (st != SWE_OK) return st;
  // AUTO: the tiled kernel, except for one reverse Cuthill-McKee-ordered
  // mesh, whose tiles are thin strips of its breadth-first levels (2.7 face
  // records and 2 halo cells per cell at 512-cell tiles): the edge kernel
  // runs it faster (34 against 29 G cell-updates/s at 10M triangles, FP32).
  const bool autok = (params ? params->kernel : SWE_KERNEL_AUTO) == SWE_KERNEL_AUTO;
  if (autok && n == 1 && p.order == SWE_ORDER_RCM && !p.compensated_depth) p.kernel = SWE_KERNEL_EDGE;
  const int kernel = p.kernel;
  if (kernel == SWE_KERNEL_EDGE && n > 1) return SWE_EINVAL;
  const int tile = p.tile;

  // Host-side construction and validation first (scenarios on parallel host
  // threads): no device is touched for an invalid mesh.
  std::vector<swe::HostMesh> hm(n);
  std::vector<int> rc(n, 0);
  {
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const int nthr = (int)std::min<unsigned>((unsigned)n, std::min(16u, hw));
    std::atomic<int> next{0};
    auto work = [&]() {
      for (int i = next++; i < n; i = next++)
        rc[i] = swe::build_host_mesh(xy[i], n_nodes[i], tri[i], n_tris[i], p.order,
                                     kernel == SWE_KERNEL_TILED ? tile : 0,
                                     kernel == SWE_KERNEL_EDGE, hm[i],
                                     kernel == SWE_KERNEL_TILED && p.precision == SWE_F32);
    };
    std::vector<std::thread> pool;
    try {  // the calling thread takes every scenario no worker takes
      for (int k = 1; k < nthr; ++k) pool.emplace_back(work);
    } catch (...) {
    }
    work();
    for (auto& t : pool) t.join();
  }
  for (int i = 0; i < n; ++i) {
    if (rc[i] == -2) return SWE_EMESH;
    if (rc[i] != 0) return SWE_EINVAL;
  }

  int dev = 0;
  CK(cudaGetDevice(&dev));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));

  swe_mesh* m = new swe_mesh();
  m->prm = p;
  m->device = dev;
  m->sms = sms;
  m->kernel = kernel;
  m->tile = tile;
  m->stages = p.stages;
  m->cpt = p.cells_per_thread;
  m->scen.resize(n);
  int64_t caller = 0, cells = 0, tiles = 0, recs = 0, halos = 0, rec_cap = 0, halo_cap = 0;
  for (int i = 0; i < n; ++i) {
    Scenario& sc = m->scen[i];
    sc.caller0 = caller;
    sc.ncells = hm[i].T;
    sc.cell0 = cells;
    sc.tile0 = tiles;
    sc.ntiles = hm[i].ntiles;
    caller += hm[i].T;
    cells += (kernel == SWE_KERNEL_TILED) ? hm[i].ntiles * tile : hm[i].T;
    tiles += hm[i].ntiles;
    recs += (int64_t)hm[i].tA.size();
    halos += (int64_t)hm[i].hidx.size();
    rec_cap = std::max(rec_cap, hm[i].rec_cap);
    halo_cap = std::max(halo_cap, hm[i].halo_cap);
    m->V += hm[i].V;
    m->E += hm[i].E;
    m->Eb += hm[i].Eb;
  }
  m->T = caller;
  m->Tp = cells;
  m->ntiles = tiles;
  m->records = recs;
  m->halos = halos;
  if (m->Tp >= INT32_MAX || recs >= INT32_MAX) {
    delete m;
    return SWE_EINVAL;
  }
  if (cuda_stream) {
    m->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cuda_failed(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking))) {
      delete m;
      return SWE_ECUDA;
    }
    m->own_stream = true;
  }
  const size_t w = real_size(m);
  const int geo_arrays = (p.precision == SWE_F64) ? 3 : 2;

  // Work chunks of the tiled kernels (see swe::Chunk). One scenario: one
  // wave of resident blocks with ceil(ntiles / resident) tiles each. Several
  // scenarios: about kEnsembleWaves waves; scenario s is split into
  // ceil(ntiles_s / per) interleaved chunks, and the chunks are launched
  // largest first so that the block scheduler, which starts blocks in index
  // order as slots free up, balances the SMs (longest-processing-time order).
  std::vector<swe::Chunk> chunks;
  if (kernel == SWE_KERNEL_TILED) {
    const bool want_pipe = p.halo_schedule == 2 && p.precision == SWE_F32 && m->stages == 2;
    m->layout = swe::make_tile_layout((uint32_t)w, (uint32_t)geo_arrays, (uint32_t)tile,
                                      (uint32_t)m->stages, (uint32_t)rec_cap, (uint32_t)halo_cap,
                                      (uint32_t)(tile / m->cpt), want_pipe ? 2u : 1u);
    if (want_pipe && !m->layout.hreg)  // the pipelined kernel needs halo indices in registers
      m->layout = swe::make_tile_layout((uint32_t)w, (uint32_t)geo_arrays, (uint32_t)tile,
                                        (uint32_t)m->stages, (uint32_t)rec_cap, (uint32_t)halo_cap,
                                        (uint32_t)(tile / m->cpt));
    m->layout.pipe = (want_pipe && m->layout.hreg) ? 1u : 0u;
    m->layout.early =
        (m->layout.hreg && p.halo_schedule == 1 && p.precision == SWE_F32 && m->stages == 2) ? 1u : 0u;
    const int occ = (p.precision == SWE_F64) ? blocks_per_sm_tiled<double>(m)
                                             : blocks_per_sm_tiled<float>(m);
    if (occ < 1) {
      g_cuda_msg = "tiled kernel layout does not fit in shared memory";
      swe_mesh_destroy(m);
      return SWE_ECUDA;
    }
    const int64_t resident = (int64_t)sms * occ;
    const int64_t waves = (n == 1) ? 1 : kEnsembleWaves;
    const int64_t per = std::max<int64_t>(1, (tiles + resident * waves - 1) / (resident * waves));
    for (int i = 0; i < n; ++i) {
      Scenario& sc = m->scen[i];
      sc.chunk0 = (int64_t)chunks.size();
      sc.nchunks = (sc.ntiles + per - 1) / per;
      for (int64_t r = 0; r < sc.nchunks; ++r) {
        swe::Chunk c{};
        c.scen = i;
        c.tile0 = (int32_t)(sc.tile0 + r);
        c.ntiles = (int32_t)((sc.ntiles - r + sc.nchunks - 1) / sc.nchunks);
        c.stride = (int32_t)sc.nchunks;
        c.part = (int32_t)(sc.chunk0 + r);
        c.cell_end = (int32_t)(sc.cell0 + sc.ncells);
        chunks.push_back(c);
      }
    }
    if (n > 1)
      std::stable_sort(chunks.begin(), chunks.end(),
                       [](const swe::Chunk& a, const swe::Chunk& b) { return a.ntiles > b.ntiles; });
    m->nchunks = (int64_t)chunks.size();
  } else {
    if (p.precision == SWE_F64) set_edge_grids<double>(m);
    else set_edge_grids<float>(m);
  }
  m->max_grid = (int)std::max<int64_t>(std::max(m->grid_cell, m->grid_cfl), m->nchunks);

  // Device layout.
  const int64_t T = m->T, Tp = m->Tp, E = m->E, R = recs, H = halos;
  const int64_t C = m->nchunks;
  Layout L;
  L.add(4 * Tp);  // perm
  L.add(w * Tp);  // area
  L.add(w * Tp);  // irP
  const bool with_rarea = kernel == SWE_KERNEL_TILED && p.precision == SWE_F64;
  if (with_rarea) L.add(w * Tp);  // 1 / area
  L.add(4 * T);                   // caller cell -> internal cell
  if (kernel == SWE_KERNEL_EDGE) {
    L.add(4 * E); L.add(4 * E);
    L.add(w * E); L.add(w * E); L.add(w * E);
    L.add(4 * T); L.add(4 * T); L.add(4 * T);
  } else {
    L.add(8 * (tiles + 1)); L.add(8 * (tiles + 1));
    if (geo_arrays > 2) {
      L.add(4 * R);                                   // FP64: side codes
      for (int g = 0; g < geo_arrays; ++g) L.add(w * R);  // and geometry arrays
    } else {
      L.add(16 * R);  // FP32: interleaved records
    }
    L.add(4 * H);
    L.add(sizeof(swe::Chunk) * C);
    L.add(sizeof(swe::Chunk) * C);  // the same chunks walked backwards
    L.add(sizeof(swe::Chunk) * C);  // the step's chunks with tile pools, forwards
    L.add(sizeof(swe::Chunk) * C);  // and backwards
    if (m->layout.hreg) L.add(4 * tiles * (int64_t)m->layout.halo_cap);
  }
  if (cudaMalloc((void**)&m->arena.base, L.total) != cudaSuccess) {
    cudaGetLastError();
    swe_mesh_destroy(m);
    return SWE_ENOMEM;
  }
  m->arena.size = L.total;
  st = SWE_OK;
  auto chk = [&](swe_status r) { if (st == SWE_OK) st = r; };
  if (cuda_failed(cudaMemsetAsync(m->arena.base, 0, L.total, m->stream))) chk(SWE_ECUDA);
  m->perm = (int32_t*)m->arena.take(4 * Tp);
  m->area = m->arena.take(w * Tp);
  m->irP = m->arena.take(w * Tp);
  if (with_rarea) m->rarea = m->arena.take(w * Tp);
  m->iperm = (int32_t*)m->arena.take(4 * T);
  if (kernel == SWE_KERNEL_EDGE) {
    m->eL = (int32_t*)m->arena.take(4 * E);
    m->eR = (int32_t*)m->arena.take(4 * E);
    m->nx = m->arena.take(w * E);
    m->ny = m->arena.take(w * E);
    m->len = m->arena.take(w * E);
    for (int k = 0; k < 3; ++k) m->cf[k] = (int32_t*)m->arena.take(4 * T);
  } else {
    m->toff = (int64_t*)m->arena.take(8 * (tiles + 1));
    m->hoff = (int64_t*)m->arena.take(8 * (tiles + 1));
    if (geo_arrays > 2) {  // FP64: side codes and geometry in separate arrays
      m->tS = (int32_t*)m->arena.take(4 * R);
      m->tg0 = m->arena.take(w * R);
      m->tg1 = m->arena.take(w * R);
      m->tg2 = m->arena.take(w * R);
    } else {  // FP32: interleaved 16-byte records
      m->trec = m->arena.take(16 * R);
    }
    m->hidx = (int32_t*)m->arena.take(4 * H);
    m->chunks = (swe::Chunk*)m->arena.take(sizeof(swe::Chunk) * C);
    m->chunks_back = (swe::Chunk*)m->arena.take(sizeof(swe::Chunk) * C);
    m->chunks_pool = (swe::Chunk*)m->arena.take(sizeof(swe::Chunk) * C);
    m->chunks_pool_back = (swe::Chunk*)m->arena.take(sizeof(swe::Chunk) * C);
    if (m->layout.hreg)
      m->hpad = (int32_t*)m->arena.take(4 * tiles * (int64_t)m->layout.halo_cap);
  }
  if (m->arena.overflow) {
    g_cuda_msg = "mesh arena layout";
    chk(SWE_ECUDA);
  }

  // Concatenated host arrays, uploaded one at a time.
  if (st == SWE_OK) {
    std::vector<int32_t> perm(Tp, -1);
    std::vector<double> area(Tp, 0.0), irp(Tp, 0.0), rarea;
    for (int i = 0; i < n; ++i) {
      const Scenario& sc = m->scen[i];
      for (int64_t j = 0; j < sc.ncells; ++j) {
        perm[sc.cell0 + j] = (int32_t)(sc.caller0 + hm[i].perm[j]);
        area[sc.cell0 + j] = hm[i].area[j];
        irp[sc.cell0 + j] = hm[i].perim[j] / hm[i].area[j];
        // a ghost cell (a copy of another sub-domain's cell) is marked by
        // perimeter / area = 0: it adds nothing to the CFL rate or the mass
        if (ghost && ghost[sc.caller0 + hm[i].perm[j]]) irp[sc.cell0 + j] = 0.0;
      }
    }
    chk(upload(m, perm, m->perm));
    {
      std::vector<int32_t> iperm(T, -1);
      for (int64_t j = 0; j < Tp; ++j)
        if (perm[j] >= 0) iperm[perm[j]] = (int32_t)j;
      chk(upload(m, iperm, m->iperm));
    }
    chk(upload_real(m, area, m->area));
    chk(upload_real(m, irp, m->irP));
    if (with_rarea) {
      rarea.assign(Tp, 0.0);  // padding cells: 0 (never updated)
      for (int64_t j = 0; j < Tp; ++j)
        if (area[j] > 0.0) rarea[j] = 1.0 / area[j];
      chk(upload_real(m, rarea, m->rarea));
    }
  }
  if (st == SWE_OK && kernel == SWE_KERNEL_EDGE) {
    const swe::HostMesh& h0 = hm[0];
    chk(upload(m, h0.eL, m->eL));
    chk(upload(m, h0.eR, m->eR));
    chk(upload_real(m, h0.nx, m->nx));
    chk(upload_real(m, h0.ny, m->ny));
    chk(upload_real(m, h0.len, m->len));
    for (int k = 0; k < 3; ++k) chk(upload(m, h0.cface[k], m->cf[k]));
  } else if (st == SWE_OK) {
    std::vector<int64_t> toff(tiles + 1, 0), hoff(tiles + 1, 0);
    std::vector<int32_t> packed(R), hidx(H);
    std::vector<double> g0(R), g1(R), g2(R);
    auto code = [](int32_t v) { return v == swe::kWall ? (int32_t)swe::kSideWall : v; };
    bool fits = true;
    int64_t r_at = 0, h_at = 0;
    for (int i = 0; i < n; ++i) {
      const swe::HostMesh& hmi = hm[i];
      const Scenario& sc = m->scen[i];
      for (int64_t t = 0; t < hmi.ntiles; ++t) {
        toff[sc.tile0 + t] = r_at + hmi.toff[t];
        hoff[sc.tile0 + t] = h_at + hmi.hoff[t];
      }
      // Sides as int16 codes packed in one word (A high, B low). Local and
      // halo codes are relative to the tile, so they need no offset.
      for (size_t r = 0; r < hmi.tA.size(); ++r) {
        const int32_t a = code(hmi.tA[r]), b = code(hmi.tB[r]);
        fits = fits && a >= -32768 && a <= 32767 && b >= -32768 && b <= 32767;
        packed[r_at + r] = (int32_t)(((uint32_t)(uint16_t)a << 16) | (uint32_t)(uint16_t)b);
        g0[r_at + r] = hmi.tnx[r];
        g1[r_at + r] = hmi.tny[r];
        g2[r_at + r] = hmi.tlen[r];
      }
      for (size_t q = 0; q < hmi.hidx.size(); ++q) hidx[h_at + q] = (int32_t)(sc.cell0 + hmi.hidx[q]);
      r_at += (int64_t)hmi.tA.size();
      h_at += (int64_t)hmi.hidx.size();
    }
    toff[tiles] = r_at;
    hoff[tiles] = h_at;
    if (!fits) chk(SWE_EINVAL);
    chk(upload(m, toff, m->toff));
    chk(upload(m, hoff, m->hoff));
    if (geo_arrays > 2) {
      chk(upload(m, packed, m->tS));
      chk(upload_real(m, g0, m->tg0));
      chk(upload_real(m, g1, m->tg1));
      chk(upload_real(m, g2, m->tg2));
    } else {
      // FP32 record r: {packed sides, nx, ny, l} as one 16-byte word (the
      // geometry rounded once from FP64)
      std::vector<int32_t> rec(4 * R);
      for (int64_t r = 0; r < R; ++r) {
        const float f[3] = {(float)g0[r], (float)g1[r], (float)g2[r]};
        rec[4 * r] = packed[r];
        std::memcpy(&rec[4 * r + 1], f, sizeof f);
      }
      chk(upload(m, rec, m->trec));
    }
    chk(upload(m, hidx, m->hidx));
    chk(upload(m, chunks, m->chunks));
    // Every chunk's tiles in the opposite order (last tile first, negative
    // stride). Steps alternate between the two walks, so that a step starts
    // on the tiles the previous one finished with, whose records and cells
    // are still in L2. The order of the tiles does not change any result.
    std::vector<swe::Chunk> back(chunks);
    for (swe::Chunk& c : back) {
      c.tile0 += (c.ntiles - 1) * c.stride;
      c.stride = -c.stride;
    }
    chk(upload(m, back, m->chunks_back));
    // The step's tables: the blocks of one SM progress at different speeds
    // (the warp scheduler favours the oldest; on the 10M mesh the three
    // blocks of an SM end their equal shares about 109, 114 and 127 us into
    // a step), so a chunk keeps the tiles of all but the last kPoolWaves
    // waves of its scenario's walk and those last waves form the scenario's
    // pool, from which the faster blocks take more tiles. Each pool entry
    // costs an atomic on one address; measured best at 3 waves (a pool of
    // every tile was 1.6 % slower than none). Only for a single FP32
    // scenario with at least 5 kPoolWaves tiles per chunk: where the pool
    // would be a larger share of the tiles (the 1M-cell meshes, ensembles)
    // and on the FP64 step it measured 0.5-5 % slower.
    constexpr int64_t kPoolWaves = 3;
    const bool use_pool = n == 1 && p.precision == SWE_F32 && !m->layout.early;
    std::vector<swe::Chunk> pooled(chunks), pooled_back(back);
    for (size_t q = 0; q < chunks.size() && use_pool; ++q) {
      const Scenario& sc = m->scen[chunks[q].scen];
      const int64_t S = sc.nchunks, N = sc.ntiles, ns = m->stages;
      const int64_t W = std::max<int64_t>(ns, N / S - kPoolWaves);  // static tiles per chunk
      if (N < 5 * kPoolWaves * S || W * S >= N) continue;
      const int64_t r = chunks[q].tile0 - sc.tile0;
      swe::Chunk& f = pooled[q];
      f.ntiles = (int32_t)W;
      f.pool_first = (int32_t)(sc.tile0 + W * S);
      f.pool_count = (int32_t)(N - W * S);
      swe::Chunk& b = pooled_back[q];
      b.tile0 = (int32_t)(sc.tile0 + N - 1 - r);
      b.ntiles = (int32_t)W;
      b.stride = -(int32_t)S;
      b.pool_first = (int32_t)(sc.tile0 + N - 1 - W * S);
      b.pool_count = (int32_t)(N - W * S);
    }
    for (const swe::Chunk& c : pooled) m->pooled = m->pooled || c.pool_count > 0;
    chk(upload(m, pooled, m->chunks_pool));
    chk(upload(m, pooled_back, m->chunks_pool_back));
    if (m->layout.hreg) {
      // tile t's halo list at t * halo_cap, padded with the tile's first cell
      const int64_t hc = m->layout.halo_cap;
      std::vector<int32_t> hpad(tiles * hc);
      for (int i = 0; i < n; ++i) {
        const Scenario& sc = m->scen[i];
        for (int64_t t = 0; t < sc.ntiles; ++t) {
          const int64_t tg = sc.tile0 + t;
          const int64_t q0 = hoff[tg], nq = hoff[tg + 1] - q0;
          for (int64_t q = 0; q < hc; ++q)
            hpad[tg * hc + q] = q < nq ? hidx[q0 + q] : (int32_t)(sc.cell0 + t * tile);
        }
      }
      chk(upload(m, hpad, m->hpad));
    }
  }
  if (st != SWE_OK) {
    swe_mesh_destroy(m);
    return st;
  }
  *out = m;
  return SWE_OK;
}

// Integrates every scenario's mass into its control word. The tiled step
// does not integrate it; k_cfl_tiled does, from the current state, leaving
// the step control (time step, end-time clamp, stop flag) as it is.
void refresh_mass(const swe_state* s) {
  const swe_mesh* m = s->mesh;
  if (m->kernel == SWE_KERNEL_TILED) {
    if (m->prm.precision == SWE_F64) launch_cfl<double>(s, swe::kMassOnly);
    else launch_cfl<float>(s, swe::kMassOnly);
  }
  swe::k_mass_sum<<<nscen(m), 256, 0, m->stream>>>(s->ctl, s->partial);
}

}  // namespace

namespace swe_host {

swe_status read_ctl(const swe_state* s) {
  CK(cudaMemcpyAsync(s->host_ctl, s->ctl, sizeof(swe::Ctl) * nscen(s->mesh), cudaMemcpyDeviceToHost,
                     s->mesh->stream));
  CK(cudaStreamSynchronize(s->mesh->stream));
  return SWE_OK;
}

static void free_mesh(swe_mesh* m) {
  if (m->arena.base) cudaFree(m->arena.base);
  if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
  delete m;
}

void retain_mesh(swe_mesh* m) { m->refs += 1; }

void release_mesh(swe_mesh* m) {
  m->refs -= 1;
  if (m->dead && m->refs == 0) free_mesh(m);
}

template <typename Real>
static void launch_forward_t(const swe_mesh* m, const swe::DevState<Real>& ds, cudaStream_t st,
                             bool back) {
  constexpr bool comp = sizeof(Real) == 4;
  swe::DevMesh<Real> dm = dev_mesh<Real>(m);
  if (m->pooled)  // the pooled k_tiled_step
    dm.chunks = back ? m->chunks_pool_back : m->chunks_pool;
  else if (back && m->chunks_back)
    dm.chunks = m->chunks_back;
  const swe::Num num = num_of(m);
  if (m->kernel == SWE_KERNEL_EDGE) {
    swe::k_edge_flux<Real><<<m->grid_edge, 256, 0, st>>>(dm, ds, num);
    swe::k_cell_update<Real, comp><<<m->grid_cell, 256, 0, st>>>(dm, ds, num);
  } else if (m->cpt == 2) {
    launch_tiled_cpt<Real, comp, 2>(m, dm, ds, num, st);
  } else {
    launch_tiled_cpt<Real, comp, 1>(m, dm, ds, num, st);
  }
}

void launch_forward(const swe_mesh* m, const swe::DevState<float>& ds, cudaStream_t st, bool back) {
  launch_forward_t<float>(m, ds, st, back);
}
void launch_forward(const swe_mesh* m, const swe::DevState<double>& ds, cudaStream_t st, bool back) {
  launch_forward_t<double>(m, ds, st, back);
}

void gather_any(const swe_mesh* m, const double* src, void* dst, int stride) {
  if (m->prm.precision == SWE_F64) launch_gather<double>(m, src, dst, stride);
  else launch_gather<float>(m, src, dst, stride);
}

void scatter_any(const swe_mesh* m, const void* src, double* dst, int stride) {
  if (m->prm.precision == SWE_F64) launch_scatter<double>(m, src, dst, stride);
  else launch_scatter<float>(m, src, dst, stride);
}

swe_status make_open_ended(swe_state* s) {
  open_end(s);
  CK(cudaGetLastError());
  return SWE_OK;
}

}  // namespace swe_host

extern "C" {

void swe_params_default(swe_params* p) {
  if (!p) return;
  p->g = 9.81;
  p->courant = 0.7;
  p->h_eps = 1e-6;
  p->precision = SWE_F64;
  p->order = SWE_ORDER_MORTON;
  p->kernel = SWE_KERNEL_AUTO;
  p->tile = 0;
  p->stages = 0;
  p->cells_per_thread = 0;
  p->halo_schedule = 0;
  p->wait_rounds = 0;
  p->compensated_depth = 0;
}

const char* swe_strerror(swe_status s) {
  switch (s) {
    case SWE_OK: return "ok";
    case SWE_EINVAL: return "invalid argument";
    case SWE_EMESH: return "invalid mesh";
    case SWE_ENOMEM: return "out of memory";
    case SWE_ECUDA: return "CUDA error";
    case SWE_ENAN: return "non-finite value in the state";
    case SWE_ETIMEOUT: return "device wait timed out";
    case SWE_EDRY: return "no wet cell: CFL time step undefined";
    case SWE_ESTATE: return "call not valid for this handle";
    default: return "unknown status";
  }
}

const char* swe_last_cuda_error(void) { return g_cuda_msg.c_str(); }

swe_status swe_mesh_create(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tris,
                           const swe_params* params, void* cuda_stream, swe_mesh** out) {
  return swe::guarded([&] { return create_batch(1, &xy, &n_nodes, &tri, &n_tris, params, cuda_stream, out); });
}

swe_status swe_mesh_create_part(const double* xy, int64_t n_nodes, const int32_t* tri,
                                int64_t n_tris, const uint8_t* ghost, const swe_params* params,
                                void* cuda_stream, swe_mesh** out) {
  if (!out) return SWE_EINVAL;
  *out = nullptr;
  if (!ghost) return SWE_EINVAL;
  swe_params p;
  swe_status st = resolve_params(params, p);
  if (st != SWE_OK) return st;
  if (p.kernel != SWE_KERNEL_TILED) return SWE_EINVAL;
  st = swe::guarded([&] { return create_batch(1, &xy, &n_nodes, &tri, &n_tris, &p, cuda_stream, out, ghost); });
  if (st == SWE_OK) (*out)->ghosts = true;
  return st;
}

swe_status swe_mesh_create_batch(int32_t n_scenarios, const double* const* xy,
                                 const int64_t* n_nodes, const int32_t* const* tri,
                                 const int64_t* n_tris, const swe_params* params,
                                 void* cuda_stream, swe_mesh** out) {
  return swe::guarded(
      [&] { return create_batch(n_scenarios, xy, n_nodes, tri, n_tris, params, cuda_stream, out); });
}

swe_status swe_mesh_counts(const swe_mesh* m, int64_t* counts) {
  if (!m || !counts) return SWE_EINVAL;
  counts[0] = m->V; counts[1] = m->T; counts[2] = m->E; counts[3] = m->Eb;
  return SWE_OK;
}

swe_status swe_mesh_scenarios(const swe_mesh* m, int32_t* n_scenarios, int64_t* n_tris) {
  if (!m || !n_scenarios) return SWE_EINVAL;
  *n_scenarios = nscen(m);
  if (n_tris)
    for (int i = 0; i < nscen(m); ++i) n_tris[i] = m->scen[i].ncells;
  return SWE_OK;
}

swe_status swe_mesh_device_bytes(const swe_mesh* m, int64_t* bytes) {
  if (!m || !bytes) return SWE_EINVAL;
  *bytes = (int64_t)m->arena.size;
  return SWE_OK;
}

void swe_mesh_destroy(swe_mesh* m) {
  if (!m) return;
  m->dead = true;
  m->refs += 1;  // the caller's own use, dropped at once
  release_mesh(m);
}

}  // extern "C"

namespace {

// swe_state_init and swe_state_init_device: the fields come from host
// arrays, or (on_device) from device arrays written on caller_stream.
swe_status state_init(swe_mesh* m, const double* h, const double* hu, const double* hv,
                      const double* z, const double* manning, double manning_const,
                      bool on_device, void* caller_stream, swe_state** out) {
  if (!out) return SWE_EINVAL;
  *out = nullptr;
  if (!m || !h || !hu || !hv || !z) return SWE_EINVAL;
  if (!manning && !(manning_const >= 0.0)) return SWE_EINVAL;
  const size_t w = real_size(m);
  const int64_t T = m->T, E = m->E, Tp = m->Tp;
  const int n = nscen(m);
  swe_state* s = new swe_state();
  s->mesh = m;
  retain_mesh(m);
  const bool interleaved = (m->kernel == SWE_KERNEL_TILED);
  Layout L;
  if (interleaved) {
    L.add(4 * w * Tp); L.add(4 * w * Tp);     // cells (h, hu, hv, z) x 2
  } else {
    for (int k = 0; k < 6; ++k) L.add(w * Tp);  // h, hu, hv x 2
    L.add(w * Tp);                              // z
  }
  L.add(w * Tp);                                // gn2
  if (m->kernel == SWE_KERNEL_EDGE) for (int k = 0; k < 5; ++k) L.add(w * E);
  L.add(8 * (size_t)m->max_grid);
  L.add(8 * T);                                 // staging
  const bool with_hlo = m->prm.compensated_depth != 0;
  if (with_hlo) L.add(4 * Tp);                  // depth residual (FP32)
  L.add(sizeof(swe::Ctl) * n);
  if (cudaMalloc((void**)&s->arena.base, L.total) != cudaSuccess) {
    cudaGetLastError();
    swe_state_destroy(s);
    return SWE_ENOMEM;
  }
  s->arena.size = L.total;
  if (cuda_failed(cudaMemsetAsync(s->arena.base, 0, L.total, m->stream))) {
    swe_state_destroy(s);
    return SWE_ECUDA;
  }
  if (interleaved) {
    s->stride = 4;
    for (int b = 0; b < 2; ++b) {
      char* c = (char*)s->arena.take(4 * w * Tp);
      s->h[b] = c;
      s->hu[b] = c + w;
      s->hv[b] = c + 2 * w;
    }
    s->z = (char*)s->h[0] + 3 * w;  // the step carries z into the other buffer
  } else {
    for (int b = 0; b < 2; ++b) {
      s->h[b] = s->arena.take(w * Tp);
      s->hu[b] = s->arena.take(w * Tp);
      s->hv[b] = s->arena.take(w * Tp);
    }
    s->z = s->arena.take(w * Tp);
  }
  s->gn2 = s->arena.take(w * Tp);
  if (m->kernel == SWE_KERNEL_EDGE) for (int k = 0; k < 5; ++k) s->fx[k] = s->arena.take(w * E);
  s->partial = (double*)s->arena.take(8 * (size_t)m->max_grid);
  s->stage = (double*)s->arena.take(8 * T);
  if (with_hlo) s->hlo = s->arena.take(4 * Tp);
  s->ctl = (swe::Ctl*)s->arena.take(sizeof(swe::Ctl) * n);
  swe_status st = SWE_OK;
  if (s->arena.overflow) {
    g_cuda_msg = "state arena layout";
    swe_state_destroy(s);
    return SWE_ECUDA;
  }
  if (cudaMallocHost((void**)&s->host_ctl, sizeof(swe::Ctl) * n) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    swe_state_destroy(s);
    return SWE_ECUDA;
  }
  if (on_device) st = wait_for_caller(m, caller_stream);
  // Bed and friction coefficient g n^2 (FP64, caller order): formed on the
  // host from host arrays or a constant n, on the device from a device n.
  std::vector<double> gn2;
  if (!(on_device && manning)) {
    gn2.resize(T);
    for (int64_t i = 0; i < T; ++i) {
      const double nn = manning ? manning[i] : manning_const;
      gn2[i] = m->prm.g * (nn * nn);
    }
  } else if (st == SWE_OK) {
    const int gg = grid_for(m->Tp, 256, m->sms * 16);
    if (m->prm.precision == SWE_F64)
      swe::k_gather_gn2<double><<<gg, 256, 0, m->stream>>>(manning, m->perm, (double*)s->gn2, m->Tp, m->prm.g);
    else
      swe::k_gather_gn2<float><<<gg, 256, 0, m->stream>>>(manning, m->perm, (float*)s->gn2, m->Tp, m->prm.g);
  }
  if (st == SWE_OK) {  // z lives in the cells, g n^2 is its own array
    const double* zf[3] = {z, nullptr, nullptr};
    void* zd[3] = {s->z, nullptr, nullptr};
    st = put_fields<double>(s, zf, zd, s->stride, on_device);
  }
  if (st == SWE_OK && !gn2.empty()) {  // else g n^2 was gathered on the device
    const double* nf[3] = {gn2.data(), nullptr, nullptr};
    void* nd[3] = {s->gn2, nullptr, nullptr};
    st = put_fields<double>(s, nf, nd, 1, false);
  }
  if (st == SWE_OK && cuda_failed(cudaStreamSynchronize(m->stream))) st = SWE_ECUDA;
  if (st == SWE_OK) st = upload_state_fields<double>(s, h, hu, hv, on_device);
  if (st == SWE_OK) st = reset_and_cfl(s);
  if (st != SWE_OK) {
    swe_state_destroy(s);
    return st;
  }
  *out = s;
  return SWE_OK;
}

}  // namespace

extern "C" {

swe_status swe_state_init(swe_mesh* m, const double* h, const double* hu, const double* hv,
                          const double* z, const double* manning, double manning_const,
                          swe_state** out) {
  return swe::guarded(
      [&] { return state_init(m, h, hu, hv, z, manning, manning_const, false, nullptr, out); });
}

swe_status swe_state_init_device(swe_mesh* m, const double* h, const double* hu, const double* hv,
                                 const double* z, const double* manning, double manning_const,
                                 void* cuda_stream, swe_state** out) {
  return swe::guarded(
      [&] { return state_init(m, h, hu, hv, z, manning, manning_const, true, cuda_stream, out); });
}

swe_status swe_state_set(swe_state* s, const double* h, const double* hu, const double* hv) {
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  swe_status st = upload_state_fields<double>(s, h, hu, hv);
  if (st != SWE_OK) return st;
  return reset_and_cfl(s);
}

swe_status swe_state_set_f32(swe_state* s, const float* h, const float* hu, const float* hv) {
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  swe_status st = upload_state_fields<float>(s, h, hu, hv);
  if (st != SWE_OK) return st;
  return reset_and_cfl(s);
}

swe_status swe_state_set_device(swe_state* s, const double* h, const double* hu, const double* hv,
                                void* cuda_stream) {
  if (!s || !h || !hu || !hv) return SWE_EINVAL;
  swe_status st = wait_for_caller(s->mesh, cuda_stream);
  if (st == SWE_OK) st = upload_state_fields<double>(s, h, hu, hv, true);
  if (st != SWE_OK) return st;
  return reset_and_cfl(s);
}

swe_status swe_step(swe_state* s, double* dt_used) {
  if (!s) return SWE_EINVAL;
  swe_status st = swe_sync(s);
  if (st != SWE_OK) return st;
  cudaStream_t str = s->mesh->stream;
  open_end(s);
  launch_one_step(s, str);
  CK(cudaGetLastError());
  st = read_ctl(s);
  if (st != SWE_OK) return st;
  if (dt_used) *dt_used = s->host_ctl[0].dt_last;
  return status_all(s);
}

swe_status swe_run(swe_state* s, int64_t n_steps) {
  if (!s || n_steps < 0) return SWE_EINVAL;
  open_end(s);
  if (n_steps == 0) return ensure_graph(s);  // prepare the graph, take no step
  return queue_steps(s, n_steps);
}

swe_status swe_advance(swe_state* s, double t_end, int64_t* n_steps) {
  if (!s || !(t_end == t_end)) return SWE_EINVAL;
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  const long long start = s->host_ctl[0].steps;
  set_end(s, t_end);
  s->open_ended = false;
  CK(cudaGetLastError());
  for (;;) {
    st = read_ctl(s);
    if (st != SWE_OK) return st;
    if (all_done(s)) break;
    st = queue_steps(s, kStepsPerGraph);
    if (st != SWE_OK) return st;
  }
  if (n_steps) *n_steps = s->host_ctl[0].steps - start;
  return status_all(s);
}

swe_status swe_sync(swe_state* s) {
  if (!s) return SWE_EINVAL;
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  return status_all(s);
}

}  // extern "C"

namespace {

template <typename Host>
void launch_take(const swe_state* s, int b, int64_t c0, int64_t c1, Host* const f[3]) {
  const swe_mesh* m = s->mesh;
  if (c1 <= c0 || (!f[0] && !f[1] && !f[2])) return;
  const int grid = grid_for(c1 - c0, 256, m->sms * 16);
  if (m->prm.precision == SWE_F64)
    swe::k_take_fields<double, Host><<<grid, 256, 0, m->stream>>>(
        (const double*)s->h[b], (const double*)s->hu[b], (const double*)s->hv[b], nullptr,
        m->iperm, c0, c1, f[0], f[1], f[2], s->stride);
  else
    swe::k_take_fields<float, Host><<<grid, 256, 0, m->stream>>>(
        (const float*)s->h[b], (const float*)s->hu[b], (const float*)s->hv[b],
        (const float*)s->hlo, m->iperm, c0, c1, f[0], f[1], f[2], s->stride);
}

// swe_copy_out[_f32] and swe_copy_out_device (to_device: h, hu, hv are
// device arrays). Each scenario's cells are read from the buffer its
// control word names (scenarios that stopped at different step counts sit
// in different buffers); consecutive scenarios in the same buffer form one
// range of caller cells. Device arrays and page-locked host arrays are
// written by one kernel per range; other host arrays through the staging
// buffer, one field at a time.
template <typename Host>
swe_status copy_out(const swe_state* s, Host* h, Host* hu, Host* hv, double* t, double* mass,
                    bool to_device) {
  if (!s) return SWE_EINVAL;
  const swe_mesh* m = s->mesh;
  const int n = nscen(m);
  if (mass) refresh_mass(s);
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  struct Range {
    int64_t c0, c1;
    int b;
  };
  std::vector<Range> ranges;
  for (int i = 0; i < n; ++i) {
    const Scenario& sc = m->scen[i];
    const int b = s->host_ctl[i].cur;
    if (!ranges.empty() && ranges.back().b == b && ranges.back().c1 == sc.caller0)
      ranges.back().c1 = sc.caller0 + sc.ncells;
    else
      ranges.push_back({sc.caller0, sc.caller0 + sc.ncells, b});
  }
  Host* dst[3] = {h, hu, hv};
  Host* direct[3] = {nullptr, nullptr, nullptr};
  for (int k = 0; k < 3; ++k)
    if (dst[k]) direct[k] = to_device ? dst[k] : (Host*)mapped_host(dst[k]);
  for (const Range& r : ranges) launch_take<Host>(s, r.b, r.c0, r.c1, direct);
  for (int k = 0; k < 3; ++k) {
    if (!dst[k] || direct[k]) continue;
    Host* one[3] = {nullptr, nullptr, nullptr};
    one[k] = (Host*)s->stage;
    for (const Range& r : ranges) launch_take<Host>(s, r.b, r.c0, r.c1, one);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(dst[k], s->stage, m->T * sizeof(Host), cudaMemcpyDeviceToHost, m->stream));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(m->stream));
  if (t) *t = s->host_ctl[0].t;
  if (mass) {
    double sum = 0.0;
    for (int i = 0; i < n; ++i) sum += s->host_ctl[i].mass;
    *mass = sum;
  }
  return status_all(s);
}

}  // namespace

extern "C" {

swe_status swe_copy_out(const swe_state* s, double* h, double* hu, double* hv, double* t,
                        double* mass) {
  return copy_out<double>(s, h, hu, hv, t, mass, false);
}

swe_status swe_copy_out_f32(const swe_state* s, float* h, float* hu, float* hv, double* t,
                            double* mass) {
  return copy_out<float>(s, h, hu, hv, t, mass, false);
}

swe_status swe_copy_out_device(const swe_state* s, double* h, double* hu, double* hv, double* t,
                               double* mass, void* cuda_stream) {
  if (!s) return SWE_EINVAL;
  // the destinations may still be in use by the caller's earlier work
  swe_status st = wait_for_caller(s->mesh, cuda_stream);
  if (st != SWE_OK) return st;
  return copy_out<double>(s, h, hu, hv, t, mass, true);
}

swe_status swe_state_info(const swe_state* s, int64_t* info) {
  if (!s || !info) return SWE_EINVAL;
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  info[0] = s->host_ctl[0].steps;
  info[1] = 0;
  info[2] = 0;
  for (int i = 0; i < nscen(s->mesh); ++i) {
    info[1] += s->host_ctl[i].neg;
    info[2] |= s->host_ctl[i].err;
  }
  return SWE_OK;
}

swe_status swe_scenario_info(const swe_state* s, int32_t scenario, double* t, double* mass,
                             int64_t* steps, double* dt_next) {
  if (!s || scenario < 0 || scenario >= nscen(s->mesh)) return SWE_EINVAL;
  if (mass) refresh_mass(s);
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  const swe::Ctl& c = s->host_ctl[scenario];
  if (t) *t = c.t;
  if (mass) *mass = c.mass;
  if (steps) *steps = c.steps;
  if (dt_next) *dt_next = c.dt_cfl;
  return status_from_err(c.err);
}

swe_status swe_next_dt(const swe_state* s, double* dt) {
  if (!s || !dt) return SWE_EINVAL;
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  *dt = s->host_ctl[0].dt_cfl;
  return status_all(s);
}

void swe_state_destroy(swe_state* s) {
  if (!s) return;
  swe_mesh* m = s->mesh;
  if (m && m->stream) cudaStreamSynchronize(m->stream);
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->capture) cudaStreamDestroy(s->capture);
  if (s->host_ctl) cudaFreeHost(s->host_ctl);
  if (s->arena.base) cudaFree(s->arena.base);
  delete s;
  if (m) release_mesh(m);
}

}  // extern "C"
