// swe_step_edges_static: one FP64 step of the two-launch kernels (per-edge
// face outputs, then the per-cell gather and update) that allocates nothing.
//
// Some callers cannot call cudaMalloc: programs that must not allocate once
// they are running (fixed memory budgets, real-time loops whose timing an
// allocation would disturb), and hosts whose device memory belongs to their
// own pool or arena, where a foreign cudaMalloc would bypass that pool's
// accounting and may synchronise the device. This entry point takes every
// input and output as a device pointer from the caller, and keeps its
// scratch (the per-edge face outputs, the per-block mass partial sums and
// the step control word) in the file-scope device array below, sized at
// build time.
//
// The scratch array exists once per GPU that loads this library and stays
// allocated until the process exits. Every call uses the same array and
// leaves the previous call's contents in it; each call resets the control
// word before use and overwrites the rest. Calls whose work overlaps on the
// GPU (other streams, other host threads) race on the array and give wrong
// results: serialise them.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <utility>

#include "../../include/swe.h"
#include "swe_kernels.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)SWE_STATIC_SCRATCH_BYTES;
constexpr int kMaxBlocks = 4096;          // cap on the update grid (mass partials)
constexpr size_t kHeadBytes = 64 * 1024;  // control word + partials, at the front

static_assert(256 + 8 * kMaxBlocks <= kHeadBytes && sizeof(swe::Ctl) <= 256, "scratch head too small");
static_assert(kHeadBytes + 5 * 8 * (size_t)SWE_STATIC_MAX_EDGES <= kScratchBytes, "scratch too small");

// The scratch. Device code could name it directly; host code must not pass
// its host-side name to a kernel (that is a stand-in, not a device address),
// so the address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
int g_grid_cell[kMaxDevices] = {};
int g_grid_edge[kMaxDevices] = {};

// Per-device set-up, done by the first call on each device with that device
// current: device address of the scratch and launch sizes.
swe_status setup(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[dev]) return SWE_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return SWE_ECUDA;
  }
  int sms = 0, occ_c = 0, occ_e = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, swe::k_cell_update<double, false>, 256, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_e, swe::k_edge_flux<double>, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    return SWE_ECUDA;
  }
  g_sms[dev] = sms;
  g_grid_cell[dev] = std::min(kMaxBlocks, sms * (occ_c > 0 ? occ_c : 1));
  g_grid_edge[dev] = sms * (occ_e > 0 ? occ_e : 1) * 4;
  g_addr[dev] = p;
  return SWE_OK;
}

// Resets the control word for one step of length dt from buffer 0.
__global__ void k_static_begin(swe::Ctl* ctl, double dt) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  swe::Ctl c{};
  c.t = 0.0;
  c.t_end = __longlong_as_double(0x7ff0000000000000ll);  // +inf
  c.dt = dt;
  c.dt_cfl = dt;
  *ctl = c;
}

// Launches kernel<<<grid, block, 0, stream>>>(args...) and returns the
// launch's own status.
template <typename... Params, typename... Args>
cudaError_t launch(void (*kernel)(Params...), int grid, int block, cudaStream_t stream,
                   Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace

extern "C" swe_status swe_step_edges_static(
    int64_t n_cells, int64_t n_edges, const int32_t* edge_left, const int32_t* edge_right,
    const double* edge_nx, const double* edge_ny, const double* edge_len, const int32_t* cell_face,
    const double* cell_area, const double* cell_perim_over_area, const double* gn2,
    const double* z, const double* h, const double* hu, const double* hv, double g,
    double courant, double h_eps, double dt, double* h_out, double* hu_out, double* hv_out,
    double* next_dt, double* mass, void* cuda_stream) {
  if (n_cells <= 0 || n_edges <= 0 || !edge_left || !edge_right || !edge_nx || !edge_ny ||
      !edge_len || !cell_face || !cell_area || !cell_perim_over_area || !gn2 || !z || !h || !hu ||
      !hv || !h_out || !hu_out || !hv_out || !(dt >= 0.0) || !std::isfinite(dt) || !(g > 0.0) ||
      !(courant > 0.0) || !(h_eps >= 0.0))
    return SWE_EINVAL;
  if (n_edges > SWE_STATIC_MAX_EDGES || n_cells > n_edges) return SWE_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SWE_ECUDA;
  }
  swe_status st = setup(dev);
  if (st != SWE_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  char* base = (char*)g_addr[dev];
  swe::Ctl* ctl = (swe::Ctl*)base;
  double* partial = (double*)(base + 256);
  double* faces = (double*)(base + kHeadBytes);

  swe::DevMesh<double> m{};
  m.T = n_cells;
  m.E = n_edges;
  m.area = cell_area;
  m.irP = cell_perim_over_area;
  m.eL = edge_left;
  m.eR = edge_right;
  m.nx = edge_nx;
  m.ny = edge_ny;
  m.len = edge_len;
  m.cf0 = cell_face;
  m.cf1 = cell_face + n_cells;
  m.cf2 = cell_face + 2 * n_cells;
  swe::DevState<double> s{};
  s.h[0] = const_cast<double*>(h);
  s.hu[0] = const_cast<double*>(hu);
  s.hv[0] = const_cast<double*>(hv);
  s.h[1] = h_out;
  s.hu[1] = hu_out;
  s.hv[1] = hv_out;
  s.stride = 1;
  s.z = z;
  s.gn2 = gn2;
  for (int k = 0; k < 5; ++k) s.fx[k] = faces + (size_t)k * n_edges;
  s.partial = partial;
  s.ctl = ctl;
  const swe::Num num = swe::make_num(g, courant, h_eps);

  const int ge = (int)std::min<int64_t>((n_edges + 255) / 256, g_grid_edge[dev]);
  const int gc = (int)std::min<int64_t>((n_cells + 255) / 256, g_grid_cell[dev]);
  // Each launch's own status is checked (a CUDA error left pending by the
  // caller's earlier work is neither reported as this call's nor cleared).
  auto launch_failed = [](cudaError_t e) {
    if (e == cudaSuccess) return false;
    cudaGetLastError();  // clear this launch's error
    return true;
  };
  if (launch_failed(launch(k_static_begin, 1, 1, stream, ctl, dt)) ||
      launch_failed(launch(swe::k_edge_flux<double>, ge, 256, stream, m, s, num)) ||
      launch_failed(launch(swe::k_cell_update<double, false>, gc, 256, stream, m, s, num)) ||
      (mass && launch_failed(launch(swe::k_mass_sum, 1, 256, stream, ctl, partial))))
    return SWE_ECUDA;
  if (next_dt || mass) {
    swe::Ctl c;
    if (cudaMemcpyAsync(&c, ctl, sizeof(c), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
      cudaGetLastError();
      return SWE_ECUDA;
    }
    if (next_dt) *next_dt = c.dt_cfl;
    if (mass) *mass = c.mass;
    if (c.err & swe::kErrNan) return SWE_ENAN;
    if (c.err & swe::kErrDry) return SWE_EDRY;
  }
  return SWE_OK;
}
