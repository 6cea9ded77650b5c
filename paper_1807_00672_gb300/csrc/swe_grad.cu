// Gradients through many steps (swe_grad_record / swe_grad, include/swe.h).
//
// swe_grad_record runs n steps forward on a state, as swe_run does, and
// keeps a tape: the dt of every step (held fixed for the derivative), the
// depths at the gauge cells after every step, and the state every K steps
// (checkpoints). swe_grad then runs the adjoint backwards through the steps:
// segment by segment, from the last checkpoint to the first, it recomputes
// the segment's inner states from its checkpoint with the forward kernel
// (the forward is deterministic, so the replay reproduces the recorded
// states bit for bit; the replay's dt is checked against the recorded one;
// the segment's last state is the next checkpoint, or the final state, and
// is not recomputed) and applies the tiled adjoint kernel step by step,
// adding the gauge-loss seeds as it passes their steps. The replay of the
// next segment runs on a second stream while the current segment's adjoint
// steps run, each into its own ring of states. Memory: ceil(n / K) + 1
// checkpoints, 2 (K - 1) replayed states and two adjoint states. K = 1
// keeps every state and replays nothing.
#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "../../include/swe.h"
#include "swe_adjoint.cuh"
#include "mesh_build.h"
#include "swe_handles.cuh"
#include "swe_kernels.cuh"

using namespace swe_host;

namespace {

#define cuda_failed(call) swe_host::cuda_failed_at((call), #call, __FILE__, __LINE__)
#define CK(call)                              \
  do {                                        \
    if (cuda_failed(call)) return SWE_ECUDA;  \
  } while (0)

constexpr int kErrReplay = 8;  // a replayed step did not reproduce the recorded dt

// After forward step k: its dt and the gauge depths of the new state.
template <typename Real>
__global__ void k_record_step(const swe::Ctl* ctl, const Real* b0, const Real* b1, double* dts,
                              int64_t k, const int32_t* cells, int G, double* gauge) {
  const Real* U = ctl->cur ? b1 : b0;
  if (blockIdx.x == 0 && threadIdx.x == 0) dts[k] = ctl->dt_last;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < G; j += gridDim.x * blockDim.x)
    gauge[k * (int64_t)G + j] = (double)U[4 * (int64_t)cells[j]];
}

// Copies the current buffer (n interleaved cells) to dst.
template <typename Real>
__global__ void k_copy_current(const swe::Ctl* ctl, const Real* b0, const Real* b1, Real* dst,
                               int64_t n) {
  const Real* U = ctl->cur ? b1 : b0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const swe::V4<Real> v = swe::ld4(U + 4 * i);
    swe::st4(dst + 4 * i, v.x, v.y, v.z, v.w);
  }
}

// Replay control word: buffer 0 current, the recorded dt, no end time.
__global__ void k_replay_begin(swe::Ctl* ctl, double dt, long long part0, long long nparts) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  swe::Ctl c{};
  c.t = 0.0;
  c.t_end = __longlong_as_double(0x7ff0000000000000ll);  // +inf
  c.dt = dt;
  c.dt_cfl = dt;
  c.part0 = part0;
  c.nparts = nparts;
  *ctl = c;
}

// The last replayed step must have used the recorded dt.
__global__ void k_replay_check(const swe::Ctl* ctl, double dt, int* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (ctl->dt_last != dt || ctl->err) atomicOr(err, kErrReplay | ctl->err);
}

// dL/dn = dL/d(g n^2) * 2 g n with n = sqrt(g n^2 / g) >= 0.
template <typename Real>
__global__ void k_finish_dn(const Real* dgn2, const Real* gn2, double g, Real* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = Real((double)dgn2[i] * 2.0 * sqrt(g * (double)gn2[i]));
}

// Programmatic dependent launch: a step's blocks fetch their first tiles'
// tape and mesh data while the previous adjoint step's last blocks finish,
// and wait for it (griddepcontrol.wait) before reading its output.
template <typename Real, int NT, int CPT>
void launch_adjoint_nt(const swe_mesh* m, const swe::DevMesh<Real>& dm, const swe::AdjArgs<Real>& a,
                       const swe::AdjLayout& L, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = L.total;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, swe::k_tiled_adjoint<Real, NT, 2, CPT>, dm, a, num_of(m), L);
}

template <typename Real, int CPT>
void launch_adjoint_cpt(const swe_mesh* m, const swe::DevMesh<Real>& dm, const swe::AdjArgs<Real>& a,
                        const swe::AdjLayout& L, int grid, cudaStream_t st) {
  switch (m->tile / CPT) {
    case 32: launch_adjoint_nt<Real, 32, CPT>(m, dm, a, L, grid, st); break;
    case 64: launch_adjoint_nt<Real, 64, CPT>(m, dm, a, L, grid, st); break;
    case 128: launch_adjoint_nt<Real, 128, CPT>(m, dm, a, L, grid, st); break;
    default: launch_adjoint_nt<Real, 256, CPT>(m, dm, a, L, grid, st); break;
  }
}

// The adjoint runs on its own chunk table (one wave at its own occupancy).
template <typename Real>
void launch_adjoint(const swe_mesh* m, const swe::Chunk* chunks, int grid,
                    const swe::AdjArgs<Real>& a, const swe::AdjLayout& L, cudaStream_t st) {
  swe::DevMesh<Real> dm = dev_mesh<Real>(m);
  dm.chunks = chunks;
  if (m->cpt == 2) launch_adjoint_cpt<Real, 2>(m, dm, a, L, grid, st);
  else launch_adjoint_cpt<Real, 1>(m, dm, a, L, grid, st);
}

// Opts the adjoint kernel into its shared memory; resident blocks per SM.
template <typename Real, int NT, int CPT>
int prepare_adjoint_nt(const swe::AdjLayout& L) {
  auto k = swe::k_tiled_adjoint<Real, NT, 2, CPT>;
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

template <typename Real, int CPT>
int prepare_adjoint_cpt(const swe_mesh* m, const swe::AdjLayout& L) {
  switch (m->tile / CPT) {
    case 32: return prepare_adjoint_nt<Real, 32, CPT>(L);
    case 64: return prepare_adjoint_nt<Real, 64, CPT>(L);
    case 128: return prepare_adjoint_nt<Real, 128, CPT>(L);
    default: return prepare_adjoint_nt<Real, 256, CPT>(L);
  }
}

template <typename Real>
int prepare_adjoint(const swe_mesh* m, const swe::AdjLayout& L) {
  return m->cpt == 2 ? prepare_adjoint_cpt<Real, 2>(m, L) : prepare_adjoint_cpt<Real, 1>(m, L);
}

int grid_for(int64_t n, int cap) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

}  // namespace

struct swe_tape {
  swe_mesh* mesh = nullptr;
  cudaStream_t stream = nullptr;
  int64_t N = 0, K = 0, nck = 0;
  int G = 0;
  size_t w = 8;
  int64_t Tp = 0, T = 0;
  Arena arena;
  char* ck = nullptr;    // nck + 1 states of Tp interleaved cells: U^0, U^K, U^2K, ..., U^N
  // Two rings of K - 1 replayed states U^{j0+1} .. U^{j0+K-1}: segment seg
  // uses ring seg % 2, so the replay of the next segment (on the side
  // stream) overlaps the adjoint steps of the current one. The last
  // segment's inner states are kept from the recording in `tail`, so a
  // backward sweep starts with adjoint steps instead of a replay.
  char* ring[2] = {nullptr, nullptr};
  char* tail = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t replayed[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  char* lam[2] = {nullptr, nullptr};
  void* gn2 = nullptr;   // copy of the state's g n^2
  void* dgn2 = nullptr;
  void* scratch = nullptr;
  double* stage = nullptr;  // T doubles
  double* dts_dev = nullptr;
  double* gauge_dev = nullptr;
  double* gseed_dev = nullptr;
  int32_t* gcells = nullptr;
  swe::Chunk* chunks = nullptr;  // work of the adjoint kernel's blocks
  int64_t nchunks = 0;
  swe::Ctl* ctl = nullptr;      // two replay control words (one per ring)
  double* partial = nullptr;    // two arrays of per-chunk mass partials
  int* err = nullptr;
  unsigned int* ticket = nullptr;
  std::vector<double> dts;
  swe::AdjLayout adj{};
  float record_ms = 0.f, grad_ms = 0.f;
  cudaEvent_t ev[2] = {nullptr, nullptr};

  size_t state_bytes() const { return 4 * w * (size_t)Tp; }
  int64_t seg_len(int64_t seg) const { return std::min(N, (seg + 1) * K) - seg * K; }
  void* slot(int64_t seg, int64_t r) const {  // state U^{seg K + r} of segment seg
    if (r == 0) return ck + seg * state_bytes();
    if (r == seg_len(seg)) return ck + (seg + 1) * state_bytes();
    if (seg == nck - 1) return tail + (r - 1) * state_bytes();
    return ring[seg % 2] + (r - 1) * state_bytes();
  }
};

namespace {

void free_tape(swe_tape* t) {
  if (t->mesh && t->stream) cudaStreamSynchronize(t->stream);
  if (t->side) cudaStreamSynchronize(t->side);
  for (auto& e : t->ev)
    if (e) cudaEventDestroy(e);
  for (int i = 0; i < 2; ++i) {
    if (t->replayed[i]) cudaEventDestroy(t->replayed[i]);
    if (t->consumed[i]) cudaEventDestroy(t->consumed[i]);
  }
  if (t->side) cudaStreamDestroy(t->side);
  if (t->arena.base) cudaFree(t->arena.base);
  swe_mesh* m = t->mesh;
  delete t;
  if (m) release_mesh(m);
}

// Device state view of replay step r of segment seg (input slot r, output
// slot r + 1; the current buffer alternates as the replay control word says).
template <typename Real>
swe::DevState<Real> replay_state(const swe_tape* t, int64_t seg, int64_t r) {
  swe::DevState<Real> d{};
  Real* in = (Real*)t->slot(seg, r);
  Real* out = (Real*)t->slot(seg, r + 1);
  Real* b0 = (r % 2 == 0) ? in : out;
  Real* b1 = (r % 2 == 0) ? out : in;
  d.h[0] = b0; d.hu[0] = b0 + 1; d.hv[0] = b0 + 2;
  d.h[1] = b1; d.hu[1] = b1 + 1; d.hv[1] = b1 + 2;
  d.stride = 4;
  d.z = b0 + 3;
  d.gn2 = (const Real*)t->gn2;
  d.partial = t->partial + (seg % 2) * std::max<int64_t>(1, t->mesh->nchunks);
  d.ctl = t->ctl + seg % 2;
  return d;
}

template <typename Real>
swe_status record_t(swe_state* s, swe_tape* t) {
  swe_mesh* m = s->mesh;
  cudaStream_t st = m->stream;
  const int gs = grid_for(t->Tp, m->sms * 8);
  const Real* b0 = (const Real*)s->h[0];
  const Real* b1 = (const Real*)s->h[1];
  k_copy_current<Real><<<gs, 256, 0, st>>>(s->ctl, b0, b1, (Real*)t->ck, t->Tp);
  CK(cudaMemcpyAsync(t->gn2, s->gn2, t->w * t->Tp, cudaMemcpyDeviceToDevice, st));
  CK(cudaEventRecord(t->ev[0], st));
  const int64_t j_tail = (t->nck - 1) * t->K;  // first step of the last segment
  for (int64_t k = 0; k < t->N; ++k) {
    launch_forward(m, dev_state<Real>(s), st);
    k_record_step<Real><<<1, 128, 0, st>>>(s->ctl, b0, b1, t->dts_dev, k, t->gcells, t->G,
                                           t->gauge_dev);
    if (k + 1 > j_tail && k + 1 < t->N)  // an inner state of the last segment
      k_copy_current<Real><<<gs, 256, 0, st>>>(s->ctl, b0, b1,
                                               (Real*)t->slot(t->nck - 1, k + 1 - j_tail), t->Tp);
    if ((k + 1) % t->K == 0 || k + 1 == t->N)
      k_copy_current<Real><<<gs, 256, 0, st>>>(s->ctl, b0, b1,
                                               (Real*)(t->ck + ((k + t->K) / t->K) * t->state_bytes()),
                                               t->Tp);
  }
  CK(cudaEventRecord(t->ev[1], st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  CK(cudaEventElapsedTime(&t->record_ms, t->ev[0], t->ev[1]));
  return SWE_OK;
}

// Recomputes the inner states U^{j0+1} .. U^{j1-1} of segment seg into its
// ring, on stream st.
template <typename Real>
void replay_segment(swe_tape* t, int64_t seg, cudaStream_t st) {
  const swe_mesh* m = t->mesh;
  const Scenario& sc = m->scen[0];
  const int64_t j0 = seg * t->K, j1 = std::min(t->N, j0 + t->K);
  if (j1 - j0 <= 1) return;
  swe::Ctl* ctl = t->ctl + seg % 2;
  k_replay_begin<<<1, 1, 0, st>>>(ctl, t->dts[j0], sc.chunk0, sc.nchunks);
  for (int64_t r = 0; r + 1 < j1 - j0; ++r) launch_forward(m, replay_state<Real>(t, seg, r), st);
  k_replay_check<<<1, 1, 0, st>>>(ctl, t->dts[j1 - 2], t->err);
}

template <typename Real>
swe_status grad_t(swe_tape* t, bool seeds_gauge, int* lam_cur) {
  swe_mesh* m = t->mesh;
  cudaStream_t st = m->stream;
  int cur = 0;
  if (seeds_gauge)
    swe::k_inject_gauges<Real><<<1, 1, 0, st>>>((Real*)t->lam[cur], t->gcells, t->gseed_dev, t->N - 1, t->G);
  // Replays run one segment ahead on the side stream: segment seg - 1's
  // replay (ring (seg - 1) % 2) overlaps segment seg's adjoint steps; it
  // first waits for the adjoint of segment seg + 1, the ring's last user.
  // The last segment needs none (its states are in the tail).
  CK(cudaEventRecord(t->consumed[0], st));
  CK(cudaEventRecord(t->consumed[1], st));
  for (int64_t seg = t->nck - 1; seg >= 0; --seg) {
    const int64_t j0 = seg * t->K, j1 = std::min(t->N, j0 + t->K);
    if (seg >= 1) {
      CK(cudaStreamWaitEvent(t->side, t->consumed[(seg - 1) % 2], 0));
      replay_segment<Real>(t, seg - 1, t->side);
      CK(cudaEventRecord(t->replayed[(seg - 1) % 2], t->side));
    }
    if (seg < t->nck - 1) CK(cudaStreamWaitEvent(st, t->replayed[seg % 2], 0));
    for (int64_t j = j1 - 1; j >= j0; --j) {
      const int64_t r = j - j0;
      swe::AdjArgs<Real> a{};
      a.un = (const Real*)t->slot(seg, r);
      a.u1 = (const Real*)t->slot(seg, r + 1);
      a.lam_in = (const Real*)t->lam[cur];
      a.lam_out = (Real*)t->lam[cur ^ 1];
      a.gn2 = (const Real*)t->gn2;
      a.dgn2 = (Real*)t->dgn2;
      a.dt = Real(t->dts[j]);
      a.err = t->err;
      a.gcells = t->gcells;
      a.gseed = t->gseed_dev;
      a.G = t->G;
      a.gstep = (seeds_gauge && j >= 1) ? (long long)(j - 1) : -1ll;  // lambda^j gets dL/dh^j
      a.ticket = t->ticket;
      launch_adjoint<Real>(m, t->chunks, (int)t->nchunks, a, t->adj, st);
      cur ^= 1;
    }
    CK(cudaEventRecord(t->consumed[seg % 2], st));
  }
  CK(cudaGetLastError());
  *lam_cur = cur;
  return SWE_OK;
}

swe_status grad_record(swe_state* s, int64_t n_steps, int64_t checkpoint_every,
                       const int32_t* gauge_cells, int32_t n_gauges, double* gauge_h,
                       swe_tape** out) {
  if (!out) return SWE_EINVAL;
  *out = nullptr;
  if (!s || n_steps <= 0 || checkpoint_every <= 0 || n_gauges < 0 || (n_gauges > 0 && !gauge_cells))
    return SWE_EINVAL;
  swe_mesh* m = s->mesh;
  if (m->kernel != SWE_KERNEL_TILED || nscen(m) != 1 || m->ghosts || m->tile / m->cpt > 256 ||
      m->prm.compensated_depth)
    return SWE_ESTATE;
  for (int j = 0; j < n_gauges; ++j)
    if (gauge_cells[j] < 0 || gauge_cells[j] >= m->T) return SWE_EINVAL;
  swe_status st = read_ctl(s);
  if (st != SWE_OK) return st;
  if (s->host_ctl[0].err) return SWE_ESTATE;

  swe_tape* t = new swe_tape();
  t->mesh = m;
  retain_mesh(m);
  t->stream = m->stream;
  t->N = n_steps;
  t->K = std::min(checkpoint_every, n_steps);
  t->nck = (n_steps + t->K - 1) / t->K;
  t->G = n_gauges;
  t->w = m->prm.precision == SWE_F64 ? 8 : 4;
  t->Tp = m->Tp;
  t->T = m->T;
  const int geo_arrays = (m->prm.precision == SWE_F64) ? 3 : 2;
  t->adj = swe::make_adj_layout((uint32_t)t->w, (uint32_t)geo_arrays, (uint32_t)m->tile, 2u,
                                (uint32_t)m->layout.rec_cap, (uint32_t)m->layout.halo_cap);
  const int occ = m->prm.precision == SWE_F64 ? prepare_adjoint<double>(m, t->adj)
                                              : prepare_adjoint<float>(m, t->adj);
  if (occ < 1) {
    g_cuda_msg = "adjoint kernel layout does not fit in shared memory";
    free_tape(t);
    return SWE_ECUDA;
  }
  // adjoint chunk table: one wave of resident blocks over the scenario's tiles
  std::vector<swe::Chunk> chunks;
  {
    const Scenario& sc = m->scen[0];
    const int64_t resident = (int64_t)m->sms * occ;
    const int64_t per = std::max<int64_t>(1, (sc.ntiles + resident - 1) / resident);
    const int64_t nc = (sc.ntiles + per - 1) / per;
    for (int64_t r = 0; r < nc; ++r) {
      swe::Chunk c{};
      c.scen = 0;
      c.tile0 = (int32_t)(sc.tile0 + r);
      c.ntiles = (int32_t)((sc.ntiles - r + nc - 1) / nc);
      c.stride = (int32_t)nc;
      c.part = (int32_t)r;
      c.cell_end = (int32_t)(sc.cell0 + sc.ncells);
      chunks.push_back(c);
    }
    t->nchunks = nc;
  }
  const size_t sb = t->state_bytes();
  Layout L;
  L.add(sb * (t->nck + 1));
  L.add(sb * std::max<int64_t>(1, t->K - 1));
  L.add(sb * std::max<int64_t>(1, t->K - 1));
  L.add(sb * std::max<int64_t>(1, t->K - 1));  // tail
  L.add(sb); L.add(sb);
  L.add(t->w * t->Tp);  // gn2
  L.add(t->w * t->Tp);  // dgn2
  L.add(t->w * t->Tp);  // scratch
  L.add(8 * t->T);      // stage
  L.add(8 * t->N);      // dts
  L.add(8 * t->N * std::max(1, t->G));  // gauge depths
  L.add(8 * t->N * std::max(1, t->G));  // gauge seeds
  L.add(4 * std::max(1, t->G));
  L.add(sizeof(swe::Chunk) * chunks.size());
  L.add(2 * sizeof(swe::Ctl));
  L.add(2 * 8 * (size_t)std::max<int64_t>(1, m->nchunks));
  L.add(sizeof(int));
  L.add(sizeof(unsigned int));
  if (cudaMalloc((void**)&t->arena.base, L.total) != cudaSuccess) {
    cudaGetLastError();
    free_tape(t);
    return SWE_ENOMEM;
  }
  t->arena.size = L.total;
  t->ck = (char*)t->arena.take(sb * (t->nck + 1));
  t->ring[0] = (char*)t->arena.take(sb * std::max<int64_t>(1, t->K - 1));
  t->ring[1] = (char*)t->arena.take(sb * std::max<int64_t>(1, t->K - 1));
  t->tail = (char*)t->arena.take(sb * std::max<int64_t>(1, t->K - 1));
  t->lam[0] = (char*)t->arena.take(sb);
  t->lam[1] = (char*)t->arena.take(sb);
  t->gn2 = t->arena.take(t->w * t->Tp);
  t->dgn2 = t->arena.take(t->w * t->Tp);
  t->scratch = t->arena.take(t->w * t->Tp);
  t->stage = (double*)t->arena.take(8 * t->T);
  t->dts_dev = (double*)t->arena.take(8 * t->N);
  t->gauge_dev = (double*)t->arena.take(8 * t->N * std::max(1, t->G));
  t->gseed_dev = (double*)t->arena.take(8 * t->N * std::max(1, t->G));
  t->gcells = (int32_t*)t->arena.take(4 * std::max(1, t->G));
  t->chunks = (swe::Chunk*)t->arena.take(sizeof(swe::Chunk) * chunks.size());
  t->ctl = (swe::Ctl*)t->arena.take(2 * sizeof(swe::Ctl));
  t->partial = (double*)t->arena.take(2 * 8 * (size_t)std::max<int64_t>(1, m->nchunks));
  t->err = (int*)t->arena.take(sizeof(int));
  t->ticket = (unsigned int*)t->arena.take(sizeof(unsigned int));
  if (t->arena.overflow) {
    g_cuda_msg = "tape arena layout";
    free_tape(t);
    return SWE_ECUDA;
  }
  auto fail = [&](swe_status r) { free_tape(t); return r; };
  if (cuda_failed(cudaMemsetAsync(t->arena.base, 0, L.total, m->stream)) ||
      cuda_failed(cudaEventCreate(&t->ev[0])) || cuda_failed(cudaEventCreate(&t->ev[1])) ||
      cuda_failed(cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking)))
    return fail(SWE_ECUDA);
  for (int i = 0; i < 2; ++i)
    if (cuda_failed(cudaEventCreateWithFlags(&t->replayed[i], cudaEventDisableTiming)) ||
        cuda_failed(cudaEventCreateWithFlags(&t->consumed[i], cudaEventDisableTiming)))
      return fail(SWE_ECUDA);
  if (cuda_failed(cudaMemcpyAsync(t->chunks, chunks.data(), sizeof(swe::Chunk) * chunks.size(),
                                  cudaMemcpyHostToDevice, m->stream)) ||
      cuda_failed(cudaStreamSynchronize(m->stream)))
    return fail(SWE_ECUDA);
  // gauge cells in internal order
  if (t->G > 0) {
    std::vector<int32_t> perm(m->Tp), inv(m->T, -1), gi(t->G);
    if (cuda_failed(cudaMemcpyAsync(perm.data(), m->perm, 4 * m->Tp, cudaMemcpyDeviceToHost, m->stream)) ||
        cuda_failed(cudaStreamSynchronize(m->stream)))
      return fail(SWE_ECUDA);
    for (int64_t j = 0; j < m->Tp; ++j)
      if (perm[j] >= 0) inv[perm[j]] = (int32_t)j;
    for (int j = 0; j < t->G; ++j) gi[j] = inv[gauge_cells[j]];
    if (cuda_failed(cudaMemcpyAsync(t->gcells, gi.data(), 4 * t->G, cudaMemcpyHostToDevice, m->stream)) ||
        cuda_failed(cudaStreamSynchronize(m->stream)))
      return fail(SWE_ECUDA);
  }
  const int64_t steps0 = s->host_ctl[0].steps;
  st = make_open_ended(s);  // end time +inf: every step takes its CFL dt
  if (st != SWE_OK) return fail(st);
  st = m->prm.precision == SWE_F64 ? record_t<double>(s, t) : record_t<float>(s, t);
  if (st != SWE_OK) return fail(st);
  st = read_ctl(s);
  if (st != SWE_OK) return fail(st);
  if (s->host_ctl[0].err) {
    const int e = s->host_ctl[0].err;
    free_tape(t);
    return (e & swe::kErrTimeout) ? SWE_ETIMEOUT : (e & swe::kErrNan) ? SWE_ENAN : SWE_EDRY;
  }
  if (s->host_ctl[0].steps - steps0 != t->N) return fail(SWE_ESTATE);
  t->dts.resize(t->N);
  if (cuda_failed(cudaMemcpyAsync(t->dts.data(), t->dts_dev, 8 * t->N, cudaMemcpyDeviceToHost, m->stream)) ||
      (gauge_h && t->G > 0 &&
       cuda_failed(cudaMemcpyAsync(gauge_h, t->gauge_dev, 8 * t->N * t->G, cudaMemcpyDeviceToHost, m->stream))) ||
      cuda_failed(cudaStreamSynchronize(m->stream)))
    return fail(SWE_ECUDA);
  *out = t;
  return SWE_OK;
}


// swe_grad and swe_grad_device: seeds and outputs in host memory, or
// (on_device) in device memory ordered on caller_stream.
swe_status grad(swe_tape* t, const double* g_h, const double* g_hu, const double* g_hv,
                const double* g_gauge, double* d_h0, double* d_hu0, double* d_hv0, double* d_z,
                double* d_n, bool on_device, void* caller_stream) {
  if (!t) return SWE_EINVAL;
  swe_mesh* m = t->mesh;
  cudaStream_t st = m->stream;
  const size_t sb = t->state_bytes();
  if (on_device && caller_stream && (cudaStream_t)caller_stream != st) {
    // the seeds were written, and the outputs may still be read, on the
    // caller's stream
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, (cudaStream_t)caller_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    CK(e);
  }
  const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemsetAsync(t->lam[0], 0, sb, st));
  CK(cudaMemsetAsync(t->lam[1], 0, sb, st));
  CK(cudaMemsetAsync(t->dgn2, 0, t->w * t->Tp, st));
  CK(cudaMemsetAsync(t->err, 0, sizeof(int), st));
  CK(cudaMemsetAsync(t->ticket, 0, sizeof(unsigned int), st));
  const double* seeds[3] = {g_h, g_hu, g_hv};
  for (int c = 0; c < 3; ++c) {
    if (!seeds[c]) continue;
    const double* from = seeds[c];
    if (!on_device) {
      CK(cudaMemcpyAsync(t->stage, seeds[c], 8 * t->T, cudaMemcpyHostToDevice, st));
      from = t->stage;
    }
    gather_any(m, from, t->lam[0] + c * t->w, 4);
  }
  const bool gseed = g_gauge && t->G > 0;
  if (gseed) CK(cudaMemcpyAsync(t->gseed_dev, g_gauge, 8 * t->N * t->G, in_kind, st));
  CK(cudaEventRecord(t->ev[0], st));
  int cur = 0;
  swe_status r = m->prm.precision == SWE_F64 ? grad_t<double>(t, gseed, &cur)
                                             : grad_t<float>(t, gseed, &cur);
  if (r != SWE_OK) return r;
  CK(cudaEventRecord(t->ev[1], st));
  double* outs[4] = {d_h0, d_hu0, d_hv0, d_z};
  for (int c = 0; c < 4; ++c) {
    if (!outs[c]) continue;
    if (on_device) {
      scatter_any(m, t->lam[cur] + c * t->w, outs[c], 4);
      continue;
    }
    scatter_any(m, t->lam[cur] + c * t->w, t->stage, 4);
    CK(cudaMemcpyAsync(outs[c], t->stage, 8 * t->T, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  if (d_n) {
    const int gs = grid_for(t->Tp, m->sms * 8);
    if (m->prm.precision == SWE_F64)
      k_finish_dn<double><<<gs, 256, 0, st>>>((const double*)t->dgn2, (const double*)t->gn2,
                                              m->prm.g, (double*)t->scratch, t->Tp);
    else
      k_finish_dn<float><<<gs, 256, 0, st>>>((const float*)t->dgn2, (const float*)t->gn2, m->prm.g,
                                             (float*)t->scratch, t->Tp);
    if (on_device) {
      scatter_any(m, t->scratch, d_n, 1);
    } else {
      scatter_any(m, t->scratch, t->stage, 1);
      CK(cudaMemcpyAsync(d_n, t->stage, 8 * t->T, cudaMemcpyDeviceToHost, st));
    }
  }
  int err = 0;
  CK(cudaMemcpyAsync(&err, t->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  CK(cudaEventElapsedTime(&t->grad_ms, t->ev[0], t->ev[1]));
  if (err & swe::kErrTimeout) return SWE_ETIMEOUT;
  if (err) return SWE_ESTATE;  // the replay did not reproduce the recorded steps
  return SWE_OK;
}

}  // namespace

extern "C" {

swe_status swe_grad_record(swe_state* s, int64_t n_steps, int64_t checkpoint_every,
                           const int32_t* gauge_cells, int32_t n_gauges, double* gauge_h,
                           swe_tape** out) {
  if (out) *out = nullptr;
  return swe::guarded(
      [&] { return grad_record(s, n_steps, checkpoint_every, gauge_cells, n_gauges, gauge_h, out); });
}

swe_status swe_grad(swe_tape* t, const double* g_h, const double* g_hu, const double* g_hv,
                    const double* g_gauge, double* d_h0, double* d_hu0, double* d_hv0, double* d_z,
                    double* d_n) {
  return grad(t, g_h, g_hu, g_hv, g_gauge, d_h0, d_hu0, d_hv0, d_z, d_n, false, nullptr);
}

swe_status swe_grad_device(swe_tape* t, const double* g_h, const double* g_hu, const double* g_hv,
                           const double* g_gauge, double* d_h0, double* d_hu0, double* d_hv0,
                           double* d_z, double* d_n, void* cuda_stream) {
  return grad(t, g_h, g_hu, g_hv, g_gauge, d_h0, d_hu0, d_hv0, d_z, d_n, true, cuda_stream);
}

swe_status swe_tape_gauges_device(const swe_tape* t, double* gauge_h, void* cuda_stream) {
  if (!t || (!gauge_h && t->G > 0)) return SWE_EINVAL;
  if (t->G == 0) return SWE_OK;
  cudaStream_t st = t->mesh->stream;
  if (cuda_stream && (cudaStream_t)cuda_stream != st) {
    cudaEvent_t ev = nullptr;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, (cudaStream_t)cuda_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
    CK(e);
  }
  CK(cudaMemcpyAsync(gauge_h, t->gauge_dev, 8 * t->N * t->G, cudaMemcpyDeviceToDevice, st));
  CK(cudaStreamSynchronize(st));
  return SWE_OK;
}

swe_status swe_tape_info(const swe_tape* t, double* info) {
  if (!t || !info) return SWE_EINVAL;
  info[0] = (double)t->N;
  info[1] = (double)t->K;
  info[2] = (double)t->record_ms;
  info[3] = (double)t->grad_ms;
  info[4] = (double)t->arena.size;
  return SWE_OK;
}

void swe_tape_destroy(swe_tape* t) {
  if (!t) return;
  free_tape(t);
}

}  // extern "C"
