// Device side of the domain decomposition (sub-domain meshes with ghost
// cells, see partition.cpp and swe_mesh_create_part): packing the owned
// cells another sub-domain holds as ghosts into a contiguous FP64 buffer,
// unpacking a received buffer into the ghost cells, and the global CFL time
// step as the minimum over the sub-domains' own (the step's reduction of
// Sec. 2.2 across sub-domains). The buffers are what a transport moves
// between sub-domains: NCCL send/recv or peer copies between GPUs, a
// device-to-device copy when several sub-domains share one GPU.
#include <algorithm>
#include <cmath>

#include "../../include/swe.h"
#include "swe_handles.cuh"
#include "swe_kernels.cuh"

using namespace swe_host;

namespace {

#define cuda_failed(call) swe_host::cuda_failed_at((call), #call, __FILE__, __LINE__)
#define CK(call)                              \
  do {                                        \
    if (cuda_failed(call)) return SWE_ECUDA;  \
  } while (0)

// buf[3 k + f] = field f (h, hu, hv) of caller cell cells[k], current buffer.
// Entries outside [0, T) are skipped.
template <typename Real>
__global__ void k_halo_pack(const swe::Ctl* ctl, swe::DevState<Real> s, const int32_t* iperm,
                            int64_t T, const int32_t* cells, int64_t n, double* buf) {
  const int cur = ctl->cur;
  const Real* h = cur ? s.h[1] : s.h[0];
  const Real* hu = cur ? s.hu[1] : s.hu[0];
  const Real* hv = cur ? s.hv[1] : s.hv[0];
  const int64_t sd = s.stride;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cells[k];
    if (c < 0 || c >= T) continue;
    const int64_t j = iperm[c];
    buf[3 * k] = (double)h[j * sd];
    buf[3 * k + 1] = (double)hu[j * sd];
    buf[3 * k + 2] = (double)hv[j * sd];
  }
}

// The reverse: field f of caller cell cells[k] = buf[3 k + f].
template <typename Real>
__global__ void k_halo_unpack(const swe::Ctl* ctl, swe::DevState<Real> s, const int32_t* iperm,
                              int64_t T, const int32_t* cells, int64_t n, const double* buf) {
  const int cur = ctl->cur;
  Real* h = cur ? s.h[1] : s.h[0];
  Real* hu = cur ? s.hu[1] : s.hu[0];
  Real* hv = cur ? s.hv[1] : s.hv[0];
  const int64_t sd = s.stride;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cells[k];
    if (c < 0 || c >= T) continue;
    const int64_t j = iperm[c];
    h[j * sd] = (Real)buf[3 * k];
    hu[j * sd] = (Real)buf[3 * k + 1];
    hv[j * sd] = (Real)buf[3 * k + 2];
  }
}

__global__ void k_dt_out(const swe::Ctl* ctl, double* dt) { *dt = ctl->dt_cfl; }

// The next step's time step: the smallest of n candidates (the sub-domains'
// CFL steps; min is exact, so every sub-domain gets the same value).
__global__ void k_dt_set_min(swe::Ctl* ctl, const double* dts, int n) {
  if (ctl->done) return;  // an error is latched: no further step
  double m = dts[0];
  for (int i = 1; i < n; ++i) m = fmin(m, dts[i]);
  if (!(m < INFINITY)) {  // no wet cell in any sub-domain
    atomicOr(&ctl->err, swe::kErrDry);
    ctl->done = 1;
    ctl->dt = 0.0;
    return;
  }
  ctl->dt = m;
  ctl->dt_cfl = m;
  ctl->clamped = 0;
}

swe_status halo_io(const swe_state* s, const int32_t* cells, int64_t n, double* buf, bool pack) {
  if (!s || n < 0 || (n > 0 && (!cells || !buf))) return SWE_EINVAL;
  const swe_mesh* m = s->mesh;
  if (!m->ghosts || !m->iperm) return SWE_ESTATE;
  if (n == 0) return SWE_OK;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)m->sms * 8);
  if (m->prm.precision == SWE_F64) {
    if (pack) k_halo_pack<double><<<grid, 256, 0, m->stream>>>(s->ctl, dev_state<double>(s), m->iperm, m->T, cells, n, buf);
    else k_halo_unpack<double><<<grid, 256, 0, m->stream>>>(s->ctl, dev_state<double>(s), m->iperm, m->T, cells, n, buf);
  } else {
    if (pack) k_halo_pack<float><<<grid, 256, 0, m->stream>>>(s->ctl, dev_state<float>(s), m->iperm, m->T, cells, n, buf);
    else k_halo_unpack<float><<<grid, 256, 0, m->stream>>>(s->ctl, dev_state<float>(s), m->iperm, m->T, cells, n, buf);
  }
  CK(cudaGetLastError());
  return SWE_OK;
}

}  // namespace

extern "C" {

swe_status swe_state_halo_pack(const swe_state* s, const int32_t* cells, int64_t n, double* buf) {
  return halo_io(s, cells, n, buf, true);
}

swe_status swe_state_halo_unpack(swe_state* s, const int32_t* cells, int64_t n, const double* buf) {
  return halo_io(s, cells, n, const_cast<double*>(buf), false);
}

swe_status swe_state_dt_device(const swe_state* s, double* dt) {
  if (!s || !dt) return SWE_EINVAL;
  if (nscen(s->mesh) != 1) return SWE_ESTATE;
  k_dt_out<<<1, 1, 0, s->mesh->stream>>>(s->ctl, dt);
  CK(cudaGetLastError());
  return SWE_OK;
}

swe_status swe_state_set_dt_min_device(swe_state* s, const double* dts, int32_t n) {
  if (!s || !dts || n < 1) return SWE_EINVAL;
  if (nscen(s->mesh) != 1) return SWE_ESTATE;
  swe_status st = make_open_ended(s);  // the step must not clamp to an end time
  if (st != SWE_OK) return st;
  k_dt_set_min<<<1, 1, 0, s->mesh->stream>>>(s->ctl, dts, n);
  CK(cudaGetLastError());
  return SWE_OK;
}

}  // extern "C"
