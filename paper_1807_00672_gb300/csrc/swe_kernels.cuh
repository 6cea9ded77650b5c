// CUDA kernels of the shallow-water step (sm_103a), templated on the
// arithmetic type (double = FP64 path, float = FP32 path).
//
// The step follows Sec. 2.2 of Zaoui's paper: per-face HLLC fluxes with
// hydrostatic reconstruction of the bed (Eq. 3), per-cell face sums and the
// explicit Euler update (Eq. 4), semi-implicit Manning friction, and the CFL
// time step with Courant number 0.7 for the next step.
//
// Determinism: every face contribution is written to its own slot and each
// cell sums its three faces in a fixed order; the grid-wide CFL rate is an
// integer max on non-negative IEEE bit patterns; the FP64 mass integral is a
// per-block sum finished by the last block in block order. No float atomics.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace swe {

// Step control word in device memory. Written by the last block of each
// update kernel, read by every block of the next launch.
struct Ctl {
  double t;          // simulated time of the current state
  double t_end;      // end time (+inf for open-ended runs)
  double dt;         // dt of the next step (CFL, clamped to t_end - t)
  double dt_cfl;     // unclamped CFL dt of the current state
  double mass;       // sum of area * h of the current state (FP64)
  double dt_last;    // dt of the last step taken
  unsigned long long rate_bits;  // running max of the CFL rate (bits of a double >= 0)
  long long steps;   // steps taken
  long long neg;     // cells whose depth was clipped at zero
  int cur;           // buffer (0/1) holding the current state
  int done;          // no more steps: t reached t_end or an error latched
  int clamped;       // dt == t_end - t
  int err;           // latched error bits
  unsigned int ticket;  // blocks finished in the current launch
  int pad_;
};

constexpr int kErrNan = 1;
constexpr int kErrDry = 2;

struct Num {
  double g;
  double courant;
  double h_eps;
};

template <typename Real>
struct DevMesh {
  int64_t T;
  int64_t E;
  // cells (internal order)
  const Real* area;
  const Real* irP;  // perimeter / area
  // two-launch layout
  const int32_t* eL;
  const int32_t* eR;
  const Real* nx;
  const Real* ny;
  const Real* len;
  const int32_t* cf0;
  const int32_t* cf1;
  const int32_t* cf2;
  // tiled layout
  int64_t ntiles;
  const int64_t* toff;
  const int32_t* tA;
  const int32_t* tB;
  const Real* tnx;
  const Real* tny;
  const Real* tlen;
};

template <typename Real>
struct DevState {
  Real* h[2];
  Real* hu[2];
  Real* hv[2];
  const Real* z;
  const Real* gn2;  // g * n^2 per cell
  // scratch
  Real* fx[5];      // two-launch face outputs: c0, cA1, cA2, cB1, cB2
  double* partial;  // per-block mass partial sums
  Ctl* ctl;
};

constexpr int32_t kWallSide = INT32_MIN;

// ---------------------------------------------------------------------------
// Exact arithmetic helpers (never contracted into FMAs).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double cbrt_(double a) { return cbrt(a); }
__device__ __forceinline__ float cbrt_(float a) { return cbrtf(a); }

// Knuth's TwoSum: s + e == a + b exactly.
template <typename Real>
__device__ __forceinline__ void two_sum(Real a, Real b, Real& s, Real& e) {
  s = add_rn(a, b);
  Real bp = sub_rn(s, a);
  Real ap = sub_rn(s, bp);
  e = add_rn(sub_rn(a, ap), sub_rn(b, bp));
}

// ---------------------------------------------------------------------------
// HLLC flux in the face frame (Toro's shallow-water form). hA, hB are the
// reconstructed depths, 0 meaning dry. Returns mass, normal and tangential
// momentum fluxes.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void hllc(Real hA, Real unA, Real utA, Real hB, Real unB, Real utB,
                                     Real g, Real& F0, Real& F1, Real& F2) {
  const Real zero = Real(0), half = Real(0.5);
  if (hA == zero && hB == zero) {
    F0 = zero; F1 = zero; F2 = zero;
    return;
  }
  const Real cA = sqrt(g * hA);
  const Real cB = sqrt(g * hB);
  Real SA, SB;
  if (hA == zero) {
    SA = unB - Real(2) * cB;
    SB = unB + cB;
  } else if (hB == zero) {
    SA = unA - cA;
    SB = unA + Real(2) * cA;
  } else {
    const Real us = (unA + unB) * half + cA - cB;
    const Real cs = (cA + cB) * half + (unA - unB) * Real(0.25);
    SA = fmin(unA - cA, us - cs);
    SB = fmax(unB + cB, us + cs);
  }
  const Real qA = hA * unA;
  const Real qB = hB * unB;
  if (SA >= zero) {
    F0 = qA; F1 = qA * unA + half * g * hA * hA; F2 = qA * utA;
    return;
  }
  if (SB <= zero) {
    F0 = qB; F1 = qB * unB + half * g * hB * hB; F2 = qB * utB;
    return;
  }
  const Real FA1 = qA * unA + half * g * hA * hA;
  const Real FB1 = qB * unB + half * g * hB * hB;
  const Real inv = Real(1) / (SB - SA);
  F0 = (SB * qA - SA * qB + SA * SB * (hB - hA)) * inv;
  F1 = (SB * FA1 - SA * FB1 + SA * SB * (qB - qA)) * inv;
  // Contact speed S* = num / den with den < 0 whenever a side is wet, so
  // S* >= 0 exactly when num <= 0: no division needed for the upwind choice.
  const Real num = SA * hB * (unB - SB) - SB * hA * (unA - SA);
  F2 = F0 * (num <= zero ? utA : utB);
}

// One face: states of sides A (the edge's left cell) and B, unit normal n
// from A to B, length len. Produces the contribution to A's residual
// (c0, cA1, cA2) and the one subtracted from B's residual (c0, cB1, cB2):
// l (F + P_side n) with the hydrostatic-reconstruction bed pressure P_side.
template <typename Real>
__device__ __forceinline__ void face_flux(Real hA, Real huA, Real hvA, Real zA,
                                          Real hB, Real huB, Real hvB, Real zB, bool wall,
                                          Real nx, Real ny, Real len, const Num& num,
                                          Real& c0, Real& cA1, Real& cA2, Real& cB1, Real& cB2) {
  const Real zero = Real(0), half = Real(0.5);
  const Real g = Real(num.g);
  const double eps = num.h_eps;
  Real uA = zero, vA = zero;
  if ((double)hA > eps) { uA = huA / hA; vA = hvA / hA; }
  const Real unA = uA * nx + vA * ny;
  const Real utA = vA * nx - uA * ny;
  Real unB, utB;
  if (wall) {
    hB = hA; zB = zA; unB = -unA; utB = utA;
  } else {
    Real uB = zero, vB = zero;
    if ((double)hB > eps) { uB = huB / hB; vB = hvB / hB; }
    unB = uB * nx + vB * ny;
    utB = vB * nx - uB * ny;
  }
  // Hydrostatic reconstruction at the face.
  const Real zs = fmax(zA, zB);
  Real hAs = fmax(zero, hA + zA - zs);
  Real hBs = fmax(zero, hB + zB - zs);
  if ((double)hAs <= eps) hAs = zero;
  if ((double)hBs <= eps) hBs = zero;
  Real F0, F1, F2;
  hllc(hAs, unA, utA, hBs, unB, utB, g, F0, F1, F2);
  if (wall) { F0 = zero; F2 = zero; }
  const Real Fx = F1 * nx - F2 * ny;
  const Real Fy = F1 * ny + F2 * nx;
  const Real PA = half * g * (hA * hA - hAs * hAs);
  const Real PB = wall ? zero : half * g * (hB * hB - hBs * hBs);
  c0 = len * F0;
  cA1 = len * (Fx + PA * nx);
  cA2 = len * (Fy + PA * ny);
  cB1 = len * (Fx + PB * nx);
  cB2 = len * (Fy + PB * ny);
}

// Per-cell end of the step: residual -> Euler update (Eq. 4) -> friction ->
// next-step CFL rate. r*_hi/_lo: the residual as an unevaluated sum (lo = 0
// for the plain path). Writes the new state and accumulates mass/rate.
template <typename Real, bool Comp>
__device__ __forceinline__ void cell_finish(Real h, Real hu, Real hv, Real area, Real irP, Real gn2,
                                            Real dt, const Real rhi[3], const Real rlo[3],
                                            const Num& num, Real& h1, Real& hu1, Real& hv1,
                                            double& mass, double& rate, int& bad, int& neg) {
  const Real zero = Real(0);
  const Real a = dt / area;
  Real U[3] = {h, hu, hv};
  Real out[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (Comp) {
      // U - a (rhi + rlo) with the product error and the sum error carried.
      const Real p = mul_rn(a, rhi[c]);
      const Real pe = fma_rn(a, rhi[c], -p);
      Real s, e;
      two_sum(U[c], -p, s, e);
      out[c] = add_rn(s, sub_rn(sub_rn(e, pe), mul_rn(a, rlo[c])));
    } else {
      out[c] = U[c] - a * rhi[c];
    }
  }
  Real hs = out[0], qx = out[1], qy = out[2];
  if (hs < zero) { hs = zero; neg += 1; }
  const double eps = num.h_eps;
  if ((double)hs > eps) {
    const Real q = sqrt(qx * qx + qy * qy);
    const Real d = Real(1) + dt * gn2 * q / (hs * hs * cbrt_(hs));
    qx = qx / d;
    qy = qy / d;
    const Real lam = sqrt(qx * qx + qy * qy) / hs + sqrt(Real(num.g) * hs);
    rate = fmax(rate, (double)(lam * irP));
  } else {
    qx = zero;
    qy = zero;
  }
  if (!isfinite(hs) || !isfinite(qx) || !isfinite(qy)) bad = 1;
  h1 = hs; hu1 = qx; hv1 = qy;
  mass += (double)area * (double)hs;
}

// ---------------------------------------------------------------------------
// Block reductions and the last-block step finalisation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Every thread of the block calls this once at the end of an update launch.
// stepped: the launch advanced the state by ctl->dt (false: CFL/mass only).
template <int NT>
__device__ void finish_launch(Ctl* ctl, double* partial, double mass, double rate, int bad, int neg,
                              bool stepped, double courant) {
  __shared__ double s_mass[NT / 32];
  __shared__ double s_rate[NT / 32];
  __shared__ int s_bad[NT / 32];
  __shared__ int s_neg[NT / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  mass = warp_sum(mass);
  rate = warp_max(rate);
  const int wbad = __any_sync(0xffffffffu, bad);
  int wneg = neg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wneg += __shfl_xor_sync(0xffffffffu, wneg, o);
  if (lane == 0) { s_mass[wid] = mass; s_rate[wid] = rate; s_bad[wid] = wbad; s_neg[wid] = wneg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, r = 0.0;
    int b = 0, n = 0;
    for (int w = 0; w < NT / 32; ++w) { m += s_mass[w]; r = fmax(r, s_rate[w]); b |= s_bad[w]; n += s_neg[w]; }
    atomicMax(&ctl->rate_bits, (unsigned long long)__double_as_longlong(r));
    if (b) atomicOr(&ctl->err, kErrNan);
    if (n) atomicAdd((unsigned long long*)&ctl->neg, (unsigned long long)n);
    partial[blockIdx.x] = m;
    __threadfence();
    const unsigned int ticket = atomicAdd(&ctl->ticket, 1u);
    s_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // Last block: the mass integral over all blocks, in block order per thread.
  double s = 0.0;
  for (unsigned int j = threadIdx.x; j < gridDim.x; j += NT) s += __ldcg(&partial[j]);
  s = warp_sum(s);
  __syncthreads();
  if (lane == 0) s_mass[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < NT / 32; ++w) m += s_mass[w];
    const unsigned long long bits = atomicExch(&ctl->rate_bits, 0ull);
    ctl->ticket = 0u;
    double t = ctl->t;
    if (stepped) {
      ctl->dt_last = ctl->dt;
      t = ctl->clamped ? ctl->t_end : t + ctl->dt;
      ctl->t = t;
      ctl->steps += 1;
      ctl->cur ^= 1;
    }
    ctl->mass = m;
    int err = atomicOr(&ctl->err, 0);
    const double maxrate = __longlong_as_double((long long)bits);
    if (!(maxrate > 0.0)) err |= kErrDry;
    if (err) {
      atomicOr(&ctl->err, err);
      ctl->done = 1;
      ctl->dt = 0.0;
      ctl->dt_cfl = 0.0;
    } else {
      const double dt_cfl = courant / maxrate;
      const double rest = ctl->t_end - t;
      ctl->dt_cfl = dt_cfl;
      if (t >= ctl->t_end) ctl->done = 1;
      if (dt_cfl >= rest) { ctl->dt = rest; ctl->clamped = 1; }
      else { ctl->dt = dt_cfl; ctl->clamped = 0; }
    }
  }
}

// ---------------------------------------------------------------------------
// Two-launch step, launch 1: one thread per edge writes its face outputs.
// ---------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) k_edge_flux(DevMesh<Real> m, DevState<Real> s, Num num) {
  const Ctl* ctl = s.ctl;
  if (ctl->done) return;
  const int cur = ctl->cur;
  const Real* __restrict__ h = cur ? s.h[1] : s.h[0];
  const Real* __restrict__ hu = cur ? s.hu[1] : s.hu[0];
  const Real* __restrict__ hv = cur ? s.hv[1] : s.hv[0];
  const Real* __restrict__ z = s.z;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m.E;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t A = m.eL[e], B = m.eR[e];
    const bool wall = B < 0;
    const Real hA = h[A], huA = hu[A], hvA = hv[A], zA = z[A];
    Real hB = 0, huB = 0, hvB = 0, zB = 0;
    if (!wall) { hB = h[B]; huB = hu[B]; hvB = hv[B]; zB = z[B]; }
    Real c0, cA1, cA2, cB1, cB2;
    face_flux<Real>(hA, huA, hvA, zA, hB, huB, hvB, zB, wall, m.nx[e], m.ny[e], m.len[e], num,
                    c0, cA1, cA2, cB1, cB2);
    s.fx[0][e] = c0;
    s.fx[1][e] = cA1;
    s.fx[2][e] = cA2;
    s.fx[3][e] = cB1;
    s.fx[4][e] = cB2;
  }
}

// Two-launch step, launch 2: one thread per cell gathers its three faces.
template <typename Real, bool Comp>
__global__ void __launch_bounds__(256) k_cell_update(DevMesh<Real> m, DevState<Real> s, Num num) {
  Ctl* ctl = s.ctl;
  if (ctl->done) return;
  const int cur = ctl->cur;
  const Real dt = Real(ctl->dt);
  const Real* __restrict__ h = cur ? s.h[1] : s.h[0];
  const Real* __restrict__ hu = cur ? s.hu[1] : s.hu[0];
  const Real* __restrict__ hv = cur ? s.hv[1] : s.hv[0];
  Real* __restrict__ h1 = cur ? s.h[0] : s.h[1];
  Real* __restrict__ hu1 = cur ? s.hu[0] : s.hu[1];
  Real* __restrict__ hv1 = cur ? s.hv[0] : s.hv[1];
  double mass = 0.0, rate = 0.0;
  int bad = 0, neg = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m.T;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t f[3] = {m.cf0[i], m.cf1[i], m.cf2[i]};
    Real rhi[3] = {Real(0), Real(0), Real(0)}, rlo[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const bool right = f[k] < 0;
      const int32_t e = f[k] & 0x7fffffff;
      Real c[3];
      c[0] = s.fx[0][e];
      if (!right) { c[1] = s.fx[1][e]; c[2] = s.fx[2][e]; }
      else { c[0] = -c[0]; c[1] = -s.fx[3][e]; c[2] = -s.fx[4][e]; }
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (Comp) {
          Real sum, err;
          two_sum(rhi[q], c[q], sum, err);
          rhi[q] = sum;
          rlo[q] = add_rn(rlo[q], err);
        } else {
          rhi[q] = rhi[q] + c[q];
        }
      }
    }
    Real a1, b1, c1;
    cell_finish<Real, Comp>(h[i], hu[i], hv[i], m.area[i], m.irP[i], s.gn2[i], dt, rhi, rlo, num,
                            a1, b1, c1, mass, rate, bad, neg);
    h1[i] = a1;
    hu1[i] = b1;
    hv1[i] = c1;
  }
  finish_launch<256>(ctl, s.partial, mass, rate, bad, neg, true, num.courant);
}

// ---------------------------------------------------------------------------
// Tiled one-launch step. A persistent block walks tiles of NT consecutive
// cells: (1) stage the tile's states in shared memory, (2) compute every face
// record of the tile once (interior faces of the tile serve both of their
// cells; faces to other tiles are recomputed there), writing each
// contribution into its cell's face slot, (3) sum each cell's three slots in
// face order and update. Remote neighbour states come from global memory
// (L2 hits under the locality ordering).
// ---------------------------------------------------------------------------
template <typename Real, bool Comp, int NT>
__global__ void __launch_bounds__(NT) k_tiled_step(DevMesh<Real> m, DevState<Real> s, Num num) {
  __shared__ Real sh_h[NT], sh_hu[NT], sh_hv[NT], sh_z[NT];
  __shared__ Real sh_c[3][3 * NT];
  Ctl* ctl = s.ctl;
  if (ctl->done) return;
  const int cur = ctl->cur;
  const Real dt = Real(ctl->dt);
  const Real* __restrict__ h = cur ? s.h[1] : s.h[0];
  const Real* __restrict__ hu = cur ? s.hu[1] : s.hu[0];
  const Real* __restrict__ hv = cur ? s.hv[1] : s.hv[0];
  const Real* __restrict__ z = s.z;
  Real* __restrict__ h1 = cur ? s.h[0] : s.h[1];
  Real* __restrict__ hu1 = cur ? s.hu[0] : s.hu[1];
  Real* __restrict__ hv1 = cur ? s.hv[0] : s.hv[1];
  double mass = 0.0, rate = 0.0;
  int bad = 0, neg = 0;
  const int tid = threadIdx.x;
  for (int64_t tile = blockIdx.x; tile < m.ntiles; tile += gridDim.x) {
    const int64_t base = tile * NT;
    const int nc = (int)min((int64_t)NT, m.T - base);
    Real myh = 0, myhu = 0, myhv = 0;
    if (tid < nc) {
      myh = h[base + tid]; myhu = hu[base + tid]; myhv = hv[base + tid];
      sh_h[tid] = myh; sh_hu[tid] = myhu; sh_hv[tid] = myhv; sh_z[tid] = z[base + tid];
    }
    __syncthreads();
    const int64_t r0 = m.toff[tile], r1 = m.toff[tile + 1];
    for (int64_t r = r0 + tid; r < r1; r += NT) {
      const int32_t a = m.tA[r];
      if (a == kWallSide) continue;  // padding record
      const int32_t b = m.tB[r];
      Real hA, huA, hvA, zA, hB = 0, huB = 0, hvB = 0, zB = 0;
      if (a < 0) {
        const int j = (-1 - a) / 3;
        hA = sh_h[j]; huA = sh_hu[j]; hvA = sh_hv[j]; zA = sh_z[j];
      } else {
        hA = h[a]; huA = hu[a]; hvA = hv[a]; zA = z[a];
      }
      const bool wall = (b == kWallSide);
      if (!wall) {
        if (b < 0) {
          const int j = (-1 - b) / 3;
          hB = sh_h[j]; huB = sh_hu[j]; hvB = sh_hv[j]; zB = sh_z[j];
        } else {
          hB = h[b]; huB = hu[b]; hvB = hv[b]; zB = z[b];
        }
      }
      Real c0, cA1, cA2, cB1, cB2;
      face_flux<Real>(hA, huA, hvA, zA, hB, huB, hvB, zB, wall, m.tnx[r], m.tny[r], m.tlen[r], num,
                      c0, cA1, cA2, cB1, cB2);
      if (a < 0) {
        const int sl = -1 - a;
        sh_c[0][sl] = c0; sh_c[1][sl] = cA1; sh_c[2][sl] = cA2;
      }
      if (b < 0 && !wall) {
        const int sl = -1 - b;
        sh_c[0][sl] = -c0; sh_c[1][sl] = -cB1; sh_c[2][sl] = -cB2;
      }
    }
    __syncthreads();
    if (tid < nc) {
      Real rhi[3] = {Real(0), Real(0), Real(0)}, rlo[3] = {Real(0), Real(0), Real(0)};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const Real c = sh_c[q][3 * tid + k];
          if (Comp) {
            Real sum, err;
            two_sum(rhi[q], c, sum, err);
            rhi[q] = sum;
            rlo[q] = add_rn(rlo[q], err);
          } else {
            rhi[q] = rhi[q] + c;
          }
        }
      }
      const int64_t i = base + tid;
      Real a1, b1, c1;
      cell_finish<Real, Comp>(myh, myhu, myhv, m.area[i], m.irP[i], s.gn2[i], dt, rhi, rlo, num,
                              a1, b1, c1, mass, rate, bad, neg);
      h1[i] = a1;
      hu1[i] = b1;
      hv1[i] = c1;
    }
    __syncthreads();
  }
  finish_launch<NT>(ctl, s.partial, mass, rate, bad, neg, true, num.courant);
}

// CFL rate and mass of the current state, no step (initialisation).
template <typename Real>
__global__ void __launch_bounds__(256) k_cfl(DevMesh<Real> m, DevState<Real> s, Num num) {
  Ctl* ctl = s.ctl;
  const int cur = ctl->cur;
  const Real* __restrict__ h = cur ? s.h[1] : s.h[0];
  const Real* __restrict__ hu = cur ? s.hu[1] : s.hu[0];
  const Real* __restrict__ hv = cur ? s.hv[1] : s.hv[0];
  double mass = 0.0, rate = 0.0;
  int bad = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m.T;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Real hh = h[i], qx = hu[i], qy = hv[i];
    if ((double)hh > num.h_eps) {
      const Real lam = sqrt(qx * qx + qy * qy) / hh + sqrt(Real(num.g) * hh);
      rate = fmax(rate, (double)(lam * m.irP[i]));
    }
    if (!isfinite(hh) || !isfinite(qx) || !isfinite(qy)) bad = 1;
    mass += (double)m.area[i] * (double)hh;
  }
  finish_launch<256>(ctl, s.partial, mass, rate, bad, 0, false, num.courant);
}

// Caller order (double) -> internal order (Real): dst[j] = src[perm[j]].
template <typename Real>
__global__ void k_gather(const double* __restrict__ src, const int32_t* __restrict__ perm,
                         Real* __restrict__ dst, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    dst[j] = Real(src[perm[j]]);
}

// Internal order (Real) -> caller order (double): dst[perm[j]] = src[j].
template <typename Real>
__global__ void k_scatter(const Real* __restrict__ src, const int32_t* __restrict__ perm,
                          double* __restrict__ dst, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    dst[perm[j]] = double(src[j]);
}

}  // namespace swe
