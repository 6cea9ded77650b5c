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
// integer max on non-negative IEEE bit patterns; the mass integral is a set
// of per-block sums added up in a fixed order (k_mass_sum). No float atomics.
//
// Precision. The FP64 path uses IEEE square roots, and reciprocals,
// quotients and h^{-1/3} by Newton-Raphson iteration to within a few ulps
// (rcp_nr, icbrt_nr). The FP32 path uses the hardware's approximate reciprocal and reciprocal
// square root and exp2/log2 for h^{-7/3}; its face sums and Euler update are
// compensated (TwoSum with exact FMA products); its dry-depth tests decide
// exactly as an FP64 comparison of the same value would (see Num::h_eps_f32);
// its mass integral uses exact FP32 products with compensated per-thread sums
// finished in FP64.
#pragma once

#include <cmath>
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
  long long part0;   // first mass partial sum of this scenario
  long long nparts;  // mass partial sums written by the last launch (one per block)
  unsigned long long rate_bits;  // running max of the CFL rate (bits of a double >= 0)
  long long steps;   // steps taken
  long long neg;     // cells whose depth was clipped at zero
  int cur;           // buffer (0/1) holding the current state
  int done;          // no more steps: t reached t_end or an error latched
  int clamped;       // dt == t_end - t
  int err;           // latched error bits
  unsigned int ticket;  // blocks of this scenario finished in the current launch
  unsigned int pool_next;  // next free entry of the step's tile pool (see Chunk)
  int subdomain;     // 1: a sub-domain of a decomposed mesh (its CFL step may be
                     // +inf when none of its own cells is wet; not an error here)
};
// A mesh holds one or more independent scenarios (an ensemble); each has its
// own control word, and a launch's blocks each work for one scenario.

constexpr int kErrNan = 1;
constexpr int kErrDry = 2;
constexpr int kErrTimeout = 4;

// Bounded device waits: a waiting thread sleeps in try_wait for up to
// kSuspendNs per round instead of spinning; after kWaitLimit rounds (about a
// second) the wait gives up and the kernel latches kErrTimeout.
constexpr uint32_t kSuspendNs = 20000;
constexpr uint32_t kWaitLimit = 50000;

struct Num {
  double g;
  double courant;
  double h_eps;
  // Largest float <= h_eps: for a float h, (double)h > h_eps exactly when
  // h > h_eps_f32 (no float lies in (h_eps_f32, h_eps]), so the FP32 path
  // takes every dry-depth decision as an FP64 comparison would.
  float h_eps_f32;
  // Rounds a step's bounded waits for its copies try before giving up
  // (kWaitLimit by default; 0 gives up at once). Waits that drain copies
  // already in flight before a block exits always use kWaitLimit.
  uint32_t wait_rounds;
};

// Numerics of a run; h_eps_f32 derived from h_eps on the host. wait: the
// wait_rounds setting of swe_params (0 default, -1 none, else rounds).
inline Num make_num(double g, double courant, double h_eps, int32_t wait = 0) {
  float f = (float)h_eps;
  if ((double)f > h_eps) f = std::nextafter(f, -INFINITY);
  const uint32_t rounds = wait == 0 ? kWaitLimit : (wait < 0 ? 0u : (uint32_t)wait);
  return Num{g, courant, h_eps, f, rounds};
}

// Work of one block of the tiled kernels: the ntiles tiles tile0 + k stride
// (k = 0, 1, ...) of scenario scen, whose cells end at cell_end. The chunks
// of one scenario interleave (stride = their count), so the blocks resident
// at any moment sweep neighbouring tiles together and a tile's halo cells
// are mostly still in L2 from the neighbours' copies. The same chunks walked
// backwards (tile0 the last tile, stride negative) serve every other step.
// The step's own tables add a pool: a block works its ntiles tiles, then
// takes further tiles one at a time from its scenario's pool, the
// pool_count tiles pool_first, pool_first + 1, ... (in the walk's direction,
// pool_first - 1, ... for a negative stride) in the order blocks ask for
// them (Ctl::pool_next), so that the blocks of an SM, which the warp
// scheduler does not serve equally, finish closer together. A pooled
// chunk keeps at least NS static tiles (those fetched before the
// dependency wait). part: the chunk's
// mass partial slot (the scenario's slots are contiguous from its
// control word's part0).
struct Chunk {
  int32_t scen, tile0, ntiles, stride;
  int32_t part, cell_end, pool_first, pool_count;
};

template <typename Real>
struct DevMesh {
  int64_t T;
  int64_t E;
  // cells (internal order; the tiled layout pads them to whole tiles)
  const Real* area;
  const Real* irP;  // perimeter / area
  const Real* rarea;  // 1 / area (FP64 tiled layout only, else null)
  // two-launch layout
  const int32_t* eL;
  const int32_t* eR;
  const Real* nx;
  const Real* ny;
  const Real* len;
  const int32_t* cf0;
  const int32_t* cf1;
  const int32_t* cf2;
  // tiled layout: block b of a launch works chunk chunks[b]
  const struct Chunk* chunks;
  int64_t ntiles;
  const int64_t* toff;
  const int64_t* hoff;
  const int32_t* hidx;
  // the same halo lists padded to halo_cap entries per tile (tile t's at
  // t * halo_cap; padding repeats the tile's first cell), when TileLayout's
  // hreg is set
  const int32_t* hpad;
  // face records: both sides packed as int16 codes (side A in the high half,
  // side B in the low half; see kSideWall), then the geometry arrays of
  // Geo<Real>
  const int32_t* tS;
  const Real* tg0;
  const Real* tg1;
  const Real* tg2;
  const int4* trec;  // FP32: interleaved records {packed sides, nx, ny, l}
};

// Cell state of one buffer b: h[b][i * stride], hu[b][i * stride],
// hv[b][i * stride]. stride 1: separate arrays (two-launch kernels);
// stride 4: interleaved cells (h, hu, hv, z), h[b] the cell array's base
// (tiled kernel), z also read from h[b] + 3.
template <typename Real>
struct DevState {
  Real* h[2];
  Real* hu[2];
  Real* hv[2];
  int stride;
  const Real* z;
  const Real* gn2;  // g * n^2 per cell
  // FP32 states with a depth residual (tiled kernel): per cell the part of
  // h its FP32 value does not hold (h + hlo is the depth); else null
  Real* hlo;
  // scratch
  Real* fx[5];      // two-launch face outputs: c0, cA1, cA2, cB1, cB2
  double* partial;  // per-block mass partial sums
  Ctl* ctl;
};

// Side codes of packed face records (int16): -1 - slot for a cell of the
// tile, TC + q (its place in the staged cells) for the cell at index q of
// the tile's halo list, kSideWall for a wall (and for side A of a padding
// record).
constexpr int kSideWall = -32768;

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

// Knuth's TwoSum: s + e == a + b exactly.
template <typename Real>
__device__ __forceinline__ void two_sum(Real a, Real b, Real& s, Real& e) {
  s = add_rn(a, b);
  Real bp = sub_rn(s, a);
  Real ap = sub_rn(s, bp);
  e = add_rn(sub_rn(a, ap), sub_rn(b, bp));
}

// Paired FP32 arithmetic (two IEEE round-to-nearest operations per
// instruction, sm_100 and later). x - y is formed as fma(y, -1, x): the
// product is exact, so the result is x - y rounded once.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// TwoSum on both lanes of a pair.
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = add2(a, b);
  const float2 bp = sub2(s, a);
  const float2 ap = sub2(s, bp);
  e = add2(sub2(a, ap), sub2(b, bp));
}

// ---------------------------------------------------------------------------
// Precision-specific operations.
// ---------------------------------------------------------------------------
template <typename Real>
struct Ops;

// FP64 reciprocal and inverse cube root by Newton-Raphson iteration (the
// textbook method: each step about squares the relative error), written
// with fused multiply-adds:
//   1/b:       y <- y + y (1 - b y), from the hardware approximation of the
//              leading bits (rcp.approx.ftz.f64, relative error about 2^-20);
//              two steps reach the last bit;
//   x^{-1/3}:  y <- y + (y / 3) (1 - x y^3), from an FP32 seed
//              2^{-log2(x) / 3} (ex2/lg2 approximations, about 2^-21); two
//              steps reach within a few ulps.
// Both are checked against IEEE division and cbrt by a GPU test. Square
// roots stay IEEE sqrt (cheaper on this hardware than any refinement tried).
__device__ __forceinline__ double rcp_approx64(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  return r;
}
__device__ __forceinline__ double rcp_nr(double b) {
  double y = rcp_approx64(b);
  double e = fma(-b, y, 1.0);
  y = fma(y, e, y);
  e = fma(-b, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float ex2_approx(float x);
__device__ __forceinline__ float lg2_approx(float x);
__device__ __forceinline__ double icbrt_nr(double x) {
  double y = (double)ex2_approx(-lg2_approx((float)x) * (1.0f / 3.0f));
  const double third = 1.0 / 3.0;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double y3 = y * y * y;
    y = fma(y * third, fma(-x, y3, 1.0), y);
  }
  return y;
}

template <>
struct Ops<double> {
  static __device__ __forceinline__ double div(double a, double b) { return a * rcp_nr(b); }
  static __device__ __forceinline__ double rcp(double b) { return rcp_nr(b); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ bool wet(double h, const Num& n) { return h > n.h_eps; }
  // dt g n^2 |q| / h^{7/3}, h^{-7/3} = y^7 with y = h^{-1/3}
  static __device__ __forceinline__ double friction(double dt, double gn2, double q, double h) {
    const double y = icbrt_nr(h);
    const double y2 = y * y;
    const double y7 = (y2 * y2) * (y2 * y);
    return dt * gn2 * q * y7;
  }
};

// FP32: single-instruction hardware approximations (reciprocal and square
// root about 1 ulp, exp2/log2 about 2 ulp), flushing subnormals to zero.
// Every divisor here is an area, a wet depth (> h_eps), a friction factor
// (>= 1) or a wave-speed span (>= one wave celerity); every square-root
// argument is a depth or a squared speed, where a subnormal value and zero
// give the same update.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float r;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

template <>
struct Ops<float> {
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp_approx(b); }
  static __device__ __forceinline__ float rcp(float b) { return rcp_approx(b); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrt_approx(x); }
  static __device__ __forceinline__ bool wet(float h, const Num& n) { return h > n.h_eps_f32; }
  static __device__ __forceinline__ float friction(float dt, float gn2, float q, float h) {
    // h^{-7/3} = 2^{-(7/3) log2 h}; only called for h > h_eps > 0
    return dt * gn2 * q * ex2_approx(-2.3333333333333335f * lg2_approx(h));
  }
};

// Face geometry of the tiled records: unit normal and length as computed on
// the host. FP64 keeps the side codes and the three values in separate
// arrays (tS, tg0, tg1, tg2); FP32 keeps each record as one 16-byte word
// {side codes, nx, ny, l} (trec), read with a single 128-bit load.
template <typename Real>
struct Geo;

template <>
struct Geo<double> {
  static constexpr int kArrays = 3;
  static __device__ __forceinline__ void get(const double* g0, const double* g1, const double* g2,
                                             int r, double& nx, double& ny, double& len) {
    nx = g0[r];
    ny = g1[r];
    len = g2[r];
  }
};

// Bytes of one staged face record and its geometry (all arrays together).
template <typename Real>
__host__ __device__ constexpr uint32_t rec_bytes() { return sizeof(Real) == 4 ? 16u : 4u + 3u * 8u; }

// FP32 record r of an interleaved record array: side codes and geometry.
__device__ __forceinline__ void rec_f32(const void* base, int r, int32_t& packed, float& nx,
                                        float& ny, float& len) {
  const int4 v = reinterpret_cast<const int4*>(base)[r];
  packed = v.x;
  nx = __int_as_float(v.y);
  ny = __int_as_float(v.z);
  len = __int_as_float(v.w);
}

// Mass integral accumulator: plain FP64, or for FP32 exact products and a
// compensated running sum, converted to FP64 at the end.
template <typename Real>
struct MassAcc;

template <>
struct MassAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double h) { s += a * h; }
  __device__ __forceinline__ double value() const { return s; }
};

template <>
struct MassAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a, float h) {
    const float p = __fmul_rn(a, h);
    const float pe = __fmaf_rn(a, h, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Stand-in accumulator for launches that do not integrate the mass (the
// tiled step: the mass is integrated on demand by k_cfl_tiled).
template <typename Real>
struct NoMass {
  __device__ __forceinline__ void add(Real, Real) {}
  __device__ __forceinline__ double value() const { return 0.0; }
};

// Four consecutive values (one interleaved cell or one face slot).
template <typename Real>
struct V4 {
  Real x, y, z, w;
};
__device__ __forceinline__ V4<float> ld4(const float* p) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float* p, float x, float y, float z, float w) {
  *reinterpret_cast<float4*>(p) = make_float4(x, y, z, w);
}
__device__ __forceinline__ void st4(double* p, double x, double y, double z, double w) {
  reinterpret_cast<double2*>(p)[0] = make_double2(x, y);
  reinterpret_cast<double2*>(p)[1] = make_double2(z, w);
}

// ---------------------------------------------------------------------------
// HLLC flux in the face frame (Toro's shallow-water form). hA, hB are the
// reconstructed depths, 0 meaning dry. Returns mass, normal and tangential
// momentum fluxes.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void hllc(Real hA, Real unA, Real utA, Real hB, Real unB, Real utB,
                                     Real g, Real& F0, Real& F1, Real& F2) {
  // Straight-line form (no divergent branches). The HLL formula is evaluated
  // with the clamped speeds S- = min(SA, 0) and S+ = max(SB, 0): it then
  // equals the upwind flux F_A when SA >= 0 and F_B when SB <= 0, the cases
  // of the case analysis, so mass and normal momentum need no case selection.
  using O = Ops<Real>;
  const Real zero = Real(0), half = Real(0.5);
  const bool wetA = hA > zero, wetB = hB > zero;
  const Real ghA = g * hA, ghB = g * hB;
  const Real cA = O::sqrt_(ghA);
  const Real cB = O::sqrt_(ghB);
  // wave speeds: two-rarefaction estimates when both sides are wet, Toro's
  // dry-bed speeds when one side is dry
  const Real us = (unA + unB) * half + cA - cB;
  const Real cs = (cA + cB) * half + (unA - unB) * Real(0.25);
  const Real SA = wetA ? (wetB ? fmin(unA - cA, us - cs) : unA - cA) : unB - Real(2) * cB;
  const Real SB = wetA ? (wetB ? fmax(unB + cB, us + cs) : unA + Real(2) * cA) : unB + cB;
  const Real Sm = fmin(SA, zero), Sp = fmax(SB, zero);
  const Real qA = hA * unA, qB = hB * unB;
  const Real FA1 = qA * unA + half * ghA * hA;
  const Real FB1 = qB * unB + half * ghB * hB;
  const Real inv = O::div(Real(1), Sp - Sm);
  const Real SS = Sm * Sp;
  const Real H0 = (Sp * qA - Sm * qB + SS * (hB - hA)) * inv;
  const Real H1 = (Sp * FA1 - Sm * FB1 + SS * (qB - qA)) * inv;
  // Transverse momentum from the upwind side of the contact: S* = num / den
  // with den < 0 whenever a side is wet, so S* >= 0 exactly when num <= 0
  // (no division); the supersonic cases take their own side.
  const Real num = SA * hB * (unB - SB) - SB * hA * (unA - SA);
  const Real ut = SA >= zero ? utA : (SB <= zero ? utB : (num <= zero ? utA : utB));
  const bool dry = !wetA && !wetB;
  F0 = dry ? zero : H0;
  F1 = dry ? zero : H1;
  F2 = dry ? zero : H0 * ut;
}

// Velocity of a cell: (hu, hv) / h when wet, else 0.
template <typename Real>
__device__ __forceinline__ void velocity(Real h, Real hu, Real hv, const Num& num, Real& u, Real& v) {
  const bool w = Ops<Real>::wet(h, num);
  if constexpr (sizeof(Real) == 8) {
    const double r = w ? rcp_nr(h) : 0.0;  // one reciprocal for both components
    u = hu * r;
    v = hv * r;
  } else {
    const float r = rcp_approx(h);
    u = w ? hu * r : 0.0f;
    v = w ? hv * r : 0.0f;
  }
}

// One face: depth, velocity and bed of sides A (the edge's left cell) and B,
// unit normal n from A to B, length len. Produces the contribution to A's
// residual (c0, cA1, cA2) and the one subtracted from B's residual
// (c0, cB1, cB2): l (F + P_side n) with the hydrostatic-reconstruction bed
// pressure P_side.
template <typename Real>
__device__ __forceinline__ void face_flux(Real hA, Real uA, Real vA, Real zA,
                                          Real hB, Real uB, Real vB, Real zB, bool wall,
                                          Real nx, Real ny, Real len, const Num& num,
                                          Real& c0, Real& cA1, Real& cA2, Real& cB1, Real& cB2) {
  const Real zero = Real(0), half = Real(0.5);
  const Real g = Real(num.g);
  const Real unA = uA * nx + vA * ny;
  const Real utA = vA * nx - uA * ny;
  Real unB, utB;
  if (wall) {
    hB = hA; zB = zA; unB = -unA; utB = utA;
  } else {
    unB = uB * nx + vB * ny;
    utB = vB * nx - uB * ny;
  }
  // Hydrostatic reconstruction at the face.
  const Real zs = fmax(zA, zB);
  Real hAs = fmax(zero, hA + zA - zs);
  Real hBs = fmax(zero, hB + zB - zs);
  if (!Ops<Real>::wet(hAs, num)) hAs = zero;
  if (!Ops<Real>::wet(hBs, num)) hBs = zero;
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

// FP32 face of the tiled kernel: velocity + face_flux<float> + hllc in
// fewer instructions, the same flux up to rounding:
//  - a dry cell's reciprocal depth is 0, so its velocity comes out 0;
//  - a reconstructed depth is x if x > h_eps, else 0 (max(0, x) and the dry
//    test in one);
//  - the transverse momentum is upwinded by the sign of the HLL mass flux
//    F0: S* = F_hll / h_hll with h_hll > 0, so in the subsonic case F0 >= 0
//    exactly when S* >= 0; when S_A >= 0, F0 = q_A >= 0 (side A, as S* >= 0),
//    when S_B <= 0, F0 = q_B <= 0 (side B); where F0 = 0 the choice does not
//    matter (F2 = F0 ut);
//  - with both sides dry every numerator is 0; the wave-speed span is
//    clamped away from 0, so the flux is 0 without a selection (and the
//    dry-bed wave speeds come from the same formula, see below);
//  - the contributions use the scaled normal (gx, gy) = l n:
//    l (F_n n + F_t t + P n) = (F_n + P) (gx, gy) + F_t (-gy, gx).
// A, B: interleaved cells (h, hu, hv, z); Wall: B is ignored (mirror of A).
template <bool Wall>
__device__ __forceinline__ void face_flux_f32(const V4<float>& A, const V4<float>& B, float nx,
                                              float ny, float len, const Num& num, float& c0,
                                              float& cA1, float& cA2, float& cB1, float& cB2) {
  const float g = (float)num.g, eps = num.h_eps_f32;
  const float gx = len * nx, gy = len * ny;
  const float rA = A.x > eps ? rcp_approx(A.x) : 0.0f;
  const float uA = A.y * rA, vA = A.z * rA;
  const float unA = uA * nx + vA * ny;
  const float utA = vA * nx - uA * ny;
  float hB, zB, unB, utB;
  if (Wall) {
    hB = A.x; zB = A.w; unB = -unA; utB = utA;
  } else {
    const float rB = B.x > eps ? rcp_approx(B.x) : 0.0f;
    const float uB = B.y * rB, vB = B.z * rB;
    hB = B.x; zB = B.w;
    unB = uB * nx + vB * ny;
    utB = vB * nx - uB * ny;
  }
  // hydrostatic reconstruction
  const float zs = fmaxf(A.w, zB);
  const float xA = A.x + A.w - zs, xB = hB + zB - zs;
  const bool wA = xA > eps, wB = xB > eps;  // wet sides: h* > 0 exactly when x > h_eps >= 0
  const float hAs = wA ? xA : 0.0f;
  const float hBs = wB ? xB : 0.0f;
  // HLLC wave speeds (see hllc). A dry side takes the normal velocity
  // un_B - 2 c_B (A dry) or un_A + 2 c_A (B dry): the two-rarefaction
  // estimates then reduce exactly to Toro's dry-bed speeds (c* = 0,
  // u* = that velocity), so no case selection is needed; a dry side's
  // discharge stays 0 (h* = 0).
  const float hg = 0.5f * g;
  const float ghA = g * hAs, ghB = g * hBs;
  const float cA = sqrt_approx(ghA), cB = sqrt_approx(ghB);
  const float vnA = wA ? unA : unB - 2.0f * cB;
  const float vnB = wB ? unB : unA + 2.0f * cA;
  const float us = (vnA + vnB) * 0.5f + cA - cB;
  const float cs = (cA + cB) * 0.5f + (vnA - vnB) * 0.25f;
  const float Sm = fminf(fminf(vnA - cA, us - cs), 0.0f);
  const float Sp = fmaxf(fmaxf(vnB + cB, us + cs), 0.0f);
  // HLL fluxes with the clamped speeds; e = g/2 h*^2 serves both the
  // hydrostatic flux term and the bed pressure g/2 (h^2 - h*^2)
  const float qA = hAs * unA, qB = hBs * unB;
  const float eA = hg * hAs * hAs, eB = hg * hBs * hBs;
  const float FA1 = qA * unA + eA;
  const float FB1 = qB * unB + eB;
  const float inv = rcp_approx(fmaxf(Sp - Sm, 1e-30f));
  const float SS = Sm * Sp;
  float F0 = (Sp * qA - Sm * qB + SS * (hBs - hAs)) * inv;
  const float F1 = (Sp * FA1 - Sm * FB1 + SS * (qB - qA)) * inv;
  float F2 = F0 * (F0 >= 0.0f ? utA : utB);
  if (Wall) { F0 = 0.0f; F2 = 0.0f; }
  const float t1 = F2 * gy, t2 = F2 * gx;
  c0 = len * F0;
  const float FA = F1 + (hg * A.x * A.x - eA);
  cA1 = FA * gx - t1;
  cA2 = FA * gy + t2;
  if (!Wall) {
    // side B's contributions negated (its residual subtracts them)
    const float FB = F1 + (hg * hB * hB - eB);
    cB1 = t1 - FB * gx;
    cB2 = -t2 - FB * gy;
  } else {
    cB1 = 0.0f;
    cB2 = 0.0f;
  }
}

// FP64 face of the tiled kernel: the straight-line form of face_flux_f32
// (clamped-speed HLL, dry-bed speeds by substitution, transverse momentum
// upwinded by the sign of F0, contributions from (gx, gy) = l n; the same
// flux as face_flux up to rounding) on cells whose velocities were formed
// once per cell: A, B are (h, u, v, z), u = v = 0 on a dry cell. Wall: B is
// ignored (mirror of A).
template <bool Wall>
__device__ __forceinline__ void face_flux_f64(const V4<double>& A, const V4<double>& B, double nx,
                                              double ny, double len, const Num& num, double& c0,
                                              double& cA1, double& cA2, double& cB1, double& cB2) {
  const double g = num.g, eps = num.h_eps;
  const double gx = len * nx, gy = len * ny;
  const double unA = A.y * nx + A.z * ny;
  const double utA = A.z * nx - A.y * ny;
  double hB, zB, unB, utB;
  if (Wall) {
    hB = A.x; zB = A.w; unB = -unA; utB = utA;
  } else {
    hB = B.x; zB = B.w;
    unB = B.y * nx + B.z * ny;
    utB = B.z * nx - B.y * ny;
  }
  // hydrostatic reconstruction. Comparisons against non-negative constants
  // and sign tests are made on the IEEE bit patterns (as 64-bit integers they
  // order non-negative doubles as their values, and every negative value,
  // -0 included, below them), which keeps them off the FP64 pipe.
  const double zs = fmax(A.w, zB);
  const double xA = A.x + A.w - zs, xB = hB + zB - zs;
  const long long beps = __double_as_longlong(eps);
  const bool wA = __double_as_longlong(xA) > beps, wB = __double_as_longlong(xB) > beps;
  const double hAs = wA ? xA : 0.0;  // x > h_eps, else dry
  const double hBs = wB ? xB : 0.0;
  // HLLC wave speeds, a dry side entering with un_B - 2 c_B (A dry) or
  // un_A + 2 c_A (B dry)
  const double hg = 0.5 * g;
  const double cA = sqrt(g * hAs), cB = sqrt(g * hBs);
  const double vnA = wA ? unA : unB - 2.0 * cB;
  const double vnB = wB ? unB : unA + 2.0 * cA;
  const double us = (vnA + vnB) * 0.5 + cA - cB;
  const double cs = (cA + cB) * 0.5 + (vnA - vnB) * 0.25;
  const double m1 = fmin(vnA - cA, us - cs), p1 = fmax(vnB + cB, us + cs);
  const double Sm = __double_as_longlong(m1) < 0 ? m1 : 0.0;  // min(m1, 0)
  const double Sp = __double_as_longlong(p1) > 0 ? p1 : 0.0;  // max(p1, 0)
  // HLL fluxes with the clamped speeds; e = g/2 h*^2 serves the flux and
  // the bed pressure g/2 (h^2 - h*^2)
  const double qA = hAs * unA, qB = hBs * unB;
  const double eA = hg * hAs * hAs, eB = hg * hBs * hBs;
  const double FA1 = qA * unA + eA;
  const double FB1 = qB * unB + eB;
  const double span = Sp - Sm;  // >= 0
  const double inv = rcp_nr(__double_as_longlong(span) > __double_as_longlong(1e-300) ? span : 1e-300);
  const double SS = Sm * Sp;
  double F0 = (Sp * qA - Sm * qB + SS * (hBs - hAs)) * inv;
  const double F1 = (Sp * FA1 - Sm * FB1 + SS * (qB - qA)) * inv;
  double F2 = F0 * (__double_as_longlong(F0) >= 0 ? utA : utB);  // side A where F0 >= +0
  if (Wall) { F0 = 0.0; F2 = 0.0; }
  const double t1 = F2 * gy, t2 = F2 * gx;
  c0 = len * F0;
  const double FA = F1 + (hg * A.x * A.x - eA);
  cA1 = FA * gx - t1;
  cA2 = FA * gy + t2;
  if (!Wall) {
    const double FB = F1 + (hg * hB * hB - eB);
    cB1 = FB * gx - t1;
    cB2 = FB * gy + t2;
  } else {
    cB1 = 0.0;
    cB2 = 0.0;
  }
}

// Per-cell end of the step: residual -> Euler update (Eq. 4) -> friction ->
// next-step CFL rate. R: the residual (for Comp, the compensated face sum
// rounded once, and U - a R is then one FMA). Writes the new state and
// accumulates mass/rate. Recip: `area` holds 1 / area (a = dt / area is then
// one product; no mass is accumulated). CH (FP32 with Comp): *lo is the
// depth's residual, h + *lo the depth; the update h + *lo - a R[0] is
// carried exactly up to the final rounding (the product's error from an
// FMA, the sum's from TwoSum), and *lo receives what that rounding left, so
// updates below half an ulp of h accumulate instead of being lost.
template <typename Real, bool Comp, typename Acc, bool Recip = false, bool CH = false>
__device__ __forceinline__ void cell_finish(Real h, Real hu, Real hv, Real area, Real irP, Real gn2,
                                            Real dt, const Real R[3], const Num& num, Real& h1,
                                            Real& hu1, Real& hv1, Acc& mass, Real& rate, Real& chk,
                                            int& neg, Real* lo = nullptr) {
  using O = Ops<Real>;
  const Real zero = Real(0);
  const Real a = Recip ? dt * area : O::div(dt, area);
  Real out[3];
  if constexpr (Comp && sizeof(Real) == 4) {
    if constexpr (CH) {
      const float t = mul_rn(-a, R[0]);
      const float e1 = fma_rn(-a, R[0], -t);  // -a R[0] = t + e1 exactly
      float s0, e2;
      two_sum(h, t, s0, e2);                   // h + t = s0 + e2 exactly
      const float r = add_rn(*lo, add_rn(e1, e2));
      two_sum(s0, r, out[0], *lo);             // new depth and residual
    } else {
      out[0] = fma_rn(-a, R[0], h);
    }
    const float2 o = fma2(make_float2(-a, -a), make_float2(R[1], R[2]), make_float2(hu, hv));
    out[1] = o.x;
    out[2] = o.y;
  } else {
    const Real U[3] = {h, hu, hv};
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = Comp ? fma_rn(-a, R[c], U[c]) : U[c] - a * R[c];
  }
  Real hs = out[0], qx = out[1], qy = out[2];
  if (hs < zero) {
    hs = zero;
    neg += 1;
    if constexpr (CH) *lo = zero;
  }
  if (O::wet(hs, num)) {
    const Real q = O::sqrt_(qx * qx + qy * qy);
    const Real d = Real(1) + O::friction(dt, gn2, q, hs);
    const Real rd = O::div(Real(1), d);
    if constexpr (sizeof(Real) == 4) {
      const float2 qq = mul2(make_float2(qx, qy), make_float2(rd, rd));
      qx = qq.x;
      qy = qq.y;
    } else {
      qx = qx * rd;
      qy = qy * rd;
    }
    const Real qn = q * rd;  // |q| after friction
    const Real lam = O::div(qn, hs) + O::sqrt_(Real(num.g) * hs);
    rate = fmax(rate, lam * irP);
  } else {
    qx = zero;
    qy = zero;
  }
  // chk stays 0 unless a value is NaN or infinite (0 x that = NaN)
  chk = fma_rn(hs + qx + qy, Real(0), chk);
  h1 = hs; hu1 = qx; hv1 = qy;
  if constexpr (!Recip) mass.add(area, hs);
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

// What a launch that ends with finish_launch did.
enum LaunchKind { kStepped = 0, kCflOnly = 1, kMassOnly = 2 };

// Every thread of the block calls this once at the end of an update launch.
// The block is one of `nblocks` working for the scenario of `ctl`; its mass
// partial sum goes to partial[part], the scenario's partials being
// partial[part0 .. part0 + nblocks). kind: kStepped, the launch advanced the
// state by ctl->dt; kCflOnly, the CFL step of the current state is set
// (initialisation); kMassOnly, only the mass partials are refreshed and the
// step control (time, time step, stop flag) stays as it is. err: kErr* bits
// seen by this thread.
template <int NT>
__device__ void finish_launch(Ctl* ctl, double* partial, long long part, long long part0,
                              int nblocks, double mass, double rate, int err_bits, int neg,
                              int kind, double courant) {
  const bool stepped = kind == kStepped;
  __shared__ double s_mass[NT / 32];
  __shared__ double s_rate[NT / 32];
  __shared__ int s_bad[NT / 32];
  __shared__ int s_neg[NT / 32];
  __shared__ int s_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  mass = warp_sum(mass);
  rate = warp_max(rate);
  int wbad = err_bits, wneg = neg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    wneg += __shfl_xor_sync(0xffffffffu, wneg, o);
    wbad |= __shfl_xor_sync(0xffffffffu, wbad, o);
  }
  if (lane == 0) { s_mass[wid] = mass; s_rate[wid] = rate; s_bad[wid] = wbad; s_neg[wid] = wneg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0, r = 0.0;
    int b = 0, n = 0;
    for (int w = 0; w < NT / 32; ++w) { m += s_mass[w]; r = fmax(r, s_rate[w]); b |= s_bad[w]; n += s_neg[w]; }
    atomicMax(&ctl->rate_bits, (unsigned long long)__double_as_longlong(r));
    if (b) atomicOr(&ctl->err, b);
    if (n) atomicAdd((unsigned long long*)&ctl->neg, (unsigned long long)n);
    partial[part] = m;
    __threadfence();
    const unsigned int ticket = atomicAdd(&ctl->ticket, 1u);
    s_last = (ticket == (unsigned int)nblocks - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // Last block: the step's control update. The mass partial sums stay in
  // `partial` and are added up by k_mass_sum when the host asks for them.
  if (threadIdx.x == 0) {
    ctl->part0 = part0;
    ctl->nparts = nblocks;
    const unsigned long long bits = atomicExch(&ctl->rate_bits, 0ull);
    ctl->ticket = 0u;
    ctl->pool_next = 0u;  // every block has taken its last tile
    if (kind == kMassOnly) return;  // errors this launch saw are latched above
    double t = ctl->t;
    if (stepped) {
      ctl->dt_last = ctl->dt;
      t = ctl->clamped ? ctl->t_end : t + ctl->dt;
      ctl->t = t;
      ctl->steps += 1;
      ctl->cur ^= 1;
    }
    int err = atomicOr(&ctl->err, 0);
    const double maxrate = __longlong_as_double((long long)bits);
    // blocks that gave up add no rate; a sub-domain with no wet cell of its
    // own gets dt_cfl = +inf (the global minimum decides)
    if (!(maxrate > 0.0) && !(err & kErrTimeout) && !ctl->subdomain) err |= kErrDry;
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
    const Real hA = h[A], zA = z[A];
    Real uA, vA;
    velocity(hA, hu[A], hv[A], num, uA, vA);
    Real hB = 0, uB = 0, vB = 0, zB = 0;
    if (!wall) {
      hB = h[B];
      zB = z[B];
      velocity(hB, hu[B], hv[B], num, uB, vB);
    }
    Real c0, cA1, cA2, cB1, cB2;
    face_flux<Real>(hA, uA, vA, zA, hB, uB, vB, zB, wall, m.nx[e], m.ny[e], m.len[e], num,
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
  MassAcc<Real> mass;
  Real rate = Real(0), chk = Real(0);
  int neg = 0;
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
    Real R[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) R[q] = Comp ? add_rn(rhi[q], rlo[q]) : rhi[q];
    Real a1, b1, c1;
    cell_finish<Real, Comp>(h[i], hu[i], hv[i], m.area[i], m.irP[i], s.gn2[i], dt, R, num, a1, b1,
                            c1, mass, rate, chk, neg);
    h1[i] = a1;
    hu1[i] = b1;
    hv1[i] = c1;
  }
  finish_launch<256>(ctl, s.partial, blockIdx.x, 0, gridDim.x, mass.value(), (double)rate,
                     chk != Real(0) ? kErrNan : 0, neg, kStepped, num.courant);
}

// ---------------------------------------------------------------------------
// TMA bulk copies, cp.async gathers and mbarriers (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Expect `bytes` more on the current phase without arriving.
__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// Programmatic dependent launch: let the next kernel in the stream start
// (its blocks run until their own pdl_wait), and wait until the previous
// kernel has completed with its memory visible.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1D bulk copy global -> shared; src, dst 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity: at most `rounds` rounds
// of try_wait; false if the phase never came.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t rounds = kWaitLimit) {
  for (uint32_t i = 0; i < rounds; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// One value global -> shared, asynchronously (completed by cp_async_wait_all).
__device__ __forceinline__ void cp_async(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// 16 bytes global -> shared (both 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Shared-memory plan of k_tiled_step, sized on the host from the mesh's
// largest per-tile record and halo counts. Each of the NS stages holds one
// tile: its interleaved cells (h, hu, hv, z), the tile's tc cells followed by
// its halo cells; its packed face records and their geometry arrays; its halo
// index list (unless hreg). After the stages: the face slots per face of each tile cell,
// face-major, and the NS mbarriers. A slot is (c0, c1, c2, -) in FP64 and
// (c0, -, c1, c2) in FP32, where the momentum pair sits in the aligned half
// that the paired FP32 instructions read. Every offset is a multiple of 16
// bytes.
struct TileLayout {
  uint32_t ext, rec_cap, halo_cap;
  uint32_t off_cells, off_tS, off_g0, off_g1, off_g2, off_hidx;
  uint32_t stage;
  uint32_t off_slots, off_bars, total;
  uint32_t hreg;   // 1: halo lists read from DevMesh::hpad into registers, not staged
  uint32_t early;  // 1 (with hreg): launch the Early kernel (halo_schedule 1)
  uint32_t slot_bytes;  // one set of face slots
  uint32_t pipe;   // 1 (with hreg, FP32, 2 stages, two slot sets): launch
                   // k_tiled_step_pipe (halo_schedule 2)
};

// nt: threads per block. When no tile has more halo cells than the block has
// threads, each thread prefetches at most one halo index into a register and
// the stages hold no halo list.
// Face slots: face k of tile cell j sits at k (TC + kSlotPad) + j (in slot
// units), which puts one cell's three slots in different shared-memory bank
// groups. Measured 0.7 % faster than k TC + j on a 10M-cell mesh, with the
// same shared-memory bank-conflict count. slot_pad maps a side code's slot
// k TC + j to its place.
constexpr int kSlotPad = 3;
template <int TC>
__device__ __forceinline__ int slot_pad(int s) { return s + (s / TC) * kSlotPad; }

inline TileLayout make_tile_layout(uint32_t w, uint32_t geo_arrays, uint32_t tc, uint32_t ns,
                                   uint32_t rec_cap, uint32_t halo_cap, uint32_t nt,
                                   uint32_t slot_sets = 1) {
  auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  TileLayout L{};
  L.rec_cap = rec_cap;
  L.halo_cap = halo_cap;
  L.hreg = halo_cap <= nt ? 1u : 0u;
  L.ext = tc + halo_cap;
  uint32_t o = 0;
  L.off_cells = o; o += a16(L.ext * 4 * w);
  if (w == 4) {  // FP32: interleaved 16-byte records
    L.off_tS = o; o += a16(rec_cap * 16);
    L.off_g0 = L.off_g1 = L.off_g2 = o;
  } else {
    L.off_tS = o; o += a16(rec_cap * 4);
    L.off_g0 = o; o += a16(rec_cap * w);
    L.off_g1 = o; o += a16(rec_cap * w);
    L.off_g2 = o; o += geo_arrays > 2 ? a16(rec_cap * w) : 0u;
  }
  L.off_hidx = o; o += L.hreg ? 0u : a16(halo_cap * 4);
  L.stage = o;
  o = ns * L.stage;
  L.slot_bytes = a16(3 * (tc + kSlotPad) * 4 * w);
  L.off_slots = o; o += slot_sets * L.slot_bytes;
  L.off_bars = o; o += a16(ns * 8);
  L.total = o;
  return L;
}

// ---------------------------------------------------------------------------
// Tiled one-launch step on interleaved cells (h, hu, hv, z). A block of NT
// threads walks the tiles of its work chunk (TC = NT * CPT consecutive cells
// each; see Chunk), then, in the Pool variant, tiles of its scenario's pool,
// through NS shared-memory stages:
//   - thread 0 queues bulk async copies (TMA) of tile k+NS-1's cell arrays
//     and face records (and its halo list, unless the layout's hreg has each
//     thread load its halo index into a register) while the block works on
//     tile k;
//   - once tile k+1's copies have landed (mid-iteration k; with Early, at the
//     start of iteration k, which needs only the register indices), every
//     thread gathers its halo cells (16 bytes each) with cp.async;
//   (1) every face record of the tile once, velocities formed per side:
//       interior faces of the tile fill
//       both of their cells' slots, faces shared with another tile fill only
//       this tile's slot (that tile computes the same face from the same
//       inputs), walls mirror; slots are face-major (face k of tile cell j at
//       k (TC + kSlotPad) + j);
//   (2) each cell sums its three face slots in face order and is updated.
// Two block barriers per tile. Cell arrays are padded to whole tiles so every
// copy moves TC values.
// ---------------------------------------------------------------------------
// Resident blocks per SM the tiled kernel is compiled for (register budget):
// 768 threads per SM for FP32 (shared memory allows 6 blocks of 128 threads
// anyway; up to 85 registers), 512 for FP64.
template <typename Real, int NT>
constexpr int tiled_min_blocks() { return (sizeof(Real) == 4 ? 768 : 512) / NT; }

// NT threads per block, tiles of TC cells (a power of two, NT <= TC); a
// thread updates the tile cells tid, tid + NT, ... (CPT = ceil(TC / NT)).
// Early: a tile's halo gather is issued at the start of the previous tile's
// iteration (launched only on layouts with hreg). CH: FP32 with a depth
// residual per cell (s.hlo, read and written by the cell's own thread).
// Pool: the chunk table has tile pools (see Chunk); without it a block works
// its static tiles only and no tile bookkeeping goes through shared memory.
template <typename Real, bool Comp, int NT, int NS, int TC, bool Early = false, bool CH = false,
          bool Pool = false>
__global__ void __launch_bounds__(NT, tiled_min_blocks<Real, NT>())
    k_tiled_step(DevMesh<Real> m, DevState<Real> s, Num num, TileLayout L) {
  constexpr int CPT = (TC + NT - 1) / NT;
  static_assert((TC & (TC - 1)) == 0 && NT <= TC && NT % 32 == 0, "tile shape");
  __shared__ int s_nrec[NS], s_nh[NS];  // record and halo counts of each stage's tile
  __shared__ int s_tile[8];  // tile of iteration j in slot j & 7 (-1: none), written by thread 0
  extern __shared__ __align__(128) unsigned char smem[];
  Real* slots = reinterpret_cast<Real*>(smem + L.off_slots);  // [3 (TC + kSlotPad)][4]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.off_bars);

  // This block's work: tiles t_first + k t_step (k < n_tiles) of one scenario,
  // then tiles from the scenario's pool (see Chunk).
  const Chunk ch = m.chunks[blockIdx.x];
  const int t_first = ch.tile0, n_tiles = ch.ntiles, t_step = ch.stride;
  const int pool_first = ch.pool_first, pool_count = ch.pool_count;
  const int cell_end = ch.cell_end;
  Ctl* ctl = s.ctl + ch.scen;
  const int tid = threadIdx.x;
  // Thread 0 takes pool entries in iteration order, only after pdl_wait (the
  // previous step's last block resets the pool): entries for iterations
  // 0..3 in one atomic before the first tile, then the entry of iteration
  // k + 4 with an atomic issued at the start of iteration k whose result is
  // first used at its end, so that its latency is hidden. Once the pool is
  // empty every later iteration gets -1.
  bool exhausted = !Pool || pool_count <= 0;
  unsigned int q_next = 0u;
  auto pool_tile = [&](unsigned int q) -> int {
    return t_step > 0 ? pool_first + (int)q : pool_first - (int)q;
  };
  // Thread 0: the tile of iteration j >= 4 at the end of iteration j - 4
  // (its pool entry, if any, taken with the atomic issued at its start).
  auto publish = [&](int j) {
    int t = -1;
    if (j < n_tiles) {
      t = t_first + j * t_step;
    } else if (!exhausted && q_next < (unsigned int)pool_count) {
      t = pool_tile(q_next);
    } else {
      exhausted = true;
    }
    s_tile[j & 7] = t;
  };
  // The state and the control word are read only after pdl_wait (they are
  // the previous step's output); mesh data may be fetched before it.
  const Real* __restrict__ U = nullptr;  // interleaved cells (h, hu, hv, z)
  Real* __restrict__ U1 = nullptr;
  Real dt = Real(0);

  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // Thread 0 tracks, per stage, the parity of the next phase to wait for and
  // whether a copy is in flight (bit st of each mask).
  uint32_t parity_bits = 0, pending = 0;
  // Thread 0: record and halo offsets of the next tile to queue, loaded one
  // iteration before they are used so that their latency stays hidden.
  int64_t o_r0 = 0, o_r1 = 0, o_h0 = 0, o_h1 = 0;
  const bool hreg = L.hreg != 0;
  constexpr bool early = Early;
  auto load_offsets = [&](int t) {
    o_r0 = m.toff[t];
    o_r1 = m.toff[t + 1];
    if (!hreg) {
      o_h0 = m.hoff[t];
      o_h1 = m.hoff[t + 1];
    }
  };
  // Thread 0: queue the bulk copies of tile t's mesh data (offsets already
  // loaded) into stage st: face records and halo list. The stage's phase
  // completes once issue_cells has arrived as well.
  auto issue_mesh = [&](int st) {
    unsigned char* p = smem + st * L.stage;
    const int64_t r0 = o_r0, h0 = o_h0;
    const uint32_t nrec = (uint32_t)(o_r1 - r0);
    const uint32_t nh = (uint32_t)(o_h1 - h0);
    s_nrec[st] = (int)nrec;
    s_nh[st] = (int)nh;
    const uint32_t rb = nrec * (uint32_t)sizeof(Real);
    fence_proxy_async();
    mbar_expect_tx_only(&bar[st], nrec * rec_bytes<Real>() + nh * 4);
    if constexpr (sizeof(Real) == 4) {
      bulk_g2s(p + L.off_tS, m.trec + r0, nrec * 16, &bar[st]);
    } else {
      bulk_g2s(p + L.off_tS, m.tS + r0, nrec * 4, &bar[st]);
      bulk_g2s(p + L.off_g0, m.tg0 + r0, rb, &bar[st]);
      bulk_g2s(p + L.off_g1, m.tg1 + r0, rb, &bar[st]);
      bulk_g2s(p + L.off_g2, m.tg2 + r0, rb, &bar[st]);
    }
    if (nh > 0) bulk_g2s(p + L.off_hidx, m.hidx + h0, nh * 4, &bar[st]);  // never with hreg
    pending |= 1u << st;
  };
  // Thread 0: queue tile t's state cells into stage st (arrives on its phase).
  auto issue_cells = [&](int st, int t) {
    unsigned char* p = smem + st * L.stage;
    const uint32_t cells = TC * 4 * (uint32_t)sizeof(Real);
    mbar_expect_tx(&bar[st], cells);
    bulk_g2s(p + L.off_cells, U + 4 * (int64_t)t * TC, cells, &bar[st]);
  };
  auto issue = [&](int st, int t) {
    issue_mesh(st);
    issue_cells(st, t);
  };
  // Thread 0: wait for stage st's copies.
  auto wait_stage = [&](int st) -> bool {
    const bool ok = mbar_wait(&bar[st], (parity_bits >> st) & 1u, num.wait_rounds);
    if (ok) {
      parity_bits ^= 1u << st;
      pending &= ~(1u << st);
    }
    return ok;
  };
  // All threads: gather the halo cells of stage st's tile (after its copies
  // landed), one interleaved cell per cp.async group. Lane l of warp w takes
  // entries l W + w (W warps), so every warp gathers about nh / W cells.
  // With hreg the thread's one entry q_h was prefetched into h_q by
  // load_halo, and all halo_cap entries are gathered (the padding ones copy
  // the tile's first cell into slots no record names).
  constexpr int W = NT / 32;
  const int q_h = (tid & 31) * W + (tid >> 5);
  int32_t h_q = 0;
  auto load_halo = [&](int t) {
    if (q_h < (int)L.halo_cap) h_q = __ldg(m.hpad + (int64_t)t * L.halo_cap + q_h);
  };
  auto gather_halo = [&](int st) {
    unsigned char* p = smem + st * L.stage;
    Real* xc = reinterpret_cast<Real*>(p + L.off_cells) + 4 * TC;
    auto copy_cell = [&](int q, int32_t i) {
      const Real* src = U + 4 * (int64_t)i;
#pragma unroll
      for (int b = 0; b < (int)sizeof(Real) / 4; ++b)
        cp_async16(xc + 4 * q + b * (16 / sizeof(Real)), src + b * (16 / sizeof(Real)));
    };
    if (hreg) {
      if (q_h < (int)L.halo_cap) copy_cell(q_h, h_q);
      return;
    }
    const int32_t* hl = reinterpret_cast<const int32_t*>(p + L.off_hidx);
    const int nh = s_nh[st];
    for (int q = q_h; q < nh; q += NT) copy_cell(q, hl[q]);
  };

  // FP64: the staged cells (h, hu, hv, z) become (h, u, v, z) in place once
  // they have landed, u = hu / h on a wet cell (one reciprocal for both
  // components) and 0 on a dry one, so that the face loop divides nothing
  // (the same values the faces would form, once per cell instead of once
  // per face side). Each thread converts its own cells of the tile, keeping
  // their (hu, hv) in registers for the update, and the halo cells it
  // gathered itself.
  constexpr bool kVel = sizeof(Real) == 8;
  Real own_q[CPT][2], next_q[CPT][2];
  auto to_velocity = [&](Real* c, Real& hu, Real& hv) {
    const V4<Real> x = ld4(c);
    Real u, v;
    velocity(x.x, x.y, x.z, num, u, v);
    hu = x.y;
    hv = x.z;
    st4(c, x.x, u, v, x.w);
  };
  auto own_velocities = [&](int st, Real (&q)[CPT][2]) {
    Real* xc = reinterpret_cast<Real*>(smem + st * L.stage + L.off_cells);
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int j = tid + cc * NT;
      if (TC % NT != 0 && j >= TC) break;
      to_velocity(xc + 4 * j, q[cc][0], q[cc][1]);
    }
  };
  auto halo_velocities = [&](int st) {
    Real* xc = reinterpret_cast<Real*>(smem + st * L.stage + L.off_cells) + 4 * TC;
    Real a, b;
    if (hreg) {
      if (q_h < (int)L.halo_cap) to_velocity(xc + 4 * q_h, a, b);
      return;
    }
    const int nh = s_nh[st];
    for (int q = q_h; q < nh; q += NT) to_velocity(xc + 4 * q, a, b);
  };

  NoMass<Real> mass;  // integrated on demand (k_cfl_tiled), not every step
  Real rate = Real(0);
  Real chk = Real(0);  // non-zero once a new value is NaN or infinite
  int neg = 0, timeout = 0;
  // Mesh data of the first tiles, then wait for the previous step.
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NS - 1; ++i)
      if (i < n_tiles) {
        load_offsets(t_first + i * t_step);
        issue_mesh(i);
      }
  }
  if (hreg && n_tiles > 0) load_halo(t_first);
  pdl_trigger();
  pdl_wait();
  if (ctl->done) {
    // no step: let the mesh copies already queued land before exiting
    if (tid == 0) {
#pragma unroll
      for (int i = 0; i < NS - 1; ++i)
        if (i < n_tiles) {
          asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar[i])) : "memory");
          mbar_wait(&bar[i], 0u);
        }
    }
    return;
  }
  {
    const int cur = ctl->cur;
    dt = Real(ctl->dt);
    U = cur ? s.h[1] : s.h[0];
    U1 = cur ? s.h[0] : s.h[1];
  }
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NS - 1; ++i)
      if (i < n_tiles) issue_cells(i, t_first + i * t_step);
    if constexpr (Pool) {
      // the tiles of iterations 0..3: static ones, then pool entries taken
      // with one atomic
      const int ndyn = n_tiles >= 4 ? 0 : 4 - n_tiles;
      const unsigned int q0 =
          (!exhausted && ndyn > 0) ? atomicAdd(&ctl->pool_next, (unsigned int)ndyn) : 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int t = -1;
        if (j < n_tiles) {
          t = t_first + j * t_step;
        } else if (!exhausted && q0 + (unsigned int)(j - n_tiles) < (unsigned int)pool_count) {
          t = pool_tile(q0 + (unsigned int)(j - n_tiles));
        } else {
          exhausted = true;
        }
        s_tile[j] = t;
      }
    }
    if (NS - 1 < n_tiles) load_offsets(t_first + (NS - 1) * t_step);
  }
  if (n_tiles > 0) {
    if (early) {
      // the gather needs only the indices in registers, not the stage
      gather_halo(0);
      if (n_tiles > 1) load_halo(t_first + t_step);
    }
    const bool ok = (tid == 0) ? wait_stage(0) : true;
    if (__syncthreads_or(!ok)) {
      timeout = 1;
      cp_async_wait_all();  // the early gather of tile 0 may be in flight
    } else {
      if (!early) gather_halo(0);
      cp_async_wait_all();
      if constexpr (kVel) {
        own_velocities(0, own_q);
        halo_velocities(0);
      }
      __syncthreads();
    }
  }
  // Each iteration: the face records of tile k, then the cell updates of
  // tile k while tile k+1's halo gather is in flight (with `early`, issued
  // before the face records). Two block barriers.
  // Pool: every thread keeps the tiles of iterations k, k + 1 and k + 2
  // (from the ring, published at least one barrier earlier). Otherwise the
  // tiles follow from k.
  int tile_c = 0, tile_n = -1, tile_n2 = -1;
  if constexpr (Pool) {
    tile_c = s_tile[0];
    tile_n = s_tile[1];
    tile_n2 = s_tile[2];
  }
  for (int k = 0; !timeout && (Pool || k < n_tiles); ++k) {
    const int tile = Pool ? tile_c : t_first + k * t_step;
    if (Pool && tile < 0) break;
    const int st = k % NS;
    const bool has_next = Pool ? tile_n >= 0 : k + 1 < n_tiles;
    // the pool entry of iteration k + 4 (published at the end of this one)
    if (Pool && tid == 0 && !exhausted && k + 4 >= n_tiles) q_next = atomicAdd(&ctl->pool_next, 1u);
    // The stage that receives tile k+NS-1 was released by the barrier that
    // ended iteration k-1.
    if constexpr (Pool) {
      if (tid == 0) {
        const int t_issue = NS == 2 ? tile_n : tile_n2;
        const int t_offs = NS == 2 ? tile_n2 : s_tile[(k + 3) & 7];
        if (t_issue >= 0) {
          issue((k + NS - 1) % NS, t_issue);
          if (t_offs >= 0) load_offsets(t_offs);
        }
      }
    } else if (tid == 0 && k + NS - 1 < n_tiles) {
      issue((k + NS - 1) % NS, tile + (NS - 1) * t_step);
      if (k + NS < n_tiles) load_offsets(tile + NS * t_step);
    }
    if (early) {
      // Tile k+1's gather starts now, from indices loaded an iteration ago:
      // its destination, the halo part of the stage the previous iteration
      // released, is not written by the stage's bulk copies. Then the
      // indices of tile k+2.
      if (has_next) {
        gather_halo((k + 1) % NS);
        if (Pool ? tile_n2 >= 0 : k + 2 < n_tiles) load_halo(Pool ? tile_n2 : tile + 2 * t_step);
      }
    } else if (hreg && has_next) {
      load_halo(Pool ? tile_n : tile + t_step);  // used by tile k+1's gather after the face loop
    }
    const unsigned char* p = smem + st * L.stage;
    const Real* xc = reinterpret_cast<const Real*>(p + L.off_cells);  // [ext][4]
    const int32_t* rS = reinterpret_cast<const int32_t*>(p + L.off_tS);
    const Real* rg0 = reinterpret_cast<const Real*>(p + L.off_g0);
    const Real* rg1 = reinterpret_cast<const Real*>(p + L.off_g1);
    const Real* rg2 = reinterpret_cast<const Real*>(p + L.off_g2);
    const int base = tile * TC;
    const int nc = min(TC, cell_end - base);
    const int nrec = s_nrec[st];
    // this thread's cells' area, perimeter/area and g n^2 (cell arrays are
    // padded to whole tiles, so the loads are always in bounds)
    Real c_area[CPT], c_irP[CPT], c_gn2[CPT], c_lo[CPT];
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int j = tid + cc * NT;
      if (TC % NT != 0 && j >= TC) break;
      c_area[cc] = kVel ? m.rarea[base + j] : m.area[base + j];  // FP64: 1 / area
      c_irP[cc] = m.irP[base + j];
      c_gn2[cc] = s.gn2[base + j];
      if constexpr (CH) c_lo[cc] = s.hlo[base + j];
    }

    // face records, the highest threads first: a partial last round falls
    // on the last warps, away from warp 0, which also queues the copies
    for (int r = NT - 1 - tid; r < nrec; r += NT) {
      int32_t packed;
      float fnx = 0.0f, fny = 0.0f, flen = 0.0f;
      if constexpr (sizeof(Real) == 4) rec_f32(rS, r, packed, fnx, fny, flen);
      else packed = rS[r];
      const int a = packed >> 16;                       // side A code
      const int b = (int)(int16_t)(packed & 0xffff);   // side B code
      if constexpr (sizeof(Real) == 4) {
        float c0, cA1, cA2, cB1, cB2;
        if (b == kSideWall) {
          if (a == kSideWall) continue;  // padding record
          const V4<Real> A = ld4(xc + 4 * ((-1 - a) & (TC - 1)));
          face_flux_f32<true>(A, A, fnx, fny, flen, num, c0, cA1, cA2, cB1, cB2);
          st4(slots + 4 * slot_pad<TC>(-1 - a), c0, 0.0f, cA1, cA2);
          continue;
        }
        const int ia = a < 0 ? ((-1 - a) & (TC - 1)) : a;
        const int ib = b < 0 ? ((-1 - b) & (TC - 1)) : b;
        const V4<Real> A = ld4(xc + 4 * ia);
        const V4<Real> B = ld4(xc + 4 * ib);
        face_flux_f32<false>(A, B, fnx, fny, flen, num, c0, cA1, cA2, cB1, cB2);
        if (a < 0) st4(slots + 4 * slot_pad<TC>(-1 - a), c0, 0.0f, cA1, cA2);
        if (b < 0) st4(slots + 4 * slot_pad<TC>(-1 - b), -c0, 0.0f, cB1, cB2);
      } else {
        Real nx, ny, len;
        Geo<Real>::get(rg0, rg1, rg2, r, nx, ny, len);
        Real c0, cA1, cA2, cB1, cB2;
        if (b == kSideWall) {
          // Wall (side A is the tile cell owning the edge) or padding record;
          // these are the last records of a tile.
          if (a == kSideWall) continue;
          const V4<Real> A = ld4(xc + 4 * ((-1 - a) & (TC - 1)));  // (h, u, v, z)
          face_flux_f64<true>(A, A, nx, ny, len, num, c0, cA1, cA2, cB1, cB2);
          st4(slots + 4 * slot_pad<TC>(-1 - a), c0, cA1, cA2, Real(0));
          continue;
        }
        const int ia = a < 0 ? ((-1 - a) & (TC - 1)) : a;
        const int ib = b < 0 ? ((-1 - b) & (TC - 1)) : b;
        const V4<Real> A = ld4(xc + 4 * ia);  // (h, u, v, z)
        const V4<Real> B = ld4(xc + 4 * ib);
        face_flux_f64<false>(A, B, nx, ny, len, num, c0, cA1, cA2, cB1, cB2);
        if (a < 0) st4(slots + 4 * slot_pad<TC>(-1 - a), c0, cA1, cA2, Real(0));
        if (b < 0) st4(slots + 4 * slot_pad<TC>(-1 - b), -c0, -cB1, -cB2, Real(0));
      }
    }
    // The next tile's copies must have landed before its halo is gathered
    // (with `early` they are waited for at the end of the iteration).
    const bool ok = (!early && tid == 0 && has_next) ? wait_stage((k + 1) % NS) : true;
    if (__syncthreads_or(!ok)) {
      timeout = 1;
      break;
    }
    if (!early && has_next) gather_halo((k + 1) % NS);
    if constexpr (kVel) {
      if (has_next) own_velocities((k + 1) % NS, next_q);
    }

    // cell updates of tile k
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int j = tid + cc * NT;
      if (j >= nc) break;
      // the three face contributions (faces k = 0, 1, 2) of each field
      const V4<Real> f0 = ld4(slots + 4 * j);
      const V4<Real> f1 = ld4(slots + 4 * (TC + kSlotPad + j));
      const V4<Real> f2 = ld4(slots + 4 * (2 * (TC + kSlotPad) + j));
      Real R[3];
      if constexpr (Comp && sizeof(Real) == 4) {
        // (f0 + f1) + f2 with both TwoSum errors added back, rounded once;
        // h alone, (hu, hv) as a pair
        Real s1, e1, s2, e2;
        two_sum(f0.x, f1.x, s1, e1);
        two_sum(s1, f2.x, s2, e2);
        R[0] = add_rn(s2, add_rn(e1, e2));
        float2 p1, q1, p2, q2;
        two_sum2(make_float2(f0.z, f0.w), make_float2(f1.z, f1.w), p1, q1);
        two_sum2(p1, make_float2(f2.z, f2.w), p2, q2);
        const float2 r = add2(p2, add2(q1, q2));
        R[1] = r.x;
        R[2] = r.y;
      } else {
        constexpr bool kPad = sizeof(Real) == 4;
        const Real a0[3] = {f0.x, kPad ? f0.z : f0.y, kPad ? f0.w : f0.z};
        const Real a1[3] = {f1.x, kPad ? f1.z : f1.y, kPad ? f1.w : f1.z};
        const Real a2[3] = {f2.x, kPad ? f2.z : f2.y, kPad ? f2.w : f2.z};
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          if (Comp) {
            Real s1, e1, s2, e2;
            two_sum(a0[q], a1[q], s1, e1);
            two_sum(s1, a2[q], s2, e2);
            R[q] = add_rn(s2, add_rn(e1, e2));
          } else {
            R[q] = a0[q] + a1[q] + a2[q];
          }
        }
      }
      const V4<Real> c = ld4(xc + 4 * j);
      // FP64: the staged cell holds (h, u, v, z); its (hu, hv) are in registers
      const Real qx = kVel ? own_q[cc][0] : c.y, qy = kVel ? own_q[cc][1] : c.z;
      Real a1, b1, c1;
      cell_finish<Real, Comp, NoMass<Real>, kVel, CH>(c.x, qx, qy, c_area[cc], c_irP[cc],
                                                      c_gn2[cc], dt, R, num, a1, b1, c1, mass,
                                                      rate, chk, neg, &c_lo[cc]);
      st4(U1 + 4 * (int64_t)(base + j), a1, b1, c1, c.w);
      if constexpr (CH) s.hlo[base + j] = c_lo[cc];
    }
    if constexpr (kVel) {
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) {
        own_q[cc][0] = next_q[cc][0];
        own_q[cc][1] = next_q[cc][1];
      }
    }
    // Slot (k + 4) & 7 held iteration k - 4's tile, which nobody reads now.
    if (Pool && tid == 0) publish(k + 4);
    if (early) {
      const bool ok_end = (tid == 0 && has_next) ? wait_stage((k + 1) % NS) : true;
      cp_async_wait_all();
      if (__syncthreads_or(!ok_end)) {
        timeout = 1;
        break;
      }
    } else {
      cp_async_wait_all();
      if constexpr (kVel) {
        if (has_next) halo_velocities((k + 1) % NS);
      }
      __syncthreads();
    }
    if constexpr (Pool) {
      tile_c = tile_n;
      tile_n = tile_n2;
      tile_n2 = s_tile[(k + 3) & 7];
    }
  }
  // After a timed-out wait, let every copy still in flight land before the
  // block's shared memory is released (bounded as well).
  if (timeout && tid == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if ((pending >> i) & 1u) mbar_wait(&bar[i], (parity_bits >> i) & 1u);
  }
  finish_launch<NT>(ctl, s.partial, ch.part, ctl->part0, (int)ctl->nparts, mass.value(),
                    (double)rate, (chk != Real(0) ? kErrNan : 0) | (timeout ? kErrTimeout : 0), neg,
                    kStepped, num.courant);
}

// ---------------------------------------------------------------------------
// FP32 tiled step with one block barrier per tile (halo_schedule 2). The
// same tiles, records, halo prefetch and arithmetic as k_tiled_step (the
// same bits), software-pipelined across tiles: iteration k updates the
// cells of tile k-1 and then computes the face records of tile k, with two
// sets of face slots (tile k-1's are read while tile k's are written). The
// tile's own cells (h, hu, hv, z) and its area, perimeter/area and g n^2
// are taken into registers in the iteration of its faces, so its stage is
// free again when tile k+1's copies are queued at the start of iteration k.
// Needs the layout's hreg (halo indices in registers) and two slot sets;
// 2 stages.
// ---------------------------------------------------------------------------
// Resident blocks per SM the pipelined kernel is compiled for: 1,024
// threads per SM with one cell per thread (4 blocks of 256 fit its shared
// memory at 256-cell tiles; up to 64 registers), else as k_tiled_step.
template <int NT, int TC>
constexpr int pipe_min_blocks() { return (TC == NT ? 1024 : 768) / NT; }

template <int NT, int TC>
__global__ void __launch_bounds__(NT, pipe_min_blocks<NT, TC>())
    k_tiled_step_pipe(DevMesh<float> m, DevState<float> s, Num num, TileLayout L) {
  using Real = float;
  constexpr int NS = 2;
  constexpr int CPT = TC / NT;
  static_assert((TC & (TC - 1)) == 0 && NT <= TC && NT % 32 == 0 && TC % NT == 0, "tile shape");
  __shared__ int s_nrec[NS];
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.off_bars);
  auto slot_set = [&](int k) {  // [3 (TC + kSlotPad)][4], as k_tiled_step's
    return reinterpret_cast<Real*>(smem + L.off_slots + (k & 1) * L.slot_bytes);
  };

  const Chunk ch = m.chunks[blockIdx.x];
  const int t_first = ch.tile0, n_tiles = ch.ntiles, t_step = ch.stride;
  const int cell_end = ch.cell_end;
  Ctl* ctl = s.ctl + ch.scen;
  const int tid = threadIdx.x;
  const Real* __restrict__ U = nullptr;
  Real* __restrict__ U1 = nullptr;
  Real dt = Real(0);

  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t parity_bits = 0, pending = 0;  // thread 0: per stage
  int64_t o_r0 = 0, o_r1 = 0;             // thread 0: next tile's record offsets
  auto load_offsets = [&](int t) {
    o_r0 = m.toff[t];
    o_r1 = m.toff[t + 1];
  };
  auto issue_mesh = [&](int st) {
    unsigned char* p = smem + st * L.stage;
    const int64_t r0 = o_r0;
    const uint32_t nrec = (uint32_t)(o_r1 - r0);
    s_nrec[st] = (int)nrec;
    fence_proxy_async();
    mbar_expect_tx_only(&bar[st], nrec * 16u);
    bulk_g2s(p + L.off_tS, m.trec + r0, nrec * 16, &bar[st]);
    pending |= 1u << st;
  };
  auto issue_cells = [&](int st, int t) {
    unsigned char* p = smem + st * L.stage;
    const uint32_t cells = TC * 4 * (uint32_t)sizeof(Real);
    mbar_expect_tx(&bar[st], cells);
    bulk_g2s(p + L.off_cells, U + 4 * (int64_t)t * TC, cells, &bar[st]);
  };
  auto wait_stage = [&](int st) -> bool {
    const bool ok = mbar_wait(&bar[st], (parity_bits >> st) & 1u, num.wait_rounds);
    if (ok) {
      parity_bits ^= 1u << st;
      pending &= ~(1u << st);
    }
    return ok;
  };
  constexpr int W = NT / 32;
  const int q_h = (tid & 31) * W + (tid >> 5);
  int32_t h_q = 0;
  auto load_halo = [&](int t) {
    if (q_h < (int)L.halo_cap) h_q = __ldg(m.hpad + (int64_t)t * L.halo_cap + q_h);
  };
  auto gather_halo = [&](int st) {
    Real* xc = reinterpret_cast<Real*>(smem + st * L.stage + L.off_cells) + 4 * TC;
    if (q_h < (int)L.halo_cap) cp_async16(xc + 4 * q_h, U + 4 * (int64_t)h_q);
  };

  NoMass<Real> mass;
  Real rate = Real(0), chk = Real(0);
  int neg = 0, timeout = 0;
  if (tid == 0 && n_tiles > 0) {
    load_offsets(t_first);
    issue_mesh(0);
  }
  if (n_tiles > 0) load_halo(t_first);
  pdl_trigger();
  pdl_wait();
  if (ctl->done) {
    if (tid == 0 && n_tiles > 0) {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar[0])) : "memory");
      mbar_wait(&bar[0], 0u);
    }
    return;
  }
  {
    const int cur = ctl->cur;
    dt = Real(ctl->dt);
    U = cur ? s.h[1] : s.h[0];
    U1 = cur ? s.h[0] : s.h[1];
  }
  if (n_tiles > 0) {
    if (tid == 0) {
      issue_cells(0, t_first);
      if (n_tiles > 1) load_offsets(t_first + t_step);
    }
    gather_halo(0);
    if (n_tiles > 1) load_halo(t_first + t_step);
    const bool ok = (tid == 0) ? wait_stage(0) : true;
    cp_async_wait_all();
    if (__syncthreads_or(!ok)) timeout = 1;
  }
  // The thread's cells of the tile whose faces were computed last: state
  // and per-cell constants, used by the next iteration's cell updates.
  V4<Real> cst[CPT];
  Real c_area[CPT], c_irP[CPT], c_gn2[CPT];  // tile k-1's, used in iteration k
  Real n_area[CPT], n_irP[CPT], n_gn2[CPT];  // tile k's, loaded at the start of iteration k
  int prev_base = 0, prev_nc = 0;
  for (int k = 0; !timeout && k <= n_tiles; ++k) {
    const int st = k & 1;
    const int tile = t_first + k * t_step;
    const bool has_tile = k < n_tiles, has_next = k + 1 < n_tiles;
    // Tile k+1: copies into the other stage (free since the barrier that
    // ended iteration k-1) and its halo gather, from indices in registers.
    if (has_next) {
      if (tid == 0) {
        issue_mesh(st ^ 1);
        issue_cells(st ^ 1, tile + t_step);
        if (k + 2 < n_tiles) load_offsets(tile + 2 * t_step);
      }
      gather_halo(st ^ 1);
      if (k + 2 < n_tiles) load_halo(tile + 2 * t_step);
    }
    // tile k's per-cell constants (global loads, consumed next iteration)
    if (has_tile) {
      const int base = tile * TC;
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) {
        const int j = tid + cc * NT;
        n_area[cc] = m.area[base + j];
        n_irP[cc] = m.irP[base + j];
        n_gn2[cc] = s.gn2[base + j];
      }
    }
    // cell updates of tile k-1 (its slots were completed by the last barrier)
    if (k >= 1) {
      const Real* slots = slot_set(k - 1);
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) {
        const int j = tid + cc * NT;
        if (j >= prev_nc) break;
        const V4<Real> f0 = ld4(slots + 4 * j);
        const V4<Real> f1 = ld4(slots + 4 * (TC + kSlotPad + j));
        const V4<Real> f2 = ld4(slots + 4 * (2 * (TC + kSlotPad) + j));
        Real R[3];
        Real s1, e1, s2, e2;
        two_sum(f0.x, f1.x, s1, e1);
        two_sum(s1, f2.x, s2, e2);
        R[0] = add_rn(s2, add_rn(e1, e2));
        float2 p1, q1, p2, q2;
        two_sum2(make_float2(f0.z, f0.w), make_float2(f1.z, f1.w), p1, q1);
        two_sum2(p1, make_float2(f2.z, f2.w), p2, q2);
        const float2 r = add2(p2, add2(q1, q2));
        R[1] = r.x;
        R[2] = r.y;
        const V4<Real> c = cst[cc];
        Real a1, b1, c1;
        cell_finish<Real, true>(c.x, c.y, c.z, c_area[cc], c_irP[cc], c_gn2[cc], dt, R, num, a1, b1,
                                c1, mass, rate, chk, neg);
        st4(U1 + 4 * (int64_t)(prev_base + j), a1, b1, c1, c.w);
      }
    }
    if (has_tile) {
      const unsigned char* p = smem + st * L.stage;
      const Real* xc = reinterpret_cast<const Real*>(p + L.off_cells);
      const int32_t* rS = reinterpret_cast<const int32_t*>(p + L.off_tS);
      Real* slots = slot_set(k);
      const int base = tile * TC;
      const int nrec = s_nrec[st];
      // face records of tile k, the highest threads first
      for (int r = NT - 1 - tid; r < nrec; r += NT) {
        int32_t packed;
        float fnx, fny, flen;
        rec_f32(rS, r, packed, fnx, fny, flen);
        const int a = packed >> 16;
        const int b = (int)(int16_t)(packed & 0xffff);
        float c0, cA1, cA2, cB1, cB2;
        if (b == kSideWall) {
          if (a == kSideWall) continue;  // padding record
          const V4<Real> A = ld4(xc + 4 * ((-1 - a) & (TC - 1)));
          face_flux_f32<true>(A, A, fnx, fny, flen, num, c0, cA1, cA2, cB1, cB2);
          st4(slots + 4 * slot_pad<TC>(-1 - a), c0, 0.0f, cA1, cA2);
          continue;
        }
        const int ia = a < 0 ? ((-1 - a) & (TC - 1)) : a;
        const int ib = b < 0 ? ((-1 - b) & (TC - 1)) : b;
        const V4<Real> A = ld4(xc + 4 * ia);
        const V4<Real> B = ld4(xc + 4 * ib);
        face_flux_f32<false>(A, B, fnx, fny, flen, num, c0, cA1, cA2, cB1, cB2);
        if (a < 0) st4(slots + 4 * slot_pad<TC>(-1 - a), c0, 0.0f, cA1, cA2);
        if (b < 0) st4(slots + 4 * slot_pad<TC>(-1 - b), -c0, 0.0f, cB1, cB2);
      }
      // this tile's own cells and constants, for the next iteration
#pragma unroll
      for (int cc = 0; cc < CPT; ++cc) {
        const int j = tid + cc * NT;
        cst[cc] = ld4(xc + 4 * j);
        c_area[cc] = n_area[cc];
        c_irP[cc] = n_irP[cc];
        c_gn2[cc] = n_gn2[cc];
      }
      prev_base = base;
      prev_nc = min(TC, cell_end - base);
    }
    // tile k+1's copies and halo must have landed before its faces; tile
    // k's slots must be complete before its cell updates
    const bool ok = (tid == 0 && has_next) ? wait_stage(st ^ 1) : true;
    cp_async_wait_all();
    if (__syncthreads_or(!ok)) {
      timeout = 1;
      break;
    }
  }
  if (timeout && tid == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if ((pending >> i) & 1u) mbar_wait(&bar[i], (parity_bits >> i) & 1u);
  }
  finish_launch<NT>(ctl, s.partial, ch.part, ctl->part0, (int)ctl->nparts, mass.value(),
                    (double)rate, (chk != Real(0) ? kErrNan : 0) | (timeout ? kErrTimeout : 0), neg,
                    kStepped, num.courant);
}

// CFL rate and mass of the current state, no step (initialisation), one
// scenario in separate arrays (two-launch layout).
template <typename Real>
__global__ void __launch_bounds__(256) k_cfl(DevMesh<Real> m, DevState<Real> s, Num num) {
  using O = Ops<Real>;
  Ctl* ctl = s.ctl;
  const int cur = ctl->cur;
  const Real* __restrict__ h = cur ? s.h[1] : s.h[0];
  const Real* __restrict__ hu = cur ? s.hu[1] : s.hu[0];
  const Real* __restrict__ hv = cur ? s.hv[1] : s.hv[0];
  MassAcc<Real> mass;
  Real rate = Real(0);
  int bad = 0;
  const int64_t sd = s.stride;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m.T;
       i += (int64_t)gridDim.x * blockDim.x) {
    const Real hh = h[i * sd], qx = hu[i * sd], qy = hv[i * sd];
    if (O::wet(hh, num)) {
      const Real lam = O::div(O::sqrt_(qx * qx + qy * qy), hh) + O::sqrt_(Real(num.g) * hh);
      rate = fmax(rate, lam * m.irP[i]);
    }
    if (!isfinite(hh + qx + qy)) bad = 1;
    mass.add(m.area[i], hh);
  }
  finish_launch<256>(ctl, s.partial, blockIdx.x, 0, gridDim.x, mass.value(), (double)rate,
                     bad ? kErrNan : 0, 0, kCflOnly, num.courant);
}

// The same on interleaved cells, over the tiled layout's work chunks (every
// scenario of the mesh). TC: cells per tile. kind: kCflOnly (set the CFL
// step) or kMassOnly (mass on demand, step control untouched).
template <typename Real>
__global__ void __launch_bounds__(256) k_cfl_tiled(DevMesh<Real> m, DevState<Real> s, Num num,
                                                   int TC, int kind) {
  using O = Ops<Real>;
  const Chunk ch = m.chunks[blockIdx.x];
  Ctl* ctl = s.ctl + ch.scen;
  const int cur = ctl->cur;
  const Real* __restrict__ U = cur ? s.h[1] : s.h[0];
  const int64_t cell_end = ch.cell_end;
  MassAcc<Real> mass;
  Real rate = Real(0);
  int bad = 0;
  for (int k = 0; k < ch.ntiles; ++k) {
    const int64_t c0 = (int64_t)(ch.tile0 + k * ch.stride) * TC;
    const int64_t c1 = min(c0 + (int64_t)TC, cell_end);
    for (int64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
      const Real hh = U[4 * i], qx = U[4 * i + 1], qy = U[4 * i + 2];
      if (O::wet(hh, num)) {
        const Real lam = O::div(O::sqrt_(qx * qx + qy * qy), hh) + O::sqrt_(Real(num.g) * hh);
        rate = fmax(rate, lam * m.irP[i]);
      }
      if (!isfinite(hh + qx + qy)) bad = 1;
      if (m.irP[i] != Real(0)) {  // 0: a ghost (or padding) cell
        mass.add(m.area[i], hh);
        if (s.hlo) mass.add(m.area[i], s.hlo[i]);  // the depth's residual
      }
    }
  }
  finish_launch<256>(ctl, s.partial, ch.part, ctl->part0, (int)ctl->nparts, mass.value(),
                     (double)rate, bad ? kErrNan : 0, 0, kind, num.courant);
}

// Mass integral of each scenario's latest launch: the sum of its per-block
// partial sums, in a fixed order (block s of 256 threads for scenario s).
static __global__ void __launch_bounds__(256) k_mass_sum(Ctl* ctls, const double* __restrict__ partial) {
  __shared__ double sh[256];
  Ctl* ctl = ctls + blockIdx.x;
  const long long n = ctl->nparts, p0 = ctl->part0;
  double acc = 0.0;
  for (long long j = threadIdx.x; j < n; j += 256) acc += partial[p0 + j];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) ctl->mass = sh[0];
}

// Caller order (double) -> internal order (Real): dst[j * stride] = src[perm[j]]
// for every internal cell j < n (perm[j] < 0 marks tile padding: skipped).
template <typename Real>
__global__ void k_gather(const double* __restrict__ src, const int32_t* __restrict__ perm,
                         Real* __restrict__ dst, int64_t n, int stride) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = perm[j];
    if (c >= 0) dst[j * stride] = Real(src[c]);
  }
}

// Internal order (Real) -> caller order (double): dst[perm[j]] = src[j * stride].
template <typename Real>
__global__ void k_scatter(const Real* __restrict__ src, const int32_t* __restrict__ perm,
                          double* __restrict__ dst, int64_t n, int stride) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = perm[j];
    if (c >= 0) dst[c] = double(src[j * stride]);
  }
}

}  // namespace swe
