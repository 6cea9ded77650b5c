// Reverse mode (adjoint) of one explicit step, for gradients of a loss with
// respect to the initial state, the bed z and Manning's n (through g n^2).
//
// One step maps U^n to U^{n+1} with a fixed dt (Sec. 2.2, Eq. 4 and the
// semi-implicit friction):
//   U*_i     = U^n_i - (dt / Omega_i) R_i,  R_i = sum over faces of s l (F + P n)
//   U^{n+1}_i = friction(U*_i)              (clip of h at 0, momentum / d)
// Given lambda = dL/dU^{n+1}, the adjoint step forms, per cell,
//   mu_i  = dL/dU*_i          (friction transposed; needs only U^{n+1}, g n^2, dt)
//   rho_i = dL/dR_i = -(dt / Omega_i) mu_i
// and per face the vector-Jacobian product of its two residual contributions
// with (rho_A, rho_B), giving dL/d(h, hu, hv, z) of both sides. Then
//   dL/dU^n_i = mu_i + sum over the cell's faces of its side's part,
//   dL/dz_i  += sum of the z parts,  dL/d(g n^2)_i += friction part.
// Every branch (wet/dry tests, the HLLC case, the min/max of the wave-speed
// estimates and of the reconstruction) is taken as the forward step takes
// it; where the forward picks between two equal values (a tie of max(zA, zB)
// or of the speed estimates) the derivative follows the first argument, the
// convention of the FP64 reference the gradients are checked against.
//
// The friction factor d is recovered from U^{n+1}: with c = dt g n^2 h^{-7/3}
// and q1 = |q^{n+1}|, d = 1 + c |q*| = 1 / (1 - c q1) exactly, so the adjoint
// needs no per-step copy of U* (relative error about eps * d).
// A depth clipped at 0 (never under the CFL step; the forward counts it) is
// differentiated as if it were not clipped.
#pragma once

#include "swe_kernels.cuh"

namespace swe {

// dL/dU* of one cell from its post-step state (h1, q1x, q1y) and lambda:
// mu (3 values) and the derivative with respect to its g n^2.
template <typename Real>
__device__ __forceinline__ void cell_vjp(Real h1, Real q1x, Real q1y, Real lh, Real lx, Real ly,
                                         Real gn2, Real dt, const Num& num, Real& mh, Real& mx,
                                         Real& my, Real& bgn2) {
  using O = Ops<Real>;
  const Real zero = Real(0);
  if (O::wet(h1, num)) {
    const Real q1n = O::sqrt_(q1x * q1x + q1y * q1y);
    const Real ch = O::friction(dt, Real(1), Real(1), h1);  // dt h^{-7/3}
    const Real c = ch * gn2;
    const Real cq = c * q1n;        // (d - 1) / d
    const Real rd = Real(1) - cq;   // 1 / d
    const Real ql = q1x * lx + q1y * ly;
    const Real k = q1n > zero ? O::div(c * ql, q1n) : zero;
    mx = rd * (lx - k * q1x);
    my = rd * (ly - k * q1y);
    mh = lh + Real(7.0 / 3.0) * O::div(cq, h1) * ql;
    bgn2 = -q1n * ch * ql;
  } else {
    mh = lh;
    mx = zero;
    my = zero;
    bgn2 = zero;
  }
}

// Vector-Jacobian product of one face, with both sides' contributions:
// inputs the sides' cells (h, hu, hv, z) as the forward step read them, the
// geometry, and rho = dL/dR of side A (the face adds c_A to R_A) and side B
// (the face subtracts c_B from R_B); outputs gA, gB = dL/d(h, hu, hv, z) of
// each side through this face. The face is the clamped form of the flux the
// tiled steps compute (face_flux_f32, face_flux_f64): one HLL formula with
// the clamped speeds S- = min(S_A, 0), S+ = max(S_B, 0), the dry side's
// normal velocity replaced by un_B - 2 c_B (or un_A + 2 c_A) in the
// wave-speed estimates, the transverse momentum upwinded by the sign of F0.
// It is the same function of the inputs as the HLLC case analysis (the
// clamped speeds reproduce the supersonic cases: with S_A >= 0, S- = 0 and
// F = F_A, whose derivative with respect to S_A is 0), so the derivatives
// agree with the case analysis's away from ties; it has no case branches.
// Ties follow fixed conventions: max(zA, zB) and the speed estimates take
// the first argument, S_A = 0 counts as S_A >= 0 and S_B = 0 as S_B <= 0.
// For a wall B is ignored (the mirror of A folds into gA, gB = 0).
template <typename Real, bool Wall>
__device__ __forceinline__ void face_vjp_clamped(const V4<Real>& A, const V4<Real>& B, Real nx,
                                                 Real ny, Real len, const Num& num, Real rA0,
                                                 Real rA1, Real rA2, Real rB0, Real rB1, Real rB2,
                                                 Real gA[4], Real gB[4]) {
  using O = Ops<Real>;
  const Real zero = Real(0), half = Real(0.5), quarter = Real(0.25);
  const Real g = Real(num.g), hg = half * g;
  // ---- forward, keeping what the reverse sweep needs
  const Real rA = O::wet(A.x, num) ? O::div(Real(1), A.x) : zero;  // 0 on a dry cell
  const Real uA = A.y * rA, vA = A.z * rA;
  const Real unA = uA * nx + vA * ny;
  const Real utA = vA * nx - uA * ny;
  Real hB, zB, unB, utB, uB = zero, vB = zero, rB = zero;
  if (Wall) {
    hB = A.x; zB = A.w; unB = -unA; utB = utA;
  } else {
    rB = O::wet(B.x, num) ? O::div(Real(1), B.x) : zero;
    uB = B.y * rB;
    vB = B.z * rB;
    hB = B.x; zB = B.w;
    unB = uB * nx + vB * ny;
    utB = vB * nx - uB * ny;
  }
  const bool zsA = A.w >= zB;  // max(zA, zB) taken from A on a tie
  const Real zs = zsA ? A.w : zB;
  const Real xA = A.x + A.w - zs, xB = hB + zB - zs;
  const bool wetA = O::wet(xA, num), wetB = O::wet(xB, num);  // reconstructed sides wet
  const Real hAs = wetA ? xA : zero, hBs = wetB ? xB : zero;
  const Real cA = O::sqrt_(g * hAs), cB = O::sqrt_(g * hBs);
  const Real vnA = wetA ? unA : unB - Real(2) * cB;
  const Real vnB = wetB ? unB : unA + Real(2) * cA;
  const Real us = (vnA + vnB) * half + cA - cB;
  const Real cs = (cA + cB) * half + (vnA - vnB) * quarter;
  const Real a1 = vnA - cA, a2 = us - cs, b1 = vnB + cB, b2 = us + cs;
  const bool firstA = a1 <= a2, firstB = b1 >= b2;
  const Real SA = firstA ? a1 : a2, SB = firstB ? b1 : b2;
  const bool negA = SA < zero, posB = SB > zero;
  const Real Sm = negA ? SA : zero, Sp = posB ? SB : zero;
  const Real qA = hAs * unA, qB = hBs * unB;
  const Real FA1 = qA * unA + hg * hAs * hAs, FB1 = qB * unB + hg * hBs * hBs;
  const bool live = wetA || wetB;  // both sides dry: F = 0 whatever the speeds
  const Real inv = live ? O::div(Real(1), Sp - Sm) : zero;
  const Real SS = Sm * Sp, dh = hBs - hAs, dq = qB - qA;
  const Real N0 = Sp * qA - Sm * qB + SS * dh;
  const Real N1 = Sp * FA1 - Sm * FB1 + SS * dq;
  const Real F0 = N0 * inv;
  const bool upA = F0 >= zero;  // transverse momentum from A where F0 >= 0

  // ---- reverse sweep
  // residual contributions: A gets +l (F0, Fx + PA nx, Fy + PA ny), B gets
  // -l (F0, Fx + PB nx, Fy + PB ny), Fx = F1 nx - F2 ny, Fy = F1 ny + F2 nx
  const Real bFx = len * (rA1 - rB1), bFy = len * (rA2 - rB2);
  const Real bF1 = bFx * nx + bFy * ny;
  Real bF0 = zero, bF2 = zero;
  if (!Wall) {
    bF0 = len * (rA0 - rB0);
    bF2 = bFy * nx - bFx * ny;
  }
  const Real bPA = len * (rA1 * nx + rA2 * ny);
  const Real bPB = Wall ? zero : -len * (rB1 * nx + rB2 * ny);
  // P = g/2 (h^2 - h*^2)
  Real bhA = g * A.x * bPA, bhB = g * hB * bPB;
  Real bhAs = -g * hAs * bPA, bhBs = -g * hBs * bPB;
  // F2 = F0 ut
  bF0 += bF2 * (upA ? utA : utB);
  const Real but = bF2 * F0;
  Real butA = upA ? but : zero, butB = upA ? zero : but;
  // F0 = N0 / D, F1 = N1 / D, D = S+ - S-
  const Real bN0 = bF0 * inv, bN1 = bF1 * inv;
  const Real bD = -(bF0 * N0 + bF1 * N1) * inv * inv;
  const Real bSp = bD + bN0 * (qA + Sm * dh) + bN1 * (FA1 + Sm * dq);
  const Real bSm = -bD + bN0 * (Sp * dh - qB) + bN1 * (Sp * dq - FB1);
  Real bqA = bN0 * Sp - bN1 * SS, bqB = bN1 * SS - bN0 * Sm;
  bhBs += bN0 * SS;
  bhAs -= bN0 * SS;
  const Real bFA1 = bN1 * Sp, bFB1 = -bN1 * Sm;
  // F1 of each side = q un + g/2 h*^2, q = h* un
  bqA += bFA1 * unA;
  bqB += bFB1 * unB;
  Real bunA = bFA1 * qA + bqA * hAs, bunB = bFB1 * qB + bqB * hBs;
  bhAs += bFA1 * g * hAs + bqA * unA;
  bhBs += bFB1 * g * hBs + bqB * unB;
  // S- = min(S_A, 0), S+ = max(S_B, 0); the speed estimates
  const Real bSA = negA ? bSm : zero, bSB = posB ? bSp : zero;
  Real bvnA = zero, bvnB = zero, bcA = zero, bcB = zero, bus = zero, bcs = zero;
  if (firstA) { bvnA += bSA; bcA -= bSA; } else { bus += bSA; bcs -= bSA; }
  if (firstB) { bvnB += bSB; bcB += bSB; } else { bus += bSB; bcs += bSB; }
  bvnA += half * bus + quarter * bcs;
  bvnB += half * bus - quarter * bcs;
  bcA += bus + half * bcs;
  bcB += half * bcs - bus;
  // a dry side's velocity in the estimates
  if (wetA) { bunA += bvnA; } else { bunB += bvnA; bcB -= Real(2) * bvnA; }
  if (wetB) { bunB += bvnB; } else { bunA += bvnB; bcA += Real(2) * bvnB; }
  // c = sqrt(g h*): dc/dh* = g / (2 c) on a wet side (c = 0 and no term on a dry one)
  if (wetA) bhAs += bcA * O::div(hg, cA);
  if (wetB) bhBs += bcB * O::div(hg, cB);
  // reconstruction h* = h + z - max(zA, zB) where it stays wet
  Real bzA = zero, bzB = zero, bzs = zero;
  if (wetA) { bhA += bhAs; bzA += bhAs; bzs -= bhAs; }
  if (wetB) { bhB += bhBs; bzB += bhBs; bzs -= bhBs; }
  if (zsA) bzA += bzs; else bzB += bzs;
  if (Wall) {  // B mirrors A: hB = hA, zB = zA, unB = -unA, utB = utA
    bhA += bhB;
    bzA += bzB;
    bunA -= bunB;
    butA += butB;
  }
  // face frame -> x, y velocities -> conserved variables (u = hu r, r = 1/h
  // on a wet cell, 0 on a dry one)
  const Real buA = bunA * nx - butA * ny, bvA = bunA * ny + butA * nx;
  gA[0] = bhA - (buA * uA + bvA * vA) * rA;
  gA[1] = buA * rA;
  gA[2] = bvA * rA;
  gA[3] = bzA;
  if (Wall) {
    gB[0] = zero; gB[1] = zero; gB[2] = zero; gB[3] = zero;
  } else {
    const Real buB = bunB * nx - butB * ny, bvB = bunB * ny + butB * nx;
    gB[0] = bhB - (buB * uB + bvB * vB) * rB;
    gB[1] = buB * rB;
    gB[2] = bvB * rB;
    gB[3] = bzB;
  }
}

// Inputs and outputs of one adjoint launch (interleaved cells, internal
// order, padded to whole tiles).
template <typename Real>
struct AdjArgs {
  const Real* un;      // U^n (h, hu, hv, z)
  const Real* u1;      // U^{n+1} (h, hu, hv, z)
  const Real* lam_in;  // dL/dU^{n+1} (h, hu, hv, accumulated dL/dz)
  Real* lam_out;       // dL/dU^n, same layout
  const Real* gn2;     // g n^2 per cell
  Real* dgn2;          // accumulated dL/d(g n^2) per cell (read-modify-write)
  Real dt;
  int* err;            // kErr* bits (timeouts)
  // Gauge seeds added to the depth adjoint of lam_out once every block is
  // done (by the last block): lam_out[4 gcells[j]] += gseed[gstep G + j],
  // j < G; gstep < 0 adds nothing. ticket: a zeroed counter.
  const int32_t* gcells;
  const double* gseed;
  int G;
  long long gstep;
  unsigned int* ticket;
};

// Shared-memory plan of k_tiled_adjoint. Per stage: the tile's and its
// halo's cells of U^n; the halo cells' U^{n+1}, lambda, areas and g n^2 (a
// tile's own cells read theirs straight from global memory into registers);
// the face records with their geometry; the halo list. After the stages:
// rho per tile and halo cell, the face slots (dh, dhu, dhv, dz) per face of
// each tile cell, face-major, and the NS mbarriers.
struct AdjLayout {
  uint32_t ext, rec_cap, halo_cap;
  uint32_t off_un, off_u1, off_lam, off_harea, off_hgn2, off_tS, off_g0, off_g1, off_g2, off_hidx;
  uint32_t stage;
  uint32_t off_rho, off_slots, off_bars, total;
};

inline AdjLayout make_adj_layout(uint32_t w, uint32_t geo_arrays, uint32_t tc, uint32_t ns,
                                 uint32_t rec_cap, uint32_t halo_cap) {
  auto a16 = [](uint32_t x) { return (x + 15u) & ~15u; };
  AdjLayout L{};
  L.rec_cap = rec_cap;
  L.halo_cap = halo_cap;
  L.ext = tc + halo_cap;
  uint32_t o = 0;
  L.off_un = o; o += a16(L.ext * 4 * w);
  L.off_u1 = o; o += a16(halo_cap * 4 * w);
  L.off_lam = o; o += a16(halo_cap * 4 * w);
  L.off_harea = o; o += a16(halo_cap * w);
  L.off_hgn2 = o; o += a16(halo_cap * w);
  if (w == 4) {  // FP32: interleaved 16-byte records
    L.off_tS = o; o += a16(rec_cap * 16);
    L.off_g0 = L.off_g1 = L.off_g2 = o;
  } else {
    L.off_tS = o; o += a16(rec_cap * 4);
    L.off_g0 = o; o += a16(rec_cap * w);
    L.off_g1 = o; o += a16(rec_cap * w);
    L.off_g2 = o; o += geo_arrays > 2 ? a16(rec_cap * w) : 0u;
  }
  L.off_hidx = o; o += a16(halo_cap * 4);
  L.stage = o;
  o = ns * L.stage;
  L.off_rho = o; o += a16(L.ext * 4 * w);
  L.off_slots = o; o += a16(3 * tc * 4 * w);
  L.off_bars = o; o += a16(ns * 8);
  L.total = o;
  return L;
}

// Tiled adjoint of one step over the same tiles, records and work chunks as
// k_tiled_step (scenario of each chunk, interleaved tile walk, NS-stage TMA
// pipeline with the halo gathered by cp.async). Per tile:
//   (A) mu and rho of every tile and halo cell (rho to shared memory, mu of
//       the thread's own cells kept in registers);
//   (B) the vector-Jacobian product of every face record into the slots of
//       the tile's cells (a face shared with another tile gives only this
//       tile's side, as in the forward);
//   (C) each cell: dL/dU^n = mu + its three slots in face order, the z parts
//       added to the running dL/dz, and its dL/d(g n^2) accumulated.
// (A) of the next tile runs right after (C), so two block barriers per tile.
template <typename Real, int NT, int NS, int CPT>
__global__ void __launch_bounds__(NT)
    k_tiled_adjoint(DevMesh<Real> m, AdjArgs<Real> A, Num num, AdjLayout L) {
  using O = Ops<Real>;
  constexpr int TC = NT * CPT;
  __shared__ int s_nrec[NS], s_nh[NS];
  extern __shared__ __align__(128) unsigned char smem[];
  Real* rho = reinterpret_cast<Real*>(smem + L.off_rho);      // [ext][4]
  Real* slots = reinterpret_cast<Real*>(smem + L.off_slots);  // [3 TC][4]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.off_bars);

  const Chunk ch = m.chunks[blockIdx.x];
  const int t_first = ch.tile0, n_tiles = ch.ntiles, t_step = ch.stride;
  const int cell_end = ch.cell_end;
  const Real dt = A.dt;
  const int tid = threadIdx.x;

  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    fence_mbar_init();
  }
  __syncthreads();

  uint32_t parity_bits = 0, pending = 0;
  auto issue = [&](int st, int t) {
    unsigned char* p = smem + st * L.stage;
    const int64_t base = (int64_t)t * TC;
    const int64_t r0 = m.toff[t], h0 = m.hoff[t];
    const uint32_t nrec = (uint32_t)(m.toff[t + 1] - r0);
    const uint32_t nh = (uint32_t)(m.hoff[t + 1] - h0);
    const uint32_t cells = TC * 4 * (uint32_t)sizeof(Real);
    s_nrec[st] = (int)nrec;
    s_nh[st] = (int)nh;
    const uint32_t rb = nrec * (uint32_t)sizeof(Real);
    fence_proxy_async();
    mbar_expect_tx(&bar[st], cells + nrec * rec_bytes<Real>() + nh * 4);
    bulk_g2s(p + L.off_un, A.un + 4 * base, cells, &bar[st]);
    if constexpr (sizeof(Real) == 4) {
      bulk_g2s(p + L.off_tS, m.trec + r0, nrec * 16, &bar[st]);
    } else {
      bulk_g2s(p + L.off_tS, m.tS + r0, nrec * 4, &bar[st]);
      bulk_g2s(p + L.off_g0, m.tg0 + r0, rb, &bar[st]);
      bulk_g2s(p + L.off_g1, m.tg1 + r0, rb, &bar[st]);
      bulk_g2s(p + L.off_g2, m.tg2 + r0, rb, &bar[st]);
    }
    if (nh > 0) bulk_g2s(p + L.off_hidx, m.hidx + h0, nh * 4, &bar[st]);
    pending |= 1u << st;
  };
  auto wait_stage = [&](int st) -> bool {
    const bool ok = mbar_wait(&bar[st], (parity_bits >> st) & 1u, num.wait_rounds);
    if (ok) {
      parity_bits ^= 1u << st;
      pending &= ~(1u << st);
    }
    return ok;
  };
  // halo cells of stage st: three interleaved cells and two scalars each
  auto gather_halo = [&](int st) {
    unsigned char* p = smem + st * L.stage;
    const int32_t* hl = reinterpret_cast<const int32_t*>(p + L.off_hidx);
    Real* dun = reinterpret_cast<Real*>(p + L.off_un) + 4 * TC;
    Real* du1 = reinterpret_cast<Real*>(p + L.off_u1);
    Real* dla = reinterpret_cast<Real*>(p + L.off_lam);
    Real* dar = reinterpret_cast<Real*>(p + L.off_harea);
    Real* dgn = reinterpret_cast<Real*>(p + L.off_hgn2);
    const int nh = s_nh[st];
    constexpr int kV = 16 / (int)sizeof(Real);  // values per 16-byte copy
    for (int q = tid; q < nh; q += NT) {
      const int64_t c = hl[q];
#pragma unroll
      for (int b = 0; b < 4 / kV; ++b) {
        cp_async16(dun + 4 * q + b * kV, A.un + 4 * c + b * kV);
        cp_async16(du1 + 4 * q + b * kV, A.u1 + 4 * c + b * kV);
        cp_async16(dla + 4 * q + b * kV, A.lam_in + 4 * c + b * kV);
      }
      cp_async(dar + q, m.area + c);
      cp_async(dgn + q, A.gn2 + c);
    }
  };

  // Per-cell inputs of the thread's own cells, loaded one tile ahead into
  // registers (their latency hides behind the previous tile's face loop).
  // load_tape_cells: U^{n+1}, g n^2 and area (tape and mesh data);
  // load_adj_cells: lambda and dL/d(g n^2) (the previous launch's output).
  V4<Real> nu1[CPT], nla[CPT];
  Real ngn[CPT], nar[CPT], ndg[CPT];
  auto load_tape_cells = [&](int t) {
    const int64_t b0 = (int64_t)t * TC;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int64_t i = b0 + tid + cc * NT;
      nu1[cc] = ld4(A.u1 + 4 * i);
      ngn[cc] = A.gn2[i];
      nar[cc] = m.area[i];
    }
  };
  auto load_adj_cells = [&](int t) {
    const int64_t b0 = (int64_t)t * TC;
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int64_t i = b0 + tid + cc * NT;
      nla[cc] = ld4(A.lam_in + 4 * i);
      ndg[cc] = A.dgn2[i];
    }
  };
  auto load_cells = [&](int t) {
    load_tape_cells(t);
    load_adj_cells(t);
  };
  // (A) of a tile: mu (registers) and the friction and dL/dz parts of the
  // thread's own cells from the registers load_cells filled, rho of those
  // cells and of the halo cells this thread gathered (gather_halo's
  // assignment, so no barrier is needed after its own copies land).
  Real mu[CPT][3], bg[CPT], dzr[CPT];
  auto phase_a = [&](int st, int tile) {
    const unsigned char* p = smem + st * L.stage;
    const Real* su1 = reinterpret_cast<const Real*>(p + L.off_u1);
    const Real* sla = reinterpret_cast<const Real*>(p + L.off_lam);
    const Real* har = reinterpret_cast<const Real*>(p + L.off_harea);
    const Real* hgn = reinterpret_cast<const Real*>(p + L.off_hgn2);
    const int nc = min(TC, cell_end - tile * TC);
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int j = tid + cc * NT;
      const V4<Real> c1 = nu1[cc];
      const V4<Real> la = nla[cc];
      dzr[cc] = la.w;
      cell_vjp<Real>(c1.x, c1.y, c1.z, la.x, la.y, la.z, ngn[cc], dt, num, mu[cc][0], mu[cc][1],
                     mu[cc][2], bg[cc]);
      bg[cc] += ndg[cc];
      const Real a = j < nc ? -O::div(dt, nar[cc]) : Real(0);  // padding: area 0
      st4(rho + 4 * j, a * mu[cc][0], a * mu[cc][1], a * mu[cc][2], Real(0));
    }
    const int nh = s_nh[st];
    for (int q = tid; q < nh; q += NT) {
      const int j = TC + q;
      const V4<Real> c1 = ld4(su1 + 4 * q);
      const V4<Real> la = ld4(sla + 4 * q);
      Real mh, mx, my, b;
      cell_vjp<Real>(c1.x, c1.y, c1.z, la.x, la.y, la.z, hgn[q], dt, num, mh, mx, my, b);
      const Real a = -O::div(dt, har[q]);
      st4(rho + 4 * j, a * mh, a * mx, a * my, Real(0));
    }
  };
  int timeout = 0;
  // Programmatic dependent launch: the first tiles' tape states, records and
  // halo lists and the own cells' tape inputs are fetched while the previous
  // adjoint step finishes; lambda and dL/d(g n^2), its output, only after
  // griddepcontrol.wait.
  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < NS - 1; ++i)
      if (i < n_tiles) issue(i, t_first + i * t_step);
  }
  if (n_tiles > 0) load_tape_cells(t_first);
  pdl_trigger();
  pdl_wait();
  if (n_tiles > 0) load_adj_cells(t_first);
  if (n_tiles > 0) {
    const bool ok = (tid == 0) ? wait_stage(0) : true;
    if (__syncthreads_or(!ok)) {
      timeout = 1;
    } else {
      gather_halo(0);
      cp_async_wait_all();
      phase_a(0, t_first);
      __syncthreads();
    }
  }
  // Each iteration: (B) the faces of tile k, then (C) its cells followed by
  // (A) of tile k+1 (rho is free once every face of tile k is done). Two
  // block barriers per tile.
  for (int k = 0; !timeout && k < n_tiles; ++k) {
    const int st = k % NS;
    const int tile = t_first + k * t_step;
    const bool has_next = k + 1 < n_tiles;
    if (tid == 0 && k + NS - 1 < n_tiles) issue((k + NS - 1) % NS, tile + (NS - 1) * t_step);
    // the next tile's own-cell inputs, into registers while the faces run
    if (has_next) load_cells(tile + t_step);
    const unsigned char* p = smem + st * L.stage;
    const Real* sun = reinterpret_cast<const Real*>(p + L.off_un);
    const int32_t* rS = reinterpret_cast<const int32_t*>(p + L.off_tS);
    const Real* rg0 = reinterpret_cast<const Real*>(p + L.off_g0);
    const Real* rg1 = reinterpret_cast<const Real*>(p + L.off_g1);
    const Real* rg2 = reinterpret_cast<const Real*>(p + L.off_g2);
    const int base = tile * TC;
    const int nc = min(TC, cell_end - base);
    const int nrec = s_nrec[st];

    // (B) face records
    for (int r = tid; r < nrec; r += NT) {
      int32_t packed;
      Real nx, ny, len;
      if constexpr (sizeof(Real) == 4) {
        rec_f32(rS, r, packed, nx, ny, len);
      } else {
        packed = rS[r];
        Geo<Real>::get(rg0, rg1, rg2, r, nx, ny, len);
      }
      const int a = packed >> 16;
      if (a == kSideWall) continue;  // padding record
      const int b = (int)(int16_t)(packed & 0xffff);
      Real gA[4], gB[4];
      if (b == kSideWall) {  // wall: side A is the tile cell owning the edge
        const int ia = (-1 - a) & (TC - 1);
        const V4<Real> UA = ld4(sun + 4 * ia);
        const V4<Real> RA = ld4(rho + 4 * ia);
        face_vjp_clamped<Real, true>(UA, UA, nx, ny, len, num, RA.x, RA.y, RA.z, Real(0), Real(0),
                                     Real(0), gA, gB);
        st4(slots + 4 * (-1 - a), gA[0], gA[1], gA[2], gA[3]);
        continue;
      }
      const int ia = a < 0 ? ((-1 - a) & (TC - 1)) : a;
      const int ib = b < 0 ? ((-1 - b) & (TC - 1)) : b;
      const V4<Real> UA = ld4(sun + 4 * ia);
      const V4<Real> UB = ld4(sun + 4 * ib);
      const V4<Real> RA = ld4(rho + 4 * ia);
      const V4<Real> RB = ld4(rho + 4 * ib);
      face_vjp_clamped<Real, false>(UA, UB, nx, ny, len, num, RA.x, RA.y, RA.z, RB.x, RB.y, RB.z,
                                    gA, gB);
      if (a < 0) st4(slots + 4 * (-1 - a), gA[0], gA[1], gA[2], gA[3]);
      if (b < 0) st4(slots + 4 * (-1 - b), gB[0], gB[1], gB[2], gB[3]);
    }
    const bool ok = (tid == 0 && has_next) ? wait_stage((k + 1) % NS) : true;
    if (__syncthreads_or(!ok)) {
      timeout = 1;
      break;
    }
    if (has_next) gather_halo((k + 1) % NS);

    // (C) cells
#pragma unroll
    for (int cc = 0; cc < CPT; ++cc) {
      const int j = tid + cc * NT;
      if (j >= nc) break;
      const V4<Real> f0 = ld4(slots + 4 * j);
      const V4<Real> f1 = ld4(slots + 4 * (TC + j));
      const V4<Real> f2 = ld4(slots + 4 * (2 * TC + j));
      st4(A.lam_out + 4 * (int64_t)(base + j), mu[cc][0] + f0.x + f1.x + f2.x,
          mu[cc][1] + f0.y + f1.y + f2.y, mu[cc][2] + f0.z + f1.z + f2.z,
          dzr[cc] + f0.w + f1.w + f2.w);
      A.dgn2[base + j] = bg[cc];
    }
    cp_async_wait_all();
    if (has_next) phase_a((k + 1) % NS, tile + t_step);
    __syncthreads();
  }
  if (timeout && tid == 0) {
#pragma unroll
    for (int i = 0; i < NS; ++i)
      if ((pending >> i) & 1u) mbar_wait(&bar[i], (parity_bits >> i) & 1u);
    atomicOr(A.err, kErrTimeout);
  }
  // The last block to finish adds the gauge seeds (one thread, fixed order,
  // so repeated gauge cells add up deterministically).
  if (A.gstep >= 0) {
    __shared__ int s_last;
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      s_last = atomicAdd(A.ticket, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (s_last && tid == 0) {
      __threadfence();
      for (int j = 0; j < A.G; ++j)
        A.lam_out[4 * (int64_t)A.gcells[j]] += Real(A.gseed[A.gstep * A.G + j]);
      *A.ticket = 0u;
    }
  }
}

// Adds g[k * G + j] to the depth adjoint of cell cells[j] for j < G (one
// thread, so repeated gauge cells add up in a fixed order).
template <typename Real>
__global__ void k_inject_gauges(Real* lam, const int32_t* cells, const double* g, int64_t k, int G) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int j = 0; j < G; ++j) lam[4 * (int64_t)cells[j]] += Real(g[k * (int64_t)G + j]);
}

}  // namespace swe
