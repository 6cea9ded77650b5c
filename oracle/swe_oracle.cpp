// FP64 CPU oracle for the cell-centred HLLC finite-volume shallow-water step.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may call this code:
// only the tests, the package's smoke check and the benchmark's CPU-baseline
// leg load it. It shares no code with the CUDA library.
//
// What it follows (Zaoui, "A GPU-enabled finite volume solver for large
// shallow water simulations"):
//   Sec. 2.1, Eq. 1   U = (h, hu, hv), fluxes G, H, source S = gh(S0 + Sf)
//   Sec. 2.2, Eq. 2-3 cell-centred finite volumes on triangles, the flux
//                     integral as a sum over the three faces F_k . n_k l_k
//   Sec. 2.2, Eq. 4   explicit Euler update of U_i
//   Sec. 2.2          CFL time step with Courant number 0.7; HLLC Riemann
//                     solver at the interfaces; hydrostatic reconstruction of
//                     the bed (S0); semi-implicit friction (Sf)
//   Sec. 3            reflective (wall) boundaries
// The paper names the HLLC solver, the hydrostatic reconstruction and the
// semi-implicit friction without writing them out. Readings taken here:
//   * HLLC for shallow water in the form of Toro (2001): two-rarefaction
//     wave-speed estimates, Toro's dry-bed speeds, HLL for mass and normal
//     momentum, transverse momentum upwinded by the sign of the contact
//     speed S*.
//   * Hydrostatic reconstruction of Audusse et al. (2004): z* = max(zL, zR),
//     h_side* = max(0, h_side + z_side - z*), plus the bed-pressure term
//     g/2 (h_side^2 - h_side*^2) n on that side's momentum flux. A side with
//     h* <= h_eps enters the Riemann problem as dry (h* = 0).
//   * Friction: linearised implicit Manning after the flux update,
//     q^{n+1} = q* / (1 + dt g n^2 |q*| / h^{7/3}), h = h^{n+1};
//     momentum is zeroed where h^{n+1} <= h_eps.
//   * dt = C min over wet cells of (Omega_i / P_i) / (|u_i| + sqrt(g h_i)),
//     P_i the perimeter, C = 0.7.
//   * Walls: mirror ghost (h and z copied, normal velocity negated,
//     tangential kept); the wall mass flux is exactly 0.
//
// Structure: one loop over edges writing per-edge fluxes, one loop over cells
// summing them and updating (the paper's two parallel loops, Sec. 2.3).
// Scalar, plain double (compiled with -ffp-contract=off), no blocking or
// reordering. The state-dependent arithmetic is templated on the number type
// so a forward-mode dual number instantiates the same steps.
//
// Parity pins (tests under tests/): HLLC consistency, antisymmetry, rotation
// invariance, S* = HLL mass flux / HLL depth, exact two-rarefaction and dry-bed
// wave speeds, the wall flux closed form, lake at rest over a bumpy bed with
// dry islands, exact mass conservation with walls, the Stoker and Ritter
// dam-break closed forms, the closed-form friction decay, and Euler's formula
// and closure of the mesh geometry.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <type_traits>
#include <vector>

namespace oracle {

struct Params {
  double g;
  double courant;
  double h_eps;
};

enum Status {
  OK = 0,
  E_INVAL = -1,
  E_MESH = -2,
  E_DRY = -8,
};

// ---------------------------------------------------------------------------
// Forward-mode dual number with a fixed number of tangent directions.
// ---------------------------------------------------------------------------
template <int N>
struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v + b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v - b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r(-a.v); for (int i = 0; i < N; ++i) r.d[i] = -a.d[i]; return r; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v * b.v); for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r(a.v / b.v);
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v);
  return r; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) { return a * Dual<N>(b); }
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) { return Dual<N>(a) * b; }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline bool operator<(const Dual<N>& a, const Dual<N>& b) { return a.v < b.v; }
template <int N> inline bool operator<=(const Dual<N>& a, const Dual<N>& b) { return a.v <= b.v; }
template <int N> inline bool operator>(const Dual<N>& a, const Dual<N>& b) { return a.v > b.v; }
template <int N> inline bool operator>=(const Dual<N>& a, const Dual<N>& b) { return a.v >= b.v; }
template <int N> inline bool operator==(const Dual<N>& a, const Dual<N>& b) { return a.v == b.v; }
template <int N> inline Dual<N> sqrt_(const Dual<N>& a) {
  Dual<N> r(std::sqrt(a.v));
  for (int i = 0; i < N; ++i) r.d[i] = (a.v > 0.0) ? a.d[i] / (2.0 * r.v) : 0.0;
  return r; }
template <int N> inline Dual<N> cbrt_(const Dual<N>& a) {
  Dual<N> r(std::cbrt(a.v));
  for (int i = 0; i < N; ++i) r.d[i] = (a.v != 0.0) ? a.d[i] / (3.0 * r.v * r.v) : 0.0;
  return r; }
template <int N> inline double value_of(const Dual<N>& a) { return a.v; }

inline double sqrt_(double a) { return std::sqrt(a); }
inline double cbrt_(double a) { return std::cbrt(a); }
inline double value_of(double a) { return a; }

// max/min written as comparisons so dual numbers follow the selected branch.
template <class R> inline R vmax(const R& a, const R& b) { return (a >= b) ? a : b; }
template <class R> inline R vmin(const R& a, const R& b) { return (a <= b) ? a : b; }

// ---------------------------------------------------------------------------
// Mesh: oriented triangles, edges with left/right cells, geometry (Eq. 3).
// ---------------------------------------------------------------------------
struct Mesh {
  int64_t V = 0, T = 0, E = 0, Eb = 0;
  std::vector<double> xy;         // 2V
  std::vector<int32_t> tri;       // 3T, counter-clockwise
  std::vector<double> area;       // Omega_i
  std::vector<double> perim;      // P_i = sum of the cell's edge lengths
  std::vector<int32_t> eL, eR;    // eR = -1 for a wall edge
  std::vector<double> nx, ny, len;  // unit normal pointing out of eL, length
  std::vector<int32_t> cell_edge;   // 3T: edge k of cell i joins its nodes k, k+1
};

// Builds edges and geometry. Interior edge: eL = the lower cell index.
// Returns OK, or E_MESH for a bad node index, a degenerate triangle or an
// edge shared by more than two triangles.
static int build_mesh(const double* xy, int64_t V, const int32_t* tri, int64_t T, Mesh& m) {
  if (V < 0 || T < 0) return E_INVAL;
  m.V = V; m.T = T;
  m.xy.assign(xy, xy + 2 * V);
  m.tri.assign(tri, tri + 3 * T);
  m.area.assign(T, 0.0);
  m.perim.assign(T, 0.0);
  for (int64_t i = 0; i < T; ++i) {
    for (int k = 0; k < 3; ++k) {
      int32_t a = m.tri[3 * i + k];
      if (a < 0 || a >= V) return E_MESH;
    }
    int32_t a = m.tri[3 * i], b = m.tri[3 * i + 1], c = m.tri[3 * i + 2];
    if (a == b || b == c || a == c) return E_MESH;
    double x0 = xy[2 * a], y0 = xy[2 * a + 1];
    double x1 = xy[2 * b], y1 = xy[2 * b + 1];
    double x2 = xy[2 * c], y2 = xy[2 * c + 1];
    double s = 0.5 * ((x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0));
    if (!(s != 0.0) || !std::isfinite(s)) return E_MESH;
    if (s < 0.0) {  // make the node order counter-clockwise
      m.tri[3 * i + 1] = c;
      m.tri[3 * i + 2] = b;
      s = -s;
    }
    m.area[i] = s;
  }
  // Every half-edge (cell i, local edge k) keyed by its unordered node pair.
  struct Half { uint64_t key; int64_t cell; int k; };
  std::vector<Half> hs;
  hs.reserve(3 * T);
  for (int64_t i = 0; i < T; ++i)
    for (int k = 0; k < 3; ++k) {
      uint64_t a = (uint32_t)m.tri[3 * i + k], b = (uint32_t)m.tri[3 * i + (k + 1) % 3];
      uint64_t lo = std::min(a, b), hi = std::max(a, b);
      hs.push_back({(lo << 32) | hi, i, k});
    }
  std::sort(hs.begin(), hs.end(), [](const Half& p, const Half& q) {
    if (p.key != q.key) return p.key < q.key;
    return p.cell < q.cell;
  });
  m.cell_edge.assign(3 * T, -1);
  m.eL.clear(); m.eR.clear(); m.nx.clear(); m.ny.clear(); m.len.clear();
  m.Eb = 0;
  size_t j = 0;
  while (j < hs.size()) {
    size_t r = j + 1;
    while (r < hs.size() && hs[r].key == hs[j].key) ++r;
    if (r - j > 2) return E_MESH;
    const Half& left = hs[j];  // lower cell index
    int32_t e = (int32_t)m.eL.size();
    int32_t a = m.tri[3 * left.cell + left.k];
    int32_t b = m.tri[3 * left.cell + (left.k + 1) % 3];
    double dx = xy[2 * b] - xy[2 * a];
    double dy = xy[2 * b + 1] - xy[2 * a + 1];
    double l = std::sqrt(dx * dx + dy * dy);
    m.eL.push_back((int32_t)left.cell);
    m.nx.push_back(dy / l);   // outward for a counter-clockwise cell
    m.ny.push_back(-dx / l);
    m.len.push_back(l);
    m.cell_edge[3 * left.cell + left.k] = e;
    if (r - j == 2) {
      const Half& right = hs[j + 1];
      if (right.cell == left.cell) return E_MESH;
      m.eR.push_back((int32_t)right.cell);
      m.cell_edge[3 * right.cell + right.k] = e;
    } else {
      m.eR.push_back(-1);
      ++m.Eb;
    }
    j = r;
  }
  m.E = (int64_t)m.eL.size();
  for (int64_t i = 0; i < T; ++i) {
    double p = 0.0;
    for (int k = 0; k < 3; ++k) p = p + m.len[m.cell_edge[3 * i + k]];
    m.perim[i] = p;
  }
  return OK;
}

// ---------------------------------------------------------------------------
// HLLC flux in the edge frame (normal n, tangent t = (-ny, nx)).
// Inputs: reconstructed depths (0 means dry), normal and tangential
// velocities of both sides. Output: (mass, normal momentum, tangential
// momentum) fluxes.
// ---------------------------------------------------------------------------
template <class R>
struct Speeds { R SL, SR, Sstar; };

template <class R>
static Speeds<R> hllc_speeds(const R& hL, const R& unL, const R& hR, const R& unR, double g) {
  Speeds<R> s;
  R cL = sqrt_(g * hL);
  R cR = sqrt_(g * hR);
  if (value_of(hL) == 0.0) {          // dry left: right rarefaction into dry bed
    s.SL = unR - 2.0 * cR;
    s.SR = unR + cR;
  } else if (value_of(hR) == 0.0) {   // dry right
    s.SL = unL - cL;
    s.SR = unL + 2.0 * cL;
  } else {                             // two-rarefaction estimates
    R ustar = (unL + unR) / 2.0 + cL - cR;
    R cstar = (cL + cR) / 2.0 + (unL - unR) / 4.0;
    s.SL = vmin(unL - cL, ustar - cstar);
    s.SR = vmax(unR + cR, ustar + cstar);
  }
  s.Sstar = (s.SL * hR * (unR - s.SR) - s.SR * hL * (unL - s.SL)) /
            (hR * (unR - s.SR) - hL * (unL - s.SL));
  return s;
}

template <class R>
static void hllc_flux(const R& hL, const R& unL, const R& utL,
                      const R& hR, const R& unR, const R& utR, double g, R F[3]) {
  if (value_of(hL) == 0.0 && value_of(hR) == 0.0) {
    F[0] = R(0.0); F[1] = R(0.0); F[2] = R(0.0);
    return;
  }
  Speeds<R> s = hllc_speeds(hL, unL, hR, unR, g);
  R qL = hL * unL;
  R qR = hR * unR;
  R FL0 = qL, FL1 = qL * unL + 0.5 * g * hL * hL, FL2 = qL * utL;
  R FR0 = qR, FR1 = qR * unR + 0.5 * g * hR * hR, FR2 = qR * utR;
  if (s.SL >= R(0.0)) { F[0] = FL0; F[1] = FL1; F[2] = FL2; return; }
  if (s.SR <= R(0.0)) { F[0] = FR0; F[1] = FR1; F[2] = FR2; return; }
  F[0] = (s.SR * FL0 - s.SL * FR0 + s.SL * s.SR * (hR - hL)) / (s.SR - s.SL);
  F[1] = (s.SR * FL1 - s.SL * FR1 + s.SL * s.SR * (qR - qL)) / (s.SR - s.SL);
  F[2] = (s.Sstar >= R(0.0)) ? F[0] * utL : F[0] * utR;
}

// Per-edge result: flux out of the left cell in x-y components, and the two
// bed-pressure terms of the hydrostatic reconstruction.
template <class R>
struct EdgeOut { R F[3]; R PL, PR; };

template <class R>
static void velocity(const R& h, const R& hu, const R& hv, double h_eps, R& u, R& v) {
  if (value_of(h) > h_eps) { u = hu / h; v = hv / h; }
  else { u = R(0.0); v = R(0.0); }
}

template <class R>
static EdgeOut<R> edge_flux(const Mesh& m, const Params& p, int64_t e,
                            const R* h, const R* hu, const R* hv, const R* z) {
  const double nx = m.nx[e], ny = m.ny[e];
  const int32_t L = m.eL[e], Rc = m.eR[e];
  const bool wall = (Rc < 0);
  R hL = h[L], zL = z[L], uL, vL;
  velocity(hL, hu[L], hv[L], p.h_eps, uL, vL);
  R unL = uL * nx + vL * ny;
  R utL = vL * nx - uL * ny;
  R hR, zR, unR, utR;
  if (wall) {
    hR = hL; zR = zL; unR = -unL; utR = utL;
  } else {
    R uR, vR;
    hR = h[Rc]; zR = z[Rc];
    velocity(hR, hu[Rc], hv[Rc], p.h_eps, uR, vR);
    unR = uR * nx + vR * ny;
    utR = vR * nx - uR * ny;
  }
  // Hydrostatic reconstruction (Audusse et al. 2004).
  R zs = vmax(zL, zR);
  R hLs = vmax(R(0.0), hL + zL - zs);
  R hRs = vmax(R(0.0), hR + zR - zs);
  if (value_of(hLs) <= p.h_eps) hLs = R(0.0);
  if (value_of(hRs) <= p.h_eps) hRs = R(0.0);
  R Fn[3];
  hllc_flux(hLs, unL, utL, hRs, unR, utR, p.g, Fn);
  if (wall) { Fn[0] = R(0.0); Fn[2] = R(0.0); }
  EdgeOut<R> o;
  o.F[0] = Fn[0];
  o.F[1] = Fn[1] * nx - Fn[2] * ny;   // back from the edge frame to x-y
  o.F[2] = Fn[1] * ny + Fn[2] * nx;
  o.PL = 0.5 * p.g * (hL * hL - hLs * hLs);
  o.PR = wall ? R(0.0) : 0.5 * p.g * (hR * hR - hRs * hRs);
  return o;
}

// Contribution of face e to the residual of cell i: s * l * (F + P_side n),
// s = +1 when i is the edge's left cell, -1 otherwise (Eq. 3).
template <class R>
static void add_face(const Mesh& m, int64_t i, int32_t e, const EdgeOut<R>& o, R res[3]) {
  bool left = (m.eL[e] == i);
  R P = left ? o.PL : o.PR;
  double l = m.len[e];
  R c0 = l * o.F[0];
  R c1 = l * (o.F[1] + P * m.nx[e]);
  R c2 = l * (o.F[2] + P * m.ny[e]);
  if (left) { res[0] = res[0] + c0; res[1] = res[1] + c1; res[2] = res[2] + c2; }
  else      { res[0] = res[0] - c0; res[1] = res[1] - c1; res[2] = res[2] - c2; }
}

// Residual of cell i: its three faces summed in local edge order k = 0, 1, 2.
template <class R>
static void cell_residual(const Mesh& m, int64_t i, const std::vector<EdgeOut<R>>& fl, R res[3]) {
  res[0] = R(0.0); res[1] = R(0.0); res[2] = R(0.0);
  for (int k = 0; k < 3; ++k) {
    int32_t e = m.cell_edge[3 * i + k];
    add_face(m, i, e, fl[e], res);
  }
}

// Euler update (Eq. 4) then semi-implicit friction. Returns 1 if the depth
// went negative and was clipped to zero.
template <class R>
static int cell_update(const Mesh& m, const Params& p, int64_t i, const R& dt, const R res[3],
                       const R* h, const R* hu, const R* hv, const R* n,
                       R& h1, R& hu1, R& hv1) {
  R a = dt / m.area[i];
  R hs = h[i] - a * res[0];
  R qx = hu[i] - a * res[1];
  R qy = hv[i] - a * res[2];
  int neg = 0;
  if (value_of(hs) < 0.0) { hs = R(0.0); neg = 1; }
  if (value_of(hs) > p.h_eps) {
    R q = sqrt_(qx * qx + qy * qy);
    R fr = dt * p.g * (n[i] * n[i]) * q / (hs * hs * cbrt_(hs));
    R d = 1.0 + fr;
    qx = qx / d;
    qy = qy / d;
  } else {
    qx = R(0.0);
    qy = R(0.0);
  }
  h1 = hs; hu1 = qx; hv1 = qy;
  return neg;
}

// Host threads for the FP64 loops over edges and cells (1 = serial, the
// default). Every edge and every cell writes only its own outputs, the
// clipped-depth count is an integer sum and the CFL step a minimum, so the
// results do not depend on the thread count. Dual numbers always run serially.
static int g_threads = 1;

// Per-cell CFL ratio (Omega/P) / (|u| + sqrt(g h)); false for a dry cell.
template <class R>
static bool cfl_ratio(const Mesh& m, const Params& p, const R* h, const R* hu, const R* hv,
                      int64_t i, R& r) {
  if (!(value_of(h[i]) > p.h_eps)) return false;
  R u = hu[i] / h[i], v = hv[i] / h[i];
  R lam = sqrt_(u * u + v * v) + sqrt_(p.g * h[i]);
  r = (m.area[i] / m.perim[i]) / lam;
  return true;
}

// CFL time step from the current state; E_DRY when no cell is wet.
template <class R>
static int cfl_dt(const Mesh& m, const Params& p, const R* h, const R* hu, const R* hv, R& dt) {
  if constexpr (std::is_same<R, double>::value) {
    if (g_threads > 1) {
      // several threads: each finds the smallest ratio of its cells, then the
      // smallest of those is taken (a minimum does not depend on the order)
      double best = std::numeric_limits<double>::infinity();
      int any = 0;
#pragma omp parallel for num_threads(g_threads) reduction(min : best) reduction(max : any) schedule(static)
      for (int64_t i = 0; i < m.T; ++i) {
        double r;
        if (cfl_ratio(m, p, h, hu, hv, i, r)) {
          if (r < best) best = r;
          any = 1;
        }
      }
      if (!any) return E_DRY;
      dt = p.courant * best;
      return OK;
    }
  }
  bool any = false;
  R best(std::numeric_limits<double>::infinity());
  for (int64_t i = 0; i < m.T; ++i) {
    R r;
    if (!cfl_ratio(m, p, h, hu, hv, i, r)) continue;
    if (!any || r < best) best = r;
    any = true;
  }
  if (!any) return E_DRY;
  dt = p.courant * best;
  return OK;
}

// One explicit Euler step with a given dt: all edges, then all cells.
template <class R>
static int64_t step(const Mesh& m, const Params& p, const R& dt,
                    const R* h, const R* hu, const R* hv, const R* z, const R* n,
                    R* h1, R* hu1, R* hv1) {
  const int nt = std::is_same<R, double>::value ? g_threads : 1;
  std::vector<EdgeOut<R>> fl(m.E);
#pragma omp parallel for num_threads(nt) schedule(static)
  for (int64_t e = 0; e < m.E; ++e) fl[e] = edge_flux(m, p, e, h, hu, hv, z);
  int64_t neg = 0;
#pragma omp parallel for num_threads(nt) reduction(+ : neg) schedule(static)
  for (int64_t i = 0; i < m.T; ++i) {
    R res[3];
    cell_residual(m, i, fl, res);
    neg += cell_update(m, p, i, dt, res, h, hu, hv, n, h1[i], hu1[i], hv1[i]);
  }
  return neg;
}

}  // namespace oracle

// ===========================================================================
// C interface for the Python tests (ctypes).
// ===========================================================================
using namespace oracle;

extern "C" {

typedef struct { double g, courant, h_eps; } oracle_params;

static Params P(const oracle_params* p) { return Params{p->g, p->courant, p->h_eps}; }

// Host threads of the FP64 edge and cell loops (values < 1 mean 1).
void oracle_set_threads(int n) { g_threads = n < 1 ? 1 : n; }

void* oracle_mesh_new(const double* xy, int64_t n_nodes, const int32_t* tri, int64_t n_tris,
                      int* status) {
  Mesh* m = new Mesh();
  int s = build_mesh(xy, n_nodes, tri, n_tris, *m);
  if (status) *status = s;
  if (s != OK) { delete m; return nullptr; }
  return m;
}

void oracle_mesh_free(void* mp) { delete static_cast<Mesh*>(mp); }

// counts[0..3] = V, T, E, wall edges
void oracle_mesh_counts(const void* mp, int64_t* counts) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  counts[0] = m->V; counts[1] = m->T; counts[2] = m->E; counts[3] = m->Eb;
}

// Cell geometry: area, perimeter, oriented triangles, per-cell edge ids.
void oracle_mesh_cells(const void* mp, double* area, double* perim, int32_t* tri,
                       int32_t* cell_edge) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  if (area) std::memcpy(area, m->area.data(), sizeof(double) * m->T);
  if (perim) std::memcpy(perim, m->perim.data(), sizeof(double) * m->T);
  if (tri) std::memcpy(tri, m->tri.data(), sizeof(int32_t) * 3 * m->T);
  if (cell_edge) std::memcpy(cell_edge, m->cell_edge.data(), sizeof(int32_t) * 3 * m->T);
}

void oracle_mesh_edges(const void* mp, int32_t* L, int32_t* R, double* nx, double* ny,
                       double* len) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  std::memcpy(L, m->eL.data(), sizeof(int32_t) * m->E);
  std::memcpy(R, m->eR.data(), sizeof(int32_t) * m->E);
  std::memcpy(nx, m->nx.data(), sizeof(double) * m->E);
  std::memcpy(ny, m->ny.data(), sizeof(double) * m->E);
  std::memcpy(len, m->len.data(), sizeof(double) * m->E);
}

// Edge-frame HLLC flux for given reconstructed states (unit tests).
void oracle_hllc(double hL, double unL, double utL, double hR, double unR, double utR,
                 double g, double* F) {
  hllc_flux(hL, unL, utL, hR, unR, utR, g, F);
}

// Wave-speed estimates S_L, S_R and contact speed S* (unit tests).
void oracle_hllc_speeds(double hL, double unL, double hR, double unR, double g, double* S) {
  Speeds<double> s = hllc_speeds(hL, unL, hR, unR, g);
  S[0] = s.SL; S[1] = s.SR; S[2] = s.Sstar;
}

// Flux of one interface between two arbitrary cell states (no mesh):
// state = (h, hu, hv, z) per side, unit normal (nx, ny), wall flag.
// out = (F_h, F_hu, F_hv, PL, PR).
void oracle_interface_flux(const double* sL, const double* sR, double nx, double ny, int wall,
                           const oracle_params* p, double* out) {
  Mesh m;
  m.E = 1; m.T = wall ? 1 : 2;
  m.eL = {0}; m.eR = {wall ? -1 : 1};
  m.nx = {nx}; m.ny = {ny}; m.len = {1.0};
  double h[2] = {sL[0], sR[0]}, hu[2] = {sL[1], sR[1]}, hv[2] = {sL[2], sR[2]}, z[2] = {sL[3], sR[3]};
  EdgeOut<double> o = edge_flux(m, P(p), 0, h, hu, hv, z);
  out[0] = o.F[0]; out[1] = o.F[1]; out[2] = o.F[2]; out[3] = o.PL; out[4] = o.PR;
}

// All per-edge outputs for a state: out is 5 x E (F_h, F_hu, F_hv, PL, PR).
void oracle_edge_fluxes(const void* mp, const oracle_params* p, const double* h, const double* hu,
                        const double* hv, const double* z, double* out) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  for (int64_t e = 0; e < m->E; ++e) {
    EdgeOut<double> o = edge_flux(*m, P(p), e, h, hu, hv, z);
    out[e] = o.F[0]; out[m->E + e] = o.F[1]; out[2 * m->E + e] = o.F[2];
    out[3 * m->E + e] = o.PL; out[4 * m->E + e] = o.PR;
  }
}

int oracle_cfl_dt(const void* mp, const oracle_params* p, const double* h, const double* hu,
                  const double* hv, double* dt) {
  return cfl_dt(*static_cast<const Mesh*>(mp), P(p), h, hu, hv, *dt);
}

double oracle_mass(const void* mp, const double* h) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  double s = 0.0;
  for (int64_t i = 0; i < m->T; ++i) s = s + m->area[i] * h[i];
  return s;
}

// One step with the given dt; state arrays updated in place. Returns the
// number of cells whose depth was clipped at zero.
int64_t oracle_step(const void* mp, const oracle_params* p, double dt, double* h, double* hu,
                    double* hv, const double* z, const double* n) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  std::vector<double> h1(m->T), hu1(m->T), hv1(m->T);
  int64_t neg = step(*m, P(p), dt, h, hu, hv, z, n, h1.data(), hu1.data(), hv1.data());
  std::memcpy(h, h1.data(), sizeof(double) * m->T);
  std::memcpy(hu, hu1.data(), sizeof(double) * m->T);
  std::memcpy(hv, hv1.data(), sizeof(double) * m->T);
  return neg;
}

// n_steps CFL steps (no end time). dts[k] receives the k-th dt if non-null.
// Returns OK or E_DRY; *neg accumulates clipped-depth counts.
int oracle_run(const void* mp, const oracle_params* p, int64_t n_steps, double* h, double* hu,
               double* hv, const double* z, const double* n, double* dts, int64_t* neg) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  Params pp = P(p);
  std::vector<double> h1(m->T), hu1(m->T), hv1(m->T);
  int64_t negs = 0;
  for (int64_t s = 0; s < n_steps; ++s) {
    double dt;
    int st = cfl_dt(*m, pp, h, hu, hv, dt);
    if (st != OK) { if (neg) *neg = negs; return st; }
    if (dts) dts[s] = dt;
    negs += step(*m, pp, dt, h, hu, hv, z, n, h1.data(), hu1.data(), hv1.data());
    std::memcpy(h, h1.data(), sizeof(double) * m->T);
    std::memcpy(hu, hu1.data(), sizeof(double) * m->T);
    std::memcpy(hv, hv1.data(), sizeof(double) * m->T);
  }
  if (neg) *neg = negs;
  return OK;
}

// Steps from time *t until t == t_end: dt = min(CFL dt, t_end - t), and the
// step that reaches t_end sets t = t_end exactly. Stops early (E_INVAL) after
// max_steps. *n_steps receives the number of steps taken.
int oracle_advance(const void* mp, const oracle_params* p, double t_end, int64_t max_steps,
                   double* h, double* hu, double* hv, const double* z, const double* n,
                   double* t, int64_t* n_steps, int64_t* neg) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  Params pp = P(p);
  std::vector<double> h1(m->T), hu1(m->T), hv1(m->T);
  int64_t k = 0, negs = 0;
  int st = OK;
  while (*t < t_end) {
    if (k >= max_steps) { st = E_INVAL; break; }
    double dt;
    st = cfl_dt(*m, pp, h, hu, hv, dt);
    if (st != OK) break;
    double rest = t_end - *t;
    bool last = (dt >= rest);
    if (last) dt = rest;
    negs += step(*m, pp, dt, h, hu, hv, z, n, h1.data(), hu1.data(), hv1.data());
    std::memcpy(h, h1.data(), sizeof(double) * m->T);
    std::memcpy(hu, hu1.data(), sizeof(double) * m->T);
    std::memcpy(hv, hv1.data(), sizeof(double) * m->T);
    *t = last ? t_end : (*t + dt);
    ++k;
  }
  if (n_steps) *n_steps = k;
  if (neg) *neg = negs;
  return st;
}

// Forward-mode derivative of n_steps steps with the PRESCRIBED time steps
// dts[0 .. n_steps) (the dt sequence is data, not a function of the state).
// (h, hu, hv) are advanced in place; (dh, dhu, dhv) carry the tangent of the
// initial state in and the tangent of the final state out; dz and dn are the
// tangents of the bed and of Manning's n (NULL = zero). If gauges is given,
// gauge_h[k * n_gauges + j] and gauge_dh[...] receive h and its tangent at
// cell gauges[j] after step k + 1 (either may be NULL). Every step is the
// plain step above instantiated on a one-direction dual number, so the
// derivative follows the branch each comparison takes (Sec. 2.2 scheme,
// differentiated piecewise).
int64_t oracle_run_tangent(const void* mp, const oracle_params* p, int64_t n_steps,
                           const double* dts, double* h, double* hu, double* hv, const double* z,
                           const double* n, double* dh, double* dhu, double* dhv,
                           const double* dz, const double* dn, const int32_t* gauges,
                           int64_t n_gauges, double* gauge_h, double* gauge_dh) {
  using D = Dual<1>;
  const Mesh* m = static_cast<const Mesh*>(mp);
  Params pp = P(p);
  const int64_t T = m->T;
  std::vector<D> H(T), HU(T), HV(T), Z(T), NN(T), H1(T), HU1(T), HV1(T);
  for (int64_t i = 0; i < T; ++i) {
    H[i] = D(h[i]); H[i].d[0] = dh[i];
    HU[i] = D(hu[i]); HU[i].d[0] = dhu[i];
    HV[i] = D(hv[i]); HV[i].d[0] = dhv[i];
    Z[i] = D(z[i]); Z[i].d[0] = dz ? dz[i] : 0.0;
    NN[i] = D(n[i]); NN[i].d[0] = dn ? dn[i] : 0.0;
  }
  int64_t negs = 0;
  for (int64_t k = 0; k < n_steps; ++k) {
    negs += step(*m, pp, D(dts[k]), H.data(), HU.data(), HV.data(), Z.data(), NN.data(),
                 H1.data(), HU1.data(), HV1.data());
    H.swap(H1); HU.swap(HU1); HV.swap(HV1);
    for (int64_t j = 0; j < n_gauges; ++j) {
      const D& v = H[gauges[j]];
      if (gauge_h) gauge_h[k * n_gauges + j] = v.v;
      if (gauge_dh) gauge_dh[k * n_gauges + j] = v.d[0];
    }
  }
  for (int64_t i = 0; i < T; ++i) {
    h[i] = H[i].v; hu[i] = HU[i].v; hv[i] = HV[i].v;
    dh[i] = H[i].d[0]; dhu[i] = HU[i].d[0]; dhv[i] = HV[i].d[0];
  }
  return negs;
}

// n_steps steps with the prescribed time steps dts (plain values; the
// finite-difference side of the derivative checks). Gauges as above.
int64_t oracle_run_dts(const void* mp, const oracle_params* p, int64_t n_steps, const double* dts,
                       double* h, double* hu, double* hv, const double* z, const double* n,
                       const int32_t* gauges, int64_t n_gauges, double* gauge_h) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  Params pp = P(p);
  std::vector<double> h1(m->T), hu1(m->T), hv1(m->T);
  int64_t negs = 0;
  for (int64_t k = 0; k < n_steps; ++k) {
    negs += step(*m, pp, dts[k], h, hu, hv, z, n, h1.data(), hu1.data(), hv1.data());
    std::memcpy(h, h1.data(), sizeof(double) * m->T);
    std::memcpy(hu, hu1.data(), sizeof(double) * m->T);
    std::memcpy(hv, hv1.data(), sizeof(double) * m->T);
    for (int64_t j = 0; j < n_gauges; ++j)
      if (gauge_h) gauge_h[k * n_gauges + j] = h[gauges[j]];
  }
  return negs;
}

// Updated state of selected cells only, for one step of length dt from the
// given state (used to check full-size runs cell by cell). out is 3 x m.
void oracle_cells_after_step(const void* mp, const oracle_params* p, double dt, const double* h,
                             const double* hu, const double* hv, const double* z, const double* n,
                             const int64_t* cells, int64_t count, double* out) {
  const Mesh* m = static_cast<const Mesh*>(mp);
  Params pp = P(p);
  for (int64_t j = 0; j < count; ++j) {
    int64_t i = cells[j];
    // Fluxes of the cell's three faces only.
    double res[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
      int32_t e = m->cell_edge[3 * i + k];
      add_face(*m, i, e, edge_flux(*m, pp, e, h, hu, hv, z), res);
    }
    double h1, hu1, hv1;
    cell_update(*m, pp, i, dt, res, h, hu, hv, n, h1, hu1, hv1);
    out[j] = h1; out[count + j] = hu1; out[2 * count + j] = hv1;
  }
}

}  // extern "C"
