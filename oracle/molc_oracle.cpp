// TEST INFRASTRUCTURE ONLY — the oracle.
//
// A plain, slow, CPU-only implementation of the high-order sweep of the method of long characteristics
// (Coale & Anistratov, "Multilevel method for thermal radiative transfer problems with method of long
// characteristics for the Boltzmann transport equation", Sec. 3).  Only the tests, the smoke check and the
// benchmark's CPU-baseline leg may load this library.  It shares no code, header or table with the CUDA
// library; both sides only consume the same seeded input arrays.
//
// Everything is templated on the real type R and instantiated twice: R = double, and R = IEEE binary128
// (__float128 with libquadmath on x86-64, long double on AArch64).  The binary128 instance is the reference
// the GPU paths are checked against; the double instance is the timed CPU baseline.
//
// What it computes, in the paper's order and notation (Sec. 3):
//   * characteristic grid: for each direction, parallel characteristics of width w_k, cut into segments at
//     every crossing with a material-cell boundary; l is the in-plane segment length (Sec. 3, paragraph
//     on the construction of the characteristic grid; reading: l is measured in the x-y plane and the 3D
//     path is l / sin(zeta), which is the only reading consistent with Eq. (13));
//   * per segment: kappa~ = kappa + 1/(c dt), Q = kappa B + I^{n-1}/(c dt)                  (Eq. 11)
//                  tau = kappa~ l / sin(zeta), alpha = 1/tau - e^-tau / (1 - e^-tau)       (Eq. 13)
//                  I_{s+1} = I_s e^-tau + (Q/kappa~)(1 - e^-tau), Ibar = alpha I_s + (1-alpha) I_{s+1}  (Eq. 12)
//                  A = l w                                                                 (Eq. 14)
//   * cell moments with weights omega_m A: E = (1/c) int I dOmega, F = int Omega I dOmega (Sec. 2, after
//     Eq. 4) and the Eddington-tensor numerator int Omega Omega I dOmega (Eq. 7 / Eq. 15), all cell averages.
// Readings where the paper is silent: I^{n-1} in Q is the previous step's segment average on the same
// segment, direction and group; the cell tensor of Eq. (15) uses the segment average Ibar; each direction
// with mu > 0 also stands for its mirror through the x-y plane (weights sum to 4 pi).  The characteristic grid
// is defined by its double-precision evaluation: the unit direction (c, s) / sqrt(c^2 + s^2), the grid lines
// x0 + i lx/nx, the characteristic offsets and widths are formed in double (this file is compiled without
// FMA contraction), and a direction and its opposite share the same lines; the crossings, segment lengths and
// everything after are then evaluated in R.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

#if defined(__aarch64__)
typedef long double real128;  // IEEE binary128 on AArch64 Linux
static inline real128 q_exp(real128 x) { return expl(x); }
static inline real128 q_expm1(real128 x) { return expm1l(x); }
static inline real128 q_sqrt(real128 x) { return sqrtl(x); }
static inline real128 q_floor(real128 x) { return floorl(x); }
static inline real128 q_ceil(real128 x) { return ceill(x); }
#else
extern "C" {
#include <quadmath.h>
}
typedef __float128 real128;
static inline real128 q_exp(real128 x) { return expq(x); }
static inline real128 q_expm1(real128 x) { return expm1q(x); }
static inline real128 q_sqrt(real128 x) { return sqrtq(x); }
static inline real128 q_floor(real128 x) { return floorq(x); }
static inline real128 q_ceil(real128 x) { return ceilq(x); }
#endif

template <class R> struct Fn;
template <> struct Fn<double> {
  static double exp(double x) { return std::exp(x); }
  static double expm1(double x) { return std::expm1(x); }
  static double sqrt(double x) { return std::sqrt(x); }
  static double floor(double x) { return std::floor(x); }
  static double ceil(double x) { return std::ceil(x); }
};
template <> struct Fn<real128> {
  static real128 exp(real128 x) { return q_exp(x); }
  static real128 expm1(real128 x) { return q_expm1(x); }
  static real128 sqrt(real128 x) { return q_sqrt(x); }
  static real128 floor(real128 x) { return q_floor(x); }
  static real128 ceil(real128 x) { return q_ceil(x); }
};
template <class R> static inline R rabs(R x) { return x < 0 ? -x : x; }

extern "C" {
// Problem geometry and angular quadrature, as plain arrays (host memory).
typedef struct {
  int nx, ny;                 // material cells; cell index = iy * nx + ix
  double x0, y0, lx, ly;      // domain [x0, x0+lx] x [y0, y0+ly], cm
  int ndir;                   // directions with mu > 0
  const double *mu;           // cos(zeta)
  const double *cos_phi;      // in-plane direction (normalised here)
  const double *sin_phi;
  const double *w;            // omega_m, sum 4 pi
  double spacing;             // h_moc: ray spacing (uniform layout) or maximum width (paper layout)
  int layout;                 // 0: uniform parallel rays, 1: paper's vertex-band construction
  int renorm;                 // 1: scale areas so that sum_{C(i,m)} A = V_i
} oracle_geom;

// Rounding-error model of a sweep that carries the deviation psi = I - B_cell along each characteristic (the
// form the GPU paths compute Eq. 12 in), for a first-order running error bound (test infrastructure: it bounds the
// arithmetic of a path, it is not part of the method).  path 0: every operation in a precision of unit roundoff u
// with exp and expm1 of relative error <= e_exp; path 1: FP32 operations (unit roundoff u) with the exponential
// formed as 2^x by an approximation of relative error <= e_exp and 1/x of relative error <= e_rcp, the average
// E1 = (1 - e^-tau)/tau below tau = 1/2 taken as e^-tau/2 sinh(tau/2)/(tau/2) by its series to the (tau/2)^6 term.
// k_sum: roundings of relative u a moment term passes through on its way into the cell sums, beyond those of its
// segment average (path 1; path 0 sums terms one by one in any order, bounded by gamma_{n-1} per cell).
// abs_unit: the absolute error of one operation whose result falls below the path's normal range (FP32 in scaled
// units: 2^-126 divided by the state's scale), added for every operation of a segment.
typedef struct {
  int path;
  double u, e_exp, e_rcp, k_sum, abs_unit;
  const double *Bref;         // [G][ncell] Planck intensity the path's stored deviations refer to, or NULL (= B)
} oracle_errmodel;
}

enum { EDGE_L = 0, EDGE_R = 1, EDGE_B = 2, EDGE_T = 3 };

// One characteristic of one direction.
template <class R> struct Ray {
  R width;
  int entry;                  // edge the characteristic enters through
  std::vector<int> cell;      // segments in traversal order
  std::vector<int> face;      // face each segment enters through (its upwind face; numbering in face_of)
  std::vector<R> len;         // in-plane length l
  std::vector<R> area;        // A = l w (after optional renormalisation)
};

template <class R> struct Dir {
  R dx, dy;                   // unit in-plane direction
  std::vector<Ray<R>> rays;   // ordered by increasing offset along n = (-dy, dx)
};

// Offsets t (along the normal n) and widths of the characteristics of one direction (Sec. 3, construction of
// the characteristic grid; uniform spacing or the vertex bands halved to h_moc, reading c4).
// (evaluated in double: part of the definition of the characteristic grid)
static void characteristic_offsets(const oracle_geom &g, double dx, double dy, std::vector<double> &t,
                                   std::vector<double> &w) {
  const double x0 = g.x0, y0 = g.y0, x1 = g.x0 + g.lx, y1 = g.y0 + g.ly;
  auto proj = [&](double x, double y) { return -dy * x + dx * y; };
  t.clear();
  w.clear();
  if (g.layout == 0) {
    double c[4] = {proj(x0, y0), proj(x1, y0), proj(x0, y1), proj(x1, y1)};
    double tmin = c[0], tmax = c[0];
    for (int i = 1; i < 4; ++i) { tmin = std::min(tmin, c[i]); tmax = std::max(tmax, c[i]); }
    double Lp = tmax - tmin;
    long n = (long)std::ceil(Lp / g.spacing - 1e-9);
    if (n < 1) n = 1;
    double wk = Lp / (double)n;
    for (long k = 0; k < n; ++k) { t.push_back(tmin + ((double)k + 0.5) * wk); w.push_back(wk); }
    return;
  }
  // Paper layout: project every vertex of the material grid onto n; each gap between consecutive distinct
  // projections is one initial characteristic (it contains no vertex).  Halve until w <= h_moc.
  const double hx = g.lx / g.nx, hy = g.ly / g.ny;
  std::vector<double> v;
  v.reserve((size_t)(g.nx + 1) * (g.ny + 1));
  for (int b = 0; b <= g.ny; ++b)
    for (int a = 0; a <= g.nx; ++a) v.push_back(proj(g.x0 + a * hx, g.y0 + b * hy));
  std::sort(v.begin(), v.end());
  const double Lp = v.back() - v.front();
  const double merge = 1e-13 * Lp;
  std::vector<double> u;
  for (double x : v)
    if (u.empty() || x - u.back() > merge) u.push_back(x);
  for (size_t i = 0; i + 1 < u.size(); ++i) {
    double gap = u[i + 1] - u[i];
    long pieces = 1;
    while (gap / (double)pieces > g.spacing) pieces *= 2;
    double wk = gap / (double)pieces;
    for (long p = 0; p < pieces; ++p) { t.push_back(u[i] + ((double)p + 0.5) * wk); w.push_back(wk); }
  }
}

// Cut the line {p : p.n = t} into segments at every crossing with a grid line (Sec. 3).  Crossing
// parameters closer than eps are one crossing (the characteristic passes through a vertex); the cell of a
// segment is the cell holding its midpoint.
template <class R>
static bool trace(const oracle_geom &g, R dx, R dy, R t, R width, Ray<R> &ray) {
  const double hxd = g.lx / g.nx, hyd = g.ly / g.ny;
  const R hx = hxd, hy = hyd;
  const R x0 = g.x0, y0 = g.y0, x1 = g.x0 + g.lx, y1 = g.y0 + g.ly;
  const R eps = R(1e-12) * std::min(hx, hy);
  // p(u) = t n + u d with n = (-dy, dx): x(u) = -t dy + u dx, y(u) = t dx + u dy
  const R bx = -t * dy, by = t * dx;
  R ulo = R(-1e300), uhi = R(1e300);
  R ux = R(-1e300), uy = R(-1e300);
  if (dx != R(0)) {
    R a = (x0 - bx) / dx, b = (x1 - bx) / dx;
    if (a > b) std::swap(a, b);
    ux = a;
    ulo = std::max(ulo, a);
    uhi = std::min(uhi, b);
  } else if (bx < x0 || bx > x1) {
    return false;
  }
  if (dy != R(0)) {
    R a = (y0 - by) / dy, b = (y1 - by) / dy;
    if (a > b) std::swap(a, b);
    uy = a;
    ulo = std::max(ulo, a);
    uhi = std::min(uhi, b);
  } else if (by < y0 || by > y1) {
    return false;
  }
  if (uhi - ulo <= eps) return false;
  // Entry edge: the boundary whose entry parameter is the larger; on a tie, the vertical (x) edge.
  bool xedge = (dy == R(0)) || (dx != R(0) && ux >= uy - eps);
  ray.entry = xedge ? (dx > R(0) ? EDGE_L : EDGE_R) : (dy > R(0) ? EDGE_B : EDGE_T);
  std::vector<R> cut;
  cut.push_back(ulo);
  if (dx != R(0))
    for (int i = 1; i < g.nx; ++i) {
      R u = (R(g.x0 + i * hxd) - bx) / dx;
      if (u > ulo && u < uhi) cut.push_back(u);
    }
  if (dy != R(0))
    for (int j = 1; j < g.ny; ++j) {
      R u = (R(g.y0 + j * hyd) - by) / dy;
      if (u > ulo && u < uhi) cut.push_back(u);
    }
  cut.push_back(uhi);
  std::sort(cut.begin(), cut.end());
  ray.width = width;
  ray.cell.clear();
  ray.len.clear();
  ray.area.clear();
  for (size_t i = 0; i + 1 < cut.size(); ++i) {
    R a = cut[i], b = cut[i + 1];
    if (b - a <= eps) continue;
    R m = R(0.5) * (a + b);
    long ix = (long)Fn<R>::floor((bx + m * dx - x0) / hx);
    long iy = (long)Fn<R>::floor((by + m * dy - y0) / hy);
    ix = std::min<long>(std::max<long>(ix, 0), g.nx - 1);
    iy = std::min<long>(std::max<long>(iy, 0), g.ny - 1);
    ray.cell.push_back((int)(iy * g.nx + ix));
    ray.len.push_back(b - a);
    ray.area.push_back((b - a) * width);
  }
  // Upwind face of every segment (Sec. 3, Eq. 16): the first enters through the entry edge; the others through
  // the face shared with the previous segment's cell.  Faces: x-face (i, j) = the line x = x0 + i hx in row j,
  // numbered j (nx + 1) + i; y-face (i, j) = the line y = y0 + j hy in column i, numbered (nx + 1) ny + j nx + i.
  // A characteristic through a vertex (a diagonal step) is counted on the x-face of the cell it enters.
  ray.face.clear();
  const int nxf = (g.nx + 1) * g.ny;
  for (size_t s = 0; s < ray.cell.size(); ++s) {
    const int ix = ray.cell[s] % g.nx, iy = ray.cell[s] / g.nx;
    int f;
    if (s == 0) {
      f = ray.entry == EDGE_L ? iy * (g.nx + 1) : ray.entry == EDGE_R ? iy * (g.nx + 1) + g.nx
        : ray.entry == EDGE_B ? nxf + ix : nxf + g.ny * g.nx + ix;
    } else {
      const int px = ray.cell[s - 1] % g.nx, py = ray.cell[s - 1] / g.nx;
      f = px != ix ? iy * (g.nx + 1) + std::max(px, ix) : nxf + std::max(py, iy) * g.nx + ix;
    }
    ray.face.push_back(f);
  }
  return !ray.cell.empty();
}

// Unit in-plane direction (cos phi, sin phi) of direction m (Sec. 3; quadrature of reading c9).
// (evaluated in double: part of the definition of the characteristic grid)
static void unit_dir(const oracle_geom &g, int m, double &dx, double &dy) {
  const double c = g.cos_phi[m], s = g.sin_phi[m];
  const double n = std::sqrt(c * c + s * s);
  dx = c / n;
  dy = s / n;
}

// The characteristics of one in-plane direction with their segments (cells, in-plane lengths l, areas A = l w of
// Eq. 14, entry edges), Sec. 3.
template <class R> static int build_dir(const oracle_geom &g, int m, Dir<R> &d) {
  double dxd, dyd;
  unit_dir(g, m, dxd, dyd);
  d.dx = dxd;
  d.dy = dyd;
  // A characteristic is a line: the direction and its opposite share the same lines.  The lines are built for
  // the sense with sin > 0 (or sin = 0, cos > 0); for the opposite sense the offsets along n = (-dy, dx) are
  // their exact negations, in reverse order (increasing offset again).
  std::vector<double> t, w;
  const bool minus = dyd < 0 || (dyd == 0 && dxd < 0);
  if (!minus) {
    characteristic_offsets(g, dxd, dyd, t, w);
  } else {
    std::vector<double> tp, wp;
    characteristic_offsets(g, -dxd, -dyd, tp, wp);
    for (size_t k = tp.size(); k-- > 0;) {
      t.push_back(-tp[k]);
      w.push_back(wp[k]);
    }
  }
  d.rays.clear();
  for (size_t k = 0; k < t.size(); ++k) {
    Ray<R> r;
    if (trace<R>(g, d.dx, d.dy, R(t[k]), R(w[k]), r)) d.rays.push_back(std::move(r));
  }
  if (g.renorm) {
    const R V = R(g.lx / g.nx) * R(g.ly / g.ny);
    std::vector<R> sum((size_t)g.nx * g.ny, R(0));
    for (auto &r : d.rays)
      for (size_t s = 0; s < r.cell.size(); ++s) sum[r.cell[s]] += r.area[s];
    for (size_t i = 0; i < sum.size(); ++i)
      if (!(sum[i] > R(0))) return -3;  // a cell no characteristic of this direction crosses
    for (auto &r : d.rays)
      for (size_t s = 0; s < r.cell.size(); ++s) r.area[s] = r.area[s] * (V / sum[r.cell[s]]);
  }
  return 0;
}

// Argument checks of the geometry (no counterpart in the paper).
static int check_geom(const oracle_geom *g) {
  if (!g || g->nx < 1 || g->ny < 1 || !(g->lx > 0) || !(g->ly > 0) || g->ndir < 1 || !(g->spacing > 0)) return -1;
  if (!g->mu || !g->cos_phi || !g->sin_phi || !g->w) return -1;
  for (int m = 0; m < g->ndir; ++m) {
    if (!(g->mu[m] > 0 && g->mu[m] <= 1)) return -1;
    if (g->cos_phi[m] == 0 && g->sin_phi[m] == 0) return -1;
  }
  return 0;
}

// Geometry is identical for directions with the same in-plane direction; build it once per distinct one.
template <class R> struct Geometry {
  std::vector<Dir<R>> dirs;        // distinct in-plane directions
  std::vector<int> of;             // direction m -> index into dirs
  int build(const oracle_geom &g) {
    of.assign(g.ndir, -1);
    for (int m = 0; m < g.ndir; ++m) {
      for (int j = 0; j < m; ++j)
        if (g.cos_phi[j] == g.cos_phi[m] && g.sin_phi[j] == g.sin_phi[m]) { of[m] = of[j]; break; }
      if (of[m] >= 0) continue;
      of[m] = (int)dirs.size();
      dirs.emplace_back();
      int rc = build_dir<R>(g, m, dirs.back());
      if (rc) return rc;
    }
    return 0;
  }
};

// Segment counts per direction (canonical order: direction m, then its characteristics by increasing
// offset along n = (-dy, dx), then segments in traversal order); bookkeeping, no counterpart in the paper.
template <class R> static void canonical_offsets(const oracle_geom &g, const Geometry<R> &geo,
                                                 std::vector<int64_t> &seg_dir_off) {
  seg_dir_off.assign(g.ndir + 1, 0);
  for (int m = 0; m < g.ndir; ++m) {
    int64_t n = 0;
    for (auto &r : geo.dirs[geo.of[m]].rays) n += (int64_t)r.cell.size();
    seg_dir_off[m + 1] = seg_dir_off[m] + n;
  }
}

// Moments accumulated per block of directions (fixed blocks, merged in block order: results do not depend
// on the number of threads).
enum { MOM_D = 0, MOM_FX, MOM_FY, MOM_NXX, MOM_NXY, MOM_NYY, MOM_NZZ, MOM_AFX, MOM_AFY, MOM_ANXY, MOM_BNXY, MOM_BFX,
       MOM_BFY, N_MOM };
// With an error model: per cell, for each of the six outputs k (D, Fx, Fy, Nxx, Nxy, Nyy) the sum of
// omega A |factor_k| times the bound of the term's segment average (ERR), the magnitude of the deviation terms
// omega A |factor_k| |Ibar - B| (DEV) and of the Planck terms omega A |factor_k| B (PLK), and the term count.
enum { ERR0 = 0, DEV0 = 6, PLK0 = 12, ECNT = 18, N_ERR = 19 };

// First-order bound of the errors of one segment's computed segment-average deviation (bar) and outgoing
// deviation (out) under an error model, from the magnitudes of the exact values: tau, e = e^-tau, om = 1 - e^-tau,
// E1 = om / tau, x = psi_in - d, pbar = Ibar - B, pout = I_out - B, the bounds eps_in of psi_in and eps_d of
// d = S - B, and mu = cos(zeta).  The path computes pbar = d + x E1, and pout = psi_in - x om below tau = 1/2 and
// d + x e above (each a fused multiply-add): pbar carries E1 eps_in + (1 - E1) eps_d, pout e eps_in + om eps_d,
// plus the roundings of x, of the product's factor (relative bound r*) and of the result.  Near tau = 1/2 the path
// may take either form; the larger bound is kept.
struct SegBound {
  double bar, out;
};
static SegBound segment_bound(const oracle_errmodel &em, double tau, double e, double om, double E1, double x,
                              double pbar, double pout, double eps_in, double eps_d, double mu) {
  const double u = em.u;
  const bool may_thin = tau < 0.5 * (1 + 1e-4), may_thick = tau >= 0.5 * (1 - 1e-4);
  double rE1 = 0, rom = 0, re = 0;
  if (em.path == 1) {
    // a = tau/2 from four FP32 roundings of its factors and two products: 5u; 2^(-a log2 e) with the argument
    // rounded twice more: relative error 7u a + e_exp; e^-tau = h^2
    const double rh = 3.5 * u * tau + em.e_exp;
    re = 2 * rh + u;
    const double rhp = rh + 4 * u + u + 5e-11;   // series in FP32 FMAs (4u), product h p (u), truncation
    const double r1me = u + (om > 0 ? e / om : 0.0) * re;
    const double ritau = 5 * u + em.e_rcp;        // 1/tau = sin(zeta) rcp(kappa~ l): 3u + e_rcp + 2u
    const double rE1_thin = rhp, rE1_thick = r1me + ritau + u;
    rE1 = std::max(may_thin ? rE1_thin : 0.0, may_thick ? rE1_thick : 0.0);
    rom = 5 * u + rhp + u;                        // om = (a + a) h p
  } else {
    // tau = kappa~ l / sin(zeta): kappa~ 3u, l u, 1/sin(zeta) from sqrt(1 - mu^2) in the path's precision
    const double rtau = (9.0 + mu * mu / (1.0 - mu * mu)) * u;
    rom = rtau + em.e_exp;                        // -expm1(-tau): argument sensitivity <= rtau
    re = tau * rtau + em.e_exp;
    rE1 = rom + rtau + u;
  }
  SegBound b;
  const double au = 16 * em.abs_unit;   // results below the normal range: the operations of one segment
  b.bar = E1 * eps_in + (1 - E1) * eps_d + E1 * u * x + x * E1 * rE1 + u * pbar + au;
  const double out_thin = e * eps_in + om * eps_d + om * u * x + x * om * rom + u * pout + au;
  const double out_thick = e * eps_in + om * eps_d + e * u * x + x * e * re + u * pout + au;
  b.out = std::max(may_thin ? out_thin : 0.0, may_thick ? out_thick : 0.0);
  return b;
}

template <class R>
static void sweep_direction(const oracle_geom &g, const Geometry<R> &geo, int m, int gi, int G, int gsel,
                            const double *kappa, const double *B, R inv_cdt, const double *bnd,
                            const double *I_prev, int64_t seg0, double *I_new, double *I_exit, int64_t ray0,
                            int Gsub, int store_dev, int prev_dev, std::vector<R> *acc, std::vector<R> *facc,
                            const oracle_errmodel *em, const double *Ierr_prev, double *Ierr_new,
                            std::vector<double> *eacc) {
  const Dir<R> &d = geo.dirs[geo.of[m]];
  const int64_t ncell = (int64_t)g.nx * g.ny;
  const R mu = g.mu[m];
  const R sinz = Fn<R>::sqrt(R(1) - mu * mu);
  const R om = g.w[m];
  const R Ox = sinz * d.dx, Oy = sinz * d.dy;
  const double *kap = kappa + (int64_t)gsel * ncell;
  const double *Bg = B + (int64_t)gsel * ncell;
  const double *Brg = em && em->Bref ? em->Bref + (int64_t)gsel * ncell : Bg;
  // error model: magnitudes of the angular factors of the six outputs, and (path 0) the roundings of the
  // factors omega (A/V) Omega.. that multiply each segment average on its way into the sums
  const double mud = (double)mu, oxd = std::fabs((double)Ox), oyd = std::fabs((double)Oy);
  const double fk[6] = {1.0, oxd, oyd, oxd * oxd, oxd * oyd, oyd * oyd};
  const double kterm = em && em->path == 0 ? 16.0 + 2.0 * mud * mud / (1.0 - mud * mud) : 0.0;
  int64_t seg = seg0;
  for (size_t k = 0; k < d.rays.size(); ++k) {
    const Ray<R> &r = d.rays[k];
    R I = bnd[r.entry * G + gsel];                 // I_{k,1}: isotropic incoming boundary intensity
    double eps_out = 0.0, b_prev = (double)I;      // error model: bound of the outgoing deviation; B before
    for (size_t s = 0; s < r.cell.size(); ++s, ++seg) {
      const int i = r.cell[s];
      const R kap_i = kap[i];
      const R B_i = Bg[i];
      const R Iprev = I_prev ? (prev_dev ? B_i + R(I_prev[seg * Gsub + gi]) : R(I_prev[seg * Gsub + gi])) : B_i;
      const R kt = kap_i + inv_cdt;                                 // Eq. (11)
      const R Q = kap_i * B_i + inv_cdt * Iprev;                    // Eq. (11)
      const R tau = kt * r.len[s] / sinz;                           // Eq. (13)
      const R one_m_e = -Fn<R>::expm1(-tau);                        // 1 - e^-tau
      const R e = Fn<R>::exp(-tau);
      const R Iout = I * e + (Q / kt) * one_m_e;                    // Eq. (12)
      const R alpha = R(1) / tau - e / one_m_e;                     // Eq. (13)
      const R Ibar = alpha * I + (R(1) - alpha) * Iout;             // Eq. (12)
      if (em) {
        // running error bound of the path's deviation-form evaluation of this segment (see segment_bound);
        // all quantities are magnitudes of the exact values, formed from this oracle's own
        const double u = em->u, Bc = (double)B_i, Br = Brg[i];
        const double jump = std::fabs(b_prev - Bc);
        const double psi_in = (double)(I - B_i);
        // the step of B the path adds at the crossing (FP32: B in two words, 2^-48 of each B)
        const double ej = (em->path == 1 ? 2 * u * jump + 4 * u * u * (std::fabs(b_prev) + Bc) : u * jump) +
                          4 * em->abs_unit;
        const double eps_in = s == 0 ? ej : eps_out + ej + u * std::fabs(psi_in);
        const double rr = (double)(inv_cdt / kt);                   // 1 / (c dt kappa~)
        const double dstate = (double)Iprev - Br;                   // the path's stored deviation
        const double eps_state = Ierr_prev ? Ierr_prev[seg * Gsub + gi] : 0.0;
        const double dd = (double)(Q / kt - B_i);
        const double eps_d = (em->path == 1
            ? u * (3 * std::fabs(dstate * rr) + 5 * std::fabs((Br - Bc) * rr) + std::fabs(dd)) + rr * eps_state
            : u * rr * (std::fabs(Br - Bc) + 8 * std::fabs((double)Iprev - Bc)) + rr * eps_state) +
                             4 * em->abs_unit;
        const double taud = (double)tau, ed = (double)e, omd = (double)one_m_e;
        const double pbar = (double)(Ibar - B_i);
        const SegBound sb = segment_bound(*em, taud, ed, omd, omd / taud, std::fabs((double)(I - Q / kt)),
                                          std::fabs(pbar), std::fabs((double)(Iout - B_i)), eps_in, eps_d, mud);
        eps_out = sb.out;
        b_prev = Bc;
        const double wA = (double)(om * r.area[s]);
        double *ea = eacc->data();
        for (int q = 0; q < 6; ++q) {
          ea[(ERR0 + q) * ncell + i] += wA * fk[q] * (sb.bar + kterm * u * std::fabs(pbar));
          ea[(DEV0 + q) * ncell + i] += wA * fk[q] * std::fabs(pbar);
          ea[(PLK0 + q) * ncell + i] += wA * fk[q] * Bc;
        }
        ea[ECNT * ncell + i] += 1.0;
        // the bound of the path's stored deviation, plus this oracle's rounding of its own to double
        if (Ierr_new) Ierr_new[seg * Gsub + gi] = sb.bar + 0x1p-53 * std::fabs(pbar);
      }
      if (facc) {   // Eq. (16): omega_m w_k times the intensity at the segment's upwind face
        const int64_t nf = (int64_t)(g.nx + 1) * g.ny + (int64_t)g.nx * (g.ny + 1);
        const int f = r.face[s];
        const R ww = om * r.width;
        R *fa = facc->data();
        fa[MOM_D * nf + f] += ww * I;
        fa[MOM_FX * nf + f] += ww * Ox * I;
        fa[MOM_FY * nf + f] += ww * Oy * I;
        fa[MOM_NXX * nf + f] += ww * Ox * Ox * I;
        fa[MOM_NXY * nf + f] += ww * Ox * Oy * I;
        fa[MOM_NYY * nf + f] += ww * Oy * Oy * I;
      }
      const R wA = om * r.area[s];                                  // omega_m A_{k,s}, Eq. (14)-(15)
      const R dev = rabs(Ibar - B_i);
      R *a = acc->data();
      a[MOM_D * ncell + i] += wA * Ibar;
      a[MOM_FX * ncell + i] += wA * Ox * Ibar;
      a[MOM_FY * ncell + i] += wA * Oy * Ibar;
      a[MOM_NXX * ncell + i] += wA * Ox * Ox * Ibar;
      a[MOM_NXY * ncell + i] += wA * Ox * Oy * Ibar;
      a[MOM_NYY * ncell + i] += wA * Oy * Oy * Ibar;
      a[MOM_NZZ * ncell + i] += wA * mu * mu * Ibar;
      a[MOM_AFX * ncell + i] += wA * rabs(Ox) * dev;
      a[MOM_AFY * ncell + i] += wA * rabs(Oy) * dev;
      a[MOM_ANXY * ncell + i] += wA * rabs(Ox * Oy) * dev;
      a[MOM_BNXY * ncell + i] += wA * rabs(Ox * Oy) * B_i;
      a[MOM_BFX * ncell + i] += wA * rabs(Ox) * B_i;
      a[MOM_BFY * ncell + i] += wA * rabs(Oy) * B_i;
      if (I_new) I_new[seg * Gsub + gi] = store_dev ? (double)(Ibar - B_i) : (double)Ibar;
      I = Iout;
    }
    if (I_exit) I_exit[(ray0 + (int64_t)k) * Gsub + gi] = (double)I;
  }
}

template <class R>
static int run_sweep(const oracle_geom *g, int G, const double *kappa, const double *B, double c, double dt,
                     const double *bnd, const double *I_prev, const int *groups, int ngroups, double *out,
                     double *I_new, double *I_exit, int nthreads, int store_dev, int prev_dev, double *face_out,
                     const oracle_errmodel *em, const double *Ierr_prev, double *Ierr_new, double *err_out) {
  if (check_geom(g)) return -1;
  if (G < 1 || !kappa || !B || !bnd || !(c > 0) || !(dt > 0) || !out) return -1;
  Geometry<R> geo;
  int rc = geo.build(*g);
  if (rc) return rc;
  std::vector<int> gl;
  if (groups) {
    for (int i = 0; i < ngroups; ++i) {
      if (groups[i] < 0 || groups[i] >= G) return -1;
      gl.push_back(groups[i]);
    }
  } else {
    for (int i = 0; i < G; ++i) gl.push_back(i);
  }
  const int Gsub = (int)gl.size();
  std::vector<int64_t> seg_off;
  canonical_offsets<R>(*g, geo, seg_off);
  std::vector<int64_t> ray_off(g->ndir + 1, 0);
  for (int m = 0; m < g->ndir; ++m) ray_off[m + 1] = ray_off[m] + (int64_t)geo.dirs[geo.of[m]].rays.size();
  const int64_t ncell = (int64_t)g->nx * g->ny;
  const R inv_cdt = R(1) / (R(c) * R(dt));
  const R V = R(g->lx / g->nx) * R(g->ly / g->ny);
  const int nblk = std::min(g->ndir, 16);
  if (nthreads < 1) nthreads = 1;
  std::vector<std::vector<R>> acc(nblk), facc(face_out ? nblk : 0);
  std::vector<std::vector<double>> eacc(em ? nblk : 0);
  const int64_t nf = (int64_t)(g->nx + 1) * g->ny + (int64_t)g->nx * (g->ny + 1);
  for (int gi = 0; gi < Gsub; ++gi) {
    for (auto &a : acc) a.assign((size_t)N_MOM * ncell, R(0));
    for (auto &a : facc) a.assign((size_t)6 * nf, R(0));
    for (auto &a : eacc) a.assign((size_t)N_ERR * ncell, 0.0);
    auto work = [&](int tid) {
      for (int b = tid; b < nblk; b += nthreads) {
        int m0 = (int)((int64_t)g->ndir * b / nblk), m1 = (int)((int64_t)g->ndir * (b + 1) / nblk);
        for (int m = m0; m < m1; ++m)
          sweep_direction<R>(*g, geo, m, gi, G, gl[gi], kappa, B, inv_cdt, bnd, I_prev, seg_off[m], I_new,
                             I_exit, ray_off[m], Gsub, store_dev, prev_dev, &acc[b], face_out ? &facc[b] : nullptr,
                             em, Ierr_prev, Ierr_new, em ? &eacc[b] : nullptr);
      }
    };
    int nt = std::min(nthreads, nblk);
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
    work(0);
    for (auto &t : th) t.join();
    std::vector<R> tot((size_t)N_MOM * ncell, R(0));
    for (int b = 0; b < nblk; ++b)
      for (size_t q = 0; q < tot.size(); ++q) tot[q] += acc[b][q];
    // Cell averages: E = (1/(c V)) sum omega A Ibar;  F, N, |.|-moments = (1/V) sum ...   (Sec. 2, Eq. 15)
    for (int q = 0; q < N_MOM; ++q) {
      double *o = out + ((int64_t)q * Gsub + gi) * ncell;
      const R scale = q == MOM_D ? R(1) / (R(c) * V) : R(1) / V;
      for (int64_t i = 0; i < ncell; ++i) o[i] = (double)(tot[(size_t)q * ncell + i] * scale);
    }
    if (em) {
      // bounds of the six outputs (E, Fx, Fy, Nxx, Nxy, Nyy, in the units of `out`): the propagated segment-average
      // bounds, the summation (path 1: k_sum roundings per term; path 0: recursive summation of the cell's n terms
      // in any order, gamma_{n-1}), and the cell assembly in FP64 (the Planck part B times per-cell geometric
      // moments formed in double-double, plus the deviation sum: 8 units of 2^-53 of both magnitudes)
      std::vector<double> et((size_t)N_ERR * ncell, 0.0);
      for (int b = 0; b < nblk; ++b)
        for (size_t q = 0; q < et.size(); ++q) et[q] += eacc[b][q];
      const double u64 = 0x1p-53;
      for (int q = 0; q < 6; ++q) {
        const double scale = q == 0 ? 1.0 / (c * (double)V) : 1.0 / (double)V;
        double *ob = err_out + ((int64_t)q * Gsub + gi) * ncell;
        double *od = err_out + ((int64_t)(6 + q) * Gsub + gi) * ncell;
        double *op = err_out + ((int64_t)(12 + q) * Gsub + gi) * ncell;
        for (int64_t i = 0; i < ncell; ++i) {
          const double E = et[(size_t)(ERR0 + q) * ncell + i], D = et[(size_t)(DEV0 + q) * ncell + i],
                       P = et[(size_t)(PLK0 + q) * ncell + i], n = et[(size_t)ECNT * ncell + i];
          const double ksum = em->path == 1 ? em->k_sum : std::max(n - 1.0, 0.0);
          ob[i] = (E + ksum * em->u * D + 8 * u64 * (D + P)) * scale;
          od[i] = D * scale;
          op[i] = P * scale;
        }
      }
    }
    if (face_out) {
      // face averages over the face length: E_f = (1/(c |f|)) sum omega w I, F_f, N_f = (1/|f|) sum ...
      std::vector<R> ft((size_t)6 * nf, R(0));
      for (int b = 0; b < nblk; ++b)
        for (size_t q = 0; q < ft.size(); ++q) ft[q] += facc[b][q];
      const R hx = R(g->lx / g->nx), hy = R(g->ly / g->ny);
      const int64_t nxf = (int64_t)(g->nx + 1) * g->ny;
      for (int q = 0; q < 6; ++q) {
        double *o = face_out + ((int64_t)q * Gsub + gi) * nf;
        for (int64_t f = 0; f < nf; ++f) {
          const R len = f < nxf ? hy : hx;
          const R scale = q == MOM_D ? R(1) / (R(c) * len) : R(1) / len;
          o[f] = (double)(ft[(size_t)q * nf + f] * scale);
        }
      }
    }
  }
  return 0;
}

// The characteristic grid of Sec. 3 (every direction's characteristics and segments) in canonical order.
template <class R>
static int run_tracks(const oracle_geom *g, int64_t *counts, int64_t *dir_ray_off, int64_t *ray_seg_off,
                      double *width, int *entry, int *cell, double *len, double *area, int *face) {
  if (check_geom(g)) return -1;
  Geometry<R> geo;
  int rc = geo.build(*g);
  if (rc) return rc;
  int64_t nr = 0, ns = 0;
  for (int m = 0; m < g->ndir; ++m)
    for (auto &r : geo.dirs[geo.of[m]].rays) { nr++; ns += (int64_t)r.cell.size(); }
  if (counts) { counts[0] = nr; counts[1] = ns; }
  if (!dir_ray_off) return 0;
  int64_t ri = 0, si = 0;
  dir_ray_off[0] = 0;
  ray_seg_off[0] = 0;
  for (int m = 0; m < g->ndir; ++m) {
    for (auto &r : geo.dirs[geo.of[m]].rays) {
      width[ri] = (double)r.width;
      entry[ri] = r.entry;
      for (size_t s = 0; s < r.cell.size(); ++s, ++si) {
        cell[si] = r.cell[s];
        if (face) face[si] = r.face[s];
        len[si] = (double)r.len[s];
        area[si] = (double)r.area[s];
      }
      ray_seg_off[++ri] = si;
    }
    dir_ray_off[m + 1] = ri;
  }
  return 0;
}

extern "C" {

// Sizes of the characteristic grid (Sec. 3): counts[0] = characteristics summed over directions, counts[1] = segments
// summed over directions (the length of the canonical per-group intensity array).  Returns 0 on success.
int oracle_count(const oracle_geom *g, int64_t *counts) {
  return run_tracks<double>(g, counts, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
}

// The characteristic grid of Sec. 3 in canonical order.  precision: 0 = double, 1 = binary128 (values rounded to double).
int oracle_tracks(const oracle_geom *g, int precision, int64_t *dir_ray_off, int64_t *ray_seg_off,
                  double *width, int *entry, int *cell, double *len, double *area, int *face) {
  if (!dir_ray_off || !ray_seg_off || !width || !entry || !cell || !len || !area) return -1;
  int64_t counts[2];
  return precision ? run_tracks<real128>(g, counts, dir_ray_off, ray_seg_off, width, entry, cell, len, area, face)
                   : run_tracks<double>(g, counts, dir_ray_off, ray_seg_off, width, entry, cell, len, area, face);
}

// One backward-Euler sweep of every direction, characteristic and (selected) group.
//   kappa, B   [G][ncell]        opacity (cm^-1) and group Planck intensity
//   bnd        [4][G]            isotropic incoming intensity per edge (left, right, bottom, top)
//   I_prev     [nseg][Gsub]      canonical previous-step segment averages, or NULL for I^{n-1} = B of the cell;
//                                with prev_dev != 0 their deviations from this step's B of the segment's cell
//                                (I^{n-1} = B + I_prev formed in the oracle's precision)
//   groups     [ngroups]         subset of groups to sweep, or NULL for all (Gsub = G)
//   out        [13][Gsub][ncell] E, Fx, Fy, Nxx, Nxy, Nyy, Nzz, then the conditioning magnitudes
//                                (1/V) sum omega A |Omega_x| |Ibar - B|, same with |Omega_y|, |Omega_x Omega_y|,
//                                and the Planck parts (1/V) sum omega A |Omega_x Omega_y| B, same with |Omega_x|,
//                                |Omega_y|
//   I_new      [nseg][Gsub]      canonical segment averages Ibar (may be NULL); with store_dev != 0 the
//                                deviations Ibar - B of the segment's cell, formed in the oracle's precision
//   I_exit     [nrays][Gsub]     intensity leaving each characteristic (may be NULL)
//   face_out   [6][Gsub][nfaces] face averages E, Fx, Fy, Nxx, Nxy, Nyy of the intensity at the upwind face of
//                                every segment, weighted by omega w (Eq. 16), or NULL; faces numbered as in
//                                trace(): x-faces (nx+1) ny first, then y-faces nx (ny+1)
//   em         error model of a path to bound, or NULL (then Ierr_prev, Ierr_new and err_out are unused)
//   Ierr_prev  [nseg][Gsub]      bound of the error of that path's stored deviations entering this step, or NULL (0)
//   Ierr_new   [nseg][Gsub]      bound of the error of the path's new deviations (plus this oracle's rounding of
//                                its own to double), or NULL
//   err_out    [18][Gsub][ncell] bound of the path's error in E, Fx, Fy, Nxx, Nxy, Nyy; then the magnitudes of
//                                their deviation terms and of their Planck terms (same six, same units as out)
int oracle_sweep(const oracle_geom *g, int precision, int G, const double *kappa, const double *B, double c,
                 double dt, const double *bnd, const double *I_prev, const int *groups, int ngroups, double *out,
                 double *I_new, double *I_exit, int nthreads, int store_dev, int prev_dev, double *face_out,
                 const oracle_errmodel *em, const double *Ierr_prev, double *Ierr_new, double *err_out) {
  if (em && (!err_out || !(em->u > 0) || (em->path != 0 && em->path != 1))) return -1;
  return precision ? run_sweep<real128>(g, G, kappa, B, c, dt, bnd, I_prev, groups, ngroups, out, I_new, I_exit,
                                       nthreads, store_dev, prev_dev, face_out, em, Ierr_prev, Ierr_new, err_out)
                   : run_sweep<double>(g, G, kappa, B, c, dt, bnd, I_prev, groups, ngroups, out, I_new, I_exit,
                                       nthreads, store_dev, prev_dev, face_out, em, Ierr_prev, Ierr_new, err_out);
}

// Bits of the oracle's real type (bookkeeping, no counterpart in the paper).
int oracle_real_bits(int precision) { return precision ? (int)(sizeof(real128) * 8) : 64; }

}  // extern "C"
