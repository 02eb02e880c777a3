// Host side of libmolc: argument checking, the characteristic-grid planner (Sec. 3) and the C ABI.
//
// The planner builds, for every azimuth pair (phi, phi + pi), the parallel characteristics of the chosen
// layout, cuts each at its crossings with the material grid lines, and stores the segments once per pair:
// the + sense walks them forward, the - sense backward, and all polar cosines of the pair share them (the
// in-plane track depends only on the azimuth; the 3D path length is l / sin(zeta), Eq. 13).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "molc_internal.h"
#include "molc_tiles.h"
#include "molc_tune.h"

using namespace molc;

namespace {

thread_local std::string g_last_error;

molc_status fail(molc_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

molc_status cuda_fail(cudaError_t e, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? MOLC_ERR_OUT_OF_MEMORY : MOLC_ERR_CUDA, "%s: %s", what,
              cudaGetErrorString(e));
}
molc_status cuda_fail(cudaError_t e, const char *who, const char *what) {
  return fail(e == cudaErrorMemoryAllocation ? MOLC_ERR_OUT_OF_MEMORY : MOLC_ERR_CUDA, "%s: %s: %s", who, what,
              cudaGetErrorString(e));
}

// Compensated (double-double) accumulator for the per-cell geometric moments.
struct Acc2 {
  double hi = 0, lo = 0;
  void add(double x) {
    double s = hi + x;
    double bp = s - hi;
    double err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
  }
  double value() const { return hi + lo; }
};

struct HostTrack {
  double width;
  int entry_plus, entry_minus;
  int64_t seg_off;
  int nseg;
};

}  // namespace

struct molc_plan {
  int device = 0;
  molc_grid grid{};
  int G = 0, n_dir = 0, n_pairs = 0, n_polar = 0;
  double spacing = 0;
  molc_layout layout = MOLC_RAYS_UNIFORM;
  unsigned flags = 0;
  bool host_only = false;
  int n_split_cells = 0;      // FP32 moments: cells whose entry list is summed in parts (known to host-only plans too)
  double hx = 0, hy = 0, V = 0;
  // host copies of the characteristic grid
  std::vector<PairDev> pairs;
  std::vector<PolarDev> polar;                 // [pair][p]
  std::vector<int64_t> pair_track_off;         // [n_pairs + 1]
  std::vector<HostTrack> tracks;
  std::vector<int> seg_cell;
  std::vector<double> seg_len, seg_afrac;
  std::vector<int> dir_pair, dir_sense, dir_polar;
  std::vector<int64_t> dir_seg_off;
  // device
  TrackDev *d_tracks = nullptr;
  int2 *d_seg32 = nullptr;
  int *d_seg_cell = nullptr;
  double *d_seg_len = nullptr, *d_seg_afrac = nullptr;
  PairDev *d_pairs = nullptr;
  PolarDev *d_polar = nullptr;
  double *d_geo = nullptr;
  int64_t *d_dir_seg_off = nullptr;
  int *d_status = nullptr;
  float4 *d_cdat = nullptr;
  float *d_cdB = nullptr;
  double *d_acc = nullptr;
  int2 *d_items32 = nullptr;
  int64_t n_items32 = 0;
  int64_t *d_cell_off = nullptr;
  int4 *d_gent = nullptr;
  int64_t *d_boff = nullptr;
  int2 *d_seg_face = nullptr;
  unsigned long long *d_balance = nullptr;   // MOLC_BALANCE: largest per-ray relative residual (double bits)
  int2 *d_munit = nullptr;
  int4 *d_mmulti = nullptr;
  double *d_mscratch = nullptr;
  double *d_facc = nullptr;
  size_t facc_elems = 0;
  int *d_block_order = nullptr;
  int64_t bundle_slots = 0;   // FP32 state: step slots of all bundles (boff[n_blocks])
  int64_t n_blocks32 = 0;     // FP32 sweep blocks (bundles)
  size_t acc_elems = 0;
  size_t device_bytes = 0;
  PlanView view{};
  // tiled FP32 sweep (plans without MOLC_FACES / MOLC_BALANCE): tables, plan-owned workspace, launch shape
  bool tiled = false;
  TileView tv{};
  TileShape tshape{};
  int np_class = 0;          // polar count the sweep kernel is compiled for (1, 2, 4, 8)
  int tgrid = 0;             // blocks of the persistent sweep launch
  int tthreads = 256;        // threads of one of its blocks
  int64_t tstate_floats = 0;
  int64_t tn_pieces = 0;
  int n_tprep = 0;
  TileInst *d_tinst = nullptr;   // the instance of this plan's own launches (written by the prep launch)
  int2 *d_tqueue = nullptr;
  int4 *d_tprep = nullptr;
  int4 *d_tpiece = nullptr;
  int64_t *d_tpiece_off = nullptr;
  std::vector<void *> tdev;  // every tiled allocation (freed with the plan)
  // benchmark timing of the sweep kernel
  std::string tune_key;      // MOLC_AUTOTUNE: the plan's signature in the tuning cache
  bool tuned_from_cache = false;
  bool timing = false;
  std::vector<cudaEvent_t> ev;   // pairs
  int n_timed = 0;
};

namespace {

// RAII guard: make the plan's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// f(i) for i in [0, n) on up to the host's hardware threads (each index once, in no fixed order); the planner's
// independent loops (one azimuth pair, one chunk's entries) write disjoint outputs, so the plan is the same as
// from a serial loop.
// Small plans (threaded = false) run the loop serially: starting the threads would cost more than the work.
template <class F>
void parallel_for(int64_t n, F f, bool threaded = true) {
  const int64_t nt =
      threaded ? std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)std::thread::hardware_concurrency())) : 1;
  if (nt <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> th;
  th.reserve((size_t)nt);
  for (int64_t k = 0; k < nt; ++k)
    th.emplace_back([&]() {
      for (int64_t i; (i = next.fetch_add(1)) < n;) f(i);
    });
  for (auto &x : th) x.join();
}

// Offsets (along n = (-s, c)) and widths of the characteristics of one azimuth, ordered by offset.
void characteristic_offsets(const molc_grid &g, double c, double s, double spacing, molc_layout layout,
                            std::vector<double> &t, std::vector<double> &w) {
  t.clear();
  w.clear();
  const double xs[2] = {g.x0, g.x0 + g.lx}, ys[2] = {g.y0, g.y0 + g.ly};
  if (layout == MOLC_RAYS_UNIFORM) {
    double tmin = 1e300, tmax = -1e300;
    for (double x : xs)
      for (double y : ys) {
        double v = -s * x + c * y;
        tmin = std::min(tmin, v);
        tmax = std::max(tmax, v);
      }
    const double Lp = tmax - tmin;
    long n = (long)std::ceil(Lp / spacing - 1e-9);
    if (n < 1) n = 1;
    const double wk = Lp / (double)n;
    t.reserve(n);
    for (long k = 0; k < n; ++k) {
      t.push_back(tmin + ((double)k + 0.5) * wk);
      w.push_back(wk);
    }
    return;
  }
  // The paper's rule: every gap between projections of grid vertices is a characteristic free of vertices;
  // split into halves until the width is at most h_moc.
  const double hx = g.lx / g.nx, hy = g.ly / g.ny;
  std::vector<double> proj;
  proj.reserve((size_t)(g.nx + 1) * (g.ny + 1));
  for (int b = 0; b <= g.ny; ++b)
    for (int a = 0; a <= g.nx; ++a) proj.push_back(-s * (g.x0 + a * hx) + c * (g.y0 + b * hy));
  std::sort(proj.begin(), proj.end());
  const double merge = 1e-13 * (proj.back() - proj.front());
  double last = proj.front();
  for (size_t i = 1; i < proj.size(); ++i) {
    if (proj[i] - last <= merge) continue;
    const double gap = proj[i] - last;
    long pieces = 1;
    while (gap / (double)pieces > spacing) pieces *= 2;
    const double wk = gap / (double)pieces;
    for (long q = 0; q < pieces; ++q) {
      t.push_back(last + ((double)q + 0.5) * wk);
      w.push_back(wk);
    }
    last = proj[i];
  }
}

// Double-double helpers (error-free transformations) for the crossing parameters.
struct DD {
  double hi, lo;
};
inline DD two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
inline DD fast_two_sum(double hi, double lo) {
  const double s = hi + lo;
  return {s, lo - (s - hi)};
}
inline bool dd_less(const DD &a, const DD &b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
// (X + t q) / d to ~106 bits: the parameter where the line {p : p.n = t} meets a grid line.
inline DD crossing(double X, double t, double q, double d) {
  const double p = t * q, pe = std::fma(t, q, -p);
  const DD n0 = two_sum(X, p);
  const DD n = fast_two_sum(n0.hi, n0.lo + pe);
  const double q1 = n.hi / d;
  const double r = std::fma(-q1, d, n.hi) + n.lo;
  return fast_two_sum(q1, r / d);
}

// Cut one characteristic into cell segments.  The characteristic grid is defined by double-precision
// evaluation of the direction, grid lines and offsets (this file is compiled without FMA contraction); the
// crossing parameters are then evaluated in double-double so that every segment length is accurate relative
// to itself, short corner segments included.  Crossings with vertical and horizontal grid lines form two
// increasing sequences that are merged; a gap <= eps between consecutive cut points is not a segment (the
// characteristic passes within eps of a vertex, i.e. steps diagonally).  A segment belongs to the cell that
// contains its midpoint.  Returns false if the line misses the domain.
bool cut_characteristic(const molc_grid &g, double hx, double hy, double c, double s, double t,
                        std::vector<int> &cells, std::vector<double> &lens, std::vector<double> &lens_lo,
                        int &entry_plus, int &entry_minus) {
  const double eps = 1e-12 * std::min(hx, hy);
  const double bx = -t * s, by = t * c;  // the point of the line at u = 0
  const double x1 = g.x0 + g.lx, y1 = g.y0 + g.ly;
  const DD lo_inf{-1e300, 0}, hi_inf{1e300, 0};
  DD xlo = lo_inf, xhi = hi_inf, ylo = lo_inf, yhi = hi_inf;
  if (c != 0.0) {
    xlo = crossing(g.x0, t, s, c);   // (x0 - bx) / c
    xhi = crossing(x1, t, s, c);
    if (dd_less(xhi, xlo)) std::swap(xlo, xhi);
  } else if (bx < g.x0 || bx > x1) {
    return false;
  }
  if (s != 0.0) {
    ylo = crossing(g.y0, t, -c, s);  // (y0 - by) / s
    yhi = crossing(y1, t, -c, s);
    if (dd_less(yhi, ylo)) std::swap(ylo, yhi);
  } else if (by < g.y0 || by > y1) {
    return false;
  }
  const DD uin = dd_less(xlo, ylo) ? ylo : xlo, uout = dd_less(xhi, yhi) ? xhi : yhi;
  if ((uout.hi - uin.hi) + (uout.lo - uin.lo) <= eps) return false;
  // entry of the + sense: the larger lower bound (tie -> the vertical edge); exit likewise with upper bounds.
  const bool x_in = c != 0.0 && (s == 0.0 || xlo.hi >= ylo.hi - eps);
  entry_plus = x_in ? (c > 0 ? 0 : 1) : (s > 0 ? 2 : 3);
  const bool x_out = c != 0.0 && (s == 0.0 || xhi.hi <= yhi.hi + eps);
  entry_minus = x_out ? (c > 0 ? 1 : 0) : (s > 0 ? 3 : 2);
  // crossing parameters, each list increasing in u
  std::vector<DD> ux, uy;
  if (c != 0.0) {
    for (int i = 1; i < g.nx; ++i) {
      const int ii = c > 0 ? i : g.nx - i;
      const DD u = crossing(g.x0 + ii * hx, t, s, c);
      if (dd_less(uin, u) && dd_less(u, uout)) ux.push_back(u);
    }
  }
  if (s != 0.0) {
    for (int j = 1; j < g.ny; ++j) {
      const int jj = s > 0 ? j : g.ny - j;
      const DD u = crossing(g.y0 + jj * hy, t, -c, s);
      if (dd_less(uin, u) && dd_less(u, uout)) uy.push_back(u);
    }
  }
  cells.clear();
  lens.clear();
  lens_lo.clear();
  size_t ix = 0, iy = 0;
  DD a = uin;
  while (true) {
    DD b;
    bool last = false;
    if (ix < ux.size() && (iy >= uy.size() || !dd_less(uy[iy], ux[ix])))
      b = ux[ix++];
    else if (iy < uy.size())
      b = uy[iy++];
    else {
      b = uout;
      last = true;
    }
    const DD ld = fast_two_sum(b.hi - a.hi, b.lo - a.lo);  // b.hi - a.hi is exact where it matters (close)
    const double len = ld.hi;
    if (len > eps) {
      const double m = a.hi + 0.5 * len;
      int cx = (int)std::floor((bx + m * c - g.x0) / hx);
      int cy = (int)std::floor((by + m * s - g.y0) / hy);
      cx = std::min(std::max(cx, 0), g.nx - 1);
      cy = std::min(std::max(cy, 0), g.ny - 1);
      cells.push_back(cy * g.nx + cx);
      lens.push_back(len);
      lens_lo.push_back(ld.lo);
    }
    a = b;
    if (last) break;
  }
  return !cells.empty();
}

template <class T> molc_status upload(T **dst, const T *src, size_t n, size_t &total, const char *what) {
  *dst = nullptr;
  if (n == 0) return MOLC_OK;
  cudaError_t e = cudaMalloc((void **)dst, n * sizeof(T));
  if (e != cudaSuccess) return cuda_fail(e, what);
  total += n * sizeof(T);
  if (src) {
    e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, what);
  }
  return MOLC_OK;
}

constexpr int kMaxTimed = 4096;

void free_events(molc_plan *p) {
  for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
  p->ev.clear();
  p->n_timed = 0;
}

void free_device(molc_plan *p) {
  free_events(p);
  void *ptrs[] = {p->d_tracks, p->d_seg32, p->d_seg_cell, p->d_seg_len, p->d_seg_afrac, p->d_pairs, p->d_polar,
                  p->d_geo, p->d_dir_seg_off, p->d_status, p->d_cdat, p->d_cdB, p->d_acc, p->d_items32,
                  p->d_cell_off, p->d_gent, p->d_boff, p->d_block_order, p->d_seg_face, p->d_facc,
                  p->d_munit, p->d_mmulti, p->d_mscratch, p->d_balance};
  for (void *q : ptrs)
    if (q) cudaFree(q);
  for (void *q : p->tdev)
    if (q) cudaFree(q);
  p->tdev.clear();
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0; }

// Workspace of a tiled sweep, in the order it is carved: control words, item flags, quadrant arrival counts,
// cell tables, quadrant moment partials, boundary buffer.  Each part is rounded up to 256 bytes.
struct TileWorkspace {
  size_t ctrl, flags, cnt, cdat, cdB, part, bbuf, total;
};
TileWorkspace tile_workspace(const TileView &t, int G, int np, int64_t n_pieces) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  TileWorkspace w;
  w.ctrl = 256;
  w.flags = up((size_t)t.n_items * sizeof(int));
  w.cnt = up((size_t)t.n_tiles * t.n_gt * sizeof(int));
  w.cdat = up((size_t)t.n_tiles * G * t.TS2p * sizeof(float4));
  w.cdB = up((size_t)t.n_tiles * G * t.TS2p * sizeof(float));
  w.part = up((size_t)t.n_tiles * t.n_gt * 4 * kOutputs * t.GT * t.TS2p * sizeof(double));
  w.bbuf = up((size_t)n_pieces * G * (np + 2) * sizeof(float));
  w.total = w.ctrl + w.flags + w.cnt + w.cdat + w.cdB + w.part + w.bbuf;
  return w;
}
// Point a view's workspace into `base` (at least tile_workspace().total bytes, 256-byte aligned).
void tile_carve(TileView &t, char *base, const TileWorkspace &w) {
  t.ctrl = (int *)base;
  base += w.ctrl;
  t.flags = (int *)base;
  base += w.flags;
  t.cnt = (int *)base;
  base += w.cnt;
  t.cdat = (float4 *)base;
  base += w.cdat;
  t.cdB = (float *)base;
  base += w.cdB;
  t.part = (double *)base;
  base += w.part;
  t.bbuf = (float *)base;
}

size_t state_bytes_fp32(const molc_plan *p);
double *bref_ptr(const molc_plan *p, molc_precision prec, void *I);
double *header_ptr(const molc_plan *p, molc_precision prec, void *I);

// Autotuner of the FP32 sweep: times each compiled staging depth on this plan and keeps the fastest.  The
// temporary inputs have about one optical depth per cell (kappa = 1/min(hx, hy), B = boundary = 1, c = dt = 1),
// so that both branches of the attenuation run; the FP32 state starts from B.  Each depth is warmed up once,
// then timed over enough launches to fill about half a millisecond, in two rounds that alternate the depths;
// a depth's time is its better round.  The default depth is kept unless another is at least 2 % faster (the
// depths differ by a few percent, less than one short timing's noise).  The depth changes no arithmetic, only
// the timing.  Allocates its temporaries for the duration of the call.
molc_status autotune(molc_plan *p, double *best_ms_out) {
  DeviceGuard dg(p->device);
  const int64_t cg = (int64_t)p->G * p->view.ncell;
  void *I = nullptr;
  double *in = nullptr;   // kappa, B [G][cell], bnd [4][G]
  double *mom = nullptr;  // 6 x [G][cell]
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&I, state_bytes_fp32(p));
  if (e == cudaSuccess) e = cudaMalloc((void **)&in, (2 * cg + 4 * (int64_t)p->G) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&mom, 6 * cg * sizeof(double));
  if (e == cudaSuccess) {
    std::vector<double> h((size_t)(2 * cg + 4 * (int64_t)p->G), 1.0);
    std::fill(h.begin(), h.begin() + cg, 1.0 / std::min(p->hx, p->hy));
    e = cudaMemcpy(in, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  constexpr int kDefault = 4;
  const int nd = (int)(sizeof(kSweepDepths) / sizeof(kSweepDepths[0]));
  std::vector<float> t(nd, 0.f);   // best time per launch of each depth
  int reps = 2;
  if (e == cudaSuccess) {
    SweepArgs a{};
    a.kappa = in;
    a.B = in + cg;
    a.bnd = in + 2 * cg;
    a.c = a.dt = 1.0;
    a.inv_c = a.inv_cdt = 1.0;
    a.I = I;
    a.Bref = bref_ptr(p, MOLC_FP32, I);
    a.scale = header_ptr(p, MOLC_FP32, I);
    a.out = molc_moments{mom, mom + cg, mom + 2 * cg, mom + 3 * cg, mom + 4 * cg, mom + 5 * cg};
    a.cdat = p->d_cdat;
    a.cdB = p->d_cdB;
    a.items = p->d_items32;
    a.n_items = p->n_items32;
    e = cudaMemset(I, 0, state_bytes_fp32(p));
    if (e == cudaSuccess) e = cudaMemcpy(a.Bref, a.B, cg * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = launch_set_scale(p->view, MOLC_FP32, a.B, const_cast<double *>(a.scale), nullptr);
    if (e == cudaSuccess) e = launch_prep(p->view, MOLC_FP32, a, nullptr);
    auto timed = [&](int d, int n, float &ms) {
      PlanView v = p->view;
      v.sweep_depth = d;
      cudaError_t r = cudaEventRecord(e0, nullptr);
      for (int k = 0; k < n && r == cudaSuccess; ++k) r = launch_sweep_fp32(v, a, nullptr);
      if (r == cudaSuccess) r = cudaEventRecord(e1, nullptr);
      if (r == cudaSuccess) r = cudaEventSynchronize(e1);
      if (r == cudaSuccess) r = cudaEventElapsedTime(&ms, e0, e1);
      return r;
    };
    float one = 0.f;
    for (int i = 0; i < nd && e == cudaSuccess; ++i) {   // warm-up; the default depth's launch sets the count
      float ms = 0.f;
      e = timed(kSweepDepths[i], 1, ms);
      if (kSweepDepths[i] == kDefault) one = ms;
    }
    if (one > 0.f) reps = std::max(2, std::min(20, (int)std::ceil(0.5f / one)));
    for (int round = 0; round < 2 && e == cudaSuccess; ++round)
      for (int i = 0; i < nd && e == cudaSuccess; ++i) {
        float ms = 0.f;
        e = timed(kSweepDepths[i], reps, ms);
        if (e == cudaSuccess && (t[i] == 0.f || ms / reps < t[i])) t[i] = ms / reps;
      }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (mom) cudaFree(mom);
  if (in) cudaFree(in);
  if (I) cudaFree(I);
  if (e != cudaSuccess) return cuda_fail(e, "create: autotune");
  int best = kDefault;
  float t_def = 0.f, t_best = 0.f;
  for (int i = 0; i < nd; ++i)
    if (kSweepDepths[i] == kDefault) t_def = t_best = t[i];
  for (int i = 0; i < nd; ++i)
    if (t[i] > 0.f && t[i] < 0.98f * t_def && t[i] < t_best) {
      t_best = t[i];
      best = kSweepDepths[i];
    }
  p->view.sweep_depth = best;
  if (best_ms_out) *best_ms_out = t_best;
  int code = 0;
  cudaMemcpy(&code, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemset(p->d_status, 0, sizeof(int));   // the temporaries' checks leave no trace
  return MOLC_OK;
}

// Tiled FP32 sweep of a plan: cut its characteristic grid into per-tile pieces (tile size and groups per item
// chosen by plan_tiles, or pinned by force_ts / force_gt), upload the tables, allocate the workspace (zeroed) and
// fix the launch shape.  Replaces an earlier tiled build of the plan.
molc_status build_tiled(molc_plan *p, int force_ts, int force_gt, bool *fits = nullptr, int threads = 0) {
  const int64_t T = (int64_t)p->tracks.size();
  std::vector<TileTrack> tt((size_t)T);
  for (int j = 0; j < p->n_pairs; ++j)
    for (int64_t k = p->pair_track_off[j]; k < p->pair_track_off[j + 1]; ++k) {
      const HostTrack &h = p->tracks[k];
      tt[k] = TileTrack{h.seg_off, h.nseg, j, h.entry_plus, h.entry_minus};
    }
  std::vector<double> pc(p->n_pairs), ps(p->n_pairs);
  for (int j = 0; j < p->n_pairs; ++j) {
    pc[j] = p->pairs[j].c;
    ps[j] = p->pairs[j].s;
  }
  TilePlanInput in{p->grid.nx, p->grid.ny, p->G, p->n_pairs, p->n_polar, pc.data(), ps.data(), &tt,
                   p->seg_cell.data(), p->seg_len.data(), p->seg_afrac.data()};
  TileTables tb;
  std::string why;
  if (!plan_tiles(in, tb, why, force_ts, force_gt)) {
    if (fits) *fits = false;
    return fail(MOLC_ERR_INVALID_ARG, "create: tiled FP32 sweep: %s", why.c_str());
  }
  if (fits) *fits = true;
  for (void *q : p->tdev)
    if (q) cudaFree(q);
  p->tdev.clear();
  p->d_tinst = nullptr;
  p->d_tqueue = nullptr;
  p->d_tprep = nullptr;
  p->d_tpiece = nullptr;
  p->d_tpiece_off = nullptr;
  TileView t{};
  t.TS = tb.TS;
  t.TS2p = tb.TS2p;
  t.ntx = tb.ntx;
  t.nty = tb.nty;
  t.n_tiles = tb.n_tiles;
  t.n_geoms = tb.n_geoms;
  t.GT = tb.GT;
  t.n_gt = tb.n_gt;
  t.n_items = tb.n_items;
  t.max_item_floats = tb.max_item_floats;
  t.max_len = tb.max_len;
  p->tstate_floats = tb.state_floats;
  p->tn_pieces = tb.n_pieces;
  if (p->host_only) {   // the layout's sizes only (plan information); nothing on the device
    p->tv = t;
    return MOLC_OK;
  }
  std::vector<int2> queue(tb.queue.size());
  for (size_t i = 0; i < queue.size(); ++i) queue[i] = make_int2(0, tb.queue[i]);
  std::vector<int4> prep;
  const int tpb = std::max(1, 256 / (tb.TS * tb.TS));
  for (int g = 0; g < p->G; ++g)
    for (int t0 = 0; t0 < tb.n_tiles; t0 += tpb) prep.push_back(make_int4(0, t0, g, g == 0 && t0 == 0));
  molc_status st = MOLC_OK;
  size_t &tot = p->device_bytes;
  auto up = [&](auto **dst, const auto &vec, const char *what) {
    if (st == MOLC_OK) st = upload(dst, vec.data(), vec.size(), tot, what);
    p->tdev.push_back((void *)*dst);
  };
  TileGeom *geoms = nullptr;
  int *Ptab = nullptr;
  int4 *pieces = nullptr, *units = nullptr;
  int2 *recs = nullptr, *ents = nullptr, *cu = nullptr;
  int64_t *item_off = nullptr;
  up(&geoms, tb.geoms, "tile geometries");
  up(&Ptab, tb.Ptab, "tile step offsets");
  up(&pieces, tb.pieces, "tile pieces");
  up(&recs, tb.recs, "tile records");
  up(&ents, tb.ents, "tile moment entries");
  up(&units, tb.units, "tile moment units");
  up(&cu, tb.cell_units, "tile cell units");
  up(&item_off, tb.item_off, "tile state offsets");
  up(&p->d_tqueue, queue, "tile queue");
  up(&p->d_tprep, prep, "tile prep map");
  up(&p->d_tpiece, tb.tpiece, "tile piece list");
  up(&p->d_tpiece_off, tb.tpiece_off, "tile piece offsets");
  if (st != MOLC_OK) return st;
  t.geoms = geoms;
  t.Ptab = Ptab;
  t.pieces = pieces;
  t.recs = recs;
  t.ents = ents;
  t.units = units;
  t.cell_units = cu;
  t.item_off = item_off;
  const TileWorkspace w = tile_workspace(t, p->G, p->n_polar, tb.n_pieces);
  char *ws = nullptr;
  cudaError_t e = cudaMalloc((void **)&ws, w.total);
  if (e == cudaSuccess) {
    p->tdev.push_back(ws);
    tot += w.total;
    e = cudaMemset(ws, 0, w.ctrl + w.flags + w.cnt);   // control words, flags and counts start at zero
  }
  if (e == cudaSuccess) {
    e = cudaMalloc((void **)&p->d_tinst, sizeof(TileInst));
    if (e == cudaSuccess) {
      p->tdev.push_back(p->d_tinst);
      tot += sizeof(TileInst);
    }
  }
  if (e != cudaSuccess) return cuda_fail(e, "create: tiled sweep workspace");
  tile_carve(t, ws, w);
  p->tv = t;
  p->n_tprep = (int)prep.size();
  p->np_class = p->n_polar <= 1 ? 1 : p->n_polar <= 2 ? 2 : p->n_polar <= 4 ? 4 : 8;
  p->tshape = tile_shape(tb, p->n_pairs, p->n_polar);
  // block threads: as asked, else the fewer that still cover an item's (piece, group) tasks in one or two rounds
  int max_tasks = 0;
  for (const TileGeom &gm : tb.geoms) max_tasks = std::max(max_tasks, gm.n_pieces * tb.GT);
  p->tthreads = threads > 0 ? threads : (max_tasks <= 2 * 128 ? 128 : 256);
  p->tgrid = tile_sweep_grid(p->np_class, tile_sweep_smem(p->tshape, p->np_class), p->tthreads);
  return MOLC_OK;
}

// Build identifier in the tuning cache: the build script defines MOLC_BUILD_ID as one token (a hash of the
// sources); made a string here.
#ifndef MOLC_BUILD_ID
#define MOLC_BUILD_ID unversioned
#endif
#define MOLC_STRINGIFY2(x) #x
#define MOLC_STRINGIFY(x) MOLC_STRINGIFY2(x)
const char *const kBuildId = MOLC_STRINGIFY(MOLC_BUILD_ID);

// Signature of a plan in the tuning cache: what molc_create was given that decides the plan's kernels and their
// launch shapes (grid, directions, groups, ray spacing and layout, the flags that change the sweep), readable
// sizes followed by a 64-bit FNV-1a hash of the exact values.
std::string plan_signature(const molc_grid &g, const molc_quadrature *q, int G, double spacing, int layout,
                           unsigned flags) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void *data, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(data);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  const unsigned f = flags & (MOLC_AREA_RENORM | MOLC_FACES | MOLC_BALANCE | MOLC_TILED);
  const double gd[4] = {g.x0, g.y0, g.lx, g.ly};
  const int gi[5] = {g.nx, g.ny, q->n, G, layout};
  mix(gd, sizeof gd);
  mix(gi, sizeof gi);
  mix(&spacing, sizeof spacing);
  mix(&f, sizeof f);
  for (const double *a : {q->mu, q->cos_phi, q->sin_phi, q->w}) mix(a, sizeof(double) * (size_t)q->n);
  char buf[200];
  std::snprintf(buf, sizeof buf, "%dx%d cells, %d groups, %d directions, spacing %.6g, layout %d, flags %u, %016llx",
                g.nx, g.ny, G, q->n, spacing, layout, f, (unsigned long long)h);
  return buf;
}

// The kind of device a tuned configuration holds for: name, SM count, compute capability.
std::string device_signature(int dev) {
  cudaDeviceProp pr{};
  if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown device";
  }
  char buf[320];
  std::snprintf(buf, sizeof buf, "%s, %d SMs, sm_%d%d", pr.name, pr.multiProcessorCount, pr.major, pr.minor);
  return buf;
}

}  // namespace

extern "C" {

// MOLC_AUTOTUNE at the end of molc_create (defined below, after the tiled step)
static molc_status tune_plan(molc_plan *p);

const char *molc_last_error(void) { return g_last_error.c_str(); }

molc_status molc_quadrature_product(int n_polar, int n_azim, double *mu, double *cos_phi, double *sin_phi,
                                    double *w) {
  if (n_polar < 1 || n_polar > 64 || n_azim < 4 || n_azim % 4 || !mu || !cos_phi || !sin_phi || !w)
    return fail(MOLC_ERR_INVALID_ARG, "quadrature_product: need 1 <= n_polar <= 64, n_azim a multiple of 4");
  // Gauss-Legendre nodes on (-1, 1): Newton's method on P_n from the guesses cos(pi (i + 3/4) / (n + 1/2)),
  // P_n and P_{n-1} by the three-term recurrence, weights 2 / ((1 - x^2) P_n'(x)^2); mapped to (0, 1) below.
  std::vector<double> x(n_polar), W(n_polar);
  const double pi = 3.14159265358979323846;
  auto legendre = [n_polar](double z, double &pn, double &dpn) {
    double p_prev = 1.0, p_cur = z;
    if (n_polar == 1) {
      pn = z;
      dpn = 1.0;
      return;
    }
    for (int k = 1; k < n_polar; ++k) {
      const double p_next = ((2.0 * k + 1.0) * z * p_cur - k * p_prev) / (k + 1.0);
      p_prev = p_cur;
      p_cur = p_next;
    }
    pn = p_cur;
    dpn = n_polar * (z * p_cur - p_prev) / (z * z - 1.0);
  };
  for (int i = 0; i < n_polar; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n_polar + 0.5)), pn, dpn;
    for (int it = 0; it < 100; ++it) {
      legendre(z, pn, dpn);
      const double dz = pn / dpn;
      z -= dz;
      if (std::fabs(dz) <= 1e-16 * std::fabs(z) + 1e-300) break;
    }
    legendre(z, pn, dpn);
    x[i] = z;
    W[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
  }
  std::vector<int> order(n_polar);
  for (int i = 0; i < n_polar; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return x[a] < x[b]; });
  // Chebyshev azimuths, first octant evaluated, the rest by exact swaps and sign flips.
  const int Q = n_azim / 4;
  std::vector<double> c1(Q), s1(Q), c(n_azim), s(n_azim);
  for (int j = 0; j < (Q + 1) / 2; ++j) {
    const double phi = (j + 0.5) * 2.0 * pi / n_azim;
    c1[j] = std::cos(phi);
    s1[j] = std::sin(phi);
    c1[Q - 1 - j] = s1[j];
    s1[Q - 1 - j] = c1[j];
  }
  if (Q % 2) c1[Q / 2] = s1[Q / 2] = std::sqrt(0.5);
  for (int j = 0; j < n_azim; ++j) {
    if (j < Q) { c[j] = c1[j]; s[j] = s1[j]; }
    else if (j < 2 * Q) { c[j] = -c1[2 * Q - 1 - j]; s[j] = s1[2 * Q - 1 - j]; }
    else if (j < 3 * Q) { c[j] = -c1[j - 2 * Q]; s[j] = -s1[j - 2 * Q]; }
    else { c[j] = c1[4 * Q - 1 - j]; s[j] = -s1[4 * Q - 1 - j]; }
  }
  for (int p = 0; p < n_polar; ++p)
    for (int j = 0; j < n_azim; ++j) {
      const int m = p * n_azim + j;
      mu[m] = 0.5 * (x[order[p]] + 1.0);
      cos_phi[m] = c[j];
      sin_phi[m] = s[j];
      w[m] = 4.0 * pi * (0.5 * W[order[p]]) / n_azim;
    }
  return MOLC_OK;
}

molc_status molc_create(const molc_grid *grid, const molc_quadrature *quad, const molc_groups *groups,
                        double ray_spacing, molc_layout layout, unsigned flags, molc_plan **out) {
  if (!out) return fail(MOLC_ERR_INVALID_ARG, "create: out is NULL");
  *out = nullptr;
  if (!grid || !quad || !groups) return fail(MOLC_ERR_INVALID_ARG, "create: NULL argument");
  const molc_grid g = *grid;
  if (g.nx < 1 || g.ny < 1 || !finite_pos(g.lx) || !finite_pos(g.ly) || !std::isfinite(g.x0) ||
      !std::isfinite(g.y0))
    return fail(MOLC_ERR_INVALID_ARG, "create: bad grid");
  if ((int64_t)g.nx * g.ny > (int64_t)1 << 28) return fail(MOLC_ERR_INVALID_ARG, "create: grid too large");
  if (groups->G < 1 || groups->G > 4096) return fail(MOLC_ERR_INVALID_ARG, "create: need 1 <= G <= 4096");
  if (!finite_pos(ray_spacing)) return fail(MOLC_ERR_INVALID_ARG, "create: ray_spacing must be > 0");
  if (layout != MOLC_RAYS_UNIFORM && layout != MOLC_RAYS_PAPER) return fail(MOLC_ERR_INVALID_ARG, "create: layout");
  if (flags & ~(MOLC_AREA_RENORM | MOLC_HOST_ONLY | MOLC_AUTOTUNE | MOLC_FACES | MOLC_BALANCE | MOLC_TILED))
    return fail(MOLC_ERR_INVALID_ARG, "create: unknown flags");
  if ((flags & MOLC_BALANCE) && (flags & MOLC_FACES))
    return fail(MOLC_ERR_INVALID_ARG, "create: MOLC_BALANCE and MOLC_FACES cannot be combined");
  const int n = quad->n;
  if (n < 2 || !quad->mu || !quad->cos_phi || !quad->sin_phi || !quad->w)
    return fail(MOLC_ERR_INVALID_ARG, "create: bad quadrature");
  for (int m = 0; m < n; ++m) {
    if (!(quad->mu[m] > 0 && quad->mu[m] < 1) || !std::isfinite(quad->cos_phi[m]) ||
        !std::isfinite(quad->sin_phi[m]) || (quad->cos_phi[m] == 0 && quad->sin_phi[m] == 0) ||
        !finite_pos(quad->w[m]))
      return fail(MOLC_ERR_INVALID_ARG, "create: direction %d: need 0 < mu < 1, a nonzero in-plane vector, w > 0", m);
  }
  if (ray_spacing * 1e7 < std::max(g.lx, g.ly)) return fail(MOLC_ERR_INVALID_ARG, "create: ray_spacing too small");

  auto p = new molc_plan();
  p->grid = g;
  p->G = groups->G;
  p->n_dir = n;
  p->spacing = ray_spacing;
  p->layout = layout;
  p->flags = flags;
  p->host_only = flags & MOLC_HOST_ONLY;
  p->hx = g.lx / g.nx;
  p->hy = g.ly / g.ny;
  p->V = p->hx * p->hy;
  if (!p->host_only) cudaGetDevice(&p->device);

  // ---- azimuth pairs: + sense has sin > 0 (or sin == 0 and cos > 0); the - sense is its exact negation.
  std::map<std::pair<double, double>, std::vector<int>> az;
  std::vector<std::pair<double, double>> az_order;
  for (int m = 0; m < n; ++m) {
    auto key = std::make_pair(quad->cos_phi[m], quad->sin_phi[m]);
    if (!az.count(key)) az_order.push_back(key);
    az[key].push_back(m);
  }
  p->dir_pair.assign(n, -1);
  p->dir_sense.assign(n, -1);
  p->dir_polar.assign(n, -1);
  for (auto &key : az_order) {
    const double c = key.first, s = key.second;
    if (!(s > 0 || (s == 0 && c > 0))) continue;
    auto neg = std::make_pair(-c, -s);
    if (!az.count(neg)) {
      delete p;
      return fail(MOLC_ERR_INVALID_ARG, "create: direction (%g, %g) has no exactly opposite direction", c, s);
    }
    const auto &plus = az[key], &minus = az[neg];
    if (p->n_pairs == 0) p->n_polar = (int)plus.size();
    if ((int)plus.size() != p->n_polar || minus.size() != plus.size()) {
      delete p;
      return fail(MOLC_ERR_INVALID_ARG, "create: every azimuth must carry the same number of polar cosines");
    }
    const int j = p->n_pairs++;
    const double nrm = std::sqrt(c * c + s * s);
    PairDev pd;
    pd.c = c / nrm;
    pd.s = s / nrm;
    pd.cf = (float)pd.c;
    pd.sf = (float)pd.s;
    p->pairs.push_back(pd);
    std::vector<bool> used(minus.size(), false);
    for (int q = 0; q < p->n_polar; ++q) {
      const int mp = plus[q];
      int mm = -1;
      for (size_t r = 0; r < minus.size(); ++r)
        if (!used[r] && quad->mu[minus[r]] == quad->mu[mp] && quad->w[minus[r]] == quad->w[mp]) {
          mm = minus[r];
          used[r] = true;
          break;
        }
      if (mm < 0) {
        delete p;
        return fail(MOLC_ERR_INVALID_ARG, "create: direction %d has no opposite with equal mu and w", mp);
      }
      PolarDev pl;
      const double mu = quad->mu[mp];
      pl.w = quad->w[mp];
      pl.sinz = std::sqrt(1.0 - mu * mu);
      pl.inv_sinz = 1.0 / pl.sinz;
      pl.wf = (float)pl.w;
      pl.sinzf = (float)pl.sinz;
      pl.inv_sinzf = (float)pl.inv_sinz;
      pl.dir_plus = mp;
      pl.dir_minus = mm;
      p->polar.push_back(pl);
      p->dir_pair[mp] = p->dir_pair[mm] = j;
      p->dir_sense[mp] = 0;
      p->dir_sense[mm] = 1;
      p->dir_polar[mp] = p->dir_polar[mm] = q;
    }
  }
  for (int m = 0; m < n; ++m)
    if (p->dir_pair[m] < 0) {
      delete p;
      return fail(MOLC_ERR_INVALID_ARG, "create: direction %d is not paired", m);
    }

  // ---- characteristics and segments, pair by pair
  const int ncell = g.nx * g.ny;
  // each pair traced on its own (in parallel), then concatenated in pair order
  struct PairTracks {
    std::vector<HostTrack> tracks;   // seg_off relative to this pair's first segment
    std::vector<int> cell;
    std::vector<double> len, afrac, len_lo;
    bool too_long = false;
  };
  std::vector<PairTracks> per_pair((size_t)p->n_pairs);
  const bool big = (int64_t)ncell * p->n_pairs >= ((int64_t)1 << 17);   // threads pay off (from ~1e5 cell-pairs)
  parallel_for(p->n_pairs, [&](int64_t j) {
    PairTracks &o = per_pair[(size_t)j];
    std::vector<double> t, wv, lens, lens_lo;
    std::vector<int> cells;
    const double c = p->pairs[j].c, s = p->pairs[j].s;
    characteristic_offsets(g, c, s, ray_spacing, layout, t, wv);
    for (size_t k = 0; k < t.size(); ++k) {
      int ep, em;
      if (!cut_characteristic(g, p->hx, p->hy, c, s, t[k], cells, lens, lens_lo, ep, em)) continue;
      if (cells.size() > (size_t)1 << 30) {
        o.too_long = true;
        return;
      }
      o.tracks.push_back(HostTrack{wv[k], ep, em, (int64_t)o.cell.size(), (int)cells.size()});
      for (size_t q = 0; q < cells.size(); ++q) {
        o.cell.push_back(cells[q]);
        o.len.push_back(lens[q]);
        o.afrac.push_back(lens[q] * wv[k]);  // A for now
        o.len_lo.push_back(lens_lo[q]);
      }
    }
  }, big);
  // offsets of each pair's tracks and segments, then every pair copied into place (in parallel)
  std::vector<int64_t> seg_base((size_t)p->n_pairs + 1, 0);
  p->pair_track_off.assign((size_t)p->n_pairs + 1, 0);
  for (int j = 0; j < p->n_pairs; ++j) {
    const PairTracks &o = per_pair[(size_t)j];
    if (o.too_long) {
      delete p;
      return fail(MOLC_ERR_INVALID_ARG, "create: characteristic too long");
    }
    p->pair_track_off[(size_t)j + 1] = p->pair_track_off[(size_t)j] + (int64_t)o.tracks.size();
    seg_base[(size_t)j + 1] = seg_base[(size_t)j] + (int64_t)o.cell.size();
  }
  std::vector<double> seg_len_lo((size_t)seg_base[(size_t)p->n_pairs]);
  p->tracks.resize((size_t)p->pair_track_off[(size_t)p->n_pairs]);
  p->seg_cell.resize(seg_len_lo.size());
  p->seg_len.resize(seg_len_lo.size());
  p->seg_afrac.resize(seg_len_lo.size());
  parallel_for(p->n_pairs, [&](int64_t j) {
    PairTracks &o = per_pair[(size_t)j];
    const int64_t t0 = p->pair_track_off[(size_t)j], s0 = seg_base[(size_t)j];
    for (size_t k = 0; k < o.tracks.size(); ++k) {
      p->tracks[(size_t)t0 + k] = o.tracks[k];
      p->tracks[(size_t)t0 + k].seg_off += s0;
    }
    std::copy(o.cell.begin(), o.cell.end(), p->seg_cell.begin() + s0);
    std::copy(o.len.begin(), o.len.end(), p->seg_len.begin() + s0);
    std::copy(o.afrac.begin(), o.afrac.end(), p->seg_afrac.begin() + s0);
    std::copy(o.len_lo.begin(), o.len_lo.end(), seg_len_lo.begin() + s0);
    o = PairTracks{};   // released as they are copied
  }, big);
  const int64_t T = (int64_t)p->tracks.size();
  const int64_t S = (int64_t)p->seg_cell.size();
  if (T == 0) {
    delete p;
    return fail(MOLC_ERR_INVALID_ARG, "create: no characteristic crosses the domain");
  }
  // ---- areas (Eq. 14), optional renormalisation per (cell, pair), area fractions a = A / V, geometric moments
  //   G_ab(i) = sum_m omega_m Omega_a Omega_b sum_{C(i,m)} A / V = sum_j W_ab(j) (1 + e_ij),
  // with W_ab(j) the pair's angular weight and e_ij = sum_{C(i,j)} A / V - 1 the area defect.  With
  // renormalisation e_ij = 0 by construction.  Otherwise e_ij is formed from double-double lengths and sums: for
  // the paper's layout it is ~1e-15 (double band edges), and N_xy's B part, sum_j W_xy(j) e_ij, is a small
  // sum that must not carry the rounding of sum_j W_xy(j) (which is exactly zero for a symmetric set).
  const bool renorm = flags & MOLC_AREA_RENORM;
  std::vector<Acc2> g0(ncell), gxx(ncell), gxy(ncell), gyy(ncell);
  Acc2 w0_all, wxx_all, wxy_all, wyy_all;
  // per pair (in parallel): the area sums of its characteristics per cell, the area fractions, and without
  // renormalisation the area defects e_ij; a pair that misses a cell records the first such cell
  std::vector<std::vector<double>> defect(renorm ? 0 : (size_t)p->n_pairs);
  std::vector<int> missed((size_t)p->n_pairs, -1);
  parallel_for(p->n_pairs, [&](int64_t j) {
    std::vector<double> asum(ncell, 0.0);
    std::vector<Acc2> asum_dd(renorm ? 0 : ncell);
    const int64_t s0 = p->tracks[p->pair_track_off[j]].seg_off;
    const int64_t s1 = p->pair_track_off[j + 1] < T ? p->tracks[p->pair_track_off[j + 1]].seg_off : S;
    for (int64_t k = p->pair_track_off[j]; k < p->pair_track_off[j + 1]; ++k) {
      const double w = p->tracks[k].width;
      for (int64_t q = p->tracks[k].seg_off; q < p->tracks[k].seg_off + p->tracks[k].nseg; ++q) {
        const int i = p->seg_cell[q];
        asum[i] += p->seg_afrac[q];
        if (!renorm) {
          const double pa = p->seg_len[q] * w;
          asum_dd[i].add(pa);
          asum_dd[i].add(std::fma(p->seg_len[q], w, -pa));
          asum_dd[i].add(seg_len_lo[q] * w);
        }
      }
    }
    if (renorm) {
      for (int i = 0; i < ncell; ++i)
        if (!(asum[i] > 0)) {
          missed[(size_t)j] = i;
          return;
        }
      for (int64_t q = s0; q < s1; ++q) p->seg_afrac[q] /= asum[p->seg_cell[q]];
    } else {
      for (int64_t q = s0; q < s1; ++q) p->seg_afrac[q] /= p->V;
      std::vector<double> &e = defect[(size_t)j];
      e.resize(ncell);
      for (int i = 0; i < ncell; ++i) e[i] = ((asum_dd[i].hi - p->V) + asum_dd[i].lo) / p->V;
    }
  }, big);
  for (int j = 0; j < p->n_pairs; ++j)
    if (missed[(size_t)j] >= 0) {
      const int i = missed[(size_t)j];
      delete p;
      return fail(MOLC_ERR_INVALID_ARG,
                  "create: cell %d is crossed by no characteristic of azimuth pair %d; reduce ray_spacing", i, j);
    }
  // in pair order: the pairs' angular weights and, without renormalisation, the defect terms of the geometric
  // moments
  for (int j = 0; j < p->n_pairs; ++j) {
    // sum over the pair's directions of omega (times Omega components)
    double w0 = 0, wxx = 0, wxy = 0, wyy = 0;
    const double c = p->pairs[j].c, s = p->pairs[j].s;
    for (int q = 0; q < p->n_polar; ++q) {
      const PolarDev &pl = p->polar[(size_t)j * p->n_polar + q];
      const double ww = 2.0 * pl.w, s2 = pl.sinz * pl.sinz;
      w0 += ww;
      wxx += ww * s2 * c * c;
      wxy += ww * s2 * c * s;
      wyy += ww * s2 * s * s;
    }
    w0_all.add(w0);
    wxx_all.add(wxx);
    wxy_all.add(wxy);
    wyy_all.add(wyy);
    if (!renorm) {
      const std::vector<double> &e = defect[(size_t)j];
      for (int i = 0; i < ncell; ++i) {
        g0[i].add(w0 * e[i]);
        gxx[i].add(wxx * e[i]);
        gxy[i].add(wxy * e[i]);
        gyy[i].add(wyy * e[i]);
      }
      std::vector<double>().swap(defect[(size_t)j]);
    }
  }
  for (int i = 0; i < ncell; ++i) {
    g0[i].add(w0_all.value());
    gxx[i].add(wxx_all.value());
    gxy[i].add(wxy_all.value());
    gyy[i].add(wyy_all.value());
  }
  std::vector<double> geo(4 * (size_t)ncell);
  for (int i = 0; i < ncell; ++i) {
    geo[i] = g0[i].value();
    geo[ncell + i] = gxx[i].value();
    geo[2 * (size_t)ncell + i] = gxy[i].value();
    geo[3 * (size_t)ncell + i] = gyy[i].value();
  }

  // ---- device track table with canonical offsets
  std::vector<TrackDev> td(T);
  std::vector<int64_t> pair_nseg(p->n_pairs, 0);
  for (int j = 0; j < p->n_pairs; ++j)
    for (int64_t k = p->pair_track_off[j]; k < p->pair_track_off[j + 1]; ++k) pair_nseg[j] += p->tracks[k].nseg;
  for (int j = 0; j < p->n_pairs; ++j) {
    const int64_t seg_base = p->tracks[p->pair_track_off[j]].seg_off;
    for (int64_t k = p->pair_track_off[j]; k < p->pair_track_off[j + 1]; ++k) {
      const HostTrack &h = p->tracks[k];
      TrackDev &d = td[k];
      d.seg_off = h.seg_off;
      d.nseg = h.nseg;
      d.pair = j;
      d.entry_plus = h.entry_plus;
      d.entry_minus = h.entry_minus;
      d.width = h.width;
      d.canon_plus = h.seg_off - seg_base;
      d.canon_minus = pair_nseg[j] - (h.seg_off - seg_base) - h.nseg;
    }
  }
  p->dir_seg_off.assign(n + 1, 0);
  for (int m = 0; m < n; ++m) p->dir_seg_off[m + 1] = p->dir_seg_off[m] + pair_nseg[p->dir_pair[m]];

  std::vector<int2> seg32(S);   // FP32 sweep records {cell, l (f32 bits)}
  for (int64_t q = 0; q < S; ++q) {
    float lf = (float)p->seg_len[q];
    int2 r;
    r.x = p->seg_cell[q];
    std::memcpy(&r.y, &lf, 4);
    seg32[q] = r;
  }

  // ---- FP32 work items: one thread per (track, sense, group), numbered chunk-major, then by azimuth pair,
  // sense, track (the tracks of a pair are adjacent in space) and group.  Groups are tiled in chunks of up to
  // 32; the threads of one (track, sense) are consecutive, so a warp's record and cell-table loads are shared
  // by up to 32 lanes, and a sweep block (128 consecutive items) holds neighbouring parallel tracks of one
  // sense, which cross neighbouring cells at the same steps.  Blocks are launched longest first (block_order)
  // for load balance.
  // MOLC_TILED plans without the face or balance reductions use the tiled sweep when a tile of one cell or more
  // keeps a work item within shared memory; the others the bundle sweep and the moment gather below
  p->tiled = (flags & MOLC_TILED) && p->n_polar <= kMaxPolarFP32 && !(flags & (MOLC_FACES | MOLC_BALANCE));
  if (p->tiled) {
    bool fits = true;
    const molc_status ts = build_tiled(p, 0, 0, &fits);
    if (ts != MOLC_OK && fits) {
      free_device(p);
      delete p;
      return ts;
    }
    if (!fits) {
      p->tiled = false;
      g_last_error.clear();
    }
  }
  const int gc32 = std::min(p->G, 32);
  const int nch32 = p->n_polar <= kMaxPolarFP32 && !p->tiled ? (p->G + gc32 - 1) / gc32 : 0;
  if (T > (int64_t)0x3fffffff) {
    delete p;
    return fail(MOLC_ERR_INVALID_ARG, "create: too many characteristics");
  }
  std::vector<int2> items;
  items.reserve((size_t)T * 2 * p->G);
  std::vector<std::pair<int, int>> ts_order;   // (track, sense) in item order
  ts_order.reserve((size_t)(2 * T));
  for (int j = 0; j < p->n_pairs; ++j)
    for (int sense = 0; sense < 2; ++sense)
      for (int64_t k = p->pair_track_off[j]; k < p->pair_track_off[j + 1]; ++k) {
        td[k].pos[sense] = (int)ts_order.size();
        ts_order.emplace_back((int)k, sense);
      }
  for (int ch = 0; ch < nch32; ++ch) {
    const int gcount = std::min(gc32, p->G - ch * gc32);
    for (const auto &ks : ts_order)
      for (int gi = 0; gi < gcount; ++gi)
        items.push_back(make_int2(ks.first, ks.second | (gi << 1) | (ch << 16)));
  }
  p->n_items32 = (int64_t)items.size();
  p->acc_elems = (size_t)ncell * kOutputs * p->G;   // FP64 sweep accumulators
  // FP32 state bundles: block b of the sweep owns as many step slots as its longest item
  const int64_t n_blocks32 = (p->n_items32 + kSweepBlock - 1) / kSweepBlock;
  if (n_blocks32 > (int64_t)0x7fffffff) {
    delete p;
    return fail(MOLC_ERR_INVALID_ARG, "create: too many work items");
  }
  std::vector<int64_t> boff(n_blocks32 + 1, 0);
  std::vector<int> blen(n_blocks32), block_order(n_blocks32);
  for (int64_t b = 0; b < n_blocks32; ++b) {
    int longest = 0;
    for (int64_t i = b * kSweepBlock; i < std::min(p->n_items32, (b + 1) * kSweepBlock); ++i)
      longest = std::max(longest, td[items[i].x].nseg);
    blen[b] = longest;
    boff[b + 1] = boff[b] + longest;
    block_order[b] = (int)b;
  }
  std::stable_sort(block_order.begin(), block_order.end(), [&](int x, int y) { return blen[x] > blen[y]; });
  p->bundle_slots = boff[n_blocks32];
  p->n_blocks32 = n_blocks32;

  // ---- FP32 cell moments are gathered per cell from the swept state: for every cell, one entry per (track,
  // sense) segment crossing it, {item position of the (track, sense), step along that sense, A/V (f32 bits),
  // 2 pair + sense}; the + sense reaches the track's j-th segment at step j, the - sense at step nseg - 1 - j.
  // Entries of a cell are in track order (so grouped by azimuth pair), and the gathered sums deterministic.
  if (2 * S > (int64_t)0x7fffffff) {
    delete p;
    return fail(MOLC_ERR_INVALID_ARG, "create: too many segments for the FP32 state rows");
  }
  // Each cell's list is padded to a multiple of kGatherPad entries with zero-area copies of its last entry.
  if ((size_t)p->n_pairs * (3 * p->n_polar + 2) * sizeof(float) > kMaxGatherSmem) {
    delete p;
    return fail(MOLC_ERR_INVALID_ARG, "create: too many azimuth pairs for the FP32 moment kernel");
  }
  std::vector<int64_t> cell_off(nch32 ? (size_t)ncell + 1 : 0, 0);
  std::vector<int4> gent;
  if (nch32) {
    std::vector<int64_t> cnt(ncell, 0);
    for (int64_t q = 0; q < S; ++q) cnt[p->seg_cell[q]] += 2;
    for (int i = 0; i < ncell; ++i) cell_off[i + 1] = cell_off[i] + (cnt[i] + kGatherPad - 1) / kGatherPad * kGatherPad;
    gent.assign((size_t)cell_off[ncell], make_int4(0, 0, 0, 0));
    std::vector<int64_t> pos(cell_off.begin(), cell_off.end() - 1);
    // in parallel over ranges of cells: every range scans all tracks in order and writes its own cells' entries,
    // so each list is in track order as from one serial scan
    const int64_t n_ranges = std::min<int64_t>(ncell, 4 * (int64_t)std::max(1u, std::thread::hardware_concurrency()));
    parallel_for(n_ranges, [&](int64_t r) {
      const int c_lo = (int)(ncell * r / n_ranges), c_hi = (int)(ncell * (r + 1) / n_ranges);
      for (int64_t k = 0; k < T; ++k) {
        const TrackDev &t = td[k];
        for (int j = 0; j < t.nseg; ++j) {
          const int64_t q = t.seg_off + j;
          const int c = p->seg_cell[q];
          if (c < c_lo || c >= c_hi) continue;
          const float af = (float)p->seg_afrac[q];
          int afb;
          std::memcpy(&afb, &af, 4);
          gent[pos[c]++] = make_int4(t.pos[0], j, afb, 2 * t.pair);
          gent[pos[c]++] = make_int4(t.pos[1], t.nseg - 1 - j, afb, 2 * t.pair + 1);
        }
      }
      for (int i = c_lo; i < c_hi; ++i)
        for (int64_t e = pos[i]; e < cell_off[i + 1]; ++e) {
          gent[e] = gent[pos[i] - 1];
          gent[e].z = 0;   // zero area
        }
    }, big);
    // Per chunk, the (item position, step) of each entry becomes the state slot of the chunk's group 0 plus the
    // bundle length and lane (gather_slot); chunks 1.. are written from the chunk-0 list first, chunk 0 last,
    // in place.
    const int64_t n_ent = cell_off[ncell];
    gent.resize((size_t)(n_ent * nch32));
    std::atomic<bool> too_large(false);
    for (int ch = nch32 - 1; ch >= 0; --ch) {
      const int gcount = std::min(gc32, p->G - ch * gc32);
      const int64_t item_base = (int64_t)ch * 2 * T * gc32;
      const int64_t n_blocks = (n_ent + 65535) / 65536;   // entries in blocks of 64 Ki, in parallel
      parallel_for(n_blocks, [&](int64_t blk) {
        const int64_t e1 = std::min(n_ent, (blk + 1) * 65536);
        for (int64_t e = blk * 65536; e < e1; ++e) {
          int4 r = gent[e];
          const int64_t item = item_base + (int64_t)r.x * gcount;
          const int64_t b = item / kSweepBlock;
          const int lane = (int)(item % kSweepBlock);
          const int64_t slot = (boff[b] + r.y) * kSweepBlock + lane;
          const int64_t blen = boff[b + 1] - boff[b];
          if ((slot >> (32 + (32 - kGatherSlotHiShift))) != 0 || blen > (int64_t)kGatherBlenMask) {
            too_large = true;
            return;
          }
          r.x = (int)(uint32_t)(slot & 0xffffffffLL);
          r.y = (int)(((uint32_t)(slot >> 32) << kGatherSlotHiShift) | ((uint32_t)blen << 7) | (uint32_t)lane);
          gent[(size_t)(ch * n_ent + e)] = r;
        }
      }, big);
      if (too_large) {
        delete p;
        return fail(MOLC_ERR_INVALID_ARG, "create: FP32 state too large for the moment-gather entries");
      }
    }
  }
  // Work units of the moment gather: each cell's entry list in parts of at most kPartEntries entries, so that a
  // cell crossed by very many characteristics (fine ray spacing) is summed by several threads; the parts of a
  // split cell are added in order by a second kernel (deterministic).
  std::vector<int2> munit;
  std::vector<int4> mmulti;
  if (nch32) {
    static_assert(kPartEntries % kGatherPad == 0, "parts must hold whole gather batches");
    for (int i = 0; i < ncell; ++i) {
      const int64_t n = cell_off[i + 1] - cell_off[i];
      const int parts = (int)std::max<int64_t>(1, (n + kPartEntries - 1) / kPartEntries);
      if (parts > 1) mmulti.push_back(make_int4(i, (int)munit.size(), parts, 0));
      for (int k = 0; k < parts; ++k) munit.push_back(make_int2(i, k));
    }
  }
  p->n_split_cells = (int)mmulti.size();

  PlanView &v = p->view;
  v.nx = g.nx;
  v.ny = g.ny;
  v.ncell = ncell;
  v.G = p->G;
  v.n_pairs = p->n_pairs;
  v.n_polar = p->n_polar;
  v.n_tracks = T;
  v.n_track_segments = S;
  v.gc32 = gc32;
  v.sweep_depth = 4;
  v.hx = p->hx;
  v.hy = p->hy;
  // ---- face moments (Eq. 16, MOLC_FACES): the face each segment enters through, per sense.  The first segment
  // of a sense enters through the boundary face of its entry edge; the others through the face they share with
  // the cell walked before (a step through a vertex counts on the x-face of the cell entered).  Faces: x-face
  // (i, j) = line x = x0 + i hx in row j, numbered j (nx + 1) + i; y-face (i, j) = line y = y0 + j hy in column
  // i, numbered (nx + 1) ny + j nx + i.
  std::vector<int2> seg_face;
  const int nxf = (g.nx + 1) * g.ny;
  v.n_faces = (flags & MOLC_FACES) ? nxf + g.nx * (g.ny + 1) : 0;
  if (flags & MOLC_FACES) {
    seg_face.assign((size_t)S, make_int2(0, 0));
    auto edge_face = [&](int edge, int cell) {
      const int ix = cell % g.nx, iy = cell / g.nx;
      return edge == 0 ? iy * (g.nx + 1) : edge == 1 ? iy * (g.nx + 1) + g.nx
           : edge == 2 ? nxf + ix : nxf + g.ny * g.nx + ix;
    };
    auto between = [&](int prev, int cell) {
      const int ix = cell % g.nx, iy = cell / g.nx, px = prev % g.nx, py = prev / g.nx;
      return px != ix ? iy * (g.nx + 1) + std::max(px, ix) : nxf + std::max(py, iy) * g.nx + ix;
    };
    for (int64_t k = 0; k < T; ++k) {
      const TrackDev &t = td[k];
      for (int j = 0; j < t.nseg; ++j) {
        const int64_t q = t.seg_off + j;
        const int c = p->seg_cell[q];
        seg_face[q].x = j == 0 ? edge_face(t.entry_plus, c) : between(p->seg_cell[q - 1], c);
        seg_face[q].y = j == t.nseg - 1 ? edge_face(t.entry_minus, c) : between(p->seg_cell[q + 1], c);
      }
    }
    // accumulators shared by both precisions: [chunk][face][6][gc] (FP32 chunks of gc32 groups, FP64 one chunk of G)
    p->facc_elems = (size_t)v.n_faces * kOutputs * std::max<int64_t>((int64_t)nch32 * gc32, p->G);
  }
  if (p->host_only) {
    *out = p;
    return MOLC_OK;
  }
  // ---- upload
  molc_status st = MOLC_OK;
  size_t &tot = p->device_bytes;
#define UP(dst, src, cnt, what)                            \
  if (st == MOLC_OK) st = upload(&p->dst, src, cnt, tot, what);
  UP(d_tracks, td.data(), (size_t)T, "tracks")
  UP(d_seg32, seg32.data(), (size_t)S, "segments")
  UP(d_seg_cell, p->seg_cell.data(), (size_t)S, "segment cells")
  UP(d_seg_len, p->seg_len.data(), (size_t)S, "segment lengths")
  UP(d_seg_afrac, p->seg_afrac.data(), (size_t)S, "segment areas")
  UP(d_pairs, p->pairs.data(), p->pairs.size(), "pairs")
  UP(d_polar, p->polar.data(), p->polar.size(), "polar")
  UP(d_geo, geo.data(), geo.size(), "geometric moments")
  UP(d_dir_seg_off, p->dir_seg_off.data(), p->dir_seg_off.size(), "direction offsets")
  UP(d_status, (const int *)nullptr, 1, "status")
  UP(d_cell_off, cell_off.data(), cell_off.size(), "cell entry offsets")
  UP(d_gent, gent.data(), gent.size(), "cell entries")
  UP(d_boff, boff.data(), boff.size(), "state bundles")
  UP(d_seg_face, seg_face.data(), seg_face.size(), "segment faces")
  UP(d_munit, munit.data(), munit.size(), "moment units")
  UP(d_mmulti, mmulti.data(), mmulti.size(), "split cells")
  UP(d_mscratch, (const double *)nullptr, mmulti.empty() ? 0 : (size_t)nch32 * munit.size() * kOutputs * gc32,
     "moment partials")
  UP(d_facc, (const double *)nullptr, p->facc_elems, "face accumulators")
  UP(d_balance, (const unsigned long long *)nullptr, (flags & MOLC_BALANCE) ? 2 : 0, "balance residual")
  UP(d_block_order, block_order.data(), block_order.size(), "block order")
  UP(d_cdat, (const float4 *)nullptr, (size_t)nch32 * gc32 * ncell, "cell table")
  UP(d_cdB, (const float *)nullptr, (size_t)nch32 * gc32 * ncell, "cell table")
  UP(d_acc, (const double *)nullptr, p->acc_elems, "accumulators")
  UP(d_items32, items.data(), items.size(), "items")
#undef UP
  if (st == MOLC_OK) {
    cudaError_t e = cudaMemset(p->d_status, 0, sizeof(int));
    if (e == cudaSuccess && p->d_balance) e = cudaMemset(p->d_balance, 0, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) st = cuda_fail(e, "status");
  }
  if (st != MOLC_OK) {
    free_device(p);
    delete p;
    return st;
  }
  v.tracks = p->d_tracks;
  v.seg32 = p->d_seg32;
  v.seg_cell = p->d_seg_cell;
  v.seg_len = p->d_seg_len;
  v.seg_afrac = p->d_seg_afrac;
  v.pairs = p->d_pairs;
  v.polar = p->d_polar;
  v.geo = p->d_geo;
  v.dir_seg_off = p->d_dir_seg_off;
  v.status = p->d_status;
  v.cell_off = p->d_cell_off;
  v.gent = p->d_gent;
  v.gent_chunk = nch32 ? cell_off[ncell] : 0;
  v.boff = p->d_boff;
  v.block_order = p->d_block_order;
  v.seg_face = p->d_seg_face;
  v.facc = p->d_facc;
  v.munit = p->d_munit;
  v.n_munits = (int64_t)munit.size();
  v.mmulti = p->d_mmulti;
  v.n_mmulti = (int)mmulti.size();
  v.mscratch = p->d_mscratch;
  p->tune_key = plan_signature(g, quad, p->G, ray_spacing, layout, flags);
  if ((flags & MOLC_AUTOTUNE) && !p->host_only && (nch32 || p->tiled)) {
    st = tune_plan(p);
    if (st != MOLC_OK) {
      free_device(p);
      delete p;
      return st;
    }
  }
  v.balance = p->d_balance;   // after the autotuner, which times the plain sweep

  *out = p;
  return MOLC_OK;
}

molc_status molc_plan_get_info(const molc_plan *p, molc_plan_info *info) {
  if (!p || !info) return fail(MOLC_ERR_INVALID_ARG, "plan_get_info: NULL argument");
  info->G = p->G;
  info->nx = p->grid.nx;
  info->ny = p->grid.ny;
  info->n_dir = p->n_dir;
  info->n_azim_pairs = p->n_pairs;
  info->n_polar = p->n_polar;
  info->n_tracks = p->view.n_tracks;
  info->n_track_segments = p->view.n_track_segments;
  info->n_segments = 2 * (int64_t)p->n_polar * p->view.n_track_segments;
  info->n_updates = info->n_segments * p->G;
  info->fp32_groups_per_warp = p->view.gc32;
  info->device_bytes = p->device_bytes;
  info->fp32_sweep_depth = p->view.sweep_depth;
  info->n_faces = p->view.n_faces;
  info->n_split_cells = p->n_split_cells;
  info->fp32_tile_cells = p->tiled ? p->tv.TS : 0;
  info->fp32_tile_groups = p->tiled ? p->tv.GT : 0;
  info->fp32_tile_items = p->tiled ? p->tv.n_items : 0;
  info->fp32_sweep_blocks = p->tiled ? p->tgrid : 0;
  info->fp32_block_threads = p->tiled ? p->tthreads : 0;
  info->tuned_from_cache = p->tuned_from_cache ? 1 : 0;
  return MOLC_OK;
}

int64_t molc_intensity_count(const molc_plan *p) {
  return p ? 2 * (int64_t)p->n_polar * p->view.n_track_segments * p->G : 0;
}

// Elements of the stored deviations: FP64, one per (segment, direction, group); FP32, the bundle slots.
static int64_t state_elems(const molc_plan *p, molc_precision prec) {
  if (prec == MOLC_FP64) return molc_intensity_count(p);
  return p->tiled ? p->tstate_floats : p->bundle_slots * kSweepBlock * p->n_polar;
}

size_t molc_intensity_bytes(const molc_plan *p, molc_precision prec) {
  if (!p) return 0;
  return header_offset(state_elems(p, prec), prec == MOLC_FP64 ? 8 : 4, p->G, p->view.ncell) + kHeaderBytes;
}

static double *bref_of(const molc_plan *p, molc_precision prec, void *I) {
  return (double *)((char *)I + bref_offset(state_elems(p, prec), prec == MOLC_FP64 ? 8 : 4));
}

extern "C++" {
namespace {
size_t state_bytes_fp32(const molc_plan *p) { return molc_intensity_bytes(p, MOLC_FP32); }
}  // namespace
}

static double *header_of(const molc_plan *p, molc_precision prec, void *I) {
  return (double *)((char *)I +
                    header_offset(state_elems(p, prec), prec == MOLC_FP64 ? 8 : 4, p->G, p->view.ncell));
}

extern "C++" {
namespace {
double *bref_ptr(const molc_plan *p, molc_precision prec, void *I) { return bref_of(p, prec, I); }
double *header_ptr(const molc_plan *p, molc_precision prec, void *I) { return header_of(p, prec, I); }
}  // namespace
}

static molc_status check_prec(const molc_plan *p, molc_precision prec, const char *who) {
  if (p->host_only) return fail(MOLC_ERR_INVALID_ARG, "%s: the plan was created with MOLC_HOST_ONLY", who);
  if (prec != MOLC_FP64 && prec != MOLC_FP32) return fail(MOLC_ERR_INVALID_ARG, "%s: bad precision", who);
  if (prec == MOLC_FP32 && p->n_polar > kMaxPolarFP32)
    return fail(MOLC_ERR_INVALID_ARG, "%s: the FP32 sweep supports at most %d polar cosines per azimuth", who,
                kMaxPolarFP32);
  return MOLC_OK;
}

molc_status molc_intensity_init(molc_plan *p, molc_precision prec, void *I, const double *B, molc_stream stream) {
  if (!p || !I || !B) return fail(MOLC_ERR_INVALID_ARG, "intensity_init: NULL argument");
  molc_status s = check_prec(p, prec, "intensity_init");
  if (s) return s;
  DeviceGuard dg(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nb = (size_t)p->G * p->view.ncell * sizeof(double);
  cudaError_t e = cudaMemsetAsync(I, 0, bref_offset(state_elems(p, prec), prec == MOLC_FP64 ? 8 : 4), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bref_of(p, prec, I), B, nb, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = launch_set_scale(p->view, prec, B, header_of(p, prec, I), st);
  return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "intensity_init");
}

// One tiled FP32 step after the scale update: the prep launch (cell tables, ticket, epoch; it also stores this
// call's instance for the sweep) and the persistent sweep.  ev: events {.., before sweep, after, after} or null.
static cudaError_t tile_step(molc_plan *p, const SweepArgs &a, const TileView &tv, cudaStream_t st,
                             cudaEvent_t *ev) {
  TileInst ti;
  ti.v = p->view;
  ti.t = tv;
  ti.a = a;
  cudaError_t e = launch_tile_prep_one(ti, p->d_tinst, p->d_tprep, p->n_tprep, tv.ctrl, st);
  if (e == cudaSuccess && ev) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess)
    e = launch_tile_sweep(p->d_tinst, p->d_tqueue, tv.n_items, tv.ctrl, p->np_class, p->tshape, p->tgrid,
                          p->tthreads, st);
  if (e == cudaSuccess && ev) {
    e = cudaEventRecord(ev[2], st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3], st);
  }
  return e;
}

// Autotuner of the tiled FP32 sweep: the planner's configuration and its neighbours (half and twice the tile
// side, half and twice the groups per work item, the other block size), each laid out and timed (one warm-up and
// two timed steps of prep + persistent sweep on temporary zero inputs, an FP32 state of that layout); the fastest
// is laid out again and kept.  Configurations the planner rejects (a work item beyond shared memory) are skipped.
// The configuration changes no segment update and no output beyond the moment summation order.
static molc_status autotune_tiled(molc_plan *p, double *best_ms_out) {
  DeviceGuard dg(p->device);
  const int ts0 = p->tv.TS, gt0 = p->tv.GT, th0 = p->tthreads;
  std::vector<std::array<int, 3>> cand = {{ts0, gt0, th0}, {ts0, gt0, th0 == 128 ? 256 : 128}};
  if (ts0 / 2 >= 2) cand.push_back({ts0 / 2, gt0, th0});
  cand.push_back({2 * ts0, gt0, th0});
  if (gt0 / 2 >= 1) cand.push_back({ts0, gt0 / 2, th0});
  if (2 * gt0 <= std::min(p->G, 32)) cand.push_back({ts0, 2 * gt0, th0});
  const int64_t cg = (int64_t)p->G * p->view.ncell;
  double *in = nullptr, *mom = nullptr;   // kappa, B [G][cell], bnd [4][G]; 6 x [G][cell]
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void **)&in, (2 * cg + 4 * (int64_t)p->G) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&mom, 6 * cg * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(in, 0, (2 * cg + 4 * (int64_t)p->G) * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  std::array<int, 3> best = cand[0];
  float best_ms = 0;
  molc_status st = MOLC_OK;
  for (const auto &c : cand) {
    if (e != cudaSuccess || st != MOLC_OK) break;
    bool fits = true;
    st = build_tiled(p, c[0], c[1], &fits, c[2]);
    if (st != MOLC_OK) {
      if (fits) break;   // a device failure, not a rejected configuration
      st = MOLC_OK;
      g_last_error.clear();
      continue;
    }
    void *I = nullptr;
    e = cudaMalloc(&I, state_bytes_fp32(p));
    if (e != cudaSuccess) break;
    SweepArgs a{};
    a.kappa = in;
    a.B = in + cg;
    a.bnd = in + 2 * cg;
    a.c = a.dt = 1.0;
    a.inv_c = a.inv_cdt = 1.0;
    a.I = I;
    a.Bref = bref_ptr(p, MOLC_FP32, I);
    a.scale = header_ptr(p, MOLC_FP32, I);
    a.out = molc_moments{mom, mom + cg, mom + 2 * cg, mom + 3 * cg, mom + 4 * cg, mom + 5 * cg};
    e = cudaMemset(I, 0, state_bytes_fp32(p));
    if (e == cudaSuccess) e = cudaMemcpy(a.Bref, a.B, cg * sizeof(double), cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess) e = launch_set_scale(p->view, MOLC_FP32, a.B, const_cast<double *>(a.scale), nullptr);
    if (e == cudaSuccess) e = tile_step(p, a, p->tv, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = tile_step(p, a, p->tv, nullptr, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaFree(I);
    if (e == cudaSuccess && (best_ms == 0 || ms < best_ms)) {
      best_ms = ms;
      best = {p->tv.TS, p->tv.GT, p->tthreads};
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (mom) cudaFree(mom);
  if (in) cudaFree(in);
  if (st != MOLC_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "create: autotune (tiled)");
  st = build_tiled(p, best[0], best[1], nullptr, best[2]);
  if (st != MOLC_OK) return st;
  if (best_ms_out) *best_ms_out = best_ms / 2.0;
  int code = 0;
  cudaMemcpy(&code, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemset(p->d_status, 0, sizeof(int));   // the temporaries' checks leave no trace
  return code == kStatusTimeout ? fail(MOLC_ERR_TIMEOUT, "create: autotune (tiled): a bounded wait gave up")
                                : MOLC_OK;
}

// MOLC_AUTOTUNE: the configuration recorded in the tuning cache for this plan, device and build when there is
// one (nothing timed), else the autotuner's choice, then recorded.  A cache that cannot be written leaves the
// plan tuned and the file as it was.
static molc_status tune_plan(molc_plan *p) {
  const std::string dev = device_signature(p->device);
  TuneRecord rec;
  if (tune_cache_enabled() && tune_cache_lookup(p->tune_key, dev, kBuildId, rec)) {
    bool applied = false;
    if (p->tiled && rec.tile_cells > 0) {
      bool fits = true;
      const molc_status st = build_tiled(p, rec.tile_cells, rec.tile_groups, &fits, rec.block_threads);
      if (st != MOLC_OK && fits) return st;
      applied = st == MOLC_OK;
      if (!applied) g_last_error.clear();
    } else if (!p->tiled) {
      for (int d : kSweepDepths)
        if (d == rec.sweep_depth) applied = true;
      if (applied) p->view.sweep_depth = rec.sweep_depth;
    }
    if (applied) {
      p->tuned_from_cache = true;
      return MOLC_OK;
    }
  }
  double ms = 0;
  const molc_status st = p->tiled ? autotune_tiled(p, &ms) : autotune(p, &ms);
  if (st != MOLC_OK) return st;
  if (tune_cache_enabled()) {
    rec = TuneRecord{};
    rec.key = p->tune_key;
    rec.device = dev;
    rec.build = kBuildId;
    rec.sweep_depth = p->tiled ? 0 : p->view.sweep_depth;
    rec.tile_cells = p->tiled ? p->tv.TS : 0;
    rec.tile_groups = p->tiled ? p->tv.GT : 0;
    rec.block_threads = p->tiled ? p->tthreads : 0;
    rec.best_ms = ms;
    std::string why;
    tune_cache_store(rec, why);
  }
  return MOLC_OK;
}

molc_status molc_tune_cache(const char *path, int *n_entries) {
  std::string why;
  const int n = tune_cache_set(path, why);
  if (n < 0) return fail(MOLC_ERR_INVALID_ARG, "tune_cache: %s", why.c_str());
  if (n_entries) *n_entries = n;
  return MOLC_OK;
}

// molc_sweep, and with factor outputs molc_sweep_closure (`who` names the entry point in error messages).
static molc_status sweep_step(molc_plan *p, molc_precision prec, const double *kappa, const double *B, double c,
                              double dt, void *I, const double *bnd, const molc_moments *out, double *fxx,
                              double *fxy, double *fyy, molc_stream stream, const char *who) {
  if (!p || !kappa || !B || !I || !bnd || !out) return fail(MOLC_ERR_INVALID_ARG, "%s: NULL argument", who);
  if (!out->E || !out->Fx || !out->Fy || !out->Nxx || !out->Nxy || !out->Nyy)
    return fail(MOLC_ERR_INVALID_ARG, "%s: NULL moment array", who);
  if (!finite_pos(c) || !finite_pos(dt)) return fail(MOLC_ERR_INVALID_ARG, "%s: need c > 0 and dt > 0", who);
  molc_status s = check_prec(p, prec, who);
  if (s) return s;
  DeviceGuard dg(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  SweepArgs a{};
  a.kappa = kappa;
  a.B = B;
  a.bnd = bnd;
  a.c = c;
  a.dt = dt;
  a.inv_c = 1.0 / c;
  a.inv_cdt = 1.0 / (c * dt);
  a.I = I;
  a.Bref = bref_of(p, prec, I);
  a.scale = header_of(p, prec, I);
  a.out = *out;
  a.cdat = p->d_cdat;
  a.cdB = p->d_cdB;
  a.acc = p->d_acc;
  a.items = p->d_items32;
  a.n_items = p->n_items32;
  a.fxx = fxx;
  a.fxy = fxy;
  a.fyy = fyy;
  cudaError_t e = cudaSuccess;
  if (p->d_facc) {
    e = cudaMemsetAsync(p->d_facc, 0, p->facc_elems * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, who, "clear face accumulators");
  }
  if (p->d_balance) {
    e = cudaMemsetAsync(p->d_balance, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_balance_scale(p->view, B, bnd, st);
    if (e != cudaSuccess) return cuda_fail(e, who, "balance check set-up");
  }
  if (prec == MOLC_FP64) {   // the FP32 path gathers its moments and has no accumulators
    e = cudaMemsetAsync(p->d_acc, 0, (size_t)p->G * p->view.ncell * kOutputs * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, who, "clear accumulators");
  } else {
    e = launch_update_scale(p->view, B, bnd, header_of(p, prec, I), st);
    if (e != cudaSuccess) return cuda_fail(e, who, "scale");
  }
  const bool timed = p->timing && p->n_timed < kMaxTimed;
  cudaEvent_t *ev = timed ? &p->ev[4 * (size_t)p->n_timed] : nullptr;
  if (prec == MOLC_FP32 && p->tiled) {
    if (timed) cudaEventRecord(ev[0], st);
    e = tile_step(p, a, p->tv, st, timed ? ev : nullptr);
    if (e != cudaSuccess) return cuda_fail(e, who, "tiled sweep");
    if (timed) ++p->n_timed;
    return MOLC_OK;
  }
  if (timed) cudaEventRecord(ev[0], st);
  e = launch_prep(p->view, prec, a, st);
  if (e != cudaSuccess) return cuda_fail(e, who, "prep");
  if (timed) cudaEventRecord(ev[1], st);
  e = prec == MOLC_FP64 ? launch_sweep_fp64(p->view, a, st) : launch_sweep_fp32(p->view, a, st);
  if (e != cudaSuccess) return cuda_fail(e, who, "sweep kernel");
  if (timed) cudaEventRecord(ev[2], st);
  e = launch_finalize(p->view, prec, a, st);
  if (e != cudaSuccess) return cuda_fail(e, who, "finalize");
  if (timed) {
    cudaEventRecord(ev[3], st);
    ++p->n_timed;
  }
  return MOLC_OK;
}

molc_status molc_sweep(molc_plan *p, molc_precision prec, const double *kappa, const double *B, double c,
                       double dt, void *I, const double *bnd, const molc_moments *out, molc_stream stream) {
  return sweep_step(p, prec, kappa, B, c, dt, I, bnd, out, nullptr, nullptr, nullptr, stream, "sweep");
}

molc_status molc_sweep_closure(molc_plan *p, molc_precision prec, const double *kappa, const double *B, double c,
                               double dt, void *I, const double *bnd, const molc_moments *out, double *fxx,
                               double *fxy, double *fyy, molc_stream stream) {
  if (!fxx || !fxy || !fyy) return fail(MOLC_ERR_INVALID_ARG, "sweep_closure: NULL factor array");
  return sweep_step(p, prec, kappa, B, c, dt, I, bnd, out, fxx, fxy, fyy, stream, "sweep_closure");
}

molc_status molc_sweep_static_scratch(molc_plan *p, molc_precision prec, const double *kappa, const double *B,
                                      double c, double dt, void *I, const double *bnd, const molc_moments *out,
                                      molc_stream stream) {
  if (!p || !kappa || !B || !I || !bnd || !out)
    return fail(MOLC_ERR_INVALID_ARG, "sweep_static_scratch: NULL argument");
  if (!out->E || !out->Fx || !out->Fy || !out->Nxx || !out->Nxy || !out->Nyy)
    return fail(MOLC_ERR_INVALID_ARG, "sweep_static_scratch: NULL moment array");
  if (!finite_pos(c) || !finite_pos(dt))
    return fail(MOLC_ERR_INVALID_ARG, "sweep_static_scratch: need c > 0 and dt > 0");
  molc_status s = check_prec(p, prec, "sweep_static_scratch");
  if (s) return s;
  if (prec == MOLC_FP32 && p->tiled) {
    // workspace carved from the static array: control words, item flags, quadrant counts (left at zero by every
    // completed call; the array starts at zero), cell tables (rewritten by every call), quadrant partials and the
    // boundary buffer (written before they are read within the call)
    TileView tv = p->tv;
    const TileWorkspace w = tile_workspace(tv, p->G, p->n_polar, p->tn_pieces);
    if (w.total > kStaticScratchBytes)
      return fail(MOLC_ERR_INVALID_ARG,
                  "sweep_static_scratch: this plan needs %zu bytes of workspace (%d cells x %d groups), more than "
                  "the %zu-byte static scratch; use molc_sweep",
                  w.total, p->view.ncell, p->G, kStaticScratchBytes);
    DeviceGuard dg(p->device);
    cudaStream_t st = (cudaStream_t)stream;
    void *base = nullptr;
    cudaError_t e = static_scratch_address(&base);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: scratch address");
    tile_carve(tv, (char *)base, w);
    // the control words, flags and counts start at zero on every call: other calls (an FP64 one, another plan's)
    // leave other data in the array
    e = cudaMemsetAsync(base, 0, w.ctrl + w.flags + w.cnt, st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: clear control words");
    SweepArgs a{};
    a.kappa = kappa;
    a.B = B;
    a.bnd = bnd;
    a.c = c;
    a.dt = dt;
    a.inv_c = 1.0 / c;
    a.inv_cdt = 1.0 / (c * dt);
    a.I = I;
    a.Bref = bref_of(p, prec, I);
    a.scale = header_of(p, prec, I);
    a.out = *out;
    e = launch_update_scale(p->view, B, bnd, header_of(p, prec, I), st);
    if (e == cudaSuccess) e = tile_step(p, a, tv, st, nullptr);
    return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "sweep_static_scratch: tiled sweep");
  }
  // workspace carved from the static array: FP64, the accumulators [cell][6][G] (must start at zero, cleared
  // below on every call); FP32, the cell tables [chunk][cell][gc] (fully written by prep_kernel)
  const Layout L = layout_for(p->view, prec);
  const size_t rows = (size_t)L.n_chunks * L.gc * p->view.ncell;
  auto up256 = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t acc_bytes = prec == MOLC_FP64 ? up256(rows * kOutputs * sizeof(double)) : 0;
  const size_t cdat_bytes = prec == MOLC_FP32 ? up256(rows * sizeof(float4)) : 0;
  const size_t cdB_bytes = prec == MOLC_FP32 ? up256(rows * sizeof(float)) : 0;
  const size_t need = acc_bytes + cdat_bytes + cdB_bytes;
  if (need > kStaticScratchBytes)
    return fail(MOLC_ERR_INVALID_ARG,
                "sweep_static_scratch: this plan needs %zu bytes of workspace (%d cells x %d groups), more than "
                "the %zu-byte static scratch; use molc_sweep",
                need, p->view.ncell, p->G, kStaticScratchBytes);
  DeviceGuard dg(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  void *base = nullptr;
  cudaError_t e = static_scratch_address(&base);
  if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: scratch address");
  char *b = (char *)base;
  SweepArgs a{};
  a.kappa = kappa;
  a.B = B;
  a.bnd = bnd;
  a.c = c;
  a.dt = dt;
  a.inv_c = 1.0 / c;
  a.inv_cdt = 1.0 / (c * dt);
  a.I = I;
  a.Bref = bref_of(p, prec, I);
  a.scale = header_of(p, prec, I);
  a.out = *out;
  a.acc = prec == MOLC_FP64 ? (double *)b : nullptr;
  a.cdat = prec == MOLC_FP32 ? (float4 *)b : nullptr;
  a.cdB = prec == MOLC_FP32 ? (float *)(b + cdat_bytes) : nullptr;
  a.items = p->d_items32;
  a.n_items = p->n_items32;
  if (p->d_facc) {
    e = cudaMemsetAsync(p->d_facc, 0, p->facc_elems * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: clear face accumulators");
  }
  if (p->d_balance) {
    // the balance floor (word 1) follows this call's B and boundary; the residual record (word 0) is kept
    e = cudaMemsetAsync(p->d_balance + 1, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = launch_balance_scale(p->view, B, bnd, st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: balance check set-up");
  }
  if (prec == MOLC_FP64) {
    e = cudaMemsetAsync(a.acc, 0, rows * kOutputs * sizeof(double), st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: clear accumulators");
  } else {
    e = launch_update_scale(p->view, B, bnd, header_of(p, prec, I), st);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: scale");
  }
  e = launch_prep(p->view, prec, a, st);
  if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: prep");
  e = prec == MOLC_FP64 ? launch_sweep_fp64(p->view, a, st) : launch_sweep_fp32(p->view, a, st);
  if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: sweep kernel");
  e = launch_finalize(p->view, prec, a, st);
  if (e != cudaSuccess) return cuda_fail(e, "sweep_static_scratch: finalize");
  return MOLC_OK;
}

}  // extern "C"

struct molc_batch {
  int device = 0;
  std::vector<molc_plan *> plans;
  molc::BatchInst *d_inst = nullptr;
  std::vector<molc::BatchInst> h_inst;
  int4 *d_prep = nullptr;
  int n_prep = 0;
  struct SweepClass {
    int n_polar, depth;
    int2 *d_map;
    int n;
  };
  struct MomentClass {
    int n_polar;
    int4 *d_map;
    int n;
    size_t smem;
  };
  std::vector<SweepClass> sweeps;
  std::vector<MomentClass> moments;
  int4 *d_combine = nullptr;
  int n_combine = 0;
  bool bound = false;
  // tiled plans: one prep and one persistent sweep launch over the items of every instance
  bool tiled = false;
  molc::TileInst *d_tinst = nullptr;
  std::vector<molc::TileInst> h_tinst;
  int2 *d_tqueue = nullptr;
  int n_tqueue = 0;
  int4 *d_tprep = nullptr;
  int n_tprep = 0;
  int *d_ticket = nullptr;
  molc::TileShape shape{};
  int np_max = 0, grid = 0, threads = 0;
  // the scale update over several blocks per instance: int4 {instance, block, blocks of the instance, 0}
  int4 *d_scale_map = nullptr;
  int n_scale = 0;
};

namespace {
void batch_free(molc_batch *b) {
  DeviceGuard dg(b->device);
  for (void *q : {(void *)b->d_tinst, (void *)b->d_tqueue, (void *)b->d_tprep, (void *)b->d_ticket,
                  (void *)b->d_scale_map})
    if (q) cudaFree(q);
  if (b->d_inst) cudaFree(b->d_inst);
  if (b->d_prep) cudaFree(b->d_prep);
  if (b->d_combine) cudaFree(b->d_combine);
  for (auto &c : b->sweeps)
    if (c.d_map) cudaFree(c.d_map);
  for (auto &c : b->moments)
    if (c.d_map) cudaFree(c.d_map);
  delete b;
}

template <class T> cudaError_t upload_vec(T **dst, const std::vector<T> &v) {
  *dst = nullptr;
  if (v.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void **)dst, v.size() * sizeof(T));
  if (e == cudaSuccess) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}
}  // namespace

extern "C" {

molc_status molc_batch_create(molc_plan *const *plans, int n, molc_batch **out) {
  if (!out) return fail(MOLC_ERR_INVALID_ARG, "batch_create: out is NULL");
  *out = nullptr;
  if (!plans || n < 1) return fail(MOLC_ERR_INVALID_ARG, "batch_create: need n >= 1 plans");
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return fail(MOLC_ERR_INVALID_ARG, "batch_create: plan %d is NULL", i);
    if (plans[i]->host_only) return fail(MOLC_ERR_INVALID_ARG, "batch_create: plan %d is MOLC_HOST_ONLY", i);
    if (plans[i]->n_polar > kMaxPolarFP32 || (plans[i]->n_items32 == 0 && !plans[i]->tiled))
      return fail(MOLC_ERR_INVALID_ARG, "batch_create: plan %d has no FP32 sweep (more than %d polar cosines)", i,
                  kMaxPolarFP32);
    if (plans[i]->device != dev) return fail(MOLC_ERR_INVALID_ARG, "batch_create: plan %d is on another device", i);
    if (plans[i]->d_balance)
      return fail(MOLC_ERR_INVALID_ARG, "batch_create: plan %d was created with MOLC_BALANCE (the check runs in "
                                        "molc_sweep only)", i);
    if (plans[i]->d_facc)
      return fail(MOLC_ERR_INVALID_ARG, "batch_create: plan %d was created with MOLC_FACES (face moments come from "
                                        "molc_sweep only)", i);
  }
  int n_tiled = 0;
  for (int i = 0; i < n; ++i) n_tiled += plans[i]->tiled ? 1 : 0;
  if (n_tiled != 0 && n_tiled != n)
    return fail(MOLC_ERR_INVALID_ARG, "batch_create: plans with and without the tiled FP32 sweep cannot be batched "
                                      "together (%d of %d are tiled)", n_tiled, n);
  auto b = new molc_batch();
  b->device = dev;
  b->plans.assign(plans, plans + n);
  {
    std::vector<int4> smap;
    for (int i = 0; i < n; ++i) {
      const int64_t cg = (int64_t)plans[i]->G * plans[i]->view.ncell;
      const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(64, (cg + 16383) / 16384));
      for (int k = 0; k < nb; ++k) smap.push_back(make_int4(i, k, nb, 0));
    }
    b->n_scale = (int)smap.size();
    if (upload_vec(&b->d_scale_map, smap) != cudaSuccess) {
      batch_free(b);
      return fail(MOLC_ERR_CUDA, "batch_create: scale map");
    }
  }
  if (n_tiled) {
    // items of all instances, those with the longest remaining wavefront first (an item's upstream items have a
    // longer one, so they come earlier); prep blocks of all instances
    b->tiled = true;
    b->h_tinst.resize(n);
    std::vector<std::pair<std::pair<int, int>, int2>> items;   // ((-remaining, instance), {instance, item})
    std::vector<int4> prep;
    TileShape sh{0, 0, 0, 0, 0, plans[0]->n_polar};
    for (int i = 0; i < n; ++i) {
      const molc_plan *p = plans[i];
      const TileView &t = p->tv;
      std::vector<int2> q(t.n_items);
      std::vector<TileGeom> geoms(t.n_geoms);
      cudaError_t e = cudaMemcpy(q.data(), p->d_tqueue, q.size() * sizeof(int2), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess)
        e = cudaMemcpy(geoms.data(), t.geoms, geoms.size() * sizeof(TileGeom), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) {
        batch_free(b);
        return cuda_fail(e, "batch_create: reading the tiled queue");
      }
      const int D = t.ntx + t.nty - 1;
      for (const int2 &x : q) {
        const TileGeom &gm = geoms[x.y % t.n_geoms];
        items.push_back({{-(D - 1 - gm.delta), i}, make_int2(i, x.y)});
      }
      const int tpb = std::max(1, 256 / (t.TS * t.TS));
      for (int g = 0; g < p->G; ++g)
        for (int t0 = 0; t0 < t.n_tiles; t0 += tpb) prep.push_back(make_int4(i, t0, g, g == 0 && t0 == 0));
      sh.max_item_floats = std::max(sh.max_item_floats, p->tshape.max_item_floats);
      sh.cd_entries = std::max(sh.cd_entries, p->tshape.cd_entries);
      sh.max_len = std::max(sh.max_len, p->tshape.max_len);
      sh.n_pairs = std::max(sh.n_pairs, p->tshape.n_pairs);
      sh.split_units = std::max(sh.split_units, p->tshape.split_units);
      if (p->n_polar != sh.np_exact) sh.np_exact = 0;
      b->np_max = std::max(b->np_max, p->np_class);
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<std::pair<int, int>, int2> &x, const std::pair<std::pair<int, int>, int2> &y) {
                       return x.first.first < y.first.first;
                     });
    std::vector<int2> queue(items.size());
    for (size_t k = 0; k < items.size(); ++k) queue[k] = items[k].second;
    b->shape = sh;
    b->n_tqueue = (int)queue.size();
    b->n_tprep = (int)prep.size();
    cudaError_t e = cudaMalloc((void **)&b->d_tinst, n * sizeof(TileInst));
    if (e == cudaSuccess) e = upload_vec(&b->d_tqueue, queue);
    if (e == cudaSuccess) e = upload_vec(&b->d_tprep, prep);
    if (e == cudaSuccess) e = cudaMalloc((void **)&b->d_ticket, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_ticket, 0, sizeof(int));
    if (e != cudaSuccess) {
      batch_free(b);
      return cuda_fail(e, "batch_create");
    }
    for (int i = 0; i < n; ++i) b->threads = std::max(b->threads, plans[i]->tthreads);
    b->grid = tile_sweep_grid(b->np_max, tile_sweep_smem(sh, b->np_max), b->threads);
    *out = b;
    return MOLC_OK;
  }
  b->h_inst.resize(n);
  // block maps
  std::vector<int4> prep;
  std::map<std::pair<int, int>, std::vector<std::pair<int, int2>>> sw;   // (np, depth) -> (length, block)
  std::map<int, std::vector<int4>> mo;
  std::map<int, size_t> mo_smem;
  std::vector<int4> comb;
  for (int i = 0; i < n; ++i) {
    const molc_plan *p = plans[i];
    const PlanView &v = p->view;
    const Layout L = layout_for(v, MOLC_FP32);
    const int n_tiles = (v.ncell + 31) / 32;
    for (int ch = 0; ch < L.n_chunks; ++ch)
      for (int t = 0; t < n_tiles; ++t) prep.push_back(make_int4(i, ch, t, ch == 0 && t == 0));
    // bundle lengths from the plan's host copy of the offsets
    std::vector<int64_t> boff(p->n_blocks32 + 1);
    if (cudaMemcpy(boff.data(), p->d_boff, boff.size() * sizeof(int64_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
      batch_free(b);
      return fail(MOLC_ERR_CUDA, "batch_create: reading bundle offsets");
    }
    auto &cls = sw[{p->n_polar, v.sweep_depth}];
    for (int64_t k = 0; k < p->n_blocks32; ++k)
      cls.push_back({(int)(boff[k + 1] - boff[k]), make_int2(i, (int)k)});
    auto &m = mo[p->n_polar];
    for (int ch = 0; ch < L.n_chunks; ++ch) {
      const int gcount = std::min(L.gc, v.G - ch * L.gc);
      const int64_t nb = (v.n_munits * gcount + 127) / 128;
      for (int64_t k = 0; k < nb; ++k) m.push_back(make_int4(i, ch, (int)k, 0));
      const int64_t nc = ((int64_t)v.n_mmulti * gcount + 127) / 128;
      for (int64_t k = 0; k < nc; ++k) comb.push_back(make_int4(i, ch, (int)k, 0));
    }
    mo_smem[p->n_polar] = std::max(mo_smem[p->n_polar], (size_t)v.n_pairs * (3 * v.n_polar + 2) * sizeof(float));
  }
  cudaError_t e = cudaMalloc((void **)&b->d_inst, n * sizeof(BatchInst));
  if (e == cudaSuccess) e = upload_vec(&b->d_prep, prep);
  b->n_prep = (int)prep.size();
  if (e == cudaSuccess) e = upload_vec(&b->d_combine, comb);
  b->n_combine = (int)comb.size();
  for (auto &kv : sw) {
    if (e != cudaSuccess) break;
    auto &lst = kv.second;
    std::stable_sort(lst.begin(), lst.end(), [](const std::pair<int, int2> &x, const std::pair<int, int2> &y) {
      return x.first > y.first;   // longest bundles first, across instances
    });
    std::vector<int2> map(lst.size());
    for (size_t k = 0; k < lst.size(); ++k) map[k] = lst[k].second;
    molc_batch::SweepClass c{kv.first.first, kv.first.second, nullptr, (int)map.size()};
    e = upload_vec(&c.d_map, map);
    b->sweeps.push_back(c);
  }
  for (auto &kv : mo) {
    if (e != cudaSuccess) break;
    molc_batch::MomentClass c{kv.first, nullptr, (int)kv.second.size(), mo_smem[kv.first]};
    e = upload_vec(&c.d_map, kv.second);
    b->moments.push_back(c);
  }
  if (e != cudaSuccess) {
    batch_free(b);
    return cuda_fail(e, "batch_create");
  }
  *out = b;
  return MOLC_OK;
}

molc_status molc_batch_bind(molc_batch *b, const molc_sweep_args *args) {
  if (!b || !args) return fail(MOLC_ERR_INVALID_ARG, "batch_bind: NULL argument");
  for (size_t i = 0; i < b->plans.size(); ++i) {
    const molc_sweep_args &x = args[i];
    const molc_plan *p = b->plans[i];
    if (!x.kappa || !x.B || !x.I || !x.bnd || !x.out.E || !x.out.Fx || !x.out.Fy || !x.out.Nxx || !x.out.Nxy ||
        !x.out.Nyy)
      return fail(MOLC_ERR_INVALID_ARG, "batch_bind: instance %zu: NULL argument", i);
    if (!finite_pos(x.c) || !finite_pos(x.dt))
      return fail(MOLC_ERR_INVALID_ARG, "batch_bind: instance %zu: need c > 0 and dt > 0", i);
    const bool f = x.fxx || x.fxy || x.fyy;
    if (f && !(x.fxx && x.fxy && x.fyy))
      return fail(MOLC_ERR_INVALID_ARG, "batch_bind: instance %zu: give all of fxx, fxy, fyy or none", i);
    SweepArgs a0{};
    SweepArgs &a = b->tiled ? a0 : b->h_inst[i].a;
    if (!b->tiled) {
      b->h_inst[i].v = p->view;
      b->h_inst[i].L = layout_for(p->view, MOLC_FP32);
    }
    a = SweepArgs{};
    a.kappa = x.kappa;
    a.B = x.B;
    a.bnd = x.bnd;
    a.c = x.c;
    a.dt = x.dt;
    a.inv_c = 1.0 / x.c;
    a.inv_cdt = 1.0 / (x.c * x.dt);
    a.I = x.I;
    a.Bref = bref_of(p, MOLC_FP32, x.I);
    a.scale = header_of(p, MOLC_FP32, x.I);
    a.out = x.out;
    a.cdat = p->d_cdat;
    a.cdB = p->d_cdB;
    a.acc = nullptr;
    a.items = p->d_items32;
    a.n_items = p->n_items32;
    a.fxx = x.fxx;   // factors formed where the moments are assembled
    a.fxy = x.fxy;
    a.fyy = x.fyy;
    if (b->tiled) {
      a.cdat = nullptr;
      a.cdB = nullptr;
      a.items = nullptr;
      a.n_items = 0;
      TileInst &ti = b->h_tinst[i];
      ti.v = p->view;
      ti.t = p->tv;
      ti.a = a;
    }
  }
  DeviceGuard dg(b->device);
  cudaError_t e = b->tiled ? cudaMemcpy(b->d_tinst, b->h_tinst.data(), b->h_tinst.size() * sizeof(TileInst),
                                        cudaMemcpyHostToDevice)
                           : cudaMemcpy(b->d_inst, b->h_inst.data(), b->h_inst.size() * sizeof(BatchInst),
                                        cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch_bind");
  b->bound = true;
  return MOLC_OK;
}

molc_status molc_batch_sweep(molc_batch *b, molc_stream stream) {
  if (!b) return fail(MOLC_ERR_INVALID_ARG, "batch_sweep: NULL batch");
  if (!b->bound) return fail(MOLC_ERR_INVALID_ARG, "batch_sweep: no arguments bound (molc_batch_bind)");
  DeviceGuard dg(b->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (b->tiled) {
    cudaError_t e = launch_update_scale_map(nullptr, b->d_tinst, b->d_scale_map, b->n_scale, st);
    if (e == cudaSuccess) e = launch_tile_prep(b->d_tinst, b->d_tprep, b->n_tprep, b->d_ticket, st);
    if (e == cudaSuccess)
      e = launch_tile_sweep(b->d_tinst, b->d_tqueue, b->n_tqueue, b->d_ticket, b->np_max, b->shape, b->grid,
                            b->threads, st);
    return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "batch_sweep");
  }
  cudaError_t e = launch_update_scale_map(b->d_inst, nullptr, b->d_scale_map, b->n_scale, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch_sweep: scale");
  e = launch_prep_batch(b->d_inst, b->d_prep, b->n_prep, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch_sweep: prep");
  // one launch per kernel class, in order on the caller's stream (classes launched on concurrent streams were
  // slower: each class fills the GPU by itself; so was one persistent launch over all classes' bundles)
  for (const auto &c : b->sweeps) {
    e = launch_sweep_fp32_batch(b->d_inst, c.d_map, c.n, c.n_polar, c.depth, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch_sweep: sweep");
  }
  for (const auto &c : b->moments) {
    e = launch_moments_fp32_batch(b->d_inst, c.d_map, c.n, c.n_polar, c.smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch_sweep: moments");
  }
  e = launch_moments_combine_batch(b->d_inst, b->d_combine, b->n_combine, st);
  if (e != cudaSuccess) return cuda_fail(e, "batch_sweep: moments (split cells)");
  return MOLC_OK;
}

void molc_batch_destroy(molc_batch *b) {
  if (b) batch_free(b);
}

molc_status molc_ray_balance(const molc_plan *p, double *max_rel_residual) {
  if (!p || !max_rel_residual) return fail(MOLC_ERR_INVALID_ARG, "ray_balance: NULL argument");
  if (p->host_only) return fail(MOLC_ERR_INVALID_ARG, "ray_balance: the plan was created with MOLC_HOST_ONLY");
  if (!p->d_balance) return fail(MOLC_ERR_INVALID_ARG, "ray_balance: the plan was created without MOLC_BALANCE");
  DeviceGuard dg(p->device);
  unsigned long long bits = 0;
  cudaError_t e = cudaMemcpy(&bits, p->d_balance, sizeof bits, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "ray_balance");
  std::memcpy(max_rel_residual, &bits, sizeof bits);
  return MOLC_OK;
}

molc_status molc_closure(const molc_plan *p, const molc_moments *m, double c, double *fxx, double *fxy,
                         double *fyy, double *f_grey, molc_stream stream) {
  if (!p || !m || !m->E || !m->Nxx || !m->Nxy || !m->Nyy || !fxx || !fxy || !fyy)
    return fail(MOLC_ERR_INVALID_ARG, "closure: NULL argument");
  if (!finite_pos(c)) return fail(MOLC_ERR_INVALID_ARG, "closure: need c > 0");
  if (p->host_only) return fail(MOLC_ERR_INVALID_ARG, "closure: the plan was created with MOLC_HOST_ONLY");
  DeviceGuard dg(p->device);
  cudaError_t e = launch_closure(p->view, *m, c, fxx, fxy, fyy, f_grey, (cudaStream_t)stream);
  return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "closure");
}

molc_status molc_face_moments(const molc_plan *p, molc_precision prec, const void *I, double c, const molc_moments *out,
                              molc_stream stream) {
  if (!p || !I || !out || !out->E || !out->Fx || !out->Fy || !out->Nxx || !out->Nxy || !out->Nyy)
    return fail(MOLC_ERR_INVALID_ARG, "face_moments: NULL argument");
  if (!finite_pos(c)) return fail(MOLC_ERR_INVALID_ARG, "face_moments: need c > 0");
  molc_status s = check_prec(p, prec, "face_moments");
  if (s) return s;
  if (!p->d_facc) return fail(MOLC_ERR_INVALID_ARG, "face_moments: the plan was created without MOLC_FACES");
  DeviceGuard dg(p->device);
  const double *scale = prec == MOLC_FP32 ? header_of(p, prec, const_cast<void *>(I)) : nullptr;
  cudaError_t e = launch_face_moments(p->view, prec, scale, c, *out, (cudaStream_t)stream);
  return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "face_moments");
}

molc_status molc_grey_coefficients(const molc_plan *p, const molc_moments *m, const double *kappa, const double *B,
                                   double *out, molc_stream stream) {
  if (!p || !m || !m->E || !m->Fx || !m->Fy || !kappa || !B || !out)
    return fail(MOLC_ERR_INVALID_ARG, "grey_coefficients: NULL argument");
  if (p->host_only)
    return fail(MOLC_ERR_INVALID_ARG, "grey_coefficients: the plan was created with MOLC_HOST_ONLY");
  DeviceGuard dg(p->device);
  cudaError_t e = launch_grey(p->view, *m, kappa, B, out, (cudaStream_t)stream);
  return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "grey_coefficients");
}

static molc_status intensity_copy(const molc_plan *p, molc_precision prec, void *I, int g_begin, int g_count,
                                  double *canon, const double *B, bool to_canon, molc_stream stream,
                                  const char *who) {
  if (!p || !I || !canon || (!to_canon && !B)) return fail(MOLC_ERR_INVALID_ARG, "%s: NULL argument", who);
  molc_status s = check_prec(p, prec, who);
  if (s) return s;
  if (g_begin < 0 || g_count < 1 || g_begin + g_count > p->G)
    return fail(MOLC_ERR_INVALID_ARG, "%s: group range [%d, %d) outside [0, %d)", who, g_begin, g_begin + g_count,
                p->G);
  DeviceGuard dg(p->device);
  cudaStream_t st = (cudaStream_t)stream;
  double *bref = bref_of(p, prec, I);
  cudaError_t e = cudaSuccess;
  if (!to_canon) {  // the imported groups refer to the given B from now on
    const size_t off = (size_t)g_begin * p->view.ncell;
    e = cudaMemcpyAsync(bref + off, B + off, (size_t)g_count * p->view.ncell * sizeof(double),
                        cudaMemcpyDeviceToDevice, st);
  }
  if (e == cudaSuccess) {
    if (prec == MOLC_FP32 && p->tiled)
      e = launch_tile_intensity_copy(p->view, p->tv, p->d_tpiece, p->d_tpiece_off, (float *)I, bref,
                                     header_of(p, prec, I), g_begin, g_count, canon, to_canon, st);
    else
      e = launch_intensity_copy(p->view, prec, I, bref, header_of(p, prec, I), g_begin, g_count, canon, to_canon,
                                st);
  }
  return e == cudaSuccess ? MOLC_OK : cuda_fail(e, who);
}

molc_status molc_intensity_export(const molc_plan *p, molc_precision prec, const void *I, int g_begin, int g_count,
                                  double *canon, molc_stream stream) {
  return intensity_copy(p, prec, const_cast<void *>(I), g_begin, g_count, canon, nullptr, true, stream,
                        "intensity_export");
}

molc_status molc_intensity_import(molc_plan *p, molc_precision prec, void *I, int g_begin, int g_count,
                                  const double *canon, const double *B, molc_stream stream) {
  return intensity_copy(p, prec, I, g_begin, g_count, const_cast<double *>(canon), B, false, stream,
                        "intensity_import");
}

molc_status molc_tracks_export(const molc_plan *p, int64_t *dir_ray_off, int64_t *ray_seg_off, double *width,
                               int *entry, int *cell, double *len, double *area) {
  if (!p || !dir_ray_off || !ray_seg_off || !width || !entry || !cell || !len || !area)
    return fail(MOLC_ERR_INVALID_ARG, "tracks_export: NULL argument");
  int64_t ri = 0, si = 0;
  dir_ray_off[0] = 0;
  ray_seg_off[0] = 0;
  for (int m = 0; m < p->n_dir; ++m) {
    const int j = p->dir_pair[m], sense = p->dir_sense[m];
    const int64_t k0 = p->pair_track_off[j], k1 = p->pair_track_off[j + 1];
    for (int64_t kk = 0; kk < k1 - k0; ++kk) {
      const HostTrack &h = p->tracks[sense == 0 ? k0 + kk : k1 - 1 - kk];
      width[ri] = h.width;
      entry[ri] = sense == 0 ? h.entry_plus : h.entry_minus;
      for (int q = 0; q < h.nseg; ++q, ++si) {
        const int64_t sg = sense == 0 ? h.seg_off + q : h.seg_off + h.nseg - 1 - q;
        cell[si] = p->seg_cell[sg];
        len[si] = p->seg_len[sg];
        area[si] = p->seg_afrac[sg] * p->V;
      }
      ray_seg_off[++ri] = si;
    }
    dir_ray_off[m + 1] = ri;
  }
  return MOLC_OK;
}

molc_status molc_kernel_timing(molc_plan *p, int enable) {
  if (!p) return fail(MOLC_ERR_INVALID_ARG, "kernel_timing: NULL plan");
  if (p->host_only) return fail(MOLC_ERR_INVALID_ARG, "kernel_timing: the plan was created with MOLC_HOST_ONLY");
  DeviceGuard dg(p->device);
  if (enable && p->ev.empty()) {
    p->ev.resize(4 * (size_t)kMaxTimed);
    for (auto &e : p->ev) {
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) {
        e = nullptr;
        return cuda_fail(r, "kernel_timing");
      }
    }
  }
  p->timing = enable != 0;
  p->n_timed = 0;
  return MOLC_OK;
}

molc_status molc_kernel_time_parts(molc_plan *p, double *parts_ms, int *launches) {
  if (!p || !parts_ms || !launches) return fail(MOLC_ERR_INVALID_ARG, "kernel_time: NULL argument");
  if (p->host_only) return fail(MOLC_ERR_INVALID_ARG, "kernel_time: the plan was created with MOLC_HOST_ONLY");
  DeviceGuard dg(p->device);
  double tot[3] = {0, 0, 0};
  if (p->n_timed > 0) {
    cudaError_t r = cudaEventSynchronize(p->ev[4 * (size_t)p->n_timed - 1]);
    if (r != cudaSuccess) return cuda_fail(r, "kernel_time");
    for (int i = 0; i < p->n_timed; ++i)
      for (int k = 0; k < 3; ++k) {
        float ms = 0;
        r = cudaEventElapsedTime(&ms, p->ev[4 * (size_t)i + k], p->ev[4 * (size_t)i + k + 1]);
        if (r != cudaSuccess) return cuda_fail(r, "kernel_time");
        tot[k] += ms;
      }
  }
  for (int k = 0; k < 3; ++k) parts_ms[k] = tot[k];
  *launches = p->n_timed;
  p->n_timed = 0;
  return MOLC_OK;
}

molc_status molc_kernel_time(molc_plan *p, double *total_ms, int *launches) {
  if (!total_ms) return fail(MOLC_ERR_INVALID_ARG, "kernel_time: NULL argument");
  double parts[3];
  molc_status s = molc_kernel_time_parts(p, parts, launches);
  if (s == MOLC_OK) *total_ms = parts[1];
  return s;
}

molc_status molc_plan_retile(molc_plan *p, const molc_tile_config *cfg) {
  if (!p || !cfg) return fail(MOLC_ERR_INVALID_ARG, "plan_retile: NULL argument");
  if (!p->tiled) return fail(MOLC_ERR_INVALID_ARG, "plan_retile: the plan has no tiled FP32 sweep");
  if (cfg->tile_cells < 0 || cfg->tile_groups < 0 || cfg->block_threads < 0 || cfg->block_threads % 32 ||
      cfg->block_threads > 512)
    return fail(MOLC_ERR_INVALID_ARG, "plan_retile: bad configuration");
  DeviceGuard dg(p->device);
  if (!p->host_only) {
    cudaError_t e = cudaDeviceSynchronize();   // the tables about to be replaced may be in use
    if (e != cudaSuccess) return cuda_fail(e, "plan_retile");
  }
  bool fits = true;
  const molc_status st = build_tiled(p, cfg->tile_cells, cfg->tile_groups, &fits, cfg->block_threads);
  if (st != MOLC_OK && !fits) {   // keep a working layout: rebuild the default one
    const std::string msg = g_last_error;
    if (build_tiled(p, 0, 0) != MOLC_OK) return fail(MOLC_ERR_INTERNAL, "plan_retile: %s", msg.c_str());
    return fail(MOLC_ERR_INVALID_ARG, "%s", msg.c_str());
  }
  return st;
}

molc_status molc_fp64_fma_rate(double *flops_per_s) {
  if (!flops_per_s) return fail(MOLC_ERR_INVALID_ARG, "fp64_fma_rate: NULL argument");
  cudaError_t e = fp64_fma_rate(flops_per_s);
  return e == cudaSuccess ? MOLC_OK : cuda_fail(e, "fp64_fma_rate");
}

molc_status molc_device_status(molc_plan *p, int *code) {
  if (!p || !code) return fail(MOLC_ERR_INVALID_ARG, "device_status: NULL argument");
  if (p->host_only) return fail(MOLC_ERR_INVALID_ARG, "device_status: the plan was created with MOLC_HOST_ONLY");
  DeviceGuard dg(p->device);
  int h = 0;
  cudaError_t e = cudaMemcpy(&h, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "device_status");
  e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "device_status");
  *code = (h & kStatusNonfinite) ? MOLC_ERR_NONFINITE_INPUT
          : (h & kStatusRange)   ? MOLC_ERR_RANGE
          : (h & kStatusTimeout) ? MOLC_ERR_TIMEOUT
                                 : MOLC_OK;
  return MOLC_OK;
}

void molc_destroy(molc_plan *p) {
  if (!p) return;
  if (p->host_only) {
    delete p;
    return;
  }
  DeviceGuard dg(p->device);
  free_device(p);
  delete p;
}

}  // extern "C"
