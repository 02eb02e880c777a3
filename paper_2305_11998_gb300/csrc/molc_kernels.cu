// CUDA kernels of libmolc (sm_103a): the MOLC high-order sweep of Sec. 3 in two precisions, the cell
// assembly of the moments, the Eddington closure and the intensity-state utilities.
//
// Both sweeps walk each characteristic in the deviation form psi = I - B_i (B_i the Planck intensity of
// the current cell).  With S = Q / kappa~ (Eq. 11) and E1(tau) = (1 - e^-tau) / tau, Eqs. (12)-(13) become
//     psi_out  = d + (psi_in - d) e^-tau,     psibar = d + (psi_in - d) E1(tau),
//     d = S - B_i = (I^{n-1} - B_i) / (c dt kappa~),
// (alpha I_s + (1 - alpha) I_{s+1} = S + (I_s - S) E1 exactly), and at a cell crossing
// psi_in(next) = psi_out + (B_prev - B_next).  The stored state is the deviation delta = Ibar - B_ref of each
// segment average from the Planck intensity B_ref its cell had when it was written, so
// d = (delta + B_ref - B) / (c dt kappa~) keeps the precision of the deviation (exactly 0 after
// molc_intensity_init, in any precision).  The cell moments then carry the deviations, and the B_i part
// is added analytically from per-cell geometric moments (it cancels exactly in F: the two senses of a track
// have opposite Omega and equal areas).  This keeps the cancelling sums F and N_xy accurate in optically
// thick cells, where |F| can be ~1e-8 c E.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

#include "molc_internal.h"

namespace molc {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// Not (x >= 0 and finite), decided on the bits (integer pipe; the FP64 pipe is narrow): +0, -0 and the positive
// finite numbers pass.
__device__ __forceinline__ bool bad_input(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  return !(u < 0x7FF0000000000000ull || u == 0x8000000000000000ull);
}

// FP32 -> FP64 by integer operations (the FP64 conversion pipe is narrow on this GPU): exponent rebiased by
// 1023 - 127 and mantissa shifted into place, exact for normal numbers.  Zeros and subnormals (|x| < 2^-126)
// map to a value of the same sign and magnitude below 2^-126; the FP32 sweep works in units where max B is
// ~2^100, so that is below 1e-68 of max B.
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned hi = (u & 0x80000000u) | (((u >> 3) & 0x0fffffffu) + 0x38000000u);
  return __hiloint2double((int)hi, (int)(u << 29));
}

// Exact FP32 -> FP64 for every finite x: the integer route for normal numbers, the conversion instruction for
// zeros and subnormals.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  return (__float_as_uint(x) & 0x7f800000u) ? f32_to_f64(x) : (double)x;
}

// Track holding row r of the intensity layout (rows are (track, sense, step); a track owns 2 nseg rows).
__device__ __forceinline__ int64_t find_track(const TrackDev *tr, int64_t T, int64_t row) {
  int64_t lo = 0, hi = T - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (2 * tr[mid].seg_off <= row)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------------------------
// prep: input checks; FP32 path also tabulates per (chunk, cell, group) {kappa~, 1/(c dt kappa~), B_hi, B_lo}
// with B = B_hi + B_lo split so that B differences between neighbouring cells keep ~48 bits.
// ---------------------------------------------------------------------------------------------------------
constexpr int kPrepCells = 32;   // cells per tile of prep_kernel

// Tiles of kPrepCells cells x the groups of one chunk: [g][cell] inputs are read along cells, the
// [chunk][cell][gc] tables are staged in shared memory and written out contiguously.  A block takes tiles
// tile0, tile0 + tstride, ...; check_bnd: this block also checks the boundary values.
__device__ __forceinline__ void prep_tiles(const PlanView &v, const SweepArgs &a, const Layout &L, int fp32,
                                           int chunk, int tile0, int tstride, bool check_bnd) {
  __shared__ float4 t4[kPrepCells * 32];
  __shared__ float t1[kPrepCells * 32];
  const float inv_cdt_f = (float)a.inv_cdt;
  const double sc = a.scale[0];
  const int g0 = chunk * L.gc;
  const int gcount = min(L.gc, v.G - g0);
  bool bad = false, range = false;
  const int n_tiles = (v.ncell + kPrepCells - 1) / kPrepCells;
  for (int tile = tile0; tile < n_tiles; tile += tstride) {
    const int c0 = tile * kPrepCells;
    const int nc = min(kPrepCells, v.ncell - c0);
#pragma unroll 4
    for (int k = threadIdx.x; k < kPrepCells * gcount; k += blockDim.x) {
      const int gl = k / kPrepCells, c = k - gl * kPrepCells;
      if (c >= nc) continue;
      const int64_t idx = (int64_t)(g0 + gl) * v.ncell + c0 + c;
      const double kap = a.kappa[idx], B = a.B[idx];
      bad |= bad_input(kap) | bad_input(B);
      if (fp32) {
        // FP64 only where a difference or a split needs it (the FP64 pipe is narrow): kappa~ and
        // 1/(c dt kappa~) are rounded to FP32 anyway and are formed in FP32
        const float kt = (float)(kap + a.inv_cdt);
        const float r = __fdiv_rn(inv_cdt_f, kt);
        const double Bs = B * sc;
        // !(Bs < kScaledMax) on the bits: signed order is value order for non-negative doubles and -0
        range |= __double_as_longlong(Bs) >= __double_as_longlong(kScaledMax);
        const float bhi = (float)Bs;
        const float blo = (float)(Bs - f32_to_f64_exact(bhi));
        t4[c * gcount + gl] = make_float4(kt, r, bhi, blo);
        t1[c * gcount + gl] = (float)((a.Bref[idx] - B) * sc) * r;
      }
    }
    if (fp32) {
      __syncthreads();
      // [chunk][cell][gc]: the chunk's stride is gc also in a partial last chunk (as the sweep reads it)
      const int64_t o = (int64_t)g0 * v.ncell + (int64_t)c0 * L.gc;
      for (int k = threadIdx.x; k < nc * gcount; k += blockDim.x) {
        const int c = k / gcount, gl = k - c * gcount;
        a.cdat[o + (int64_t)c * L.gc + gl] = t4[k];
        a.cdB[o + (int64_t)c * L.gc + gl] = t1[k];
      }
      __syncthreads();
    }
  }
  if (check_bnd)
    for (int i = threadIdx.x; i < 4 * v.G; i += blockDim.x) {
      bad |= bad_input(a.bnd[i]);
      range |= fp32 && !(a.bnd[i] * sc < kScaledMax);
    }
  if (bad) atomicOr(v.status, kStatusNonfinite);
  if (range && !bad) atomicOr(v.status, kStatusRange);
}

__global__ void __launch_bounds__(128) prep_kernel(PlanView v, SweepArgs a, Layout L, int fp32) {
  prep_tiles(v, a, L, fp32, blockIdx.y, blockIdx.x, gridDim.x, blockIdx.x == 0 && blockIdx.y == 0);
}

// Batched (FP32): block j prepares tile map[j].z of chunk map[j].y of instance map[j].x.
__global__ void __launch_bounds__(128) prep_batch_kernel(const BatchInst *inst, const int4 *map) {
  const int4 m = map[blockIdx.x];
  const BatchInst &b = inst[m.x];
  prep_tiles(b.v, b.a, b.L, 1, m.y, m.z, 1 << 30, m.w != 0);
}

// ---------------------------------------------------------------------------------------------------------
// FP64 plain sweep: one thread per (track, sense, group, polar cosine), all arithmetic in FP64, one FP64
// atomic per output and update into the [cell][6][G] accumulators.
// Per-ray balance (MOLC_BALANCE): R = I_in - I_out + sum_s tau_s (d_s - psibar_s), which is the integral of the
// transport equation along the characteristic, I_in - I_out + sum_s (Q_s - kappa~_s Ibar_s) l_s / sin zeta, in the
// deviation variables (Q - kappa~ Ibar = kappa~ (d - psibar)).  Segment by segment it reads
// I_in,s - I_out,s + tau_s (d_s - psibar_s) = 0, and the crossings add I_out,s - I_in,s+1 = 0 (the steps of B the
// deviation form takes there); S is the sum of the magnitudes of all these terms in the variables the sweep
// rounds (|I_in,s|, |I_out,s| and their deviations |psi_in,s|, |psi_out,s| from the cell's B, tau_s |B_s + d_s| =
// |Q_s| l_s / sin zeta, tau_s |B_s + psibar_s| = kappa~_s |Ibar_s| l_s / sin zeta, the B steps), so that |R| / S
// is a few units of the working precision's rounding when the arithmetic is consistent.  The largest |R| / S goes
// into *word by an integer atomicMax (non-negative doubles order like their bits).
// Rays whose terms sum to less than kBalanceFloor of max(B, boundary) (word[1], in the units of R and S after the
// factor `units`) carry no radiation at the working precision and are left out.
constexpr double kBalanceFloor = 1e-30;
__device__ __forceinline__ void ray_balance_max(unsigned long long *word, double R, double S, double units) {
  const double floor = kBalanceFloor * __longlong_as_double((long long)word[1]) * units;
  if (!(S > floor) || !(S > 0.0)) return;
  atomicMax(word, (unsigned long long)__double_as_longlong(fabs(R) / S));
}

// ---------------------------------------------------------------------------------------------------------
template <bool BAL>   // BAL: with the per-ray balance check (MOLC_BALANCE)
__global__ void __launch_bounds__(128) sweep_fp64_kernel(PlanView v, SweepArgs a) {
  const int NP = v.n_polar, Q = v.G * NP;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= v.n_tracks * 2 * Q) return;
  const int q = (int)(idx % Q);
  const int64_t rest = idx / Q;
  const int sense = (int)(rest & 1);
  const int64_t t = rest >> 1;
  const int g = q / NP, p = q - g * NP;
  const TrackDev tr = v.tracks[t];
  const PolarDev pd = v.polar[tr.pair * NP + p];
  const PairDev pr = v.pairs[tr.pair];
  const double sg = sense ? -1.0 : 1.0;
  const double Ox = sg * pd.sinz * pr.c, Oy = sg * pd.sinz * pr.s;
  const double inv_cdt = 1.0 / (a.c * a.dt);
  const double *kap = a.kappa + (int64_t)g * v.ncell;
  const double *Bg = a.B + (int64_t)g * v.ncell;
  const double *Bref = a.Bref + (int64_t)g * v.ncell;
  double *I = (double *)a.I + (2 * tr.seg_off + (int64_t)sense * tr.nseg) * Q + q;
  const int nseg = tr.nseg;
  const double Iin = a.bnd[(sense ? tr.entry_minus : tr.entry_plus) * v.G + g];
  double psi = 0.0, Bprev = 0.0;
  double rb = 0.0, sb = 0.0;   // MOLC_BALANCE: sum of tau (d - psibar) and the magnitudes of the terms
  for (int s = 0; s < nseg; ++s) {
    const int64_t sgi = sense ? tr.seg_off + nseg - 1 - s : tr.seg_off + s;
    const int cell = v.seg_cell[sgi];
    const double len = v.seg_len[sgi], af = v.seg_afrac[sgi];
    const double Bc = Bg[cell];
    const double kt = kap[cell] + inv_cdt;
    const double jump = s == 0 ? Iin - Bc : Bprev - Bc;
    psi = s == 0 ? jump : psi + jump;
    if constexpr (BAL) sb += fabs(jump);
    if (v.facc) {   // Eq. (16): omega w times the intensity at the segment's upwind face
      const int2 fc = v.seg_face[sgi];
      double *fa = v.facc + (int64_t)(sense ? fc.y : fc.x) * kOutputs * v.G + g;
      const double wi = pd.w * tr.width * (psi + Bc);
      atomicAdd(fa + 0 * v.G, wi);
      atomicAdd(fa + 1 * v.G, wi * Ox);
      atomicAdd(fa + 2 * v.G, wi * Oy);
      atomicAdd(fa + 3 * v.G, wi * Ox * Ox);
      atomicAdd(fa + 4 * v.G, wi * Ox * Oy);
      atomicAdd(fa + 5 * v.G, wi * Oy * Oy);
    }
    const double d = (I[(int64_t)s * Q] + (Bref[cell] - Bc)) * (inv_cdt / kt);
    const double tau = kt * len * pd.inv_sinz;
    const double one_m_e = -expm1(-tau);
    const double ex = exp(-tau);
    const double E1 = one_m_e / tau;
    const double pin = psi;
    const double x = pin - d;
    const double pb = fma(x, E1, d);
    // thin: psi_in - (psi_in - d)(1 - e^-tau), the change to the accuracy of expm1; thick: d + (psi_in - d) e^-tau,
    // the transmitted part to the accuracy of exp
    psi = tau < 0.5 ? fma(-x, one_m_e, pin) : fma(x, ex, d);
    I[(int64_t)s * Q] = pb;
    if constexpr (BAL) {
      rb += tau * (d - pb);
      sb += fabs(Bc + pin) + fabs(Bc + psi) + fabs(pin) + fabs(psi) + tau * (fabs(Bc + d) + fabs(Bc + pb));
    }
    const double wv = pd.w * af * pb;
    double *acc = a.acc + (int64_t)cell * kOutputs * v.G + g;
    atomicAdd(acc + 0 * v.G, wv);
    atomicAdd(acc + 1 * v.G, wv * Ox);
    atomicAdd(acc + 2 * v.G, wv * Oy);
    atomicAdd(acc + 3 * v.G, wv * Ox * Ox);
    atomicAdd(acc + 4 * v.G, wv * Ox * Oy);
    atomicAdd(acc + 5 * v.G, wv * Oy * Oy);
    Bprev = Bc;
  }
  if (BAL && nseg > 0) {
    const double Iout = psi + Bprev;
    ray_balance_max(v.balance, Iin - Iout + rb, sb, 1.0);
  }
}

// ---------------------------------------------------------------------------------------------------------
// FP32 production sweep.  One thread per (track, sense, group): the thread walks its track in its sense and
// carries all NP polar cosines of the azimuth in registers (the in-plane track is shared by them).  Threads of
// a warp hold consecutive groups of the same track-sense, so the record and cell-table loads are shared and
// coalesced; the previous-step deviations stream in and out in the bundle layout (a block's 128 threads read
// and write 128 * NP contiguous values per step).  The sweep does no reduction: the cell moments are gathered
// afterwards from the swept state (moments_fp32_kernel).
// ---------------------------------------------------------------------------------------------------------

// 2^x (ex2.approx.ftz.f32: the SFU's base-2 exponential).
__device__ __forceinline__ float ex2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// E1 = (1 - e^-tau)/tau, e^-tau and, for tau < 1/2, om = 1 - e^-tau in FP32, from a = tau/2.  With
// h = e^-a = 2^(-a log2 e):
//   tau < 1/2:  E1 = h sinh(a) / a, the even Taylor series in y = a^2 to y^3 (truncation < 5e-11 relative),
//               free of cancellation, and om = tau E1 (= 2 h sinh(a));
//   tau >= 1/2: E1 = (1 - e^-tau) / tau (1 - e^-tau > 0.39, no cancellation).
// e^-tau = h^2.  inv_tau is 1/tau.  The outgoing intensity is taken as psi_in - (psi_in - d) om below tau = 1/2
// and as d + (psi_in - d) e^-tau above: equal in exact arithmetic, but across a thin segment the first keeps the
// change to the relative accuracy of om where the second would carry the rounding of e^-tau on all of psi_in - d,
// and across a thick one the second keeps the small transmitted part to the relative accuracy of e^-tau.
__device__ __forceinline__ void attenuation(float a, float inv_tau, float &E1, float &om, float &ex, bool &thin) {
  constexpr float kMinusLog2e = -1.4426950408889634f;
  const float h = ex2_approx(a * kMinusLog2e);
  ex = h * h;
  const float y = a * a;
  float p = fmaf(y, 1.f / 5040.f, 1.f / 120.f);
  p = fmaf(p, y, 1.f / 6.f);
  p = fmaf(p, y, 1.f);
  const float hp = h * p;
  thin = a < 0.25f;
  E1 = thin ? hp : (1.f - ex) * inv_tau;
  om = (a + a) * hp;
}

// L2 eviction policy (sm_80+ createpolicy) for the streamed state, which each pass touches once: evict-first,
// so that the cell tables and segment records stay in L2.
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// NP consecutive FP32 deviations of one thread: vector accesses where the alignment allows (the row offset is
// a multiple of NP elements and the state is 256-byte aligned), evict-first in L2, no L1 allocation.
template <int NP>
__device__ __forceinline__ void load_dev(const float *p, float (&v)[NP], unsigned long long pol) {
  if constexpr (NP % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 4)
      asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
          : "=f"(v[i]), "=f"(v[i + 1]), "=f"(v[i + 2]), "=f"(v[i + 3])
          : "l"(p + i), "l"(pol));
  } else if constexpr (NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 2)
      asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
          : "=f"(v[i]), "=f"(v[i + 1])
          : "l"(p + i), "l"(pol));
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i)
      asm volatile("ld.global.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v[i]) : "l"(p + i), "l"(pol));
  }
}
// The same through L2 with the default policy (ld.global.cg): the moment gather reads pieces of the state that
// share sectors with pieces other cells read at about the same time.
template <int NP>
__device__ __forceinline__ void load_dev_cg(const float *p, float (&v)[NP]) {
  if constexpr (NP % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 4) {
      const float4 t = __ldcg(reinterpret_cast<const float4 *>(p + i));
      v[i] = t.x;
      v[i + 1] = t.y;
      v[i + 2] = t.z;
      v[i + 3] = t.w;
    }
  } else if constexpr (NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 2) {
      const float2 t = __ldcg(reinterpret_cast<const float2 *>(p + i));
      v[i] = t.x;
      v[i + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) v[i] = __ldcg(p + i);
  }
}
template <int NP>
__device__ __forceinline__ void store_dev(float *p, const float (&v)[NP], unsigned long long pol) {
  if constexpr (NP % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 4)
      asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p + i),
                   "f"(v[i]), "f"(v[i + 1]), "f"(v[i + 2]), "f"(v[i + 3]), "l"(pol)
                   : "memory");
  } else if constexpr (NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 2)
      asm volatile("st.global.L1::no_allocate.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(p + i), "f"(v[i]),
                   "f"(v[i + 1]), "l"(pol)
                   : "memory");
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i)
      asm volatile("st.global.L1::no_allocate.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p + i), "f"(v[i]), "l"(pol)
                   : "memory");
  }
}

// One cp.async of `bytes` (4, 8 or 16) from global to shared memory; with the L2 policy `pol` when HINT.  The
// hinted form is used only where every copy's address is formed in registers with no constant offset folded into
// the instruction (up to 4 polar cosines: one copy per thread or one piece per lane); the other polar counts copy
// several pieces at constant offsets from one address and take the plain form.
template <bool HINT, int BYTES>
__device__ __forceinline__ void cp_async_piece(unsigned dst, const float *src, unsigned long long pol) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async copies 4, 8 or 16 bytes");
  if constexpr (HINT) {
    if constexpr (BYTES == 16)
      asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "l"(pol)
                   : "memory");
    else
      asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;" ::"r"(dst), "l"(src),
                   "n"(BYTES), "l"(pol)
                   : "memory");
  } else {
    if constexpr (BYTES == 16)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    else
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(dst), "l"(src), "n"(BYTES) : "memory");
  }
}

// Asynchronous copies (cp.async, sm_80+) of NP consecutive FP32 deviations from global to shared memory:
// 16-byte pieces where NP * 4 bytes allow, else 8- or 4-byte pieces (the thread's deviations start at a multiple
// of NP * 4 bytes of a 256-byte aligned state).  The streamed state is read with the L2 policy `pol`
// (evict-first), so that it does not push the cell tables and segment records out of L2 (up to 4 polar cosines).
template <int NP>
__device__ __forceinline__ void copy_dev_async(float *dst_smem, const float *src, unsigned long long pol) {
  constexpr bool kHint = NP <= 4;
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  if constexpr (NP % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 4) cp_async_piece<kHint, 16>(d + 4 * i, src + i, pol);
  } else if constexpr (NP % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NP; i += 2) cp_async_piece<kHint, 8>(d + 4 * i, src + i, pol);
  } else {
#pragma unroll
    for (int i = 0; i < NP; ++i) cp_async_piece<kHint, 4>(d + 4 * i, src + i, pol);
  }
}
// Warp-cooperative forms for odd NP: the 32 threads of a warp hold 32 x NP consecutive floats of a bundle step
// slot (128 NP bytes, 16-byte aligned), moved as 8 NP pieces of 16 bytes by the first 8 NP lanes (one
// instruction per lane for NP <= 4) instead of NP scalar accesses per thread.
template <int NP>
__device__ __forceinline__ void copy_warp_chunk_async(float *dst_smem, const float *src, int lane,
                                                      unsigned long long pol) {
  constexpr int kPieces = 8 * NP;
  constexpr bool kHint = NP <= 4;
#pragma unroll
  for (int j = 0; j < (kPieces + 31) / 32; ++j) {
    const int k = lane + 32 * j;
    if (k < kPieces)
      cp_async_piece<kHint, 16>((unsigned)__cvta_generic_to_shared(dst_smem + 4 * k), src + 4 * k, pol);
  }
}
template <int NP>
__device__ __forceinline__ void store_warp_chunk(float *dst, const float *src_smem, int lane,
                                                 unsigned long long pol) {
  constexpr int kPieces = 8 * NP;
#pragma unroll
  for (int j = 0; j < (kPieces + 31) / 32; ++j) {
    const int k = lane + 32 * j;
    if (k < kPieces) {
      const float4 t = *reinterpret_cast<const float4 *>(src_smem + 4 * k);
      asm volatile("st.global.L1::no_allocate.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(dst + 4 * k),
                   "f"(t.x), "f"(t.y), "f"(t.z), "f"(t.w), "l"(pol)
                   : "memory");
    }
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void copy16_async(void *dst_smem, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void copy4_async(void *dst_smem, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ int2 ld_record(const int2 *p) {
  int2 v;
  // volatile: a load the compiler cannot see as one must not be executed speculatively (callers guard the
  // address range with a condition)
  asm volatile("ld.global.nc.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

// Software pipeline of the FP32 sweep, per thread, in rings of D slots (D = staging depth, chosen per plan by
// the autotuner; the step loop is unrolled by D so that every slot index is a constant): at step s the thread
//   - issues asynchronous copies of its previous-step deviations for step s+D-1 and of the cell table entry of
//     step s+D-2 (whose record arrived two steps earlier) into shared memory, as one cp.async group,
//   - waits until the groups holding step s's deviations and table entry have landed,
//   - computes step s and stores its new deviations to global memory,
//   - loads the record of step s+D into a register.
// Group accounting: the prologue commits D-1 groups (deviations of steps 0..D-2, table entries of steps
// 0..D-3) and step s commits one; step s's deviations are in group s and its table entry in group s+1 (group s
// for s <= D-3), so waiting until at most D-2 groups are pending is enough.
// For odd NP the deviations of a step are copied for the whole warp by its first 8 NP lanes (every lane then
// runs the warp's longest track's steps, the copies and commits warp-uniform, a __syncwarp making the landed
// copies visible to the other lanes and ordering the reads of a slot before its refill), and the new deviations
// go back through the slot: each thread writes its own, the warp stores the slot's chunk in 16-byte pieces.  A thread whose track has ended leaves its part of the slot as it was copied,
// so the padding it stores back is unchanged.
// What an FP32 sweep adds to the segment update: nothing, the face reductions of Eq. 16 (MOLC_FACES), or the
// per-ray balance check (MOLC_BALANCE).
enum SweepExtra { kSweepPlain = 0, kSweepFaces = 1, kSweepBalance = 2 };

// Shared memory of one FP32 sweep block: D staged steps of its 128 threads' deviations, cell-table entries and
// B_ref differences.
template <int NP, int D>
struct __align__(16) SweepSmem {
  float dev[D][kSweepBlock * NP];
  float4 tab[D][kSweepBlock];
  float dB[D][kSweepBlock];
};

template <int NP, int D, int EXTRA = kSweepPlain>
__device__ __forceinline__ void sweep_fp32_body(const PlanView &v, const SweepArgs &a, const Layout &L, int bundle,
                                                SweepSmem<NP, D> &sm) {
  static_assert(D >= 3, "the staging depth needs D >= 3");
  constexpr bool FACES = EXTRA == kSweepFaces, BAL = EXTRA == kSweepBalance;
  constexpr bool COOP = NP % 2 != 0;       // warp-cooperative copies and stores of the deviations (odd NP; even NP
  constexpr bool COOP_ST = COOP;           // already copies 8 or 16 bytes per thread, and NP = 2 measured slower)
  constexpr int kSteps = D;
  auto &sdev = sm.dev;
  auto &stab = sm.tab;
  auto &sdB = sm.dB;
  const int tid = threadIdx.x;
  const int64_t item = (int64_t)bundle * kSweepBlock + tid;
  const bool live = item < a.n_items;
  const int2 it = live ? a.items[item] : make_int2(0, 0);
  const TrackDev tr = v.tracks[it.x];
  const int sense = it.y & 1, gi = (it.y >> 1) & 0x7fff, ch = it.y >> 16;
  const int g0 = ch * L.gc;
  const int gcount = min(L.gc, v.G - g0);
  const int g = g0 + gi;
  const int nseg = live ? tr.nseg : 0;
  // warp-uniform trip count
  int nmax = nseg;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(kFull, nmax, o));
  if (nmax == 0) return;

  const unsigned long long pol_stream = policy_evict_first();
  // floats between consecutive steps of one item (bundle layout); a run-time value, so that the copies below
  // address through registers
  const int64_t stride = (int64_t)kSweepBlock * v.n_polar;
  float *I = (float *)a.I + (v.boff[bundle] * kSweepBlock + tid) * NP;
  const int lane = tid & 31, wofs = (tid & ~31) * NP;   // this warp's chunk in a slot (COOP)
  float *Iw = (float *)a.I + v.boff[bundle] * kSweepBlock * NP + wofs;
  const int nlim = COOP ? nmax : nseg;   // steps this thread copies and commits for
  const int2 *rec = v.seg32 + (sense ? tr.seg_off + nseg - 1 : tr.seg_off);
  const int rstep = sense ? -1 : 1;
  const int64_t cbase = (int64_t)ch * v.ncell * L.gc + gi;
  const float4 *cd = a.cdat + cbase;
  const float *cdB = a.cdB + cbase;

  float half_inv_sinz[NP], sinz[NP], wf[FACES ? NP : 1];   // 1/(2 sin zeta): tau/2 = kappa~ l half_inv_sinz
#pragma unroll
  for (int p = 0; p < NP; ++p) {
    const PolarDev pd = v.polar[tr.pair * NP + p];
    half_inv_sinz[p] = 0.5f * pd.inv_sinzf;
    sinz[p] = pd.sinzf;
    if constexpr (FACES) wf[p] = pd.wf;
  }
  // face moments (Eq. 16): faces of this sense's segments, in traversal order like the records
  const int2 *sface = FACES ? v.seg_face + (sense ? tr.seg_off + nseg - 1 : tr.seg_off) : nullptr;
  const float fx = FACES ? (float)((sense ? -1.0 : 1.0) * v.pairs[tr.pair].c) : 0.f;
  const float fy = FACES ? (float)((sense ? -1.0 : 1.0) * v.pairs[tr.pair].s) : 0.f;
  const float width = FACES ? (float)tr.width : 0.f;
  // entering intensity (scaled), split like B so that I_in - B keeps the precision of the difference
  const double bin = live ? a.bnd[(sense ? tr.entry_minus : tr.entry_plus) * v.G + g] * a.scale[0] : 0.0;
  const float in_hi = (float)bin, in_lo = (float)(bin - (double)in_hi);
  const float rescale = (float)a.scale[3];   // power of two: the stored deviations to this step's scale

  // prologue: records of steps 0..D-1; groups 0..D-2 = {deviations k, table k (k <= D-3)}
  int2 recs[kSteps];
#pragma unroll
  for (int k = 0; k < kSteps; ++k) recs[k] = k < nseg ? ld_record(rec + k * rstep) : make_int2(0, 0);
#pragma unroll
  for (int k = 0; k < kSteps - 1; ++k) {
    if constexpr (COOP) {
      if (k < nmax) copy_warp_chunk_async<NP>(&sdev[k][wofs], Iw + k * stride, lane, pol_stream);
    }
    if (k < nseg) {
      if constexpr (!COOP) copy_dev_async<NP>(&sdev[k][tid * NP], I + k * stride, pol_stream);
      if (k < kSteps - 2) {
        copy16_async(&stab[k][tid], cd + (int64_t)recs[k].x * L.gc);
        copy4_async(&sdB[k][tid], cdB + (int64_t)recs[k].x * L.gc);
      }
    }
    cp_async_commit();
  }
  float psi[NP];
#pragma unroll
  for (int p = 0; p < NP; ++p) psi[p] = 0.f;
  float bhi_prev = in_hi, blo_prev = in_lo;   // the boundary acts as the "previous cell" of step 0
  // MOLC_BALANCE, in FP64 from this sweep's FP32 values: per polar cosine the sum of tau (d - psibar) and of the
  // magnitudes of the terms; the crossing steps are common to the polar cosines; B of the last cell
  double rb[BAL ? NP : 1], sb[BAL ? NP : 1], jsum = 0.0, blast = 0.0;
  if constexpr (BAL) {
#pragma unroll
    for (int p = 0; p < NP; ++p) rb[p] = sb[p] = 0.0;
  }
  for (int s0 = 0; s0 < nmax; s0 += kSteps) {
#pragma unroll
    for (int u = 0; u < kSteps; ++u) {
      const int s = s0 + u;
      if (s < nlim) {
        // group s+D-1: deviations of step s+D-1, table entry of step s+D-2
        if constexpr (COOP) {
          __syncwarp();   // every lane is done with the slot refilled here (read at step s-1)
          if (s + kSteps - 1 < nmax)
            copy_warp_chunk_async<NP>(&sdev[(u + kSteps - 1) % kSteps][wofs], Iw + (kSteps - 1) * stride, lane,
                                      pol_stream);
        } else {
          if (s + kSteps - 1 < nseg)
            copy_dev_async<NP>(&sdev[(u + kSteps - 1) % kSteps][tid * NP], I + (kSteps - 1) * stride, pol_stream);
        }
        if (s + kSteps - 2 < nseg) {
          const int c2 = recs[(u + kSteps - 2) % kSteps].x;
          copy16_async(&stab[(u + kSteps - 2) % kSteps][tid], cd + (int64_t)c2 * L.gc);
          copy4_async(&sdB[(u + kSteps - 2) % kSteps][tid], cdB + (int64_t)c2 * L.gc);
        }
        cp_async_commit();
        cp_async_wait<kSteps - 2>();   // deviations and table entry of step s have landed
        if constexpr (COOP) __syncwarp();   // ... including the pieces other lanes copied
        if (s < nseg) {
          float dv[NP];
          if constexpr (NP % 4 == 0) {
#pragma unroll
            for (int p = 0; p < NP; p += 4) {
              const float4 t4 = *reinterpret_cast<const float4 *>(&sdev[u][tid * NP + p]);
              dv[p] = t4.x;
              dv[p + 1] = t4.y;
              dv[p + 2] = t4.z;
              dv[p + 3] = t4.w;
            }
          } else {
#pragma unroll
            for (int p = 0; p < NP; ++p) dv[p] = sdev[u][tid * NP + p];
          }
          const float4 q = stab[u][tid];
          const float qy = q.y * rescale;   // rescale (a power of two) brings the stored deviations to this scale
          const float dB = sdB[u][tid];
          // step s
          const float len = __int_as_float(recs[u].y);
          const float jump = (bhi_prev - q.z) + (blo_prev - q.w);
          const float kl = q.x * len;
          const float rkl = rcp_approx(kl);
#pragma unroll
          for (int p = 0; p < NP; ++p) psi[p] += jump;
          double bcell = 0.0;
          if constexpr (BAL) {
            jsum += fabs(f32_to_f64_exact(jump));
            bcell = f32_to_f64_exact(q.z) + f32_to_f64_exact(q.w);
            blast = bcell;
          }
          if constexpr (FACES) {
            // the intensity entering the segment, in scaled units: psi (relative to this cell) + B of this cell
            const float Bc = q.z + q.w;
            float S0 = 0.f, S1 = 0.f, S2 = 0.f;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
              const float t0 = wf[p] * (psi[p] + Bc);
              S0 += t0;
              const float t1 = t0 * sinz[p];
              S1 += t1;
              S2 = fmaf(t1, sinz[p], S2);
            }
            const int2 fc = __ldg(sface + s * rstep);
            double *fa = v.facc + ((int64_t)ch * v.n_faces + (sense ? fc.y : fc.x)) * kOutputs * L.gc + gi;
            S0 *= width;
            S1 *= width;
            S2 *= width;
            atomicAdd(fa, f32_to_f64(S0));
            atomicAdd(fa + L.gc, f32_to_f64(fx * S1));
            atomicAdd(fa + 2 * L.gc, f32_to_f64(fy * S1));
            atomicAdd(fa + 3 * L.gc, f32_to_f64(fx * fx * S2));
            atomicAdd(fa + 4 * L.gc, f32_to_f64(fx * fy * S2));
            atomicAdd(fa + 5 * L.gc, f32_to_f64(fy * fy * S2));
          }
#pragma unroll
          for (int p = 0; p < NP; ++p) {
            float E1, om, ex;
            bool thin;
            const float ahalf = kl * half_inv_sinz[p];   // tau / 2
            attenuation(ahalf, sinz[p] * rkl, E1, om, ex, thin);
            const float d = fmaf(dv[p], qy, dB);
            const float pin = psi[p];
            const float x = pin - d;
            dv[p] = fmaf(x, E1, d);
            psi[p] = thin ? fmaf(-x, om, pin) : fmaf(x, ex, d);
            if constexpr (BAL) {
              const double tau = 2.0 * f32_to_f64_exact(ahalf), dd = f32_to_f64_exact(d),
                           pb = f32_to_f64_exact(dv[p]);
              rb[p] += tau * (dd - pb);
              const double pi = f32_to_f64_exact(pin), po = f32_to_f64_exact(psi[p]);
              sb[p] += fabs(bcell + pi) + fabs(bcell + po) + fabs(pi) + fabs(po) +
                       tau * (fabs(bcell + dd) + fabs(bcell + pb));
            }
        }
        if constexpr (COOP_ST) {
#pragma unroll
          for (int p = 0; p < NP; ++p) sdev[u][tid * NP + p] = dv[p];
        } else {
          store_dev<NP>(I, dv, pol_stream);
        }
        bhi_prev = q.z;
        blo_prev = q.w;
        I += stride;
        if (s + kSteps < nseg) recs[u] = ld_record(rec + (s + kSteps) * rstep);
        }
        if constexpr (COOP_ST) {
          __syncwarp();
          store_warp_chunk<NP>(Iw, &sdev[u][wofs], lane, pol_stream);
        }
        Iw += stride;
      }
    }
  }
  cp_async_wait<0>();
  if constexpr (BAL) {
    if (nseg > 0) {
      const double Iin = f32_to_f64_exact(in_hi) + f32_to_f64_exact(in_lo);
      double R = 0.0, S = 0.0, worst = -1.0;
#pragma unroll
      for (int p = 0; p < NP; ++p) {   // the polar cosine with the largest relative residual
        const double Iout = f32_to_f64_exact(psi[p]) + blast;
        const double r = Iin - Iout + rb[p], sm = sb[p] + jsum;
        const double rel = sm > 0.0 ? fabs(r) / sm : 0.0;
        if (rel > worst) {
          worst = rel;
          R = r;
          S = sm;
        }
      }
      ray_balance_max(v.balance, R, S, a.scale[0]);   // R, S in the state's scaled units
    }
  }
}

template <int NP, int D, int EXTRA = kSweepPlain>
__global__ void __launch_bounds__(kSweepBlock) sweep_fp32_kernel(PlanView v, SweepArgs a, Layout L) {
  __shared__ SweepSmem<NP, D> sm;
  sweep_fp32_body<NP, D, EXTRA>(v, a, L, v.block_order[blockIdx.x], sm);
}

// Batched: block j sweeps bundle map[j].y of instance map[j].x (blocks of all instances, longest first).
template <int NP, int D>
__global__ void __launch_bounds__(kSweepBlock) sweep_fp32_batch_kernel(const BatchInst *inst, const int2 *map) {
  __shared__ SweepSmem<NP, D> sm;
  const int2 m = map[blockIdx.x];
  const BatchInst &b = inst[m.x];
  sweep_fp32_body<NP, D>(b.v, b.a, b.L, m.y, sm);
}

// FP32 path, cell moments: one thread per (chunk, cell, group), consecutive groups of a cell in consecutive
// lanes.  The thread sums, over the (track, sense) segments crossing its cell, the swept deviations of its group
// (NP contiguous values per segment; the lanes of a cell read one contiguous block) weighted by
// omega (A/V) (1, Omega, Omega Omega).  A cell's entries come grouped by azimuth pair: within a pair the
// polar folds S0 = sum_p w_p dev_p, S1 = sum_p w_p sin(zeta_p) dev_p (signed by the sense),
// S2 = sum_p w_p sin^2(zeta_p) dev_p are summed in FP32 (runs of at most kPairRun segments); across runs the six sums
// are carried as unevaluated pairs of FP32 words (hi + lo, TwoSum: a 48-bit significand), then assembled in FP64:
//   E = (B geo0 + D)/c, F = D_F, N_ab = B geo_ab + D_ab, and B_ref := B.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

// Entries are taken kGatherBatch at a time so that their state loads are in flight together (each cell's entry
// list is padded to a multiple of kGatherPad with zero-area entries of its last pair, so the batch must equal it).
constexpr int kGatherBatch = kGatherPad;
// An FP32 partial sum takes at most kPairRun entries (one azimuth pair) before it is added to the two-word sums:
// a cell crossed by many characteristics of one pair (fine ray spacing) keeps the FP32 error of a few terms.
constexpr int kPairRun = 8;

// Eddington factors of one (cell, group) from the moments just assembled (Eq. 7 with the cell averages of
// Eq. 15): f = N / (c E), 0 where E = 0.  The same operations as closure_cells, so molc_sweep_closure and
// molc_sweep + molc_closure give the same bits.
__device__ __forceinline__ void eddington_factors(const SweepArgs &a, int64_t idx, double E, double nxx, double nxy,
                                                  double nyy) {
  const double inv = E > 0 ? 1.0 / (a.c * E) : 0.0;
  a.fxx[idx] = nxx * inv;
  a.fxy[idx] = nxy * inv;
  a.fyy[idx] = nyy * inv;
}

// Assembly of one (cell, group) from its six deviation sums D (state units; is = 1/scale):
//   E = (B geo0 + D0 is)/c, F = D_F is, N_ab = B geo_ab + D_ab is, and B_ref := B.
__device__ __forceinline__ void assemble_cell(const PlanView &v, const SweepArgs &a, int cell, int g,
                                              const double (&D)[kOutputs]) {
  const double is = a.scale[1];   // the deviations are in the state's scaled units (exact power of two)
  const int64_t idx = (int64_t)g * v.ncell + cell;
  const double B = a.B[idx];
  const double E = (B * v.geo[cell] + D[0] * is) * a.inv_c;
  const double nxx = B * v.geo[v.ncell + cell] + D[3] * is;
  const double nxy = B * v.geo[2 * (int64_t)v.ncell + cell] + D[4] * is;
  const double nyy = B * v.geo[3 * (int64_t)v.ncell + cell] + D[5] * is;
  a.out.E[idx] = E;
  a.out.Fx[idx] = D[1] * is;
  a.out.Fy[idx] = D[2] * is;
  a.out.Nxx[idx] = nxx;
  a.out.Nxy[idx] = nxy;
  a.out.Nyy[idx] = nyy;
  a.Bref[idx] = B;   // the new deviations refer to this step's B
  if (a.fxx) eddington_factors(a, idx, E, nxx, nxy, nyy);
}

// One block: threads t0 .. t0+127 of chunk ch ((unit, group) pairs, groups fastest; a unit is one part of a
// cell's entry list).  A cell in one part is assembled here; the parts of a split cell go to the scratch
// partials, summed in order by moments_combine.
template <int NP>
__device__ __forceinline__ void moments_fp32_body(const PlanView &v, const SweepArgs &a, const Layout &L, int ch,
                                                  int64_t t0) {
  extern __shared__ float coef[];   // [pair][3][NP] {w, w sin, w sin^2}, then [pair][2] {cos, sin}
  float *csn = coef + 3 * NP * v.n_pairs;
  for (int i = threadIdx.x; i < v.n_pairs * NP; i += blockDim.x) {
    const int pr = i / NP, p = i - pr * NP;
    const float w = v.polar[i].wf, sz = v.polar[i].sinzf;
    coef[(pr * 3 + 0) * NP + p] = w;
    coef[(pr * 3 + 1) * NP + p] = w * sz;
    coef[(pr * 3 + 2) * NP + p] = (w * sz) * sz;
  }
  for (int i = threadIdx.x; i < v.n_pairs; i += blockDim.x) {
    csn[2 * i] = v.pairs[i].cf;
    csn[2 * i + 1] = v.pairs[i].sf;
  }
  __syncthreads();
  const int g0 = ch * L.gc;
  const int gcount = min(L.gc, v.G - g0);
  const int64_t t = t0 + threadIdx.x;
  if (ch == 0 && t == 0) const_cast<double *>(a.scale)[3] = 1.0;   // the state is in this step's scale now
  if (t >= v.n_munits * gcount) return;
  const int64_t unit = t / gcount;
  const int gi = (int)(t - unit * gcount);
  const int2 um = v.n_mmulti ? v.munit[unit] : make_int2((int)unit, 0);   // no split cell: unit = cell
  const int cell = um.x;
  const int g = g0 + gi;
  const int4 *gent = v.gent + ch * v.gent_chunk;
  const float *I = (const float *)a.I;
  float hi[kOutputs], lo[kOutputs];
#pragma unroll
  for (int k = 0; k < kOutputs; ++k) hi[k] = lo[k] = 0.f;
  const int64_t ce0 = v.cell_off[cell], ce1 = v.cell_off[cell + 1];
  const int64_t e0 = ce0 + (int64_t)um.y * kPartEntries;
  const int ne = (int)min(ce1 - e0, (int64_t)kPartEntries);   // entries of this part (a multiple of kGatherBatch)
  const bool split = ce1 - ce0 > kPartEntries;
  const int4 *ep = gent + e0;
  int cur = ne > 0 ? (__ldg(&ep->w) >> 1) : 0;
  int run = 0;   // entries in the current FP32 partial sums
  float P0 = 0.f, P1 = 0.f, P2 = 0.f;
  auto flush = [&]() {
    const float cf = csn[2 * cur], sf = csn[2 * cur + 1];
    two_sum_add(hi[0], lo[0], P0);
    two_sum_add(hi[1], lo[1], cf * P1);
    two_sum_add(hi[2], lo[2], sf * P1);
    two_sum_add(hi[3], lo[3], (cf * cf) * P2);
    two_sum_add(hi[4], lo[4], (cf * sf) * P2);
    two_sum_add(hi[5], lo[5], (sf * sf) * P2);
  };
  // up to 3 polar cosines the entries of the next batch are loaded while this batch's state loads are in flight;
  // at 4 that costs the occupancy it buys (measured with the factors formed here), so each batch loads its own
  constexpr bool kPrefetch = NP <= 3;
  int4 en[kGatherBatch];
  if (kPrefetch && ne > 0) {
#pragma unroll
    for (int b = 0; b < kGatherBatch; ++b) en[b] = __ldg(ep + b);
  }
  for (int e = 0; e < ne; e += kGatherBatch) {
    if constexpr (!kPrefetch) {
      // the line holding the entries two batches ahead is fetched into L2 now (no registers held): the entry
      // loads below then hit in cache instead of waiting on DRAM before the state loads that depend on them
      if (e + 2 * kGatherBatch < ne)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(ep + e + 2 * kGatherBatch));
#pragma unroll
      for (int b = 0; b < kGatherBatch; ++b) en[b] = __ldg(ep + e + b);
    }
    float dv[kGatherBatch][NP];
#pragma unroll
    for (int b = 0; b < kGatherBatch; ++b) load_dev_cg<NP>(I + gather_slot(en[b].x, en[b].y, gi) * NP, dv[b]);
    int2 zw[kGatherBatch];
#pragma unroll
    for (int b = 0; b < kGatherBatch; ++b) zw[b] = make_int2(en[b].z, en[b].w);
    if (kPrefetch && e + kGatherBatch < ne) {
#pragma unroll
      for (int b = 0; b < kGatherBatch; ++b) en[b] = __ldg(ep + e + kGatherBatch + b);
    }
#pragma unroll
    for (int b = 0; b < kGatherBatch; ++b) {
      const int pr = zw[b].y >> 1;
      if (pr != cur || run == kPairRun) {
        flush();
        cur = pr;
        run = 0;
        P0 = P1 = P2 = 0.f;
      }
      ++run;
      const float *c0 = coef + pr * 3 * NP;
      float S0 = 0.f, S1 = 0.f, S2 = 0.f;
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        S0 = fmaf(c0[p], dv[b][p], S0);
        S1 = fmaf(c0[NP + p], dv[b][p], S1);
        S2 = fmaf(c0[2 * NP + p], dv[b][p], S2);
      }
      const float af = __int_as_float(zw[b].x);
      P0 = fmaf(af, S0, P0);
      P1 = fmaf((zw[b].y & 1) ? -af : af, S1, P1);
      P2 = fmaf(af, S2, P2);
    }
  }
  if (ne > 0) flush();
  // FP64 work here is per (cell, group), not per update: conversions by integer operations, one add per sum
  double D[kOutputs];
#pragma unroll
  for (int k = 0; k < kOutputs; ++k) D[k] = f32_to_f64(hi[k]) + f32_to_f64(lo[k]);
  if (!split) {
    assemble_cell(v, a, cell, g, D);
  } else {
    double *ps = v.mscratch + (((int64_t)ch * v.n_munits + unit) * kOutputs) * L.gc + gi;
#pragma unroll
    for (int k = 0; k < kOutputs; ++k) ps[k * L.gc] = D[k];
  }
}

// Split cells: the parts' partial sums added in part order (FP64), then assembled.  One thread per (split
// cell, group) of chunk ch, threads t0 ...
__device__ __forceinline__ void moments_combine_body(const PlanView &v, const SweepArgs &a, const Layout &L, int ch,
                                                     int64_t t0) {
  const int g0 = ch * L.gc;
  const int gcount = min(L.gc, v.G - g0);
  const int64_t t = t0 + threadIdx.x;
  if (t >= (int64_t)v.n_mmulti * gcount) return;
  const int m = (int)(t / gcount), gi = (int)(t - (int64_t)m * gcount);
  const int4 mc = v.mmulti[m];
  double D[kOutputs] = {0, 0, 0, 0, 0, 0};
  for (int k = 0; k < mc.z; ++k) {
    const double *ps = v.mscratch + (((int64_t)ch * v.n_munits + mc.y + k) * kOutputs) * L.gc + gi;
#pragma unroll
    for (int o = 0; o < kOutputs; ++o) D[o] += ps[o * L.gc];
  }
  assemble_cell(v, a, mc.x, g0 + gi, D);
}

__global__ void __launch_bounds__(128) moments_combine_kernel(PlanView v, SweepArgs a, Layout L) {
  moments_combine_body(v, a, L, blockIdx.y, (int64_t)blockIdx.x * blockDim.x);
}

__global__ void __launch_bounds__(128) moments_combine_batch_kernel(const BatchInst *inst, const int4 *map) {
  const int4 m = map[blockIdx.x];
  const BatchInst &b = inst[m.x];
  moments_combine_body(b.v, b.a, b.L, m.y, (int64_t)m.z * blockDim.x);
}

// blocks per SM: 7 up to 3 polar cosines (72 registers: the next batch's entries are loaded while the current
// batch's state loads are in flight), 8 at 4, 5 beyond
template <int NP>
__global__ void __launch_bounds__(128, NP <= 3 ? 7 : NP == 4 ? 8 : 5)
    moments_fp32_kernel(PlanView v, SweepArgs a, Layout L) {
  moments_fp32_body<NP>(v, a, L, blockIdx.y, (int64_t)blockIdx.x * blockDim.x);
}

// Batched: block j handles threads 128 map[j].z .. of chunk map[j].y of instance map[j].x.
template <int NP>
__global__ void __launch_bounds__(128, NP <= 3 ? 7 : NP == 4 ? 8 : 5)
    moments_fp32_batch_kernel(const BatchInst *inst, const int4 *map) {
  const int4 m = map[blockIdx.x];
  const BatchInst &b = inst[m.x];
  moments_fp32_body<NP>(b.v, b.a, b.L, m.y, (int64_t)m.z * blockDim.x);
}

// ---------------------------------------------------------------------------------------------------------
// finalize: cell assembly.  acc holds sum_m omega_m sum_{C(i,m)} (A/V) psibar (times Omega components);
// the B_i part uses the geometric moments geo = sum_m omega_m sum_{C(i,m)} A/V (times Omega components).
//   E = (B geo0 + D)/c, F = acc, N_ab = B geo_ab + acc_ab.  (The B part of F is zero by symmetry.)
// ---------------------------------------------------------------------------------------------------------
__global__ void finalize_kernel(PlanView v, SweepArgs a, Layout L) {
  const double inv_c = 1.0 / a.c;
  const double is = a.scale[1];   // accumulators are in the state's scaled units (exact power of two)
  // one thread per cell, looping over groups: the cell's accumulator block is read contiguously (through L1)
  // and every output [g][cell] is written coalesced across threads
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < v.ncell; cell += gridDim.x * blockDim.x) {
    const double g0v = v.geo[cell], gxx = v.geo[v.ncell + cell], gxy = v.geo[2 * (int64_t)v.ncell + cell],
                 gyy = v.geo[3 * (int64_t)v.ncell + cell];
    for (int g = 0; g < v.G; ++g) {
      const int64_t idx = (int64_t)g * v.ncell + cell;
      const int g0 = g / L.gc * L.gc, gc = L.gc;   // [chunk][cell][6][gc], as the sweeps accumulate
      const double *ac = a.acc + (int64_t)kOutputs * g0 * v.ncell + (int64_t)cell * kOutputs * gc + (g - g0);
      const double B = a.B[idx];
      const double E = (B * g0v + __ldg(ac + 0 * gc) * is) * inv_c;
      const double nxx = B * gxx + __ldg(ac + 3 * gc) * is;
      const double nxy = B * gxy + __ldg(ac + 4 * gc) * is;
      const double nyy = B * gyy + __ldg(ac + 5 * gc) * is;
      a.out.E[idx] = E;
      a.out.Fx[idx] = __ldg(ac + 1 * gc) * is;
      a.out.Fy[idx] = __ldg(ac + 2 * gc) * is;
      a.out.Nxx[idx] = nxx;
      a.out.Nxy[idx] = nxy;
      a.out.Nyy[idx] = nyy;
      a.Bref[idx] = B;   // the new deviations refer to this step's B
      if (a.fxx) eddington_factors(a, idx, E, nxx, nxy, nyy);
    }
  }
}

// f = N / (c E) per group (Eq. 7 with the cell averages of Eq. 15); <f>_E = sum_g N_g / (c sum_g E_g).
__device__ __forceinline__ void closure_cells(const PlanView &v, const molc_moments &m, double c, double *fxx,
                                              double *fxy, double *fyy, double *fgrey, int cell0, int cstride) {
  for (int cell = cell0; cell < v.ncell; cell += cstride) {
    double se = 0, sxx = 0, sxy = 0, syy = 0;
    for (int g = 0; g < v.G; ++g) {
      const int64_t i = (int64_t)g * v.ncell + cell;
      const double E = m.E[i], nxx = m.Nxx[i], nxy = m.Nxy[i], nyy = m.Nyy[i];
      const double inv = E > 0 ? 1.0 / (c * E) : 0.0;
      fxx[i] = nxx * inv;
      fxy[i] = nxy * inv;
      fyy[i] = nyy * inv;
      se += E;
      sxx += nxx;
      sxy += nxy;
      syy += nyy;
    }
    if (fgrey) {
      const double inv = se > 0 ? 1.0 / (c * se) : 0.0;
      fgrey[cell] = sxx * inv;
      fgrey[v.ncell + cell] = sxy * inv;
      fgrey[2 * (int64_t)v.ncell + cell] = syy * inv;
    }
  }
}

// Grey-problem coefficients (Eqs. 8-9), one thread per cell, all in FP64: <kappa>_E, <kappa>_B, the flux-weighted
// K_R = diag(<kappa>_|Fx|, <kappa>_|Fy|) and eta = sum_g (kappa_g - K_R) F_g / sum_g E_g.
__global__ void grey_kernel(PlanView v, molc_moments m, const double *kappa, const double *B, double *out) {
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < v.ncell; cell += gridDim.x * blockDim.x) {
    double se = 0, ske = 0, sb = 0, skb = 0, sfx = 0, skfx = 0, sfy = 0, skfy = 0;
    for (int g = 0; g < v.G; ++g) {
      const int64_t i = (int64_t)g * v.ncell + cell;
      const double k = kappa[i], E = m.E[i], b = B[i], fx = fabs(m.Fx[i]), fy = fabs(m.Fy[i]);
      se += E;
      ske += k * E;
      sb += b;
      skb += k * b;
      sfx += fx;
      skfx += k * fx;
      sfy += fy;
      skfy += k * fy;
    }
    const double kE = se > 0 ? ske / se : 0.0, kB = sb > 0 ? skb / sb : 0.0;
    const double kx = sfx > 0 ? skfx / sfx : 0.0, ky = sfy > 0 ? skfy / sfy : 0.0;
    double ex = 0, ey = 0;
    for (int g = 0; g < v.G; ++g) {
      const int64_t i = (int64_t)g * v.ncell + cell;
      ex += (kappa[i] - kx) * m.Fx[i];
      ey += (kappa[i] - ky) * m.Fy[i];
    }
    const int64_t n = v.ncell;
    out[cell] = kE;
    out[n + cell] = kB;
    out[2 * n + cell] = kx;
    out[3 * n + cell] = ky;
    out[4 * n + cell] = se > 0 ? ex / se : 0.0;
    out[5 * n + cell] = se > 0 ? ey / se : 0.0;
  }
}

__global__ void closure_kernel(PlanView v, molc_moments m, double c, double *fxx, double *fxy, double *fyy,
                               double *fgrey) {
  closure_cells(v, m, c, fxx, fxy, fyy, fgrey, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}


// Canonical segment averages <-> deviation state: one thread per row (track, sense, step) of the layout,
// looping over polar cosines and the selected groups.  Ibar = B_ref(cell) + delta.
template <class T>
__global__ void intensity_copy_kernel(PlanView v, Layout L, T *I, const double *Bref, const double *scale,
                                      int g_begin, int g_count, double *canon, int to_canon, int bundle) {
  const int NP = v.n_polar;
  const double sc = scale[0], is = scale[1];
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < L.rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = find_track(v.tracks, v.n_tracks, row);
    const TrackDev tr = v.tracks[t];
    const int64_t local = row - 2 * tr.seg_off;
    const int sense = local >= tr.nseg;
    const int s = (int)(local - (int64_t)sense * tr.nseg);
    const int cell = v.seg_cell[sense ? tr.seg_off + tr.nseg - 1 - s : tr.seg_off + s];
    for (int p = 0; p < NP; ++p) {
      const PolarDev pd = v.polar[tr.pair * NP + p];
      const int dir = sense ? pd.dir_minus : pd.dir_plus;
      const int64_t cs = v.dir_seg_off[dir] + (sense ? tr.canon_minus : tr.canon_plus) + s;
      for (int g = g_begin; g < g_begin + g_count; ++g) {
        const int ch = g / L.gc, gl = g - ch * L.gc, gcount = min(L.gc, v.G - ch * L.gc);
        T *el = bundle ? I + bundle_index(v.boff,
                                          (int64_t)ch * 2 * v.n_tracks * L.gc +
                                              (int64_t)tr.pos[sense] * gcount + gl,
                                          s, NP) + p
                       : I + L.rows * (int64_t)NP * (ch * L.gc) + row * (int64_t)(gcount * NP) + gl * NP + p;
        const double br = Bref[(int64_t)g * v.ncell + cell];
        double *cv = canon + cs * g_count + (g - g_begin);
        if (to_canon)
          *cv = br + (double)*el * is;
        else
          *el = (T)((*cv - br) * sc);
      }
    }
  }
}

// max over finite non-negative B of the IEEE bits (ordered like the values for x >= 0)
__global__ void max_bits_kernel(const double *B, int64_t n, unsigned long long *mx) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double b = B[i];
    if (b >= 0.0 && isfinite(b)) m = max(m, (unsigned long long)__double_as_longlong(b));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

// scale = 2^(100 - e) with max B = f 2^e, f in [1/2, 1) (2^100 if max B = 0); 1 for FP64 states.
__global__ void set_scale_kernel(const unsigned long long *mx, double *header, int fp32) {
  double s = 1.0;
  if (fp32) {
    const double m = __longlong_as_double((long long)*mx);
    int e = 0;
    if (m > 0.0) frexp(m, &e);
    s = ldexp(1.0, kScaleTargetExp - e);
  }
  header[0] = s;
  header[1] = 1.0 / s;
  header[3] = 1.0;
  reinterpret_cast<unsigned long long *>(header)[2] = 0;   // the sweep-time reduction starts from zero
  reinterpret_cast<unsigned int *>(header + 4)[0] = 0;     // and with no block counted
}

// Sweep-time scale of an FP32 state: the scale follows max(B, boundary) so that the largest scaled intensity
// stays near 2^100.  It is kept while that maximum, scaled, has its exponent in [93, 108]; otherwise it is reset
// to 2^(100 - e), max = f 2^e.  header[3] = new scale / old scale (a power of two) is the factor by which this
// step's sweep multiplies the stored deviations as it reads them; the moment kernel sets it back to 1.
__device__ __forceinline__ void update_scale(unsigned long long mbits, double *header) {
  const double m = __longlong_as_double((long long)mbits);
  const double s = header[0];
  double f = 1.0;
  if (m > 0.0 && isfinite(m)) {
    int em = 0, es = 0;
    frexp(m, &em);
    frexp(s, &es);
    const int e = em + es - 1;   // exponent of m * s (s is a power of two)
    if (e < 93 || e > 108) {
      const double sn = ldexp(1.0, kScaleTargetExp - em);
      f = sn / s;
      header[0] = sn;
      header[1] = 1.0 / sn;
    }
  }
  header[3] = f;
}

// One launch: every block folds its share of B (block 0 also the boundary) into header[2] by atomicMax; the
// last block to finish (counted in header[4]) updates the scale and leaves both words at zero for the next call.
__global__ void __launch_bounds__(256) update_scale_kernel(const double *B, int64_t n, const double *bnd, int nb,
                                                         double *header) {
  __shared__ unsigned long long red[8];
  unsigned long long *mx = reinterpret_cast<unsigned long long *>(header + 2);
  unsigned int *cnt = reinterpret_cast<unsigned int *>(header + 4);
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = B[i];
    if (x >= 0.0 && isfinite(x)) m = max(m, (unsigned long long)__double_as_longlong(x));
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
      const double x = bnd[i];
      if (x >= 0.0 && isfinite(x)) m = max(m, (unsigned long long)__double_as_longlong(x));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(kFull, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    if (m) atomicMax(mx, m);
    __threadfence();
    if (atomicAdd(cnt, 1u) == gridDim.x - 1) {   // last block: every other block's maximum is in place
      __threadfence();
      const unsigned long long all = atomicMax(mx, 0ull);
      update_scale(all, header);
      *mx = 0;
      *cnt = 0;
    }
  }
}

// Batched, several blocks per instance: map[block] = {instance, block of the instance, blocks of the instance, 0}.
// Each block folds its share of the instance's B (its block 0 also the boundary) into the instance's header[2] by
// atomicMax; the last of the instance's blocks (counted in header[4]) updates that instance's scale, as
// update_scale_kernel does for one plan.
template <class Inst>
__global__ void __launch_bounds__(256) update_scale_map_kernel(const Inst *inst, const int4 *map) {
  __shared__ unsigned long long red[8];
  const int4 m = map[blockIdx.x];
  const Inst &b = inst[m.x];
  double *header = const_cast<double *>(b.a.scale);
  unsigned long long *mx = reinterpret_cast<unsigned long long *>(header + 2);
  unsigned int *cnt = reinterpret_cast<unsigned int *>(header + 4);
  const int64_t n = (int64_t)b.v.G * b.v.ncell;
  unsigned long long v = 0;
  for (int64_t i = (int64_t)m.y * blockDim.x + threadIdx.x; i < n; i += (int64_t)m.z * blockDim.x) {
    const double x = b.a.B[i];
    if (x >= 0.0 && isfinite(x)) v = max(v, (unsigned long long)__double_as_longlong(x));
  }
  if (m.y == 0)
    for (int i = threadIdx.x; i < 4 * b.v.G; i += blockDim.x) {
      const double x = b.a.bnd[i];
      if (x >= 0.0 && isfinite(x)) v = max(v, (unsigned long long)__double_as_longlong(x));
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = max(v, red[w]);
    if (v) atomicMax(mx, v);
    __threadfence();
    if (atomicAdd(cnt, 1u) == (unsigned)m.z - 1) {   // last block of this instance
      __threadfence();
      const unsigned long long all = atomicMax(mx, 0ull);
      update_scale(all, header);
      *mx = 0;
      *cnt = 0;
    }
  }
}

int grid_for(int64_t n, int block) {
  int64_t b = (n + block - 1) / block;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (int)b;
}

}  // namespace

cudaError_t launch_prep(const PlanView &v, molc_precision prec, const SweepArgs &a, cudaStream_t st) {
  Layout L = layout_for(v, prec);
  if (prec == MOLC_FP64) L.gc = L.n_chunks = 1;   // input checks only: one group per tile row, all groups
  if (L.gc > 32 || L.n_chunks > 65535) return cudaErrorInvalidConfiguration;
  const int n_tiles = (v.ncell + kPrepCells - 1) / kPrepCells;
  const dim3 grid((unsigned)std::min(n_tiles, 152 * 16), (unsigned)(prec == MOLC_FP64 ? v.G : L.n_chunks));
  prep_kernel<<<grid, 128, 0, st>>>(v, a, L, prec == MOLC_FP32);
  return cudaGetLastError();
}

cudaError_t launch_sweep_fp64(const PlanView &v, const SweepArgs &a, cudaStream_t st) {
  const int64_t threads = v.n_tracks * 2 * (int64_t)v.G * v.n_polar;
  const int64_t blocks = (threads + 127) / 128;
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  if (v.balance)
    sweep_fp64_kernel<true><<<(unsigned)blocks, 128, 0, st>>>(v, a);
  else
    sweep_fp64_kernel<false><<<(unsigned)blocks, 128, 0, st>>>(v, a);
  return cudaGetLastError();
}

template <int D>
static cudaError_t sweep_fp32_depth(const PlanView &v, const SweepArgs &a, const Layout &L, dim3 grid,
                                    cudaStream_t st) {
  switch (v.n_polar) {
    case 1: sweep_fp32_kernel<1, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 2: sweep_fp32_kernel<2, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 3: sweep_fp32_kernel<3, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 4: sweep_fp32_kernel<4, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 5: sweep_fp32_kernel<5, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 6: sweep_fp32_kernel<6, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 7: sweep_fp32_kernel<7, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 8: sweep_fp32_kernel<8, D><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int EXTRA>
cudaError_t sweep_fp32_extra(const PlanView &v, const SweepArgs &a, const Layout &L, dim3 grid, cudaStream_t st) {
  switch (v.n_polar) {
    case 1: sweep_fp32_kernel<1, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 2: sweep_fp32_kernel<2, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 3: sweep_fp32_kernel<3, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 4: sweep_fp32_kernel<4, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 5: sweep_fp32_kernel<5, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 6: sweep_fp32_kernel<6, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 7: sweep_fp32_kernel<7, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    case 8: sweep_fp32_kernel<8, 4, EXTRA><<<grid, kSweepBlock, 0, st>>>(v, a, L); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_fp32(const PlanView &v, const SweepArgs &a, cudaStream_t st) {
  const Layout L = layout_for(v, MOLC_FP32);
  const int64_t blocks = (a.n_items + kSweepBlock - 1) / kSweepBlock;
  if (blocks > 0x7fffffff) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)blocks);
  if (v.facc) return sweep_fp32_extra<kSweepFaces>(v, a, L, grid, st);       // face reductions, depth 4
  if (v.balance) return sweep_fp32_extra<kSweepBalance>(v, a, L, grid, st);  // per-ray balance check, depth 4
  switch (v.sweep_depth) {
    case 3: return sweep_fp32_depth<3>(v, a, L, grid, st);
    case 4: return sweep_fp32_depth<4>(v, a, L, grid, st);
    case 6: return sweep_fp32_depth<6>(v, a, L, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_finalize(const PlanView &v, molc_precision prec, const SweepArgs &a, cudaStream_t st) {
  const Layout L = layout_for(v, prec);
  if (prec == MOLC_FP64) {
    finalize_kernel<<<grid_for(v.ncell, 128), 128, 0, st>>>(v, a, L);
    return cudaGetLastError();
  }
  const int64_t blocks = (v.n_munits * L.gc + 127) / 128;
  if (blocks > 0x7fffffff || L.n_chunks > 65535) return cudaErrorInvalidConfiguration;
  const dim3 grid((unsigned)blocks, (unsigned)L.n_chunks);
  const size_t smem = (size_t)v.n_pairs * (3 * v.n_polar + 2) * sizeof(float);
  if (smem > kMaxGatherSmem) return cudaErrorInvalidConfiguration;
  switch (v.n_polar) {
#define MOLC_MOMENTS(NP)                                                                                       \
  case NP:                                                                                                     \
    if (smem > 48 * 1024) {                                                                                    \
      cudaError_t e = cudaFuncSetAttribute(moments_fp32_kernel<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem);                                                         \
      if (e != cudaSuccess) return e;                                                                          \
    }                                                                                                          \
    moments_fp32_kernel<NP><<<grid, 128, smem, st>>>(v, a, L);                                                 \
    break;
    MOLC_MOMENTS(1)
    MOLC_MOMENTS(2)
    MOLC_MOMENTS(3)
    MOLC_MOMENTS(4)
    MOLC_MOMENTS(5)
    MOLC_MOMENTS(6)
    MOLC_MOMENTS(7)
    MOLC_MOMENTS(8)
#undef MOLC_MOMENTS
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || v.n_mmulti == 0) return e;
  const dim3 cgrid((unsigned)(((int64_t)v.n_mmulti * L.gc + 127) / 128), (unsigned)L.n_chunks);
  moments_combine_kernel<<<cgrid, 128, 0, st>>>(v, a, L);
  return cudaGetLastError();
}

// Face moments from the face sums: E_f = D is / (c |f|), F_f, N_f = sums is / |f|; is = 1/scale of the state
// (1 for FP64), |f| = hy on x-faces, hx on y-faces.  One thread per (face, group).
__global__ void face_moments_kernel(PlanView v, Layout L, const double *scale, double c, double hx, double hy,
                                    molc_moments out) {
  const int64_t n = (int64_t)v.n_faces * v.G;
  const int nxf = (v.nx + 1) * v.ny;
  const double is = scale ? scale[1] : 1.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int g = (int)(i / v.n_faces), f = (int)(i - (int64_t)g * v.n_faces);
    const int ch = g / L.gc, gl = g - ch * L.gc;
    const double *fa = v.facc + ((int64_t)ch * v.n_faces + f) * kOutputs * L.gc + gl;
    const double r = is / (f < nxf ? hy : hx);
    out.E[i] = fa[0] * r / c;
    out.Fx[i] = fa[L.gc] * r;
    out.Fy[i] = fa[2 * L.gc] * r;
    out.Nxx[i] = fa[3 * L.gc] * r;
    out.Nxy[i] = fa[4 * L.gc] * r;
    out.Nyy[i] = fa[5 * L.gc] * r;
  }
}

cudaError_t launch_face_moments(const PlanView &v, molc_precision prec, const double *scale, double c,
                                const molc_moments &out, cudaStream_t st) {
  const Layout L = layout_for(v, prec);
  face_moments_kernel<<<grid_for((int64_t)v.n_faces * v.G, 256), 256, 0, st>>>(v, L, scale, c, v.hx, v.hy, out);
  return cudaGetLastError();
}

cudaError_t launch_grey(const PlanView &v, const molc_moments &m, const double *kappa, const double *B,
                        double *out, cudaStream_t st) {
  grey_kernel<<<grid_for(v.ncell, 128), 128, 0, st>>>(v, m, kappa, B, out);
  return cudaGetLastError();
}

cudaError_t launch_closure(const PlanView &v, const molc_moments &m, double c, double *fxx, double *fxy,
                           double *fyy, double *f_grey, cudaStream_t st) {
  closure_kernel<<<grid_for(v.ncell, 256), 256, 0, st>>>(v, m, c, fxx, fxy, fyy, f_grey);
  return cudaGetLastError();
}

cudaError_t launch_update_scale(const PlanView &v, const double *B, const double *bnd, double *header,
                                cudaStream_t st) {
  const int64_t n = (int64_t)v.G * v.ncell;
  update_scale_kernel<<<std::min(grid_for(n, 256), 152 * 4), 256, 0, st>>>(B, n, bnd, 4 * v.G, header);
  return cudaGetLastError();
}

cudaError_t launch_update_scale_map(const BatchInst *inst, const TileInst *tinst, const int4 *map, int blocks,
                                    cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  if (tinst)
    update_scale_map_kernel<TileInst><<<blocks, 256, 0, st>>>(tinst, map);
  else
    update_scale_map_kernel<BatchInst><<<blocks, 256, 0, st>>>(inst, map);
  return cudaGetLastError();
}

cudaError_t launch_prep_batch(const BatchInst *inst, const int4 *map, int blocks, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  prep_batch_kernel<<<blocks, 128, 0, st>>>(inst, map);
  return cudaGetLastError();
}

template <int D>
static cudaError_t sweep_fp32_batch_depth(const BatchInst *inst, const int2 *map, int blocks, int n_polar,
                                          cudaStream_t st) {
  switch (n_polar) {
    case 1: sweep_fp32_batch_kernel<1, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 2: sweep_fp32_batch_kernel<2, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 3: sweep_fp32_batch_kernel<3, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 4: sweep_fp32_batch_kernel<4, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 5: sweep_fp32_batch_kernel<5, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 6: sweep_fp32_batch_kernel<6, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 7: sweep_fp32_batch_kernel<7, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    case 8: sweep_fp32_batch_kernel<8, D><<<blocks, kSweepBlock, 0, st>>>(inst, map); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep_fp32_batch(const BatchInst *inst, const int2 *map, int blocks, int n_polar, int depth,
                                    cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  switch (depth) {
    case 3: return sweep_fp32_batch_depth<3>(inst, map, blocks, n_polar, st);
    case 4: return sweep_fp32_batch_depth<4>(inst, map, blocks, n_polar, st);
    case 6: return sweep_fp32_batch_depth<6>(inst, map, blocks, n_polar, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_moments_fp32_batch(const BatchInst *inst, const int4 *map, int blocks, int n_polar,
                                      size_t smem, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  if (smem > kMaxGatherSmem) return cudaErrorInvalidConfiguration;
  switch (n_polar) {
#define MOLC_MOMENTS_B(NP)                                                                                     \
  case NP:                                                                                                     \
    if (smem > 48 * 1024) {                                                                                    \
      cudaError_t e = cudaFuncSetAttribute(moments_fp32_batch_kernel<NP>,                                      \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);            \
      if (e != cudaSuccess) return e;                                                                          \
    }                                                                                                          \
    moments_fp32_batch_kernel<NP><<<blocks, 128, smem, st>>>(inst, map);                                       \
    break;
    MOLC_MOMENTS_B(1)
    MOLC_MOMENTS_B(2)
    MOLC_MOMENTS_B(3)
    MOLC_MOMENTS_B(4)
    MOLC_MOMENTS_B(5)
    MOLC_MOMENTS_B(6)
    MOLC_MOMENTS_B(7)
    MOLC_MOMENTS_B(8)
#undef MOLC_MOMENTS_B
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_moments_combine_batch(const BatchInst *inst, const int4 *map, int blocks, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  moments_combine_batch_kernel<<<blocks, 128, 0, st>>>(inst, map);
  return cudaGetLastError();
}


cudaError_t launch_intensity_copy(const PlanView &v, molc_precision prec, void *I, const double *Bref,
                                  const double *scale, int g_begin, int g_count, double *canon, bool to_canon,
                                  cudaStream_t st) {
  const Layout L = layout_for(v, prec);
  if (prec == MOLC_FP64)
    intensity_copy_kernel<double><<<grid_for(L.rows, 128), 128, 0, st>>>(v, L, (double *)I, Bref, scale, g_begin,
                                                                         g_count, canon, to_canon, 0);
  else
    intensity_copy_kernel<float><<<grid_for(L.rows, 128), 128, 0, st>>>(v, L, (float *)I, Bref, scale, g_begin,
                                                                       g_count, canon, to_canon, 1);
  return cudaGetLastError();
}

cudaError_t launch_balance_scale(const PlanView &v, const double *B, const double *bnd, cudaStream_t st) {
  unsigned long long *mx = v.balance + 1;
  max_bits_kernel<<<grid_for((int64_t)v.G * v.ncell, 256), 256, 0, st>>>(B, (int64_t)v.G * v.ncell, mx);
  max_bits_kernel<<<1, 256, 0, st>>>(bnd, 4 * (int64_t)v.G, mx);
  return cudaGetLastError();
}

cudaError_t launch_set_scale(const PlanView &v, molc_precision prec, const double *B, double *header,
                             cudaStream_t st) {
  unsigned long long *mx = reinterpret_cast<unsigned long long *>(header + 2);
  cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  max_bits_kernel<<<grid_for((int64_t)v.G * v.ncell, 256), 256, 0, st>>>(B, (int64_t)v.G * v.ncell, mx);
  set_scale_kernel<<<1, 1, 0, st>>>(mx, header, prec == MOLC_FP32);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------------------
// FP64 FMA throughput of this GPU (the bound of the plain FP64 sweep, which spends its time in FP64 exp/expm1
// and FP64 atomics): every thread runs kFmaChains independent chains of kFmaIters dependent FMAs, so the FP64
// pipe, not latency, limits the rate.  The chains' sum is compared with a value it never takes and stored, if it
// did, to a static device variable, so that the work cannot be dropped and no pointer is needed.
// ---------------------------------------------------------------------------------------------------------
constexpr int kFmaChains = 8, kFmaIters = 4096;
__device__ double g_fma_sink;
__global__ void __launch_bounds__(256) fp64_fma_kernel(double a, double b) {
  double x[kFmaChains];
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) x[k] = threadIdx.x * 1e-3 + k;
  for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
    for (int k = 0; k < kFmaChains; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < kFmaChains; ++k) s += x[k];
  if (s == 12345.678) g_fma_sink = s;   // never true for the arguments used; keeps the chains live
}

cudaError_t fp64_fma_rate(double *flops_per_s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * 8, threads = 256;
  float best = 0.f;
  for (int rep = 0; e == cudaSuccess && rep < 4; ++rep) {   // first run warms up; best of the other three
    cudaEventRecord(e0, 0);
    fp64_fma_kernel<<<blocks, threads>>>(0.999999, 1e-7);
    cudaEventRecord(e1, 0);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return e;
  *flops_per_s = 2.0 * (double)blocks * threads * kFmaChains * kFmaIters / (best * 1e-3);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------------------------------------
// Static scratch of molc_sweep_static_scratch: the per-sweep workspace (moment accumulators, FP32 cell table)
// in an array fixed at build time, reserved when the module is loaded on a device, so that entry point
// allocates nothing.  The host name g_static_scratch is not a device address: its address on a device comes
// from cudaGetSymbolAddress with that device current, looked up once per device and cached.
// ---------------------------------------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

cudaError_t static_scratch_address(void **ptr) {
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static void *cached[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < kMaxDevices && cached[dev]) {
    *ptr = cached[dev];
    return cudaSuccess;
  }
  void *addr = nullptr;
  e = cudaGetSymbolAddress(&addr, g_static_scratch);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kMaxDevices) cached[dev] = addr;
  *ptr = addr;
  return cudaSuccess;
}


// =========================================================================================================
// Tiled FP32 sweep: the characteristic grid cut into per-tile pieces (molc_tiles.cpp), one persistent launch
// over work items (tile, quadrant, group tile) taken from an atomic ticket in wavefront order.  Per item:
//   1. one thread starts bulk copies (cp.async.bulk, completion on an mbarrier) of the item's previous-step state
//      (its pieces' deviations, packed step by step exactly as the item walks them) and of its cell table into
//      shared memory, and waits (bounded) until the items upstream in its quadrant have finished this step;
//   2. each thread walks one (piece, group): the deviation-form update of Eqs. 11-13, arithmetic identical to
//      sweep_fp32_body, with the state read and rewritten in shared memory and the records (cell, l) prefetched
//      four steps ahead from L2; the intensity leaving the tile goes to the next piece's slot of the boundary
//      buffer (L2), the item's flag is raised, and the new state is bulk-copied back;
//   3. each thread sums one cell's moment entries of this quadrant from the new state in shared memory (polar
//      fold in FP32, runs of one pair in FP32, two-word FP32 across runs) and writes the quadrant's partial
//      moments (FP64); the last of the four quadrant items of a (tile, group tile) adds the four partials in
//      quadrant order and assembles E, F, N (and f) like the moment gather.
// No block waits on a block that has not started: a ticket is taken only by a running block, and an item waits
// only on items of earlier tickets.  Every wait is bounded and records kStatusTimeout when it gives up.
// =========================================================================================================
namespace {

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16), completing on `bar`
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// shared -> global bulk copy in the issuing thread's bulk group
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// order this thread's shared-memory writes before later bulk copies (async proxy) read them
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr unsigned kBulkChunk = 32768;   // bytes per bulk-copy instruction

// shared memory of one block: state | cdat (float4) | cdB | P | direction table | split-cell partials (double)
struct TileSmem {
  size_t state, cdat, cdB, P, dir, split, total;
};
__host__ __device__ inline size_t up16(size_t b) { return (b + 15) / 16 * 16; }
__host__ __device__ inline TileSmem tile_smem_layout(int max_item_floats, int TS2p, int GT, int max_len,
                                                     int n_pairs, int np, int split_units) {
  TileSmem m;
  m.state = 0;
  m.cdat = up16((size_t)max_item_floats * 4);
  m.cdB = m.cdat + (size_t)GT * TS2p * 16;
  m.P = m.cdB + up16((size_t)GT * TS2p * 4);
  m.dir = m.P + up16((size_t)(max_len + 1) * 4);
  m.split = m.dir + up16((size_t)n_pairs * (3 * np + 2) * 4);
  m.total = m.split + (size_t)split_units * GT * kOutputs * 8;
  return m;
}

// Bounded spin of one thread on a flag reaching `epoch`; false (and the status recorded) if it gave up.  Once a
// wait of the plan has given up, later ones do not wait at all (the step's results are void anyway).
__device__ bool wait_flag(const int *flag, int epoch, int *status) {
  for (int it = 0; it < kTileWaitLimit; ++it) {
    if (ld_acquire_gpu(flag) >= epoch) return true;
    if ((it & 255) == 255 && (*(volatile int *)status & kStatusTimeout)) return false;
    __nanosleep(it < 64 ? 32 : 256);
  }
  atomicOr(status, kStatusTimeout);
  return false;
}

// Cell tables of the tiles (prep_tiles, laid out [tile][G][TS2p], the state's rescale folded into the second
// entry), the input checks, the ticket reset of the coming sweep launch and the plan's step epoch.
__device__ __forceinline__ void tile_prep_body(const PlanView &v, const TileView &t, const SweepArgs &a, int4 m,
                                               int *ticket) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;
  if (m.w && threadIdx.x == 0) t.ctrl[1] += 1;   // a new step of this plan: flags of earlier steps are stale
  const int TS = t.TS, TS2 = TS * TS;
  const int tpb = max(1, (int)blockDim.x / TS2);
  const int tile = m.y + threadIdx.x / TS2, cl = threadIdx.x % TS2;
  const int g = m.z;
  bool bad = false, range = false;
  if (threadIdx.x < tpb * TS2 && tile < t.n_tiles) {
    const int ix = (tile % t.ntx) * TS + cl % TS, iy = (tile / t.ntx) * TS + cl / TS;
    if (ix < v.nx && iy < v.ny) {
      const float inv_cdt_f = (float)a.inv_cdt;
      const double sc = a.scale[0];
      const float rescale = (float)a.scale[3];
      const int64_t idx = (int64_t)g * v.ncell + (int64_t)iy * v.nx + ix;
      const double kap = a.kappa[idx], B = a.B[idx];
      bad = bad_input(kap) | bad_input(B);
      const float kt = (float)(kap + a.inv_cdt);
      const float r = __fdiv_rn(inv_cdt_f, kt);
      const double Bs = B * sc;
      range = __double_as_longlong(Bs) >= __double_as_longlong(kScaledMax);
      const float bhi = (float)Bs;
      const float blo = (float)(Bs - f32_to_f64_exact(bhi));
      const int64_t o = ((int64_t)tile * v.G + g) * t.TS2p + cl;
      t.cdat[o] = make_float4(kt, r * rescale, bhi, blo);
      t.cdB[o] = (float)((a.Bref[idx] - B) * sc) * r;
    }
  }
  if (m.w)
    for (int i = threadIdx.x; i < 4 * v.G; i += blockDim.x) {
      bad |= bad_input(a.bnd[i]);
      range |= !(a.bnd[i] * a.scale[0] < kScaledMax);
    }
  if (bad) atomicOr(v.status, kStatusNonfinite);
  if (range && !bad) atomicOr(v.status, kStatusRange);
}

// map[block] = {instance, first tile, group, 1: this block also checks the boundary and starts the plan's step}
__global__ void __launch_bounds__(256) tile_prep_kernel(const TileInst *inst, const int4 *map, int *ticket) {
  const int4 m = map[blockIdx.x];
  const TileInst &I = inst[m.x];
  tile_prep_body(I.v, I.t, I.a, m, ticket);
}

// One plan: the call's instance comes by value and is stored for the sweep launch that follows.
__global__ void __launch_bounds__(256) tile_prep_one_kernel(TileInst ov, TileInst *dst, const int4 *map,
                                                            int *ticket) {
  const int4 m = map[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) *dst = ov;
  tile_prep_body(ov.v, ov.t, ov.a, m, ticket);
}

// Moments of one cell unit (entries [e0, e1) of the geometry) from the new state in shared memory: polar fold
// in FP32, runs of at most kPairRun entries of one pair in FP32, two-word FP32 across runs (as the moment
// gather), then FP64.
template <int NPM, bool EXACT>
__device__ __forceinline__ void tile_unit_sums(const TileView &t, const TileGeom &gm, int np, int gcnt, int gl,
                                               const float *sst, const float *dirt, int e0, int e1,
                                               double (&D)[kOutputs]) {
  float hi[kOutputs], lo[kOutputs];
#pragma unroll
  for (int k = 0; k < kOutputs; ++k) hi[k] = lo[k] = 0.f;
  const int dstride = 3 * np + 2;
  int cur = -1, run = 0;
  float P0 = 0.f, P1 = 0.f, P2 = 0.f;
  auto flush = [&]() {
    if (cur < 0) return;
    const float cf = dirt[cur * dstride + 3 * np], sf = dirt[cur * dstride + 3 * np + 1];
    two_sum_add(hi[0], lo[0], P0);
    two_sum_add(hi[1], lo[1], cf * P1);
    two_sum_add(hi[2], lo[2], sf * P1);
    two_sum_add(hi[3], lo[3], (cf * cf) * P2);
    two_sum_add(hi[4], lo[4], (cf * sf) * P2);
    two_sum_add(hi[5], lo[5], (sf * sf) * P2);
  };
  const int2 *ent = t.ents + gm.ent_off;
  constexpr int kBatch = 8;   // entries loaded together (their L2 latencies overlap)
  for (int eb = e0; eb < e1; eb += kBatch) {
    int2 enb[kBatch];
#pragma unroll
    for (int b = 0; b < kBatch; ++b) enb[b] = eb + b < e1 ? __ldg(ent + eb + b) : make_int2(0, 0);
#pragma unroll
    for (int b = 0; b < kBatch; ++b) {
      if (eb + b >= e1) break;
      const int2 en = enb[b];
      const int slot = en.x & 0xFFFFFF, pr = (int)((unsigned)en.x >> 24);
      if (pr != cur || run == kPairRun) {
        flush();
        cur = pr;
        run = 0;
        P0 = P1 = P2 = 0.f;
      }
      ++run;
      const float *dv = sst + ((int64_t)slot * gcnt + gl) * np;
      const float *c0 = dirt + pr * dstride;
      float S0 = 0.f, S1 = 0.f, S2 = 0.f;
#pragma unroll
      for (int p = 0; p < NPM; ++p)
        if (EXACT || p < np) {
          const float x = dv[p];
          S0 = fmaf(c0[p], x, S0);
          S1 = fmaf(c0[np + p], x, S1);
          S2 = fmaf(c0[2 * np + p], x, S2);
        }
      const float af = __int_as_float(en.y);
      P0 = fmaf(af, S0, P0);
      P1 = fmaf(af, S1, P1);
      P2 = fmaf(af, S2, P2);
    }
  }
  flush();
#pragma unroll
  for (int k = 0; k < kOutputs; ++k) D[k] = f32_to_f64(hi[k]) + f32_to_f64(lo[k]);
}

template <int NPM, bool EXACT>
__global__ void __launch_bounds__(512) tile_sweep_kernel(const TileInst *inst, const int2 *queue, int n_queue,
                                                        int *ticket, TileSmem lay) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ unsigned long long bar;
  __shared__ int s_q, s_last;
  float *sst = reinterpret_cast<float *>(smem + lay.state);
  float4 *scd = reinterpret_cast<float4 *>(smem + lay.cdat);
  float *scdB = reinterpret_cast<float *>(smem + lay.cdB);
  int *sP = reinterpret_cast<int *>(smem + lay.P);
  float *sdir = reinterpret_cast<float *>(smem + lay.dir);
  double *ssplit = reinterpret_cast<double *>(smem + lay.split);
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_proxy_async_smem();
  }
  __syncthreads();
  unsigned phase = 0;
  bool stored = false;   // a bulk store of this block may still be reading shared memory
  int next_q = 0;        // thread 0: the ticket taken for the next item while this one runs
  if (tid == 0) next_q = atomicAdd(ticket, 1);
  for (;;) {
    if (tid == 0) s_q = next_q;
    __syncthreads();
    const int qi = s_q;
    if (qi >= n_queue) break;
    // Take the next ticket now (its latency overlaps this item).  Still no block waits on one that has not
    // started: the smallest unfinished ticket is either some block's current item (its upstream items hold
    // smaller tickets, all finished) or a block's next item whose current item, smaller still, is unfinished.
    if (tid == 0) next_q = atomicAdd(ticket, 1);
    const int2 qe = queue[qi];
    const TileInst &I = inst[qe.x];
    const PlanView &v = I.v;
    const TileView &t = I.t;
    const SweepArgs &a = I.a;
    const int item = qe.y;
    const int gt = item / t.n_geoms, gidx = item - gt * t.n_geoms;
    const TileGeom gm = t.geoms[gidx];
    const int np = EXACT ? NPM : v.n_polar;
    const int g0 = gt * t.GT, gcnt = min(t.GT, v.G - g0);
    const int epoch = t.ctrl[1];
    float *state_g = (float *)a.I + t.item_off[item];
    const unsigned state_bytes = (unsigned)((((int64_t)gm.n_slots * gcnt * np + 3) / 4 * 4) * 4);
    const int64_t cd_off = ((int64_t)gm.tile * v.G + g0) * t.TS2p;
    // 1. stage the state and the cell table (one thread), wait for the upstream items (one thread)
    if (tid == 0) {
      if (stored) bulk_wait_read_all();   // the previous item's store has read the buffer
      const unsigned cd_bytes = (unsigned)gcnt * t.TS2p * 16, cdB_bytes = (unsigned)gcnt * t.TS2p * 4;
      mbar_arrive_expect_tx(&bar, state_bytes + cd_bytes + cdB_bytes);
      for (unsigned o = 0; o < state_bytes; o += kBulkChunk)
        bulk_load((char *)sst + o, (const char *)state_g + o, min(kBulkChunk, state_bytes - o), &bar);
      bulk_load(scd, t.cdat + cd_off, cd_bytes, &bar);
      bulk_load(scdB, t.cdB + cd_off, cdB_bytes, &bar);
    }
    for (int i = tid; i <= gm.max_len; i += nthr) sP[i] = t.Ptab[gm.P_off + i];
    {
      // direction table of this quadrant: per pair the polar folds {w, w sin, w sin^2} and the in-plane
      // direction of the pair's sense that points into q
      const int dstride = 3 * np + 2;
      for (int i = tid; i < v.n_pairs * dstride; i += nthr) {
        const int pr = i / dstride, k = i - pr * dstride;
        float val;
        if (k < 3 * np) {
          const int p = k % np, kind = k / np;
          const PolarDev pd = v.polar[pr * np + p];
          val = kind == 0 ? pd.wf : kind == 1 ? pd.wf * pd.sinzf : (pd.wf * pd.sinzf) * pd.sinzf;
        } else {
          const PairDev pp = v.pairs[pr];
          const bool minus = ((pp.c < 0) != ((gm.q & 1) != 0)) || ((pp.s < 0) != ((gm.q & 2) != 0));
          const float cf = minus ? -pp.cf : pp.cf, sf = minus ? -pp.sf : pp.sf;
          val = k == 3 * np ? cf : sf;
        }
        sdir[i] = val;
      }
    }
    if (tid == 0) {
      const int base = gt * t.n_geoms;
      if (gm.up_x >= 0) wait_flag(t.flags + base + gm.up_x, epoch, v.status);
      if (gm.up_y >= 0) wait_flag(t.flags + base + gm.up_y, epoch, v.status);
      int it = 0;
      while (!mbar_try_wait(&bar, phase) && ++it < kTileWaitLimit) {
        if ((it & 255) == 0 && (*(volatile int *)v.status & kStatusTimeout)) break;   // the step is void already
        __nanosleep(32);
      }
      if (it >= kTileWaitLimit) atomicOr(v.status, kStatusTimeout);
    }
    __syncthreads();
    // all threads observe the completed phase (the copies' data is visible to them after this wait)
    {
      int it = 0;
      while (!mbar_try_wait(&bar, phase) && ++it < kTileWaitLimit) {
        if ((it & 255) == 0 && (*(volatile int *)v.status & kStatusTimeout)) break;
        __nanosleep(32);
      }
    }
    phase ^= 1;
    // 2. walk the pieces
    const double sc = a.scale[0];
    for (int k = tid; k < gm.n_pieces * gcnt; k += nthr) {
      const int r = k / gcnt, gl = k - r * gcnt, g = g0 + gl;
      const int4 pc = t.pieces[gm.piece_off + r];
      const int len = pc.y >> 1;
      const int pair = v.tracks[pc.x].pair;
      float half_inv_sinz[NPM], sinz[NPM], psi[NPM];
#pragma unroll
      for (int p = 0; p < NPM; ++p) {
        half_inv_sinz[p] = sinz[p] = psi[p] = 0.f;
        if (EXACT || p < np) {
          const PolarDev pd = v.polar[pair * np + p];
          half_inv_sinz[p] = 0.5f * pd.inv_sinzf;
          sinz[p] = pd.sinzf;
        }
      }
      float bhi_prev, blo_prev;
      if (pc.z < 0) {   // the piece starts on the domain boundary: entering intensity, split like B
        const double bin = a.bnd[(-1 - pc.z) * v.G + g] * sc;
        bhi_prev = (float)bin;
        blo_prev = (float)(bin - (double)bhi_prev);
      } else {          // from the previous piece of the characteristic (through L2)
        const float *bb = t.bbuf + ((int64_t)pc.z * v.G + g) * (np + 2);
#pragma unroll
        for (int p = 0; p < NPM; ++p)
          if (EXACT || p < np) psi[p] = __ldcg(bb + p);
        bhi_prev = __ldcg(bb + np);
        blo_prev = __ldcg(bb + np + 1);
      }
      const int2 *rec = t.recs + gm.slot_base + r;
      int2 rr[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) rr[u] = u < len ? ld_record(rec + sP[u]) : make_int2(0, 0);
      for (int s0 = 0; s0 < len; s0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int s = s0 + u;
          if (s < len) {
            const int2 rc = rr[u];
            if (s + 4 < len) rr[u] = ld_record(rec + sP[s + 4]);
            float *sv = sst + ((int64_t)(sP[s] + r) * gcnt + gl) * np;
            const float4 q = scd[gl * t.TS2p + rc.x];
            const float dB = scdB[gl * t.TS2p + rc.x];
            const float len_f = __int_as_float(rc.y);
            const float jump = (bhi_prev - q.z) + (blo_prev - q.w);
            const float kl = q.x * len_f;
            const float rkl = rcp_approx(kl);
            float dv[NPM];
            if constexpr (NPM == 4) {
              if (EXACT) {
                const float4 d4 = *reinterpret_cast<const float4 *>(sv);
                dv[0] = d4.x;
                dv[1] = d4.y;
                dv[2] = d4.z;
                dv[3] = d4.w;
              } else {
#pragma unroll
                for (int p = 0; p < NPM; ++p) dv[p] = p < np ? sv[p] : 0.f;
              }
            } else {
#pragma unroll
              for (int p = 0; p < NPM; ++p) dv[p] = (EXACT || p < np) ? sv[p] : 0.f;
            }
#pragma unroll
            for (int p = 0; p < NPM; ++p) psi[p] += jump;
#pragma unroll
            for (int p = 0; p < NPM; ++p) {
              if (EXACT || p < np) {
                float E1, om, ex;
                bool thin;
                const float ahalf = kl * half_inv_sinz[p];
                attenuation(ahalf, sinz[p] * rkl, E1, om, ex, thin);
                const float d = fmaf(dv[p], q.y, dB);
                const float pin = psi[p];
                const float x = pin - d;
                dv[p] = fmaf(x, E1, d);
                psi[p] = thin ? fmaf(-x, om, pin) : fmaf(x, ex, d);
              }
            }
            if constexpr (NPM == 4) {
              if (EXACT) {
                *reinterpret_cast<float4 *>(sv) = make_float4(dv[0], dv[1], dv[2], dv[3]);
              } else {
#pragma unroll
                for (int p = 0; p < NPM; ++p)
                  if (p < np) sv[p] = dv[p];
              }
            } else {
#pragma unroll
              for (int p = 0; p < NPM; ++p)
                if (EXACT || p < np) sv[p] = dv[p];
            }
            bhi_prev = q.z;
            blo_prev = q.w;
          }
        }
      }
      if (pc.w >= 0) {   // hand the outgoing intensity to the next piece
        float *bb = t.bbuf + ((int64_t)pc.w * v.G + g) * (np + 2);
#pragma unroll
        for (int p = 0; p < NPM; ++p)
          if (EXACT || p < np) __stcg(bb + p, psi[p]);
        __stcg(bb + np, bhi_prev);
        __stcg(bb + np + 1, blo_prev);
      }
    }
    fence_proxy_async_smem();   // this thread's state writes before the bulk store reads them
    __syncthreads();
    if (tid == 0) {
      if (state_bytes) {
        for (unsigned o = 0; o < state_bytes; o += kBulkChunk)
          bulk_store((char *)state_g + o, (const char *)sst + o, min(kBulkChunk, state_bytes - o));
        bulk_commit();
        stored = true;
      }
      __threadfence();   // every thread's boundary writes (ordered by the barrier) before the flag
      st_release_gpu(t.flags + item, epoch);
    }
    // 3. moments of this quadrant: split cells' parts into shared memory first, then one task per (cell, group)
    const int TS2 = t.TS * t.TS;
    const int2 *cu = t.cell_units + gm.cu_off;
    const int4 *un = t.units + gm.unit_off;
    if (lay.total > lay.split) {
      for (int k = tid; k < gm.n_units * gcnt; k += nthr) {
        const int u = k / gcnt, gl = k - u * gcnt;
        const int4 uu = un[u];
        if (cu[uu.x].y > 1) {
          double D[kOutputs];
          tile_unit_sums<NPM, EXACT>(t, gm, np, gcnt, gl, sst, sdir, uu.y, uu.z, D);
#pragma unroll
          for (int o = 0; o < kOutputs; ++o) ssplit[((int64_t)u * gcnt + gl) * kOutputs + o] = D[o];
        }
      }
      __syncthreads();
    }
    double *part = t.part + (((int64_t)gm.tile * t.n_gt + gt) * 4 + gm.q) * kOutputs * t.GT * t.TS2p;
    for (int k = tid; k < TS2 * gcnt; k += nthr) {
      const int gl = k / TS2, cl = k - gl * TS2;
      const int2 c = cu[cl];
      double D[kOutputs] = {0, 0, 0, 0, 0, 0};
      if (c.y == 1) {
        const int4 uu = un[c.x];
        tile_unit_sums<NPM, EXACT>(t, gm, np, gcnt, gl, sst, sdir, uu.y, uu.z, D);
      } else {
        for (int j = 0; j < c.y; ++j)
#pragma unroll
          for (int o = 0; o < kOutputs; ++o) D[o] += ssplit[((int64_t)(c.x + j) * gcnt + gl) * kOutputs + o];
      }
#pragma unroll
      for (int o = 0; o < kOutputs; ++o) part[((int64_t)o * t.GT + gl) * t.TS2p + cl] = D[o];
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      int *cnt = t.cnt + (int64_t)gm.tile * t.n_gt + gt;
      const int prev = atomicAdd(cnt, 1);
      s_last = prev == 3;
      if (prev == 3) {
        *cnt = 0;   // ready for the next step (its items start after this launch ends)
        __threadfence();
      }
    }
    __syncthreads();
    if (s_last) {   // the four quadrant partials are in place: assemble the tile's cells
      const double *pt = t.part + ((int64_t)gm.tile * t.n_gt + gt) * 4 * kOutputs * t.GT * t.TS2p;
      const int tx = gm.tile % t.ntx, ty = gm.tile / t.ntx;
      for (int k = tid; k < TS2 * gcnt; k += nthr) {
        const int gl = k / TS2, cl = k - gl * TS2;
        const int ix = tx * t.TS + cl % t.TS, iy = ty * t.TS + cl / t.TS;
        if (ix >= v.nx || iy >= v.ny) continue;
        double D[kOutputs] = {0, 0, 0, 0, 0, 0};
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int o = 0; o < kOutputs; ++o)
            D[o] += __ldcg(pt + (((int64_t)q * kOutputs + o) * t.GT + gl) * t.TS2p + cl);
        assemble_cell(v, a, iy * v.nx + ix, g0 + gl, D);
      }
    }
    __syncthreads();
  }
  if (tid == 0 && stored) bulk_wait_all();   // the last state store has completed
}

// Canonical segment averages <-> tiled FP32 state: one thread per row (track, sense, step), looping over polar
// cosines and the selected groups (as intensity_copy_kernel; only the element address differs).
__global__ void tile_intensity_copy_kernel(PlanView v, TileView t, const int4 *tpiece, const int64_t *tpiece_off,
                                           float *I, const double *Bref, const double *scale, int g_begin,
                                           int g_count, double *canon, int to_canon, int64_t rows) {
  const int NP = v.n_polar;
  const double sc = scale[0], is = scale[1];
  for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = find_track(v.tracks, v.n_tracks, row);
    const TrackDev tr = v.tracks[k];
    const int64_t local = row - 2 * tr.seg_off;
    const int sense = local >= tr.nseg;
    const int s = (int)(local - (int64_t)sense * tr.nseg);
    const int cell = v.seg_cell[sense ? tr.seg_off + tr.nseg - 1 - s : tr.seg_off + s];
    // the piece holding step s of this sense
    const int64_t a0 = tpiece_off[2 * k + sense], a1 = tpiece_off[2 * k + sense + 1];
    int64_t pi = a0;
    while (pi + 1 < a1 && tpiece[pi + 1].z <= s) ++pi;
    const int4 tp = tpiece[pi];
    const TileGeom gm = t.geoms[tp.x];
    const int slot = t.Ptab[gm.P_off + (s - tp.z)] + tp.y;
    for (int p = 0; p < NP; ++p) {
      const PolarDev pd = v.polar[tr.pair * NP + p];
      const int dir = sense ? pd.dir_minus : pd.dir_plus;
      const int64_t cs = v.dir_seg_off[dir] + (sense ? tr.canon_minus : tr.canon_plus) + s;
      for (int g = g_begin; g < g_begin + g_count; ++g) {
        const int gt = g / t.GT, gl = g - gt * t.GT, gcnt = min(t.GT, v.G - gt * t.GT);
        float *el = I + t.item_off[(int64_t)gt * t.n_geoms + tp.x] + ((int64_t)slot * gcnt + gl) * NP + p;
        const double br = Bref[(int64_t)g * v.ncell + cell];
        double *cv = canon + cs * g_count + (g - g_begin);
        if (to_canon)
          *cv = br + (double)*el * is;
        else
          *el = (float)((*cv - br) * sc);
      }
    }
  }
}

// Allow a kernel the device's largest dynamic shared memory (the opt-in limit less its static shared memory).
cudaError_t allow_max_dynamic_smem(const void *fn) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) cudaGetLastError();   // do not leave the error for a later launch check
  return e;
}

template <int NPM, bool EXACT>
cudaError_t launch_tile_np(const TileInst *inst, const int2 *queue, int n_queue, int *ticket, const TileSmem &lay,
                           int grid, int threads, cudaStream_t st) {
  static bool attr = false;   // once per instantiation
  if (!attr) {
    cudaError_t e = allow_max_dynamic_smem((const void *)tile_sweep_kernel<NPM, EXACT>);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  tile_sweep_kernel<NPM, EXACT><<<grid, threads, lay.total, st>>>(inst, queue, n_queue, ticket, lay);
  return cudaGetLastError();
}

}  // namespace

size_t tile_sweep_smem(const TileShape &sh, int np_max) {
  return tile_smem_layout(sh.max_item_floats, sh.cd_entries, 1, sh.max_len, sh.n_pairs, np_max, sh.split_units).total;
}

cudaError_t launch_tile_prep(const TileInst *inst, const int4 *map, int blocks, int *ticket, cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  tile_prep_kernel<<<blocks, 256, 0, st>>>(inst, map, ticket);
  return cudaGetLastError();
}

cudaError_t launch_tile_prep_one(const TileInst &ov, TileInst *dst, const int4 *map, int blocks, int *ticket,
                                 cudaStream_t st) {
  if (blocks <= 0) return cudaSuccess;
  tile_prep_one_kernel<<<blocks, 256, 0, st>>>(ov, dst, map, ticket);
  return cudaGetLastError();
}

cudaError_t launch_tile_sweep(const TileInst *inst, const int2 *queue, int n_queue, int *ticket, int np_max,
                              const TileShape &sh, int grid, int threads, cudaStream_t st) {
  const TileSmem lay = tile_smem_layout(sh.max_item_floats, sh.cd_entries, 1, sh.max_len, sh.n_pairs, np_max,
                                        sh.split_units);
  const bool exact = sh.np_exact == np_max;
  switch (np_max) {
    case 1: return exact ? launch_tile_np<1, true>(inst, queue, n_queue, ticket, lay, grid, threads, st)
                         : launch_tile_np<1, false>(inst, queue, n_queue, ticket, lay, grid, threads, st);
    case 2: return exact ? launch_tile_np<2, true>(inst, queue, n_queue, ticket, lay, grid, threads, st)
                         : launch_tile_np<2, false>(inst, queue, n_queue, ticket, lay, grid, threads, st);
    case 3: case 4: return exact && np_max == 4 ? launch_tile_np<4, true>(inst, queue, n_queue, ticket, lay, grid, threads, st)
                                                : launch_tile_np<4, false>(inst, queue, n_queue, ticket, lay, grid, threads, st);
    default: return exact && np_max == 8 ? launch_tile_np<8, true>(inst, queue, n_queue, ticket, lay, grid, threads, st)
                                         : launch_tile_np<8, false>(inst, queue, n_queue, ticket, lay, grid, threads, st);
  }
}

int tile_sweep_grid(int np_max, size_t smem, int threads) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void *fn = np_max <= 1 ? (const void *)tile_sweep_kernel<1, true>
                 : np_max <= 2 ? (const void *)tile_sweep_kernel<2, true>
                 : np_max <= 4 ? (const void *)tile_sweep_kernel<4, true> : (const void *)tile_sweep_kernel<8, true>;
  allow_max_dynamic_smem(fn);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem) != cudaSuccess || per < 1) {
    cudaGetLastError();
    per = 1;
  }
  return sms * per;
}

cudaError_t launch_tile_intensity_copy(const PlanView &v, const TileView &t, const int4 *tpiece,
                                       const int64_t *tpiece_off, float *I, const double *Bref,
                                       const double *scale, int g_begin, int g_count, double *canon, bool to_canon,
                                       cudaStream_t st) {
  const int64_t rows = 2 * v.n_track_segments;
  tile_intensity_copy_kernel<<<grid_for(rows, 128), 128, 0, st>>>(v, t, tpiece, tpiece_off, I, Bref, scale, g_begin,
                                                                  g_count, canon, to_canon, rows);
  return cudaGetLastError();
}

}  // namespace molc
