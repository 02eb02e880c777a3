"""Emulations of the two working-precision evaluations of Eq. 12 (test helper, CPU only).

They restate, in numpy, the arithmetic of a sweep that carries the deviation psi = I - B_cell along each
characteristic (Sec. 3, Eqs. 11-13 rewritten exactly: Ibar = S + (I_s - S) E1, I_{s+1} = S + (I_s - S) e^-tau):

* `emulate(..., "fp32")`: every operation rounded to IEEE binary32 in the order a GB300 FP32 path evaluates it,
  with 2^x and 1/x correctly rounded or (`approx`) given a relative error up to the hardware approximations'
  stated accuracy, B split in two FP32 words, and the state in units scaled by a power of two;
* `emulate(..., "fp64")`: every operation in binary64, with numpy's exp/expm1.

They walk the oracle's own characteristic grid in its canonical order and return the segment-average
deviations Ibar - B of the cell, canonical [nseg][G], so that the error of each can be set against the oracle's
first-order bound of that arithmetic.  Nothing here is imported by the library or by the oracle.
"""
import numpy as np

f32 = np.float32


def _fma32(a, b, c):
    """a * b + c with one rounding to binary32 (the product of two binary32 numbers is exact in binary64)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(f32)


def _r32(x):
    return np.asarray(x, np.float64).astype(f32)


def _fma64(a, b, c):
    """a * b + c in binary64 with the product kept exact (Veltkamp split and error-free sums): one rounding
    except for rare double roundings of the final addition."""
    a, b, c = (np.asarray(v, np.float64) for v in (a, b, c))
    p = a * b
    sp = 134217729.0   # 2^27 + 1
    ah = a * sp - (a * sp - a)
    al = a - ah
    bh = b * sp - (b * sp - b)
    bl = b - bh
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl   # p + e = a b exactly
    s = p + c
    bp = s - p
    t = (p - (s - bp)) + (c - bp)                        # s + t = p + c exactly
    return s + (t + e)


def emulate(tr, mu, kappa, B, c, dt, bnd, prec, dev_prev=None, Bref=None, approx=None):
    """One sweep; tr = oracle.tracks(geometry); mu [ndir]; kappa, B [G][ncell]; bnd [4][G]; dev_prev: canonical
    [nseg][G] stored deviations from Bref (None: 0, i.e. I^{n-1} = B); Bref [G][ncell] (None: B).  approx (FP32
    only): (rel_ex2, rel_rcp, seed) to give every 2^x and 1/x a relative error of +-rel (seeded signs) before
    its rounding to binary32, as the hardware approximations may; None: correctly rounded.  Returns the new
    canonical deviations from B (float64 array of the path's values)."""
    kappa = np.asarray(kappa, np.float64)
    B = np.asarray(B, np.float64)
    Bref = B if Bref is None else np.asarray(Bref, np.float64)
    G, ncell = B.shape
    nseg = tr["cell"].size
    out = np.zeros((nseg, G))
    inv_cdt = 1.0 / (c * dt)
    if prec == "fp32":
        # state scale: a power of two that maps max(B, boundary) to [2^99, 2^100)
        m = max(float(B.max()), float(np.max(bnd)))
        e = np.frexp(m)[1] if m > 0 else 0
        sc = 2.0 ** (100 - e)
        kt = _r32(kappa + inv_cdt)                      # [G][ncell]
        r = (_r32(np.full_like(kappa, inv_cdt)) / kt).astype(f32)   # correctly rounded division
        Bs = B * sc
        bhi = _r32(Bs)
        blo = _r32(Bs - bhi.astype(np.float64))
        dB = (_r32((Bref - B) * sc) * r).astype(f32)
        minus_log2e = f32(-1.4426950408889634)
        c5040, c120, c6 = f32(1.0 / 5040.0), f32(1.0 / 120.0), f32(1.0 / 6.0)
    if approx is not None:
        rel_ex2, rel_rcp, seed = approx
        rng = np.random.default_rng(seed)
        perturb = lambda v, rel: v * (1.0 + rel * rng.choice((-1.0, 1.0), size=np.shape(v)))
    else:
        perturb = lambda v, rel: v
        rel_ex2 = rel_rcp = 0.0
    seg = 0
    for m in range(mu.size):
        sinz = np.sqrt(1.0 - mu[m] * mu[m])
        if prec == "fp32":
            half_inv_sinz = f32(0.5) * _r32(1.0 / sinz)
            sinzf = _r32(sinz)
        for k in range(tr["dir_ray_off"][m], tr["dir_ray_off"][m + 1]):
            s0, s1 = tr["ray_seg_off"][k], tr["ray_seg_off"][k + 1]
            edge = tr["entry"][k]
            if prec == "fp32":
                bin_ = bnd[edge] * sc
                bh_prev = _r32(bin_)
                bl_prev = _r32(bin_ - bh_prev.astype(np.float64))
                psi = np.zeros(G, f32)
            else:
                Iin = np.asarray(bnd[edge], np.float64)
                psi = np.zeros(G)
                Bprev = None
            for q in range(s0, s1):
                i = tr["cell"][q]
                dv = np.zeros(G) if dev_prev is None else dev_prev[seg]
                if prec == "fp32":
                    jump = (_r32(bh_prev - bhi[:, i]) + _r32(bl_prev - blo[:, i])).astype(f32)
                    kl = (kt[:, i] * _r32(tr["len"][q])).astype(f32)
                    rkl = _r32(perturb(1.0 / kl.astype(np.float64), rel_rcp))
                    psi = (psi + jump).astype(f32)
                    a = (kl * half_inv_sinz).astype(f32)
                    h = _r32(perturb(np.exp2((a * minus_log2e).astype(np.float64)), rel_ex2))
                    ex = (h * h).astype(f32)
                    y = (a * a).astype(f32)
                    p = _fma32(y, c5040, c120)
                    p = _fma32(p, y, c6)
                    p = _fma32(p, y, f32(1.0))
                    hp = (h * p).astype(f32)
                    thin = a < f32(0.25)
                    inv_tau = (sinzf * rkl).astype(f32)
                    E1 = np.where(thin, hp, ((f32(1.0) - ex).astype(f32) * inv_tau).astype(f32))
                    om = ((a + a).astype(f32) * hp).astype(f32)
                    d = _fma32(_r32(dv * sc), r[:, i], dB[:, i])
                    x = (psi - d).astype(f32)
                    pbar = _fma32(x, E1, d)
                    psi = np.where(thin, _fma32(-x, om, psi), _fma32(x, ex, d))
                    # the stored deviation refers to this cell's B: back to unscaled units (exact)
                    out[seg] = pbar.astype(np.float64) / sc
                    bh_prev, bl_prev = bhi[:, i], blo[:, i]
                else:
                    Bc = B[:, i]
                    kt64 = kappa[:, i] + inv_cdt
                    jump = (Iin - Bc) if Bprev is None else (Bprev - Bc)
                    psi = jump if Bprev is None else psi + jump
                    d = (dv + (Bref[:, i] - Bc)) * (inv_cdt / kt64)
                    tau = kt64 * tr["len"][q] * (1.0 / sinz)
                    ome = -np.expm1(-tau)
                    ex = np.exp(-tau)
                    E1 = ome / tau
                    x = psi - d
                    pbar = _fma64(x, E1, d)
                    psi = np.where(tau < 0.5, _fma64(-x, ome, psi), _fma64(x, ex, d))
                    out[seg] = pbar
                    Bprev = Bc
                seg += 1
    return out
