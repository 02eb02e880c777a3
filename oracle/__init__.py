"""The oracle: a plain CPU implementation of the MOLC high-order sweep (Sec. 3), in double and binary128.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It never imports the CUDA library's package, and the library never imports it.

``build()`` compiles ``molc_oracle.cpp`` with g++ into ``oracle/_build/``; everything else is ctypes glue
that hands numpy arrays to the C++ code and returns numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "molc_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "libmolc_oracle.so")
_lib = None

MOMENTS = ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy", "Nzz", "absFx", "absFy", "absNxy", "absBNxy", "absBFx", "absBFy")
PREC = {"double": 0, "quad": 1}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, IEEE arithmetic; libquadmath on x86-64)."""
    if not force and os.path.exists(_OUT) and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC):
        return _OUT
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", _OUT + ".tmp",
           _SRC]
    if platform.machine() in ("x86_64", "AMD64"):
        cmd.append("-lquadmath")
    subprocess.run(cmd, check=True)
    os.replace(_OUT + ".tmp", _OUT)
    return _OUT


class _Geom(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double),
                ("lx", C.c_double), ("ly", C.c_double), ("ndir", C.c_int),
                ("mu", C.POINTER(C.c_double)), ("cos_phi", C.POINTER(C.c_double)),
                ("sin_phi", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double)),
                ("spacing", C.c_double), ("layout", C.c_int), ("renorm", C.c_int)]


class _ErrModel(C.Structure):
    _fields_ = [("path", C.c_int), ("u", C.c_double), ("e_exp", C.c_double), ("e_rcp", C.c_double),
                ("k_sum", C.c_double), ("abs_unit", C.c_double), ("Bref", C.POINTER(C.c_double))]


def _load():
    """The oracle library: the one build() makes, or the prebuilt library named by MOLC_ORACLE_LIB (the mutation
    test loads copies of the oracle with a planted mistake this way, in subprocesses of its own)."""
    global _lib
    if _lib is None:
        lib = C.CDLL(os.environ.get("MOLC_ORACLE_LIB") or build())
        i64p = C.POINTER(C.c_int64)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lib.oracle_count.argtypes = [C.POINTER(_Geom), i64p]
        lib.oracle_tracks.argtypes = [C.POINTER(_Geom), C.c_int, i64p, i64p, dp, ip, ip, dp, dp, ip]
        lib.oracle_sweep.argtypes = [C.POINTER(_Geom), C.c_int, C.c_int, dp, dp, C.c_double, C.c_double, dp, dp,
                                     ip, C.c_int, dp, dp, dp, C.c_int, C.c_int, C.c_int, dp, C.POINTER(_ErrModel),
                                     dp, dp, dp]
        for f in (lib.oracle_count, lib.oracle_tracks, lib.oracle_sweep):
            f.restype = C.c_int
        lib.oracle_real_bits.argtypes = [C.c_int]
        lib.oracle_real_bits.restype = C.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


@dataclass
class Geometry:
    """Material grid, angular quadrature and characteristic-grid rule (Sec. 3; readings c4, c9)."""
    nx: int
    ny: int
    lx: float
    ly: float
    mu: np.ndarray
    cos_phi: np.ndarray
    sin_phi: np.ndarray
    w: np.ndarray
    spacing: float
    layout: int = 0          # 0 uniform parallel rays, 1 the paper's vertex bands halved to <= spacing
    renorm: int = 1
    x0: float = 0.0
    y0: float = 0.0

    def _c(self):
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (self.mu, self.cos_phi, self.sin_phi,
                                                                            self.w)]
        return _Geom(self.nx, self.ny, self.x0, self.y0, self.lx, self.ly, int(self.mu.size),
                     *[_dp(a) for a in self._keep], self.spacing, self.layout, self.renorm)

    @property
    def ncell(self) -> int:
        return self.nx * self.ny

    @classmethod
    def from_workload(cls, wl, quad=None, spacing=None, layout=0, renorm=1):
        q = quad if quad is not None else wl.quadrature()
        return cls(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w,
                   wl.spacing if spacing is None else spacing, layout, renorm)


def counts(geom: Geometry):
    """(characteristics, segments) of the characteristic grid of Sec. 3, both summed over directions."""
    lib = _load()
    g = geom._c()
    out = np.zeros(2, dtype=np.int64)
    rc = lib.oracle_count(C.byref(g), out.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc:
        raise RuntimeError(f"oracle_count failed ({rc})")
    return int(out[0]), int(out[1])


def tracks(geom: Geometry, precision: str = "quad") -> dict:
    """The characteristic grid of Sec. 3 in canonical order (direction, characteristic by offset, segment)."""
    lib = _load()
    nr, ns = counts(geom)
    g = geom._c()
    d = dict(dir_ray_off=np.zeros(geom.mu.size + 1, np.int64), ray_seg_off=np.zeros(nr + 1, np.int64),
             width=np.zeros(nr), entry=np.zeros(nr, np.int32), cell=np.zeros(ns, np.int32), len=np.zeros(ns),
             area=np.zeros(ns), face=np.zeros(ns, np.int32))
    i64 = C.POINTER(C.c_int64)
    ip = C.POINTER(C.c_int)
    rc = lib.oracle_tracks(C.byref(g), PREC[precision], d["dir_ray_off"].ctypes.data_as(i64),
                           d["ray_seg_off"].ctypes.data_as(i64), _dp(d["width"]), d["entry"].ctypes.data_as(ip),
                           d["cell"].ctypes.data_as(ip), _dp(d["len"]), _dp(d["area"]), d["face"].ctypes.data_as(ip))
    if rc:
        raise RuntimeError(f"oracle_tracks failed ({rc})")
    return d


FACE_MOMENTS = ("face_E", "face_Fx", "face_Fy", "face_Nxx", "face_Nxy", "face_Nyy")


def n_faces(geom: Geometry) -> int:
    """Faces of the material grid that carry the face moments of Eq. 16: x-faces (nx + 1) ny, then y-faces
    nx (ny + 1)."""
    return (geom.nx + 1) * geom.ny + geom.nx * (geom.ny + 1)


BOUND_NAMES = ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy")


def sweep(geom: Geometry, kappa, B, c, dt, bnd, I_prev=None, groups=None, precision: str = "quad",
          want_I=True, want_exit=False, threads=None, I_as_deviation=False, I_prev_is_deviation=False,
          want_faces=False, errmodel=None, I_err=None) -> dict:
    """One backward-Euler sweep (Sec. 3: Eqs. 11-13 along every characteristic, Eqs. 14-15 and the Sec. 2
    moment definitions per cell).  kappa, B: [G][ncell]; bnd: [4][G]; I_prev: canonical [nseg][Gsub] or None
    (I^{n-1} = B of the segment's cell); with I_prev_is_deviation, I_prev holds deviations from B of the
    segment's cell (so a state carried between steps as deviations keeps its precision).  Returns the cell
    moments as [Gsub][ncell] arrays keyed by name,
    plus 'I' (canonical [nseg][Gsub] segment averages, or their deviations from the cell's B formed in the
    oracle's precision when I_as_deviation) and 'I_exit' ([nrays][Gsub]) when asked.

    errmodel: {path: 0 (all operations in one precision) or 1 (FP32 with approximate 2^x and 1/x), u, e_exp,
    e_rcp, k_sum, abs_unit, Bref (optional [G][ncell])} describes the arithmetic of a path that evaluates Eq. 12 in the
    deviation form; the sweep then also returns 'bound' (the first-order bound of that path's error in E, Fx, Fy,
    Nxx, Nxy, Nyy, [Gsub][ncell] each), 'dev' and 'plk' (the magnitudes of their deviation and Planck terms) and
    'I_err' (the bound of the path's stored deviations, canonical [nseg][Gsub]).  I_err: the bound of the stored
    deviations entering this step (from the previous step's 'I_err'), or None for an exact state."""
    lib = _load()
    kappa = np.ascontiguousarray(kappa, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    bnd = np.ascontiguousarray(bnd, dtype=np.float64)
    G = kappa.shape[0]
    assert kappa.shape == (G, geom.ncell) and B.shape == kappa.shape and bnd.shape == (4, G)
    gl = None
    if groups is not None:
        gl = np.ascontiguousarray(groups, dtype=np.int32)
    Gsub = G if gl is None else gl.size
    nr, ns = counts(geom)
    if I_prev is not None:
        I_prev = np.ascontiguousarray(I_prev, dtype=np.float64)
        assert I_prev.shape == (ns, Gsub)
    out = np.zeros((len(MOMENTS), Gsub, geom.ncell))
    I_new = np.zeros((ns, Gsub)) if want_I else None
    I_exit = np.zeros((nr, Gsub)) if want_exit else None
    fout = np.zeros((6, Gsub, n_faces(geom))) if want_faces else None
    em = err_out = Ierr_new = Bref = None
    if errmodel is not None:
        if errmodel.get("Bref") is not None:
            Bref = np.ascontiguousarray(errmodel["Bref"], dtype=np.float64)
            assert Bref.shape == B.shape
        em = _ErrModel(int(errmodel["path"]), float(errmodel["u"]), float(errmodel["e_exp"]),
                       float(errmodel.get("e_rcp", 0.0)), float(errmodel.get("k_sum", 0.0)),
                       float(errmodel.get("abs_unit", 0.0)), _dp(Bref))
        err_out = np.zeros((18, Gsub, geom.ncell))
        Ierr_new = np.zeros((ns, Gsub))
        if I_err is not None:
            I_err = np.ascontiguousarray(I_err, dtype=np.float64)
            assert I_err.shape == (ns, Gsub)
    g = geom._c()
    nthreads = threads or max(1, min(os.cpu_count() or 1, 64))
    rc = lib.oracle_sweep(C.byref(g), PREC[precision], G, _dp(kappa), _dp(B), float(c), float(dt), _dp(bnd),
                          _dp(I_prev), gl.ctypes.data_as(C.POINTER(C.c_int)) if gl is not None else None,
                          0 if gl is None else int(gl.size), _dp(out), _dp(I_new), _dp(I_exit), int(nthreads),
                          int(bool(I_as_deviation)), int(bool(I_prev_is_deviation)), _dp(fout),
                          C.byref(em) if em is not None else None, _dp(I_err if em is not None else None),
                          _dp(Ierr_new), _dp(err_out))
    if rc:
        raise RuntimeError(f"oracle_sweep failed ({rc})")
    res = {k: out[i] for i, k in enumerate(MOMENTS)}
    if em is not None:
        res["bound"] = {k: err_out[i] for i, k in enumerate(BOUND_NAMES)}
        res["dev"] = {k: err_out[6 + i] for i, k in enumerate(BOUND_NAMES)}
        res["plk"] = {k: err_out[12 + i] for i, k in enumerate(BOUND_NAMES)}
        res["I_err"] = Ierr_new
    if want_I:
        res["I"] = I_new
    if want_exit:
        res["I_exit"] = I_exit
    if want_faces:
        res.update({k: fout[i] for i, k in enumerate(FACE_MOMENTS)})
    return res


def closure(E, Nxx, Nxy, Nyy, c):
    """Eddington factors f = N / (c E) (Eq. 7 / Eq. 15); f_zz = 1 - f_xx - f_yy."""
    cE = c * np.asarray(E)
    fxx = np.asarray(Nxx) / cE
    fxy = np.asarray(Nxy) / cE
    fyy = np.asarray(Nyy) / cE
    return fxx, fxy, fyy


def grey_eddington(E, Nxx, Nxy, Nyy, c):
    """The E-weighted spectral average of the Eddington factors, <f>_E = sum_g f_g E_g / sum_g E_g (Sec. 2, Eq. 8
    with u = f), from [G][ncell] arrays; f_g = N_g / (c E_g) per group (0 where E_g = 0), and the average is 0
    where sum_g E_g = 0.  Returns (xx, xy, yy), each [ncell]."""
    E = np.asarray(E, dtype=np.float64)
    pos = E > 0
    se = E.sum(0)
    out = []
    for N in (Nxx, Nxy, Nyy):
        f = np.where(pos, np.asarray(N, dtype=np.float64) / np.where(pos, c * E, 1.0), 0.0)
        out.append(np.where(se > 0, (f * E).sum(0) / np.where(se > 0, se, 1.0), 0.0))
    return tuple(out)


def real_bits(precision: str) -> int:
    """Bits of the oracle's real type for a precision name (bookkeeping)."""
    return _load().oracle_real_bits(PREC[precision])


def grey_coefficients(E, Fx, Fy, kappa, B):
    """Spectrum averages of the effective grey problem (Sec. 2, Eqs. 8-9) per cell, from [G][ncell] arrays:
    <kappa>_E = sum kappa E / sum E, <kappa>_B = sum kappa B / sum B, K_R = diag(<kappa>_|Fx|, <kappa>_|Fy|)
    with <u>_|F| = sum u |F| / sum |F|, and eta = sum (kappa - K_R) F / sum E.  Zero where a denominator is zero."""
    E, Fx, Fy, kappa, B = (np.asarray(a, dtype=np.float64) for a in (E, Fx, Fy, kappa, B))

    def avg(w):
        den = w.sum(0)
        return np.where(den > 0, (kappa * w).sum(0) / np.where(den > 0, den, 1.0), 0.0)

    kE, kB, kx, ky = avg(E), avg(B), avg(np.abs(Fx)), avg(np.abs(Fy))
    se = E.sum(0)
    safe = np.where(se > 0, se, 1.0)
    ex = np.where(se > 0, ((kappa - kx) * Fx).sum(0) / safe, 0.0)
    ey = np.where(se > 0, ((kappa - ky) * Fy).sum(0) / safe, 0.0)
    return dict(kappa_E=kE, kappa_B=kB, KRx=kx, KRy=ky, eta_x=ex, eta_y=ey)

