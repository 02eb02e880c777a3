"""Thin Python binding of libmolc (include/molc.h): argument marshalling only.

Every step of the sweep runs in the library's CUDA kernels; PyTorch supplies device memory and the current
stream.  There is no fallback: if the compiled library cannot be loaded, importing raises.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

FP64, FP32 = 0, 1
RAYS_UNIFORM, RAYS_PAPER = 0, 1
AREA_RENORM = 1
HOST_ONLY = 2
AUTOTUNE = 4
FACES = 8
BALANCE = 16
TILED = 32
PREC = {"fp64": FP64, "fp32": FP32, FP64: FP64, FP32: FP32}
LAYOUT = {"uniform": RAYS_UNIFORM, "paper": RAYS_PAPER, RAYS_UNIFORM: RAYS_UNIFORM, RAYS_PAPER: RAYS_PAPER}
STATUS = {0: "MOLC_OK", 1: "MOLC_ERR_INVALID_ARG", 2: "MOLC_ERR_OUT_OF_MEMORY", 3: "MOLC_ERR_CUDA",
          4: "MOLC_ERR_NONFINITE_INPUT", 5: "MOLC_ERR_TIMEOUT", 6: "MOLC_ERR_INTERNAL", 7: "MOLC_ERR_RANGE"}
MOMENTS = ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy")

# every symbol include/molc.h declares
EXPORTED = ("molc_quadrature_product", "molc_create", "molc_plan_get_info", "molc_intensity_count",
            "molc_intensity_bytes", "molc_intensity_init", "molc_sweep", "molc_closure", "molc_intensity_export",
            "molc_intensity_import", "molc_tracks_export", "molc_kernel_timing", "molc_kernel_time",
            "molc_device_status", "molc_last_error", "molc_destroy", "molc_sweep_static_scratch",
            "molc_kernel_time_parts", "molc_batch_create", "molc_batch_bind", "molc_batch_sweep",
            "molc_batch_destroy", "molc_grey_coefficients", "molc_face_moments", "molc_sweep_closure",
            "molc_ray_balance", "molc_fp64_fma_rate", "molc_plan_retile", "molc_tune_cache")


class MolcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("x0", C.c_double), ("y0", C.c_double), ("lx", C.c_double),
                ("ly", C.c_double)]


class _Quad(C.Structure):
    _fields_ = [("n", C.c_int), ("mu", C.POINTER(C.c_double)), ("cos_phi", C.POINTER(C.c_double)),
                ("sin_phi", C.POINTER(C.c_double)), ("w", C.POINTER(C.c_double))]


class _Groups(C.Structure):
    _fields_ = [("G", C.c_int), ("edges", C.POINTER(C.c_double))]


class _Moments(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in MOMENTS]


class _Info(C.Structure):
    _fields_ = [("G", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("n_dir", C.c_int), ("n_azim_pairs", C.c_int),
                ("n_polar", C.c_int), ("n_tracks", C.c_int64), ("n_track_segments", C.c_int64),
                ("n_segments", C.c_int64), ("n_updates", C.c_int64), ("fp32_groups_per_warp", C.c_int),
                ("device_bytes", C.c_size_t), ("fp32_sweep_depth", C.c_int), ("n_faces", C.c_int),
                ("n_split_cells", C.c_int), ("fp32_tile_cells", C.c_int), ("fp32_tile_groups", C.c_int),
                ("fp32_tile_items", C.c_int), ("fp32_sweep_blocks", C.c_int), ("fp32_block_threads", C.c_int),
                ("tuned_from_cache", C.c_int)]


class _TileConfig(C.Structure):
    _fields_ = [("tile_cells", C.c_int), ("tile_groups", C.c_int), ("block_threads", C.c_int)]


class _SweepArgs(C.Structure):
    _fields_ = [("kappa", C.c_void_p), ("B", C.c_void_p), ("c", C.c_double), ("dt", C.c_double),
                ("I", C.c_void_p), ("bnd", C.c_void_p), ("out", _Moments), ("fxx", C.c_void_p),
                ("fxy", C.c_void_p), ("fyy", C.c_void_p)]


_lib = None


def load(build_if_needed: bool = True):
    """Load libmolc.so (building it first when the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_needed else _build.LIB
    if not os.path.exists(path):
        raise OSError(f"libmolc is not built ({path}); run paper_2305_11998_gb300.build.build()")
    lib = C.CDLL(path)
    dp, vp, i64p, ip = C.POINTER(C.c_double), C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int)
    sig = {
        "molc_quadrature_product": (C.c_int, [C.c_int, C.c_int, dp, dp, dp, dp]),
        "molc_create": (C.c_int, [C.POINTER(_Grid), C.POINTER(_Quad), C.POINTER(_Groups), C.c_double, C.c_int,
                                  C.c_uint, C.POINTER(vp)]),
        "molc_plan_get_info": (C.c_int, [vp, C.POINTER(_Info)]),
        "molc_intensity_count": (C.c_int64, [vp]),
        "molc_intensity_bytes": (C.c_size_t, [vp, C.c_int]),
        "molc_intensity_init": (C.c_int, [vp, C.c_int, vp, vp, vp]),
        "molc_sweep": (C.c_int, [vp, C.c_int, vp, vp, C.c_double, C.c_double, vp, vp, C.POINTER(_Moments), vp]),
        "molc_sweep_static_scratch": (C.c_int, [vp, C.c_int, vp, vp, C.c_double, C.c_double, vp, vp,
                                                C.POINTER(_Moments), vp]),
        "molc_closure": (C.c_int, [vp, C.POINTER(_Moments), C.c_double, vp, vp, vp, vp, vp]),
        "molc_ray_balance": (C.c_int, [vp, dp]),
        "molc_sweep_closure": (C.c_int, [vp, C.c_int, vp, vp, C.c_double, C.c_double, vp, vp, C.POINTER(_Moments),
                                         vp, vp, vp, vp]),
        "molc_grey_coefficients": (C.c_int, [vp, C.POINTER(_Moments), vp, vp, vp, vp]),
        "molc_face_moments": (C.c_int, [vp, C.c_int, vp, C.c_double, C.POINTER(_Moments), vp]),
        "molc_intensity_export": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_int, vp, vp]),
        "molc_intensity_import": (C.c_int, [vp, C.c_int, vp, C.c_int, C.c_int, vp, vp, vp]),
        "molc_tracks_export": (C.c_int, [vp, i64p, i64p, dp, ip, ip, dp, dp]),
        "molc_kernel_timing": (C.c_int, [vp, C.c_int]),
        "molc_kernel_time": (C.c_int, [vp, C.POINTER(C.c_double), ip]),
        "molc_kernel_time_parts": (C.c_int, [vp, C.POINTER(C.c_double), ip]),
        "molc_device_status": (C.c_int, [vp, ip]),
        "molc_fp64_fma_rate": (C.c_int, [dp]),
        "molc_plan_retile": (C.c_int, [vp, C.POINTER(_TileConfig)]),
        "molc_tune_cache": (C.c_int, [C.c_char_p, ip]),
        "molc_last_error": (C.c_char_p, []),
        "molc_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.POINTER(vp)]),
        "molc_batch_bind": (C.c_int, [vp, C.POINTER(_SweepArgs)]),
        "molc_batch_sweep": (C.c_int, [vp, vp]),
        "molc_batch_destroy": (None, [vp]),
        "molc_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != 0:
        raise MolcError(rc, load().molc_last_error().decode())


def _check_f64(t, n: int, name: str):
    if t.dtype != torch.float64 or t.numel() != n:
        raise ValueError(f"{name}: expected {n} float64 elements")


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def fp64_fma_rate() -> float:
    """molc_fp64_fma_rate: FP64 FMA throughput of the current device in FLOP/s (synchronises)."""
    r = C.c_double()
    _check(load().molc_fp64_fma_rate(C.byref(r)))
    return r.value


def tune_cache(path) -> int:
    """molc_tune_cache: use the JSON file `path` as the process-wide MOLC_AUTOTUNE cache (None: off); returns the
    number of entries read."""
    n = C.c_int(0)
    _check(load().molc_tune_cache(None if path is None else os.fsencode(path), C.byref(n)))
    return n.value


def quadrature_product(n_polar: int, n_azim: int):
    """Gauss-Legendre x Chebyshev product set from the library: (mu, cos_phi, sin_phi, w) numpy arrays."""
    n = n_polar * n_azim
    arrs = [np.zeros(n) for _ in range(4)]
    _check(load().molc_quadrature_product(n_polar, n_azim, *[_dp(a) for a in arrs]))
    return tuple(arrs)


@dataclass
class PlanInfo:
    G: int
    nx: int
    ny: int
    n_dir: int
    n_azim_pairs: int
    n_polar: int
    n_tracks: int
    n_track_segments: int
    n_segments: int
    n_updates: int
    fp32_groups_per_warp: int
    device_bytes: int
    fp32_sweep_depth: int
    n_faces: int
    n_split_cells: int
    fp32_tile_cells: int
    fp32_tile_groups: int
    fp32_tile_items: int
    fp32_sweep_blocks: int
    fp32_block_threads: int
    tuned_from_cache: int


class Plan:
    """molc_create / molc_sweep / molc_closure on torch tensors (float64, CUDA, contiguous)."""

    def __init__(self, nx, ny, lx, ly, mu, cos_phi, sin_phi, w, G, spacing, layout="uniform", renorm=True,
                 x0=0.0, y0=0.0, edges=None, host_only=False, autotune=False, faces=False, balance=False,
                 tiled=False):
        lib = load()
        self._lib = lib
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (mu, cos_phi, sin_phi, w)]
        grid = _Grid(nx, ny, x0, y0, lx, ly)
        quad = _Quad(self._keep[0].size, *[_dp(a) for a in self._keep])
        e = None if edges is None else np.ascontiguousarray(edges, dtype=np.float64)
        groups = _Groups(G, _dp(e) if e is not None else None)
        h = C.c_void_p()
        _check(lib.molc_create(C.byref(grid), C.byref(quad), C.byref(groups), float(spacing), LAYOUT[layout],
                               (AREA_RENORM if renorm else 0) | (HOST_ONLY if host_only else 0) |
                               (AUTOTUNE if autotune else 0) | (FACES if faces else 0) |
                               (BALANCE if balance else 0) | (TILED if tiled else 0), C.byref(h)))
        self._h = h
        inf = _Info()
        _check(lib.molc_plan_get_info(h, C.byref(inf)))
        self.info = PlanInfo(**{k: getattr(inf, k) for k, _ in _Info._fields_})
        self.G, self.nx, self.ny = G, nx, ny
        self.ncell = nx * ny

    @classmethod
    def from_workload(cls, wl, quad=None, spacing=None, layout="uniform", renorm=True, host_only=False,
                      autotune=False, faces=False, balance=False, tiled=False, groups=None):
        """A plan for a synth.Workload; `groups` (a range) builds it over that contiguous group range only (a shard
        of the instance: the same characteristic grid, those groups' edges)."""
        q = quad if quad is not None else wl.quadrature()
        edges = wl.edges()
        G = wl.G
        if groups is not None:
            edges = edges[groups.start: groups.stop + 1]
            G = len(groups)
        return cls(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, G,
                   wl.spacing if spacing is None else spacing, layout, renorm, edges=edges, host_only=host_only,
                   autotune=autotune, faces=faces, balance=balance, tiled=tiled)

    def retile(self, tile_cells=0, tile_groups=0, block_threads=0):
        """molc_plan_retile: re-cut the tiled FP32 sweep (FP32 states must be re-initialised afterwards)."""
        cfg = _TileConfig(int(tile_cells), int(tile_groups), int(block_threads))
        _check(self._lib.molc_plan_retile(self._h, C.byref(cfg)))
        inf = _Info()
        _check(self._lib.molc_plan_get_info(self._h, C.byref(inf)))
        self.info = PlanInfo(**{k: getattr(inf, k) for k, _ in _Info._fields_})

    def close(self):
        if getattr(self, "_h", None):
            self._lib.molc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- intensity state
    def intensity_count(self) -> int:
        return int(self._lib.molc_intensity_count(self._h))

    def intensity_bytes(self, prec) -> int:
        return int(self._lib.molc_intensity_bytes(self._h, PREC[prec]))

    def new_intensity(self, prec="fp32", device="cuda"):
        """Uninitialised device storage for the opaque intensity state (a byte tensor)."""
        return torch.empty(self.intensity_bytes(prec), dtype=torch.uint8, device=device)

    def intensity_init(self, prec, I, B, stream=None):
        self._state(prec, I)
        self._fields(B=B)
        _check(self._lib.molc_intensity_init(self._h, PREC[prec], _ptr(I), _ptr(B), _stream(stream)))

    def intensity_export(self, prec, I, g_begin=0, g_count=None, out=None, stream=None):
        g_count = self.G - g_begin if g_count is None else g_count
        ns = self.info.n_segments
        if out is None:
            out = torch.empty((ns, g_count), dtype=torch.float64, device=I.device)
        self._state(prec, I)
        _check_f64(out, ns * g_count, "out")
        _check(self._lib.molc_intensity_export(self._h, PREC[prec], _ptr(I), g_begin, g_count, _ptr(out),
                                               _stream(stream)))
        return out

    def intensity_import(self, prec, I, canon, B, g_begin=0, stream=None):
        g_count = canon.shape[1]
        self._state(prec, I)
        self._fields(B=B)
        _check_f64(canon, self.info.n_segments * g_count, "canon")
        _check(self._lib.molc_intensity_import(self._h, PREC[prec], _ptr(I), g_begin, g_count, _ptr(canon),
                                               _ptr(B), _stream(stream)))

    # ---- argument checks (sizes and types of the tensors whose raw pointers cross the C ABI; a mismatch is
    # rejected here, before any kernel could read or write past a buffer)
    def _fields(self, kappa=None, B=None, bnd=None):
        n = self.G * self.ncell
        if kappa is not None:
            _check_f64(kappa, n, "kappa")
        if B is not None:
            _check_f64(B, n, "B")
        if bnd is not None:
            _check_f64(bnd, 4 * self.G, "bnd")

    def _state(self, prec, I):
        if I.numel() * I.element_size() < self.intensity_bytes(prec):
            raise ValueError(f"I: needs {self.intensity_bytes(prec)} bytes for {prec}")

    def _moments(self, m, per=None):
        n = self.G * (self.ncell if per is None else per)
        for k in MOMENTS:
            _check_f64(m[k], n, k)
        return _Moments(*[_ptr(m[k]).value for k in MOMENTS])

    # ---- the sweep
    def new_moments(self, device="cuda"):
        return {k: torch.empty((self.G, self.ncell), dtype=torch.float64, device=device) for k in MOMENTS}

    def sweep(self, prec, kappa, B, c, dt, I, bnd, out=None, stream=None):
        out = out if out is not None else self.new_moments(kappa.device)
        self._fields(kappa, B, bnd)
        self._state(prec, I)
        m = self._moments(out)
        _check(self._lib.molc_sweep(self._h, PREC[prec], _ptr(kappa), _ptr(B), float(c), float(dt), _ptr(I),
                                    _ptr(bnd), C.byref(m), _stream(stream)))
        return out

    def sweep_closure(self, prec, kappa, B, c, dt, I, bnd, out=None, f=None, stream=None):
        """molc_sweep_closure: one step and its Eddington factors in one call; returns (moments, factors), the
        factors {fxx, fxy, fyy} ([G][ncell] each, written into `f` when given)."""
        out = out if out is not None else self.new_moments(kappa.device)
        f = f if f is not None else {k: torch.empty((self.G, self.ncell), dtype=torch.float64, device=kappa.device)
                                     for k in ("fxx", "fxy", "fyy")}
        for k in ("fxx", "fxy", "fyy"):
            _check_f64(f[k], self.G * self.ncell, k)
        self._fields(kappa, B, bnd)
        self._state(prec, I)
        m = self._moments(out)
        _check(self._lib.molc_sweep_closure(self._h, PREC[prec], _ptr(kappa), _ptr(B), float(c), float(dt), _ptr(I),
                                            _ptr(bnd), C.byref(m), _ptr(f["fxx"]), _ptr(f["fxy"]), _ptr(f["fyy"]),
                                            _stream(stream)))
        return out, f

    def sweep_static_scratch(self, prec, kappa, B, c, dt, I, bnd, out=None, stream=None):
        """molc_sweep_static_scratch: as sweep(), with the workspace taken from the library's fixed device array
        (no device allocation by the library; plans up to its size limit only; calls that overlap in time on
        one device race).  `out` is allocated here by torch when not given: pass it for a call that allocates
        nothing at all."""
        out = out if out is not None else self.new_moments(kappa.device)
        self._fields(kappa, B, bnd)
        self._state(prec, I)
        m = self._moments(out)
        _check(self._lib.molc_sweep_static_scratch(self._h, PREC[prec], _ptr(kappa), _ptr(B), float(c), float(dt),
                                                   _ptr(I), _ptr(bnd), C.byref(m), _stream(stream)))
        return out

    def closure(self, moments, c, grey=False, stream=None, out=None):
        """molc_closure: {fxx, fxy, fyy} ([G][ncell] each, written into `out` when given) and, with grey, the
        E-weighted spectral averages [3][ncell]."""
        f = out if out is not None else {
            k: torch.empty((self.G, self.ncell), dtype=torch.float64, device=moments["E"].device)
            for k in ("fxx", "fxy", "fyy")}
        for k in ("fxx", "fxy", "fyy"):
            _check_f64(f[k], self.G * self.ncell, k)
        fg = torch.empty((3, self.ncell), dtype=torch.float64, device=moments["E"].device) if grey else None
        m = self._moments(moments)
        _check(self._lib.molc_closure(self._h, C.byref(m), float(c), _ptr(f["fxx"]), _ptr(f["fxy"]),
                                      _ptr(f["fyy"]), _ptr(fg), _stream(stream)))
        if grey:
            f["grey"] = fg
        return f

    def face_moments(self, prec, I, c, stream=None):
        """molc_face_moments: {E, Fx, Fy, Nxx, Nxy, Nyy} of the faces, each [G][n_faces], of the last sweep."""
        nf = self.info.n_faces
        out = {k: torch.empty((self.G, nf), dtype=torch.float64, device=I.device) for k in MOMENTS}
        self._state(prec, I)
        m = self._moments(out, per=nf)
        _check(self._lib.molc_face_moments(self._h, PREC[prec], _ptr(I), float(c), C.byref(m), _stream(stream)))
        return out

    GREY = ("kappa_E", "kappa_B", "KRx", "KRy", "eta_x", "eta_y")

    def grey_coefficients(self, moments, kappa, B, stream=None):
        """molc_grey_coefficients: {name: [cell] tensor} for kappa_E, kappa_B, KRx, KRy, eta_x, eta_y."""
        out = torch.empty((6, self.ncell), dtype=torch.float64, device=kappa.device)
        self._fields(kappa, B)
        m = self._moments(moments)
        _check(self._lib.molc_grey_coefficients(self._h, C.byref(m), _ptr(kappa), _ptr(B), _ptr(out),
                                                _stream(stream)))
        return dict(zip(self.GREY, out))

    def ray_balance(self) -> float:
        """molc_ray_balance: the largest per-ray relative balance residual of the last sweep (plans created with
        balance=True; synchronises)."""
        r = C.c_double()
        _check(self._lib.molc_ray_balance(self._h, C.byref(r)))
        return r.value

    def kernel_timing(self, enable: bool = True):
        _check(self._lib.molc_kernel_timing(self._h, int(enable)))

    def kernel_time(self):
        """(summed milliseconds, launches) of the sweep kernels timed since the last call."""
        ms = C.c_double()
        n = C.c_int()
        _check(self._lib.molc_kernel_time(self._h, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def kernel_time_parts(self):
        """({"prep", "sweep", "moments"} summed milliseconds, timed calls) since the last call."""
        ms = (C.c_double * 3)()
        n = C.c_int()
        _check(self._lib.molc_kernel_time_parts(self._h, ms, C.byref(n)))
        return dict(zip(("prep", "sweep", "moments"), list(ms))), n.value

    def device_status(self) -> int:
        code = C.c_int()
        _check(self._lib.molc_device_status(self._h, C.byref(code)))
        return code.value

    def tracks(self) -> dict:
        nr = 2 * self.info.n_polar * self.info.n_tracks
        ns = self.info.n_segments
        d = dict(dir_ray_off=np.zeros(self.info.n_dir + 1, np.int64), ray_seg_off=np.zeros(nr + 1, np.int64),
                 width=np.zeros(nr), entry=np.zeros(nr, np.int32), cell=np.zeros(ns, np.int32), len=np.zeros(ns),
                 area=np.zeros(ns))
        i64 = C.POINTER(C.c_int64)
        ip = C.POINTER(C.c_int)
        _check(self._lib.molc_tracks_export(self._h, d["dir_ray_off"].ctypes.data_as(i64),
                                            d["ray_seg_off"].ctypes.data_as(i64), _dp(d["width"]),
                                            d["entry"].ctypes.data_as(ip), d["cell"].ctypes.data_as(ip),
                                            _dp(d["len"]), _dp(d["area"])))
        return d


class Batch:
    """molc_batch_*: one batched FP32 step over many plans (instances) on one device."""

    def __init__(self, plans):
        self._lib = load()
        self.plans = list(plans)
        arr = (C.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        h = C.c_void_p()
        _check(self._lib.molc_batch_create(arr, len(self.plans), C.byref(h)))
        self._h = h
        self._args = None

    def bind(self, args):
        """args: one dict per instance with kappa, B, c, dt, I, bnd, out (moments dict) and optionally f
        (dict fxx, fxy, fyy)."""
        arr = (_SweepArgs * len(self.plans))()
        if len(args) != len(self.plans):
            raise ValueError(f"bind: need {len(self.plans)} argument sets")
        for i, (a, P) in enumerate(zip(args, self.plans)):
            f = a.get("f")
            P._fields(a["kappa"], a["B"], a["bnd"])
            P._state("fp32", a["I"])
            m = P._moments(a["out"])
            if f:
                for k in ("fxx", "fxy", "fyy"):
                    _check_f64(f[k], P.G * P.ncell, k)
            arr[i] = _SweepArgs(_ptr(a["kappa"]), _ptr(a["B"]), float(a["c"]), float(a["dt"]), _ptr(a["I"]),
                                _ptr(a["bnd"]), m,
                                *([_ptr(f["fxx"]), _ptr(f["fxy"]), _ptr(f["fyy"])] if f else [None] * 3))
        _check(self._lib.molc_batch_bind(self._h, arr))
        self._args = args     # keep the tensors alive while bound

    def sweep(self, stream=None):
        _check(self._lib.molc_batch_sweep(self._h, _stream(stream)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.molc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

