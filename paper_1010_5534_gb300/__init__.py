"""Python binding of the GB300 adaptive image ray-tracing (AIR) library.

Thin ctypes layer over the C ABI in include/air.h: it marshals arguments,
allocates outputs (torch device tensors, or pinned host tensors) and passes
torch's current CUDA stream. Every step of the method runs in the library's
CUDA kernels; there is no fallback. If the shared library is missing, calls
raise RuntimeError.

Method: E. R. Parkin (2010), "Adaptive image ray-tracing for astrophysical
simulations", Section 2 (the AIR steps) and Section 3 (Eq. 1, Eq. 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_HERE, "libair_gb300.so")
SOURCES = ["air_api.cu", "air_grid.cu", "air_march.cu", "air_refine.cu", "air_static.cu",
           "air_batch.cu", "air_mlp.cu", "air_learned.cu", "air_tune.cu", "air_raster.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden"]

AIR_OK, AIR_ERR_ARG, AIR_ERR_OOM, AIR_ERR_CUDA, AIR_ERR_CAPACITY, AIR_ERR_TIMEOUT, \
    AIR_ERR_NUMERIC = range(7)
AIR_HOST, AIR_DEVICE = 0, 1
RASTER_MODES = {"nearest": 0, "bilinear": 1}
RASTER_QUANTITIES = {"I": 0, "p": 1, "N": 2}

EXPORTED = ["air_load_grid", "air_set_stream", "air_render_fixed", "air_render_adaptive",
            "air_render_batch", "air_mlp_create", "air_mlp_set_stream", "air_mlp_params",
            "air_mlp_forward", "air_mlp_loss_grad", "air_mlp_train", "air_mlp_free",
            "air_learn_samples", "air_render_learned", "air_autotune", "air_set_tuning",
            "air_get_tuning",
            "air_profile_enable", "air_profile_read", "air_band_flux_static", "air_render_raster",
            "air_render_adaptive_spectra", "air_render_adaptive_sharded",
            "air_render_batch_learned",
            "air_free",
            "air_last_error", "air_version"]
PHASES = ("march", "scan", "balance", "refine", "output", "batch", "learn")


def _nvcc():
    for c in ("/usr/local/cuda/bin/nvcc", "nvcc"):
        if os.path.sep not in c or os.path.exists(c):
            return c
    return "nvcc"


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a (one nvcc per translation unit, in
    parallel) and link paper_1010_5534_gb300/libair_gb300.so."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith(".cuh")] + \
        [os.path.join(_HERE, "..", "include", "air.h")]
    newest = max(os.path.getmtime(p) for p in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()
    procs, objs = [], []
    for s in srcs:
        o = os.path.join(_BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        cmd = [nvcc, *NVCC_FLAGS, "-c", s, "-o", o]
        if verbose:
            print(" ".join(cmd))
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{out.decode(errors='replace')}")
        if verbose and out:
            print(out.decode(errors="replace"))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp, *objs]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout.decode(errors='replace')}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ---------------------------------------------------------------- structures
class GridDesc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("brick", C.c_int32), ("max_level", C.c_int32),
                ("n_bricks", C.c_int32), ("brick_level", C.c_void_p),
                ("brick_origin", C.c_void_p), ("field_dtype", C.c_int32), ("rho", C.c_void_p),
                ("temp", C.c_void_p), ("n_bands", C.c_int32), ("emis_mode", C.c_int32),
                ("lambda_table", C.c_void_p), ("n_tbins", C.c_int32), ("logT_lo", C.c_double),
                ("logT_hi", C.c_double), ("kappa", C.c_void_p)]


class View(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("up", C.c_double * 3), ("center", C.c_double * 3),
                ("half_extent", C.c_double)]


class Params(C.Structure):
    _fields_ = [("base_res", C.c_int32), ("max_level", C.c_int32), ("xi_crit", C.c_double),
                ("xi_norm", C.c_int32), ("refine_on", C.c_int32), ("fp64_level", C.c_int32),
                ("include_interior", C.c_int32)]


EXCHANGE_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p,
                          C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p)


class Shard(C.Structure):
    _fields_ = [("rank", C.c_int32), ("world", C.c_int32), ("exchange", EXCHANGE_FN),
                ("user", C.c_void_p)]


class _DeviceArray:
    """A view of library-owned device memory for torch.as_tensor (CUDA array
    interface, no copy)."""

    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


class BatchOpts(C.Structure):
    _fields_ = [("bands_per_thread", C.c_int32), ("use_graph", C.c_int32),
                ("wait_timeout_ms", C.c_double), ("test_stall_barrier", C.c_int32)]


class Tuning(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("bands_per_thread", C.c_int32),
                ("batch_bands_per_thread", C.c_int32), ("batch_blocks_per_sm", C.c_int32),
                ("best_ms", C.c_double * 3), ("trials", C.c_int32)]


class LearnedOpts(C.Structure):
    _fields_ = [("quantile", C.c_double)]


class LearnedStats(C.Structure):
    _fields_ = [("proposed_rays", C.c_int64), ("used_rays", C.c_int64),
                ("wasted_rays", C.c_int64), ("fallback_rays", C.c_int64), ("waves", C.c_int32),
                ("sweeps", C.c_int32), ("under_predicted", C.c_int64),
                ("over_predicted", C.c_int64)]


class Image(C.Structure):
    _fields_ = [("mem", C.c_int32), ("capacity", C.c_int64), ("n_out", C.c_int64),
                ("n_leaves", C.c_int64), ("n_rays", C.c_int64), ("n_steps", C.c_int64),
                ("n_sweeps", C.c_int32), ("level", C.c_void_p), ("i", C.c_void_p),
                ("j", C.c_void_p), ("is_leaf", C.c_void_p), ("coldens", C.c_void_p),
                ("intensity", C.c_void_p), ("p", C.c_void_p), ("band_flux", C.c_void_p)]


_lib = None
_lock = threading.Lock()


def lib():
    """The loaded C library. Raises RuntimeError if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "paper_1010_5534_gb300.build() (nvcc, sm_103a)")
            L = C.CDLL(LIB_PATH)
            L.air_load_grid.restype = C.c_int
            L.air_load_grid.argtypes = [C.POINTER(GridDesc), C.c_void_p, C.POINTER(C.c_void_p)]
            L.air_set_stream.restype = C.c_int
            L.air_set_stream.argtypes = [C.c_void_p, C.c_void_p]
            L.air_render_fixed.restype = C.c_int
            L.air_render_fixed.argtypes = [C.c_void_p, C.POINTER(View), C.c_int32, C.c_int32,
                                           C.POINTER(Image)]
            L.air_render_adaptive.restype = C.c_int
            L.air_render_adaptive.argtypes = [C.c_void_p, C.POINTER(View), C.POINTER(Params),
                                              C.POINTER(Image)]
            L.air_render_batch.restype = C.c_int
            L.air_render_batch.argtypes = [C.c_void_p, C.POINTER(View), C.c_int32,
                                           C.POINTER(Params), C.POINTER(BatchOpts),
                                           C.POINTER(Image)]
            L.air_mlp_create.restype = C.c_int
            L.air_mlp_create.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
            L.air_mlp_set_stream.restype = C.c_int
            L.air_mlp_set_stream.argtypes = [C.c_void_p, C.c_void_p]
            L.air_mlp_params.restype = C.c_int
            L.air_mlp_params.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.air_mlp_forward.restype = C.c_int
            L.air_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
            L.air_mlp_loss_grad.restype = C.c_int
            L.air_mlp_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                                            C.c_void_p, C.POINTER(C.c_double)]
            L.air_mlp_train.restype = C.c_int
            L.air_mlp_train.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                        C.c_int32, C.c_float, C.c_void_p]
            L.air_mlp_free.restype = None
            L.air_mlp_free.argtypes = [C.c_void_p]
            L.air_learn_samples.restype = C.c_int
            L.air_learn_samples.argtypes = [C.c_void_p, C.POINTER(View), C.POINTER(Params),
                                            C.c_void_p, C.c_void_p]
            L.air_render_learned.restype = C.c_int
            L.air_render_learned.argtypes = [C.c_void_p, C.POINTER(View), C.POINTER(Params),
                                             C.c_void_p, C.POINTER(LearnedOpts), C.POINTER(Image),
                                             C.POINTER(LearnedStats)]
            L.air_autotune.restype = C.c_int
            L.air_autotune.argtypes = [C.c_void_p, C.POINTER(View), C.POINTER(Params), C.c_int32,
                                       C.POINTER(Tuning)]
            L.air_set_tuning.restype = C.c_int
            L.air_set_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
            L.air_get_tuning.restype = C.c_int
            L.air_get_tuning.argtypes = [C.c_void_p, C.POINTER(Tuning)]
            L.air_profile_enable.restype = C.c_int
            L.air_profile_enable.argtypes = [C.c_void_p, C.c_int32]
            L.air_profile_read.restype = C.c_int
            L.air_profile_read.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.air_band_flux_static.restype = C.c_int
            L.air_band_flux_static.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.c_void_p,
                                               C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                               C.c_void_p]
            L.air_render_batch_learned.restype = C.c_int
            L.air_render_batch_learned.argtypes = [C.c_void_p, C.POINTER(View), C.c_int32,
                                                   C.POINTER(Params), C.POINTER(BatchOpts),
                                                   C.c_void_p, C.POINTER(LearnedOpts),
                                                   C.POINTER(Image), C.POINTER(LearnedStats)]
            L.air_render_adaptive_sharded.restype = C.c_int
            L.air_render_adaptive_sharded.argtypes = [C.c_void_p, C.POINTER(View), C.POINTER(Params),
                                                      C.POINTER(Shard), C.POINTER(Image)]
            L.air_render_adaptive_spectra.restype = C.c_int
            L.air_render_adaptive_spectra.argtypes = [C.c_void_p, C.POINTER(View), C.POINTER(Params),
                                                      C.POINTER(Image), C.c_void_p, C.c_int64]
            L.air_render_raster.restype = C.c_int
            L.air_render_raster.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                            C.c_int64]
            L.air_free.restype = None
            L.air_free.argtypes = [C.c_void_p]
            L.air_last_error.restype = C.c_char_p
            L.air_version.restype = C.c_char_p
            _lib = L
    return _lib


class AirError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"AIR error {status}: {msg}")
        self.status = status


def _check(status):
    if status != AIR_OK:
        raise AirError(status, lib().air_last_error().decode(errors="replace"))


def _view(v) -> View:
    s = View()
    s.dir[:] = [float(x) for x in v.dir]
    s.up[:] = [float(x) for x in v.up]
    s.center[:] = [float(x) for x in v.center]
    s.half_extent = float(v.half_extent)
    return s


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Grid:
    """A simulation grid resident on the GPU (air_load_grid).

    `desc` is any object with the attributes kind ("uniform" | "amr"), n, lo,
    hi, rho, and optionally temp, brick, max_level, brick_level, brick_origin,
    emis_mode, lambda_table, logT_lo, logT_hi, kappa."""

    def __init__(self, desc):
        d = GridDesc()
        keep = []
        d.kind = 0 if desc.kind == "uniform" else 1
        d.n[:] = [int(x) for x in desc.n]
        d.lo[:] = [float(x) for x in desc.lo]
        d.hi[:] = [float(x) for x in desc.hi]
        rho = np.ascontiguousarray(desc.rho)
        dt = np.float64 if rho.dtype == np.float64 else np.float32
        rho = np.ascontiguousarray(rho, dtype=dt)
        d.field_dtype = 1 if dt == np.float64 else 0
        d.rho = rho.ctypes.data
        keep.append(rho)
        if getattr(desc, "temp", None) is not None:
            t = np.ascontiguousarray(desc.temp, dtype=dt)
            d.temp = t.ctypes.data
            keep.append(t)
        if d.kind == 1:
            bl = np.ascontiguousarray(desc.brick_level, dtype=np.int32)
            bo = np.ascontiguousarray(desc.brick_origin, dtype=np.int32)
            d.brick, d.max_level, d.n_bricks = int(desc.brick), int(desc.max_level), len(bl)
            d.brick_level, d.brick_origin = bl.ctypes.data, bo.ctypes.data
            keep += [bl, bo]
        kappa = np.ascontiguousarray(desc.kappa, dtype=np.float64)
        d.n_bands = len(kappa)
        d.kappa = kappa.ctypes.data
        keep.append(kappa)
        d.emis_mode = int(getattr(desc, "emis_mode", 0))
        if d.emis_mode == 1:
            tab = np.ascontiguousarray(desc.lambda_table, dtype=np.float32)
            d.lambda_table = tab.ctypes.data
            d.n_tbins = tab.shape[1]
            d.logT_lo, d.logT_hi = float(desc.logT_lo), float(desc.logT_hi)
            keep.append(tab)
        self.n_bands = d.n_bands
        h = C.c_void_p()
        _check(lib().air_load_grid(C.byref(d), _stream(), C.byref(h)))
        self._h = h
        self._cap_hint = 0

    def close(self):
        if getattr(self, "_h", None):
            lib().air_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, view, base_res, max_level, xi_crit, n_views_batch=0, xi_norm=0,
                 refine_on=0, fp64_level=-1):
        """Time launch configurations on this grid and keep the fastest."""
        _check(lib().air_set_stream(self._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 0)
        t = Tuning()
        _check(lib().air_autotune(self._h, C.byref(_view(view)), C.byref(p), int(n_views_batch),
                                  C.byref(t)))
        return {f: (list(getattr(t, f)) if f == "best_ms" else getattr(t, f))
                for f, _ in Tuning._fields_}

    def set_tuning(self, tile_w=0, bands_per_thread=0, batch_bands_per_thread=0,
                   batch_blocks_per_sm=0):
        t = Tuning(int(tile_w), int(bands_per_thread), int(batch_bands_per_thread),
                   int(batch_blocks_per_sm))
        _check(lib().air_set_tuning(self._h, C.byref(t)))

    def profile(self, on=True):
        """Enable (and reset) or disable per-phase device timing."""
        _check(lib().air_profile_enable(self._h, 1 if on else 0))

    def profile_read(self):
        ms = np.zeros(len(PHASES))
        ln = np.zeros(len(PHASES), dtype=np.int64)
        _check(lib().air_profile_read(self._h, ms.ctypes.data, ln.ctypes.data))
        return {p: (float(ms[k]), int(ln[k])) for k, p in enumerate(PHASES)}

    # ---------------------------------------------------------- outputs
    def _alloc(self, n, mem, fields):
        import torch
        nb = self.n_bands
        cap = max(int(n), 1)
        if mem == "device":
            dev = dict(device="cuda")
        else:
            dev = dict(device="cpu", pin_memory=True)
        out = {}
        spec = dict(level=(torch.int32, (cap,)), i=(torch.int32, (cap,)), j=(torch.int32, (cap,)),
                    is_leaf=(torch.uint8, (cap,)), coldens=(torch.float32, (cap,)),
                    intensity=(torch.float32, (nb, cap)), p=(torch.float32, (cap,)),
                    band_flux=(torch.float64, (nb,)))
        for k in fields:
            dt, shp = spec[k]
            out[k] = torch.empty(shp, dtype=dt, **dev)
        im = Image()
        im.mem = AIR_DEVICE if mem == "device" else AIR_HOST
        im.capacity = cap
        for k, t in out.items():
            setattr(im, k, t.data_ptr())
        return im, out

    def alloc_image(self, capacity, mem="device", fields=None):
        """Output arrays for `capacity` nodes (a dict of tensors, page-locked for
        mem="host"), to pass as `out=` to render_adaptive call after call."""
        return self._alloc(capacity, mem, fields or self.ALL)[1]

    def _image_of(self, out, mem):
        """Image struct over caller-provided output tensors (see alloc_image)."""
        import torch
        spec = dict(level=torch.int32, i=torch.int32, j=torch.int32, is_leaf=torch.uint8,
                    coldens=torch.float32, intensity=torch.float32, p=torch.float32,
                    band_flux=torch.float64)
        on_dev = mem == "device"
        cap = None
        im = Image()
        im.mem = AIR_DEVICE if on_dev else AIR_HOST
        for k, t in out.items():
            if k not in spec or t.dtype != spec[k] or not t.is_contiguous():
                raise ValueError(f"output {k!r}: wrong name, dtype or layout")
            if t.is_cuda != on_dev:
                raise ValueError(f"output {k!r} is not in {mem} memory")
            if k == "band_flux":
                if t.numel() < self.n_bands:
                    raise ValueError("band_flux holds fewer than n_bands values")
            else:
                if k == "intensity" and (t.dim() != 2 or t.shape[0] != self.n_bands):
                    raise ValueError("intensity must be [n_bands, capacity]")
                n = t.shape[-1]
                cap = n if cap is None else min(cap, n)
            setattr(im, k, t.data_ptr())
        im.capacity = max(int(cap or 1), 1)
        return im

    @staticmethod
    def _result(im, out):
        n = im.n_out
        res = {k: (v[..., :n] if k != "band_flux" else v) for k, v in out.items()}
        res.update(n_out=im.n_out, n_leaves=im.n_leaves, n_rays=im.n_rays,
                   n_steps=im.n_steps, n_sweeps=im.n_sweeps)
        return res

    ALL = ("level", "i", "j", "is_leaf", "coldens", "intensity", "p", "band_flux")

    def render_fixed(self, view, res, fp64_level=-1, mem="device", fields=ALL):
        """Fixed res x res image (row-major)."""
        _check(lib().air_set_stream(self._h, _stream()))
        im, out = self._alloc(res * res, mem, fields)
        _check(lib().air_render_fixed(self._h, C.byref(_view(view)), int(res), int(fp64_level),
                                      C.byref(im)))
        return self._result(im, out)

    def render_batch(self, views, base_res, max_level, xi_crit, xi_norm=0, refine_on=0,
                     fp64_level=-1, include_interior=False, mem="device", fields=ALL,
                     bands_per_thread=0, use_graph=True, wait_timeout_ms=2000.0,
                     test_stall_barrier=False, capacity=None):
        """Batched adaptive images of several views in one persistent launch;
        returns one result dict per view (as render_adaptive)."""
        _check(lib().air_set_stream(self._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 1 if include_interior else 0)
        o = BatchOpts(int(bands_per_thread), 1 if use_graph else 0, float(wait_timeout_ms),
                      1 if test_stall_barrier else 0)
        hints = getattr(self, "_batch_hint", {})
        caps = [capacity or hints.get(k, 4 * base_res * base_res) for k in range(len(views))]
        st, ims, outs = _batch_call(self, views, p, o, caps, mem, fields)
        if st == AIR_ERR_CAPACITY and all(im.n_out > 0 for im in ims):
            caps = [max(int(im.n_out), 1) for im in ims]
            st, ims, outs = _batch_call(self, views, p, o, caps, mem, fields)
        self._raster_src = None
        _check(st)
        self._batch_hint = {k: int(im.n_out) for k, im in enumerate(ims)}
        return [self._result(im, out) for im, out in zip(ims, outs)]

    def render_batch_learned(self, views, base_res, max_level, xi_crit, mlp, quantile=0.8,
                             xi_norm=0, refine_on=0, fp64_level=-1, include_interior=False,
                             mem="device", fields=ALL, bands_per_thread=0, wait_timeout_ms=2000.0,
                             capacity=None):
        """air_render_batch_learned: batched images with the learned proposal;
        returns (one result dict per view, stats summed over the views)."""
        _check(lib().air_set_stream(self._h, _stream()))
        _check(lib().air_mlp_set_stream(mlp._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 1 if include_interior else 0)
        o = BatchOpts(int(bands_per_thread), 0, float(wait_timeout_ms), 0)
        lo = LearnedOpts(float(quantile))
        stats = LearnedStats()
        hints = getattr(self, "_batch_hint", {})
        caps = [capacity or hints.get(k, 4 * base_res * base_res) for k in range(len(views))]
        st, ims, outs = _batch_call(self, views, p, o, caps, mem, fields, (mlp, lo, stats))
        if st == AIR_ERR_CAPACITY and all(im.n_out > 0 for im in ims):
            caps = [max(int(im.n_out), 1) for im in ims]
            st, ims, outs = _batch_call(self, views, p, o, caps, mem, fields, (mlp, lo, stats))
        self._raster_src = None
        _check(st)
        self._batch_hint = {k: int(im.n_out) for k, im in enumerate(ims)}
        sd = {f: getattr(stats, f) for f, _ in LearnedStats._fields_}
        return [self._result(im, out) for im, out in zip(ims, outs)], sd

    def learn_samples(self, view, base_res, max_level, xi_crit, xi_norm=0, refine_on=0,
                      fp64_level=-1, labels=True):
        """(x, y): features [4 n0^2, 16] (BF16 bits as int16) and depth labels
        [4 n0^2] (int32) of one view's quadrant samples (sample 4 b + q:
        level-1 pixel q of base pixel b, row-major), on the GPU."""
        import torch
        _check(lib().air_set_stream(self._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 0)
        nb = 4 * base_res * base_res
        x = torch.empty((nb, 16), dtype=torch.int16, device="cuda")
        y = torch.empty(nb, dtype=torch.int32, device="cuda") if labels else None
        _check(lib().air_learn_samples(self._h, C.byref(_view(view)), C.byref(p),
                                       C.c_void_p(x.data_ptr()),
                                       C.c_void_p(y.data_ptr()) if y is not None else None))
        return x, y

    def render_learned(self, view, base_res, max_level, xi_crit, mlp, quantile=0.8, xi_norm=0,
                       refine_on=0, fp64_level=-1, include_interior=False, mem="device",
                       fields=ALL, capacity=None):
        """Adaptive image with the learned proposal; returns (result, stats)."""
        _check(lib().air_set_stream(self._h, _stream()))
        _check(lib().air_mlp_set_stream(mlp._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 1 if include_interior else 0)
        o = LearnedOpts(float(quantile))
        stats = LearnedStats()
        cap = capacity or max(self._cap_hint, 4 * base_res * base_res)
        im, out = self._alloc(cap, mem, fields)
        st = lib().air_render_learned(self._h, C.byref(_view(view)), C.byref(p), mlp._h,
                                      C.byref(o), C.byref(im), C.byref(stats))
        if st == AIR_ERR_CAPACITY:
            im, out = self._alloc(im.n_out, mem, fields)
            st = lib().air_render_learned(self._h, C.byref(_view(view)), C.byref(p), mlp._h,
                                          C.byref(o), C.byref(im), C.byref(stats))
        _check(st)
        self._cap_hint = max(self._cap_hint, int(im.n_out))
        self._raster_src = (int(base_res), int(max_level))
        sd = {f: getattr(stats, f) for f, _ in LearnedStats._fields_}
        return self._result(im, out), sd

    def render_adaptive(self, view, base_res, max_level, xi_crit, xi_norm=0, refine_on=0,
                        fp64_level=-1, include_interior=False, mem="device", fields=ALL,
                        capacity=None, out=None):
        """Adaptive image; leaves (or all traced nodes) in creation order. With
        `out` (from alloc_image) the image is written into those arrays; the
        call fails if they are too small."""
        _check(lib().air_set_stream(self._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 1 if include_interior else 0)
        if out is not None:
            im = self._image_of(out, mem)
            _check(lib().air_render_adaptive(self._h, C.byref(_view(view)), C.byref(p),
                                             C.byref(im)))
            self._raster_src = (int(base_res), int(max_level))
            return self._result(im, out)
        cap = capacity or max(self._cap_hint, 4 * base_res * base_res)
        im, out = self._alloc(cap, mem, fields)
        st = lib().air_render_adaptive(self._h, C.byref(_view(view)), C.byref(p), C.byref(im))
        if st == AIR_ERR_CAPACITY:
            need = im.n_out
            im, out = self._alloc(need, mem, fields)
            st = lib().air_render_adaptive(self._h, C.byref(_view(view)), C.byref(p), C.byref(im))
        _check(st)
        self._cap_hint = max(self._cap_hint, int(im.n_out))
        self._raster_src = (int(base_res), int(max_level))
        return self._result(im, out)

    def render_adaptive_sharded(self, view, base_res, max_level, xi_crit, group=None, xi_norm=0,
                                refine_on=0, fp64_level=-1, include_interior=False, mem="device",
                                fields=ALL, capacity=None):
        """air_render_adaptive_sharded over the torch.distributed group: this
        rank traces its slice of every sweep's rays, the slices are exchanged
        (shard.exchange_slices), and every rank returns the whole image."""
        import torch
        import torch.distributed as dist
        from . import shard as _shard
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        errors = []

        def exchange(user, first, count, nb, N, I, stride, p, steps):
            try:
                arrs = [torch.as_tensor(_DeviceArray(N + 4 * first, count, "<f4"), device="cuda"),
                        torch.as_tensor(_DeviceArray(p + 4 * first, count, "<f4"), device="cuda"),
                        torch.as_tensor(_DeviceArray(steps + 4 * first, count, "<i4"), device="cuda")]
                arrs += [torch.as_tensor(_DeviceArray(I + 4 * (b * stride + first), count, "<f4"),
                                         device="cuda") for b in range(nb)]
                _shard.exchange_slices(arrs, rank, world, group)
                torch.cuda.current_stream().synchronize()
                return 0
            except Exception as e:  # reported after the call returns
                errors.append(e)
                return 1

        cb = EXCHANGE_FN(exchange)
        sh = Shard(rank, world, cb, None)
        _check(lib().air_set_stream(self._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 1 if include_interior else 0)
        cap = capacity or max(self._cap_hint, 4 * base_res * base_res)
        for _ in range(2):
            im, out = self._alloc(cap, mem, fields)
            st = lib().air_render_adaptive_sharded(self._h, C.byref(_view(view)), C.byref(p),
                                                   C.byref(sh), C.byref(im))
            if errors:
                raise errors[0]
            if st != AIR_ERR_CAPACITY:
                break
            cap = int(im.n_out)
        _check(st)
        self._cap_hint = max(self._cap_hint, int(im.n_out))
        return self._result(im, out)

    def render_adaptive_spectra(self, view, base_res, max_level, xi_crit, xi_norm=0, refine_on=0,
                                fp64_level=-1, mem="device", fields=("level", "i", "j", "is_leaf",
                                                                     "coldens", "p", "band_flux"),
                                spectra_cap=None):
        """air_render_adaptive_spectra: every traced node (creation order) and
        its spectrum in a page-locked host tensor [n_bands, spectra_cap]
        (float32, node k in column k). Returns (result, spectra)."""
        import torch
        fields = tuple(f for f in fields if f != "intensity")
        _check(lib().air_set_stream(self._h, _stream()))
        p = Params(int(base_res), int(max_level), float(xi_crit), int(xi_norm), int(refine_on),
                   int(fp64_level), 1)
        cap = spectra_cap or max(self._cap_hint, 4 * base_res * base_res)
        for _ in range(2):
            spec = torch.empty((self.n_bands, cap), dtype=torch.float32, pin_memory=True)
            im, out = self._alloc(cap, mem, fields)
            st = lib().air_render_adaptive_spectra(self._h, C.byref(_view(view)), C.byref(p),
                                                   C.byref(im), C.c_void_p(spec.data_ptr()),
                                                   C.c_int64(cap))
            if st != AIR_ERR_CAPACITY:
                break
            cap = max(int(im.n_rays), int(im.n_out), cap)
        _check(st)
        self._cap_hint = max(self._cap_hint, int(im.n_out))
        self._raster_src = (int(base_res), int(max_level))
        return self._result(im, out), spec[:, :int(im.n_out)]

    def raster(self, quantity="p", band=0, mode="bilinear", mem="device"):
        """air_render_raster: finest-level raster [(n0 2^Lm), (n0 2^Lm)] (index
        [y, x]) of the most recent single-view adaptive image, float32."""
        import torch
        src = getattr(self, "_raster_src", None)
        if src is None:
            raise AirError(AIR_ERR_ARG, "no single-view adaptive image to rasterise")
        nf = src[0] << src[1]
        out = torch.empty((nf, nf), dtype=torch.float32, device="cuda" if mem == "device" else "cpu",
                          pin_memory=(mem != "device"))
        _check(lib().air_set_stream(self._h, _stream()))
        _check(lib().air_render_raster(self._h, RASTER_QUANTITIES[quantity], int(band),
                                       RASTER_MODES[mode], C.c_void_p(out.data_ptr()),
                                       C.c_int64(nf * nf)))
        return out


def _batch_call(grid, views, p, opts, caps, mem, fields, learned=None):
    ims, outs = [], []
    for c in caps:
        im, out = grid._alloc(c, mem, fields)
        ims.append(im)
        outs.append(out)
    arr_v = (View * len(views))(*[_view(v) for v in views])
    arr_i = (Image * len(views))(*ims)
    if learned is None:
        st = lib().air_render_batch(grid._h, arr_v, len(views), C.byref(p), C.byref(opts), arr_i)
    else:
        mlp, lo, stats = learned
        st = lib().air_render_batch_learned(grid._h, arr_v, len(views), C.byref(p), C.byref(opts),
                                            mlp._h, C.byref(lo), arr_i, C.byref(stats))
    return st, arr_i, outs


def band_flux_static(intensity, n, area0, level=None, is_leaf=None, out=None):
    """air_band_flux_static: band flux of a device image with no allocation in
    the library. `intensity` is a [n_bands, stride] CUDA tensor (row stride
    `stride`), `level` / `is_leaf` optional CUDA tensors, `out` a float64 CUDA
    tensor of n_bands entries (allocated here if None, by the caller's torch)."""
    import torch
    if intensity.dim() != 2 or intensity.dtype != torch.float32 or intensity.stride(1) != 1:
        raise ValueError("intensity must be a float32 [n_bands, stride] tensor with unit column stride")
    nb = intensity.shape[0]
    n = int(n)
    if not 0 <= n <= intensity.shape[1]:
        raise ValueError(f"n = {n} outside [0, {intensity.shape[1]}]")
    dev = intensity.device
    for name, t, dt in (("level", level, torch.int32), ("is_leaf", is_leaf, torch.uint8)):
        if t is not None:
            if t.dtype != dt or t.dim() != 1 or t.stride(0) != 1 or t.numel() < n:
                raise ValueError(f"{name} must be a contiguous {dt} tensor of at least n entries")
            if t.device != dev:
                raise ValueError(f"{name} is on {t.device}, intensity on {dev}")
    if out is None:
        out = torch.empty(nb, dtype=torch.float64, device=dev)
    elif out.dtype != torch.float64 or out.numel() < nb or not out.is_contiguous() or out.device != dev:
        raise ValueError("out must be a contiguous float64 tensor of n_bands entries on intensity's device")
    with torch.cuda.device(dev):
        st = lib().air_band_flux_static(
            C.c_void_p(intensity.data_ptr()), int(intensity.stride(0)), int(nb),
            C.c_void_p(level.data_ptr()) if level is not None else None,
            C.c_void_p(is_leaf.data_ptr()) if is_leaf is not None else None, n, float(area0),
            C.c_void_p(out.data_ptr()), _stream())
    _check(st)
    return out


MLP_NPARAMS = 16 * 64 + 64 + 64 * 64 + 64 + 64 * 5 + 5


class MLP:
    """The refinement-depth network (air_mlp_*). Features: uint16 BF16 bit
    patterns [n, 16] on the GPU; labels int32 [n]; parameters FP32 [5573]."""

    def __init__(self, params=None):
        h = C.c_void_p()
        arr = None
        if params is not None:
            arr = np.ascontiguousarray(params, dtype=np.float32)
            assert arr.size == MLP_NPARAMS
        _check(lib().air_mlp_create(arr.ctypes.data if arr is not None else None, _stream(),
                                    C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().air_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self, set=None):
        out = np.empty(MLP_NPARAMS, dtype=np.float32)
        arr = None if set is None else np.ascontiguousarray(set, dtype=np.float32)
        _check(lib().air_mlp_set_stream(self._h, _stream()))
        _check(lib().air_mlp_params(self._h, out.ctypes.data,
                                    arr.ctypes.data if arr is not None else None))
        return out

    def forward(self, x):
        import torch
        n = x.shape[0]
        out = torch.empty((n, 5), dtype=torch.float32, device=x.device)
        _check(lib().air_mlp_set_stream(self._h, _stream()))
        _check(lib().air_mlp_forward(self._h, C.c_void_p(x.data_ptr()), n, C.c_void_p(out.data_ptr())))
        return out

    def loss_grad(self, x, y):
        import torch
        g = torch.empty(MLP_NPARAMS, dtype=torch.float32, device=x.device)
        loss = C.c_double()
        _check(lib().air_mlp_set_stream(self._h, _stream()))
        _check(lib().air_mlp_loss_grad(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                       x.shape[0], C.c_void_p(g.data_ptr()), C.byref(loss)))
        return loss.value, g

    def train(self, x, y, batch=4096, epochs=1, lr=1e-3):
        hist = np.zeros(max(epochs, 1))
        _check(lib().air_mlp_set_stream(self._h, _stream()))
        _check(lib().air_mlp_train(self._h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                   x.shape[0], int(batch), int(epochs), float(lr),
                                   hist.ctypes.data))
        return hist[:epochs]


def version() -> str:
    return lib().air_version().decode()
