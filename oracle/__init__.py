"""FP64 CPU oracle for adaptive image ray-tracing (AIR) -- test infrastructure.

Only tests/, the smoke check and the benchmark's CPU-baseline leg import this
package. The product library (paper_1010_5534_gb300) never imports it, and the
two share no code; the only shared inputs come from the `scenes` module.

The arithmetic lives in air_oracle.c (plain C, FP64, no FMA contraction); this
module compiles it with gcc and wraps it with ctypes. See air_oracle.c for the
passages of the paper each part follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "air_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liborc.so (gcc, FP64, -ffp-contract=off so
    that no multiply-add is fused, OpenMP over independent rays)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "air_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Scene(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n", C.c_int32 * 3), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3), ("brick", C.c_int32), ("max_level", C.c_int32),
                ("n_bricks", C.c_int32), ("brick_level", C.c_void_p),
                ("brick_origin", C.c_void_p), ("rho", C.c_void_p), ("temp", C.c_void_p),
                ("n_bands", C.c_int32), ("emis_mode", C.c_int32),
                ("lambda_table", C.c_void_p), ("n_tbins", C.c_int32),
                ("logT_lo", C.c_double), ("logT_hi", C.c_double), ("kappa", C.c_void_p),
                ("field_f32", C.c_int32)]


class ViewS(C.Structure):
    _fields_ = [("dir", C.c_double * 3), ("up", C.c_double * 3), ("center", C.c_double * 3),
                ("half_extent", C.c_double)]


class Params(C.Structure):
    _fields_ = [("base_res", C.c_int32), ("max_level", C.c_int32), ("xi_crit", C.c_double),
                ("xi_norm", C.c_int32), ("refine_on", C.c_int32)]


class Replay(C.Structure):
    _fields_ = [("n", C.c_int64), ("level", C.c_void_p), ("i", C.c_void_p), ("j", C.c_void_p),
                ("p_int", C.c_void_p), ("p_col", C.c_void_p)]


class Hybrid(C.Structure):
    _fields_ = [("rtol", C.c_double), ("margin", C.c_double), ("n_decisions", C.c_int64),
                ("n_undecided", C.c_int64), ("n_taken_from_other", C.c_int64),
                ("n_unresolved", C.c_int64)]


class Tree(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("n_nodes", C.c_int64), ("n_leaves", C.c_int64),
                ("n_refined", C.c_int64), ("n_sweeps", C.c_int64), ("n_steps", C.c_int64),
                ("level", C.c_void_p), ("i", C.c_void_p), ("j", C.c_void_p),
                ("leaf", C.c_void_p), ("parent", C.c_void_p), ("col", C.c_void_p),
                ("inten", C.c_void_p), ("p_int", C.c_void_p), ("steps", C.c_void_p)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            L.orc_prepare.restype = C.c_void_p
            L.orc_prepare.argtypes = [C.POINTER(Scene), C.POINTER(C.c_int32)]
            L.orc_release.argtypes = [C.c_void_p]
            L.orc_trace.restype = C.c_int32
            L.orc_trace.argtypes = [C.c_void_p, C.POINTER(ViewS), C.c_int32, C.c_int64,
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p]
            L.orc_air.restype = C.c_int32
            L.orc_air.argtypes = [C.c_void_p, C.POINTER(ViewS), C.POINTER(Params),
                                  C.POINTER(Tree), C.POINTER(Replay)]
            L.orc_air_hybrid.restype = C.c_int32
            L.orc_air_hybrid.argtypes = [C.c_void_p, C.POINTER(ViewS), C.POINTER(Params),
                                         C.POINTER(Tree), C.POINTER(Replay), C.POINTER(Hybrid)]
            L.orc_xi.restype = C.c_double
            L.orc_xi.argtypes = [C.c_void_p, C.c_int32]
            L.orc_lambda.restype = C.c_double
            L.orc_lambda.argtypes = [C.c_void_p, C.c_int32, C.c_double]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def _view(v) -> ViewS:
    s = ViewS()
    s.dir[:] = [float(x) for x in v.dir]
    s.up[:] = [float(x) for x in v.up]
    s.center[:] = [float(x) for x in v.center]
    s.half_extent = float(v.half_extent)
    return s


class Oracle:
    """Holds a prepared scene for repeated calls. FP32 fields are read in place
    (each value widens exactly to FP64 on use), others as FP64 copies."""

    def __init__(self, scene):
        self.scene = scene
        self._keep = []
        s = Scene()
        s.kind = 0 if scene.kind == "uniform" else 1
        s.n[:] = [int(x) for x in scene.n]
        s.lo[:] = [float(x) for x in scene.lo]
        s.hi[:] = [float(x) for x in scene.hi]
        f32 = scene.rho.dtype == np.float32 and (scene.temp is None or scene.temp.dtype == np.float32)
        fdt = np.float32 if f32 else np.float64
        s.field_f32 = 1 if f32 else 0
        self.rho = np.ascontiguousarray(scene.rho, dtype=fdt)
        s.rho = _p(self.rho)
        if scene.temp is not None:
            self.temp = np.ascontiguousarray(scene.temp, dtype=fdt)
            s.temp = _p(self.temp)
        if scene.kind == "amr":
            self.blev = np.ascontiguousarray(scene.brick_level, dtype=np.int32)
            self.borg = np.ascontiguousarray(scene.brick_origin, dtype=np.int32)
            s.brick, s.max_level, s.n_bricks = scene.brick, scene.max_level, len(self.blev)
            s.brick_level, s.brick_origin = _p(self.blev), _p(self.borg)
        self.kappa = np.ascontiguousarray(scene.kappa, dtype=np.float64)
        s.n_bands = len(self.kappa)
        s.kappa = _p(self.kappa)
        s.emis_mode = scene.emis_mode
        if scene.emis_mode == 1:
            self.tab = np.ascontiguousarray(scene.lambda_table, dtype=np.float64)
            s.lambda_table = _p(self.tab)
            s.n_tbins = self.tab.shape[1]
            s.logT_lo, s.logT_hi = scene.logT_lo, scene.logT_hi
        self._s = s
        err = C.c_int32(0)
        self.ctx = lib().orc_prepare(C.byref(s), C.byref(err))
        if not self.ctx:
            raise OracleError(f"orc_prepare failed ({err.value})")
        self.n_bands = s.n_bands

    def __del__(self):
        if getattr(self, "ctx", None):
            lib().orc_release(self.ctx)
            self.ctx = None

    def trace(self, view, n0, L, I, J):
        L = np.ascontiguousarray(L, dtype=np.int32)
        I = np.ascontiguousarray(I, dtype=np.int32)
        J = np.ascontiguousarray(J, dtype=np.int32)
        n = len(L)
        col = np.zeros(n)
        inten = np.zeros((n, self.n_bands))
        steps = np.zeros(n, dtype=np.int64)
        e = lib().orc_trace(self.ctx, C.byref(_view(view)), int(n0), n, _p(L), _p(I), _p(J),
                            _p(col), _p(inten), _p(steps))
        if e:
            raise OracleError(f"orc_trace failed ({e})")
        return col, inten, steps

    def fixed(self, view, res):
        """Fixed-resolution image: every pixel of a res x res image, row-major."""
        jj, ii = np.meshgrid(np.arange(res), np.arange(res), indexing="ij")
        col, inten, steps = self.trace(view, res, np.zeros(res * res), ii.ravel(), jj.ravel())
        return dict(i=ii.ravel().astype(np.int32), j=jj.ravel().astype(np.int32), col=col,
                    inten=inten, steps=steps)

    def air(self, view, base_res, max_level, xi_crit, xi_norm=0, refine_on=0,
            capacity=None, replay=None, other=None, rtol=1e-5, margin=2.0):
        """The AIR sweep loop. Returns every traced node (interior ones included)
        in creation order; `leaf` marks the pixels of the final image.

        replay: take pixel values from this table (level, i, j, p_int, p_col)
        instead of tracing. other: trace, but take every undecided flag
        decision (|xi - xi_crit| within `margin` x the first-order change of xi
        when each stencil value moves by `rtol` of itself) from this table's
        values; the counts come back under "hybrid"."""
        if capacity is None:
            capacity = sum((base_res << l) ** 2 for l in range(max_level + 1))
        nb = self.n_bands
        out = dict(level=np.zeros(capacity, np.int32), i=np.zeros(capacity, np.int32),
                   j=np.zeros(capacity, np.int32), leaf=np.zeros(capacity, np.int32),
                   parent=np.zeros(capacity, np.int32), col=np.zeros(capacity),
                   inten=np.zeros((capacity, nb)), p_int=np.zeros(capacity),
                   steps=np.zeros(capacity, np.int64))
        t = Tree()
        t.capacity = capacity
        for k in ("level", "i", "j", "leaf", "parent", "col", "inten", "p_int", "steps"):
            setattr(t, k, _p(out[k]))
        p = Params(base_res, max_level, float(xi_crit), xi_norm, refine_on)
        keep = []

        def table(src):
            arrs = [np.ascontiguousarray(src[k], dtype=dt) for k, dt in
                    (("level", np.int32), ("i", np.int32), ("j", np.int32),
                     ("p_int", np.float64), ("p_col", np.float64))]
            keep.extend(arrs)
            return Replay(len(arrs[0]), *[_p(a) for a in arrs])

        hy = None
        if other is not None:
            if replay is not None:
                raise ValueError("replay and other are exclusive")
            hy = Hybrid(float(rtol), float(margin), 0, 0, 0, 0)
            e = lib().orc_air_hybrid(self.ctx, C.byref(_view(view)), C.byref(p), C.byref(t),
                                     C.byref(table(other)), C.byref(hy))
        else:
            rp = table(replay) if replay is not None else None
            e = lib().orc_air(self.ctx, C.byref(_view(view)), C.byref(p), C.byref(t),
                              C.byref(rp) if rp is not None else None)
        if e:
            raise OracleError(f"orc_air failed ({e})")
        n = t.n_nodes
        res = {k: v[:n] for k, v in out.items()}
        res.update(n_nodes=n, n_leaves=t.n_leaves, n_refined=t.n_refined,
                   n_sweeps=t.n_sweeps, n_steps=t.n_steps)
        H = view.half_extent
        lv = res["level"][res["leaf"] == 1]
        area = (2.0 * H / (base_res * 2.0 ** lv)) ** 2
        res["band_flux"] = (res["inten"][res["leaf"] == 1] * area[:, None]).sum(axis=0)
        if hy is not None:
            res["hybrid"] = dict(decisions=hy.n_decisions, undecided=hy.n_undecided,
                                 taken_from_other=hy.n_taken_from_other,
                                 unresolved=hy.n_unresolved)
        return res

    def lam(self, band, T):
        return lib().orc_lambda(self.ctx, band, float(T))


def xi(stencil, xi_norm=0) -> float:
    """Eq. 2 on a 3x3 stencil indexed [dj+1][di+1]."""
    s = np.ascontiguousarray(np.asarray(stencil, dtype=np.float64).reshape(9))
    return lib().orc_xi(_p(s), xi_norm)
