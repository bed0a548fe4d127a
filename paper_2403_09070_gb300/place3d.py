"""Thin Python binding of the place3d C ABI (include/place3d.h).

Argument marshalling only: every step of the evaluation runs in the CUDA
kernels of libplace3d.so.  There is no CPU fallback: if the library cannot be
loaded the constructor raises.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory; CUDA tensors are used in place on the handle's stream).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FP64, FP32, FP32_TC = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "fp32_tc": FP32_TC}
F64, F32 = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1
FLAG_CHECKS = 1
FLAG_MACRO_GATHER_SCAN, FLAG_MACRO_GATHER_DIRECT, FLAG_SERIAL, FLAG_TILES, FLAG_NO_TILES = 2, 4, 8, 16, 32
WL_FORMS = ((1, 1), (1, 2), (1, 4), (2, 2), (4, 1), (2, 4), (8, 1), (4, 4), (16, 1), (8, 4), (32, 1), (16, 4), (32, 2),
            (32, 4))
MAP_RHO_FIXED, MAP_EX, MAP_EY, MAP_EZ = 0, 1, 2, 3
MODE_3D, MODE_2D = 0, 1
ERRORS = {-1: "INVALID_ARG", -2: "BAD_CSR", -3: "OUT_OF_RANGE", -4: "CUDA", -5: "OOM", -6: "TIMEOUT",
          -7: "UNSUPPORTED"}


class Place3DError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"place3d error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Problem(C.Structure):
    _fields_ = [
        ("n_inst", C.c_int32), ("is_macro", C.c_void_p), ("z_fixed", C.c_void_p),
        ("w_bot", C.c_void_p), ("h_bot", C.c_void_p), ("w_top", C.c_void_p), ("h_top", C.c_void_p),
        ("n_net", C.c_int32), ("n_pin", C.c_int32), ("net_start", C.c_void_p), ("pin_inst", C.c_void_p),
        ("pin_off_bot_x", C.c_void_p), ("pin_off_bot_y", C.c_void_p),
        ("pin_off_top_x", C.c_void_p), ("pin_off_top_y", C.c_void_p),
        ("xl", C.c_double), ("yl", C.c_double), ("xh", C.c_double), ("yh", C.c_double),
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("gamma", C.c_double), ("gamma_z", C.c_double), ("alpha", C.c_double), ("lam", C.c_double),
        ("precision", C.c_int32), ("flags", C.c_int32),
        ("mode", C.c_int32), ("is_hbt", C.c_void_p), ("lam_layer", C.c_double * 3),
    ]


class Result(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d", "n_cross",
                                           "g_scale", "s_x", "s_y", "s_z")] + [("energy_layer", C.c_double * 3),
                                                                                ("overflow", C.c_double)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "energy_layer"}
        d["energy_layer"] = list(self.energy_layer)
        return d


EXPORTS = ("place3d_create", "place3d_geometry", "place3d_alpha", "place3d_set_positions",
           "place3d_eval_objective_and_grad", "place3d_get_result", "place3d_copy_map",
           "place3d_copy_wl_parts", "place3d_set_profiling", "place3d_num_stages", "place3d_stage_name",
           "place3d_stage_times", "place3d_launches_per_eval", "place3d_last_error", "place3d_destroy",
           "place3d_density_map_noalloc", "place3d_tc_selftest", "place3d_autotune", "place3d_wl_forms",
           "place3d_set_wl_form", "place3d_result_to_device", "place3d_set_params", "place3d_eval_graph",
           "place3d_batch_create", "place3d_batch_eval", "place3d_batch_destroy", "place3d_set_layer_weights",
           "place3d_tc_timeout_selftest", "place3d_debug_fail_alloc", "place3d_ll2f_selftest",
           "place3d_graph_captures", "place3d_nesterov_init", "place3d_nesterov_precondition",
           "place3d_nesterov_update", "place3d_nesterov_step", "place3d_set_wl_plan", "place3d_tc_tiles",
           "place3d_set_tc_tiles", "place3d_batch_shared_stages")
NOALLOC_MAX_BINS = 262144

_lib = None


def library_path() -> str:
    return _build.SO


def load_library(build_if_missing: bool = True):
    """Load libplace3d.so (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.SO
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing; run paper_2403_09070_gb300.build.build()")
        _build.build()
    L = C.CDLL(path)
    vp, i32, d = C.c_void_p, C.c_int, C.c_double
    L.place3d_create.argtypes = [C.POINTER(_Problem), i32, vp, C.POINTER(vp)]
    L.place3d_geometry.argtypes = [vp, vp]
    L.place3d_alpha.argtypes = [d] * 6
    L.place3d_alpha.restype = d
    L.place3d_set_positions.argtypes = [vp, vp, vp, vp, i32, i32]
    L.place3d_eval_objective_and_grad.argtypes = [vp, C.POINTER(Result), vp, vp, vp, i32, i32]
    L.place3d_get_result.argtypes = [vp, C.POINTER(Result)]
    L.place3d_copy_map.argtypes = [vp, i32, vp, i32]
    L.place3d_copy_wl_parts.argtypes = [vp, vp, vp, vp, vp]
    L.place3d_set_profiling.argtypes = [vp, i32]
    L.place3d_num_stages.argtypes = []
    L.place3d_stage_name.argtypes = [i32]
    L.place3d_stage_name.restype = C.c_char_p
    L.place3d_stage_times.argtypes = [vp, vp, vp, vp, i32]
    L.place3d_launches_per_eval.argtypes = [vp]
    L.place3d_last_error.argtypes = [vp]
    L.place3d_last_error.restype = C.c_char_p
    L.place3d_destroy.argtypes = [vp]
    L.place3d_destroy.restype = None
    L.place3d_autotune.argtypes = [vp, i32]
    L.place3d_set_wl_form.argtypes = [vp, i32, i32, i32]
    L.place3d_result_to_device.argtypes = [vp, vp]
    L.place3d_eval_graph.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32]
    L.place3d_batch_create.argtypes = [vp, i32, C.POINTER(vp)]
    L.place3d_batch_eval.argtypes = [vp, vp, vp, vp, vp, vp, vp, i32, vp]
    L.place3d_batch_destroy.argtypes = [vp]
    L.place3d_batch_destroy.restype = None
    L.place3d_batch_shared_stages.argtypes = [vp]
    L.place3d_set_params.argtypes = [vp, d, d, d, d]
    L.place3d_set_layer_weights.argtypes = [vp, vp]
    L.place3d_wl_forms.argtypes = [vp, vp, vp, vp, i32]
    L.place3d_set_wl_plan.argtypes = [vp, vp, vp, vp, i32]
    L.place3d_tc_tiles.argtypes = [vp, vp, i32]
    L.place3d_set_tc_tiles.argtypes = [vp, vp, i32]
    L.place3d_tc_selftest.argtypes = [i32, i32, i32, i32, vp, vp, vp, vp]
    L.place3d_tc_timeout_selftest.argtypes = [C.c_longlong, vp]
    L.place3d_debug_fail_alloc.argtypes = [i32]
    L.place3d_debug_fail_alloc.restype = None
    L.place3d_ll2f_selftest.argtypes = [vp, vp, i32, vp]
    L.place3d_graph_captures.argtypes = [vp]
    L.place3d_graph_captures.restype = C.c_longlong
    L.place3d_nesterov_init.argtypes = [vp] * 4 + [d]
    L.place3d_nesterov_precondition.argtypes = [vp] * 4
    L.place3d_nesterov_update.argtypes = [vp] * 10 + [d]
    L.place3d_nesterov_step.argtypes = [vp, vp]
    L.place3d_density_map_noalloc.argtypes = [i32] + [vp] * 8 + [d] * 4 + [i32] * 3 + [vp, vp]
    _lib = L
    return L


def alpha(dx, dz, beta=10.0, w_hbt=1.0, rh_top=0.8, rh_bot=1.0) -> float:
    """HBT penalty factor of Sec. V-A (computed by the library)."""
    return float(load_library().place3d_alpha(dx, dz, beta, w_hbt, rh_top, rh_bot))


def _is_torch(a):
    return hasattr(a, "data_ptr") and hasattr(a, "is_cuda")


def _buf(a):
    """(pointer, dtype code, mem kind, keepalive) of a numpy array / torch tensor."""
    if _is_torch(a):
        import torch
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        dt = {torch.float64: F64, torch.float32: F32}.get(a.dtype)
        if dt is None:
            raise ValueError(f"unsupported dtype {a.dtype}")
        return a.data_ptr(), dt, (MEM_DEVICE if a.is_cuda else MEM_HOST), a
    a = np.ascontiguousarray(a)
    dt = {np.dtype(np.float64): F64, np.dtype(np.float32): F32}.get(a.dtype)
    if dt is None:
        raise ValueError(f"unsupported dtype {a.dtype}")
    return a.ctypes.data, dt, MEM_HOST, a


class Place3D:
    """One placement problem on one GPU (owns a place3d handle)."""

    def __init__(self, prob: dict, precision: str | int = "fp32", device: int = 0, stream=None,
                 alpha: float | None = None, flags: int = 0):
        L = load_library()
        self._L = L
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        self.precision = precision
        keep = {}

        def arr(k, dt):
            a = np.ascontiguousarray(prob[k], dtype=dt)
            keep[k] = a
            return a.ctypes.data

        n = int(prob["n_inst"])
        zf = prob.get("z_fixed")
        p = _Problem()
        p.n_inst = n
        p.is_macro = arr("is_macro", np.uint8)
        p.z_fixed = arr("z_fixed", np.uint8) if zf is not None else None
        p.w_bot, p.h_bot = arr("w_bot", np.float64), arr("h_bot", np.float64)
        p.w_top, p.h_top = arr("w_top", np.float64), arr("h_top", np.float64)
        p.n_net, p.n_pin = int(prob["n_net"]), int(prob["n_pin"])
        p.net_start, p.pin_inst = arr("net_start", np.int32), arr("pin_inst", np.int32)
        p.pin_off_bot_x, p.pin_off_bot_y = arr("off_bx", np.float64), arr("off_by", np.float64)
        p.pin_off_top_x, p.pin_off_top_y = arr("off_tx", np.float64), arr("off_ty", np.float64)
        p.xl, p.yl, p.xh, p.yh = (float(prob[k]) for k in ("xl", "yl", "xh", "yh"))
        p.nx, p.ny, p.nz = int(prob["nx"]), int(prob["ny"]), int(prob["nz"])
        p.gamma, p.gamma_z = float(prob["gamma"]), float(prob.get("gamma_z", 0.0))
        if alpha is None and p.nx > 0 and p.ny > 0:
            wb = (p.xh - p.xl) / p.nx
            hb = (p.yh - p.yl) / p.ny
            dz = p.nz * 0.5 * (wb + hb)
            alpha = L.place3d_alpha(p.xh - p.xl, dz, prob.get("beta", 10.0), prob.get("w_hbt", 1.0),
                                    prob.get("rh_top", 0.8), prob.get("rh_bot", 1.0))
        p.alpha = float(alpha) if alpha is not None else 0.0
        p.lam = float(prob["lam"])
        p.precision = int(precision)
        p.flags = int(flags)
        p.mode = int(prob.get("mode", MODE_3D))
        p.is_hbt = arr("is_hbt", np.uint8) if prob.get("is_hbt") is not None else None
        p.lam_layer = (C.c_double * 3)(*[float(v) for v in prob.get("lam_layer", (prob["lam"],) * 3)])
        self.mode = p.mode
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = C.c_void_p()
        rc = L.place3d_create(C.byref(p), int(device), C.c_void_p(stream or 0), C.byref(h))
        if rc != 0:
            raise Place3DError(rc, L.place3d_last_error(None).decode())
        self._h = h
        self.n = n
        self.alpha = p.alpha
        self.nb = p.nx * p.ny * p.nz
        self.shape = (p.nz, p.ny, p.nx)
        self._keep = None

    # -- plumbing --
    def _check(self, rc):
        if rc != 0:
            raise Place3DError(rc, self._L.place3d_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._L.place3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API --
    def geometry(self) -> dict:
        out = np.zeros(6)
        self._check(self._L.place3d_geometry(self._h, out.ctypes.data))
        return dict(wb=out[0], hb=out[1], db=out[2], dx=out[3], dy=out[4], dz=out[5])

    def set_positions(self, x, y, z):
        bx, by, bz = _buf(x), _buf(y), _buf(z)
        if len({bx[1], by[1], bz[1]}) != 1 or len({bx[2], by[2], bz[2]}) != 1:
            raise ValueError("x, y, z must share dtype and memory kind")
        self._keep = (bx[3], by[3], bz[3])
        self._check(self._L.place3d_set_positions(self._h, bx[0], by[0], bz[0], bx[1], bx[2]))

    def eval(self, gx=None, gy=None, gz=None, sync: bool = True):
        """Enqueue one evaluation; with sync return the scalars as a dict."""
        res = Result()
        if gx is None:
            ptrs, dt, mem = (None, None, None), F64, MEM_HOST
        else:
            b = [_buf(a) for a in (gx, gy, gz)]
            ptrs, dt, mem = tuple(v[0] for v in b), b[0][1], b[0][2]
            self._gkeep = [v[3] for v in b]
        self._check(self._L.place3d_eval_objective_and_grad(
            self._h, C.byref(res) if sync else None, *ptrs, dt, mem))
        return res.as_dict() if sync else None

    def result_to_device(self, dst):
        """Enqueue the last evaluation's 10 scalars into a CUDA float64 tensor."""
        self._check(self._L.place3d_result_to_device(self._h, dst.data_ptr()))

    def set_params(self, gamma: float, gamma_z: float, alpha: float, lam: float):
        self._check(self._L.place3d_set_params(self._h, float(gamma), float(gamma_z), float(alpha), float(lam)))
        self.alpha = float(alpha)

    def set_layer_weights(self, lam_bot: float, lam_top: float, lam_hbt: float):
        """2D mode: the density weights (lambda-, lambda+, lambda') of eq. 2d-place."""
        self._check(self._L.place3d_set_layer_weights(self._h, (C.c_double * 3)(lam_bot, lam_top, lam_hbt)))

    def eval_graph(self, x, y, z, gx, gy, gz):
        """Pack + evaluate as one CUDA-graph launch (CUDA tensors; the graph is
        re-captured only when a tensor's address, the dtype, gamma, gamma_z, alpha or a
        reduction form changes; a new lambda is read from device memory)."""
        b = [_buf(a) for a in (x, y, z, gx, gy, gz)]
        if any(v[2] != MEM_DEVICE for v in b) or len({v[1] for v in b}) != 1:
            raise ValueError("eval_graph takes CUDA tensors of one dtype")
        self._gkeep = [v[3] for v in b]
        self._check(self._L.place3d_eval_graph(self._h, *[v[0] for v in b], b[0][1]))

    def get_result(self) -> dict:
        res = Result()
        self._check(self._L.place3d_get_result(self._h, C.byref(res)))
        return res.as_dict()

    def copy_map(self, which: int) -> np.ndarray:
        if which == MAP_RHO_FIXED:
            out = np.zeros(self.shape, np.int64)
        else:
            out = np.zeros(self.shape, np.float64 if self.precision == FP64 else np.float32)
        self._check(self._L.place3d_copy_map(self._h, which, out.ctypes.data, MEM_HOST))
        return out

    def wl_parts(self) -> dict:
        g = [np.zeros(self.n) for _ in range(4)]
        self._check(self._L.place3d_copy_wl_parts(self._h, *[a.ctypes.data for a in g]))
        return dict(gx=g[0], gy=g[1], gfd=g[2], gwaz=g[3])

    def set_profiling(self, on: bool):
        self._check(self._L.place3d_set_profiling(self._h, int(bool(on))))

    def stage_times(self, reset: bool = False) -> dict:
        ns = self._L.place3d_num_stages()
        ms = np.zeros(ns)
        ln = np.zeros(ns, np.int64)
        ev = np.zeros(1, np.int64)
        self._check(self._L.place3d_stage_times(self._h, ms.ctypes.data, ln.ctypes.data, ev.ctypes.data,
                                                int(reset)))
        names = [self._L.place3d_stage_name(k).decode() for k in range(ns)]
        return dict(evals=int(ev[0]), stages={nm: (float(ms[k]), int(ln[k])) for k, nm in enumerate(names)})

    def autotune(self, repeats: int = 3):
        """Pick the fastest reduction form per net-degree bucket (call after set_positions)."""
        self._check(self._L.place3d_autotune(self._h, int(repeats)))

    def wl_forms(self) -> list:
        """[(largest degree, lanes per net, pins per lane)] per degree bucket."""
        cap = 16
        a, b, c = (np.zeros(cap, np.int32) for _ in range(3))
        k = self._L.place3d_wl_forms(self._h, a.ctypes.data, b.ctypes.data, c.ctypes.data, cap)
        return [(int(a[i]), int(b[i]), int(c[i])) for i in range(min(k, cap))]

    def set_wl_form(self, bucket: int, lanes: int, pins: int):
        self._check(self._L.place3d_set_wl_form(self._h, int(bucket), int(lanes), int(pins)))

    def set_wl_plan(self, plan):
        """Set the wirelength launch plan [(largest degree, lanes, pins)], as
        wl_forms() lists it; [] restores the default plan."""
        d, l_, p_ = (np.ascontiguousarray([int(v[k]) for v in plan], dtype=np.int32) for k in range(3))
        self._check(self._L.place3d_set_wl_plan(self._h, d.ctypes.data, l_.ctypes.data, p_.ctypes.data,
                                                len(plan)))

    def tc_tiles(self) -> list:
        """Tile widths of the four tensor-core product groups ([] without them)."""
        a = np.zeros(4, np.int32)
        k = self._L.place3d_tc_tiles(self._h, a.ctypes.data, 4)
        return [int(v) for v in a[:k]]

    def set_tc_tiles(self, cols):
        a = np.ascontiguousarray(cols, dtype=np.int32)
        self._check(self._L.place3d_set_tc_tiles(self._h, a.ctypes.data, int(a.size)))

    def _dev(self, arrs):
        b = [_buf(a) for a in arrs]
        want = F64 if self.precision == PRECISIONS["fp64"] else F32
        if any(v[2] != MEM_DEVICE or v[1] != want for v in b):
            raise ValueError("the Nesterov helpers take CUDA tensors in the handle's precision")
        return [v[0] for v in b]

    def nesterov_init(self, g, init_step: float):
        """g <- the last evaluation's gradient / H; step <- init_step / max |g|
        (device, no sync; the evaluation: eval() without gradient arrays)."""
        self._check(self._L.place3d_nesterov_init(self._h, *self._dev(list(g)), float(init_step)))

    def nesterov_precondition(self, g):
        """g <- the last evaluation's gradient / H (eq. improved-precond);
        step <- |dv| / |dg| (device, no sync)."""
        self._check(self._L.place3d_nesterov_precondition(self._h, *self._dev(list(g))))

    def nesterov_update(self, u, v, g, coef: float):
        """u <- P(v - step g); v <- P(u_new + coef (u_new - u)), also the
        positions of the next evaluation (device, no sync)."""
        self._check(self._L.place3d_nesterov_update(self._h, *self._dev(list(u) + list(v) + list(g)), float(coef)))

    def nesterov_step(self) -> float:
        s = C.c_double(0)
        self._check(self._L.place3d_nesterov_step(self._h, C.byref(s)))
        return s.value

    def graph_captures(self) -> int:
        """CUDA-graph captures made by this handle so far."""
        return int(self._L.place3d_graph_captures(self._h))

    def launches_per_eval(self) -> int:
        return int(self._L.place3d_launches_per_eval(self._h))


def density_map_noalloc(x, y, z, w_bot, h_bot, w_top, h_top, is_macro, region, grid, rho, stream=None):
    """Allocation-free fixed-point density map (place3d_density_map_noalloc).

    All arrays are CUDA tensors on the current device (float64, is_macro
    uint8); rho ([nz, ny, nx] float64) is written on `stream` (asynchronous).
    For callers that cannot allocate device memory at this point; the
    library's scratch for it is a fixed array shared by all calls on a
    device, so calls must not overlap on the GPU."""
    L = load_library()
    n = int(x.numel())
    xl, yl, xh, yh = (float(v) for v in region)
    nx, ny, nz = (int(v) for v in grid)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    rc = L.place3d_density_map_noalloc(n, *[t.data_ptr() for t in (x, y, z, w_bot, h_bot, w_top, h_top,
                                                                     is_macro)],
                                       xl, yl, xh, yh, nx, ny, nz, rho.data_ptr(), C.c_void_p(stream or 0))
    if rc != 0:
        raise Place3DError(rc, "place3d_density_map_noalloc failed")


def debug_fail_alloc(nth: int):
    """Make the nth device allocation of the next create on this thread fail
    as out of memory (nth <= 0 clears it)."""
    load_library().place3d_debug_fail_alloc(int(nth))


def ll2f_selftest(vals):
    """Convert int64 values with the density pass's int64 -> FP32 routine on
    the GPU; returns (results as float32, count differing from the hardware
    conversion)."""
    L = load_library()
    v = np.ascontiguousarray(vals, dtype=np.int64)
    out = np.zeros(v.size, np.float32)
    bad = C.c_int(0)
    rc = L.place3d_ll2f_selftest(v.ctypes.data, out.ctypes.data, int(v.size), C.byref(bad))
    if rc != 0:
        raise Place3DError(rc, L.place3d_last_error(None).decode())
    return out, bad.value


def tc_timeout_selftest(wait_cycles: int = 200_000_000):
    """Run the tensor-core kernel with a producer that loads nothing and every
    wait bounded by wait_cycles SM clocks; returns (status, wait error code)."""
    L = load_library()
    e = C.c_int(0)
    rc = L.place3d_tc_timeout_selftest(int(wait_cycles), C.byref(e))
    return rc, e.value


def tc_selftest(A, W):
    """The tensor-core split-BF16 product out[b][n][m] = sum_k A[b][m][k] W[n][k]
    (place3d_tc_selftest) on host float32 arrays; returns (out, wait_error)."""
    L = load_library()
    A = np.ascontiguousarray(A, dtype=np.float32)
    W = np.ascontiguousarray(W, dtype=np.float32)
    batches, M, K = A.shape
    N = W.shape[0]
    out = np.zeros((batches, N, M), np.float32)
    err = np.zeros(1, np.int32)
    rc = L.place3d_tc_selftest(M, N, K, batches, A.ctypes.data, W.ctypes.data, out.ctypes.data, err.ctypes.data)
    if rc != 0:
        raise Place3DError(rc, f"place3d_tc_selftest failed (wait error {int(err[0])})")
    return out, int(err[0])


class Batch:
    """Independent placement problems evaluated by one CUDA-graph launch."""

    def __init__(self, handles):
        L = load_library()
        self._L = L
        self.handles = list(handles)
        arr = (C.c_void_p * len(self.handles))(*[h._h.value for h in self.handles])
        b = C.c_void_p()
        rc = L.place3d_batch_create(arr, len(self.handles), C.byref(b))
        if rc != 0:
            raise Place3DError(rc, L.place3d_last_error(None).decode())
        self._b = b

    def eval(self, xs, ys, zs, gxs, gys, gzs, stream=None):
        """Per-instance CUDA tensors (lists); launches the batch graph."""
        cols = [xs, ys, zs, gxs, gys, gzs]
        bufs = [[_buf(a) for a in col] for col in cols]
        dts = {v[1] for col in bufs for v in col}
        if len(dts) != 1 or any(v[2] != MEM_DEVICE for col in bufs for v in col):
            raise ValueError("batch eval takes CUDA tensors of one dtype")
        self._keep = [v[3] for col in bufs for v in col]
        arrs = [(C.c_void_p * len(col))(*[v[0] for v in col]) for col in bufs]
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        rc = self._L.place3d_batch_eval(self._b, *arrs, dts.pop(), C.c_void_p(stream or 0))
        if rc != 0:
            raise Place3DError(rc, "place3d_batch_eval: " + self._L.place3d_last_error(None).decode())

    def shared_stages(self) -> int:
        """1 when the last captured batch graph shares the wirelength stage's
        launches among its instances, 0 when each instance runs its own."""
        return int(self._L.place3d_batch_shared_stages(self._b))

    def close(self):
        if getattr(self, "_b", None):
            self._L.place3d_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
