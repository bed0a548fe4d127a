"""ctypes wrapper of the FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``; the library path never imports it.  It is
independent of the CUDA path: it shares no code with it and never calls it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = [os.path.join(_HERE, f) for f in ("oracle.c", "oracle.h", "oracle_fixed.inc")]
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FP contraction, so that every
    floating-point step is one IEEE rounding)."""
    newest = max(os.path.getmtime(f) for f in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, os.path.join(_HERE, "oracle.c"), "-lm"])
        os.replace(tmp, _SO)
    return _SO


class Problem(C.Structure):
    _fields_ = [
        ("n_inst", C.c_int), ("is_macro", C.c_void_p), ("z_fixed", C.c_void_p),
        ("w_bot", C.c_void_p), ("h_bot", C.c_void_p), ("w_top", C.c_void_p), ("h_top", C.c_void_p),
        ("n_net", C.c_int), ("n_pin", C.c_int), ("net_start", C.c_void_p), ("pin_inst", C.c_void_p),
        ("off_bx", C.c_void_p), ("off_by", C.c_void_p), ("off_tx", C.c_void_p), ("off_ty", C.c_void_p),
        ("xl", C.c_double), ("yl", C.c_double), ("xh", C.c_double), ("yh", C.c_double),
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("gamma", C.c_double), ("gamma_z", C.c_double), ("alpha", C.c_double), ("lam", C.c_double),
        ("is_hbt", C.c_void_p), ("mode", C.c_int), ("lam_layer", C.c_double * 3),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.POINTER(Problem)
        vp, d = C.c_void_p, C.c_double
        L.orc_geometry.argtypes = [P, vp]
        L.orc_alpha.argtypes = [d] * 6
        L.orc_alpha.restype = d
        L.orc_attributes.argtypes = [P] + [vp] * 9
        L.orc_density_direct.argtypes = [P, vp, vp, vp, vp]
        L.orc_macro_corner_map.argtypes = [P, vp, vp, vp, vp]
        L.orc_prefix_sum3.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.orc_prefix_sum3_i64.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.orc_density_fixed.argtypes = [P, vp, vp, vp, C.c_int, vp]
        L.orc_poisson.argtypes = [P] + [vp] * 8
        L.orc_poisson_series_direct.argtypes = [P] + [vp] * 6
        L.orc_density_grad_gather.argtypes = [P] + [vp] * 9
        L.orc_macro_grad_suffix.argtypes = [P] + [vp] * 9
        L.orc_density_grad_exact.argtypes = [P] + [vp] * 7
        L.orc_wirelength.argtypes = [P, vp, vp, vp, C.c_int, vp, vp, vp, vp, vp]
        L.orc_eval.argtypes = [P, vp, vp, vp, C.c_int, C.c_int, vp, vp, vp, vp]
        L.orc_filler_plan.argtypes = [P, vp, d, d, vp]
        L.orc_eval2d.argtypes = [P, vp, vp, vp, C.c_int, vp, vp, vp]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """Holds contiguous copies of a problem dict and calls the C oracle."""

    def __init__(self, prob: dict, alpha: float | None = None):
        self.p = prob
        f64 = lambda k: np.ascontiguousarray(prob[k], dtype=np.float64)
        self._keep = dict(
            is_macro=np.ascontiguousarray(prob["is_macro"], dtype=np.uint8),
            z_fixed=np.ascontiguousarray(prob["z_fixed"], dtype=np.uint8),
            net_start=np.ascontiguousarray(prob["net_start"], dtype=np.int32),
            pin_inst=np.ascontiguousarray(prob["pin_inst"], dtype=np.int32),
            is_hbt=(np.ascontiguousarray(prob["is_hbt"], dtype=np.uint8) if prob.get("is_hbt") is not None
                    else None),
            **{k: f64(k) for k in ("w_bot", "h_bot", "w_top", "h_top",
                                   "off_bx", "off_by", "off_tx", "off_ty")})
        k = self._keep
        self.geom = None
        self.s = Problem(
            int(prob["n_inst"]), _ptr(k["is_macro"]), _ptr(k["z_fixed"]),
            _ptr(k["w_bot"]), _ptr(k["h_bot"]), _ptr(k["w_top"]), _ptr(k["h_top"]),
            int(prob["n_net"]), int(prob["n_pin"]), _ptr(k["net_start"]), _ptr(k["pin_inst"]),
            _ptr(k["off_bx"]), _ptr(k["off_by"]), _ptr(k["off_tx"]), _ptr(k["off_ty"]),
            float(prob["xl"]), float(prob["yl"]), float(prob["xh"]), float(prob["yh"]),
            int(prob["nx"]), int(prob["ny"]), int(prob["nz"]),
            float(prob["gamma"]), float(prob.get("gamma_z", 0.0)), 0.0, float(prob["lam"]),
            _ptr(k["is_hbt"]), int(prob.get("mode", 0)),
            (C.c_double * 3)(*[float(v) for v in prob.get("lam_layer", (prob["lam"],) * 3)]))
        g = self.geometry()
        self.s.alpha = float(alpha) if alpha is not None else self.alpha_default()
        self.nb = int(prob["nx"]) * int(prob["ny"]) * int(prob["nz"])
        self.shape = (int(prob["nz"]), int(prob["ny"]), int(prob["nx"]))
        self.n = int(prob["n_inst"])
        del g

    # -- helpers --
    def geometry(self):
        out = np.zeros(6)
        lib().orc_geometry(C.byref(self.s), _ptr(out))
        return dict(wb=out[0], hb=out[1], db=out[2], dx=out[3], dy=out[4], dz=out[5])

    def alpha_default(self):
        g = self.geometry()
        p = self.p
        return lib().orc_alpha(g["dx"], g["dz"], p.get("beta", 10.0), p.get("w_hbt", 1.0),
                               p.get("rh_top", 0.8), p.get("rh_bot", 1.0))

    @property
    def alpha(self):
        return self.s.alpha

    @staticmethod
    def _xyz(x, y, z):
        return tuple(np.ascontiguousarray(a, dtype=np.float64) for a in (x, y, z))

    # -- steps --
    def attributes(self, x, y, z):
        x, y, z = self._xyz(x, y, z)
        n = self.n
        delta = np.zeros(n, np.int32)
        out = [np.zeros(n) for _ in range(5)]
        lib().orc_attributes(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), _ptr(delta),
                             *[_ptr(a) for a in out])
        return dict(delta=delta, w=out[0], h=out[1], sw=out[2], sh=out[3], omega=out[4])

    def filler_plan(self, z, u_top: float, u_bot: float) -> dict:
        """Eqs. filler-vol / free-filler-vol at initial depths z."""
        z = np.ascontiguousarray(z, dtype=np.float64)
        o = np.zeros(11)
        lib().orc_filler_plan(C.byref(self.s), _ptr(z), float(u_top), float(u_bot), _ptr(o))
        keys = ("vol_a", "vol_f_top", "vol_f_bot", "vol_fr", "w_top", "h_top", "w_bot", "h_bot")
        d = dict(zip(keys, o[:8].tolist()))
        d.update(n_top=int(o[8]), n_bot=int(o[9]), n_free=int(o[10]))
        return d

    def eval2d(self, x, y, z, density_mode: int = 1, grads: bool = True) -> dict:
        """Multi-die 2D objective and gradient (eq. 2d-place); the problem
        has mode = 1, nz = 3 and optionally is_hbt / lam_layer."""
        x, y, z = self._xyz(x, y, z)
        out = np.zeros(7)
        gx = np.zeros(self.n) if grads else None
        gy = np.zeros(self.n) if grads else None
        lib().orc_eval2d(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), int(density_mode), _ptr(out),
                         _ptr(gx), _ptr(gy))
        keys = ("obj", "wl", "e_bot", "e_top", "e_hbt", "hpwl_d2d", "n_cross")
        r = dict(zip(keys, out.tolist()))
        r["gx"], r["gy"] = gx, gy
        return r

    def density_direct(self, x, y, z):
        x, y, z = self._xyz(x, y, z)
        rho = np.zeros(self.shape)
        lib().orc_density_direct(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), _ptr(rho))
        return rho

    def macro_corner_map(self, x, y, z):
        x, y, z = self._xyz(x, y, z)
        A = np.zeros(self.shape)
        lib().orc_macro_corner_map(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), _ptr(A))
        return A

    @staticmethod
    def prefix_sum3(a):
        a = np.array(a, dtype=a.dtype, order="C", copy=True)
        nz, ny, nx = a.shape
        if a.dtype == np.int64:
            lib().orc_prefix_sum3_i64(_ptr(a), nx, ny, nz)
        else:
            a = a.astype(np.float64)
            lib().orc_prefix_sum3(_ptr(a), nx, ny, nz)
        return a

    def density_fixed(self, x, y, z, use_float: bool):
        x, y, z = self._xyz(x, y, z)
        q = np.zeros(self.shape, np.int64)
        lib().orc_density_fixed(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), int(use_float), _ptr(q))
        return q

    def poisson(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        outs = {k: np.zeros(self.shape) for k in ("a", "psi", "phi", "ex", "ey", "ez")}
        e = np.zeros(max(self.shape[0], 1))
        lib().orc_poisson(C.byref(self.s), _ptr(rho), *[_ptr(outs[k]) for k in
                                                         ("a", "psi", "phi", "ex", "ey", "ez")], _ptr(e))
        outs["energy"] = float(e[0])
        if self.s.mode == 1:
            outs["energy_layers"] = e.tolist()  # 2D mode: one energy per layer
        return outs

    def poisson_series_direct(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        outs = {k: np.zeros(self.shape) for k in ("a", "phi", "ex", "ey", "ez")}
        lib().orc_poisson_series_direct(C.byref(self.s), _ptr(rho),
                                        *[_ptr(outs[k]) for k in ("a", "phi", "ex", "ey", "ez")])
        return outs

    def density_grad_gather(self, x, y, z, ex, ey, ez):
        x, y, z = self._xyz(x, y, z)
        E = [np.ascontiguousarray(a, dtype=np.float64) for a in (ex, ey, ez)]
        g = [np.zeros(self.n) for _ in range(3)]
        lib().orc_density_grad_gather(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z),
                                      *[_ptr(a) for a in E], *[_ptr(a) for a in g])
        return g

    def macro_grad_suffix(self, x, y, z, ex, ey, ez):
        x, y, z = self._xyz(x, y, z)
        E = [np.ascontiguousarray(a, dtype=np.float64) for a in (ex, ey, ez)]
        g = [np.zeros(self.n) for _ in range(3)]
        lib().orc_macro_grad_suffix(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z),
                                    *[_ptr(a) for a in E], *[_ptr(a) for a in g])
        return g

    def density_grad_exact(self, x, y, z, phi):
        x, y, z = self._xyz(x, y, z)
        phi = np.ascontiguousarray(phi, dtype=np.float64)
        g = [np.zeros(self.n) for _ in range(3)]
        lib().orc_density_grad_exact(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), _ptr(phi),
                                     *[_ptr(a) for a in g])
        return g

    def wirelength(self, x, y, z, fd_mode: int = 1):
        x, y, z = self._xyz(x, y, z)
        out = np.zeros(4)
        g = [np.zeros(self.n) for _ in range(4)]
        lib().orc_wirelength(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), int(fd_mode), _ptr(out),
                             *[_ptr(a) for a in g])
        return dict(wl_bi=out[0], wl_z=out[1], hpwl_d2d=out[2], n_cross=out[3],
                    gx=g[0], gy=g[1], gfd=g[2], gwaz=g[3])

    def eval(self, x, y, z, density_mode: int = 1, fd_mode: int = 1, grads: bool = True):
        """density_mode: 0 direct FP64, 1 fixed-point (double), 2 fixed-point (float)."""
        x, y, z = self._xyz(x, y, z)
        out = np.zeros(10)
        g = [np.zeros(self.n) for _ in range(3)] if grads else [None] * 3
        lib().orc_eval(C.byref(self.s), _ptr(x), _ptr(y), _ptr(z), int(density_mode), int(fd_mode),
                       _ptr(out), *[_ptr(a) for a in g])
        keys = ("obj", "wl_bi", "wl_z", "energy", "hpwl_d2d", "n_cross", "g_scale", "Sx", "Sy", "Sz")
        r = {k: float(v) for k, v in zip(keys, out)}
        r["gx"], r["gy"], r["gz"] = g
        return r
