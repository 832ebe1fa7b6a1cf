"""Thin ctypes binding of libmd (include/md.h): argument marshalling only.

Every md_* function here has the name, arguments and meaning of the C function of the
same name; the `MD` class only bundles a handle with its sizes.  All computation runs
in the CUDA kernels of libmd.so; there is no CPU fallback: importing this module on a
machine without the built library or without a GPU raises.
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Optional, Sequence

import numpy as np

from . import build_lib

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS_JSON = os.path.join(HERE, "cr_c_params.json")

MD_OK, MD_ERR_ARG, MD_ERR_CUDA, MD_ERR_NBR_OVERFLOW, MD_ERR_SKIN_VIOLATION, MD_ERR_LOST_ATOM, MD_ERR_STATE = range(7)
MD_FP64, MD_MIXED = 0, 1
ERR_NAMES = {1: "MD_ERR_ARG", 2: "MD_ERR_CUDA", 3: "MD_ERR_NBR_OVERFLOW", 4: "MD_ERR_SKIN_VIOLATION",
             5: "MD_ERR_LOST_ATOM", 6: "MD_ERR_STATE"}


class md_params(C.Structure):
    _fields_ = [("r_e", C.c_double), ("f_e", C.c_double), ("beta", C.c_double),
                ("F_o", C.c_double), ("n", C.c_double), ("rho_e", C.c_double),
                ("alpha", C.c_double), ("P_e", C.c_double),
                ("a", C.c_double * 4), ("d", C.c_double),
                ("D_o", C.c_double), ("alpha_x", C.c_double), ("y_eq", C.c_double),
                ("rc", C.c_double), ("rc_morse", C.c_double),
                ("shifted", C.c_int32), ("tabulated", C.c_int32),
                ("r_min", C.c_double), ("h", C.c_double)]


class md_system(C.Structure):
    _fields_ = [("n_cr", C.c_int32), ("n_c", C.c_int32),
                ("x_cr", C.c_void_p), ("v_cr", C.c_void_p), ("x_c", C.c_void_p),
                ("fixed", C.c_void_p),
                ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("periodic", C.c_int32 * 3),
                ("z_indenter0", C.c_double), ("v_indenter", C.c_double), ("dt", C.c_double),
                ("mass_cr", C.c_double)]


class md_options(C.Structure):
    _fields_ = [("pot", C.POINTER(md_params)), ("precision", C.c_int32), ("skin", C.c_double),
                ("rebuild_every", C.c_int32), ("kmax", C.c_int32), ("kcmax", C.c_int32),
                ("tpa", C.c_int32), ("block", C.c_int32), ("use_graph", C.c_int32),
                ("inner_skin", C.c_double), ("debug_checks", C.c_int32)]


class md_energy(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("embed", "pair", "mterm", "morse", "kinetic", "potential", "total",
                                           "temperature", "load", "depth", "z_indenter")] + \
               [("step", C.c_int64), ("rebuilds", C.c_int64)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class md_phase_times(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("skin", "rebuild", "verlet1", "density", "morse", "force", "reduce")] + \
               [("steps", C.c_int64), ("rebuilds", C.c_int64)]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class MDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None
EXPORTS = ["md_init", "md_build_neighbors", "md_compute_forces", "md_step", "md_step_profiled",
           "md_get_energy", "md_get_forces", "md_get_indenter_load", "md_get_state", "md_set_state",
           "md_get_neighbors", "md_get_info", "md_last_error", "md_free", "md_version", "md_forces_small",
           "md_set_indenter_velocity", "md_get_virial", "md_probe_fp64_fma", "md_check_lists", "md_step_io"]


def lib(build: bool = True):
    """Load libmd.so (building it first when its sources are newer); raises when it cannot."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        build_lib.build()
    if not os.path.exists(build_lib.LIB):
        raise RuntimeError(f"libmd.so not built ({build_lib.LIB}); run paper_1507_07068_gb300.build_lib.build()")
    L = C.CDLL(build_lib.LIB)
    vp = C.c_void_p
    L.md_init.argtypes = [C.POINTER(md_system), C.c_int32, C.POINTER(md_options), vp, C.POINTER(vp)]
    L.md_build_neighbors.argtypes = [vp]
    L.md_compute_forces.argtypes = [vp]
    L.md_step.argtypes = [vp, C.c_int64]
    L.md_step_profiled.argtypes = [vp, C.c_int64, C.POINTER(md_phase_times)]
    L.md_get_energy.argtypes = [vp, C.c_int32, C.POINTER(md_energy)]
    L.md_get_forces.argtypes = [vp, C.c_int32, vp]
    L.md_get_indenter_load.argtypes = [vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.md_get_state.argtypes = [vp, C.c_int32, vp, vp, vp, vp]
    L.md_set_state.argtypes = [vp, C.c_int32, vp, vp, C.c_double, C.c_int64]
    L.md_step_io.argtypes = [vp, C.c_int32, vp, vp, C.c_double, C.c_int64, C.c_int64, vp, vp, C.POINTER(md_energy)]
    L.md_set_indenter_velocity.argtypes = [vp, C.c_int32, C.c_double]
    L.md_get_virial.argtypes = [vp, C.c_int32, vp]
    L.md_probe_fp64_fma.argtypes = [vp, vp]
    L.md_get_neighbors.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp, C.c_int32]
    L.md_get_info.argtypes = [vp, vp]
    L.md_check_lists.argtypes = [vp, C.c_double, vp]
    L.md_last_error.argtypes = [vp]
    L.md_last_error.restype = C.c_char_p
    L.md_free.argtypes = [vp]
    L.md_free.restype = None
    L.md_version.restype = C.c_int
    L.md_forces_small.argtypes = [C.POINTER(md_params), C.c_int32, vp, C.c_int32, vp, C.POINTER(C.c_double),
                                  C.POINTER(C.c_double), C.POINTER(C.c_int32), vp, vp, vp, C.c_char_p, C.c_size_t]
    for name in EXPORTS:
        if name not in ("md_last_error", "md_free", "md_version"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def load_params(path: Optional[str] = None) -> dict:
    with open(path or PARAMS_JSON) as fh:
        return json.load(fh)


def make_params(p: dict, **override) -> md_params:
    q = dict(p)
    q.update(override)
    st = md_params()
    for name in ("r_e", "f_e", "beta", "F_o", "n", "rho_e", "alpha", "P_e", "d", "D_o", "alpha_x", "y_eq",
                 "r_min", "h"):
        setattr(st, name, float(q[name]))
    st.a[:] = [float(q["a0"]), float(q["a1"]), float(q["a2"]), float(q["a3"])]
    st.rc = float(q["rc"])
    st.rc_morse = float(q.get("rc_morse", q.get("rc_m")))
    st.shifted = int(q["shifted"])
    st.tabulated = int(q["tabulated"])
    return st


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(h, code: int):
    if code != MD_OK:
        msg = lib().md_last_error(h)
        raise MDError(code, msg.decode() if msg else "")


def current_stream() -> int:
    """cudaStream_t of torch's current stream (PyTorch provides the stream)."""
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libmd needs a CUDA GPU; torch.cuda.is_available() is False")
    return int(torch.cuda.current_stream().cuda_stream)


# ----------------------------------------------------------------------------- same-name calls

def md_init(systems: Sequence[md_system], options: md_options, stream: int):
    arr = (md_system * len(systems))(*systems)
    h = C.c_void_p()
    rc = lib().md_init(arr, len(systems), C.byref(options), C.c_void_p(stream), C.byref(h))
    _check(None, rc)
    return h


def md_build_neighbors(h):
    _check(h, lib().md_build_neighbors(h))


def md_compute_forces(h):
    _check(h, lib().md_compute_forces(h))


def md_step(h, n: int):
    _check(h, lib().md_step(h, int(n)))


def md_step_profiled(h, n: int) -> dict:
    t = md_phase_times()
    _check(h, lib().md_step_profiled(h, int(n), C.byref(t)))
    return t.as_dict()


def md_get_energy(h, replica: int = 0) -> dict:
    e = md_energy()
    _check(h, lib().md_get_energy(h, int(replica), C.byref(e)))
    return e.as_dict()


def md_get_forces(h, replica: int, n_cr: int, out: Optional[np.ndarray] = None) -> np.ndarray:
    out = np.empty((n_cr, 3)) if out is None else out
    _check(h, lib().md_get_forces(h, int(replica), _ptr(out)))
    return out


def md_get_indenter_load(h, replica: int = 0):
    l = C.c_double(); d = C.c_double()
    _check(h, lib().md_get_indenter_load(h, int(replica), C.byref(l), C.byref(d)))
    return l.value, d.value


def md_get_state(h, replica: int, n_cr: int, x: Optional[np.ndarray] = None, v: Optional[np.ndarray] = None):
    x = np.empty((n_cr, 3)) if x is None else x
    v = np.empty((n_cr, 3)) if v is None else v
    z = C.c_double(); st = C.c_int64()
    _check(h, lib().md_get_state(h, int(replica), _ptr(x), _ptr(v), C.cast(C.pointer(z), C.c_void_p),
                                 C.cast(C.pointer(st), C.c_void_p)))
    return x, v, z.value, st.value


def md_set_state(h, replica: int, x: Optional[np.ndarray], v: Optional[np.ndarray], z_ind: float, step: int):
    _check(h, lib().md_set_state(h, int(replica), _ptr(x), _ptr(v), float(z_ind), int(step)))


def md_step_io(h, replica: int, x: np.ndarray, v: np.ndarray, z_ind: float, step: int, n: int = 1,
               x_out: Optional[np.ndarray] = None, v_out: Optional[np.ndarray] = None):
    """md_step_io: set replica's state, advance n steps, read its state back; returns
    (x_out, v_out, energy dict).  x_out, v_out may be x, v."""
    x_out = np.empty_like(x) if x_out is None else x_out
    v_out = np.empty_like(v) if v_out is None else v_out
    for a in (x, v, x_out, v_out):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != x.shape:
            raise ValueError("md_step_io: C-contiguous float64 arrays of one shape (n, 3)")
    e = md_energy()
    _check(h, lib().md_step_io(h, int(replica), _ptr(x), _ptr(v), float(z_ind), int(step), int(n),
                               _ptr(x_out), _ptr(v_out), C.byref(e)))
    return x_out, v_out, e.as_dict()


def md_get_virial(h, replica: int, n_cr: int, out: Optional[np.ndarray] = None):
    out = np.empty((n_cr, 6)) if out is None else out
    _check(h, lib().md_get_virial(h, int(replica), _ptr(out)))
    return out


def md_probe_fp64_fma() -> float:
    """FP64 FMA rate of the current device's CUDA cores (flop/s, 2 per FMA)."""
    f = C.c_double(); ms = C.c_double()
    code = lib().md_probe_fp64_fma(C.cast(C.pointer(f), C.c_void_p), C.cast(C.pointer(ms), C.c_void_p))
    if code != MD_OK:
        raise MDError(code, "md_probe_fp64_fma failed")
    return f.value


def md_set_indenter_velocity(h, replica: int, v_ind: float):
    _check(h, lib().md_set_indenter_velocity(h, int(replica), float(v_ind)))


def md_get_neighbors(h, replica: int, which: int, n_cr: int, kmax: int):
    cell = np.zeros((n_cr, 3), np.int32)
    cnt = np.zeros(n_cr, np.int32)
    nbr = np.full((n_cr, kmax), -1, np.int32)
    _check(h, lib().md_get_neighbors(h, int(replica), int(which), _ptr(cell), _ptr(cnt), _ptr(nbr), int(kmax)))
    return cell, cnt, nbr


def md_get_info(h) -> dict:
    out = np.zeros(9, np.int64)
    _check(h, lib().md_get_info(h, _ptr(out)))
    keys = ("replicas", "n_cr", "n_c", "slots", "cells", "kmax", "kcmax", "max_cnt", "max_cntc")
    return dict(zip(keys, (int(v) for v in out)))


CHECK_KINDS = ("out_of_range", "over_capacity", "wrong_direction", "beyond_radius", "missing", "one_way",
               "bad_cr_c", "inner_not_in_verlet")


def md_check_lists(h, radius: float = 0.0) -> dict:
    out = np.zeros(8, np.int64)
    _check(h, lib().md_check_lists(h, float(radius), _ptr(out)))
    return dict(zip(CHECK_KINDS, (int(v) for v in out)))


def md_free(h):
    if h:
        lib().md_free(h)


def md_last_error(h=None) -> str:
    msg = lib().md_last_error(h)
    return msg.decode() if msg else ""


def md_version() -> int:
    return int(lib().md_version())


MD_SMALL_MAX_ATOMS = 16384


def md_forces_small(params: md_params, n_cr: int, x_cr: int, n_c: int, x_c: Optional[int], box_lo, box_hi,
                    periodic, F: int, energy: int, stream: int = 0):
    """The allocation-free entry point.  x_cr, x_c, F and energy are device addresses of
    caller-owned buffers (x_cr, F: n_cr x 3 doubles; x_c: n_c x 3; energy: 4 doubles)."""
    lo = (C.c_double * 3)(*[float(t) for t in box_lo])
    hi = (C.c_double * 3)(*[float(t) for t in box_hi])
    per = (C.c_int32 * 3)(*[int(t) for t in periodic])
    msg = C.create_string_buffer(256)
    rc = lib().md_forces_small(C.byref(params), int(n_cr), x_cr, int(n_c), x_c, lo, hi, per, F, energy,
                               C.c_void_p(stream), msg, len(msg))
    if rc != MD_OK:
        raise MDError(rc, msg.value.decode())


# ----------------------------------------------------------------------------- convenience

def system_from(rep) -> tuple:
    """md_system for an object with x_cr, v_cr, fixed, x_c, box_lo, box_hi, periodic,
    z_indenter0, v_indenter, dt, mass_cr; returns (struct, arrays kept alive)."""
    x = np.ascontiguousarray(rep.x_cr, np.float64)
    v = np.ascontiguousarray(rep.v_cr, np.float64)
    xc = np.ascontiguousarray(rep.x_c, np.float64).reshape(-1, 3)
    fx = np.ascontiguousarray(rep.fixed, np.uint8)
    s = md_system()
    s.n_cr = len(x); s.n_c = len(xc)
    s.x_cr = _ptr(x); s.v_cr = _ptr(v); s.x_c = _ptr(xc) if len(xc) else None; s.fixed = _ptr(fx)
    s.box_lo[:] = [float(t) for t in rep.box_lo]
    s.box_hi[:] = [float(t) for t in rep.box_hi]
    s.periodic[:] = [int(t) for t in rep.periodic]
    s.z_indenter0 = float(rep.z_indenter0); s.v_indenter = float(rep.v_indenter)
    s.dt = float(rep.dt); s.mass_cr = float(rep.mass_cr)
    return s, (x, v, xc, fx)


class MD:
    """One libmd handle over a list of replicas."""

    def __init__(self, replicas, params: Optional[dict] = None, precision: str = "mixed", skin: float = 0.3,
                 rebuild_every: int = 0, kmax: int = 0, kcmax: int = 0, tpa: int = 0, block: int = 0,
                 use_graph: bool = True, stream: Optional[int] = None, inner_skin: float = 0.0,
                 debug_checks: bool = False, **pot_override):
        self.replicas = list(replicas)
        self.n = [r.n_cr for r in self.replicas]
        self._params = make_params(params or load_params(), **pot_override)
        systems, self._keep = [], []
        for r in self.replicas:
            s, keep = system_from(r)
            systems.append(s); self._keep.append(keep)
        opt = md_options()
        opt.pot = C.pointer(self._params)
        opt.precision = MD_MIXED if precision == "mixed" else MD_FP64
        opt.skin = float(skin); opt.rebuild_every = int(rebuild_every)
        opt.kmax = int(kmax); opt.kcmax = int(kcmax); opt.tpa = int(tpa); opt.block = int(block)
        opt.use_graph = 1 if use_graph else 0
        opt.inner_skin = float(inner_skin)
        opt.debug_checks = 1 if debug_checks else 0
        self._opt = opt
        self.stream = current_stream() if stream is None else int(stream)
        self.h = md_init(systems, opt, self.stream)
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            md_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n: int = 1):
        md_step(self.h, n)

    def step_profiled(self, n: int) -> dict:
        return md_step_profiled(self.h, n)

    def build_neighbors(self):
        md_build_neighbors(self.h)

    def compute_forces(self):
        md_compute_forces(self.h)

    def energy(self, r: int = 0) -> dict:
        return md_get_energy(self.h, r)

    def forces(self, r: int = 0) -> np.ndarray:
        return md_get_forces(self.h, r, self.n[r])

    def state(self, r: int = 0):
        return md_get_state(self.h, r, self.n[r])

    def set_state(self, r: int, x, v, z_ind: float, step: int):
        x = None if x is None else np.ascontiguousarray(x, np.float64)
        v = None if v is None else np.ascontiguousarray(v, np.float64)
        md_set_state(self.h, r, x, v, z_ind, step)

    def step_io(self, r: int, x, v, z_ind: float, step: int, n: int = 1, x_out=None, v_out=None):
        """Set replica r's state, advance every replica n steps, return r's (x, v, energies)."""
        x = np.ascontiguousarray(x, np.float64)
        v = np.ascontiguousarray(v, np.float64)
        if x.shape != (self.n[r], 3):
            raise ValueError(f"step_io: x must be ({self.n[r]}, 3)")
        return md_step_io(self.h, r, x, v, z_ind, step, n, x_out, v_out)

    def virial(self, r: int = 0):
        """Per-atom virial (n, 6: xx, yy, zz, xy, xz, yz; eV) of replica r."""
        return md_get_virial(self.h, r, self.n[r])

    def set_indenter_velocity(self, r: int, v_ind: float):
        md_set_indenter_velocity(self.h, r, v_ind)

    def neighbors(self, r: int = 0, which: int = 0, kmax: Optional[int] = None):
        info = md_get_info(self.h)
        k = kmax or (info["kcmax"] if which else info["kmax"])
        return md_get_neighbors(self.h, r, which, self.n[r], k)

    def info(self) -> dict:
        return md_get_info(self.h)

    def check_lists(self, radius: float = 0.0) -> dict:
        return md_check_lists(self.h, radius)
