"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and by
the benchmark's CPU-baseline leg; never by the library product.  The oracle is a
plain, slow FP64 restatement of the paper's method (Appendix Eqs. A1-A13, Eq. (1),
Sec. 2.1 Tasks 1-5, Sec. 2.6, Fig. 5); see oracle.c for what each function follows.

Parity status of each oracle function (what pins it, in tests/test_oracle_*.py):
  potential functions f, Phi, phi, F, M ... closed forms A6-A9, finite differences,
                                            Hermite error bound, special cases
  neighbour sets ........................ brute force == cell list; symmetry
  energies and forces .................... -grad E by central differences per term;
                                            Newton's third law; BCC closed form
                                            (E = -E_c, dE/da = 0, F = 0); dimer
  time loop .............................. time reversibility, NVE conservation,
                                            momentum conservation, indenter travel
The physical outputs of Sec. 4.3 (load, modulus, hardness) stay unpinned: the
potential parameters of the paper's refs. [42] and [34] are not printed.
"""
from __future__ import annotations

import ctypes as C
import json
import os
import subprocess
import threading
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")
# optimisation levels the oracle is built at: -O2 as the paper's own build (Sec. 2.3),
# -O3 beside it for the CPU baseline (no -march=native: one build serves x86 and Arm hosts)
OPT_LIBS = {"O2": LIB, "O3": os.path.join(HERE, "liboracle_O3.so")}

_lock = threading.Lock()
_lib = None
_libs = {}
_opt = "O2"

OR_F, OR_PHI, OR_MORSE, OR_EMBED, OR_MTERM, OR_F_RAW, OR_PHI_AN, OR_MORSE_RAW = range(8)


class OrParams(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("r_e", "f_e", "beta", "F_o", "n", "rho_e", "alpha", "P_e",
                 "a0", "a1", "a2", "a3", "d", "D_o", "alpha_x", "y_eq", "rc", "rc_m")] + \
               [("shifted", C.c_int32), ("tabulated", C.c_int32), ("r_min", C.c_double), ("h", C.c_double)]


def build(force: bool = False, opt: str = "O2") -> str:
    """Compile oracle.c into liboracle.so (-O2) or liboracle_O3.so (-O3): gcc, FP64, no FMA
    contraction, OpenMP if available."""
    out = OPT_LIBS[opt]
    with _lock:
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
            return out
        base = ["gcc", "-" + opt, "-std=c99", "-ffp-contract=off", "-fPIC", "-shared", SRC, "-o", out + ".tmp", "-lm"]
        try:
            subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
        except subprocess.CalledProcessError:
            subprocess.run(base, check=True, capture_output=True)
        os.replace(out + ".tmp", out)
        return out


def select(opt: str) -> None:
    """Use the oracle built at -O2 (default) or -O3 for the objects created from now on."""
    global _lib, _opt
    if opt not in OPT_LIBS:
        raise ValueError(opt)
    _opt, _lib = opt, _libs.get(opt)


def lib():
    global _lib
    if _lib is None:
        if _opt in _libs:
            _lib = _libs[_opt]
            return _lib
        path = build(opt=_opt)
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        L.or_pot_new.restype = C.c_void_p
        L.or_pot_new.argtypes = [C.POINTER(OrParams)]
        L.or_pot_free.argtypes = [C.c_void_p]
        L.or_eval.restype = C.c_int
        L.or_eval.argtypes = [C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.or_neumaier.restype = C.c_double
        L.or_neumaier.argtypes = [dp, C.c_int64]
        L.or_grid.restype = C.c_int
        L.or_grid.argtypes = [dp, dp, ip, C.c_double, ip, dp]
        L.or_cell_coords.restype = C.c_int
        L.or_cell_coords.argtypes = [C.c_int32, dp, dp, dp, ip, C.c_double, ip]
        L.or_neighbors.restype = C.c_int64
        L.or_neighbors.argtypes = [C.c_int32, dp, dp, dp, ip, C.c_double, C.c_int32, lp, ip, C.c_int64,
                                   C.POINTER(C.c_int64)]
        L.or_cneighbors.restype = C.c_int64
        L.or_cneighbors.argtypes = [C.c_int32, dp, C.c_int32, dp, dp, dp, ip, C.c_double, lp, ip, C.c_int64,
                                    C.POINTER(C.c_int64)]
        L.or_forces.restype = C.c_int
        L.or_forces.argtypes = [C.c_void_p, C.c_int32, dp, dp, dp, ip, C.c_int32, dp, C.c_int32,
                                dp, dp, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_sim_new.restype = C.c_void_p
        L.or_sim_new.argtypes = [C.c_void_p, C.c_int32, dp, dp, up, C.c_int32, dp, dp, dp, ip,
                                 C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_int32]
        L.or_sim_free.argtypes = [C.c_void_p]
        L.or_sim_set_v_ind.argtypes = [C.c_void_p, C.c_double]
        L.or_sim_virial.restype = C.c_int
        L.or_sim_virial.argtypes = [C.c_void_p, dp]
        L.or_forces_given.restype = C.c_int
        L.or_forces_given.argtypes = [C.c_void_p, C.c_int32, dp, dp, dp, ip, C.c_int32, dp, up, dp, dp, dp, dp, dp]
        L.or_virial.restype = C.c_int
        L.or_virial.argtypes = [C.c_void_p, C.c_int32, dp, dp, dp, ip, C.c_int32, dp, C.c_int32, dp, dp, dp]
        L.or_sim_step.restype = C.c_int
        L.or_sim_step.argtypes = [C.c_void_p, C.c_int64]
        L.or_sim_get.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_sim_list.restype = C.c_int64
        L.or_sim_list.argtypes = [C.c_void_p, C.c_int32, lp, ip, C.c_int64]
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int32]
        _lib = _libs[_opt] = L
    return _lib


def set_threads(n: int) -> int:
    """Set the OpenMP thread count (0 = leave); returns the count in use."""
    return int(lib().or_set_threads(int(n)))


def _arr(a, dt=np.float64):
    return np.ascontiguousarray(np.asarray(a, dtype=dt))


def load_params(path: Optional[str] = None) -> dict:
    """The derived parameter set shipped with the package (a JSON file written by derive_params.py)."""
    if path is None:
        path = os.path.join(os.path.dirname(HERE), "paper_1507_07068_gb300", "cr_c_params.json")
    with open(path) as fh:
        return json.load(fh)


class Potential:
    """The oracle's potential functions with a given parameter dict."""

    def __init__(self, params: dict, **override):
        p = dict(params)
        p.update(override)
        self.params = p
        st = OrParams()
        for name, _ in OrParams._fields_:
            setattr(st, name, int(p[name]) if name in ("shifted", "tabulated") else float(p[name]))
        self._st = st
        self._L = lib()   # the build (-O2 / -O3) this potential belongs to
        self.h = self._L.or_pot_new(C.byref(st))
        if not self.h:
            raise MemoryError("or_pot_new failed")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._L.or_pot_free(self.h)
                self.h = None
        except Exception:
            pass

    def eval(self, which: int, x: float):
        v = C.c_double(); d = C.c_double()
        if self._L.or_eval(self.h, int(which), float(x), C.byref(v), C.byref(d)):
            raise ValueError(which)
        return v.value, d.value

    def evalv(self, which: int, xs: Sequence[float]):
        out = np.array([self.eval(which, float(x)) for x in xs])
        return out[:, 0], out[:, 1]


def neumaier(x) -> float:
    x = _arr(x)
    return float(lib().or_neumaier(x, x.size))


def grid(lo, hi, periodic, cut):
    n = np.zeros(3, np.int32); w = np.zeros(3)
    err = lib().or_grid(_arr(lo), _arr(hi), _arr(periodic, np.int32), float(cut), n, w)
    if err:
        raise ValueError(f"or_grid: {err}")
    return n, w


def cell_coords(x, lo, hi, periodic, cut) -> np.ndarray:
    x = _arr(x).reshape(-1, 3)
    out = np.zeros((len(x), 3), np.int32)
    if lib().or_cell_coords(len(x), x, _arr(lo), _arr(hi), _arr(periodic, np.int32), float(cut), out):
        raise ValueError("or_cell_coords")
    return out


def _csr_call(fn, n, *args):
    cap = 64 * max(n, 1)
    while True:
        off = np.zeros(n + 1, np.int64); idx = np.zeros(max(cap, 1), np.int32); need = C.c_int64()
        tot = fn(*args, off, idx, cap, C.byref(need))
        if tot >= 0:
            return off, idx[:tot].copy()
        if need.value <= cap:
            raise RuntimeError("oracle neighbour build failed")
        cap = int(need.value)


def neighbors(x, lo, hi, periodic, cut, method: int = 1):
    """CSR (off, idx) of all j != i within `cut` (method 0 brute force, 1 cell list)."""
    x = _arr(x).reshape(-1, 3)
    return _csr_call(lib().or_neighbors, len(x), len(x), x, _arr(lo), _arr(hi), _arr(periodic, np.int32),
                     float(cut), int(method))


def cneighbors(x, xc, lo, hi, periodic, cut):
    x = _arr(x).reshape(-1, 3); xc = _arr(xc).reshape(-1, 3)
    return _csr_call(lib().or_cneighbors, len(x), len(x), x, len(xc), xc if len(xc) else np.zeros(3),
                     _arr(lo), _arr(hi), _arr(periodic, np.int32), float(cut))


def forces(pot: Potential, x, lo, hi, periodic, xc=None, method: int = 1, want_atoms: bool = False):
    """Stateless evaluation: returns dict with F (n,3), energy components, load (and rho, P, e_atom)."""
    x = _arr(x).reshape(-1, 3)
    xc = np.zeros((0, 3)) if xc is None else _arr(xc).reshape(-1, 3)
    n = len(x)
    F = np.zeros((n, 3)); ep = np.zeros(5)
    rho = np.zeros(n) if want_atoms else None
    P = np.zeros(n) if want_atoms else None
    ea = np.zeros(n) if want_atoms else None
    ptr = lambda a: a.ctypes.data_as(C.c_void_p) if a is not None else None
    err = pot._L.or_forces(pot.h, n, x, _arr(lo), _arr(hi), _arr(periodic, np.int32), len(xc),
                          xc if len(xc) else np.zeros(3), int(method), F, ep, ptr(rho), ptr(P), ptr(ea))
    if err:
        raise RuntimeError(f"or_forces: {err}")
    out = dict(F=F, embed=ep[0], pair=ep[1], mterm=ep[2], morse=ep[3], load=ep[4],
               potential=ep[0] + ep[1] + ep[2] + ep[3])
    if want_atoms:
        out.update(rho=rho, P=P, e_atom=ea)
    return out


def forces_given(pot: Potential, x, lo, hi, periodic, xc=None, given=None, fm_in=None):
    """The two passes of Task 4 with an exchange between them (the paper's F', M'
    Allgatherv, Sec. 3.3.2): returns F, fm (F'(rho_i), M'(P_i) from this call's own first
    pass, (n, 2)), the per-atom energies and the energy sums; atoms with given[i] != 0 enter
    the second pass with fm_in[i] instead of their own first-pass values."""
    x = _arr(x).reshape(-1, 3)
    xc = np.zeros((0, 3)) if xc is None else _arr(xc).reshape(-1, 3)
    n = len(x)
    g = np.zeros(n, np.uint8) if given is None else _arr(given, np.uint8)
    fin = np.zeros((n, 2)) if fm_in is None else _arr(fm_in).reshape(n, 2)
    F = np.zeros((n, 3)); ep = np.zeros(5); fm = np.zeros((n, 2)); ea = np.zeros(n)
    err = pot._L.or_forces_given(pot.h, n, x, _arr(lo), _arr(hi), _arr(periodic, np.int32), len(xc),
                                xc if len(xc) else np.zeros(3), g, fin, fm, F, ep, ea)
    if err:
        raise RuntimeError(f"or_forces_given: {err}")
    return dict(F=F, fm=fm, e_atom=ea, embed=ep[0], pair=ep[1], mterm=ep[2], morse=ep[3], load=ep[4])


def virial(pot: Potential, x, lo, hi, periodic, xc=None, method: int = 1):
    """Per-atom virial (n, 6: xx, yy, zz, xy, xz, yz) at the given positions: each pair term
    c (x_j - x_i) (x) (x_j - x_i) with c = (dE/dr) / r, half to each atom of the pair (a Cr-C
    pair's half to the Cr atom).  Also returns the forces and energies of `forces`."""
    x = _arr(x).reshape(-1, 3)
    xc = np.zeros((0, 3)) if xc is None else _arr(xc).reshape(-1, 3)
    n = len(x)
    F = np.zeros((n, 3)); ep = np.zeros(5); W = np.zeros((n, 6))
    err = pot._L.or_virial(pot.h, n, x, _arr(lo), _arr(hi), _arr(periodic, np.int32), len(xc),
                          xc if len(xc) else np.zeros(3), int(method), F, ep, W)
    if err:
        raise RuntimeError(f"or_virial: {err}")
    return dict(W=W, F=F, embed=ep[0], pair=ep[1], mterm=ep[2], morse=ep[3], load=ep[4],
                potential=ep[0] + ep[1] + ep[2] + ep[3])


class Sim:
    """Oracle time loop (Fig. 5): Verlet lists with skin, Tasks 1-5 per step."""

    def __init__(self, pot: Potential, rep, skin: float = 0.3, rebuild_every: int = 0, method: int = 1,
                 x=None, v=None):
        self.pot = pot
        self.n = rep.n_cr
        self.nc = rep.n_c
        self._keep = [pot]
        x = _arr(rep.x_cr if x is None else x).reshape(-1, 3)
        v = _arr(rep.v_cr if v is None else v).reshape(-1, 3)
        xc = _arr(rep.x_c).reshape(-1, 3) if rep.n_c else np.zeros((1, 3))
        self._L = pot._L
        self.h = self._L.or_sim_new(pot.h, self.n, x, v, _arr(rep.fixed, np.uint8), self.nc, xc,
                                  _arr(rep.box_lo), _arr(rep.box_hi), _arr(rep.periodic, np.int32),
                                  float(rep.z_indenter0), float(rep.v_indenter), float(rep.dt),
                                  float(rep.mass_cr), float(skin), int(rebuild_every), int(method))
        if not self.h:
            raise RuntimeError("or_sim_new failed")

    def __del__(self):
        try:
            if getattr(self, "h", None):
                self._L.or_sim_free(self.h)
                self.h = None
        except Exception:
            pass

    def step(self, n: int = 1):
        if self._L.or_sim_step(self.h, int(n)):
            raise RuntimeError("or_sim_step failed")

    def set_indenter_velocity(self, v_ind: float):
        self._L.or_sim_set_v_ind(self.h, float(v_ind))

    def virial(self):
        """Per-atom virial (n, 6: xx, yy, zz, xy, xz, yz) of the current state."""
        W = np.zeros((self.n, 6))
        if self._L.or_sim_virial(self.h, W):
            raise RuntimeError("or_sim_virial failed")
        return W

    def state(self):
        x = np.zeros((self.n, 3)); v = np.zeros((self.n, 3)); F = np.zeros((self.n, 3))
        e = np.zeros(8); z = np.zeros(1); cnt = np.zeros(2, np.int64)
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        self._L.or_sim_get(self.h, p(x), p(v), p(F), p(e), p(z), p(cnt))
        return dict(x=x, v=v, F=F, embed=e[0], pair=e[1], mterm=e[2], morse=e[3], kinetic=e[4],
                    potential=e[5], total=e[6], load=e[7], z_ind=z[0], step=int(cnt[0]), rebuilds=int(cnt[1]))

    def verlet_list(self, which: int = 0):
        cap = 128 * max(self.n, 1)
        off = np.zeros(self.n + 1, np.int64); idx = np.zeros(cap, np.int32)
        tot = self._L.or_sim_list(self.h, int(which), off, idx, cap)
        if tot < 0:
            raise RuntimeError("list capacity")
        return off, idx[:tot].copy()
