"""ctypes wrapper of the FP64 CPU oracle (misa_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and
by the CPU-baseline / reference leg of bench.py, never by the library.  It
shares no code with the CUDA path.  build() compiles the C source with gcc
(OpenMP when available) into oracle/liboracle.so.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "misa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle; tries OpenMP first, then a serial build."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", _LIB, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.or_spline_slopes.argtypes = [_D, C.c_int, C.c_double, _D]
        L.or_spline_eval.argtypes = [_D, _D, C.c_int, C.c_double, C.c_double, _D]
        L.or_spline_eval.restype = C.c_double
        L.or_spline_weights.argtypes = [C.c_int, C.c_double, C.c_double, _I32, _D, _D]
        L.or_pot_new.argtypes = [C.c_int, C.c_double, C.c_double, _D, _D, _D]
        L.or_pot_new.restype = C.c_void_p
        L.or_pot_free.argtypes = [C.c_void_p]
        L.or_pot_eval.argtypes = [C.c_void_p, C.c_int, C.c_double, _D]
        L.or_pot_eval.restype = C.c_double
        L.or_site_index.argtypes = [C.c_int] * 5
        L.or_site_index.restype = C.c_int64
        L.or_site_position.argtypes = [C.c_int, C.c_int, C.c_double, C.c_int64, _D]
        L.or_nearest_site.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _D]
        L.or_nearest_site.restype = C.c_int64
        L.or_pka_site.argtypes = [C.c_int, C.c_int, C.c_int]
        L.or_pka_site.restype = C.c_int64
        L.or_alloy_new.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _D, _D, _D]
        L.or_alloy_new.restype = C.c_void_p
        L.or_alloy_free.argtypes = [C.c_void_p]
        L.or_eam_alloy.argtypes = [C.c_void_p, C.c_int64, _D, C.c_void_p, _D, C.c_int, C.c_int, _D, _D, _D, _D]
        L.or_ws_defects.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64, _D,
                                    C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.or_eam.argtypes = [C.c_void_p, C.c_int64, _D, _D, C.c_int, C.c_int, _D, _D, _D, _D]
        L.or_eam_sample.argtypes = [C.c_void_p, C.c_int64, _D, _D, C.c_int, C.c_int64, _I64, _D, _D, _D]
        L.or_pair_list.argtypes = [C.c_int64, _D, _D, C.c_double, C.c_int, C.c_int64, _I64, _I64, _D]
        L.or_pair_list.restype = C.c_int64
        L.or_next_dt.argtypes = [C.c_int64, _D, C.c_double, C.c_double]
        L.or_next_dt.restype = C.c_double
        L.or_insert_pka.argtypes = [_D, C.c_int64, C.c_double, C.c_double, _D]
        L.or_kinetic.argtypes = [C.c_int64, _D, C.c_double]
        L.or_kinetic.restype = C.c_double
        L.or_md_run.argtypes = [C.c_void_p, C.c_int64, _D, _D, _D, C.c_int, _D, C.c_double, C.c_double,
                                C.c_double, C.c_int, C.c_int, C.c_int, _D]
        L.or_md_run.restype = C.c_double
        L.or_lattice_new.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double]
        L.or_lattice_new.restype = C.c_void_p
        L.or_lattice_free.argtypes = [C.c_void_p]
        L.or_lattice_assign.argtypes = [C.c_void_p, C.c_int64, _D]
        L.or_lattice_update.argtypes = [C.c_void_p, C.c_int64, _D]
        L.or_lattice_site_atom.argtypes = [C.c_void_p, _I64]
        L.or_lattice_site_atom.restype = C.c_int64
        L.or_lattice_runaways.argtypes = [C.c_void_p, _I64]
        L.or_lattice_runaways.restype = C.c_int64
        L.or_lattice_pairs.argtypes = [C.c_void_p, _D, C.c_double, C.c_int64, _I64, _I64, _D]
        L.or_lattice_pairs.restype = C.c_int64
        L.or_offsets.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int, _I32]
        L.or_offsets.restype = C.c_int
        L.or_loss_grad.argtypes = [C.c_void_p, C.c_int64, _D, _D, C.c_int, _D, C.c_double, _D, _D, _D]
        L.or_loss_grad.restype = C.c_double
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D)


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().or_num_threads())


# ---------------------------------------------------------------------------
# spline
# ---------------------------------------------------------------------------

def spline_slopes(y, h):
    y = _c64(y)
    m = np.empty_like(y)
    lib().or_spline_slopes(_d(y), len(y), h, _d(m))
    return m


def spline_eval(y, h, x):
    """Value and derivative of the knot spline at each x."""
    y = _c64(y)
    m = spline_slopes(y, h)
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    v = np.empty_like(xs)
    dv = np.empty_like(xs)
    d = C.c_double()
    for q, xq in enumerate(xs):
        v[q] = lib().or_spline_eval(_d(y), _d(m), len(y), h, float(xq), C.byref(d))
        dv[q] = d.value
    return v, dv


def spline_weights(n, h, x):
    idx = (C.c_int * 8)()
    w = np.zeros(8)
    dw = np.zeros(8)
    c = lib().or_spline_weights(n, h, float(x), idx, _d(w), _d(dw))
    return np.array(idx[:c]), w[:c], dw[:c]


# ---------------------------------------------------------------------------
# potential
# ---------------------------------------------------------------------------

class Pot:
    """Three spline tables: f(r), phi(r) on [0, rc], F(rho) on [0, rho_max]."""

    def __init__(self, pot):
        self.n, self.rc, self.rho_max = pot.n, pot.rc, pot.rho_max
        self._keep = [_c64(pot.f), _c64(pot.phi), _c64(pot.F)]
        self.h = lib().or_pot_new(pot.n, pot.rc, pot.rho_max, *[_d(a) for a in self._keep])
        if not self.h:
            raise ValueError("bad potential tables")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_pot_free(self.h)
            self.h = None

    def eval(self, which: int, x):
        xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
        v = np.empty_like(xs)
        dv = np.empty_like(xs)
        d = C.c_double()
        for q, xq in enumerate(xs):
            v[q] = lib().or_pot_eval(self.h, which, float(xq), C.byref(d))
            dv[q] = d.value
        return v, dv


# ---------------------------------------------------------------------------
# lattice
# ---------------------------------------------------------------------------

def site_index(bx, by, x, y, z) -> int:
    return int(lib().or_site_index(bx, by, x, y, z))


def site_position(bx, by, a0, sid) -> np.ndarray:
    r = np.zeros(3)
    lib().or_site_position(bx, by, a0, sid, _d(r))
    return r


def nearest_site(bx, by, bz, a0, p) -> int:
    p = _c64(p)
    return int(lib().or_nearest_site(bx, by, bz, a0, _d(p)))


class Alloy:
    """Oracle alloy potential: per-species density and embedding tables,
    pair tables for a <= b in row-major upper-triangle order."""

    def __init__(self, al):
        nsp = al.nsp
        f = _c64(al.f).reshape(nsp, al.n)
        F = _c64(al.F).reshape(nsp, al.n)
        phi = _c64(al.phi).reshape(nsp * (nsp + 1) // 2, al.n)
        self.h = lib().or_alloy_new(al.n, nsp, al.rc, al.rho_max, _d(f), _d(F), _d(phi))
        if not self.h:
            raise ValueError("bad alloy tables")
        self.nsp = nsp

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_alloy_free(self.h)
            self.h = None


def eam_alloy(al: Alloy, x, types, L, mode: int = 0, nthreads: int = 0):
    """rho, F'(rho), per-atom energy, forces of an alloy configuration."""
    x = _c64(x).reshape(-1, 3)
    L = _c64(L)
    t = np.ascontiguousarray(types, dtype=np.int8)
    n = x.shape[0]
    rho, fp, e = np.empty(n), np.empty(n), np.empty(n)
    f = np.empty((n, 3))
    rc = lib().or_eam_alloy(al.h, n, _d(x), t.ctypes.data_as(C.c_void_p), _d(L), mode, nthreads, _d(rho), _d(fp),
                            _d(e), _d(f))
    if rc != 0:
        raise ValueError(f"or_eam_alloy failed ({rc})")
    return rho, fp, e, f


def ws_defects(bx, by, bz, a0, x):
    """(vacancies, interstitials) of the Wigner-Seitz analysis of positions x."""
    x = _c64(x).reshape(-1, 3)
    v, i = C.c_int64(), C.c_int64()
    lib().or_ws_defects(bx, by, bz, a0, x.shape[0], _d(x), C.byref(v), C.byref(i))
    return int(v.value), int(i.value)


def pka_site(bx, by, bz) -> int:
    return int(lib().or_pka_site(bx, by, bz))


def offsets(a0, R, par):
    buf = (C.c_int * (3 * 4096))()
    n = lib().or_offsets(a0, R, par, 4096, buf)
    return np.array(buf[:3 * n], dtype=np.int64).reshape(n, 3)


# ---------------------------------------------------------------------------
# EAM
# ---------------------------------------------------------------------------

def eam(pot: Pot, x, L, mode: int = 0, nthreads: int = 0):
    """rho, F'(rho), per-atom energy E_i and force F_i (N, 3) of every atom."""
    x = _c64(x).reshape(-1, 3)
    L = _c64(L)
    n = x.shape[0]
    rho, fp, e = np.empty(n), np.empty(n), np.empty(n)
    f = np.empty((n, 3))
    lib().or_eam(pot.h, n, _d(x), _d(L), mode, nthreads, _d(rho), _d(fp), _d(e), _d(f))
    return rho, fp, e, f


def eam_sample(pot: Pot, x, L, targets, nthreads: int = 0):
    """rho, E_i and F_i of the target atoms only (cell list)."""
    x = _c64(x).reshape(-1, 3)
    L = _c64(L)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    rho, e = np.empty(len(t)), np.empty(len(t))
    f = np.empty((len(t), 3))
    lib().or_eam_sample(pot.h, x.shape[0], _d(x), _d(L), nthreads, len(t), t.ctypes.data_as(_I64),
                        _d(rho), _d(e), _d(f))
    return rho, e, f


def pair_list(x, L, rc, mode: int = 0, cap: int = 10_000_000):
    x = _c64(x).reshape(-1, 3)
    L = _c64(L)
    n = lib().or_pair_list(x.shape[0], _d(x), _d(L), rc, mode, 0, None, None, None)
    pi, pj, pr = np.empty(n, np.int64), np.empty(n, np.int64), np.empty(n)
    lib().or_pair_list(x.shape[0], _d(x), _d(L), rc, mode, n, pi.ctypes.data_as(_I64),
                       pj.ctypes.data_as(_I64), _d(pr))
    return pi, pj, pr


# ---------------------------------------------------------------------------
# MD
# ---------------------------------------------------------------------------

def next_dt(v, dt_max, dx_max) -> float:
    v = _c64(v)
    return float(lib().or_next_dt(v.shape[0], _d(v), dt_max, dx_max))


def insert_pka(v, atom, mass, energy, direction):
    d = _c64(direction)
    lib().or_insert_pka(_d(v), atom, mass, energy, _d(d))


def kinetic(v, mass) -> float:
    v = _c64(v)
    return float(lib().or_kinetic(v.shape[0], _d(v), mass))


def md_run(pot: Pot, x, v, L, mass, dt_max, dx_max, nsteps, mode=1, nthreads=0, a=None, log=False):
    """Velocity-Verlet NVE run.  Returns (x, v, a, t, log[nsteps, 3] = dt, PE, KE)."""
    x = _c64(x).reshape(-1, 3).copy()
    v = _c64(v).reshape(-1, 3).copy()
    acc_valid = 1 if a is not None else 0
    a = _c64(a).copy() if a is not None else np.zeros_like(x)
    L = _c64(L)
    lg = np.zeros((max(nsteps, 1), 3)) if log else None
    t = lib().or_md_run(pot.h, x.shape[0], _d(x), _d(v), _d(a), acc_valid, _d(L), mass, dt_max, dx_max,
                        nsteps, mode, nthreads, _d(lg) if log else None)
    return x, v, a, t, (lg[:nsteps] if log else None)


# ---------------------------------------------------------------------------
# lattice list
# ---------------------------------------------------------------------------

class Lattice:
    def __init__(self, bx, by, bz, a0, skin):
        self.bx, self.by, self.bz = bx, by, bz
        self.h = lib().or_lattice_new(bx, by, bz, a0, skin)
        self.ns = 2 * bx * by * bz

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_lattice_free(self.h)
            self.h = None

    def assign(self, x):
        x = _c64(x).reshape(-1, 3)
        lib().or_lattice_assign(self.h, x.shape[0], _d(x))

    def update(self, x):
        x = _c64(x).reshape(-1, 3)
        lib().or_lattice_update(self.h, x.shape[0], _d(x))

    def site_atom(self):
        out = np.empty(self.ns, np.int64)
        lib().or_lattice_site_atom(self.h, out.ctypes.data_as(_I64))
        return out

    def runaways(self):
        out = np.empty(self.ns, np.int64)
        n = lib().or_lattice_runaways(self.h, out.ctypes.data_as(_I64))
        return out[:n].copy()

    def pairs(self, x, rc):
        x = _c64(x).reshape(-1, 3)
        n = lib().or_lattice_pairs(self.h, _d(x), rc, 0, None, None, None)
        pi, pj, pr = np.empty(n, np.int64), np.empty(n, np.int64), np.empty(n)
        lib().or_lattice_pairs(self.h, _d(x), rc, n, pi.ctypes.data_as(_I64), pj.ctypes.data_as(_I64),
                               _d(pr))
        return pi, pj, pr


# ---------------------------------------------------------------------------
# knot gradient
# ---------------------------------------------------------------------------

def loss_grad(pot: Pot, x, L, Fref, Eref, mode=0):
    """Loss (1/3N) sum |F - Fref|^2 + ((E - Eref)/N)^2 and its gradient with
    respect to the 3n knot values (f, phi, F)."""
    x = _c64(x).reshape(-1, 3)
    L = _c64(L)
    Fr = _c64(Fref).reshape(-1, 3)
    g = np.zeros(3 * pot.n)
    E = C.c_double()
    F = np.empty_like(x)
    loss = lib().or_loss_grad(pot.h, x.shape[0], _d(x), _d(L), mode, _d(Fr), float(Eref), _d(g),
                              C.byref(E), _d(F))
    return float(loss), g, float(E.value), F
