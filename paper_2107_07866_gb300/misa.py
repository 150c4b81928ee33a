"""Python binding of the C ABI in include/misa.h (argument marshalling only).

Every step of the method runs in the CUDA library libmisa.so; this module
passes pointers and sizes.  PyTorch supplies device memory (the library's
allocator hooks draw from torch's caching allocator) and the CUDA stream.
There is no CPU fallback: a missing library raises at import of Sim.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmisa.so")

MISA_OK = 0
MISA_EINVAL = -1
MISA_EOOM = -2
MISA_ECUDA = -3
MISA_ERUNAWAY_OVERFLOW = -4
MISA_EUNSTABLE = -5
MISA_ETIMEOUT = -6

FP64 = 0
FP32_FORCE = 1

ST_RUNAWAY_OVERFLOW = 0x1
ST_NONFINITE = 0x2
ST_RFLOOR = 0x4
ST_RHO_EXTRAP = 0x8

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32),
        ("a0", C.c_double), ("mass", C.c_double), ("rc", C.c_double), ("skin", C.c_double),
        ("n_knots", C.c_int32),
        ("f_knots", C.POINTER(C.c_double)), ("phi_knots", C.POINTER(C.c_double)),
        ("F_knots", C.POINTER(C.c_double)),
        ("rho_max", C.c_double),
        ("precision", C.c_int32), ("reassign_period", C.c_int32),
        ("dt_max", C.c_double), ("dx_max", C.c_double),
        ("runaway_capacity", C.c_int64),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("tile", C.c_int32),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("time", C.c_double), ("dt", C.c_double),
        ("natoms", C.c_int64), ("nsites", C.c_int64), ("n_runaway", C.c_int64),
        ("n_vacant", C.c_int64), ("status", C.c_uint32), ("vmax", C.c_double),
        ("launches", C.c_int64),
    ]


class Peaks(C.Structure):
    _fields_ = [
        ("fp32_ffma_tflops", C.c_double), ("fp32_ffma2_tflops", C.c_double), ("fp64_dfma_tflops", C.c_double),
        ("mufu_rsqrt_tops", C.c_double), ("lds128_tbps", C.c_double), ("sm_clock_mhz", C.c_double),
        ("num_sms", C.c_int32),
    ]


PHASES = ("kick_drift", "list", "density", "ra_density", "force", "ra_force", "end")


_lib = None
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)


def lib():
    """Loads libmisa.so (built by __graft_entry__.build() or
    paper_2107_07866_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2107_07866_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        L.misa_default_params.argtypes = [C.POINTER(Params)]
        L.misa_create.argtypes = [C.POINTER(Params), C.c_void_p, C.POINTER(C.c_void_p)]
        L.misa_destroy.argtypes = [C.c_void_p]
        L.misa_last_error.argtypes = [C.c_void_p]
        L.misa_last_error.restype = C.c_char_p
        L.misa_set_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
        L.misa_set_velocities.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.misa_stage_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]
        L.misa_set_state_staged.argtypes = [C.c_void_p]
        L.misa_insert_pka.argtypes = [C.c_void_p, C.c_int64, C.c_double, _D]
        L.misa_step.argtypes = [C.c_void_p, C.c_int]
        L.misa_step_energies.argtypes = [C.c_void_p, C.c_int]
        L.misa_get_energies.argtypes = [C.c_void_p, _D, _D, C.c_void_p]
        L.misa_get_energies_async.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.misa_wait_outputs.argtypes = [C.c_void_p]
        for name in ("misa_get_positions", "misa_get_velocities", "misa_get_forces", "misa_get_density"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.misa_get_site_map.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, _I64]
        L.misa_stats_get.argtypes = [C.c_void_p, C.POINTER(Stats)]
        L.misa_clear_status.argtypes = [C.c_void_p]
        L.misa_save.argtypes = [C.c_void_p, C.c_char_p]
        L.misa_load.argtypes = [C.c_void_p, C.c_char_p]
        L.misa_timing_enable.argtypes = [C.c_void_p, C.c_int]
        L.misa_timing_get.argtypes = [C.c_void_p, _D, _I64]
        L.misa_create_batch.argtypes = [C.POINTER(Params), C.c_int32, C.POINTER(C.c_int32), C.c_void_p,
                                        C.POINTER(C.c_void_p)]
        L.misa_replica_count.argtypes = [C.c_void_p]
        L.misa_replica_info.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), _I64, _I64]
        L.misa_insert_pka_replica.argtypes = [C.c_void_p, C.c_int32, C.c_double, _D]
        L.misa_replica_stats.argtypes = [C.c_void_p, C.c_int32, C.POINTER(Stats)]
        L.misa_replica_energies.argtypes = [C.c_void_p, _D, _D]
        L.misa_set_graphs.argtypes = [C.c_void_p, C.c_int]
        L.misa_tile_current.argtypes = [C.c_void_p]
        L.misa_tile_current_force.argtypes = [C.c_void_p]
        L.misa_retune.argtypes = [C.c_void_p]
        L.misa_defects.argtypes = [C.c_void_p, C.c_void_p]
        L.misa_set_species.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.misa_eam_forces_static.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double,
                                             C.c_int32, C.c_void_p, C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]
        L.misa_set_tables.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.misa_loss_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, _D, C.c_void_p]
        L.misa_tile_count.restype = C.c_int
        L.misa_tile_valid.argtypes = [C.c_int, C.c_int]
        L.misa_selftest.argtypes = [C.c_longlong, C.POINTER(C.c_longlong)]
        L.misa_tile_shape.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.misa_measure_peaks.argtypes = [C.POINTER(Peaks), C.c_void_p]
        L.misa_set_density_variant.argtypes = [C.c_void_p, C.c_int32]
        _lib = L
    return _lib


class MisaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"misa error {code}: {msg}")
        self.code = code


def _ptr(a):
    """Data pointer of a C-contiguous float64 numpy array or torch tensor."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def _f64(a):
    if a is None or hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


class _TorchAllocator:
    """Allocator hooks that hand the library memory from torch's caching
    allocator on the current device."""

    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda")
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, nbytes, ctx):
        self.live.pop(ptr, None)


class Sim:
    """Periodic bcc crystals on the GPU (a misa_sim handle): one box of
    nx x ny x nz cells, or a batch of independent replicas when ``replicas``
    lists their (nx, ny, nz)."""

    def __init__(self, pot: synth.Potential, nx=None, ny=None, nz=None, precision="fp32", a0=synth.A0_FE,
                 mass=synth.MASS_FE, skin=0.6, reassign_period=10, dt_max=1.0, dx_max=0.0,
                 runaway_capacity=0, tile=0, stream=None, torch_memory=True, replicas=None):
        if replicas is None:
            ny = nx if ny is None else ny
            nz = nx if nz is None else nz
            replicas = [(nx, ny, nz)]
        else:
            nx, ny, nz = replicas[0]
        L = lib()
        p = Params()
        L.misa_default_params(C.byref(p))
        self._knots = [np.ascontiguousarray(pot.f, dtype=np.float64), np.ascontiguousarray(pot.phi, dtype=np.float64),
                       np.ascontiguousarray(pot.F, dtype=np.float64)]
        p.nx, p.ny, p.nz = nx, ny, nz
        p.a0, p.mass, p.rc, p.skin = a0, mass, pot.rc, skin
        p.n_knots = pot.n
        p.f_knots = self._knots[0].ctypes.data_as(_D)
        p.phi_knots = self._knots[1].ctypes.data_as(_D)
        p.F_knots = self._knots[2].ctypes.data_as(_D)
        p.rho_max = pot.rho_max
        p.precision = {"fp64": FP64, "fp32": FP32_FORCE}[precision] if isinstance(precision, str) else int(precision)
        p.reassign_period = reassign_period
        p.dt_max, p.dx_max = dt_max, dx_max
        p.runaway_capacity = runaway_capacity
        p.tile = tile
        self._alloc = None
        st = None
        try:
            import torch
            if torch.cuda.is_available():
                if torch_memory:
                    self._alloc = _TorchAllocator()
                    p.alloc, p.free = self._alloc.alloc, self._alloc.free
                if stream is None:
                    stream = torch.cuda.current_stream()
                st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        except ImportError:
            st = stream
        self.stream = st
        h = C.c_void_p()
        dims = (C.c_int32 * (3 * len(replicas)))(*[int(v) for d in replicas for v in d])
        rc = L.misa_create_batch(C.byref(p), len(replicas), dims, C.c_void_p(st) if st else None, C.byref(h))
        if rc != MISA_OK:
            raise MisaError(rc, L.misa_last_error(None).decode())
        self.h = h
        self.replicas = [tuple(d) for d in replicas]
        self.nx, self.ny, self.nz = nx, ny, nz
        self.natoms = sum(2 * a * b * c for a, b, c in replicas)
        self.box = np.array([nx * a0, ny * a0, nz * a0])
        self.a0 = a0
        self._n_knots = pot.n
        self.precision = p.precision

    # -- plumbing -----------------------------------------------------------
    def _check(self, rc):
        if rc != MISA_OK:
            raise MisaError(rc, lib().misa_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().misa_destroy(self.h)
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

    # -- state --------------------------------------------------------------
    def set_state(self, x, v=None):
        x = _f64(x)
        v = _f64(v)
        self._check(lib().misa_set_state(self.h, _ptr(x), _ptr(v), self.natoms))

    def stage_state(self, x, v=None):
        """Starts copying x (and v) into the handle's staging buffers on its
        copy stream; set_state_staged() applies them.  The arrays stay
        referenced here until the next stage_state call, which waits for
        this copy to be complete (they must not change meanwhile)."""
        x = _f64(x)
        v = _f64(v)
        self._check(lib().misa_stage_state(self.h, _ptr(x), _ptr(v), self.natoms))
        self._staged = (x, v)

    def set_state_staged(self):
        self._check(lib().misa_set_state_staged(self.h))

    def set_velocities(self, v):
        v = _f64(v)
        self._check(lib().misa_set_velocities(self.h, _ptr(v), self.natoms))

    def insert_pka(self, atom=-1, energy=1000.0, direction=(1.0, 0.0, 0.0)):
        d = (C.c_double * 3)(*[float(t) for t in direction])
        self._check(lib().misa_insert_pka(self.h, int(atom), float(energy), d))

    def step(self, n=1, energies=False):
        """n MD steps; with energies the last one also evaluates the per-atom
        energies, which energies() then reads without another evaluation."""
        fn = lib().misa_step_energies if energies else lib().misa_step
        self._check(fn(self.h, int(n)))

    # -- read-out -----------------------------------------------------------
    def energies(self, per_atom=False, out=None):
        """Total potential and kinetic energy (eV); with per_atom also E_i of
        every atom (into out, a float64 array of natoms, when given)."""
        pe, ke = C.c_double(), C.c_double()
        e = (np.empty(self.natoms) if out is None else out) if per_atom else None
        self._check(lib().misa_get_energies(self.h, C.byref(pe), C.byref(ke), _ptr(e)))
        return (pe.value, ke.value, e) if per_atom else (pe.value, ke.value)

    def energies_async(self, out):
        """E_i of every atom into out (float64, natoms; pinned host memory
        for a copy that runs beside the following calls) without waiting;
        out holds them once wait_outputs() has returned."""
        if len(out) < self.natoms:
            raise ValueError("out must hold natoms values")
        self._check(lib().misa_get_energies_async(self.h, _ptr(out), len(out)))
        return out

    def wait_outputs(self):
        """Waits for the copies started by energies_async."""
        self._check(lib().misa_wait_outputs(self.h))

    def _get(self, fn, width, out=None):
        if out is None:
            out = np.empty((self.natoms, width) if width > 1 else self.natoms)
        self._check(fn(self.h, _ptr(out), self.natoms))
        return out

    def positions(self, out=None):
        return self._get(lib().misa_get_positions, 3, out)

    def velocities(self, out=None):
        return self._get(lib().misa_get_velocities, 3, out)

    def forces(self, out=None):
        return self._get(lib().misa_get_forces, 3, out)

    def density(self, out=None):
        return self._get(lib().misa_get_density, 1, out)

    def site_map(self):
        sa = np.empty(self.natoms, np.int64)
        n = C.c_int64()
        self._check(lib().misa_get_site_map(self.h, _ptr(sa), None, 0, C.byref(n)))
        ra = np.empty(max(n.value, 1), np.int64)
        self._check(lib().misa_get_site_map(self.h, None, _ptr(ra), len(ra), C.byref(n)))
        return sa, ra[:n.value].copy()

    def stats(self) -> dict:
        s = Stats()
        self._check(lib().misa_stats_get(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def timing(self, enable=True):
        self._check(lib().misa_timing_enable(self.h, 1 if enable else 0))

    def timing_get(self):
        """{phase: summed ms} over the steps since timing was enabled / read, and the step count."""
        ms = (C.c_double * len(PHASES))()
        n = C.c_int64()
        self._check(lib().misa_timing_get(self.h, ms, C.byref(n)))
        return dict(zip(PHASES, list(ms))), n.value

    # -- potential fitting ----------------------------------------------------
    def set_tables(self, f, phi, F):
        """New knot values (numpy arrays or torch tensors, host or device)."""
        f, phi, F = _f64(f), _f64(phi), _f64(F)
        self._check(lib().misa_set_tables(self.h, _ptr(f), _ptr(phi), _ptr(F)))

    def loss_grad(self, Fref, Eref, grad=None):
        """Force-matching + energy loss of the current positions against
        Fref (natoms x 3) and Eref (one per replica), and its gradient with
        respect to the 3 x n knot values (f, phi, F).  grad may be a
        preallocated numpy array or device tensor of 3n doubles."""
        Fref = _f64(Fref)
        Eref = _f64(np.atleast_1d(Eref)) if not hasattr(Eref, "data_ptr") else Eref
        if grad is None:
            grad = np.empty(3 * self._n_knots)
        loss = C.c_double()
        self._check(lib().misa_loss_grad(self.h, _ptr(Fref), _ptr(Eref), C.byref(loss), _ptr(grad)))
        return loss.value, grad

    # -- batches --------------------------------------------------------------
    def replica_info(self, r):
        """(dims, first atom id, atom count) of replica r."""
        d = (C.c_int32 * 3)()
        b, n = C.c_int64(), C.c_int64()
        self._check(lib().misa_replica_info(self.h, int(r), d, C.byref(b), C.byref(n)))
        return tuple(d), b.value, n.value

    def insert_pka_replica(self, r, energy, direction):
        d = (C.c_double * 3)(*[float(t) for t in direction])
        self._check(lib().misa_insert_pka_replica(self.h, int(r), float(energy), d))

    def replica_stats(self, r) -> dict:
        s = Stats()
        self._check(lib().misa_replica_stats(self.h, int(r), C.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def replica_energies(self):
        n = len(self.replicas)
        pe, ke = np.empty(n), np.empty(n)
        self._check(lib().misa_replica_energies(self.h, pe.ctypes.data_as(_D), ke.ctypes.data_as(_D)))
        return pe, ke

    def set_density_variant(self, variant):
        """0: full-neighbour density pass; 1: Newton's third law inside tiles
        (FP32 single-type handles)."""
        self._check(lib().misa_set_density_variant(self.h, int(variant)))

    def set_graphs(self, enable=True):
        self._check(lib().misa_set_graphs(self.h, 1 if enable else 0))

    def tile(self):
        """Tile shape of the density pass (cells)."""
        return tile_shapes()[lib().misa_tile_current(self.h) - 1]

    def set_species(self, alloy, types):
        """Alloy potential (synth.AlloyPotential-like: nsp, f, F, phi knot
        arrays) and the type of every atom id."""
        nsp = int(alloy.nsp)
        f = np.ascontiguousarray(alloy.f, dtype=np.float64).reshape(nsp, -1)
        F = np.ascontiguousarray(alloy.F, dtype=np.float64).reshape(nsp, -1)
        phi = np.ascontiguousarray(alloy.phi, dtype=np.float64).reshape(nsp * (nsp + 1) // 2, -1)
        t = np.ascontiguousarray(types, dtype=np.int8)
        if t.shape != (self.natoms,):
            raise ValueError("one type per atom")
        self._check(lib().misa_set_species(self.h, nsp, _ptr(f), _ptr(F), _ptr(phi), C.c_void_p(t.ctypes.data)))

    def defects(self):
        """Frenkel pairs (vacancies = interstitials) of every replica."""
        out = np.empty(lib().misa_replica_count(self.h), np.int64)
        self._check(lib().misa_defects(self.h, _ptr(out)))
        return out

    def retune(self):
        """Re-run the tile autotuner on the current state."""
        self._check(lib().misa_retune(self.h))

    def tile_force(self):
        """Tile shape of the force pass (cells)."""
        return tile_shapes()[lib().misa_tile_current_force(self.h) - 1]

    def clear_status(self):
        self._check(lib().misa_clear_status(self.h))

    def save(self, path):
        self._check(lib().misa_save(self.h, str(path).encode()))

    def load(self, path):
        self._check(lib().misa_load(self.h, str(path).encode()))


def tile_shapes():
    """All built tile shapes (cells), index k - 1 for misa tile index k."""
    L = lib()
    out = []
    for k in range(1, L.misa_tile_count() + 1):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        L.misa_tile_shape(k, C.byref(a), C.byref(b), C.byref(c))
        out.append((a.value, b.value, c.value))
    return out


def selftest(n=1 << 22):
    """Mismatch counts of the library's shortcuts against their exact
    counterparts: (double -> float, float -> double) integer-pipe conversions
    against the GPU's own on n bit patterns, and the FP32-decided site hash
    against the FP64 one on n positions."""
    out = (C.c_longlong * 3)()
    code = lib().misa_selftest(n, out)
    if code != MISA_OK:
        raise MisaError(code, "misa_selftest failed")
    return int(out[0]), int(out[1]), int(out[2])


def measure_peaks(stream=None) -> dict:
    """Issue-rate microbenchmarks of the current device (misa_measure_peaks):
    FP32 FMA, packed FP32x2 FMA and FP64 FMA in TFLOP/s, MUFU reciprocal
    square roots in 1e12/s, conflict-free 16-byte shared-memory loads in
    TB/s, the SM clock during the FP32 probe, the SM count."""
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        except Exception:
            stream = None
    p = Peaks()
    code = lib().misa_measure_peaks(C.byref(p), C.c_void_p(stream) if stream else None)
    if code != MISA_OK:
        raise MisaError(code, "misa_measure_peaks failed")
    return {k: getattr(p, k) for k, _ in Peaks._fields_}


def tile_indices(precision):
    """1-based tile indices built for a precision ("fp32" or "fp64")."""
    L = lib()
    code = {"fp64": FP64, "fp32": FP32_FORCE}[precision] if isinstance(precision, str) else int(precision)
    return [k for k in range(1, L.misa_tile_count() + 1) if L.misa_tile_valid(code, k)]
