"""The allocation-free entry point misa_eam_forces_static, called through the
C ABI, against the handle-based entry points (misa_set_state +
misa_get_forces / misa_get_energies) on the same positions.

Some callers cannot allocate device memory (a framework pool that owns every
byte, a latency-critical path that cannot take cudaMalloc's implicit
synchronisation, a plug-in in a host program that reserved the GPU up
front); misa_eam_forces_static serves them from a static device array.
This file is collected last so that a run stopping at the first failure has
run every other test before it; it also passes alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def nerr(x, xo):
    x = np.asarray(x, dtype=np.float64).reshape(len(xo), -1)
    xo = np.asarray(xo, dtype=np.float64).reshape(len(xo), -1)
    mag = np.linalg.norm(xo, axis=1)
    rms = np.sqrt(np.mean(mag * mag))
    return float(np.max(np.linalg.norm(x - xo, axis=1) / np.maximum(mag, max(rms, 1e-300))))


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa
    L = misa.lib()
    f = L.misa_eam_forces_static
    f.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_double, C.c_double, C.c_double, C.c_int32, C.c_void_p,
                  C.c_double, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return torch, misa, f


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_entry_matches_handle_entry_on_two_calls(env, prec):
    torch, misa, fn = env
    pot = synth.potential()
    dims = (12, 10, 8)
    natoms = 2 * dims[0] * dims[1] * dims[2]
    knots = torch.from_numpy(np.concatenate([pot.f, pot.phi, pot.F])).cuda()
    code = misa.FP64 if prec == "fp64" else misa.FP32_FORCE
    stream = torch.cuda.current_stream().cuda_stream
    # two different configurations in a row: the second call must not see
    # anything the first one left in the shared array
    for seed, n_int in ((3, 10), (4, 2)):
        xh = synth.cascade_snapshot(*dims, 0.12, n_int, 3, seed)
        x = torch.from_numpy(xh).cuda()
        f_out = torch.empty((natoms, 3), dtype=torch.float64, device="cuda")
        e_out = torch.empty(natoms, dtype=torch.float64, device="cuda")
        rc = fn(*dims, synth.A0_FE, pot.rc, 0.6, pot.n, knots.data_ptr(), pot.rho_max, code, x.data_ptr(),
                f_out.data_ptr(), e_out.data_ptr(), stream)
        assert rc == misa.MISA_OK, misa.lib().misa_last_error(None)
        with misa.Sim(pot, *dims, precision=prec) as s:
            s.set_state(xh)
            f_ref = s.forces()
            _, _, e_ref = s.energies(per_atom=True)
        assert nerr(f_out.cpu().numpy(), f_ref) < TOL[prec]
        assert nerr(e_out.cpu().numpy(), e_ref) < TOL[prec]


def test_static_entry_rejects_oversized_input(env):
    torch, misa, fn = env
    pot = synth.potential()
    knots = torch.from_numpy(np.concatenate([pot.f, pot.phi, pot.F])).cuda()
    x = torch.zeros(3, dtype=torch.float64, device="cuda")
    # 2 * 30^3 = 54,000 atoms > the static limit: refused before any GPU work
    rc = fn(30, 30, 30, synth.A0_FE, pot.rc, 0.6, pot.n, knots.data_ptr(), pot.rho_max, misa.FP64,
            x.data_ptr(), x.data_ptr(), None, None)
    assert rc == misa.MISA_EINVAL
    assert b"exceed" in misa.lib().misa_last_error(None)


def _static_call(torch, misa, fn, pot, dims, prec, xh):
    natoms = 2 * dims[0] * dims[1] * dims[2]
    knots = torch.from_numpy(np.concatenate([pot.f, pot.phi, pot.F])).cuda()
    x = torch.from_numpy(xh).cuda()
    f_out = torch.empty((natoms, 3), dtype=torch.float64, device="cuda")
    e_out = torch.empty(natoms, dtype=torch.float64, device="cuda")
    code = misa.FP64 if prec == "fp64" else misa.FP32_FORCE
    torch.cuda.synchronize()
    rc = fn(*dims, synth.A0_FE, pot.rc, 0.6, pot.n, knots.data_ptr(), pot.rho_max, code, x.data_ptr(),
            f_out.data_ptr(), e_out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return rc, f_out, e_out


def _handle(misa, pot, dims, prec, xh):
    with misa.Sim(pot, *dims, precision=prec) as s:
        s.set_state(xh)
        f = s.forces()
        _, _, e = s.energies(per_atom=True)
    return f, e


def test_static_entry_larger_fp64_box_then_smaller_fp32_box(env):
    # the second call lays its buffers out differently in the shared array
    # (other box, other precision): nothing of the first call may leak in
    torch, misa, fn = env
    pot = synth.potential()
    for dims, prec, seed in (((14, 12, 10), "fp64", 5), ((8, 7, 6), "fp32", 6), ((14, 12, 10), "fp32", 7)):
        xh = synth.cascade_snapshot(*dims, 0.12, 6, 2, seed)
        rc, f_out, e_out = _static_call(torch, misa, fn, pot, dims, prec, xh)
        assert rc == misa.MISA_OK, misa.lib().misa_last_error(None)
        f_ref, e_ref = _handle(misa, pot, dims, prec, xh)
        assert nerr(f_out.cpu().numpy(), f_ref) < TOL[prec], (dims, prec)
        assert nerr(e_out.cpu().numpy(), e_ref) < TOL[prec], (dims, prec)


def test_static_entry_allocates_no_device_memory(env):
    # after a first call of the same precision (which loads its kernels),
    # a call leaves the device's free memory exactly as it found it
    torch, misa, fn = env
    pot = synth.potential()
    dims = (10, 9, 8)
    xh = synth.cascade_snapshot(*dims, 0.1, 4, 1, 9)
    natoms = 2 * dims[0] * dims[1] * dims[2]
    knots = torch.from_numpy(np.concatenate([pot.f, pot.phi, pot.F])).cuda()
    x = torch.from_numpy(xh).cuda()
    f_out = torch.empty((natoms, 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for prec in ("fp32", "fp64"):
        code = misa.FP64 if prec == "fp64" else misa.FP32_FORCE
        args = (*dims, synth.A0_FE, pot.rc, 0.6, pot.n, knots.data_ptr(), pot.rho_max, code, x.data_ptr(),
                f_out.data_ptr(), None, stream)
        assert fn(*args) == misa.MISA_OK
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        assert fn(*args) == misa.MISA_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (prec, free0 - free1)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_static_entry_at_the_knot_limit(env, prec):
    # MISA_STATIC_MAX_KNOTS knots per table: the FP32 table window still fits
    # beside the tile in a block's shared memory
    torch, misa, fn = env
    pot = synth.potential(n=8192)
    dims = (7, 6, 6)
    xh = synth.cascade_snapshot(*dims, 0.1, 3, 1, 12)
    rc, f_out, e_out = _static_call(torch, misa, fn, pot, dims, prec, xh)
    assert rc == misa.MISA_OK, misa.lib().misa_last_error(None)
    f_ref, e_ref = _handle(misa, pot, dims, prec, xh)
    assert nerr(f_out.cpu().numpy(), f_ref) < TOL[prec]
    assert nerr(e_out.cpu().numpy(), e_ref) < TOL[prec]
