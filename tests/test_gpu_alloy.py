"""Alloys on the GPU (Sec. 2.2, Eq. eam_base and Eq. eam_force_ij with atom
types) through the C ABI, against the FP64 oracle's alloy evaluation.
Same error norm and bounds as the single-type parity tests: 1e-12 (FP64),
1e-5 (FP32)."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def misa():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa as M_
    return M_


def nerr(x, xo):
    x, xo = x.reshape(len(x), -1), xo.reshape(len(xo), -1)
    mag = np.linalg.norm(xo, axis=1)
    rms = np.sqrt(np.mean(mag ** 2))
    return float(np.max(np.linalg.norm(x - xo, axis=1) / np.maximum(mag, rms)))


CASES = {
    "thermal_2sp_11x9x8": (2, (11, 9, 8), lambda: synth.thermal_snapshot(11, 9, 8, 0.12, 21), (0.7, 0.3)),
    "cascade_3sp_10x9x12": (3, (10, 9, 12), lambda: synth.cascade_snapshot(10, 9, 12, 0.12, 16, 6, 22), (0.6, 0.25, 0.15)),
    "cascade_2sp_6x6x6": (2, (6, 6, 6), lambda: synth.cascade_snapshot(6, 6, 6, 0.1, 5, 3, 23), (0.5, 0.5)),
}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_alloy_parity(misa, oracle, prec, case):
    nsp, dims, mk, frac = CASES[case]
    al = synth.alloy_potential(nsp)
    x = mk()
    t = synth.random_types(len(x), frac, 31)
    rho_o, _, e_o, f_o = oracle.eam_alloy(oracle.Alloy(al), x, t, synth.box(*dims), mode=1)
    with misa.Sim(al.species(0), *dims, precision=prec) as s:
        s.set_species(al, t)
        s.set_state(x)
        f, rho = s.forces(), s.density()
        pe, _, e = s.energies(per_atom=True)
        st = s.stats()
    assert nerr(f, f_o) < TOL[prec], nerr(f, f_o)
    assert nerr(rho, rho_o) < TOL[prec], nerr(rho, rho_o)
    assert nerr(e, e_o) < TOL[prec], nerr(e, e_o)
    assert abs(pe - e_o.sum()) / len(x) < TOL[prec]
    if case.startswith("cascade"):
        assert st["n_runaway"] > 0


@pytest.mark.parametrize("case", ["cascade_3sp_10x9x12", "cascade_2sp_6x6x6"])
def test_alloy_tile_shapes_bitwise_equal(misa, oracle, case):
    # FP32 alloy gathers: per-site sums do not depend on the tile shape (tiles
    # wider than the box included), and every shape meets the oracle bound
    nsp, dims, mk, frac = CASES[case]
    al = synth.alloy_potential(nsp)
    x = mk()
    t = synth.random_types(len(x), frac, 32)
    rho_o, _, e_o, f_o = oracle.eam_alloy(oracle.Alloy(al), x, t, synth.box(*dims), mode=1)
    ref = None
    for k in misa.tile_indices("fp32"):
        with misa.Sim(al.species(0), *dims, precision="fp32", tile=k) as s:
            s.set_species(al, t)
            s.set_state(x)
            got = (s.forces(), s.density(), s.energies(per_atom=True)[2])
        assert nerr(got[0], f_o) < TOL["fp32"], (k, nerr(got[0], f_o))
        assert nerr(got[1], rho_o) < TOL["fp32"], (k, nerr(got[1], rho_o))
        assert nerr(got[2], e_o) < TOL["fp32"], (k, nerr(got[2], e_o))
        if ref is None:
            ref = got
        else:
            for a_, b_ in zip(ref, got):
                np.testing.assert_array_equal(a_, b_)


def test_identical_species_match_single_type(misa):
    pot = synth.potential()
    nsp = 3
    al = synth.AlloyPotential(nsp, pot.n, pot.rc, pot.rho_max, np.stack([pot.f] * nsp), np.stack([pot.F] * nsp),
                              np.stack([pot.phi] * (nsp * (nsp + 1) // 2)))
    x = synth.cascade_snapshot(9, 8, 10, 0.12, 10, 4, 24)
    t = synth.random_types(len(x), (0.4, 0.3, 0.3), 25)
    out = []
    for species in (False, True):
        with misa.Sim(pot, 9, 8, 10, precision="fp64") as s:
            if species:
                s.set_species(al, t)
            s.set_state(x)
            out.append(s.forces())
    assert nerr(out[1], out[0]) < 1e-12


def test_one_species_is_the_single_type_path(misa):
    al = synth.alloy_potential(2)
    one = synth.AlloyPotential(1, al.n, al.rc, al.rho_max, al.f[:1], al.F[:1], al.phi[:1])
    x = synth.thermal_snapshot(8, 8, 8, 0.1, 26)
    out = []
    for k in range(2):
        with misa.Sim(al.species(0), 8, precision="fp32", tile=1) as s:
            if k:
                s.set_species(one, np.zeros(len(x), np.int8))
            s.set_state(x)
            out.append(s.forces())
    np.testing.assert_array_equal(out[0], out[1])


def test_alloy_cascade_run_matches_oracle(misa, oracle):
    nsp, n = 3, 10
    al = synth.alloy_potential(nsp)
    x = synth.thermal_snapshot(n, n, n, 0.08, 27)
    t = synth.random_types(len(x), (0.6, 0.25, 0.15), 28)
    with misa.Sim(al.species(0), n, precision="fp64", dx_max=0.02, reassign_period=5) as s:
        s.set_species(al, t)
        s.set_state(x, synth.maxwell_velocities(len(x), 300.0, synth.MASS_FE, 29))
        s.insert_pka(-1, 1500.0, synth.random_direction(30))
        pe0, ke0 = s.energies()
        s.step(200)
        pe1, ke1 = s.energies()
        st = s.stats()
        xp, f = s.positions(), s.forces()
    assert st["status"] == 0 and st["n_runaway"] > 0
    _, _, _, f_o = oracle.eam_alloy(oracle.Alloy(al), xp, t, synth.box(n, n, n), mode=1)
    assert nerr(f, f_o) < 1e-12
    assert abs((pe1 + ke1) - (pe0 + ke0)) / len(x) < 1e-4


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_alloy_replicas_equal_single_boxes(misa, prec):
    al = synth.alloy_potential(2)
    dims = [(7, 8, 6), (9, 7, 8)]
    xs = [synth.cascade_snapshot(*d, 0.1, 4, 2, 40 + k) for k, d in enumerate(dims)]
    ts = [synth.random_types(len(x), (0.7, 0.3), 50 + k) for k, x in enumerate(xs)]
    single = []
    for d, x, t in zip(dims, xs, ts):
        with misa.Sim(al.species(0), *d, precision=prec, tile=1) as s:
            s.set_species(al, t)
            s.set_state(x)
            s.step(20)
            single.append(s.forces())
    with misa.Sim(al.species(0), replicas=dims, precision=prec, tile=1) as s:
        s.set_species(al, np.concatenate(ts))
        s.set_state(np.concatenate(xs))
        s.step(20)
        fb = s.forces()
    np.testing.assert_array_equal(fb, np.concatenate(single))


def test_alloy_parity_at_benchmark_size(misa, oracle):
    # the alloy benchmark's box (100^3 cells, three species 70/20/10 %) in the
    # launch configuration it times: tiles retuned on the state, steps replayed
    # from a captured graph, adaptive dt, knock-on atom, hash update every 10
    # steps; then every atom against the oracle on the GPU's own positions
    n, nsp = 100, 3
    natoms = 2 * n ** 3
    al = synth.alloy_potential(nsp)
    t = synth.random_types(natoms, (0.7, 0.2, 0.1), 80)
    with misa.Sim(al.species(0), n, precision="fp32", dt_max=1.0, dx_max=0.02, reassign_period=10) as s:
        s.set_species(al, t)
        s.set_velocities(synth.maxwell_velocities(natoms, 600.0, synth.MASS_FE, 3))
        s.retune()
        s.insert_pka(-1, 5000.0, synth.random_direction(20))
        s.step(30)
        st = s.stats()
        assert st["status"] == 0 and st["step"] == 30
        x, f, rho = s.positions(), s.forces(), s.density()
        _, _, e = s.energies(per_atom=True)
    rho_o, _, e_o, f_o = oracle.eam_alloy(oracle.Alloy(al), x, t, synth.box(n, n, n), mode=1)
    assert nerr(f, f_o) < TOL["fp32"], nerr(f, f_o)
    assert nerr(rho, rho_o) < TOL["fp32"], nerr(rho, rho_o)
    assert nerr(e, e_o) < TOL["fp32"], nerr(e, e_o)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_alloy_energy_step_equals_separate_evaluation(misa, prec):
    # the alloy passes of the energy step (misa_step_energies) write the
    # same per-atom energies as a separate evaluation after plain steps
    nsp, dims, mk, frac = CASES["cascade_3sp_10x9x12"]
    al = synth.alloy_potential(nsp)
    x = mk()
    t = synth.random_types(len(x), frac, 33)
    v = synth.maxwell_velocities(len(x), 600.0, synth.MASS_FE, 6)
    out = []
    for energies in (False, True):
        with misa.Sim(al.species(0), *dims, precision=prec, dx_max=0.02, reassign_period=3) as s:
            s.set_species(al, t)
            s.set_state(x, v)
            s.step(6, energies=energies)
            if energies:
                # the asynchronous read-out of the same energies
                e_async = np.zeros(len(x))
                s.energies_async(e_async)
                s.wait_outputs()
            pe, ke, e = s.energies(per_atom=True)
            out.append((s.positions(), pe, ke, e))
    for a_, b_ in zip(out[0], out[1]):
        np.testing.assert_array_equal(a_, b_)
    np.testing.assert_array_equal(e_async, out[1][3])
