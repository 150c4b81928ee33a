"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: forces within 1e-12 relative for the FP64
path and 1e-5 for the FP32 force path; the same normalised error is applied
to densities and per-atom energies.  Normalised error of a per-atom
quantity X: max_i |X_i - X_i^o| / max(|X_i^o|, rms_i |X^o|), the rms floor
keeping near-zero forces from dividing by zero.
"""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}
M = synth.MASS_FE


def nerr(x, xo):
    x = np.asarray(x, dtype=np.float64)
    xo = np.asarray(xo, dtype=np.float64)
    if x.ndim == 1:
        x, xo = x[:, None], xo[:, None]
    mag = np.linalg.norm(xo, axis=1)
    rms = np.sqrt(np.mean(mag * mag))
    return float(np.max(np.linalg.norm(x - xo, axis=1) / np.maximum(mag, max(rms, 1e-300))))


@pytest.fixture(scope="module")
def misa():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa as M_
    return M_


CASES = {
    # ragged against every tile shape (8x8x8 etc.), several tiles
    "thermal_13x11x9": (lambda: synth.thermal_snapshot(13, 11, 9, 0.12, 1), (13, 11, 9)),
    # interstitials (run-aways + vacancies) and close pairs down to 1 A
    "cascade_12x9x10": (lambda: synth.cascade_snapshot(12, 9, 10, 0.12, 24, 8, 2), (12, 9, 10)),
    # smallest box the library takes
    "cascade_6x6x6": (lambda: synth.cascade_snapshot(6, 6, 6, 0.1, 5, 3, 3), (6, 6, 6)),
}


@pytest.fixture(scope="module")
def oracle_results(oracle, opot):
    out = {}
    for name, (mk, dims) in CASES.items():
        x = mk()
        L = synth.box(*dims)
        rho, fp, e, f = oracle.eam(opot, x, L, mode=1)
        out[name] = (x, dims, rho, e, f)
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_density_energy_force_parity(misa, pot, oracle_results, prec, case):
    x, dims, rho_o, e_o, f_o = oracle_results[case]
    with misa.Sim(pot, *dims, precision=prec) as s:
        s.set_state(x)
        f = s.forces()
        rho = s.density()
        pe, ke, e = s.energies(per_atom=True)
        st = s.stats()
    assert nerr(f, f_o) < TOL[prec], nerr(f, f_o)
    assert nerr(rho, rho_o) < TOL[prec], nerr(rho, rho_o)
    assert nerr(e, e_o) < TOL[prec], nerr(e, e_o)
    assert abs(pe - e_o.sum()) / len(x) < TOL[prec]
    assert ke == 0.0
    if case.startswith("cascade"):
        assert st["n_runaway"] > 0
    assert st["status"] & ~0x8 == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_perfect_crystal_zero_force(misa, pot, oracle, opot, prec):
    n = 10
    with misa.Sim(pot, n, precision=prec) as s:
        f = s.forces()
        pe, ke, e = s.energies(per_atom=True)
        x = s.positions()
    np.testing.assert_allclose(x, synth.bcc_positions(n, n, n), atol=1e-12)
    _, _, e_o, _ = oracle.eam(opot, synth.bcc_positions(n, n, n), synth.box(n, n, n), mode=1)
    # pair forces of the first shell are ~0.3 eV/A; their sum vanishes by symmetry
    assert np.abs(f).max() < (1e-12 if prec == "fp64" else 1e-5)
    np.testing.assert_allclose(e, e_o, rtol=0, atol=TOL[prec] * 9.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["cascade_12x9x10", "cascade_6x6x6"])
def test_tile_shapes_bitwise_equal(misa, pot, oracle_results, prec, case):
    # every shape, including tiles more than twice as wide as the 6-cell box
    # (run-away pairs then span several periodic images of the tile)
    x, dims, _, _, f_o = oracle_results[case]
    ref = None
    for t in misa.tile_indices(prec):
        with misa.Sim(pot, *dims, precision=prec, tile=t) as s:
            s.set_state(x)
            f = s.forces()
        assert nerr(f, f_o) < TOL[prec], (misa.tile_shapes()[t - 1], nerr(f, f_o))
        if ref is None:
            ref = f
        else:
            # the per-site sum order does not depend on the tile shape
            np.testing.assert_array_equal(f, ref)


def test_fp64_trajectory_matches_oracle(misa, pot, oracle, opot):
    # the plain FP64 workload: 10^3 cells, 600 K (seed 0), dt = 1 fs, 100 steps
    n = 10
    x0 = synth.bcc_positions(n, n, n)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 0)
    L = synth.box(n, n, n)
    with misa.Sim(pot, n, precision="fp64", dt_max=1.0, dx_max=0.0, reassign_period=1) as s:
        s.set_velocities(v0)
        s.step(100)
        x = s.positions()
        v = s.velocities()
        st = s.stats()
    xo, vo, _, t, _ = oracle.md_run(opot, x0, v0, L, M, 1.0, 0.0, 100, mode=1)
    d = x - xo
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(v, vo, rtol=0, atol=1e-9)
    assert st["step"] == 100 and abs(st["time"] - 100.0) < 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cascade_trajectory_with_runaways(misa, pot, oracle, opot, prec):
    # knock-on atom, adaptive timestep, atoms leaving and re-entering sites:
    # the run-away list, demotion, re-homing and promotion all move atoms
    # between storage kinds while the physics must follow the oracle
    n = 8
    x0 = synth.cascade_snapshot(n, n, n, 0.1, 6, 2, 11)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 4)
    pka = synth.pka_atom(n, n, n)
    d = synth.random_direction(9)
    oracle.insert_pka(v0, pka, M, 300.0, d)
    L = synth.box(n, n, n)
    steps = 60
    with misa.Sim(pot, n, precision=prec, dt_max=1.0, dx_max=0.02, reassign_period=3) as s:
        s.set_state(x0, v0)
        n_ra0 = s.stats()["n_runaway"]
        s.step(steps)
        x = s.positions()
        st = s.stats()
        sa, ra = s.site_map()
    xo, vo, _, t, _ = oracle.md_run(opot, x0, v0, L, M, 1.0, 0.02, steps, mode=1)
    dd = x - xo
    dd -= L * np.round(dd / L)
    tol = 1e-8 if prec == "fp64" else 2e-5
    assert np.abs(dd).max() < tol, np.abs(dd).max()
    assert abs(st["time"] - t) < (1e-10 if prec == "fp64" else 1e-6)
    assert n_ra0 > 0 and st["status"] & 0x3 == 0
    # storage: every atom exactly once
    allid = np.concatenate([sa[sa >= 0], ra])
    assert len(allid) == len(x0) and len(np.unique(allid)) == len(x0)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_nve_drift(misa, pot, prec):
    # per-atom total-energy drift below 1e-4 eV over 1000 steps of 1 fs
    n = 10
    with misa.Sim(pot, n, precision=prec, dt_max=1.0) as s:
        s.set_velocities(synth.maxwell_velocities(2 * n ** 3, 600.0, M, 0))
        pe0, ke0 = s.energies()
        es = []
        for _ in range(10):
            s.step(100)
            pe, ke = s.energies()
            es.append(pe + ke)
    drift = np.max(np.abs(np.array(es) - (pe0 + ke0))) / (2 * n ** 3)
    assert drift < 1e-4, drift


def test_nve_drift_cascade_adaptive_dt(misa, pot):
    # the same bound through a knock-on cascade: adaptive timestep, run-aways,
    # hash updates every 5 steps, 1000 steps
    n = 10
    with misa.Sim(pot, n, precision="fp32", dt_max=1.0, dx_max=0.02, reassign_period=5) as s:
        s.set_velocities(synth.maxwell_velocities(2 * n ** 3, 300.0, M, 11))
        s.insert_pka(-1, 1000.0, synth.random_direction(12))
        pe0, ke0 = s.energies()
        es = []
        for _ in range(10):
            s.step(100)
            pe, ke = s.energies()
            es.append(pe + ke)
        st = s.stats()
    assert st["status"] == 0 and st["step"] == 1000
    drift = np.max(np.abs(np.array(es) - (pe0 + ke0))) / (2 * n ** 3)
    assert drift < 1e-4, drift


def test_alg2_invariants_on_device(misa, pot, oracle):
    n, skin = 8, 0.6
    x0 = synth.cascade_snapshot(n, n, n, 0.12, 12, 4, 5)
    v0 = synth.maxwell_velocities(len(x0), 900.0, M, 5)
    oracle.insert_pka(v0, synth.pka_atom(n, n, n), M, 500.0, synth.random_direction(2))
    with misa.Sim(pot, n, precision="fp32", dx_max=0.05, reassign_period=1, skin=skin) as s:
        s.set_state(x0, v0)
        s.step(40)
        x = s.positions()
        sa, ra = s.site_map()
    L = synth.box(n, n, n)
    sites = synth.bcc_positions(n, n, n)
    allid = np.concatenate([sa[sa >= 0], ra])
    assert len(allid) == len(x) and len(np.unique(allid)) == len(x)
    occ = np.flatnonzero(sa >= 0)
    d = x[sa[occ]] - sites[occ]
    d -= L * np.round(d / L)
    assert np.linalg.norm(d, axis=1).max() <= skin + 1e-9
    # after a hash update no run-away sits within the skin of an empty nearest site
    for i in ra:
        s_ = oracle.nearest_site(n, n, n, synth.A0_FE, x[i])
        dd = x[i] - sites[s_]
        dd -= L * np.round(dd / L)
        assert not (sa[s_] < 0 and np.linalg.norm(dd) <= skin - 1e-9)
    # run-away list is kept in ascending atom id
    assert np.all(np.diff(ra) > 0)


def test_determinism_and_checkpoint(misa, pot, tmp_path):
    n = 8
    x0 = synth.cascade_snapshot(n, n, n, 0.1, 8, 2, 6)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 6)

    def run(k1, k2, ck=None):
        with misa.Sim(pot, n, precision="fp32", dx_max=0.02, reassign_period=2) as s:
            s.set_state(x0, v0)
            s.step(k1)
            if ck is not None:
                s.save(ck)
            s.step(k2)
            return s.positions(), s.velocities()

    xa, va = run(20, 20)
    xb, vb = run(20, 20, tmp_path / "c.bin")
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(va, vb)
    with misa.Sim(pot, n, precision="fp32", dx_max=0.02, reassign_period=2) as s:
        s.load(tmp_path / "c.bin")
        s.step(20)
        xc, vc = s.positions(), s.velocities()
    np.testing.assert_array_equal(xa, xc)
    np.testing.assert_array_equal(va, vc)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_staged_state_equals_set_state(misa, pot, prec):
    import torch
    n = 8
    x0 = synth.cascade_snapshot(n, n, n, 0.1, 8, 2, 6)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 6)
    x1 = synth.cascade_snapshot(n, n, n, 0.12, 6, 3, 9)
    v1 = synth.maxwell_velocities(len(x1), 900.0, M, 9)

    def direct(x, v, k):
        with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=2) as s:
            s.set_state(x, v)
            s.step(k)
            return s.positions(), s.velocities(), s.forces()

    ref0, ref1 = direct(x0, v0, 7), direct(x1, v1, 5)
    with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=2) as s:
        with pytest.raises(misa.MisaError) as e:
            s.set_state_staged()
        assert e.value.code == misa.MISA_EINVAL
        # pinned host tensors, the second state streaming in during the steps
        s.stage_state(torch.from_numpy(x0).pin_memory(), torch.from_numpy(v0).pin_memory())
        s.set_state_staged()
        s.stage_state(torch.from_numpy(x1).pin_memory(), torch.from_numpy(v1).pin_memory())
        s.step(7)
        got0 = (s.positions(), s.velocities(), s.forces())
        s.set_state_staged()
        s.step(5)
        got1 = (s.positions(), s.velocities(), s.forces())
        # numpy host arrays; without velocities the atoms start at rest
        s.stage_state(x0)
        s.set_state_staged()
        assert not np.any(s.velocities())
        with pytest.raises(misa.MisaError):
            s.set_state_staged()
    for ref, got in ((ref0, got0), (ref1, got1)):
        for a, b in zip(ref, got):
            np.testing.assert_array_equal(a, b)


def test_pka_and_adaptive_dt(misa, pot):
    n = 8
    with misa.Sim(pot, n, precision="fp64", dt_max=1.0, dx_max=0.02) as s:
        d = np.array([1.0, 2.0, 2.0])
        s.insert_pka(-1, 5000.0, d)
        v = s.velocities()
        pka = synth.pka_atom(n, n, n)
        ke = 0.5 * M * np.dot(v[pka], v[pka]) * synth.EV_PER_AMU_A2_FS2
        assert ke == pytest.approx(5000.0, rel=1e-12)
        np.testing.assert_allclose(v[pka] / np.linalg.norm(v[pka]), d / 3.0, atol=1e-14)
        st = s.stats()
        assert st["dt"] == pytest.approx(0.02 / np.linalg.norm(v[pka]), rel=1e-12)
        s.step(3)
        st = s.stats()
        assert st["time"] < 0.1


def test_runaway_overflow_is_reported(misa, pot):
    x = synth.cascade_snapshot(8, 8, 8, 0.1, 12, 0, 7)
    with misa.Sim(pot, 8, precision="fp32", runaway_capacity=4) as s:
        s.set_state(x)
        with pytest.raises(misa.MisaError) as e:
            s.forces()
        assert e.value.code == misa.MISA_ERUNAWAY_OVERFLOW
        assert s.stats()["status"] & misa.ST_RUNAWAY_OVERFLOW


def test_shortcuts_match_exact_counterparts(misa):
    # the FP64 integration kernels convert float <-> double with integer
    # operations; they must agree bit for bit with the GPU's conversions.
    # Setting a state hashes atoms with the site decided in FP32 under a
    # certifying margin; it must agree bit for bit with the FP64 hash.
    assert misa.selftest(1 << 22) == (0, 0, 0)


def test_frenkel_pairs_match_oracle(misa, pot, oracle):
    # Wigner-Seitz count on the device (site array + run-away homes) against
    # the oracle's nearest-site occupancy of the same positions: after
    # set_state on cascade snapshots, and after a knock-on cascade has run
    a0 = synth.A0_FE
    for dims, x in (((12, 9, 10), synth.cascade_snapshot(12, 9, 10, 0.12, 24, 8, 2)),
                    ((6, 6, 6), synth.cascade_snapshot(6, 6, 6, 0.1, 5, 3, 3))):
        with misa.Sim(pot, *dims, precision="fp32") as s:
            s.set_state(x)
            nf = s.defects()
            nv, ni = oracle.ws_defects(*dims, a0, s.positions())
            assert nv == ni == int(nf[0]) > 0
    n = 10
    with misa.Sim(pot, n, precision="fp32", dx_max=0.02, reassign_period=5) as s:
        s.set_state(synth.thermal_snapshot(n, n, n, 0.08, 5),
                    synth.maxwell_velocities(2 * n ** 3, 300.0, synth.MASS_FE, 6))
        s.insert_pka(-1, 2000.0, synth.random_direction(7))
        counts = []
        for _ in range(6):
            s.step(100)
            nv, ni = oracle.ws_defects(n, n, n, a0, s.positions())
            counts.append(int(s.defects()[0]))
            assert nv == ni == counts[-1]
        assert max(counts) > 0


def edge_snapshot(n=8, seed=13):
    """A thermal crystal with the two edge readings of Sec. 2.2 built in:
    one atom moved 5e-5 A from a lattice atom and two atoms 5e-5 A apart at
    an octahedral interstitial point (pairs below r_floor = 1e-4 A: values at
    r_floor, no force), and six atoms moved to 0.5 A around a lattice atom
    along the axes (densities above rho_max: linear embedding tail).  The
    moved atoms become run-aways and leave vacancies behind."""
    x = synth.thermal_snapshot(n, n, n, 0.05, seed)
    a0 = synth.A0_FE
    rng = np.random.default_rng(seed)
    movers = rng.choice(np.arange(2, len(x), 2), 9, replace=False)
    host_a, host_c = 2 * (n * n * 2 + n * 2 + 2), 2 * (n * n * 5 + n * 5 + 5) + 1
    assert host_a not in movers and host_c not in movers
    x[movers[0]] = x[host_a] + 5e-5 * np.array([0.6, 0.0, 0.8])
    octa = np.array([4.5, 4.0, 3.0]) * a0  # face centre of a cube: an octahedral site
    x[movers[1]] = octa
    x[movers[2]] = octa + 5e-5 * np.array([0.0, 0.8, 0.6])
    for k, (d, s) in enumerate([(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)]):
        e = np.zeros(3)
        e[d] = 0.5 * s
        x[movers[3 + k]] = x[host_c] + e
    return np.mod(x, synth.box(n, n, n)), (host_a, host_c, movers)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_edge_readings_against_oracle(misa, pot, oracle, opot, prec):
    # the CUDA path leaves the plain formula in two places -- pairs closer
    # than r_floor and densities above rho_max -- and must follow the
    # oracle's readings there atom by atom, reporting both status bits
    n = 8
    x, (host_a, host_c, movers) = edge_snapshot(n)
    L = synth.box(n, n, n)
    rho_o, _, e_o, f_o = oracle.eam(opot, x, L, mode=1)
    assert np.sum(rho_o > pot.rho_max) >= 7
    with misa.Sim(pot, n, precision=prec) as s:
        s.set_state(x)
        f = s.forces()
        rho = s.density()
        _, _, e = s.energies(per_atom=True)
        st = s.stats()
    assert st["n_runaway"] >= 8
    assert st["status"] & misa.ST_RFLOOR and st["status"] & misa.ST_RHO_EXTRAP
    assert st["status"] & 0x3 == 0
    assert nerr(f, f_o) < TOL[prec], nerr(f, f_o)
    assert nerr(rho, rho_o) < TOL[prec], nerr(rho, rho_o)
    assert nerr(e, e_o) < TOL[prec], nerr(e, e_o)
    # the dimers' partners pull on nothing: the oracle's force on the two
    # interstitials 5e-5 A apart is the crystal's alone, and the GPU agrees
    # with it there to the same bound
    sel = np.concatenate([[host_a, host_c], movers])
    assert nerr(f[sel], f_o[sel]) < TOL[prec]


@pytest.mark.parametrize("case", list(CASES))
def test_newton3_density_variant_against_oracle(misa, pot, oracle_results, case):
    # the density pass with Newton's third law inside tiles (Sec. 4.2's pair
    # halving, no atomics): every tile shape bitwise equal to every other, and
    # densities, energies and forces within the FP32 bound of the oracle
    x, dims, rho_o, e_o, f_o = oracle_results[case]
    ref = None
    for t in misa.tile_indices("fp32"):
        with misa.Sim(pot, *dims, precision="fp32", tile=t) as s:
            s.set_density_variant(1)
            s.set_state(x)
            f = s.forces()
            rho = s.density()
            _, _, e = s.energies(per_atom=True)
            st = s.stats()
        assert st["status"] & 0x3 == 0
        assert nerr(f, f_o) < TOL["fp32"], (t, nerr(f, f_o))
        assert nerr(rho, rho_o) < TOL["fp32"], (t, nerr(rho, rho_o))
        assert nerr(e, e_o) < TOL["fp32"], (t, nerr(e, e_o))
        if ref is None:
            ref = (f, rho, e)
        else:
            for a_, b_ in zip(ref, (f, rho, e)):
                np.testing.assert_array_equal(a_, b_)


def test_newton3_density_variant_trajectory(misa, pot, oracle, opot):
    # the cascade trajectory of test_cascade_trajectory_with_runaways through
    # the Newton-3 density pass, and the variant switched back and forth
    n = 8
    x0 = synth.cascade_snapshot(n, n, n, 0.1, 6, 2, 11)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 4)
    oracle.insert_pka(v0, synth.pka_atom(n, n, n), M, 300.0, synth.random_direction(9))
    L = synth.box(n, n, n)
    with misa.Sim(pot, n, precision="fp32", dt_max=1.0, dx_max=0.02, reassign_period=3) as s:
        s.set_state(x0, v0)
        s.set_density_variant(1)
        s.step(30)
        s.set_density_variant(0)
        s.set_density_variant(1)
        s.step(30)
        x = s.positions()
        st = s.stats()
    xo, _, _, t, _ = oracle.md_run(opot, x0, v0, L, M, 1.0, 0.02, 60, mode=1)
    dd = x - xo
    dd -= L * np.round(dd / L)
    assert np.abs(dd).max() < 2e-5, np.abs(dd).max()
    assert abs(st["time"] - t) < 1e-6 and st["status"] & 0x3 == 0
    with misa.Sim(pot, n, precision="fp64") as s:
        with pytest.raises(misa.MisaError) as e:
            s.set_density_variant(1)
        assert e.value.code == misa.MISA_EINVAL


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("dims,nint", [((12, 12, 12), 1100), ((13, 9, 10), 300)])
def test_runaway_index_with_many_interstitials(misa, pot, oracle, opot, prec, dims, nint):
    # atoms on octahedral interstitial points.  12^3 cells, 1,100 of them: the
    # per-tile run-away index of a large tile overflows its sortable segment
    # (the tile scans the whole list), small tiles are indexed.  13 x 9 x 10
    # cells: 4-cell tiles leave partial last tiles of 1-2 cells, so a
    # run-away's window across the periodic wrap meets four tiles along an
    # axis.  Every tile shape gives bitwise the same result, and the oracle's
    x = synth.interstitial_snapshot(*dims, 0.05, nint, 21)
    L = synth.box(*dims)
    rho_o, _, e_o, f_o = oracle.eam(opot, x, L, mode=1)
    ref = None
    for t in misa.tile_indices(prec):
        with misa.Sim(pot, *dims, precision=prec, tile=t) as s:
            s.set_state(x)
            f = s.forces()
            rho = s.density()
            _, _, e = s.energies(per_atom=True)
            st = s.stats()
        assert st["n_runaway"] == nint and st["status"] & 0x3 == 0
        assert nerr(f, f_o) < TOL[prec], (t, nerr(f, f_o))
        assert nerr(rho, rho_o) < TOL[prec] and nerr(e, e_o) < TOL[prec]
        if ref is None:
            ref = (f, rho, e)
        else:
            for a_, b_ in zip(ref, (f, rho, e)):
                np.testing.assert_array_equal(a_, b_)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_energy_step_equals_separate_evaluation(misa, pot, prec):
    # energies evaluated inside the last step's passes (misa_step_energies)
    # are bitwise those of a separate evaluation after plain steps, for the
    # direct and the graph-replayed step; a later plain step invalidates them
    n = 8
    x0 = synth.cascade_snapshot(n, n, n, 0.1, 6, 2, 11)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 4)
    out = []
    for energies, graphs in ((False, True), (True, True), (True, False)):
        with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=3) as s:
            s.set_graphs(graphs)
            s.set_state(x0, v0)
            s.insert_pka(-1, 300.0, synth.random_direction(9))
            s.step(7, energies=energies)
            l0 = s.stats()["launches"]
            pe, ke, e = s.energies(per_atom=True)
            evaluated = s.stats()["launches"] - l0
            out.append((s.positions(), s.velocities(), pe, ke, e, evaluated))
            s.step(2, energies=energies)
            s.step(1)
            pe2, _, e2 = s.energies(per_atom=True)
            out[-1] = out[-1] + (pe2, e2)
    ref = out[0]
    for got in out[1:]:
        for k in (0, 1, 4, 7):
            np.testing.assert_array_equal(got[k], ref[k])
        assert got[2] == ref[2] and got[3] == ref[3] and got[6] == ref[6]
    # the energy step saved the evaluation's launches
    assert out[1][5] < ref[5] and out[2][5] < ref[5]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("nint", [12, 300])
def test_runaway_index_follows_state_changes(misa, pot, prec, nint, tmp_path):
    # A force evaluation outside a step reuses the per-tile run-away index
    # while the run-away list is unchanged; set_state, steps and a checkpoint
    # load must rebuild it.  Each result is compared bitwise with a fresh
    # handle's.  12 run-aways: the walkers scan the whole list; 300: they
    # use the index.
    n = 10
    xa = synth.interstitial_snapshot(n, n, n, 0.05, nint, 31)
    xb = synth.interstitial_snapshot(n, n, n, 0.05, nint + 7, 32)
    vb = synth.maxwell_velocities(len(xb), 600.0, M, 5)

    def fields(s):
        _, _, e = s.energies(per_atom=True)
        return s.forces(), s.density(), e

    with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=2) as s:
        s.set_state(xa)
        first = fields(s)
        np.testing.assert_array_equal(fields(s)[0], first[0])  # evaluation with the cached index
        s.set_state(xb, vb)
        got_b = fields(s)
        s.step(5)
        got_c = fields(s)
        ck = str(tmp_path / "state.ckpt")
        s.save(ck)
        st = s.stats()
    assert st["n_runaway"] >= nint and st["status"] & 0x3 == 0
    with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=2) as t:
        t.set_state(xb, vb)
        ref_b = fields(t)
    for a_, b_ in zip(got_b, ref_b):
        np.testing.assert_array_equal(a_, b_)
    with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=2) as t:
        t.set_state(xa)
        fields(t)
        t.load(ck)
        ref_c = fields(t)
    for a_, b_ in zip(got_c, ref_c):
        np.testing.assert_array_equal(a_, b_)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_energies_async_equal_synchronous_read(misa, pot, prec):
    # misa_get_energies_async hands back, once misa_wait_outputs has
    # returned, bitwise the E_i that misa_get_energies reads; steps issued
    # after it run beside the copy and do not disturb it; a second call
    # waits for the first copy before it overwrites the handle's buffer
    import torch
    n = 8
    x0 = synth.cascade_snapshot(n, n, n, 0.1, 6, 2, 13)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 7)
    ref = []
    with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=3) as s:
        s.set_state(x0, v0)
        for _ in range(2):
            s.step(4, energies=True)
            ref.append(s.energies(per_atom=True)[2].copy())
    bufs = [torch.zeros(len(x0), dtype=torch.float64).pin_memory() for _ in range(2)]
    with misa.Sim(pot, n, precision=prec, dx_max=0.02, reassign_period=3) as s:
        s.set_state(x0, v0)
        for k in range(2):
            s.step(4, energies=True)
            s.energies_async(bufs[k])
        s.step(3)  # runs beside the second copy
        s.wait_outputs()
        for k in range(2):
            np.testing.assert_array_equal(bufs[k].numpy(), ref[k])
        # without a preceding energy step the call evaluates the potential
        pe, _, e = s.energies(per_atom=True)
        out = np.zeros(len(x0))
        s.step(1)
        s.energies_async(out)
        s.wait_outputs()
        _, _, e1 = s.energies(per_atom=True)
        np.testing.assert_array_equal(out, e1)


def test_destroy_waits_for_async_energies(misa, pot):
    # closing the handle right after misa_get_energies_async waits for the
    # copy: the host buffer holds the energies afterwards
    import torch
    n = 8
    x0 = synth.thermal_snapshot(n, n, n, 0.1, 17)
    buf = torch.zeros(len(x0), dtype=torch.float64).pin_memory()
    with misa.Sim(pot, n, precision="fp32") as s:
        s.set_state(x0)
        ref = s.energies(per_atom=True)[2].copy()
        s.energies_async(buf)
    np.testing.assert_array_equal(buf.numpy(), ref)
