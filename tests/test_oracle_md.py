"""Pins of the oracle's MD loop (Fig. 1 read as kick-drift-kick velocity
Verlet, adaptive timestep, PKA insertion of Sec. 5.1): NVE energy
conservation, time reversibility, momentum conservation, the displacement
bound of the adaptive step, and the PKA's kinetic energy."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

M = synth.MASS_FE


def test_nve_energy_conservation(oracle, opot):
    n = 6
    x = synth.bcc_positions(n, n, n)
    v = synth.maxwell_velocities(len(x), 600.0, M, 0)
    L = synth.box(n, n, n)
    # the criterion's length: per-atom drift below 1e-4 eV over 1000 steps
    _, _, _, _, log = oracle.md_run(opot, x, v, L, M, 1.0, 0.0, 1000, mode=1, log=True)
    et = log[:, 1] + log[:, 2]
    assert len(et) >= 1000
    assert (et.max() - et.min()) / len(x) < 1e-4


def test_time_reversibility(oracle, opot):
    n = 5
    x0 = synth.thermal_snapshot(n, n, n, 0.08, 1)
    v0 = synth.maxwell_velocities(len(x0), 600.0, M, 1)
    L = synth.box(n, n, n)
    x1, v1, a1, _, _ = oracle.md_run(opot, x0, v0, L, M, 1.0, 0.0, 50, mode=0)
    x2, v2, _, _, _ = oracle.md_run(opot, x1, -v1, L, M, 1.0, 0.0, 50, mode=0, a=a1)
    d = x2 - x0
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-v2, v0, atol=1e-10)


def test_momentum_conserved_and_pka_energy(oracle, opot):
    n = 6
    x = synth.bcc_positions(n, n, n)
    v = synth.maxwell_velocities(len(x), 300.0, M, 2)
    L = synth.box(n, n, n)
    pka = oracle.pka_site(n, n, n)
    assert pka == synth.pka_atom(n, n, n)
    np.testing.assert_allclose(x[pka], L / 2, atol=1e-12)  # the box centre
    d = synth.random_direction(3)
    v2 = v.copy()
    oracle.insert_pka(v2, pka, M, 500.0, d)
    assert 0.5 * M * np.dot(v2[pka], v2[pka]) * synth.EV_PER_AMU_A2_FS2 == pytest.approx(500.0, rel=1e-12)
    np.testing.assert_allclose(v2[pka] / np.linalg.norm(v2[pka]), d, atol=1e-12)
    p0 = v2.sum(0)
    _, v3, _, _, _ = oracle.md_run(opot, x, v2, L, M, 1.0, 0.02, 30, mode=1)
    np.testing.assert_allclose(v3.sum(0), p0, atol=1e-9)


def test_adaptive_step_bounds_displacement(oracle, opot):
    n = 6
    x = synth.bcc_positions(n, n, n)
    v = synth.maxwell_velocities(len(x), 600.0, M, 4)
    oracle.insert_pka(v, oracle.pka_site(n, n, n), M, 2000.0, synth.random_direction(5))
    L = synth.box(n, n, n)
    dx_max = 0.02
    xs, vs = x, v
    a = None
    for _ in range(10):
        vmax = np.sqrt((vs * vs).sum(1)).max()
        x1, v1, a, t, _ = oracle.md_run(opot, xs, vs, L, M, 1.0, dx_max, 1, mode=1, a=a)
        assert t == pytest.approx(min(1.0, dx_max / vmax), rel=1e-12)
        d = x1 - xs
        d -= L * np.round(d / L)
        # v dt <= dx_max; the half-kick adds at most a dt^2 / 2
        amax = np.sqrt((a * a).sum(1)).max()
        assert np.sqrt((d * d).sum(1)).max() <= dx_max + amax * t * t
        xs, vs = x1, v1
