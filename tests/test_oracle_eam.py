"""Pins of the oracle's EAM evaluation (Eq. eam_base, Eq. eam_force_ij, the
five steps of Sec. 2.2): closed forms on the perfect crystal and on a dimer,
reduction to a plain pair potential, forces as the negative energy gradient,
Newton's third law, and brute force == cell list == sampled evaluation."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

A0 = synth.A0_FE


def _shell_closed_form(rc=synth.RC):
    fs, _ = synth.truncated(synth.f_analytic, synth.df_analytic, rc)
    ps, _ = synth.truncated(synth.phi_analytic, synth.dphi_analytic, rc)
    rho = 0.0
    pair = 0.0
    m = 6
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                if (i % 2 == j % 2 == k % 2) and (i or j or k):
                    d = 0.5 * A0 * np.sqrt(i * i + j * j + k * k)
                    if d < rc:
                        rho += float(fs(d))
                        pair += 0.5 * float(ps(d))
    return rho, float(synth.embed_analytic(rho)) + pair


def test_perfect_crystal_closed_form_and_zero_force(oracle, opot):
    rho_eq, e_coh = _shell_closed_form()
    assert e_coh == pytest.approx(-8.97196806, abs=1e-7)
    x = synth.bcc_positions(6, 5, 7)
    L = synth.box(6, 5, 7)
    for mode in (0, 1):
        rho, fp, e, f = oracle.eam(opot, x, L, mode=mode)
        np.testing.assert_allclose(rho, rho_eq, rtol=0, atol=1e-9)
        np.testing.assert_allclose(e, e_coh, rtol=0, atol=1e-9)
        np.testing.assert_allclose(fp, -0.9 / np.sqrt(rho_eq), rtol=0, atol=1e-9)
        # inversion symmetry: zero force up to the rounding of the positions
        assert np.abs(f).max() < 1e-11


def test_dimer_closed_form(oracle, opot):
    # two atoms in a box much larger than rc: rho = f(r) for both,
    # E = 2 F(f(r)) + phi(r), |F| = 2 F'(f(r)) f'(r) + phi'(r) along the bond
    L = np.array([30.0, 30.0, 30.0])
    fs, dfs = synth.truncated(synth.f_analytic, synth.df_analytic)
    ps, dps = synth.truncated(synth.phi_analytic, synth.dphi_analytic)
    # (rho stays above ~0.3, where the sqrt embedding table is accurate)
    for r in [1.9, 2.5, 3.0, 3.4]:
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r / np.sqrt(3), 10.0 + r / np.sqrt(3), 10.0 + r / np.sqrt(3)]])
        rho, fp, e, f = oracle.eam(opot, x, L, mode=0)
        rho_a = float(fs(r))
        np.testing.assert_allclose(rho, rho_a, rtol=1e-9)
        e_a = 2 * float(synth.embed_analytic(rho_a)) + float(ps(r))
        assert e.sum() == pytest.approx(e_a, rel=1e-8)
        mag = 2 * (-0.9 / np.sqrt(rho_a)) * float(dfs(r)) + float(dps(r))
        u = (x[0] - x[1]) / r
        np.testing.assert_allclose(f[0], -mag * u, rtol=1e-6, atol=1e-9)
        np.testing.assert_allclose(f[1], mag * u, rtol=1e-6, atol=1e-9)


def test_pair_potential_limit(oracle, pot):
    # F == 0: EAM is the plain pair potential phi; compare with a direct
    # numpy pair sum of the analytic truncated phi'.
    p0 = synth.Potential(pot.n, pot.rc, pot.rho_max, pot.f, pot.phi, np.zeros_like(pot.F))
    op = oracle.Pot(p0)
    x = synth.thermal_snapshot(5, 5, 5, 0.12, 4)
    L = synth.box(5, 5, 5)
    _, _, e, f = oracle.eam(op, x, L, mode=0)
    ps, dps = synth.truncated(synth.phi_analytic, synth.dphi_analytic)
    d = x[:, None, :] - x[None, :, :]
    d -= L * np.round(d / L)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    inside = r < pot.rc
    fr = np.where(inside, dps(np.where(inside, r, 1.0)), 0.0)
    fref = -(fr / r)[:, :, None] * d
    np.testing.assert_allclose(f, fref.sum(1), rtol=0, atol=2e-8)
    eref = 0.5 * np.where(inside, ps(np.where(inside, r, 1.0)), 0.0).sum(1)
    np.testing.assert_allclose(e, eref, rtol=0, atol=1e-9)


def _total_energy(oracle, op, x, L):
    return oracle.eam(op, x, L, mode=0)[2].sum()


def test_force_is_minus_energy_gradient(oracle, opot):
    x = synth.cascade_snapshot(5, 5, 5, 0.15, 3, 2, 7)
    L = synth.box(5, 5, 5)
    _, _, _, f = oracle.eam(opot, x, L, mode=0)
    h = 1e-5
    rng = np.random.default_rng(5)
    for i in rng.choice(len(x), 6, replace=False):
        for d in range(3):
            xp = x.copy(); xp[i, d] += h
            xm = x.copy(); xm[i, d] -= h
            g = (_total_energy(oracle, opot, xp, L) - _total_energy(oracle, opot, xm, L)) / (2 * h)
            assert -g == pytest.approx(f[i, d], rel=1e-7, abs=1e-7 * max(1.0, abs(f[i, d])))


def test_newton_third_law_and_modes_agree(oracle, opot):
    x = synth.cascade_snapshot(6, 6, 6, 0.15, 5, 3, 9)
    L = synth.box(6, 6, 6)
    r0, fp0, e0, f0 = oracle.eam(opot, x, L, mode=0)
    r1, fp1, e1, f1 = oracle.eam(opot, x, L, mode=1)
    np.testing.assert_allclose(r1, r0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(e1, e0, rtol=0, atol=1e-12)
    np.testing.assert_allclose(f1, f0, rtol=0, atol=1e-11)
    assert np.abs(f0.sum(0)).max() < 1e-10 * max(1.0, np.abs(f0).max() * len(x))
    t = np.array([0, 17, 99, 250, 431])
    rs, es, fs = oracle.eam_sample(opot, x, L, t)
    np.testing.assert_allclose(rs, r0[t], atol=1e-12)
    np.testing.assert_allclose(es, e0[t], atol=1e-12)
    np.testing.assert_allclose(fs, f0[t], atol=1e-11)


def test_small_box_explicit_images(oracle, opot):
    # boxes of 3 and 4 cells (8.6 and 11.4 A) are shorter than rc or 2 rc, so
    # atoms meet several periodic images of the same neighbour (or of
    # themselves); the perfect crystal still gives the closed-form energy
    rho_eq, e_coh = _shell_closed_form()
    for n in (3, 4):
        x = synth.bcc_positions(n, n, n)
        L = synth.box(n, n, n)
        rho, _, e, f = oracle.eam(opot, x, L, mode=0)
        np.testing.assert_allclose(rho, rho_eq, atol=1e-9)
        np.testing.assert_allclose(e, e_coh, atol=1e-9)
        assert np.abs(f).max() < 1e-10
