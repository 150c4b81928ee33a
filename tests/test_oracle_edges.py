"""Pins of the oracle's two edge readings of Sec. 2.2 / Sec. 4.1, where the
plain formula has no value:

* r < r_floor = 1e-4 A (a head-on collision brings two atoms together): the
  pair contributes the tables' values at r_floor and no force, since the
  direction of the pair is undefined;
* rho > rho_max (the embedding table ends at 4 rho_eq): F continues linearly
  with the table's end value and slope; the knot gradient of the fitting loss
  then takes the linear tail's weights.

Each pin checks the oracle against the analytic potential the tables were
made from (not against the oracle's own spline), against central
differences of the oracle's energy or loss, or against both."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

R_FLOOR = 1e-4
BIG = np.array([30.0, 30.0, 30.0])  # no periodic image within rc


def _analytic():
    fs, dfs = synth.truncated(synth.f_analytic, synth.df_analytic)
    ps, dps = synth.truncated(synth.phi_analytic, synth.dphi_analytic)
    return fs, dfs, ps, dps


def test_close_pair_below_r_floor_has_floor_values_and_no_force(oracle, opot):
    # a dimer at r = 5e-5 A: both atoms see f(r_floor) and half of
    # phi(r_floor); neither feels a force
    fs, _, ps, _ = _analytic()
    r = 5e-5
    u = np.array([1.0, 2.0, 2.0]) / 3.0
    x = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0] + r * u])
    for mode in (0, 1):
        rho, fp, e, f = oracle.eam(opot, x, BIG, mode=mode)
        rho_a = float(fs(R_FLOOR))
        np.testing.assert_allclose(rho, rho_a, rtol=1e-9)
        e_a = 2.0 * float(synth.embed_analytic(rho_a)) + float(ps(R_FLOOR))
        assert e.sum() == pytest.approx(e_a, rel=1e-7)
        # the value at r itself differs by phi'(0) * 5e-5 A ~ 0.26 eV (1.6e-4
        # relative): a floor that is not applied fails the bound above
        e_at_r = 2.0 * float(synth.embed_analytic(float(fs(r)))) + float(ps(r))
        assert abs(e_at_r - e_a) > 1e3 * 1e-7 * abs(e_a)
        assert np.all(f == 0.0)


def test_close_pair_just_above_r_floor_has_the_analytic_force(oracle, opot):
    # the floor branch covers r < r_floor only: at 3 r_floor the force is the
    # analytic 2 F'(f) f' + phi' along the bond
    fs, dfs, ps, dps = _analytic()
    r = 3e-4
    u = np.array([2.0, -1.0, 2.0]) / 3.0
    x = np.array([[10.0, 11.0, 12.0], [10.0, 11.0, 12.0] + r * u])
    _, _, e, f = oracle.eam(opot, x, BIG, mode=0)
    rho_a = float(fs(r))
    mag = 2.0 * (-0.9 / np.sqrt(rho_a)) * float(dfs(r)) + float(dps(r))
    # Hermite end slopes are second order next to r = 0: ~1e-5 relative there
    np.testing.assert_allclose(f[0], mag * u, rtol=2e-5)
    np.testing.assert_allclose(f[1], -mag * u, rtol=2e-5)
    assert e.sum() == pytest.approx(2.0 * float(synth.embed_analytic(rho_a)) + float(ps(r)), rel=1e-7)


def _cluster():
    """An atom with six neighbours at 0.5 A along the axes (rho ~ 64 at the
    centre, ~50 at the six: all above rho_max = 47.3), one atom at 2.3 A
    (below rho_max), and apart from them a dimer at 5e-5 A (below r_floor)."""
    c = np.array([8.0, 9.0, 10.0])
    x = [c]
    for d in range(3):
        for s in (-1.0, 1.0):
            e = np.zeros(3)
            e[d] = s * 0.5
            x.append(c + e)
    x.append(c + np.array([1.3, 1.2, -1.4]))
    far = np.array([20.0, 21.0, 22.0])
    x.append(far)
    x.append(far + 5e-5 * np.array([0.0, 0.6, 0.8]))
    return np.array(x)


def _linear_tail_energy(rho, rho_max):
    """F(rho) of the analytic embedding, continued linearly above rho_max."""
    F = synth.embed_analytic
    dF = -0.9 / np.sqrt(rho_max)
    return np.where(rho > rho_max, float(F(rho_max)) + dF * (rho - rho_max), F(np.minimum(rho, rho_max)))


def test_density_above_rho_max_continues_linearly(oracle, pot, opot):
    fs, _, ps, _ = _analytic()
    x = _cluster()
    rho, fp, e, f = oracle.eam(opot, x, BIG, mode=0)
    # plain analytic sums over all pairs (r_floor applied to the dimer)
    d = x[:, None, :] - x[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    inside = r < synth.RC
    rr = np.where(inside, np.maximum(r, R_FLOOR), 1.0)
    rho_a = np.where(inside, fs(rr), 0.0).sum(1)
    np.testing.assert_allclose(rho, rho_a, rtol=1e-8)
    above = rho_a > pot.rho_max
    assert above.sum() == 7 and (~above).sum() == 3
    e_a = _linear_tail_energy(rho_a, pot.rho_max) + 0.5 * np.where(inside, ps(rr), 0.0).sum(1)
    np.testing.assert_allclose(e, e_a, rtol=1e-7)
    # F'(rho) above rho_max is the end slope of the table: F'(rho_max)
    np.testing.assert_allclose(fp[above], -0.9 / np.sqrt(pot.rho_max), rtol=1e-6)


def test_forces_above_rho_max_are_minus_the_energy_gradient(oracle, opot):
    x = _cluster()
    _, _, _, f = oracle.eam(opot, x, BIG, mode=0)
    h = 1e-6
    for i in (0, 1, 4, 7):
        for d in range(3):
            xp = x.copy(); xp[i, d] += h
            xm = x.copy(); xm[i, d] -= h
            ep = oracle.eam(opot, xp, BIG, mode=0)[2].sum()
            em = oracle.eam(opot, xm, BIG, mode=0)[2].sum()
            g = (ep - em) / (2 * h)
            assert -g == pytest.approx(f[i, d], rel=2e-7, abs=1e-6)
    # the close dimer feels nothing from its partner below r_floor
    assert np.all(f[8:] == 0.0)


def _loss(oracle, pot, x, L, Fref, Eref):
    return oracle.loss_grad(oracle.Pot(pot), x, L, Fref, Eref)[0]


def test_gradient_above_rho_max_and_below_r_floor_matches_central_differences(oracle, pot):
    # the knot gradient where the linear tail of F and the r_floor values are
    # used: F knots that fix the tail (the last three define the end slope),
    # f and phi knots of the 0.5-1.1 A pairs, and the first f and phi knots
    # (the dimer's values at r_floor)
    x = _cluster()
    ef, ep, eF = synth.knot_perturbation(pot.n, 0.02, 31)
    target = pot.scaled(ef, ep, eF)
    _, _, e_t, f_t = oracle.eam(oracle.Pot(target), x, BIG, mode=0)
    Eref = e_t.sum() + 3.0  # a nonzero energy residual
    loss, g, _, _ = oracle.loss_grad(oracle.Pot(pot), x, BIG, f_t, Eref)
    assert loss > 0
    n = pot.n
    hr = pot.rc / (n - 1)
    seg = lambda r: int(r / hr)
    idx = [2 * n + n - 1, 2 * n + n - 2, 2 * n + n - 3]                 # F tail
    idx += [seg(0.5), seg(0.5) + 1, seg(0.7071), seg(1.0) + 1]          # f
    idx += [n + seg(0.5), n + seg(0.7071) + 1, n + seg(1.0)]            # phi
    idx += [0, 1, n, n + 1]                                             # r_floor values
    # the tail knots carry weight only through atoms above rho_max
    assert np.all(g[idx[:3]] != 0.0)
    h = 1e-6
    for k in idx:
        tab, j = divmod(int(k), n)
        arrs = [pot.f.copy(), pot.phi.copy(), pot.F.copy()]
        step = h * max(1.0, abs(arrs[tab][j]))
        arrs[tab][j] += step
        lp = _loss(oracle, synth.Potential(n, pot.rc, pot.rho_max, *arrs), x, BIG, f_t, Eref)
        arrs[tab][j] -= 2 * step
        lm = _loss(oracle, synth.Potential(n, pot.rc, pot.rho_max, *arrs), x, BIG, f_t, Eref)
        fd = (lp - lm) / (2 * step)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9 * np.abs(g).max()), (k, g[k], fd)
