"""Pins of the oracle's knot gradient of the force-matching + energy loss
(no counterpart in the paper; used to fit potentials): central finite
differences on seeded knots, and the loss at the target tables is zero."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth


def _loss(oracle, pot, x, L, Fref, Eref):
    l, _, _, _ = oracle.loss_grad(oracle.Pot(pot), x, L, Fref, Eref)
    return l


def test_gradient_matches_central_differences(oracle, pot):
    n = 5
    x = synth.thermal_snapshot(n, n, n, 0.12, 21)
    L = synth.box(n, n, n)
    ef, ep, eF = synth.knot_perturbation(pot.n, 0.02, 5)
    target = pot.scaled(ef, ep, eF)
    _, _, e_t, f_t = oracle.eam(oracle.Pot(target), x, L, mode=0)
    Eref = e_t.sum()
    loss, g, _, _ = oracle.loss_grad(oracle.Pot(pot), x, L, f_t, Eref)
    assert loss > 0
    # knots the configuration actually touches: f/phi segments of occupied
    # distances, F segments around the densities; plus a few random ones
    rho = oracle.eam(oracle.Pot(pot), x, L, mode=0)[0]
    hr = pot.rc / (pot.n - 1)
    hrho = pot.rho_max / (pot.n - 1)
    rng = np.random.default_rng(8)
    idx = list(rng.choice(np.flatnonzero(np.abs(g[:pot.n]) > 0), 10, replace=False))
    idx += list(pot.n + rng.choice(np.flatnonzero(np.abs(g[pot.n:2 * pot.n]) > 0), 10, replace=False))
    idx += list(2 * pot.n + np.unique((rho / hrho).astype(int))[:8])
    idx += list(rng.choice(3 * pot.n, 4, replace=False))
    h = 1e-6
    for k in idx:
        tab, j = divmod(int(k), pot.n)
        arrs = [pot.f.copy(), pot.phi.copy(), pot.F.copy()]
        step = h * max(1.0, abs(arrs[tab][j]))
        arrs[tab][j] += step
        lp = _loss(oracle, synth.Potential(pot.n, pot.rc, pot.rho_max, *arrs), x, L, f_t, Eref)
        arrs[tab][j] -= 2 * step
        lm = _loss(oracle, synth.Potential(pot.n, pot.rc, pot.rho_max, *arrs), x, L, f_t, Eref)
        fd = (lp - lm) / (2 * step)
        assert g[k] == pytest.approx(fd, rel=2e-4, abs=1e-9 * max(1.0, np.abs(g).max()))


def test_loss_vanishes_at_target(oracle, pot):
    n = 5
    x = synth.thermal_snapshot(n, n, n, 0.1, 2)
    L = synth.box(n, n, n)
    _, _, e, f = oracle.eam(oracle.Pot(pot), x, L, mode=0)
    loss, g, _, _ = oracle.loss_grad(oracle.Pot(pot), x, L, f, e.sum())
    assert loss < 1e-28
    assert np.abs(g).max() < 1e-12
