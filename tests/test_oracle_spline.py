"""Pins of the oracle's spline tables (Sec. 4.1 reading: local cubic Hermite,
slopes from central differences).  Each check is fixed by mathematics, not by
retyping the oracle: polynomial reproduction, interpolation, C1 continuity,
the interpolation error bound, and the linear dependence on the knots."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth


def test_reproduces_quadratics_everywhere(oracle):
    n, h = 40, 0.25
    xk = np.arange(n) * h
    y = 1.5 - 2.0 * xk + 0.75 * xk ** 2
    xs = np.linspace(0.0, xk[-1], 777)
    v, dv = oracle.spline_eval(y, h, xs)
    np.testing.assert_allclose(v, 1.5 - 2.0 * xs + 0.75 * xs ** 2, rtol=0, atol=1e-12)
    np.testing.assert_allclose(dv, -2.0 + 1.5 * xs, rtol=0, atol=1e-11)


def test_reproduces_cubics_on_interior_segments(oracle):
    # 4th-order central slopes are exact on cubics (and quartics); segments
    # whose two end knots both use them reproduce a cubic exactly.
    n, h = 50, 0.1
    xk = np.arange(n) * h
    p = lambda x: 0.3 - x + 0.5 * x ** 2 - 0.2 * x ** 3
    dp = lambda x: -1.0 + x - 0.6 * x ** 2
    xs = np.linspace(xk[2], xk[n - 3], 501)
    v, dv = oracle.spline_eval(p(xk), h, xs)
    np.testing.assert_allclose(v, p(xs), rtol=0, atol=1e-11)
    np.testing.assert_allclose(dv, dp(xs), rtol=0, atol=1e-10)


def test_knot_slopes_exact_on_quartic(oracle):
    n, h = 30, 0.2
    xk = np.arange(n) * h
    y = xk ** 4 - 3 * xk ** 3
    m = oracle.spline_slopes(y, h)
    np.testing.assert_allclose(m[2:-2], 4 * xk[2:-2] ** 3 - 9 * xk[2:-2] ** 2, rtol=1e-12, atol=1e-9)


def test_interpolates_and_is_c1(oracle):
    rng = np.random.default_rng(3)
    n, h = 64, 0.05
    y = rng.normal(size=n)
    xk = np.arange(n) * h
    v, _ = oracle.spline_eval(y, h, xk)
    np.testing.assert_allclose(v, y, rtol=0, atol=1e-13)
    eps = 1e-11
    lo, dlo = oracle.spline_eval(y, h, xk[1:-1] - eps)
    hi, dhi = oracle.spline_eval(y, h, xk[1:-1] + eps)
    np.testing.assert_allclose(lo, hi, atol=1e-7)
    np.testing.assert_allclose(dlo, dhi, atol=1e-6)
    # the derivative at a knot is that knot's slope
    m = oracle.spline_slopes(y, h)
    _, dk = oracle.spline_eval(y, h, xk[1:-1] + 1e-13)
    np.testing.assert_allclose(dk, m[1:-1], atol=1e-9)


def test_error_bound_on_analytic_tables(oracle, pot):
    # Hermite interpolation with O(h^4) slopes: error ~ h^4 max|g''''|; at
    # h = rc/4999 that is far below 1e-9 for the smooth f and phi.
    h = pot.rc / (pot.n - 1)
    fs, dfs = synth.truncated(synth.f_analytic, synth.df_analytic)
    ps, dps = synth.truncated(synth.phi_analytic, synth.dphi_analytic)
    r = np.linspace(0.5, pot.rc - 1e-6, 2001)
    v, dv = oracle.spline_eval(pot.f, h, r)
    np.testing.assert_allclose(v, fs(r), rtol=0, atol=1e-10)
    np.testing.assert_allclose(dv, dfs(r), rtol=0, atol=1e-7)
    v, dv = oracle.spline_eval(pot.phi, h, r)
    np.testing.assert_allclose(v, ps(r), rtol=0, atol=1e-9 * max(1.0, np.abs(ps(r)).max()))
    np.testing.assert_allclose(dv, dps(r), rtol=1e-6, atol=1e-6)
    hr = pot.rho_max / (pot.n - 1)
    rho = np.linspace(5.0, pot.rho_max, 1001)
    v, dv = oracle.spline_eval(pot.F, hr, rho)
    np.testing.assert_allclose(v, -1.8 * np.sqrt(rho), rtol=0, atol=1e-11)
    # interior slopes are 4th order; the end knot's one-sided slope is 2nd
    # order: h^2/3 |F'''(rho_max)| ~ 1.3e-9
    np.testing.assert_allclose(dv[:-20], -0.9 / np.sqrt(rho[:-20]), rtol=0, atol=1e-10)
    np.testing.assert_allclose(dv, -0.9 / np.sqrt(rho), rtol=0, atol=5e-9)


def test_weights_give_the_same_spline(oracle):
    rng = np.random.default_rng(11)
    n, h = 20, 0.3
    y = rng.normal(size=n)
    for x in [0.0, 0.01, 0.29, 0.3, 1.7, 2.55, 5.1, 5.4, (n - 1) * h]:
        idx, w, dw = oracle.spline_weights(n, h, x)
        v, dv = oracle.spline_eval(y, h, x)
        assert abs(np.dot(w, y[idx]) - v[0]) < 1e-12
        assert abs(np.dot(dw, y[idx]) - dv[0]) < 1e-11


def test_potential_zero_beyond_cutoff_and_linear_embedding_tail(oracle, pot, opot):
    v, dv = opot.eval(0, [pot.rc, pot.rc + 0.3])
    assert np.all(v == 0.0) and np.all(dv == 0.0)
    v, dv = opot.eval(1, [pot.rc, 7.0])
    assert np.all(v == 0.0) and np.all(dv == 0.0)
    # above rho_max the embedding continues along its end tangent
    e0, d0 = opot.eval(2, [pot.rho_max])
    e1, d1 = opot.eval(2, [pot.rho_max + 2.0])
    assert d1[0] == pytest.approx(d0[0], abs=1e-12)
    assert e1[0] == pytest.approx(e0[0] + 2.0 * d0[0], abs=1e-12)
