"""Pins of the oracle's alloy evaluation (Sec. 2.2, Eq. eam_base and
Eq. eam_force_ij with atom types): identical species reduce to the
single-species oracle; a two-species dimer against the analytic closed
form; forces against central differences of the energy; momentum; and
invariance under relabelling the species."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth


@pytest.fixture(scope="module")
def alloy3():
    return synth.alloy_potential(3)


def test_identical_species_reduce_to_single_species(oracle):
    pot = synth.potential()
    nsp = 3
    al = synth.AlloyPotential(nsp, pot.n, pot.rc, pot.rho_max, np.stack([pot.f] * nsp), np.stack([pot.F] * nsp),
                              np.stack([pot.phi] * (nsp * (nsp + 1) // 2)))
    x = synth.cascade_snapshot(5, 5, 5, 0.15, 4, 2, 3)
    t = synth.random_types(len(x), (0.5, 0.3, 0.2), 4)
    L = synth.box(5, 5, 5)
    ra, fa, ea, Fa = oracle.eam_alloy(oracle.Alloy(al), x, t, L, mode=0)
    rs, fs, es, Fs = oracle.eam(oracle.Pot(pot), x, L, mode=0)
    np.testing.assert_allclose(ra, rs, rtol=1e-14, atol=0)
    np.testing.assert_allclose(ea, es, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(Fa, Fs, rtol=0, atol=1e-12 * np.abs(Fs).max())


@pytest.mark.parametrize("a,b", [(0, 1), (1, 2), (2, 0)])
def test_dimer_closed_form(oracle, alloy3, a, b):
    dens, emb, pair = synth.alloy_functions(3)
    rc = synth.RC

    def trunc(g, dg, r):
        return g(r) - g(rc) - (r - rc) * dg(rc), dg(r) - dg(rc)

    n = 12
    L = synth.box(n, n, n)
    for r in (2.4, 2.9, 3.5):
        x = np.array([[10.0, 10.0, 10.0], [10.0 + r, 10.0, 10.0]])
        _, _, e, f = oracle.eam_alloy(oracle.Alloy(alloy3), x, np.array([a, b], np.int8), L, mode=0)
        ra, dra = trunc(*dens(a), r)
        rb, drb = trunc(*dens(b), r)
        p, dp = trunc(*pair(a, b), r)
        Fa, dFa = emb(a)[0](rb), emb(a)[1](rb)
        Fb, dFb = emb(b)[0](ra), emb(b)[1](ra)
        assert e[0] == pytest.approx(Fa + 0.5 * p, rel=1e-6)
        assert e[1] == pytest.approx(Fb + 0.5 * p, rel=1e-6)
        dE = dFa * drb + dFb * dra + dp  # d(E_0 + E_1)/dr
        # a dimer's densities are ~1, where -c sqrt(rho) bends sharply: the
        # derivative of the cubic Hermite interpolant is accurate to
        # O(h_rho^3 d4F/drho4) ~ 1e-5 there (h_rho = rho_max / 4999)
        assert f[0, 0] == pytest.approx(dE, rel=5e-5)   # atom 0 is pulled along +x when dE/dr > 0
        assert f[1, 0] == pytest.approx(-dE, rel=5e-5)
        assert np.abs(f[:, 1:]).max() < 1e-12


def test_forces_are_minus_energy_gradient(oracle, alloy3):
    n = 4
    x = synth.thermal_snapshot(n, n, n, 0.12, 8)
    t = synth.random_types(len(x), (0.6, 0.25, 0.15), 9)
    L = synth.box(n, n, n)
    al = oracle.Alloy(alloy3)
    _, _, _, f = oracle.eam_alloy(al, x, t, L, mode=0)
    rng = np.random.default_rng(10)
    h = 1e-5
    for i in rng.choice(len(x), 6, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            ep = oracle.eam_alloy(al, xp, t, L, mode=0)[2].sum()
            em = oracle.eam_alloy(al, xm, t, L, mode=0)[2].sum()
            assert f[i, d] == pytest.approx(-(ep - em) / (2 * h), rel=1e-6, abs=1e-8)
    assert np.abs(f.sum(axis=0)).max() < 1e-11 * np.abs(f).max() * len(x)


def test_relabelling_species_changes_nothing(oracle, alloy3):
    perm = np.array([2, 0, 1])  # new label of old species s
    inv = np.argsort(perm)
    nsp = 3
    phi = np.empty_like(alloy3.phi)
    for a in range(nsp):
        for b in range(a, nsp):
            phi[synth.pair_index(perm[a], perm[b], nsp)] = alloy3.phi[synth.pair_index(a, b, nsp)]
    swapped = synth.AlloyPotential(nsp, alloy3.n, alloy3.rc, alloy3.rho_max, alloy3.f[inv], alloy3.F[inv], phi)
    x = synth.cascade_snapshot(5, 5, 5, 0.12, 4, 2, 11)
    t = synth.random_types(len(x), (0.4, 0.4, 0.2), 12)
    L = synth.box(5, 5, 5)
    r1 = oracle.eam_alloy(oracle.Alloy(alloy3), x, t, L, mode=1)
    r2 = oracle.eam_alloy(oracle.Alloy(swapped), x, perm[t].astype(np.int8), L, mode=1)
    for u, v in zip(r1, r2):
        np.testing.assert_array_equal(u, v)
