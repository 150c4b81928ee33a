"""Pins of the oracle's lattice list (Sec. 3, Alg. 1, Alg. 2): the paper's
worked index example, the bcc neighbour shells, the nearest-site hash against
brute force, the Alg. 2 post-conditions, and the lattice-list pair set
against the brute-force pair set."""
import json
import os

import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
A0 = synth.A0_FE


def test_worked_index_example(oracle):
    g = json.load(open(os.path.join(GOLDEN, "lattice_index_example.json")))
    assert oracle.site_index(g["box_x"], g["box_y"], g["x"], g["y"], g["z"]) == g["index"]


def test_index_matches_generator_order_and_positions(oracle):
    nx, ny, nz = 5, 6, 7
    x = synth.bcc_positions(nx, ny, nz)
    rng = np.random.default_rng(0)
    for sid in rng.integers(0, len(x), 50):
        np.testing.assert_allclose(oracle.site_position(nx, ny, A0, int(sid)), x[sid], atol=1e-12)
    # the id is a bijection onto [0, 2 nx ny nz)
    ids = {oracle.site_index(nx, ny, xx, yy, zz) for zz in range(nz) for yy in range(ny) for xx in range(2 * nx)}
    assert ids == set(range(2 * nx * ny * nz))


def test_nearest_site_is_brute_force_nearest(oracle):
    nx = ny = nz = 5
    sites = synth.bcc_positions(nx, ny, nz)
    L = synth.box(nx, ny, nz)
    rng = np.random.default_rng(1)
    for p in rng.uniform(0, 1, (300, 3)) * L:
        d = sites - p
        d -= L * np.round(d / L)
        r = np.sqrt((d * d).sum(1))
        best = np.flatnonzero(r <= r.min() + 1e-12)
        assert oracle.nearest_site(nx, ny, nz, A0, p) == best.min()


def _bcc_shells(R):
    """Cartesian bcc lattice vectors within R, counted directly."""
    m = int(np.ceil(2 * R / A0)) + 1
    out = []
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            for k in range(-m, m + 1):
                if (i % 2 == j % 2 == k % 2) and (i or j or k):
                    v = 0.5 * A0 * np.array([i, j, k])
                    if np.linalg.norm(v) <= R:
                        out.append(v)
    return np.array(out)


@pytest.mark.parametrize("R,count", [(5.6, 58), (6.8, 112)])
def test_offset_index_is_parity_dependent_bcc_shell_set(oracle, R, count):
    ref = _bcc_shells(R)
    assert len(ref) == count
    for par in (0, 1):
        off = oracle.offsets(A0, R, par)
        assert len(off) == count
        # turn (dx2, dy, dz) lattice-id offsets back into Cartesian vectors
        tp = (par + off[:, 0]) & 1
        cx = (par + off[:, 0] - tp) // 2
        vec = A0 * np.stack([cx + 0.5 * tp - 0.5 * par, off[:, 1] + 0.5 * tp - 0.5 * par,
                             off[:, 2] + 0.5 * tp - 0.5 * par], 1)
        a = np.array(sorted(map(tuple, np.round(vec, 9))))
        b = np.array(sorted(map(tuple, np.round(ref, 9))))
        np.testing.assert_array_equal(a, b)
    # same Cartesian set, different id offsets for corner and centre sites
    assert set(map(tuple, oracle.offsets(A0, R, 0))) != set(map(tuple, oracle.offsets(A0, R, 1)))


def test_initial_crystal_has_no_clash(oracle):
    lt = oracle.Lattice(5, 5, 6, A0, 0.6)
    lt.assign(synth.bcc_positions(5, 5, 6))
    assert len(lt.runaways()) == 0
    np.testing.assert_array_equal(lt.site_atom(), np.arange(2 * 5 * 5 * 6))


def _check_invariants(oracle, lt, x, nx, ny, nz, skin):
    sa = lt.site_atom()
    ra = lt.runaways()
    n = len(x)
    placed = sa[sa >= 0]
    # (1) every atom stored exactly once: one slot or the run-away list
    allid = np.concatenate([placed, ra])
    assert len(allid) == n and len(np.unique(allid)) == n
    L = synth.box(nx, ny, nz)
    sites = synth.bcc_positions(nx, ny, nz)
    for s in np.flatnonzero(sa >= 0):
        d = x[sa[s]] - sites[s]
        d -= L * np.round(d / L)
        assert np.linalg.norm(d) <= skin + 1e-12
    # (2) a site nobody is nearest to holds no atom: the atom a site holds
    # has that site as its nearest one
    near = np.array([oracle.nearest_site(nx, ny, nz, A0, np.mod(p, L)) for p in x])
    for s in np.flatnonzero(sa >= 0):
        assert near[sa[s]] == s
    # (3) no run-away whose nearest site is empty and within the skin
    for i in ra:
        s = near[i]
        d = np.mod(x[i], L) - sites[s]
        d -= L * np.round(d / L)
        assert not (sa[s] < 0 and np.linalg.norm(d) <= skin)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_alg2_invariants(oracle, seed):
    nx, ny, nz, skin = 5, 6, 5, 0.6
    x0 = synth.cascade_snapshot(nx, ny, nz, 0.15, 6, 3, seed)
    lt = oracle.Lattice(nx, ny, nz, A0, skin)
    lt.assign(x0)
    _check_invariants(oracle, lt, x0, nx, ny, nz, skin)
    rng = np.random.default_rng(seed)
    x1 = x0 + rng.normal(0, 0.2, x0.shape)
    lt.update(x1)
    _check_invariants(oracle, lt, x1, nx, ny, nz, skin)


@pytest.mark.parametrize("dims,seed", [((5, 5, 5), 0), ((6, 5, 7), 1), ((7, 7, 7), 2)])
def test_lattice_list_pair_set_equals_brute_force(oracle, dims, seed):
    nx, ny, nz = dims
    skin, rc = 0.6, synth.RC
    x = synth.cascade_snapshot(nx, ny, nz, 0.15, 8, 4, seed)
    L = synth.box(nx, ny, nz)
    lt = oracle.Lattice(nx, ny, nz, A0, skin)
    lt.assign(x)
    assert len(lt.runaways()) >= 8
    bi, bj, br = oracle.pair_list(x, L, rc, mode=0)
    li, lj, lr = lt.pairs(x, rc)
    a = sorted(zip(bi.tolist(), bj.tolist()))
    b = sorted(zip(li.tolist(), lj.tolist()))
    assert a == b
    np.testing.assert_allclose(np.sort(br), np.sort(lr), atol=1e-12)
    # the cell list enumerates the same set where it applies
    ci, cj, _ = oracle.pair_list(x, L, rc, mode=1)
    assert sorted(zip(ci.tolist(), cj.tolist())) == a


def test_offset_memory_independent_of_system_size(oracle):
    # O(M) offsets vs O(MN) neighbour lists (Sec. 3): the offset index depends
    # on a0 and the radius only
    assert len(oracle.offsets(A0, 6.8, 0)) == len(oracle.offsets(A0, 6.8, 1)) == 112


# --- Wigner-Seitz defect count (Frenkel pairs, Sec. 5.1) --------------------

def _ws_brute(nx, ny, nz, a0, x):
    """Occupancy by brute force: each atom to the closest site over all sites
    and periodic images (ties to the lower site index)."""
    sites = synth.bcc_positions(nx, ny, nz, a0)
    L = synth.box(nx, ny, nz, a0)
    occ = np.zeros(len(sites), int)
    for p in x:
        d = sites - p
        d -= L * np.round(d / L)
        r2 = np.einsum("ij,ij->i", d, d)
        occ[int(np.flatnonzero(r2 <= r2.min() + 1e-12)[0])] += 1
    return int((occ == 0).sum()), int(np.maximum(occ - 1, 0).sum())


def test_ws_defects_perfect_crystal(oracle):
    x = synth.bcc_positions(6, 5, 7)
    assert oracle.ws_defects(6, 5, 7, synth.A0_FE, x) == (0, 0)


def test_ws_defects_single_frenkel_pair(oracle):
    a0 = synth.A0_FE
    x = synth.bcc_positions(6, 6, 6, a0)
    # an octahedral interstitial position (face centre of a cube): nearest
    # sites are occupied corners, so one vacancy and one interstitial
    x[17] = np.array([2.5, 2.5, 2.0]) * a0 + 0.01
    assert oracle.ws_defects(6, 6, 6, a0, x) == (1, 1)
    # a second atom into the first one's empty cell: still one pair
    x[40] = synth.bcc_positions(6, 6, 6, a0)[17] + 0.3
    assert oracle.ws_defects(6, 6, 6, a0, x) == (1, 1)


def test_ws_defects_match_brute_force(oracle):
    a0 = synth.A0_FE
    for seed in range(3):
        x = synth.cascade_snapshot(5, 5, 5, 0.25, 6, 2, seed)
        got = oracle.ws_defects(5, 5, 5, a0, x)
        assert got == _ws_brute(5, 5, 5, a0, x)
        assert got[0] == got[1] > 0  # atoms = sites: vacancies = interstitials
