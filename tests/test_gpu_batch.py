"""Batched replicas (Sec. 1 feature list: batch execution of simulations):
several uneven boxes in one handle, every step kernel launched once for all
of them.  A replica of a batch must evolve exactly as the same box alone
(same kernels, same per-site sum order), the captured step graph must
reproduce the directly launched step, and every replica of an uneven batch
must follow the FP64 oracle's run of that box alone."""
import numpy as np
import pytest

from paper_2107_07866_gb300 import synth

pytestmark = pytest.mark.gpu

M = synth.MASS_FE


@pytest.fixture(scope="module")
def misa():
    import torch
    assert torch.cuda.is_available()
    from paper_2107_07866_gb300 import build
    build.build()
    from paper_2107_07866_gb300 import misa as M_
    return M_


def _inputs(dims, seed, pka_eV):
    x = synth.cascade_snapshot(*dims, 0.1, 3, 1, seed)
    v = synth.maxwell_velocities(len(x), 300.0 + 100 * seed, M, seed)
    if pka_eV:
        a = synth.pka_atom(*dims)
        d = synth.random_direction(seed + 5)
        v[a] = np.sqrt(2 * pka_eV / M / synth.EV_PER_AMU_A2_FS2) * d
    return x, v


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_replicas_evolve_as_single_boxes(misa, pot, prec):
    reps = [(6, 7, 8), (9, 6, 6), (8, 8, 7)]
    ins = [_inputs(d, k, 200.0 * (k + 1)) for k, d in enumerate(reps)]
    kw = dict(precision=prec, dx_max=0.02, reassign_period=2, tile=2)
    with misa.Sim(pot, replicas=reps, **kw) as b:
        assert b.natoms == sum(2 * a * c * e for a, c, e in reps)
        b.set_state(np.concatenate([x for x, _ in ins]), np.concatenate([v for _, v in ins]))
        b.step(25)
        xb, fb = b.positions(), b.forces()
        stb = [b.replica_stats(r) for r in range(len(reps))]
        peb, keb = b.replica_energies()
    off = 0
    for r, (d, (x, v)) in enumerate(zip(reps, ins)):
        n = 2 * d[0] * d[1] * d[2]
        with misa.Sim(pot, *d, **kw) as s:
            s.set_state(x, v)
            s.step(25)
            np.testing.assert_array_equal(xb[off:off + n], s.positions())
            np.testing.assert_array_equal(fb[off:off + n], s.forces())
            st = s.stats()
            pe, ke = s.energies()
        # each replica has its own adaptive timestep and run-away list
        assert stb[r]["time"] == st["time"] and stb[r]["n_runaway"] == st["n_runaway"]
        assert peb[r] == pytest.approx(pe, rel=1e-12) and keb[r] == pytest.approx(ke, rel=1e-12)
        off += n
    assert len({s_["time"] for s_ in stb}) == len(reps)


def test_graph_replay_equals_direct_launches(misa, pot):
    x, v = _inputs((8, 8, 8), 3, 400.0)
    out = []
    for graphs in (True, False):
        with misa.Sim(pot, 8, precision="fp32", dx_max=0.02, reassign_period=3) as s:
            s.set_graphs(graphs)
            s.set_state(x, v)
            s.step(15)
            s.step(15)
            out.append((s.positions(), s.velocities(), s.stats()["step"]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert out[0][2] == out[1][2] == 30


def test_autotuner_picks_a_built_tile(misa, pot):
    with misa.Sim(pot, 12, precision="fp32", tile=0) as s:
        assert s.tile() in misa.tile_shapes() and s.tile_force() in misa.tile_shapes()


def test_batch_pka_per_replica(misa, pot):
    reps = [(6, 6, 6), (7, 6, 8)]
    with misa.Sim(pot, replicas=reps, precision="fp64", dx_max=0.02) as b:
        d = np.array([0.0, 0.6, 0.8])
        b.insert_pka_replica(1, 1000.0, d)
        v = b.velocities()
        _, base, n = b.replica_info(1)
        a = base + synth.pka_atom(*reps[1])
        assert 0.5 * M * np.dot(v[a], v[a]) * synth.EV_PER_AMU_A2_FS2 == pytest.approx(1000.0, rel=1e-12)
        assert np.count_nonzero(np.linalg.norm(v, axis=1)) == 1
        b.step(4)
        t0, t1 = b.replica_stats(0)["time"], b.replica_stats(1)["time"]
        assert t0 == pytest.approx(4.0) and t1 < 0.5


def test_retune_changes_speed_not_results(misa, pot):
    # the autotuner re-run on a thermal state may pick other tile shapes for
    # the two passes; per-site sums do not depend on the shapes
    x = synth.thermal_snapshot(16, 12, 14, 0.12, 3)
    v = synth.maxwell_velocities(len(x), 600.0, synth.MASS_FE, 4)
    out = []
    for tile in (0, 1):
        with misa.Sim(pot, 16, 12, 14, precision="fp32", tile=tile) as s:
            s.set_state(x, v)
            f0 = s.forces()
            s.retune()
            assert s.tile() in misa.tile_shapes() and s.tile_force() in misa.tile_shapes()
            np.testing.assert_array_equal(s.forces(), f0)
            s.step(5)
            out.append((s.positions(), s.forces()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _nerr(x, xo):
    x, xo = np.asarray(x).reshape(len(x), -1), np.asarray(xo).reshape(len(xo), -1)
    mag = np.linalg.norm(xo, axis=1)
    rms = np.sqrt(np.mean(mag ** 2))
    return float(np.max(np.linalg.norm(x - xo, axis=1) / np.maximum(mag, rms)))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_uneven_batch_matches_oracle_per_replica(misa, pot, oracle, opot, prec):
    # four boxes of different dims in one handle, each with its own knock-on
    # atom, run-aways (cascade snapshots) and adaptive timestep: every
    # replica's trajectory is the oracle's MD run of that box alone, and the
    # densities, energies and forces of its final state are the oracle's
    reps = [(6, 7, 8), (9, 6, 6), (8, 8, 7), (7, 9, 6)]
    ins = []
    for k, d in enumerate(reps):
        x = synth.cascade_snapshot(*d, 0.1, 4 + k, 1, 40 + k)
        v = synth.maxwell_velocities(len(x), 300.0 + 150 * k, M, 40 + k)
        oracle.insert_pka(v, synth.pka_atom(*d), M, 120.0 + 90.0 * k, synth.random_direction(50 + k))
        ins.append((x, v))
    steps = 40
    with misa.Sim(pot, replicas=reps, precision=prec, dt_max=1.0, dx_max=0.02, reassign_period=3) as b:
        b.set_state(np.concatenate([x for x, _ in ins]), np.concatenate([v for _, v in ins]))
        ra0 = [b.replica_stats(r)["n_runaway"] for r in range(len(reps))]
        b.step(steps)
        xb, fb, rhob = b.positions(), b.forces(), b.density()
        _, _, eb = b.energies(per_atom=True)
        stb = [b.replica_stats(r) for r in range(len(reps))]
        info = [b.replica_info(r) for r in range(len(reps))]
    assert min(ra0) > 0
    tol_x = 1e-8 if prec == "fp64" else 2e-5
    for r, (d, (x0, v0)) in enumerate(zip(reps, ins)):
        _, base, n = info[r]
        L = synth.box(*d)
        sl = slice(base, base + n)
        xo, _, _, t, _ = oracle.md_run(opot, x0, v0, L, M, 1.0, 0.02, steps, mode=1)
        dd = xb[sl] - xo
        dd -= L * np.round(dd / L)
        assert np.abs(dd).max() < tol_x, (r, np.abs(dd).max())
        assert stb[r]["step"] == steps and stb[r]["status"] & 0x3 == 0
        assert abs(stb[r]["time"] - t) < (1e-10 if prec == "fp64" else 1e-6), (r, stb[r]["time"], t)
        rho_o, _, e_o, f_o = oracle.eam(opot, xb[sl], L, mode=1)
        assert _nerr(fb[sl], f_o) < TOL[prec], (r, _nerr(fb[sl], f_o))
        assert _nerr(rhob[sl], rho_o) < TOL[prec]
        assert _nerr(eb[sl], e_o) < TOL[prec]
    # the replicas took different timesteps
    assert len({s_["time"] for s_ in stb}) == len(reps)
