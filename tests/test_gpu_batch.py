"""Batched replicas: forces, energies and pair lists of every replica against the FP64 oracle,
trajectories against single-system runs and the oracle, graph replay against plain launches,
device-decided rebuilds, and the autotuner."""
import numpy as np
import pytest

import oracle as O
from paper_1012_2677_gb300 import ljmd, synth

pytestmark = pytest.mark.gpu

RC, MARGIN = 2.5, 0.3


def _workload(R=6, seed=77, n_range=(700, 3000)):
    n, box, x, v, T = synth.batch_workload(R, seed, n_range=n_range)
    return n, box, synth.dyadic(x), v


def _split(a, n):
    return np.split(a, np.cumsum(n)[:-1])


def _min_image(d, L):
    return d - L * np.round(d / L)


def test_batch_forces_energies_and_pairs_match_oracle():
    n, box, x, v = _workload()
    with ljmd.Batch(n, box, cutoff=RC, margin=MARGIN) as b:
        b.set_state(x, v)
        pe, ke, vir = b.energies()
        gx, gv, gf = b.get_state()
        pairs = [b.pairs(r) for r in range(len(n))]
    for r, (xr, vr, fr, Lr) in enumerate(zip(_split(x, n), _split(v, n), _split(gf, n), box)):
        F, pe_o, vir_o = O.forces(xr, Lr)
        rms = np.sqrt((F ** 2).sum(1).mean())
        assert np.sqrt(((fr - F) ** 2).sum(1)).max() / rms <= 1e-5
        assert pe[r] == pytest.approx(pe_o, rel=1e-6)
        assert vir[r] == pytest.approx(vir_o, rel=1e-6)
        assert ke[r] == pytest.approx(O.kinetic(vr), rel=1e-12)
        assert np.array_equal(pairs[r], O.pairs_within(xr, Lr, RC + MARGIN))
    assert np.array_equal(gv, v)


def test_batch_trajectory_matches_single_systems_and_oracle():
    n, box, x, v = _workload(R=5, seed=78)
    dt, steps = 0.004, 20
    with ljmd.Batch(n, box, cutoff=RC, margin=MARGIN) as b:
        b.set_state(x, v)
        b.step(dt, steps, graph_steps=5)
        bx, bv, _ = b.get_state()
    for r, (xr, vr, Lr) in enumerate(zip(_split(x, n), _split(v, n), box)):
        with ljmd.System(cutoff=RC, margin=MARGIN, precision=ljmd.LJ_MIXED) as s:
            s.set_state(xr, vr, Lr)
            s.step(dt, steps)
            sx, sv, _, _ = s.get_state()
        bxr = _split(bx, n)[r]
        assert np.abs(_min_image(bxr - sx, Lr)).max() < 1e-5
        if r < 2:
            xo, vo, *_ = O.vv_run(xr, vr, Lr, dt, steps)
            assert np.abs(_min_image(bxr - xo, Lr)).max() < 1e-4


def test_batch_graph_replay_equals_plain_launches():
    """A graph replay runs the same kernels in the same order as plain launches: bit-identical
    states.  ljmd_batch_step(24, K = 8) runs 1 plain step, two 8-step replays and 7 plain steps,
    each call ending on the full-step velocity, so the plain reference uses the same chunks."""
    n, box, x, v = _workload(R=4, seed=79)
    out = []
    for chunks, K in (((1, 8, 8, 7), 0), ((24,), 8)):
        with ljmd.Batch(n, box, cutoff=RC, margin=MARGIN) as b:
            b.set_state(x, v)
            for c in chunks:
                b.step(0.004, c, graph_steps=K)
            out.append(b.get_state())
            st = b.stats()
        assert st["steps"] == 24 and st["status_word"] == 0
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_batch_device_rebuilds_keep_lists_valid():
    """Over a run long enough for many device-decided rebuilds, every pair within r_c is listed."""
    n, box, x, v = _workload(R=4, seed=80)
    with ljmd.Batch(n, box, cutoff=RC, margin=MARGIN) as b:
        b.set_state(x, v)
        b.step(0.004, 150, graph_steps=10)
        st = b.stats()
        gx, _, _ = b.get_state()
        for r, (xr, Lr) in enumerate(zip(_split(gx, n), box)):
            listed = set(map(tuple, b.pairs(r).tolist()))
            d = _min_image(xr[None, :, :] - xr[:, None, :], Lr)
            i, j = np.nonzero(np.triu((d ** 2).sum(-1) < RC * RC, k=1))
            assert set(zip(i.tolist(), j.tolist())) <= listed
    assert st["rebuilds"] >= 3 and st["status_word"] == 0


def test_batch_autotune_keeps_results():
    n, box, x, v = _workload(R=4, seed=81)
    with ljmd.Batch(n, box, cutoff=RC, margin=MARGIN) as b:
        b.set_state(x, v)
        tile, lanes, ms = b.autotune(trials=2)
        _, _, gf = b.get_state()
    assert tile in (2, 3, 4, 6) and lanes in (2, 4, 8) and ms > 0
    for fr, xr, Lr in zip(_split(gf, n), _split(x, n), box):
        F, _, _ = O.forces(xr, Lr)
        rms = np.sqrt((F ** 2).sum(1).mean())
        assert np.sqrt(((fr - F) ** 2).sum(1)).max() / rms <= 1e-5


def test_batch_rejects_boxes_under_two_search_lengths():
    """A box under 2 (r_s + margin) could hold two images of one partner within reach of a key."""
    with pytest.raises(ljmd.LjmdError) as e:
        ljmd.Batch([300, 800], [6.1, 9.5], cutoff=RC, margin=MARGIN)
    assert e.value.code == ljmd.LJ_EINVAL


def test_batch_with_two_cell_replicas():
    """Replicas under 3 r_s (N = 500 at rho 0.9 is L = 8.22 < 3 x 2.8: 2 cells per side) beside
    ordinary ones: pairs bit-exact and forces against the oracle, and a 20-step run against single
    systems (whose two-cell boxes take the whole-box path)."""
    spec = [(500, 0.9), (480, 0.85), (600, 0.9), (2000, 0.5)]
    xs, vs, box = [], [], []
    for r, (N, rho) in enumerate(spec):
        x, L = synth.fcc_thinned(N, rho, 300 + r)
        x = np.mod(x + synth.displacements(N, 0.1, 500 + r), L)  # off the lattice: forces well away from zero
        xs.append(synth.dyadic(x))
        vs.append(synth.thermal_velocities(N, 1.0, 400 + r))
        box.append(L)
    n = np.array([N for N, _ in spec])
    box = np.array(box)
    assert box[0] < 3 * (RC + MARGIN) and box[1] < 3 * (RC + MARGIN)
    x, v = np.concatenate(xs), np.concatenate(vs)
    with ljmd.Batch(n, box, cutoff=RC, margin=MARGIN) as b:
        b.set_state(x, v)
        _, _, gf = b.get_state()
        pairs = [b.pairs(r) for r in range(len(n))]
        b.step(0.004, 20, graph_steps=5)
        bx, _, _ = b.get_state()
        st = b.stats()
    assert st["status_word"] == 0
    for r, (xr, fr, Lr) in enumerate(zip(xs, _split(gf, n), box)):
        F, _, _ = O.forces(xr, Lr)
        rms = np.sqrt((F ** 2).sum(1).mean())
        assert np.sqrt(((fr - F) ** 2).sum(1)).max() / rms <= 1e-5, r
        assert np.array_equal(pairs[r], O.pairs_within(xr, Lr, RC + MARGIN)), r
    for r, (xr, vr, Lr) in enumerate(zip(xs, vs, box)):
        with ljmd.System(cutoff=RC, margin=MARGIN, precision=ljmd.LJ_MIXED) as s:
            s.set_state(xr, vr, Lr)
            s.step(0.004, 20)
            sx, _, _, _ = s.get_state()
        assert np.abs(_min_image(_split(bx, n)[r] - sx, Lr)).max() < 1e-5, r
