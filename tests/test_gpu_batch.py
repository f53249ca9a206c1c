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


def test_batch_rejects_boxes_under_three_cells():
    with pytest.raises(ljmd.LjmdError) as e:
        ljmd.Batch([500, 800], [7.0, 9.5], cutoff=RC, margin=MARGIN)
    assert e.value.code == ljmd.LJ_ERANGE
