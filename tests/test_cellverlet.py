"""The CPU Verlet-list baseline (oracle/cellverlet.c: cell grid, sort, half list, Alg. 4-6) against
the all-pairs FP64 oracle on the small FP64 configuration (FCC 10^3 x 4, rho 0.5, L = 20), before it
is timed as a CPU baseline."""
import numpy as np
import pytest

import oracle as O
from oracle import cellverlet as CV
from paper_1012_2677_gb300 import synth


def _state(steps=40):
    x, L = O.fcc_lattice(10, 0.5)
    v = O.init_velocities(len(x), 1.0, 1)
    x, v, *_ = O.vv_run(x, v, L, 0.005, steps)
    return O.wrap(x, L), v, L


def test_forces_energies_and_pair_count_match_the_oracle():
    x, v, L = _state()
    r = CV.run(x, v, L, 0.005, 0, 0.5)
    F, pe, vir = O.forces(x, L)
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((r["f"] - F) ** 2).sum(1)).max() <= 1e-12 * rms
    assert r["pe"] == pytest.approx(pe, rel=1e-12) and r["vir"] == pytest.approx(vir, rel=1e-12)
    assert r["pairs"] == len(O.pairs_within(x, L, 3.0))
    assert np.array_equal(r["x"], x)


def test_two_cells_per_side_falls_back_to_all_pairs():
    L = 7.2
    x = synth.uniform_positions(300, L, 3)
    r = CV.run(x, None, L, 0.005, 0, 0.3)
    assert r["pairs"] == len(O.pairs_within(x, L, 2.8))


def test_trajectory_with_rebuilds_matches_the_oracle():
    x, v, L = _state()
    xo, vo, Fo, pe, ke, _ = O.vv_run(x, v, L, 0.005, 60)
    r = CV.run(x, v, L, 0.005, 60, 0.5)
    assert r["rebuilds"] >= 3
    assert np.abs(r["x"] - xo).max() < 1e-9
    assert np.abs(r["v"] - vo).max() < 1e-8
    assert r["pe"] == pytest.approx(pe[-1], rel=1e-10) and r["ke"] == pytest.approx(ke[-1], rel=1e-10)
