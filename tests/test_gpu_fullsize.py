"""Parity at the benchmark's sizes, in the launch configuration the benchmark times: forces on a
seeded sample of particles against the oracle's all-pairs sum for those particles (16.4M at rho
0.5 and 0.8, the 256-replica batch), total force (Newton's third law) against zero, the pipelined
force kernel against the single-buffer one (bit-identical: same per-key arithmetic and summation
order), and the 32,000-particle differentiable trajectory in the mixed form against the FP64 form."""
import numpy as np
import pytest

import oracle as O
from paper_1012_2677_gb300 import ljmd, synth

pytestmark = pytest.mark.gpu

RC, MARGIN, DT = 2.5, 0.5, 0.005


def _run(M, steps, tile=0, lanes=0, nbuf=0, seed=3):
    with ljmd.System(cutoff=RC, margin=MARGIN, precision=ljmd.LJ_MIXED) as s:
        s.set_tuning(tile, lanes, 0, nbuf)
        s.init_lattice(M, 0.5, 1.0, seed)
        s.step(DT, steps)
        x, _, f, _ = s.get_state()
        st = s.stats()
    return x, f, st


def _check_sample(x, f, L, n_sample=4096, seed=11, tol=1e-5):
    """Forces of n_sample particles against the oracle's all-pairs sums for them: half the sample
    at random, half among particles within 1.5 of a face (their partners include periodic images,
    some of particles that drifted below the position offset).  Returns rms(F) of the sample."""
    rng = np.random.default_rng(seed)
    xw = np.mod(x, L)
    near = np.flatnonzero(((xw < 1.5) | (xw > L - 1.5)).any(1))
    idx = np.concatenate([rng.choice(x.shape[0], n_sample // 2, replace=False),
                          rng.choice(near, n_sample - n_sample // 2, replace=False)])
    F = O.forces_sample(x, L, idx)
    rms = np.sqrt((F ** 2).sum(1).mean())
    err = np.sqrt(((f[idx] - F) ** 2).sum(1)).max() / rms
    assert err <= tol, err
    return rms


def test_full_size_forces_sampled():
    """16,384,000 particles (160^3 FCC cells at rho 0.5), 10 steps with the default tuning."""
    x, f, st = _run(160, 10)
    assert st["n"] == 16384000 and st["status_word"] == 0
    rms = _check_sample(x, f, st["box"])
    # sum of forces: each FP32 pair force enters twice with opposite signs up to rounding
    assert np.abs(f.sum(0)).max() < 1e-6 * rms * st["n"]


@pytest.mark.parametrize("tile,lanes", [(4, 4), (8, 2), (3, 8)])
def test_pipelined_force_kernel_matches_single_buffer(tile, lanes):
    """1,048,576 particles: thousands of tiles per launch, so each CTA reuses both buffers and all
    three bookkeeping slots many times; interior and periodic tiles both occur."""
    x1, f1, st1 = _run(64, 4, tile, lanes, 1)
    x2, f2, st2 = _run(64, 4, tile, lanes, 2)
    assert st1["status_word"] == 0 and st2["status_word"] == 0
    assert np.array_equal(x1, x2) and np.array_equal(f1, f2)
    _check_sample(x2, f2, st2["box"])


@pytest.mark.parametrize("nbuf", [1, 2])
def test_fp64_half_list_force_kernels(nbuf):
    """FP64 form with the half list, 1,048,576 particles: the single-buffer kernel (nbuf 1) and the
    pipelined one (nbuf 2: the producer writes shift codes and sorted indices, the consumers
    scatter with atomics) against the oracle on a sample, FP64 tolerance."""
    with ljmd.System(cutoff=RC, margin=MARGIN, precision=ljmd.LJ_FP64, list_form=ljmd.LJ_LIST_HALF) as s:
        s.set_tuning(4, 4, 0, nbuf)
        s.init_lattice(64, 0.5, 1.0, 3)
        s.step(DT, 3)
        x, _, f, _ = s.get_state()
        st = s.stats()
    assert st["status_word"] == 0 and st["list_form"] == ljmd.LJ_LIST_HALF
    _check_sample(x, f, st["box"], tol=1e-11)


def test_full_size_dense_variant_takes_the_half_list():
    """The dense variant of the largest run: 16,384,000 particles at rho 0.8, T 0.9, 10 steps with
    the automatic list form, which takes the half list there (force scatter with atomics)."""
    with ljmd.System(cutoff=RC, margin=MARGIN, precision=ljmd.LJ_MIXED, list_form=ljmd.LJ_LIST_AUTO) as s:
        s.init_lattice(160, 0.8, 0.9, 4)
        s.step(DT, 10)
        x, _, f, _ = s.get_state()
        st = s.stats()
    assert st["list_form"] == ljmd.LJ_LIST_HALF and st["status_word"] == 0
    rms = _check_sample(x, f, st["box"])
    assert np.abs(f.sum(0)).max() < 1e-6 * rms * st["n"]


def test_batched_workload_sampled():
    """The batched workload the bench times: 256 replicas (N in [500, 50000], rho in [0.3, 0.9],
    T in [0.7, 1.5], 6.2M particles), autotuned tiles, 20 steps as 10-step graph replays; forces
    of sampled particles of six replicas against the oracle's all-pairs sum on each replica."""
    n, box, x, v, _ = synth.batch_workload(256, 1000)
    with ljmd.Batch(n, box, cutoff=RC, margin=0.3) as b:
        b.set_state(x, v)
        b.autotune(trials=2)
        b.step(0.004, 20, graph_steps=10)
        gx, _, gf = b.get_state()
        st = b.stats()
    assert st["status_word"] == 0 and st["steps"] >= 20
    offs = np.concatenate([[0], np.cumsum(n)])
    rng = np.random.default_rng(3)
    for r in rng.choice(len(n), 6, replace=False):
        xr, fr = gx[offs[r]:offs[r + 1]], gf[offs[r]:offs[r + 1]]
        idx = rng.choice(len(xr), 16, replace=False)
        F = O.forces_sample(xr, float(box[r]), idx)
        rms = np.sqrt((F ** 2).sum(1).mean())
        assert np.sqrt(((fr[idx] - F) ** 2).sum(1)).max() / rms <= 1e-5, r


def test_differentiable_workload_mixed_against_fp64():
    """The differentiable workload the bench times: 32,000 particles (FCC thinned, rho 0.6, T 1.2),
    50 steps, loss over the last 10, checkpoints every 10: the mixed form's loss and gradients
    against the FP64 form's (relative 1e-3, the stated gradient tolerance)."""
    x, L = synth.fcc_thinned(32000, 0.6, 5)
    v = synth.thermal_velocities(len(x), 1.2, 5)
    out = {}
    for prec in (ljmd.LJ_MIXED, ljmd.LJ_FP64):
        with ljmd.System(cutoff=RC, margin=MARGIN, precision=prec, energy_every=0) as s:
            out[prec] = s.traj_loss_grad(x, v, L, 0.005, 50, 10, 10)
    (lm, gxm, gvm, thm), (ld, gxd, gvd, thd) = out[ljmd.LJ_MIXED], out[ljmd.LJ_FP64]
    assert lm == pytest.approx(ld, rel=1e-5)
    for a, b in ((gxm, gxd), (gvm, gvd)):
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b)
    for a, b in zip(thm, thd):
        assert a == pytest.approx(b, rel=1e-3)
