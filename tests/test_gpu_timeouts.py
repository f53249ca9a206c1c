"""Bounded device waits.  With a wait budget far too small for a tile's bulk copies to land, the
list kernel, the single-buffer force kernel and the pipelined force kernel (producer and
consumer warps waiting for each other) give up, record LJ_ST_TIMEOUT in the device status word
and leave after their copies have landed; the device stays usable, which a fresh system then
shows by matching the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_1012_2677_gb300 import ljmd, synth

pytestmark = pytest.mark.gpu

TINY = 16  # SM clock cycles: no bulk copy lands that fast


def _system(nbuf=0):
    s = ljmd.System(cutoff=2.5, margin=0.5, precision=ljmd.LJ_MIXED)
    s.set_tuning(0, 0, 0, nbuf)
    return s


def _device_still_usable():
    x, L = O.fcc_lattice(8, 0.6)
    x = synth.dyadic(x + np.random.default_rng(5).normal(0.0, 0.05, x.shape))
    F, _, _ = O.forces(x, L)
    with _system() as s:
        s.set_state(x, None, L)
        s.compute_forces()
        _, _, gf, _ = s.get_state()
        assert s.stats()["status_word"] == 0
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= 1e-5


def test_list_construction_wait_times_out():
    with _system() as s:
        s.init_lattice(20, 0.5, 1.0, 1)  # 32,000 particles, 13 cells per side
        ljmd.ljmd_set_wait_budget(TINY)
        try:
            with pytest.raises(ljmd.LjmdError) as e:
                s.build_pairlist()
        finally:
            ljmd.ljmd_set_wait_budget(0)
        assert e.value.code == ljmd.LJ_EDEVICE
        assert s.stats()["status_word"] & ljmd.LJ_ST_TIMEOUT
    _device_still_usable()


@pytest.mark.parametrize("nbuf", [1, 2])
def test_force_kernel_waits_time_out(nbuf):
    """nbuf 1: the single-buffer kernel (CTA waits for its tile's copies); nbuf 2: the pipelined
    kernel, where consumers also wait for producers and producers for consumers."""
    with _system(nbuf) as s:
        s.init_lattice(20, 0.5, 1.0, 1)
        s.build_pairlist()  # the default budget: a valid list
        ljmd.ljmd_set_wait_budget(TINY)
        try:
            try:
                s.compute_forces()
            except ljmd.LjmdError as e:
                assert e.code == ljmd.LJ_EDEVICE
        finally:
            ljmd.ljmd_set_wait_budget(0)
        assert s.stats()["status_word"] & ljmd.LJ_ST_TIMEOUT
    _device_still_usable()


def test_wait_budget_rejects_negative():
    with pytest.raises(ljmd.LjmdError) as e:
        ljmd.ljmd_set_wait_budget(-1)
    assert e.value.code == ljmd.LJ_EINVAL
