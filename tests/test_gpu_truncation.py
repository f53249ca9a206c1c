"""Energy conservation under each truncation of the potential (Sec. 2.1): Eq. 2 (constant and
quadratic terms, V(r_c) = V'(r_c) = 0), the constant shift alone (V(r_c) = 0, force discontinuous at
r_c) and the plain cut (both discontinuous), at r_c = 2.5 and the longer 3.0.

The small FP64 configuration (FCC 10^3 x 4 at rho 0.5, T 1, seed 1, dt 0.005) runs 1000 steps on
the GPU in both precision forms; its energy drift must be no worse than 1.5x the FP64 oracle's on the
same start.  The oracle's drifts are in tests/golden/truncation_drift_c1.txt, written by
tests/golden/make_truncation_drift.py from the oracle alone."""
import os

import numpy as np
import pytest

from paper_1012_2677_gb300 import ljmd

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "truncation_drift_c1.txt")
MODES = {"quadratic": ljmd.LJ_TRUNC_QUADRATIC, "shift": ljmd.LJ_TRUNC_SHIFT, "cut": ljmd.LJ_TRUNC_CUT}
STEPS, DT = 1000, 0.005


def _oracle_drifts():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        rc, mode, mx, rms, slope = line.split()
        out[(float(rc), mode)] = (float(mx), float(rms), float(slope))
    return out


def drift_stats(E, n, dt):
    """(max |E(t) - E(0)| / |E(0)|, rms of (E(t) - E(0)) / |E(0)|, least-squares slope of E / N)."""
    e0 = abs(E[0])
    t = np.arange(len(E)) * dt
    return (float(np.abs(E - E[0]).max() / e0), float(np.sqrt(((E - E[0]) ** 2).mean()) / e0),
            float(np.polyfit(t, E / n, 1)[0]))


def gpu_drift(rc, trunc, precision):
    import torch
    log = torch.zeros((STEPS + 8, 4), dtype=torch.float64, device="cuda")
    with ljmd.System(cutoff=rc, margin=0.5, truncation=trunc, precision=precision, list_form=ljmd.LJ_LIST_AUTO,
                     energy_every=1) as s:
        s.init_lattice(10, 0.5, 1.0, 1)
        s.set_energy_log(log)
        s.step(DT, STEPS)
        st = s.stats()
    rec = log.cpu().numpy()[:STEPS + 1]
    assert st["status_word"] == 0
    assert np.array_equal(rec[:, 0], np.arange(STEPS + 1))
    return drift_stats(rec[:, 1] + rec[:, 2], st["n"], DT)


@pytest.mark.parametrize("precision", [ljmd.LJ_FP64, ljmd.LJ_MIXED])
@pytest.mark.parametrize("rc", [2.5, 3.0])
@pytest.mark.parametrize("mode", list(MODES))
def test_truncation_drift_no_worse_than_oracle(mode, rc, precision):
    ref = _oracle_drifts()[(rc, mode)]
    got = gpu_drift(rc, MODES[mode], precision)
    assert got[0] <= 1.5 * ref[0], (got, ref)
    assert got[1] <= 1.5 * ref[1], (got, ref)

