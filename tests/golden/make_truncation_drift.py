"""Write truncation_drift_c1.txt: energy drift of the FP64 oracle's NVE run for each truncation of
the potential (Sec. 2.1: Eq. 2, the constant shift only, the plain cut) at r_c = 2.5 and 3.0.

Workload (the small FP64 configuration): FCC 10^3 x 4 at density 0.5 (L = 20), Gaussian velocities
at T = 1 from SplitMix64 seed 1 with zero momentum, velocity-Verlet with dt = 0.005, 1000 steps.
Per case: max_t |E(t) - E(0)| / |E(0)|, the rms of (E(t) - E(0)) / |E(0)|, and the least-squares
slope of E(t) / N against t.  Calls only the oracle.  Run from the repository root:
    python tests/golden/make_truncation_drift.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle as O  # noqa: E402

STEPS, DT = 1000, 0.005
MODES = {"quadratic": O.TRUNC_QUADRATIC, "shift": O.TRUNC_SHIFT, "cut": O.TRUNC_CUT}


def drift_stats(E, n, dt):
    e0 = abs(E[0])
    t = np.arange(len(E)) * dt
    return (float(np.abs(E - E[0]).max() / e0), float(np.sqrt(((E - E[0]) ** 2).mean()) / e0),
            float(np.polyfit(t, E / n, 1)[0]))


def main():
    x, L = O.fcc_lattice(10, 0.5)
    v = O.init_velocities(len(x), 1.0, 1)
    lines = ["# Energy drift of the FP64 oracle, FCC 10^3 x 4 at rho 0.5, T 1 (seed 1), dt 0.005, 1000 steps.",
             "# Written by tests/golden/make_truncation_drift.py (oracle only).",
             "# rc mode max_rel_drift rms_rel_drift slope_per_particle"]
    for rc in (2.5, 3.0):
        for name, mode in MODES.items():
            p = O.LJParams(rc_over_sigma=rc, mode=mode)
            _, pe0, _ = O.forces(x, L, p)
            _, _, _, pe, ke, _ = O.vv_run(x, v, L, DT, STEPS, p)
            E = np.concatenate([[pe0 + O.kinetic(v)], pe + ke])
            mx, rms, slope = drift_stats(E, len(x), DT)
            lines.append("%.1f %s %.6e %.6e %.6e" % (rc, name, mx, rms, slope))
            print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "truncation_drift_c1.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
