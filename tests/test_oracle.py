"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself:
a symbolic solve, finite differences, an ODE solver, a published test vector,
an invariant, an independent brute force on tiny inputs, or a number printed
in the paper (fixtures under tests/golden/ with their citations).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1012_2677_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P = O.LJParams()


def _golden(name):
    out = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#")[0].strip()
        if "=" in line:
            k, v = (s.strip() for s in line.split("=", 1))
            out[k] = float(v) if any(c in v for c in ".e") else int(v)
    return out


def _perturbed_fcc(M, rho, amp, seed):
    x, L = O.fcc_lattice(M, rho)
    return O.wrap(x + synth.displacements(len(x), amp, seed), L), L


# ---------------------------------------------------------------- potential

def test_truncation_coefficients_solve_eq2_conditions():
    """Eq. 2: c2, c0 are fixed by V(rc) = V'(rc) = 0 (Sec. 2.1); solved here by sympy."""
    sp = pytest.importorskip("sympy")
    x, c2, c0 = sp.symbols("x c2 c0")
    V = x ** -12 - x ** -6 + c2 * x ** 2 + c0
    for xc in (sp.Rational(5, 2), sp.Integer(3), sp.Rational(11, 4)):
        sol = sp.solve([V.subs(x, xc), sp.diff(V, x).subs(x, xc)], [c2, c0], dict=True)[0]
        oc2, oc0 = O.trunc_coeffs(float(xc))
        assert oc2 == pytest.approx(float(sol[c2]), rel=1e-14)
        assert oc0 == pytest.approx(float(sol[c0]), rel=1e-14)
    # constant-shift variant: c2 = 0 and V(rc) = 0 only
    sol = sp.solve([(x ** -12 - x ** -6 + c0).subs(x, sp.Rational(5, 2))], [c0], dict=True)[0]
    s2, s0 = O.trunc_coeffs(2.5, O.TRUNC_SHIFT)
    assert s2 == 0.0 and s0 == pytest.approx(float(sol[c0]), rel=1e-14)


def test_truncated_potential_and_force_vanish_at_cutoff():
    """V(rc) = V'(rc) = 0: V(rc - d) is O(d^2), the force O(d); zero at and beyond rc (Alg. 5)."""
    rc = P.rc
    v1, v2 = O.pair_v((rc - 1e-3) ** 2), O.pair_v((rc - 5e-4) ** 2)
    assert abs(v1) < 1e-4 and v1 / v2 == pytest.approx(4.0, rel=2e-3)
    f1, f2 = O.pair_f((rc - 1e-3) ** 2), O.pair_f((rc - 5e-4) ** 2)
    assert f1 / f2 == pytest.approx(2.0, rel=2e-3)
    assert O.pair_v(rc * rc) == 0.0 and O.pair_f(rc * rc) == 0.0
    assert O.pair_v(9.0) == 0.0 and O.pair_f(9.0) == 0.0


def test_eq1_minimum():
    """Eq. 1: V(2^(1/6) sigma) = -eps and the force vanishes there, for any eps, sigma."""
    for eps, sigma in ((1.0, 1.0), (1.7, 0.8)):
        rm = 2.0 ** (1.0 / 6.0) * sigma
        assert O.v_raw(rm, eps, sigma) == pytest.approx(-eps, abs=1e-14)
        assert abs(O.f_raw(rm, eps, sigma)) < 1e-13
    # the Eq. 2 potential is shifted and tilted: its value at 2^(1/6) is not -1
    assert O.pair_v(2.0 ** (1.0 / 3.0)) == pytest.approx(-0.944761, abs=1e-6)


def test_alg6_force_is_minus_gradient():
    """Alg. 6 coefficient: f r = dV/dr (force on i from j is f (q_j - q_i)), by central differences."""
    for p in (P, O.LJParams(eps=1.3, sigma=0.9), O.LJParams(mode=O.TRUNC_SHIFT), O.LJParams(mode=O.TRUNC_CUT)):
        for r in np.linspace(0.85 * p.sigma, p.rc - 0.01, 37):
            h = 1e-6
            dvdr = (O.pair_v((r + h) ** 2, p) - O.pair_v((r - h) ** 2, p)) / (2 * h)
            assert O.pair_f(r * r, p) * r == pytest.approx(dvdr, rel=1e-7, abs=1e-8)


def test_shift_only_truncation_keeps_raw_force():
    """Sec. 2.1: with c2 = 0 the force equals the untruncated Eq. 1 force."""
    p = O.LJParams(mode=O.TRUNC_SHIFT)
    for r in (0.9, 1.1, 1.5, 2.2, 2.49):
        assert -O.pair_f(r * r, p) * r == pytest.approx(O.f_raw(r), rel=1e-13)
        assert O.pair_v(r * r, p) - O.v_raw(r) == pytest.approx(O.pair_v(2.45 ** 2, p) - O.v_raw(2.45), abs=1e-12)


# ---------------------------------------------------------------- forces, energies

def test_forces_are_minus_gradient_of_pe():
    x, L = _perturbed_fcc(3, 0.5, 0.25, 11)
    F, pe, _ = O.forces(x, L)
    w = synth.gaussian(x.shape, 12)
    h = 1e-6
    dpe = (O.forces(x + h * w, L)[1] - O.forces(x - h * w, L)[1]) / (2 * h)
    assert np.sum(F * w) == pytest.approx(-dpe, rel=1e-7)


def test_newton_third_law_total_force_zero():
    x, L = _perturbed_fcc(4, 0.8, 0.15, 13)
    F, _, _ = O.forces(x, L)
    assert np.abs(F.sum(0)).max() < 1e-11 * np.abs(F).sum()


def test_virial_is_volume_derivative():
    """W = sum_{i<j} r_ij . F_ij = -dPE/dlambda under uniform scaling of positions and box."""
    x, L = _perturbed_fcc(3, 0.6, 0.2, 14)
    _, _, W = O.forces(x, L)
    h = 1e-6
    dpe = (O.forces(x * (1 + h), L * (1 + h))[1] - O.forces(x * (1 - h), L * (1 - h))[1]) / (2 * h)
    assert W == pytest.approx(-dpe, rel=1e-7)


def test_forces_sample_matches_full():
    x, L = _perturbed_fcc(3, 0.5, 0.2, 15)
    F, _, _ = O.forces(x, L)
    idx = np.array([0, 7, 50, 107])
    assert np.array_equal(O.forces_sample(x, L, idx), F[idx])


# ---------------------------------------------------------------- pair set, grid, sorted list

def _numpy_pairs(x, L, rs):
    d = x[None, :, :] - x[:, None, :]
    d = np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))
    r2 = d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1] + d[..., 2] * d[..., 2]
    i, j = np.nonzero(np.triu(r2 < rs * rs, k=1))
    return np.stack([i, j], 1)


@pytest.mark.parametrize("N,L,rs,seed", [(300, 7.0, 3.0, 1), (500, 9.5, 2.8, 2), (64, 6.1, 3.0, 3)])
def test_pair_set_equals_independent_brute_force(N, L, rs, seed):
    x = synth.uniform_positions(N, L, seed)
    assert np.array_equal(O.pairs_within(x, L, rs), _numpy_pairs(x, L, rs))


def test_pair_set_strict_inequality_and_periodic_images():
    L, rs = 10.0, 2.5
    x = np.array([[1.0, 1.0, 1.0], [3.5, 1.0, 1.0],            # exactly rs apart: excluded
                  [5.0, 5.0, 5.0], [5.0, 5.0, 7.5 - 2 ** -40],  # just inside
                  [0.25, 9.0, 9.0], [9.75, 9.0, 9.0]])          # across the boundary, 0.5 apart
    assert [tuple(p) for p in O.pairs_within(x, L, rs)] == [(2, 3), (4, 5)]


def test_cell_side_puts_partners_in_adjacent_cells():
    """Sec. 2.2: with cell side >= rs every interacting pair is in the same or an adjacent cell."""
    L, rs = 13.0, 3.0
    x = synth.uniform_positions(800, L, 4)
    n = O.cells_per_side(L, rs)
    assert L / n >= rs and L / (n + 1) < rs
    lab = O.cell_labels(x, L, n)
    cz, cy, cx = lab % n, (lab // n) % n, lab // (n * n)
    for i, j in O.pairs_within(x, L, rs):
        for c in (cx, cy, cz):
            dc = (c[j] - c[i]) % n
            assert dc in (0, 1, n - 1)


def _fig3_pointer_procedure(labels, ncells):
    """Sec. 2.2 / Fig. 3 written as a loop: count, set pointers, place and advance."""
    count = [0] * ncells
    for c in labels:
        count[c] += 1
    pointer = [0] * ncells
    for c in range(1, ncells):
        pointer[c] = pointer[c - 1] + count[c - 1]
    start = list(pointer)
    out = [None] * len(labels)
    for i, c in enumerate(labels):
        out[pointer[c]] = i
        pointer[c] += 1
    return count, start, out


def test_grid_list_counting_sort_like_fig3():
    labels = [int(c) for c in synth.rng(5).integers(0, 4, size=14)]  # 14 particles, 4 cells
    cnt, ptr, order = O.grid_list(labels, 4)
    c2, s2, o2 = _fig3_pointer_procedure(labels, 4)
    assert list(cnt) == c2 and list(ptr[:-1]) == s2 and list(order) == o2 and ptr[-1] == 14
    labels = [int(c) for c in synth.rng(6).integers(0, 27, size=500)]
    cnt, ptr, order = O.grid_list(labels, 27)
    c2, s2, o2 = _fig3_pointer_procedure(labels, 27)
    assert list(cnt) == c2 and list(ptr[:-1]) == s2 and list(order) == o2


def test_sorted_pair_list_like_fig6():
    x = synth.uniform_positions(120, 7.0, 7)
    pairs = O.pairs_within(x, 7.0, 3.0)
    shuffled = pairs[synth.rng(8).permutation(len(pairs))][:, ::-1]  # any order, either orientation
    kp, sl = O.sorted_pair_list(shuffled, 120)
    # Fig. 6 as a loop: count partners per key, set pointers, place partners
    cnt = [0] * 120
    for a, b in shuffled:
        cnt[min(a, b)] += 1
    ptr = [0] * 121
    for i in range(120):
        ptr[i + 1] = ptr[i] + cnt[i]
    assert list(kp) == ptr and kp[-1] == len(pairs)
    for i in range(120):
        partners = sorted(max(a, b) for a, b in pairs if min(a, b) == i)
        assert list(sl[kp[i]:kp[i + 1]]) == partners


# ---------------------------------------------------------------- initial state

def test_fcc_lattice_matches_paper_benchmark_box():
    """Sec. 4.5: 500,000 particles at density 0.5 fill a 100^3 box per process."""
    g = _golden("paper_benchmark_pairs.txt")
    M = round((g["particles_per_process"] / 4) ** (1 / 3))
    x, L = O.fcc_lattice(M, g["density"])
    assert len(x) == g["particles_per_process"] and L == pytest.approx(g["box_per_process"], rel=1e-14)
    assert x.min() >= 0.0 and x.max() < L


def test_fcc_nearest_neighbours():
    x, L = O.fcc_lattice(3, 0.8)
    a = (4 / 0.8) ** (1 / 3)
    assert np.all(O.neighbor_counts(x, L, a / math.sqrt(2) * 1.001) == 12)
    assert np.all(O.neighbor_counts(x, L, a / math.sqrt(2) * 0.999) == 0)
    assert len(x) / L ** 3 == pytest.approx(0.8, rel=1e-13)


def test_splitmix64_published_vectors():
    g = _golden("splitmix64_vectors.txt")
    for k in range(5):
        assert O.splitmix_at(g["seed"], k) == g["out%d" % k]


def test_velocities_zero_momentum_temperature_and_gaussian():
    scipy_stats = pytest.importorskip("scipy.stats")
    N, T = 4000, 1.3
    v = O.init_velocities(N, T, 1)
    assert np.abs(v.sum(0)).max() < 1e-11
    assert (v ** 2).sum() == pytest.approx(3 * (N - 1) * T, rel=1e-13)
    raw = O.gaussian_raw(N, 1).ravel()
    assert scipy_stats.kstest(raw, "norm").pvalue > 1e-3
    assert np.array_equal(O.init_velocities(N, T, 1), v) and not np.array_equal(O.init_velocities(N, T, 2), v)


# ---------------------------------------------------------------- integrator

def test_velocity_verlet_two_particles_against_ode_solver():
    """Two particles on a line: VV converges to the exact relative motion at second order."""
    integ = pytest.importorskip("scipy.integrate")
    L, r0, tend = 12.0, 1.6, 1.0
    x0 = np.array([[4.0, 6.0, 6.0], [4.0 + r0, 6.0, 6.0]])

    def rhs(t, y):  # relative coordinate r, reduced mass 1/2: r'' = -2 V'(r) = -2 f r
        r, vr = y
        return [vr, -2.0 * O.pair_f(r * r) * r]

    ref = integ.solve_ivp(rhs, (0, tend), [r0, 0.0], method="DOP853", rtol=1e-13, atol=1e-14)
    errs = []
    for dt in (0.01, 0.005):
        n = round(tend / dt)
        x, v, *_ = O.vv_run(x0, np.zeros_like(x0), L, dt, n)
        errs.append(abs((x[1, 0] - x[0, 0]) - ref.y[0, -1]))
    assert errs[0] < 2e-3 and errs[0] / errs[1] == pytest.approx(4.0, rel=0.05)


def test_velocity_verlet_time_reversible():
    x0, L = _perturbed_fcc(3, 0.6, 0.15, 16)
    v0 = O.init_velocities(len(x0), 1.0, 3)
    x, v, *_ = O.vv_run(x0, v0, L, 0.005, 40)
    xb, vb, *_ = O.vv_run(x, -v, L, 0.005, 40)
    assert np.abs(xb - x0).max() < 1e-10 and np.abs(vb + v0).max() < 1e-9


def test_nve_energy_conservation_and_dt2_scaling():
    x0, L = O.fcc_lattice(4, 0.5)
    v0 = O.init_velocities(len(x0), 1.0, 1)
    spread = []
    for dt, n in ((0.004, 100), (0.002, 200)):
        _, _, _, pe, ke, _ = O.vv_run(x0, v0, L, dt, n)
        e = pe + ke
        spread.append(e.max() - e.min())
        assert spread[-1] / abs(e[0]) < 2e-3
    assert 2.5 < spread[0] / spread[1] < 6.0


# ---------------------------------------------------------------- derivatives (differentiable form)

def test_hvp_matches_finite_differences_of_forces():
    x, L = _perturbed_fcc(3, 0.6, 0.2, 17)
    w = synth.gaussian(x.shape, 18)
    h = 1e-5
    fd = -(O.forces(x + h * w, L)[0] - O.forces(x - h * w, L)[0]) / (2 * h)
    hv = O.hvp(x, L, w)
    assert np.linalg.norm(hv - fd) < 1e-6 * np.linalg.norm(fd)


def test_dense_hessian_symmetric_and_consistent():
    x, L = _perturbed_fcc(2, 0.3, 0.2, 19)  # 32 particles, L = 7.1
    H = O.hessian(x, L)
    assert np.abs(H - H.T).max() < 1e-10 * np.abs(H).max()
    w = synth.gaussian(x.shape, 20)
    assert np.allclose(H @ w.ravel(), O.hvp(x, L, w).ravel(), rtol=1e-12, atol=1e-12 * np.abs(H).max())
    h = 1e-5
    for col in (0, 17, 50):
        e = np.zeros(x.size)
        e[col] = h
        fd = -(O.forces(x + e.reshape(x.shape), L)[0] - O.forces(x - e.reshape(x.shape), L)[0]).ravel() / (2 * h)
        assert np.linalg.norm(H[:, col] - fd) < 1e-6 * max(np.linalg.norm(fd), 1.0)


def test_parameter_derivatives():
    x, L = _perturbed_fcc(3, 0.6, 0.2, 21)
    p = O.LJParams(eps=1.2, sigma=0.95)
    lam = synth.gaussian(x.shape, 22)
    dpe, vjp = O.param_derivs(x, L, p, lam)
    pe = O.forces(x, L, p)[1]
    assert dpe[0] == pytest.approx(pe / p.eps, rel=1e-13)
    h = 1e-6
    for k, (pp, pm) in enumerate(((O.LJParams(eps=1.2 + h, sigma=0.95), O.LJParams(eps=1.2 - h, sigma=0.95)),
                                  (O.LJParams(eps=1.2, sigma=0.95 + h), O.LJParams(eps=1.2, sigma=0.95 - h)))):
        Fp, pep, _ = O.forces(x, L, pp)
        Fm, pem, _ = O.forces(x, L, pm)
        assert dpe[k] == pytest.approx((pep - pem) / (2 * h), rel=1e-6)
        assert vjp[k] == pytest.approx(np.sum(lam * (Fp - Fm)) / (2 * h), rel=1e-6)


def test_trajectory_gradient_matches_finite_differences():
    x0, L = _perturbed_fcc(3, 0.6, 0.1, 23)
    v0 = O.init_velocities(len(x0), 1.2, 5)
    p = O.LJParams(eps=1.0, sigma=1.0)
    dt, n, npe = 0.005, 20, 5
    loss, gx, gv, (ge, gs) = O.traj_loss_grad(x0, v0, L, dt, n, npe, p)
    assert loss == pytest.approx(O.traj_loss(x0, v0, L, dt, n, npe, p), rel=1e-14)
    h = 1e-5
    f = lambda pp, xx=x0, vv=v0: O.traj_loss(xx, vv, L, dt, n, npe, pp)
    assert ge == pytest.approx((f(O.LJParams(eps=1 + h)) - f(O.LJParams(eps=1 - h))) / (2 * h), rel=1e-6)
    assert gs == pytest.approx((f(O.LJParams(sigma=1 + h)) - f(O.LJParams(sigma=1 - h))) / (2 * h), rel=1e-6)
    for (i, k) in ((0, 0), (13, 2), (77, 1)):
        e = np.zeros_like(x0)
        e[i, k] = h
        assert gx[i, k] == pytest.approx((f(p, x0 + e) - f(p, x0 - e)) / (2 * h), rel=1e-5, abs=1e-10)
        assert gv[i, k] == pytest.approx((f(p, x0, v0 + e) - f(p, x0, v0 - e)) / (2 * h), rel=1e-5, abs=1e-10)


# ---------------------------------------------------------------- the paper's printed pair count

@pytest.mark.slow
def test_pair_count_of_paper_benchmark_final_state():
    """Sec. 5.4 prints 11,629,010..11,656,318 search-length pairs per 500,000-particle process at
    the end of the Sec. 4.5 run.  A 4,000-particle replica of that run, with cross-border pairs of a
    100^3 process domain counted by both sides as a domain-decomposed list does, lands within 1%."""
    g = _golden("paper_benchmark_pairs.txt")
    x, L = O.fcc_lattice(10, g["density"])
    v = g["speed"] * synth.unit_vectors(len(x), 6)
    x, v, *_ = O.vv_run(x, v, L, g["dt"], g["steps_total"])
    xw = O.wrap(x, L)
    pairs = O.pairs_within(xw, L, g["search_length"])
    d = xw[pairs[:, 1]] - xw[pairs[:, 0]]
    d = np.where(d > 0.5 * L, d - L, np.where(d < -0.5 * L, d + L, d))
    per_process = (len(pairs) + np.abs(d).sum() / g["box_per_process"]) / len(x)
    paper = 0.5 * (g["pairs_max"] + g["pairs_min"]) / g["particles_per_process"]
    assert per_process == pytest.approx(paper, rel=0.01)


# ---------------------------------------------------------------- truncation variants over a run

def test_stored_truncation_drifts_order_as_the_paper_argues():
    """Sec. 2.1: a potential that jumps at r_c (the plain cut) conserves energy far worse than the
    forms with V(r_c) = 0, and a longer cutoff narrows the gap.  Checked on the oracle runs stored
    in truncation_drift_c1.txt (written by make_truncation_drift.py, oracle only), which the GPU
    drift tests compare against."""
    d = {}
    for line in open(os.path.join(GOLDEN, "truncation_drift_c1.txt")):
        if line.strip() and not line.startswith("#"):
            rc, mode, mx, rms, slope = line.split()
            d[(float(rc), mode)] = float(rms)
    assert len(d) == 6
    for rc in (2.5, 3.0):
        assert d[(rc, "cut")] > 4 * max(d[(rc, "quadratic")], d[(rc, "shift")])
    assert d[(3.0, "cut")] < d[(2.5, "cut")]
