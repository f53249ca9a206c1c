"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Inputs come from the seeded generators and the oracle only, rounded to a dyadic grid so the
library stores them bit for bit.  Tolerances (from the specification of the method's
targets): forces max|dF| / rms|F| <= 1e-5, 10-step positions within 1e-4 sigma, energy drift
no worse than the oracle's (x1.5), pair lists bit-exact as sets of id pairs.
"""
import numpy as np
import pytest

import oracle as O
from paper_1012_2677_gb300 import ljmd, synth

pytestmark = pytest.mark.gpu

FORMS = [(ljmd.LJ_MIXED, ljmd.LJ_LIST_FULL), (ljmd.LJ_MIXED, ljmd.LJ_LIST_HALF),
         (ljmd.LJ_FP64, ljmd.LJ_LIST_FULL), (ljmd.LJ_FP64, ljmd.LJ_LIST_HALF)]
FORCE_TOL = {ljmd.LJ_MIXED: 1e-5, ljmd.LJ_FP64: 1e-11}


def _system(precision=ljmd.LJ_MIXED, list_form=ljmd.LJ_LIST_FULL, cutoff=2.5, margin=0.5, lanes=0, **kw):
    return ljmd.System(cutoff=cutoff, margin=margin, precision=precision, list_form=list_form, lanes=lanes, **kw)


def _thermal_state(M, rho, T, seed, steps=60, dt=0.005):
    """Oracle-equilibrated FCC start (positions folded, dyadic)."""
    x, L = O.fcc_lattice(M, rho)
    v = O.init_velocities(len(x), T, seed)
    x, v, *_ = O.vv_run(x, v, L, dt, steps)
    return synth.dyadic(O.wrap(x, L)), v, L


_CACHE = {}


def thermal(M, rho, T, seed):
    key = (M, rho, T, seed)
    if key not in _CACHE:
        _CACHE[key] = _thermal_state(M, rho, T, seed)
    return _CACHE[key]


def _pairs_set(P):
    return set(map(tuple, np.asarray(P).tolist()))


def _brute_pairs_numpy(x, L, r):
    """Pairs (i < j) closer than r by direct numpy evaluation (a property check of the
    library's own state, independent of the oracle)."""
    d = x[None, :, :] - x[:, None, :]
    d -= L * np.round(d / L)
    i, j = np.nonzero(np.triu((d ** 2).sum(-1) < r * r, k=1))
    return np.stack([i, j], 1)


# ------------------------------------------------------------------------------------ initial state

def test_init_lattice_matches_oracle():
    with _system(precision=ljmd.LJ_FP64) as s:
        s.init_lattice(6, 0.5, 1.0, 1)
        x, v, f, img = s.get_state()
    xo, L = O.fcc_lattice(6, 0.5)
    vo = O.init_velocities(len(xo), 1.0, 1)
    assert s.box == pytest.approx(L, rel=1e-15)
    assert np.abs(x - xo).max() < 1e-12
    assert np.abs(v - vo).max() < 1e-12 * np.abs(vo).max()
    assert not img.any()


# ------------------------------------------------------------------------------------ pair list

@pytest.mark.parametrize("precision,list_form", FORMS)
@pytest.mark.parametrize("N,L,rs_margin,seed", [
    (700, 12.0, (2.5, 0.5), 1),     # 4 cells per side, cell side exactly r_s
    (900, 17.3, (2.5, 0.3), 2),     # 6 cells, ragged
    (300, 7.2, (2.5, 0.3), 3),      # 2 cells per side (neighbour cells alias)
    (150, 6.3, (2.5, 0.3), 4),      # 2 cells, L just above 2 (r_s + margin)
    (1, 9.0, (2.5, 0.5), 5),        # a single particle: empty list
])
def test_pair_list_bit_exact(precision, list_form, N, L, rs_margin, seed):
    rc, margin = rs_margin
    x = synth.dyadic(synth.uniform_positions(N, L, seed))
    with _system(precision, list_form, cutoff=rc, margin=margin) as s:
        s.set_state(x, None, L)
        s.build_pairlist()
        got = s.pairs()
        st = s.stats()
    ref = O.pairs_within(x, L, rc + margin)
    assert np.array_equal(got, ref)
    assert st["list_entries"] == (2 if list_form == ljmd.LJ_LIST_FULL else 1) * len(ref)


@pytest.mark.parametrize("list_form", [ljmd.LJ_LIST_FULL, ljmd.LJ_LIST_HALF])
def test_pair_list_edge_cases(list_form):
    """Particles on cell faces and pairs at r_s to the last bit (the FP64 band decides)."""
    L, rc, margin = 12.0, 2.5, 0.5
    rs = rc + margin
    e = 2.0 ** -40
    pts = [[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [6.0, 6.0, 6.0], [9.0, 9.0, 9.0],  # cell faces (h = 3)
           [1.0, 1.0, 1.0], [1.0 + rs, 1.0, 1.0],                               # exactly r_s: out
           [5.0, 1.0, 1.0], [5.0, 1.0 + rs - e, 1.0],                            # r_s - 2^-40: in
           [1.0, 5.0, 7.0], [1.0, 5.0, 7.0 + rs + e],                            # r_s + 2^-40: out
           [0.5, 11.0, 4.0], [12.0 - 2.5, 11.0, 4.0],                            # across the boundary
           [11.999, 3.0, 3.0], [0.0, 3.0, 3.0]]
    x = np.array(pts)
    x = np.vstack([x, synth.dyadic(synth.uniform_positions(200, L, 9))])
    with _system(ljmd.LJ_MIXED, list_form, cutoff=rc, margin=margin) as s:
        s.set_state(x, None, L)
        s.build_pairlist()
        got = s.pairs()
    assert np.array_equal(got, O.pairs_within(x, L, rs))


def _clustered_state(seed=21):
    """A dense FCC cluster (rho 2.0, nearest neighbours 0.89 apart) inside a sparse jittered cubic
    background (spacing 2): the cluster's cells hold about 54 particles, so a key's three-cell
    windows run to about 160 candidates and its row to about 220 entries.  The list kernel's
    bit pool and segment staging then overflow, and it takes its slower paths (tested again,
    written to global memory directly); the force kernels read such long segments from HBM."""
    a = (4.0 / 2.0) ** (1.0 / 3.0)
    g = np.arange(6)
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
    cells = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 1, 3)
    cluster = 3.0 + ((cells + basis[None]) * a).reshape(-1, 3)
    lo, hi = 3.0 - 1.0, 3.0 + 6 * a + 1.0
    s = np.arange(12) * 2.0 + 1.0
    bg = np.stack(np.meshgrid(s, s, s, indexing="ij"), -1).reshape(-1, 3)
    bg = bg[~np.all((bg > lo) & (bg < hi), axis=1)]
    bg = bg + synth.displacements(len(bg), 0.3, seed)
    cluster = cluster + synth.displacements(len(cluster), 0.05, seed + 1)
    return synth.dyadic(O.wrap(np.vstack([cluster, bg]), 24.0)), 24.0


@pytest.mark.parametrize("precision,list_form", FORMS)
def test_dense_cluster_list_and_forces(precision, list_form):
    """Pair list bit-exact and forces within tolerance where the list kernel's shared-memory areas
    overflow (see _clustered_state)."""
    x, L = _clustered_state()
    with _system(precision, list_form) as s:
        s.set_state(x, None, L)
        s.build_pairlist()
        got = s.pairs()
        s.compute_forces()
        _, _, gf, _ = s.get_state()
        st = s.stats()
    assert st["status_word"] == 0
    ref = O.pairs_within(x, L, 3.0)
    assert np.array_equal(got, ref)
    assert np.bincount(ref.ravel(), minlength=len(x)).max() > 150  # rows long enough to overflow
    F, _, _ = O.forces(x, L)
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= FORCE_TOL[precision]


def _oracle_grid(x, L, rs):
    n = O.cells_per_side(L, rs)
    count, pointer, order = O.grid_list(O.cell_labels(O.wrap(x, L), L, n), n ** 3)
    return count, pointer, order


@pytest.mark.parametrize("precision", [ljmd.LJ_MIXED, ljmd.LJ_FP64])
def test_cell_grid_matches_counting_sort(precision):
    """The library's cell grid is the oracle's counting sort (Sec. 2.2, Fig. 3) element by element:
    GridParticleNumber (the pointer differences), GridPointer and GridList (labels ascending, ties in
    id order), on a random state, on particles placed exactly on cell faces, and after a run whose
    rebuilds left the particles in a cell order unrelated to their ids (the stable order must still
    come out by id)."""
    L, rc, margin = 14.0, 2.5, 0.5
    rs = rc + margin
    n = O.cells_per_side(L, rs)
    h = L / n
    x = synth.dyadic(synth.uniform_positions(1500, L, 12))
    faces = synth.dyadic(np.array([[i * h, j * h, (i + j) % n * h] for i in range(n) for j in range(n)]))
    x = np.vstack([x, faces])
    with _system(precision, cutoff=rc, margin=margin) as s:
        s.set_state(x, None, L)
        s.build_pairlist()
        ptr, lst = s.grid()
        assert s.stats()["cells_per_side"] == n
    count, pointer, order = _oracle_grid(x, L, rs)
    assert np.array_equal(ptr, pointer)
    assert np.array_equal(np.diff(ptr), count)
    assert np.array_equal(lst, order)
    # a liquid run: rebuilds re-sort the particles, so the order entering the next sort is not by id
    x, v, L = thermal(8, 0.6, 1.2, 9)
    with _system(precision, cutoff=rc, margin=margin) as s:
        s.set_state(x, v, L)
        s.step(0.005, 40)
        assert s.stats()["rebuilds"] >= 2
        s.build_pairlist()                      # the grid of the current (folded) positions
        gx, _, _, _ = s.get_state()
        ptr, lst = s.grid()
    count, pointer, order = _oracle_grid(gx, L, rs)
    assert np.array_equal(ptr, pointer)
    assert np.array_equal(lst, order)


# ------------------------------------------------------------------------------------ forces

@pytest.mark.parametrize("precision,list_form", FORMS)
@pytest.mark.parametrize("lanes", [0, 1, 4, 32])
def test_forces_and_energies_match_oracle(precision, list_form, lanes):
    x, v, L = thermal(10, 0.5, 1.0, 1)
    F, pe, vir = O.forces(x, L)
    with _system(precision, list_form, lanes=lanes) as s:
        s.set_state(x, v, L)
        s.compute_forces()
        gx, gv, gf, _ = s.get_state()
        gpe, gke, gvir = s.energies()
    assert np.array_equal(gx, x)
    rms = np.sqrt((F ** 2).sum(1).mean())
    err = np.sqrt(((gf - F) ** 2).sum(1)).max() / rms
    assert err <= FORCE_TOL[precision], err
    etol = 1e-6 if precision == ljmd.LJ_MIXED else 1e-12
    assert gpe == pytest.approx(pe, rel=etol)
    assert gvir == pytest.approx(vir, rel=etol)
    assert gke == pytest.approx(O.kinetic(v), rel=1e-6 if precision == ljmd.LJ_MIXED else 1e-13)
    assert np.abs(gf.sum(0)).max() < (1e-4 if precision == ljmd.LJ_MIXED else 1e-9) * rms


@pytest.mark.parametrize("precision,list_form", FORMS)
@pytest.mark.parametrize("tile,lanes,nbuf", [(1, 4, 1), (2, 2, 2), (4, 8, 2), (8, 4, 1), (14, 16, 2), (5, 1, 2)])
def test_forces_and_list_under_tuning_knobs(precision, list_form, tile, lanes, nbuf):
    """Every tile shape / lanes / buffering choice gives the oracle's forces and the exact list."""
    x, v, L = thermal(8, 0.6, 1.2, 9)  # 2048 particles, 5 cells per side (ragged tiles for T = 2, 4)
    F, pe, vir = O.forces(x, L)
    with _system(precision, list_form) as s:
        s.set_tuning(tile, lanes, 0, nbuf)
        s.set_state(x, v, L)
        s.compute_forces()
        _, _, gf, _ = s.get_state()
        gpe, _, gvir = s.energies()
        got = s.pairs()
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= FORCE_TOL[precision]
    etol = 1e-6 if precision == ljmd.LJ_MIXED else 1e-12
    assert gpe == pytest.approx(pe, rel=etol) and gvir == pytest.approx(vir, rel=etol)
    assert np.array_equal(got, O.pairs_within(x, L, 3.0))


@pytest.mark.parametrize("precision,list_form", FORMS)
@pytest.mark.parametrize("nbuf", [1, 2])
def test_forces_after_face_layer_drifts_below_offset(precision, list_form, nbuf):
    """FCC start: one lattice layer lies exactly on each lower face, so within a few steps half of
    it drifts below the position offset (the finer hi grid of the binade below) while the list
    is kept; its +L images meet the upper-face layer at nearest-neighbour distance, where an
    inexact image shift of hi would show as ~1e-4 relative force error."""
    with _system(precision, list_form) as s:
        s.set_tuning(0, 0, 0, nbuf)
        s.init_lattice(8, 0.5, 1.0, 5)
        s.step(0.005, 4)
        x, _, gf, _ = s.get_state()
        L = s.stats()["box"]
        assert s.stats()["rebuilds"] == 1
    assert (x.min(0) < 0).all()  # some particles left through every lower face
    F, _, _ = O.forces(x, L)
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= FORCE_TOL[precision]


@pytest.mark.parametrize("precision,rho,expect", [(ljmd.LJ_MIXED, 0.5, ljmd.LJ_LIST_FULL),
                                                  (ljmd.LJ_MIXED, 0.8, ljmd.LJ_LIST_HALF),
                                                  (ljmd.LJ_FP64, 0.5, ljmd.LJ_LIST_HALF)])
def test_auto_list_form(precision, rho, expect):
    """LJ_LIST_AUTO: the full list in the mixed form below 75 full-list partners per particle
    ((4/3) pi r_s^3 rho: 56.5 at rho 0.5, 90 at rho 0.8), the half list above and in the FP64 form;
    forces, energies and the pair set are the oracle's either way."""
    x, v, L = thermal(8, rho, 1.0, 6)
    F, pe, vir = O.forces(x, L)
    with _system(precision, ljmd.LJ_LIST_AUTO) as s:
        s.set_state(x, v, L)
        s.compute_forces()
        st = s.stats()
        _, _, gf, _ = s.get_state()
        gpe, _, gvir = s.energies()
        got = s.pairs()
    assert st["list_form"] == expect
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= FORCE_TOL[precision]
    etol = 1e-6 if precision == ljmd.LJ_MIXED else 1e-12
    assert gpe == pytest.approx(pe, rel=etol) and gvir == pytest.approx(vir, rel=etol)
    assert np.array_equal(got, O.pairs_within(x, L, 3.0))


def test_adjoint_requires_the_full_list():
    """The adjoint kernel reads every partner of a key from the key's own row: an explicit half
    list is refused, an automatic one switches to the full list and the HVP is the oracle's."""
    x, v, L = thermal(8, 0.8, 1.0, 6)
    w = np.random.default_rng(12).normal(size=x.shape)
    with _system(ljmd.LJ_MIXED, ljmd.LJ_LIST_HALF) as s:
        s.set_state(x, v, L)
        with pytest.raises(ljmd.LjmdError) as e:
            s.hvp(w)
        assert e.value.code == ljmd.LJ_ESTATE
    ref = O.hvp(x, L, w)
    with _system(ljmd.LJ_MIXED, ljmd.LJ_LIST_AUTO) as s:
        s.set_state(x, v, L)
        assert s.stats()["list_form"] == ljmd.LJ_LIST_HALF
        hw, _ = s.hvp(w)
        assert s.stats()["list_form"] == ljmd.LJ_LIST_FULL
    rms = np.sqrt((ref ** 2).sum(1).mean())
    assert np.sqrt(((hw - ref) ** 2).sum(1)).max() / rms <= 2e-4


@pytest.mark.parametrize("precision", [ljmd.LJ_MIXED, ljmd.LJ_FP64])
def test_forces_dense_liquid(precision):
    x, v, L = thermal(8, 0.8, 0.9, 4)
    F, pe, _ = O.forces(x, L)
    with _system(precision) as s:
        s.set_state(x, v, L)
        s.compute_forces()
        _, _, gf, _ = s.get_state()
        gpe, _, _ = s.energies()
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= FORCE_TOL[precision]
    assert gpe == pytest.approx(pe, rel=1e-6)


@pytest.mark.parametrize("trunc", [ljmd.LJ_TRUNC_SHIFT, ljmd.LJ_TRUNC_CUT])
def test_truncation_variants(trunc):
    x, v, L = thermal(8, 0.5, 1.0, 2)
    p = O.LJParams(mode=trunc)
    F, pe, _ = O.forces(x, L, p)
    with _system(ljmd.LJ_FP64, truncation=trunc) as s:
        s.set_state(x, v, L)
        s.compute_forces()
        _, _, gf, _ = s.get_state()
        gpe, _, _ = s.energies()
    rms = np.sqrt((F ** 2).sum(1).mean())
    assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= 1e-11
    assert gpe == pytest.approx(pe, rel=1e-12)


def test_eps_sigma_parameters():
    x, v, L = thermal(8, 0.5, 1.0, 3)
    p = O.LJParams(eps=1.3, sigma=0.95)
    F, pe, _ = O.forces(x, L, p)
    for precision, tol in ((ljmd.LJ_FP64, 1e-11), (ljmd.LJ_MIXED, 1e-5)):
        with ljmd.System(eps=1.3, sigma=0.95, cutoff=2.5 * 0.95, margin=0.5, precision=precision) as s:
            s.set_state(x, v, L)
            s.compute_forces()
            _, _, gf, _ = s.get_state()
            gpe, _, _ = s.energies()
        rms = np.sqrt((F ** 2).sum(1).mean())
        assert np.sqrt(((gf - F) ** 2).sum(1)).max() / rms <= tol
        assert gpe == pytest.approx(pe, rel=max(tol, 1e-6))


# ------------------------------------------------------------------------------------ trajectories

@pytest.mark.parametrize("precision,list_form", FORMS)
def test_ten_step_trajectory(precision, list_form):
    x, v, L = thermal(10, 0.5, 1.0, 1)
    xo, vo, Fo, *_ = O.vv_run(x, v, L, 0.005, 10)
    with _system(precision, list_form) as s:
        s.set_state(x, v, L)
        s.step(0.005, 10)
        gx, gv, gf, img = s.get_state()
    gx_unwrapped = gx + img * L
    tol = 1e-4 if precision == ljmd.LJ_MIXED else 1e-10
    assert np.abs(gx_unwrapped - xo).max() < tol
    assert np.abs(gv - vo).max() < (1e-3 if precision == ljmd.LJ_MIXED else 1e-8)


@pytest.mark.parametrize("precision", [ljmd.LJ_MIXED, ljmd.LJ_FP64])
def test_nve_drift_no_worse_than_oracle(precision):
    """Config 1 of the workload (FCC 10^3 x 4, rho 0.5, T 1, dt 0.005, 100 steps)."""
    xo, L = O.fcc_lattice(10, 0.5)
    vo = O.init_velocities(len(xo), 1.0, 1)
    _, _, _, pe, ke, _ = O.vv_run(xo, vo, L, 0.005, 100)
    Fo, pe0, _ = O.forces(xo, L)
    e_or = np.concatenate([[pe0 + O.kinetic(vo)], pe + ke])
    import torch
    log = torch.zeros((128, 4), dtype=torch.float64, device="cuda")
    with _system(precision, energy_every=1) as s:
        s.init_lattice(10, 0.5, 1.0, 1)
        s.set_energy_log(log)
        s.step(0.005, 100)
        st = s.stats()
    rec = log.cpu().numpy()[:101]
    assert np.array_equal(rec[:, 0], np.arange(101))
    e_gpu = rec[:, 1] + rec[:, 2]
    drift_or = np.abs(e_or - e_or[0]).max() / abs(e_or[0])
    drift_gpu = np.abs(e_gpu - e_gpu[0]).max() / abs(e_gpu[0])
    assert drift_gpu <= 1.5 * drift_or, (drift_gpu, drift_or)
    assert np.abs(e_gpu - e_or).max() / abs(e_or[0]) < 1e-4
    assert st["rebuilds"] >= 1 and st["status_word"] == 0


def test_list_stays_valid_during_run():
    """After every step no pair within r_c is missing from the list (displacement rule)."""
    x, v, L = thermal(6, 0.6, 1.5, 6)
    rc, margin = 2.5, 0.3
    with _system(ljmd.LJ_MIXED, cutoff=rc, margin=margin) as s:
        s.set_state(x, v, L)
        rebuilds = []
        for _ in range(40):
            s.step(0.005, 1)
            gx, _, _, _ = s.get_state()
            listed = _pairs_set(s.pairs())
            inner = _pairs_set(_brute_pairs_numpy(gx, L, rc))
            assert inner <= listed
            rebuilds.append(s.stats()["rebuilds"])
    assert rebuilds[-1] > rebuilds[0]  # the run did cross list lifetimes


def test_status_word_flags_nonfinite():
    x, v, L = thermal(6, 0.5, 1.0, 7)
    v = v.copy()
    v[3, 1] = np.nan
    with _system(ljmd.LJ_MIXED) as s:
        s.set_state(x, v, L)
        with pytest.raises(ljmd.LjmdError) as e:
            s.step(0.005, 2)
        assert e.value.code == ljmd.LJ_EDEVICE


def test_invalid_box_rejected():
    with _system(ljmd.LJ_MIXED, cutoff=2.5, margin=0.5) as s:
        with pytest.raises(ljmd.LjmdError) as e:
            s.set_state(np.zeros((4, 3)), None, 6.9)  # < 2 (r_s + margin) = 7
        assert e.value.code == ljmd.LJ_EINVAL


# ------------------------------------------------------------------------------------ list validity rules

@pytest.mark.parametrize("mode", [ljmd.LJ_VALID_HALF_MARGIN, ljmd.LJ_VALID_DUTC, ljmd.LJ_VALID_DUTC_LDC,
                                  ljmd.LJ_VALID_HALF_MARGIN_LDC])
def test_validity_rules_never_miss_a_pair(mode):
    """Under every rule (Sec. 2.3, Alg. 2), after every step each pair within r_c is listed."""
    x, v, L = thermal(6, 0.6, 1.5, 6)
    rc, margin = 2.5, 0.3
    with _system(ljmd.LJ_MIXED, cutoff=rc, margin=margin) as s:
        s.set_validity(mode, 256)
        s.set_state(x, v, L)
        for _ in range(60):
            s.step(0.005, 1)
            gx, _, _, _ = s.get_state()
            listed = _pairs_set(s.pairs())
            assert _pairs_set(_brute_pairs_numpy(gx, L, rc)) <= listed
        st = s.stats()
    assert st["validity"] == mode and st["status_word"] == 0 and st["rebuilds"] >= 2


@pytest.mark.parametrize("precision", [ljmd.LJ_FP64, ljmd.LJ_MIXED])
def test_margin_rule_at_its_limit(precision):
    """Two particles, just outside r_s, approach each other by margin/2 + 1.9e-9 each in one step, so
    that they end inside r_c.  (margin/2)^2 = 0.04 has an FP32 neighbour below it that a
    displacement this close to the limit would round to; the measured maximum must not undershoot
    (Sec. 2.3: a rebuild once any particle moved more than margin/2), so the pair is listed after
    the step."""
    rc, margin, L = 2.5, 0.4, 16.0
    rs = rc + margin
    delta = 128 * 2.0 ** -36                   # 1.86e-9
    x = np.array([[4.0, 8.0, 8.0], [4.0 + rs + 2.0 ** -30, 8.0, 8.0]])
    dt = 0.5
    u = (0.5 * margin + delta) / dt
    v = np.array([[u, 0.0, 0.0], [-u, 0.0, 0.0]])
    with _system(precision, ljmd.LJ_LIST_FULL, cutoff=rc, margin=margin) as s:
        s.set_state(x, v, L)
        s.build_pairlist()
        assert len(s.pairs()) == 0             # r_s + 2^-30 apart: not listed
        s.step(dt, 1)
        gx, _, _, _ = s.get_state()
        r = np.linalg.norm(gx[1] - gx[0])
        assert r < rc                          # now interacting
        assert _pairs_set(s.pairs()) == {(0, 1)}
        assert s.stats()["rebuilds"] == 2


def test_ldc_extends_list_lifetime_with_same_trajectory():
    """The large displacement check keeps lists the margin/2 rule would drop (fewer rebuilds, Alg. 2)
    and the trajectory is the same to FP32 summation order; DUTC alone rebuilds at least as often
    as the displacement rule."""
    x, v, L = thermal(8, 0.5, 1.0, 12)
    out = {}
    for mode in (ljmd.LJ_VALID_HALF_MARGIN, ljmd.LJ_VALID_HALF_MARGIN_LDC, ljmd.LJ_VALID_DUTC, ljmd.LJ_VALID_DUTC_LDC):
        with _system(ljmd.LJ_MIXED, cutoff=2.5, margin=0.5) as s:
            s.set_validity(mode, 4096)
            s.set_state(x, v, L)
            s.step(0.005, 150)
            gx, _, _, img = s.get_state()
            out[mode] = (s.stats(), gx + img * L)
    base = out[ljmd.LJ_VALID_HALF_MARGIN]
    ldc = out[ljmd.LJ_VALID_HALF_MARGIN_LDC]
    assert ldc[0]["rebuilds"] < base[0]["rebuilds"] and ldc[0]["ldc_kept"] > 0
    assert np.abs(ldc[1] - base[1]).max() < 1e-4
    assert out[ljmd.LJ_VALID_DUTC][0]["rebuilds"] >= base[0]["rebuilds"]
    assert out[ljmd.LJ_VALID_DUTC_LDC][0]["rebuilds"] <= out[ljmd.LJ_VALID_DUTC][0]["rebuilds"]


@pytest.mark.parametrize("list_form", [ljmd.LJ_LIST_FULL, ljmd.LJ_LIST_HALF])
@pytest.mark.parametrize("precision", [ljmd.LJ_MIXED, ljmd.LJ_FP64])
def test_pair_list_clustered(list_form, precision):
    """A dense blob over a dilute background: cells far above the mean occupancy take the list
    kernel's fallback path (too many work units for the unit tables); the list stays bit-exact."""
    L = 21.0
    rng = synth.rng(41)
    blob = 10.0 + 1.5 * rng.standard_normal((1200, 3))
    back = synth.uniform_positions(1500, L, 42)
    x = synth.dyadic(np.vstack([blob, back]) % L)
    with _system(precision, list_form, cutoff=2.5, margin=0.5) as s:
        s.set_state(x, None, L)
        s.build_pairlist()
        got = s.pairs()
    assert np.array_equal(got, O.pairs_within(x, L, 3.0))
