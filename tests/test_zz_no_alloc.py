"""The allocation-free pair export (ljmd_get_pairs_static) against ljmd_get_pairs.

Collected last on purpose: it must give the same pairs when its static device scratch is used
for the first time in the process and after every other test has run.
"""
import os
import re

import numpy as np
import pytest

from paper_1012_2677_gb300 import ljmd, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FORMS = [(ljmd.LJ_MIXED, ljmd.LJ_LIST_FULL), (ljmd.LJ_MIXED, ljmd.LJ_LIST_HALF),
         (ljmd.LJ_FP64, ljmd.LJ_LIST_FULL), (ljmd.LJ_FP64, ljmd.LJ_LIST_HALF)]


def _system(precision, list_form, cutoff=2.5, margin=0.5):
    return ljmd.System(cutoff=cutoff, margin=margin, precision=precision, list_form=list_form)


def _two_calls_match(s):
    ref = s.pairs()
    for _ in range(2):
        got, n = s.pairs_static()
        assert n == len(ref)
        assert np.array_equal(got, ref)
    return ref


def test_static_export_body_has_no_allocation():
    """The entry point and its kernels' file call no allocating function."""
    src = open(os.path.join(ROOT, "paper_1012_2677_gb300", "csrc", "ljmd_api.cu")).read()
    body = src[src.index("int ljmd_get_pairs_static("):]
    body = body[:body.index("\n}\n")]
    kern = open(os.path.join(ROOT, "paper_1012_2677_gb300", "csrc", "kernels_pairs_static.cu")).read()
    for text in (body, kern):
        assert not re.search(r"cudaMalloc|cudaFree|dalloc|std::vector|\bnew\b|malloc\(", text)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,list_form", FORMS)
@pytest.mark.parametrize("N,L,seed", [(900, 17.3, 2), (300, 7.2, 3), (1500, 12.0, 4)])
def test_static_export_matches_get_pairs(precision, list_form, N, L, seed):
    x = synth.dyadic(synth.uniform_positions(N, L, seed))
    with _system(precision, list_form, margin=0.3) as s:
        s.set_state(x, None, L)
        s.build_pairlist()
        ref = _two_calls_match(s)
        assert len(ref) > 0


@pytest.mark.gpu
@pytest.mark.parametrize("list_form", [ljmd.LJ_LIST_FULL, ljmd.LJ_LIST_HALF])
def test_static_export_during_a_run(list_form):
    """Lists rebuilt by the integrator (particles re-sorted) export the same way."""
    with _system(ljmd.LJ_MIXED, list_form, margin=0.3) as s:
        s.init_lattice(6, 0.6, 1.5, 11)
        s.step(0.005, 1)
        first = _two_calls_match(s)
        r0 = s.stats()["rebuilds"]
        s.step(0.005, 60)
        assert s.stats()["rebuilds"] > r0
        later = _two_calls_match(s)
        assert not np.array_equal(first, later)


@pytest.mark.gpu
def test_static_export_prefix_and_handles():
    """cap < npairs returns the first cap pairs of the sorted list; two handles share the
    scratch one call after the other."""
    xa = synth.dyadic(synth.uniform_positions(800, 13.0, 21))
    xb = synth.dyadic(synth.uniform_positions(600, 11.0, 22))
    with _system(ljmd.LJ_MIXED, ljmd.LJ_LIST_FULL) as a, _system(ljmd.LJ_FP64, ljmd.LJ_LIST_HALF) as b:
        a.set_state(xa, None, 13.0)
        b.set_state(xb, None, 11.0)
        a.build_pairlist()
        b.build_pairlist()
        ra, rb = a.pairs(), b.pairs()
        for _ in range(2):
            ga, na = a.pairs_static()
            gb, nb = b.pairs_static()
            assert np.array_equal(ga, ra) and np.array_equal(gb, rb)
        head, n = a.pairs_static(cap=17)
        assert n == len(ra) and np.array_equal(head, ra[:17])
        none, n = a.pairs_static(cap=0)
        assert n == len(ra) and len(none) == 0


@pytest.mark.gpu
def test_static_export_empty_and_errors():
    with _system(ljmd.LJ_MIXED, ljmd.LJ_LIST_FULL) as s:
        s.set_state(np.array([[1.0, 2.0, 3.0]]), None, 9.0)
        with pytest.raises(ljmd.LjmdError) as e:
            s.pairs_static()  # no list yet: constructing one could allocate
        assert e.value.code == ljmd.LJ_ESTATE
        s.build_pairlist()
        got, n = s.pairs_static()
        assert n == 0 and len(got) == 0 and len(s.pairs()) == 0
    # 16384 particles at rho = 0.5 with r_s = 3: about 9e5 full-list entries, beyond 2^19
    with _system(ljmd.LJ_MIXED, ljmd.LJ_LIST_FULL) as s:
        s.init_lattice(16, 0.5, 1.0, 3)
        s.build_pairlist()
        assert s.stats()["list_entries"] > ljmd.LJ_PAIRS_STATIC_MAX_ENTRIES
        with pytest.raises(ljmd.LjmdError) as e:
            s.pairs_static(cap=1)
        assert e.value.code == ljmd.LJ_ERANGE
        assert len(s.pairs()) > 0  # the handle is still usable


@pytest.mark.gpu
def test_static_export_leaves_free_device_memory_unchanged():
    """After the first call (which resolves the scratch address), further calls change the free
    device memory by nothing: no allocation anywhere below the entry point, helpers included."""
    torch = pytest.importorskip("torch")
    x = synth.dyadic(synth.uniform_positions(1200, 14.0, 31))
    with _system(ljmd.LJ_MIXED, ljmd.LJ_LIST_FULL) as s:
        s.set_state(x, None, 14.0)
        s.build_pairlist()
        ref, _ = s.pairs_static()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(5):
            got, n = s.pairs_static()
            assert n == len(ref) and np.array_equal(got, ref)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
