"""GPU checks of the cut-off autotuner (hrp_autotune): the tree it returns is one of its
candidates, keeps the given precisions, factors as accurately as the given tree on an
independent matrix, is not slower than the given tree, and is cached in the handle."""
import time

import numpy as np
import pytest

from synth import dominant_spd, seed_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrp_mod():
    import torch
    import paper_2601_08082_gb300 as hrp
    assert torch.cuda.is_available()
    return hrp


@pytest.fixture(scope="module")
def handle(hrp_mod):
    h = hrp_mod.Handle(0)
    yield h
    h.close()


def _median_ms(hrp, h, tree, A0, reps=5):
    import torch
    ts = []
    for _ in range(reps + 1):
        A = A0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = h.potrf(tree, A)
        e1.record()
        torch.cuda.synchronize()
        assert info == 0
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts[1:])), A


@pytest.mark.parametrize("spec,n", [("[F16,F32|F64@128]", 2048), ("[F64]", 1024)])
def test_autotune_choice(hrp_mod, handle, spec, n):
    t = hrp_mod.tree_parse(spec, leaf=128)
    best, ms = handle.autotune(t, n, reps=3, retune=True)
    assert ms > 0
    cands = hrp_mod.autotune_candidates(t)
    assert any((c.leaf, c.trsm_leaf, c.tile_occupancy) == (best.leaf, best.trsm_leaf, best.tile_occupancy)
               for c in cands)
    assert hrp_mod.tree_format(best) == hrp_mod.tree_format(t)

    # cached: the same key returns the same choice without running anything
    t0 = time.perf_counter()
    best2, ms2 = handle.autotune(t, n, reps=3)
    assert time.perf_counter() - t0 < 0.05
    assert (best2.leaf, best2.trsm_leaf, best2.tile_occupancy, ms2) == (best.leaf, best.trsm_leaf,
                                                                         best.tile_occupancy, ms)

    # an independent matrix of another family: as accurate (backward error within the
    # tuner's own 4x acceptance rule) and not slower (10% for timing noise)
    A0 = hrp_mod.colmajor(dominant_spd(n, 2.0, seed_for(0, 78))).cuda()
    ms_given, L_given = _median_ms(hrp_mod, handle, t, A0)
    ms_best, L_best = _median_ms(hrp_mod, handle, best, A0)
    be_given = handle.backward_error(A0, L_given)
    be_best = handle.backward_error(A0, L_best)
    assert be_best <= 4 * be_given + 1e-15
    assert ms_best <= 1.10 * ms_given + 0.05


def test_autotune_of_an_f8_tree_returns_it(hrp_mod, handle):
    t = hrp_mod.tree_parse("[F8,F16,F32|F64@128]", leaf=128)
    best, ms = handle.autotune(t, 1024, reps=1)
    assert (best.leaf, best.trsm_leaf or best.leaf) == (128, 128) and ms > 0


def test_batched_systems_take_the_cut_offs_tuned_for_their_order(hrp_mod, handle):
    """hrp_autotune_orders tunes a few orders; a batched system of order n then runs with the
    cut-offs and tile rule tuned at the largest tuned order <= n: bitwise the factor of a
    single hrp_potrf with that tuned tree."""
    import torch
    h = hrp_mod.Handle(0)
    try:
        h.set_batched_mode(False)          # stream pool: the single factorization's kernels
        t = hrp_mod.tree_parse("[F16,F32|F64@128]", leaf=128)
        h.autotune_orders(t, [256, 1024], reps=1)
        tuned = {o: h.autotune(t, o, reps=1)[0] for o in (256, 1024)}
        sizes = [200, 300, 1100, 700]
        mats = [dominant_spd(n, 2.0, seed_for(0, 90 + i)) for i, n in enumerate(sizes)]
        As = [hrp_mod.colmajor(A).cuda() for A in mats]
        d_info = torch.zeros(len(sizes), dtype=torch.int32, device="cuda")
        h.potrf_batched(t, As, d_info)
        torch.cuda.synchronize()
        assert d_info.cpu().tolist() == [0] * len(sizes)
        for n, A, At in zip(sizes, mats, As):
            ref_tree = t if n < 256 else tuned[1024 if n >= 1024 else 256]
            single = hrp_mod.colmajor(A).cuda()
            assert h.potrf(ref_tree, single) == 0
            assert torch.equal(torch.tril(single.T), torch.tril(At.T)), n
    finally:
        h.close()
