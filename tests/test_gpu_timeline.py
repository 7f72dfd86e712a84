"""GPU test of hrp_get_timeline (timing mode's per-launch record).

For a lookahead factorization of order 2048 with leaf 128, the timeline must hold every launch
(as many rows as hrp_last_launch_count), classes in range, streams 0 (critical) or a side
stream, start <= end, and on the critical stream the 16 leaves in column order, none
overlapping the next launch on that stream.
"""
import numpy as np
import pytest

from synth import dominant_spd, seed_for

pytestmark = pytest.mark.gpu


def test_timeline_records_every_launch():
    import torch
    import paper_2601_08082_gb300 as hrp
    n = 2048
    A = hrp.colmajor(dominant_spd(n, 2.0, seed_for(0, 960))).cuda()
    h = hrp.Handle(0)
    try:
        tree = hrp.tree_parse("[F16,F16,F32|F64@128]", leaf=128)
        classes = h.timing(tree, A.clone())
        tl = h.timeline()
        assert len(tl) == h.launch_count() == sum(c["launches"] for c in classes.values())
        assert np.all((tl[:, 0] >= 0) & (tl[:, 0] <= 4))
        assert np.all(tl[:, 1] >= 0)
        assert np.all(tl[:, 2] <= tl[:, 3])
        crit = tl[tl[:, 1] == 0]
        leaves = crit[crit[:, 0] == 0]
        assert len(leaves) == n // 128
        assert np.all(np.diff(leaves[:, 2]) > 0)            # in enqueue order
        assert np.all(crit[1:, 2] >= crit[:-1, 3] - 1e-3)   # one stream: no overlap (event resolution)
    finally:
        h.close()
