"""The allocation-free solve entry point, hrp_potrs_noalloc.

Some callers cannot allocate device memory where they solve (their memory belongs to
an application pool, or cudaMalloc's implicit synchronization is not acceptable in
their loop).  hrp_potrs_noalloc serves them from a fixed array inside the library.
This test calls it through the C ABI twice in a row and checks each result against the
handle-based hrp_potrs and against the CPU oracle's solve with the same factor, with the
tolerance of the other POTRS parity tests (1e-12 relative).  A second case uses an
order close to the array's limit (n = 8150: 128 row blocks, the last
inverse slot and the mailboxes beside it) and 20 right-hand sides (two sweeps of 16 and 4).
It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import dense
from synth import dominant_spd, rhs, seed_for

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,nrhs_pair", [(1000, (3, 17)), (8150, (20, 1))])
def test_noalloc_solve_matches_handle_solve_on_two_calls(n, nrhs_pair):
    import torch

    import paper_2601_08082_gb300 as hrp

    lib = hrp.load()
    h = hrp.Handle(0)
    A = dominant_spd(n, 1.0, seed_for(0, 4242), shift=1.0)
    L_t = hrp.colmajor(A).cuda()
    assert h.potrf(hrp.tree_parse("[F16,F32|F64@128]", leaf=128), L_t) == 0
    L = np.tril(hrp.from_colmajor(L_t))
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, nrhs in enumerate(nrhs_pair):
        B = rhs(n, nrhs, seed_for(0, 5000 + call))
        B_ref = hrp.colmajor(B).cuda()
        h.potrs(L_t, B_ref)
        B_na = hrp.colmajor(B).cuda()
        st = lib.hrp_potrs_noalloc(n, nrhs, ctypes.c_void_p(L_t.data_ptr()), L_t.shape[1],
                                   ctypes.c_void_p(B_na.data_ptr()), B_na.shape[1], stream)
        assert st == 0
        torch.cuda.synchronize()
        X_ref = hrp.from_colmajor(B_ref)
        X_na = hrp.from_colmajor(B_na)
        assert not np.any(np.isnan(X_na))
        assert np.max(np.abs(X_na - X_ref)) <= 1e-12 * np.max(np.abs(X_ref)), call
        X_cpu = dense.potrs(L, B)
        assert np.max(np.abs(X_na - X_cpu)) <= 1e-12 * np.max(np.abs(X_cpu)), call
    # sizes beyond the fixed scratch are rejected before any work is enqueued
    assert lib.hrp_potrs_noalloc(8193, 1, ctypes.c_void_p(L_t.data_ptr()), 8193,
                                 ctypes.c_void_p(L_t.data_ptr()), 8193, stream) == 1
    h.close()
