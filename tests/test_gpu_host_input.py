"""GPU tests of hrp_potrf_host: Alg. 1 on a matrix in host memory, the transfer of its lower
triangle overlapped with the factorization (each node waits only for the column blocks it
reads).

The overlap changes only when kernels may start, not what they compute, so the factor must be
bit for bit the one hrp_potrf_async computes from a device copy of the same matrix, for every
tree, order and mode (lookahead, dynamic scaling), also when a call follows another on the
same handle.  Entries above the 128 x 128 diagonal blocks are not transferred and must keep
what dA held.  A matrix that is not positive definite reports the same column.
"""
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


def _both(hrp, A, spec, leaf, scaling=False, lookahead=True, sentinel=7.0):
    import torch
    h = hrp.Handle(0)
    try:
        h.set_lookahead(lookahead)
        if scaling:
            h.set_scaling(True)
        tree = hrp.tree_parse(spec, leaf=leaf)
        n = A.shape[0]
        info = torch.zeros(2, dtype=torch.int32, device="cuda")
        Ad = hrp.colmajor(A).cuda()
        h.potrf_async(tree, Ad, info[0:1])
        hA = hrp.colmajor(A).pin_memory()
        Ah = torch.full_like(Ad, sentinel)
        for _ in range(2):                   # twice: the handle's copy events are reused
            Ah.fill_(sentinel)
            h.potrf_host(tree, hA, Ah, info[1:2])
        torch.cuda.synchronize()
        return hrp.from_colmajor(Ad), hrp.from_colmajor(Ah), [int(v) for v in info.cpu()]
    finally:
        h.close()


@pytest.mark.parametrize("n,spec,leaf", [
    (1, "[F64]", 64), (100, "[F64]", 64), (300, "[F16,F32|F64@64]", 64), (1000, "[F64]", 128),
    (1000, "[F16,F32|F64@128]", 128), (2048, "[F16,F16,F32|F64@128]", 128),
    (4096, "[F16,F16,F16,F32|F64@128]", 128), (2048, "[F8,F16,F32|F64@128]", 128),
])
def test_host_input_factor_is_the_device_factor(hrp_mod, n, spec, leaf):
    A = dominant_spd(n, 1.5, seed_for(0, 900 + n), shift=1.0)
    Ld, Lh, info = _both(hrp_mod, A, spec, leaf)
    assert info == [0, 0]
    il = np.tril_indices(n)
    assert np.array_equal(Lh[il], Ld[il])
    # above the diagonal blocks nothing was written
    i, j = np.triu_indices(n, 1)
    far = (i // 128) < (j // 128)
    assert np.all(Lh[i[far], j[far]] == 7.0)


def test_host_input_without_lookahead_and_with_scaling(hrp_mod):
    n = 1500
    A = dominant_spd(n, 1.5, seed_for(0, 950))
    for kw in ({"lookahead": False}, {"scaling": True}):
        Ld, Lh, info = _both(hrp_mod, A, "[F16,F32|F64@128]", 128, **kw)
        assert info == [0, 0]
        il = np.tril_indices(n)
        assert np.array_equal(Lh[il], Ld[il]), kw


def test_host_input_reports_failing_column(hrp_mod):
    n = 700
    A = dominant_spd(n, 2.0, seed_for(0, 951))
    A[400, 400] = -1.0
    _, _, info = _both(hrp_mod, A, "[F16,F32|F64@128]", 128)
    assert info[0] == info[1] == 401


def test_host_input_argument_errors(hrp_mod):
    import ctypes
    import torch
    hrp = hrp_mod
    h = hrp.Handle(0)
    lib = hrp.load()
    tree = hrp.tree_parse("[F64]", leaf=64)
    hA = torch.zeros((8, 8), dtype=torch.float64).pin_memory()
    dA = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    vp = ctypes.c_void_p
    s = vp(torch.cuda.current_stream().cuda_stream)
    assert lib.hrp_potrf_host(h._h, ctypes.byref(tree), -1, vp(hA.data_ptr()), 8, vp(dA.data_ptr()), 8,
                              vp(info.data_ptr()), s) == 1
    assert lib.hrp_last_arg(h._h) == -3
    assert lib.hrp_potrf_host(h._h, ctypes.byref(tree), 8, vp(hA.data_ptr()), 7, vp(dA.data_ptr()), 8,
                              vp(info.data_ptr()), s) == 1
    assert lib.hrp_last_arg(h._h) == -5
    assert lib.hrp_potrf_host(h._h, ctypes.byref(tree), 8, vp(0), 8, vp(dA.data_ptr()), 8,
                              vp(info.data_ptr()), s) == 1
    assert lib.hrp_last_arg(h._h) == -4
    h.close()


def test_host_input_with_padded_leading_dimensions(hrp_mod):
    # ldha and lda larger than n: the copies walk both pitches
    import torch
    hrp = hrp_mod
    n, ldh, ldd = 700, 731, 760
    A = dominant_spd(n, 1.5, seed_for(0, 952))
    h = hrp.Handle(0)
    try:
        tree = hrp.tree_parse("[F16,F32|F64@128]", leaf=128)
        info = torch.zeros(2, dtype=torch.int32, device="cuda")
        hA = torch.zeros((n, ldh), dtype=torch.float64)
        hA[:, :n] = hrp.colmajor(A)
        hA = hA.pin_memory()
        Ah = torch.full((n, ldd), 7.0, dtype=torch.float64, device="cuda")
        h.potrf_host(tree, hA, Ah, info[1:2], n=n)
        Ad = torch.zeros((n, ldd), dtype=torch.float64, device="cuda")
        Ad[:, :n] = hrp.colmajor(A).cuda()
        h.potrf_async(tree, Ad, info[0:1], n=n)
        torch.cuda.synchronize()
        assert [int(v) for v in info.cpu()] == [0, 0]
        Ld, Lh = hrp.from_colmajor(Ad)[:n, :n], hrp.from_colmajor(Ah)[:n, :n]
        il = np.tril_indices(n)
        assert np.array_equal(Lh[il], Ld[il])
        assert torch.all(Ah[:, n:] == 7.0)                 # padding rows of every column untouched
    finally:
        h.close()
