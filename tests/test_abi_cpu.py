"""Host-side checks of the C ABI that need no GPU: the library builds, loads and exports
every entry point include/hrp.h declares, and the tree descriptor parses the notation
of Sec. 4.2 the same way the oracle reads it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hrp.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hrp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2601_08082_gb300 import build as b, hrp
    if not os.path.exists(hrp.LIB_PATH):
        b.build()
    return hrp.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    from paper_2601_08082_gb300 import hrp
    assert sorted(hrp.EXPORTED) == names


@pytest.mark.parametrize("spec,levels,inner,size", [
    ("[F64]", [0], 0, 0),
    ("[F16,F16,F16,F16,F32|F64@128]", [2, 2, 2, 2, 1], 0, 128),
    ("[F8,F16,F16,F32|F64@128]", [3, 2, 2, 1], 0, 128),
    ("[F16, F32, F64]", [2, 1, 0], 0, 0),
])
def test_tree_parse_matches_oracle_reading(lib, spec, levels, inner, size):
    from paper_2601_08082_gb300 import hrp
    from oracle import tree as otree
    t = hrp.tree_parse(spec, leaf=128)
    assert list(t.level[: t.depth]) == levels
    assert t.inner_size == size
    o = otree.parse(spec)
    assert [hrp.PREC[p] for p in o.levels] == levels and o.inner_size == size
    assert hrp.tree_format(t).replace(" ", "") == spec.replace(" ", "")


@pytest.mark.parametrize("bad", ["F16", "[F12]", "[]", "[F16|F16@12]", "[F64|F64@]", "[F32]x"])
def test_tree_parse_rejects(lib, bad):
    from paper_2601_08082_gb300 import hrp
    t = hrp.Tree()
    assert lib.hrp_tree_parse(bad.encode(), 128, ctypes.byref(t)) == 1


def test_status_strings(lib):
    assert lib.hrp_status_string(0) == b"HRP_OK"
    assert lib.hrp_status_string(2) == b"HRP_ERR_NOT_SPD"
    assert lib.hrp_status_string(6) == b"HRP_ERR_TIMEOUT"


def test_null_handle_is_rejected_without_a_gpu(lib):
    from paper_2601_08082_gb300 import hrp
    t = hrp.tree_parse("[F64]", 64)
    assert lib.hrp_potrf(None, ctypes.byref(t), 4, None, 4, None, None) == 1
    assert lib.hrp_potrs(None, 4, 1, None, 4, None, 4, None) == 1


@pytest.mark.parametrize("spec,leaf,trsm_leaf", [
    ("[F16,F32|F64@128]", 128, 0), ("[F64]", 64, 0), ("[F32]", 100, 50), ("[F16,F16,F32]", 128, 64)])
def test_autotune_candidates_keep_the_precisions(lib, spec, leaf, trsm_leaf):
    # host-only enumeration: the given tree first, then valid cut-offs, no duplicates; the
    # precision list, inner region and TRSM arithmetic are those of the given tree
    from paper_2601_08082_gb300 import hrp
    t = hrp.tree_parse(spec, leaf=leaf, trsm_leaf=trsm_leaf)
    cands = hrp.autotune_candidates(t)
    assert (cands[0].leaf, cands[0].trsm_leaf) == (leaf, trsm_leaf)
    seen = set()
    for c in cands:
        tl = c.trsm_leaf or c.leaf
        assert 1 <= c.leaf <= 128 and 1 <= tl <= c.leaf
        assert (c.leaf, tl, c.tile_occupancy) not in seen
        seen.add((c.leaf, tl, c.tile_occupancy))
        assert hrp.tree_format(c) == hrp.tree_format(t)
        assert (c.depth, list(c.level)[:c.depth], c.inner, c.inner_size, c.trsm_compute) == \
            (t.depth, list(t.level)[:t.depth], t.inner, t.inner_size, t.trsm_compute)
    assert {(128, 128, 0), (64, 64, 0), (64, 32, 0)} <= seen
    occ = {o for _, _, o in seen}
    assert occ == ({0, 2, 4} if "F16" in spec else {0})     # tile rule only with tensor-core levels


def test_autotune_candidates_for_an_f8_tree_keep_its_cut_offs(lib):
    from paper_2601_08082_gb300 import hrp
    t = hrp.tree_parse("[F8,F16,F16,F32|F64@128]", leaf=128)
    cands = hrp.autotune_candidates(t)
    assert all(c.leaf == 128 and (c.trsm_leaf or 128) == 128 for c in cands)
    assert sorted(c.tile_occupancy for c in cands) == [0, 2, 4]      # only the tile rule varies


def test_autotune_rejects_bad_arguments_without_a_gpu(lib):
    from paper_2601_08082_gb300 import hrp
    t = hrp.tree_parse("[F64]", leaf=64)
    t.leaf = 0
    assert lib.hrp_autotune_candidates(ctypes.byref(t), None, 0) == -1
    assert lib.hrp_autotune(None, ctypes.byref(t), 64, 1, 0, ctypes.byref(hrp.Tree()), None, None) != 0


def _prototypes():
    """name -> number of parameters, from the prototypes in include/hrp.h."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for m in re.finditer(r"\b(hrp_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        args = m.group(2).strip()
        depth, n = 0, (0 if args in ("", "void") else 1)
        for ch in args:
            depth += ch == "("
            depth -= ch == ")"
            n += ch == "," and depth == 0
        out[m.group(1)] = n
    return out


def test_binding_declares_every_prototype_with_its_arity(lib):
    protos = _prototypes()
    assert set(protos) == set(_declared())
    for name, nargs in protos.items():
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None, f"{name}: no argtypes in the binding"
        assert len(argtypes) == nargs, (name, len(argtypes), nargs)
