"""HRP: hierarchical recursive precision Cholesky for GB300 (sm_103a).

The product is the C-ABI library ``libhrp.so`` (include/hrp.h) built from csrc/;
``hrp`` is its thin Python binding.  Build with ``build.build()``.
"""
from . import hrp  # noqa: F401
from .hrp import (STATUS, Handle, HrpError, Tree, autotune_candidates, colmajor, from_colmajor, load,  # noqa: F401
                  mlp_param_count, policy_tree, tree_format, tree_parse)
