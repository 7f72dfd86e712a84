"""HRP: hierarchical recursive precision Cholesky for GB300 (sm_103a).

The product is the C-ABI library ``libhrp.so`` (include/hrp.h) built from csrc/;
``hrp`` is its thin Python binding.  Build with ``build.build()``.
"""
from . import hrp  # noqa: F401
from .hrp import (Handle, HrpError, Tree, colmajor, from_colmajor, load, mlp_param_count,  # noqa: F401
                  policy_tree, tree_format, tree_parse)
