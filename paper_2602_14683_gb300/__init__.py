"""paper_2602_14683_gb300 -- GB300 (sm_103a) kernels for unfolding-free beta-divergence
majorization-minimization of nonnegative CP and Tucker decompositions (arXiv 2602.14683).

The computation lives in libntf.so (C ABI declared in include/ntf.h); this package is its
thin Python binding.  Build the library with ``paper_2602_14683_gb300.build.build()``.
"""
from ._lib import (  # noqa: F401
    Context, Coo, NtfError, beta_div, coo_stable_perm, cp_beta_div_noalloc, cp_mu_sweep, cp_mu_sweep_extrap,
    cp_jcomm_outer_extrap, default_context, jcomm_outer, nesterov_weights,
    make_opts, plan_cut, raw_library, tucker_jcomm_outer_extrap, tucker_mu_sweep, tucker_mu_sweep_extrap, Batch, Server, LIB_PATH, EXPORTED,
)
