"""BQRRP (arXiv 2507.00976) for B300: sm_103a CUDA kernels behind a C ABI.

``binding`` marshals arguments to ``libbqrrp.so`` (built by ``build``);
``workloads`` generates the seeded synthetic inputs.  The CUDA library is only
loaded on first use, and loading fails loudly if it has not been built.
"""
from . import binding  # noqa: F401  (ctypes wrappers; the .so loads lazily)
from .binding import (  # noqa: F401
    bqrrp_factor, bqrrp_factor_host, bqrrp_workspace_query, bqrrp_workspace_query_host, bqrrp_sketch_operator,
    bqrrp_sketch_apply, bqrrp_qrcp_wide, bqrrp_col_perm, bqrrp_cholqr_panel, bqrrp_geqrf, bqrrp_dgemm,
    bqrrp_probe_fp64_peak, factor, colmajor_empty, to_colmajor, make_opts, last_error,
    BatchPlan, bqrrp_batch_autotune, factor_batched, Server,
)
