"""GB300 (sm_103a) mixed-precision LOBPCG (Kressner, Ma, Shao, arXiv 2302.12528).

Thin Python binding of the C ABI in ``include/mplobpcg.h`` and
``include/mplobpcg_steps.h``: every function here only marshals arguments
(pointers, sizes, the CUDA stream) and calls the library, whose CUDA kernels
do all of the work.  PyTorch supplies device memory and streams.

Import fails loudly when the CUDA library has not been built
(``python -c "import __graft_entry__ as g; g.build()"``).
"""
from .binding import (  # noqa: F401
    LIB_PATH, Batch, MPL_C128, MPL_D_DCHOL, MPL_D_SCHOL, MPL_MP_SCHOL, MPL_R64, POLICIES, MplError,
    Stats, Handle, analyze_host, create_csr, create_dense, eigsh_csr, fv_assemble, fv_assemble_adjoint,
    fv_values, lib, lowp_syrk, probe_fma_rate, residual_noalloc, split_gemm, start_block,
)
