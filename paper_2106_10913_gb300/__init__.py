"""GB300 (sm_103a) AWG preconditioned conjugate gradient (arXiv 2106.10913).

The solver is the C-ABI library ``lib/libawg.so`` (declared in
``include/awg.h``); this package is its Python binding.
"""

from .awg import (  # noqa: F401
    AWGError, AWGSolver, EXPORTED, FP64, MIXED_BF16, MIXED_FP16, MIXED_FP32, H3_AD, H3_HYB, H3_INEX, LIB_PATH,
    H2_NN_HYB, H2_ASP_HYB, H2_ASP_AD, H2_AS_HYB,
    STAGE, awg_apply, awg_apply_stage, awg_destroy, awg_get_array, awg_get_info, awg_pcg,
    awg_profile, awg_profile_read, awg_profile_trace, awg_setup, default_options, load_library, PROF_NAMES, PROF_SERIAL, PROF_COUNT,
    awg_apply_hnn_noalloc, awg_learned_data, awg_learned_forward, awg_learned_grad,
    awg_learned_train, awg_apply_block, awg_coarse_apply_block, awg_pcg_block, awg_pcg_block_async, awg_save, awg_load,
    LEARNED_NPARAM, LEARNED_NFEAT, GENEO_DENSE, GENEO_BLOCK, GENEO_LEARNED,
)
