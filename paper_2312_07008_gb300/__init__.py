"""GB300 (sm_103a) FNO SA-DSRG-PT2 hot path (arXiv:2312.07008).

The computation lives in libdsrg_fno.so (hand-written CUDA behind a C ABI,
include/dsrg_fno.h); this package is its thin ctypes binding.
"""
from .binding import (  # noqa: F401
    FP64, SLICED_BF16, BF16X3, TF32, MODE_PO, MODE_PV, MODE_NKAPPA, MODE_FIXED, DsrgFnoError, Problem, problem_from_synth,
    dsrg_fno_pt2_energy, dsrg_fno_pt2_energy_mr, dsrg_fno_vv_opdm, dsrg_fno_vv_opdm_lambda3, dsrg_fno_sa_lambda3, dsrg_fno_truncate,
    dsrg_fno_truncate_noalloc, dsrg_fno_cut, dsrg_fno_naf, dsrg_fno_ladder,
    dsrg_fno_discarded_correction, dsrg_fno_discarded_correction_mr, dsrg_fno_sa_densities, dsrg_fno_batch_run, dsrg_fno_batch_last_workers,
    dsrg_fno_release, dsrg_fno_profile_enable, dsrg_fno_profile_query, dsrg_fno_launch_count,
    dsrg_fno_debug_workspace_bytes, dsrg_fno_debug_eig_batch, dsrg_fno_set_log_callback, dsrg_fno_debug_pair_tiles,
    dsrg_fno_debug_set_barrier_limit, dsrg_fno_debug_set_fused_epilogue, dsrg_fno_debug_set_syrk_planes, dsrg_fno_debug_set_eig_colpair,
    load, LIB_PATH, EXPORTED,
)
