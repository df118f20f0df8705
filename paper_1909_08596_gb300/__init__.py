"""GB300-native embedded two-electron-integral transformation of periodic ab initio DMET
(Cui, Zhu & Chan, arXiv 1909.08596, section 2.1, Algorithm 1).

The computation lives in libdmetemb.so (C ABI: include/dmet_emb.h, CUDA kernels for
sm_103a under csrc/); `binding` exposes the same entry points to Python.
"""
from . import binding
from .binding import (DmetError, dmet_emb_autotune, dmet_emb_batch_mode, dmet_emb_split_parts, dmet_emb_destroy, dmet_emb_tile_widths, dmet_emb_eri, dmet_emb_eri_bytes, dmet_emb_eri_fftdf, dmet_emb_eri_noalloc, dmet_emb_graph,
                      dmet_emb_bath, dmet_emb_fock, dmet_emb_jk_df, dmet_emb_last_error, dmet_fftdf_plane_waves, dmet_emb_problem_ms,
                      dmet_emb_l_pairs, dmet_emb_launch_count, dmet_emb_plan, dmet_emb_profile, dmet_emb_profile_count,
                      dmet_emb_profile_read, dmet_emb_schedule, dmet_emb_status, dmet_emb_transform_3idx, dmet_emb_wait_limit,
                      make_desc)
