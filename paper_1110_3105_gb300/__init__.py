"""GB300 recursive-skeletonization fast direct solver (Ho & Greengard, 1110.3105).

The compute path is librs.so (CUDA, sm_103a) behind the C ABI of
include/rs.h; this package only binds it (``_lib``) and builds it
(``build``).  Importing the package does not load the library; the first
call of any binding does, and raises if the library is missing.
"""
from ._lib import (RS_HELMHOLTZ2D, RS_LAPLACE2D, RS_LAPLACE3D, RS_PREC_FP32,  # noqa: F401
                   RS_PREC_FP64, Handle, RSError, Server, load, rs_box_ranks, rs_build, rs_free, rs_gmres_patches,
                   rs_green, rs_launch_count, rs_matvec, rs_profile_enable, rs_profile_read, rs_profile_records,
                   rs_path_counts, rs_probe_fma_peak, rs_profile_tiles, rs_set_fault, rs_set_path, rs_solve, rs_solve_noalloc, rs_solve_refined, rs_tc_selftest,
                   rs_tree_level, rs_tree_perm, rs_version)
