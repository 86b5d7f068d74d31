"""GB300-native U(1)-symmetric MPS two-site TEBD update (arXiv:2303.11409, Sec. II).

The hot path is the C-ABI CUDA library built from csrc/ (declared in
include/mps_gb300.h); this package is its ctypes binding plus host-side model
set-up.  Importing it fails if the library has not been built.
"""
from ._binding import (EXPORTED, LIB_PATH, MPS, MPS_BF16X3, MPS_EINVAL, MPS_ECHARGE, MPS_ENOCONV,  # noqa: F401
                       MPS_ENOMEM, MPS_ECUDA, MPS_ETIMEOUT, MPS_FP64, MPS_MAX_D, MPS_OK, MPS_TF32,
                       JacobiNotConverged, KERNEL_KINDS, MPSError, apply_gate2_batch, gate_length, launch_count, lib,
                       plan_sectors, plan_sectors_rule, gate_layout,
                       svd_sectors, svd_work_bytes)
from ._binding import MPS_NOALLOC_SCRATCH_BYTES, svd_sectors_noalloc  # noqa: F401
from ._binding import Executor, footprint_bytes, fp64_peak_probe, zgemm_tc  # noqa: F401
from ._binding import tc_inject_stall, svd_mixed_min_k, svd_mixed_sweeps, svd_cluster_min_k  # noqa: F401
from ._binding import (autotune_clear, autotune_force, autotune_freeze, autotune_min_flops,  # noqa: F401
                       autotune_stats, autotune_table)
from . import models, tebd, serve  # noqa: F401
