"""GB300-native normal variate generators after Brent, "Fast Normal Random
Number Generators for Vector Processors" (TR-CS-93-04, 1993): Box-Muller
Algorithm B1 and Polar Algorithm P (Sec. 2), Methods B2 and B3 (Sec. 3),
Method P2 (Sec. 4) and the Ratio method R (Sec. 5), on Philox4x32-10
uniforms, as hand-written sm_103a CUDA kernels behind the C ABI of
include/nrng.h.  The binding functions carry the C entry points' names."""
from ._lib import NrngError, load  # noqa: F401
from .nrng import (  # noqa: F401
    ACCURATE, B1, B2, FAST, POINTS_B3, POINTS_P2, POINTS_RATIO, POLAR, STREAM_DESC, BatchedGraph, Reparam,
    broadcast_layout, descriptors_to_device,
    nrng_batched, nrng_batched_autotune, nrng_batched_config_count, nrng_batched_config_info,
    nrng_batched_get_config, nrng_batched_set_config, nrng_batched_workspace_size, nrng_boxmuller,
    nrng_boxmuller_b3, nrng_eval_points, nrng_get_status, nrng_polar, nrng_polar_max_blocks, nrng_polar_noalloc, nrng_polar_p2,
    nrng_polar_twopass, nrng_polar_twopass_workspace_size, nrng_polar_workspace_size, nrng_ratio,
    nrng_ratio_workspace_size, nrng_reparam_bwd, nrng_reparam_fwd, nrng_uniform, nrng_philox_ceiling, polar_workspace,
    raise_on_status, ratio_workspace, stream_descriptors,
)
