"""GB300-native probabilistic shape-from-silhouette (Section 2.2.2 of
"Digitize Your Body and Action in 3-D at Over 10 FPS").

The computation lives in libpsfs (hand-written CUDA for sm_103a behind the C
ABI of include/psfs.h); `psfs` is its ctypes binding with the same names, and
`autograd` wraps the adjoint in a torch.autograd.Function.
"""

from .psfs import (  # noqa: F401
    MAP_DTYPES,
    PSFS_ERR_CAPACITY,
    PSFS_ERR_CUDA,
    PSFS_ERR_INVALID_ARG,
    PSFS_ERR_NOMEM,
    PSFS_ERR_NOT_READY,
    PSFS_ERR_TIMEOUT,
    PSFS_MAP_BF16,
    PSFS_MAP_F16,
    PSFS_MAP_F32,
    PSFS_MAX_CAMS,
    PSFS_OK,
    PsfsError,
    Reconstructor,
    load,
    FUSE_CONFIGS,
    psfs_autotune,
    BATCH_CONFIGS,
    psfs_batch_autotune,
    psfs_batch_create,
    psfs_batch_destroy,
    psfs_batch_run,
    psfs_batch_set_config,
    psfs_batch_sync,
    psfs_backward,
    psfs_backward_slm,
    psfs_get_fuse_config,
    psfs_set_fuse_config,
    psfs_create,
    psfs_destroy,
    psfs_fuse_slm,
    psfs_get_likelihood,
    psfs_last_error_message,
    psfs_params_default,
    psfs_profile_enable,
    psfs_profile_read,
    psfs_reconstruct,
    psfs_reconstruct_host,
    psfs_reconstruct_noalloc,
    psfs_reconstruct_sequence,
    psfs_set_background,
    psfs_status_string,
    psfs_sync,
    voxel_list,
)
