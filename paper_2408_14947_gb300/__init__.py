"""GB300 (sm_103a) CUDA implementation of the ERX per-line step.

ERX (Garske et al., Sec. III) scores each pixel of an incoming hyperspectral
line by its Mahalanobis distance to an exponentially moving background mean
and covariance.  All arithmetic runs in the CUDA library ``liberx.so`` behind
the C ABI of ``include/erx.h``; this package only marshals arguments to it.
"""
from .erx import (  # noqa: F401
    ERX_OK, ERX_EINVAL, ERX_ENOMEM, ERX_ECUDA, ERX_ENOTPD, ERX_ERANGE, ERX_ESTATE,
    ERX_EUNSUPPORTED, ERX_ETIMEOUT, ERX_FLAG_SIMT_STATS, ERX_PROJ_NONE, ERX_PROJ_SRP, ERX_UPDATE_THEN_SCORE, ERX_SCORE_THEN_UPDATE,
    ERX_U16, ERX_F32, ERX_F64, ERX_FORM_FP64, ERX_FORM_FP32, ERX_FORM_TF32, ERX_FORM_BF16,
    ErxConfig, ErxError, load_library, lib_path,
    erx_config_default, erx_create, erx_push_lines, erx_push_lines_host, erx_sync, erx_reset,
    erx_get_state, erx_set_state, erx_dim, erx_get_projection, erx_srp_weights, erx_destroy,
    erx_status_str, Detector, erx_profile_enable, erx_profile_read, erx_kernel_name,
    ERX_K_COUNT, erx_push_lines_static, Batch, Encoder, erx_train_opts_default,
    ERX_PROJ_LEARNED, ERX_FORM_TF32X3, ERX_FLAG_PIPELINE, ERX_AVG_EMA, ERX_AVG_IMC,
    ERX_AVG_POOLED, ERX_EIO, roc_metrics, selftest_bounded_wait,
)
