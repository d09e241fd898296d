"""GB300-native (sm_103a) kernel-SVM trainer: SMO with adaptive shrinking and
gradient reconstruction (arXiv:1406.5161) behind a small C ABI.

The compute path is the CUDA library ``libsvmgb.so`` (sources in ``csrc/``,
ABI in ``include/svm_gb300.h``); this package only builds and binds it.
``synth`` draws the seeded synthetic workloads.
"""
from ._abi import (  # noqa: F401
    SVM_OK, SVM_NOT_CONVERGED, SVM_PENDING, SVM_ERR_ARG, SVM_ERR_OOM, SVM_ERR_BUDGET,
    SVM_ERR_TIMEOUT, SVM_ERR_CUDA, SVM_ERR_CANCELLED, SVM_ERR_UNSUPPORTED,
    SVM_FP64, SVM_MIXED_BF16, SVM_MIXED_BF16_SIMT, SVM_SHRINK_NONE, SVM_SHRINK_FIXED, SVM_SHRINK_FRACTION,
    SVM_RECON_SINGLE, SVM_RECON_MULTI, SVM_FLAG_STREAM_ROWS, SVM_FLAG_PHASE_TIMES, SVM_FLAG_NO_CLUSTERS, SVM_FLAG_CSR_ROWS, SVM_FLAG_WSS2, SVM_FLAG_NO_RELAYOUT, SVM_FLAG_CUDA_CORE_ROWS, SVM_FLAG_TENSOR_ROWS, SVM_FLAG_FULL_RECON, SVM_KERNEL_RBF, SVM_KERNEL_LINEAR, SVM_KERNEL_POLY, SVM_KERNEL_SIGMOID, SvmError, DeviceCSR, to_device, load, lib_path,
    svm_train, svm_decision, svm_last_error, svm_version, svm_kernel_launches, svm_diag_wait_timeout, svm_diag_sfu_rate,
    svm_train_fixed_workspace, svm_train_batch, svm_batch_autotune, Server, Model,
)

# Table 3 of the paper as (kind, value, reconstruction) shrink policies.
POLICIES = {
    "Original": None,
    "Single2": (SVM_SHRINK_FIXED, 2, SVM_RECON_SINGLE),
    "Single500": (SVM_SHRINK_FIXED, 500, SVM_RECON_SINGLE),
    "Single1000": (SVM_SHRINK_FIXED, 1000, SVM_RECON_SINGLE),
    "Single5pc": (SVM_SHRINK_FRACTION, 0.05, SVM_RECON_SINGLE),
    "Single10pc": (SVM_SHRINK_FRACTION, 0.10, SVM_RECON_SINGLE),
    "Single50pc": (SVM_SHRINK_FRACTION, 0.50, SVM_RECON_SINGLE),
    "Multi2": (SVM_SHRINK_FIXED, 2, SVM_RECON_MULTI),
    "Multi500": (SVM_SHRINK_FIXED, 500, SVM_RECON_MULTI),
    "Multi1000": (SVM_SHRINK_FIXED, 1000, SVM_RECON_MULTI),
    "Multi5pc": (SVM_SHRINK_FRACTION, 0.05, SVM_RECON_MULTI),
    "Multi10pc": (SVM_SHRINK_FRACTION, 0.10, SVM_RECON_MULTI),
    "Multi50pc": (SVM_SHRINK_FRACTION, 0.50, SVM_RECON_MULTI),
}
# the paper's heuristic classes: aggressive (star), average (diamond), conservative (bullet)
AGGRESSIVE, AVERAGE, LAZY = POLICIES["Multi5pc"], POLICIES["Multi10pc"], POLICIES["Multi50pc"]
