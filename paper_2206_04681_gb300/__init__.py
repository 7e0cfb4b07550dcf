"""GB300-native Fourier local Laplacian filtering (arXiv 2206.04681).

The filter runs in ``libfllf.so`` (hand-written sm_103a CUDA kernels behind
the C ABI of ``include/fllf.h``).  This package holds the ctypes binding
(``_lib``), the build step (``build``), the seeded synthetic inputs
(``synth``) and a torch marshalling helper; PyTorch only supplies device
memory and streams.
"""

from ._lib import (FllfError, fllf_params, make_params, make_fast_params, lib,
                   FLLF_METHOD_FOURIER, FLLF_METHOD_FAST, fllf_params_validate, fllf_coeffs,
                   fllf_optimal_period, fllf_run_adaptive, fllf_run_luma, fllf_tuning,
                   fllf_plan_get_tuning, fllf_plan_set_tuning, fllf_plan_autotune,
                   fllf_plan_set_timing_mask,
                   fllf_batch_get_ctas, fllf_batch_set_ctas, fllf_batch_autotune,
                   fllf_batch_get_mode, fllf_batch_set_mode,
                   fllf_plan_scratch_bytes, fllf_plan_create, fllf_plan_destroy,
                   fllf_plan_params, fllf_plan_coeffs, fllf_run, fllf_run_host, fllf_submit, fllf_submit_host,
                   fllf_poll, fllf_batch_create, fllf_batch_destroy, fllf_batch_run,
                   fllf_batch_check, fllf_batch_run_plans, fllf_plan_set_wait_test, fllf_dataflow_check, POLL_MAX_US,
                   fllf_run_noalloc, NOALLOC_SCRATCH_BYTES,
                   fllf_plan_enable_timing, fllf_plan_stage_times, STAGES,
                   fllf_server_stats, fllf_server_create, fllf_server_destroy, fllf_server_submit,
                   fllf_server_poll, fllf_server_stats_get, fllf_server_stats_reset,
                   FLLF_OK, FLLF_EINVAL, FLLF_ENOMEM, FLLF_ECUDA, FLLF_EAGAIN,
                   FLLF_ETIMEOUT, FLLF_EBUSY, FLLF_FP32, FLLF_FP16, FLLF_BF16,
                   FLLF_COEFF_QUADRATURE, FLLF_COEFF_CLOSED_FORM, PRECISIONS)


def run_tensor(plan, x, out, stream=None):
    """fllf_run on torch CUDA tensors (C, H, W) float32, contiguous; marshalling only."""
    import torch
    p = fllf_plan_params(plan)
    shape = (p.C, p.H, p.W)
    for t, name in ((x, "input"), (out, "output")):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
        if tuple(t.shape[-3:]) != shape and not (p.C == 1 and tuple(t.shape) == shape[1:]):
            raise ValueError(f"{name} shape {tuple(t.shape)} does not match the plan {shape}")
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    fllf_run(plan, x.data_ptr(), out.data_ptr(), s.cuda_stream)
    return out
