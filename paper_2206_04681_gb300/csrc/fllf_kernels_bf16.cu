// Per-stage kernels with the Fourier pyramids stored as __nv_bfloat16.
#define FLLF_STORAGE __nv_bfloat16
#define FLLF_LAUNCH_NAME(stage) launch_##stage##_bf16
#include "fllf_kernels.inl"
