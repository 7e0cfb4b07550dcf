// Per-stage kernels with the Fourier pyramids stored as __half.
#define FLLF_STORAGE __half
#define FLLF_LAUNCH_NAME(stage) launch_##stage##_f16
#include "fllf_kernels.inl"
