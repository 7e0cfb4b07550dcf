// Per-stage kernels with the Fourier pyramids stored as float.
#define FLLF_STORAGE float
#define FLLF_STORAGE_IS_F32 1
#define FLLF_LAUNCH_NAME(stage) launch_##stage##_f32
#include "fllf_kernels.inl"
