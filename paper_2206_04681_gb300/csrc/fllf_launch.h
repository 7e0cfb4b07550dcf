// fllf_launch.h -- host-side launchers of the per-stage kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "fllf_device.cuh"

namespace fllf {

// One set of launchers per storage precision of the Fourier pyramids.  `cps`
// caps the persistent grid at that many resident CTAs per SM (0: as many as
// fit); launch_occupancy_<suffix>(kind, batched) reports how many fit.
#define FLLF_DECLARE_LAUNCHERS(suffix)                                                                   \
  cudaError_t launch_up0_##suffix(const Up0Args& a, cudaStream_t s, int cps);                            \
  cudaError_t launch_up_##suffix(const UpArgs& a, cudaStream_t s, int cps);                              \
  cudaError_t launch_down_##suffix(const DownArgs& a, cudaStream_t s, int cps);                          \
  cudaError_t launch_down_s_##suffix(const DownArgs& a, cudaStream_t s, int cps);                        \
  cudaError_t launch_down0_##suffix(const Down0Args& a, cudaStream_t s, int cps);                        \
  cudaError_t launch_down10_##suffix(const Down10Args& a, cudaStream_t s, int cps);                      \
  cudaError_t launch_chain_##suffix(const ChainArgs& a, cudaStream_t s, int cps);                        \
  cudaError_t launch_graph_##suffix(const GraphArgs& a, cudaStream_t s, int cps, int with_d10);          \
  cudaError_t launch_up0_batch_##suffix(const BatchTable<Up0Args>& t, cudaStream_t s, int cps);          \
  cudaError_t launch_up_batch_##suffix(const BatchTable<UpArgs>& t, cudaStream_t s, int cps);            \
  cudaError_t launch_down_batch_##suffix(const BatchTable<DownArgs>& t, cudaStream_t s, int cps);        \
  cudaError_t launch_down0_batch_##suffix(const BatchTable<Down0Args>& t, cudaStream_t s, int cps);      \
  cudaError_t launch_down10_batch_##suffix(const BatchTable<Down10Args>& t, cudaStream_t s, int cps);    \
  int launch_occupancy_##suffix(int kind, int batched);
// REDUCE of one float plane (the gain map of pixel-adaptive runs).
cudaError_t launch_map_reduce(const float* src, int sh, int sw, int spitch, float* dst, int dh, int dw,
                              int dpitch, cudaStream_t s);
// Luma of a planar RGB image (n pixels per plane), and the luma change added back.
cudaError_t launch_luma(const float* rgb, float* y, long long n, const float w[3], cudaStream_t s);
cudaError_t launch_luma_apply(const float* rgb, const float* y, const float* yf, float* out, long long n,
                              cudaStream_t s);
// Copies `rows` dense rows of W floats to a row pitch of `pitch` floats.
cudaError_t launch_pad_rows(const float* src, int W, long long rows, float* dst, int pitch, cudaStream_t s);
// The staging copies of a batch: n PadRow entries, prefix[n + 1] row sums.
cudaError_t launch_pad_batch(const PadRow* tab, const int* prefix, int n, int total, cudaStream_t s);
// Copies status[0] (the fault word) into a host-mapped word (one thread).
cudaError_t launch_status_snapshot(const unsigned* status, unsigned* host_word, cudaStream_t s);
FLLF_DECLARE_LAUNCHERS(f32)
FLLF_DECLARE_LAUNCHERS(f16)
FLLF_DECLARE_LAUNCHERS(bf16)
#undef FLLF_DECLARE_LAUNCHERS

}  // namespace fllf
