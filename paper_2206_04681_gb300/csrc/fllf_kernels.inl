// fllf_kernels.inl -- per-stage __global__ kernels for one storage type
// FLLF_STORAGE; included by one translation unit per precision.
#include "fllf_launch.h"

namespace fllf {

template <typename S>
__global__ void __launch_bounds__(kThreads) k_up0(const Up0Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  up0_tile<S>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_up(const UpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  up_tile<S>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_down(const DownArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  down_tile<S>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_down0(const Down0Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  down0_tile<S>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

static inline unsigned cdiv(int a, int b) { return (unsigned)((a + b - 1) / b); }

cudaError_t FLLF_LAUNCH_NAME(up0)(const Up0Args& a, int planes, cudaStream_t s) {
  dim3 grid(cdiv(a.dst.w, kUpTW), cdiv(a.dst.h, kUpTH), planes);
  k_up0<FLLF_STORAGE><<<grid, kThreads, kUpSmemBytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(up)(const UpArgs& a, int planes, cudaStream_t s) {
  dim3 grid(cdiv(a.dst.w, kUpTW), cdiv(a.dst.h, kUpTH), planes);
  k_up<FLLF_STORAGE><<<grid, kThreads, kUpSmemBytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(down)(const DownArgs& a, int planes, cudaStream_t s) {
  dim3 grid(cdiv(a.fine.w, kDnOW), cdiv(a.fine.h, kDnOH), planes);
  k_down<FLLF_STORAGE><<<grid, kThreads, kDnSmemBytes, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(down0)(const Down0Args& a, int planes, cudaStream_t s) {
  dim3 grid(cdiv(a.w0, kDnOW), cdiv(a.h0, kDnOH), planes);
  k_down0<FLLF_STORAGE><<<grid, kThreads, kDnSmemBytes, s>>>(a);
  return cudaGetLastError();
}

}  // namespace fllf
