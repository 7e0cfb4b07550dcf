// fllf_noalloc.cu -- Fourier LLF with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool
// or allocator it does not own (an allocator callback, a host that forbids
// allocation after start-up), real-time loops where an allocation could block
// or fragment memory, or plugin hosts that hand out only the input and output
// buffers.  fllf_run_noalloc serves them: it runs the same kernels as
// fllf_run, but the pyramids live in one file-scope device array that the
// library image carries, so the call itself never allocates device memory.
//
// Rules a caller must know (also stated in include/fllf.h):
//   * The array is FLLF_NOALLOC_SCRATCH_BYTES (32 MiB) per GPU, held by every
//     GPU that loads the library until the process exits.  A parameter set
//     whose scratch (coefficients + guide, Fourier and residual pyramids)
//     does not fit is rejected with FLLF_EINVAL before any work is queued.
//   * All calls on one GPU share the array and it keeps the last call's
//     contents.  Calls whose GPU work overlaps (two streams, two host
//     threads) race on it; serialise them on one stream.  The pyramids need
//     no clearing (every word a kernel reads was written earlier in the same
//     call); the status words are cleared at the start of every call, by the
//     same small kernel that writes the coefficients.
//   * The coefficients travel to that kernel as a by-value argument, so the
//     call reads no host memory after it returns.
//   * The first call on a device resolves the array's device address with
//     cudaGetSymbolAddress (with that device current), which may load the
//     module; make that first call before any stream capture.  The address
//     is kept for the life of the process: do not use this entry point
//     across a cudaDeviceReset.
//   * A bounded wait that gives up inside the kernels (a TMA copy that never
//     lands, about 2 s) is not reported by this call: it has returned long
//     before.  The output is then incomplete.
#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FLLF_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

constexpr size_t kHeadBytes = 512;  // a_1..a_64 (float32) at 0, the 256-byte status block at 256, then the pyramids
constexpr int kMaxOrders = 64;

fllf_status noalloc_fail(fllf_status s, const std::string& why) {
  fllf::set_last_error(why);
  return s;
}

// The coefficients of one call, passed by value.
struct Coeffs {
  float a[kMaxOrders];
};

// Writes a_1..a_K into the head of the array and clears its status block
// (fault word, grid-barrier words, wait-limit words): one block of 64 threads.
__global__ void k_noalloc_setup(float* a_dst, Coeffs c, int K, unsigned* status) {
  const int t = threadIdx.x;
  if (t < K) a_dst[t] = c.a[t];
  status[t] = 0u;   // 64 words = 256 bytes
}

}  // namespace

extern "C" fllf_status fllf_run_noalloc(const fllf_params* user, const float* d_in, float* d_out,
                                        void* stream) {
  fllf_status st = fllf::validate(user);
  if (st != FLLF_OK) return st;
  const fllf_params np = fllf::normalized(*user);
  const fllf_params* p = &np;
  if (!d_in || !d_out) return noalloc_fail(FLLF_EINVAL, "input or output pointer is NULL");
  const size_t n = sizeof(float) * (size_t)p->H * p->W * p->C;
  const char *a = reinterpret_cast<const char*>(d_in), *b = reinterpret_cast<const char*>(d_out);
  if (a < b + n && b < a + n) return noalloc_fail(FLLF_EINVAL, "input and output buffers overlap");

  std::vector<fllf::Level> lv;
  const size_t need = fllf::layout(*p, &lv);
  if (need + kHeadBytes > (size_t)FLLF_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(FLLF_EINVAL,
                        "fllf_run_noalloc: this image needs " + std::to_string(need + kHeadBytes) +
                            " bytes of scratch, above the fixed " +
                            std::to_string((size_t)FLLF_NOALLOC_SCRATCH_BYTES) + "-byte array");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(FLLF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(FLLF_EINVAL, "device index out of range");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // Host code only holds a stand-in for the device array; ask the runtime
      // for its address on the current device.
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();   // leave no sticky error behind for later launch checks
        return noalloc_fail(FLLF_ECUDA, std::string("cudaGetSymbolAddress of the scratch array: ") +
                                            cudaGetErrorString(e));
      }
      g_noalloc_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_noalloc_ptr[dev];
  }

  // Coefficients in float64 on the host, written as float32 into the head of
  // the array by a small kernel that takes them by value and also clears the
  // status block.
  double a64[kMaxOrders];
  Coeffs c{};
  for (int k = 0; k < p->K; ++k) a64[k] = 0.0;   // fast LLF: unused
  if (p->method == FLLF_METHOD_FOURIER) fllf::compute_coeffs(*p, a64);
  for (int k = 0; k < p->K; ++k) c.a[k] = (float)a64[k];
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* d_a = reinterpret_cast<float*>(base);
  unsigned* fault = reinterpret_cast<unsigned*>(base + 256);
  k_noalloc_setup<<<1, 64, 0, s>>>(d_a, c, p->K, fault);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return noalloc_fail(FLLF_ECUDA, std::string("coefficient set-up kernel: ") + cudaGetErrorString(e));

  unsigned char* pyr = base + kHeadBytes;
  const int L = p->levels;
  for (int l = 0; l < L; ++l) {
    fllf::Level& v = lv[l];
    if (l == 0) {
      v.G = nullptr;
      v.Z = nullptr;
      v.E = nullptr;
      continue;
    }
    v.G = reinterpret_cast<float*>(pyr + reinterpret_cast<size_t>(v.G));
    v.Z = pyr + reinterpret_cast<size_t>(v.Z);
    v.E = (l <= L - 2) ? reinterpret_cast<float*>(pyr + reinterpret_cast<size_t>(v.E)) : nullptr;
  }
  if (!fllf::check_layout(*p, lv, pyr, (size_t)FLLF_NOALLOC_SCRATCH_BYTES - kHeadBytes))
    return noalloc_fail(FLLF_EINVAL, "internal error: scratch layout outside the fixed array");
  fllf::PathMaps maps;
  if (L > 1 && !fllf::build_maps(*p, lv, &maps))
    return noalloc_fail(FLLF_ECUDA, "TMA tensor map encoding failed (cuTensorMapEncodeTiled)");

  e = fllf::enqueue_path(*p, lv, maps, d_a, fault, d_in, d_out, s);
  if (e != cudaSuccess) return noalloc_fail(FLLF_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return FLLF_OK;
}
