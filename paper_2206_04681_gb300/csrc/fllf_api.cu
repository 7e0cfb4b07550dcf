// fllf_api.cu -- the C ABI of include/fllf.h: parameters, coefficients, plans,
// run / submit / poll.  Host code; the kernels live in fllf_kernels_*.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"
#include "fllf_launch.h"

namespace {

thread_local std::string g_last_error;

fllf_status fail(fllf_status s, const std::string& why) {
  g_last_error = why;
  return s;
}

fllf_status cuda_fail(cudaError_t e, const char* what) {
  return fail(FLLF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Keeps the caller's current device across a call that switches devices.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

namespace fllf {

void set_last_error(const std::string& s) { g_last_error = s; }

// ---- Fourier coefficients (Eqs. (9)-(11)) ------------------------------------------
// Gauss-Legendre nodes on [-1, 1]: roots of P_n by Newton's method from the
// asymptotic guesses cos(pi (i - 1/4) / (n + 1/2)); P_n and P_n' from the
// three-term recurrence (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1}.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 1; j < n; ++j) {
        const double p2 = ((2.0 * j + 1.0) * z * p1 - j * p0) / (j + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void compute_coeffs(const fllf_params& p, double* a) {
  const double pi = 3.14159265358979323846;
  const int K = p.K;
  const double s = p.sigma_r, T = p.T, g = p.m - 1.0;
  if (p.coeff_mode == FLLF_COEFF_CLOSED_FORM) {
    for (int k = 1; k <= K; ++k) {
      const double om = 2.0 * pi * k / T;
      const double alpha = s * std::sqrt(2.0 * pi) / T * std::exp(-0.5 * (om * s) * (om * s));
      a[k - 1] = g * 2.0 * s * s * alpha * om;
    }
    return;
  }
  // (2/T) * integral_{-T/2}^{T/2} f(x) sin(w_k x) dx; the integrand is even,
  // so integrate over [0, T/2] and double.  Composite 16-node Gauss-Legendre
  // on panels no wider than a quarter of sigma_r and of the period of the
  // highest order (at least 64 panels, at most 4096): each panel holds a
  // smooth, slowly varying piece of the integrand, where the rule is exact
  // to rounding.  At each node, sin(k w_1 x) for k = 1..K follows from
  // sin(w_1 x), cos(w_1 x) by the rotation (c, s) <- (c c1 - s s1, s c1 + c s1).
  const int nodes = 16;
  static const std::vector<double> gl = [] {
    std::vector<double> x, w;
    gauss_legendre(16, x, w);
    x.insert(x.end(), w.begin(), w.end());
    return x;
  }();
  const double* gx = gl.data();
  const double* gw = gl.data() + nodes;
  const double half = T / 2.0, scale = std::min(s, T / K) / 4.0;
  const int panels = (int)std::min(4096.0, std::max(64.0, std::ceil(half / scale)));
  for (int k = 0; k < K; ++k) a[k] = 0.0;
  const double h = half / panels, w1 = 2.0 * pi / T;
  for (int q = 0; q < panels; ++q) {
    const double mid = q * h + 0.5 * h;
    for (int i = 0; i < nodes; ++i) {
      const double x = mid + 0.5 * h * gx[i];
      const double wf = 0.5 * h * gw[i] * g * x * std::exp(-x * x / (2.0 * s * s));
      const double s1 = std::sin(w1 * x), c1 = std::cos(w1 * x);
      double sk = s1, ck = c1;
      for (int k = 0; k < K; ++k) {
        a[k] += wf * sk;
        const double sn = sk * c1 + ck * s1;
        ck = ck * c1 - sk * s1;
        sk = sn;
      }
    }
  }
  for (int k = 0; k < K; ++k) a[k] *= 2.0 * (2.0 / T);
}

fllf_status validate(const fllf_params* p) {
  if (!p) return fail(FLLF_EINVAL, "params is NULL");
  if (p->H < 1 || p->W < 1 || p->H > 65536 || p->W > 65536)
    return fail(FLLF_EINVAL, "H and W must be in [1, 65536]");
  if (p->C < 1 || p->C > 64) return fail(FLLF_EINVAL, "C must be in [1, 64]");
  if (p->levels < 1 || p->levels > 16) return fail(FLLF_EINVAL, "levels must be in [1, 16]");
  if (p->method != FLLF_METHOD_FOURIER && p->method != FLLF_METHOD_FAST)
    return fail(FLLF_EINVAL, "method must be FLLF_METHOD_FOURIER or FLLF_METHOD_FAST");
  const bool fast = p->method == FLLF_METHOD_FAST;
  if (fast && (p->samples < 2 || p->samples > 128)) return fail(FLLF_EINVAL, "samples must be in [2, 128]");
  if (!fast && (p->K < 1 || p->K > 64)) return fail(FLLF_EINVAL, "K must be in [1, 64]");
  if (!std::isfinite(p->m)) return fail(FLLF_EINVAL, "m must be finite");
  if (!(p->sigma_r > 0.0) || !std::isfinite(p->sigma_r))
    return fail(FLLF_EINVAL, "sigma_r must be finite and > 0");
  if (!fast && (!(p->T > 0.0) || !std::isfinite(p->T))) return fail(FLLF_EINVAL, "T must be finite and > 0");
  if (p->precision < FLLF_FP32 || p->precision > FLLF_BF16)
    return fail(FLLF_EINVAL, "precision must be FLLF_FP32, FLLF_FP16 or FLLF_BF16");
  if (!fast && p->coeff_mode != FLLF_COEFF_QUADRATURE && p->coeff_mode != FLLF_COEFF_CLOSED_FORM)
    return fail(FLLF_EINVAL, "coeff_mode must be quadrature or closed form");
  return FLLF_OK;
}

// A fast LLF plan holds its S sampled pyramids as ceil(S/2) complex planes:
// every pyramid, map and kernel sees K = ceil(S/2); T and coeff_mode are
// fixed to values that the Fourier-only code paths accept.
fllf_params normalized(const fllf_params& p) {
  fllf_params q = p;
  if (p.method == FLLF_METHOD_FAST) {
    q.K = (p.samples + 1) / 2;
    q.T = 2.0;
    q.coeff_mode = FLLF_COEFF_QUADRATURE;
  } else {
    q.samples = 0;
  }
  return q;
}

// Scratch layout: per level l = 1..levels-1, G_l, Z_l and (l <= levels-2) E_l
// for all planes, each buffer 256-byte aligned; row pitch rounded up to 16
// elements so that rows start on 64-byte (G, E) / 64-128-byte (Z) boundaries.
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t layout(const fllf_params& p, std::vector<Level>* out) {
  const size_t zsize = p.precision == FLLF_FP32 ? 8 : 4;
  size_t off = 0;
  int h = p.H, w = p.W;
  if (out) out->assign(p.levels, Level{});
  for (int l = 0; l < p.levels; ++l) {
    Level lv{};
    lv.h = h;
    lv.w = w;
    if (l > 0) {
      lv.pitch = (w + 15) & ~15;
      lv.gplane = (long long)h * lv.pitch;
      lv.zk = (long long)h * lv.pitch;
      lv.zplane = lv.zk * p.K;
      const size_t gbytes = align256(sizeof(float) * (size_t)lv.gplane * p.C);
      const size_t zbytes = align256(zsize * (size_t)lv.zplane * p.C);
      lv.G = reinterpret_cast<float*>(off);
      off += gbytes;
      lv.Z = reinterpret_cast<void*>(off);
      off += zbytes;
      if (l <= p.levels - 2) {
        lv.E = reinterpret_cast<float*>(off);
        off += gbytes;
      }
    } else {
      lv.pitch = w;
      lv.gplane = (long long)h * w;
    }
    if (out) (*out)[l] = lv;
    h = (h + 1) / 2;
    w = (w + 1) / 2;
  }
  return off;
}

// Every level buffer must lie inside the scratch allocation.
bool check_layout(const fllf_params& p, const std::vector<Level>& lv, const unsigned char* base,
                  size_t bytes) {
  const size_t zsize = p.precision == FLLF_FP32 ? 8 : 4;
  auto inside = [&](const void* ptr, size_t n) {
    const unsigned char* q = static_cast<const unsigned char*>(ptr);
    return q != nullptr && q >= base && q + n <= base + bytes;
  };
  for (int l = 1; l < p.levels; ++l) {
    const size_t g = sizeof(float) * (size_t)lv[l].gplane * p.C;
    const size_t z = zsize * (size_t)lv[l].zplane * p.C;
    if (lv[l].pitch < lv[l].w) return false;
    if (!inside(lv[l].G, g) || !inside(lv[l].Z, z)) return false;
    if (l <= p.levels - 2 && !inside(lv[l].E, g)) return false;
    if (l == p.levels - 1 && lv[l].E != nullptr) return false;
  }
  return true;
}

}  // namespace fllf

using namespace fllf;



namespace {

std::mutex g_ticket_mu;
struct Ticket {
  cudaEvent_t ev;
  int device;
  fllf_plan* plan;
  int snap = -1;  // the plan's snapshot word of the fault word, or -1 (read the device word)
};
std::unordered_map<uint64_t, Ticket> g_tickets;
uint64_t g_next_ticket = 1;

void free_plan(fllf_plan* pl) {
  if (!pl) return;
  if (pl->d_a) cudaFree(pl->d_a);
  if (pl->d_fault) cudaFree(pl->d_fault);
  if (pl->scratch) cudaFree(pl->scratch);
  if (pl->d_io_in) cudaFree(pl->d_io_in);
  if (pl->d_io_out) cudaFree(pl->d_io_out);
  if (pl->d_mpyr) cudaFree(pl->d_mpyr);
  if (pl->d_luma) cudaFree(pl->d_luma);
  if (pl->d_stage) cudaFree(pl->d_stage);
  plan_graph_destroy(pl->graph);
  for (cudaEvent_t e : pl->io_ev)
    if (e) cudaEventDestroy(e);
  for (HostSlot& h : pl->host_slots) {
    if (h.d_in) cudaFree(h.d_in);
    if (h.d_out) cudaFree(h.d_out);
    for (cudaEvent_t e : {h.copied_in, h.filtered, h.copied_out})
      if (e) cudaEventDestroy(e);
  }
  if (pl->h_snap) cudaFreeHost(pl->h_snap);
  if (pl->io_h2d) cudaStreamDestroy(pl->io_h2d);
  if (pl->io_d2h) cudaStreamDestroy(pl->io_d2h);
  delete pl->timer;
  delete pl;
}

// The two copy streams of the host-buffer paths (first use).
fllf_status copy_streams(fllf_plan* pl) {
  cudaError_t e;
  if (!pl->io_h2d && (e = cudaStreamCreateWithFlags(&pl->io_h2d, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "copy stream creation");
  if (!pl->io_d2h && (e = cudaStreamCreateWithFlags(&pl->io_d2h, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(e, "copy stream creation");
  return FLLF_OK;
}

// The staging slots of fllf_submit_host (first use): all or none.
fllf_status host_slots_setup(fllf_plan* pl) {
  if (!pl->host_slots.empty()) return FLLF_OK;
  fllf_status st = copy_streams(pl);
  if (st != FLLF_OK) return st;
  const size_t bytes = sizeof(float) * (size_t)pl->p.H * pl->p.W * pl->p.C;
  std::vector<HostSlot> slots(kHostSlots);
  auto undo = [&]() {
    for (HostSlot& h : slots) {
      if (h.d_in) cudaFree(h.d_in);
      if (h.d_out) cudaFree(h.d_out);
      for (cudaEvent_t e : {h.copied_in, h.filtered, h.copied_out})
        if (e) cudaEventDestroy(e);
    }
  };
  for (HostSlot& h : slots) {
    if (cudaMalloc(&h.d_in, bytes) != cudaSuccess || cudaMalloc(&h.d_out, bytes) != cudaSuccess) {
      cudaGetLastError();
      undo();
      return fail(FLLF_ENOMEM, "host staging slot allocation failed");
    }
    for (cudaEvent_t* e : {&h.copied_in, &h.filtered, &h.copied_out}) {
      const cudaError_t ce = cudaEventCreateWithFlags(e, cudaEventDisableTiming);
      if (ce != cudaSuccess) {
        cudaGetLastError();
        *e = nullptr;
        undo();
        return cuda_fail(ce, "cudaEventCreate");
      }
    }
  }
  pl->host_slots = std::move(slots);
  pl->next_slot = 0;
  return FLLF_OK;
}

// The plan's host-mapped fault-word snapshots (first use).  Without them
// (allocation failed) tickets read the device word instead.
void snap_setup(fllf_plan* pl) {
  if (pl->h_snap) return;
  unsigned* h = nullptr;
  unsigned* d = nullptr;
  if (cudaHostAlloc(reinterpret_cast<void**>(&h), sizeof(unsigned) * kSnapWords, cudaHostAllocMapped) !=
          cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&d), h, 0) != cudaSuccess) {
    cudaGetLastError();
    if (h) cudaFreeHost(h);
    return;
  }
  std::lock_guard<std::mutex> lk(g_ticket_mu);
  pl->h_snap = h;
  pl->d_snap = d;
  pl->snap_free.clear();
  for (int i = kSnapWords - 1; i >= 0; --i) pl->snap_free.push_back(i);
}

// Ends a submitted run on stream s: a snapshot of the plan's fault word into
// a free host-mapped word (none free: the poll reads the device word), a
// completion event, and the ticket.
fllf_status enqueue_ticket(fllf_plan* plan, cudaStream_t s, uint64_t* ticket) {
  snap_setup(plan);
  int snap = -1;
  {
    std::lock_guard<std::mutex> lk(g_ticket_mu);
    if (!plan->snap_free.empty()) {
      snap = plan->snap_free.back();
      plan->snap_free.pop_back();
    }
  }
  auto give_back = [&]() {
    if (snap < 0) return;
    std::lock_guard<std::mutex> lk(g_ticket_mu);
    plan->snap_free.push_back(snap);
  };
  cudaError_t e;
  if (snap >= 0 && (e = launch_status_snapshot(plan->d_fault, plan->d_snap + snap, s)) != cudaSuccess) {
    give_back();
    return cuda_fail(e, "status snapshot");
  }
  cudaEvent_t ev;
  if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) {
    give_back();
    return cuda_fail(e, "cudaEventCreate");
  }
  if ((e = cudaEventRecord(ev, s)) != cudaSuccess) {
    cudaEventDestroy(ev);
    give_back();
    return cuda_fail(e, "cudaEventRecord");
  }
  std::lock_guard<std::mutex> lk(g_ticket_mu);
  *ticket = g_next_ticket++;
  g_tickets[*ticket] = Ticket{ev, plan->device, plan, snap};
  return FLLF_OK;
}

// One-plane views of a plan (levels offset to plane c, maps of one plane) and
// the streams and events of the host-buffer plane pipeline; built once.
fllf_status plane_pipeline_setup(fllf_plan* pl) {
  const int C = pl->p.C, L = pl->p.levels;
  if ((int)pl->plane_lv.size() == C) return FLLF_OK;
  fllf_params p1 = pl->p;
  p1.C = 1;
  std::vector<std::vector<Level>> lvs(C);
  std::vector<PathMaps> maps(C);
  for (int c = 0; c < C; ++c) {
    lvs[c] = pl->lv;
    for (int l = 1; l < L; ++l) {
      Level& v = lvs[c][l];
      const size_t zs = pl->p.precision == FLLF_FP32 ? 8 : 4;
      if (v.G) v.G += (size_t)c * v.gplane;
      if (v.E) v.E += (size_t)c * v.gplane;
      if (v.Z) v.Z = static_cast<unsigned char*>(v.Z) + (size_t)c * v.zplane * zs;
    }
    if (L > 1 && !build_maps(p1, lvs[c], &maps[c]))
      return fail(FLLF_ECUDA, "TMA tensor map encoding failed (cuTensorMapEncodeTiled)");
  }
  fllf_status st = copy_streams(pl);
  if (st != FLLF_OK) return st;
  cudaError_t e;
  while ((int)pl->io_ev.size() < 2 * C) {
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
      return cuda_fail(e, "cudaEventCreate");
    pl->io_ev.push_back(ev);
  }
  pl->plane_lv = std::move(lvs);
  pl->plane_maps = std::move(maps);
  return FLLF_OK;
}

}  // namespace


// Clears the plan's status block (fault word and grid-barrier words) and
// reports the timeout a kernel's bounded wait recorded there.
static fllf_status report_fault(fllf_plan* plan) {
  cudaMemset(plan->d_fault, 0, 256);
  return fail(FLLF_ETIMEOUT, "a kernel's bounded wait for a shared-memory copy ran out");
}

// Reads and clears the plan's fault word (after the plan's work completed).
static fllf_status check_fault(fllf_plan* plan) {
  unsigned f = 0;
  cudaError_t e = cudaMemcpy(&f, plan->d_fault, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "fault word read");
  return f ? report_fault(plan) : FLLF_OK;
}

namespace {

// Period of Eq. (12): T minimising E(T) = erfc(a / T) + erfc((T - R) / sigma)
// with a = pi sigma (2K + 1).  For R < T < a the first term's slope,
// (2/sqrt(pi)) (a / T^2) exp(-a^2 / T^2), rises with T and the second's
// magnitude, (2/sqrt(pi)) exp(-(T - R)^2 / sigma^2) / sigma, falls, so the
// minimum is the single root of
//   h(T) = log(a / T^2) - a^2 / T^2 + log(sigma) + (T - R)^2 / sigma^2,
// found by bisection in float64 (log space keeps both slopes from
// underflowing).  Without a sign change in (R, min(a, R + 40 sigma)) the
// minimum of E is searched directly by golden sections instead.
double optimal_period(double sigma, int K, double R) {
  const double a = M_PI * sigma * (2.0 * K + 1.0);
  auto E = [&](double T) { return std::erfc(a / T) + std::erfc((T - R) / sigma); };
  auto h = [&](double T) {
    const double u = a / T, v = (T - R) / sigma;
    return std::log(a / (T * T)) - u * u + std::log(sigma) + v * v;
  };
  double lo = R * (1.0 + 1e-12) + 1e-300, hi = std::min(a, R + 40.0 * sigma);
  if (hi > lo && h(lo) < 0.0 && h(hi) > 0.0) {
    for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
      const double mid = 0.5 * (lo + hi);
      (h(mid) < 0.0 ? lo : hi) = mid;
    }
    return 0.5 * (lo + hi);
  }
  lo = R;
  hi = R + 40.0 * sigma + a;
  const double g = 0.5 * (std::sqrt(5.0) - 1.0);
  double c = hi - g * (hi - lo), d = lo + g * (hi - lo);
  for (int it = 0; it < 400 && hi - lo > 1e-13 * hi; ++it) {
    if (E(c) < E(d)) {
      hi = d;
      d = c;
      c = hi - g * (hi - lo);
    } else {
      lo = c;
      c = d;
      d = lo + g * (hi - lo);
    }
  }
  return 0.5 * (lo + hi);
}

}  // namespace

extern "C" {

const char* fllf_status_str(fllf_status s) {
  switch (s) {
    case FLLF_OK: return "FLLF_OK";
    case FLLF_EINVAL: return "FLLF_EINVAL";
    case FLLF_ENOMEM: return "FLLF_ENOMEM";
    case FLLF_ECUDA: return "FLLF_ECUDA";
    case FLLF_EAGAIN: return "FLLF_EAGAIN";
    case FLLF_ETIMEOUT: return "FLLF_ETIMEOUT";
    case FLLF_EBUSY: return "FLLF_EBUSY";
  }
  return "FLLF_UNKNOWN";
}

const char* fllf_last_error(void) { return g_last_error.c_str(); }

fllf_status fllf_params_validate(const fllf_params* p) { return validate(p); }

fllf_status fllf_coeffs(const fllf_params* p, double* a_out) {
  fllf_status st = validate(p);
  if (st != FLLF_OK) return st;
  if (!a_out) return fail(FLLF_EINVAL, "a_out is NULL");
  if (p->method == FLLF_METHOD_FAST) return fail(FLLF_EINVAL, "fast LLF has no Fourier coefficients");
  compute_coeffs(*p, a_out);
  return FLLF_OK;
}

fllf_status fllf_optimal_period(double sigma_r, int K, double R, double* T_out) {
  if (!T_out) return fail(FLLF_EINVAL, "T_out is NULL");
  if (!(sigma_r > 0.0) || !std::isfinite(sigma_r) || !(R > 0.0) || !std::isfinite(R) || K < 1 || K > 64)
    return fail(FLLF_EINVAL, "fllf_optimal_period needs sigma_r > 0, R > 0 (finite) and 1 <= K <= 64");
  *T_out = optimal_period(sigma_r, K, R);
  return FLLF_OK;
}

size_t fllf_plan_scratch_bytes(const fllf_params* p) {
  if (validate(p) != FLLF_OK) return 0;
  return layout(normalized(*p), nullptr);
}

fllf_status fllf_plan_create(const fllf_params* user, int device, fllf_plan** out) {
  if (!out) return fail(FLLF_EINVAL, "out is NULL");
  *out = nullptr;
  fllf_status st = validate(user);
  if (st != FLLF_OK) return st;
  const fllf_params np = normalized(*user);
  const fllf_params* p = &np;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(FLLF_EINVAL, "device out of range");
  DeviceGuard guard(device);
  if (!guard.ok) return fail(FLLF_ECUDA, "cudaSetDevice failed");

  fllf_plan* pl = new (std::nothrow) fllf_plan();
  if (!pl) return fail(FLLF_ENOMEM, "host allocation of the plan failed");
  pl->p = *p;
  pl->device = device;
  pl->a64.assign(p->K, 0.0);   // fast LLF: zeros (unused)
  if (p->method == FLLF_METHOD_FOURIER) compute_coeffs(*p, pl->a64.data());
  std::vector<float> a32(p->K);
  for (int k = 0; k < p->K; ++k) a32[k] = (float)pl->a64[k];

  if ((e = cudaMalloc(&pl->d_a, sizeof(float) * p->K)) != cudaSuccess) {
    free_plan(pl);
    return fail(FLLF_ENOMEM, std::string("coefficient allocation: ") + cudaGetErrorString(e));
  }
  if ((e = cudaMemcpy(pl->d_a, a32.data(), sizeof(float) * p->K, cudaMemcpyHostToDevice)) !=
      cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "coefficient upload");
  }
  std::vector<Level> rel;
  pl->scratch_bytes = layout(*p, &rel);
  if (pl->scratch_bytes) {
    if ((e = cudaMalloc(&pl->scratch, pl->scratch_bytes)) != cudaSuccess) {
      cudaGetLastError();
      free_plan(pl);
      return fail(FLLF_ENOMEM, std::string("scratch allocation: ") + cudaGetErrorString(e));
    }
  }
  // layout() returns byte offsets (the first buffer sits at offset 0): rebase
  // by level role -- G and Z exist at every level l >= 1, E at 1 <= l <= L-2.
  pl->lv = rel;
  const int L = p->levels;
  for (int l = 0; l < L; ++l) {
    Level& lv = pl->lv[l];
    if (l == 0) {
      lv.G = nullptr;
      lv.Z = nullptr;
      lv.E = nullptr;
      continue;
    }
    lv.G = reinterpret_cast<float*>(pl->scratch + reinterpret_cast<size_t>(rel[l].G));
    lv.Z = pl->scratch + reinterpret_cast<size_t>(rel[l].Z);
    lv.E = (l <= L - 2) ? reinterpret_cast<float*>(pl->scratch + reinterpret_cast<size_t>(rel[l].E))
                        : nullptr;
  }
  if (!check_layout(*p, pl->lv, pl->scratch, pl->scratch_bytes)) {
    free_plan(pl);
    return fail(FLLF_EINVAL, "internal error: scratch layout outside the allocation");
  }
  if ((e = cudaMalloc(&pl->d_fault, 256)) != cudaSuccess) {
    cudaGetLastError();
    pl->d_fault = nullptr;
    free_plan(pl);
    return fail(FLLF_ENOMEM, "fault word allocation failed");
  }
  if ((e = cudaMemset(pl->d_fault, 0, 256)) != cudaSuccess) {
    free_plan(pl);
    return cuda_fail(e, "fault word clear");
  }
  if (p->levels > 1 && (p->W % 4) != 0) {
    // rows of W floats do not start on 16-byte boundaries: the input is
    // staged at a padded pitch for the level-0 TMA loads
    const size_t bytes = sizeof(float) * (size_t)staged_pitch(p->W) * p->H * p->C;
    if ((e = cudaMalloc(&pl->d_stage, bytes)) != cudaSuccess) {
      cudaGetLastError();
      pl->d_stage = nullptr;
      free_plan(pl);
      return fail(FLLF_ENOMEM, "input staging buffer allocation failed");
    }
  }
  if (p->levels > 1 && !build_maps(*p, pl->lv, &pl->maps)) {
    free_plan(pl);
    return fail(FLLF_ECUDA, "TMA tensor map encoding failed (cuTensorMapEncodeTiled)");
  }
  if (p->levels > 1 && p->method == FLLF_METHOD_FOURIER) {
    // the dataflow launch: task list and argument tables of this image
    GraphGrain g = pl->tune.grain;
    g.lo = pl->tune.dataflow == 3 ? (g.lo >= 2 ? g.lo : 3) : 0;
    pl->graph = plan_graph_create(pl, g, pl->tune.dataflow != 2, &e);
    if (!pl->graph) {
      free_plan(pl);
      return e == cudaErrorMemoryAllocation ? fail(FLLF_ENOMEM, "dataflow task table allocation failed")
                                            : cuda_fail(e, "dataflow task table");
    }
  }
  *out = pl;
  return FLLF_OK;
}

fllf_status fllf_plan_destroy(fllf_plan* plan) {
  if (!plan) return FLLF_OK;
  DeviceGuard guard(plan->device);
  free_plan(plan);
  return FLLF_OK;
}

fllf_status fllf_plan_params(const fllf_plan* plan, fllf_params* out) {
  if (!plan || !out) return fail(FLLF_EINVAL, "plan or out is NULL");
  *out = plan->p;
  return FLLF_OK;
}

fllf_status fllf_plan_coeffs(const fllf_plan* plan, double* a_out) {
  if (!plan || !a_out) return fail(FLLF_EINVAL, "plan or a_out is NULL");
  if (plan->p.method != FLLF_METHOD_FOURIER) return fail(FLLF_EINVAL, "fast LLF has no Fourier coefficients");
  std::memcpy(a_out, plan->a64.data(), sizeof(double) * plan->p.K);
  return FLLF_OK;
}

fllf_status fllf_run(fllf_plan* plan, const float* d_in, float* d_out, void* stream) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (!d_in || !d_out) return fail(FLLF_EINVAL, "input or output pointer is NULL");
  const size_t n = (size_t)plan->p.H * plan->p.W * plan->p.C;
  const char *a = reinterpret_cast<const char*>(d_in), *b = reinterpret_cast<const char*>(d_out);
  if (a < b + n * sizeof(float) && b < a + n * sizeof(float))
    return fail(FLLF_EINVAL, "input and output buffers overlap");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(FLLF_ECUDA, "cudaSetDevice failed");
  cudaError_t e = enqueue_path(plan->p, plan->lv, plan->maps, plan->d_a, plan->d_fault, d_in, d_out,
                               reinterpret_cast<cudaStream_t>(stream), plan->timer, nullptr, 0.f,
                               &plan->tune, plan->graph, plan->d_stage);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return FLLF_OK;
}

fllf_status fllf_run_adaptive(fllf_plan* plan, const float* d_in, const float* d_gain, float* d_out,
                              void* stream) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (!d_in || !d_out || !d_gain) return fail(FLLF_EINVAL, "input, gain or output pointer is NULL");
  const fllf_params& p = plan->p;
  if (p.method != FLLF_METHOD_FOURIER) return fail(FLLF_EINVAL, "fllf_run_adaptive needs a Fourier LLF plan");
  if (p.m == 1.0)
    return fail(FLLF_EINVAL, "fllf_run_adaptive needs a plan with m != 1 (its coefficients are rescaled "
                             "per pixel by (m_p - 1) / (m - 1))");
  const size_t n = (size_t)p.H * p.W * p.C;
  const char *a = reinterpret_cast<const char*>(d_in), *b = reinterpret_cast<const char*>(d_out);
  const char* g = reinterpret_cast<const char*>(d_gain);
  if (a < b + n * sizeof(float) && b < a + n * sizeof(float))
    return fail(FLLF_EINVAL, "input and output buffers overlap");
  if (g < b + n * sizeof(float) && b < g + (size_t)p.H * p.W * sizeof(float))
    return fail(FLLF_EINVAL, "gain map and output buffers overlap");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(FLLF_ECUDA, "cudaSetDevice failed");
  const int L = p.levels;
  std::vector<Level> lv = plan->lv;
  std::vector<size_t> off(L, 0);
  size_t bytes = 0;
  for (int l = 1; l <= L - 2; ++l) {
    off[l] = bytes;
    bytes += align256(sizeof(float) * (size_t)lv[l].h * lv[l].pitch);
  }
  if (bytes && !plan->d_mpyr) {
    cudaError_t e = cudaMalloc(&plan->d_mpyr, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      plan->d_mpyr = nullptr;
      return fail(FLLF_ENOMEM, "gain-map pyramid allocation failed");
    }
  }
  for (int l = 1; l <= L - 2; ++l)
    lv[l].M = reinterpret_cast<const float*>(reinterpret_cast<unsigned char*>(plan->d_mpyr) + off[l]);
  cudaError_t e = enqueue_path(p, lv, plan->maps, plan->d_a, plan->d_fault, d_in, d_out,
                               reinterpret_cast<cudaStream_t>(stream), plan->timer, d_gain,
                               (float)(1.0 / (p.m - 1.0)), &plan->tune, nullptr, plan->d_stage);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return FLLF_OK;
}

fllf_status fllf_run_luma(fllf_plan* plan, const float* d_rgb_in, float* d_rgb_out, void* stream) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (!d_rgb_in || !d_rgb_out) return fail(FLLF_EINVAL, "input or output pointer is NULL");
  const fllf_params& p = plan->p;
  if (p.C != 1) return fail(FLLF_EINVAL, "fllf_run_luma needs a plan with C == 1 (it filters the luma plane)");
  const size_t n = (size_t)p.H * p.W;
  const char *a = reinterpret_cast<const char*>(d_rgb_in), *b = reinterpret_cast<const char*>(d_rgb_out);
  if (a < b + 3 * n * sizeof(float) && b < a + 3 * n * sizeof(float))
    return fail(FLLF_EINVAL, "input and output buffers overlap");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(FLLF_ECUDA, "cudaSetDevice failed");
  if (!plan->d_luma) {
    cudaError_t e = cudaMalloc(&plan->d_luma, 2 * n * sizeof(float));
    if (e != cudaSuccess) {
      cudaGetLastError();
      plan->d_luma = nullptr;
      return fail(FLLF_ENOMEM, "luma buffer allocation failed");
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float* y = plan->d_luma;
  float* yf = plan->d_luma + n;
  static const float kLuma[3] = {0.299f, 0.587f, 0.114f};  // BT.601
  cudaError_t e;
  if ((e = launch_luma(d_rgb_in, y, (long long)n, kLuma, s)) != cudaSuccess) return cuda_fail(e, "luma");
  if ((e = enqueue_path(p, plan->lv, plan->maps, plan->d_a, plan->d_fault, y, yf, s, plan->timer,
                        nullptr, 0.f, &plan->tune, nullptr, plan->d_stage)) != cudaSuccess)
    return cuda_fail(e, "kernel launch");
  if ((e = launch_luma_apply(d_rgb_in, y, yf, d_rgb_out, (long long)n, s)) != cudaSuccess)
    return cuda_fail(e, "luma apply");
  return FLLF_OK;
}

fllf_status fllf_run_host(fllf_plan* plan, const float* h_in, float* h_out, void* stream) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (!h_in || !h_out) return fail(FLLF_EINVAL, "input or output pointer is NULL");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(FLLF_ECUDA, "cudaSetDevice failed");
  const size_t bytes = sizeof(float) * (size_t)plan->p.H * plan->p.W * plan->p.C;
  cudaError_t e;
  if (!plan->d_io_in) {
    if ((e = cudaMalloc(&plan->d_io_in, bytes)) != cudaSuccess) {
      cudaGetLastError();
      plan->d_io_in = nullptr;
      return fail(FLLF_ENOMEM, "device input buffer allocation failed");
    }
  }
  if (!plan->d_io_out) {
    if ((e = cudaMalloc(&plan->d_io_out, bytes)) != cudaSuccess) {
      cudaGetLastError();
      plan->d_io_out = nullptr;
      return fail(FLLF_ENOMEM, "device output buffer allocation failed");
    }
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int C = plan->p.C;
  if (C == 1 || plan->p.levels == 1) {
    if ((e = cudaMemcpyAsync(plan->d_io_in, h_in, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return cuda_fail(e, "host-to-device copy");
    if ((e = enqueue_path(plan->p, plan->lv, plan->maps, plan->d_a, plan->d_fault, plan->d_io_in,
                          plan->d_io_out, s, plan->timer, nullptr, 0.f, &plan->tune, plan->graph,
                          plan->d_stage)) != cudaSuccess)
      return cuda_fail(e, "kernel launch");
    if ((e = cudaMemcpyAsync(h_out, plan->d_io_out, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
      return cuda_fail(e, "device-to-host copy");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return check_fault(plan);
  }
  // C >= 2: the planes are independent, so plane c's host-to-device copy, the
  // filtering of plane c-1 and the device-to-host copy of plane c-2 overlap
  // (two copy streams and the caller's stream; each plane runs the path on a
  // one-plane view of the scratch, with the same arithmetic per pixel).
  fllf_status st = plane_pipeline_setup(plan);
  if (st != FLLF_OK) return st;
  fllf_params p1 = plan->p;
  p1.C = 1;
  const size_t pn = (size_t)plan->p.H * plan->p.W, pb = sizeof(float) * pn;
  // the copy streams start after the caller's earlier work on s
  cudaEvent_t* ev = plan->io_ev.data();
  if ((e = cudaEventRecord(ev[0], s)) != cudaSuccess || (e = cudaStreamWaitEvent(plan->io_h2d, ev[0], 0)) != cudaSuccess)
    return cuda_fail(e, "stream ordering");
  for (int c = 0; c < C; ++c) {
    if ((e = cudaMemcpyAsync(plan->d_io_in + c * pn, h_in + c * pn, pb, cudaMemcpyHostToDevice, plan->io_h2d)) !=
            cudaSuccess ||
        (e = cudaEventRecord(ev[2 * c], plan->io_h2d)) != cudaSuccess)
      return cuda_fail(e, "host-to-device copy");
  }
  for (int c = 0; c < C; ++c) {
    if ((e = cudaStreamWaitEvent(s, ev[2 * c], 0)) != cudaSuccess) return cuda_fail(e, "stream ordering");
    if ((e = enqueue_path(p1, plan->plane_lv[c], plan->plane_maps[c], plan->d_a, plan->d_fault,
                          plan->d_io_in + c * pn, plan->d_io_out + c * pn, s, plan->timer, nullptr, 0.f,
                          &plan->tune, nullptr,
                          plan->d_stage ? plan->d_stage + (size_t)c * staged_pitch(p1.W) * p1.H : nullptr)) !=
        cudaSuccess)
      return cuda_fail(e, "kernel launch");
    if ((e = cudaEventRecord(ev[2 * c + 1], s)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(plan->io_d2h, ev[2 * c + 1], 0)) != cudaSuccess)
      return cuda_fail(e, "stream ordering");
    if ((e = cudaMemcpyAsync(h_out + c * pn, plan->d_io_out + c * pn, pb, cudaMemcpyDeviceToHost,
                             plan->io_d2h)) != cudaSuccess)
      return cuda_fail(e, "device-to-host copy");
  }
  if ((e = cudaStreamSynchronize(plan->io_d2h)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
  return check_fault(plan);
}

fllf_status fllf_submit(fllf_plan* plan, const float* d_in, float* d_out, void* stream,
                        uint64_t* ticket) {
  if (!ticket) return fail(FLLF_EINVAL, "ticket is NULL");
  fllf_status st = fllf_run(plan, d_in, d_out, stream);
  if (st != FLLF_OK) return st;
  DeviceGuard guard(plan->device);
  return enqueue_ticket(plan, reinterpret_cast<cudaStream_t>(stream), ticket);
}

fllf_status fllf_submit_host(fllf_plan* plan, const float* h_in, float* h_out, void* stream,
                             uint64_t* ticket) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (!h_in || !h_out || !ticket) return fail(FLLF_EINVAL, "input, output or ticket pointer is NULL");
  DeviceGuard guard(plan->device);
  if (!guard.ok) return fail(FLLF_ECUDA, "cudaSetDevice failed");
  fllf_status st = host_slots_setup(plan);
  if (st != FLLF_OK) return st;
  HostSlot& h = plan->host_slots[plan->next_slot];
  const size_t bytes = sizeof(float) * (size_t)plan->p.H * plan->p.W * plan->p.C;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  // input: after the slot's previous frame was filtered (its input read)
  if ((e = cudaStreamWaitEvent(plan->io_h2d, h.filtered, 0)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h.d_in, h_in, bytes, cudaMemcpyHostToDevice, plan->io_h2d)) != cudaSuccess ||
      (e = cudaEventRecord(h.copied_in, plan->io_h2d)) != cudaSuccess)
    return cuda_fail(e, "host-to-device copy");
  // filtering: after the input arrived and the slot's previous output left
  if ((e = cudaStreamWaitEvent(s, h.copied_in, 0)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(s, h.copied_out, 0)) != cudaSuccess)
    return cuda_fail(e, "stream ordering");
  if ((e = enqueue_path(plan->p, plan->lv, plan->maps, plan->d_a, plan->d_fault, h.d_in, h.d_out, s, plan->timer,
                        nullptr, 0.f, &plan->tune, plan->graph, plan->d_stage)) != cudaSuccess)
    return cuda_fail(e, "kernel launch");
  if ((e = cudaEventRecord(h.filtered, s)) != cudaSuccess) return cuda_fail(e, "stream ordering");
  // output: after the filtering
  if ((e = cudaStreamWaitEvent(plan->io_d2h, h.filtered, 0)) != cudaSuccess ||
      (e = cudaMemcpyAsync(h_out, h.d_out, bytes, cudaMemcpyDeviceToHost, plan->io_d2h)) != cudaSuccess ||
      (e = cudaEventRecord(h.copied_out, plan->io_d2h)) != cudaSuccess)
    return cuda_fail(e, "device-to-host copy");
  plan->next_slot = (plan->next_slot + 1) % kHostSlots;
  // the fault word as it stands after this frame goes to a host-mapped word
  // that fllf_poll reads, so no device-to-host copy queues behind the frame
  // copies on the copy engine
  return enqueue_ticket(plan, plan->io_d2h, ticket);
}

fllf_status fllf_poll(uint64_t ticket, int timeout_us) {
  Ticket tk;
  {
    std::lock_guard<std::mutex> lk(g_ticket_mu);
    auto it = g_tickets.find(ticket);
    if (it == g_tickets.end()) return fail(FLLF_EINVAL, "unknown or consumed ticket");
    tk = it->second;
  }
  DeviceGuard guard(tk.device);
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t e = cudaEventQuery(tk.ev);
    if (e == cudaSuccess || (e != cudaErrorNotReady)) {
      unsigned snapped = 1;
      {
        std::lock_guard<std::mutex> lk(g_ticket_mu);
        g_tickets.erase(ticket);
        if (tk.snap >= 0) {
          snapped = reinterpret_cast<volatile unsigned*>(tk.plan->h_snap)[tk.snap];
          tk.plan->snap_free.push_back(tk.snap);
        }
      }
      cudaEventDestroy(tk.ev);
      if (e != cudaSuccess) return cuda_fail(e, "submitted work failed");
      // the snapshot decides for a host-frame ticket (a set word is reported
      // even when an earlier poll already cleared the device word)
      if (tk.snap >= 0) return snapped ? report_fault(tk.plan) : FLLF_OK;
      return check_fault(tk.plan);
    }
    if (timeout_us == 0) return FLLF_EAGAIN;
    const auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                        std::chrono::steady_clock::now() - t0).count();
    const long long limit = timeout_us > 0 ? timeout_us : (long long)FLLF_POLL_MAX_US;
    if (us >= limit) return fail(FLLF_ETIMEOUT, "ticket still pending");
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

fllf_status fllf_plan_enable_timing(fllf_plan* plan, int enable) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  DeviceGuard guard(plan->device);
  if (enable && !plan->timer) plan->timer = new (std::nothrow) StageTimer();
  if (enable && !plan->timer) return fail(FLLF_ENOMEM, "timer allocation failed");
  if (enable) plan->timer->mask = 0xffffffffu;
  if (!enable) {
    delete plan->timer;
    plan->timer = nullptr;
  }
  return FLLF_OK;
}

fllf_status fllf_plan_set_timing_mask(fllf_plan* plan, unsigned mask) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (mask == 0) return fllf_plan_enable_timing(plan, 0);
  const fllf_status st = fllf_plan_enable_timing(plan, 1);
  if (st == FLLF_OK) plan->timer->mask = mask;
  return st;
}

fllf_status fllf_plan_set_wait_test(fllf_plan* plan, long long wait_cycles, unsigned extra_arrivals) {
  if (!plan) return fail(FLLF_EINVAL, "plan is NULL");
  if (wait_cycles < 0) return fail(FLLF_EINVAL, "wait_cycles must be >= 0");
  DeviceGuard guard(plan->device);
  // status words 4..5: the wait limit; word 6: extra grid-barrier arrivals
  unsigned words[4] = {0u, 0u, extra_arrivals, 0u};
  std::memcpy(words, &wait_cycles, sizeof(wait_cycles));
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
  if ((e = cudaMemcpy(plan->d_fault + fllf::kStatusLimitWord, words, sizeof(words), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return cuda_fail(e, "status block write");
  return FLLF_OK;
}

fllf_status fllf_plan_stage_times(fllf_plan* plan, double* ms, int* launches) {
  if (!plan || !ms || !launches) return fail(FLLF_EINVAL, "plan, ms or launches is NULL");
  for (int i = 0; i < FLLF_NSTAGE; ++i) {
    ms[i] = 0.0;
    launches[i] = 0;
  }
  if (!plan->timer) return FLLF_OK;
  DeviceGuard guard(plan->device);
  StageTimer* t = plan->timer;
  fllf_status st = FLLF_OK;
  for (auto& p : t->pending) {
    float x = 0.f;
    cudaError_t e = cudaEventSynchronize(p.e);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, p.b, p.e);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "stage timing");
    } else {
      ms[p.stage] += x;
      launches[p.stage] += 1;
    }
    t->pool.push_back(p.b);
    t->pool.push_back(p.e);
  }
  t->pending.clear();
  if (t->failed) st = fail(FLLF_ECUDA, "event creation failed during timing");
  t->failed = false;
  return st;
}

}  // extern "C"
