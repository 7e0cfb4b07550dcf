// fllf_server.cu -- continuous batching of filter requests on one GPU.
//
// One device pool (the HBM budget) holds every admitted request's pyramids;
// a first-fit allocator hands out 256-byte aligned ranges, so serving never
// calls cudaMalloc / cudaFree per request.  A worker thread
//   1. retires waves whose completion event fired (records latency, frees
//      the requests' pool ranges and slots),
//   2. admits queued requests in FIFO order while a slot, pool memory and a
//      free wave context are available (all requests of one wave share the
//      storage precision), building their plans inside the pool from the
//      server's resident plan data (below),
//   3. launches the admitted group as one batched wave on the context's
//      stream (argument tables uploaded from pinned memory, then the batched
//      stage kernels), and records the wave's event.
// Waves on different streams overlap on the device, and requests that arrive
// while waves run are admitted as soon as resources free up.
//
// Resident plan data: the Fourier coefficients of every parameter set the
// server has seen (m, sigma_r, T, K, coefficient mode) are kept in a cache,
// on the host and in a device slot, as long as a request uses them and
// afterwards until the cache is full (least recently used first out).  The
// quadrature of a new parameter set runs in fllf_server_submit, on the
// caller's thread; admission only takes the cached slot (uploading the
// coefficients once, when a set first gets a slot) and encodes the request's
// tensor maps for its pool range.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"

using namespace fllf;

namespace {

using Clock = std::chrono::steady_clock;

double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing of free ranges.
class RangeAlloc {
 public:
  explicit RangeAlloc(size_t size = 0) { reset(size); }
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = peak_ = 0;
  }
  bool alloc(size_t n, size_t* off) {
    n = (n + 255) & ~size_t(255);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= n) {
        *off = it->first;
        const size_t rest = it->second - n, start = it->first + n;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += n;
        peak_ = std::max(peak_, used_);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t n) {
    n = (n + 255) & ~size_t(255);
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t peak() const { return peak_; }
  void reset_peak() { peak_ = used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0, peak_ = 0;
};

enum ReqState { kPending = 0, kAdmitted = 1, kDone = 2, kFailed = 3 };

// The parameters the coefficients depend on.
struct CoefKey {
  double m, sigma_r, T;
  int K, mode;
  bool operator==(const CoefKey& o) const {
    return m == o.m && sigma_r == o.sigma_r && T == o.T && K == o.K && mode == o.mode;
  }
};
struct CoefKeyHash {
  size_t operator()(const CoefKey& k) const {
    const uint64_t a = std::hash<double>()(k.m), b = std::hash<double>()(k.sigma_r),
                   c = std::hash<double>()(k.T);
    return (size_t)(a * 0x9E3779B97F4A7C15ull ^ (b + 0x632BE59BD9B4E019ull) * 31 ^ c * 17 ^ (uint64_t)k.K * 131 ^
                    (uint64_t)k.mode);
  }
};
// A cached coefficient set: float32 values, its device slot (-1: none yet),
// the requests that hold it and when it was last used.
struct CoefEntry {
  std::vector<float> a32;
  int slot = -1;
  int refs = 0;
  uint64_t tick = 0;
};
constexpr int kCoefSlots = 4096;         // device slots of 64 floats
constexpr int kCoefCache = 2 * kCoefSlots;  // cached sets (with or without a slot)

struct Request {
  uint64_t id = 0;
  fllf_params p{};
  const float* in = nullptr;
  float* out = nullptr;
  double t_submit = 0, t_done = 0;
  int state = kPending;
  size_t off = 0, bytes = 0;      // pool range
  fllf_plan plan;                 // plan living inside the pool range
  CoefEntry* coef = nullptr;      // its cached coefficient set (held until it finishes)
  std::string err;                // why the request failed (the worker's errors are its own)
};

// Bytes of one request in the pool: its pyramids.
// Pyramid scratch, then (rows not 16-byte aligned) the input staging copy.
size_t stage_offset(const fllf_params& p) { return (layout(p, nullptr) + 255) & ~size_t(255); }
size_t request_bytes(const fllf_params& p) {
  if (p.levels < 2 || (p.W % 4) == 0) return layout(p, nullptr);
  return stage_offset(p) + sizeof(float) * (size_t)staged_pitch(p.W) * p.H * p.C;
}

// Status block after the pool: 16 waves x 64 bytes.
constexpr size_t kStatusBytes = 1024;

struct Wave {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  unsigned char* d_tab = nullptr;  // device argument tables
  unsigned char* h_tab = nullptr;  // pinned staging of the tables
  size_t cap = 0;
  unsigned* d_fault = nullptr;      // this wave's fault word (status block of the pool)
  volatile unsigned* h_fault = nullptr;  // pinned copy, read back after the wave's stages
  std::vector<Request*> reqs;
  bool busy = false;
  double t_launch = 0;
};

}  // namespace

struct fllf_server {
  int device = 0;
  size_t budget = 0;
  int max_slots = 0, max_queue = 0;
  unsigned char* pool = nullptr;
  unsigned* d_status = nullptr;  // status block: one 64-byte fault line per wave
  unsigned* h_status = nullptr;  // pinned mirror of the fault words
  RangeAlloc alloc;
  std::mutex mu;
  std::condition_variable cv;  // wakes the worker (submissions) and pollers (completions)
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> reqs;
  std::vector<Wave> waves;
  std::thread worker;
  bool stop = false;
  uint64_t next_id = 1;
  int active = 0;
  // statistics
  uint64_t submitted = 0, completed = 0, rejected = 0;
  std::vector<double> lat_ms;
  double px_done = 0, t_first = 0, t_last = 0;
  int max_active = 0, nwaves = 0;
  // resident plan data
  std::unordered_map<CoefKey, CoefEntry, CoefKeyHash> coefs;
  float* d_coef = nullptr;         // kCoefSlots x 64 floats
  std::vector<int> free_slots;
  uint64_t tick = 0, cache_hits = 0, cache_misses = 0, admission_quadratures = 0;
};

namespace {

fllf_status sfail(fllf_status s, const std::string& why) {
  set_last_error(why);
  return s;
}

// Builds request r's plan inside the pool (host work only).
bool build_request_plan(fllf_server* sv, Request* r) {
  std::vector<Level> rel;
  layout(r->p, &rel);
  unsigned char* base = sv->pool + r->off;
  fllf_plan& pl = r->plan;
  pl.p = r->p;
  pl.device = sv->device;
  pl.lv = rel;
  const int L = r->p.levels;
  for (int l = 0; l < L; ++l) {
    Level& v = pl.lv[l];
    if (l == 0) {
      v.G = nullptr;
      v.Z = nullptr;
      v.E = nullptr;
      continue;
    }
    v.G = reinterpret_cast<float*>(base + reinterpret_cast<size_t>(rel[l].G));
    v.Z = base + reinterpret_cast<size_t>(rel[l].Z);
    v.E = (l <= L - 2) ? reinterpret_cast<float*>(base + reinterpret_cast<size_t>(rel[l].E)) : nullptr;
  }
  if (!check_layout(r->p, pl.lv, base, r->bytes)) return false;
  pl.d_fault = sv->d_status;
  pl.scratch = nullptr;  // owned by the pool
  pl.d_stage = (L > 1 && (r->p.W % 4) != 0) ? reinterpret_cast<float*>(base + stage_offset(r->p)) : nullptr;
  if (L > 1 && !build_maps(r->p, pl.lv, &pl.maps)) return false;
  // the cached coefficients: a device slot, filled when the set first gets one
  CoefEntry& ce = *r->coef;
  if (ce.slot < 0) {
    if (sv->free_slots.empty()) {
      // take the slot of the least recently used set no request holds
      CoefEntry* lru = nullptr;
      for (auto& kv : sv->coefs)
        if (kv.second.slot >= 0 && kv.second.refs == 0 && (!lru || kv.second.tick < lru->tick)) lru = &kv.second;
      if (!lru) return false;
      sv->free_slots.push_back(lru->slot);
      lru->slot = -1;
    }
    ce.slot = sv->free_slots.back();
    sv->free_slots.pop_back();
    if (cudaMemcpy(sv->d_coef + 64 * (size_t)ce.slot, ce.a32.data(), sizeof(float) * ce.a32.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      sv->free_slots.push_back(ce.slot);
      ce.slot = -1;
      return false;
    }
  }
  ce.tick = ++sv->tick;
  pl.d_a = sv->d_coef + 64 * (size_t)ce.slot;
  return true;
}

// Releases a request's hold on its cached coefficients (lock held).
void release_coef(Request* r) {
  if (r->coef) --r->coef->refs;
  r->coef = nullptr;
}

// Enqueues a wave: coefficient uploads, argument tables, batched stages.
cudaError_t launch_wave(fllf_server* sv, Wave& w) {
  std::vector<const fllf_plan*> plans;
  std::vector<const float*> ins;
  std::vector<float*> outs;
  for (Request* r : w.reqs) {
    plans.push_back(&r->plan);
    ins.push_back(r->in);
    outs.push_back(r->out);
  }
  BatchBlob bb;
  build_batch_blob(plans, w.reqs.front()->p.precision, &bb);
  set_blob_fault(bb, w.d_fault);
  set_blob_io(bb, ins.data(), outs.data());
  const size_t need = bb.blob.size();
  cudaError_t e;
  if (need > w.cap) {
    if (w.h_tab) cudaFreeHost(w.h_tab);
    if (w.d_tab) cudaFree(w.d_tab);
    w.h_tab = nullptr;
    w.d_tab = nullptr;
    w.cap = 0;
    const size_t cap = need * 2;
    if ((e = cudaMallocHost(&w.h_tab, cap)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&w.d_tab, cap)) != cudaSuccess) return e;
    w.cap = cap;
  }
  std::memcpy(w.h_tab, bb.blob.data(), bb.blob.size());
  *w.h_fault = 0;
  if ((e = cudaMemsetAsync(w.d_fault, 0, sizeof(unsigned), w.stream)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(w.d_tab, w.h_tab, need, cudaMemcpyHostToDevice, w.stream)) != cudaSuccess)
    return e;
  for (int i : bb.copy_img) {
    const fllf_params& p = w.reqs[i]->p;
    if ((e = cudaMemcpyAsync(outs[i], ins[i], sizeof(float) * (size_t)p.H * p.W * p.C,
                             cudaMemcpyDeviceToDevice, w.stream)) != cudaSuccess)
      return e;
  }
  if ((e = launch_batch_pad(bb, w.d_tab, w.stream)) != cudaSuccess) return e;
  if ((e = launch_batch_stages(bb.stages, w.d_tab, w.reqs.front()->p.precision, w.stream)) !=
      cudaSuccess)
    return e;
  if ((e = cudaMemcpyAsync(const_cast<unsigned*>(w.h_fault), w.d_fault, sizeof(unsigned),
                           cudaMemcpyDeviceToHost, w.stream)) != cudaSuccess)
    return e;
  return cudaEventRecord(w.done, w.stream);
}

void worker_loop(fllf_server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    bool progress = false;
    // 1. retire finished waves
    for (Wave& w : sv->waves) {
      if (!w.busy) continue;
      cudaError_t q = cudaEventQuery(w.done);
      if (q == cudaErrorNotReady) continue;
      std::string why;
      if (q != cudaSuccess) {
        why = std::string("wave: ") + cudaGetErrorString(q);
      } else if (*w.h_fault != 0) {
        why = "wave: a bounded wait gave up (fault word " + std::to_string(*w.h_fault) + ")";
        q = cudaErrorLaunchFailure;
      }
      const double t = now_s();
      for (Request* r : w.reqs) {
        r->t_done = t;
        r->err = why;
        r->state = (q == cudaSuccess) ? kDone : kFailed;
        sv->alloc.release(r->off, r->bytes);
        release_coef(r);
        --sv->active;
        if (q == cudaSuccess) {
          ++sv->completed;
          sv->lat_ms.push_back((t - r->t_submit) * 1e3);
          sv->px_done += (double)r->p.H * r->p.W;
          sv->t_last = t;
        }
      }
      w.reqs.clear();
      w.busy = false;
      progress = true;
    }
    if (progress) sv->cv.notify_all();
    if (sv->stop) {
      bool busy = false;
      for (Wave& w : sv->waves) busy |= w.busy;
      if (!busy) break;
    }
    // 2. admit queued requests into a free wave context and launch it
    Wave* free_w = nullptr;
    for (Wave& w : sv->waves)
      if (!w.busy) {
        free_w = &w;
        break;
      }
    if (free_w && !sv->stop && !sv->pending.empty()) {
      const int prec = sv->pending.front()->p.precision;
      while (!sv->pending.empty() && sv->active < sv->max_slots) {
        Request* r = sv->pending.front();
        if (r->p.precision != prec) break;
        size_t off;
        if (!sv->alloc.alloc(r->bytes, &off)) break;  // wait for memory (FIFO order)
        r->off = off;
        sv->pending.pop_front();
        if (!build_request_plan(sv, r)) {
          sv->alloc.release(off, r->bytes);
          release_coef(r);
          r->err = "plan construction inside the pool failed";
          r->state = kFailed;
          ++sv->rejected;
          progress = true;
          continue;
        }
        r->state = kAdmitted;
        free_w->reqs.push_back(r);
        ++sv->active;
      }
      sv->max_active = std::max(sv->max_active, sv->active);
      if (!free_w->reqs.empty()) {
        free_w->busy = true;
        free_w->t_launch = now_s();
        ++sv->nwaves;
        lk.unlock();
        const cudaError_t e = launch_wave(sv, *free_w);
        lk.lock();
        if (e != cudaSuccess) {
          cudaGetLastError();
          for (Request* r : free_w->reqs) {
            r->err = std::string("wave launch: ") + cudaGetErrorString(e);
            r->state = kFailed;
            sv->alloc.release(r->off, r->bytes);
            release_coef(r);
            --sv->active;
          }
          free_w->reqs.clear();
          free_w->busy = false;
          set_last_error(std::string("wave launch: ") + cudaGetErrorString(e));
        }
        progress = true;
      }
    }
    if (progress) {
      sv->cv.notify_all();
      continue;
    }
    // 3. nothing to do right now: wait for a submission or poll the events again
    sv->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

}  // namespace

static void free_server(fllf_server* sv) {
  if (sv->d_coef) cudaFree(sv->d_coef);
  for (Wave& w : sv->waves) {
    if (w.stream) cudaStreamDestroy(w.stream);
    if (w.done) cudaEventDestroy(w.done);
    if (w.h_tab) cudaFreeHost(w.h_tab);
    if (w.d_tab) cudaFree(w.d_tab);
  }
  if (sv->h_status) cudaFreeHost(sv->h_status);
  if (sv->pool) cudaFree(sv->pool);
  delete sv;
}

extern "C" {

fllf_status fllf_server_create(int device, size_t hbm_budget, int max_slots, int max_queue,
                               int max_waves, fllf_server** out) {
  if (!out) return sfail(FLLF_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget < (1u << 20) || max_slots < 1 || max_slots > 4096 || max_queue < 1 || max_waves < 1 ||
      max_waves > 16)
    return sfail(FLLF_EINVAL, "hbm_budget >= 1 MiB, max_slots 1..4096, max_queue >= 1, max_waves 1..16");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return sfail(FLLF_EINVAL, "device out of range");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  fllf_server* sv = new (std::nothrow) fllf_server();
  if (!sv) return sfail(FLLF_ENOMEM, "server allocation failed");
  sv->device = device;
  sv->budget = (hbm_budget + 255) & ~size_t(255);
  sv->max_slots = max_slots;
  sv->max_queue = max_queue;
  cudaError_t e = cudaMalloc(&sv->pool, sv->budget + kStatusBytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    sv->pool = nullptr;
    free_server(sv);
    if (prev >= 0) cudaSetDevice(prev);
    return sfail(FLLF_ENOMEM, std::string("pool allocation: ") + cudaGetErrorString(e));
  }
  // The status block after the pool's budget holds one fault line per wave.
  sv->d_status = reinterpret_cast<unsigned*>(sv->pool + sv->budget);
  if (cudaMemset(sv->d_status, 0, kStatusBytes) != cudaSuccess ||
      cudaMallocHost(&sv->h_status, kStatusBytes) != cudaSuccess) {
    free_server(sv);
    if (prev >= 0) cudaSetDevice(prev);
    return sfail(FLLF_ECUDA, "status block allocation failed");
  }
  std::memset(sv->h_status, 0, kStatusBytes);
  if (cudaMalloc(&sv->d_coef, sizeof(float) * 64 * kCoefSlots) != cudaSuccess) {
    cudaGetLastError();
    sv->d_coef = nullptr;
    free_server(sv);
    if (prev >= 0) cudaSetDevice(prev);
    return sfail(FLLF_ENOMEM, "coefficient slots allocation failed");
  }
  for (int j = kCoefSlots - 1; j >= 0; --j) sv->free_slots.push_back(j);
  sv->alloc.reset(sv->budget);
  sv->waves.resize(max_waves);
  for (int i = 0; i < max_waves; ++i) {
    Wave& w = sv->waves[i];
    w.d_fault = sv->d_status + 16 * i;
    w.h_fault = sv->h_status + 16 * i;
    // Argument tables sized for a full wave of deep pyramids, so that growing
    // them (which synchronises the device) stays rare.
    w.cap = (64u << 10) + (size_t)std::min(max_slots, 256) * (16u << 10);
    if (cudaMallocHost(&w.h_tab, w.cap) != cudaSuccess || cudaMalloc(&w.d_tab, w.cap) != cudaSuccess) {
      w.cap = 0;
      free_server(sv);
      if (prev >= 0) cudaSetDevice(prev);
      return sfail(FLLF_ENOMEM, "argument table allocation failed");
    }
    if (cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming) != cudaSuccess) {
      free_server(sv);
      if (prev >= 0) cudaSetDevice(prev);
      return sfail(FLLF_ECUDA, "stream / event creation failed");
    }
  }
  sv->worker = std::thread(worker_loop, sv);
  if (prev >= 0) cudaSetDevice(prev);
  *out = sv;
  return FLLF_OK;
}

fllf_status fllf_server_destroy(fllf_server* sv) {
  if (!sv) return FLLF_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (Request* r : sv->pending) {
      r->state = kFailed;
      release_coef(r);
    }
    sv->pending.clear();
  }
  sv->cv.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(sv->device);
  free_server(sv);
  if (prev >= 0) cudaSetDevice(prev);
  return FLLF_OK;
}

fllf_status fllf_server_submit(fllf_server* sv, const fllf_params* p, const float* d_in, float* d_out,
                               uint64_t* ticket) {
  if (!sv || !ticket) return sfail(FLLF_EINVAL, "server or ticket is NULL");
  fllf_status st = validate(p);
  if (st != FLLF_OK) return st;
  if (p->method != FLLF_METHOD_FOURIER) return sfail(FLLF_EINVAL, "the server runs Fourier LLF requests only");
  if (!d_in || !d_out) return sfail(FLLF_EINVAL, "input or output pointer is NULL");
  const size_t n = sizeof(float) * (size_t)p->H * p->W * p->C;
  const char *a = reinterpret_cast<const char*>(d_in), *b = reinterpret_cast<const char*>(d_out);
  if (a < b + n && b < a + n) return sfail(FLLF_EINVAL, "input and output buffers overlap");
  const size_t bytes = request_bytes(*p);
  if (bytes > sv->budget) {
    std::lock_guard<std::mutex> lk(sv->mu);
    ++sv->rejected;
    return sfail(FLLF_ENOMEM, "request needs " + std::to_string(bytes) + " bytes, above the " +
                                  std::to_string(sv->budget) + "-byte pool");
  }
  auto r = std::make_unique<Request>();
  r->p = *p;
  r->in = d_in;
  r->out = d_out;
  r->bytes = bytes;
  // the coefficient set: from the cache, or computed here (on the caller's
  // thread, outside the server's lock) and cached
  const CoefKey key{p->m, p->sigma_r, p->T, p->K, p->coeff_mode};
  std::vector<float> fresh;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->coefs.find(key) == sv->coefs.end()) fresh.resize(1);
  }
  if (!fresh.empty()) {
    std::vector<double> a64(p->K);
    compute_coeffs(*p, a64.data());
    fresh.assign(a64.begin(), a64.end());
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return sfail(FLLF_EINVAL, "server is stopping");
    if ((int)sv->pending.size() >= sv->max_queue) {
      ++sv->rejected;
      return sfail(FLLF_EBUSY, "request queue is full");
    }
    auto it = sv->coefs.find(key);
    if (it == sv->coefs.end()) {
      if (fresh.empty()) {   // evicted since the look-up above: compute under the lock (rare)
        std::vector<double> a64(p->K);
        compute_coeffs(*p, a64.data());
        fresh.assign(a64.begin(), a64.end());
      }
      if ((int)sv->coefs.size() >= kCoefCache) {
        // make room: drop the least recently used sets no request holds
        std::vector<std::pair<uint64_t, CoefKey>> idle;
        for (auto& kv : sv->coefs)
          if (kv.second.refs == 0) idle.push_back({kv.second.tick, kv.first});
        std::sort(idle.begin(), idle.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        for (size_t j = 0; j < idle.size() && j < (size_t)kCoefCache / 4; ++j) {
          auto e = sv->coefs.find(idle[j].second);
          if (e->second.slot >= 0) sv->free_slots.push_back(e->second.slot);
          sv->coefs.erase(e);
        }
      }
      it = sv->coefs.emplace(key, CoefEntry{}).first;
      it->second.a32 = std::move(fresh);
      ++sv->cache_misses;
    } else {
      ++sv->cache_hits;
    }
    ++it->second.refs;
    it->second.tick = ++sv->tick;
    r->coef = &it->second;
    r->id = sv->next_id++;
    r->t_submit = now_s();
    if (sv->submitted == 0 || sv->t_first == 0) sv->t_first = r->t_submit;
    ++sv->submitted;
    *ticket = r->id;
    sv->pending.push_back(r.get());
    sv->reqs.emplace(r->id, std::move(r));
  }
  sv->cv.notify_all();
  return FLLF_OK;
}

fllf_status fllf_server_poll(fllf_server* sv, uint64_t ticket, int timeout_us) {
  if (!sv) return sfail(FLLF_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return sfail(FLLF_EINVAL, "unknown or consumed ticket");
  Request* r = it->second.get();
  auto finished = [&] { return r->state == kDone || r->state == kFailed; };
  if (!finished()) {
    if (timeout_us == 0) return FLLF_EAGAIN;
    const long long limit = timeout_us > 0 ? timeout_us : (long long)FLLF_POLL_MAX_US;
    if (!sv->cv.wait_for(lk, std::chrono::microseconds(limit), finished))
      return sfail(FLLF_ETIMEOUT, "request still pending");
  }
  const bool ok = r->state == kDone;
  const std::string why = r->err.empty() ? "request cancelled (server stopping)" : r->err;
  sv->reqs.erase(it);
  if (!ok) return sfail(FLLF_ECUDA, why);
  return FLLF_OK;
}

fllf_status fllf_server_stats_get(fllf_server* sv, fllf_server_stats* out) {
  if (!sv || !out) return sfail(FLLF_EINVAL, "server or out is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  fllf_server_stats s{};
  s.submitted = sv->submitted;
  s.completed = sv->completed;
  s.rejected = sv->rejected;
  if (!sv->lat_ms.empty()) {
    std::vector<double> v = sv->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) {
      const double pos = q * (v.size() - 1);
      const size_t i = (size_t)pos;
      const double f = pos - i;
      return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
    };
    s.p50_ms = pct(0.50);
    s.p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    s.mean_ms = sum / v.size();
    s.max_ms = v.back();
  }
  const double span = sv->t_last - sv->t_first;
  s.mpixel_per_s = span > 0 ? sv->px_done / span / 1e6 : 0.0;
  s.pool_bytes = sv->budget;
  s.pool_peak_bytes = sv->alloc.peak();
  s.max_active = sv->max_active;
  s.waves = sv->nwaves;
  s.plan_cache_hits = sv->cache_hits;
  s.plan_cache_misses = sv->cache_misses;
  s.admission_quadratures = sv->admission_quadratures;
  *out = s;
  return FLLF_OK;
}

fllf_status fllf_server_stats_reset(fllf_server* sv) {
  if (!sv) return sfail(FLLF_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->submitted = sv->completed = sv->rejected = 0;
  sv->lat_ms.clear();
  sv->px_done = sv->t_first = sv->t_last = 0;
  sv->max_active = sv->active;
  sv->nwaves = 0;
  sv->cache_hits = sv->cache_misses = sv->admission_quadratures = 0;
  sv->alloc.reset_peak();
  return FLLF_OK;
}

}  // extern "C"
