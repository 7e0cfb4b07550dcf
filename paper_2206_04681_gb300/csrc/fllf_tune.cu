// fllf_tune.cu -- launch tuning of plans and batches, and the autotuner.
//
// The kernels' tile shapes and orders per chunk are compile-time constants:
// they fix the TMA box geometry and the thread mappings.  What varies at
// run time is how the work is launched, and the autotuner picks that by
// timing the plan (or batch) on the caller's own images with CUDA events:
//   * where the chained launch of the small levels starts (levels >= 2 whose
//     planes hold at most chain_pixels pixels run in one cooperative launch
//     with grid barriers; larger levels run one launch per stage);
//   * below which size a level's combine runs on 32 x 16 tiles with two
//     pixels per thread rather than 64 x 32 tiles with eight;
//   * the persistent grid of every stage kind: how many CTAs per SM are
//     resident (fewer leaves each CTA more L2 and DRAM bandwidth, more
//     hides latency);
//   * the order in which the level 1 -> 2 REDUCE visits its work items
//     (last to first reads what the level-0 REDUCE wrote last from L2).
// Each timed run starts after an L2 flush (a write of twice the L2 size to a
// buffer the tuner allocates for the search and frees after it).  The
// search is coordinate descent from the current setting; a candidate
// replaces it only when it is at least 1% faster, so timing noise does not
// move the setting.  Every setting computes the same output, bit for bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <string>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"

using namespace fllf;

namespace {

fllf_status tfail(fllf_status s, const std::string& why) {
  set_last_error(why);
  return s;
}

struct Guard {
  int prev = -1;
  bool ok = false;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Milliseconds per call of `run`: one untimed call, then `reps` calls each
// timed on its own with events, right after a write of `flush_bytes` to
// `flush` (twice the L2), so that every timed call starts with a cold L2 as
// in steady use on frames larger than the cache; negative on a CUDA error.
double time_calls(const std::function<cudaError_t()>& run, int reps, cudaStream_t s, void* flush,
                  size_t flush_bytes) {
  std::vector<cudaEvent_t> ev(2 * reps, nullptr);
  bool ok = true;
  for (auto& e : ev) ok = ok && cudaEventCreate(&e) == cudaSuccess;
  ok = ok && run() == cudaSuccess;
  for (int i = 0; i < reps && ok; ++i) {
    if (flush) ok = cudaMemsetAsync(flush, i & 0xff, flush_bytes, s) == cudaSuccess;
    ok = ok && cudaEventRecord(ev[2 * i], s) == cudaSuccess && run() == cudaSuccess &&
         cudaEventRecord(ev[2 * i + 1], s) == cudaSuccess;
  }
  double ms = -1.0;
  if (ok && cudaEventSynchronize(ev[2 * reps - 1]) == cudaSuccess) {
    double sum = 0.0;
    for (int i = 0; i < reps && ok; ++i) {
      float t = 0.f;
      ok = cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]) == cudaSuccess;
      sum += t;
    }
    if (ok) ms = sum / reps;
  }
  for (auto e : ev)
    if (e) cudaEventDestroy(e);
  return ms;
}

// A device buffer of twice the L2 size for the flushes (freed by the owner).
size_t flush_size(int device) {
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device);
  return 2 * (size_t)(l2 > 0 ? l2 : (64 << 20));
}

constexpr double kGain = 0.99;  // a candidate must be >= 1% faster to be taken

void to_public(const Tuning& t, fllf_tuning* o) {
  o->chain_pixels = t.chain_px;
  for (int k = 0; k < FLLF_NSTAGE; ++k) o->ctas_per_sm[k] = t.cps[k];
  o->reduce_reverse = t.reverse;
  o->small_pixels = t.small_px;
  o->dataflow = t.dataflow;
  const int g[5] = {t.grain.up0, t.grain.up, t.grain.dns, t.grain.d10, t.grain.d0};
  for (int k = 0; k < 5; ++k) o->task_items[k] = g[k];
  o->dataflow_level = t.grain.lo;
  o->reduce_bands = t.bands;
}

// Task sizes of a public tuning (0: the default of that kind).
GraphGrain grain_of(const fllf_tuning* t) {
  GraphGrain g;
  int* f[5] = {&g.up0, &g.up, &g.dns, &g.d10, &g.d0};
  for (int k = 0; k < 5; ++k)
    if (t->task_items[k] > 0) *f[k] = t->task_items[k];
  g.lo = t->dataflow_level;
  return g;
}
bool same_grain(const GraphGrain& a, const GraphGrain& b) {
  return a.up0 == b.up0 && a.up == b.up && a.dns == b.dns && a.d10 == b.d10 && a.d0 == b.d0 && a.lo == b.lo;
}

// Replaces the plan's dataflow task list by one with the given task sizes
// and fused-combine mode (dataflow 2: the fused level-1/level-0 combine runs
// as its own kernel).
// The task list a mode runs: every stage (modes 1, 2), or the levels from
// grain.lo up (mode 3; level 3 when unset).
GraphGrain built_grain(const GraphGrain& g, int dataflow) {
  GraphGrain b = g;
  b.lo = dataflow == 3 ? (g.lo >= 2 ? g.lo : 3) : 0;
  return b;
}

fllf_status regrain(fllf_plan* plan, const GraphGrain& g, int dataflow) {
  const bool with_d10 = dataflow != 2;
  const GraphGrain b = built_grain(g, dataflow);
  if (!plan->graph || (same_grain(plan->tune.grain, g) && plan->graph->gb.with_d10 == with_d10 &&
                       plan->graph->gb.lo == b.lo)) {
    plan->tune.grain = g;
    return FLLF_OK;
  }
  cudaError_t e = cudaDeviceSynchronize();   // the old tables may be in use
  if (e != cudaSuccess) return tfail(FLLF_ECUDA, std::string("device synchronize: ") + cudaGetErrorString(e));
  PlanGraph* ng = plan_graph_create(plan, b, with_d10, &e);
  if (!ng) return tfail(FLLF_ENOMEM, std::string("dataflow task table: ") + cudaGetErrorString(e));
  plan_graph_destroy(plan->graph);
  plan->graph = ng;
  plan->tune.grain = g;
  return FLLF_OK;
}

}  // namespace

extern "C" {

fllf_status fllf_plan_get_tuning(const fllf_plan* plan, fllf_tuning* out) {
  if (!plan || !out) return tfail(FLLF_EINVAL, "plan or out is NULL");
  to_public(plan->tune, out);
  return FLLF_OK;
}

fllf_status fllf_plan_set_tuning(fllf_plan* plan, const fllf_tuning* t) {
  if (!plan || !t) return tfail(FLLF_EINVAL, "plan or tuning is NULL");
  if (t->chain_pixels < 0) return tfail(FLLF_EINVAL, "chain_pixels must be >= 0");
  if (t->small_pixels < 0) return tfail(FLLF_EINVAL, "small_pixels must be >= 0");
  for (int k = 0; k < FLLF_NSTAGE; ++k)
    if (t->ctas_per_sm[k] < 0 || t->ctas_per_sm[k] > 32) return tfail(FLLF_EINVAL, "ctas_per_sm must be 0..32");
  if (t->reduce_reverse != 0 && t->reduce_reverse != 1) return tfail(FLLF_EINVAL, "reduce_reverse must be 0 or 1");
  if (t->dataflow < 0 || t->dataflow > 3) return tfail(FLLF_EINVAL, "dataflow must be 0, 1, 2 or 3");
  if (t->dataflow_level != 0 && (t->dataflow_level < 2 || t->dataflow_level > 15))
    return tfail(FLLF_EINVAL, "dataflow_level must be 0 or 2..15");
  if (t->reduce_bands < 0 || t->reduce_bands > 256) return tfail(FLLF_EINVAL, "reduce_bands must be 0..256");
  for (int k = 0; k < 5; ++k)
    if (t->task_items[k] < 0 || t->task_items[k] > 4096) return tfail(FLLF_EINVAL, "task_items must be 0..4096");
  {
    Guard guard(plan->device);
    const fllf_status st = regrain(plan, grain_of(t), t->dataflow);
    if (st != FLLF_OK) return st;
  }
  plan->tune.dataflow = t->dataflow;
  plan->tune.bands = t->reduce_bands > 1 ? t->reduce_bands : 1;
  plan->tune.chain_px = t->chain_pixels;
  for (int k = 0; k < FLLF_NSTAGE; ++k) plan->tune.cps[k] = t->ctas_per_sm[k];
  plan->tune.reverse = t->reduce_reverse;
  plan->tune.small_px = t->small_pixels;
  return FLLF_OK;
}

fllf_status fllf_plan_autotune(fllf_plan* plan, const float* d_in, float* d_out, int reps, void* stream,
                               double* best_ms) {
  if (!plan || !d_in || !d_out) return tfail(FLLF_EINVAL, "plan, input or output is NULL");
  if (reps < 1 || reps > 10000) return tfail(FLLF_EINVAL, "reps must be 1..10000");
  Guard guard(plan->device);
  if (!guard.ok) return tfail(FLLF_ECUDA, "cudaSetDevice failed");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fllf_params& p = plan->p;
  const size_t fbytes = flush_size(plan->device);
  void* flush = nullptr;
  if (cudaMalloc(&flush, fbytes) != cudaSuccess) {
    cudaGetLastError();
    return tfail(FLLF_ENOMEM, "autotune: the L2 flush buffer could not be allocated");
  }
  PlanGraph* best_graph = plan->graph;   // the task list the best setting runs with
  auto measure = [&](const Tuning& t, const PlanGraph* g) {
    return time_calls(
        [&] {
          return enqueue_path(p, plan->lv, plan->maps, plan->d_a, plan->d_fault, d_in, d_out, s, nullptr,
                              nullptr, 0.f, &t, g, plan->d_stage);
        },
        reps, s, flush, fbytes);
  };
  Tuning best = plan->tune;
  double best_t = measure(best, best_graph);
  if (best_t < 0) {
    cudaFree(flush);
    return tfail(FLLF_ECUDA, "autotune: a timed run failed");
  }
  auto consider = [&](const Tuning& t) {
    const double m = measure(t, best_graph);
    if (m < 0) return false;
    if (m < kGain * best_t) {
      best = t;
      best_t = m;
    }
    return true;
  };
  bool ok = true;
  // keeps the candidate (and its task list) when it is at least 1% faster
  auto consider_graph = [&](const Tuning& t, PlanGraph* g) {
    const double m = measure(t, g);
    if (m < 0) {
      cudaStreamSynchronize(s);
      plan_graph_destroy(g);
      return false;
    }
    cudaStreamSynchronize(s);
    if (m < kGain * best_t) {
      if (best_graph != plan->graph && best_graph != g) plan_graph_destroy(best_graph);
      best_graph = g;
      best = t;
      best_t = m;
    } else if (g != best_graph && g != plan->graph) {
      plan_graph_destroy(g);
    }
    return true;
  };
  // 0. one dataflow launch, the dataflow launch followed by the fused
  // level-1/level-0 combine, or one launch per stage kind and level
  if (best_graph) {
    for (int mode = 0; mode <= 3 && ok; ++mode)
      for (int lo : {2, 3, 4}) {
        if (!ok || (mode != 3 && lo != 2)) continue;
        Tuning t = best;
        t.dataflow = mode;
        if (mode == 3) t.grain.lo = lo;
        if (mode == best.dataflow && (mode != 3 || lo == best.grain.lo)) continue;
        if (mode == 0) {
          ok = consider(t);
          continue;
        }
        if (mode == 3 && lo > p.levels - 2) continue;
        cudaError_t e;
        PlanGraph* g = plan_graph_create(plan, built_grain(t.grain, mode), mode != 2, &e);
        ok = g != nullptr && consider_graph(t, g);
      }
  }
  if (ok && best_graph && best.dataflow) {
    // its resident CTAs per SM, then the task size of each stage kind (a
    // new task list per candidate)
    const int occ = stage_occupancy(p.precision, FLLF_STAGE_GRAPH, false);
    for (int c = 1; c <= occ && ok; ++c) {
      Tuning t = best;
      t.cps[FLLF_STAGE_GRAPH] = c == occ ? 0 : c;
      if (t.cps[FLLF_STAGE_GRAPH] == best.cps[FLLF_STAGE_GRAPH]) continue;
      ok = consider(t);
    }
    const std::vector<std::vector<int>> cand = {{1, 2, 4, 8, 16}, {2, 4, 8, 16, 32}, {1, 2, 4, 8}, {1, 2, 4}};
    for (int k = 0; k < 4 && ok; ++k)
      for (int v : cand[k]) {
        if (!ok) break;
        Tuning t = best;
        int* f[4] = {&t.grain.up0, &t.grain.up, &t.grain.dns, &t.grain.d10};
        if (*f[k] == v) continue;
        *f[k] = v;
        cudaError_t e;
        PlanGraph* g = plan_graph_create(plan, built_grain(t.grain, best.dataflow), best.dataflow != 2, &e);
        ok = g != nullptr && consider_graph(t, g);
      }
  }
  if (best.dataflow && best_graph) {
    // the per-stage settings below do not apply to the dataflow launch
    if (best_graph != plan->graph) {
      cudaStreamSynchronize(s);
      plan_graph_destroy(plan->graph);
      plan->graph = best_graph;
    }
    plan->tune = best;
    cudaStreamSynchronize(s);
    cudaFree(flush);
    if (!ok) return tfail(FLLF_ECUDA, "autotune: a timed run failed");
    if (best_ms) *best_ms = best_t;
    return FLLF_OK;
  }
  if (best_graph != plan->graph) {   // a task list tried but the per-stage launches won
    cudaStreamSynchronize(s);
    plan_graph_destroy(best_graph);
    best.grain = plan->tune.grain;
  }
  // 1. where the chained launch of the small levels starts
  for (long long px : {0ll, 1ll << 15, 1ll << 17, 1ll << 19, 1ll << 21, 1ll << 23}) {
    Tuning t = best;
    t.chain_px = px;
    ok = ok && consider(t);
  }
  // 2. the size below which a combine runs on the small tiles: none, or
  // each level size from the finest combined level (>= 2) down
  {
    std::vector<long long> cand{0};
    for (int l = 2; l <= p.levels - 2; ++l) cand.push_back((long long)plan->lv[l].h * plan->lv[l].w * p.C);
    for (long long px : cand) {
      if (!ok) break;
      Tuning t = best;
      t.small_px = px;
      if (t.small_px == best.small_px) continue;
      ok = consider(t);
    }
  }
  // 3. resident CTAs per SM of each stage kind
  for (int kind = 0; kind < FLLF_STAGE_GRAPH && ok; ++kind) {
    const int occ = stage_occupancy(p.precision, kind, false);
    for (int c = 1; c <= occ && ok; ++c) {
      Tuning t = best;
      t.cps[kind] = c == occ ? 0 : c;
      if (t.cps[kind] == best.cps[kind]) continue;
      ok = consider(t);
    }
  }
  // 4. visiting order of the level 1 -> 2 REDUCE
  if (ok) {
    Tuning t = best;
    t.reverse = 1 - t.reverse;
    ok = consider(t);
  }
  // 5. the level-0 and level 1 -> 2 REDUCE in row bands
  for (int nb : {1, 2, 4, 6, 8, 12, 16}) {
    if (!ok || nb == best.bands || p.levels < 3) continue;
    Tuning t = best;
    t.bands = nb;
    ok = consider(t);
  }
  plan->tune = best;
  cudaStreamSynchronize(s);
  cudaFree(flush);
  if (!ok) return tfail(FLLF_ECUDA, "autotune: a timed run failed");
  if (best_ms) *best_ms = best_t;
  return FLLF_OK;
}

}  // extern "C"
