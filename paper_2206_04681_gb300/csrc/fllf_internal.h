// fllf_internal.h -- host helpers shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "fllf.h"
#include "fllf_device.cuh"

namespace fllf {

void set_last_error(const std::string& s);
fllf_status validate(const fllf_params* p);
// The parameters a plan runs with: for fast LLF, K = ceil(samples / 2) (the
// complex planes holding the sampled pyramids).
fllf_params normalized(const fllf_params& p);
// a_1..a_K in float64 (quadrature over one period, or the closed form).
void compute_coeffs(const fllf_params& p, double* a);
// Scratch layout of a plan; returns its size in bytes.  With `out`, fills
// the per-level descriptors with offsets (to be rebased on the allocation).
size_t layout(const fllf_params& p, std::vector<Level>* out);
// True when every level buffer of `lv` lies inside [base, base + bytes).
bool check_layout(const fllf_params& p, const std::vector<Level>& lv, const unsigned char* base,
                  size_t bytes);
// Optional hook called before and after every kernel launch of a path
// (stage kind, begin?) -- used by the per-stage timing diagnostics.
struct StageHook {
  virtual ~StageHook() = default;
  virtual void mark(int stage, bool begin, cudaStream_t s) = 0;
};

// Records a pair of events around every launch; events are pooled per plan.
struct StageTimer : StageHook {
  struct Pair { int stage; cudaEvent_t b, e; };
  std::vector<cudaEvent_t> pool;
  std::vector<Pair> pending;
  cudaEvent_t open = nullptr;
  bool failed = false;
  unsigned mask = 0xffffffffu;  // stage kinds to time (bit k = stage kind k)
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t ev = pool.back();
      pool.pop_back();
      return ev;
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreate(&ev) != cudaSuccess) failed = true;
    return ev;
  }
  void mark(int stage, bool begin, cudaStream_t s) override {
    if (!((mask >> stage) & 1u)) return;
    cudaEvent_t ev = get();
    if (!ev) return;
    cudaEventRecord(ev, s);
    if (begin) {
      open = ev;
    } else if (open) {
      pending.push_back({stage, open, ev});
      open = nullptr;
    }
  }
  ~StageTimer() override {
    for (auto& p : pending) {
      cudaEventDestroy(p.b);
      cudaEventDestroy(p.e);
    }
    for (auto ev : pool) cudaEventDestroy(ev);
  }
};

// TMA tensor maps of a plan's pyramid levels (indexed by level).
struct PathMaps {
  std::vector<CUtensorMap> z_dn;  // Z_l read as the coarse level of a combine
  std::vector<CUtensorMap> e_dn;  // E_l read as the coarse level of a combine
  std::vector<CUtensorMap> z_up;  // Z_l read as the source of a REDUCE
  std::vector<CUtensorMap> g_up;  // G_l read as the source of a REDUCE
  std::vector<CUtensorMap> z_dn1; // Z_l read as the coarse level of a level >= 1 combine (kKC1 orders)
  std::vector<CUtensorMap> z_fn;  // Z_l read as the fine level of a combine (kKC1 orders)
  std::vector<CUtensorMap> g_fn;  // G_l read as the fine level of a combine
  // the same four roles on the 32 x 16 tiles of the small-level combine (kKCS orders)
  std::vector<CUtensorMap> z_cs;  // Z_l as the coarse level (20 x 10 window)
  std::vector<CUtensorMap> e_cs;  // E_l as the coarse level (20 x 10 window)
  std::vector<CUtensorMap> z_fs;  // Z_l as the fine level (36 x 16 box)
  std::vector<CUtensorMap> g_fs;  // G_l as the fine level (36 x 16 box)
  CUtensorMap z_st1{};            // Z_1 written by the level-0 REDUCE (TMA store boxes)
  // fused level-1/level-0 combine (levels >= 3)
  CUtensorMap g1_d10{};           // G_1 on the level-1 window
  CUtensorMap z2_d10{};           // Z_2 on the level-2 window
  CUtensorMap e2_d10{};           // E_2 on the level-2 window (levels >= 4)
};
// Encodes the maps for the level buffers in `lv` (device addresses).
bool build_maps(const fllf_params& p, const std::vector<Level>& lv, PathMaps* m);
// Tiled map of a planar C x H x W float image with the given box (zero fill
// outside); false when the image does not allow one (W % 4 != 0, a base not
// 16-byte aligned) or the encoding fails.
// Level-0 image map (x = column, y = row, z = plane) with a row pitch of
// `pitch` floats (0: W).  False when the rows do not start on 16-byte
// boundaries (pitch % 4 != 0 or a misaligned base): the kernels then read
// the input with plain loads.
bool encode_image_map(CUtensorMap* m, const float* base, int W, int H, int C, uint32_t box_w, uint32_t box_h,
                      int pitch = 0);
// Row pitch (floats) of a plan's input staging copy: W rounded up to 4.
inline int staged_pitch(int W) { return (W + 3) & ~3; }

// ---- dataflow launch (one persistent grid over every stage) -------------------
// Work items per task of each stage kind (the REDUCE at levels >= 1 and the
// small-tile combines: at their finest level, halved per level above).
struct GraphGrain {
  int up0 = 4, up = 8, dns = 4, d10 = 2, d0 = 4;
  // 0: every stage; lo >= 2: only the REDUCE from level lo up and the
  // combines from the top down to level lo (the stages below run as their
  // own kernels, before and after)
  int lo = 0;
};
// The host image of a dataflow launch: argument tables, the ordered task
// list, the dependency list and the zeroed completion counters.
struct GraphBuild {
  std::vector<unsigned char> blob;
  size_t up0_off = 0, ups_off = 0, dns_off = 0, d10_off = 0, d0_off = 0, tasks_off = 0, bands_off = 0,
         cons_off = 0, seeds_off = 0, rt_off = 0;
  size_t rt_words = 0;       // the run state, zeroed before every run
  int ntasks = 0, nbands = 0, nseeds = 0, n_up0 = 0, n_ups = 0, n_dns = 0, n_d10 = 0, n_d0 = 0;
  bool ok = false;
  bool with_d10 = true;      // the fused level-1/level-0 combine is part of the task list
  int lo = 0;                // first level of the task list (0: every stage)
  Up0Args up0_inline{};      // level-0 argument blocks when they are passed inline (one image)
  Down10Args d10_inline{};
  Down0Args d0_inline{};
  std::vector<int> up0_img, d10_img, d0_img, copy_img;  // image of each table entry / single-level images
};
// Builds the task graph of the plans (same storage precision, Fourier LLF,
// no gain map).  inline0: one image whose level-0 argument blocks travel in
// the kernel parameters (set per run) instead of the tables.  with_d10: the
// fused level-1/level-0 combine of the images with >= 3 levels is in the
// task list (otherwise the caller launches it after the dataflow kernel).
void build_graph(const std::vector<const fllf_plan*>& plans, int prec, const GraphGrain& gr, bool inline0,
                 bool with_d10, GraphBuild* out);
// Runs the queue on one (host) worker: true when every task is made ready
// exactly once, only after the bands it reads are complete, and every band
// completes.
bool check_graph(const GraphBuild& gb, std::string* why);
// Kernel arguments for the tables uploaded at d_base (inline blocks copied).
GraphArgs graph_args(const GraphBuild& gb, const unsigned char* d_base, unsigned* d_fault);
// Clears the run state and launches the dataflow kernel.
cudaError_t launch_graph(int prec, const GraphArgs& g, size_t rt_bytes, cudaStream_t s, int cps,
                         bool with_d10);
// A plan's own dataflow launch (one image, level-0 blocks inline).
struct PlanGraph {
  GraphBuild gb;
  unsigned char* d_mem = nullptr;
  GraphArgs args{};   // table pointers; the level-0 blocks are completed per run
};

// Launch tuning of a plan (the autotuner's knobs).  chain_px: levels >= 2
// whose planes hold at most this many pixels in all run in the chained
// launch (0: none); small_px: the other combines at levels >= 2 with at most
// this many pixels run on the 32 x 16 tiles (0: none); cps[kind]:
// resident-CTA cap per SM of the stage kind's persistent grid (0: as many as
// fit); reverse: the level 1->2 REDUCE visits its items last to first.
struct Tuning {
  long long chain_px = 0;
  long long small_px = 1ll << 40;
  int cps[FLLF_NSTAGE] = {0, 0, 0, 0, 0, 0};
  int reverse = 1;
  // 0: the per-stage kernels (default: measured faster); 1: one persistent
  // dataflow launch; 2: the dataflow launch without the fused level-1/level-0
  // combine, which follows as its own kernel; 3: the per-stage kernels for
  // the levels below grain.lo and one dataflow launch for the levels from
  // grain.lo up
  int dataflow = 0;
  GraphGrain grain;   // work items per task of the dataflow launch
  // > 1: the level-0 and level 1 -> 2 REDUCE in this many row bands, each
  // level-1 band right after the level-0 band it reads (its Z_1 from L2)
  int bands = 1;
};
// Resident CTAs per SM of a stage kind's kernel for a storage precision.
int stage_occupancy(int prec, int kind, bool batched);

// Builds and uploads a plan's own dataflow launch (Fourier LLF, >= 2 levels);
// null with *err set on failure.  Destroy frees its device tables.
PlanGraph* plan_graph_create(const fllf_plan* plan, const GraphGrain& gr, bool with_d10, cudaError_t* err);
void plan_graph_destroy(PlanGraph* g);

// Enqueues the whole Fourier LLF path of one image on stream s.  `fault`
// is a device word that kernels set when a bounded wait runs out.  With a
// gain map d_gain (H x W, pitch W) the levels' M pointers must hold its
// pyramid buffers (levels 1..levels-2); the path builds the pyramid and
// scales each level's Fourier term by (m_{l,p} - 1) * mscale.
// With d_stage (C x H x staged_pitch(W) floats), an input whose rows are not
// 16-byte aligned is first copied there at the padded pitch, so that the
// level-0 kernels load it by TMA.
cudaError_t enqueue_path(const fllf_params& p, const std::vector<Level>& lv, const PathMaps& maps,
                         const float* d_a, unsigned* fault, const float* d_in, float* d_out,
                         cudaStream_t s, StageHook* hook = nullptr, const float* d_gain = nullptr,
                         float mscale = 0.f, const Tuning* tune = nullptr, const PlanGraph* graph = nullptr,
                         float* d_stage = nullptr);

// ---- batched argument tables (shared by batches and the server) ---------------
// kStageDown10 (the fused level-1/level-0 combine of the images with >= 3
// levels) shares the CTA cap of kStageDown0.
enum BatchStageKind { kStageUp0 = 0, kStageUp = 1, kStageDown = 2, kStageDown0 = 3, kStageDown10 = 4 };
struct StageRec {
  int kind;
  size_t args_off;    // byte offset of the argument blocks in the table image
  size_t prefix_off;  // byte offset of the work-item prefix sums
  int n, total;
};
struct BatchBlob {
  std::vector<unsigned char> blob;  // host image of the device tables
  std::vector<StageRec> stages;     // launch order
  std::vector<int> up0_img, down0_img, down10_img, copy_img;
  size_t up0_off = 0, down0_off = 0, down10_off = 0, status_off = 0;
  // input staging (images whose plan has d_stage): per image the staging
  // buffer or null, and the PadRow table with its row prefix sums
  std::vector<float*> stage;
  std::vector<int> pad_img;
  size_t pad_off = 0, pad_prefix_off = 0;
  int pad_total = 0;
};
// Argument tables for `plans` (same storage precision `prec`).
void build_batch_blob(const std::vector<const fllf_plan*>& plans, int prec, BatchBlob* out);
// Points every argument block's fault word at d_fault.
void set_blob_fault(BatchBlob& bb, unsigned* d_fault);
// Writes the level-0 input / output pointers of each image, and the input's
// tensor maps, into the tables u (up0), d0 (level-0 combine) and d10 (fused
// level-1/level-0 combine), which hold bb's entries in bb's order.
// With staging, the maps point at the staging buffers and pad (bb's PadRow
// entries, may be null when bb has none) gets this run's sources.
void set_level0_io(const BatchBlob& bb, Up0Args* u, Down0Args* d0, Down10Args* d10, PadRow* pad,
                   const float* const* d_in, float* const* d_out);
// The level-0 input map of image `img` of bb for a box, at its staging
// buffer when it has one (then use_tma needs the staging copy first).
bool encode_level0_map(const BatchBlob& bb, int img, const float* in, int W, int H, int C, CUtensorMap* m,
                       uint32_t box_w, uint32_t box_h);
// Enqueues the batch's input staging copies (one launch; none without).
cudaError_t launch_batch_pad(const BatchBlob& bb, const unsigned char* d_base, cudaStream_t s);
// The same on the table image inside bb.
void set_blob_io(BatchBlob& bb, const float* const* d_in, float* const* d_out);
// Enqueues the batched stage kernels reading the tables uploaded at d_base.
cudaError_t launch_batch_stages(const std::vector<StageRec>& stages, const unsigned char* d_base,
                                int prec, cudaStream_t s, const int* cps = nullptr);

}  // namespace fllf

// A filter plan (opaque to callers): parameters, float32 coefficients on the
// device, the scratch pyramids, their TMA maps and a device status block.
namespace fllf {
// A staging slot of fllf_submit_host: device copies of one frame's input and
// output, and the events that order the slot's reuse (input copied, frame
// filtered, output copied back).
struct HostSlot {
  float* d_in = nullptr;
  float* d_out = nullptr;
  cudaEvent_t copied_in = nullptr, filtered = nullptr, copied_out = nullptr;
};
constexpr int kHostSlots = 2;
constexpr int kSnapWords = 64;  // host-mapped fault-word snapshots, one per pending host-buffer ticket
}  // namespace fllf

struct fllf_plan {
  fllf_params p{};
  int device = 0;
  std::vector<double> a64;
  float* d_a = nullptr;
  unsigned char* scratch = nullptr;
  size_t scratch_bytes = 0;
  std::vector<fllf::Level> lv;    // device addresses
  float* d_io_in = nullptr;
  float* d_io_out = nullptr;
  fllf::StageTimer* timer = nullptr;  // per-stage timing diagnostics (optional)
  fllf::PathMaps maps;                // TMA tensor maps of the level buffers
  unsigned* d_fault = nullptr;        // device status block (fault word, grid-barrier words)
  float* d_mpyr = nullptr;            // gain-map pyramid of pixel-adaptive runs (first use)
  float* d_luma = nullptr;            // Y and filtered Y of colour-by-luma runs (first use)
  float* d_stage = nullptr;           // input staged at a 16-byte row pitch (W % 4 != 0 only)
  fllf::Tuning tune;                  // launch tuning (fllf_plan_set_tuning / fllf_plan_autotune)
  fllf::PlanGraph* graph = nullptr;   // the plan's dataflow launch (Fourier LLF, >= 2 levels)
  // Host-buffer runs of C >= 2 planes: one-plane views of the scratch (levels
  // and maps) and the copy streams of the plane pipeline (first use).
  std::vector<std::vector<fllf::Level>> plane_lv;
  std::vector<fllf::PathMaps> plane_maps;
  cudaStream_t io_h2d = nullptr, io_d2h = nullptr;
  std::vector<cudaEvent_t> io_ev;     // per plane: input copied, plane filtered
  // fllf_submit_host: staging slots used in turn (first use)
  std::vector<fllf::HostSlot> host_slots;
  int next_slot = 0;
  // fault-word snapshots of pending fllf_submit_host tickets: pinned,
  // device-mapped words and the free ones (guarded by the ticket lock)
  unsigned* h_snap = nullptr;
  unsigned* d_snap = nullptr;
  std::vector<int> snap_free;
};
