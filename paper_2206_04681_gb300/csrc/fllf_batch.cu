// fllf_batch.cu -- batched execution of many plans: one launch per stage kind
// covers every image (uneven sizes, own K / sigma_r / m / levels); the
// launch sequence of a batch object is captured once in a CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"
#include "fllf_launch.h"

namespace fllf {

namespace {

// Work-item counts; these mirror the device-side definitions exactly.
int up0_items_h(const Level& l1, int planes) { return cdiv(l1.w, kUpTW) * cdiv(l1.h, kUpTH) * planes; }
int up_items_h(const Level& dst, int planes, int K, int write_g, int prec) {
  const int kcu = prec == FLLF_FP32 ? Smem<8>::up_kc : Smem<4>::up_kc;
  return cdiv(dst.w, kRsTW) * cdiv(dst.h, kRsTH) * planes * (cdiv(K, kcu) + (write_g ? 1 : 0));
}
int combine_tiles_h(int h, int w, int planes) { return cdiv(w + kDnX0, kDnOW) * cdiv(h, kDnOH) * planes; }
int small_tiles_h(int h, int w, int planes) { return cdiv(w + kDnX0, kSmW) * cdiv(h, kSmH) * planes; }

template <typename T>
size_t push(std::vector<unsigned char>& blob, const T* data, size_t n, size_t align) {
  const size_t off = (blob.size() + align - 1) / align * align;
  blob.resize(off + sizeof(T) * n);
  std::copy(reinterpret_cast<const unsigned char*>(data), reinterpret_cast<const unsigned char*>(data + n),
            blob.begin() + off);
  return off;
}

cudaError_t launch_stage_at(const unsigned char* d_base, const StageRec& st, int prec, cudaStream_t s,
                            int cps) {
  const int* prefix = reinterpret_cast<const int*>(d_base + st.prefix_off);
  switch (st.kind) {
    case kStageUp0: {
      BatchTable<Up0Args> t{reinterpret_cast<const Up0Args*>(d_base + st.args_off), prefix, st.n, st.total};
      return prec == FLLF_FP16 ? launch_up0_batch_f16(t, s, cps)
             : prec == FLLF_BF16 ? launch_up0_batch_bf16(t, s, cps) : launch_up0_batch_f32(t, s, cps);
    }
    case kStageUp: {
      BatchTable<UpArgs> t{reinterpret_cast<const UpArgs*>(d_base + st.args_off), prefix, st.n, st.total};
      return prec == FLLF_FP16 ? launch_up_batch_f16(t, s, cps)
             : prec == FLLF_BF16 ? launch_up_batch_bf16(t, s, cps) : launch_up_batch_f32(t, s, cps);
    }
    case kStageDown: {
      BatchTable<DownArgs> t{reinterpret_cast<const DownArgs*>(d_base + st.args_off), prefix, st.n, st.total};
      return prec == FLLF_FP16 ? launch_down_batch_f16(t, s, cps)
             : prec == FLLF_BF16 ? launch_down_batch_bf16(t, s, cps) : launch_down_batch_f32(t, s, cps);
    }
    case kStageDown10: {
      BatchTable<Down10Args> t{reinterpret_cast<const Down10Args*>(d_base + st.args_off), prefix, st.n,
                               st.total};
      return prec == FLLF_FP16 ? launch_down10_batch_f16(t, s, cps)
             : prec == FLLF_BF16 ? launch_down10_batch_bf16(t, s, cps) : launch_down10_batch_f32(t, s, cps);
    }
    default: {
      BatchTable<Down0Args> t{reinterpret_cast<const Down0Args*>(d_base + st.args_off), prefix, st.n, st.total};
      return prec == FLLF_FP16 ? launch_down0_batch_f16(t, s, cps)
             : prec == FLLF_BF16 ? launch_down0_batch_bf16(t, s, cps) : launch_down0_batch_f32(t, s, cps);
    }
  }
}

}  // namespace

void build_batch_blob(const std::vector<const fllf_plan*>& plans, int prec, BatchBlob* out) {
  out->stages.clear();
  out->up0_img.clear();
  out->down0_img.clear();
  out->down10_img.clear();
  out->copy_img.clear();
  out->up0_off = out->down0_off = out->down10_off = 0;
  std::vector<unsigned char>& blob = out->blob;
  blob.clear();
  int maxL = 1;
  for (const fllf_plan* p : plans) maxL = std::max(maxL, p->p.levels);
  auto add_stage = [&](int kind, const auto& args, const std::vector<int>& counts) {
    if (args.empty()) return;
    StageRec st{};
    st.kind = kind;
    st.n = (int)args.size();
    std::vector<int> pre(st.n + 1, 0);
    for (int j = 0; j < st.n; ++j) pre[j + 1] = pre[j] + counts[j];
    st.total = pre[st.n];
    st.args_off = push(blob, args.data(), args.size(), 128);
    st.prefix_off = push(blob, pre.data(), pre.size(), 16);
    out->stages.push_back(st);
  };
  // A 256-byte status block first (fault word, barrier words).
  const std::vector<unsigned> status(64, 0u);
  out->status_off = push(blob, status.data(), status.size(), 256);
  {
    // input staging of the images whose plans stage their input (rows not
    // 16-byte aligned); the sources are set per run
    out->stage.assign(plans.size(), nullptr);
    out->pad_img.clear();
    out->pad_off = out->pad_prefix_off = 0;
    out->pad_total = 0;
    std::vector<PadRow> rows;
    std::vector<int> pre(1, 0);
    for (int i = 0; i < (int)plans.size(); ++i) {
      const fllf_plan* pl = plans[i];
      if (pl->p.levels < 2 || !pl->d_stage) continue;
      out->stage[i] = pl->d_stage;
      out->pad_img.push_back(i);
      PadRow r{};
      r.dst = pl->d_stage;
      r.W = pl->p.W;
      r.pitch = staged_pitch(pl->p.W);
      r.rows = pl->p.H * pl->p.C;
      rows.push_back(r);
      pre.push_back(pre.back() + r.rows);
    }
    if (!rows.empty()) {
      out->pad_off = push(blob, rows.data(), rows.size(), 64);
      out->pad_prefix_off = push(blob, pre.data(), pre.size(), 16);
      out->pad_total = pre.back();
    }
  }
  {
    std::vector<Up0Args> args;
    std::vector<int> counts;
    for (int i = 0; i < (int)plans.size(); ++i) {
      const fllf_plan* pl = plans[i];
      if (pl->p.levels < 2) {
        out->copy_img.push_back(i);
        continue;
      }
      Up0Args u{};
      u.a = pl->d_a;
      u.h0 = pl->p.H;
      u.w0 = pl->p.W;
      u.planes = pl->p.C;
      u.dst = pl->lv[1];
      u.zstmap = pl->maps.z_st1;
      u.K = pl->p.K;
      u.turns = (float)(2.0 / pl->p.T);
      u.use_tma = 0;  // the input and its map are set per run (set_level0_io)
      args.push_back(u);
      counts.push_back(up0_items_h(pl->lv[1], pl->p.C));
      out->up0_img.push_back(i);
    }
    add_stage(kStageUp0, args, counts);
    if (!args.empty()) out->up0_off = out->stages.back().args_off;
  }
  for (int l = 1; l <= maxL - 2; ++l) {
    std::vector<UpArgs> args;
    std::vector<int> counts;
    for (const fllf_plan* pl : plans) {
      const int L = pl->p.levels;
      if (l > L - 2) continue;
      UpArgs u{};
      u.zmap = pl->maps.z_up[l];
      u.gmap = pl->maps.g_up[l];
      u.src = pl->lv[l];
      u.dst = pl->lv[l + 1];
      u.planes = pl->p.C;
      u.K = pl->p.K;
      u.write_g = (l + 1 <= L - 2) ? 1 : 0;
      args.push_back(u);
      counts.push_back(up_items_h(pl->lv[l + 1], pl->p.C, pl->p.K, u.write_g, prec));
    }
    add_stage(kStageUp, args, counts);
  }
  // combines at levels >= 2 (level 1 runs inside the fused level-0 stage of
  // the images with >= 3 levels; images with 2 levels combine level 0 only)
  for (int l = maxL - 2; l >= 2; --l) {
    std::vector<DownArgs> args;
    std::vector<int> counts;
    for (const fllf_plan* pl : plans) {
      const int L = pl->p.levels;
      if (l > L - 2) continue;
      DownArgs d{};   // the 32 x 16 tiles of the batched combine
      d.zmap = pl->maps.z_cs[l + 1];
      d.emap = pl->maps.e_cs[l + 1];
      d.zfmap = pl->maps.z_fs[l];
      d.gfmap = pl->maps.g_fs[l];
      d.fine = pl->lv[l];
      d.coarse = pl->lv[l + 1];
      d.planes = pl->p.C;
      d.K = pl->p.K;
      d.turns = (float)(2.0 / pl->p.T);
      d.has_e = (l + 1 <= L - 2) ? 1 : 0;
      args.push_back(d);
      counts.push_back(small_tiles_h(pl->lv[l].h, pl->lv[l].w, pl->p.C));
    }
    add_stage(kStageDown, args, counts);
  }
  {
    std::vector<Down10Args> a10;
    std::vector<int> c10;
    std::vector<Down0Args> args;
    std::vector<int> counts;
    for (int idx : out->up0_img) {
      const fllf_plan* pl = plans[idx];
      if (pl->p.levels >= 3) {
        Down10Args d{};
        d.z1map = pl->maps.z_dn[1];
        d.g1map = pl->maps.g1_d10;
        d.z2map = pl->maps.z2_d10;
        d.e2map = pl->maps.e2_d10;
        d.h0 = pl->p.H;
        d.w0 = pl->p.W;
        d.planes = pl->p.C;
        d.l1 = pl->lv[1];
        d.l2 = pl->lv[2];
        d.K = pl->p.K;
        d.turns = (float)(2.0 / pl->p.T);
        d.has_e2 = pl->p.levels >= 4 ? 1 : 0;
        d.use_tma = 0;  // the input and its map are set per run (set_level0_io)
        a10.push_back(d);
        c10.push_back(combine_tiles_h(pl->p.H, pl->p.W, pl->p.C));
        out->down10_img.push_back(idx);
        continue;
      }
      Down0Args d{};
      d.zmap = pl->maps.z_dn[1];
      d.emap = pl->maps.e_dn[1];
      d.h0 = pl->p.H;
      d.w0 = pl->p.W;
      d.planes = pl->p.C;
      d.coarse = pl->lv[1];
      d.K = pl->p.K;
      d.turns = (float)(2.0 / pl->p.T);
      d.has_e = pl->p.levels >= 3 ? 1 : 0;
      args.push_back(d);
      counts.push_back(combine_tiles_h(pl->p.H, pl->p.W, pl->p.C));
      out->down0_img.push_back(idx);
    }
    add_stage(kStageDown10, a10, c10);
    if (!a10.empty()) out->down10_off = out->stages.back().args_off;
    add_stage(kStageDown0, args, counts);
    if (!args.empty()) out->down0_off = out->stages.back().args_off;
  }
}

void set_blob_fault(BatchBlob& bb, unsigned* d_fault) {
  for (const StageRec& st : bb.stages) {
    unsigned char* base = bb.blob.data() + st.args_off;
    for (int j = 0; j < st.n; ++j) {
      switch (st.kind) {
        case kStageUp0: reinterpret_cast<Up0Args*>(base)[j].fault = d_fault; break;
        case kStageUp: reinterpret_cast<UpArgs*>(base)[j].fault = d_fault; break;
        case kStageDown: reinterpret_cast<DownArgs*>(base)[j].fault = d_fault; break;
        case kStageDown10: reinterpret_cast<Down10Args*>(base)[j].fault = d_fault; break;
        default: reinterpret_cast<Down0Args*>(base)[j].fault = d_fault; break;
      }
    }
  }
}

bool encode_level0_map(const BatchBlob& bb, int img, const float* in, int W, int H, int C, CUtensorMap* m,
                       uint32_t box_w, uint32_t box_h) {
  float* st = img < (int)bb.stage.size() ? bb.stage[img] : nullptr;
  return st ? encode_image_map(m, st, W, H, C, box_w, box_h, staged_pitch(W))
            : encode_image_map(m, in, W, H, C, box_w, box_h);
}

void set_level0_io(const BatchBlob& bb, Up0Args* u, Down0Args* d0, Down10Args* d10, PadRow* pad,
                   const float* const* d_in, float* const* d_out) {
  // the input's maps for the level-0 REDUCE and the fused combine are encoded
  // per run (the kernels order them for the tensor-map proxy before use), at
  // the staging copy for images that have one; where the image allows no
  // map, the kernels read the input with plain loads
  for (size_t j = 0; j < bb.up0_img.size(); ++j) {
    Up0Args& a = u[j];
    a.I = d_in[bb.up0_img[j]];
    a.use_tma = encode_level0_map(bb, bb.up0_img[j], a.I, a.w0, a.h0, a.planes, &a.imap, kUpIW, kUpIR) ? 1 : 0;
  }
  for (size_t j = 0; j < bb.down0_img.size(); ++j) {
    d0[j].I = d_in[bb.down0_img[j]];
    d0[j].O = d_out[bb.down0_img[j]];
  }
  for (size_t j = 0; j < bb.down10_img.size(); ++j) {
    Down10Args& a = d10[j];
    a.I = d_in[bb.down10_img[j]];
    a.O = d_out[bb.down10_img[j]];
    a.use_tma =
        encode_level0_map(bb, bb.down10_img[j], a.I, a.w0, a.h0, a.planes, &a.imap, kD0IW, kDnOH) ? 1 : 0;
  }
  if (pad)
    for (size_t j = 0; j < bb.pad_img.size(); ++j) pad[j].src = d_in[bb.pad_img[j]];
}

void set_blob_io(BatchBlob& bb, const float* const* d_in, float* const* d_out) {
  unsigned char* b = bb.blob.data();
  set_level0_io(bb, reinterpret_cast<Up0Args*>(b + bb.up0_off), reinterpret_cast<Down0Args*>(b + bb.down0_off),
                reinterpret_cast<Down10Args*>(b + bb.down10_off),
                bb.pad_img.empty() ? nullptr : reinterpret_cast<PadRow*>(b + bb.pad_off), d_in, d_out);
}

cudaError_t launch_batch_pad(const BatchBlob& bb, const unsigned char* d_base, cudaStream_t s) {
  if (bb.pad_img.empty()) return cudaSuccess;
  return launch_pad_batch(reinterpret_cast<const PadRow*>(d_base + bb.pad_off),
                          reinterpret_cast<const int*>(d_base + bb.pad_prefix_off), (int)bb.pad_img.size(),
                          bb.pad_total, s);
}

cudaError_t launch_batch_stages(const std::vector<StageRec>& stages, const unsigned char* d_base,
                                int prec, cudaStream_t s, const int* cps) {
  for (const StageRec& st : stages) {
    const int ck = st.kind == kStageDown10 ? kStageDown0 : st.kind;
    const cudaError_t e = launch_stage_at(d_base, st, prec, s, cps ? cps[ck] : 0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace fllf

using namespace fllf;

namespace {

fllf_status bfail(fllf_status s, const std::string& why) {
  set_last_error(why);
  return s;
}

struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int dev) {
    cudaGetDevice(&prev);
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

struct fllf_batch {
  std::vector<fllf_plan*> plans;
  int device = 0, precision = 0;
  BatchBlob bb;
  unsigned char* d_mem = nullptr;  // device copy of the tables
  unsigned* d_fault = nullptr;
  Up0Args* h_up0 = nullptr;        // pinned per-run mirrors of the level-0 tables
  Down0Args* h_down0 = nullptr;
  Down10Args* h_down10 = nullptr;
  PadRow* h_pad = nullptr;         // pinned per-run mirror of the input staging table
  cudaEvent_t copied = nullptr;
  bool copied_pending = false;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  int cps[4] = {0, 0, 0, 0};       // resident-CTA cap per batched stage kind (0: as many as fit)
  // the launch mode (0, the default, measured faster on mixed batches: one
  // launch per stage kind and level; 1: the dataflow launch, every stage of
  // every image in one launch; 2: the same without the fused level-1/level-0
  // combine, which follows as one batched launch)
  int mode = 0;
  GraphGrain grain;
  GraphBuild flow;
  unsigned char* d_flow = nullptr;
  size_t flow_prefix_off = 0;      // tile prefix sums of the fused combine's table (mode 2)
  Up0Args* h_fup0 = nullptr;       // pinned per-run mirrors of the dataflow's level-0 tables
  Down10Args* h_fd10 = nullptr;
  Down0Args* h_fd0 = nullptr;
};

static void free_flow(fllf_batch* b) {
  if (b->d_flow) cudaFree(b->d_flow);
  if (b->h_fup0) cudaFreeHost(b->h_fup0);
  if (b->h_fd10) cudaFreeHost(b->h_fd10);
  if (b->h_fd0) cudaFreeHost(b->h_fd0);
  b->d_flow = nullptr;
  b->h_fup0 = nullptr;
  b->h_fd10 = nullptr;
  b->h_fd0 = nullptr;
  b->flow = GraphBuild{};
}

// Builds and uploads the batch's dataflow task list for its mode and grain.
static fllf_status build_flow(fllf_batch* b) {
  free_flow(b);
  std::vector<const fllf_plan*> plans(b->plans.begin(), b->plans.end());
  build_graph(plans, b->precision, b->grain, false, b->mode != 2, &b->flow);
  if (!b->flow.ok) return bfail(FLLF_EINVAL, "internal error: dataflow task list");
  // tile prefix sums of the fused combine's table, for its batched launch
  std::vector<int> pre(b->flow.n_d10 + 1, 0);
  for (int j = 0; j < b->flow.n_d10; ++j) {
    const fllf_params& p = b->plans[b->flow.d10_img[j]]->p;
    pre[j + 1] = pre[j] + cdiv(p.W + kDnX0, kDnOW) * cdiv(p.H, kDnOH) * p.C;
  }
  b->flow_prefix_off = push(b->flow.blob, pre.data(), pre.size(), 16);
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_flow, b->flow.blob.size())) != cudaSuccess) {
    cudaGetLastError();
    b->d_flow = nullptr;
    return bfail(FLLF_ENOMEM, "dataflow table allocation failed");
  }
  // every argument block's fault word is the batch's
  unsigned char* hb = b->flow.blob.data();
  auto fault = [&](auto* a, int n) {
    for (int j = 0; j < n; ++j) a[j].fault = b->d_fault;
  };
  fault(reinterpret_cast<Up0Args*>(hb + b->flow.up0_off), b->flow.n_up0);
  fault(reinterpret_cast<UpArgs*>(hb + b->flow.ups_off), b->flow.n_ups);
  fault(reinterpret_cast<DownArgs*>(hb + b->flow.dns_off), b->flow.n_dns);
  fault(reinterpret_cast<Down10Args*>(hb + b->flow.d10_off), b->flow.n_d10);
  fault(reinterpret_cast<Down0Args*>(hb + b->flow.d0_off), b->flow.n_d0);
  if ((e = cudaMemcpy(b->d_flow, hb, b->flow.blob.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return bfail(FLLF_ECUDA, std::string("dataflow table upload: ") + cudaGetErrorString(e));
  const size_t n0 = std::max(1, b->flow.n_up0), n10 = std::max(1, b->flow.n_d10), nd0 = std::max(1, b->flow.n_d0);
  if (cudaMallocHost(&b->h_fup0, sizeof(Up0Args) * n0) != cudaSuccess ||
      cudaMallocHost(&b->h_fd10, sizeof(Down10Args) * n10) != cudaSuccess ||
      cudaMallocHost(&b->h_fd0, sizeof(Down0Args) * nd0) != cudaSuccess) {
    cudaGetLastError();
    return bfail(FLLF_ENOMEM, "pinned dataflow tables");
  }
  std::copy(reinterpret_cast<const Up0Args*>(hb + b->flow.up0_off),
            reinterpret_cast<const Up0Args*>(hb + b->flow.up0_off) + b->flow.n_up0, b->h_fup0);
  std::copy(reinterpret_cast<const Down10Args*>(hb + b->flow.d10_off),
            reinterpret_cast<const Down10Args*>(hb + b->flow.d10_off) + b->flow.n_d10, b->h_fd10);
  std::copy(reinterpret_cast<const Down0Args*>(hb + b->flow.d0_off),
            reinterpret_cast<const Down0Args*>(hb + b->flow.d0_off) + b->flow.n_d0, b->h_fd0);
  return FLLF_OK;
}

// The dataflow launch of the batch (and, in mode 2, the batched fused combine).
static cudaError_t launch_flow(fllf_batch* b, cudaStream_t s) {
  GraphArgs g = graph_args(b->flow, b->d_flow, b->d_fault);
  const bool with_d10 = b->mode != 2;
  cudaError_t e = launch_graph(b->precision, g, sizeof(unsigned) * b->flow.rt_words, s, b->cps[kStageUp0], with_d10);
  if (e != cudaSuccess || with_d10 || b->flow.n_d10 == 0) return e;
  const int* pre = reinterpret_cast<const int*>(b->d_flow + b->flow_prefix_off);
  const int total = reinterpret_cast<const int*>(b->flow.blob.data() + b->flow_prefix_off)[b->flow.n_d10];
  BatchTable<Down10Args> t{g.d10s, pre, b->flow.n_d10, total};
  switch (b->precision) {
    case FLLF_FP16: return launch_down10_batch_f16(t, s, b->cps[kStageDown0]);
    case FLLF_BF16: return launch_down10_batch_bf16(t, s, b->cps[kStageDown0]);
    default: return launch_down10_batch_f32(t, s, b->cps[kStageDown0]);
  }
}

static void free_batch(fllf_batch* b) {
  if (!b) return;
  free_flow(b);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->copied) cudaEventDestroy(b->copied);
  if (b->h_up0) cudaFreeHost(b->h_up0);
  if (b->h_down0) cudaFreeHost(b->h_down0);
  if (b->h_down10) cudaFreeHost(b->h_down10);
  if (b->h_pad) cudaFreeHost(b->h_pad);
  if (b->d_mem) cudaFree(b->d_mem);
  delete b;
}

extern "C" {

fllf_status fllf_batch_create(fllf_plan* const* plans, int n, fllf_batch** out) {
  if (!out) return bfail(FLLF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!plans || n < 1 || n > 4096) return bfail(FLLF_EINVAL, "need 1..4096 plans");
  for (int i = 0; i < n; ++i)
    if (!plans[i]) return bfail(FLLF_EINVAL, "plan is NULL");
  const int dev = plans[0]->device, prec = plans[0]->p.precision;
  for (int i = 1; i < n; ++i)
    if (plans[i]->device != dev || plans[i]->p.precision != prec)
      return bfail(FLLF_EINVAL, "all plans of a batch need the same device and precision");
  for (int i = 0; i < n; ++i)
    if (plans[i]->p.method != FLLF_METHOD_FOURIER) return bfail(FLLF_EINVAL, "batches hold Fourier LLF plans only");
  DeviceScope scope(dev);
  if (!scope.ok) return bfail(FLLF_ECUDA, "cudaSetDevice failed");
  fllf_batch* b = new (std::nothrow) fllf_batch();
  if (!b) return bfail(FLLF_ENOMEM, "batch allocation failed");
  b->plans.assign(plans, plans + n);
  b->device = dev;
  b->precision = prec;
  build_batch_blob(std::vector<const fllf_plan*>(plans, plans + n), prec, &b->bb);
  cudaError_t e;
  if ((e = cudaMalloc(&b->d_mem, b->bb.blob.size())) != cudaSuccess) {
    cudaGetLastError();
    b->d_mem = nullptr;
    free_batch(b);
    return bfail(FLLF_ENOMEM, "batch table allocation failed");
  }
  b->d_fault = reinterpret_cast<unsigned*>(b->d_mem + b->bb.status_off);
  set_blob_fault(b->bb, b->d_fault);
  if ((e = cudaMemcpy(b->d_mem, b->bb.blob.data(), b->bb.blob.size(), cudaMemcpyHostToDevice)) !=
      cudaSuccess) {
    free_batch(b);
    return bfail(FLLF_ECUDA, std::string("batch table upload: ") + cudaGetErrorString(e));
  }
  const size_t nu = std::max<size_t>(1, b->bb.up0_img.size());
  if (cudaMallocHost(&b->h_up0, sizeof(Up0Args) * nu) != cudaSuccess ||
      cudaMallocHost(&b->h_down0, sizeof(Down0Args) * nu) != cudaSuccess ||
      cudaMallocHost(&b->h_down10, sizeof(Down10Args) * nu) != cudaSuccess ||
      cudaMallocHost(&b->h_pad, sizeof(PadRow) * std::max<size_t>(1, b->bb.pad_img.size())) != cudaSuccess) {
    cudaGetLastError();
    free_batch(b);
    return bfail(FLLF_ENOMEM, "pinned host tables");
  }
  if (!b->bb.up0_img.empty()) {
    const Up0Args* u = reinterpret_cast<const Up0Args*>(b->bb.blob.data() + b->bb.up0_off);
    const Down0Args* d = reinterpret_cast<const Down0Args*>(b->bb.blob.data() + b->bb.down0_off);
    const Down10Args* f = reinterpret_cast<const Down10Args*>(b->bb.blob.data() + b->bb.down10_off);
    std::copy(u, u + b->bb.up0_img.size(), b->h_up0);
    std::copy(d, d + b->bb.down0_img.size(), b->h_down0);
    std::copy(f, f + b->bb.down10_img.size(), b->h_down10);
  }
  if (!b->bb.pad_img.empty()) {
    const PadRow* r = reinterpret_cast<const PadRow*>(b->bb.blob.data() + b->bb.pad_off);
    std::copy(r, r + b->bb.pad_img.size(), b->h_pad);
  }
  if (cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    free_batch(b);
    return bfail(FLLF_ECUDA, "batch event / stream creation failed");
  }
  const fllf_status fs = build_flow(b);
  if (fs != FLLF_OK) {
    const std::string why = fllf_last_error();
    free_batch(b);
    return bfail(fs, why);
  }
  *out = b;
  return FLLF_OK;
}

fllf_status fllf_batch_destroy(fllf_batch* b) {
  if (!b) return FLLF_OK;
  DeviceScope scope(b->device);
  free_batch(b);
  return FLLF_OK;
}

fllf_status fllf_batch_run(fllf_batch* b, const float* const* d_in, float* const* d_out, void* stream) {
  if (!b || !d_in || !d_out) return bfail(FLLF_EINVAL, "batch, d_in or d_out is NULL");
  const int n = (int)b->plans.size();
  for (int i = 0; i < n; ++i) {
    if (!d_in[i] || !d_out[i]) return bfail(FLLF_EINVAL, "an image pointer is NULL");
    const fllf_params& p = b->plans[i]->p;
    const size_t bytes = sizeof(float) * (size_t)p.H * p.W * p.C;
    const char *x = reinterpret_cast<const char*>(d_in[i]), *y = reinterpret_cast<const char*>(d_out[i]);
    if (x < y + bytes && y < x + bytes) return bfail(FLLF_EINVAL, "input and output buffers overlap");
  }
  DeviceScope scope(b->device);
  if (!scope.ok) return bfail(FLLF_ECUDA, "cudaSetDevice failed");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  // The pinned mirrors may still feed the previous run's copies.
  if (b->copied_pending && (e = cudaEventSynchronize(b->copied)) != cudaSuccess)
    return bfail(FLLF_ECUDA, std::string("batch copy wait: ") + cudaGetErrorString(e));
  const BatchBlob& bb = b->bb;
  if (b->mode == 0) {
    set_level0_io(bb, b->h_up0, b->h_down0, b->h_down10, b->h_pad, d_in, d_out);
    auto upload = [&](size_t off, const void* src, size_t bytes) {
      return bytes ? cudaMemcpyAsync(b->d_mem + off, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    if ((e = upload(bb.up0_off, b->h_up0, sizeof(Up0Args) * bb.up0_img.size())) != cudaSuccess ||
        (e = upload(bb.down0_off, b->h_down0, sizeof(Down0Args) * bb.down0_img.size())) != cudaSuccess ||
        (e = upload(bb.down10_off, b->h_down10, sizeof(Down10Args) * bb.down10_img.size())) != cudaSuccess)
      return bfail(FLLF_ECUDA, std::string("batch table update: ") + cudaGetErrorString(e));
  } else {
    // the dataflow tables' level-0 blocks: this run's inputs, outputs and input maps
    const GraphBuild& f = b->flow;
    for (int j = 0; j < f.n_up0; ++j) {
      Up0Args& a = b->h_fup0[j];
      a.I = d_in[f.up0_img[j]];
      a.use_tma = encode_level0_map(bb, f.up0_img[j], a.I, a.w0, a.h0, a.planes, &a.imap, kUpIW, kUpIR) ? 1 : 0;
    }
    for (int j = 0; j < f.n_d10; ++j) {
      Down10Args& a = b->h_fd10[j];
      a.I = d_in[f.d10_img[j]];
      a.O = d_out[f.d10_img[j]];
      a.use_tma =
          encode_level0_map(bb, f.d10_img[j], a.I, a.w0, a.h0, a.planes, &a.imap, kD0IW, kDnOH) ? 1 : 0;
    }
    for (int j = 0; j < f.n_d0; ++j) {
      b->h_fd0[j].I = d_in[f.d0_img[j]];
      b->h_fd0[j].O = d_out[f.d0_img[j]];
    }
    auto upload = [&](size_t off, const void* src, size_t bytes) {
      return bytes ? cudaMemcpyAsync(b->d_flow + off, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    if ((e = upload(f.up0_off, b->h_fup0, sizeof(Up0Args) * f.n_up0)) != cudaSuccess ||
        (e = upload(f.d10_off, b->h_fd10, sizeof(Down10Args) * f.n_d10)) != cudaSuccess ||
        (e = upload(f.d0_off, b->h_fd0, sizeof(Down0Args) * f.n_d0)) != cudaSuccess)
      return bfail(FLLF_ECUDA, std::string("batch table update: ") + cudaGetErrorString(e));
  }
  if (!bb.pad_img.empty()) {
    // this run's staging sources
    for (size_t j = 0; j < bb.pad_img.size(); ++j) b->h_pad[j].src = d_in[bb.pad_img[j]];
    if ((e = cudaMemcpyAsync(b->d_mem + bb.pad_off, b->h_pad, sizeof(PadRow) * bb.pad_img.size(),
                             cudaMemcpyHostToDevice, s)) != cudaSuccess)
      return bfail(FLLF_ECUDA, std::string("batch table update: ") + cudaGetErrorString(e));
  }
  if ((e = cudaEventRecord(b->copied, s)) != cudaSuccess)
    return bfail(FLLF_ECUDA, std::string("batch event: ") + cudaGetErrorString(e));
  b->copied_pending = true;
  for (int i : bb.copy_img) {
    const fllf_params& p = b->plans[i]->p;
    if ((e = cudaMemcpyAsync(d_out[i], d_in[i], sizeof(float) * (size_t)p.H * p.W * p.C,
                             cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      return bfail(FLLF_ECUDA, std::string("single-level copy: ") + cudaGetErrorString(e));
  }
  if (bb.stages.empty()) return FLLF_OK;
  if (!b->graph) {
    // Capture the launch sequence once; the tables are read from device
    // memory, so the graph stays valid for every later run.
    cudaGraph_t g = nullptr;
    if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
      return bfail(FLLF_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaError_t le = launch_batch_pad(bb, b->d_mem, b->cap);
    if (le == cudaSuccess)
      le = b->mode == 0 ? launch_batch_stages(bb.stages, b->d_mem, b->precision, b->cap, b->cps)
                        : launch_flow(b, b->cap);
    e = cudaStreamEndCapture(b->cap, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return bfail(FLLF_ECUDA, std::string("graph capture: ") +
                                   cudaGetErrorString(le != cudaSuccess ? le : e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return bfail(FLLF_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
  }
  if ((e = cudaGraphLaunch(b->graph, s)) != cudaSuccess)
    return bfail(FLLF_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
  return FLLF_OK;
}

fllf_status fllf_batch_get_mode(const fllf_batch* b, int* mode, int* task_items) {
  if (!b || !mode) return bfail(FLLF_EINVAL, "batch or mode is NULL");
  *mode = b->mode;
  if (task_items) {
    const int g[5] = {b->grain.up0, b->grain.up, b->grain.dns, b->grain.d10, b->grain.d0};
    std::copy(g, g + 5, task_items);
  }
  return FLLF_OK;
}

fllf_status fllf_batch_set_mode(fllf_batch* b, int mode, const int* task_items) {
  if (!b) return bfail(FLLF_EINVAL, "batch is NULL");
  if (mode < 0 || mode > 2) return bfail(FLLF_EINVAL, "mode must be 0, 1 or 2");
  GraphGrain g = b->grain;
  if (task_items) {
    for (int k = 0; k < 5; ++k)
      if (task_items[k] < 1 || task_items[k] > 4096) return bfail(FLLF_EINVAL, "task_items must be 1..4096");
    g.up0 = task_items[0];
    g.up = task_items[1];
    g.dns = task_items[2];
    g.d10 = task_items[3];
    g.d0 = task_items[4];
  }
  const bool regrain = g.up0 != b->grain.up0 || g.up != b->grain.up || g.dns != b->grain.dns ||
                       g.d10 != b->grain.d10 || g.d0 != b->grain.d0 || ((mode == 2) != (b->mode == 2));
  if (mode == b->mode && !regrain) return FLLF_OK;
  DeviceScope scope(b->device);
  // the launch sequence is captured in the graph, and the tables may be in use
  cudaDeviceSynchronize();
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->copied_pending = false;
  b->mode = mode;
  b->grain = g;
  if (regrain) return build_flow(b);
  return FLLF_OK;
}

fllf_status fllf_batch_get_ctas(const fllf_batch* b, int* ctas_per_sm) {
  if (!b || !ctas_per_sm) return bfail(FLLF_EINVAL, "batch or ctas_per_sm is NULL");
  std::copy(b->cps, b->cps + 4, ctas_per_sm);
  return FLLF_OK;
}

fllf_status fllf_batch_set_ctas(fllf_batch* b, const int* ctas_per_sm) {
  if (!b || !ctas_per_sm) return bfail(FLLF_EINVAL, "batch or ctas_per_sm is NULL");
  for (int k = 0; k < 4; ++k)
    if (ctas_per_sm[k] < 0 || ctas_per_sm[k] > 32) return bfail(FLLF_EINVAL, "ctas_per_sm must be 0..32");
  if (!std::equal(ctas_per_sm, ctas_per_sm + 4, b->cps)) {
    DeviceScope scope(b->device);
    // the launch shapes are baked into the captured graph: capture again
    if (b->graph) {
      cudaStreamSynchronize(b->cap);
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    std::copy(ctas_per_sm, ctas_per_sm + 4, b->cps);
  }
  return FLLF_OK;
}

fllf_status fllf_batch_autotune(fllf_batch* b, const float* const* d_in, float* const* d_out, int reps,
                                void* stream, double* best_ms) {
  if (!b || !d_in || !d_out) return bfail(FLLF_EINVAL, "batch, d_in or d_out is NULL");
  if (reps < 1 || reps > 10000) return bfail(FLLF_EINVAL, "reps must be 1..10000");
  DeviceScope scope(b->device);
  if (!scope.ok) return bfail(FLLF_ECUDA, "cudaSetDevice failed");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return bfail(FLLF_ECUDA, "autotune: event creation failed");
  }
  // L2 flush before every timed run (twice the L2, allocated for the search)
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device);
  const size_t fbytes = 2 * (size_t)(l2 > 0 ? l2 : (64 << 20));
  void* flush = nullptr;
  if (cudaMalloc(&flush, fbytes) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return bfail(FLLF_ENOMEM, "autotune: the L2 flush buffer could not be allocated");
  }
  // ms per batched run with the given caps (negative on failure)
  auto measure = [&](const int* cps) -> double {
    if (fllf_batch_set_ctas(b, cps) != FLLF_OK) return -1.0;
    if (fllf_batch_run(b, d_in, d_out, stream) != FLLF_OK) return -1.0;  // captures the graph
    double sum = 0.0;
    for (int i = 0; i < reps; ++i) {
      float t = 0.f;
      if (cudaMemsetAsync(flush, i & 0xff, fbytes, s) != cudaSuccess || cudaEventRecord(e0, s) != cudaSuccess ||
          fllf_batch_run(b, d_in, d_out, stream) != FLLF_OK || cudaEventRecord(e1, s) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)
        return -1.0;
      sum += t;
    }
    return sum / reps;
  };
  int best[4];
  std::copy(b->cps, b->cps + 4, best);
  double best_t = measure(best);
  bool ok = best_t >= 0;
  // 1. the launch mode (one launch per stage kind and level, the dataflow
  // launch, the dataflow launch followed by the batched fused combine), each
  // with every CTA cap at "as many as fit"
  {
    int mode_best = b->mode;
    const int zero[4] = {0, 0, 0, 0};
    for (int m = 0; m <= 2 && ok; ++m) {
      if (m == mode_best) continue;
      const int prev = b->mode;
      ok = fllf_batch_set_mode(b, m, nullptr) == FLLF_OK;
      const double t = ok ? measure(zero) : -1.0;
      ok = ok && t >= 0;
      if (ok && t < 0.99 * best_t) {
        mode_best = m;
        best_t = t;
        std::copy(zero, zero + 4, best);
      } else if (ok) {
        ok = fllf_batch_set_mode(b, prev, nullptr) == FLLF_OK;
      }
    }
    if (ok) ok = fllf_batch_set_mode(b, mode_best, nullptr) == FLLF_OK && fllf_batch_set_ctas(b, best) == FLLF_OK;
  }
  // 2. the CTA caps of the kinds the mode launches (the dataflow kernel takes
  // the first cap, its batched fused combine the fourth)
  for (int kind = 0; kind < 4 && ok; ++kind) {
    if (b->mode != 0 && kind != 0 && !(b->mode == 2 && kind == 3)) continue;
    const int occ = b->mode != 0 && kind == 0 ? stage_occupancy(b->precision, FLLF_STAGE_GRAPH, false)
                                              : stage_occupancy(b->precision, kind, true);
    for (int c = 1; c <= occ && ok; ++c) {
      int t[4];
      std::copy(best, best + 4, t);
      t[kind] = c == occ ? 0 : c;
      if (t[kind] == best[kind]) continue;
      const double m = measure(t);
      ok = m >= 0;
      if (ok && m < 0.99 * best_t) {   // at least 1% faster
        std::copy(t, t + 4, best);
        best_t = m;
      }
    }
  }
  if (ok) ok = fllf_batch_set_ctas(b, best) == FLLF_OK;
  // 3. the dataflow launch's task sizes
  if (ok && b->mode != 0) {
    const std::vector<std::vector<int>> cand = {{1, 2, 4, 8, 16}, {2, 4, 8, 16, 32}, {1, 2, 4, 8}, {1, 2, 4}};
    for (int k = 0; k < 4 && ok; ++k)
      for (int v : cand[k]) {
        int cur[5];
        int mode = 0;
        fllf_batch_get_mode(b, &mode, cur);
        if (cur[k] == v) continue;
        int t[5];
        std::copy(cur, cur + 5, t);
        t[k] = v;
        ok = fllf_batch_set_mode(b, mode, t) == FLLF_OK;
        const double m = ok ? measure(best) : -1.0;
        ok = ok && m >= 0;
        if (ok && m < 0.99 * best_t) best_t = m;
        else if (ok) ok = fllf_batch_set_mode(b, mode, cur) == FLLF_OK;
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(flush);
  const fllf_status st = ok ? fllf_batch_set_ctas(b, best) : FLLF_ECUDA;
  if (!ok) return bfail(FLLF_ECUDA, "autotune: a timed batched run failed");
  if (best_ms) *best_ms = best_t;
  return st;
}

fllf_status fllf_batch_check(fllf_batch* b) {
  if (!b) return bfail(FLLF_EINVAL, "batch is NULL");
  DeviceScope scope(b->device);
  unsigned f = 0;
  const cudaError_t e = cudaMemcpy(&f, b->d_fault, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bfail(FLLF_ECUDA, std::string("fault word read: ") + cudaGetErrorString(e));
  if (f) {
    cudaMemset(b->d_fault, 0, 256);
    return bfail(FLLF_ETIMEOUT, "a kernel's bounded wait for a shared-memory copy ran out");
  }
  return FLLF_OK;
}

fllf_status fllf_batch_run_plans(fllf_plan* const* plans, const float* const* d_in, float* const* d_out, int n,
                                 void* stream) {
  fllf_batch* b = nullptr;
  fllf_status st = fllf_batch_create(plans, n, &b);
  if (st != FLLF_OK) return st;
  st = fllf_batch_run(b, d_in, d_out, stream);
  if (st == FLLF_OK) {
    DeviceScope scope(b->device);
    const cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    st = e != cudaSuccess ? bfail(FLLF_ECUDA, std::string("stream synchronize: ") + cudaGetErrorString(e))
                          : fllf_batch_check(b);
  } else {
    // the tables may be in use by work already enqueued before the failure
    DeviceScope scope(b->device);
    cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  }
  const std::string keep = st == FLLF_OK ? std::string() : std::string(fllf_last_error());
  fllf_batch_destroy(b);
  if (st != FLLF_OK) return bfail(st, keep);
  return FLLF_OK;
}

}  // extern "C"
