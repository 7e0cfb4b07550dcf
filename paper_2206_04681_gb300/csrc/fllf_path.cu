// fllf_path.cu -- host side of the path: TMA tensor maps of the pyramid
// levels and the launch sequence of one image (up pass, then down pass).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"
#include "fllf_launch.h"

namespace fllf {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D tiled map (x = column, y = row, z = plane) with zero fill outside.
// 4-D tiled map of a Fourier level (x = column, y = row, z = order, w = plane).
bool encode4(CUtensorMap* m, CUtensorMapDataType dt, const void* base, uint64_t w, uint64_t h,
             uint64_t K, uint64_t planes, uint64_t row_bytes, uint64_t order_bytes, uint64_t plane_bytes,
             uint32_t bx, uint32_t by, uint32_t bz) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[4] = {w, h, K, planes};
  cuuint64_t strides[3] = {row_bytes, order_bytes, plane_bytes};
  cuuint32_t box[4] = {bx, by, bz, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, dt, 4, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode3(CUtensorMap* m, CUtensorMapDataType dt, size_t esize, const void* base, uint64_t w,
             uint64_t h, uint64_t planes, uint64_t row_bytes, uint64_t plane_bytes, uint32_t bx,
             uint32_t by, uint32_t bz) {
  auto enc = encoder();
  if (!enc) return false;
  cuuint64_t dims[3] = {w, h, planes};
  cuuint64_t strides[2] = {row_bytes, plane_bytes};
  cuuint32_t box[3] = {bx, by, bz};
  cuuint32_t estr[3] = {1, 1, 1};
  (void)esize;
  return enc(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t launch_up0(int prec, const Up0Args& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_up0_f16(a, s, cps);
    case FLLF_BF16: return launch_up0_bf16(a, s, cps);
    default: return launch_up0_f32(a, s, cps);
  }
}
cudaError_t launch_up(int prec, const UpArgs& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_up_f16(a, s, cps);
    case FLLF_BF16: return launch_up_bf16(a, s, cps);
    default: return launch_up_f32(a, s, cps);
  }
}
cudaError_t launch_down(int prec, const DownArgs& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_down_f16(a, s, cps);
    case FLLF_BF16: return launch_down_bf16(a, s, cps);
    default: return launch_down_f32(a, s, cps);
  }
}
cudaError_t launch_down_s(int prec, const DownArgs& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_down_s_f16(a, s, cps);
    case FLLF_BF16: return launch_down_s_bf16(a, s, cps);
    default: return launch_down_s_f32(a, s, cps);
  }
}
cudaError_t launch_chain(int prec, const ChainArgs& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_chain_f16(a, s, cps);
    case FLLF_BF16: return launch_chain_bf16(a, s, cps);
    default: return launch_chain_f32(a, s, cps);
  }
}
cudaError_t launch_down10(int prec, const Down10Args& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_down10_f16(a, s, cps);
    case FLLF_BF16: return launch_down10_bf16(a, s, cps);
    default: return launch_down10_f32(a, s, cps);
  }
}
cudaError_t launch_down0(int prec, const Down0Args& a, cudaStream_t s, int cps) {
  switch (prec) {
    case FLLF_FP16: return launch_down0_f16(a, s, cps);
    case FLLF_BF16: return launch_down0_bf16(a, s, cps);
    default: return launch_down0_f32(a, s, cps);
  }
}

}  // namespace

int stage_occupancy(int prec, int kind, bool batched) {
  switch (prec) {
    case FLLF_FP16: return launch_occupancy_f16(kind, batched ? 1 : 0);
    case FLLF_BF16: return launch_occupancy_bf16(kind, batched ? 1 : 0);
    default: return launch_occupancy_f32(kind, batched ? 1 : 0);
  }
}

bool encode_image_map(CUtensorMap* m, const float* base, int W, int H, int C, uint32_t box_w, uint32_t box_h,
                      int pitch) {
  if (pitch <= 0) pitch = W;
  if ((pitch % 4) != 0 || pitch < W || (reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
  return encode3(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, W, H, C, 4ull * pitch, 4ull * pitch * H, box_w,
                 box_h, 1);
}

bool build_maps(const fllf_params& p, const std::vector<Level>& lv, PathMaps* m) {
  const int L = p.levels;
  m->z_dn.assign(L, CUtensorMap{});
  m->e_dn.assign(L, CUtensorMap{});
  m->z_up.assign(L, CUtensorMap{});
  m->g_up.assign(L, CUtensorMap{});
  m->z_dn1.assign(L, CUtensorMap{});
  m->z_fn.assign(L, CUtensorMap{});
  m->g_fn.assign(L, CUtensorMap{});
  m->z_cs.assign(L, CUtensorMap{});
  m->e_cs.assign(L, CUtensorMap{});
  m->z_fs.assign(L, CUtensorMap{});
  m->g_fs.assign(L, CUtensorMap{});
  const bool f32 = p.precision == FLLF_FP32;
  const size_t zs = f32 ? 8 : 4;
  const CUtensorMapDataType zdt = f32 ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  const uint32_t up_kc = f32 ? 1 : 2;
  // Z_1 as the level-0 REDUCE writes it: per warp a box of its 4 level-1
  // columns, the tile's kUpTH rows and a chunk of kKC orders
  if (L >= 2 && !encode4(&m->z_st1, zdt, lv[1].Z, lv[1].w, lv[1].h, p.K, p.C, zs * lv[1].pitch,
                         zs * (uint64_t)lv[1].zk, zs * (uint64_t)lv[1].zplane, kUpRun, kUpTH, kKC))
    return false;
  for (int l = 1; l < L; ++l) {
    const Level& v = lv[l];
    const uint64_t zrow = zs * v.pitch, zplane = zs * (uint64_t)v.zk;
    const uint64_t grow = 4ull * v.pitch, gplane = 4ull * (uint64_t)v.gplane;
    const uint64_t zplanes = (uint64_t)p.K * p.C;
    // as the coarse level of a combine: 36 x 18 window, kKC orders
    if (!encode4(&m->z_dn[l], zdt, v.Z, v.w, v.h, p.K, p.C, zrow, zs * (uint64_t)v.zk,
                 zs * (uint64_t)v.zplane, kDnCW, kDnCH, kKC))
      return false;
    // level >= 1 combines: Z_l as the coarse window (l >= 2), Z_l and G_l as the fine boxes (l <= L-2)
    if (l >= 2 && !encode4(&m->z_dn1[l], zdt, v.Z, v.w, v.h, p.K, p.C, zrow, zs * (uint64_t)v.zk,
                           zs * (uint64_t)v.zplane, kDnCW, kDnCH, kKC1))
      return false;
    if (l <= L - 2) {
      if (!encode4(&m->z_fn[l], zdt, v.Z, v.w, v.h, p.K, p.C, zrow, zs * (uint64_t)v.zk,
                   zs * (uint64_t)v.zplane, kD0IW, kDnOH, kKC1))
        return false;
      if (!encode3(&m->g_fn[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v.G, v.w, v.h, p.C, grow, gplane,
                   kD0IW, kDnOH, 1))
        return false;
    }
    // the small-tile combine (levels >= 1 as the fine level, >= 2 as the coarse one)
    if (l >= 2 && !encode4(&m->z_cs[l], zdt, v.Z, v.w, v.h, p.K, p.C, zrow, zs * (uint64_t)v.zk,
                           zs * (uint64_t)v.zplane, kSmCW, kSmCH, kKCS))
      return false;
    if (l <= L - 2) {
      if (!encode4(&m->z_fs[l], zdt, v.Z, v.w, v.h, p.K, p.C, zrow, zs * (uint64_t)v.zk,
                   zs * (uint64_t)v.zplane, kSmIW, kSmH, kKCS))
        return false;
      if (!encode3(&m->g_fs[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v.G, v.w, v.h, p.C, grow, gplane,
                   kSmIW, kSmH, 1))
        return false;
    }
    // as the source of a REDUCE: 68 x 35 box, up_kc orders; plus the guide
    if (l <= L - 2) {
      if (!encode3(&m->z_up[l], zdt, zs, v.Z, v.w, v.h, zplanes, zrow, zplane, kRsBW, kRsIR, up_kc))
        return false;
      if (!encode3(&m->g_up[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v.G, v.w, v.h, p.C, grow, gplane,
                   kRsBW, kRsIR, 1))
        return false;
    }
    if (v.E) {
      if (!encode3(&m->e_dn[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v.E, v.w, v.h, p.C, grow, gplane,
                   kDnCW, kDnCH, 1))
        return false;
      if (l >= 2 && !encode3(&m->e_cs[l], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v.E, v.w, v.h, p.C, grow,
                             gplane, kSmCW, kSmCH, 1))
        return false;
    }
  }
  if (L >= 3) {
    // fused level-1/level-0 combine: G_1 on the 36 x 18 level-1 window, Z_2 and
    // E_2 on the 20 x 11 level-2 window
    const Level& v1 = lv[1];
    const Level& v2 = lv[2];
    if (!encode3(&m->g1_d10, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v1.G, v1.w, v1.h, p.C, 4ull * v1.pitch,
                 4ull * (uint64_t)v1.gplane, kDnCW, kDnCH, 1))
      return false;
    if (!encode4(&m->z2_d10, zdt, v2.Z, v2.w, v2.h, p.K, p.C, zs * v2.pitch, zs * (uint64_t)v2.zk,
                 zs * (uint64_t)v2.zplane, kD2W, kD2H, kKC))
      return false;
    if (v2.E && !encode3(&m->e2_d10, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, v2.E, v2.w, v2.h, p.C,
                         4ull * v2.pitch, 4ull * (uint64_t)v2.gplane, kD2W, kD2H, 1))
      return false;
  }
  return true;
}

namespace {

// Fast LLF (Sec. II-D): the sampled detail images' pyramids (level-0 REDUCE,
// then the REDUCE kernels unchanged), the interpolating combines on the
// 32 x 16 tiles from the top down to level 2, and levels 1 and 0 in the
// fused level-0 tiles (the level-0 combine alone with 2 levels).
cudaError_t enqueue_fast(const fllf_params& p, const std::vector<Level>& lv, const PathMaps& maps,
                         const float* d_a, unsigned* fault, const float* d_in, float* d_out, cudaStream_t s,
                         StageHook* hook, const Tuning& tn, const float* tin, int tpitch) {
  const int L = p.levels, C = p.C, prec = p.precision;
  FastArgs fa{};
  fa.S = p.samples;
  fa.tau = (float)(1.0 / (p.samples - 1));
  fa.fm1 = (float)(p.m - 1.0);
  fa.c2 = (float)(1.4426950408889634 / (2.0 * p.sigma_r * p.sigma_r));   // log2(e) / (2 sigma_r^2)
  {
    // The level-0 REDUCE may step the Gaussian factor through each chunk of
    // 2 kKC samples by products instead of one exp2 per sample when, for
    // every pixel value in [0, 1]: the ratio's exponent stays within
    // +-60 (c2 tau (2 + tau)); and the chunk's start factor stays a normal
    // float (exponent >= -126) wherever a factor inside the chunk is not
    // negligible (>= 2^-24), i.e. (sqrt(24) + (2 kKC - 1) tau sqrt(c2))^2 <= 126.
    const double c2 = 1.4426950408889634 / (2.0 * p.sigma_r * p.sigma_r), tau = 1.0 / (p.samples - 1);
    const double spread = std::sqrt(24.0) + (2 * kKC - 1) * tau * std::sqrt(c2);
    fa.rec = (c2 * tau * (2.0 + tau) <= 60.0 && spread * spread <= 126.0) ? 1 : 0;
    fa.k2 = (float)std::exp2(-2.0 * c2 * tau * tau);
  }
  auto mark = [&](int st, bool b) {
    if (hook) hook->mark(st, b, s);
  };
  cudaError_t e;
  Up0Args u0{};
  u0.I = d_in;
  u0.a = d_a;
  u0.h0 = p.H;
  u0.w0 = p.W;
  u0.planes = C;
  u0.dst = lv[1];
  u0.zstmap = maps.z_st1;
  u0.K = p.K;
  u0.fault = fault;
  u0.fast = fa;
  u0.use_tma = encode_image_map(&u0.imap, tin, p.W, p.H, C, kUpIW, kUpIR, tpitch) ? 1 : 0;
  mark(FLLF_STAGE_UP0, true);
  if ((e = launch_up0(prec, u0, s, tn.cps[FLLF_STAGE_UP0])) != cudaSuccess) return e;
  mark(FLLF_STAGE_UP0, false);
  for (int l = 1; l <= L - 2; ++l) {
    UpArgs u{};
    u.zmap = maps.z_up[l];
    u.gmap = maps.g_up[l];
    u.src = lv[l];
    u.dst = lv[l + 1];
    u.planes = C;
    u.K = p.K;
    u.write_g = (l + 1 <= L - 2) ? 1 : 0;
    u.reverse = (l == 1 && tn.reverse) ? 1 : 0;
    u.fault = fault;
    mark(FLLF_STAGE_UP, true);
    if ((e = launch_up(prec, u, s, tn.cps[FLLF_STAGE_UP])) != cudaSuccess) return e;
    mark(FLLF_STAGE_UP, false);
  }
  // with >= 3 levels, level 1 runs inside the level-0 tiles (as for Fourier LLF)
  const int down_lo = L >= 3 ? 2 : 1;
  for (int l = L - 2; l >= down_lo; --l) {
    DownArgs d{};
    d.zmap = maps.z_cs[l + 1];
    d.emap = maps.e_cs[l + 1];
    d.zfmap = maps.z_fs[l];
    d.gfmap = maps.g_fs[l];
    d.fine = lv[l];
    d.coarse = lv[l + 1];
    d.planes = C;
    d.K = p.K;
    d.has_e = (l + 1 <= L - 2) ? 1 : 0;
    d.fault = fault;
    d.fast = fa;
    mark(FLLF_STAGE_DOWN_S, true);
    if ((e = launch_down_s(prec, d, s, tn.cps[FLLF_STAGE_DOWN_S])) != cudaSuccess) return e;
    mark(FLLF_STAGE_DOWN_S, false);
  }
  mark(FLLF_STAGE_DOWN0, true);
  if (L >= 3) {
    Down10Args d{};
    d.z1map = maps.z_dn[1];
    d.g1map = maps.g1_d10;
    d.z2map = maps.z2_d10;
    d.e2map = maps.e2_d10;
    d.I = d_in;
    d.O = d_out;
    d.h0 = p.H;
    d.w0 = p.W;
    d.planes = C;
    d.l1 = lv[1];
    d.l2 = lv[2];
    d.K = p.K;
    d.has_e2 = (L >= 4) ? 1 : 0;
    d.use_tma = (u0.use_tma && encode_image_map(&d.imap, tin, p.W, p.H, C, kD0IW, kDnOH, tpitch)) ? 1 : 0;
    d.fault = fault;
    d.fast = fa;
    if ((e = launch_down10(prec, d, s, tn.cps[FLLF_STAGE_DOWN0])) != cudaSuccess) return e;
  } else {
    Down0Args d0{};
    d0.zmap = maps.z_dn[1];
    d0.emap = maps.e_dn[1];
    d0.I = d_in;
    d0.O = d_out;
    d0.h0 = p.H;
    d0.w0 = p.W;
    d0.planes = C;
    d0.coarse = lv[1];
    d0.K = p.K;
    d0.has_e = 0;
    d0.fault = fault;
    d0.fast = fa;
    if ((e = launch_down0(prec, d0, s, tn.cps[FLLF_STAGE_DOWN0])) != cudaSuccess) return e;
  }
  mark(FLLF_STAGE_DOWN0, false);
  return cudaSuccess;
}

}  // namespace

cudaError_t enqueue_path(const fllf_params& p, const std::vector<Level>& lv, const PathMaps& maps,
                         const float* d_a, unsigned* fault, const float* d_in, float* d_out,
                         cudaStream_t s, StageHook* hook, const float* d_gain, float mscale,
                         const Tuning* tune, const PlanGraph* graph, float* d_stage) {
  static const Tuning kDefault{};
  const Tuning& tn = tune ? *tune : kDefault;
  const int L = p.levels, C = p.C, prec = p.precision;
  const float turns = (float)(2.0 / p.T);
  if (L == 1) {
    // Only the top level: L_0[O] = G_0[I] = I.
    return cudaMemcpyAsync(d_out, d_in, sizeof(float) * (size_t)p.H * p.W * C,
                           cudaMemcpyDeviceToDevice, s);
  }
  auto mark = [&](int st, bool b) {
    if (hook) hook->mark(st, b, s);
  };
  cudaError_t e;
  // The level-0 kernels load the input by TMA when its rows start on 16-byte
  // boundaries; otherwise a staging buffer takes a copy at a padded pitch
  // (one pass, counted with the level-0 REDUCE), else they use plain loads.
  const float* tin = d_in;
  int tpitch = p.W;
  if (d_stage && ((p.W % 4) != 0 || (reinterpret_cast<uintptr_t>(d_in) & 15) != 0)) {
    tpitch = staged_pitch(p.W);
    mark(FLLF_STAGE_UP0, true);
    if ((e = launch_pad_rows(d_in, p.W, (long long)p.H * C, d_stage, tpitch, s)) != cudaSuccess) return e;
    mark(FLLF_STAGE_UP0, false);
    tin = d_stage;
  }
  if (p.method == FLLF_METHOD_FAST)
    return enqueue_fast(p, lv, maps, d_a, fault, d_in, d_out, s, hook, tn, tin, tpitch);

  if (graph && (tn.dataflow == 1 || tn.dataflow == 2) && !d_gain) {
    // one persistent dataflow launch over every stage (the plan's task list;
    // the level-0 argument blocks carry this run's input and output), or
    // over every stage but the fused level-1/level-0 combine, which then
    // follows as its own kernel
    GraphArgs g = graph->args;
    g.up0.I = d_in;
    g.up0.use_tma = encode_image_map(&g.up0.imap, tin, p.W, p.H, C, kUpIW, kUpIR, tpitch) ? 1 : 0;
    if (L >= 3) {
      g.d10.I = d_in;
      g.d10.O = d_out;
      g.d10.use_tma = (g.up0.use_tma && encode_image_map(&g.d10.imap, tin, p.W, p.H, C, kD0IW, kDnOH, tpitch)) ? 1 : 0;
    } else {
      g.d0.I = d_in;
      g.d0.O = d_out;
    }
    const bool with_d10 = graph->gb.with_d10;
    mark(FLLF_STAGE_GRAPH, true);
    if ((e = launch_graph(prec, g, sizeof(unsigned) * graph->gb.rt_words, s, tn.cps[FLLF_STAGE_GRAPH],
                          with_d10)) != cudaSuccess)
      return e;
    mark(FLLF_STAGE_GRAPH, false);
    if (L >= 3 && !with_d10) {
      mark(FLLF_STAGE_DOWN0, true);
      if ((e = launch_down10(prec, g.d10, s, tn.cps[FLLF_STAGE_DOWN0])) != cudaSuccess) return e;
      mark(FLLF_STAGE_DOWN0, false);
    }
    return cudaSuccess;
  }

  Up0Args u0{};
  u0.I = d_in;
  u0.a = d_a;
  u0.h0 = p.H;
  u0.w0 = p.W;
  u0.planes = C;
  u0.dst = lv[1];
  u0.zstmap = maps.z_st1;
  u0.K = p.K;
  u0.turns = turns;
  u0.fault = fault;
  u0.use_tma = encode_image_map(&u0.imap, tin, p.W, p.H, C, kUpIW, kUpIR, tpitch) ? 1 : 0;
  // The level 1 -> 2 REDUCE exists with >= 3 levels, and the chained or
  // dataflow launches only start at level 2 or above.
  const bool banded = tn.bands > 1 && L >= 3;
  if (!banded) {
    mark(FLLF_STAGE_UP0, true);
    if ((e = launch_up0(prec, u0, s, tn.cps[FLLF_STAGE_UP0])) != cudaSuccess) return e;
    mark(FLLF_STAGE_UP0, false);
  } else {
    // Row bands: the level-0 REDUCE of tile rows [r0, r1) of all planes in
    // turn (plane-major), each followed by the level 1 -> 2 REDUCE of the
    // level-2 tile rows whose level-1 inputs are then complete.
    const int ntx0 = cdiv(lv[1].w, kUpTW), nty0 = cdiv(lv[1].h, kUpTH), rows0 = nty0 * C;
    const int kcu = prec == FLLF_FP32 ? Smem<8>::up_kc : Smem<4>::up_kc;
    const int ntx2 = cdiv(lv[2].w, kRsTW), nty2 = cdiv(lv[2].h, kRsTH), rows2 = nty2 * C;
    const int per2 = ntx2 * (cdiv(p.K, kcu) + ((2 <= L - 2) ? 1 : 0));
    UpArgs u1{};
    u1.zmap = maps.z_up[1];
    u1.gmap = maps.g_up[1];
    u1.src = lv[1];
    u1.dst = lv[2];
    u1.planes = C;
    u1.K = p.K;
    u1.write_g = (2 <= L - 2) ? 1 : 0;
    u1.fault = fault;
    // level-0 REDUCE tile rows (plane-major index) a level-2 tile row reads
    auto needs = [&](int r2) {
      const int pl = r2 / nty2, ty2 = r2 % nty2;
      const int last1 = std::min(lv[1].h - 1, 2 * std::min(kRsTH * ty2 + kRsTH - 1, lv[2].h - 1) + 2);
      return pl * nty0 + last1 / kUpTH;
    };
    const int nb = std::min(tn.bands, rows0);
    int done2 = 0;
    for (int c = 0; c < nb; ++c) {
      const int r0 = (int)((long long)rows0 * c / nb), r1 = (int)((long long)rows0 * (c + 1) / nb);
      Up0Args ub = u0;
      ub.item0 = r0 * ntx0;
      ub.item1 = r1 * ntx0;
      mark(FLLF_STAGE_UP0, true);
      if ((e = launch_up0(prec, ub, s, tn.cps[FLLF_STAGE_UP0])) != cudaSuccess) return e;
      mark(FLLF_STAGE_UP0, false);
      int ready2 = done2;
      while (ready2 < rows2 && needs(ready2) < r1) ++ready2;
      if (c == nb - 1) ready2 = rows2;
      if (ready2 > done2) {
        UpArgs ua = u1;
        ua.item0 = done2 * per2;
        ua.item1 = ready2 * per2;
        mark(FLLF_STAGE_UP, true);
        if ((e = launch_up(prec, ua, s, tn.cps[FLLF_STAGE_UP])) != cudaSuccess) return e;
        mark(FLLF_STAGE_UP, false);
        done2 = ready2;
      }
    }
  }
  if (d_gain) {
    // Gaussian pyramid of the gain map, levels 1..L-2 (the levels that combine)
    for (int l = 1; l <= L - 2; ++l) {
      const float* src = l == 1 ? d_gain : lv[l - 1].M;
      const int sp = l == 1 ? p.W : lv[l - 1].pitch;
      if ((e = launch_map_reduce(src, lv[l - 1].h, lv[l - 1].w, sp, const_cast<float*>(lv[l].M), lv[l].h,
                                 lv[l].w, lv[l].pitch, s)) != cudaSuccess)
        return e;
    }
  }

  // With a chain threshold (tuning; 0 by default), levels >= c0 run as one
  // chained cooperative launch: from the first level (>= 2) whose pixels over
  // all planes fit in chain_px, the REDUCE stages up to the top and the
  // combines back down to c0.
  //
  // With dataflow 3, the levels from the plan's task-list level up (>= 2) run
  // instead as one dataflow launch: the REDUCE from that level to the top and
  // the combines back down to it, each task starting once the row bands it
  // reads are complete.
  const bool flow_small = graph && tn.dataflow == 3 && !d_gain && graph->gb.lo >= 2 && graph->gb.lo <= L - 2;
  const long long chain_px = tn.chain_px;
  int c0 = L - 1;
  if (flow_small) {
    c0 = graph->gb.lo;
  } else {
    for (int l = 2; l <= L - 2; ++l)
      if ((long long)lv[l].h * lv[l].w * C <= chain_px) {
        c0 = l;
        break;
      }
    if (L - 1 - c0 > kChainMax) c0 = L - 1 - kChainMax;
  }
  auto up_args = [&](int l) {
    UpArgs u{};
    u.zmap = maps.z_up[l];
    u.gmap = maps.g_up[l];
    u.src = lv[l];
    u.dst = lv[l + 1];
    u.planes = C;
    u.K = p.K;
    u.write_g = (l + 1 <= L - 2) ? 1 : 0;
    u.fault = fault;
    return u;
  };
  auto down_args = [&](int l) {
    DownArgs d{};
    d.zmap = maps.z_dn1[l + 1];
    d.emap = maps.e_dn[l + 1];
    d.zfmap = maps.z_fn[l];
    d.gfmap = maps.g_fn[l];
    d.fine = lv[l];
    d.coarse = lv[l + 1];
    d.planes = C;
    d.K = p.K;
    d.turns = turns;
    d.has_e = (l + 1 <= L - 2) ? 1 : 0;
    d.mscale = mscale;
    d.fault = fault;
    return d;
  };
  for (int l = 1; l <= L - 2 && l < c0; ++l) {
    UpArgs u = up_args(l);
    if (l == 1 && banded) {
      // The level 1 -> 2 REDUCE in row bands, each launched right after the
      // level-0 REDUCE band it reads (below), while that band's Z_1 is still
      // in L2: nothing to launch here.
      continue;
    }
    u.reverse = (l == 1 && tn.reverse) ? 1 : 0;   // the level-0 REDUCE wrote Z_1 first to last
    mark(FLLF_STAGE_UP, true);
    if ((e = launch_up(prec, u, s, tn.cps[FLLF_STAGE_UP])) != cudaSuccess) return e;
    mark(FLLF_STAGE_UP, false);
  }
  if (c0 <= L - 2 && flow_small) {
    mark(FLLF_STAGE_GRAPH, true);
    if ((e = launch_graph(prec, graph->args, sizeof(unsigned) * graph->gb.rt_words, s, tn.cps[FLLF_STAGE_GRAPH],
                          false)) != cudaSuccess)
      return e;
    mark(FLLF_STAGE_GRAPH, false);
  } else if (c0 <= L - 2) {
    ChainArgs ca{};
    for (int l = c0; l <= L - 2; ++l) ca.up[ca.n_up++] = up_args(l);
    for (int l = L - 2; l >= c0; --l) {
      DownArgs d = down_args(l);
      const bool small = (long long)lv[l].h * lv[l].w * C <= tn.small_px;
      if (small) {   // the 32 x 16 tiles, as outside the chain
        d.zmap = maps.z_cs[l + 1];
        d.emap = maps.e_cs[l + 1];
        d.zfmap = maps.z_fs[l];
        d.gfmap = maps.g_fs[l];
      }
      ca.dn_small[ca.n_dn] = small ? 1 : 0;
      ca.dn[ca.n_dn++] = d;
    }
    ca.sync = fault + 32;
    ca.fault = fault;
    mark(FLLF_STAGE_CHAIN, true);
    if ((e = launch_chain(prec, ca, s, tn.cps[FLLF_STAGE_CHAIN])) != cudaSuccess) return e;
    mark(FLLF_STAGE_CHAIN, false);
  }
  // With levels >= 3 the level-1 combine runs inside the level-0 tiles.
  const int down_lo = L >= 3 ? 2 : 1;
  for (int l = (c0 <= L - 2 ? c0 - 1 : L - 2); l >= down_lo; --l) {
    DownArgs d = down_args(l);
    if (l >= 2 && (long long)lv[l].h * lv[l].w * C <= tn.small_px) {
      // small level: the same combine on 32 x 16 tiles
      d.zmap = maps.z_cs[l + 1];
      d.emap = maps.e_cs[l + 1];
      d.zfmap = maps.z_fs[l];
      d.gfmap = maps.g_fs[l];
      mark(FLLF_STAGE_DOWN_S, true);
      if ((e = launch_down_s(prec, d, s, tn.cps[FLLF_STAGE_DOWN_S])) != cudaSuccess) return e;
      mark(FLLF_STAGE_DOWN_S, false);
      continue;
    }
    mark(FLLF_STAGE_DOWN, true);
    if ((e = launch_down(prec, d, s, tn.cps[FLLF_STAGE_DOWN])) != cudaSuccess) return e;
    mark(FLLF_STAGE_DOWN, false);
  }
  if (L >= 3) {
    Down10Args d{};
    d.z1map = maps.z_dn[1];
    d.g1map = maps.g1_d10;
    d.z2map = maps.z2_d10;
    d.e2map = maps.e2_d10;
    d.I = d_in;
    d.O = d_out;
    d.h0 = p.H;
    d.w0 = p.W;
    d.planes = C;
    d.l1 = lv[1];
    d.l2 = lv[2];
    d.K = p.K;
    d.turns = turns;
    d.has_e2 = (L >= 4) ? 1 : 0;
    d.M0 = d_gain;
    d.mscale = mscale;
    d.use_tma = (u0.use_tma && encode_image_map(&d.imap, tin, p.W, p.H, C, kD0IW, kDnOH, tpitch)) ? 1 : 0;
    d.fault = fault;
    mark(FLLF_STAGE_DOWN0, true);
    if ((e = launch_down10(prec, d, s, tn.cps[FLLF_STAGE_DOWN0])) != cudaSuccess) return e;
    mark(FLLF_STAGE_DOWN0, false);
    return cudaSuccess;
  }
  Down0Args d0{};
  d0.zmap = maps.z_dn[1];
  d0.emap = maps.e_dn[1];
  d0.I = d_in;
  d0.O = d_out;
  d0.h0 = p.H;
  d0.w0 = p.W;
  d0.planes = C;
  d0.coarse = lv[1];
  d0.K = p.K;
  d0.turns = turns;
  d0.has_e = (L >= 3) ? 1 : 0;
  d0.M0 = d_gain;
  d0.mscale = mscale;
  d0.fault = fault;
  mark(FLLF_STAGE_DOWN0, true);
  if ((e = launch_down0(prec, d0, s, tn.cps[FLLF_STAGE_DOWN0])) != cudaSuccess) return e;
  mark(FLLF_STAGE_DOWN0, false);
  return cudaSuccess;
}

}  // namespace fllf
