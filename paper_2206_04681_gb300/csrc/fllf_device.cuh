// fllf_device.cuh -- shared device code of the Fourier LLF hot path (sm_103a).
//
// The filter (Sec. III-A, Eq. (14), Fig. 1) needs the guide Gaussian
// pyramid G_l[I] and 2K Gaussian Fourier pyramids C~_{l,k} = G_l[cos(w_k I)],
// S~_{l,k} = G_l[sin(w_k I)].  They are stored as K complex planes
// Z_{l,k} = C~_{l,k} + i S~_{l,k}; the per-pixel coefficient pair of
// Fig. 1 is a_k (cos(w_k g), sin(w_k g)) with g = G_l[I]_p, and
//
//   L_l[O]_p - L_l[I]_p = sum_k a_k Im( e^{-i w_k g} (Z_{l,k} - up(Z_{l+1,k}))_p ).
//
// The collapse (Eq. (4)) is carried in residual form: with
// E_l = O_l - G_l[I] (O_l the partial collapse down to level l),
// E_top = 0, E_l = Delta_l + up(E_{l+1}) and O = I + E_0, which follows
// from L_l[I] = G_l - up(G_{l+1}) and O_l = L_l[O] + up(O_{l+1}).  At
// level 0, g = I_p and the Z_0 term cancels exactly (r(I, I_p) = I), so
// Delta_0 = -sum_k a_k Im(e^{-i w_k I_p} up(Z_{1,k})_p).
//
// Borders: reflect-101 at every level for REDUCE; EXPAND is zero insertion
// followed by the kernel with reflect-101 at the fine size, which on the
// coarse grid means index -1 -> 1 and index m -> m-2 (fine size odd) or m-1
// (fine size even); a coarse level of size 1 expands to the identity.
//
// Tiles are staged in shared memory by the Tensor Memory Accelerator
// (cp.async.bulk.tensor, completion on an mbarrier), double-buffered so that
// the next chunk or tile is in flight while the current one is computed.
// TMA fills out-of-range elements with zeros; border tiles then rewrite
// those elements in shared memory from their reflected sources.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace fllf {

constexpr int kThreads = 256;  // every kernel runs 256 threads per CTA

// ---- storage of one complex Fourier sample (C~, S~) ---------------------------------
template <typename S> struct Cplx;
template <> struct Cplx<float> {
  using T = float2;
  static __device__ __forceinline__ float2 cvt(T v) { return v; }
  static __device__ __forceinline__ void st(T* p, float2 v) { *p = v; }
};
template <> struct Cplx<__half> {
  using T = __half2;
  static __device__ __forceinline__ float2 cvt(T v) { return __half22float2(v); }
  static __device__ __forceinline__ void st(T* p, float2 v) { *p = __float22half2_rn(v); }
};
template <> struct Cplx<__nv_bfloat16> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ float2 cvt(T v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ void st(T* p, float2 v) { *p = __float22bfloat162_rn(v); }
};

// One pyramid level of every plane of a batch.
struct Level {
  int h, w;             // level size
  int pitch;            // row pitch in elements (floats for G/E, complex for Z)
  long long gplane;     // elements between planes of G and E
  long long zk;         // complex elements between orders of Z
  long long zplane;     // complex elements between planes of Z
  float* G;             // guide level G_l[I] (null at level 0)
  void* Z;              // K complex Fourier planes
  float* E;             // residual E_l (null at l = levels-1)
  const float* M;       // gain map G_l[M] of pixel-adaptive runs (one plane, this pitch), else null
};

// Kernel arguments.  Tensor maps describe the level buffers as 3-D tensors
// (x = column, y = row, z = plane); Z maps read by a REDUCE have
// z = plane * K + k, Z maps read by a combine are 4-D (column, row, order,
// plane), so that orders k >= K of a chunk read as zeros.
// Fast LLF (Sec. II-D): S samples g_j = tau j of [0, 1] and the sampled
// detail images F_j = f(I - g_j), f(d) = fm1 d 2^(-c2 d^2) (the Gaussian
// detail with fm1 = m - 1, c2 = log2(e) / (2 sigma_r^2)); F_{2k} and F_{2k+1}
// are the real and imaginary parts of complex plane k (the imaginary part of
// the last plane is zero when S is odd).  S = 0: Fourier LLF.
// rec = 1: within a chunk of 2 kKC consecutive samples the Gaussian factor
// E_j = 2^(-c2 (i - tau j)^2) follows E_{j+1} = E_j r_j, r_{j+1} = r_j k2
// (r_j = 2^(-c2 tau (2 (tau j - i) + tau)), k2 = 2^(-2 c2 tau^2)) from one
// exact start per chunk; the host sets it only where neither r nor the start
// leaves the float range for any pixel in [0, 1].
struct FastArgs {
  int S;
  float tau, fm1, c2;
  int rec;
  float k2;
};

// Input staging of one image of a batch: `rows` dense rows of W floats from
// src to rows of `pitch` floats (a multiple of 4) at dst.
struct PadRow {
  const float* src;
  float* dst;
  int W, pitch, rows, pad_;
};

struct Up0Args {
  CUtensorMap imap;     // level-0 input (valid when use_tma)
  CUtensorMap zstmap;   // Z_1 as a TMA store target: (4 columns, kUpTH rows, kKC orders) boxes
  const float* I;       // level-0 input planes, pitch w0, plane stride h0*w0
  const float* a;       // a_1..a_K (float32): order k is stored as a_k Z_{1,k}
  int h0, w0, planes;
  Level dst;            // level 1
  int K;
  float turns;          // 2/T: w_1 x = pi * (turns * x)
  int use_tma;          // input rows 16-byte aligned (w0 % 4 == 0, aligned base)
  unsigned* fault;      // bounded-wait fault word
  FastArgs fast;        // fast LLF: plane k holds (F_{2k}, F_{2k+1}) unweighted
  int item0, item1;     // the launch's tiles [item0, item1) (item1 = 0: every tile)
};

struct UpArgs {
  CUtensorMap zmap;     // source Z_l
  CUtensorMap gmap;     // source G_l
  Level src;            // level l >= 1
  Level dst;            // level l+1
  int planes, K;
  int write_g;          // G_{l+1} needed (l+1 <= levels-2)
  int reverse;          // visit the work items last to first (L2 reuse of the level just written)
  unsigned* fault;
  int item0, item1;     // the launch's work items [item0, item1) (item1 = 0: every item)
};

// The boxes are those of the 64 x 32 combine (k_down), or of the 32 x 16
// small-level combine (k_down_s: 20 x 10 x kKCS, 20 x 10, 36 x 16 x kKCS and
// 36 x 16).
struct DownArgs {
  CUtensorMap zmap;     // coarse Z_{l+1}: 36 x 18 x kKC1 window
  CUtensorMap emap;     // coarse E_{l+1}: 36 x 18 window
  CUtensorMap zfmap;    // fine Z_l: 68 x 32 x kKC1 box from (X0 - 2, Y0)
  CUtensorMap gfmap;    // fine G_l: 68 x 32 box from (X0 - 2, Y0)
  Level fine;           // level l >= 1: G, Z read, E written
  Level coarse;         // level l+1
  int planes, K;
  float turns;
  int has_e;            // E_{l+1} exists (l+1 <= levels-2)
  float mscale;         // 1/(m - 1): the gain map's scale of the Fourier term (fine.M set)
  unsigned* fault;
  FastArgs fast;        // fast LLF: interpolate the bracketing samples' differences
};

struct Down0Args {
  CUtensorMap zmap;     // Z_1
  CUtensorMap emap;     // E_1
  const float* I;       // level-0 input, pitch w0
  float* O;             // level-0 output, pitch w0
  int h0, w0, planes;
  Level coarse;         // level 1
  int K;
  float turns;
  int has_e;            // E_1 exists (levels >= 3)
  const float* M0;      // level-0 gain map (pitch w0) of pixel-adaptive runs, else null
  float mscale;         // 1/(m - 1)
  unsigned* fault;
  FastArgs fast;        // fast LLF
};

// Fused combine of levels 1 and 0 (levels >= 3): the level-1 combine runs on
// the window of level-1 cells that the level-0 EXPAND reads, so E_1 stays in
// shared memory.
struct Down10Args {
  CUtensorMap imap;     // level-0 input tile (68 x 32 from (X0 - 2, Y0); valid when use_tma)
  CUtensorMap z1map;    // Z_1 as the coarse window of level 0 (36 x 18 x kKC)
  CUtensorMap g1map;    // G_1 on the same window (36 x 18)
  CUtensorMap z2map;    // Z_2 window of the level-1 cells (20 x 11 x kKC)
  CUtensorMap e2map;    // E_2 on the level-2 window (20 x 11)
  const float* I;       // level-0 input, pitch w0
  float* O;             // level-0 output, pitch w0
  int h0, w0, planes;
  Level l1, l2;         // levels 1 and 2
  int K;
  float turns;
  int has_e2;           // E_2 exists (levels >= 4)
  int use_tma;          // input rows 16-byte aligned (w0 % 4 == 0, aligned base)
  const float* M0;      // level-0 gain map (pitch w0) of pixel-adaptive runs, else null;
                        // the level-1 map is l1.M
  float mscale;         // 1/(m - 1)
  unsigned* fault;
  FastArgs fast;        // fast LLF: interpolating combines at levels 1 and 0
};

// Batched stage launch: argument blocks of the images that have the stage
// (device memory) and exclusive prefix sums of their work-item counts
// (prefix[0] = 0, prefix[n] = total).
template <typename A>
struct BatchTable {
  const A* args;
  const int* prefix;
  int n, total;
};

// Dataflow launch: one persistent grid runs every stage of one or many images
// as tasks (a run of consecutive work items of one row band of one stage).
// A band becomes ready when every band it reads is complete; its tasks are
// then pushed onto a device queue, from which the CTAs pop ready tasks only.
// The bands that read nothing (the level-0 REDUCE) are the queue's seeds.
enum GraphKind { kGUp0 = 0, kGUp = 1, kGDownS = 2, kGDown10 = 3, kGDown0 = 4 };
struct GraphTask {
  int kind;        // GraphKind
  int args;        // index into the kind's argument table (-1: the inline block of GraphArgs)
  int first, count;// work items [first, first + count) of the stage
  int band;        // the row band the task belongs to
};
struct GraphBand {
  unsigned total;  // work items of the band
  int task0, ntasks;  // its tasks: [task0, task0 + ntasks)
  int ndeps;       // bands it reads
  int cons0, cons1;   // bands that read it: cons[cons0 .. cons1)
};

struct GraphArgs {
  Up0Args up0;          // inline level-0 argument blocks of a single image (inline0 = 1)
  Down10Args d10;
  Down0Args d0;
  const Up0Args* up0s;  // argument tables in device memory
  const UpArgs* ups;
  const DownArgs* dns;
  const Down10Args* d10s;
  const Down0Args* d0s;
  const GraphTask* tasks;
  const GraphBand* bands;
  const int* cons;      // consumer band lists
  const int* seeds;     // the seed tasks, in the order they are popped
  // run state (zeroed before every run): [0] queue head, [1] queue tail,
  // then per band the items done and the bands it reads that are complete,
  // then the queue slots (task + 1; 0 = not yet pushed)
  unsigned* rt;
  unsigned* fault;
  int ntasks, nbands, nseeds;
  int inline0;
};

// Chained small levels: REDUCE stages then combine stages in one cooperative
// launch, with a grid barrier between consecutive stages.
constexpr int kChainMax = 12;
struct ChainArgs {
  UpArgs up[kChainMax];     // REDUCE stages, finest first
  DownArgs dn[kChainMax];   // combine stages, coarsest first
  int dn_small[kChainMax];  // combine stage on the 32 x 16 tiles (its maps are those boxes)
  int n_up, n_dn;
  unsigned* sync;           // grid barrier: [0] arrivals, [1] generation (zeroed by the plan)
  unsigned* fault;
};

// ---- tiling constants ---------------------------------------------------------------
constexpr int kKC = 4;                    // complex orders per combine / up0 chunk

// up0: 32 x 14 level-1 outputs per tile.
constexpr int kUpTW = 32, kUpTH = 14;
constexpr int kUpRun = 4;                 // coarse outputs per horizontal item
constexpr int kUpSeg = kUpTW / kUpRun;    // items per input row (8)
constexpr int kUpIR = 2 * kUpTH + 3;      // fine input rows (31)
constexpr int kUpIPX = 2 * kUpRun + 3;    // fine inputs per item (11)
constexpr int kUpItems = kUpIR * kUpSeg;  // 248 horizontal items
constexpr int kUpVRows = kUpTH / 2;       // coarse rows per vertical thread (7)
constexpr int kUpCS = 36;                 // staged rows per column (36 x 8 B: 2 mod 8 bank groups)
// staged input columns (box from 2*X1-4, 16-B aligned; 70 are read): a row
// pitch of 76 floats (12 banks mod 32) puts the 8 rows of a quarter-warp's
// 16-byte loads on distinct banks, where 72 (8 mod 32) made them 2-way
constexpr int kUpIW = 76;
static_assert(kUpItems <= kThreads, "REDUCE items exceed the block");
static_assert(kUpSeg * 32 == kThreads && kUpIR <= 32, "up0 items: one warp per run segment, one lane per row");
static_assert(kKC * 2 * kUpRun == 32 && kUpRun * kUpVRows <= 32, "up0 vertical pass: one warp per segment");
static_assert(kKC % 2 == 0, "up0 order recurrence: the two registers' roles repeat every chunk");
static_assert(2 * kUpVRows + 2 * (kUpVRows + 2) <= kUpCS && 4 * (kUpVRows - 1) + 8 <= kUpCS &&
                  kUpIR <= kUpCS,
              "up0 vertical reads stay in the staged column");
static_assert(2 * kUpRun * (kUpSeg - 1) + 16 <= kUpIW, "up0 run reads stay inside the staged row");
static_assert(kKC * kUpTW * 2 == kThreads, "vertical REDUCE mapping");

// up (levels >= 1): 30 x 16 coarse outputs per tile.
constexpr int kRsTW = 30, kRsTH = 16;
constexpr int kRsIR = 2 * kRsTH + 3;      // fine rows read (35)
constexpr int kRsBW = 68;                 // staged fine columns (box from 2*X1-4)
constexpr int kRsVW = 64;                 // vertical-pass columns (63 used)
constexpr int kUpSlots = 2;               // TMA ring slots of the REDUCE stage (1 load in flight)

// combine: 64 x 32 fine outputs per tile; fine tile origin 64*tx-6 so that the
// coarse window origin 32*tx-4 is 16-byte aligned for both element sizes.
constexpr int kDnOW = 64, kDnOH = 32;
constexpr int kDnCW = 36;                 // staged coarse columns (34 used)
constexpr int kDnCH = kDnOH / 2 + 2;      // staged coarse rows (18)
constexpr int kDnX0 = 6;                  // fine tile origin offset
static_assert((kDnOW / 4) * (kDnOH / 2) == kThreads, "combine thread mapping");
// fused level-1/level-0 combine: the level-2 window of the level-1 cells
// (origin (cx0/2 - 2, (cy0 - 1)/2), 19 x 11 used) and the 2 x 2 cell blocks
// of the level-1 threads over the 34 x 18 used level-1 cells.
constexpr int kD2W = 20, kD2H = 11;
constexpr int kB1X = 17, kB1Y = 9;
constexpr int kKC1 = 2;                   // orders per chunk of the level >= 1 combine
constexpr int kD0IW = kDnOW + 4;          // staged level-0 input columns (from X0 - 2)
static_assert(kB1X * kB1Y <= kThreads && 2 * kB1X == kDnCW - 2 && 2 * kB1Y == kDnCH,
              "level-1 blocks cover the used window");
static_assert(kB1X + 2 < kD2W && kB1Y + 1 < kD2H, "level-1 blocks read inside the level-2 window");

// combine at the small levels (>= 1): 32 x 16 fine outputs per tile and one
// fine column by two rows per thread (more tiles and a quarter of the work
// per thread of the 64 x 32 combine, for levels too small to fill the GPU
// with those).  Tile origin 32*tx-6, so the coarse window starts at 16*tx-4
// (16-byte aligned for both element sizes).
constexpr int kSmW = 32, kSmH = 16;
constexpr int kSmIW = kSmW + 4;           // staged fine columns (from X0 - 2)
constexpr int kSmCW = 20;                 // staged coarse columns (18 used)
constexpr int kSmCH = kSmH / 2 + 2;       // staged coarse rows (10)
constexpr int kKCS = 4;                   // orders per chunk of the small combine
static_assert(kSmW * (kSmH / 2) == kThreads, "small combine thread mapping");

__host__ __device__ constexpr int cdiv(int a, int b) { return (a + b - 1) / b; }
__host__ __device__ constexpr size_t align128(size_t x) { return (x + 127) & ~size_t(127); }

// Shared-memory plans (bytes).
template <int ESZ>  // bytes per complex sample
struct Smem {
  // up0
  static constexpr size_t up0_it = align128(sizeof(float) * kUpIR * kUpIW);
  static constexpr size_t up0_hz = sizeof(float2) * kKC * kUpTW * kUpCS;
  static constexpr size_t up0_hg = sizeof(float) * kUpTW * kUpCS;
  // the vertical pass's Z_1 outputs of one chunk, per warp a (4, kUpTH,
  // kKC) box for its TMA store; two chunks in flight
  static constexpr size_t up0_st = (size_t)ESZ * kUpRun * kUpTH * kKC * (kThreads / 32);
  static constexpr size_t up0 = 2 * up0_it + align128(up0_hz) + align128(up0_hg) + 2 * align128(up0_st) + 64;
  // fast LLF (80 registers): one chunk in flight, which keeps 3 CTAs per SM
  static constexpr size_t up0_fast = 2 * up0_it + align128(up0_hz) + align128(up0_hg) + align128(up0_st) + 64;
  // up
  static constexpr int up_kc = ESZ == 8 ? 1 : 2;  // orders per chunk
  // ring slot: one chunk of orders, or the guide plane (smaller)
  static constexpr size_t up_slot = align128((size_t)ESZ * up_kc * kRsIR * kRsBW);
  static constexpr size_t up_vb = align128(sizeof(float2) * up_kc * kRsTH * kRsVW);
  static constexpr size_t up_vg = align128(sizeof(float) * kRsTH * kRsVW);
  static constexpr size_t up = kUpSlots * up_slot + up_vb + up_vg + 64;
  static_assert(sizeof(float) * kRsIR * kRsBW <= up_slot, "the guide box fits a ring slot");
  // combine
  static constexpr size_t dn_z = align128((size_t)ESZ * kKC * kDnCH * kDnCW);
  static constexpr size_t dn_e = align128(sizeof(float) * kDnCH * kDnCW);
  static constexpr size_t dn_buf = dn_z + dn_e;
  static constexpr size_t dn = 2 * dn_buf + 64;
  // combine at level >= 1: fine Z_l and G_l boxes, coarse Z_{l+1} and E_{l+1} windows
  static constexpr size_t dn1_zf = align128((size_t)ESZ * kKC1 * kDnOH * kD0IW);
  static constexpr size_t dn1_zc = align128((size_t)ESZ * kKC1 * kDnCH * kDnCW);
  static constexpr size_t dn1_e = align128(sizeof(float) * kDnCH * kDnCW);
  static constexpr size_t dn1_g = align128(sizeof(float) * kDnOH * kD0IW);
  static constexpr size_t dn1_buf = dn1_zf + dn1_zc + dn1_e + dn1_g;
  static constexpr size_t dn1 = 2 * dn1_buf + 64;
  // small-level combine: the same four boxes on 32 x 16 tiles
  static constexpr size_t sm_zf = align128((size_t)ESZ * kKCS * kSmH * kSmIW);
  static constexpr size_t sm_zc = align128((size_t)ESZ * kKCS * kSmCH * kSmCW);
  static constexpr size_t sm_e = align128(sizeof(float) * kSmCH * kSmCW);
  static constexpr size_t sm_g = align128(sizeof(float) * kSmH * kSmIW);
  static constexpr size_t sm_buf = sm_zf + sm_zc + sm_e + sm_g;
  static constexpr size_t dns = 2 * sm_buf + 64;
  // fused level-1/level-0 combine
  static constexpr size_t d10_z1 = dn_z;
  static constexpr size_t d10_z2 = align128((size_t)ESZ * kKC * kD2H * kD2W);
  static constexpr size_t d10_g1 = align128(sizeof(float) * kDnCH * kDnCW);
  static constexpr size_t d10_e2 = align128(sizeof(float) * kD2H * kD2W);
  static constexpr size_t d10_i = align128(sizeof(float) * kDnOH * kD0IW);
  static constexpr size_t d10_buf = d10_z1 + d10_z2 + d10_g1 + d10_e2 + d10_i;
  static constexpr size_t d10_e1 = align128(sizeof(float) * kDnCH * kDnCW);
  static constexpr size_t d10 = 2 * d10_buf + d10_e1 + 64;
};

// ---- small helpers ------------------------------------------------------------------
__device__ __forceinline__ int refl101(int i, int n) {
  if (n == 1) return 0;
  while (i < 0 || i >= n) i = (i < 0) ? -i : 2 * (n - 1) - i;
  return i;
}
__device__ __forceinline__ int refl_fast(int i, int n) {
  return (unsigned)i < (unsigned)n ? i : refl101(i, n);
}

// Coarse index seen by EXPAND at a fine level of size n (coarse size m).
__device__ __forceinline__ int ext_coarse(int j, int m, int n) {
  if (m == 1) return 0;
  if (j < 0) return 1;
  if (j >= m) return (n & 1) ? m - 2 : m - 1;
  return j;
}

// x / d and x % d for 0 <= x < 2^22 and 1 <= d (work-item and tile indices):
// the float quotient is off by at most one, which one correction step fixes.
// A few instructions instead of the generic 32-bit division sequence.
__device__ __forceinline__ int div_fast(int x, int d, int& rem) {
  int q = __float2int_rz(__int2float_rn(x) * __frcp_rn(__int2float_rn(d)));
  int r = x - q * d;
  if (r < 0) {
    --q;
    r += d;
  } else if (r >= d) {
    ++q;
    r -= d;
  }
  rem = r;
  return q;
}
// Tile t of a grid ntx x nty x planes (x fastest).
struct TileXY {
  int tx, ty, pl;
};
__device__ __forceinline__ TileXY tile_of(int t, int ntx, int nty) {
  TileXY o;
  const int r = div_fast(t, ntx, o.tx);
  o.pl = div_fast(r, nty, o.ty);
  return o;
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 splat(float v) { return make_float2(v, v); }

// (cos(pi t), sin(pi t)).  The argument is reduced to r = t - 2 round(t/2) in
// [-1, 1] (exact), the hardware sine/cosine are evaluated on pi r, and where
// |sin| < 1/2 the cosine is recomputed as +-sqrt(1 - sin^2), where the sine
// is accurate in relative terms and the hardware cosine is not.
__device__ __forceinline__ float2 cos_sin_turns(float t) {
  const float n = rintf(0.5f * t);
  const float r = fmaf(-2.f, n, t);
  const float ang = 3.14159265358979323846f * r;
  const float s = __sinf(ang);
  const float c = __cosf(ang);
  const float q = fmaf(-s, s, 1.f);
  const float cq = copysignf(q * rsqrtf(q), c);
  return make_float2(fabsf(s) < 0.5f ? cq : c, s);
}

// Horner step over the orders, P <- P w + D (complex), and Im(P w).  With
// w = e^{-i w_1 g} and D_k the a_k-weighted Fourier difference of order k,
// running k = K .. 1 gives sum_k Im(w^k D_k) = Im(P w).
__device__ __forceinline__ float2 horner(float2 P, float2 w, float2 D) {
  return make_float2(fmaf(P.x, w.x, fmaf(-P.y, w.y, D.x)), fmaf(P.x, w.y, fmaf(P.y, w.x, D.y)));
}
__device__ __forceinline__ float im_mul(float2 P, float2 w) { return fmaf(P.x, w.y, P.y * w.x); }

// Fast LLF: the sampled detail f(i - g_j) and the hat weight of sample s at
// t = g (S - 1) clamped to [0, S-1], which is 1 - a for the lower and a for
// the upper of the two samples bracketing g and 0 for the others.
__device__ __forceinline__ float fast_detail(const FastArgs& f, float i, int j) {
  const float d = fmaf(-f.tau, (float)j, i);
  return f.fm1 * d * exp2f(-f.c2 * d * d);
}
__device__ __forceinline__ float fast_pos(const FastArgs& f, float g) {
  return fminf(fmaxf(g * (float)(f.S - 1), 0.f), (float)(f.S - 1));
}
__device__ __forceinline__ float fast_hat(float t, int s) { return fmaxf(0.f, 1.f - fabsf(t - (float)s)); }

// 5-tap binomial sums without the 1/16.
__device__ __forceinline__ float tap5(float a, float b, float c, float d, float e) {
  return fmaf(6.f, c, fmaf(4.f, b + d, a + e));
}
__device__ __forceinline__ float2 tap5(float2 a, float2 b, float2 c, float2 d, float2 e) {
  return fma2(splat(6.f), c, fma2(splat(4.f), add2(b, d), add2(a, e)));
}

// ---- mbarrier + TMA ------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (TMA) writes to the same buffer.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ uint32_t mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok;
}
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z,
                                          uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(saddr(b))
      : "memory");
}

__device__ __forceinline__ void tma_load4(void* dst, const CUtensorMap* map, int x, int y, int z, int v,
                                          uint64_t* b) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(v), "r"(saddr(b))
      : "memory");
}

// TMA store of a 4-D box from shared memory (bulk-group completion), and
// the bulk-group accounting of the issuing thread: commit the stores issued
// so far as a group; wait until at most N groups are pending, for their
// reads of shared memory (.read) or for their completion.
__device__ __forceinline__ void tma_store4(const CUtensorMap* map, const void* src, int x, int y, int z, int v) {
  asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(saddr(src)), "r"(x), "r"(y), "r"(z), "r"(v)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// the per-warp Z_1 staging boxes of the level-0 REDUCE are TMA store sources,
// which must start on 128-byte boundaries
static_assert(Smem<8>::up0_st / (kThreads / 32) % 128 == 0 && Smem<4>::up0_st / (kThreads / 32) % 128 == 0,
              "TMA store sources start on 128-byte boundaries");

// Status block of a run (device, zeroed when it is allocated): word 0 holds
// the fault bits a bounded wait sets when it gives up, words 1..2 a grid
// barrier's arrivals and generation, words 4..5 an optional shorter wait
// limit in SM cycles (0: the default of about 2 s), word 6 arrivals a grid
// barrier waits for beyond the grid (0 normally; a test sets it to make the
// barrier's wait run out).  All of it lies in the first 64 bytes.
constexpr int kStatusLimitWord = 4;
constexpr int kStatusExtraArrivals = 6;

// Bounded waits give up after about 2 s of SM clock, or after the status
// block's shorter limit.
constexpr long long kWaitCycles = 4000000000LL;
__device__ __forceinline__ long long wait_limit(const unsigned* status) {
  if (!status) return kWaitCycles;
  const long long v = *reinterpret_cast<const volatile long long*>(status + kStatusLimitWord);
  return (v > 0 && v < kWaitCycles) ? v : kWaitCycles;
}

// Bounded wait on an mbarrier phase.  The outcome is made uniform over the
// CTA; on a timeout the fault word records it and the caller leaves the
// kernel.
__device__ __forceinline__ bool mbar_wait_cta(uint64_t* b, uint32_t parity, unsigned* fault) {
  int ok = 1;
  if (!mbar_test(b, parity)) {
    const long long lim = wait_limit(fault);
    const long long t0 = clock64();
    while (!mbar_test(b, parity)) {
      if (clock64() - t0 > lim) {
        ok = 0;
        break;
      }
    }
  }
  const int all = __syncthreads_and(ok);
  if (!all && threadIdx.x == 0 && fault) atomicOr(fault, 1u);
  return all != 0;
}

// Bounded wait on an mbarrier phase by the calling thread alone (no CTA
// barrier).  On a timeout, or once another thread of the CTA has timed out,
// the fault word and the CTA's shared abort flag are set; the CTA leaves at
// its next barrier, where every thread reads the flag.
__device__ __forceinline__ void mbar_wait_thread(uint64_t* b, uint32_t parity, unsigned* fault,
                                                 volatile int* abort) {
  if (mbar_test(b, parity)) return;
  const long long lim = wait_limit(fault);
  const long long t0 = clock64();
  while (!mbar_test(b, parity)) {
    if (*abort || clock64() - t0 > lim) {
      if (fault) atomicOr(fault, 1u);
      *abort = 1;
      return;
    }
  }
}

// Rewrites the out-of-range cells of a staged box (planes x bh x bw elements
// of type E, box origin (x0, y0), valid extent w x h) from their sources
// under `map` (reflect-101 or the EXPAND extension): rows first, then
// columns, so that corners take both mappings.  Only the out-of-range rows
// and columns are visited.  Cells whose source lies outside the box keep
// TMA's zero fill (they feed no stored output).
template <typename E, typename MapY, typename MapX>
__device__ __forceinline__ void fix_borders(E* buf, int planes, int bh, int bw, int x0, int y0,
                                            int w, int h, MapY mapy, MapX mapx) {
  if (x0 >= 0 && y0 >= 0 && x0 + bw <= w && y0 + bh <= h) return;   // window inside the level
  const int top = min(max(-y0, 0), bh), bot = min(max(y0 + bh - h, 0), bh - top);
  const int lft = min(max(-x0, 0), bw), rgt = min(max(x0 + bw - w, 0), bw - lft);
  if (top + bot > 0) {
    const int nr = top + bot, n = planes * nr * bw;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
      const int pl = idx / (nr * bw), rem = idx - pl * nr * bw;
      const int ri = rem / bw, c = rem - ri * bw;
      const int r = ri < top ? ri : bh - bot + (ri - top);
      const int sr = mapy(y0 + r) - y0;
      if (sr >= 0 && sr < bh) buf[(pl * bh + r) * bw + c] = buf[(pl * bh + sr) * bw + c];
    }
    __syncthreads();
  }
  if (lft + rgt > 0) {
    const int nc = lft + rgt, n = planes * bh * nc;
    for (int idx = threadIdx.x; idx < n; idx += kThreads) {
      const int pl = idx / (bh * nc), rem = idx - pl * bh * nc;
      const int r = rem / nc, ci = rem - r * nc;
      const int c = ci < lft ? ci : bw - rgt + (ci - lft);
      const int sc = mapx(x0 + c) - x0;
      if (sc >= 0 && sc < bw) buf[(pl * bh + r) * bw + c] = buf[(pl * bh + r) * bw + sc];
    }
    __syncthreads();
  }
}

}  // namespace fllf
