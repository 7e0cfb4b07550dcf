// fllf_device.cuh -- device tile functions of the Fourier LLF hot path (sm_103a).
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
// Four tile functions implement the path; each is a __device__ function of
// (tile, plane) so that the per-stage kernels and the batched persistent
// kernel share them:
//   up0_tile    level 0 -> 1: trig of I on the fly + REDUCE of I and all Z.
//   up_tile     level l -> l+1 (l >= 1): REDUCE of G_l and Z_l.
//   down_tile   level l >= 1: expand-subtract-accumulate of the 2K pyramids
//               fused with the residual collapse; writes E_l only.
//   down0_tile  level 0: the same with the Z_0 cancellation, writes O.
// The 2K Laplacian pyramids are never written to memory.
//
// Borders: reflect-101 at every level for REDUCE; EXPAND is zero insertion
// followed by the kernel with reflect-101 at the fine size, which on the
// coarse grid means index -1 -> 1 and index m -> m-2 (fine size odd) or m-1
// (fine size even); a coarse level of size 1 expands to the identity.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace fllf {

constexpr int kThreads = 256;  // every tile function runs with 256 threads
constexpr int kKC = 4;         // complex orders processed per shared-memory pass

// ---- REDUCE tiling: 32 x 14 coarse outputs per tile --------------------------
constexpr int kUpTW = 32;                      // coarse columns per tile
constexpr int kUpTH = 14;                      // coarse rows per tile
constexpr int kUpRun = 4;                      // coarse outputs per horizontal item
constexpr int kUpSeg = kUpTW / kUpRun;         // items per input row
constexpr int kUpIR = 2 * kUpTH + 3;           // fine input rows per tile
constexpr int kUpIPX = 2 * kUpRun + 3;         // fine inputs per item
constexpr int kUpItems = kUpIR * kUpSeg;       // 248 horizontal items
constexpr int kUpVRows = kUpTH / 2;            // coarse rows per vertical thread
static_assert(kUpItems <= kThreads, "REDUCE items exceed the block");
static_assert(kKC * kUpTW * 2 == kThreads, "vertical REDUCE mapping");

// ---- combine tiling: 64 x 32 fine outputs per tile ------------------------------
constexpr int kDnOW = 64;                      // fine columns per tile
constexpr int kDnOH = 32;                      // fine rows per tile
constexpr int kDnCW = kDnOW / 2 + 2;           // coarse columns staged (34)
constexpr int kDnCH = kDnOH / 2 + 2;           // coarse rows staged (18)
static_assert((kDnOW / 4) * (kDnOH / 2) == kThreads, "combine thread mapping");

constexpr size_t kUpSmemBytes =
    sizeof(float2) * kKC * kUpIR * kUpTW + sizeof(float) * kUpIR * kUpTW;
constexpr size_t kDnSmemBytes =
    sizeof(float2) * kKC * kDnCH * kDnCW + sizeof(float) * kDnCH * kDnCW;

// ---- storage of one complex Fourier sample (C~, S~) ---------------------------
template <typename S> struct Cplx;
template <> struct Cplx<float> {
  using T = float2;
  static __device__ __forceinline__ float2 ld(const T* p) { return *p; }
  static __device__ __forceinline__ void st(T* p, float2 v) { *p = v; }
};
template <> struct Cplx<__half> {
  using T = __half2;
  static __device__ __forceinline__ float2 ld(const T* p) { return __half22float2(*p); }
  static __device__ __forceinline__ void st(T* p, float2 v) { *p = __float22half2_rn(v); }
};
template <> struct Cplx<__nv_bfloat16> {
  using T = __nv_bfloat162;
  static __device__ __forceinline__ float2 ld(const T* p) { return __bfloat1622float2(*p); }
  static __device__ __forceinline__ void st(T* p, float2 v) { *p = __float22bfloat162_rn(v); }
};

// One pyramid level of every plane of a batch.
struct Level {
  int h, w;             // level size
  int pitch;            // row pitch in elements (floats for G/E, complex for Z)
  long long gplane;     // elements between planes of G and E
  long long zk;         // complex elements between orders of Z
  long long zplane;     // complex elements between planes of Z
  float* G;             // guide level G_l[I] (may be null when unused)
  void* Z;              // K complex Fourier planes
  float* E;             // residual E_l (null at l = levels-1)
};

struct Up0Args {
  const float* I;       // level-0 input planes, pitch w0, plane stride h0*w0
  int h0, w0;
  Level dst;            // level 1
  int K;
  float turns;          // 2/T: w_1 x = pi * (turns * x)
};

struct UpArgs {
  Level src;            // level l >= 1
  Level dst;            // level l+1
  int K;
  int write_g;          // G_{l+1} needed (l+1 <= levels-2)
};

struct DownArgs {
  Level fine;           // level l >= 1: G, Z read, E written
  Level coarse;         // level l+1: Z and (if has_e) E read
  const float* a;       // a_1..a_K (float32)
  int K;
  float turns;
  int has_e;            // E_{l+1} exists (l+1 <= levels-2)
};

struct Down0Args {
  const float* I;       // level-0 input, pitch w0
  float* O;             // level-0 output, pitch w0
  int h0, w0;
  Level coarse;         // level 1
  const float* a;
  int K;
  float turns;
  int has_e;            // E_1 exists (levels >= 3)
};

__device__ __forceinline__ int refl101(int i, int n) {
  if (n == 1) return 0;
  while (i < 0 || i >= n) i = (i < 0) ? -i : 2 * (n - 1) - i;
  return i;
}

// Coarse index seen by EXPAND at a fine level of size n (coarse size m).
__device__ __forceinline__ int ext_coarse(int j, int m, int n) {
  if (m == 1) return 0;
  if (j < 0) return 1;
  if (j >= m) return (n & 1) ? m - 2 : m - 1;
  return j;
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 f2fma(float s, float2 a, float2 b) {
  return make_float2(fmaf(s, a.x, b.x), fmaf(s, a.y, b.y));
}

// 5-tap binomial sum of v[2q..2q+4] without the 1/16.
template <typename V>
__device__ __forceinline__ V tap5(const V& a, const V& b, const V& c, const V& d, const V& e);
template <>
__device__ __forceinline__ float tap5<float>(const float& a, const float& b, const float& c,
                                             const float& d, const float& e) {
  return fmaf(6.f, c, fmaf(4.f, b + d, a + e));
}
template <>
__device__ __forceinline__ float2 tap5<float2>(const float2& a, const float2& b, const float2& c,
                                               const float2& d, const float2& e) {
  return f2fma(6.f, c, f2fma(4.f, f2add(b, d), f2add(a, e)));
}

// ---------------------------------------------------------------------------------
// Vertical REDUCE of a horizontal-pass buffer (rows 2j..2j+4 -> coarse row j).
// buf: [kUpIR][kUpTW] (row-major), scale = 1/256.
template <typename V, typename Store>
__device__ __forceinline__ void up_vertical(const V* buf, int col, int grp, int x, int y0,
                                            int h, int w, Store store) {
  const int r0 = 2 * kUpVRows * grp;
  V win[2 * kUpVRows + 3];
#pragma unroll
  for (int t = 0; t < 2 * kUpVRows + 3; ++t) win[t] = buf[(r0 + t) * kUpTW + col];
  if (x >= w) return;
#pragma unroll
  for (int j = 0; j < kUpVRows; ++j) {
    const int y = y0 + grp * kUpVRows + j;
    if (y < h) store(y, tap5<V>(win[2 * j], win[2 * j + 1], win[2 * j + 2], win[2 * j + 3], win[2 * j + 4]));
  }
}

// ---------------------------------------------------------------------------------
// up0: level 0 -> 1.  Each horizontal item holds 11 fine pixels of one input
// row; it evaluates e^{i k w_1 x} for k = 1..K by the Chebyshev recurrence
// cos((k+1)t) = 2 cos t cos kt - cos((k-1)t) (same for sin) from one
// sincospi per pixel, and writes 4 horizontally reduced complex values per
// order into shared memory; the vertical pass finishes REDUCE and stores Z_1.
template <typename S>
__device__ void up0_tile(const Up0Args& a, int tx, int ty, int plane, unsigned char* smem) {
  using CT = typename Cplx<S>::T;
  float2* hz = reinterpret_cast<float2*>(smem);
  float* hg = reinterpret_cast<float*>(hz + kKC * kUpIR * kUpTW);
  const int tid = threadIdx.x;
  const int X1 = tx * kUpTW, Y1 = ty * kUpTH;
  const float* Ip = a.I + (long long)plane * a.h0 * a.w0;

  const bool item = tid < kUpItems;
  const int r = tid / kUpSeg, s = tid % kUpSeg;
  float two_c[kUpIPX], cp[kUpIPX], cc[kUpIPX], sp[kUpIPX], sc[kUpIPX];
  if (item) {
    const int gy = refl101(2 * Y1 - 2 + r, a.h0);
    float v[kUpIPX];
#pragma unroll
    for (int j = 0; j < kUpIPX; ++j) {
      const int gx = refl101(2 * X1 - 2 + 2 * kUpRun * s + j, a.w0);
      v[j] = __ldg(Ip + (long long)gy * a.w0 + gx);
      float sn, cs;
      sincospif(a.turns * v[j], &sn, &cs);
      two_c[j] = 2.f * cs; cp[j] = 1.f; sp[j] = 0.f; cc[j] = cs; sc[j] = sn;
    }
#pragma unroll
    for (int q = 0; q < kUpRun; ++q)
      hg[r * kUpTW + kUpRun * s + q] = tap5<float>(v[2 * q], v[2 * q + 1], v[2 * q + 2], v[2 * q + 3], v[2 * q + 4]);
  }
  const int nch = (a.K + kKC - 1) / kKC;
  CT* Z = reinterpret_cast<CT*>(a.dst.Z) + (long long)plane * a.dst.zplane;
  for (int ch = 0; ch < nch; ++ch) {
    if (item) {
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
#pragma unroll
        for (int q = 0; q < kUpRun; ++q) {
          const float re = tap5<float>(cc[2 * q], cc[2 * q + 1], cc[2 * q + 2], cc[2 * q + 3], cc[2 * q + 4]);
          const float im = tap5<float>(sc[2 * q], sc[2 * q + 1], sc[2 * q + 2], sc[2 * q + 3], sc[2 * q + 4]);
          hz[(kk * kUpIR + r) * kUpTW + kUpRun * s + q] = make_float2(re, im);
        }
#pragma unroll
        for (int j = 0; j < kUpIPX; ++j) {
          const float cn = fmaf(two_c[j], cc[j], -cp[j]);
          const float sn = fmaf(two_c[j], sc[j], -sp[j]);
          cp[j] = cc[j]; cc[j] = cn; sp[j] = sc[j]; sc[j] = sn;
        }
      }
    }
    __syncthreads();
    {
      const int kk = tid / (2 * kUpTW), grp = (tid / kUpTW) & 1, col = tid % kUpTW;
      const int k = ch * kKC + kk;
      if (k < a.K) {
        CT* Zk = Z + (long long)k * a.dst.zk;
        const int x = X1 + col;
        const int pitch = a.dst.pitch;
        up_vertical<float2>(hz + kk * kUpIR * kUpTW, col, grp, x, Y1, a.dst.h, a.dst.w,
                            [&](int y, float2 v) {
                              Cplx<S>::st(Zk + (long long)y * pitch + x,
                                          make_float2(v.x * (1.f / 256.f), v.y * (1.f / 256.f)));
                            });
      }
      if (ch == 0 && tid < 2 * kUpTW) {
        float* G = a.dst.G + (long long)plane * a.dst.gplane;
        const int x = X1 + col;
        const int pitch = a.dst.pitch;
        up_vertical<float>(hg, col, grp, x, Y1, a.dst.h, a.dst.w,
                           [&](int y, float v) { G[(long long)y * pitch + x] = v * (1.f / 256.f); });
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// up: level l -> l+1 for l >= 1 (REDUCE of G_l and of the K complex planes).
template <typename S>
__device__ void up_tile(const UpArgs& a, int tx, int ty, int plane, unsigned char* smem) {
  using CT = typename Cplx<S>::T;
  float2* hz = reinterpret_cast<float2*>(smem);
  float* hg = reinterpret_cast<float*>(hz + kKC * kUpIR * kUpTW);
  const int tid = threadIdx.x;
  const int X1 = tx * kUpTW, Y1 = ty * kUpTH;
  const bool item = tid < kUpItems;
  const int r = tid / kUpSeg, s = tid % kUpSeg;
  int gy = 0, gx[kUpIPX];
  if (item) {
    gy = refl101(2 * Y1 - 2 + r, a.src.h);
#pragma unroll
    for (int j = 0; j < kUpIPX; ++j) gx[j] = refl101(2 * X1 - 2 + 2 * kUpRun * s + j, a.src.w);
    if (a.write_g) {
      const float* G = a.src.G + (long long)plane * a.src.gplane + (long long)gy * a.src.pitch;
      float v[kUpIPX];
#pragma unroll
      for (int j = 0; j < kUpIPX; ++j) v[j] = __ldg(G + gx[j]);
#pragma unroll
      for (int q = 0; q < kUpRun; ++q)
        hg[r * kUpTW + kUpRun * s + q] = tap5<float>(v[2 * q], v[2 * q + 1], v[2 * q + 2], v[2 * q + 3], v[2 * q + 4]);
    }
  }
  const int nch = (a.K + kKC - 1) / kKC;
  const CT* Zs = reinterpret_cast<const CT*>(a.src.Z) + (long long)plane * a.src.zplane;
  CT* Zd = reinterpret_cast<CT*>(a.dst.Z) + (long long)plane * a.dst.zplane;
  for (int ch = 0; ch < nch; ++ch) {
    if (item) {
#pragma unroll
      for (int kk = 0; kk < kKC; ++kk) {
        const int k = ch * kKC + kk;
        if (k < a.K) {
          const CT* row = Zs + (long long)k * a.src.zk + (long long)gy * a.src.pitch;
          float2 v[kUpIPX];
#pragma unroll
          for (int j = 0; j < kUpIPX; ++j) v[j] = Cplx<S>::ld(row + gx[j]);
#pragma unroll
          for (int q = 0; q < kUpRun; ++q)
            hz[(kk * kUpIR + r) * kUpTW + kUpRun * s + q] =
                tap5<float2>(v[2 * q], v[2 * q + 1], v[2 * q + 2], v[2 * q + 3], v[2 * q + 4]);
        }
      }
    }
    __syncthreads();
    {
      const int kk = tid / (2 * kUpTW), grp = (tid / kUpTW) & 1, col = tid % kUpTW;
      const int k = ch * kKC + kk;
      if (k < a.K) {
        CT* Zk = Zd + (long long)k * a.dst.zk;
        const int x = X1 + col;
        const int pitch = a.dst.pitch;
        up_vertical<float2>(hz + kk * kUpIR * kUpTW, col, grp, x, Y1, a.dst.h, a.dst.w,
                            [&](int y, float2 v) {
                              Cplx<S>::st(Zk + (long long)y * pitch + x,
                                          make_float2(v.x * (1.f / 256.f), v.y * (1.f / 256.f)));
                            });
      }
      if (ch == 0 && a.write_g && tid < 2 * kUpTW) {
        float* G = a.dst.G + (long long)plane * a.dst.gplane;
        const int x = X1 + col;
        const int pitch = a.dst.pitch;
        up_vertical<float>(hg, col, grp, x, Y1, a.dst.h, a.dst.w,
                           [&](int y, float v) { G[(long long)y * pitch + x] = v * (1.f / 256.f); });
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Combine helpers.  A thread owns fine rows 2j, 2j+1 and fine columns
// 4c..4c+3 of the tile, i.e. coarse rows j-1..j+1 and coarse columns
// 2c-1..2c+2 (tile-local +1 offsets below).  EXPAND of the 3 x 4 coarse
// window gives the 2 x 4 fine values; the weights are 1/8 (1, 6, 1) at even
// fine positions and 1/2 (1, 1) at odd ones, per axis.

// Unscaled 2-D EXPAND of a 3 x 4 window into 2 x 4 fine values; the per-position
// scales (1/64, 1/16, 1/16, 1/4) are applied by the caller.
template <typename V>
__device__ __forceinline__ void expand_2x4(const V w[3][4], V out[2][4]) {
  V ve[4], vo[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    if constexpr (sizeof(V) == sizeof(float)) {
      ve[c] = fmaf(6.f, w[1][c], w[0][c] + w[2][c]);
      vo[c] = w[1][c] + w[2][c];
    } else {
      ve[c] = f2fma(6.f, w[1][c], f2add(w[0][c], w[2][c]));
      vo[c] = f2add(w[1][c], w[2][c]);
    }
  }
  const V* rows[2] = {ve, vo};
#pragma unroll
  for (int rr = 0; rr < 2; ++rr) {
    const V* v = rows[rr];
    if constexpr (sizeof(V) == sizeof(float)) {
      out[rr][0] = fmaf(6.f, v[1], v[0] + v[2]);
      out[rr][1] = v[1] + v[2];
      out[rr][2] = fmaf(6.f, v[2], v[1] + v[3]);
      out[rr][3] = v[2] + v[3];
    } else {
      out[rr][0] = f2fma(6.f, v[1], f2add(v[0], v[2]));
      out[rr][1] = f2add(v[1], v[2]);
      out[rr][2] = f2fma(6.f, v[2], f2add(v[1], v[3]));
      out[rr][3] = f2add(v[2], v[3]);
    }
  }
}

// EXPAND scale of fine position (row parity rr, column index cc in 0..3).
__device__ __forceinline__ float expand_scale(int rr, int cc) {
  const float sr = rr ? 0.5f : 0.125f;
  const float sc = (cc & 1) ? 0.5f : 0.125f;
  return sr * sc;
}

// Stage one chunk of coarse complex planes (orders k0..k0+kKC-1) and,
// optionally, the coarse residual into shared memory.
template <typename S>
__device__ __forceinline__ void stage_coarse(const Level& c, int plane, int cy0, int cx0,
                                             int fine_h, int fine_w, int k0, int K,
                                             float2* cz, float* ce, bool with_e) {
  using CT = typename Cplx<S>::T;
  const CT* Z = reinterpret_cast<const CT*>(c.Z) + (long long)plane * c.zplane;
  constexpr int n = kKC * kDnCH * kDnCW;
  for (int idx = threadIdx.x; idx < n; idx += kThreads) {
    const int kk = idx / (kDnCH * kDnCW);
    const int rem = idx - kk * kDnCH * kDnCW;
    const int rr = rem / kDnCW, cc = rem - rr * kDnCW;
    const int k = k0 + kk;
    if (k < K) {
      const int y = ext_coarse(cy0 + rr, c.h, fine_h);
      const int x = ext_coarse(cx0 + cc, c.w, fine_w);
      cz[idx] = Cplx<S>::ld(Z + (long long)k * c.zk + (long long)y * c.pitch + x);
    }
  }
  if (with_e) {
    const float* E = c.E + (long long)plane * c.gplane;
    for (int idx = threadIdx.x; idx < kDnCH * kDnCW; idx += kThreads) {
      const int rr = idx / kDnCW, cc = idx - rr * kDnCW;
      const int y = ext_coarse(cy0 + rr, c.h, fine_h);
      const int x = ext_coarse(cx0 + cc, c.w, fine_w);
      ce[idx] = __ldg(E + (long long)y * c.pitch + x);
    }
  }
}

// Shared body of the combine at level l (fine level), LEVEL0 selects the
// level-0 form (g = I_p, no Z_0 term, output O = I + E_0).
template <typename S, bool LEVEL0>
__device__ __forceinline__ void combine_tile(const Level* fine, const float* I, float* O, int h,
                                             int w, const Level& coarse, const float* acoef, int K,
                                             float turns, int has_e, int tx, int ty, int plane,
                                             unsigned char* smem) {
  using CT = typename Cplx<S>::T;
  float2* cz = reinterpret_cast<float2*>(smem);
  float* ce = reinterpret_cast<float*>(cz + kKC * kDnCH * kDnCW);
  const int tid = threadIdx.x;
  const int X0 = tx * kDnOW, Y0 = ty * kDnOH;
  const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
  const int tr = tid / (kDnOW / 4), tc = tid % (kDnOW / 4);
  const int fy0 = Y0 + 2 * tr, fx0 = X0 + 4 * tc;

  // Guide value g and its Chebyshev state for the thread's 2 x 4 pixels.
  float two_c[2][4], cp[2][4], cc[2][4], sp[2][4], sc[2][4], acc[2][4];
  const long long gpitch = LEVEL0 ? (long long)w : (long long)fine->pitch;
  const float* gsrc = LEVEL0 ? I + (long long)plane * h * w
                             : fine->G + (long long)plane * fine->gplane;
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int y = min(fy0 + rr, h - 1), x = min(fx0 + q, w - 1);
      const float g = __ldg(gsrc + (long long)y * gpitch + x);
      float sn, cs;
      sincospif(turns * g, &sn, &cs);
      two_c[rr][q] = 2.f * cs; cp[rr][q] = 1.f; sp[rr][q] = 0.f; cc[rr][q] = cs; sc[rr][q] = sn;
      acc[rr][q] = LEVEL0 ? g : 0.f;
    }

  const CT* Zf = nullptr;
  if constexpr (!LEVEL0) Zf = reinterpret_cast<const CT*>(fine->Z) + (long long)plane * fine->zplane;

  const int nch = (K + kKC - 1) / kKC;
  for (int ch = 0; ch < nch; ++ch) {
    stage_coarse<S>(coarse, plane, cy0, cx0, h, w, ch * kKC, K, cz, ce, ch == 0 && has_e);
    __syncthreads();
    if (ch == 0 && has_e) {
      float win[3][4], up[2][4];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) win[i][q] = ce[(tr + i) * kDnCW + 2 * tc + q];
      expand_2x4<float>(win, up);
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[rr][q] = fmaf(expand_scale(rr, q), up[rr][q], acc[rr][q]);
    }
#pragma unroll
    for (int kk = 0; kk < kKC; ++kk) {
      const int k = ch * kKC + kk;
      if (k < K) {
        const float ak = __ldg(acoef + k);
        float2 win[3][4], up[2][4];
        const float2* base = cz + kk * kDnCH * kDnCW;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) win[i][q] = base[(tr + i) * kDnCW + 2 * tc + q];
        expand_2x4<float2>(win, up);
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float sfac = expand_scale(rr, q);
            float t;
            if constexpr (LEVEL0) {
              // Delta_0 = -sum_k a_k Im(e^{-i k t} up(Z_1))
              t = fmaf(cc[rr][q], up[rr][q].y, -sc[rr][q] * up[rr][q].x);
              acc[rr][q] = fmaf(-ak * sfac, t, acc[rr][q]);
            } else {
              const int y = min(fy0 + rr, h - 1), x = min(fx0 + q, w - 1);
              const float2 z = Cplx<S>::ld(Zf + (long long)k * fine->zk + (long long)y * fine->pitch + x);
              const float2 d = make_float2(fmaf(-sfac, up[rr][q].x, z.x), fmaf(-sfac, up[rr][q].y, z.y));
              t = fmaf(cc[rr][q], d.y, -sc[rr][q] * d.x);
              acc[rr][q] = fmaf(ak, t, acc[rr][q]);
            }
            const float cn = fmaf(two_c[rr][q], cc[rr][q], -cp[rr][q]);
            const float sn = fmaf(two_c[rr][q], sc[rr][q], -sp[rr][q]);
            cp[rr][q] = cc[rr][q]; cc[rr][q] = cn; sp[rr][q] = sc[rr][q]; sc[rr][q] = sn;
          }
      }
    }
    __syncthreads();
  }

  float* dst;
  long long dpitch;
  if constexpr (LEVEL0) {
    dst = O + (long long)plane * h * w;
    dpitch = w;
  } else {
    dst = fine->E + (long long)plane * fine->gplane;
    dpitch = fine->pitch;
  }
#pragma unroll
  for (int rr = 0; rr < 2; ++rr)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int y = fy0 + rr, x = fx0 + q;
      if (y < h && x < w) dst[(long long)y * dpitch + x] = acc[rr][q];
    }
}

template <typename S>
__device__ void down_tile(const DownArgs& a, int tx, int ty, int plane, unsigned char* smem) {
  combine_tile<S, false>(&a.fine, nullptr, nullptr, a.fine.h, a.fine.w, a.coarse, a.a, a.K, a.turns,
                         a.has_e, tx, ty, plane, smem);
}

template <typename S>
__device__ void down0_tile(const Down0Args& a, int tx, int ty, int plane, unsigned char* smem) {
  combine_tile<S, true>(nullptr, a.I, a.O, a.h0, a.w0, a.coarse, a.a, a.K, a.turns, a.has_e, tx, ty,
                        plane, smem);
}

}  // namespace fllf
