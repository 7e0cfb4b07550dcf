// fllf_kernels.inl -- the kernels of the path for one storage type
// FLLF_STORAGE; included by one translation unit per precision.
//
// Every stage is a persistent device function over a stream of work items
// (tiles, or (tile, chunk of orders) pairs).  CTA b of a grid of G takes
// items b, b + G, ...; a 2-deep ring of shared-memory buffers keeps the TMA
// copy of the next item in flight while the current one is computed.  Items
// are mapped to their image by a resolver: one image for the per-image
// kernels (arguments in the parameter block), many images for the batched
// kernels (argument tables in device memory, with prefix sums of the item
// counts).
#include "fllf_launch.h"

namespace fllf {

namespace {

// Waits (bounded) for a TMA copy still in flight before a CTA leaves early.
__device__ __forceinline__ void drain(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(b, parity) && clock64() - t0 < kWaitCycles) {
  }
}

// Completed uses of the two TMA buffers of a CTA (identical in every thread);
// the parity of a buffer's next phase is use[buf] & 1.  Carried across the
// stages of the chained kernel.
struct Pipe {
  uint32_t use[2];
};

__device__ __forceinline__ void init_bars(uint64_t* bar) {
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
}

// Entry j of a prefix table holding item x (prefix[0] = 0, prefix[n] = total).
__device__ __forceinline__ int find_entry(const int* prefix, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(prefix + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------------------
// up0: level 0 -> 1.  Item = tile of 32 x 14 level-1 outputs.  Item (row r,
// segment s) of the horizontal pass holds 11 fine pixels of one staged input
// row; it evaluates e^{i k w_1 x} for k = 1..K with the Chebyshev recurrence
// z_{k+1} = 2 cos(w_1 x) z_k - z_{k-1} (one packed FMA per order) from one
// hardware sincos per pixel and writes 4 horizontally reduced complex values
// per order to column-major staging; the vertical pass finishes REDUCE
// (Eq. (1)) and stores G_1 and Z_1.
__device__ __forceinline__ int up0_tiles(const Up0Args& a) {
  return cdiv(a.dst.w, kUpTW) * cdiv(a.dst.h, kUpTH) * a.planes;
}

template <typename S, typename Res>
__device__ __forceinline__ bool stage_up0(Res res, int total, unsigned char* smem, uint64_t* bar,
                                          Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  float* itb[2] = {reinterpret_cast<float*>(smem), reinterpret_cast<float*>(smem + SM::up0_it)};
  float2* hz = reinterpret_cast<float2*>(smem + 2 * SM::up0_it);
  float* hg = reinterpret_cast<float*>(smem + 2 * SM::up0_it + align128(SM::up0_hz));
  const int tid = threadIdx.x;
  auto issue = [&](const Up0Args& a, int t, int buf) {
    const int ntx = cdiv(a.dst.w, kUpTW), nty = cdiv(a.dst.h, kUpTH);
    const int tx = t % ntx, r = t / ntx, ty = r % nty, pl = r / nty;
    mbar_expect_tx(&bar[buf], sizeof(float) * kUpIR * kUpIW);
    tma_load3(itb[buf], &a.imap, 2 * tx * kUpTW - 4, 2 * ty * kUpTH - 2, pl, &bar[buf]);
  };
  if (b < total && tid == 0) {
    int lt;
    const Up0Args* a0 = res(b, lt);
    if (a0->use_tma) {
      fence_proxy_async();
      issue(*a0, lt, 0);
    }
  }
  int n = 0;
  for (int gt = b; gt < total; gt += G, ++n) {
    const int buf = n & 1;
    int t;
    const Up0Args& a = *res(gt, t);
    const int ntx = cdiv(a.dst.w, kUpTW), nty = cdiv(a.dst.h, kUpTH);
    const int tx = t % ntx, rt = t / ntx, ty = rt % nty, pl = rt / nty;
    const int X1 = tx * kUpTW, Y1 = ty * kUpTH;
    const int xs = 2 * X1 - 4, ys = 2 * Y1 - 2;
    const int nch = cdiv(a.K, kKC);
    float* it = itb[buf];
    const int gn = gt + G;
    if (tid == 0 && gn < total) {
      int tn;
      const Up0Args* an = res(gn, tn);
      if (an->use_tma) {
        fence_proxy_async();
        issue(*an, tn, buf ^ 1);
      }
    }
    if (a.use_tma) {
      if (!mbar_wait_cta(&bar[buf], pp.use[buf] & 1, a.fault)) {
        if (tid == 0 && gn < total) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
        return false;
      }
      ++pp.use[buf];
      fix_borders(it, 1, kUpIR, kUpIW, xs, ys, a.w0, a.h0,
                  [&](int y) { return refl101(y, a.h0); }, [&](int x) { return refl101(x, a.w0); });
    } else {
      const float* Ip = a.I + (long long)pl * a.h0 * a.w0;
      for (int idx = tid; idx < kUpIR * kUpIW; idx += kThreads) {
        const int rr = idx / kUpIW, cc = idx - rr * kUpIW;
        it[idx] = __ldg(Ip + (long long)refl_fast(ys + rr, a.h0) * a.w0 + refl_fast(xs + cc, a.w0));
      }
      __syncthreads();
    }

    // Warp s owns coarse columns 4s .. 4s+3 of the tile, and does both passes
    // for them; only a warp sync separates the passes.
    // Horizontal pass: lane r takes fine row r of the run segment. The run's 11
    // inputs (columns 8s+2 .. 8s+12 of the staged row) are read as four 16-byte
    // words: rows are 72 floats apart, so scalar reads of consecutive rows
    // would hit the same 4 banks.
    const int r = tid & 31, s = tid >> 5;
    const bool item = r < kUpIR;
    float2* hzw = hz + s * (kKC * kUpRun * kUpCS);  // [order][column][fine row]
    float* hgw = hg + s * (kUpRun * kUpCS);          // [column][fine row]
    float2 zc[kUpIPX], zp[kUpIPX], tc[kUpIPX];
    if (item) {
      float v[kUpIPX];
      {
        const float4* row = reinterpret_cast<const float4*>(it + r * kUpIW + 2 * kUpRun * s);
        const float4 q0 = row[0], q1 = row[1], q2 = row[2], q3 = row[3];
        v[0] = q0.z; v[1] = q0.w;
        v[2] = q1.x; v[3] = q1.y; v[4] = q1.z; v[5] = q1.w;
        v[6] = q2.x; v[7] = q2.y; v[8] = q2.z; v[9] = q2.w;
        v[10] = q3.x;
      }
#pragma unroll
      for (int j = 0; j < kUpIPX; ++j) {
        const float2 z = cos_sin_turns(a.turns * v[j]);
        zc[j] = z;
        zp[j] = make_float2(1.f, 0.f);
        tc[j] = splat(2.f * z.x);
      }
#pragma unroll
      for (int q = 0; q < kUpRun; ++q)
        hgw[q * kUpCS + r] = tap5(v[2 * q], v[2 * q + 1], v[2 * q + 2], v[2 * q + 3], v[2 * q + 4]);
    }
    // Every warp has read its inputs: the buffer may be refilled (the TMA
    // load of the tile after next is issued after this barrier).
    __syncthreads();
    // Vertical pass: lane = (order kk, row group grp, column q). With a column
    // stride of 36 float2 the 8 lanes of a quarter-warp read 8 distinct
    // 16-byte bank groups.
    const int vq = tid & 3, vgrp = (tid >> 2) & 1, vkk = (tid >> 3) & 3;
    const int xo = X1 + kUpRun * s + vq;
    for (int ch = 0; ch < nch; ++ch) {
      if (item) {
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
#pragma unroll
          for (int q = 0; q < kUpRun; ++q)
            hzw[(kk * kUpRun + q) * kUpCS + r] =
                tap5(zc[2 * q], zc[2 * q + 1], zc[2 * q + 2], zc[2 * q + 3], zc[2 * q + 4]);
#pragma unroll
          for (int j = 0; j < kUpIPX; ++j) {
            const float2 zn = fma2(tc[j], zc[j], make_float2(-zp[j].x, -zp[j].y));
            zp[j] = zc[j];
            zc[j] = zn;
          }
        }
      }
      __syncwarp();
      {
        const int k = ch * kKC + vkk;
        if (k < a.K && xo < a.dst.w) {
          CT* Zk = reinterpret_cast<CT*>(a.dst.Z) + (long long)pl * a.dst.zplane +
                   (long long)k * a.dst.zk + xo;
          const float4* p =
              reinterpret_cast<const float4*>(hzw + (vkk * kUpRun + vq) * kUpCS + 2 * kUpVRows * vgrp);
          float2 w[2 * kUpVRows + 4];
#pragma unroll
          for (int u = 0; u < kUpVRows + 2; ++u) {
            const float4 q4 = p[u];
            w[2 * u] = make_float2(q4.x, q4.y);
            w[2 * u + 1] = make_float2(q4.z, q4.w);
          }
#pragma unroll
          for (int j = 0; j < kUpVRows; ++j) {
            const int y = Y1 + vgrp * kUpVRows + j;
            if (y < a.dst.h)
              Cplx<S>::st(Zk + (long long)y * a.dst.pitch,
                          mul2(splat(1.f / 256.f),
                               tap5(w[2 * j], w[2 * j + 1], w[2 * j + 2], w[2 * j + 3], w[2 * j + 4])));
          }
        }
        if (ch == 0 && tid % 32 < kUpRun * kUpVRows) {
          // guide: lane = (column gq, pair of coarse rows gp)
          const int gq = (tid & 31) % kUpRun, gp = (tid & 31) / kUpRun, xg = X1 + kUpRun * s + gq;
          if (xg < a.dst.w) {
            float* Gp = a.dst.G + (long long)pl * a.dst.gplane + xg;
            const float2* p = reinterpret_cast<const float2*>(hgw + gq * kUpCS + 4 * gp);
            float w[8];  // staged rows 4gp .. 4gp+7 (6 used for the two outputs' taps + 1)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float2 q2 = p[u];
              w[2 * u] = q2.x;
              w[2 * u + 1] = q2.y;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
              const int y = Y1 + 2 * gp + j;
              if (y < a.dst.h)
                Gp[(long long)y * a.dst.pitch] =
                    (1.f / 256.f) * tap5(w[2 * j], w[2 * j + 1], w[2 * j + 2], w[2 * j + 3], w[2 * j + 4]);
            }
          }
        }
      }
      __syncwarp();
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// up: level l -> l+1 for l >= 1 (REDUCE of G_l and the K complex planes).
// Item = (tile of 30 x 16 coarse outputs, chunk of KCU orders): orders reduce
// independently, so small levels still spread over many CTAs.  TMA stages
// the 35 x 68 source box of each order of the chunk (plus G_l with chunk 0);
// the vertical pass reads one staged column per thread and keeps the reduced
// rows in registers; the horizontal pass reads 5 staged columns per output.
template <typename S>
__device__ __forceinline__ int up_items(const UpArgs& a) {
  return cdiv(a.dst.w, kRsTW) * cdiv(a.dst.h, kRsTH) * a.planes *
         cdiv(a.K, Smem<sizeof(typename Cplx<S>::T)>::up_kc);
}

template <typename S, typename Res>
__device__ __forceinline__ bool stage_up(Res res, int total, unsigned char* smem, uint64_t* bar,
                                         Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  constexpr int KCU = SM::up_kc;
  constexpr int RG = kThreads / (KCU * kRsVW);  // vertical row groups
  constexpr int VOUT = kRsTH / RG;              // coarse rows per vertical thread
  constexpr int HQ = kThreads / (KCU * kRsTW);  // horizontal row groups
  constexpr int HOUT = kRsTH / HQ;
  static_assert(RG * KCU * kRsVW == kThreads, "vertical mapping");
  static_assert(kRsTH % HQ == 0, "horizontal mapping");
  unsigned char* bufs[2] = {smem, smem + SM::up_buf};
  float2* vb = reinterpret_cast<float2*>(smem + 2 * SM::up_buf);
  float* vg = reinterpret_cast<float*>(smem + 2 * SM::up_buf + SM::up_vb);
  const int tid = threadIdx.x;
  const int nitems = b < total ? (total - b + G - 1) / G : 0;
  auto issue = [&](int gi, int buf) {
    int li;
    const UpArgs& a = *res(gi, li);
    const int nch = cdiv(a.K, KCU), t = li / nch, ch = li % nch;
    const int ntx = cdiv(a.dst.w, kRsTW), nty = cdiv(a.dst.h, kRsTH);
    const int tx = t % ntx, r = t / ntx, ty = r % nty, pl = r / nty;
    const int x = 2 * tx * kRsTW - 4, y = 2 * ty * kRsTH - 2;
    const bool g = ch == 0 && a.write_g;
    mbar_expect_tx(&bar[buf], (uint32_t)(sizeof(CT) * KCU * kRsIR * kRsBW +
                                         (g ? sizeof(float) * kRsIR * kRsBW : 0)));
    tma_load3(bufs[buf], &a.zmap, x, y, pl * a.K + ch * KCU, &bar[buf]);
    if (g) tma_load3(bufs[buf] + SM::up_src, &a.gmap, x, y, pl, &bar[buf]);
  };
  if (tid == 0 && nitems > 0) {
    fence_proxy_async();
    issue(b, 0);
  }
  for (int i = 0; i < nitems; ++i) {
    const int buf = i & 1;
    int li;
    const UpArgs& a = *res(b + i * G, li);
    const int nch = cdiv(a.K, KCU), t = li / nch, ch = li % nch;
    const int ntx = cdiv(a.dst.w, kRsTW), nty = cdiv(a.dst.h, kRsTH);
    const int tx = t % ntx, rt = t / ntx, ty = rt % nty, pl = rt / nty;
    const int X1 = tx * kRsTW, Y1 = ty * kRsTH;
    const int xs = 2 * X1 - 4, ys = 2 * Y1 - 2;
    const bool g = ch == 0 && a.write_g;
    if (tid == 0 && i + 1 < nitems) {
      fence_proxy_async();
      issue(b + (i + 1) * G, buf ^ 1);
    }
    if (!mbar_wait_cta(&bar[buf], pp.use[buf] & 1, a.fault)) {
      if (tid == 0 && i + 1 < nitems) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
      return false;
    }
    ++pp.use[buf];
    CT* src = reinterpret_cast<CT*>(bufs[buf]);
    float* gsrc = reinterpret_cast<float*>(bufs[buf] + SM::up_src);
    auto my = [&](int y) { return refl101(y, a.src.h); };
    auto mx = [&](int x) { return refl101(x, a.src.w); };
    fix_borders(src, KCU, kRsIR, kRsBW, xs, ys, a.src.w, a.src.h, my, mx);
    if (g) fix_borders(gsrc, 1, kRsIR, kRsBW, xs, ys, a.src.w, a.src.h, my, mx);

    {  // vertical half
      const int rg = tid / (KCU * kRsVW), kk = (tid / kRsVW) % KCU, c = tid % kRsVW;
      const CT* col = src + (kk * kRsIR + 2 * VOUT * rg) * kRsBW + c + 2;
      float2 v[2 * VOUT + 3];
#pragma unroll
      for (int u = 0; u < 2 * VOUT + 3; ++u) v[u] = Cplx<S>::cvt(col[u * kRsBW]);
#pragma unroll
      for (int j = 0; j < VOUT; ++j)
        vb[(kk * kRsTH + VOUT * rg + j) * kRsVW + c] =
            tap5(v[2 * j], v[2 * j + 1], v[2 * j + 2], v[2 * j + 3], v[2 * j + 4]);
      if (g) {
        const int grp = tid / kRsVW, cg = tid % kRsVW;  // 4 groups x 4 coarse rows
        const float* gc = gsrc + (8 * grp) * kRsBW + cg + 2;
        float u[11];
#pragma unroll
        for (int q = 0; q < 11; ++q) u[q] = gc[q * kRsBW];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          vg[(4 * grp + j) * kRsVW + cg] = tap5(u[2 * j], u[2 * j + 1], u[2 * j + 2], u[2 * j + 3], u[2 * j + 4]);
      }
    }
    __syncthreads();
    {  // horizontal half
      if (tid < KCU * kRsTW * HQ) {
        const int hk = tid / (kRsTW * HQ), rem = tid % (kRsTW * HQ);
        const int hq = rem / kRsTW, ic = rem % kRsTW;
        const int k = ch * KCU + hk, x = X1 + ic;
        if (k < a.K && x < a.dst.w) {
          CT* Zk = reinterpret_cast<CT*>(a.dst.Z) + (long long)pl * a.dst.zplane +
                   (long long)k * a.dst.zk + x;
#pragma unroll
          for (int j = 0; j < HOUT; ++j) {
            const int jr = hq * HOUT + j, y = Y1 + jr;
            if (y < a.dst.h) {
              const float2* p = vb + (hk * kRsTH + jr) * kRsVW + 2 * ic;
              const float4 q0 = *reinterpret_cast<const float4*>(p);
              const float4 q1 = *reinterpret_cast<const float4*>(p + 2);
              const float2 o = tap5(make_float2(q0.x, q0.y), make_float2(q0.z, q0.w),
                                    make_float2(q1.x, q1.y), make_float2(q1.z, q1.w), p[4]);
              Cplx<S>::st(Zk + (long long)y * a.dst.pitch, mul2(splat(1.f / 256.f), o));
            }
          }
        }
      }
      if (g && tid < 2 * kRsTW) {
        const int half = tid / kRsTW, ic = tid % kRsTW, x = X1 + ic;
        if (x < a.dst.w) {
          float* Gp = a.dst.G + (long long)pl * a.dst.gplane + x;
#pragma unroll
          for (int j = 0; j < kRsTH / 2; ++j) {
            const int jr = half * (kRsTH / 2) + j, y = Y1 + jr;
            if (y < a.dst.h) {
              const float* p = vg + jr * kRsVW + 2 * ic;
              Gp[(long long)y * a.dst.pitch] = (1.f / 256.f) * tap5(p[0], p[1], p[2], p[3], p[4]);
            }
          }
        }
      }
    }
    __syncthreads();
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Combine (Eq. (14) product-sum fused with the residual collapse).
// Item = (tile of 64 x 32 fine pixels, chunk of kKC orders); the chunks of a
// tile run back to back on one CTA, which keeps the per-pixel state in
// registers.  A thread owns fine rows 2j, 2j+1 and fine columns 4c..4c+3 of
// the tile (tile origin 64*tx-6), i.e. coarse rows j-1..j+1 and coarse
// columns 2c-1..2c+2, which sit at staged rows tr..tr+2 and columns
// 2tc..2tc+3.  EXPAND of the 3 x 4 complex window runs on (C~, S~) pairs
// with packed FP32x2 arithmetic; the per-pixel trig state (cos, -sin) of the
// two fine rows and the accumulators are (even row, odd row) pairs, advanced
// by complex rotation.  EXPAND weights 1/8 (1, 6, 1) at even fine positions
// and 1/2 (1, 1) at odd ones per axis are folded into the coefficients.
__device__ __forceinline__ float2 expand_scale_pair(int q) {
  return (q & 1) ? make_float2(1.f / 16.f, 1.f / 4.f) : make_float2(1.f / 64.f, 1.f / 16.f);
}

// Uniform view of the level >= 1 and level-0 combine arguments.
struct CombineView {
  const CUtensorMap* zmap;
  const CUtensorMap* emap;
  const Level* fine;    // level >= 1 only
  const float* I;       // level 0 only
  float* O;             // level 0 only
  const Level* coarse;
  const float* a;
  unsigned* fault;
  int h, w, planes, K, has_e;
  float turns;
};
__device__ __forceinline__ CombineView view_of(const DownArgs& d) {
  return CombineView{&d.zmap, &d.emap, &d.fine, nullptr, nullptr, &d.coarse, d.a, d.fault,
                     d.fine.h, d.fine.w, d.planes, d.K, d.has_e, d.turns};
}
__device__ __forceinline__ CombineView view_of(const Down0Args& d) {
  return CombineView{&d.zmap, &d.emap, nullptr, d.I, d.O, &d.coarse, d.a, d.fault,
                     d.h0, d.w0, d.planes, d.K, d.has_e, d.turns};
}
__device__ __forceinline__ int combine_tiles(const CombineView& v) {
  return cdiv(v.w + kDnX0, kDnOW) * cdiv(v.h, kDnOH) * v.planes;
}

template <typename S, bool LEVEL0, bool COH, typename Res>
__device__ __forceinline__ bool stage_combine(Res res, int total, unsigned char* smem, uint64_t* bar,
                                              Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  unsigned char* bufs[2] = {smem, smem + SM::dn_buf};
  const int tid = threadIdx.x;
  if (b >= total) return true;
  auto issue = [&](const CombineView& v, int lt, int ch, int buf) {
    const int ntx = cdiv(v.w + kDnX0, kDnOW), nty = cdiv(v.h, kDnOH);
    const int tx = lt % ntx, r = lt / ntx, ty = r % nty, pl = r / nty;
    const int cx0 = (tx * kDnOW - kDnX0) / 2 - 1, cy0 = ty * (kDnOH / 2) - 1;
    const bool e = ch == 0 && v.has_e;
    mbar_expect_tx(&bar[buf], (uint32_t)(sizeof(CT) * kKC * kDnCH * kDnCW +
                                         (e ? sizeof(float) * kDnCH * kDnCW : 0)));
    tma_load3(bufs[buf], v.zmap, cx0, cy0, pl * v.K + ch * kKC, &bar[buf]);
    if (e) tma_load3(bufs[buf] + SM::dn_z, v.emap, cx0, cy0, pl, &bar[buf]);
  };
  int t = b, lt = 0, ch = 0;
  CombineView v = res(t, lt);
  int nch = cdiv(v.K, kKC);
  if (tid == 0) {
    fence_proxy_async();
    issue(v, lt, 0, 0);
  }

  const int tc = tid % (kDnOW / 4), tr = tid / (kDnOW / 4);
  float2 cc[4], ns[4], c1[4], s1[4], ns1[4], acc[4];
  int xq[4], y0c = 0, y1c = 0, fy = 0, fx = 0, pl = 0;
  for (int i = 0;; ++i) {
    const int buf = i & 1;
    const int ntx = cdiv(v.w + kDnX0, kDnOW), nty = cdiv(v.h, kDnOH);
    const int tx = lt % ntx, rt = lt / ntx, ty = rt % nty;
    pl = rt / nty;
    const int X0 = tx * kDnOW - kDnX0, Y0 = ty * kDnOH;
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const bool more_chunks = ch + 1 < nch;
    const bool has_next = more_chunks || t + G < total;
    if (tid == 0 && has_next) {
      fence_proxy_async();
      if (more_chunks) {
        issue(v, lt, ch + 1, buf ^ 1);
      } else {
        int ln;
        const CombineView vn = res(t + G, ln);
        issue(vn, ln, 0, buf ^ 1);
      }
    }
    const int h = v.h, w = v.w;
    if (ch == 0) {
      // Per-tile state: guide value g, trig state (cos, -sin) for k = 1, accumulators.
      fy = Y0 + 2 * tr;
      fx = X0 + 4 * tc;
      y0c = min(fy, h - 1);
      y1c = min(fy + 1, h - 1);
      const long long gpitch = LEVEL0 ? (long long)w : (long long)v.fine->pitch;
      const float* gsrc = LEVEL0 ? v.I + (long long)pl * h * w : v.fine->G + (long long)pl * v.fine->gplane;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        xq[q] = min(max(fx + q, 0), w - 1);
        const float g0 = COH ? __ldcg(gsrc + y0c * gpitch + xq[q]) : __ldg(gsrc + y0c * gpitch + xq[q]);
        const float g1 = COH ? __ldcg(gsrc + y1c * gpitch + xq[q]) : __ldg(gsrc + y1c * gpitch + xq[q]);
        const float2 z0 = cos_sin_turns(v.turns * g0), z1 = cos_sin_turns(v.turns * g1);
        c1[q] = make_float2(z0.x, z1.x);
        s1[q] = make_float2(z0.y, z1.y);
        ns1[q] = make_float2(-z0.y, -z1.y);
        cc[q] = c1[q];
        ns[q] = ns1[q];
        acc[q] = LEVEL0 ? make_float2(g0, g1) : splat(0.f);
      }
    }
    if (!mbar_wait_cta(&bar[buf], pp.use[buf] & 1, v.fault)) {
      if (tid == 0 && has_next) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
      return false;
    }
    ++pp.use[buf];
    CT* zb = reinterpret_cast<CT*>(bufs[buf]);
    float* eb = reinterpret_cast<float*>(bufs[buf] + SM::dn_z);
    const Level& coarse = *v.coarse;
    auto my = [&](int y) { return ext_coarse(y, coarse.h, h); };
    auto mx = [&](int x) { return ext_coarse(x, coarse.w, w); };
    fix_borders(zb, kKC, kDnCH, kDnCW, cx0, cy0, coarse.w, coarse.h, my, mx);
    if (ch == 0 && v.has_e) {
      fix_borders(eb, 1, kDnCH, kDnCW, cx0, cy0, coarse.w, coarse.h, my, mx);
      float e3[3][4];
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        // 8-byte aligned (2*tc floats): two float2 reads
        const float2* q2 = reinterpret_cast<const float2*>(eb + (tr + r) * kDnCW + 2 * tc);
        const float2 qa = q2[0], qb = q2[1];
        e3[r][0] = qa.x; e3[r][1] = qa.y; e3[r][2] = qb.x; e3[r][3] = qb.y;
      }
      float2 p[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) p[q] = make_float2(fmaf(6.f, e3[1][q], e3[0][q] + e3[2][q]), e3[1][q] + e3[2][q]);
      acc[0] = fma2(expand_scale_pair(0), fma2(splat(6.f), p[1], add2(p[0], p[2])), acc[0]);
      acc[1] = fma2(expand_scale_pair(1), add2(p[1], p[2]), acc[1]);
      acc[2] = fma2(expand_scale_pair(2), fma2(splat(6.f), p[2], add2(p[1], p[3])), acc[2]);
      acc[3] = fma2(expand_scale_pair(3), add2(p[2], p[3]), acc[3]);
    }
#pragma unroll
    for (int kk = 0; kk < kKC; ++kk) {
      const int k = ch * kKC + kk;
      if (k < v.K) {
        const float ak = __ldg(v.a + k);
        const CT* zw = zb + kk * kDnCH * kDnCW + tr * kDnCW + 2 * tc;
        float2 wv[3][4];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          if constexpr (sizeof(CT) == 8) {
            // 16-byte aligned: (tr*36 + 2*tc) complex of 8 bytes
            const float4 qa = *reinterpret_cast<const float4*>(zw + r * kDnCW);
            const float4 qb = *reinterpret_cast<const float4*>(zw + r * kDnCW + 2);
            wv[r][0] = make_float2(qa.x, qa.y); wv[r][1] = make_float2(qa.z, qa.w);
            wv[r][2] = make_float2(qb.x, qb.y); wv[r][3] = make_float2(qb.z, qb.w);
          } else {
            // 8-byte aligned: two pairs of 4-byte complex samples
            const uint2 qa = *reinterpret_cast<const uint2*>(zw + r * kDnCW);
            const uint2 qb = *reinterpret_cast<const uint2*>(zw + r * kDnCW + 2);
            wv[r][0] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&qa.x));
            wv[r][1] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&qa.y));
            wv[r][2] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&qb.x));
            wv[r][3] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&qb.y));
          }
        }
        float2 ve[4], vo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          ve[q] = fma2(splat(6.f), wv[1][q], add2(wv[0][q], wv[2][q]));
          vo[q] = add2(wv[1][q], wv[2][q]);
        }
        float2 ue[4], uo[4];
        ue[0] = fma2(splat(6.f), ve[1], add2(ve[0], ve[2]));
        ue[1] = add2(ve[1], ve[2]);
        ue[2] = fma2(splat(6.f), ve[2], add2(ve[1], ve[3]));
        ue[3] = add2(ve[2], ve[3]);
        uo[0] = fma2(splat(6.f), vo[1], add2(vo[0], vo[2]));
        uo[1] = add2(vo[1], vo[2]);
        uo[2] = fma2(splat(6.f), vo[2], add2(vo[1], vo[3]));
        uo[3] = add2(vo[2], vo[3]);
        const float2 ce0 = mul2(splat(-ak), expand_scale_pair(0));
        const float2 ce1 = mul2(splat(-ak), expand_scale_pair(1));
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // cos(k w g) up(S~) - sin(k w g) up(C~) for the two fine rows
          const float2 tq = make_float2(fmaf(cc[q].x, ue[q].y, ns[q].x * ue[q].x),
                                        fmaf(cc[q].y, uo[q].y, ns[q].y * uo[q].x));
          acc[q] = fma2((q & 1) ? ce1 : ce0, tq, acc[q]);
        }
        if constexpr (!LEVEL0) {
          const CT* Zk = reinterpret_cast<const CT*>(v.fine->Z) + (long long)pl * v.fine->zplane +
                         (long long)k * v.fine->zk;
          const CT* r0 = Zk + (long long)y0c * v.fine->pitch;
          const CT* r1 = Zk + (long long)y1c * v.fine->pitch;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            CT zz0, zz1;
            if constexpr (COH) {
              if constexpr (sizeof(CT) == 8) {
                const float2 f0 = __ldcg(reinterpret_cast<const float2*>(r0 + xq[q]));
                const float2 f1 = __ldcg(reinterpret_cast<const float2*>(r1 + xq[q]));
                zz0 = *reinterpret_cast<const CT*>(&f0);
                zz1 = *reinterpret_cast<const CT*>(&f1);
              } else {
                const unsigned u0 = __ldcg(reinterpret_cast<const unsigned*>(r0 + xq[q]));
                const unsigned u1 = __ldcg(reinterpret_cast<const unsigned*>(r1 + xq[q]));
                zz0 = *reinterpret_cast<const CT*>(&u0);
                zz1 = *reinterpret_cast<const CT*>(&u1);
              }
            } else {
              zz0 = r0[xq[q]];
              zz1 = r1[xq[q]];
            }
            const float2 z0 = Cplx<S>::cvt(zz0), z1 = Cplx<S>::cvt(zz1);
            const float2 tq = make_float2(fmaf(cc[q].x, z0.y, ns[q].x * z0.x),
                                          fmaf(cc[q].y, z1.y, ns[q].y * z1.x));
            acc[q] = fma2(splat(ak), tq, acc[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 cn = fma2(cc[q], c1[q], mul2(ns[q], s1[q]));
          const float2 nn = fma2(ns[q], c1[q], mul2(cc[q], ns1[q]));
          cc[q] = cn;
          ns[q] = nn;
        }
      }
    }
    if (!more_chunks) {
      float* dst;
      long long dpitch;
      if constexpr (LEVEL0) {
        dst = v.O + (long long)pl * h * w;
        dpitch = w;
      } else {
        dst = v.fine->E + (long long)pl * v.fine->gplane;
        dpitch = v.fine->pitch;
      }
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int y = fy + rr;
        if (y < h) {
          float* d = dst + (long long)y * dpitch;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int x = fx + q;
            if (x >= 0 && x < w) d[x] = rr ? acc[q].y : acc[q].x;
          }
        }
      }
    }
    __syncthreads();
    if (more_chunks) {
      ++ch;
    } else {
      t += G;
      if (t >= total) break;
      v = res(t, lt);
      ch = 0;
      nch = cdiv(v.K, kKC);
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Per-image kernels (arguments in the parameter block).
template <typename S>
__global__ void __launch_bounds__(kThreads) k_up0(const __grid_constant__ Up0Args a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::up0 - 64);
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  stage_up0<S>([&](int g, int& l) { l = g; return &a; }, up0_tiles(a), smem, bar, pp, blockIdx.x,
               gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_up(const __grid_constant__ UpArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::up - 64);
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  stage_up<S>([&](int g, int& l) { l = g; return &a; }, up_items<S>(a), smem, bar, pp, blockIdx.x,
              gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_down(const __grid_constant__ DownArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dn - 64);
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  const CombineView v = view_of(a);
  stage_combine<S, false, false>([&](int g, int& l) { l = g; return v; }, combine_tiles(v), smem, bar,
                                 pp, blockIdx.x, gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads, 3) k_down0(const __grid_constant__ Down0Args a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dn - 64);
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  const CombineView v = view_of(a);
  stage_combine<S, true, false>([&](int g, int& l) { l = g; return v; }, combine_tiles(v), smem, bar,
                                pp, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------
// Batched kernels: one launch per stage kind covers every image of a batch.
// Their tensor maps live in device memory; the thread that issues the copies
// orders them for the tensor-map proxy before first use.
__device__ __forceinline__ void fence_tensormap(const void* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
template <typename A, typename F>
__device__ __forceinline__ void fence_maps(const BatchTable<A>& tb, F maps) {
  if (threadIdx.x == 0)
    for (int j = 0; j < tb.n; ++j) maps(tb.args[j]);
}
template <typename S>
__global__ void __launch_bounds__(kThreads) k_up0_batch(const BatchTable<Up0Args> tb) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::up0 - 64);
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  stage_up0<S>([&](int g, int& l) {
                 const int j = find_entry(tb.prefix, tb.n, g);
                 l = g - __ldg(tb.prefix + j);
                 return tb.args + j;
               },
               tb.total, smem, bar, pp, blockIdx.x, gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_up_batch(const BatchTable<UpArgs> tb) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::up - 64);
  fence_maps(tb, [](const UpArgs& a) {
    fence_tensormap(&a.zmap);
    fence_tensormap(&a.gmap);
  });
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  stage_up<S>([&](int g, int& l) {
                const int j = find_entry(tb.prefix, tb.n, g);
                l = g - __ldg(tb.prefix + j);
                return tb.args + j;
              },
              tb.total, smem, bar, pp, blockIdx.x, gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_down_batch(const BatchTable<DownArgs> tb) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dn - 64);
  fence_maps(tb, [](const DownArgs& a) {
    fence_tensormap(&a.zmap);
    fence_tensormap(&a.emap);
  });
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  stage_combine<S, false, false>(
      [&](int g, int& l) {
        const int j = find_entry(tb.prefix, tb.n, g);
        l = g - __ldg(tb.prefix + j);
        return view_of(tb.args[j]);
      },
      tb.total, smem, bar, pp, blockIdx.x, gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads, 3) k_down0_batch(const BatchTable<Down0Args> tb) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dn - 64);
  fence_maps(tb, [](const Down0Args& a) {
    fence_tensormap(&a.zmap);
    fence_tensormap(&a.emap);
  });
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  stage_combine<S, true, false>(
      [&](int g, int& l) {
        const int j = find_entry(tb.prefix, tb.n, g);
        l = g - __ldg(tb.prefix + j);
        return view_of(tb.args[j]);
      },
      tb.total, smem, bar, pp, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier of a cooperative launch (all CTAs resident), bounded:
// arrival counter + generation word; every thread first orders its global
// stores before later TMA (async proxy) reads of other CTAs.
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks,
                                             unsigned* fault) {
  asm volatile("fence.proxy.async.global;" ::: "memory");
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned g = ld_acquire(gen);
    if (atomicAdd(count, 1u) + 1u == nblocks) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire(gen) == g) {
        __nanosleep(32);
        if (clock64() - t0 > kWaitCycles) {
          ok = 0;
          atomicOr(fault, 2u);
          break;
        }
      }
    }
    __threadfence();
  }
  return __syncthreads_or(!ok) == 0;
}

// All stages from level c0 down: REDUCE c0 -> ... -> top, then the combines
// top-1 ... c0, in one cooperative launch with grid barriers between stages.
template <typename S>
__global__ void __launch_bounds__(kThreads) k_chain(const __grid_constant__ ChainArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  constexpr size_t kS = SM::up > SM::dn ? SM::up : SM::dn;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kS - 64);
  init_bars(bar);
  Pipe pp{{0u, 0u}};
  const int b = blockIdx.x, G = gridDim.x;
  for (int st = 0; st < a.n_up; ++st) {
    const UpArgs* u = &a.up[st];
    if (!stage_up<S>([&](int g, int& l) { l = g; return u; }, up_items<S>(*u), smem, bar, pp, b, G))
      return;
    if (!grid_barrier(a.sync, a.sync + 1, G, a.fault)) return;
  }
  for (int st = 0; st < a.n_dn; ++st) {
    const CombineView v = view_of(a.dn[st]);
    if (!stage_combine<S, false, true>([&](int g, int& l) { l = g; return v; }, combine_tiles(v),
                                       smem, bar, pp, b, G))
      return;
    if (st + 1 < a.n_dn && !grid_barrier(a.sync, a.sync + 1, G, a.fault)) return;
  }
}

// Persistent grid: at most (resident CTAs per SM) x (SMs) CTAs.
template <typename Kern>
int persistent_grid(Kern kern, size_t smem, int items) {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kThreads, smem);
    cached = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
  }
  return items < cached ? items : cached;
}

}  // namespace

using CTS = typename Cplx<FLLF_STORAGE>::T;
using SMS = Smem<sizeof(CTS)>;

cudaError_t FLLF_LAUNCH_NAME(up0)(const Up0Args& a, cudaStream_t s) {
  const int tiles = cdiv(a.dst.w, kUpTW) * cdiv(a.dst.h, kUpTH) * a.planes;
  const int grid = persistent_grid(k_up0<FLLF_STORAGE>, SMS::up0, tiles);
  k_up0<FLLF_STORAGE><<<grid, kThreads, SMS::up0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(up)(const UpArgs& a, cudaStream_t s) {
  const int items = cdiv(a.dst.w, kRsTW) * cdiv(a.dst.h, kRsTH) * a.planes * cdiv(a.K, SMS::up_kc);
  const int grid = persistent_grid(k_up<FLLF_STORAGE>, SMS::up, items);
  k_up<FLLF_STORAGE><<<grid, kThreads, SMS::up, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(down)(const DownArgs& a, cudaStream_t s) {
  const int tiles = cdiv(a.fine.w + kDnX0, kDnOW) * cdiv(a.fine.h, kDnOH) * a.planes;
  const int grid = persistent_grid(k_down<FLLF_STORAGE>, SMS::dn, tiles);
  k_down<FLLF_STORAGE><<<grid, kThreads, SMS::dn, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(down0)(const Down0Args& a, cudaStream_t s) {
  const int tiles = cdiv(a.w0 + kDnX0, kDnOW) * cdiv(a.h0, kDnOH) * a.planes;
  const int grid = persistent_grid(k_down0<FLLF_STORAGE>, SMS::dn, tiles);
  k_down0<FLLF_STORAGE><<<grid, kThreads, SMS::dn, s>>>(a);
  return cudaGetLastError();
}

cudaError_t FLLF_LAUNCH_NAME(chain)(const ChainArgs& a, cudaStream_t s) {
  constexpr size_t kChainSmem = SMS::up > SMS::dn ? SMS::up : SMS::dn;
  static int grid = 0;
  if (grid == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_chain<FLLF_STORAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kChainSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_chain<FLLF_STORAGE>, kThreads, kChainSmem);
    grid = (per > 0 ? per : 1) * (sms > 0 ? sms : 1);
  }
  void* args[] = {const_cast<ChainArgs*>(&a)};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_chain<FLLF_STORAGE>),
                                              dim3(grid), dim3(kThreads), args, kChainSmem, s);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Batched launches: the grid covers every work item of the table.
cudaError_t FLLF_LAUNCH_NAME(up0_batch)(const BatchTable<Up0Args>& tb, cudaStream_t s) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid(k_up0_batch<FLLF_STORAGE>, SMS::up0, tb.total);
  k_up0_batch<FLLF_STORAGE><<<grid, kThreads, SMS::up0, s>>>(tb);
  return cudaGetLastError();
}
cudaError_t FLLF_LAUNCH_NAME(up_batch)(const BatchTable<UpArgs>& tb, cudaStream_t s) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid(k_up_batch<FLLF_STORAGE>, SMS::up, tb.total);
  k_up_batch<FLLF_STORAGE><<<grid, kThreads, SMS::up, s>>>(tb);
  return cudaGetLastError();
}
cudaError_t FLLF_LAUNCH_NAME(down_batch)(const BatchTable<DownArgs>& tb, cudaStream_t s) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid(k_down_batch<FLLF_STORAGE>, SMS::dn, tb.total);
  k_down_batch<FLLF_STORAGE><<<grid, kThreads, SMS::dn, s>>>(tb);
  return cudaGetLastError();
}
cudaError_t FLLF_LAUNCH_NAME(down0_batch)(const BatchTable<Down0Args>& tb, cudaStream_t s) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid(k_down0_batch<FLLF_STORAGE>, SMS::dn, tb.total);
  k_down0_batch<FLLF_STORAGE><<<grid, kThreads, SMS::dn, s>>>(tb);
  return cudaGetLastError();
}

}  // namespace fllf
