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
#include <algorithm>
#include <type_traits>

#include "fllf_launch.h"

#ifndef FLLF_STORAGE_IS_F32
#define FLLF_STORAGE_IS_F32 0
#endif

namespace fllf {

namespace {

// Waits (bounded) for a TMA copy still in flight before a CTA leaves early.
__device__ __forceinline__ void drain(uint64_t* b, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_test(b, parity) && clock64() - t0 < kWaitCycles) {
  }
}

// Completed uses of the TMA buffers of a CTA (identical in every thread);
// the parity of a buffer's next phase is use[buf] & 1.  Carried across the
// stages of the chained kernel.
struct Pipe {
  uint32_t use[kUpSlots];
};

// bar[0 .. kUpSlots-1]: the buffers' mbarriers (the combine stages use the
// first two); bar[6] holds the CTA's abort flag (an int) for the stages that
// wait per thread.
static_assert(kUpSlots <= 6, "barrier area: 64 bytes");
__device__ __forceinline__ volatile int* abort_flag(uint64_t* bar) {
  return reinterpret_cast<volatile int*>(&bar[6]);
}
// Kernel entry: the CTA's barriers, then the launch dependency.  Every
// kernel of the path is launched with programmatic stream serialization, so
// its CTAs may be resident before the previous kernel of the stream has
// finished: griddepcontrol.wait blocks until that kernel has completed and its
// memory is visible, before any global access of this one (reads of what it
// wrote and writes of what it read alike).  launch_dependents then lets the
// next kernel's CTAs be scheduled (onto SMs this grid leaves free, and as its
// CTAs exit), so their launch and set-up overlap this kernel.  Both are no-ops
// in a kernel launched without the attribute.
__device__ __forceinline__ void init_bars(uint64_t* bar) {
  if (threadIdx.x == 0) {
    for (int j = 0; j < kUpSlots; ++j) mbar_init(&bar[j], 1);
    *abort_flag(bar) = 0;
    fence_mbar_init();
  }
  __syncthreads();
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Brings a tensor map of the kernel's parameters into the TMA unit's
// descriptor cache.  Issued before the launch dependency is waited for (the
// maps are parameters, not data of the previous kernel), so the fetch
// overlaps that kernel's tail instead of delaying the first copy.
__device__ __forceinline__ void prefetch_map(const CUtensorMap* m) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(m)) : "memory");
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

// Work item -> argument block of a batched stage.  The item range of the
// last entry is kept, so that the consecutive items of one image (the common
// case) skip the search.
template <typename A>
struct EntryCache {
  BatchTable<A> tb;
  int j = 0, lo = 0, hi = 0;
  __device__ __forceinline__ const A* operator()(int g, int& l) {
    if (g < lo || g >= hi) {
      j = find_entry(tb.prefix, tb.n, g);
      lo = __ldg(tb.prefix + j);
      hi = __ldg(tb.prefix + j + 1);
    }
    l = g - lo;
    return tb.args + j;
  }
};
// Stages reading their arguments through an EntryCache (a table in global
// memory) copy an item's scalars by value: the copy stays in registers across
// the stage's global stores, which could otherwise alias the table.  Kernels
// with their arguments in the parameter space read them in place.
template <class R>
struct CopiesArgs : std::false_type {};
template <class A>
struct CopiesArgs<EntryCache<A>> : std::true_type {};

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

// FAST: fast LLF (Sec. II-D) instead: complex plane k of a fine pixel is
// (F_{2k}, F_{2k+1}), the sampled detail images, computed per chunk from the
// pixel value (no recurrence), and stored unweighted.
template <typename S, bool FAST = false, typename Res>
__device__ __forceinline__ bool stage_up0(Res res, int total, unsigned char* smem, uint64_t* bar,
                                          Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  auto itb = [&](int buf) { return reinterpret_cast<float*>(smem + buf * SM::up0_it); };
  float2* hz = reinterpret_cast<float2*>(smem + 2 * SM::up0_it);
  float* hg = reinterpret_cast<float*>(smem + 2 * SM::up0_it + align128(SM::up0_hz));
  // per warp and chunk the (4 columns, kUpTH rows, kKC orders) box of Z_1 it
  // writes, stored by TMA; two chunks in flight (buffers by chunk parity)
  CT* stg = reinterpret_cast<CT*>(smem + 2 * SM::up0_it + align128(SM::up0_hz) + align128(SM::up0_hg));
  constexpr int kStBox = kUpRun * kUpTH * kKC;
  const int tid = threadIdx.x;
  int nst = 0;  // chunks stored by this CTA
  auto issue = [&](const Up0Args& a, int t, int buf) {
    const TileXY g = tile_of(t, cdiv(a.dst.w, kUpTW), cdiv(a.dst.h, kUpTH));
    mbar_expect_tx(&bar[buf], sizeof(float) * kUpIR * kUpIW);
    tma_load3(itb(buf), &a.imap, 2 * g.tx * kUpTW - 4, 2 * g.ty * kUpTH - 2, g.pl, &bar[buf]);
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
    const Up0Args* ap = res(gt, t);  // the tensor maps are read here
    std::conditional_t<CopiesArgs<Res>::value, const Up0Args, const Up0Args&> a = *ap;
    const TileXY gxy = tile_of(t, cdiv(a.dst.w, kUpTW), cdiv(a.dst.h, kUpTH));
    const int pl = gxy.pl;
    const int X1 = gxy.tx * kUpTW, Y1 = gxy.ty * kUpTH;
    const int xs = 2 * X1 - 4, ys = 2 * Y1 - 2;
    const int nch = cdiv(a.K, kKC);
    float* it = itb(buf);
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
        if ((tid & 31) == 0) bulk_wait_all();
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
    // Lane 31 repeats row 30 (kUpIR = 31 rows) into the unused staging row
    // 31, which keeps the pass free of divergence.
    const int r = tid & 31, s = tid >> 5, rl = min(r, kUpIR - 1);
    float2* hzw = hz + s * (kKC * kUpRun * kUpCS);  // [order][column][fine row]
    float* hgw = hg + s * (kUpRun * kUpCS);          // [column][fine row]
    // Orders by the recurrence z_{k+1} = 2 cos(w_1 x) z_k - z_{k-1} held in two
    // registers per pixel that take turns: at an even step of a chunk zb holds
    // the current order and za the one before, and za <- t zb - za moves to
    // the next; at an odd step the roles swap.  A chunk has an even number of
    // steps, so each chunk starts with the same roles (no register copies).
    float2 zb[kUpIPX], za[kUpIPX], tc[kUpIPX];
    float v[kUpIPX];
    // fast LLF: per pixel, the Gaussian factor of the current sample and its
    // ratio to the next (kept within 85 registers: 3 CTAs per SM)
    float fe[FAST ? kUpIPX : 1], fr[FAST ? kUpIPX : 1];
    {
      {
        const float4* row = reinterpret_cast<const float4*>(it + rl * kUpIW + 2 * kUpRun * s);
        const float4 q0 = row[0], q1 = row[1], q2 = row[2], q3 = row[3];
        v[0] = q0.z; v[1] = q0.w;
        v[2] = q1.x; v[3] = q1.y; v[4] = q1.z; v[5] = q1.w;
        v[6] = q2.x; v[7] = q2.y; v[8] = q2.z; v[9] = q2.w;
        v[10] = q3.x;
      }
      if constexpr (!FAST) {
#pragma unroll
        for (int j = 0; j < kUpIPX; ++j) {
          const float2 z = cos_sin_turns(a.turns * v[j]);
          zb[j] = z;
          za[j] = make_float2(1.f, 0.f);
          tc[j] = splat(2.f * z.x);
        }
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
    for (int ch = 0; ch < nch; ++ch) {
      {
#pragma unroll
        for (int kk = 0; kk < kKC; ++kk) {
          if constexpr (FAST) {
            const int s0 = 2 * (ch * kKC + kk);
            const bool s1 = s0 + 1 < a.fast.S;
            if (a.fast.rec) {
              // Gaussian factors by the multiplicative recurrence from the
              // chunk's first sample (exact start, two exp2 per pixel and
              // chunk): E_{j+1} = E_j r_j, r_{j+1} = r_j k2
              if (kk == 0) {
#pragma unroll
                for (int j = 0; j < kUpIPX; ++j) {
                  const float d0 = fmaf(-a.fast.tau, (float)s0, v[j]);
                  fe[j] = exp2f(-a.fast.c2 * d0 * d0);
                  fr[j] = exp2f(a.fast.c2 * a.fast.tau * fmaf(2.f, d0, -a.fast.tau));
                }
              }
#pragma unroll
              for (int j = 0; j < kUpIPX; ++j) {
                const float d0 = fmaf(-a.fast.tau, (float)s0, v[j]), d1 = d0 - a.fast.tau;
                const float f0 = a.fast.fm1 * d0 * fe[j];
                fe[j] *= fr[j];
                fr[j] *= a.fast.k2;
                const float f1 = s1 ? a.fast.fm1 * d1 * fe[j] : 0.f;
                fe[j] *= fr[j];
                fr[j] *= a.fast.k2;
                zb[j] = make_float2(f0, f1);
              }
            } else {
#pragma unroll
              for (int j = 0; j < kUpIPX; ++j)
                zb[j] = make_float2(fast_detail(a.fast, v[j], s0), s1 ? fast_detail(a.fast, v[j], s0 + 1) : 0.f);
            }
          }
          // the current order: zb at an even step, za at an odd one (fast LLF: zb)
          const float2* zk = (FAST || (kk & 1) == 0) ? zb : za;
#pragma unroll
          for (int q = 0; q < kUpRun; ++q)
            hzw[(kk * kUpRun + q) * kUpCS + r] =
                tap5(zk[2 * q], zk[2 * q + 1], zk[2 * q + 2], zk[2 * q + 3], zk[2 * q + 4]);
          if constexpr (!FAST) {
#pragma unroll
            for (int j = 0; j < kUpIPX; ++j) {
              if ((kk & 1) == 0) za[j] = fma2(tc[j], zb[j], make_float2(-za[j].x, -za[j].y));
              else zb[j] = fma2(tc[j], za[j], make_float2(-zb[j].x, -zb[j].y));
            }
          }
        }
      }
      __syncwarp();
      {
        const int k = ch * kKC + vkk;
        // Column q of order k, rows Y1 + 7 vgrp .. + 6: order k is stored
        // weighted by its coefficient, a_k Z_{1,k}, into the warp's staging
        // box [order][row][column]; the TMA store leaves out what falls
        // outside level 1 or beyond order K.
        // fast LLF keeps one staging buffer (shared memory for 3 CTAs per SM)
        constexpr int kStBufs = FAST ? 1 : 2;
        CT* sb = stg + ((nst % kStBufs) * (kThreads / 32) + s) * kStBox;
        // the box written from this buffer kStBufs chunks ago has been read
        if ((tid & 31) == 0) bulk_wait_read<kStBufs - 1>();
        __syncwarp();
        {
          const float sk = FAST ? (1.f / 256.f) : (k < a.K ? __ldg(a.a + k) : 0.f) * (1.f / 256.f);
          const float4* p =
              reinterpret_cast<const float4*>(hzw + (vkk * kUpRun + vq) * kUpCS + 2 * kUpVRows * vgrp);
          float2 w[2 * kUpVRows + 4];
#pragma unroll
          for (int u = 0; u < kUpVRows + 2; ++u) {
            const float4 q4 = p[u];
            w[2 * u] = make_float2(q4.x, q4.y);
            w[2 * u + 1] = make_float2(q4.z, q4.w);
          }
          CT* o = sb + (vkk * kUpTH + vgrp * kUpVRows) * kUpRun + vq;
#pragma unroll
          for (int j = 0; j < kUpVRows; ++j)
            Cplx<S>::st(o + j * kUpRun,
                        mul2(splat(sk), tap5(w[2 * j], w[2 * j + 1], w[2 * j + 2], w[2 * j + 3], w[2 * j + 4])));
        }
        fence_proxy_async();
        __syncwarp();
        if ((tid & 31) == 0) {
          tma_store4(&ap->zstmap, sb, X1 + kUpRun * s, Y1, ch * kKC, pl);
          bulk_commit();
        }
        ++nst;
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
  // the stores have completed (and read their staging) before the stage ends
  if ((tid & 31) == 0) bulk_wait_all();
  return true;
}

// ---------------------------------------------------------------------------------------
// up: level l -> l+1 for l >= 1 (REDUCE of G_l and the K complex planes).
// Item = (tile of 30 x 16 coarse outputs, chunk): chunks 0 .. nch-1 hold KCU
// orders each, and chunk nch (when G_{l+1} is needed) the guide plane; items
// reduce independently, so small levels still spread over many CTAs.  TMA
// stages the 35 x 68 source box of an item into a ring of kUpSlots buffers,
// kUpSlots - 1 items ahead of the one being reduced; the vertical pass reads
// one staged column per thread and keeps the reduced rows in registers, the
// horizontal pass reads 5 staged columns per output.
template <typename S>
__device__ __forceinline__ int up_chunks(const UpArgs& a) {
  return cdiv(a.K, Smem<sizeof(typename Cplx<S>::T)>::up_kc) + (a.write_g ? 1 : 0);
}
template <typename S>
__device__ __forceinline__ int up_items(const UpArgs& a) {
  return cdiv(a.dst.w, kRsTW) * cdiv(a.dst.h, kRsTH) * a.planes * up_chunks<S>(a);
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
  float2* vb = reinterpret_cast<float2*>(smem + kUpSlots * SM::up_slot);
  float* vg = reinterpret_cast<float*>(smem + kUpSlots * SM::up_slot + SM::up_vb);
  volatile int* abortp = abort_flag(bar);
  const int tid = threadIdx.x;
  const int nitems = b < total ? (total - b + G - 1) / G : 0;
  auto issue = [&](int gi, int slot) {
    int li;
    const UpArgs& a = *res(gi, li);
    int ch;
    const int nch = cdiv(a.K, KCU), t = div_fast(li, up_chunks<S>(a), ch);
    const TileXY g = tile_of(t, cdiv(a.dst.w, kRsTW), cdiv(a.dst.h, kRsTH));
    const int pl = g.pl;
    const int x = 2 * g.tx * kRsTW - 4, y = 2 * g.ty * kRsTH - 2;
    unsigned char* dst = smem + slot * SM::up_slot;
    if (ch < nch) {
      mbar_expect_tx(&bar[slot], (uint32_t)(sizeof(CT) * KCU * kRsIR * kRsBW));
      tma_load3(dst, &a.zmap, x, y, pl * a.K + ch * KCU, &bar[slot]);
    } else {
      mbar_expect_tx(&bar[slot], (uint32_t)(sizeof(float) * kRsIR * kRsBW));
      tma_load3(dst, &a.gmap, x, y, pl, &bar[slot]);
    }
  };
  if (tid == 0) {
    fence_proxy_async();
    for (int j = 0; j < kUpSlots - 1 && j < nitems; ++j) issue(b + j * G, j);
  }
  for (int i = 0; i < nitems; ++i) {
    const int slot = i % kUpSlots;
    int li;
    std::conditional_t<CopiesArgs<Res>::value, const UpArgs, const UpArgs&> a = *res(b + i * G, li);
    int ch;
    const int nch = cdiv(a.K, KCU), t = div_fast(li, up_chunks<S>(a), ch);
    const TileXY gxy = tile_of(t, cdiv(a.dst.w, kRsTW), cdiv(a.dst.h, kRsTH));
    const int pl = gxy.pl;
    const int X1 = gxy.tx * kRsTW, Y1 = gxy.ty * kRsTH;
    const int xs = 2 * X1 - 4, ys = 2 * Y1 - 2;
    if (tid == 0 && i + kUpSlots - 1 < nitems) {
      fence_proxy_async();
      issue(b + (i + kUpSlots - 1) * G, (i + kUpSlots - 1) % kUpSlots);
    }
    mbar_wait_thread(&bar[slot], pp.use[slot] & 1, a.fault, abortp);
    ++pp.use[slot];
    unsigned char* buf = smem + slot * SM::up_slot;
    auto my = [&](int y) { return refl101(y, a.src.h); };
    auto mx = [&](int x) { return refl101(x, a.src.w); };
    if (ch < nch) {
      CT* src = reinterpret_cast<CT*>(buf);
      fix_borders(src, KCU, kRsIR, kRsBW, xs, ys, a.src.w, a.src.h, my, mx);
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
      }
      __syncthreads();
      if (tid < KCU * kRsTW * HQ) {  // horizontal half
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
    } else {
      float* gsrc = reinterpret_cast<float*>(buf);
      fix_borders(gsrc, 1, kRsIR, kRsBW, xs, ys, a.src.w, a.src.h, my, mx);
      {  // vertical half: 4 groups x 4 coarse rows x 64 columns
        const int grp = tid / kRsVW, cg = tid % kRsVW;
        const float* gc = gsrc + (8 * grp) * kRsBW + cg + 2;
        float u[11];
#pragma unroll
        for (int q = 0; q < 11; ++q) u[q] = gc[q * kRsBW];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          vg[(4 * grp + j) * kRsVW + cg] = tap5(u[2 * j], u[2 * j + 1], u[2 * j + 2], u[2 * j + 3], u[2 * j + 4]);
      }
      __syncthreads();
      if (tid < kRsTW * 8) {  // horizontal half: 8 groups x 2 coarse rows x 30 columns
        const int hq = tid / kRsTW, ic = tid % kRsTW, x = X1 + ic;
        if (x < a.dst.w) {
          float* Gp = a.dst.G + (long long)pl * a.dst.gplane + x;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int jr = 2 * hq + j, y = Y1 + jr;
            if (y < a.dst.h) {
              const float* p = vg + jr * kRsVW + 2 * ic;
              Gp[(long long)y * a.dst.pitch] = (1.f / 256.f) * tap5(p[0], p[1], p[2], p[3], p[4]);
            }
          }
        }
      }
    }
    __syncthreads();
    if (*abortp) {
      // leave with no copy in flight
      if (tid == 0)
        for (int j = i + 1; j < nitems && j < i + kUpSlots; ++j)
          drain(&bar[j % kUpSlots], pp.use[j % kUpSlots] & 1);
      return false;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Combine (Eq. (14) product-sum fused with the residual collapse).
// Item = (tile of 64 x 32 fine pixels, chunk of kKC orders); the chunks of a
// tile run back to back on one CTA, from the highest order down, which keeps
// the per-pixel state in registers.  The stored Fourier planes carry their
// coefficient (a_k Z_{l,k}), so with w = e^{-i w_1 g} the sum of Eq. (14) is
// evaluated by Horner's rule over the orders: P <- P w + D_k, sum = Im(P w),
// where D_k = a_k (Z_{l,k} - up Z_{l+1,k}) at level l >= 1 and
// D_k = -a_k up Z_{1,k} at level 0 (the Z_0 term cancels).  A thread owns
// fine rows 2j, 2j+1 and fine columns 4c..4c+3 of the tile (tile origin
// 64*tx-6), i.e. coarse rows j-1..j+1 and coarse columns 2c-1..2c+2, which sit
// at staged rows tr..tr+2 and columns 2tc..2tc+3.  EXPAND weights 1/8 (1, 6, 1)
// at even fine positions and 1/2 (1, 1) at odd ones per axis are applied
// after the sum at level 0 (they are the same for every order) and per order
// at level >= 1.
__device__ __forceinline__ float2 expand_scale_pair(int q) {
  return (q & 1) ? make_float2(1.f / 16.f, 1.f / 4.f) : make_float2(1.f / 64.f, 1.f / 16.f);
}

// Unscaled EXPAND of the staged 3 x 4 complex window at zw (row pitch kDnCW)
// to the 2 x 4 fine pixels of a combine thread: ue (even fine row), uo (odd).
template <typename S>
__device__ __forceinline__ void expand_2x4(const typename Cplx<S>::T* zw, float2 ue[4], float2 uo[4]) {
  using CT = typename Cplx<S>::T;
  float2 wv[3][4];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    if constexpr (sizeof(CT) == 8) {
      // 16-byte aligned: (row*36 + 2*tc) complex of 8 bytes
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
  ue[0] = fma2(splat(6.f), ve[1], add2(ve[0], ve[2]));
  ue[1] = add2(ve[1], ve[2]);
  ue[2] = fma2(splat(6.f), ve[2], add2(ve[1], ve[3]));
  ue[3] = add2(ve[2], ve[3]);
  uo[0] = fma2(splat(6.f), vo[1], add2(vo[0], vo[2]));
  uo[1] = add2(vo[1], vo[2]);
  uo[2] = fma2(splat(6.f), vo[2], add2(vo[1], vo[3]));
  uo[3] = add2(vo[2], vo[3]);
}

// Residual EXPAND up(E) at the 2 x 4 fine pixels of a combine thread from the
// staged 3 x 4 float window at eb (row pitch kDnCW), scaled: (even, odd) rows.
__device__ __forceinline__ void expand_e_2x4(const float* eb, float2 out[4]) {
  float e3[3][4];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    // 8-byte aligned (2*tc floats): two float2 reads
    const float2* q2 = reinterpret_cast<const float2*>(eb + r * kDnCW);
    const float2 qa = q2[0], qb = q2[1];
    e3[r][0] = qa.x; e3[r][1] = qa.y; e3[r][2] = qb.x; e3[r][3] = qb.y;
  }
  float2 p[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) p[q] = make_float2(fmaf(6.f, e3[1][q], e3[0][q] + e3[2][q]), e3[1][q] + e3[2][q]);
  out[0] = mul2(expand_scale_pair(0), fma2(splat(6.f), p[1], add2(p[0], p[2])));
  out[1] = mul2(expand_scale_pair(1), add2(p[1], p[2]));
  out[2] = mul2(expand_scale_pair(2), fma2(splat(6.f), p[2], add2(p[1], p[3])));
  out[3] = mul2(expand_scale_pair(3), add2(p[2], p[3]));
}

// e^{-i pi t} as (cos, -sin).
__device__ __forceinline__ float2 conj_turns(float t) {
  const float2 z = cos_sin_turns(t);
  return make_float2(z.x, -z.y);
}

// View of the level-0 combine arguments.
struct CombineView {
  const CUtensorMap* zmap;
  const CUtensorMap* emap;
  const float* I;
  float* O;
  const Level* coarse;
  unsigned* fault;
  const float* M0;
  const FastArgs* fast;
  int h, w, planes, K, has_e;
  float turns, mscale;
};
__device__ __forceinline__ CombineView view_of(const Down0Args& d) {
  return CombineView{&d.zmap, &d.emap, d.I, d.O, &d.coarse, d.fault, d.M0, &d.fast,
                     d.h0, d.w0, d.planes, d.K, d.has_e, d.turns, d.mscale};
}
__device__ __forceinline__ int combine_tiles(int h, int w, int planes) {
  return cdiv(w + kDnX0, kDnOW) * cdiv(h, kDnOH) * planes;
}
__device__ __forceinline__ int combine_tiles(const CombineView& v) { return combine_tiles(v.h, v.w, v.planes); }

// Level-0 combine alone (levels == 2, where E_1 = 0 and no level-1 combine
// exists, the batched path, and fast LLF).
// FAST: fast LLF (Sec. II-D) at level 0: the level-0 sampled details are
// evaluated at the pixel, (1 - a) F_j + a F_{j+1} for the samples bracketing
// g = I_p, and the EXPAND of every plane is weighted by the same hat weights.
template <typename S, bool FAST = false, typename Res>
__device__ __forceinline__ bool stage_combine0(Res res, int total, unsigned char* smem, uint64_t* bar,
                                               Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  auto bufp = [&](int buf) { return smem + buf * SM::dn_buf; };
  const int tid = threadIdx.x;
  if (b >= total) return true;
  auto issue = [&](const CombineView& v, int lt, int ch, bool first, int buf) {
    const TileXY g = tile_of(lt, cdiv(v.w + kDnX0, kDnOW), cdiv(v.h, kDnOH));
    const int cx0 = (g.tx * kDnOW - kDnX0) / 2 - 1, cy0 = g.ty * (kDnOH / 2) - 1;
    const bool e = first && v.has_e;
    mbar_expect_tx(&bar[buf], (uint32_t)(sizeof(CT) * kKC * kDnCH * kDnCW +
                                         (e ? sizeof(float) * kDnCH * kDnCW : 0)));
    tma_load4(bufp(buf), v.zmap, cx0, cy0, ch * kKC, g.pl, &bar[buf]);
    if (e) tma_load3(bufp(buf) + SM::dn_z, v.emap, cx0, cy0, g.pl, &bar[buf]);
  };
  int t = b, lt = 0;
  CombineView v = res(t, lt);
  int nch = cdiv(v.K, kKC), ch = nch - 1;
  if (tid == 0) {
    fence_proxy_async();
    issue(v, lt, ch, true, 0);
  }

  const int tc = tid % (kDnOW / 4), tr = tid / (kDnOW / 4);
  float2 we[4], wo[4], Pe[4], Po[4], base[4];
  int fy = 0, fx = 0, pl = 0, X0 = 0, Y0 = 0;
  for (int i = 0;; ++i) {
    const int buf = i & 1;
    const bool first = ch == nch - 1, last = ch == 0;
    const int h = v.h, w = v.w;
    if (first) {
      const TileXY g = tile_of(lt, cdiv(w + kDnX0, kDnOW), cdiv(h, kDnOH));
      pl = g.pl;
      X0 = g.tx * kDnOW - kDnX0;
      Y0 = g.ty * kDnOH;
    }
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const bool has_next = !last || t + G < total;
    if (tid == 0 && has_next) {
      fence_proxy_async();
      if (!last) {
        issue(v, lt, ch - 1, false, buf ^ 1);
      } else {
        int ln;
        const CombineView vn = res(t + G, ln);
        issue(vn, ln, cdiv(vn.K, kKC) - 1, true, buf ^ 1);
      }
    }
    if (first) {
      // Per-tile state: e^{-i w_1 I}, Horner sums, base value I.
      fy = Y0 + 2 * tr;
      fx = X0 + 4 * tc;
      const int y0c = min(fy, h - 1), y1c = min(fy + 1, h - 1);
      const float* gsrc = v.I + (long long)pl * h * w;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int xq = min(max(fx + q, 0), w - 1);
        const float g0 = __ldg(gsrc + (long long)y0c * w + xq), g1 = __ldg(gsrc + (long long)y1c * w + xq);
        Pe[q] = Po[q] = splat(0.f);
        if constexpr (FAST) {
          const FastArgs& fa = *v.fast;
          auto level0 = [&](float g, float t) {   // (1 - a) F_j(p) + a F_{j+1}(p) at g = I_p
            const int j = min((int)t, fa.S - 2);
            const float al = t - (float)j;
            return fmaf(al, fast_detail(fa, g, j + 1), (1.f - al) * fast_detail(fa, g, j));
          };
          const float t0 = fast_pos(fa, g0), t1 = fast_pos(fa, g1);
          we[q] = make_float2(t0, 0.f);
          wo[q] = make_float2(t1, 0.f);
          base[q] = make_float2(g0 + level0(g0, t0), g1 + level0(g1, t1));
        } else {
          we[q] = conj_turns(v.turns * g0);
          wo[q] = conj_turns(v.turns * g1);
          base[q] = make_float2(g0, g1);
        }
      }
    }
    if (!mbar_wait_cta(&bar[buf], pp.use[buf] & 1, v.fault)) {
      if (tid == 0 && has_next) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
      return false;
    }
    ++pp.use[buf];
    CT* zb = reinterpret_cast<CT*>(bufp(buf));
    float* eb = reinterpret_cast<float*>(bufp(buf) + SM::dn_z);
    const Level& coarse = *v.coarse;
    auto my = [&](int y) { return ext_coarse(y, coarse.h, h); };
    auto mx = [&](int x) { return ext_coarse(x, coarse.w, w); };
    fix_borders(zb, kKC, kDnCH, kDnCW, cx0, cy0, coarse.w, coarse.h, my, mx);
    if (first && v.has_e) {
      fix_borders(eb, 1, kDnCH, kDnCW, cx0, cy0, coarse.w, coarse.h, my, mx);
      float2 ue[4];
      expand_e_2x4(eb + tr * kDnCW + 2 * tc, ue);
#pragma unroll
      for (int q = 0; q < 4; ++q) base[q] = add2(base[q], ue[q]);
    }
    // Orders k >= K of the highest chunk are staged as zeros (4-D map) and
    // come first in the descending Horner run, where they leave P at zero.
    const CT* zw = zb + tr * kDnCW + 2 * tc;
#pragma unroll
    for (int kk = kKC - 1; kk >= 0; --kk) {
      float2 ue[4], uo[4];
      expand_2x4<S>(zw + kk * kDnCH * kDnCW, ue, uo);
      if constexpr (FAST) {
        const int s0 = 2 * (ch * kKC + kk);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Pe[q].x = fmaf(fast_hat(we[q].x, s0 + 1), ue[q].y, fmaf(fast_hat(we[q].x, s0), ue[q].x, Pe[q].x));
          Po[q].x = fmaf(fast_hat(wo[q].x, s0 + 1), uo[q].y, fmaf(fast_hat(wo[q].x, s0), uo[q].x, Po[q].x));
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Pe[q] = horner(Pe[q], we[q], ue[q]);
          Po[q] = horner(Po[q], wo[q], uo[q]);
        }
      }
    }
    if (last) {
      float* dst = v.O + (long long)pl * h * w;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int y = fy + rr;
        if (y < h) {
          float* d = dst + (long long)y * w;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int x = fx + q;
            // the EXPAND weight and the sign of D_k are applied here
            const float2 sc = expand_scale_pair(q);
            float delta;
            if constexpr (FAST) delta = rr ? -sc.y * Po[q].x : -sc.x * Pe[q].x;
            else delta = rr ? -sc.y * im_mul(Po[q], wo[q]) : -sc.x * im_mul(Pe[q], we[q]);
            if (x >= 0 && x < w) {
              if (v.M0) delta *= (__ldg(v.M0 + (long long)y * w + x) - 1.f) * v.mscale;
              d[x] = (rr ? base[q].y : base[q].x) + delta;
            }
          }
        }
      }
    }
    __syncthreads();
    if (!last) {
      --ch;
    } else {
      t += G;
      if (t >= total) break;
      v = res(t, lt);
      nch = cdiv(v.K, kKC);
      ch = nch - 1;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Combine at a level l >= 1 (Eq. (14) middle case, with the residual collapse):
// E_l = sum_k Im(e^{-i k w_1 g} a_k (Z_{l,k} - up Z_{l+1,k})) + up E_{l+1}.
// Item = (tile of 64 x 32 level-l pixels, chunk of kKC1 orders), chunks from
// the highest order down.  Every operand is staged by TMA: the fine Z_l box
// (68 x 32 from (X0 - 2, Y0)) and the coarse Z_{l+1} window of each chunk,
// and with the first chunk the fine G_l box and the coarse E_{l+1} window, so
// the loads of the next chunk overlap the current one.  Thread mapping, EXPAND
// and Horner as in the level-0 combine; the EXPAND weight is applied per order
// before the difference with Z_l.
template <typename S, typename Res>
__device__ __forceinline__ bool stage_combine1(Res res, int total, unsigned char* smem, uint64_t* bar,
                                               Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  constexpr size_t kOffC = SM::dn1_zf, kOffE = kOffC + SM::dn1_zc, kOffG = kOffE + SM::dn1_e;
  auto bufp = [&](int buf) { return smem + buf * SM::dn1_buf; };
  volatile int* abortp = abort_flag(bar);
  const int tid = threadIdx.x;
  if (b >= total) return true;
  auto issue = [&](const DownArgs& a, int lt, int ch, bool first, int buf) {
    const TileXY g = tile_of(lt, cdiv(a.fine.w + kDnX0, kDnOW), cdiv(a.fine.h, kDnOH));
    const int X0 = g.tx * kDnOW - kDnX0, Y0 = g.ty * kDnOH;
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const bool e = first && a.has_e;
    uint32_t bytes = (uint32_t)(sizeof(CT) * kKC1 * (kDnOH * kD0IW + kDnCH * kDnCW));
    if (first) bytes += (uint32_t)(sizeof(float) * kDnOH * kD0IW);
    if (e) bytes += (uint32_t)(sizeof(float) * kDnCH * kDnCW);
    mbar_expect_tx(&bar[buf], bytes);
    unsigned char* p = bufp(buf);
    // x = X0 - 2 = 64 tx - 8: 16-byte aligned for every element size
    tma_load4(p, &a.zfmap, X0 - 2, Y0, ch * kKC1, g.pl, &bar[buf]);
    tma_load4(p + kOffC, &a.zmap, cx0, cy0, ch * kKC1, g.pl, &bar[buf]);
    if (first) tma_load3(p + kOffG, &a.gfmap, X0 - 2, Y0, g.pl, &bar[buf]);
    if (e) tma_load3(p + kOffE, &a.emap, cx0, cy0, g.pl, &bar[buf]);
  };
  int t = b, lt = 0;
  const DownArgs* a = res(t, lt);
  int nch = cdiv(a->K, kKC1), ch = nch - 1;
  if (tid == 0) {
    fence_proxy_async();
    issue(*a, lt, ch, true, 0);
  }

  const int tc = tid % (kDnOW / 4), tr = tid / (kDnOW / 4);
  float2 we[4], wo[4], Pe[4], Po[4], base[4];
  int fy = 0, fx = 0, pl = 0, X0 = 0, Y0 = 0;
  for (int i = 0;; ++i) {
    const int buf = i & 1;
    const bool first = ch == nch - 1, last = ch == 0;
    const int h = a->fine.h, w = a->fine.w;
    if (first) {
      const TileXY g = tile_of(lt, cdiv(w + kDnX0, kDnOW), cdiv(h, kDnOH));
      pl = g.pl;
      X0 = g.tx * kDnOW - kDnX0;
      Y0 = g.ty * kDnOH;
      fy = Y0 + 2 * tr;
      fx = X0 + 4 * tc;
    }
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const bool has_next = !last || t + G < total;
    if (tid == 0 && has_next) {
      fence_proxy_async();
      if (!last) {
        issue(*a, lt, ch - 1, false, buf ^ 1);
      } else {
        int ln;
        const DownArgs* an = res(t + G, ln);
        issue(*an, ln, cdiv(an->K, kKC1) - 1, true, buf ^ 1);
      }
    }
    mbar_wait_thread(&bar[buf], pp.use[buf] & 1, a->fault, abortp);
    ++pp.use[buf];
    const CT* zf = reinterpret_cast<const CT*>(bufp(buf));
    CT* zc = reinterpret_cast<CT*>(bufp(buf) + kOffC);
    float* eb = reinterpret_cast<float*>(bufp(buf) + kOffE);
    const Level& coarse = a->coarse;
    auto my = [&](int y) { return ext_coarse(y, coarse.h, h); };
    auto mx = [&](int x) { return ext_coarse(x, coarse.w, w); };
    fix_borders(zc, kKC1, kDnCH, kDnCW, cx0, cy0, coarse.w, coarse.h, my, mx);
    if (first) {
      // staged fine pixel (fy + rr, fx + q) at row 2 tr + rr, column 4 tc + 2 + q
      // (zero outside the level; those pixels are not stored)
      const float* gb = reinterpret_cast<const float*>(bufp(buf) + kOffG) + 2 * tr * kD0IW + 4 * tc + 2;
      const float2 a0 = *reinterpret_cast<const float2*>(gb), a1 = *reinterpret_cast<const float2*>(gb + 2);
      const float2 c0 = *reinterpret_cast<const float2*>(gb + kD0IW);
      const float2 c1 = *reinterpret_cast<const float2*>(gb + kD0IW + 2);
      const float ge[4] = {a0.x, a0.y, a1.x, a1.y}, go[4] = {c0.x, c0.y, c1.x, c1.y};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        we[q] = conj_turns(a->turns * ge[q]);
        wo[q] = conj_turns(a->turns * go[q]);
        Pe[q] = Po[q] = splat(0.f);
        base[q] = splat(0.f);
      }
      if (a->has_e) {
        fix_borders(eb, 1, kDnCH, kDnCW, cx0, cy0, coarse.w, coarse.h, my, mx);
        expand_e_2x4(eb + tr * kDnCW + 2 * tc, base);
      }
    }
    // Orders k >= K of the highest chunk are staged as zeros (4-D maps) and
    // come first in the descending Horner run, where they leave P at zero.
    const CT* zw = zc + tr * kDnCW + 2 * tc;
    const CT* zfw = zf + 2 * tr * kD0IW + 4 * tc + 2;
#pragma unroll
    for (int kk = kKC1 - 1; kk >= 0; --kk) {
      float2 ue[4], uo[4];
      expand_2x4<S>(zw + kk * kDnCH * kDnCW, ue, uo);
      float2 fe[4], fo[4];
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const CT* r = zfw + kk * kDnOH * kD0IW + rr * kD0IW;
        float2* f = rr ? fo : fe;
        if constexpr (sizeof(CT) == 8) {
          // (row * 68 + 4 tc + 2) complex of 8 bytes: 16-byte aligned
          const float4 q0 = *reinterpret_cast<const float4*>(r);
          const float4 q1 = *reinterpret_cast<const float4*>(r + 2);
          f[0] = make_float2(q0.x, q0.y); f[1] = make_float2(q0.z, q0.w);
          f[2] = make_float2(q1.x, q1.y); f[3] = make_float2(q1.z, q1.w);
        } else {
          // 8-byte aligned: two pairs of 4-byte complex samples
          const uint2 q0 = *reinterpret_cast<const uint2*>(r);
          const uint2 q1 = *reinterpret_cast<const uint2*>(r + 2);
          f[0] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&q0.x));
          f[1] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&q0.y));
          f[2] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&q1.x));
          f[3] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&q1.y));
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 sc = expand_scale_pair(q);
        Pe[q] = horner(Pe[q], we[q], fma2(splat(-sc.x), ue[q], fe[q]));
        Po[q] = horner(Po[q], wo[q], fma2(splat(-sc.y), uo[q], fo[q]));
      }
    }
    if (last) {
      float* dst = a->fine.E + (long long)pl * a->fine.gplane;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int y = fy + rr;
        if (y < h) {
          float* d = dst + (long long)y * a->fine.pitch;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int x = fx + q;
            float delta = rr ? im_mul(Po[q], wo[q]) : im_mul(Pe[q], we[q]);
            if (x >= 0 && x < w) {
              if (a->fine.M)
                delta *= (__ldg(a->fine.M + (long long)y * a->fine.pitch + x) - 1.f) * a->mscale;
              d[x] = (rr ? base[q].y : base[q].x) + delta;
            }
          }
        }
      }
    }
    __syncthreads();
    if (*abortp) {
      if (tid == 0 && has_next) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
      return false;
    }
    if (!last) {
      --ch;
    } else {
      t += G;
      if (t >= total) break;
      a = res(t, lt);
      nch = cdiv(a->K, kKC1);
      ch = nch - 1;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Combine at a small level l >= 1 (Eq. (14), l >= 1 case), on 32 x 16 tiles.
// Item = tile; its orders are staged kKCS at a time (highest chunk first, in a
// ring of two slots) and every thread runs the whole descending Horner sum
// for its two fine pixels (column X0 + tc, rows Y0 + 2 tr and + 1).  Each
// arithmetic step is the one the 64 x 32 combine takes for the same pixel, in
// the same order (EXPAND: vertical sums per coarse column, then the
// horizontal 1-6-1 or 1-1 sum; D = f - s u; Horner; Im(P w); base + delta),
// so both give the same bits and a level may run on either.  The horizontal
// sum is written once for both column parities: u = a v1 + (b v0 + v2) with
// (a, b) = (6, 1) for an even column and (1, 0) for an odd one, whose
// v1 + (0 v0 + v2) rounds exactly as v1 + v2.
//
// FAST: fast LLF (Sec. II-D).  The planes hold the sampled detail images, and
// the pixel's difference is interpolated between the two samples bracketing
// g = G_l[I]_p: Delta = sum_s hat_s(g) (F_{l,s} - up F_{l+1,s}), with the hat
// weights 1 - a, a of the bracketing pair and 0 elsewhere.
template <typename S, bool FAST = false, typename Res>
__device__ __forceinline__ bool stage_combine_s(Res res, int total, unsigned char* smem, uint64_t* bar,
                                                Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  constexpr size_t kOffC = SM::sm_zf, kOffE = kOffC + SM::sm_zc, kOffG = kOffE + SM::sm_e;
  auto bufp = [&](int buf) { return smem + buf * SM::sm_buf; };
  volatile int* abortp = abort_flag(bar);
  const int tid = threadIdx.x;
  if (b >= total) return true;
  auto issue = [&](const DownArgs& a, int lt, int ch, bool first, int buf) {
    const TileXY g = tile_of(lt, cdiv(a.fine.w + kDnX0, kSmW), cdiv(a.fine.h, kSmH));
    const int X0 = g.tx * kSmW - kDnX0, Y0 = g.ty * kSmH;
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const bool e = first && a.has_e;
    uint32_t bytes = (uint32_t)(sizeof(CT) * kKCS * (kSmH * kSmIW + kSmCH * kSmCW));
    if (first) bytes += (uint32_t)(sizeof(float) * kSmH * kSmIW);
    if (e) bytes += (uint32_t)(sizeof(float) * kSmCH * kSmCW);
    mbar_expect_tx(&bar[buf], bytes);
    unsigned char* p = bufp(buf);
    // x = X0 - 2 = 32 tx - 8 and cx0 = 16 tx - 4: 16-byte aligned for every element size
    tma_load4(p, &a.zfmap, X0 - 2, Y0, ch * kKCS, g.pl, &bar[buf]);
    tma_load4(p + kOffC, &a.zmap, cx0, cy0, ch * kKCS, g.pl, &bar[buf]);
    if (first) tma_load3(p + kOffG, &a.gfmap, X0 - 2, Y0, g.pl, &bar[buf]);
    if (e) tma_load3(p + kOffE, &a.emap, cx0, cy0, g.pl, &bar[buf]);
  };
  int t = b, lt = 0;
  // the tile's arguments (a by-value copy of the scalars for a batched
  // table); the tensor maps are read at ap
  constexpr bool kCopy = CopiesArgs<Res>::value;
  const DownArgs* ap = res(t, lt);
  DownArgs av;
  if constexpr (kCopy) av = *ap;
  const DownArgs* a = kCopy ? &av : ap;
  int nch = cdiv(a->K, kKCS), ch = nch - 1;
  if (tid == 0) {
    fence_proxy_async();
    issue(*ap, lt, ch, true, 0);
  }

  // X0 is even, so the column's parity is that of tc; its EXPAND reads the
  // staged coarse columns c0 .. c0 + 2 (an odd column uses the last two) and
  // rows tr .. tr + 2 (the odd row uses the last two).
  const int tc = tid % kSmW, tr = tid / kSmW, odd = tc & 1, c0 = tc >> 1;
  const float2 ha = splat(odd ? 1.f : 6.f), hb = splat(odd ? 0.f : 1.f);
  const float2 sc = expand_scale_pair(odd);
  float2 we = splat(0.f), wo = splat(0.f), Pe = splat(0.f), Po = splat(0.f), base = splat(0.f);
  int fy = 0, fx = 0, pl = 0, X0 = 0, Y0 = 0;
  for (int i = 0;; ++i) {
    const int buf = i & 1;
    const bool first = ch == nch - 1, last = ch == 0;
    const int h = a->fine.h, w = a->fine.w;
    if (first) {
      const TileXY g = tile_of(lt, cdiv(w + kDnX0, kSmW), cdiv(h, kSmH));
      pl = g.pl;
      X0 = g.tx * kSmW - kDnX0;
      Y0 = g.ty * kSmH;
      fy = Y0 + 2 * tr;
      fx = X0 + tc;
    }
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const bool has_next = !last || t + G < total;
    if (tid == 0 && has_next) {
      fence_proxy_async();
      if (!last) {
        issue(*ap, lt, ch - 1, false, buf ^ 1);
      } else {
        int ln;
        const DownArgs* an = res(t + G, ln);
        issue(*an, ln, cdiv(an->K, kKCS) - 1, true, buf ^ 1);
      }
    }
    mbar_wait_thread(&bar[buf], pp.use[buf] & 1, a->fault, abortp);
    ++pp.use[buf];
    const CT* zf = reinterpret_cast<const CT*>(bufp(buf));
    CT* zc = reinterpret_cast<CT*>(bufp(buf) + kOffC);
    float* eb = reinterpret_cast<float*>(bufp(buf) + kOffE);
    const Level& coarse = a->coarse;
    auto my = [&](int y) { return ext_coarse(y, coarse.h, h); };
    auto mx = [&](int x) { return ext_coarse(x, coarse.w, w); };
    fix_borders(zc, kKCS, kSmCH, kSmCW, cx0, cy0, coarse.w, coarse.h, my, mx);
    if (first) {
      // staged fine pixel (fy + rr, fx) at row 2 tr + rr, column tc + 2 (zero
      // outside the level; those pixels are not stored)
      const float* gb = reinterpret_cast<const float*>(bufp(buf) + kOffG) + 2 * tr * kSmIW + tc + 2;
      if constexpr (FAST) {
        // sample positions t = g (S - 1) of the two pixels
        we = make_float2(fast_pos(a->fast, gb[0]), 0.f);
        wo = make_float2(fast_pos(a->fast, gb[kSmIW]), 0.f);
      } else {
        we = conj_turns(a->turns * gb[0]);
        wo = conj_turns(a->turns * gb[kSmIW]);
      }
      Pe = Po = splat(0.f);
      base = splat(0.f);
      if (a->has_e) {
        fix_borders(eb, 1, kSmCH, kSmCW, cx0, cy0, coarse.w, coarse.h, my, mx);
        const float* ew = eb + tr * kSmCW + c0;
        float2 p[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float e0 = ew[c], e1 = ew[kSmCW + c], e2 = ew[2 * kSmCW + c];
          p[c] = make_float2(fmaf(6.f, e1, e0 + e2), e1 + e2);
        }
        base = mul2(sc, fma2(ha, p[1], fma2(hb, p[0], p[2])));
      }
    }
    // Orders k >= K of the highest chunk are staged as zeros (4-D maps) and
    // come first in the descending Horner run, where they leave P at zero.
    const CT* zw = zc + tr * kSmCW + c0;
    const CT* zfw = zf + 2 * tr * kSmIW + tc + 2;
#pragma unroll
    for (int kk = kKCS - 1; kk >= 0; --kk) {
      const CT* zr = zw + kk * kSmCH * kSmCW;
      float2 ve[3], vo[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2 q0 = Cplx<S>::cvt(zr[c]);
        const float2 q1 = Cplx<S>::cvt(zr[kSmCW + c]);
        const float2 q2 = Cplx<S>::cvt(zr[2 * kSmCW + c]);
        ve[c] = fma2(splat(6.f), q1, add2(q0, q2));
        vo[c] = add2(q1, q2);
      }
      const float2 ue = fma2(ha, ve[1], fma2(hb, ve[0], ve[2]));
      const float2 uo = fma2(ha, vo[1], fma2(hb, vo[0], vo[2]));
      const CT* fr = zfw + kk * kSmH * kSmIW;
      const float2 fe = Cplx<S>::cvt(fr[0]), fo = Cplx<S>::cvt(fr[kSmIW]);
      if constexpr (FAST) {
        const int s0 = 2 * (ch * kKCS + kk);
        const float2 de = fma2(splat(-sc.x), ue, fe), dd = fma2(splat(-sc.y), uo, fo);
        Pe.x = fmaf(fast_hat(we.x, s0 + 1), de.y, fmaf(fast_hat(we.x, s0), de.x, Pe.x));
        Po.x = fmaf(fast_hat(wo.x, s0 + 1), dd.y, fmaf(fast_hat(wo.x, s0), dd.x, Po.x));
      } else {
        Pe = horner(Pe, we, fma2(splat(-sc.x), ue, fe));
        Po = horner(Po, wo, fma2(splat(-sc.y), uo, fo));
      }
    }
    if (last && fx >= 0 && fx < w) {
      float* dst = a->fine.E + (long long)pl * a->fine.gplane + fx;
#pragma unroll
      for (int rr = 0; rr < 2; ++rr) {
        const int y = fy + rr;
        if (y < h) {
          float delta;
          if constexpr (FAST) delta = rr ? Po.x : Pe.x;
          else delta = rr ? im_mul(Po, wo) : im_mul(Pe, we);
          if (a->fine.M) delta *= (__ldg(a->fine.M + (long long)y * a->fine.pitch + fx) - 1.f) * a->mscale;
          dst[(long long)y * a->fine.pitch] = (rr ? base.y : base.x) + delta;
        }
      }
    }
    __syncthreads();
    if (*abortp) {
      if (tid == 0 && has_next) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
      return false;
    }
    if (!last) {
      --ch;
    } else {
      t += G;
      if (t >= total) break;
      ap = res(t, lt);
      if constexpr (kCopy) av = *ap;
      else a = ap;
      nch = cdiv(a->K, kKCS);
      ch = nch - 1;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Fused combine at levels 1 and 0 (Eq. (14), both cases; levels >= 3).
// Item = (tile of 64 x 32 level-0 pixels, chunk of kKC orders) as in the
// level-0 combine.  The level-0 EXPAND reads the 36 x 18 staged window of
// level-1 cells from (cx0, cy0) = (X0/2 - 1, Y0/2 - 1), and E_1 is needed on
// exactly that window, so the tile first runs the level-1 combine there: it
// reads the same staged Z_1 cells as the fine values of level 1, G_1 on the
// window (with the first chunk), and the 20 x 11 window of level-2 cells
// from (cx0/2 - 2, (cy0 - 1)/2) holding Z_2 and E_2.  Thread b < 153 owns the
// 2 x 2 level-1 cells (2 br + rr, 2 bc + cc).  cy0 is odd and cx0 even, so
// rr = 0 is an odd level-1 row (level-2 window rows br, br+1, weights
// 1/2 (1, 1)) and rr = 1 an even one (rows br..br+2, 1/8 (1, 6, 1)); cc = 0
// is an even column (window columns bc+1..bc+3) and cc = 1 an odd one
// (bc+2, bc+3).  After the last chunk the level-1 threads write
// E_1 = Delta_1 + up(E_2) to shared memory, the out-of-range cells take their
// EXPAND sources, and every thread finishes O = I + Delta_0 + up(E_1) for its
// 2 x 4 level-0 pixels.  E_1 never goes to memory, and each Z_1 sample is
// read once for both levels.
//
// FAST: fast LLF (Sec. II-D): the planes hold the sampled detail images, the
// Horner sums become the hat-weighted sums over the samples bracketing the
// guide (as in the small-tile and level-0 combines), and level 0 adds the
// level-0 sampled details evaluated at the pixel.
template <typename S, bool ADAPT, bool FAST = false, typename Res>
__device__ __forceinline__ bool stage_down10(Res res, int total, unsigned char* smem, uint64_t* bar,
                                            Pipe& pp, int b, int G) {
  using CT = typename Cplx<S>::T;
  using SM = Smem<sizeof(CT)>;
  constexpr size_t kOffG1 = SM::d10_z1 + SM::d10_z2, kOffE2 = kOffG1 + SM::d10_g1;
  constexpr size_t kOffI = kOffE2 + SM::d10_e2;
  auto bufp = [&](int buf) { return smem + buf * SM::d10_buf; };
  float* e1 = reinterpret_cast<float*>(smem + 2 * SM::d10_buf);
  volatile int* abortp = abort_flag(bar);
  const int tid = threadIdx.x;
  if (b >= total) return true;
  auto issue = [&](const Down10Args& a, int lt, int ch, bool first, int buf) {
    const TileXY g = tile_of(lt, cdiv(a.w0 + kDnX0, kDnOW), cdiv(a.h0, kDnOH));
    const int tx = g.tx, ty = g.ty, pl = g.pl;
    const int cx0 = (tx * kDnOW - kDnX0) / 2 - 1, cy0 = ty * (kDnOH / 2) - 1;
    const int c2x = cx0 / 2 - 2, c2y = (cy0 - 1) / 2;
    const bool e2 = first && a.has_e2, in = first && a.use_tma;
    uint32_t bytes = (uint32_t)(sizeof(CT) * kKC * (kDnCH * kDnCW + kD2H * kD2W));
    if (first) bytes += (uint32_t)(sizeof(float) * kDnCH * kDnCW);
    if (e2) bytes += (uint32_t)(sizeof(float) * kD2H * kD2W);
    if (in) bytes += (uint32_t)(sizeof(float) * kDnOH * kD0IW);
    mbar_expect_tx(&bar[buf], bytes);
    unsigned char* p = bufp(buf);
    tma_load4(p, &a.z1map, cx0, cy0, ch * kKC, pl, &bar[buf]);
    tma_load4(p + SM::d10_z1, &a.z2map, c2x, c2y, ch * kKC, pl, &bar[buf]);
    if (first) tma_load3(p + kOffG1, &a.g1map, cx0, cy0, pl, &bar[buf]);
    if (e2) tma_load3(p + kOffE2, &a.e2map, c2x, c2y, pl, &bar[buf]);
    // level-0 input from X0 - 2 = 64 tx - 8 (x 4 bytes: 16-byte aligned)
    if (in) tma_load3(p + kOffI, &a.imap, tx * kDnOW - kDnX0 - 2, ty * kDnOH, pl, &bar[buf]);
  };
  int t = b, lt = 0;
  // the tile's arguments (a by-value copy of the scalars for a batched
  // table); the tensor maps are read at ap
  constexpr bool kCopy = CopiesArgs<Res>::value;
  const Down10Args* ap = res(t, lt);
  Down10Args av;
  if constexpr (kCopy) av = *ap;
  const Down10Args* a = kCopy ? &av : ap;
  int nch = cdiv(a->K, kKC), ch = nch - 1;
  if (tid == 0) {
    fence_proxy_async();
    issue(*ap, lt, ch, true, 0);
  }

  const int tc = tid % (kDnOW / 4), tr = tid / (kDnOW / 4);
  // level-1 blocks on threads 0..152 (warps 0-4 at full width): the other
  // warps go straight to the level-0 combine, and their issue slots serve the
  // SM's other CTA meanwhile.  Threads 0..143 take block columns 0..15, a
  // half-warp per block row, so that a half-warp's window loads are one
  // contiguous run (no bank conflicts); threads 144..152 take column 16.
  static_assert(kB1X == 17, "level-1 block mapping");
  constexpr int kB1Main = (kB1X - 1) * kB1Y;
  const bool l1t = tid < kB1X * kB1Y;
  const int bc = tid < kB1Main ? (tid & 15) : kB1X - 1;
  const int br = tid < kB1Main ? (tid >> 4) : tid - kB1Main;
  float2 we[4], wo[4], Pe[4], Po[4], base[4];
  float2 w1[2][2], P1[2][2];
  float up_e2[2][2];
  int fy = 0, fx = 0, pl = 0, X0 = 0, Y0 = 0;
  // per tile, CTA-uniform: the windows lie inside levels 1 and 2 (no border
  // fix-ups, level-1 cells written unguarded), the 64 x 32 output lies
  // inside the image (stored unguarded)
  bool inner = false, full = false;
  for (int i = 0;; ++i) {
    const int buf = i & 1;
    const int h0 = a->h0, w0 = a->w0;
    const bool first = ch == nch - 1, last = ch == 0;
    if (first) {
      const TileXY g = tile_of(lt, cdiv(w0 + kDnX0, kDnOW), cdiv(h0, kDnOH));
      pl = g.pl;
      X0 = g.tx * kDnOW - kDnX0;
      Y0 = g.ty * kDnOH;
      const int wx = X0 / 2 - 1, wy = Y0 / 2 - 1, vx = wx / 2 - 2, vy = (wy - 1) / 2;
      inner = wx >= 0 && wy >= 0 && wx + kDnCW <= a->l1.w && wy + kDnCH <= a->l1.h && vx >= 0 && vy >= 0 &&
              vx + kD2W <= a->l2.w && vy + kD2H <= a->l2.h;
      full = X0 >= 0 && X0 + kDnOW <= w0 && Y0 + kDnOH <= h0;
    }
    const int cx0 = X0 / 2 - 1, cy0 = Y0 / 2 - 1;
    const int c2x = cx0 / 2 - 2, c2y = (cy0 - 1) / 2;
    const bool has_next = !last || t + G < total;
    if (tid == 0 && has_next) {
      fence_proxy_async();
      if (!last) {
        issue(*ap, lt, ch - 1, false, buf ^ 1);
      } else {
        int ln;
        const Down10Args* an = res(t + G, ln);
        issue(*an, ln, cdiv(an->K, kKC) - 1, true, buf ^ 1);
      }
    }
    // level-0 state: e^{-i w_1 I}, Horner sums, and I itself
    auto init0 = [&](int q, float g0, float g1) {
      Pe[q] = Po[q] = splat(0.f);
      if constexpr (FAST) {
        const FastArgs& fa = a->fast;
        auto level0 = [&](float g, float t) {   // (1 - a) F_j(p) + a F_{j+1}(p) at g = I_p
          const int j = min((int)t, fa.S - 2);
          const float al = t - (float)j;
          return fmaf(al, fast_detail(fa, g, j + 1), (1.f - al) * fast_detail(fa, g, j));
        };
        const float t0 = fast_pos(fa, g0), t1 = fast_pos(fa, g1);
        we[q] = make_float2(t0, 0.f);
        wo[q] = make_float2(t1, 0.f);
        base[q] = make_float2(g0 + level0(g0, t0), g1 + level0(g1, t1));
      } else {
        we[q] = conj_turns(a->turns * g0);
        wo[q] = conj_turns(a->turns * g1);
        base[q] = make_float2(g0, g1);
      }
    };
    if (first) {
      fy = Y0 + 2 * tr;
      fx = X0 + 4 * tc;
      if (!a->use_tma) {
        const int y0c = min(fy, h0 - 1), y1c = min(fy + 1, h0 - 1);
        const float* Ip = a->I + (long long)pl * h0 * w0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int xq = min(max(fx + q, 0), w0 - 1);
          init0(q, __ldg(Ip + (long long)y0c * w0 + xq), __ldg(Ip + (long long)y1c * w0 + xq));
        }
      }
    }
    mbar_wait_thread(&bar[buf], pp.use[buf] & 1, a->fault, abortp);
    ++pp.use[buf];
    CT* z1b = reinterpret_cast<CT*>(bufp(buf));
    CT* z2b = reinterpret_cast<CT*>(bufp(buf) + SM::d10_z1);
    const float* g1b = reinterpret_cast<const float*>(bufp(buf) + kOffG1);
    float* e2b = reinterpret_cast<float*>(bufp(buf) + kOffE2);
    if (first && a->use_tma) {
      // staged input: fine pixel (fy + rr, fx + q) at row 2 tr + rr, column 4 tc + 2 + q
      // (zero outside the image; those pixels are not stored)
      const float* ib = reinterpret_cast<const float*>(bufp(buf) + kOffI) + 2 * tr * kD0IW + 4 * tc + 2;
      const float2 a0 = *reinterpret_cast<const float2*>(ib), a1 = *reinterpret_cast<const float2*>(ib + 2);
      const float2 c0 = *reinterpret_cast<const float2*>(ib + kD0IW);
      const float2 c1 = *reinterpret_cast<const float2*>(ib + kD0IW + 2);
      init0(0, a0.x, c0.x);
      init0(1, a0.y, c0.y);
      init0(2, a1.x, c1.x);
      init0(3, a1.y, c1.y);
    }
    const Level& L1 = a->l1;
    const Level& L2 = a->l2;
    auto my1 = [&](int y) { return ext_coarse(y, L1.h, h0); };
    auto mx1 = [&](int x) { return ext_coarse(x, L1.w, w0); };
    auto my2 = [&](int y) { return ext_coarse(y, L2.h, L1.h); };
    auto mx2 = [&](int x) { return ext_coarse(x, L2.w, L1.w); };
    if (!inner) {
      fix_borders(z1b, kKC, kDnCH, kDnCW, cx0, cy0, L1.w, L1.h, my1, mx1);
      fix_borders(z2b, kKC, kD2H, kD2W, c2x, c2y, L2.w, L2.h, my2, mx2);
      if (first && a->has_e2) fix_borders(e2b, 1, kD2H, kD2W, c2x, c2y, L2.w, L2.h, my2, mx2);
    }

    // level-1 combine on the window cells (Horner over this chunk's orders)
    if (l1t) {
      if (first) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            w1[rr][cc] = FAST ? make_float2(fast_pos(a->fast, g1b[(2 * br + rr) * kDnCW + 2 * bc + cc]), 0.f)
                              : conj_turns(a->turns * g1b[(2 * br + rr) * kDnCW + 2 * bc + cc]);
            P1[rr][cc] = splat(0.f);
            up_e2[rr][cc] = 0.f;
          }
        if (a->has_e2) {
          const float* ew = e2b + br * kD2W + bc + 1;
          float vo[3], ve[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float e0 = ew[c], e1v = ew[kD2W + c], e2v = ew[2 * kD2W + c];
            vo[c] = e0 + e1v;
            ve[c] = fmaf(6.f, e1v, e0 + e2v);
          }
          up_e2[0][0] = (1.f / 16.f) * fmaf(6.f, vo[1], vo[0] + vo[2]);
          up_e2[0][1] = (1.f / 4.f) * (vo[1] + vo[2]);
          up_e2[1][0] = (1.f / 64.f) * fmaf(6.f, ve[1], ve[0] + ve[2]);
          up_e2[1][1] = (1.f / 16.f) * (ve[1] + ve[2]);
        }
      }
      // orders k >= K read as zeros (4-D maps) and leave P at zero
      const CT* zw2 = z2b + br * kD2W + bc + 1;
      const CT* zc1 = z1b + 2 * br * kDnCW + 2 * bc;
#pragma unroll
      for (int kk = kKC - 1; kk >= 0; --kk) {
        {
          const CT* zw = zw2 + kk * kD2H * kD2W;
          float2 vo[3], ve[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const float2 q0 = Cplx<S>::cvt(zw[c]);
            const float2 q1 = Cplx<S>::cvt(zw[kD2W + c]);
            const float2 q2 = Cplx<S>::cvt(zw[2 * kD2W + c]);
            vo[c] = add2(q0, q1);
            ve[c] = fma2(splat(6.f), q1, add2(q0, q2));
          }
          // unscaled EXPAND sums; the weights 1/16, 1/4, 1/64, 1/16 are powers
          // of two, so D = f - w U below is the same number whether w U is
          // rounded first or folded into one fused multiply-add
          float2 U[2][2];
          U[0][0] = fma2(splat(6.f), vo[1], add2(vo[0], vo[2]));
          U[0][1] = add2(vo[1], vo[2]);
          U[1][0] = fma2(splat(6.f), ve[1], add2(ve[0], ve[2]));
          U[1][1] = add2(ve[1], ve[2]);
          constexpr float kUw[2][2] = {{-1.f / 16.f, -1.f / 4.f}, {-1.f / 64.f, -1.f / 16.f}};
          const CT* zc = zc1 + kk * kDnCH * kDnCW;
#pragma unroll
          for (int rr = 0; rr < 2; ++rr) {
            float2 f[2];
            if constexpr (sizeof(CT) == 8) {
              const float4 q = *reinterpret_cast<const float4*>(zc + rr * kDnCW);  // 16-byte aligned
              f[0] = make_float2(q.x, q.y);
              f[1] = make_float2(q.z, q.w);
            } else {
              const uint2 q = *reinterpret_cast<const uint2*>(zc + rr * kDnCW);  // 8-byte aligned
              f[0] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&q.x));
              f[1] = Cplx<S>::cvt(*reinterpret_cast<const CT*>(&q.y));
            }
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
              const float2 d = fma2(splat(kUw[rr][cc]), U[rr][cc], f[cc]);
              if constexpr (FAST) {
                const int s0 = 2 * (ch * kKC + kk);
                P1[rr][cc].x = fmaf(fast_hat(w1[rr][cc].x, s0 + 1), d.y, fmaf(fast_hat(w1[rr][cc].x, s0), d.x, P1[rr][cc].x));
              } else {
                P1[rr][cc] = horner(P1[rr][cc], w1[rr][cc], d);
              }
            }
          }
        }
      }
    }

    // level-0 combine (Horner over this chunk's orders)
    const CT* zw0 = z1b + tr * kDnCW + 2 * tc;
#pragma unroll
    for (int kk = kKC - 1; kk >= 0; --kk) {
      float2 ue[4], uo[4];
      expand_2x4<S>(zw0 + kk * kDnCH * kDnCW, ue, uo);
      if constexpr (FAST) {
        const int s0 = 2 * (ch * kKC + kk);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Pe[q].x = fmaf(fast_hat(we[q].x, s0 + 1), ue[q].y, fmaf(fast_hat(we[q].x, s0), ue[q].x, Pe[q].x));
          Po[q].x = fmaf(fast_hat(wo[q].x, s0 + 1), uo[q].y, fmaf(fast_hat(wo[q].x, s0), uo[q].x, Po[q].x));
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          Pe[q] = horner(Pe[q], we[q], ue[q]);
          Po[q] = horner(Po[q], wo[q], uo[q]);
        }
      }
    }

    if (last) {
      // E_1 = Delta_1 + up(E_2) on the window cells inside level 1
      auto write_e1 = [&](auto guarded) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) {
            const int y1 = cy0 + 2 * br + rr, x1 = cx0 + 2 * bc + cc;
            if (!decltype(guarded)::value || (y1 >= 0 && y1 < L1.h && x1 >= 0 && x1 < L1.w)) {
              float d1 = FAST ? P1[rr][cc].x : im_mul(P1[rr][cc], w1[rr][cc]);
              if constexpr (ADAPT) d1 *= (__ldg(L1.M + (long long)y1 * L1.pitch + x1) - 1.f) * a->mscale;
              e1[(2 * br + rr) * kDnCW + 2 * bc + cc] = d1 + up_e2[rr][cc];
            }
          }
      };
      if (l1t) {
        if (inner) write_e1(std::false_type{});
        else write_e1(std::true_type{});
      }
      __syncthreads();
      if (!inner) fix_borders(e1, 1, kDnCH, kDnCW, cx0, cy0, L1.w, L1.h, my1, mx1);
      float2 ue[4];
      expand_e_2x4(e1 + tr * kDnCW + 2 * tc, ue);
      float* dst = a->O + (long long)pl * h0 * w0;
      // O = I + Delta_0 + up(E_1) at the thread's 2 x 4 pixels inside the image
      auto write_o = [&](auto guarded) {
#pragma unroll
        for (int rr = 0; rr < 2; ++rr) {
          const int y = fy + rr;
          if (!decltype(guarded)::value || y < h0) {
            float* d = dst + (long long)y * w0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const int x = fx + q;
              const float2 sc = expand_scale_pair(q);
              float delta;
              if constexpr (FAST) delta = rr ? -sc.y * Po[q].x : -sc.x * Pe[q].x;
              else delta = rr ? -sc.y * im_mul(Po[q], wo[q]) : -sc.x * im_mul(Pe[q], we[q]);
              if (!decltype(guarded)::value || (x >= 0 && x < w0)) {
                if constexpr (ADAPT) delta *= (__ldg(a->M0 + (long long)y * w0 + x) - 1.f) * a->mscale;
                d[x] = (rr ? base[q].y + ue[q].y : base[q].x + ue[q].x) + delta;
              }
            }
          }
        }
      };
      if (full) write_o(std::false_type{});
      else write_o(std::true_type{});
    }
    __syncthreads();
    if (*abortp) {
      if (tid == 0 && has_next) drain(&bar[buf ^ 1], pp.use[buf ^ 1] & 1);
      return false;
    }
    if (!last) {
      --ch;
    } else {
      t += G;
      if (t >= total) break;
      ap = res(t, lt);
      if constexpr (kCopy) av = *ap;
      else a = ap;
      nch = cdiv(a->K, kKC);
      ch = nch - 1;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Per-image kernels (arguments in the parameter block).
template <typename S, bool FAST>
__global__ void __launch_bounds__(kThreads) k_up0(const __grid_constant__ Up0Args a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (FAST ? SM::up0_fast : SM::up0) - 64);
  if (threadIdx.x == 0 && a.use_tma) prefetch_map(&a.imap);
  init_bars(bar);
  Pipe pp{};
  const int hi = a.item1 > 0 ? a.item1 : up0_tiles(a);
  stage_up0<S, FAST>([&](int g, int& l) { l = g; return &a; }, hi, smem, bar, pp, a.item0 + blockIdx.x,
               gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads) k_up(const __grid_constant__ UpArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::up - 64);
  if (threadIdx.x == 0) {
    prefetch_map(&a.zmap);
    if (a.write_g) prefetch_map(&a.gmap);
  }
  init_bars(bar);
  Pipe pp{};
  const int n = up_items<S>(a);
  const int hi = a.item1 > 0 ? a.item1 : n;
  // reversed order: the items of the level the previous kernel wrote last are
  // read first, while they are still in L2
  stage_up<S>([&](int g, int& l) { l = a.reverse ? n - 1 - g : g; return &a; }, hi, smem, bar, pp,
              a.item0 + blockIdx.x, gridDim.x);
}

template <typename S>
__global__ void __launch_bounds__(kThreads, 2) k_down(const __grid_constant__ DownArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dn1 - 64);
  init_bars(bar);
  Pipe pp{};
  stage_combine1<S>([&](int g, int& l) { l = g; return &a; }, combine_tiles(a.fine.h, a.fine.w, a.planes),
                    smem, bar, pp, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ int small_tiles(int h, int w, int planes) {
  return cdiv(w + kDnX0, kSmW) * cdiv(h, kSmH) * planes;
}

template <typename S, bool FAST>
__global__ void __launch_bounds__(kThreads) k_down_s(const __grid_constant__ DownArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dns - 64);
  if (threadIdx.x == 0) {
    prefetch_map(&a.zfmap);
    prefetch_map(&a.zmap);
    prefetch_map(&a.gfmap);
    if (a.has_e) prefetch_map(&a.emap);
  }
  init_bars(bar);
  Pipe pp{};
  stage_combine_s<S, FAST>([&](int g, int& l) { l = g; return &a; }, small_tiles(a.fine.h, a.fine.w, a.planes),
                     smem, bar, pp, blockIdx.x, gridDim.x);
}

template <typename S, bool FAST>
__global__ void __launch_bounds__(kThreads, 3) k_down0(const __grid_constant__ Down0Args a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dn - 64);
  init_bars(bar);
  Pipe pp{};
  const CombineView v = view_of(a);
  stage_combine0<S, FAST>([&](int g, int& l) { l = g; return v; }, combine_tiles(v), smem, bar, pp, blockIdx.x,
                    gridDim.x);
}

// ADAPT: pixel-adaptive gain map (Down10Args::M0 and l1.M set); FAST: fast LLF.
template <typename S, bool ADAPT, bool FAST>
__global__ void __launch_bounds__(kThreads, 2) k_down10(const __grid_constant__ Down10Args a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::d10 - 64);
  if (threadIdx.x == 0) {
    prefetch_map(&a.z1map);
    prefetch_map(&a.z2map);
    prefetch_map(&a.g1map);
    if (a.has_e2) prefetch_map(&a.e2map);
    if (a.use_tma) prefetch_map(&a.imap);
  }
  init_bars(bar);
  Pipe pp{};
  stage_down10<S, ADAPT, FAST>([&](int g, int& l) { l = g; return &a; }, combine_tiles(a.h0, a.w0, a.planes), smem, bar,
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
  fence_maps(tb, [](const Up0Args& a) {
    if (a.use_tma) fence_tensormap(&a.imap);
    fence_tensormap(&a.zstmap);
  });
  init_bars(bar);
  Pipe pp{};
  stage_up0<S>(EntryCache<Up0Args>{tb},
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
  Pipe pp{};
  stage_up<S>(EntryCache<UpArgs>{tb},
              tb.total, smem, bar, pp, blockIdx.x, gridDim.x);
}

// Combines at levels >= 1 of a batch: the 32 x 16 tiles (the same bits as
// the 64 x 32 combine, and the better fill for the small levels of mixed
// batches).
template <typename S>
__global__ void __launch_bounds__(kThreads) k_down_batch(const BatchTable<DownArgs> tb) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::dns - 64);
  fence_maps(tb, [](const DownArgs& a) {
    fence_tensormap(&a.zmap);
    fence_tensormap(&a.emap);
    fence_tensormap(&a.zfmap);
    fence_tensormap(&a.gfmap);
  });
  init_bars(bar);
  Pipe pp{};
  stage_combine_s<S>(
      EntryCache<DownArgs>{tb},
      tb.total, smem, bar, pp, blockIdx.x, gridDim.x);
}

// Fused level-1/level-0 combine of the batch's images with >= 3 levels (no
// gain map; the input's map is written per run).
template <typename S>
__global__ void __launch_bounds__(kThreads, 2) k_down10_batch(const BatchTable<Down10Args> tb) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + SM::d10 - 64);
  fence_maps(tb, [](const Down10Args& a) {
    fence_tensormap(&a.z1map);
    fence_tensormap(&a.g1map);
    fence_tensormap(&a.z2map);
    if (a.has_e2) fence_tensormap(&a.e2map);
    if (a.use_tma) fence_tensormap(&a.imap);
  });
  init_bars(bar);
  Pipe pp{};
  stage_down10<S, false>(
      EntryCache<Down10Args>{tb},
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
  Pipe pp{};
  stage_combine0<S>(
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
    // arrivals awaited: the grid, plus the status block's extra count (0
    // normally; a test raises it so that the wait runs out)
    const unsigned need = nblocks + *reinterpret_cast<const volatile unsigned*>(fault + kStatusExtraArrivals);
    const unsigned g = ld_acquire(gen);
    if (atomicAdd(count, 1u) + 1u == need) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const long long lim = wait_limit(fault);
      const long long t0 = clock64();
      while (ld_acquire(gen) == g) {
        __nanosleep(32);
        if (clock64() - t0 > lim) {
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
__global__ void __launch_bounds__(kThreads, 2) k_chain(const __grid_constant__ ChainArgs a) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  constexpr size_t kS = SM::up > SM::dn1 ? SM::up : SM::dn1;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kS - 64);
  init_bars(bar);
  Pipe pp{};
  const int b = blockIdx.x, G = gridDim.x;
  for (int st = 0; st < a.n_up; ++st) {
    const UpArgs* u = &a.up[st];
    if (!stage_up<S>([&](int g, int& l) { l = g; return u; }, up_items<S>(*u), smem, bar, pp, b, G))
      return;
    if (!grid_barrier(a.sync, a.sync + 1, G, a.fault)) return;
  }
  for (int st = 0; st < a.n_dn; ++st) {
    const DownArgs* d = &a.dn[st];
    const bool ok = a.dn_small[st]
                        ? stage_combine_s<S>([&](int g, int& l) { l = g; return d; },
                                             small_tiles(d->fine.h, d->fine.w, d->planes), smem, bar, pp, b, G)
                        : stage_combine1<S>([&](int g, int& l) { l = g; return d; },
                                            combine_tiles(d->fine.h, d->fine.w, d->planes), smem, bar, pp, b, G);
    if (!ok) return;
    if (st + 1 < a.n_dn && !grid_barrier(a.sync, a.sync + 1, G, a.fault)) return;
  }
}

// ---------------------------------------------------------------------------------------
// Dataflow launch (one persistent grid for every stage of one or many images).
// A CTA pops the next ready task from the device queue, runs its work items
// through the same stage function as the per-stage kernels (so the output is
// the same, bit for bit), and adds them to its band's count.  The CTA whose
// task completes a band marks the band complete in every band that reads it;
// a reader band whose inputs are now all complete has its tasks pushed.  A
// popped task never waits for another task, so no CTA depends on another
// being resident; a CTA waits (bounded) only for a queue slot to be filled,
// and every slot is filled once, by a CTA that is running a task.
// One task of each stage kind, kept out of line: each is register-allocated
// on its own (the fused combine alone needs about 125 registers), instead of
// all five inside one loop body.
template <typename S>
__device__ __noinline__ bool graph_up0(const GraphArgs& g, const GraphTask& t, unsigned char* smem, uint64_t* bar,
                                       Pipe& pp) {
  const Up0Args* a = t.args < 0 ? &g.up0 : g.up0s + t.args;
  return stage_up0<S>([&](int gi, int& l) { l = gi; return a; }, t.first + t.count, smem, bar, pp, t.first, 1);
}
template <typename S>
__device__ __noinline__ bool graph_up(const GraphArgs& g, const GraphTask& t, unsigned char* smem, uint64_t* bar,
                                      Pipe& pp) {
  const UpArgs* a = g.ups + t.args;
  return stage_up<S>([&](int gi, int& l) { l = gi; return a; }, t.first + t.count, smem, bar, pp, t.first, 1);
}
template <typename S>
__device__ __noinline__ bool graph_down_s(const GraphArgs& g, const GraphTask& t, unsigned char* smem,
                                          uint64_t* bar, Pipe& pp) {
  const DownArgs* a = g.dns + t.args;
  return stage_combine_s<S>([&](int gi, int& l) { l = gi; return a; }, t.first + t.count, smem, bar, pp,
                            t.first, 1);
}
template <typename S>
__device__ __noinline__ bool graph_down10(const GraphArgs& g, const GraphTask& t, unsigned char* smem,
                                          uint64_t* bar, Pipe& pp) {
  const Down10Args* a = t.args < 0 ? &g.d10 : g.d10s + t.args;
  return stage_down10<S, false>([&](int gi, int& l) { l = gi; return a; }, t.first + t.count, smem, bar, pp,
                                t.first, 1);
}
template <typename S>
__device__ __noinline__ bool graph_down0(const GraphArgs& g, const GraphTask& t, unsigned char* smem,
                                         uint64_t* bar, Pipe& pp) {
  const Down0Args* a = t.args < 0 ? &g.d0 : g.d0s + t.args;
  return stage_combine0<S>([&](int gi, int& l) { l = gi; return view_of(*a); }, t.first + t.count, smem, bar,
                           pp, t.first, 1);
}

// D10: the task list holds the fused level-1/level-0 combine (otherwise it
// runs as its own kernel after this one, with the registers it needs).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

template <typename S, bool D10>
__global__ void __launch_bounds__(kThreads, 2) k_graph(const __grid_constant__ GraphArgs g) {
  using SM = Smem<sizeof(typename Cplx<S>::T)>;
  constexpr size_t kS = std::max(std::max(std::max(SM::up0, SM::up), std::max(SM::dns, SM::d10)), SM::dn);
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ GraphTask s_t;
  __shared__ int s_state;   // 1: a task to run, 0: the queue is exhausted, -1: a wait gave up
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kS - 64);
  init_bars(bar);
  Pipe pp{};
  unsigned* head = g.rt;
  unsigned* tail = g.rt + 1;
  unsigned* band_done = g.rt + 2;
  unsigned* band_in = band_done + g.nbands;
  unsigned* slot = band_in + g.nbands;
  // Thread 0 takes a queue index for the next task as soon as the current one
  // starts (the slot may still be empty: it is read after the current task).
  // Safe, since every slot below ntasks is filled eventually: while tasks
  // remain, some band whose inputs are complete has tasks not yet pushed only
  // if a task of an input band is still running, and that task pushes it.
  int next = 0;
  if (threadIdx.x == 0) next = (int)atomicAdd(head, 1u);
  for (;;) {
    if (threadIdx.x == 0) {
      const int idx = next;
      int task = -1, st = 1;
      if (idx >= g.ntasks) {
        st = 0;
      } else if (idx < g.nseeds) {
        task = g.seeds[idx];
      } else {
        // a slot is filled once, by the CTA that makes its band ready
        unsigned v = ld_acquire(slot + (idx - g.nseeds));
        if (v == 0u) {
          const long long lim = wait_limit(g.fault);
          const long long t0 = clock64();
          while ((v = ld_acquire(slot + (idx - g.nseeds))) == 0u) {
            __nanosleep(64);
            if (clock64() - t0 > lim) {
              atomicOr(g.fault, 4u);
              st = -1;
              break;
            }
          }
        }
        task = (int)v - 1;
      }
      if (st == 1) {
        s_t = g.tasks[task];
        // what the producers wrote (generic proxy) is read by this task's TMA copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        next = (int)atomicAdd(head, 1u);
      }
      s_state = st;
    }
    __syncthreads();
    if (s_state <= 0) return;
    const GraphTask& t = s_t;
    bool r;
    switch (t.kind) {
      case kGUp0: r = graph_up0<S>(g, t, smem, bar, pp); break;
      case kGUp: r = graph_up<S>(g, t, smem, bar, pp); break;
      case kGDownS: r = graph_down_s<S>(g, t, smem, bar, pp); break;
      case kGDown10:
        if constexpr (D10) r = graph_down10<S>(g, t, smem, bar, pp);
        else r = false;
        break;
      default: r = graph_down0<S>(g, t, smem, bar, pp); break;
    }
    if (!r) return;
    // publish: every thread's stores of the task, then the band's count; the
    // task that completes the band pushes the bands it made ready
    asm volatile("fence.proxy.async.global;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      // release: this CTA's stores (ordered before by the barrier); acquire:
      // the other producers' stores, when this task completes the band
      const GraphBand b = g.bands[t.band];
      if (atom_add_acq_rel(band_done + t.band, (unsigned)t.count) + (unsigned)t.count == b.total) {
        for (int c = b.cons0; c < b.cons1; ++c) {
          const int rb = g.cons[c];
          const GraphBand r = g.bands[rb];
          if (atom_add_acq_rel(band_in + rb, 1u) + 1u == (unsigned)r.ndeps) {
            const unsigned pos = atomicAdd(tail, (unsigned)r.ntasks);
            for (int j = 0; j < r.ntasks; ++j)
              asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(slot + pos + j),
                           "r"((unsigned)(r.task0 + j + 1))
                           : "memory");
          }
        }
      }
    }
    __syncthreads();   // s_t is written again by the next pop
  }
}

#if FLLF_STORAGE_IS_F32
// ---------------------------------------------------------------------------------------
// REDUCE (Eq. (1)) of one float plane: the gain map's Gaussian pyramid for
// pixel-adaptive runs.  One thread per output, 5 x 5 binomial taps with
// reflect-101 at the source size.
__global__ void __launch_bounds__(kThreads) k_map_reduce(const float* __restrict__ src, int sh, int sw,
                                                          int spitch, float* __restrict__ dst, int dh,
                                                          int dw, int dpitch) {
  const int idx = blockIdx.x * kThreads + threadIdx.x;
  if (idx >= dh * dw) return;
  const int y = idx / dw, x = idx - y * dw;
  const float k5[5] = {1.f, 4.f, 6.f, 4.f, 1.f};
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float* row = src + (long long)refl_fast(2 * y + i - 2, sh) * spitch;
    float h = 0.f;
#pragma unroll
    for (int j = 0; j < 5; ++j) h = fmaf(k5[j], __ldg(row + refl_fast(2 * x + j - 2, sw)), h);
    acc = fmaf(k5[i], h, acc);
  }
  dst[(long long)y * dpitch + x] = acc * (1.f / 256.f);
}

// Colour by luma (LLF on Y of YUV, U and V kept): Y = w . RGB of a planar
// RGB image (n pixels per plane), and back: every channel moves by Y' - Y.
__global__ void __launch_bounds__(kThreads) k_luma(const float* __restrict__ rgb, float* __restrict__ y,
                                                   long long n, float wr, float wg, float wb) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    y[i] = fmaf(wr, __ldg(rgb + i), fmaf(wg, __ldg(rgb + n + i), wb * __ldg(rgb + 2 * n + i)));
}
__global__ void __launch_bounds__(kThreads) k_luma_apply(const float* __restrict__ rgb,
                                                         const float* __restrict__ y,
                                                         const float* __restrict__ yf, float* __restrict__ out,
                                                         long long n) {
  for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    const float d = __ldg(yf + i) - __ldg(y + i);
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * n + i] = __ldg(rgb + c * n + i) + d;
  }
}

// Input staging: dense rows of W floats to rows of `pitch` floats (pitch a
// multiple of 4, so every row starts on a 16-byte boundary).  A CTA copies a
// row at a time, four loads in flight per thread.
__global__ void __launch_bounds__(kThreads) k_pad_rows(const float* __restrict__ src, int W, long long rows,
                                                       float* __restrict__ dst, int pitch) {
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float* sr = src + r * W;
    float* dr = dst + r * pitch;
    for (int c0 = threadIdx.x; c0 < W; c0 += 4 * kThreads) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * kThreads;
        v[u] = c < W ? __ldg(sr + c) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * kThreads;
        if (c < W) dr[c] = v[u];
      }
    }
  }
}

// The staging copies of a batch: global row r of the table's images.
__global__ void __launch_bounds__(kThreads) k_pad_batch(const PadRow* __restrict__ tab,
                                                        const int* __restrict__ prefix, int n, int total) {
  for (int r = blockIdx.x; r < total; r += gridDim.x) {
    const int j = find_entry(prefix, n, r);
    const PadRow e = tab[j];
    const int lr = r - __ldg(prefix + j);
    const float* sr = e.src + (long long)lr * e.W;
    float* dr = e.dst + (long long)lr * e.pitch;
    for (int c0 = threadIdx.x; c0 < e.W; c0 += 4 * kThreads) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * kThreads;
        v[u] = c < e.W ? __ldg(sr + c) : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u * kThreads;
        if (c < e.W) dr[c] = v[u];
      }
    }
  }
}

// Copies a status block's fault word into a host-mapped word, so that a
// frame's completion can be checked on the host without a device-to-host copy.
__global__ void k_status_snapshot(const unsigned* __restrict__ status, unsigned* __restrict__ host_word) {
  *host_word = *reinterpret_cast<const volatile unsigned*>(status);
}
#endif

// Persistent grid: at most (resident CTAs per SM) x (SMs) CTAs, or `cps`
// CTAs per SM when 0 < cps < the resident count.  The cache (and the dynamic
// shared-memory attribute it sets) is per kernel function: the kernel is the
// template argument, not just its type.
template <auto Kern>
int resident_per_sm(size_t smem, int* sms_out) {
  static int per = 0, sms = 0;
  if (per == 0) {
    int dev = 0, p = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(Kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, Kern, kThreads, smem);
    sms = n > 0 ? n : 1;
    per = p > 0 ? p : 1;
  }
  if (sms_out) *sms_out = sms;
  return per;
}
template <auto Kern>
int persistent_grid(size_t smem, int items, int cps = 0) {
  int sms = 1;
  int per = resident_per_sm<Kern>(smem, &sms);
  if (cps > 0 && cps < per) per = cps;
  const int grid = per * sms;
  return items < grid ? items : grid;
}

// Launch with programmatic stream serialization (the kernel enters through
// init_bars, which waits for the previous kernel of the stream).
template <typename... P, typename... A>
cudaError_t launch_pdl(void (*kern)(P...), int grid, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<A&&>(args)...);
}

}  // namespace

using CTS = typename Cplx<FLLF_STORAGE>::T;
using SMS = Smem<sizeof(CTS)>;

cudaError_t FLLF_LAUNCH_NAME(up0)(const Up0Args& a, cudaStream_t s, int cps) {
  const int tiles = (a.item1 > 0 ? a.item1 : cdiv(a.dst.w, kUpTW) * cdiv(a.dst.h, kUpTH) * a.planes) - a.item0;
  if (tiles <= 0) return cudaSuccess;
  if (a.fast.S > 0) {
    const int grid = persistent_grid<k_up0<FLLF_STORAGE, true>>(SMS::up0_fast, tiles, cps);
    return launch_pdl(k_up0<FLLF_STORAGE, true>, grid, SMS::up0_fast, s, a);
  }
  const int grid = persistent_grid<k_up0<FLLF_STORAGE, false>>(SMS::up0, tiles, cps);
  return launch_pdl(k_up0<FLLF_STORAGE, false>, grid, SMS::up0, s, a);
}

cudaError_t FLLF_LAUNCH_NAME(up)(const UpArgs& a, cudaStream_t s, int cps) {
  const int all = cdiv(a.dst.w, kRsTW) * cdiv(a.dst.h, kRsTH) * a.planes * (cdiv(a.K, SMS::up_kc) + (a.write_g ? 1 : 0));
  const int items = (a.item1 > 0 ? a.item1 : all) - a.item0;
  if (items <= 0) return cudaSuccess;
  const int grid = persistent_grid<k_up<FLLF_STORAGE>>(SMS::up, items, cps);
  return launch_pdl(k_up<FLLF_STORAGE>, grid, SMS::up, s, a);
}

cudaError_t FLLF_LAUNCH_NAME(down)(const DownArgs& a, cudaStream_t s, int cps) {
  const int tiles = cdiv(a.fine.w + kDnX0, kDnOW) * cdiv(a.fine.h, kDnOH) * a.planes;
  const int grid = persistent_grid<k_down<FLLF_STORAGE>>(SMS::dn1, tiles, cps);
  return launch_pdl(k_down<FLLF_STORAGE>, grid, SMS::dn1, s, a);
}

cudaError_t FLLF_LAUNCH_NAME(down_s)(const DownArgs& a, cudaStream_t s, int cps) {
  const int tiles = cdiv(a.fine.w + kDnX0, kSmW) * cdiv(a.fine.h, kSmH) * a.planes;
  if (a.fast.S > 0) {
    const int grid = persistent_grid<k_down_s<FLLF_STORAGE, true>>(SMS::dns, tiles, cps);
    return launch_pdl(k_down_s<FLLF_STORAGE, true>, grid, SMS::dns, s, a);
  }
  const int grid = persistent_grid<k_down_s<FLLF_STORAGE, false>>(SMS::dns, tiles, cps);
  return launch_pdl(k_down_s<FLLF_STORAGE, false>, grid, SMS::dns, s, a);
}

cudaError_t FLLF_LAUNCH_NAME(down0)(const Down0Args& a, cudaStream_t s, int cps) {
  const int tiles = cdiv(a.w0 + kDnX0, kDnOW) * cdiv(a.h0, kDnOH) * a.planes;
  if (a.fast.S > 0) {
    const int grid = persistent_grid<k_down0<FLLF_STORAGE, true>>(SMS::dn, tiles, cps);
    return launch_pdl(k_down0<FLLF_STORAGE, true>, grid, SMS::dn, s, a);
  }
  const int grid = persistent_grid<k_down0<FLLF_STORAGE, false>>(SMS::dn, tiles, cps);
  return launch_pdl(k_down0<FLLF_STORAGE, false>, grid, SMS::dn, s, a);
}

cudaError_t FLLF_LAUNCH_NAME(down10)(const Down10Args& a, cudaStream_t s, int cps) {
  const int tiles = cdiv(a.w0 + kDnX0, kDnOW) * cdiv(a.h0, kDnOH) * a.planes;
  if (a.fast.S > 0) {
    const int grid = persistent_grid<k_down10<FLLF_STORAGE, false, true>>(SMS::d10, tiles, cps);
    return launch_pdl(k_down10<FLLF_STORAGE, false, true>, grid, SMS::d10, s, a);
  } else if (a.M0) {
    const int grid = persistent_grid<k_down10<FLLF_STORAGE, true, false>>(SMS::d10, tiles, cps);
    return launch_pdl(k_down10<FLLF_STORAGE, true, false>, grid, SMS::d10, s, a);
  } else {
    const int grid = persistent_grid<k_down10<FLLF_STORAGE, false, false>>(SMS::d10, tiles, cps);
    return launch_pdl(k_down10<FLLF_STORAGE, false, false>, grid, SMS::d10, s, a);
  }
}

cudaError_t FLLF_LAUNCH_NAME(chain)(const ChainArgs& a, cudaStream_t s, int cps) {
  constexpr size_t kChainSmem = SMS::up > SMS::dn1 ? SMS::up : SMS::dn1;
  int sms = 1;
  int per = resident_per_sm<k_chain<FLLF_STORAGE>>(kChainSmem, &sms);
  if (cps > 0 && cps < per) per = cps;
  const int grid = per * sms;   // cooperative: every CTA resident
  void* args[] = {const_cast<ChainArgs*>(&a)};
  cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_chain<FLLF_STORAGE>),
                                              dim3(grid), dim3(kThreads), args, kChainSmem, s);
  return e != cudaSuccess ? e : cudaGetLastError();
}

// Dataflow launch: a persistent grid of the resident CTAs (at most `cps` per
// SM), programmatic stream serialization as for the per-stage kernels.
cudaError_t FLLF_LAUNCH_NAME(graph)(const GraphArgs& a, cudaStream_t s, int cps, int with_d10) {
  constexpr size_t kS = std::max(std::max(std::max(SMS::up0, SMS::up), std::max(SMS::dns, SMS::d10)), SMS::dn);
  if (with_d10) {
    const int grid = persistent_grid<k_graph<FLLF_STORAGE, true>>(kS, a.ntasks, cps);
    return grid > 0 ? launch_pdl(k_graph<FLLF_STORAGE, true>, grid, kS, s, a) : cudaSuccess;
  }
  const int grid = persistent_grid<k_graph<FLLF_STORAGE, false>>(kS, a.ntasks, cps);
  return grid > 0 ? launch_pdl(k_graph<FLLF_STORAGE, false>, grid, kS, s, a) : cudaSuccess;
}

// Resident CTAs per SM of a stage kind's kernel (kind: 0 up0, 1 up, 2 down,
// 3 down0 -- the fused level-0/1 kernel for the per-image path --, 4 chain,
// 5 the small-level combine).
int FLLF_LAUNCH_NAME(occupancy)(int kind, int batched) {
  switch (kind) {
    case 0: return batched ? resident_per_sm<k_up0_batch<FLLF_STORAGE>>(SMS::up0, nullptr)
                           : resident_per_sm<k_up0<FLLF_STORAGE, false>>(SMS::up0, nullptr);
    case 1: return batched ? resident_per_sm<k_up_batch<FLLF_STORAGE>>(SMS::up, nullptr)
                           : resident_per_sm<k_up<FLLF_STORAGE>>(SMS::up, nullptr);
    case 2: return batched ? resident_per_sm<k_down_batch<FLLF_STORAGE>>(SMS::dns, nullptr)
                           : resident_per_sm<k_down<FLLF_STORAGE>>(SMS::dn1, nullptr);
    case 3: return batched ? resident_per_sm<k_down10_batch<FLLF_STORAGE>>(SMS::d10, nullptr)
                           : resident_per_sm<k_down10<FLLF_STORAGE, false, false>>(SMS::d10, nullptr);
    case 4: {
      constexpr size_t kChainSmem = SMS::up > SMS::dn1 ? SMS::up : SMS::dn1;
      return resident_per_sm<k_chain<FLLF_STORAGE>>(kChainSmem, nullptr);
    }
    case 6: {
      constexpr size_t kS = std::max(std::max(std::max(SMS::up0, SMS::up), std::max(SMS::dns, SMS::d10)), SMS::dn);
      return resident_per_sm<k_graph<FLLF_STORAGE, true>>(kS, nullptr);
    }
    default: return resident_per_sm<k_down_s<FLLF_STORAGE, false>>(SMS::dns, nullptr);
  }
}

#if FLLF_STORAGE_IS_F32
cudaError_t launch_luma(const float* rgb, float* y, long long n, const float w[3], cudaStream_t s) {
  const int grid = (int)std::min<long long>(cdiv((int)std::min<long long>(n, 1LL << 30), kThreads), 152 * 8);
  k_luma<<<grid, kThreads, 0, s>>>(rgb, y, n, w[0], w[1], w[2]);
  return cudaGetLastError();
}
cudaError_t launch_luma_apply(const float* rgb, const float* y, const float* yf, float* out, long long n,
                              cudaStream_t s) {
  const int grid = (int)std::min<long long>(cdiv((int)std::min<long long>(n, 1LL << 30), kThreads), 152 * 8);
  k_luma_apply<<<grid, kThreads, 0, s>>>(rgb, y, yf, out, n);
  return cudaGetLastError();
}
cudaError_t launch_pad_rows(const float* src, int W, long long rows, float* dst, int pitch, cudaStream_t s) {
  if (rows <= 0 || W <= 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(rows, 152 * 8);
  k_pad_rows<<<grid, kThreads, 0, s>>>(src, W, rows, dst, pitch);
  return cudaGetLastError();
}
cudaError_t launch_pad_batch(const PadRow* tab, const int* prefix, int n, int total, cudaStream_t s) {
  if (n <= 0 || total <= 0) return cudaSuccess;
  k_pad_batch<<<std::min(total, 152 * 8), kThreads, 0, s>>>(tab, prefix, n, total);
  return cudaGetLastError();
}
cudaError_t launch_status_snapshot(const unsigned* status, unsigned* host_word, cudaStream_t s) {
  k_status_snapshot<<<1, 1, 0, s>>>(status, host_word);
  return cudaGetLastError();
}
cudaError_t launch_map_reduce(const float* src, int sh, int sw, int spitch, float* dst, int dh, int dw,
                              int dpitch, cudaStream_t s) {
  const int n = dh * dw;
  k_map_reduce<<<cdiv(n, kThreads), kThreads, 0, s>>>(src, sh, sw, spitch, dst, dh, dw, dpitch);
  return cudaGetLastError();
}
#endif

// Batched launches: the grid covers every work item of the table.
cudaError_t FLLF_LAUNCH_NAME(up0_batch)(const BatchTable<Up0Args>& tb, cudaStream_t s, int cps) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid<k_up0_batch<FLLF_STORAGE>>(SMS::up0, tb.total, cps);
  return launch_pdl(k_up0_batch<FLLF_STORAGE>, grid, SMS::up0, s, tb);
}
cudaError_t FLLF_LAUNCH_NAME(up_batch)(const BatchTable<UpArgs>& tb, cudaStream_t s, int cps) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid<k_up_batch<FLLF_STORAGE>>(SMS::up, tb.total, cps);
  return launch_pdl(k_up_batch<FLLF_STORAGE>, grid, SMS::up, s, tb);
}
cudaError_t FLLF_LAUNCH_NAME(down_batch)(const BatchTable<DownArgs>& tb, cudaStream_t s, int cps) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid<k_down_batch<FLLF_STORAGE>>(SMS::dns, tb.total, cps);
  return launch_pdl(k_down_batch<FLLF_STORAGE>, grid, SMS::dns, s, tb);
}
cudaError_t FLLF_LAUNCH_NAME(down10_batch)(const BatchTable<Down10Args>& tb, cudaStream_t s, int cps) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid<k_down10_batch<FLLF_STORAGE>>(SMS::d10, tb.total, cps);
  return launch_pdl(k_down10_batch<FLLF_STORAGE>, grid, SMS::d10, s, tb);
}
cudaError_t FLLF_LAUNCH_NAME(down0_batch)(const BatchTable<Down0Args>& tb, cudaStream_t s, int cps) {
  if (tb.total <= 0) return cudaSuccess;
  const int grid = persistent_grid<k_down0_batch<FLLF_STORAGE>>(SMS::dn, tb.total, cps);
  return launch_pdl(k_down0_batch<FLLF_STORAGE>, grid, SMS::dn, s, tb);
}

}  // namespace fllf
