// fllf_graph.cu -- host side of the dataflow launch: the task list of one or
// many images (every stage of the path cut into row-band tasks, in an order
// where producers come first) and its launch.
//
// Stages and their row bands (a band is one tile row of one plane, the unit
// a completion counter tracks):
//   up0      level 0 -> 1 REDUCE, bands of 14 level-1 rows (kUpTH)
//   up(l)    level l -> l+1 REDUCE, bands of 16 level-(l+1) rows (kRsTH)
//   down_s(l) combine at level l >= 2 on 32 x 16 tiles, bands of 16 level-l rows
//   down10   fused level-1/level-0 combine, bands of 32 level-0 rows (kDnOH)
//   down0    level-0 combine of a 2-level image, bands of 32 level-0 rows
// A band waits for the bands of the levels it reads, over the rows its valid
// outputs need (with a margin of rows on each side, and the reflected rows at
// the borders, which lie inside those ranges).  Waiting on more rows than
// needed only delays a task; it never changes the result, which is that of
// the per-stage kernels bit for bit (the same stage functions on the same
// work items).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fllf.h"
#include "fllf_internal.h"
#include "fllf_launch.h"

namespace fllf {

namespace {

template <typename T>
size_t push(std::vector<unsigned char>& blob, const T* data, size_t n, size_t align) {
  const size_t off = (blob.size() + align - 1) / align * align;
  blob.resize(off + sizeof(T) * n);
  if (n)
    std::copy(reinterpret_cast<const unsigned char*>(data), reinterpret_cast<const unsigned char*>(data + n),
              blob.begin() + off);
  return off;
}

// One stage of one image in the task graph.
struct GStage {
  int kind = 0;       // GraphKind
  int img = 0;        // index of the image
  int level = 0;      // up: source level l; down_s: level l; others 0
  int args = -1;      // index into the kind's argument table (-1: inline)
  int ntx = 0, nty = 0, planes = 0;
  int per_tile = 1;   // work items per tile (chunks of the REDUCE)
  int band_rows = 0;  // rows per band at the stage's own output level
  int counter0 = 0;   // counter of band (pl, ty) = counter0 + pl * nty + ty
  int phase = 0;      // 0: up the pyramid, 1: down
  int rank = 0;       // order among the stages of a phase at equal positions
  int scale = 0;      // log2 of the output level (level-0 rows per output row)
  int items_per_band() const { return ntx * per_tile; }
};

}  // namespace

void build_graph(const std::vector<const fllf_plan*>& plans, int prec, const GraphGrain& gr, bool inline0,
                 bool with_d10, GraphBuild* out) {
  *out = GraphBuild{};
  out->with_d10 = with_d10;
  out->lo = gr.lo;
  const int kcu = prec == FLLF_FP32 ? Smem<8>::up_kc : Smem<4>::up_kc;
  std::vector<Up0Args> a_up0;
  std::vector<UpArgs> a_up;
  std::vector<DownArgs> a_dns;
  std::vector<Down10Args> a_d10;
  std::vector<Down0Args> a_d0;
  std::vector<GStage> st;
  // per image: the stage index of up0, up(l), down_s(l) and the level-0 combine
  struct ImgStages {
    int up0 = -1, d0 = -1;
    std::vector<int> up, dns;
  };
  std::vector<ImgStages> is(plans.size());
  int ncounters = 1;  // bands are numbered from 1
  auto add_stage = [&](GStage s) {
    s.counter0 = ncounters;
    ncounters += s.nty * s.planes;
    st.push_back(s);
    return (int)st.size() - 1;
  };
  for (int i = 0; i < (int)plans.size(); ++i) {
    const fllf_plan* pl = plans[i];
    const fllf_params& p = pl->p;
    const int L = p.levels, C = p.C;
    const float turns = (float)(2.0 / p.T);
    if (L < 2) {
      out->copy_img.push_back(i);
      continue;
    }
    is[i].up.assign(L, -1);
    is[i].dns.assign(L, -1);
    const int lo = gr.lo;   // > 0: only the levels from lo up
    if (lo == 0) {
      Up0Args u{};
      u.a = pl->d_a;
      u.h0 = p.H;
      u.w0 = p.W;
      u.planes = C;
      u.dst = pl->lv[1];
      u.dst.M = nullptr;
      u.zstmap = pl->maps.z_st1;
      u.K = p.K;
      u.turns = turns;
      u.fault = pl->d_fault;
      GStage s;
      s.kind = kGUp0;
      s.img = i;
      s.ntx = cdiv(pl->lv[1].w, kUpTW);
      s.nty = cdiv(pl->lv[1].h, kUpTH);
      s.planes = C;
      s.band_rows = kUpTH;
      s.phase = 0;
      s.rank = 0;
      s.scale = 1;
      if (inline0) {
        s.args = -1;
        out->up0_inline = u;
      } else {
        s.args = (int)a_up0.size();
        a_up0.push_back(u);
        out->up0_img.push_back(i);
      }
      is[i].up0 = add_stage(s);
    }
    for (int l = std::max(1, lo); l <= L - 2; ++l) {
      UpArgs u{};
      u.zmap = pl->maps.z_up[l];
      u.gmap = pl->maps.g_up[l];
      u.src = pl->lv[l];
      u.dst = pl->lv[l + 1];
      u.src.M = u.dst.M = nullptr;
      u.planes = C;
      u.K = p.K;
      u.write_g = (l + 1 <= L - 2) ? 1 : 0;
      u.reverse = 0;
      u.fault = pl->d_fault;
      GStage s;
      s.kind = kGUp;
      s.img = i;
      s.level = l;
      s.args = (int)a_up.size();
      a_up.push_back(u);
      s.ntx = cdiv(pl->lv[l + 1].w, kRsTW);
      s.nty = cdiv(pl->lv[l + 1].h, kRsTH);
      s.planes = C;
      s.per_tile = cdiv(p.K, kcu) + u.write_g;
      s.band_rows = kRsTH;
      s.phase = 0;
      s.rank = l;
      s.scale = l + 1;
      is[i].up[l] = add_stage(s);
    }
    for (int l = L - 2; l >= std::max(2, lo); --l) {
      DownArgs d{};
      d.zmap = pl->maps.z_cs[l + 1];
      d.emap = pl->maps.e_cs[l + 1];
      d.zfmap = pl->maps.z_fs[l];
      d.gfmap = pl->maps.g_fs[l];
      d.fine = pl->lv[l];
      d.coarse = pl->lv[l + 1];
      d.fine.M = d.coarse.M = nullptr;
      d.planes = C;
      d.K = p.K;
      d.turns = turns;
      d.has_e = (l + 1 <= L - 2) ? 1 : 0;
      d.fault = pl->d_fault;
      GStage s;
      s.kind = kGDownS;
      s.img = i;
      s.level = l;
      s.args = (int)a_dns.size();
      a_dns.push_back(d);
      s.ntx = cdiv(pl->lv[l].w + kDnX0, kSmW);
      s.nty = cdiv(pl->lv[l].h, kSmH);
      s.planes = C;
      s.band_rows = kSmH;
      s.phase = 1;
      s.rank = L - 2 - l;
      s.scale = l;
      is[i].dns[l] = add_stage(s);
    }
    if (lo > 0) continue;   // the level-0 stage runs as its own kernel
    GStage s;
    s.img = i;
    s.ntx = cdiv(p.W + kDnX0, kDnOW);
    s.nty = cdiv(p.H, kDnOH);
    s.planes = C;
    s.band_rows = kDnOH;
    s.phase = 1;
    s.rank = L;
    s.scale = 0;
    if (L >= 3) {
      Down10Args d{};
      d.z1map = pl->maps.z_dn[1];
      d.g1map = pl->maps.g1_d10;
      d.z2map = pl->maps.z2_d10;
      d.e2map = pl->maps.e2_d10;
      d.h0 = p.H;
      d.w0 = p.W;
      d.planes = C;
      d.l1 = pl->lv[1];
      d.l2 = pl->lv[2];
      d.l1.M = d.l2.M = nullptr;
      d.K = p.K;
      d.turns = turns;
      d.has_e2 = L >= 4 ? 1 : 0;
      d.fault = pl->d_fault;
      s.kind = kGDown10;
      if (inline0) {
        s.args = -1;
        out->d10_inline = d;
      } else {
        s.args = (int)a_d10.size();
        a_d10.push_back(d);
        out->d10_img.push_back(i);
      }
      // without it in the task list, the fused combine runs as its own kernel
      // (argument blocks kept for that launch)
      if (!with_d10) continue;
    } else {
      Down0Args d{};
      d.zmap = pl->maps.z_dn[1];
      d.emap = pl->maps.e_dn[1];
      d.h0 = p.H;
      d.w0 = p.W;
      d.planes = C;
      d.coarse = pl->lv[1];
      d.coarse.M = nullptr;
      d.K = p.K;
      d.turns = turns;
      d.has_e = 0;
      d.fault = pl->d_fault;
      s.kind = kGDown0;
      if (inline0) {
        s.args = -1;
        out->d0_inline = d;
      } else {
        s.args = (int)a_d0.size();
        a_d0.push_back(d);
        out->d0_img.push_back(i);
      }
    }
    is[i].d0 = add_stage(s);
  }

  // Bands: every band's producers (the bands it reads, over the rows its
  // valid outputs need), then the readers of each band and the tasks.
  std::vector<std::vector<int>> band_producers(ncounters);
  std::vector<int> band_stage(ncounters, -1);
  auto add_rows = [&](std::vector<int>& ctrs, int sidx, int pl, int lo, int hi, int h) {
    if (sidx < 0) return;   // produced by a kernel that ran before this launch
    const GStage& ps = st[sidx];
    lo = std::max(lo, 0);
    hi = std::min(hi, h - 1);
    if (hi < lo) return;
    const int b0 = lo / ps.band_rows, b1 = std::min(hi / ps.band_rows, ps.nty - 1);
    for (int b = b0; b <= b1; ++b) ctrs.push_back(ps.counter0 + pl * ps.nty + b);
  };
  for (int sidx = 0; sidx < (int)st.size(); ++sidx) {
    const GStage& s = st[sidx];
    const fllf_plan* pl = plans[s.img];
    const std::vector<Level>& lv = pl->lv;
    const int L = pl->p.levels;
    for (int plane = 0; plane < s.planes; ++plane)
      for (int ty = 0; ty < s.nty; ++ty) {
        std::vector<int> ctrs;
        switch (s.kind) {
          case kGUp0:
            break;
          case kGUp: {
            const int l = s.level, Y1 = ty * kRsTH;
            const int yv = std::min(Y1 + kRsTH - 1, lv[l + 1].h - 1);
            add_rows(ctrs, l == 1 ? is[s.img].up0 : is[s.img].up[l - 1], plane, 2 * Y1 - 3, 2 * yv + 3, lv[l].h);
            break;
          }
          case kGDownS: {
            const int l = s.level, Y0 = ty * kSmH;
            const int yv = std::min(Y0 + kSmH - 1, lv[l].h - 1);
            add_rows(ctrs, is[s.img].up[l - 1], plane, Y0 - 1, yv + 1, lv[l].h);   // Z_l, G_l
            add_rows(ctrs, is[s.img].up[l], plane, Y0 / 2 - 2, yv / 2 + 2, lv[l + 1].h);   // Z_{l+1}
            if (l + 1 <= L - 2) add_rows(ctrs, is[s.img].dns[l + 1], plane, Y0 / 2 - 2, yv / 2 + 2, lv[l + 1].h);
            break;
          }
          case kGDown10: {
            const int Y0 = ty * kDnOH;
            const int c1 = Y0 / 2 - 1;   // the level-1 window (kDnCH rows)
            add_rows(ctrs, is[s.img].up0, plane, c1 - 1, c1 + kDnCH, lv[1].h);   // Z_1, G_1
            const int c2 = (c1 - 1) / 2;  // the level-2 window (kD2H rows)
            add_rows(ctrs, is[s.img].up[1], plane, c2 - 1, c2 + kD2H, lv[2].h);   // Z_2
            if (L >= 4) add_rows(ctrs, is[s.img].dns[2], plane, c2 - 1, c2 + kD2H, lv[2].h);   // E_2
            break;
          }
          default: {  // level-0 combine of a 2-level image
            const int Y0 = ty * kDnOH;
            const int c1 = Y0 / 2 - 1;
            add_rows(ctrs, is[s.img].up0, plane, c1 - 1, c1 + kDnCH, lv[1].h);
            break;
          }
        }
        const int me = s.counter0 + plane * s.nty + ty;
        std::sort(ctrs.begin(), ctrs.end());
        ctrs.erase(std::unique(ctrs.begin(), ctrs.end()), ctrs.end());
        band_producers[me] = ctrs;
        band_stage[me] = sidx;
      }
  }
  const int nb = ncounters - 1;   // bands are numbered from 1; index 0 is unused
  // Work items per task: the given size at the finest level of a stage kind,
  // halved per level above it, so that the coarse levels (few bands, on the
  // path every finer level waits for) run as many short tasks.
  auto grain_of = [&](const GStage& s) {
    switch (s.kind) {
      case kGUp0: return std::max(1, gr.up0);
      case kGUp: return std::max(1, gr.up >> std::min(20, s.level - 1));
      case kGDownS: return std::max(1, gr.dns >> std::min(20, s.level - 2));
      case kGDown10: return std::max(1, gr.d10);
      default: return std::max(1, gr.d0);
    }
  };
  std::vector<GraphTask> tasks;
  std::vector<GraphBand> bands(nb + 1, GraphBand{});
  for (int sidx = 0; sidx < (int)st.size(); ++sidx) {
    const GStage& s = st[sidx];
    const int per = s.items_per_band(), g = grain_of(s);
    for (int plane = 0; plane < s.planes; ++plane)
      for (int ty = 0; ty < s.nty; ++ty) {
        const int band = s.counter0 + plane * s.nty + ty;
        const int first = (plane * s.nty + ty) * per;
        GraphBand& b = bands[band];
        b.total = (unsigned)per;
        b.task0 = (int)tasks.size();
        b.ndeps = (int)band_producers[band].size();
        for (int j = 0; j < per; j += g) {
          GraphTask t{};
          t.kind = s.kind;
          t.args = s.args;
          t.first = first + j;
          t.count = std::min(g, per - j);
          t.band = band;
          tasks.push_back(t);
        }
        b.ntasks = (int)tasks.size() - b.task0;
      }
  }
  std::vector<std::vector<int>> readers(nb + 1);
  for (int band = 1; band <= nb; ++band)
    for (int pb : band_producers[band]) readers[pb].push_back(band);
  std::vector<int> cons;
  for (int band = 1; band <= nb; ++band) {
    bands[band].cons0 = (int)cons.size();
    cons.insert(cons.end(), readers[band].begin(), readers[band].end());
    bands[band].cons1 = (int)cons.size();
  }
  // seeds: the tasks of the bands that read nothing (the level-0 REDUCE),
  // top rows first over every image (rows as a fraction of the height), so
  // that the levels above can start on the first rows while the rest runs
  std::vector<std::pair<double, int>> seed_keys;
  for (int band = 1; band <= nb; ++band) {
    if (bands[band].ndeps != 0) continue;
    const GStage& s = st[band_stage[band]];
    const int ty = (band - s.counter0) % s.nty;
    const double frac = (double)ty * s.band_rows * (double)(1 << s.scale) / std::max(1, plans[s.img]->p.H);
    for (int j = 0; j < bands[band].ntasks; ++j) seed_keys.push_back({frac, bands[band].task0 + j});
  }
  std::stable_sort(seed_keys.begin(), seed_keys.end());
  std::vector<int> seeds;
  for (const auto& k : seed_keys) seeds.push_back(k.second);
  const int nt = (int)tasks.size();
  // every work item of every stage in exactly one task
  out->ok = true;
  for (const GStage& s : st) {
    long long seen = 0;
    for (int b = s.counter0; b < s.counter0 + s.nty * s.planes; ++b)
      for (int j = 0; j < bands[b].ntasks; ++j) seen += tasks[bands[b].task0 + j].count;
    if (seen != (long long)s.items_per_band() * s.nty * s.planes) out->ok = false;
  }

  std::vector<unsigned char>& blob = out->blob;
  out->up0_off = push(blob, a_up0.data(), a_up0.size(), 128);
  out->ups_off = push(blob, a_up.data(), a_up.size(), 128);
  out->dns_off = push(blob, a_dns.data(), a_dns.size(), 128);
  out->d10_off = push(blob, a_d10.data(), a_d10.size(), 128);
  out->d0_off = push(blob, a_d0.data(), a_d0.size(), 128);
  out->tasks_off = push(blob, tasks.data(), tasks.size(), 16);
  out->bands_off = push(blob, bands.data(), bands.size(), 16);
  out->cons_off = push(blob, cons.data(), cons.size(), 16);
  out->seeds_off = push(blob, seeds.data(), seeds.size(), 16);
  // run state: head, tail, per band the items done and the inputs complete,
  // then one queue slot per task that is not a seed
  out->rt_words = 2 + 2 * (size_t)(nb + 1) + (size_t)(nt - (int)seeds.size());
  const std::vector<unsigned> zeros(out->rt_words, 0u);
  out->rt_off = push(blob, zeros.data(), zeros.size(), 256);
  out->ntasks = nt;
  out->nbands = nb + 1;
  out->nseeds = (int)seeds.size();
  out->n_up0 = (int)a_up0.size();
  out->n_ups = (int)a_up.size();
  out->n_dns = (int)a_dns.size();
  out->n_d10 = (int)a_d10.size();
  out->n_d0 = (int)a_d0.size();
}

bool check_graph(const GraphBuild& gb, std::string* why) {
  const GraphTask* tasks = reinterpret_cast<const GraphTask*>(gb.blob.data() + gb.tasks_off);
  const GraphBand* bands = reinterpret_cast<const GraphBand*>(gb.blob.data() + gb.bands_off);
  const int* cons = reinterpret_cast<const int*>(gb.blob.data() + gb.cons_off);
  const int* seeds = reinterpret_cast<const int*>(gb.blob.data() + gb.seeds_off);
  // run the queue on one host worker, as the CTAs do
  std::vector<unsigned> done(gb.nbands, 0u), in(gb.nbands, 0u);
  std::vector<int> queue(seeds, seeds + gb.nseeds), popped(gb.ntasks, 0);
  for (size_t q = 0; q < queue.size(); ++q) {
    const int ti = queue[q];
    if (ti < 0 || ti >= gb.ntasks || popped[ti]++) {
      *why = "task " + std::to_string(ti) + " queued twice or unknown";
      return false;
    }
    const GraphTask& t = tasks[ti];
    if (t.band < 1 || t.band >= gb.nbands || in[t.band] != (unsigned)bands[t.band].ndeps) {
      *why = "task " + std::to_string(ti) + " runs before a band it reads is complete";
      return false;
    }
    done[t.band] += (unsigned)t.count;
    if (done[t.band] == bands[t.band].total)
      for (int c = bands[t.band].cons0; c < bands[t.band].cons1; ++c) {
        const GraphBand& r = bands[cons[c]];
        if (++in[cons[c]] == (unsigned)r.ndeps)
          for (int j = 0; j < r.ntasks; ++j) queue.push_back(r.task0 + j);
      }
  }
  if ((int)queue.size() != gb.ntasks) {
    *why = std::to_string(gb.ntasks - (int)queue.size()) + " tasks are never made ready";
    return false;
  }
  for (int b = 1; b < gb.nbands; ++b)
    if (done[b] != bands[b].total) {
      *why = "band " + std::to_string(b) + " does not complete";
      return false;
    }
  if (gb.rt_words != 2 + 2 * (size_t)gb.nbands + (size_t)(gb.ntasks - gb.nseeds)) {
    *why = "run-state size";
    return false;
  }
  return true;
}

GraphArgs graph_args(const GraphBuild& gb, const unsigned char* d_base, unsigned* d_fault) {
  GraphArgs g{};
  g.up0 = gb.up0_inline;
  g.d10 = gb.d10_inline;
  g.d0 = gb.d0_inline;
  g.up0s = reinterpret_cast<const Up0Args*>(d_base + gb.up0_off);
  g.ups = reinterpret_cast<const UpArgs*>(d_base + gb.ups_off);
  g.dns = reinterpret_cast<const DownArgs*>(d_base + gb.dns_off);
  g.d10s = reinterpret_cast<const Down10Args*>(d_base + gb.d10_off);
  g.d0s = reinterpret_cast<const Down0Args*>(d_base + gb.d0_off);
  g.tasks = reinterpret_cast<const GraphTask*>(d_base + gb.tasks_off);
  g.bands = reinterpret_cast<const GraphBand*>(d_base + gb.bands_off);
  g.cons = reinterpret_cast<const int*>(d_base + gb.cons_off);
  g.seeds = reinterpret_cast<const int*>(d_base + gb.seeds_off);
  g.rt = reinterpret_cast<unsigned*>(const_cast<unsigned char*>(d_base) + gb.rt_off);
  g.fault = d_fault;
  g.ntasks = gb.ntasks;
  g.nbands = gb.nbands;
  g.nseeds = gb.nseeds;
  g.inline0 = 0;
  return g;
}

PlanGraph* plan_graph_create(const fllf_plan* plan, const GraphGrain& gr, bool with_d10, cudaError_t* err) {
  *err = cudaSuccess;
  PlanGraph* g = new PlanGraph();
  build_graph({plan}, plan->p.precision, gr, true, with_d10, &g->gb);
  if (!g->gb.ok) {
    delete g;
    *err = cudaErrorInvalidValue;
    return nullptr;
  }
  cudaError_t e = cudaMalloc(&g->d_mem, g->gb.blob.size());
  if (e == cudaSuccess) e = cudaMemcpy(g->d_mem, g->gb.blob.data(), g->gb.blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (g->d_mem) cudaFree(g->d_mem);
    delete g;
    *err = e;
    return nullptr;
  }
  g->args = graph_args(g->gb, g->d_mem, plan->d_fault);
  g->args.inline0 = 1;
  return g;
}

void plan_graph_destroy(PlanGraph* g) {
  if (!g) return;
  if (g->d_mem) cudaFree(g->d_mem);
  delete g;
}

cudaError_t launch_graph(int prec, const GraphArgs& g, size_t rt_bytes, cudaStream_t s, int cps,
                         bool with_d10) {
  cudaError_t e = cudaMemsetAsync(g.rt, 0, rt_bytes, s);
  if (e != cudaSuccess || g.ntasks == 0) return e;
  const int w = with_d10 ? 1 : 0;
  switch (prec) {
    case FLLF_FP16: return launch_graph_f16(g, s, cps, w);
    case FLLF_BF16: return launch_graph_bf16(g, s, cps, w);
    default: return launch_graph_f32(g, s, cps, w);
  }
}

}  // namespace fllf

using namespace fllf;

extern "C" fllf_status fllf_dataflow_check(const fllf_params* ps, int n, const int* task_items, int with_d10,
                                           int first_level, int* ntasks, int* nbands) {
  if (!ps || n < 1 || n > 4096) {
    set_last_error("need 1..4096 parameter sets");
    return FLLF_EINVAL;
  }
  std::vector<fllf_plan> plans(n);
  std::vector<const fllf_plan*> ptrs;
  for (int i = 0; i < n; ++i) {
    const fllf_status st = validate(&ps[i]);
    if (st != FLLF_OK) return st;
    fllf_plan& pl = plans[i];
    pl.p = normalized(ps[i]);
    if (pl.p.method != FLLF_METHOD_FOURIER || pl.p.precision != ps[0].precision) {
      set_last_error("dataflow task lists hold Fourier LLF images of one storage precision");
      return FLLF_EINVAL;
    }
    layout(pl.p, &pl.lv);   // offsets stand in for device addresses: the tables are not used
    const int L = pl.p.levels;
    PathMaps& m = pl.maps;
    for (auto* v : {&m.z_dn, &m.e_dn, &m.z_up, &m.g_up, &m.z_dn1, &m.z_fn, &m.g_fn, &m.z_cs, &m.e_cs, &m.z_fs,
                    &m.g_fs})
      v->assign(L, CUtensorMap{});
    ptrs.push_back(&pl);
  }
  GraphGrain g;
  if (task_items) {
    for (int k = 0; k < 5; ++k)
      if (task_items[k] < 1 || task_items[k] > 4096) {
        set_last_error("task_items must be 1..4096");
        return FLLF_EINVAL;
      }
    g.up0 = task_items[0];
    g.up = task_items[1];
    g.dns = task_items[2];
    g.d10 = task_items[3];
    g.d0 = task_items[4];
  }
  if (first_level != 0 && (first_level < 2 || first_level > 15)) {
    set_last_error("first_level must be 0 or 2..15");
    return FLLF_EINVAL;
  }
  g.lo = first_level;
  GraphBuild gb;
  build_graph(ptrs, ps[0].precision, g, n == 1, with_d10 != 0, &gb);
  std::string why;
  if (!gb.ok) {
    set_last_error("a task list that does not cover every work item once, or a cycle among the bands");
    return FLLF_EINVAL;
  }
  if (!check_graph(gb, &why)) {
    set_last_error(why);
    return FLLF_EINVAL;
  }
  if (ntasks) *ntasks = gb.ntasks;
  if (nbands) *nbands = gb.nbands - 1;
  return FLLF_OK;
}
