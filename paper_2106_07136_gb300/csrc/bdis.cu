// bdis.cu -- C ABI, parameter checks, workspace and the coarse-to-fine driver
// of the BDIS CUDA library (arXiv 2106.07136, Sec. 2).
//
// bdis_match enqueues, on the handle's stream:
//   level 0 with the first pyramid step (one kernel), (pyramid_level) x
//   (coarsest - 1), then for l = coarsest .. finest: search(l), densify(l),
//   and an upsample when finest > 0 (pyramid variants 1 and 0: the level-0
//   preparation, then every step; variant 0 two kernels per step).
// That is coarsest + 2 * (coarsest - finest + 1) (+1) launches per batch by
// default, independent of the number of pairs in it.
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <new>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "bdis_internal.cuh"

// Calls of bdis_match_host_async that can be in flight at once: each holds
// its own device inputs and output, reused by the call kAsyncSlots later.
constexpr int kAsyncSlots = BDIS_ASYNC_SLOTS;

struct bdis_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // kernel timing (bdis_enable_timing)
  bool timing = false;
  struct Mark {
    cudaEvent_t start, stop;
    int cls;
  };
  std::vector<cudaEvent_t> event_pool;
  std::vector<Mark> marks;
  // bdis_match_host pipeline: copy-in and copy-out streams beside `stream`,
  // and per buffer slot the events "inputs copied", "matched", "output copied"
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  // (bdis_match_host uses two slots, bdis_match_host_async kAsyncSlots)
  cudaEvent_t ev_in[kAsyncSlots] = {}, ev_done[kAsyncSlots] = {}, ev_out[kAsyncSlots] = {};
  // bdis_match_host_async: calls enqueued since the streams were last idle,
  // the next ticket, and the workspace layout those calls use (slot buffers)
  int async_pending = 0;
  uint64_t async_next = 1;
  size_t async_key[1 + 3 * kAsyncSlots] = {};
};

namespace bdis {
namespace {

thread_local char g_last_error[256] = "";

// Device allocations still to fail (bdis_inject_alloc_failures).
std::atomic<int> g_alloc_failures{0};

constexpr size_t kAlign = 256;

inline size_t align_up(size_t n) { return (n + kAlign - 1) / kAlign * kAlign; }

}  // namespace

Layout plan_layout(int w, int h, int count, const bdis_params &p, bool host_staging) {
  Layout lay;
  size_t off = 0;
  auto take = [&](size_t n) {
    size_t o = off;
    off += align_up(n);
    return o;
  };
  lay.levels = p.coarsest_scale + 1;
  const int stride = grid_stride(p.patch_size, p.overlap);
  size_t max_np = 0;
  for (int l = 0; l < lay.levels; ++l) {
    lay.lw[l] = level_dim(w, l);
    lay.lh[l] = level_dim(h, l);
    const size_t plane = (size_t)lay.lw[l] * lay.lh[l] * count * sizeof(float);
    lay.L[l] = take(plane);
    lay.R[l] = take(2 * plane);  // packed (R, R[x+1] - R[x])
    lay.G[l] = take(plane);
    if (l >= p.finest_scale && l > 0) lay.D[l] = take(plane);
    if (l >= p.finest_scale) {
      size_t np = (size_t)grid_count(lay.lw[l], p.patch_size, stride) *
                  grid_count(lay.lh[l], p.patch_size, stride);
      if (np > max_np) max_np = np;
    }
  }
  lay.d_star = take(max_np * count * sizeof(float));
  lay.weight = take(max_np * count * sizeof(float));
  lay.warm_w = level_dim(w, p.coarsest_scale + 1);
  lay.warm_h = level_dim(h, p.coarsest_scale + 1);
  lay.warm = take((size_t)lay.warm_w * lay.warm_h * count * sizeof(float));
  {
    const int top = p.coarsest_scale;
    const size_t np_top = (size_t)grid_count(lay.lw[top], p.patch_size, stride) *
                          grid_count(lay.lh[top], p.patch_size, stride) * count;
    lay.d_star2 = take(np_top * sizeof(float));
    lay.weight2 = take(np_top * sizeof(float));
    lay.post1 = take(np_top * sizeof(float));
    lay.post2 = take(np_top * sizeof(float));
    lay.flags1 = take(np_top);
    lay.flags2 = take(np_top);
    lay.prop_level = proposal_level(top);
    lay.prop = take((size_t)lay.lw[lay.prop_level] * lay.lh[lay.prop_level] * count *
                    sizeof(float));
  }
  if (host_staging) {
    lay.in_left = take((size_t)w * h * count);
    lay.in_right = take((size_t)w * h * count);
    lay.out = take((size_t)w * h * count * sizeof(float));
  }
  lay.bytes = off;
  return lay;
}

namespace {

// Let every asynchronous host match finish: all three streams idle.
cudaError_t drain_async(bdis_handle *h) {
  if (!h->async_pending) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(h->copy_in);
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  cudaError_t e3 = cudaStreamSynchronize(h->copy_out);
  h->async_pending = 0;
  return e != cudaSuccess ? e : (e2 != cudaSuccess ? e2 : e3);
}

// Every entry that uses the workspace comes through here. A call other than
// an asynchronous host match first lets those finish: its own layout may
// overlap their input and output slots.
bdis_status ensure_workspace(bdis_handle *h, size_t bytes, bool from_async = false) {
  if (!from_async || bytes > h->ws_bytes) {
    cudaError_t e = drain_async(h);
    if (e != cudaSuccess) return record_cuda(e);
  }
  if (bytes <= h->ws_bytes) return BDIS_OK;
  // The old block may still be read by work already on the stream.
  if (h->ws) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return record_cuda(e);
    cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  void *p = nullptr;
  cudaError_t e = device_alloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    snprintf(g_last_error, sizeof g_last_error, "workspace of %zu bytes: %s", bytes,
             cudaGetErrorString(e));
    return BDIS_E_NOMEM;
  }
  h->ws = p;
  h->ws_bytes = bytes;
  return BDIS_OK;
}

bdis_status check_image(const bdis_image *im) {
  if (!im || !im->data) return BDIS_E_INVALID_ARG;
  if (im->width < 1 || im->height < 1 || im->count < 1) return BDIS_E_INVALID_ARG;
  if (im->format != BDIS_U8 && im->format != BDIS_F32) return BDIS_E_INVALID_ARG;
  const size_t es = im->format == BDIS_U8 ? 1 : 4;
  if (im->pitch_bytes < (size_t)im->width * es || im->pitch_bytes % es) return BDIS_E_INVALID_ARG;
  if (im->count > 1 && im->image_stride_bytes < im->pitch_bytes * (size_t)im->height)
    return BDIS_E_INVALID_ARG;
  if (im->count > 1 && im->image_stride_bytes % es) return BDIS_E_INVALID_ARG;
  return BDIS_OK;
}

bdis_status check_pair(const bdis_image *l, const bdis_image *r) {
  bdis_status s = check_image(l);
  if (s != BDIS_OK) return s;
  s = check_image(r);
  if (s != BDIS_OK) return s;
  if (l->width != r->width || l->height != r->height || l->count != r->count ||
      l->format != r->format || l->pitch_bytes != r->pitch_bytes ||
      (l->count > 1 && l->image_stride_bytes != r->image_stride_bytes))
    return BDIS_E_INVALID_ARG;
  return BDIS_OK;
}

// Device (or managed) memory that kernels on the CURRENT device may read: a
// plain device allocation must live on that device (another GPU's memory
// without peer access would be an illegal address there, not an argument error).
bdis_status check_device_ptr(const void *p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return BDIS_E_INVALID_ARG;
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return BDIS_E_INVALID_ARG;
  if (at.type == cudaMemoryTypeDevice) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return BDIS_E_INVALID_ARG;
    }
    if (at.device != cur) return BDIS_E_INVALID_ARG;
  }
  return BDIS_OK;
}

bdis_status check_geometry(int w, int h, const bdis_params &p) {
  if (level_dim(w, p.coarsest_scale) < p.patch_size ||
      level_dim(h, p.coarsest_scale) < p.patch_size)
    return BDIS_E_INVALID_ARG;
  return BDIS_OK;
}

cudaEvent_t take_event(bdis_handle *h) {
  if (!h->event_pool.empty()) {
    cudaEvent_t e = h->event_pool.back();
    h->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Bracket one launch with events when timing is on.
// NVTX range over one host scope (a launch, a whole-method call): names are
// string literals or the per-class, per-level table below.
struct Range {
  explicit Range(const char *name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range &) = delete;
  Range &operator=(const Range &) = delete;
};

// "bdis <class> L<level>" per kernel class and pyramid level, "bdis <class>"
// without a level; built once (a function-local static).
const char *range_name(int cls, int level) {
  struct Table {
    char s[8][17][40];
    Table() {
      static const char *kClass[8] = {"prepare_level0", "pyramid", "search", "densify",
                                      "upsample", "seed_map", "proposal_net", "select_start"};
      for (int c = 0; c < 8; ++c)
        for (int l = 0; l < 17; ++l) {
          if (l < 16)
            snprintf(s[c][l], sizeof s[c][l], "bdis %s L%d", kClass[c], l);
          else
            snprintf(s[c][l], sizeof s[c][l], "bdis %s", kClass[c]);
        }
    }
  };
  static const Table t;
  if (cls < 0 || cls >= 8) return "bdis";
  return t.s[cls][level >= 0 && level < 16 ? level : 16];
}

struct Timed {
  bdis_handle *h;
  cudaEvent_t a = nullptr, b = nullptr;
  int cls;
  Range range;
  Timed(bdis_handle *h_, int cls_, int level = -1)
      : h(h_), cls(cls_), range(range_name(cls_, level)) {
    if (h->timing) {
      a = take_event(h);
      b = take_event(h);
      if (a && b) cudaEventRecord(a, h->stream);
    }
  }
  ~Timed() {
    if (a && b) {
      cudaEventRecord(b, h->stream);
      h->marks.push_back({a, b, cls});
    } else {
      if (a) h->event_pool.push_back(a);
      if (b) h->event_pool.push_back(b);
    }
  }
};

// Arguments of the search and densify launches of level l (the coarser map
// of level l+1 seeds the patches; level 0 densifies into `out`).
SearchArgs level_search_args(char *base, const Layout &lay, const bdis_params &p, int count,
                             int l, bool warm = false) {
  auto F = [&](size_t off) { return reinterpret_cast<float *>(base + off); };
  SearchArgs sa{};
  fill_search_args(sa, lay.lw[l], lay.lh[l], count, p);
  sa.L = F(lay.L[l]);
  sa.R2 = reinterpret_cast<const float2 *>(base + lay.R[l]);
  sa.G = F(lay.G[l]);
  if (l < p.coarsest_scale) {
    sa.coarse = F(lay.D[l + 1]);
    sa.cw = lay.lw[l + 1];
    sa.ch = lay.lh[l + 1];
    sa.cplane = (long long)sa.cw * sa.ch;
  } else if (warm) {
    sa.coarse = F(lay.warm);
    sa.cw = lay.warm_w;
    sa.ch = lay.warm_h;
    sa.cplane = (long long)sa.cw * sa.ch;
  }
  sa.d_star = F(lay.d_star);
  sa.weight = F(lay.weight);
  return sa;
}

DensifyArgs level_densify_args(char *base, const Layout &lay, const bdis_params &p, int count,
                               int l, float *out, bool warm = false) {
  auto F = [&](size_t off) { return reinterpret_cast<float *>(base + off); };
  DensifyArgs da{};
  fill_densify_args(da, lay.lw[l], lay.lh[l], count, p);
  da.d_star = F(lay.d_star);
  da.weight = F(lay.weight);
  if (l < p.coarsest_scale) {
    da.coarse = F(lay.D[l + 1]);
    da.cw = lay.lw[l + 1];
    da.ch = lay.lh[l + 1];
    da.cplane = (long long)da.cw * da.ch;
  } else if (warm) {
    da.coarse = F(lay.warm);
    da.cw = lay.warm_w;
    da.ch = lay.warm_h;
    da.cplane = (long long)da.cw * da.ch;
  }
  da.is_finest = (l == p.finest_scale);
  da.L = F(lay.L[l]);
  da.R2 = reinterpret_cast<const float2 *>(base + lay.R[l]);
  da.out = (l == 0) ? out : F(lay.D[l]);
  return da;
}

// The whole method on device images already checked; `out` dense device.
bdis_status run_match(bdis_handle *h, const bdis_image &left, const bdis_image &right,
                      const bdis_params &p, float *out, const Layout &lay,
                      const Tuning *tune = nullptr, const Seed *seed = nullptr) {
  Range whole(seed && seed->net ? "bdis match (learned start)"
               : seed && seed->map ? "bdis match (seeded start)"
                                   : "bdis match");
  char *base = static_cast<char *>(h->ws);
  auto F = [&](size_t off) { return reinterpret_cast<float *>(base + off); };
  auto F2 = [&](size_t off) { return reinterpret_cast<float2 *>(base + off); };
  const int count = left.count;
  cudaStream_t st = h->stream;
  cudaError_t e;
  const int top = p.coarsest_scale;
  const bool seeded = seed && (seed->map || seed->net);
  if (seed && seed->map) {
    // first, before the output (which may alias the seed) is written
    Timed tm(h, 5);
    e = launch_warm_map(seed->map, level_dim(left.width, seed->level),
                        level_dim(left.height, seed->level), top + 1 - seed->level, count,
                        F(lay.warm), st);
    if (e != cudaSuccess) return record_cuda(e);
  }
  // level 0 and (pyramid variant 2) the first pyramid step in the same launch
  const bool fuse0 = pyramid_fused() == 2 && p.coarsest_scale >= 1;
  {
    Timed tm(h, 0, 0);
    e = fuse0 ? launch_prepare_pyramid0(left, right, F(lay.L[0]), F2(lay.R[0]), F(lay.G[0]),
                                        F(lay.L[1]), F2(lay.R[1]), F(lay.G[1]), st)
              : launch_prepare_level0(left, right, F(lay.L[0]), F2(lay.R[0]), F(lay.G[0]), st);
  }
  if (e != cudaSuccess) return record_cuda(e);
  for (int l = fuse0 ? 1 : 0; l < p.coarsest_scale; ++l) {
    {
      Timed tm(h, 1, l + 1);
      e = launch_pyramid_level(F(lay.L[l]), F2(lay.R[l]), lay.lw[l], lay.lh[l], count,
                               F(lay.L[l + 1]), F2(lay.R[l + 1]), F(lay.G[l + 1]), st);
    }
    if (e != cudaSuccess) return record_cuda(e);
  }
  if (seed && seed->net) {
    // the proposal network on the level planes just built, then its seed map
    const int nl = seed->level;
    {
      Timed tm(h, 6, nl);
      bdis_status s = net_forward_on(seed->net, F(lay.L[nl]), F(lay.R[nl]), 2, lay.lw[nl],
                                     lay.lh[nl], count, F(lay.prop), st);
      if (s != BDIS_OK) return s;
    }
    Timed tm(h, 5);
    e = launch_warm_map(F(lay.prop), lay.lw[nl], lay.lh[nl], top + 1 - nl, count, F(lay.warm),
                        st);
    if (e != cudaSuccess) return record_cuda(e);
  }
  for (int l = p.coarsest_scale; l >= p.finest_scale; --l) {
    const bool two = seeded && seed->fallback && l == top;
    SearchArgs sa = level_search_args(base, lay, p, count, l, seeded);
    if (tune) apply_tuning(sa, tune->level[l]);
    if (two) {
      sa.posterior = F(lay.post1);
      sa.flags = reinterpret_cast<uint8_t *>(base + lay.flags1);
    }
    {
      Timed tm(h, 2, l);
      e = launch_search(sa, st);
    }
    if (e != cudaSuccess) return record_cuda(e);
    if (two) {
      // R16: the plain start of the same level, then the per-patch choice
      SearchArgs sb = level_search_args(base, lay, p, count, l, false);
      if (tune) apply_tuning(sb, tune->level[l]);
      sb.d_star = F(lay.d_star2);
      sb.weight = F(lay.weight2);
      sb.posterior = F(lay.post2);
      sb.flags = reinterpret_cast<uint8_t *>(base + lay.flags2);
      {
        Timed tm(h, 2, l);
        e = launch_search(sb, st);
      }
      if (e != cudaSuccess) return record_cuda(e);
      Timed tm(h, 7, l);
      e = launch_select_start(sa.d_star, sa.weight, sa.posterior, sa.flags, sb.d_star, sb.weight,
                              sb.posterior, sb.flags, sa.total, st);
      if (e != cudaSuccess) return record_cuda(e);
    }
    // carried pixels of the coarsest level: the seed, unless the fallback applies
    DensifyArgs da = level_densify_args(base, lay, p, count, l, out, seeded && !two);
    if (tune) apply_tuning(da, tune->level[l]);
    {
      Timed tm(h, 3, l);
      e = launch_densify(da, st);
    }
    if (e != cudaSuccess) return record_cuda(e);
  }
  const float *coarse = p.finest_scale == 0 ? out : F(lay.D[p.finest_scale]);
  const int cw = lay.lw[p.finest_scale], ch = lay.lh[p.finest_scale];
  if (p.finest_scale > 0) {
    Timed tm(h, 4);
    e = launch_upsample(coarse, cw, ch, p.finest_scale, left.width, left.height, count, out, st);
    if (e != cudaSuccess) return record_cuda(e);
  }
  return BDIS_OK;
}

bdis_status bind_device(const bdis_handle *h) {
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return record_cuda(e);
  if (cur != h->device) {
    e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return record_cuda(e);
  }
  return BDIS_OK;
}

}  // namespace

size_t match_scratch_bytes(int w, int h, int count, const bdis_params &p) {
  return plan_layout(w, h, count, p, false).bytes;
}

bdis_status check_match_args(const bdis_image *left, const bdis_image *right,
                             const bdis_params *p, const float *disparity_out) {
  if (!disparity_out) return BDIS_E_INVALID_ARG;
  bdis_status s = check_pair(left, right);
  if (s != BDIS_OK) return s;
  s = check_params(p);
  if (s != BDIS_OK) return s;
  return check_geometry(left->width, left->height, *p);
}

bdis_status check_match_pointers(const bdis_image *left, const bdis_image *right,
                                 const float *disparity_out) {
  if (check_device_ptr(left->data) != BDIS_OK || check_device_ptr(right->data) != BDIS_OK ||
      check_device_ptr(disparity_out) != BDIS_OK)
    return BDIS_E_INVALID_ARG;
  return BDIS_OK;
}

bdis_status run_match_in(void *scratch, size_t scratch_bytes, cudaStream_t stream,
                         const bdis_image &left, const bdis_image &right, const bdis_params &p,
                         float *out, const Tuning *tune, const Seed *seed) {
  bdis_handle view;  // borrows the caller's scratch; owns nothing, times nothing
  view.stream = stream;
  view.ws = scratch;
  view.ws_bytes = scratch_bytes;
  const Layout lay = plan_layout(left.width, left.height, left.count, p, false);
  if (lay.bytes > scratch_bytes) return BDIS_E_UNSUPPORTED;
  (void)0;
  bdis_status s = run_match(&view, left, right, p, out, lay, tune, seed);
  view.ws = nullptr;
  return s;
}

namespace {

// Mean milliseconds of `reps` back-to-back calls of fn on st, after one warm-up.
template <typename Fn>
float time_launches(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int reps, Fn fn,
                    cudaError_t *err) {
  cudaError_t e = fn();
  cudaEventRecord(e0, st);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = fn();
  cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  *err = e;
  return ms / reps;
}

}  // namespace

bdis_status autotune_match(void *scratch, size_t scratch_bytes, cudaStream_t st,
                           const bdis_image &left, const bdis_image &right,
                           const bdis_params &p, float *out, Tuning *tune) {
  *tune = Tuning{};
  // one full run fills every level's planes and the coarse maps the levels read
  bdis_status s = run_match_in(scratch, scratch_bytes, st, left, right, p, out, nullptr);
  if (s != BDIS_OK) return s;
  const Layout lay = plan_layout(left.width, left.height, left.count, p, false);
  char *base = static_cast<char *>(scratch);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const bool fixed = p.window_samples == 5 && p.window_step == 0.5f &&
                     (p.patch_size == 8 || p.patch_size == 12 || p.patch_size == 16);
  const int reps = 3;
  // lane layouts of the fixed-size kernels: 1 and the wide one (2, or 3 at
  // patch 12), and 4 columns per lane at patch 8
  const int cpls[3] = {1, 2, 4};
  const int n_cpl = !fixed ? 1 : (p.patch_size == 8 ? 3 : 2);
  for (int l = p.coarsest_scale; l >= p.finest_scale && e == cudaSuccess; --l) {
    // search: lane layout x block size x global or warp-tiled sampling
    float best = 1e30f;
    for (int ci = 0; ci < n_cpl && e == cudaSuccess; ++ci)
      for (int bt = 64; bt <= 128 && e == cudaSuccess; bt *= 2)
        for (int tiled = 0; tiled <= (fixed ? 1 : 0) && e == cudaSuccess; ++tiled) {
          SearchArgs sa = level_search_args(base, lay, p, left.count, l);
          sa.cols_per_lane = cpls[ci];
          sa.block_threads = bt;
          sa.tiled = tiled;
          const float ms =
              time_launches(st, e0, e1, reps, [&] { return launch_search(sa, st); }, &e);
          if (e == cudaSuccess && ms < best) {
            best = ms;
            tune->level[l].search_cpl = cpls[ci];
            tune->level[l].search_threads = bt;
            tune->level[l].search_tiled = tiled + 1;
          }
        }
    // densify (the separable BDIS kernels): 0 = the strip kernel where it
    // applies, else a tile height of 8, 16 or 32
    if (p.fusion == BDIS_FUSION_BDIS) {
      best = 1e30f;
      for (int ty = 0; ty <= 32 && e == cudaSuccess; ty = ty ? 2 * ty : 8) {
        DensifyArgs da = level_densify_args(base, lay, p, left.count, l, out);
        da.tile_y = ty;
        const float ms = time_launches(st, e0, e1, reps, [&] { return launch_densify(da, st); }, &e);
        if (e == cudaSuccess && ms < best) {
          best = ms;
          tune->level[l].densify_tile_y = ty;
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return record_cuda(e);
}

cudaError_t device_alloc(void **p, size_t bytes) {
  int n = g_alloc_failures.load();
  while (n > 0) {
    if (g_alloc_failures.compare_exchange_weak(n, n - 1)) return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

void set_last_error(const char *msg) { snprintf(g_last_error, sizeof g_last_error, "%s", msg); }

bdis_status record_cuda(cudaError_t e) {
  if (e == cudaSuccess) return BDIS_OK;
  snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e),
           cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BDIS_E_NOMEM : BDIS_E_CUDA;
}

bdis_status check_params(const bdis_params *p) {
  if (!p) return BDIS_E_INVALID_ARG;
  if (p->patch_size < 1 || !(p->overlap >= 0.f && p->overlap < 1.f) || p->iterations < 0 ||
      p->finest_scale < 0 || p->finest_scale > p->coarsest_scale || p->window_samples < 1 ||
      p->window_samples % 2 == 0 || !(p->sigma_r > 0.f) || !(p->sigma_s > 0.f) ||
      !(p->window_step >= 0.f) || !(p->gamma >= 0.f && p->gamma <= 1.f) ||
      (p->fusion != BDIS_FUSION_BDIS && p->fusion != BDIS_FUSION_DIS))
    return BDIS_E_INVALID_ARG;
  if (p->patch_size < 4 || p->patch_size > kMaxPatch || p->window_samples > kMaxWindow ||
      p->coarsest_scale > 15)
    return BDIS_E_UNSUPPORTED;
  return BDIS_OK;
}

}  // namespace bdis

using namespace bdis;

extern "C" {

void bdis_default_params(bdis_params *p) {
  if (!p) return;
  p->patch_size = 8;
  p->overlap = 0.75f;
  p->iterations = 12;
  p->coarsest_scale = 4;
  p->finest_scale = 0;
  p->sigma_r = 4.f;
  p->sigma_s = 4.f;
  p->window_samples = 5;
  p->window_step = 0.5f;
  p->gamma = 0.75f;
  p->normalize = 1;
  p->fusion = BDIS_FUSION_BDIS;
}

const char *bdis_status_string(bdis_status s) {
  switch (s) {
    case BDIS_OK: return "ok";
    case BDIS_E_INVALID_ARG: return "invalid argument";
    case BDIS_E_NOMEM: return "out of memory";
    case BDIS_E_CUDA: return "CUDA error";
    case BDIS_E_TIMEOUT: return "timeout";
    case BDIS_E_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *bdis_last_error_string(void) { return g_last_error; }

int bdis_version(void) { return (1 << 16) | 0; }

bdis_status bdis_level_dims(int width, int height, int level, int *lw, int *lh) {
  if (width < 1 || height < 1 || level < 0 || level > 30 || !lw || !lh) return BDIS_E_INVALID_ARG;
  *lw = level_dim(width, level);
  *lh = level_dim(height, level);
  return BDIS_OK;
}

bdis_status bdis_grid(int n, int patch_size, float overlap, int *stride, int *count) {
  if (n < 1 || patch_size < 1 || !(overlap >= 0.f && overlap < 1.f) || !stride || !count)
    return BDIS_E_INVALID_ARG;
  *stride = grid_stride(patch_size, overlap);
  *count = grid_count(n, patch_size, *stride);
  return BDIS_OK;
}

bdis_status bdis_patch_count(int width, int height, const bdis_params *p, int64_t *total) {
  bdis_status s = check_params(p);
  if (s != BDIS_OK) return s;
  if (!total || width < 1 || height < 1) return BDIS_E_INVALID_ARG;
  s = check_geometry(width, height, *p);
  if (s != BDIS_OK) return s;
  const int stride = grid_stride(p->patch_size, p->overlap);
  int64_t t = 0;
  for (int l = p->finest_scale; l <= p->coarsest_scale; ++l)
    t += (int64_t)grid_count(level_dim(width, l), p->patch_size, stride) *
         grid_count(level_dim(height, l), p->patch_size, stride);
  *total = t;
  return BDIS_OK;
}

bdis_status bdis_create(bdis_handle **out, int device, void *stream) {
  if (!out) return BDIS_E_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess) return record_cuda(e);
  if (device < 0 || device >= n) return BDIS_E_INVALID_ARG;
  bdis_handle *h = new (std::nothrow) bdis_handle();
  if (!h) return BDIS_E_NOMEM;
  h->device = device;
  h->stream = static_cast<cudaStream_t>(stream);
  *out = h;
  return BDIS_OK;
}

bdis_status bdis_reserve(bdis_handle *h, int width, int height, int count, const bdis_params *p) {
  if (!h || width < 1 || height < 1 || count < 1) return BDIS_E_INVALID_ARG;
  bdis_status s = check_params(p);
  if (s != BDIS_OK) return s;
  s = check_geometry(width, height, *p);
  if (s != BDIS_OK) return s;
  s = bind_device(h);
  if (s != BDIS_OK) return s;
  return ensure_workspace(h, plan_layout(width, height, count, *p, false).bytes);
}

size_t bdis_workspace_bytes(const bdis_handle *h) { return h ? h->ws_bytes : 0; }

void bdis_destroy(bdis_handle *h) {
  if (!h) return;
  if (bind_device(h) == BDIS_OK) {
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    for (auto &m : h->marks) {
      cudaEventDestroy(m.start);
      cudaEventDestroy(m.stop);
    }
    for (auto e : h->event_pool) cudaEventDestroy(e);
    if (h->copy_in) {
      cudaStreamSynchronize(h->copy_in);
      cudaStreamSynchronize(h->copy_out);
      cudaStreamDestroy(h->copy_in);
      cudaStreamDestroy(h->copy_out);
      for (int i = 0; i < kAsyncSlots; ++i) {
        cudaEventDestroy(h->ev_in[i]);
        cudaEventDestroy(h->ev_done[i]);
        cudaEventDestroy(h->ev_out[i]);
      }
    }
  }
  delete h;
}

bdis_status bdis_set_search_variant(int columns_per_lane) {
  if (columns_per_lane != 1 && columns_per_lane != 2 && columns_per_lane != 4)
    return BDIS_E_INVALID_ARG;
  set_search_cols_per_lane(columns_per_lane);
  return BDIS_OK;
}

int bdis_get_search_variant(void) { return search_cols_per_lane(); }

void bdis_set_search_tiling(int on) { set_search_tiled(on); }

int bdis_get_search_tiling(void) { return search_tiled(); }

bdis_status bdis_set_densify_variant(int tile_height) {
  if (tile_height != 0 && tile_height != 8 && tile_height != 16 && tile_height != 32)
    return BDIS_E_INVALID_ARG;
  set_densify_tile(tile_height);
  return BDIS_OK;
}

int bdis_get_densify_variant(void) { return densify_tile(); }

void bdis_set_pyramid_variant(int variant) { set_pyramid_fused(variant); }

int bdis_get_pyramid_variant(void) { return pyramid_fused(); }

bdis_status bdis_check_status(uint32_t *sites) {
  if (!sites) return BDIS_E_INVALID_ARG;
  unsigned s = 0u, d = 0u, p = 0u;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = take_check_search(&s);
  if (e == cudaSuccess) e = take_check_densify(&d);
  if (e == cudaSuccess) e = take_check_pyramid(&p);
  if (e != cudaSuccess) return record_cuda(e);
  *sites = s | d | p;
  return BDIS_OK;
}

int bdis_checked_build(void) {
#ifdef BDIS_CHECKED
  return 1;
#else
  return 0;
#endif
}

void bdis_set_launch_overlap(int on) { set_launch_overlap(on); }

int bdis_get_launch_overlap(void) { return launch_overlap(); }

bdis_status bdis_enable_timing(bdis_handle *h, int on) {
  if (!h) return BDIS_E_INVALID_ARG;
  h->timing = on != 0;
  return BDIS_OK;
}

bdis_status bdis_read_timing(bdis_handle *h, bdis_timing *out) {
  if (!h || !out) return BDIS_E_INVALID_ARG;
  bdis_status s = bind_device(h);
  if (s != BDIS_OK) return s;
  for (int c = 0; c < BDIS_TIMING_CLASSES; ++c) {
    out->ms[c] = 0.0;
    out->launches[c] = 0;
  }
  cudaError_t err = cudaSuccess;
  for (auto &m : h->marks) {
    cudaError_t e = cudaEventSynchronize(m.stop);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, m.start, m.stop);
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    if (m.cls >= 0 && m.cls < BDIS_TIMING_CLASSES) {
      out->ms[m.cls] += ms;
      out->launches[m.cls] += 1;
    }
    h->event_pool.push_back(m.start);
    h->event_pool.push_back(m.stop);
  }
  h->marks.clear();
  return record_cuda(err);
}

bdis_status bdis_match(bdis_handle *h, const bdis_image *left, const bdis_image *right,
                       const bdis_params *p, float *disparity_out) {
  if (!h || !disparity_out) return BDIS_E_INVALID_ARG;
  bdis_status s = check_pair(left, right);
  if (s != BDIS_OK) return s;
  s = check_params(p);
  if (s != BDIS_OK) return s;
  s = check_geometry(left->width, left->height, *p);
  if (s != BDIS_OK) return s;
  s = bind_device(h);
  if (s != BDIS_OK) return s;
  if (check_device_ptr(left->data) != BDIS_OK || check_device_ptr(right->data) != BDIS_OK ||
      check_device_ptr(disparity_out) != BDIS_OK)
    return BDIS_E_INVALID_ARG;
  const Layout lay = plan_layout(left->width, left->height, left->count, *p, false);
  s = ensure_workspace(h, lay.bytes);
  if (s != BDIS_OK) return s;
  return run_match(h, *left, *right, *p, disparity_out, lay);
}

static bdis_status match_with_seed(bdis_handle *h, const bdis_image *left,
                                   const bdis_image *right, const bdis_params *p,
                                   const Seed &seed, float *disparity_out) {
  if (!h || !disparity_out) return BDIS_E_INVALID_ARG;
  bdis_status s = check_pair(left, right);
  if (s != BDIS_OK) return s;
  s = check_params(p);
  if (s != BDIS_OK) return s;
  s = check_geometry(left->width, left->height, *p);
  if (s != BDIS_OK) return s;
  if ((seed.map || seed.net) && (seed.level < 0 || seed.level > p->coarsest_scale))
    return BDIS_E_INVALID_ARG;
  s = bind_device(h);
  if (s != BDIS_OK) return s;
  if (check_device_ptr(left->data) != BDIS_OK || check_device_ptr(right->data) != BDIS_OK ||
      check_device_ptr(disparity_out) != BDIS_OK ||
      (seed.map && check_device_ptr(seed.map) != BDIS_OK))
    return BDIS_E_INVALID_ARG;
  const Layout lay = plan_layout(left->width, left->height, left->count, *p, false);
  if (seed.net && seed.level != lay.prop_level) return BDIS_E_UNSUPPORTED;
  s = ensure_workspace(h, lay.bytes);
  if (s != BDIS_OK) return s;
  return run_match(h, *left, *right, *p, disparity_out, lay, nullptr, &seed);
}

bdis_status bdis_match_warm(bdis_handle *h, const bdis_image *left, const bdis_image *right,
                            const bdis_params *p, const float *prev, float *disparity_out) {
  Seed seed;
  seed.map = prev;
  seed.level = 0;
  return match_with_seed(h, left, right, p, seed, disparity_out);
}

bdis_status bdis_match_seeded(bdis_handle *h, const bdis_image *left, const bdis_image *right,
                              const bdis_params *p, const float *seed_map, int seed_level,
                              int fallback, float *disparity_out) {
  if (!seed_map) return BDIS_E_INVALID_ARG;
  Seed seed;
  seed.map = seed_map;
  seed.level = seed_level;
  seed.fallback = fallback ? 1 : 0;
  return match_with_seed(h, left, right, p, seed, disparity_out);
}

bdis_status bdis_match_learned(bdis_handle *h, bdis_net *net, const bdis_image *left,
                               const bdis_image *right, const bdis_params *p, int fallback,
                               float *disparity_out) {
  if (!net || !p) return BDIS_E_INVALID_ARG;
  Seed seed;
  seed.net = net;
  seed.level = proposal_level(p->coarsest_scale);
  seed.fallback = fallback ? 1 : 0;
  return match_with_seed(h, left, right, p, seed, disparity_out);
}

int bdis_proposal_level(int coarsest_scale) {
  return coarsest_scale < 0 ? -1 : proposal_level(coarsest_scale);
}

bdis_status bdis_warm_map(const float *prev, int width, int height, int level, int count,
                          float *out, void *stream) {
  if (!prev || !out || width < 1 || height < 1 || level < 1 || level > 16 || count < 1)
    return BDIS_E_INVALID_ARG;
  return record_cuda(launch_warm_map(prev, width, height, level, count, out,
                                     static_cast<cudaStream_t>(stream)));
}

namespace {

// Copy streams and events of the host pipeline, created on first use.
bdis_status ensure_pipeline(bdis_handle *h) {
  if (h->copy_in) return BDIS_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking);
  for (int i = 0; i < kAsyncSlots && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->ev_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[i], cudaEventDisableTiming);
  }
  return record_cuda(e);
}

}  // namespace

bdis_status bdis_match_host(bdis_handle *h, const uint8_t *left, const uint8_t *right, int width,
                            int height, int count, const bdis_params *p, float *disparity_out) {
  if (!h || !left || !right || !disparity_out || width < 1 || height < 1 || count < 1)
    return BDIS_E_INVALID_ARG;
  bdis_status s = check_params(p);
  if (s != BDIS_OK) return s;
  s = check_geometry(width, height, *p);
  if (s != BDIS_OK) return s;
  s = bind_device(h);
  if (s != BDIS_OK) return s;
  const size_t wh = (size_t)width * height;
  // The batch runs as chunks: chunk i's inputs are copied in (copy_in) while
  // chunk i-1 is matched (stream) and chunk i-2's result is copied out
  // (copy_out). Inputs and outputs on the device are double-buffered by slot
  // (i & 1); a slot is refilled only after the match that read it (ev_done)
  // and the copy-out that read its output (ev_out) have finished. From 32
  // pairs the first and last chunks are a sixteenth of the batch, so that
  // the copy-in before the first match and the copy-out after the last one
  // (the only copies nothing hides) are short; three equal chunks between.
  int chunk_first[5], chunk_n[5], nchunk;
  if (count >= 32) {
    const int edge = count / 16, mid = count - 2 * edge;
    nchunk = 5;
    chunk_n[0] = chunk_n[4] = edge;
    chunk_n[1] = chunk_n[2] = mid / 3;
    chunk_n[3] = mid - 2 * (mid / 3);
  } else {
    nchunk = count >= 8 ? 4 : (count >= 2 ? 2 : 1);
    const int c = (count + nchunk - 1) / nchunk;
    for (int i = 0; i < nchunk; ++i) chunk_n[i] = std::max(0, std::min(c, count - i * c));
  }
  int cs = 0;
  for (int i = 0, f = 0; i < nchunk; ++i) {
    chunk_first[i] = f;
    f += chunk_n[i];
    cs = std::max(cs, chunk_n[i]);
  }
  const Layout lay = plan_layout(width, height, cs, *p, true);
  const size_t in_b = wh * cs, out_b = wh * cs * sizeof(float);
  size_t off = lay.bytes;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += (n + 255) / 256 * 256;
    return o;
  };
  const size_t slot_l[2] = {lay.in_left, nchunk > 1 ? take(in_b) : 0};
  const size_t slot_r[2] = {lay.in_right, nchunk > 1 ? take(in_b) : 0};
  const size_t slot_o[2] = {lay.out, nchunk > 1 ? take(out_b) : 0};
  s = ensure_workspace(h, off);
  if (s != BDIS_OK) return s;
  if (nchunk > 1) {
    s = ensure_pipeline(h);
    if (s != BDIS_OK) return s;
  }
  char *base = static_cast<char *>(h->ws);
  cudaStream_t sin = nchunk > 1 ? h->copy_in : h->stream;
  cudaStream_t sout = nchunk > 1 ? h->copy_out : h->stream;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < nchunk && e == cudaSuccess; ++i) {
    const int first = chunk_first[i], n = chunk_n[i];
    if (n <= 0) break;
    const int slot = i & 1;
    const size_t ib = wh * n;
    if (nchunk > 1 && i >= 2) e = cudaStreamWaitEvent(sin, h->ev_done[slot], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + slot_l[slot], left + wh * first, ib, cudaMemcpyHostToDevice, sin);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + slot_r[slot], right + wh * first, ib, cudaMemcpyHostToDevice,
                          sin);
    if (nchunk > 1) {
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[slot], sin);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_in[slot], 0);
      if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(h->stream, h->ev_out[slot], 0);
    }
    if (e != cudaSuccess) break;
    bdis_image L{base + slot_l[slot], width, height, (size_t)width, wh, n, BDIS_U8};
    bdis_image R = L;
    R.data = base + slot_r[slot];
    float *dout = reinterpret_cast<float *>(base + slot_o[slot]);
    s = run_match(h, L, R, *p, dout, lay);
    if (s != BDIS_OK) break;
    if (nchunk > 1) {
      e = cudaEventRecord(h->ev_done[slot], h->stream);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, h->ev_done[slot], 0);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(disparity_out + wh * first, dout, ib * sizeof(float),
                          cudaMemcpyDeviceToHost, sout);
    if (e == cudaSuccess && nchunk > 1) e = cudaEventRecord(h->ev_out[slot], sout);
  }
  // leave every stream idle: the next call may resize or reuse the workspace
  cudaError_t e2 = cudaStreamSynchronize(h->stream);
  if (nchunk > 1) {
    cudaError_t e3 = cudaStreamSynchronize(h->copy_in);
    cudaError_t e4 = cudaStreamSynchronize(h->copy_out);
    if (e2 == cudaSuccess) e2 = e3 != cudaSuccess ? e3 : e4;
  }
  if (s != BDIS_OK) return s;
  if (e == cudaSuccess) e = e2;
  return record_cuda(e);
}

bdis_status bdis_match_host_async(bdis_handle *h, const uint8_t *left, const uint8_t *right,
                                  int width, int height, int count, const bdis_params *p,
                                  float *disparity_out, uint64_t *ticket) {
  if (!h || !left || !right || !disparity_out || !ticket || width < 1 || height < 1 ||
      count < 1)
    return BDIS_E_INVALID_ARG;
  bdis_status s = check_params(p);
  if (s != BDIS_OK) return s;
  s = check_geometry(width, height, *p);
  if (s != BDIS_OK) return s;
  s = bind_device(h);
  if (s != BDIS_OK) return s;
  s = ensure_pipeline(h);
  if (s != BDIS_OK) return s;
  // One whole batch per call, its device inputs and output in slot
  // (ticket % kAsyncSlots): the copy-in of this call overlaps the matches
  // before it, and its copy-out the matches after it. A slot is refilled only
  // after the match that read its inputs (ev_done) and the copy-out that read
  // its output (ev_out) of the call kAsyncSlots before have finished, so a
  // copy that runs late holds up the matches only once all slots are taken.
  const size_t wh = (size_t)width * height;
  const Layout lay = plan_layout(width, height, count, *p, true);
  const size_t in_b = wh * count, out_b = wh * count * sizeof(float);
  size_t off = lay.bytes;
  auto take = [&](size_t n) {
    const size_t o = off;
    off += (n + 255) / 256 * 256;
    return o;
  };
  size_t slot_l[kAsyncSlots], slot_r[kAsyncSlots], slot_o[kAsyncSlots];
  slot_l[0] = lay.in_left;
  slot_r[0] = lay.in_right;
  slot_o[0] = lay.out;
  for (int i = 1; i < kAsyncSlots; ++i) {
    slot_l[i] = take(in_b);
    slot_r[i] = take(in_b);
    slot_o[i] = take(out_b);
  }
  size_t key[1 + 3 * kAsyncSlots] = {off};
  for (int i = 0; i < kAsyncSlots; ++i) {
    key[1 + 3 * i] = slot_l[i];
    key[2 + 3 * i] = slot_r[i];
    key[3 + 3 * i] = slot_o[i];
  }
  static_assert(sizeof key == sizeof(((bdis_handle *)nullptr)->async_key), "key size");
  if (h->async_pending && memcmp(key, h->async_key, sizeof key) != 0) {
    cudaError_t e = drain_async(h);  // calls in flight use another layout
    if (e != cudaSuccess) return record_cuda(e);
  }
  s = ensure_workspace(h, off, true);
  if (s != BDIS_OK) return s;
  memcpy(h->async_key, key, sizeof key);
  const uint64_t t = h->async_next;
  const int slot = (int)(t % kAsyncSlots);
  char *base = static_cast<char *>(h->ws);
  cudaError_t e = cudaStreamWaitEvent(h->copy_in, h->ev_done[slot], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + slot_l[slot], left, in_b, cudaMemcpyHostToDevice, h->copy_in);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + slot_r[slot], right, in_b, cudaMemcpyHostToDevice, h->copy_in);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_in[slot], h->copy_in);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_in[slot], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->ev_out[slot], 0);
  if (e != cudaSuccess) return record_cuda(e);
  h->async_pending += 1;  // work is on the streams from here on
  bdis_image L{base + slot_l[slot], width, height, (size_t)width, wh, count, BDIS_U8};
  bdis_image R = L;
  R.data = base + slot_r[slot];
  float *dout = reinterpret_cast<float *>(base + slot_o[slot]);
  s = run_match(h, L, R, *p, dout, lay);
  if (s != BDIS_OK) return s;
  e = cudaEventRecord(h->ev_done[slot], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy_out, h->ev_done[slot], 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(disparity_out, dout, out_b, cudaMemcpyDeviceToHost, h->copy_out);
  if (e == cudaSuccess) e = cudaEventRecord(h->ev_out[slot], h->copy_out);
  if (e != cudaSuccess) return record_cuda(e);
  h->async_next = t + 1;
  *ticket = t;
  return BDIS_OK;
}

bdis_status bdis_host_wait(bdis_handle *h, uint64_t ticket) {
  if (!h || ticket == 0 || ticket >= h->async_next) return BDIS_E_INVALID_ARG;
  bdis_status s = bind_device(h);
  if (s != BDIS_OK) return s;
  if (!h->async_pending) return BDIS_OK;  // drained since (by a later call or wait)
  // The slot's copy-out event was recorded by this call or by a later one on
  // the same in-order stream: once it has completed, so has this call.
  cudaError_t e = cudaEventSynchronize(h->ev_out[ticket % kAsyncSlots]);
  if (e == cudaSuccess && ticket + 1 == h->async_next) e = drain_async(h);
  return record_cuda(e);
}

bdis_status bdis_host_wait_timeout(bdis_handle *h, uint64_t ticket, double timeout_ms) {
  if (!h || ticket == 0 || ticket >= h->async_next || !(timeout_ms >= 0.0))
    return BDIS_E_INVALID_ARG;
  bdis_status s = bind_device(h);
  if (s != BDIS_OK) return s;
  if (!h->async_pending) return BDIS_OK;
  // poll the slot's copy-out event (see bdis_host_wait) against a host deadline
  const auto deadline = std::chrono::steady_clock::now() +
                        std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                            std::chrono::duration<double, std::milli>(timeout_ms));
  while (true) {
    cudaError_t e = cudaEventQuery(h->ev_out[ticket % kAsyncSlots]);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) return record_cuda(e);
    cudaGetLastError();  // not-ready is not an error
    if (std::chrono::steady_clock::now() >= deadline) {
      set_last_error("bdis_host_wait_timeout: the call's result is not ready yet");
      return BDIS_E_TIMEOUT;
    }
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  if (ticket + 1 == h->async_next) return record_cuda(drain_async(h));
  return BDIS_OK;
}

void bdis_inject_alloc_failures(int count) { g_alloc_failures.store(count > 0 ? count : 0); }

static bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }

bdis_status bdis_prepare_level0(const bdis_image *left, const bdis_image *right, float *L0,
                                float *R0, float *G0, void *stream) {
  bdis_status s = check_pair(left, right);
  if (s != BDIS_OK) return s;
  if (!L0 || !R0 || !G0 || !aligned8(R0) || left->width < 2 || left->height < 2)
    return BDIS_E_INVALID_ARG;
  return record_cuda(launch_prepare_level0(*left, *right, L0, reinterpret_cast<float2 *>(R0), G0,
                                           static_cast<cudaStream_t>(stream)));
}

bdis_status bdis_pyramid_level(const float *L, const float *R, int width, int height, int count,
                               float *L1, float *R1, float *G1, void *stream) {
  if (!L || !R || !L1 || !R1 || !G1 || !aligned8(R) || !aligned8(R1) || width < 3 ||
      height < 3 || count < 1)
    return BDIS_E_INVALID_ARG;
  return record_cuda(launch_pyramid_level(L, reinterpret_cast<const float2 *>(R), width, height,
                                          count, L1, reinterpret_cast<float2 *>(R1), G1,
                                          static_cast<cudaStream_t>(stream)));
}

bdis_status bdis_pack_right(const float *R, int width, int height, int count, float *R2,
                            void *stream) {
  if (!R || !R2 || !aligned8(R2) || width < 1 || height < 1 || count < 1)
    return BDIS_E_INVALID_ARG;
  return record_cuda(launch_pack_right(R, width, height, count, reinterpret_cast<float2 *>(R2),
                                       static_cast<cudaStream_t>(stream)));
}

bdis_status bdis_search_level(const float *L, const float *R, const float *G, int width,
                              int height, int count, const float *coarse, int coarse_width,
                              int coarse_height, const bdis_params *p, float *d_star,
                              float *weight, const bdis_patch_debug *dbg, void *stream) {
  bdis_status s = check_params(p);
  if (s != BDIS_OK) return s;
  if (!L || !R || !G || !d_star || !weight || !aligned8(R) || count < 1 ||
      width < p->patch_size || height < p->patch_size)
    return BDIS_E_INVALID_ARG;
  if (coarse && (coarse_width < 1 || coarse_height < 1)) return BDIS_E_INVALID_ARG;
  SearchArgs a{};
  fill_search_args(a, width, height, count, *p);
  a.L = L;
  a.R2 = reinterpret_cast<const float2 *>(R);
  a.G = G;
  a.coarse = coarse;
  a.cw = coarse ? coarse_width : 0;
  a.ch = coarse ? coarse_height : 0;
  a.cplane = (long long)a.cw * a.ch;
  a.d_star = d_star;
  a.weight = weight;
  if (dbg) {
    a.u_init = dbg->u_init;
    a.posterior = dbg->posterior;
    a.energies = dbg->energies;
    a.flags = dbg->flags;
    a.n_valid = dbg->n_valid;
    a.steps = dbg->steps;
  }
  return record_cuda(launch_search(a, static_cast<cudaStream_t>(stream)));
}

bdis_status bdis_densify_level(int width, int height, int count, const bdis_params *p,
                               const float *d_star, const float *weight, const float *coarse,
                               int coarse_width, int coarse_height, int is_finest,
                               const float *L, const float *R, float *out, void *stream) {
  bdis_status s = check_params(p);
  if (s != BDIS_OK) return s;
  if (!d_star || !weight || !out || count < 1 || width < p->patch_size ||
      height < p->patch_size)
    return BDIS_E_INVALID_ARG;
  if (p->fusion == BDIS_FUSION_DIS && (!L || !R || !aligned8(R))) return BDIS_E_INVALID_ARG;
  if (coarse && (coarse_width < 1 || coarse_height < 1)) return BDIS_E_INVALID_ARG;
  DensifyArgs a{};
  fill_densify_args(a, width, height, count, *p);
  a.d_star = d_star;
  a.weight = weight;
  a.coarse = coarse;
  a.cw = coarse ? coarse_width : 0;
  a.ch = coarse ? coarse_height : 0;
  a.cplane = (long long)a.cw * a.ch;
  a.is_finest = is_finest ? 1 : 0;
  a.L = L;
  a.R2 = reinterpret_cast<const float2 *>(R);
  a.out = out;
  return record_cuda(launch_densify(a, static_cast<cudaStream_t>(stream)));
}

bdis_status bdis_select_start(float *d_star_a, float *weight_a, const float *posterior_a,
                              const uint8_t *flags_a, const float *d_star_b,
                              const float *weight_b, const float *posterior_b,
                              const uint8_t *flags_b, int64_t total, void *stream) {
  if (!d_star_a || !weight_a || !posterior_a || !flags_a || !d_star_b || !weight_b ||
      !posterior_b || !flags_b || total < 0)
    return BDIS_E_INVALID_ARG;
  return record_cuda(launch_select_start(d_star_a, weight_a, posterior_a, flags_a, d_star_b,
                                         weight_b, posterior_b, flags_b, (long long)total,
                                         static_cast<cudaStream_t>(stream)));
}

bdis_status bdis_upsample(const float *map, int map_width, int map_height, int level, int width,
                          int height, int count, float *out, void *stream) {
  if (!map || !out || map_width < 1 || map_height < 1 || level < 0 || level > 15 || width < 1 ||
      height < 1 || count < 1)
    return BDIS_E_INVALID_ARG;
  return record_cuda(launch_upsample(map, map_width, map_height, level, width, height, count, out,
                                     static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
