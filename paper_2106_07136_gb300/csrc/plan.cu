// plan.cu -- mixed-resolution batches as one CUDA graph, with autotuned launches.
//
// A plan fixes a set of groups, each a batch of equally sized pairs (for
// example 64 pairs at 320x240, 96 at 640x480, 64 at 1280x720, 32 at
// 1920x1080). Every group gets its own workspace so that the groups can run
// concurrently; the whole launch sequence (19 launches per group at 5
// scales) is captured once into a CUDA graph whose groups are independent
// branches, and each run is a single graph launch. Before capture the
// autotuner times, per group and level, the candidate lane layouts, block
// sizes and sampling (global or warp-tiled) of the search kernel and the
// densify kernels on the group's own data, and keeps the fastest.
#include <new>
#include <vector>

#include "bdis_internal.cuh"

struct bdis_plan {
  int device = 0;
  bdis_params params{};
  struct Group {
    bdis_params params{};  // the plan's, with the coarsest scale raised per group if asked
    bdis_image left{}, right{};
    float *out = nullptr;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bdis::Tuning tune{};
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
  };
  std::vector<Group> groups;
  cudaStream_t capture = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  size_t bytes = 0;
};

namespace {

void release(bdis_plan *pl) {
  if (!pl) return;
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  for (auto &g : pl->groups) {
    if (g.stream) cudaStreamSynchronize(g.stream);
    if (g.ws) cudaFree(g.ws);
    if (g.done) cudaEventDestroy(g.done);
    if (g.stream) cudaStreamDestroy(g.stream);
  }
  if (pl->fork) cudaEventDestroy(pl->fork);
  if (pl->capture) cudaStreamDestroy(pl->capture);
  delete pl;
}

// The smallest coarsest scale c at which a disparity range of a tenth of the
// width is at most 4 px at the coarsest level (2^c >= W / 40), never below
// the plan's own and lowered until the coarsest level still holds a patch.
int scaled_coarsest(const bdis_params &p, int w, int h) {
  int c = p.coarsest_scale;
  while (c < 15 && (40LL << c) < (long long)w) ++c;
  while (c > p.coarsest_scale &&
         (bdis::level_dim(w, c) < p.patch_size || bdis::level_dim(h, c) < p.patch_size))
    --c;
  return c;
}

}  // namespace

extern "C" {

bdis_status bdis_plan_create(int device, const bdis_group *groups, int n_groups,
                             const bdis_params *p, int flags, void *stream, bdis_plan **out) {
  if (!out || !groups || n_groups < 1 || n_groups > 64) return BDIS_E_INVALID_ARG;
  *out = nullptr;
  bdis_status s = bdis::check_params(p);
  if (s != BDIS_OK) return s;
  for (int i = 0; i < n_groups; ++i) {
    s = bdis::check_match_args(&groups[i].left, &groups[i].right, p, groups[i].disparity_out);
    if (s != BDIS_OK) return s;
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  if (device < 0 || device >= ndev) return BDIS_E_INVALID_ARG;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  for (int i = 0; i < n_groups; ++i) {
    s = bdis::check_match_pointers(&groups[i].left, &groups[i].right, groups[i].disparity_out);
    if (s != BDIS_OK) return s;
  }
  bdis_plan *pl = new (std::nothrow) bdis_plan();
  if (!pl) return BDIS_E_NOMEM;
  pl->device = device;
  pl->params = *p;
  pl->groups.resize(n_groups);
  cudaStream_t user = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < n_groups && e == cudaSuccess; ++i) {
    auto &g = pl->groups[i];
    g.params = *p;
    if (flags & BDIS_PLAN_SCALE_TO_WIDTH)
      g.params.coarsest_scale = scaled_coarsest(*p, groups[i].left.width, groups[i].left.height);
    g.left = groups[i].left;
    g.right = groups[i].right;
    g.out = groups[i].disparity_out;
    g.ws_bytes = bdis::match_scratch_bytes(g.left.width, g.left.height, g.left.count, g.params);
    e = bdis::device_alloc(&g.ws, g.ws_bytes);
    if (e != cudaSuccess) {
      g.ws = nullptr;
      cudaGetLastError();
      release(pl);
      return BDIS_E_NOMEM;
    }
    pl->bytes += g.ws_bytes;
    e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->capture, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    release(pl);
    return bdis::record_cuda(e);
  }
  // autotune each group on its own data (before capture: it times launches)
  if (flags & BDIS_PLAN_AUTOTUNE) {
    if (user) e = cudaStreamSynchronize(user);  // the inputs may still be written there
    for (auto &g : pl->groups) {
      if (e != cudaSuccess) break;
      s = bdis::autotune_match(g.ws, g.ws_bytes, g.stream, g.left, g.right, g.params, g.out,
                               &g.tune);
      if (s != BDIS_OK) {
        release(pl);
        return s;
      }
    }
    for (auto &g : pl->groups)
      if (e == cudaSuccess) e = cudaStreamSynchronize(g.stream);
    if (e != cudaSuccess) {
      release(pl);
      return bdis::record_cuda(e);
    }
  }
  // capture: fork from the capture stream into one branch per group, join back
  e = cudaStreamBeginCapture(pl->capture, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(pl->fork, pl->capture);
  bdis_status run_status = BDIS_OK;
  for (auto &g : pl->groups) {
    if (e != cudaSuccess || run_status != BDIS_OK) break;
    e = cudaStreamWaitEvent(g.stream, pl->fork, 0);
    if (e == cudaSuccess)
      run_status = bdis::run_match_in(g.ws, g.ws_bytes, g.stream, g.left, g.right, g.params,
                                      g.out, (flags & BDIS_PLAN_AUTOTUNE) ? &g.tune : nullptr);
    if (e == cudaSuccess && run_status == BDIS_OK) e = cudaEventRecord(g.done, g.stream);
    if (e == cudaSuccess && run_status == BDIS_OK) e = cudaStreamWaitEvent(pl->capture, g.done, 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(pl->capture, &graph);
  if (e == cudaSuccess) e = ee;
  pl->graph = graph;
  if (e == cudaSuccess && run_status == BDIS_OK)
    e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
  if (e != cudaSuccess || run_status != BDIS_OK) {
    cudaGetLastError();
    release(pl);
    return run_status != BDIS_OK ? run_status : bdis::record_cuda(e);
  }
  *out = pl;
  return BDIS_OK;
}

bdis_status bdis_plan_run(bdis_plan *pl, void *stream) {
  if (!pl || !pl->exec) return BDIS_E_INVALID_ARG;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != pl->device) e = cudaSetDevice(pl->device);
  if (e == cudaSuccess) e = cudaGraphLaunch(pl->exec, static_cast<cudaStream_t>(stream));
  return bdis::record_cuda(e);
}

bdis_status bdis_plan_info(const bdis_plan *pl, int group, int level, bdis_plan_choice *out) {
  if (!pl || !out || group < 0 || group >= (int)pl->groups.size() || level < 0 || level > 15)
    return BDIS_E_INVALID_ARG;
  const auto &t = pl->groups[group].tune.level[level];
  out->search_columns_per_lane = t.search_cpl;
  out->search_block_threads = t.search_threads;
  out->search_tiling = t.search_tiled ? t.search_tiled - 1 : bdis::search_tiled();
  out->densify_tile_height = t.densify_tile_y;
  out->workspace_bytes = pl->groups[group].ws_bytes;
  out->coarsest_scale = pl->groups[group].params.coarsest_scale;
  return BDIS_OK;
}

size_t bdis_plan_workspace_bytes(const bdis_plan *pl) { return pl ? pl->bytes : 0; }

void bdis_plan_destroy(bdis_plan *pl) {
  if (!pl) return;
  cudaSetDevice(pl->device);
  release(pl);
}

}  // extern "C"
