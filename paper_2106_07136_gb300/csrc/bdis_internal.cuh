// bdis_internal.cuh -- shared declarations of the BDIS CUDA library.
//
// The library is the GB300 (sm_103a) implementation of Bayesian Dense Inverse
// Search (arXiv 2106.07136). Kernels live in pyramid.cu (Sec. 2.1 pyramid and
// template gradient), search.cu (Eq. 1 inverse search with the Eqs. 3-4
// posterior) and densify.cu (Sec. 2.3 Gaussian-mask fusion); bdis.cu holds the
// C ABI, parameter checks, the workspace and the coarse-to-fine driver.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <utility>

#include "bdis.h"

namespace bdis {

// Saddle tolerance: a patch is dropped when another window sample beats the
// centre by more than this fraction of max(E_centre, 1) (Sec. 2.2 filter).
constexpr float kSaddleTau = 1e-6f;
// A patch is flat (no update) when its Hessian is at most this much per pixel.
constexpr float kFlatEps = 1e-4f;
// Largest final update (px) of a patch that counts as converged; patches whose
// last step is larger are dropped (Sec. 3.2 discards non-converged patches).
constexpr float kConvergeTol = 0.02f;
// A patch whose update falls below this (px) has converged and stops stepping
// (the step count is a maximum); a warp leaves the loop when all its patches have.
constexpr float kStepTol = 1e-4f;
// R16: seeded and plain results of one patch this close (px) are one solution
constexpr float kSameSolution = 0.1f;
// Pyramid level the proposal network of the learned start runs on (at most
// the coarsest level). Its map seeds the coarsest searched level L through
// block means at level L + 1 (R16), so a level near L loses nothing.
constexpr int kProposalLevel = 4;
__host__ __device__ inline int proposal_level(int coarsest) {
  return coarsest < kProposalLevel ? coarsest : kProposalLevel;
}
// Largest window the search kernel keeps track of.
constexpr int kMaxWindow = 15;
// Largest patch side (one patch per group of at most 32 lanes).
constexpr int kMaxPatch = 32;

constexpr uint8_t kFlagFlat = 1, kFlagDiverged = 2, kFlagSaddle = 4, kFlagGamma = 8,
                  kFlagEmpty = 16, kFlagUnconverged = 32;
constexpr uint8_t kDropFlags =
    kFlagDiverged | kFlagSaddle | kFlagGamma | kFlagEmpty | kFlagUnconverged;

__host__ __device__ inline int level_dim(int n, int level) {
  for (int l = 0; l < level; ++l) n = (n + 1) / 2;
  return n;
}

// Stride from size and overlap, rounded in double so that the host and any
// caller that computes in double agree on every representable overlap.
inline int grid_stride(int ps, float overlap) {
  double s = ps * (1.0 - (double)overlap) + 0.5;
  int si = (int)s;
  if ((double)si > s) --si;  // floor for positive values
  return si < 1 ? 1 : si;
}

inline int grid_count(int n, int ps, int stride) {
  if (n < ps) return 0;
  return (n - ps + stride - 1) / stride + 1;
}

__host__ __device__ __forceinline__ int grid_origin(int i, int count, int n, int ps, int stride) {
  return (i == count - 1) ? n - ps : i * stride;
}

// Smallest valid-pixel count that passes the gamma test, decided in double.
inline int gamma_min_count(float gamma, int ps) {
  const double need = (double)gamma * (double)(ps * ps);
  int n = 0;
  while (n <= ps * ps && (double)n < need) ++n;
  return n;
}

// Per-level launch choices (0 = the library default). The autotuner of
// bdis_plan_create fills them by timing the candidates on the real data.
struct LevelTuning {
  int search_cpl = 0;      // fast search path: 1, 2 or 4 columns per lane
  int search_threads = 0;  // search block size: 64 or 128
  int search_tiled = 0;    // search sampling: 1 = global memory, 2 = warp-tiled
  int densify_tile_y = 0;  // densify: 0 = strip kernel (or tiles of 32); 8, 16, 32 = tile height
};
struct Tuning {
  LevelTuning level[16];
};

// Device workspace of one match call. Offsets from the workspace base.
struct Layout {
  int levels = 0;  // coarsest + 1
  int lw[16] = {0}, lh[16] = {0};
  size_t L[16] = {0}, R[16] = {0}, G[16] = {0}, D[16] = {0};
  size_t d_star = 0, weight = 0;
  size_t warm = 0;  // seed map of the coarsest level from a previous disparity
  int warm_w = 0, warm_h = 0;
  // second search of the coarsest level (R16) and the posteriors / flags of both
  size_t d_star2 = 0, weight2 = 0, post1 = 0, post2 = 0, flags1 = 0, flags2 = 0;
  size_t prop = 0;  // network proposal at the proposal level
  int prop_level = kProposalLevel;
  size_t in_left = 0, in_right = 0, out = 0;  // host-path staging
  size_t bytes = 0;
};

Layout plan_layout(int w, int h, int count, const bdis_params &p, bool host_staging);

struct SearchArgs {
  const float *L, *G;
  const float2 *R2;  // packed right plane: (R[x], R[x+1] - R[x]) per pixel
  int w, h;
  long long plane;  // w * h
  const float *coarse;
  int cw, ch;
  long long cplane;
  int ps, stride, nx, ny, np;
  // floor(k / nx) = umulhi(k, nx_mul) for every patch index k < np (0: divide)
  unsigned nx_mul;
  long long total;  // count * np
  long long pixels; // count * plane (the extent of L, G and the packed R)
  int iters, s;
  float step, kappa;
  int nmin_valid, normalize;
  int cols_per_lane;  // fast path: columns of a patch per lane (1, 2, 3 or 4)
  int block_threads;  // 0 = 128
  int tiled;          // fast path: 1 = warp-tiled shared-memory sampling
  int fusion;         // BDIS_FUSION_*
  float *d_star, *weight;
  float *u_init, *posterior, *energies;
  uint8_t *flags;
  int32_t *n_valid;
  uint8_t *steps;
  int debug;  // any of the per-patch debug outputs above is wanted (set at launch)
};

struct DensifyArgs {
  int w, h;
  long long plane;
  long long total;  // count * plane
  int ps, stride, nx, ny, np;
  float two_s2;
  const float *d_star, *weight;
  const float *coarse;
  int cw, ch;
  long long cplane;
  int is_finest;
  int fusion;
  int tile_y;         // 0 = strip kernel where PS / stride is whole, else tiles of 32; > 0 tiles
  const float *L;     // DIS fusion: the level's left plane
  const float2 *R2;   // DIS fusion: the level's packed right plane
  float *out;
};

// Launchers (return the launch error, if any).
cudaError_t launch_prepare_level0(const bdis_image &left, const bdis_image &right, float *L0,
                                  float2 *R0, float *G0, cudaStream_t st);
// Level 0 and the first pyramid step in one kernel (the outputs of
// launch_prepare_level0 then launch_pyramid_level, bit for bit).
cudaError_t launch_prepare_pyramid0(const bdis_image &left, const bdis_image &right, float *L0,
                                    float2 *R0, float *G0, float *L1, float2 *R1, float *G1,
                                    cudaStream_t st);
cudaError_t launch_pyramid_level(const float *L, const float2 *R, int w, int h, int count,
                                 float *L1, float2 *R1, float *G1, cudaStream_t st);
cudaError_t launch_pack_right(const float *R, int w, int h, int count, float2 *R2,
                              cudaStream_t st);
cudaError_t launch_search(const SearchArgs &a, cudaStream_t st);
cudaError_t launch_densify(const DensifyArgs &a, cudaStream_t st);
cudaError_t launch_select_start(float *d_a, float *w_a, const float *p_a, const uint8_t *f_a,
                                const float *d_b, const float *w_b, const float *p_b,
                                const uint8_t *f_b, long long total, cudaStream_t st);
// The network's forward pass on the caller's stream (net.cu).
bdis_status net_forward_on(bdis_net *net, const float *L, const float *R, int r_stride, int w,
                           int h, int count, float *out, cudaStream_t st);

// How the coarsest searched level starts: 0 (plain), a given map, or the net.
struct Seed {
  const float *map = nullptr;  // a disparity map at pyramid level `level`
  int level = 0;
  bdis_net *net = nullptr;     // or: the proposal network run on pyramid level `level`
  int fallback = 0;            // R16 per-patch choice against the plain start
};

cudaError_t launch_warm_map(const float *prev, int w, int h, int level, int count, float *out,
                            cudaStream_t st);
cudaError_t launch_upsample(const float *map, int mw, int mh, int level, int w, int h, int count,
                            float *out, cudaStream_t st);

// Columns per lane of the fast search path (1 or the wide variant); tunable.
int search_cols_per_lane();
void set_search_cols_per_lane(int cpl);
int search_tiled();
void set_search_tiled(int on);
int densify_tile();
void set_densify_tile(int tile_height);
int pyramid_fused();
void set_pyramid_fused(int variant);

// ---- Bounds-checked build (-DBDIS_CHECKED; the memory-sanitizer substitute,
// libbdis_checked.so). There, the kernels' data-dependent global accesses
// check their element index against the buffer's extent; an access out of
// bounds is skipped (a read gives 0) and sets bit `site` of this translation
// unit's check word, which bdis_check_status reads. In the normal build the
// checks compile away. Sites:
enum CheckSite {
  kCheckSearchSample = 0,   // inverse search: right-plane samples (window and steps)
  kCheckSearchRows = 1,     // inverse search: template and gradient rows
  kCheckSearchOut = 2,      // inverse search: per-patch outputs
  kCheckDensifyTile = 3,    // densify: staged patch tile
  kCheckDensifyOut = 4,     // densify: dense map
  kCheckPyramidInput = 5,   // level-0 preparation: the input views
  kCheckPyramidStage = 6,   // pyramid step: the staged level
  kCheckPyramidOut = 7,     // level planes written by the pyramid kernels
};
#ifdef BDIS_CHECKED
static __device__ unsigned g_check_word;
#endif
__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
#ifdef BDIS_CHECKED
  if (i < 0 || i >= n) {
    atomicOr(&g_check_word, 1u << site);
    return false;
  }
#else
  (void)i;
  (void)n;
  (void)site;
#endif
  return true;
}
// A read-only float load that the checked build bounds-checks against
// [base, base + n).
__device__ __forceinline__ float ld_checked(const float *p, const float *base, long long n,
                                            int site) {
  if (!in_bounds(p - base, n, site)) return 0.f;
  return __ldg(p);
}
// Site wrappers: in the normal build they expand to the plain expression
// (so its code is exactly what it was without checks), in the checked build
// to the checked form. BDIS_CHECKED_ONLY(...) keeps its argument only in the
// checked build (extra parameters and arguments).
#ifdef BDIS_CHECKED
#define BDIS_CHECKED_ONLY(...) __VA_ARGS__
#define BDIS_LDG(p, base, n, site) ::bdis::ld_checked((p), (base), (n), (site))
#else
#define BDIS_CHECKED_ONLY(...)
#define BDIS_LDG(p, base, n, site) __ldg(p)
#endif
// Read and clear this translation unit's check word (always 0 in the normal
// build).
static inline cudaError_t take_check_word(unsigned *v) {
#ifdef BDIS_CHECKED
  cudaError_t e = cudaMemcpyFromSymbol(v, g_check_word, sizeof(unsigned));
  const unsigned z = 0u;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_word, &z, sizeof(unsigned));
  return e;
#else
  *v = 0u;
  return cudaSuccess;
#endif
}
cudaError_t take_check_search(unsigned *v);
cudaError_t take_check_densify(unsigned *v);
cudaError_t take_check_pyramid(unsigned *v);

// Programmatic dependent launch of the method's default kernels (pyramid,
// search, densify): a kernel may be scheduled while the previous kernel on
// the stream finishes its last blocks, so its launch and block start-up
// overlap that tail. Each such kernel first signals that its own dependents
// may be scheduled (all of its blocks have started by then, so a waiting
// dependent never holds back one of them), then waits for the previous
// grid to complete and its writes to be visible, before touching global
// memory. Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  asm volatile("griddepcontrol.wait;\n" ::: "memory");
}
int launch_overlap();
void set_launch_overlap(int on);
// SMs of the current device (looked up once per device).
int device_sms();

template <typename... KArgs, typename... Args>
cudaError_t launch_maybe_overlapped(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                    cudaStream_t st, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  // Only launches of at most 16 blocks per SM overlap. Measured: one pair's
  // latency fell 17% with the overlap, but a 512-pair step took 1.7% longer
  // (likely because the next kernel's early blocks land on whichever SMs
  // free up first, an uneven placement for the rest of that kernel).
  const long long blocks = (long long)grid.x * grid.y * grid.z;
  cfg.numAttrs = (launch_overlap() && blocks <= 16LL * device_sms()) ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Fill SearchArgs / DensifyArgs geometry from parameters (host).
void fill_search_args(SearchArgs &a, int w, int h, int count, const bdis_params &p);
void fill_densify_args(DensifyArgs &a, int w, int h, int count, const bdis_params &p);

// Every device allocation of the library goes through here, so that host-side
// fault injection (bdis_inject_alloc_failures) can make the next ones fail as
// out of memory without touching the GPU.
cudaError_t device_alloc(void **p, size_t bytes);

// Record a CUDA error for bdis_last_error_string() and map it to a status.
bdis_status record_cuda(cudaError_t e);
void set_last_error(const char *msg);
bdis_status check_params(const bdis_params *p);

// Pieces of bdis_match for entry points that bring their own scratch memory.
size_t match_scratch_bytes(int w, int h, int count, const bdis_params &p);
bdis_status check_match_args(const bdis_image *left, const bdis_image *right,
                             const bdis_params *p, const float *disparity_out);
bdis_status check_match_pointers(const bdis_image *left, const bdis_image *right,
                                 const float *disparity_out);
bdis_status run_match_in(void *scratch, size_t scratch_bytes, cudaStream_t stream,
                         const bdis_image &left, const bdis_image &right, const bdis_params &p,
                         float *out, const Tuning *tune = nullptr, const Seed *seed = nullptr);
// Fill `tune` for every searched level by timing the candidate launches on
// the given data (after one full run that fills the level planes).
bdis_status autotune_match(void *scratch, size_t scratch_bytes, cudaStream_t stream,
                           const bdis_image &left, const bdis_image &right,
                           const bdis_params &p, float *out, Tuning *tune);

inline void apply_tuning(SearchArgs &a, const LevelTuning &t) {
  if (t.search_cpl) a.cols_per_lane = t.search_cpl;
  if (t.search_threads) a.block_threads = t.search_threads;
  if (t.search_tiled) a.tiled = t.search_tiled - 1;
}
inline void apply_tuning(DensifyArgs &a, const LevelTuning &t) {
  if (t.densify_tile_y) a.tile_y = t.densify_tile_y;
}

}  // namespace bdis
