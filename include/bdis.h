/*
 * bdis.h -- C ABI of the GB300 (sm_103a) implementation of Bayesian Dense
 * Inverse Search (BDIS) stereo matching, Song et al., arXiv 2106.07136.
 *
 * The method (Sec. 2): build a coarse-to-fine image pyramid (Sec. 2.1,
 * Fig. 1); at each scale run the inverse-search Lucas-Kanade of Eq. 1 on a
 * grid of overlapping square patches; weigh every patch by the Bayesian
 * posterior of Eqs. 3-4 over a small window of disparities, dropping patches
 * that fail the convergence (saddle) test or the valid-pixel threshold gamma
 * (Sec. 2.2, Sec. 3); fuse the patches into a dense map with the spatial
 * Gaussian mask of Eq. 5 (Sec. 2.3). Pixels that no kept patch covers are
 * not estimated (Sec. 3.2).
 *
 * Conventions for every entry point:
 *   - Disparity D >= 0 with I_left(x, y) ~ I_right(x - D, y) on rectified,
 *     row-aligned pairs (Sec. 3). Intensities are gray levels 0..255.
 *   - Images and maps are row-major. "Dense" means pitch = width elements
 *     and consecutive images of a batch packed back to back.
 *   - Pointers documented as "device" must be CUDA device (or managed)
 *     memory on the handle's device (for bdis_match_static: the current
 *     device); the caller owns them. Device memory of another GPU is refused
 *     with BDIS_E_INVALID_ARG before anything is launched.
 *   - Work is enqueued on the given CUDA stream and returns before it
 *     finishes; argument errors return synchronously without enqueuing
 *     anything; a CUDA error is returned by the call that observes it.
 *   - `void *stream` is a cudaStream_t (NULL = the legacy default stream).
 *   - A handle is not thread-safe: use one handle per host thread/stream.
 *
 * Per-patch flag bits (bdis_patch_debug.flags): 1 flat (no gradient energy,
 * no update), 2 diverged (moved more than the patch size from its start, or
 * non-finite), 4 saddle (another window sample has lower energy), 8 below
 * gamma, 16 no pixel valid at every window sample, 32 not converged (last
 * update above 0.02 px). Any bit but 1 drops the patch. The window of a
 * diverged patch is not evaluated: its posterior is 0 and bits 4 and 16 stay
 * clear.
 */
#ifndef BDIS_H
#define BDIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    BDIS_OK = 0,
    BDIS_E_INVALID_ARG = 1, /* a size, pointer or parameter is out of range */
    BDIS_E_NOMEM = 2,       /* device or pinned allocation failed; handle still usable */
    BDIS_E_CUDA = 3,        /* a CUDA call failed; see bdis_last_error_string() */
    BDIS_E_TIMEOUT = 4,     /* a bounded wait ran out */
    BDIS_E_UNSUPPORTED = 5  /* valid for the method but outside this library's limits */
} bdis_status;

typedef enum { BDIS_U8 = 0, BDIS_F32 = 1 } bdis_format;

/* A batch of `count` equally sized grayscale images. data points at the first
 * pixel of the first image; rows are pitch_bytes apart and images
 * image_stride_bytes apart (ignored when count == 1). BDIS_F32 exists for
 * sub-pixel test fixtures whose warps are exact only in floating point. */
typedef struct {
    const void *data;
    int width;
    int height;
    size_t pitch_bytes;
    size_t image_stride_bytes;
    int count;
    bdis_format format;
} bdis_image;

/* Parameters of the method, names after the paper (Sec. 3):
 *   patch_size      side of the square patch in pixels (Sec. 1), 4..32;
 *   overlap         fraction shared by neighbouring patches, [0, 1); the
 *                   stride is round(patch_size * (1 - overlap)), at least 1;
 *   iterations      maximum inverse-search steps per patch and scale (Eq. 1), >= 0;
 *                   a patch stops early once its update falls below 1e-4 px;
 *   coarsest_scale  pyramid level where the search starts (level l has
 *                   ceil(W / 2^l) x ceil(H / 2^l) pixels), 0..15;
 *   finest_scale    level where it ends, 0..coarsest_scale; above 0 the map
 *                   is brought to full size by bilinear reads;
 *   sigma_r         brightness std of the likelihood, Eq. 4 (paper: 4);
 *   sigma_s         spatial std of the Gaussian mask, Eq. 5 (paper: 4);
 *   window_samples  s, disparity candidates in the window of Eq. 3, odd,
 *                   1..15 (paper: 5);
 *   window_step     spacing of the candidates in px (paper: 0.5 and 1 px
 *                   offsets, i.e. 0.5);
 *   gamma           minimum fraction of patch pixels whose right-image
 *                   sample lies inside the image (paper: 0.75 at 640x480,
 *                   0.25 at 288x360);
 *   normalize       1: subtract the patch means (DIS's normalisation);
 *   fusion          BDIS_FUSION_BDIS: the Bayesian posterior and Gaussian mask
 *                   (Sec. 2.2-2.3); BDIS_FUSION_DIS: the baseline the paper
 *                   compares against, every patch fused by its inverse
 *                   squared residual (Eq. 2; a patch that left its search
 *                   range falls back to its start). */
enum { BDIS_FUSION_BDIS = 0, BDIS_FUSION_DIS = 1 };

typedef struct {
    int patch_size;
    float overlap;
    int iterations;
    int coarsest_scale;
    int finest_scale;
    float sigma_r;
    float sigma_s;
    int window_samples;
    float window_step;
    float gamma;
    int normalize;
    int fusion;
} bdis_params;

/* Optional per-patch outputs of bdis_search_level. Any pointer may be NULL.
 * Arrays are count x n_patches (energies: count x n_patches x s), device. */
typedef struct {
    float *u_init;     /* starting disparity of each patch */
    float *posterior;  /* Eq. 3 posterior of D* within its window */
    float *energies;   /* window energies E_i, i = 0..s-1 */
    uint8_t *flags;    /* flag bits listed above */
    int32_t *n_valid;  /* pixels whose sample at D* is inside the image */
    uint8_t *steps;    /* inverse-search updates applied to D, 0..iterations */
} bdis_patch_debug;

typedef struct bdis_handle bdis_handle;
typedef struct bdis_net bdis_net; /* the learned proposal network (see below) */

/* Paper defaults (Sec. 3): patch 8, overlap 0.75, 12 iterations, scales 4..0,
 * sigma_r = sigma_s = 4, 5 samples 0.5 px apart, gamma 0.75, normalize 1,
 * BDIS fusion. */
void bdis_default_params(bdis_params *p);

const char *bdis_status_string(bdis_status s);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char *bdis_last_error_string(void);

/* ABI version: (major << 16) | minor. */
int bdis_version(void);

/* ---------------------------------------------------------------- geometry
 * Pure host functions, no GPU needed. */

/* Size of pyramid level `level` for a W x H image (Sec. 2.1): ceil halving. */
bdis_status bdis_level_dims(int width, int height, int level, int *level_width,
                            int *level_height);

/* Patch grid along an axis of n pixels: stride and number of origins
 * (origins i * stride, the last moved to n - patch_size). */
bdis_status bdis_grid(int n, int patch_size, float overlap, int *stride, int *count);

/* Total number of patches searched for one W x H pair over all levels. */
bdis_status bdis_patch_count(int width, int height, const bdis_params *p, int64_t *total);

/* ------------------------------------------------------------------ handle */

/* Create a matcher bound to CUDA device `device` and stream `stream`.
 * The handle owns a device workspace that grows on demand. */
bdis_status bdis_create(bdis_handle **out, int device, void *stream);

/* Reserve the workspace for a batch of `count` W x H pairs under `p`, so that
 * later bdis_match calls of that size or smaller allocate nothing. */
bdis_status bdis_reserve(bdis_handle *h, int width, int height, int count, const bdis_params *p);

/* Bytes of device workspace the handle currently holds. */
size_t bdis_workspace_bytes(const bdis_handle *h);

void bdis_destroy(bdis_handle *h);

/* Kernel timing. When enabled, the handle brackets each of its launches with
 * CUDA events on its stream (one pair of event records per launch, no
 * synchronisation). bdis_read_timing waits for the recorded events, adds
 * their durations per kernel class and clears them. Classes:
 * 0 level-0 preparation, 1 pyramid step, 2 inverse search + posterior,
 * 3 densification, 4 upsampling, 5 seed map, 6 proposal network, 7 the
 * per-patch choice of the seeded start.
 * Independently of this switch, every launch sits inside an NVTX range named
 * for its class and pyramid level ("bdis search L0"), and each whole-method
 * call inside one named for the entry point, so a profiler (ncu --nvtx,
 * Nsight Systems) can attribute and filter them; without a profiler attached
 * a range costs a few nanoseconds of host time. */
#define BDIS_TIMING_CLASSES 8
typedef struct {
    double ms[BDIS_TIMING_CLASSES];
    int64_t launches[BDIS_TIMING_CLASSES];
} bdis_timing;

bdis_status bdis_enable_timing(bdis_handle *h, int on);
bdis_status bdis_read_timing(bdis_handle *h, bdis_timing *out);

/* --------------------------------------------------------------- the method */

/* Dense disparity of `left->count` pairs (Sec. 2, the whole method).
 * left/right: device images, identical geometry and format.
 * disparity_out: device, count x height x width float, dense; NaN where no
 * kept patch covers the pixel (Sec. 3.2). Enqueued on the handle's stream. */
bdis_status bdis_match(bdis_handle *h, const bdis_image *left, const bdis_image *right,
                       const bdis_params *p, float *disparity_out);

/* Warm start (for video): as bdis_match, but the coarsest searched level
 * starts from `prev`, a previous disparity of the same scene (device, count x
 * H x W float, NaN allowed; e.g. the last frame's output), instead of 0. The
 * seed map at level coarsest+1 is the mean of prev's finite values over the
 * 2^(coarsest+1) block centred on each sample point, divided by
 * 2^(coarsest+1), or 0 where none is finite; it seeds the coarsest patches
 * and the pixels that level carries. prev may alias disparity_out (it is
 * read before the output is written). prev NULL = bdis_match. */
bdis_status bdis_match_warm(bdis_handle *h, const bdis_image *left, const bdis_image *right,
                            const bdis_params *p, const float *prev, float *disparity_out);

/* Proposal start (R16): the coarsest level is seeded from `seed`, a disparity
 * map at pyramid level seed_level (0..coarsest; count x ceil(H/2^l) x
 * ceil(W/2^l) floats, values in that level's pixels, NaN allowed), reduced to
 * level coarsest+1 by block means as at bdis_match_warm. With fallback = 0
 * this is the warm start from that level. With fallback = 1 the coarsest
 * level is searched twice, from the seed and from the plain start; a patch
 * keeps the seeded result only if it is kept, lies more than 0.1 px from a
 * kept plain result (closer, both found one solution and the plain result
 * stands), and the plain result is dropped or has no higher posterior; pixels of that level that no kept patch
 * covers carry the plain start: a proposal that every patch rejects gives
 * exactly bdis_match. Not in the paper (its start is 0). */
bdis_status bdis_match_seeded(bdis_handle *h, const bdis_image *left, const bdis_image *right,
                              const bdis_params *p, const float *seed, int seed_level,
                              int fallback, float *disparity_out);

/* Learned start: the proposal network runs on pyramid level
 * bdis_proposal_level(coarsest) of these pairs (inside the same launch
 * sequence) and its output seeds the coarsest level as at bdis_match_seeded. */
bdis_status bdis_match_learned(bdis_handle *h, bdis_net *net, const bdis_image *left,
                               const bdis_image *right, const bdis_params *p, int fallback,
                               float *disparity_out);

/* The pyramid level the learned start runs its network on for a given
 * coarsest scale: min(4, coarsest_scale) (-1 for a negative scale). Its map
 * is reduced to level coarsest + 1 by block means (as at bdis_match_seeded),
 * so a level near the coarsest loses no information the seed keeps; the
 * network is trained on this level. */
int bdis_proposal_level(int coarsest_scale);

/* Same, with HOST buffers: left/right are `count` dense width x height uint8
 * images in host memory, disparity_out a dense host float array. The call
 * copies in, matches, copies out and returns when the result is in
 * disparity_out. A batch of 2 or more pairs runs as 2 (4 from 8 pairs; from
 * 32 pairs 5, the first and last a sixteenth of the batch each) chunks: one
 * chunk's inputs are copied in while the previous chunk is matched and the
 * one before is copied out (two copy streams owned by the handle, device
 * buffers double-buffered). Pinned host memory makes the
 * copies asynchronous DMA; pageable memory works but is slower. */
bdis_status bdis_match_host(bdis_handle *h, const uint8_t *left, const uint8_t *right,
                            int width, int height, int count, const bdis_params *p,
                            float *disparity_out);

/* Asynchronous form of bdis_match_host, for streams of batches (video,
 * serving): the call enqueues the copy-in, the match (Sec. 2, as at
 * bdis_match) and the copy-out of one whole batch and returns at once with
 * a ticket (> 0) in *ticket. Successive calls overlap: a call's copy-in
 * runs beside earlier calls' matches, its copy-out beside later ones'. The
 * device holds BDIS_ASYNC_SLOTS (4) batches' inputs and outputs (slot =
 * ticket % 4); a slot is refilled only after the match and the copy-out of
 * the call four before have finished, so up to four calls can be in flight
 * and a copy that runs late holds up the matches only once all four slots
 * are taken. Device memory: bdis_match's workspace, whose own input and
 * output buffers are slot 0, plus three more slots of 6 bytes per pixel
 * (2 in, 4 out): 2.8 GB more for 512 pairs of 640 x 480.
 * Ownership: left, right and disparity_out stay the caller's; they must not
 * be written (inputs) or read (output) until bdis_host_wait(h, ticket) has
 * returned. Use pinned host memory: with pageable memory the copies, and so
 * the call, block. Any other call on the handle that uses its workspace
 * (bdis_match and its variants, bdis_match_host, bdis_reserve) first waits
 * for every asynchronous call in flight; so does a call with another
 * geometry, batch size or scale range.
 * Errors: argument, parameter and geometry errors as at bdis_match_host,
 * returned at once with nothing enqueued; CUDA errors of the enqueue at
 * once; CUDA errors of the work itself from bdis_host_wait. */
#define BDIS_ASYNC_SLOTS 4
bdis_status bdis_match_host_async(bdis_handle *h, const uint8_t *left, const uint8_t *right,
                                  int width, int height, int count, const bdis_params *p,
                                  float *disparity_out, uint64_t *ticket);

/* Returns when the asynchronous call `ticket` (and every call before it) has
 * finished and its result is in its disparity_out. Waiting for the latest
 * ticket leaves the handle's streams idle. BDIS_E_INVALID_ARG for a ticket
 * this handle has not issued. */
bdis_status bdis_host_wait(bdis_handle *h, uint64_t ticket);

/* Bounded form of bdis_host_wait for loops that must not block (serving):
 * polls the call's completion against a host-side deadline of timeout_ms
 * (>= 0; 0 = just look) and returns BDIS_E_TIMEOUT when the deadline passes
 * first. The call stays in flight and its buffers stay the library's until a
 * later wait returns BDIS_OK. Other errors as at bdis_host_wait. Not in the
 * paper (its program is one blocking loop). */
bdis_status bdis_host_wait_timeout(bdis_handle *h, uint64_t ticket, double timeout_ms);

/* Host-side fault injection, for tests of failure handling: the next `count`
 * device allocations the library makes (a handle's workspace grows, plan
 * workspaces, network buffers) fail as if the device were out of memory,
 * without asking the driver. The calls that hit one return BDIS_E_NOMEM and
 * leave their handle, plan or network usable. count <= 0 clears it.
 * Process-wide. Nothing on the GPU is touched. */
void bdis_inject_alloc_failures(int count);

/* ------------------------------------------------------------------ steps
 * The method's steps, one launch sequence each, on dense device batches of
 * `count` planes. bdis_match runs exactly these kernels. */

/* The right view of every level is kept PACKED: two floats per pixel,
 * (R[x], R[x+1] - R[x]), the difference 0 in the last column, so that the
 * search interpolates with one 8-byte load. Packed planes are count x H x W
 * x 2 floats and must be 8-byte aligned. */

/* Level 0 (Sec. 2.1): gray levels as float and the template gradient.
 * L0, G0: device, count x H x W float; R0: device, packed. G0 = Sobel-x / 8
 * of the left image with a mirrored (reflect-101) border. */
bdis_status bdis_prepare_level0(const bdis_image *left, const bdis_image *right, float *L0,
                                float *R0, float *G0, void *stream);

/* One pyramid step (Sec. 2.1): 5x5 binomial [1 4 6 4 1]/16 smoothing with a
 * reflect-101 border, keeping even samples, for both views; plus Sobel-x / 8
 * of the new left level. Inputs count x h x w (R, R1 packed); outputs count x
 * ceil(h/2) x ceil(w/2). */
bdis_status bdis_pyramid_level(const float *L, const float *R, int width, int height, int count,
                               float *L1, float *R1, float *G1, void *stream);

/* Pack a plain right-view plane (count x h x w float) into the packed layout
 * the search reads (for callers that bring their own pyramid). */
bdis_status bdis_pack_right(const float *R, int width, int height, int count, float *R2,
                            void *stream);

/* Inverse search of every patch of one level (Eq. 1) with the posterior and
 * patch tests (Eqs. 3-4, Sec. 2.2, Sec. 3). L, G: count x h x w device; R:
 * the packed right view of the level.
 * coarse: the next coarser dense map, count x ch x cw, or NULL at the
 * coarsest level (patches then start at 0); a patch starts from twice the
 * coarse map read bilinearly at half its centre. Outputs, count x n_patches
 * with patches row-major over the grid: d_star (D*), weight (posterior times
 * the valid-pixel fraction; 0 for a dropped patch). dbg may be NULL. */
bdis_status bdis_search_level(const float *L, const float *R, const float *G, int width,
                              int height, int count, const float *coarse, int coarse_width,
                              int coarse_height, const bdis_params *p, float *d_star,
                              float *weight, const bdis_patch_debug *dbg, void *stream);

/* Densification of one level (Sec. 2.3): each pixel is the mean of its kept
 * covering patches' D* weighted by weight_k * exp(-|x - c_k|^2 / (2 sigma_s^2)).
 * With DIS fusion the per-pixel weight is weight_k / max(r^2, 1) with r the
 * residual R(x - D*_k) - L(x) (Eq. 2), over patches whose sample is inside
 * the right image; L and R (the level's left plane and packed right plane)
 * are then required, and may be NULL otherwise. Pixels without a kept patch
 * get NaN when is_finest, otherwise twice the coarse map at half their
 * position (0 when coarse is NULL). out: count x h x w device. */
bdis_status bdis_densify_level(int width, int height, int count, const bdis_params *p,
                               const float *d_star, const float *weight, const float *coarse,
                               int coarse_width, int coarse_height, int is_finest,
                               const float *L, const float *R, float *out, void *stream);

/* The warm-start seed map alone: level `level` (1..16) of a count x H x W
 * previous disparity, as described at bdis_match_warm. out: count x
 * ceil(H/2^level) x ceil(W/2^level). */
bdis_status bdis_warm_map(const float *prev, int width, int height, int level, int count,
                          float *out, void *stream);

/* The per-patch choice on the coarsest level when it is searched twice
 * (bdis_match_seeded with fallback; R16, not in the paper): result a
 * (searched from the seed) is kept only if it is kept by the patch tests, it
 * is not within 0.1 px of a kept result b (searched from the plain start;
 * that close, both found one solution and the plain one stands), and b is
 * dropped or has no higher posterior; elsewhere b's D* and weight overwrite
 * a's. All arrays device, `total` patches (bdis_search_level's outputs and
 * its debug posterior and flags). */
bdis_status bdis_select_start(float *d_star_a, float *weight_a, const float *posterior_a,
                              const uint8_t *flags_a, const float *d_star_b,
                              const float *weight_b, const float *posterior_b,
                              const uint8_t *flags_b, int64_t total, void *stream);

/* Bring a map of level f to full size: bilinear over finite neighbours,
 * values times 2^f; NaN where no finite neighbour has weight. */
bdis_status bdis_upsample(const float *map, int map_width, int map_height, int level, int width,
                          int height, int count, float *out, void *stream);

/* Tuning: lane layout of the inverse-search kernel for patch sizes 8, 12 and
 * 16 with the paper's 5-sample window. 1 = one patch column per lane (a
 * group of 8 or 16 lanes per patch); 2 = the wide layout (2 columns per lane
 * for sizes 8 and 16, 3 for size 12); 4 = 4 columns per lane (size 8 only;
 * other sizes take 2). Results are identical up to float rounding; the
 * choice only moves speed. Process-wide; default 2. Returns
 * BDIS_E_INVALID_ARG for any other value. */
bdis_status bdis_set_search_variant(int columns_per_lane);
int bdis_get_search_variant(void);

/* Tuning: how that kernel reads the right view. 0 (default) = every sample
 * is read from global memory (through L1). 1 = warp-tiled: the patches of a
 * warp lie on one patch-grid row, and the right-view rows they can sample
 * while inside their search range are staged once in shared memory. A warp
 * whose starts spread too far for its tile reads global memory instead.
 * Results are bit-identical either way. Process-wide. */
void bdis_set_search_tiling(int on);
int bdis_get_search_tiling(void);

/* Tuning: the densification kernel (Eq. 5 fusion, BDIS mode). 0 (default) =
 * the strip kernel where the grid stride divides the patch size (overlap
 * 0.75 at patch sizes 8, 12, 16), tiles of 32 rows otherwise; 8, 16 or 32 =
 * the tiled kernel with that tile height. Results are identical whichever
 * runs. Process-wide; BDIS_E_INVALID_ARG for any other value. A plan's
 * autotuner makes its own per-level choice. */
bdis_status bdis_set_densify_variant(int tile_height);
int bdis_get_densify_variant(void);

/* Tuning: the pyramid (Sec. 2.1). 2 (default) = level 0 and the first
 * pyramid step in one kernel (the 8-bit views staged once; level 0 written
 * and never read back for level 1), later steps as in 1; 1 = the level-0
 * preparation, then one fused kernel per step (downsample into shared
 * memory, then L, packed R and the gradient written once); 0 = the
 * preparation, then per step a downsample kernel and a gradient-and-packing
 * kernel over the new level. Results are identical. Values outside 0..2 are
 * clamped. Process-wide. bdis_pyramid_level runs one step: fused unless 0. */
void bdis_set_pyramid_variant(int variant);
int bdis_get_pyramid_variant(void);

/* Tuning: launch overlap. 1 (default): launches of the default pyramid,
 * search and densify kernels and of the seed-map and seeded-start choice
 * kernels that have at most 16 blocks per SM (small batches, coarse levels)
 * are programmatic dependents of the kernel before them on the stream, so a
 * launch's start-up overlaps the previous kernel's last blocks; each kernel
 * still waits for the previous one to finish before it touches memory.
 * 0: plain stream order. Results are identical. Process-wide. */
void bdis_set_launch_overlap(int on);
int bdis_get_launch_overlap(void);

/* Bounds-checked build (libbdis_checked.so: the same sources compiled with
 * -DBDIS_CHECKED; the substitute for a memory sanitizer). There, the
 * kernels' data-dependent global accesses check their element index against
 * the buffer's extent, skip an access out of bounds (a read gives 0) and
 * record the access site. bdis_check_status waits for the device, then
 * writes the sites caught since the last call as bits and clears them:
 * bit 0 inverse-search samples of the right plane, 1 its template and
 * gradient rows, 2 its per-patch outputs, 3 the densify patch tile, 4 the
 * densify output, 5 the level-0 input views, 6 a pyramid step's input level,
 * 7 the pyramid's output planes. In the normal build it writes 0.
 * bdis_checked_build returns 1 in the checked build, else 0. */
bdis_status bdis_check_status(uint32_t *sites);
int bdis_checked_build(void);

/* Measurement utility, not part of the method: FP32 FMA throughput of the
 * current device in TFLOP/s (the roofline denominator of the inverse search).
 * Runs two launches of an FMA-chain kernel of `iterations` steps per chain on
 * `stream` and waits for them. */
bdis_status bdis_probe_fp32_tflops(int iterations, double *tflops, void *stream);

/* ------------------------------------------------------------ batch plans
 * Mixed-resolution batches (the method is per pair, Sec. 2; this is how many
 * pairs of several sizes share the GPU). A plan fixes `n_groups` groups, each
 * a batch of equally sized pairs with its device images and output, all
 * bound by ADDRESS: refill the images and rerun. Each group gets its own
 * workspace (so groups run concurrently); the whole sequence is captured once
 * into a CUDA graph with one branch per group, and bdis_plan_run is a single
 * graph launch on `stream`. With BDIS_PLAN_AUTOTUNE, creation first runs each
 * group once and times, per level, the candidate search lane layouts (1, the
 * wide layout, and 4 columns per lane at patch size 8), block sizes (64, 128)
 * and sampling (global or warp-tiled), and the densify kernels (strip, tiles
 * of 8, 16, 32 rows) on that data, keeping the fastest; results are the same
 * up to float rounding whatever is chosen. bdis_plan_create synchronises `stream`
 * (autotuning reads the inputs) and may take a second; run is asynchronous. */
#define BDIS_PLAN_AUTOTUNE 1
/* Per group, raise the coarsest scale to the smallest c >= p->coarsest_scale
 * with 2^c >= width / 40, so that a disparity range of a tenth of the width
 * (the mixed-size batch's) is at most 4 px at the coarsest level, where each
 * patch starts from 0 (Sec. 2.1); c is lowered again while the coarsest level
 * would be smaller than a patch. Not in the paper: an option of the batched
 * path. bdis_plan_info reports each group's scale. */
#define BDIS_PLAN_SCALE_TO_WIDTH 2

typedef struct {
    bdis_image left, right;  /* device, as for bdis_match */
    float *disparity_out;    /* device, count x height x width */
} bdis_group;

typedef struct {
    int search_columns_per_lane; /* 0 = default */
    int search_block_threads;    /* 0 = default (128) */
    int densify_tile_height;     /* 0 = strip kernel (stride divides the patch
                                    size), else tiles of 32; 8/16/32 = tiles */
    size_t workspace_bytes;      /* of the whole group */
    int coarsest_scale;          /* of the group (BDIS_PLAN_SCALE_TO_WIDTH may raise it) */
    int search_tiling;           /* 0 = global-memory sampling, 1 = warp-tiled */
} bdis_plan_choice;

typedef struct bdis_plan bdis_plan;

bdis_status bdis_plan_create(int device, const bdis_group *groups, int n_groups,
                             const bdis_params *p, int flags, void *stream, bdis_plan **out);
bdis_status bdis_plan_run(bdis_plan *plan, void *stream);
/* Launch choices for one group and pyramid level (after autotuning). */
bdis_status bdis_plan_info(const bdis_plan *plan, int group, int level, bdis_plan_choice *out);
size_t bdis_plan_workspace_bytes(const bdis_plan *plan);
void bdis_plan_destroy(bdis_plan *plan);

/* ------------------------------------------------- learned coarse proposal
 * Not in the paper (its coarsest level starts from 0, Sec. 2.1): a small
 * network proposes the coarsest disparity and BDIS refines it. Six 3x3
 * convolutions with dilations 1, 2, 4, 4, 2, 1; 2 -> 32 -> 32 -> 32 -> 32 ->
 * 32 -> 1 channels, ReLU between layers; input [(L - 128) / 64, (R - 128) /
 * 64] of a pyramid level, output that level's disparity in its pixels. BF16
 * weights and activations, FP32 accumulation, on the tensor cores.
 * Master weights are FP32 in this order, layer by layer: W[co][ky*3+kx][ci]
 * (bdis_net_weight_count() floats in all), then b[co]. */
int bdis_net_weight_count(void);

/* Tuning: the kernels of the network's forward convolutions, all implicit
 * GEMMs with BF16 operands and FP32 accumulation. 1 (default) = banded
 * 5th-generation tensor-core kernel for inference (bdis_net_forward,
 * bdis_match_learned): activations in a zero-padded planar layout, a band of
 * image rows with its halo staged by one bulk copy per channel plane, each
 * 3x3 tap's operand a shifted window of it, accumulators in tensor memory,
 * the next band's copy overlapping the epilogue; 2 = the per-tile tcgen05
 * kernel (a 128-pixel tile's slab staged by the threads); 0 = mma.sync
 * (warp-level BF16 MMA). Results agree up to FP32 accumulation order. The
 * training forward takes the per-tile kernel under 1 and 2; inputs too wide
 * for a kernel's shared memory take the next one down. Process-wide. */
void bdis_set_net_variant(int tensor_path);
int bdis_get_net_variant(void);

/* weights: host, bdis_net_weight_count() floats (copied). */
bdis_status bdis_net_create(int device, const float *weights, bdis_net **out);

/* Proposal for count x h x w level planes: L (float), R (float with element
 * stride r_stride: 1 plain, 2 packed) -> disparity (float, level pixels).
 * All device. Activations are held by the network object (grown on demand). */
bdis_status bdis_net_forward(bdis_net *net, const float *L, const float *R, int r_stride,
                             int width, int height, int count, float *disparity, void *stream);

/* Loss (Huber, delta 1, mean over all count*h*w pixels; NaN labels count 0)
 * and its gradient with respect to the master weights, without updating.
 * loss_out / grad_out: host pointers or NULL (then nothing is copied). */
bdis_status bdis_net_gradient(bdis_net *net, const float *L, const float *R, int r_stride,
                              int width, int height, int count, const float *label,
                              float *loss_out, float *grad_out, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on that gradient. */
bdis_status bdis_net_train_step(bdis_net *net, const float *L, const float *R, int r_stride,
                                int width, int height, int count, const float *label, float lr,
                                float *loss_out, void *stream);

/* Whether a forward pass of the network timed out since the last call:
 * waits for `stream`, then returns BDIS_E_TIMEOUT (and clears the record) if
 * a tensor-core forward kernel's bounded wait for its own MMAs (about 200 ms)
 * ran out since the last bdis_net_status; that kernel then wrote NaN for the
 * tile and returned, so a proposal (and bdis_match_learned's seed) may hold
 * NaN there, which the seed map treats as missing. BDIS_OK otherwise. The
 * forward entry points themselves return before the kernels run, so this is
 * how a caller learns of it. */
bdis_status bdis_net_status(bdis_net *net, void *stream);

/* Host-side fault injection, for tests of the path above: records a timeout
 * exactly as the kernel's timeout path does (the network's device fault word
 * is written from the host); the next bdis_net_status returns BDIS_E_TIMEOUT. */
bdis_status bdis_net_inject_timeout(bdis_net *net);

/* Copy the FP32 master weights to host memory (waits for the device). */
bdis_status bdis_net_get_weights(bdis_net *net, float *weights_out);
void bdis_net_destroy(bdis_net *net);

/* ----------------------------------------------------------- no allocation
 * Some callers cannot allocate GPU memory: a hard real-time loop that froze
 * its memory map after start-up, a plug-in that runs inside a host process
 * whose allocator owns the device, or code on a path where cudaMalloc may
 * synchronise the device or fail at run time. bdis_match_static runs the
 * same kernels as bdis_match with no handle and no allocation: its scratch
 * memory (pyramid planes, per-patch arrays) is a fixed array of
 * BDIS_STATIC_SCRATCH_BYTES compiled into this library. The paper has no
 * counterpart; this is a deployment variant of bdis_match.
 *
 *   - Arguments, output and errors as bdis_match, on the CURRENT CUDA device
 *     and the given stream (cudaStream_t, NULL = legacy default stream).
 *   - No cudaMalloc, cudaFree or other allocating call is made.
 *   - Each call looks the array's device address up on the current device
 *     (cudaGetSymbolAddress). Under CUDA's lazy module loading the FIRST call
 *     on a device is what loads the array onto that device: the driver then
 *     reserves its 24 MiB, which may synchronise and may fail (returned as
 *     BDIS_E_NOMEM). So make one call per device at start-up, as a warm-up,
 *     before any stream capture and before the path that must not allocate.
 *     From then on the device holds the array until the process exits (or
 *     until cudaDeviceReset, after which the next call loads it again).
 *   - Work whose scratch need exceeds BDIS_STATIC_SCRATCH_BYTES is refused
 *     with BDIS_E_UNSUPPORTED and a message in bdis_last_error_string(). The
 *     24 MiB hold one 1280x720 pair or three 640x480 pairs at the defaults.
 *   - All calls on a device share the one array, which keeps the last call's
 *     contents; nothing in it needs clearing (each kernel writes every
 *     element it later reads). Calls whose work overlaps on the GPU (other
 *     streams, other host threads) race on the array: serialise them. */
#define BDIS_STATIC_SCRATCH_BYTES (24u << 20)

bdis_status bdis_match_static(const bdis_image *left, const bdis_image *right,
                              const bdis_params *p, float *disparity_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BDIS_H */
