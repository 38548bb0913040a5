// search.cu -- patch-wise inverse search (Sec. 2.1, Eq. 1) with the Bayesian
// patch posterior (Sec. 2.2, Eqs. 3-4) and the patch tests, one kernel.
//
// Layout (fast path): one patch per group of G lanes, each lane owning CPL
// adjacent columns of its patch and walking the rows (default CPL = 2, G = 4,
// 8 patches per warp; the generic path takes one column per lane). The right
// image is read as packed (R[x], R[x+1] - R[x]) pairs, so one 8-byte load and
// one FMA give a linearly interpolated sample. The G lanes of a group read
// consecutive pairs of one row (coalesced); neighbouring patches overlap, so
// these loads are served from L1/L2. Reductions over the patch are
// xor-butterflies inside the group. The lane's centred gradient is kept
// through the steps, in registers or (default kernel) in shared memory; the
// template is re-read where it is used.
//
// Arithmetic per patch (the method's own, Eq. 1 and Eq. 3):
//   - rows are aligned, so the set of pixels whose sample is inside the right
//     image is a run of columns; its sums (centred gradient, Hessian,
//     template term) are recomputed only when that run changes;
//   - with mean normalisation, sum g_n (R~_n - T_n) = sum g_c R~ - sum g_c T
//     where g_c is the gradient centred on the valid set; within one integer
//     base sum g_c R~ = A + t B is linear in the fraction, so A and B are
//     re-read (one load and two FMAs per pixel) only when the base or the run
//     changes in some patch of the warp, and an update is otherwise one FMA;
//   - the window energies are sums of residuals taken relative to a per-column
//     shift (the column's first-row residual), merged exactly over the group,
//     which keeps the saddle decisions well conditioned; per row a lane reads
//     the CPL + 2 packed pairs that all five samples of its columns need once;
//   - a lane's two columns take the same operations, which run as packed
//     f32x2 adds and FMAs (per component the scalar rounding).
//
// Two instantiations: a fast path with the patch size and window length fixed
// at compile time (fully unrolled, no per-row guards) for the common settings,
// and a generic path for any patch size up to 32 and window up to 15.
//
// Roofline: instruction-issue / FP32 bound. Algorithmic work per patch
// (patch evaluations x 8 flops per pixel): ps^2 * 8 * (updates + s), the
// update count being at most `iterations` (a converged patch stops early).
// DRAM bytes per patch level: the L, G and packed R planes read once
// (16 B per pixel) plus 8 B written per patch.
#include "bdis_internal.cuh"

namespace bdis {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kSearchThreads = 128;  // the fast kernels' launch bound (threads per block)

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <int G>
__device__ __forceinline__ int group_sum_int(int v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Split a sample position x - D into integer base and fraction computed from
// D alone (exact in float): x - D = (x + k) + t with t in [0, 1).
__device__ __forceinline__ void split_disp(float D, int &k, float &t) {
  const float nd = fminf(fmaxf(-D, -1.0e7f), 1.0e7f);  // NaN -> bound, never in range
  const float f = floorf(nd);
  k = (int)f;
  t = nd - f;
}

// Sample at (i0 + t) is inside [0, w-1].
__device__ __forceinline__ bool sample_ok(int i0, float t, int w) {
  return i0 >= 0 && (i0 < w - 1 || (i0 == w - 1 && t == 0.f));
}

// The same test for several columns at one fraction: i0 in [0, last_base(t, w)].
__device__ __forceinline__ int last_base(float t, int w) { return t == 0.f ? w - 1 : w - 2; }

__device__ __forceinline__ float lerp_packed(float2 q, float t) { return fmaf(t, q.y, q.x); }

__device__ __forceinline__ float bilinear_clamped(const float *M, int w, int h, float x,
                                                  float y) {
  x = fminf(fmaxf(x, 0.f), (float)(w - 1));
  y = fminf(fmaxf(y, 0.f), (float)(h - 1));
  const int x0 = (int)floorf(x), y0 = (int)floorf(y);
  const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
  const float tx = x - x0, ty = y - y0;
  const float top = (1.f - tx) * __ldg(M + (size_t)y0 * w + x0) + tx * __ldg(M + (size_t)y0 * w + x1);
  const float bot = (1.f - tx) * __ldg(M + (size_t)y1 * w + x0) + tx * __ldg(M + (size_t)y1 * w + x1);
  return (1.f - ty) * top + ty * bot;
}

// Patch index -> (pair, origin) and the coarse-to-fine start (Sec. 2.1: twice
// the coarser map read bilinearly at half the patch centre; 0 at the top).
struct PatchPos {
  int b, x0, y0;
  float u0;
};

__device__ __forceinline__ PatchPos patch_pos(const SearchArgs &a, long long k) {
  PatchPos p;
  p.b = (int)(k / a.np);
  const int kk = (int)(k - (long long)p.b * a.np);
  const int pj = kk / a.nx, pi = kk - (kk / a.nx) * a.nx;
  p.x0 = grid_origin(pi, a.nx, a.w, a.ps, a.stride);
  p.y0 = grid_origin(pj, a.ny, a.h, a.ps, a.stride);
  p.u0 = 0.f;
  if (a.coarse) {
    const float cx = (float)p.x0 + (a.ps - 1) * 0.5f, cy = (float)p.y0 + (a.ps - 1) * 0.5f;
    p.u0 = 2.f * bilinear_clamped(a.coarse + (long long)p.b * a.cplane, a.cw, a.ch, cx * 0.5f,
                                  cy * 0.5f);
  }
  return p;
}

// Posterior of the window centre (Eq. 3 with Eq. 4 as likelihood, evaluated
// relative to the smallest energy) and the patch flags; writes the outputs.
__device__ __forceinline__ void finish_patch(const SearchArgs &a, long long k, bool write,
                                             float D, float u0, float last_step, bool flat,
                                             int steps, int nvalid, int nc, float Ec, float Eo,
                                             float pc, float z, int ps) {
  uint8_t flags = flat ? kFlagFlat : 0;
  if (!isfinite(D) || fabsf(D - u0) > (float)ps) flags |= kFlagDiverged;
  if (fabsf(last_step) > kConvergeTol) flags |= kFlagUnconverged;
  float post = 0.f;
  if (nc == 0) {
    if (!(flags & kFlagDiverged)) flags |= kFlagEmpty;  // a diverged patch reads no window
  } else {
    post = __fdividef(pc, z);  // pc = exp(-(Ec - Emin) / kappa), the centre's term of z; z in [1, s]
    if (a.s > 1 && Eo < Ec - kSaddleTau * fmaxf(Ec, 1.f)) flags |= kFlagSaddle;
  }
  if (nvalid < a.nmin_valid) flags |= kFlagGamma;
  const bool drop = (flags & kDropFlags) != 0;
  if (write BDIS_CHECKED_ONLY(&&in_bounds(k, a.total, kCheckSearchOut))) {
    if (a.fusion == BDIS_FUSION_DIS) {
      // DIS fuses every patch (Eq. 2); a runaway patch falls back to its start
      a.d_star[k] = (flags & kFlagDiverged) ? u0 : D;
      a.weight[k] = 1.f;
    } else {
      a.d_star[k] = D;
      a.weight[k] = drop ? 0.f : post * (float)nvalid / (float)(ps * ps);
    }
    if (a.debug) {
      if (a.u_init) a.u_init[k] = u0;
      if (a.posterior) a.posterior[k] = post;
      if (a.flags) a.flags[k] = flags;
      if (a.n_valid) a.n_valid[k] = nvalid;
      if (a.steps) a.steps[k] = (uint8_t)steps;
    }
  }
}

// DIS fusion needs neither the window nor the posterior: flags from the
// iterations and the gamma count only.
__device__ __forceinline__ void finish_patch_dis(const SearchArgs &a, long long k, bool write,
                                                 float D, float u0, float last_step, bool flat,
                                                 int steps, int nvalid, int ps) {
  uint8_t flags = flat ? kFlagFlat : 0;
  if (!isfinite(D) || fabsf(D - u0) > (float)ps) flags |= kFlagDiverged;
  if (fabsf(last_step) > kConvergeTol) flags |= kFlagUnconverged;
  if (nvalid < a.nmin_valid) flags |= kFlagGamma;
  if (write BDIS_CHECKED_ONLY(&&in_bounds(k, a.total, kCheckSearchOut))) {
    a.d_star[k] = (flags & kFlagDiverged) ? u0 : D;
    a.weight[k] = 1.f;
    if (a.u_init) a.u_init[k] = u0;
    if (a.posterior) a.posterior[k] = 0.f;
    if (a.flags) a.flags[k] = flags;
    if (a.n_valid) a.n_valid[k] = nvalid;
    if (a.steps) a.steps[k] = (uint8_t)steps;
  }
}

// ------------------------------------------------------------- fast path

constexpr int pow2_at_least(int n) { return n <= 1 ? 1 : 2 * pow2_at_least((n + 1) / 2); }

// Patch size PS and a 5-sample window 0.5 px apart fixed at compile time.
// Each lane owns CPL adjacent columns of its patch (G lanes per patch), so the
// per-step work that does not scale with pixels (sample split, validity vote,
// reductions, the update) is shared by CPL * PS pixels.
//
// The right rows y0 .. y0 + PS - 1 are read through `Rows`: the packed plane
// in global memory (runtime row pitch), or a warp's staged copy in shared
// memory (row pitch fixed at compile time, so every sample is one shared load
// at an immediate offset from its column).
struct GlobalRows {
  const float2 *row0;  // row y0 of the packed right plane
  int w;
#ifdef BDIS_CHECKED
  const float2 *base;  // the whole packed plane (count * plane pairs)
  long long n;
#endif
  __device__ __forceinline__ const float2 *col(int x) const { return row0 + x; }
  // a column that is always safe to read (for lanes whose sample is unused)
  __device__ __forceinline__ const float2 *col_clamped(int x) const {
    return row0 + min(max(x, 0), w - 1);
  }
#ifdef BDIS_CHECKED
  __device__ __forceinline__ float2 ld(const float2 *p, int r) const {
    const float2 *q = p + (size_t)r * w;
    if (!in_bounds(q - base, n, kCheckSearchSample)) return make_float2(0.f, 0.f);
    return __ldg(q);
  }
#else
  __device__ __forceinline__ float2 ld(const float2 *p, int r) const {
    return __ldg(p + (size_t)r * w);
  }
#endif
  __device__ __forceinline__ void ready() const {}
};

template <int TW>
struct TileRows {
  const float2 *tile;  // shared: PS rows of TW pairs, first column `lo`
  int lo, width;       // columns lo .. lo + width - 1 are staged (the rest is never written)
  __device__ __forceinline__ const float2 *col(int x) const { return tile + (x - lo); }
  __device__ __forceinline__ const float2 *col_clamped(int x) const {
    return tile + min(max(x - lo, 0), width - 1);
  }
  __device__ __forceinline__ float2 ld(const float2 *p, int r) const { return p[r * TW]; }
  // the staging copies of this lane are complete and the warp's are visible
  __device__ __forceinline__ void ready() const {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncwarp();
  }
};

// The lane's columns of the centred gradient: in registers, or (SHARED) in
// shared memory with element (j, r) of thread t at p[(j * PS + r) * kSearchThreads]
// (p = block array + t; consecutive threads hit consecutive banks). Shared
// storage frees registers where they are the occupancy limit.
template <int PS, int CPL, bool SHARED>
struct GcStore {
  float v[CPL][PS];
  __device__ __forceinline__ float &at(int j, int r) { return v[j][r]; }
};
template <int PS, int CPL>
struct GcStore<PS, CPL, true> {
  float *p;
  __device__ __forceinline__ float &at(int j, int r) { return p[(j * PS + r) * kSearchThreads]; }
};

// Inverse-search state of one patch (the group's lanes hold the same scalars).
template <int PS, int CPL, bool SH>
struct PatchState {
  float D, last_step;
  bool frozen, flat;
  int steps;
  unsigned prev;  // valid-column code the sums below were taken over
  GcStore<PS, CPL, SH> gc;
  float invH, gcT;  // 1 / Hessian, template term of the sums
  // Within one integer base the interpolated sum is linear in the fraction:
  // sum gc (R + t dR) = A + t B, A = sum gc R, B = sum gc dR at base kc.
  float A, B;
  int kc;
};

// Sums of a patch's valid column set (bit j of `code`: the lane's column j is
// valid): centred gradient (kept in st.gc where `need`), Hessian and template
// term. Every lane of the warp takes part (group reductions); only groups
// with `need` keep the result.
template <int PS, int CPL, bool SH>
__device__ __forceinline__ void patch_sums(const SearchArgs &a, PatchState<PS, CPL, SH> &st,
                                           const bool (&act)[CPL], unsigned code, bool need,
                                           const float *Lc, const float *Gc) {
  constexpr int LANES = (PS + CPL - 1) / CPL;
  constexpr int G = pow2_at_least(LANES);
  const int w = a.w;
  bool v[CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) v[j] = (code >> j) & 1u;
  float hh, ct;
  int nn;
  if constexpr (CPL % 2 == 0) {
    // column pairs as packed f32x2; the lane's own columns are always
    // readable, and an invalid column's terms are multiplied by 0
    float2 g2[CPL / 2][PS], m2[CPL / 2], s2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int jp = 0; jp < CPL / 2; ++jp)
      m2[jp] = make_float2(v[2 * jp] ? 1.f : 0.f, v[2 * jp + 1] ? 1.f : 0.f);
#pragma unroll
    for (int jp = 0; jp < CPL / 2; ++jp)
#pragma unroll
      for (int r = 0; r < PS; ++r) {
        float ge[2];
#pragma unroll
        for (int e = 0; e < 2; ++e)
          ge[e] = act[2 * jp + e] ? BDIS_LDG(Gc + (size_t)r * w + 2 * jp + e, a.G, a.pixels,
                                               kCheckSearchRows)
                                  : 0.f;
        g2[jp][r] = make_float2(ge[0], ge[1]);
        s2 = __ffma2_rn(g2[jp][r], m2[jp], s2);  // adds g where valid, exactly
      }
    const float sg = group_sum<G>(s2.x + s2.y);
    nn = PS * group_sum_int<G>(__popc(code));
    const float mg = (a.normalize && nn > 0) ? __fdividef(sg, (float)nn) : 0.f;
    const float2 nmg = make_float2(-mg, -mg);
    float2 h2 = make_float2(0.f, 0.f), c2 = make_float2(0.f, 0.f);
#pragma unroll
    for (int jp = 0; jp < CPL / 2; ++jp) {
#pragma unroll
      for (int r = 0; r < PS; ++r) {
        const float2 q = __fmul2_rn(__fadd2_rn(g2[jp][r], nmg), m2[jp]);
        if (need) {
          st.gc.at(2 * jp, r) = q.x;
          st.gc.at(2 * jp + 1, r) = q.y;
        }
        float te[2];
#pragma unroll
        for (int e = 0; e < 2; ++e)
          te[e] = act[2 * jp + e] ? BDIS_LDG(Lc + (size_t)r * w + 2 * jp + e, a.L, a.pixels,
                                               kCheckSearchRows)
                                  : 0.f;
        h2 = __ffma2_rn(q, q, h2);
        c2 = __ffma2_rn(q, make_float2(te[0], te[1]), c2);
      }
    }
    hh = h2.x + h2.y;
    ct = c2.x + c2.y;
  } else {
    float g[CPL][PS];
    float sg = 0.f;
#pragma unroll
    for (int j = 0; j < CPL; ++j)
#pragma unroll
      for (int r = 0; r < PS; ++r) {
        g[j][r] =
            v[j] ? BDIS_LDG(Gc + (size_t)r * w + j, a.G, a.pixels, kCheckSearchRows) : 0.f;
        sg += g[j][r];
      }
    sg = group_sum<G>(sg);
    nn = PS * group_sum_int<G>(__popc(code));
    const float mg = (a.normalize && nn > 0) ? __fdividef(sg, (float)nn) : 0.f;
    hh = 0.f;
    ct = 0.f;
#pragma unroll
    for (int j = 0; j < CPL; ++j)
#pragma unroll
      for (int r = 0; r < PS; ++r) {
        const float q = v[j] ? g[j][r] - mg : 0.f;
        if (need) st.gc.at(j, r) = q;
        hh = fmaf(q, q, hh);
        ct = fmaf(q,
                  act[j] ? BDIS_LDG(Lc + (size_t)r * w + j, a.L, a.pixels, kCheckSearchRows)
                         : 0.f,
                  ct);
      }
  }
  hh = group_sum<G>(hh);
  ct = group_sum<G>(ct);
  if (need) {  // implies not frozen (frozen is the same in every lane of a group)
    st.invH = hh > 0.f ? __fdividef(1.f, hh) : 0.f;  // hh is far below 2^126
    st.gcT = ct;
    st.prev = code;
    if (nn == 0 || hh <= kFlatEps * (float)nn) {  // the Hessian and count change only here
      st.frozen = true;
      st.flat = true;
    }
  }
}

// A and B of the lane's columns at integer base kd (sample columns ib + j):
// no branches inside; an invalid column has gc = 0 and reads a clamped,
// readable column, so it adds exactly 0.
template <int PS, int CPL, bool SH, class Rows>
__device__ __forceinline__ void patch_ab(const Rows &rows, PatchState<PS, CPL, SH> &st, int ib,
                                         int kd) {
  constexpr int LANES = (PS + CPL - 1) / CPL;
  constexpr int G = pow2_at_least(LANES);
  float sa[2] = {0.f, 0.f}, sb[2] = {0.f, 0.f};
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    const auto p = rows.col_clamped(ib + j);
#pragma unroll
    for (int r = 0; r < PS; ++r) {
      const float2 q = rows.ld(p, r);
      const float g = st.gc.at(j, r);
      sa[r & 1] = fmaf(g, q.x, sa[r & 1]);
      sb[r & 1] = fmaf(g, q.y, sb[r & 1]);
    }
  }
  st.A = group_sum<G>(sa[0] + sa[1]);
  st.B = group_sum<G>(sb[0] + sb[1]);
  st.kc = kd;
}

// Valid-column code of the lane at sample base ib (x - D = ib + j + t).
template <int CPL>
__device__ __forceinline__ unsigned valid_code(const bool (&act)[CPL], int ib, float t, int w) {
  const int lb = last_base(t, w);
  unsigned code = 0u;
#pragma unroll
  for (int j = 0; j < CPL; ++j) code |= (unsigned)(act[j] && ib + j >= 0 && ib + j <= lb) << j;
  return code;
}

// The patch's D* update (Eq. 1) from the step sum; a stopped patch keeps its
// state. Stops on a non-finite D, on leaving the search range (dropped
// later) or on convergence (update below kStepTol).
template <int PS, int CPL, bool SH>
__device__ __forceinline__ void patch_update(PatchState<PS, CPL, SH> &st, float Ssum, float u0) {
  const float step = (Ssum - st.gcT) * st.invH;
  const bool live = !st.frozen;
  const float D = st.D + step;
  st.D = live ? D : st.D;
  st.last_step = live ? step : st.last_step;
  st.steps += live ? 1 : 0;
  st.frozen = !live || !isfinite(D) || fabsf(D - u0) > (float)PS || fabsf(step) < kStepTol;
}

// The first update of Eq. 1 for every patch of the warp: every patch computes
// its sums (no votes, no predicated stores).
template <int PS, int CPL, bool SH, class Rows>
__device__ __forceinline__ void search_first_step(const SearchArgs &a, const Rows &rows,
                                                  PatchState<PS, CPL, SH> &st,
                                                  const bool (&act)[CPL], int xl, const float *Lc,
                                                  const float *Gc, float u0) {
  int kd;
  float t;
  split_disp(st.D, kd, t);
  const int ib = xl + kd;
  patch_sums<PS, CPL, SH>(a, st, act, valid_code<CPL>(act, ib, t, a.w), true, Lc, Gc);
  rows.ready();  // staged rows (if any) arrive while the sums above load
  patch_ab<PS, CPL, SH>(rows, st, ib, kd);
  if (!st.frozen) patch_update<PS, CPL, SH>(st, fmaf(t, st.B, st.A), u0);
}

// A later update for every patch of the warp. Returns false, taking no step,
// when every patch of the warp has already stopped. One warp reduction
// decides what the warp recomputes:
//   - a patch whose valid column set changed (group-wise) takes new sums;
//   - A and B are re-read when some patch needs new sums or moved to another
//     integer base. A patch whose base and gradient did not change gets the
//     same sums again, so its result does not depend on its neighbours.
// The valid set can only change near the image border: while every column of
// the patch samples inside [0, w - 2] (kd in [-x0, w - 1 - PS - x0]) it is the
// full set, with no per-column tests.
template <int PS, int CPL, bool SH, class Rows>
__device__ __forceinline__ bool search_next_step(const SearchArgs &a, const Rows &rows,
                                                 PatchState<PS, CPL, SH> &st,
                                                 const bool (&act)[CPL], int xl, int x0,
                                                 unsigned full, const float *Lc,
                                                 const float *Gc, unsigned gbits, float u0) {
  int kd;
  float t;
  split_disp(st.D, kd, t);
  const int ib = xl + kd;
  unsigned code = full;
  if ((unsigned)(kd + x0) > (unsigned)(a.w - 1 - PS)) code = valid_code<CPL>(act, ib, t, a.w);
  const bool chg = !st.frozen && code != st.prev;
  const bool mv = !st.frozen && kd != st.kc;
  const unsigned r = __reduce_or_sync(kFull, (chg ? 1u : 0u) | (mv ? 2u : 0u) |
                                                 (st.frozen ? 0u : 4u));
  if (!(r & 4u)) return false;  // every patch of the warp has stopped
  if (r & 1u) {
    const bool need = (__ballot_sync(kFull, chg) & gbits) != 0u;
    patch_sums<PS, CPL, SH>(a, st, act, code, need, Lc, Gc);
  }
  if (r & 3u) patch_ab<PS, CPL, SH>(rows, st, ib, kd);
  patch_update<PS, CPL, SH>(st, fmaf(t, st.B, st.A), u0);
  return true;
}

// The window's row pass for column pairs (packed f32x2). Each of the CPL + 2
// packed pairs of a row is read once and interpolated at both fractions.
// GUARD: read only the pairs a valid column samples (the others may lie
// outside the image or the staged tile); without it every pair is in both.
// An invalid column's sums are finite and are multiplied by 0 in the merge.
template <int PS, int CPL, bool GUARD, class Rows>
__device__ __forceinline__ void window_rows_pairs(BDIS_CHECKED_ONLY(const SearchArgs &a, )
                                                  const Rows &rows, int ib, float t, float th,
                                                  bool hi, const float *Lc, int w,
                                                  const bool (&act)[CPL],
                                                  const bool (&need)[CPL + 2],
                                                  const float (&cs)[CPL],
                                                  float2 (&P1)[5][CPL / 2],
                                                  float2 (&P2)[5][CPL / 2]) {
  constexpr int S = 5;
#pragma unroll
  for (int r = 0; r < PS; ++r) {
    float Lt[CPL + 2], Lh[CPL + 2];
#pragma unroll
    for (int m = 0; m < CPL + 2; ++m) {
      const float2 q = (!GUARD || need[m]) ? rows.ld(rows.col(ib - 1 + m), r)
                                            : make_float2(0.f, 0.f);
      Lt[m] = lerp_packed(q, t);
      Lh[m] = lerp_packed(q, th);
    }
#pragma unroll
    for (int jp = 0; jp < CPL / 2; ++jp) {
      const int j = 2 * jp;
      // minus (template + shift): -(T + cs) rounds to exactly -fl(T + cs)
      float tn[2];
#pragma unroll
      for (int e = 0; e < 2; ++e)
        tn[e] = -(act[j + e] ? BDIS_LDG(Lc + (size_t)r * w + j + e, a.L, a.pixels,
                                          kCheckSearchRows)
                             : 0.f) -
                cs[j + e];
      const float2 Tn = make_float2(tn[0], tn[1]);
      // samples i = 0..4 at D* - 1, -0.5, 0, +0.5, +1: columns ib + j + 1 .. ib + j - 1
      const float2 d[S] = {
          __fadd2_rn(make_float2(Lt[j + 2], Lt[j + 3]), Tn),
          __fadd2_rn(hi ? make_float2(Lh[j + 2], Lh[j + 3]) : make_float2(Lh[j + 1], Lh[j + 2]),
                     Tn),
          __fadd2_rn(make_float2(Lt[j + 1], Lt[j + 2]), Tn),
          __fadd2_rn(hi ? make_float2(Lh[j + 1], Lh[j + 2]) : make_float2(Lh[j], Lh[j + 1]), Tn),
          __fadd2_rn(make_float2(Lt[j], Lt[j + 1]), Tn)};
#pragma unroll
      for (int i = 0; i < S; ++i) {
        P1[i][jp] = __fadd2_rn(P1[i][jp], d[i]);
        P2[i][jp] = __ffma2_rn(d[i], d[i], P2[i][jp]);
      }
    }
  }
}

template <int PS, int CPL, bool SH = false, class Rows>
__device__ __forceinline__ void fixed_patch(const SearchArgs &a, const Rows &rows, long long k,
                                            bool live, int c, unsigned gbits, int b, int x0,
                                            int y0, float u0, float *sgc = nullptr) {
  constexpr int LANES = (PS + CPL - 1) / CPL;
  constexpr int G = pow2_at_least(LANES);
  constexpr int S = 5, HALF = 2;
  const int w = a.w;
  const int xl = x0 + c * CPL;  // first column of this lane
  bool act[CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j) act[j] = (c * CPL + j) < PS;
  const long long poff = (long long)b * a.plane + (long long)y0 * w;
  const float *Lc = a.L + poff + xl;
  const float *Gc = a.G + poff + xl;

  // The template T (the lane's left columns) is read where it is used: in the
  // sums of a new valid run and in the window, not held through the steps.

  // ---- inverse-search iterations (Eq. 1)
  PatchState<PS, CPL, SH> st;
  if constexpr (SH) st.gc.p = sgc + threadIdx.x;
  st.D = u0;
  st.last_step = 0.f;
  st.frozen = st.flat = false;
  st.steps = 0;
  if (a.iters > 0) {
    unsigned full = 0u;  // the lane's columns that are part of the patch
#pragma unroll
    for (int j = 0; j < CPL; ++j) full |= (unsigned)act[j] << j;
    search_first_step<PS, CPL, SH>(a, rows, st, act, xl, Lc, Gc, u0);
    for (int it = 1; it < a.iters; ++it)
      if (!search_next_step<PS, CPL, SH>(a, rows, st, act, xl, x0, full, Lc, Gc, gbits, u0))
        break;  // every patch of the warp has stopped
  }
  const float D = st.D, last_step = st.last_step;
  const bool flat = st.flat;
  const int steps = st.steps;

  rows.ready();
  // ---- Bayesian window (Eqs. 3-4): samples at D* + {-1, -0.5, 0, 0.5, 1}
  const bool fin = isfinite(D);
  // a patch that left its search range is dropped (R8) and reads no window
  const bool inr = fin && fabsf(D - u0) <= (float)PS;
  int kd;
  float t;
  split_disp(D, kd, t);
  const int ib = xl + kd;
  // samples at D* + {-1, 0, 1} have fraction t; at D* +- 0.5 fraction th, with
  // base column one further right when t >= 0.5
  const bool hi = t >= 0.5f;
  const float th = hi ? t - 0.5f : t + 0.5f;
  const int lb = last_base(t, w);
  bool vc[CPL];
  int nv_lane = 0, nc_lane = 0;
#pragma unroll
  for (int j = 0; j < CPL; ++j) {
    nv_lane += (act[j] && fin && ib + j >= 0 && ib + j <= lb) ? 1 : 0;
    vc[j] = act[j] && inr && ib + j >= 1 && ib + j + 1 <= lb;
    nc_lane += vc[j] ? 1 : 0;
  }
  const int nvalid = PS * group_sum_int<G>(nv_lane);
  if (a.fusion == BDIS_FUSION_DIS) {
    finish_patch_dis(a, k, live && c == 0, D, u0, last_step, flat, steps, nvalid, PS);
    return;
  }
  const int nc = PS * group_sum_int<G>(nc_lane);
  // One pass over the rows. Every sample of the lane's columns lies in
  // columns ib - 1 .. ib + CPL, so per row the lane reads those CPL + 2 packed
  // pairs once and interpolates each at both fractions (t for D* and D* +- 1,
  // th for D* +- 0.5). Per column j, residuals are taken relative to a shift
  // cs[j] (the column's first-row residual at D*), which removes the
  // brightness offset between the views; the group then merges the shifted
  // sums exactly: sum (d - md)^2 = S2 - 2 (md - cs) S1 + n (md - cs)^2.
  // Pairs are read only where a valid column samples them (in bounds then).
  bool need[CPL + 2];
#pragma unroll
  for (int m = 0; m < CPL + 2; ++m)
    need[m] = (m < CPL && vc[m]) || (m >= 1 && m - 1 < CPL && vc[m - 1]) ||
              (m >= 2 && m - 2 < CPL && vc[m - 2]);
  float cs[CPL];
#pragma unroll
  for (int j = 0; j < CPL; ++j)
    cs[j] = vc[j] ? lerp_packed(rows.ld(rows.col(ib + j), 0), t) -
                        BDIS_LDG(Lc + j, a.L, a.pixels, kCheckSearchRows)
                  : 0.f;
  // Merge per sample: s1 = sum of the residuals, md their mean, and
  // E = sum (d - md)^2 = S2 - 2 (md - cs) S1 + n (md - cs)^2 per column.
  const float inv_nc = nc > 0 ? __fdividef(1.f, (float)nc) : 0.f;
  float E[S];
  if constexpr (CPL % 2 == 0) {
    // Columns j and j + 1 take the same operations, so each pair runs as one
    // packed f32x2 instruction (per component the same rounding as the scalar
    // fadd / fma): half the issue slots for the residuals and both sums.
    float2 P1[S][CPL / 2], P2[S][CPL / 2];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int jp = 0; jp < CPL / 2; ++jp) P1[i][jp] = P2[i][jp] = make_float2(0.f, 0.f);
    // A warp whose patches are all in range (so their pairs lie in a staged
    // tile, if any) with all pairs in the image reads them unconditionally.
    if (__all_sync(kFull, inr && ib >= 1 && ib + CPL <= w - 1))
      window_rows_pairs<PS, CPL, false>(BDIS_CHECKED_ONLY(a, ) rows, ib, t, th, hi, Lc, w, act,
                                        need, cs, P1, P2);
    else
      window_rows_pairs<PS, CPL, true>(BDIS_CHECKED_ONLY(a, ) rows, ib, t, th, hi, Lc, w, act,
                                       need, cs, P1, P2);
    // the merge below, per column pair; an invalid column's term is x * 0
    // (every term is finite)
    const float2 kPS = make_float2((float)PS, (float)PS), kM2 = make_float2(-2.f, -2.f);
    float2 cs2[CPL / 2], ncs2[CPL / 2], vm[CPL / 2];
#pragma unroll
    for (int jp = 0; jp < CPL / 2; ++jp) {
      cs2[jp] = make_float2(cs[2 * jp], cs[2 * jp + 1]);
      ncs2[jp] = make_float2(-cs[2 * jp], -cs[2 * jp + 1]);
      vm[jp] = make_float2(vc[2 * jp] ? 1.f : 0.f, vc[2 * jp + 1] ? 1.f : 0.f);
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      float s1 = 0.f;
#pragma unroll
      for (int jp = 0; jp < CPL / 2; ++jp) {
        const float2 x = __fmul2_rn(__ffma2_rn(kPS, cs2[jp], P1[i][jp]), vm[jp]);
        s1 += x.x + x.y;
      }
      s1 = group_sum<G>(s1);
      const float md = (a.normalize && nc > 0) ? s1 * inv_nc : 0.f;
      const float2 md2 = make_float2(md, md);
      float e = 0.f;
#pragma unroll
      for (int jp = 0; jp < CPL / 2; ++jp) {
        const float2 u = __fadd2_rn(md2, ncs2[jp]);
        const float2 in = __ffma2_rn(__fmul2_rn(kPS, u), u, P2[i][jp]);
        const float2 x = __fmul2_rn(__ffma2_rn(__fmul2_rn(kM2, u), P1[i][jp], in), vm[jp]);
        e += x.x + x.y;
      }
      E[i] = group_sum<G>(e);
    }
  } else {
    float S1[S][CPL], S2[S][CPL];
#pragma unroll
    for (int i = 0; i < S; ++i)
#pragma unroll
      for (int j = 0; j < CPL; ++j) S1[i][j] = S2[i][j] = 0.f;
#pragma unroll
    for (int r = 0; r < PS; ++r) {
      float Lt[CPL + 2], Lh[CPL + 2];
#pragma unroll
      for (int m = 0; m < CPL + 2; ++m) {
        const float2 q = need[m] ? rows.ld(rows.col(ib - 1 + m), r) : make_float2(0.f, 0.f);
        Lt[m] = lerp_packed(q, t);
        Lh[m] = lerp_packed(q, th);
      }
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        const float Tj =  // template + shift
            (vc[j] ? BDIS_LDG(Lc + (size_t)r * w + j, a.L, a.pixels, kCheckSearchRows) : 0.f) +
            cs[j];
        // samples i = 0..4 at D* - 1, -0.5, 0, +0.5, +1: columns ib + j + 1 .. ib + j - 1.
        // An invalid column's sums (finite: its pairs read as 0) are not merged below.
        const float d[S] = {Lt[j + 2] - Tj, (hi ? Lh[j + 2] : Lh[j + 1]) - Tj, Lt[j + 1] - Tj,
                            (hi ? Lh[j + 1] : Lh[j]) - Tj, Lt[j] - Tj};
#pragma unroll
        for (int i = 0; i < S; ++i) {
          S1[i][j] += d[i];
          S2[i][j] = fmaf(d[i], d[i], S2[i][j]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < S; ++i) {
      float s1 = 0.f;
#pragma unroll
      for (int j = 0; j < CPL; ++j) s1 += vc[j] ? S1[i][j] + (float)PS * cs[j] : 0.f;
      s1 = group_sum<G>(s1);
      const float md = (a.normalize && nc > 0) ? s1 * inv_nc : 0.f;
      float e = 0.f;
#pragma unroll
      for (int j = 0; j < CPL; ++j) {
        if (vc[j]) {
          const float u = md - cs[j];
          e += fmaf(-2.f * u, S1[i][j], fmaf((float)PS * u, u, S2[i][j]));
        }
      }
      E[i] = group_sum<G>(e);
    }
  }
  const bool write = live && c == 0;
  if (write && a.energies) {
#pragma unroll
    for (int i = 0; i < S; ++i) a.energies[k * S + i] = E[i];
  }
  float Emin = E[0], Eo = INFINITY;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    Emin = fminf(Emin, E[i]);
    if (i != HALF) Eo = fminf(Eo, E[i]);
  }
  const float nik = -1.4426950408889634f / a.kappa;  // exp(x / -kappa) = 2^(x log2(e) / -kappa)
  float z = 0.f, pc = 0.f;
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const float ex = exp2f((E[i] - Emin) * nik);
    z += ex;
    if (i == HALF) pc = ex;
  }
  finish_patch(a, k, write, D, u0, last_step, flat, steps, nvalid, nc, E[HALF], Eo, pc, z, PS);
}

// One patch per group, pairs on blockIdx.y, patches of a pair on blockIdx.x;
// samples read from global memory (through L1).
// SH: the centred-gradient cache in shared memory (GcStore).
template <int PS, int CPL, int MINB, bool SH>
__global__ void __launch_bounds__(kSearchThreads, MINB) search_fixed_kernel(const SearchArgs a) {
  pdl_enter();
  constexpr int LANES = (PS + CPL - 1) / CPL;
  constexpr int G = pow2_at_least(LANES);
  static_assert(G <= 32, "group size");
  const int lane = threadIdx.x & 31;
  const int c = lane & (G - 1);
  const unsigned gbits = (G == 32) ? kFull : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int kk = blockIdx.x * (blockDim.x / G) + (int)(threadIdx.x / G);
  const bool live = kk < a.np;
  const int kp = live ? kk : a.np - 1;  // past the end: redo the last patch, store nothing
  const int b = blockIdx.y;
  const long long k = (long long)b * a.np + kp;
  const int pj = a.nx_mul ? (int)__umulhi((unsigned)kp, a.nx_mul) : kp / a.nx;
  const int pi = kp - pj * a.nx;
  const int w = a.w, x0 = grid_origin(pi, a.nx, w, PS, a.stride);
  const int y0 = grid_origin(pj, a.ny, a.h, PS, a.stride);
  float u0 = 0.f;
  if (a.coarse) {
    const float cx = (float)x0 + (PS - 1) * 0.5f, cy = (float)y0 + (PS - 1) * 0.5f;
    u0 = 2.f * bilinear_clamped(a.coarse + (long long)b * a.cplane, a.cw, a.ch, cx * 0.5f,
                                cy * 0.5f);
  }
  __shared__ float sgc[SH ? CPL * PS * kSearchThreads : 1];
  fixed_patch<PS, CPL, SH>(a,
                           GlobalRows{a.R2 + (long long)b * a.plane + (long long)y0 * w,
                                      w BDIS_CHECKED_ONLY(, a.R2, a.pixels)},
                           k, live, c, gbits, b, x0, y0, u0, sgc);
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// Warp-tiled variant: a warp takes 32 / G consecutive patches of one patch-grid
// row, so they share rows y0 .. y0 + PS - 1. While a patch stays in its search
// range (|D - u0| <= PS, window +-1 px) it reads columns
// [x0 + floor(-u0 - PS) - 1, x0 + PS + floor(-u0 + PS)]; the warp stages the
// union of its patches' ranges (with one more column each side for rounding
// of the range test) into shared memory and samples from there. A warp whose
// starts spread too far for TW columns reads global memory instead; results
// are identical either way (same arithmetic in the same order). The copies
// are asynchronous and the patch waits for them only before its first sample.
// Measured on GB300 its steps run ~20% faster than the global-memory kernel's
// (lower sample latency, about the same instruction count), but staging and
// the second code path cost more per patch than that saves: 5.4 vs 4.6 ms of
// search per 128 pairs at patch size 8, so it is off by default.
template <int PS, int CPL, int MINB, int TW>
__global__ void __launch_bounds__(kSearchThreads, MINB) search_tiled_kernel(const SearchArgs a) {
  constexpr int LANES = (PS + CPL - 1) / CPL;
  constexpr int G = pow2_at_least(LANES);
  constexpr int P = 32 / G;  // patches per warp
  static_assert(G <= 32 && 32 % G == 0, "group size");
  __shared__ float2 tiles[4][PS * TW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = lane & (G - 1);
  const unsigned gbits = (G == 32) ? kFull : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int chunks = (a.nx + P - 1) / P;
  const int wid = blockIdx.x * (blockDim.x >> 5) + warp;
  if (wid >= a.ny * chunks) return;  // whole warps only
  const int pj = wid / chunks, q = wid - pj * chunks;
  const int pi_raw = q * P + lane / G;
  const bool live = pi_raw < a.nx;
  const int pi = live ? pi_raw : a.nx - 1;  // past the row end: redo its last patch, store nothing
  const int b = blockIdx.y;
  const long long k = (long long)b * a.np + (long long)pj * a.nx + pi;
  const int w = a.w, x0 = grid_origin(pi, a.nx, w, PS, a.stride);
  const int y0 = grid_origin(pj, a.ny, a.h, PS, a.stride);
  float u0 = 0.f;
  if (a.coarse) {
    const float cx = (float)x0 + (PS - 1) * 0.5f, cy = (float)y0 + (PS - 1) * 0.5f;
    u0 = 2.f * bilinear_clamped(a.coarse + (long long)b * a.cplane, a.cw, a.ch, cx * 0.5f,
                                cy * 0.5f);
  }
  const float2 *row0 = a.R2 + (long long)b * a.plane + (long long)y0 * w;
  const bool bounded = fabsf(u0) < 1.0e6f;  // false for NaN
  int lo = bounded ? x0 + (int)floorf(-u0 - (float)PS) - 3 : 0;
  int hi = bounded ? x0 + PS + (int)floorf(-u0 + (float)PS) + 2 : 0;
  lo = warp_min(lo);
  hi = warp_max(hi);
  if (__all_sync(kFull, bounded) && hi - lo < TW) {
    // asynchronous copies of the needed columns lo .. hi of the PS rows (zero
    // outside the image); fixed_patch waits for them just before the first
    // sample, so they travel while the patch's first sums load
    float2 *tile = tiles[warp];
    const int width = hi - lo + 1;
    for (int i = lane; i < PS * width; i += 32) {
      const int r = i / width, cc = i - r * width, x = lo + cc;
      const bool in = x >= 0 && x < w;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + r * TW + cc);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(dst),
                   "l"(in ? row0 + (size_t)r * w + x : row0), "r"(in ? 8 : 0));
    }
    fixed_patch<PS, CPL>(a, TileRows<TW>{tile, lo, width}, k, live, c, gbits, b, x0, y0, u0);
  } else {
    fixed_patch<PS, CPL>(a, GlobalRows{row0, w BDIS_CHECKED_ONLY(, a.R2, a.pixels)}, k, live, c,
                         gbits, b, x0, y0, u0);
  }
}

// ---------------------------------------------------------- generic path

template <int G>
__global__ void __launch_bounds__(128) search_generic_kernel(const SearchArgs a) {
  const int lane = threadIdx.x & 31;
  const int c = lane & (G - 1);
  const unsigned gbits = (G == 32) ? kFull : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const bool live = gid < a.total;
  const long long k = live ? gid : a.total - 1;
  const PatchPos pp = patch_pos(a, k);
  const int ps = a.ps, w = a.w;
  const bool act = c < ps;
  const int x = pp.x0 + (act ? c : 0);
  const long long poff = (long long)pp.b * a.plane + (long long)pp.y0 * w;
  const float *Lc = a.L + poff + x;
  const float *Gc = a.G + poff + x;
  const float2 *R2 = a.R2 + poff;

  float T[G];
#pragma unroll
  for (int r = 0; r < G; ++r)
    T[r] = (act && r < ps) ? BDIS_LDG(Lc + (size_t)r * w, a.L, a.pixels, kCheckSearchRows) : 0.f;

  const float u0 = pp.u0;
  float D = u0, last_step = 0.f;
  bool frozen = false, flat = false, have = false;
  int steps = 0;
  unsigned prev = 0u;
  float gc[G];
#pragma unroll
  for (int r = 0; r < G; ++r) gc[r] = 0.f;
  float H = 0.f, gcT = 0.f;
  int n = 0;
  for (int it = 0; it < a.iters; ++it) {
    if (__all_sync(kFull, frozen)) break;
    int kd;
    float t;
    split_disp(D, kd, t);
    const int i0 = x + kd;
    const bool v = act && sample_ok(i0, t, w);
    const unsigned m = __ballot_sync(kFull, v) & gbits;
    const bool need = !frozen && (!have || m != prev);
    if (__any_sync(kFull, need)) {
      float sg = 0.f;
#pragma unroll
      for (int r = 0; r < G; ++r)
        sg += (v && r < ps) ? BDIS_LDG(Gc + (size_t)r * w, a.G, a.pixels, kCheckSearchRows) : 0.f;
      sg = group_sum<G>(sg);
      const int nn = ps * __popc(m);
      const float mg = (a.normalize && nn > 0) ? sg / (float)nn : 0.f;
      float hh = 0.f, ct = 0.f;
#pragma unroll
      for (int r = 0; r < G; ++r) {
        const float q =
            (v && r < ps) ? BDIS_LDG(Gc + (size_t)r * w, a.G, a.pixels, kCheckSearchRows) - mg
                          : 0.f;
        if (need) gc[r] = q;
        hh = fmaf(q, q, hh);
        ct = fmaf(q, T[r], ct);
      }
      hh = group_sum<G>(hh);
      ct = group_sum<G>(ct);
      if (need) {
        H = hh;
        gcT = ct;
        n = nn;
        prev = m;
        have = true;
      }
    }
    if (!frozen && (n == 0 || H <= kFlatEps * (float)n)) {
      frozen = true;
      flat = true;
    }
    float acc = 0.f;
    if (v && !frozen) {
      const float2 *p = R2 + i0;
#pragma unroll
      for (int r = 0; r < G; ++r)
        if (r < ps) acc = fmaf(gc[r], lerp_packed(__ldg(p + (size_t)r * w), t), acc);
    }
    const float Ssum = group_sum<G>(acc);
    if (!frozen) {
      last_step = (Ssum - gcT) / H;
      D += last_step;
      ++steps;
      if (!isfinite(D) || fabsf(D - u0) > (float)ps || fabsf(last_step) < kStepTol)
        frozen = true;
    }
  }

  const bool fin = isfinite(D);
  int kd;
  float t;
  split_disp(D, kd, t);
  const bool v0 = act && fin && sample_ok(x + kd, t, w);
  const int nvalid = ps * __popc(__ballot_sync(kFull, v0) & gbits);
  if (a.fusion == BDIS_FUSION_DIS) {
    finish_patch_dis(a, k, live && c == 0, D, u0, last_step, flat, steps, nvalid, ps);
    return;
  }
  const int half = (a.s - 1) / 2;
  bool vc = act && fin && fabsf(D - u0) <= (float)ps;  // a diverged patch reads no window
  for (int i = 0; i < a.s; ++i) {
    split_disp(D + (float)(i - half) * a.step, kd, t);
    vc = vc && sample_ok(x + kd, t, w);
  }
  const int nc = ps * __popc(__ballot_sync(kFull, vc) & gbits);
  const bool write = live && c == 0;
  // window energies; the normaliser z is accumulated relative to the running
  // minimum and rescaled when the minimum drops
  float Ec = 0.f, Eo = INFINITY, Emin = INFINITY, z = 0.f;
  for (int i = 0; i < a.s; ++i) {
    split_disp(D + (float)(i - half) * a.step, kd, t);
    float dres[G];
    float sd = 0.f;
#pragma unroll
    for (int r = 0; r < G; ++r) {
      dres[r] = (vc && r < ps) ? lerp_packed(__ldg(R2 + (x + kd) + (size_t)r * w), t) - T[r]
                               : 0.f;
      sd += dres[r];
    }
    float md = 0.f;
    if (a.normalize) {
      sd = group_sum<G>(sd);
      md = nc > 0 ? sd / (float)nc : 0.f;
    }
    float e = 0.f;
#pragma unroll
    for (int r = 0; r < G; ++r) {
      const float q = (vc && r < ps) ? dres[r] - md : 0.f;
      e = fmaf(q, q, e);
    }
    const float E = group_sum<G>(e);
    if (write && a.energies) a.energies[k * a.s + i] = E;
    if (i == half)
      Ec = E;
    else
      Eo = fminf(Eo, E);
    if (E < Emin) {
      z = (Emin == INFINITY ? 0.f : z * expf(-(Emin - E) / a.kappa)) + 1.f;
      Emin = E;
    } else {
      z += expf(-(E - Emin) / a.kappa);
    }
  }
  finish_patch(a, k, write, D, u0, last_step, flat, steps, nvalid, nc, Ec, Eo,
               expf(-(Ec - Emin) / a.kappa), z, ps);
}

template <int PS, int CPL, int MINB, bool SH = false>
cudaError_t launch_fixed(const SearchArgs &a, cudaStream_t st) {
  constexpr int G = pow2_at_least((PS + CPL - 1) / CPL);
  const int threads = a.block_threads == 64 ? 64 : 128, per_block = threads / G;
  const int count = (int)(a.total / a.np);
  const dim3 grid((unsigned)((a.np + per_block - 1) / per_block), (unsigned)count);
  return launch_maybe_overlapped(search_fixed_kernel<PS, CPL, MINB, SH>, grid, dim3(threads), 0, st,
                                 a);
}

template <int PS, int CPL, int MINB>
cudaError_t launch_tiled(const SearchArgs &a, cudaStream_t st) {
  constexpr int G = pow2_at_least((PS + CPL - 1) / CPL), P = 32 / G;
  constexpr int TW = (PS == 8 && CPL <= 2) ? 64 : 96;  // 4 warps x PS x TW x 8 B <= 48 KB
  const int threads = a.block_threads == 64 ? 64 : 128, wpb = threads / 32;
  const long long warps = (long long)a.ny * ((a.nx + P - 1) / P);
  const int count = (int)(a.total / a.np);
  const dim3 grid((unsigned)((warps + wpb - 1) / wpb), (unsigned)count);
  search_tiled_kernel<PS, CPL, MINB, TW><<<grid, threads, 0, st>>>(a);
  return cudaGetLastError();
}

template <int PS, int CPL, int MINB>
cudaError_t launch_fast(const SearchArgs &a, cudaStream_t st) {
  return a.tiled ? launch_tiled<PS, CPL, MINB>(a, st) : launch_fixed<PS, CPL, MINB>(a, st);
}

template <typename K>
cudaError_t launch_groups(K kernel, int G, const SearchArgs &a, cudaStream_t st) {  // 1-D grid
  const int threads = 128;
  const long long lanes = a.total * G;
  const unsigned blocks = (unsigned)((lanes + threads - 1) / threads);
  kernel<<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

// R16: keep the seeded result of a coarsest patch only if it is kept and the
// plain result is dropped or has no higher posterior; otherwise take the plain.
__global__ void select_start_kernel(float *__restrict__ d_a, float *__restrict__ w_a,
                                    const float *__restrict__ p_a, const uint8_t *__restrict__ f_a,
                                    const float *__restrict__ d_b, const float *__restrict__ w_b,
                                    const float *__restrict__ p_b, const uint8_t *__restrict__ f_b,
                                    long long total) {
  pdl_enter();
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const bool kept_a = !(f_a[k] & kDropFlags), kept_b = !(f_b[k] & kDropFlags);
  // both kept and this close: the two searches found one solution; the plain one stands
  const bool same = kept_a && kept_b && fabsf(d_a[k] - d_b[k]) <= kSameSolution;
  const bool keep_a = !same && kept_a && (!kept_b || p_a[k] >= p_b[k]);
  if (!keep_a) {
    d_a[k] = d_b[k];
    w_a[k] = w_b[k];
  }
}

}  // namespace

cudaError_t launch_select_start(float *d_a, float *w_a, const float *p_a, const uint8_t *f_a,
                                const float *d_b, const float *w_b, const float *p_b,
                                const uint8_t *f_b, long long total, cudaStream_t st) {
  if (total == 0) return cudaSuccess;
  return launch_maybe_overlapped(select_start_kernel, dim3((unsigned)((total + 255) / 256)),
                                 dim3(256), 0, st, d_a, w_a, p_a, f_a, d_b, w_b, p_b, f_b, total);
}

namespace {
int g_cols_per_lane = 2;  // process-wide choice of the fast-path variant
int g_tiled = 0;          // fast path: warp-tiled shared-memory sampling (off: slower)
}  // namespace

int search_cols_per_lane() { return g_cols_per_lane; }
void set_search_cols_per_lane(int cpl) { g_cols_per_lane = cpl; }
int search_tiled() { return g_tiled; }
void set_search_tiled(int on) { g_tiled = on ? 1 : 0; }

void fill_search_args(SearchArgs &a, int w, int h, int count, const bdis_params &p) {
  a.w = w;
  a.h = h;
  a.plane = (long long)w * h;
  a.ps = p.patch_size;
  a.stride = grid_stride(p.patch_size, p.overlap);
  a.nx = grid_count(w, p.patch_size, a.stride);
  a.ny = grid_count(h, p.patch_size, a.stride);
  a.np = a.nx * a.ny;
  // m = ceil(2^32 / nx) = (2^32 + e) / nx gives k m / 2^32 = k / nx + k e / (nx 2^32),
  // whose floor is floor(k / nx) while k e < 2^32 (the remainder is at most nx - 1)
  a.nx_mul = 0;
  if (a.nx >= 2) {
    const unsigned long long m = ((1ull << 32) + (unsigned long long)a.nx - 1) / a.nx;
    const unsigned long long e = m * (unsigned long long)a.nx - (1ull << 32);
    if ((unsigned long long)(a.np - 1) * e < (1ull << 32)) a.nx_mul = (unsigned)m;
  }
  a.total = (long long)a.np * count;
  a.pixels = a.plane * count;
  a.iters = p.iterations;
  a.s = p.window_samples;
  a.step = p.window_step;
  a.kappa = 2.f * p.sigma_r * p.sigma_r * (float)(p.window_samples * p.window_samples);
  a.nmin_valid = gamma_min_count(p.gamma, p.patch_size);
  a.normalize = p.normalize ? 1 : 0;
  a.cols_per_lane = search_cols_per_lane();
  a.tiled = search_tiled();
  a.fusion = p.fusion;
}

cudaError_t launch_search(const SearchArgs &args, cudaStream_t st) {
  if (args.total == 0) return cudaSuccess;
  SearchArgs a = args;
  a.debug = (a.u_init || a.posterior || a.flags || a.n_valid || a.steps || a.energies) ? 1 : 0;
  const int count = (int)(a.total / a.np);
  if (a.s == 5 && a.step == 0.5f && count <= 65535) {
    const int cpl = a.cols_per_lane;
    if (a.ps == 8) {
      if (cpl == 1) return launch_fast<8, 1, 8>(a, st);
      if (cpl == 4) return launch_fast<8, 4, 4>(a, st);
      // 64 registers with the gradient cache in shared memory: 8 blocks of 128 per SM
      // (the tiled variant keeps it in registers at 72: 7 blocks)
      return a.tiled ? launch_tiled<8, 2, 7>(a, st) : launch_fixed<8, 2, 8, true>(a, st);
    }
    if (a.ps == 12) return cpl == 1 ? launch_fast<12, 1, 4>(a, st) : launch_fast<12, 3, 3>(a, st);
    if (a.ps == 16) return cpl == 1 ? launch_fast<16, 1, 4>(a, st) : launch_fast<16, 2, 3>(a, st);
  }
  if (a.ps <= 4) return launch_groups(search_generic_kernel<4>, 4, a, st);
  if (a.ps <= 8) return launch_groups(search_generic_kernel<8>, 8, a, st);
  if (a.ps <= 16) return launch_groups(search_generic_kernel<16>, 16, a, st);
  return launch_groups(search_generic_kernel<32>, 32, a, st);
}

cudaError_t take_check_search(unsigned *v) { return take_check_word(v); }

}  // namespace bdis
