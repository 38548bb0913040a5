// densify.cu -- fusion of the patch disparities into a dense map (Sec. 2.3).
//
// Each pixel takes its covering patches straight from the regular grid (no
// scatter, no atomics): w = weight_k * m(x - x0_k) * m(y - y0_k), where the
// Gaussian mask m (Eq. 5, sigma_s) is separable and depends only on the
// position inside the patch. The pixel's disparity is sum w D*_k / sum w (the
// normalised form of Eq. 2 with the combined posterior as weight). Pixels
// without a kept patch are NaN at the finest level (Sec. 3.2: not
// estimated); coarser levels carry the value their patches started from.
//
// Because the mask is separable, a block computes a 32x32 tile in two passes
// through shared memory: first, for every patch row that touches the tile
// and every tile column, the x-weighted sums over the covering patches of
// that row (sum m_x (w D) and sum m_x w, w D formed once per patch); then,
// per pixel, the y-weighted sum of those over its covering rows. Work per pixel drops from (ps/stride)^2 to
// about 2 ps/stride multiply-adds per quantity.
//
// Roofline: DRAM bytes per pixel: 4 written (+4 read for the coarse map where
// carried) plus the patch arrays (8 B per patch) read once per tile.
#include "bdis_internal.cuh"

namespace bdis {
namespace {

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

// Patches covering coordinate x along one axis: the regular ones
// [lo, hi] (indices <= n - 2) plus the last one (origin n_px - ps) if it covers.
__device__ __forceinline__ void cover_range(int x, int n_px, int ps, int stride, int n, int &lo,
                                            int &hi, int &last) {
  const int a = x - ps + 1;
  lo = a <= 0 ? 0 : (a + stride - 1) / stride;
  hi = min(x / stride, n - 2);
  last = (x >= n_px - ps) ? 1 : 0;
}

constexpr int kTileX = 32, kTileY = 32, kMaxRows = kTileY + kMaxPatch;

__global__ void __launch_bounds__(256) densify_kernel(const DensifyArgs a) {
  __shared__ float mask[kMaxPatch];
  __shared__ float sA[kMaxRows][kTileX], sB[kMaxRows][kTileX];
  const int tid = threadIdx.x;
  if (tid < a.ps) {
    const float m = (float)tid - (a.ps - 1) * 0.5f;
    mask[tid] = expf(-(m * m) / a.two_s2);
  }
  const int b = blockIdx.z;
  const int tile_y = a.tile_y > 0 ? a.tile_y : kTileY;  // 8, 16 or 32
  const int X0 = blockIdx.x * kTileX, Y0 = blockIdx.y * tile_y;
  const int ylast = min(Y0 + tile_y, a.h) - 1;
  // patch rows touching the tile: regular rows [jlo, jhi] and maybe the last
  int jlo, jhi, jl_unused, hlast_lo, hlast_hi;
  cover_range(Y0, a.h, a.ps, a.stride, a.ny, jlo, jl_unused, hlast_lo);
  cover_range(ylast, a.h, a.ps, a.stride, a.ny, jl_unused, jhi, hlast_hi);
  const int nreg = max(0, jhi - jlo + 1);
  const int has_last = hlast_hi;  // the last row covers the bottom of the tile if any
  const int nrows = nreg + has_last;
  const float *wp = a.weight + (long long)b * a.np;
  const float *dp = a.d_star + (long long)b * a.np;
  __syncthreads();

  // pass 1: x-weighted sums per (patch row, tile column)
  for (int q = tid; q < nrows * kTileX; q += blockDim.x) {
    const int jj = q / kTileX, xx = q - jj * kTileX;
    const int x = X0 + xx;
    float A = 0.f, B = 0.f;
    if (x < a.w) {
      const int j = jj < nreg ? jlo + jj : a.ny - 1;
      int ilo, ihi, ilast;
      cover_range(x, a.w, a.ps, a.stride, a.nx, ilo, ihi, ilast);
      const float *wr = wp + (long long)j * a.nx;
      const float *dr = dp + (long long)j * a.nx;
      for (int ii = ilo; ii <= ihi + ilast; ++ii) {
        const int i = ii > ihi ? a.nx - 1 : ii;
        const float wk = __ldg(wr + i);
        if (wk > 0.f) {  // a dropped patch has weight 0 (its D* may be NaN)
          const float mx = mask[x - grid_origin(i, a.nx, a.w, a.ps, a.stride)];
          A = fmaf(mx, wk * __ldg(dr + i), A);
          B = fmaf(mx, wk, B);
        }
      }
    }
    sA[jj][xx] = A;
    sB[jj][xx] = B;
  }
  __syncthreads();

  // pass 2: y-weighted sums over the covering rows of each pixel
  const int xx = tid & (kTileX - 1);
  const int x = X0 + xx;
  for (int yy = tid / kTileX; yy < tile_y; yy += blockDim.x / kTileX) {
    const int y = Y0 + yy;
    if (x >= a.w || y >= a.h) continue;
    int lo, hi, last;
    cover_range(y, a.h, a.ps, a.stride, a.ny, lo, hi, last);
    float num = 0.f, den = 0.f;
    for (int j = lo; j <= hi + last; ++j) {
      const int row = j > hi ? a.ny - 1 : j;  // past the regular rows: the last row
      const int jj = j > hi ? nreg : j - jlo;
      const float my = mask[y - grid_origin(row, a.ny, a.h, a.ps, a.stride)];
      num = fmaf(my, sA[jj][xx], num);
      den = fmaf(my, sB[jj][xx], den);
    }
    float out;
    if (den > 0.f)
      out = __fdividef(num, den);  // den >= the smallest mask weight, far below 2^126
    else if (a.is_finest)
      out = __int_as_float(0x7fc00000);  // NaN: not estimated
    else if (a.coarse)
      out = 2.f * bilinear_clamped(a.coarse + (long long)b * a.cplane, a.cw, a.ch, x * 0.5f,
                                   y * 0.5f);
    else
      out = 0.f;
    a.out[(long long)b * a.plane + (long long)y * a.w + x] = out;
  }
}

// Strip variant for patch grids whose stride S divides the patch size PS
// (M = PS / S covering patch rows per pixel row; overlap 0.75 gives M = 4 for
// PS 8, 12 and 16). A thread owns one column and a strip of K pixel rows. The
// pixel rows of group g (rows gS .. gS + S - 1) are covered by the same M
// regular patch rows g - M + 1 .. g (those in [0, ny - 2]) plus, near the
// bottom, the last patch row (origin h - PS). Walking down the strip one group
// at a time adds one regular patch row, so each thread computes the x-weighted
// sums A_j, B_j of one new patch row per group and keeps the last M in
// registers; the y-weighted sums then take them in ascending j, as the tiled
// kernel does, with the same operations, so the two give identical results.
// The block's patch values are staged in shared memory once (one barrier);
// a warp's reads of them (19 patches of a row for 32 columns) are broadcasts.
// The y weights sit in registers (PS / 2 of them: the mask is symmetric). At
// PS 8 the kernel runs at up to 72 registers, 7 blocks of 128 per SM, which
// measured faster than 8 blocks at 64.
template <int PS, int S, int K>
__global__ void __launch_bounds__(128, PS == 8 ? 7 : 6) densify_strip_kernel(const DensifyArgs a) {
  constexpr int M = PS / S;
  static_assert(M * S == PS && K % S == 0, "strip geometry");
  // patch columns / rows a block (128 columns x K rows) can need, plus one
  // slot each for the last (irregular) patch column / row
  constexpr int NCMAX = (128 + S - 1) / S + M + 2, NRMAX = K / S + M + 1;
  // Whatever the image size, a block's regular patch columns number at most
  // (126 + PS) / S + 1 (all of [ilo(X0), ihi(X0 + 127)]) and its regular rows
  // at most K / S + M - 1 (rows g0 - M + 1 .. g0 + K / S - 1): with the last
  // column / row slot they fit the tile.
  static_assert((126 + PS) / S + 1 + 1 <= NCMAX && K / S + M - 1 + 1 <= NRMAX, "tile bounds");
  // column ZC is never a patch column: it holds (0, 0), the value of a patch
  // that does not cover the pixel
  constexpr int ZC = NCMAX - 1;
  static_assert((126 + PS) / S + 1 + 1 <= ZC, "zero column");
  // staged patch values as (w D*, w) pairs; a dropped patch (w <= 0) as (0, 0)
  __shared__ float2 swd[NRMAX][NCMAX];
  __shared__ float smask[PS];
  pdl_enter();
  const int X0 = blockIdx.x * 128, x = X0 + (int)threadIdx.x;
  const int Y0 = blockIdx.y * K, b = blockIdx.z;
  const bool active = x < a.w;
  const float *wp = a.weight + (long long)b * a.np;
  const float *dp = a.d_star + (long long)b * a.np;
  // The block's patch rows and columns are staged into shared memory with
  // asynchronous copies, all in flight at once (one round trip per block).
  const int xlast_b = min(X0 + 127, a.w - 1);
  const int g0 = Y0 / S, gend = (min(Y0 + K, a.h) - 1) / S;
  const int ic0 = X0 - PS + 1 <= 0 ? 0 : (X0 - PS + 1 + S - 1) / S;
  const int ic1 = min(xlast_b / S, a.nx - 2);
  const int jr0 = max(0, g0 - M + 1), jr1 = min(gend, a.ny - 2);
  const int NC = max(0, ic1 - ic0 + 1), NR = max(0, jr1 - jr0 + 1);
  {
    // thread cc copies column cc of every tile row (NC + 1 <= NCMAX < 128
    // columns): no per-element division, one column index per thread
    static_assert(NCMAX <= 128, "one tile column per thread");
    const int cc = threadIdx.x;
    if (cc <= NC) {
      const int i = cc < NC ? ic0 + cc : a.nx - 1;
      const unsigned dd0 = (unsigned)__cvta_generic_to_shared(&swd[0][cc].x);
      for (int rr = 0; rr <= NR; ++rr) {
        const int j = rr < NR ? jr0 + rr : a.ny - 1;
        const long long o = (long long)j * a.nx + i;
        const unsigned step = (unsigned)(rr * NCMAX * sizeof(float2));
        BDIS_CHECKED_ONLY(if (!in_bounds(o, a.np, kCheckDensifyTile)) {
          swd[rr][cc] = make_float2(0.f, 0.f);
          continue;
        })
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dd0 + step), "l"(dp + o));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dd0 + step + 4),
                     "l"(wp + o));
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");
      // the thread's own copies are complete: form (w D*, w), as the tiled kernel does
      for (int rr = 0; rr <= NR; ++rr) {
        const float2 v = swd[rr][cc];  // (D*, w)
        swd[rr][cc] = v.y > 0.f ? make_float2(v.y * v.x, v.y) : make_float2(0.f, 0.f);
      }
    } else if (cc == ZC) {
      for (int rr = 0; rr <= NR; ++rr) swd[rr][ZC] = make_float2(0.f, 0.f);
    }
  }
  if (threadIdx.x < PS) {  // Gaussian mask (Eq. 5): the tiled kernel's expression and values
    const float m = (float)threadIdx.x - (PS - 1) * 0.5f;
    smask[threadIdx.x] = expf(-(m * m) / a.two_s2);
  }
  __syncthreads();
  if (!active || Y0 >= a.h) return;
  auto mask_at = [&](int q) { return smask[q]; };
  // covering patches of column x: regular ilo .. ihi (<= nx - 2), then the last;
  // their x weights are fixed for the thread
  const int ilo = x - PS + 1 <= 0 ? 0 : (x - PS + 1 + S - 1) / S;
  const int ihi = min(x / S, a.nx - 2);
  const bool ilast = x >= a.w - PS;
  float mxr[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) {
    const int q = x - (ilo + k) * S;
    mxr[k] = (q >= 0 && q < PS) ? mask_at(q) : 0.f;
  }
  const float mxl = ilast ? mask_at(x - (a.w - PS)) : 0.f;
  // covering patch k of column x (k = 0..M: the regular ilo + k, then the
  // last): its tile column (ZC where there is none) and its x weight
  int cck[M + 1];
  float mxk[M + 1];
#pragma unroll
  for (int k = 0; k <= M; ++k) {
    const int ii = ilo + k;
    const bool reg = ii <= ihi;
    cck[k] = reg ? ii - ic0 : (ilast && ii == ihi + 1) ? NC : ZC;
    mxk[k] = reg ? mxr[k] : mxl;
  }
  // a patch row's (w D*, w) pairs (staged; read one row ahead of their use)
  // and its x-weighted sums, in the same order and with the same fmas as the
  // tiled kernel: a patch that is not used, or dropped, is (0, 0) and adds
  // exactly 0
  auto load_row = [&](int j, float2 *v) {
    const float2 *row = swd[j <= a.ny - 2 ? j - jr0 : NR];
#pragma unroll
    for (int k = 0; k <= M; ++k) v[k] = row[cck[k]];
  };
  auto sum_row = [&](const float2 *v, float2 &AB) {
    AB = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k <= M; ++k) AB = __ffma2_rn(make_float2(mxk[k], mxk[k]), v[k], AB);
  };
  auto row_sums = [&](int j, float2 &AB) {
    float2 v[M + 1];
    load_row(j, v);
    sum_row(v, AB);
  };
  const int ylast = a.h - PS;  // first pixel row the last patch row covers
  float2 last = make_float2(0.f, 0.f);
  bool have_last = false;
  // ring of the regular rows g - M + 1 .. g (slot k holds row g - M + 1 + k),
  // each as its (x-weighted numerator, denominator) pair
  float2 rAB[M];
#pragma unroll
  for (int k = 0; k < M - 1; ++k) {
    const int j = g0 - M + 1 + k;
    rAB[k + 1] = make_float2(0.f, 0.f);
    if (j >= 0 && j <= a.ny - 2) row_sums(j, rAB[k + 1]);
  }

  const long long obase = (long long)b * a.plane + x;
  const int yend = min(Y0 + K, a.h);
  // the y weights of the group's rows, in registers: the mask is symmetric
  // (its offsets from the centre are +-m), so PS / 2 values hold it
  float myr[PS / 2];
#pragma unroll
  for (int q = 0; q < PS / 2; ++q) myr[q] = smask[q];
  float2 nv[M + 1];  // row g's loads, issued during group g - 1
  if (g0 <= a.ny - 2) load_row(g0, nv);
  for (int g = g0; g * S < yend; ++g) {
    float2 cv[M + 1];
#pragma unroll
    for (int k = 0; k <= M; ++k) cv[k] = nv[k];
    if (g + 1 <= a.ny - 2 && (g + 1) * S < yend) load_row(g + 1, nv);
#pragma unroll
    for (int k = 0; k < M - 1; ++k) rAB[k] = rAB[k + 1];
    rAB[M - 1] = make_float2(0.f, 0.f);
    if (g <= a.ny - 2) sum_row(cv, rAB[M - 1]);
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const int y = g * S + t;
      if (y >= yend) break;
      // (numerator, denominator) as one packed f32x2 FMA per covering row:
      // per component the same fma as the tiled kernel; a ring slot outside
      // the regular rows holds (0, 0) and adds exactly 0
      float2 nd2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        const int q = t + (M - 1 - k) * S;  // known at compile time (unrolled)
        const float my = myr[q < PS / 2 ? q : PS - 1 - q];
        nd2 = __ffma2_rn(make_float2(my, my), rAB[k], nd2);
      }
      if (y >= ylast) {
        if (!have_last) {
          row_sums(a.ny - 1, last);
          have_last = true;
        }
        const float my = mask_at(y - ylast);
        nd2 = __ffma2_rn(make_float2(my, my), last, nd2);
      }
      const float num = nd2.x, den = nd2.y;
      float out;
      if (den > 0.f)
        out = __fdividef(num, den);  // den >= the smallest mask weight, far below 2^126
      else if (a.is_finest)
        out = __int_as_float(0x7fc00000);  // NaN: not estimated
      else if (a.coarse)
        out = 2.f * bilinear_clamped(a.coarse + (long long)b * a.cplane, a.cw, a.ch, x * 0.5f,
                                     y * 0.5f);
      else
        out = 0.f;
      BDIS_CHECKED_ONLY(if (!in_bounds(obase + (long long)y * a.w, a.total, kCheckDensifyOut))
                            continue;)
      a.out[obase + (long long)y * a.w] = out;
    }
  }
}

// DIS fusion (Eq. 2): per pixel, every covering patch whose sample x - D*_k is
// inside the right image, weighted by weight_k / max(r^2, 1) with r the
// photometric residual R(x - D*_k) - L(x). The weights depend on the pixel
// and the patch jointly, so this is a direct gather over the covering patches.
__global__ void __launch_bounds__(256) densify_dis_kernel(const DensifyArgs a) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= a.total) return;
  const int b = (int)(idx / a.plane);
  const int rem = (int)(idx - (long long)b * a.plane);
  const int y = rem / a.w, x = rem - (rem / a.w) * a.w;
  int ilo, ihi, ilast, jlo, jhi, jlast;
  cover_range(x, a.w, a.ps, a.stride, a.nx, ilo, ihi, ilast);
  cover_range(y, a.h, a.ps, a.stride, a.ny, jlo, jhi, jlast);
  const float *wp = a.weight + (long long)b * a.np;
  const float *dp = a.d_star + (long long)b * a.np;
  const float2 *Rrow = a.R2 + (long long)b * a.plane + (long long)y * a.w;
  const float Lx = __ldg(a.L + (long long)b * a.plane + (long long)y * a.w + x);
  float num = 0.f, den = 0.f;
  for (int jj = jlo; jj <= jhi + jlast; ++jj) {
    const int j = jj > jhi ? a.ny - 1 : jj;
    for (int ii = ilo; ii <= ihi + ilast; ++ii) {
      const int i = ii > ihi ? a.nx - 1 : ii;
      const int kk = j * a.nx + i;
      const float wk = __ldg(wp + kk);
      if (!(wk > 0.f)) continue;
      const float D = __ldg(dp + kk);
      const float nd = fminf(fmaxf(-D, -1.0e7f), 1.0e7f);
      const float f = floorf(nd);
      const int i0 = x + (int)f;
      const float t = nd - f;
      if (!(i0 >= 0 && (i0 < a.w - 1 || (i0 == a.w - 1 && t == 0.f)))) continue;
      const float2 q = __ldg(Rrow + i0);
      const float r = fmaf(t, q.y, q.x) - Lx;
      const float wpx = wk / fmaxf(r * r, 1.f);
      num = fmaf(wpx, D, num);
      den += wpx;
    }
  }
  float out;
  if (den > 0.f)
    out = __fdividef(num, den);  // den >= the smallest mask weight, far below 2^126
  else if (a.is_finest)
    out = __int_as_float(0x7fc00000);
  else if (a.coarse)
    out = 2.f * bilinear_clamped(a.coarse + (long long)b * a.cplane, a.cw, a.ch, x * 0.5f,
                                 y * 0.5f);
  else
    out = 0.f;
  a.out[idx] = out;
}

// Full-size map from level f: bilinear over finite neighbours with positive
// weight, values times 2^f.
__global__ void upsample_kernel(const float *__restrict__ M, int mw, int mh, float scale, int w,
                                int h, long long total, float *__restrict__ out) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long plane = (long long)w * h;
  const int b = (int)(idx / plane);
  const int rem = (int)(idx - (long long)b * plane);
  const int y = rem / w, x = rem - (rem / w) * w;
  const float *Mb = M + (long long)b * mw * mh;
  float fx = fminf((float)x / scale, (float)(mw - 1));
  float fy = fminf((float)y / scale, (float)(mh - 1));
  const int x0 = (int)floorf(fx), y0 = (int)floorf(fy);
  const int x1 = min(x0 + 1, mw - 1), y1 = min(y0 + 1, mh - 1);
  const float tx = fx - x0, ty = fy - y0;
  const float wt[4] = {(1.f - tx) * (1.f - ty), tx * (1.f - ty), (1.f - tx) * ty, tx * ty};
  const float v[4] = {Mb[(size_t)y0 * mw + x0], Mb[(size_t)y0 * mw + x1],
                      Mb[(size_t)y1 * mw + x0], Mb[(size_t)y1 * mw + x1]};
  float s = 0.f, sw = 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (wt[q] > 0.f && isfinite(v[q])) {
      s += wt[q] * v[q];
      sw += wt[q];
    }
  out[idx] = sw > 0.f ? scale * s / sw : __int_as_float(0x7fc00000);
}

// R15 warm start: level-`level` seed map from a previous full-size disparity:
// mean of its finite values over the 2^level block centred on the sample
// point, divided by 2^level; 0 where none is finite.
__global__ void warm_map_kernel(const float *__restrict__ P, int w, int h, int level, int mw,
                                int mh, long long total, float *__restrict__ out) {
  pdl_enter();
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long mplane = (long long)mw * mh;
  const int b = (int)(idx / mplane);
  const int rem = (int)(idx - (long long)b * mplane);
  const int Y = rem / mw, X = rem - (rem / mw) * mw;
  const int s = 1 << level;
  const int half = s / 2;
  const int x0 = max(X * s - half, 0), x1 = min(X * s + half + (s == 1 ? 1 : 0), w);
  const int y0 = max(Y * s - half, 0), y1 = min(Y * s + half + (s == 1 ? 1 : 0), h);
  const float *Pb = P + (long long)b * w * h;
  float sum = 0.f;
  int n = 0;
  for (int y = y0; y < y1; ++y)
    for (int x = x0; x < x1; ++x) {
      const float v = __ldg(Pb + (size_t)y * w + x);
      if (isfinite(v)) {
        sum += v;
        ++n;
      }
    }
  out[idx] = n ? sum / (float)n / (float)s : 0.f;
}

}  // namespace

cudaError_t launch_warm_map(const float *prev, int w, int h, int level, int count, float *out,
                            cudaStream_t st) {
  const int mw = level_dim(w, level), mh = level_dim(h, level);
  const long long total = (long long)mw * mh * count;
  if (total == 0) return cudaSuccess;
  const int threads = 128;
  return launch_maybe_overlapped(warm_map_kernel, dim3((unsigned)((total + threads - 1) / threads)),
                                 dim3(threads), 0, st, prev, w, h, level, mw, mh, total, out);
}

namespace {
int g_densify_tile = 0;  // process-wide densify kernel choice (0 = strips where they apply)
}  // namespace

int densify_tile() { return g_densify_tile; }
void set_densify_tile(int tile_height) { g_densify_tile = tile_height; }

void fill_densify_args(DensifyArgs &a, int w, int h, int count, const bdis_params &p) {
  a.tile_y = g_densify_tile;
  a.w = w;
  a.h = h;
  a.plane = (long long)w * h;
  a.total = a.plane * count;
  a.ps = p.patch_size;
  a.stride = grid_stride(p.patch_size, p.overlap);
  a.nx = grid_count(w, p.patch_size, a.stride);
  a.ny = grid_count(h, p.patch_size, a.stride);
  a.np = a.nx * a.ny;
  a.two_s2 = 2.f * p.sigma_s * p.sigma_s;
  a.fusion = p.fusion;
}

cudaError_t launch_densify(const DensifyArgs &a, cudaStream_t st) {
  if (a.total == 0) return cudaSuccess;
  if (a.fusion == BDIS_FUSION_DIS) {
    const int threads = 256;
    densify_dis_kernel<<<(unsigned)((a.total + threads - 1) / threads), threads, 0, st>>>(a);
    return cudaGetLastError();
  }
  const int count = (int)(a.total / a.plane);
  if (a.tile_y == 0 && a.nx > 0 && a.ny > 0) {  // default: strips where the geometry allows
    // A thread walks its column down a strip of K rows, one dependent step
    // per group of S rows, so a launch takes at least one strip's walk. Where
    // strips of 32 rows would not give every SM two blocks (small levels,
    // small batches), strips of 8 (9) rows spread the same rows over four
    // times the blocks. The map is the same either way: each row's
    // x-weighted sums depend only on the row and the column.
    const unsigned bx = (unsigned)((a.w + 127) / 128);
    const bool short_strips = (long long)bx * ((a.h + 31) / 32) * count < 2LL * device_sms();
    auto rows = [&](int K) { return dim3(bx, (unsigned)((a.h + K - 1) / K), (unsigned)count); };
    if (a.ps == 8 && a.stride == 2)
      return short_strips ? launch_maybe_overlapped(densify_strip_kernel<8, 2, 8>, rows(8),
                                                    dim3(128), 0, st, a)
                          : launch_maybe_overlapped(densify_strip_kernel<8, 2, 32>, rows(32),
                                                    dim3(128), 0, st, a);
    if (a.ps == 12 && a.stride == 3)
      return short_strips ? launch_maybe_overlapped(densify_strip_kernel<12, 3, 9>, rows(9),
                                                    dim3(128), 0, st, a)
                          : launch_maybe_overlapped(densify_strip_kernel<12, 3, 30>, rows(30),
                                                    dim3(128), 0, st, a);
    if (a.ps == 16 && a.stride == 4)
      return short_strips ? launch_maybe_overlapped(densify_strip_kernel<16, 4, 8>, rows(8),
                                                    dim3(128), 0, st, a)
                          : launch_maybe_overlapped(densify_strip_kernel<16, 4, 32>, rows(32),
                                                    dim3(128), 0, st, a);
  }
  const int tile_y = a.tile_y > 0 ? a.tile_y : kTileY;
  const dim3 grid((unsigned)((a.w + kTileX - 1) / kTileX), (unsigned)((a.h + tile_y - 1) / tile_y),
                  (unsigned)count);
  densify_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_upsample(const float *map, int mw, int mh, int level, int w, int h, int count,
                            float *out, cudaStream_t st) {
  const long long total = (long long)w * h * count;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  upsample_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(
      map, mw, mh, (float)(1 << level), w, h, total, out);
  return cudaGetLastError();
}

cudaError_t take_check_densify(unsigned *v) { return take_check_word(v); }

}  // namespace bdis
