// pyramid.cu -- image pyramid and template gradient (Sec. 2.1, Fig. 1).
//
// Level 0 is the input as gray levels; each coarser level smooths with the
// separable 5-tap binomial [1 4 6 4 1]/16 (reflect-101 border) and keeps the
// even samples, so level l+1 pixel X sits on level l pixel 2X. The inverse
// search needs the x-gradient of the left (template) image only: Sobel-x / 8,
// exact on linear ramps.
//
// The right view is stored packed, (R[x], R[x+1] - R[x]) per pixel (the
// difference is 0 in the last column), so that the inverse search gets a
// linearly interpolated sample from one 8-byte load and one FMA.
//
// Roofline: all kernels stream planes once (HBM/L2 bandwidth bound).
// prepare_level0: reads 2 B/px (uint8 pair), writes 16 B/px (L, packed R, G).
// pyramid_level (per output px): reads 4 input px of each view (~24 B with
// halo reuse from L1), writes 8 B; the gradient/packing pass reads 8 B and
// writes 8 B. The fused pyramid step reads 12 B per input px once (staged
// tile) and writes 16 B per output px. prepare_pyramid0 (the default first
// launch) reads 2 B per level-0 px and writes level 0 (16 B/px) and level 1
// (16 B per level-1 px): level 0 is not read back for the first step.
#include "bdis_internal.cuh"

namespace bdis {
namespace {

__device__ __forceinline__ int reflect101(int i, int n) {
  // one reflection suffices: callers keep |overhang| <= 2 and n >= 3
  i = i < 0 ? -i : i;
  return i >= n ? 2 * (n - 1) - i : i;
}

template <typename T>
__device__ __forceinline__ float load_px(const void *base, size_t pitch, int x, int y) {
  return (float)reinterpret_cast<const T *>(reinterpret_cast<const char *>(base) + (size_t)y * pitch)[x];
}

// Level 0: float copies of both views and Sobel-x / 8 of the left view.
template <typename T>
__global__ void prepare_level0_kernel(const void *left, const void *right, size_t pitch,
                                      size_t stride, int w, int h, long long total, float *L0,
                                      float2 *R0, float *G0) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long plane = (long long)w * h;
  const int b = (int)(idx / plane);
  const int rem = (int)(idx - (long long)b * plane);
  const int y = rem / w, x = rem - (rem / w) * w;
  const char *lb = reinterpret_cast<const char *>(left) + (size_t)b * stride;
  const char *rb = reinterpret_cast<const char *>(right) + (size_t)b * stride;
  L0[idx] = load_px<T>(lb, pitch, x, y);
  const float r = load_px<T>(rb, pitch, x, y);
  R0[idx] = make_float2(r, x + 1 < w ? load_px<T>(rb, pitch, x + 1, y) - r : 0.f);
  const int xm = reflect101(x - 1, w), xp = reflect101(x + 1, w);
  const int ym = reflect101(y - 1, h), yp = reflect101(y + 1, h);
  const float dm = load_px<T>(lb, pitch, xp, ym) - load_px<T>(lb, pitch, xm, ym);
  const float d0 = load_px<T>(lb, pitch, xp, y) - load_px<T>(lb, pitch, xm, y);
  const float dp = load_px<T>(lb, pitch, xp, yp) - load_px<T>(lb, pitch, xm, yp);
  G0[idx] = (dm + 2.f * d0 + dp) * 0.125f;
}

// One pyramid step for both views: out(X, Y) = sum_ij b_i b_j in(2X+i, 2Y+j).
__global__ void down_kernel(const float *__restrict__ L, const float2 *__restrict__ R, int w,
                            int h, int dw, int dh, long long total, float *__restrict__ L1,
                            float2 *__restrict__ R1) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long dplane = (long long)dw * dh;
  const int b = (int)(idx / dplane);
  const int rem = (int)(idx - (long long)b * dplane);
  const int Y = rem / dw, X = rem - (rem / dw) * dw;
  const float *Lb = L + (long long)b * w * h;
  const float2 *Rb = R + (long long)b * w * h;
  const float k[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
  int xs[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) xs[i] = reflect101(2 * X + i - 2, w);
  float accL = 0.f, accR = 0.f;
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const int yy = reflect101(2 * Y + j - 2, h);
    const float *lr = Lb + (size_t)yy * w;
    const float2 *rr = Rb + (size_t)yy * w;
    float hl = 0.f, hr = 0.f;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
      hl = fmaf(k[i], __ldg(lr + xs[i]), hl);
      hr = fmaf(k[i], __ldg(rr + xs[i]).x, hr);
    }
    accL = fmaf(k[j], hl, accL);
    accR = fmaf(k[j], hr, accR);
  }
  L1[idx] = accL;
  R1[idx].x = accR;  // the difference term is filled by the gradient pass
}

// Sobel-x / 8 of the left level and the difference term of the packed right level.
__global__ void sobel_pack_kernel(const float *__restrict__ L, float2 *__restrict__ R, int w,
                                  int h, long long total, float *__restrict__ G) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const long long plane = (long long)w * h;
  const int b = (int)(idx / plane);
  const int rem = (int)(idx - (long long)b * plane);
  const int y = rem / w, x = rem - (rem / w) * w;
  const float *Lb = L + (long long)b * plane;
  const int xm = reflect101(x - 1, w), xp = reflect101(x + 1, w);
  const int ym = reflect101(y - 1, h), yp = reflect101(y + 1, h);
  const float dm = __ldg(Lb + (size_t)ym * w + xp) - __ldg(Lb + (size_t)ym * w + xm);
  const float d0 = __ldg(Lb + (size_t)y * w + xp) - __ldg(Lb + (size_t)y * w + xm);
  const float dp = __ldg(Lb + (size_t)yp * w + xp) - __ldg(Lb + (size_t)yp * w + xm);
  G[idx] = (dm + 2.f * d0 + dp) * 0.125f;
  float2 *Rb = R + (long long)b * plane + (size_t)y * w;
  Rb[x].y = x + 1 < w ? Rb[x + 1].x - Rb[x].x : 0.f;
}

// Level 0 from 8-bit views, four pixels per thread (width, pitch and image
// stride multiples of 4): one 32-bit load per row segment plus the two
// reflected neighbour bytes, float4 stores. Row and pair come from the grid,
// so there is no per-pixel index division. Same values as the scalar kernel.
__global__ void __launch_bounds__(128) prepare_level0_x4_kernel(
    const uint8_t *__restrict__ left, const uint8_t *__restrict__ right, size_t pitch,
    size_t stride, int w, int h, float *__restrict__ L0, float2 *__restrict__ R0,
    float *__restrict__ G0) {
  const int x = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  const int y = blockIdx.y, b = blockIdx.z;
  if (x >= w) return;
  const uint8_t *lb = left + (size_t)b * stride;
  const uint8_t *rb = right + (size_t)b * stride;
  const int xm = reflect101(x - 1, w), xq = reflect101(x + 4, w);
  // v[0] = column x - 1 (reflected), v[1..4] = x .. x + 3, v[5] = x + 4 (reflected)
  auto row6 = [&](const uint8_t *row, float v[6]) {
    const uint32_t wd = __ldg(reinterpret_cast<const unsigned int *>(row + x));
    v[0] = (float)__ldg(row + xm);
#pragma unroll
    for (int i = 0; i < 4; ++i) v[1 + i] = (float)((wd >> (8 * i)) & 0xffu);
    v[5] = (float)__ldg(row + xq);
  };
  float lm[6], l0[6], lp[6], r[6];
  row6(lb + (size_t)reflect101(y - 1, h) * pitch, lm);
  row6(lb + (size_t)y * pitch, l0);
  row6(lb + (size_t)reflect101(y + 1, h) * pitch, lp);
  row6(rb + (size_t)y * pitch, r);
  const size_t o = (size_t)b * w * h + (size_t)y * w + x;
  float g[4], rd[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float dm = lm[i + 2] - lm[i];
    const float d0 = l0[i + 2] - l0[i];
    const float dp = lp[i + 2] - lp[i];
    g[i] = (dm + 2.f * d0 + dp) * 0.125f;
    rd[i] = x + i + 1 < w ? r[i + 2] - r[i + 1] : 0.f;
  }
  *reinterpret_cast<float4 *>(L0 + o) = make_float4(l0[1], l0[2], l0[3], l0[4]);
  *reinterpret_cast<float4 *>(G0 + o) = make_float4(g[0], g[1], g[2], g[3]);
  float4 *r4 = reinterpret_cast<float4 *>(R0 + o);
  r4[0] = make_float4(r[1], rd[0], r[2], rd[1]);
  r4[1] = make_float4(r[3], rd[2], r[4], rd[3]);
}

// One pyramid step fused with the gradient and packing of the new level. A
// block owns a 32 x 16 output tile and computes it plus a one-pixel halo. The
// input rows and columns the tile needs are staged in shared memory once:
// stage row r holds input row reflect101(2 Y0 - 4 + r), stage column c input
// column reflect101(2 X0 - 4 + c). A horizontal 5-tap pass per stage row and
// computed column, then a vertical 5-tap pass per computed output, give the
// binomial downsample. A halo cell is evaluated at its reflected coordinate,
// so it holds exactly the neighbour that reflect-101 asks for; every tap
// reads the same input element, in the same order, as down_kernel. Then L1,
// the packed R1 and Sobel-x / 8 of L1 are written once (as sobel_pack_kernel).
constexpr int kPyrX = 32, kPyrY = 16;
constexpr int kStX = 2 * kPyrX + 7, kStY = 2 * kPyrY + 7;  // staged input columns / rows
constexpr int kStP = 72;                                     // staged row pitch (floats)
constexpr int kCx = kPyrX + 2;                               // computed columns (with halo)

// Stage columns of tap 0 for the computed columns of this lane (cx = lane,
// and lanes 0, 1 also take 32, 33), at the reflected output coordinate.
__device__ __forceinline__ void stage_taps(int lane, int X0, int dw, int (&c0)[2], bool (&cok)[2]) {
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int cx = lane + 32 * u, Xr = X0 - 1 + cx;
    cok[u] = cx < kCx && Xr <= dw;
    c0[u] = cok[u] ? 2 * (reflect101(Xr, dw) - X0) + 2 : 0;
  }
}

// Columns of the stage this lane fills (c = lane + 32 u): the input column
// reflect101(2 X0 - 4 + c), or none past the last reflected tap.
__device__ __forceinline__ void stage_columns(int lane, int X0, int w, int (&xsrc)[3],
                                              bool (&xok)[3]) {
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int c = lane + 32 * u, xi = 2 * X0 - 4 + c;
    xok[u] = c < kStX && xi <= w + 1;
    xsrc[u] = xok[u] ? reflect101(xi, w) : 0;
  }
}

// The pyramid step on a staged tile (the stage complete and visible): a
// horizontal 5-tap pass per stage row and computed column, a vertical 5-tap
// pass per computed output, then L1, packed R1 and Sobel-x / 8 of L1. The two
// views sit side by side, (L, R) per pixel, so that every tap of both is one
// 8-byte shared load and one packed f32x2 FMA (per component the same fma, in
// the same order, as down_kernel).
__device__ __forceinline__ void pyramid_passes(const float2 (*inLR)[kStP], float2 (*hLR)[kCx],
                                               float2 (*sLR)[kCx], const int (&c0)[2],
                                               const bool (&cok)[2], int b, int X0, int Y0,
                                               int h, int dw, int dh, float *__restrict__ L1,
                                               float2 *__restrict__ R1, float *__restrict__ G1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const float k[5] = {1.f / 16, 4.f / 16, 6.f / 16, 4.f / 16, 1.f / 16};
  for (int r = warp; r < kStY; r += nwarp) {
    if (2 * Y0 - 4 + r > h + 1) break;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!cok[u]) continue;
      float2 hv = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 5; ++i) hv = __ffma2_rn(make_float2(k[i], k[i]), inLR[r][c0[u] + i], hv);
      hLR[r][lane + 32 * u] = hv;
    }
  }
  __syncthreads();
  // vertical taps: the downsampled value of every computed cell
  for (int cy = warp; cy < kPyrY + 2; cy += nwarp) {
    const int Yr = Y0 - 1 + cy;
    if (Yr > dh) break;
    const int r0 = 2 * (reflect101(Yr, dh) - Y0) + 2;  // stage row of tap 0
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (!cok[u]) continue;
      const int cx = lane + 32 * u;
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 5; ++j) acc = __ffma2_rn(make_float2(k[j], k[j]), hLR[r0 + j][cx], acc);
      sLR[cy][cx] = acc;
    }
  }
  __syncthreads();
  const int cx = 1 + lane;
  for (int cy = 1 + warp; cy <= kPyrY; cy += nwarp) {
    const int X = X0 + cx - 1, Y = Y0 + cy - 1;
    if (X >= dw || Y >= dh) continue;
    const float dm = sLR[cy - 1][cx + 1].x - sLR[cy - 1][cx - 1].x;
    const float d0 = sLR[cy][cx + 1].x - sLR[cy][cx - 1].x;
    const float dp = sLR[cy + 1][cx + 1].x - sLR[cy + 1][cx - 1].x;
    const size_t o = (size_t)b * dw * dh + (size_t)Y * dw + X;
    BDIS_CHECKED_ONLY(
        if (!in_bounds((long long)o, (long long)gridDim.z * dw * dh, kCheckPyramidOut)) continue;)
    const float2 v = sLR[cy][cx];
    L1[o] = v.x;
    G1[o] = (dm + 2.f * d0 + dp) * 0.125f;
    R1[o] = make_float2(v.y, X + 1 < dw ? sLR[cy][cx + 1].y - v.y : 0.f);
  }
}

__global__ void __launch_bounds__(256) pyramid_fused_kernel(
    const float *__restrict__ L, const float2 *__restrict__ R, int w, int h, int dw, int dh,
    float *__restrict__ L1, float2 *__restrict__ R1, float *__restrict__ G1) {
  __shared__ float2 inLR[kStY][kStP];
  __shared__ float2 hLR[kStY][kCx];
  __shared__ float2 sLR[kPyrY + 2][kCx];
  pdl_enter();
  const int b = blockIdx.z, X0 = blockIdx.x * kPyrX, Y0 = blockIdx.y * kPyrY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const float *Lb = L + (long long)b * w * h;
  const float2 *Rb = R + (long long)b * w * h;
  // Warps take stage rows, lanes take columns, so every reflected index is
  // computed once per row (warp) or once per column (lane). Stage row r holds
  // input row reflect101(2 Y0 - 4 + r), column c input column
  // reflect101(2 X0 - 4 + c); anything past the last reflected tap is skipped.
  int xsrc[3];
  bool xok[3];
  stage_columns(lane, X0, w, xsrc, xok);
  for (int r = warp; r < kStY; r += nwarp) {
    const int yi = 2 * Y0 - 4 + r;
    if (yi > h + 1) break;  // rows only grow from here
    const size_t rowoff = (size_t)reflect101(yi, h) * w;
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      if (!xok[u]) continue;
      BDIS_CHECKED_ONLY(
          if (!in_bounds((long long)rowoff + xsrc[u], (long long)w * h, kCheckPyramidStage))
              continue;)
      const int c = lane + 32 * u;
      const unsigned dl = (unsigned)__cvta_generic_to_shared(&inLR[r][c].x);
      const unsigned dr = (unsigned)__cvta_generic_to_shared(&inLR[r][c].y);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dl),
                   "l"(Lb + rowoff + xsrc[u]));
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dr),
                   "l"(Rb + rowoff + xsrc[u]));  // the value is the pair's first word
    }
  }
  int c0[2];
  bool cok[2];
  stage_taps(lane, X0, dw, c0, cok);  // while the copies travel
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  pyramid_passes(inLR, hLR, sLR, c0, cok, b, X0, Y0, h, dw, dh, L1, R1, G1);
}

// Level 0 and the first pyramid step in one pass over the input views: the
// tile of the step is staged straight from the 8-bit (or float) images, the
// block writes the level-0 pixels it owns (the 2 kPyrX x 2 kPyrY under its
// output tile: L0, packed R0 and Sobel-x / 8 of L0, the same values and
// operations as prepare_level0) from the stage, then runs the pyramid step on
// it. Level 0 is thus written once and never read back for level 1.
template <typename T>
__global__ void __launch_bounds__(256) prepare_pyramid0_kernel(
    const void *__restrict__ left, const void *__restrict__ right, size_t pitch, size_t stride,
    int w, int h, int dw, int dh, int words, float *__restrict__ L0, float2 *__restrict__ R0,
    float *__restrict__ G0, float *__restrict__ L1, float2 *__restrict__ R1,
    float *__restrict__ G1) {
  __shared__ float2 inLR[kStY][kStP];
  __shared__ float2 hLR[kStY][kCx];
  __shared__ float2 sLR[kPyrY + 2][kCx];
  pdl_enter();
  const int b = blockIdx.z, X0 = blockIdx.x * kPyrX, Y0 = blockIdx.y * kPyrY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const char *lb = reinterpret_cast<const char *>(left) + (size_t)b * stride;
  const char *rb = reinterpret_cast<const char *>(right) + (size_t)b * stride;
  int xsrc[3];
  bool xok[3];
  stage_columns(lane, X0, w, xsrc, xok);
  // 8-bit views with 4-byte aligned rows (words != 0), block inside the image
  // in x: a stage row is 18 aligned 32-bit words (columns 2 X0 - 4 ..
  // 2 X0 + 67), one per lane, and all of the warp's rows are loaded before any
  // is stored. Otherwise one element per lane and column, reflected.
  constexpr int kRowsPerWarp = (kStY + 7) / 8, kWords = (kStX + 3) / 4;
  if (sizeof(T) == 1 && words && 2 * X0 - 4 >= 0 && 2 * X0 + 4 * kWords - 4 <= w && nwarp == 8) {
    uint32_t wl[kRowsPerWarp], wr[kRowsPerWarp];
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
      const int r = warp + 8 * q, yi = 2 * Y0 - 4 + r;
      const bool rok = lane < kWords && r < kStY && yi <= h + 1;
      const size_t off = (size_t)(rok ? reflect101(yi, h) : 0) * pitch + (size_t)(2 * X0 - 4);
#ifdef BDIS_CHECKED
      // the word's last byte lies inside the view (h - 1 full rows and w bytes)
      const bool inb =
          !rok || in_bounds((long long)(off + 4 * lane + 3), (long long)(h - 1) * pitch + w,
                            kCheckPyramidInput);
      wl[q] = rok && inb ? __ldg(reinterpret_cast<const uint32_t *>(lb + off) + lane) : 0u;
      wr[q] = rok && inb ? __ldg(reinterpret_cast<const uint32_t *>(rb + off) + lane) : 0u;
#else
      wl[q] = rok ? __ldg(reinterpret_cast<const uint32_t *>(lb + off) + lane) : 0u;
      wr[q] = rok ? __ldg(reinterpret_cast<const uint32_t *>(rb + off) + lane) : 0u;
#endif
    }
#pragma unroll
    for (int q = 0; q < kRowsPerWarp; ++q) {
      const int r = warp + 8 * q;
      if (r >= kStY || 2 * Y0 - 4 + r > h + 1) break;
      if (lane >= kWords) continue;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = 4 * lane + e;
        if (c < kStX)
          inLR[r][c] = make_float2((float)((wl[q] >> (8 * e)) & 0xffu),
                                   (float)((wr[q] >> (8 * e)) & 0xffu));
      }
    }
  } else {
    for (int r = warp; r < kStY; r += nwarp) {
      const int yi = 2 * Y0 - 4 + r;
      if (yi > h + 1) break;
      const int row = reflect101(yi, h);
#pragma unroll
      for (int u = 0; u < 3; ++u) {
        if (!xok[u]) continue;
        BDIS_CHECKED_ONLY(
            if (!in_bounds((long long)row * pitch + (long long)xsrc[u] * sizeof(T),
                           (long long)(h - 1) * pitch + (long long)w * sizeof(T),
                           kCheckPyramidInput)) continue;)
        inLR[r][lane + 32 * u] = make_float2(load_px<T>(lb, pitch, xsrc[u], row),
                                             load_px<T>(rb, pitch, xsrc[u], row));
      }
    }
  }
  int c0[2];
  bool cok[2];
  stage_taps(lane, X0, dw, c0, cok);
  __syncthreads();
  // level 0: pixel (2 X0 + i, 2 Y0 + j) is stage (row j + 4, column i + 4); its
  // neighbours x +- 1, y +- 1 are the staged reflect-101 ones
  for (int j = warp; j < 2 * kPyrY; j += nwarp) {
    const int y = 2 * Y0 + j;
    if (y >= h) break;
    const int r = j + 4;
    for (int i = lane; i < 2 * kPyrX; i += 32) {
      const int x = 2 * X0 + i;
      if (x >= w) break;
      const int c = i + 4;
      const float2 v = inLR[r][c];
      const float dm = inLR[r - 1][c + 1].x - inLR[r - 1][c - 1].x;
      const float d0 = inLR[r][c + 1].x - inLR[r][c - 1].x;
      const float dp = inLR[r + 1][c + 1].x - inLR[r + 1][c - 1].x;
      const size_t o = (size_t)b * w * h + (size_t)y * w + x;
      BDIS_CHECKED_ONLY(
          if (!in_bounds((long long)o, (long long)gridDim.z * w * h, kCheckPyramidOut)) continue;)
      L0[o] = v.x;
      G0[o] = (dm + 2.f * d0 + dp) * 0.125f;
      R0[o] = make_float2(v.y, x + 1 < w ? inLR[r][c + 1].y - v.y : 0.f);
    }
  }
  pyramid_passes(inLR, hLR, sLR, c0, cok, b, X0, Y0, h, dw, dh, L1, R1, G1);
}

__global__ void pack_right_kernel(const float *__restrict__ R, int w, long long total,
                                  float2 *__restrict__ R2) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int x = (int)(idx % w);
  const float r = R[idx];
  R2[idx] = make_float2(r, x + 1 < w ? R[idx + 1] - r : 0.f);
}


inline unsigned blocks_for(long long n, int threads) {
  return (unsigned)((n + threads - 1) / threads);
}

// 2: level 0 and the first step in one kernel, later steps fused; 1: every
// step one fused kernel after the level-0 preparation; 0: downsample, then
// gradient and packing, per step
int g_pyramid_fused = 2;

}  // namespace

int pyramid_fused() { return g_pyramid_fused; }

int g_launch_overlap = 1;
int launch_overlap() { return g_launch_overlap; }
void set_launch_overlap(int on) { g_launch_overlap = on ? 1 : 0; }

int device_sms() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 152;
    }
    cache[dev] = n;
  }
  return cache[dev];
}
void set_pyramid_fused(int variant) { g_pyramid_fused = variant < 0 ? 0 : (variant > 2 ? 2 : variant); }

cudaError_t launch_prepare_pyramid0(const bdis_image &left, const bdis_image &right, float *L0,
                                    float2 *R0, float *G0, float *L1, float2 *R1, float *G1,
                                    cudaStream_t st) {
  const int w = left.width, h = left.height, dw = (w + 1) / 2, dh = (h + 1) / 2;
  if ((long long)w * h * left.count == 0) return cudaSuccess;
  const size_t stride = left.count > 1 ? left.image_stride_bytes : 0;
  const dim3 grid((unsigned)((dw + kPyrX - 1) / kPyrX), (unsigned)((dh + kPyrY - 1) / kPyrY),
                  (unsigned)left.count);
  // whole aligned 32-bit words per row for the 8-bit staging fast path
  const int words = left.format == BDIS_U8 && left.pitch_bytes % 4 == 0 && stride % 4 == 0 &&
                    right.pitch_bytes == left.pitch_bytes &&
                    (reinterpret_cast<uintptr_t>(left.data) & 3) == 0 &&
                    (reinterpret_cast<uintptr_t>(right.data) & 3) == 0;
  if (left.format == BDIS_U8)
    return launch_maybe_overlapped(prepare_pyramid0_kernel<uint8_t>, grid, dim3(256), 0, st,
                                   left.data, right.data, left.pitch_bytes, stride, w, h, dw, dh,
                                   words, L0, R0, G0, L1, R1, G1);
  return launch_maybe_overlapped(prepare_pyramid0_kernel<float>, grid, dim3(256), 0, st,
                                 left.data, right.data, left.pitch_bytes, stride, w, h, dw, dh, 0,
                                 L0, R0, G0, L1, R1, G1);
}

cudaError_t launch_prepare_level0(const bdis_image &left, const bdis_image &right, float *L0,
                                  float2 *R0, float *G0, cudaStream_t st) {
  const long long total = (long long)left.width * left.height * left.count;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const size_t stride = left.count > 1 ? left.image_stride_bytes : 0;
  const bool aligned4 = left.width % 4 == 0 && left.pitch_bytes % 4 == 0 && stride % 4 == 0 &&
                        right.pitch_bytes == left.pitch_bytes &&
                        (reinterpret_cast<uintptr_t>(left.data) & 3) == 0 &&
                        (reinterpret_cast<uintptr_t>(right.data) & 3) == 0;
  if (left.format == BDIS_U8 && aligned4 && left.height >= 2 &&
      (reinterpret_cast<uintptr_t>(L0) & 15) == 0 && (reinterpret_cast<uintptr_t>(R0) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(G0) & 15) == 0) {
    const int tpb = 128;
    const dim3 grid((unsigned)((left.width / 4 + tpb - 1) / tpb), (unsigned)left.height,
                    (unsigned)left.count);
    prepare_level0_x4_kernel<<<grid, tpb, 0, st>>>(
        static_cast<const uint8_t *>(left.data), static_cast<const uint8_t *>(right.data),
        left.pitch_bytes, stride, left.width, left.height, L0, R0, G0);
    return cudaGetLastError();
  }
  if (left.format == BDIS_U8)
    prepare_level0_kernel<uint8_t><<<blocks_for(total, threads), threads, 0, st>>>(
        left.data, right.data, left.pitch_bytes, stride, left.width, left.height, total, L0, R0,
        G0);
  else
    prepare_level0_kernel<float><<<blocks_for(total, threads), threads, 0, st>>>(
        left.data, right.data, left.pitch_bytes, stride, left.width, left.height, total, L0, R0,
        G0);
  return cudaGetLastError();
}

cudaError_t launch_pyramid_level(const float *L, const float2 *R, int w, int h, int count,
                                 float *L1, float2 *R1, float *G1, cudaStream_t st) {
  const int dw = (w + 1) / 2, dh = (h + 1) / 2;
  const long long total = (long long)dw * dh * count;
  if (total == 0) return cudaSuccess;
  if (g_pyramid_fused) {
    const dim3 grid((unsigned)((dw + kPyrX - 1) / kPyrX), (unsigned)((dh + kPyrY - 1) / kPyrY),
                    (unsigned)count);
    return launch_maybe_overlapped(pyramid_fused_kernel, grid, dim3(256), 0, st, L, R, w, h, dw,
                                   dh, L1, R1, G1);
  }
  const int threads = 256;
  down_kernel<<<blocks_for(total, threads), threads, 0, st>>>(L, R, w, h, dw, dh, total, L1, R1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  sobel_pack_kernel<<<blocks_for(total, threads), threads, 0, st>>>(L1, R1, dw, dh, total, G1);
  return cudaGetLastError();
}

cudaError_t launch_pack_right(const float *R, int w, int h, int count, float2 *R2,
                              cudaStream_t st) {
  const long long total = (long long)w * h * count;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  pack_right_kernel<<<blocks_for(total, threads), threads, 0, st>>>(R, w, total, R2);
  return cudaGetLastError();
}

cudaError_t take_check_pyramid(unsigned *v) { return take_check_word(v); }

}  // namespace bdis
