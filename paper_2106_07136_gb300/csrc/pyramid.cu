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
// writes 8 B.
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

}  // namespace

cudaError_t launch_prepare_level0(const bdis_image &left, const bdis_image &right, float *L0,
                                  float2 *R0, float *G0, cudaStream_t st) {
  const long long total = (long long)left.width * left.height * left.count;
  if (total == 0) return cudaSuccess;
  const int threads = 256;
  const size_t stride = left.count > 1 ? left.image_stride_bytes : 0;
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

}  // namespace bdis
