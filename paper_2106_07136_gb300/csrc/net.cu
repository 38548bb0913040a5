// net.cu -- the learned coarse proposal: a 6-layer 3x3 convolutional network
// on one pyramid level of the pair (level 4 of the paper's 5 scales, the
// level the learned start runs it on), BF16 weights and activations, FP32
// accumulation, forward and training kernels on the tensor cores. The
// network is fully convolutional: any level size works.
//
// Not part of the paper: the paper's method starts its coarsest level from 0
// (Sec. 2.1); this network proposes a start instead, and BDIS refines it.
//
// Architecture (all 3x3, zero padding, dilations 1, 2, 4, 4, 2, 1 so the
// receptive field spans +-14 pixels of its level):
//   x0 = [(L - 128) / 64, (R - 128) / 64]           2 channels (padded to 16)
//   a1..a5 = relu(conv(a_{i-1}) + b_i)              32 channels
//   d = conv(a5) + b6                               1 channel (padded to 16), one per pixel
// Activations are NHWC bf16 (channels innermost).
//
// Every convolution is an implicit GEMM (bf16 in, f32 accumulate): rows =
// pixels, columns = output channels, K = 9 taps x input channels. The forward
// convolutions run on the 5th-generation tensor cores (tcgen05, below) by
// default, or on mma.sync.m16n8k16; training uses mma.sync. The data-gradient of a layer is the same kernel run on the
// output gradient with transposed, tap-flipped weights and the previous
// layer's ReLU mask fused into the store; the weight-gradient is a GEMM with
// rows = output channels, columns = (tap, input channel), K = pixels,
// reduced across blocks with float atomics.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "bdis_internal.cuh"

namespace {

constexpr int kLayers = 6;
constexpr int kDil[kLayers] = {1, 2, 4, 4, 2, 1};
constexpr int kCin[kLayers] = {2, 32, 32, 32, 32, 32};    // real channels
constexpr int kCout[kLayers] = {32, 32, 32, 32, 32, 1};
constexpr int kCinP[kLayers] = {16, 32, 32, 32, 32, 32};  // padded (multiples of 16)
constexpr int kCoutP[kLayers] = {32, 32, 32, 32, 32, 16};

constexpr int master_w_offset(int l) {
  int off = 0;
  for (int i = 0; i < l; ++i) off += kCout[i] * 9 * kCin[i] + kCout[i];
  return off;
}
constexpr int kMasterCount = master_w_offset(kLayers);

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  __nv_bfloat162 v;
  v.x = lo;
  v.y = hi;
  return *reinterpret_cast<uint32_t *>(&v);
}

// D (16x8 f32) += A (16x16 bf16, row) * B (16x8 bf16, col)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// ------------------------------------------------------------ input pack

// x0[p][0] = (L - 128)/64, x0[p][1] = (R - 128)/64, channels 2..15 zero.
__global__ void pack_input_kernel(const float *__restrict__ L, const float *__restrict__ R,
                                  int r_stride, long long total, __nv_bfloat16 *__restrict__ x0) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= total) return;
  uint4 *dst = reinterpret_cast<uint4 *>(x0 + p * 16);
  const float l = (__ldg(L + p) - 128.f) * (1.f / 64.f);
  const float r = (__ldg(R + p * r_stride) - 128.f) * (1.f / 64.f);
  uint4 v0 = make_uint4(pack_bf16(l, r), 0u, 0u, 0u);
  dst[0] = v0;
  dst[1] = make_uint4(0u, 0u, 0u, 0u);
}

// ------------------------------------------------------------ conv (mma)

enum ConvMode { kFwdRelu = 0, kFwdLinearF32 = 1, kBwdDataMasked = 2 };

// One warp computes MT x 16 consecutive pixels x COUT channels (MT m-tiles
// share every weight fragment it loads); a block of 4 warps covers 64 MT
// pixels per tile and loops over tiles (persistent), so the weights (COUT x 9
// x CIN bf16) are staged in shared memory once per block.
template <int CIN, int COUT, int MODE, int MT = 4>
__global__ void __launch_bounds__(128) conv_mma_kernel(
    const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ wt,
    const float *__restrict__ bias, int dil, int H, int W, long long total,
    const __nv_bfloat16 *__restrict__ mask, void *__restrict__ out) {
  static_assert(CIN % 16 == 0 && COUT % 8 == 0, "tile");
  constexpr int NT = COUT / 8;
  __shared__ __align__(16) __nv_bfloat16 ws[COUT * 9 * CIN];
  for (int i = threadIdx.x * 8; i < COUT * 9 * CIN; i += blockDim.x * 8)
    *reinterpret_cast<uint4 *>(ws + i) = *reinterpret_cast<const uint4 *>(wt + i);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const long long plane = (long long)H * W;
  const long long per_tile = 64LL * MT;
  for (long long tile = blockIdx.x; tile * per_tile < total; tile += gridDim.x) {
    const long long p0 = tile * per_tile + (long long)warp * 16 * MT;
    // pixel rows of this thread: m-tile m feeds rows p0 + 16 m + g and + 8
    long long pr[MT][2];
    int pb[MT][2], py[MT][2], px[MT][2];
    bool pv[MT][2];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        pr[m][i] = p0 + 16 * m + g + 8 * i;
        pv[m][i] = pr[m][i] < total;
        const long long pp = pv[m][i] ? pr[m][i] : 0;
        pb[m][i] = (int)(pp / plane);
        const int rem = (int)(pp - (long long)pb[m][i] * plane);
        py[m][i] = rem / W;
        px[m][i] = rem - py[m][i] * W;
      }
    float acc[MT][NT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int n = 0; n < NT; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = (tap / 3 - 1) * dil, dx = (tap % 3 - 1) * dil;
      const __nv_bfloat16 *src[MT][2];
#pragma unroll
      for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int yy = py[m][i] + dy, xx = px[m][i] + dx;
          const bool ok = pv[m][i] && yy >= 0 && yy < H && xx >= 0 && xx < W;
          src[m][i] = ok ? in + (((long long)pb[m][i] * H + yy) * W + xx) * CIN : nullptr;
        }
#pragma unroll
      for (int kb = 0; kb < CIN / 16; ++kb) {
        const int c0 = kb * 16 + q * 2;
        uint32_t b[NT][2];
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const __nv_bfloat16 *wr = ws + ((n * 8 + g) * 9 + tap) * CIN + c0;
          b[n][0] = *reinterpret_cast<const uint32_t *>(wr);
          b[n][1] = *reinterpret_cast<const uint32_t *>(wr + 8);
        }
#pragma unroll
        for (int m = 0; m < MT; ++m) {
          uint32_t a[4];
          a[0] = src[m][0] ? *reinterpret_cast<const uint32_t *>(src[m][0] + c0) : 0u;
          a[1] = src[m][1] ? *reinterpret_cast<const uint32_t *>(src[m][1] + c0) : 0u;
          a[2] = src[m][0] ? *reinterpret_cast<const uint32_t *>(src[m][0] + c0 + 8) : 0u;
          a[3] = src[m][1] ? *reinterpret_cast<const uint32_t *>(src[m][1] + c0 + 8) : 0u;
#pragma unroll
          for (int n = 0; n < NT; ++n) mma_bf16(acc[m][n], a, b[n]);
        }
      }
    }
    // epilogue: acc[m][n][0..1] -> row 16m + g, channels 8n + 2q + {0,1}; [2..3] -> row + 8
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        if (!pv[m][i]) continue;
        const long long p = pr[m][i];
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          const int c = n * 8 + q * 2;
          float v0 = acc[m][n][2 * i], v1 = acc[m][n][2 * i + 1];
          if (MODE == kFwdRelu) {
            v0 = fmaxf(v0 + bias[c], 0.f);
            v1 = fmaxf(v1 + bias[c + 1], 0.f);
            *reinterpret_cast<uint32_t *>(reinterpret_cast<__nv_bfloat16 *>(out) + p * COUT + c) =
                pack_bf16(v0, v1);
          } else if (MODE == kFwdLinearF32) {
            float *o = reinterpret_cast<float *>(out) + p * COUT + c;
            o[0] = v0 + bias[c];
            o[1] = v1 + bias[c + 1];
          } else {  // data gradient times the previous layer's ReLU derivative
            const __nv_bfloat162 mk =
                *reinterpret_cast<const __nv_bfloat162 *>(mask + p * COUT + c);
            v0 = __bfloat162float(mk.x) > 0.f ? v0 : 0.f;
            v1 = __bfloat162float(mk.y) > 0.f ? v1 : 0.f;
            *reinterpret_cast<uint32_t *>(reinterpret_cast<__nv_bfloat16 *>(out) + p * COUT + c) =
                pack_bf16(v0, v1);
          }
        }
      }
  }
}

// ------------------------------------------------------- conv (tcgen05)

// The same forward convolutions on the 5th-generation tensor cores, as an
// implicit GEMM without an im2col copy. Pixels are numbered in a padded frame:
// each image becomes (H + 2 dil) x (W + 2 dil) with zero borders, so a tap
// (dy, dx) is the constant shift dy dil (W + 2 dil) + dx dil of that
// numbering. A block (one warpgroup, 128 threads) owns a tile of 128
// consecutive padded positions and stages, once, the slab of padded positions
// [tile - s, tile + 127 + s] (s = the largest shift) in shared memory: for each
// group of 8 channels a plane of slab rows, 16 bytes per row. In the
// no-swizzle K-major layout that is a run of core matrices (8 rows x 16 bytes,
// 128 B apart along M), so the A operand of tap t is the slab window starting
// s + shift(t) rows in (a descriptor start 16 B per row), and the two channel
// groups of one MMA (K = 16) are one plane apart (the leading offset). B (the
// COUT x 9 CIN weights) is staged once per block. One thread issues the
// 9 CIN / 16 MMAs (M 128, N COUT, K 16) into a tensor-memory accumulator and
// commits them to an mbarrier; every thread then reads its row of D (warp w
// owns tensor-memory lanes 32 w .. 32 w + 31) and, if its position is a real
// pixel, writes the layer output. Waits are bounded by the global timer: on a
// timeout the block writes NaN, sets the network's fault word (read by
// bdis_net_status), frees its tensor memory and returns.

__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);  // no swizzle
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait until the mbarrier's phase `parity` has completed, at most ~200 ms
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 200000000ull) return false;
  }
}

// slab rows of a tile: 128 positions plus the largest shift on either side
__host__ __device__ __forceinline__ int tc_slab_rows(int dil, int W) {
  return 128 + 2 * (dil * (W + 2 * dil) + dil);
}

template <int CIN, int COUT>
int tc_smem_bytes(int dil, int W) {  // the slab and the weights
  return (CIN / 8) * tc_slab_rows(dil, W) * 16 + (9 * CIN / 8) * (COUT / 8) * 128;
}

template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(128) conv_tc_kernel(
    const __nv_bfloat16 *__restrict__ in, const __nv_bfloat16 *__restrict__ wt,
    const float *__restrict__ bias, int dil, int H, int W, int count,
    void *__restrict__ out, int *__restrict__ fault) {
  static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "tile");
  static_assert(MODE == kFwdRelu || MODE == kFwdLinearF32, "forward only");
  constexpr int KG = 9 * CIN / 8;  // 8-element k-groups of the weights
  constexpr int NG = COUT / 8;
  constexpr int CG = CIN / 8;      // channel groups (slab planes)
  extern __shared__ __align__(128) uint8_t tc_smem[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  const int Wp = W + 2 * dil, Hp = H + 2 * dil;
  const int NS = tc_slab_rows(dil, W), soff = dil * Wp + dil;
  const long long planep = (long long)Hp * Wp, totalp = planep * count;
  uint8_t *Ss = tc_smem, *Bs = tc_smem + CG * NS * 16;  // slab, weights
  const int tid = threadIdx.x, warp = tid >> 5;
  // B: weight row co (K = 9 CIN contiguous) -> core (kg, co / 8), row co % 8
  for (int i = tid; i < COUT * KG; i += 128) {
    const int co = i / KG, kg = i - co * KG;
    const uint4 v = *reinterpret_cast<const uint4 *>(wt + (size_t)co * 9 * CIN + kg * 8);
    *reinterpret_cast<uint4 *>(Bs + ((kg * NG + co / 8) * 8 + co % 8) * 16) = v;
  }
  const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mbar_a));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(slot));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_slot;
  const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(Ss);
  const uint32_t b_base = (uint32_t)__cvta_generic_to_shared(Bs);
  constexpr uint32_t idesc = (1u << 4)                    // D: f32
                             | (1u << 7) | (1u << 10)     // A, B: bf16, both K-major
                             | ((uint32_t)(COUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  // a padded position -> its real pixel index, or -1 on a border or past the end
  auto real_pixel = [&](long long q) -> long long {
    if (q < 0 || q >= totalp) return -1;
    const int b = (int)(q / planep);
    const int rem = (int)(q - (long long)b * planep);
    const int y = rem / Wp - dil, x = rem - (rem / Wp) * Wp - dil;
    if (y < 0 || y >= H || x < 0 || x >= W) return -1;
    return ((long long)b * H + y) * W + x;
  };
  uint32_t parity = 0;
  bool ok = true;
  for (long long tile = blockIdx.x; tile * 128 < totalp && ok; tile += gridDim.x) {
    const long long q0 = tile * 128 - soff;  // padded position of slab row 0
    for (int i = tid; i < NS; i += 128) {
      const long long pix = real_pixel(q0 + i);
      const __nv_bfloat16 *src = pix >= 0 ? in + pix * CIN : in;
#pragma unroll
      for (int cg = 0; cg < CG; ++cg)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                         s_base + (cg * NS + i) * 16),
                     "l"(src + cg * 8), "r"(pix >= 0 ? 16 : 0));
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    const uint32_t sb = s_base;
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor cores
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (tid == 0) {
#pragma unroll 1
      for (int tap = 0; tap < 9; ++tap) {
        const int row0 = soff + (tap / 3 - 1) * dil * Wp + (tap % 3 - 1) * dil;
#pragma unroll
        for (int kk = 0; kk < CIN / 16; ++kk) {
          const uint64_t ad =
              umma_smem_desc(sb + (2 * kk * NS + row0) * 16, (uint32_t)NS * 16, 128);
          const uint64_t bd =
              umma_smem_desc(b_base + (tap * CG + 2 * kk) * NG * 128, NG * 128, 128);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
              "l"(ad), "l"(bd), "r"(idesc), "r"(tap | kk));
        }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
              mbar_a));
    }
    // every thread of the block takes the same branch below (the loads are
    // warp-collective and the loop has block barriers)
    ok = __syncthreads_and(mbar_wait(mbar_a, parity)) != 0;
    if (!ok && tid == 0) atomicOr(fault, 1);  // reported by bdis_net_status
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float d[COUT];
    if (ok) {
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
      if constexpr (COUT == 32) {
        uint32_t r[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
              "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
              "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
              "=r"(r[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int c = 0; c < COUT; ++c) d[c] = __uint_as_float(r[c]);
      } else {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
            "%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int c = 0; c < COUT; ++c) d[c] = __uint_as_float(r[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < COUT; ++c) d[c] = __int_as_float(0x7fc00000);
    }
    const long long p = real_pixel(tile * 128 + tid);
    if (p >= 0) {
      if constexpr (MODE == kFwdRelu) {
        uint32_t pk[COUT / 2];
#pragma unroll
        for (int c = 0; c < COUT; c += 2)
          pk[c / 2] = pack_bf16(fmaxf(d[c] + bias[c], 0.f), fmaxf(d[c + 1] + bias[c + 1], 0.f));
        uint4 *o = reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(out) + p * COUT);
#pragma unroll
        for (int v = 0; v < COUT / 8; ++v)
          o[v] = make_uint4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
      } else {
        float *o = reinterpret_cast<float *>(out) + p * COUT;
#pragma unroll
        for (int c = 0; c < COUT; ++c) o[c] = d[c] + bias[c];
      }
    }
    // every thread has read D and the MMAs are done: the slab and D may be rewritten
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");  // none left in flight (timeout exit)
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tmem));
}

// ------------------------------------------- conv (tcgen05, banded inference)

// The inference forward pass keeps every activation in a padded planar
// layout in global memory: each image is framed by kPad zero rows and
// columns (kPad = the largest dilation, so every tap of a real pixel lands
// inside its own frame), frames are numbered back to back, and each group of
// 8 channels is its own plane of 16-byte rows, with zero guard rows before
// and after. A 3x3 tap is then a constant shift of the position numbering, a
// plane's rows are exactly the 8-row x 16-byte core matrices of the tensor
// cores' no-swizzle K-major operand layout, and the rows any band of
// positions reads form one contiguous range per plane: one bulk copy each.
//
// The whole forward pass is one cooperative launch, one block per SM: the
// input is packed, then the six layers run in turn with a grid barrier
// between steps (a band's halo was written by other blocks). Within a layer
// the block is warp-specialised, three stages in flight:
//   - warps 8-11 (one lane each) issue each unit's MMAs (9 taps x CIN / 16
//     per 128-position tile; M 128, N = COUT, K 16; every 4th tile each)
//     into one of two tensor-memory accumulators, one COUT-column slice per
//     tile; warp 8 also stages the units (a band of BH image rows of one
//     image, all padded columns, with its halo of up to dil rows + dil
//     columns either side) by bulk copies into two slab buffers;
//   - warps 0-7 (warp w reads tensor-memory lanes 32 (w % 4) .. + 31, of
//     every other tile) take each finished accumulator, add the bias, apply
//     the ReLU, pack to bf16 and write the real pixels, then hand the
//     accumulator back; two warps per lane quarter hide each other's latency.
// So unit k's MMAs run while unit k + 1's copy travels and unit k - 1's
// epilogue drains. The MMAs bound it: measured on GB300, an M 128 x K 16
// MMA whose A operand (4 KB) is read afresh from no-swizzle shared memory
// takes about 68 cycles whether N is 32 or 64, so with 32 output channels
// the tensor pipe runs at about a quarter of its dense rate.
// Every wait is bounded by the global timer (200 ms on an mbarrier, 1 s at a
// grid barrier): on a timeout the block records it in the network's fault
// word, waits (bounded) for its own copies and MMAs in flight, writes NaN
// over its bands of the map, frees its tensor memory and returns; the other
// blocks then time out at the next grid barrier, if there is one, and do
// the same.
constexpr int kPad = 4;                // frame border = the largest dilation
constexpr int kBandCols = 256;         // tensor-memory columns per accumulator (two)
constexpr int kBandSmem = 224 * 1024;  // dynamic shared memory per block (one per SM)
constexpr int kBandEpiWarps = 8;       // two per tensor-memory lane quarter
constexpr int kBandMmaWarps = 4;       // MMA issue: one lane of each takes every 4th tile
constexpr int kBandThreads = 32 * (kBandEpiWarps + kBandMmaWarps);

__host__ __device__ __forceinline__ long long pp_guard(int W) {
  return (long long)kPad * (W + 2 * kPad) + kPad + 128;
}

// elements (bf16) between two channel planes of a padded planar buffer
__host__ __device__ __forceinline__ long long pp_plane(int H, int W, int count) {
  return ((long long)count * (H + 2 * kPad) * (W + 2 * kPad) + 2 * pp_guard(W)) * 8;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes,
                                          uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(mbar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void *band_smem_base() {
  extern __shared__ __align__(128) uint8_t band_smem[];
  return band_smem;
}

// One layer of the fused inference kernel below.
struct BandLayer {
  const __nv_bfloat16 *in, *wt;
  const float *bias;
  void *out;      // kFwdRelu: padded planar bf16; kFwdLinearF32: dense float map
  int dil, BH, nsb;  // dilation, band rows, slab rows per channel plane
};
struct BandNet {
  BandLayer layer[6];
  const float *L, *R;  // the level planes (R with element stride r_stride)
  int r_stride, H, W, count;
  int slab_bytes;      // per slab buffer (the largest layer's), two buffers
  unsigned *sync;      // grid barrier counter, zero at launch
  int *fault;          // set when a bounded wait ran out
};

// Shared state of the fused kernel's block.
struct BandShared {
  uint32_t s_base, b_base, tmem;
  uint32_t full_a[2], mma_a[2], free_a[2];
};

// Grid-wide barrier of the cooperative launch (all blocks are resident): the
// block's writes are published, one thread counts the block in and waits,
// bounded, for every block of the grid. `target` = barriers passed so far x
// gridDim.x. Returns false (on every thread) if the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned *count, unsigned target) {
  __threadfence();
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    atomicAdd(count, 1u);
    const uint64_t t0 = global_ns();
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (global_ns() - t0 > 1000000000ull) {  // 1 s
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
  }
  return __syncthreads_and(ok) != 0;
}

// One layer: the roles of the module comment over the layer's units. kg counts
// the block's units over all layers (buffer = kg & 1, barrier phase = (kg >> 1)
// & 1); on return every unit of the layer is written and its accumulators are
// handed back. MODE kFwdRelu: out is a padded planar bf16 buffer of COUT
// channels; kFwdLinearF32: out is the dense float map of channel 0.
template <int CIN, int COUT, int MODE>
__device__ bool band_layer(const BandNet &net, const BandLayer &ly, const BandShared &sh,
                           float *sbias, long long &kg) {
  static_assert(CIN % 16 == 0 && (COUT == 16 || COUT == 32), "tile");
  static_assert(MODE == kFwdRelu || MODE == kFwdLinearF32, "forward only");
  constexpr int KG = 9 * CIN / 8, NG = COUT / 8, CG = CIN / 8;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = net.H, W = net.W, count = net.count, dil = ly.dil, BH = ly.BH;
  const int nsb_max = ly.nsb, slab_bytes = net.slab_bytes;
  const int Wp = W + 2 * kPad, Hp = H + 2 * kPad;
  const long long F = (long long)Hp * Wp;
  const long long plane_in = pp_plane(H, W, count), guard = pp_guard(W);
  const int soff = dil * Wp + dil;
  const int nb = (H + BH - 1) / BH;
  const long long units = (long long)count * nb;
  // the layer's weights and bias (the previous layer's MMAs are all done)
  uint8_t *Bs = reinterpret_cast<uint8_t *>(band_smem_base()) + 2 * slab_bytes;
  for (int i = tid; i < COUT * KG; i += kBandThreads) {
    const int kgr = i / COUT, co = i - kgr * COUT;  // consecutive threads: consecutive rows
    const uint4 v = *reinterpret_cast<const uint4 *>(ly.wt + (size_t)co * 9 * CIN + kgr * 8);
    *reinterpret_cast<uint4 *>(Bs + ((kgr * NG + co / 8) * 8 + co % 8) * 16) = v;
  }
  if (tid < COUT) sbias[tid] = ly.bias[tid];
  // weights: generic-proxy writes read by the tensor cores; the input: written
  // by other blocks before the grid barrier, read by this block's bulk copies
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("fence.proxy.async.global;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  auto band = [&](long long u, long long &q_s, int &cnt, int &tiles) {
    const int b = (int)(u / nb), j = (int)(u - (long long)b * nb);
    const int rows = min(BH, H - j * BH);
    q_s = (long long)b * F + (long long)(kPad + j * BH) * Wp;
    cnt = rows * Wp;
    tiles = (cnt + 127) >> 7;
  };
  const long long nk = units > blockIdx.x ? (units - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  bool ok = true;
  if (warp >= kBandEpiWarps) {
    // ---- copies (issuer 0) and MMAs (one lane of each issuer warp)
    const int issuer = warp - kBandEpiWarps;
    if (lane == 0 && nk > 0) {
      constexpr uint32_t idesc = (1u << 4)                 // D: f32
                                 | (1u << 7) | (1u << 10)  // A, B: bf16, both K-major
                                 | ((uint32_t)(COUT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
      auto issue_load = [&](long long k) {
        long long q_s;
        int cnt, tiles;
        band(blockIdx.x + k * gridDim.x, q_s, cnt, tiles);
        const int s = (int)((kg + k) & 1), nsb = tiles * 128 + 2 * soff;
        mbar_expect_tx(sh.full_a[s], (uint32_t)(CG * nsb * 16));
        for (int cg = 0; cg < CG; ++cg)
          bulk_load(sh.s_base + (uint32_t)(s * slab_bytes + cg * nsb_max * 16),
                    ly.in + ((long long)cg * plane_in / 8 + guard + q_s - soff) * 8,
                    (uint32_t)(nsb * 16), sh.full_a[s]);
      };
      // the last unit whose copy / MMAs went to each buffer (-1: none), for the timeout path
      long long last_load[2] = {-1, -1}, last_mma[2] = {-1, -1};
      if (issuer == 0) {
        issue_load(0);
        last_load[kg & 1] = kg;
      }
      for (long long k = 0; k < nk && ok; ++k) {
        const long long g = kg + k;
        const int s = (int)(g & 1);
        const uint32_t ph = (uint32_t)((g >> 1) & 1);
        ok = mbar_wait(sh.full_a[s], ph);  // unit k's slab has landed
        if (ok && g >= 2) ok = mbar_wait(sh.free_a[s], ph ^ 1u);  // unit g - 2's epilogue is done
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        long long q_s;
        int cnt, tiles;
        band(blockIdx.x + k * gridDim.x, q_s, cnt, tiles);
        // descriptors advance in 16-byte units of their start-address field
        // (shared memory is far below the field's 256 KB reach, so no carry)
        const uint64_t a0 = umma_smem_desc(sh.s_base + (uint32_t)(s * slab_bytes),
                                           (uint32_t)nsb_max * 16, 128);
        const uint64_t b0 = umma_smem_desc(sh.b_base, NG * 128, 128);
        const uint32_t t0 = sh.tmem + (uint32_t)(s * kBandCols);
#pragma unroll 1
        for (int i = issuer; i < tiles; i += kBandMmaWarps) {
          const uint32_t d_tmem = t0 + (uint32_t)(i * COUT);
          const int rowi = soff + i * 128;
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int row0 = rowi + (tap / 3 - 1) * dil * Wp + (tap % 3 - 1) * dil;
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk) {
              const uint64_t ad = a0 + (uint64_t)(row0 + 2 * kk * nsb_max);
              const uint64_t bd = b0 + (uint64_t)((tap * CG + 2 * kk) * NG * 8);
              asm volatile(
                  "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                  " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(tap | kk));
            }
          }
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                sh.mma_a[s]));
        last_mma[s] = g;
        // the next unit's copy goes to the other slab once unit g - 1's MMAs
        // (queued ahead of unit g's) have read it
        if (issuer == 0 && k + 1 < nk) {
          if (k >= 1) ok = mbar_wait(sh.mma_a[s ^ 1], (uint32_t)(((g - 1) >> 1) & 1));
          if (!ok) break;
          issue_load(k + 1);
          last_load[s ^ 1] = g + 1;
        }
      }
      if (!ok) {
        atomicOr(net.fault, 1);  // reported by bdis_net_status
        // let the copies and MMAs this block issued land before its memory is released
        for (int b2 = 0; b2 < 2; ++b2) {
          if (last_load[b2] >= 0) mbar_wait(sh.full_a[b2], (uint32_t)((last_load[b2] >> 1) & 1));
          if (last_mma[b2] >= 0) mbar_wait(sh.mma_a[b2], (uint32_t)((last_mma[b2] >> 1) & 1));
        }
      }
    }
  } else {
    // ---- epilogue (warps 0 .. kBandEpiWarps - 1)
    const int quarter = warp & 3, parity = warp >> 2;
    const float *bs = sbias;
    for (long long k = 0; k < nk; ++k) {
      const long long g = kg + k;
      const int s = (int)(g & 1);
      long long q_s;
      int cnt, tiles;
      band(blockIdx.x + k * gridDim.x, q_s, cnt, tiles);
      ok = mbar_wait(sh.mma_a[s], (uint32_t)((g >> 1) & 1));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const int b = (int)(q_s / F);
      for (int i = parity; i < tiles; i += kBandEpiWarps / 4) {
        const uint32_t taddr = sh.tmem + ((uint32_t)(quarter * 32) << 16) +
                               (uint32_t)(s * kBandCols + i * COUT);
        float d[COUT];
        if constexpr (COUT == 32) {
          uint32_t r[32];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
              "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                "=r"(r[30]), "=r"(r[31])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int c = 0; c < COUT; ++c) d[c] = __uint_as_float(r[c]);
        } else {
          uint32_t r[16];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
              "%13,%14,%15}, [%16];\n"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
          for (int c = 0; c < COUT; ++c) d[c] = __uint_as_float(r[c]);
        }
        const int m = i * 128 + quarter * 32 + lane;  // position within the band
        const int xp = m % Wp, x = xp - kPad;
        if (m < cnt && x >= 0 && x < W) {
          const long long q = q_s + m;
          if constexpr (MODE == kFwdRelu) {
            uint32_t pk[COUT / 2];
#pragma unroll
            for (int c = 0; c < COUT; c += 2)
              pk[c / 2] = pack_bf16(fmaxf(d[c] + bs[c], 0.f), fmaxf(d[c + 1] + bs[c + 1], 0.f));
            const long long plane_out = pp_plane(H, W, count) / 8;  // in 16-byte rows
            uint4 *o = reinterpret_cast<uint4 *>(ly.out) + guard + q;
#pragma unroll
            for (int v = 0; v < COUT / 8; ++v)
              o[v * plane_out] =
                  make_uint4(pk[4 * v], pk[4 * v + 1], pk[4 * v + 2], pk[4 * v + 3]);
          } else {
            const int y = (int)((q - (long long)b * F) / Wp) - kPad;
            reinterpret_cast<float *>(ly.out)[((long long)b * H + y) * W + x] = d[0] + bs[0];
          }
        }
      }
      // this accumulator is read: the unit two later may overwrite it
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      mbar_arrive(sh.free_a[s]);
    }
  }
  kg += nk;
  return __syncthreads_and(ok ? 1 : 0) != 0;
}

// The whole inference forward pass in one cooperative launch (one block per
// SM): the input planes are packed into x0, then the six layers run in turn,
// a grid barrier between steps (a layer reads the bands around its own, which
// other blocks wrote). Weights and bias are restaged per layer; the slabs,
// barriers and tensor memory carry over.
__global__ void __launch_bounds__(kBandThreads, 1) net_forward_kernel(const BandNet net) {
  __shared__ __align__(8) uint64_t mb_full[2], mb_mma[2], mb_free[2];
  __shared__ uint32_t tmem_slot;
  __shared__ float sbias[32];
  const int tid = threadIdx.x, warp = tid >> 5;
  BandShared sh;
  for (int i = 0; i < 2; ++i) {
    sh.full_a[i] = (uint32_t)__cvta_generic_to_shared(&mb_full[i]);
    sh.mma_a[i] = (uint32_t)__cvta_generic_to_shared(&mb_mma[i]);
    sh.free_a[i] = (uint32_t)__cvta_generic_to_shared(&mb_free[i]);
  }
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(sh.full_a[i], 1);
      mbar_init(sh.mma_a[i], kBandMmaWarps);
      mbar_init(sh.free_a[i], 32 * kBandEpiWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(slot),
                 "n"(2 * kBandCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // x0: plane 0 = [(L - 128) / 64, (R - 128) / 64, 0 x 6] at every real pixel
  // (plane 1 and the borders stay zero)
  {
    const int H = net.H, W = net.W, Wp = W + 2 * kPad, Hp = H + 2 * kPad;
    const long long plane = (long long)H * W, total = plane * net.count;
    uint4 *x0 = reinterpret_cast<uint4 *>(const_cast<__nv_bfloat16 *>(net.layer[0].in));
    for (long long p = (long long)blockIdx.x * kBandThreads + tid; p < total;
         p += (long long)gridDim.x * kBandThreads) {
      const int b = (int)(p / plane);
      const int rem = (int)(p - (long long)b * plane);
      const int y = rem / W, x = rem - (rem / W) * W;
      const long long q = ((long long)b * Hp + y + kPad) * Wp + x + kPad;
      const float l = (__ldg(net.L + p) - 128.f) * (1.f / 64.f);
      const float r = (__ldg(net.R + p * net.r_stride) - 128.f) * (1.f / 64.f);
      x0[pp_guard(W) + q] = make_uint4(pack_bf16(l, r), 0u, 0u, 0u);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  sh.tmem = tmem_slot;
  sh.s_base = (uint32_t)__cvta_generic_to_shared(band_smem_base());
  sh.b_base = sh.s_base + 2u * (uint32_t)net.slab_bytes;
  long long kg = 0;
  unsigned passed = 0;
  bool ok = grid_barrier(net.sync, ++passed * gridDim.x);
  if (ok) ok = band_layer<16, 32, kFwdRelu>(net, net.layer[0], sh, sbias, kg);
  for (int l = 1; l < 5 && ok; ++l) {
    ok = grid_barrier(net.sync, ++passed * gridDim.x);
    if (ok) ok = band_layer<32, 32, kFwdRelu>(net, net.layer[l], sh, sbias, kg);
  }
  if (ok) ok = grid_barrier(net.sync, ++passed * gridDim.x);
  if (ok) ok = band_layer<32, 16, kFwdLinearF32>(net, net.layer[5], sh, sbias, kg);
  if (!ok) {
    // a wait ran out (ok is uniform over the block): record it, and mark this
    // block's bands of the map as missing (NaN), whatever was written there
    if (tid == 0) atomicOr(net.fault, 1);
    const BandLayer &ly = net.layer[5];
    const int H = net.H, W = net.W, nb = (H + ly.BH - 1) / ly.BH;
    const long long units = (long long)net.count * nb;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
      const int b = (int)(u / nb), j = (int)(u - (long long)b * nb);
      const int n = min(ly.BH, H - j * ly.BH) * W;
      float *o = reinterpret_cast<float *>(ly.out) + ((long long)b * H + j * ly.BH) * W;
      for (int i = tid; i < n; i += kBandThreads) o[i] = __int_as_float(0x7fc00000);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(sh.tmem),
                 "n"(2 * kBandCols));
}

// ------------------------------------------------------- weight gradient

// dW[co][tap][ci] += sum_p G[p][co] * X[p shifted by tap][ci]; db[co] += sum_p G[p][co].
// A block takes a run of 64 pixels at a time (grid-stride) and keeps the
// whole COUT x (9 CIN) gradient in registers over its runs, then adds it to
// global memory once. Rows = co (A = G^T), columns = (tap, ci), K = pixels.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) conv_wgrad_kernel(
    const __nv_bfloat16 *__restrict__ X, const __nv_bfloat16 *__restrict__ G, int dil, int H,
    int W, long long total, float *__restrict__ dW, float *__restrict__ db) {
  constexpr int PIX = 64;
  constexpr int NCOL = 9 * CIN;          // GEMM columns
  constexpr int NT = NCOL / 8;           // n-tiles
  constexpr int MT = COUT / 16;          // m-tiles (COUT multiple of 16)
  constexpr int NT_W = (NT + 3) / 4;     // n-tiles per warp
  static_assert(COUT % 16 == 0 && CIN % 16 == 0, "tile");
  __shared__ __align__(16) __nv_bfloat16 gs[PIX][COUT];
  __shared__ __align__(16) __nv_bfloat16 xs[9][PIX][CIN];
  __shared__ float dbs[COUT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, q = lane & 3;
  const long long plane = (long long)H * W;
  for (int c = threadIdx.x; c < COUT; c += blockDim.x) dbs[c] = 0.f;
  float acc[MT][NT_W][4];
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT_W; ++n) acc[m][n][0] = acc[m][n][1] = acc[m][n][2] = acc[m][n][3] = 0.f;
  float dbl = 0.f;  // bias partial of channel threadIdx.x (when < COUT)
  for (long long base = (long long)blockIdx.x * PIX; base < total;
       base += (long long)gridDim.x * PIX) {
    __syncthreads();
    // stage G (PIX x COUT) and the nine shifted copies of X (PIX x CIN), zero padded
    for (int i = threadIdx.x; i < PIX * COUT / 2; i += blockDim.x) {
      const int pix = i / (COUT / 2), c2 = (i - pix * (COUT / 2)) * 2;
      const long long p = base + pix;
      uint32_t v = 0u;
      if (p < total) v = *reinterpret_cast<const uint32_t *>(G + p * COUT + c2);
      *reinterpret_cast<uint32_t *>(&gs[pix][c2]) = v;
    }
    for (int i = threadIdx.x; i < 9 * PIX * CIN / 2; i += blockDim.x) {
      const int tap = i / (PIX * CIN / 2);
      const int rem = i - tap * (PIX * CIN / 2);
      const int pix = rem / (CIN / 2), c2 = (rem - pix * (CIN / 2)) * 2;
      const long long p = base + pix;
      uint32_t v = 0u;
      if (p < total) {
        const int b = (int)(p / plane);
        const int r2 = (int)(p - (long long)b * plane);
        const int y = r2 / W + (tap / 3 - 1) * dil, x = r2 % W + (tap % 3 - 1) * dil;
        if (y >= 0 && y < H && x >= 0 && x < W)
          v = *reinterpret_cast<const uint32_t *>(X + (((long long)b * H + y) * W + x) * CIN + c2);
      }
      *reinterpret_cast<uint32_t *>(&xs[tap][pix][c2]) = v;
    }
    __syncthreads();
    if (threadIdx.x < COUT) {
      float s = 0.f;
      for (int pix = 0; pix < PIX; ++pix) s += __bfloat162float(gs[pix][threadIdx.x]);
      dbl += s;
    }
#pragma unroll
    for (int k0 = 0; k0 < PIX; k0 += 16) {
#pragma unroll
      for (int m = 0; m < MT; ++m) {
        // A[co][pix]: rows co = m*16 + g (+8), cols pix = k0 + 2q (+1) (+8)
        const int co = m * 16 + g;
        uint32_t a[4];
        a[0] = pack_raw(gs[k0 + 2 * q][co], gs[k0 + 2 * q + 1][co]);
        a[1] = pack_raw(gs[k0 + 2 * q][co + 8], gs[k0 + 2 * q + 1][co + 8]);
        a[2] = pack_raw(gs[k0 + 2 * q + 8][co], gs[k0 + 2 * q + 9][co]);
        a[3] = pack_raw(gs[k0 + 2 * q + 8][co + 8], gs[k0 + 2 * q + 9][co + 8]);
#pragma unroll
        for (int n = 0; n < NT_W; ++n) {
          const int nt = warp * NT_W + n;
          if (nt >= NT) break;
          // B[pix][col]: col = nt*8 + g -> (tap, ci); rows pix = k0 + 2q (+1) (+8)
          const int col = nt * 8 + g, tap = col / CIN, ci = col - tap * CIN;
          uint32_t b[2];
          b[0] = pack_raw(xs[tap][k0 + 2 * q][ci], xs[tap][k0 + 2 * q + 1][ci]);
          b[1] = pack_raw(xs[tap][k0 + 2 * q + 8][ci], xs[tap][k0 + 2 * q + 9][ci]);
          mma_bf16(acc[m][n], a, b);
        }
      }
    }
  }
  // C[co][col]: acc[m][n][0..1] -> row m*16+g, cols nt*8 + 2q + {0,1}; [2..3] -> row +8
#pragma unroll
  for (int m = 0; m < MT; ++m)
#pragma unroll
    for (int n = 0; n < NT_W; ++n) {
      const int nt = warp * NT_W + n;
      if (nt >= NT) break;
      const int col = nt * 8 + q * 2;
      const int co = m * 16 + g;
      // dW layout [co][tap][ci] == [co][col]
      atomicAdd(dW + (long long)co * NCOL + col, acc[m][n][0]);
      atomicAdd(dW + (long long)co * NCOL + col + 1, acc[m][n][1]);
      atomicAdd(dW + (long long)(co + 8) * NCOL + col, acc[m][n][2]);
      atomicAdd(dW + (long long)(co + 8) * NCOL + col + 1, acc[m][n][3]);
    }
  if (threadIdx.x < COUT) atomicAdd(db + threadIdx.x, dbl);
}

// ------------------------------------------------------ loss, weights, adam

// Huber (delta 1) loss of channel 0 of z6 (p x 16 f32) against label
// (NaN = no label), averaged over all pixels; its gradient into g6 (p x 16 bf16).
__global__ void loss_kernel(const float *__restrict__ z6, const float *__restrict__ label,
                            long long total, float inv_n, __nv_bfloat16 *__restrict__ g6,
                            float *__restrict__ loss_sum) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f, gr = 0.f;
  if (p < total) {
    const float y = label[p];
    if (isfinite(y)) {
      const float e = z6[p * 16] - y;
      const float ae = fabsf(e);
      l = ae <= 1.f ? 0.5f * e * e : ae - 0.5f;
      gr = (ae <= 1.f ? e : copysignf(1.f, e)) * inv_n;
    }
    uint4 *dst = reinterpret_cast<uint4 *>(g6 + p * 16);
    dst[0] = make_uint4(pack_bf16(gr, 0.f), 0u, 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && loss_sum) atomicAdd(loss_sum, l * inv_n);
}

// Master weights (f32, real channels) -> padded bf16 forward weights
// [coutP][9][cinP] and, for layers > 0, the transposed tap-flipped copies the
// data gradient uses: [cinP][9][coutP] with wt_t[ci][t][co] = w[co][8-t][ci].
__global__ void pack_weights_kernel(const float *__restrict__ master, __nv_bfloat16 *fwd,
                                    __nv_bfloat16 *bwd, int layer_offset, int cin, int cout,
                                    int cinP, int coutP) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = coutP * 9 * cinP;
  if (i >= n) return;
  const int co = i / (9 * cinP), rem = i - co * 9 * cinP, t = rem / cinP, ci = rem - t * cinP;
  float v = 0.f;
  if (co < cout && ci < cin) v = master[layer_offset + (co * 9 + t) * cin + ci];
  fwd[i] = __float2bfloat16_rn(v);
  if (bwd) bwd[(ci * 9 + (8 - t)) * coutP + co] = __float2bfloat16_rn(v);
}

__global__ void bias_pad_kernel(const float *__restrict__ master, float *bias, int off, int cout,
                                int coutP) {
  const int c = threadIdx.x;
  if (c < coutP) bias[c] = c < cout ? master[off + c] : 0.f;
}

// Adam on the master weights; gradients are gathered from the padded
// per-layer gradient buffers.
__global__ void adam_kernel(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ grad, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gr = grad[i];
  const float mi = b1 * m[i] + (1.f - b1) * gr;
  const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Padded per-layer gradients [coutP][9][cinP] + [coutP] -> master order.
__global__ void gather_grad_kernel(const float *__restrict__ dWp, const float *__restrict__ dbp,
                                   float *__restrict__ grad, int off, int cin, int cout,
                                   int cinP) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int nw = cout * 9 * cin;
  if (i < nw) {
    const int co = i / (9 * cin), rem = i - co * 9 * cin, t = rem / cin, ci = rem - t * cin;
    grad[off + i] = dWp[(co * 9 + t) * cinP + ci];
  } else if (i < nw + cout) {
    grad[off + i] = dbp[i - nw];
  }
}

// Level-3 net output (channel 0 of z6) -> plain map.
__global__ void take_channel0_kernel(const float *__restrict__ z6, long long total, float *out) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < total) out[p] = z6[p * 16];
}

inline unsigned nblocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

struct bdis_net {
  int device = 0;
  // master weights and Adam state (f32, real channels, master order)
  float *w = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  // per-layer padded bf16 weights, transposed copies, padded biases, padded grads
  __nv_bfloat16 *wf[kLayers] = {}, *wb[kLayers] = {};
  float *bias[kLayers] = {}, *dW[kLayers] = {}, *db[kLayers] = {};
  float *loss = nullptr;
  long long step = 0;
  // activations for `cap` pixels
  long long cap = 0;
  __nv_bfloat16 *x0 = nullptr, *a[5] = {}, *gbuf[2] = {}, *g6 = nullptr;
  float *z6 = nullptr;
  // device word set when a forward kernel's bounded wait ran out
  int *fault = nullptr;
  unsigned *sync = nullptr;  // grid barrier counter of the fused inference kernel
  // inference activations in the padded planar layout, for pp_h x pp_w x pp_count
  __nv_bfloat16 *x0pp = nullptr, *app[5] = {};
  int pp_h = 0, pp_w = 0, pp_count = 0;
};

namespace {

void net_free_acts(bdis_net *n) {
  cudaFree(n->x0);
  for (auto &p : n->a) cudaFree(p);
  for (auto &p : n->gbuf) cudaFree(p);
  cudaFree(n->g6);
  cudaFree(n->z6);
  n->x0 = nullptr;
  for (auto &p : n->a) p = nullptr;
  for (auto &p : n->gbuf) p = nullptr;
  n->g6 = nullptr;
  n->z6 = nullptr;
  n->cap = 0;
}

void net_free_pp(bdis_net *n) {
  cudaFree(n->x0pp);
  for (auto &p : n->app) cudaFree(p);
  n->x0pp = nullptr;
  for (auto &p : n->app) p = nullptr;
  n->pp_h = n->pp_w = n->pp_count = 0;
}

// Padded planar activations of the inference pass for count h x w images,
// zeroed (borders and guards stay zero: only real pixels are ever written).
bdis_status net_reserve_pp(bdis_net *n, int h, int w, int count, cudaStream_t st) {
  if (n->pp_h == h && n->pp_w == w && n->pp_count == count) return BDIS_OK;
  net_free_pp(n);
  const size_t plane = (size_t)pp_plane(h, w, count) * sizeof(__nv_bfloat16);
  cudaError_t e = bdis::device_alloc((void **)&n->x0pp, 2 * plane);
  for (auto &p : n->app)
    if (e == cudaSuccess) e = bdis::device_alloc((void **)&p, 4 * plane);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->x0pp, 0, 2 * plane, st);
  for (auto &p : n->app)
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, 4 * plane, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    net_free_pp(n);
    return e == cudaErrorMemoryAllocation ? BDIS_E_NOMEM : bdis::record_cuda(e);
  }
  n->pp_h = h;
  n->pp_w = w;
  n->pp_count = count;
  return BDIS_OK;
}

bdis_status net_reserve(bdis_net *n, long long pixels) {
  if (pixels <= n->cap) return BDIS_OK;
  net_free_acts(n);
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = bdis::device_alloc(p, bytes);
  };
  alloc((void **)&n->x0, pixels * 16 * 2);
  for (auto &p : n->a) alloc((void **)&p, pixels * 32 * 2);
  for (auto &p : n->gbuf) alloc((void **)&p, pixels * 32 * 2);
  alloc((void **)&n->g6, pixels * 16 * 2);
  alloc((void **)&n->z6, pixels * 16 * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    net_free_acts(n);
    return BDIS_E_NOMEM;
  }
  n->cap = pixels;
  return BDIS_OK;
}

cudaError_t pack_all(bdis_net *n, cudaStream_t st) {
  for (int l = 0; l < kLayers; ++l) {
    const int cnt = kCoutP[l] * 9 * kCinP[l];
    pack_weights_kernel<<<nblocks(cnt, 256), 256, 0, st>>>(n->w, n->wf[l], l > 0 ? n->wb[l] : nullptr,
                                                           master_w_offset(l), kCin[l], kCout[l],
                                                           kCinP[l], kCoutP[l]);
    bias_pad_kernel<<<1, 32, 0, st>>>(n->w, n->bias[l],
                                      master_w_offset(l) + kCout[l] * 9 * kCin[l], kCout[l],
                                      kCoutP[l]);
  }
  return cudaGetLastError();
}

int g_sms = 0;
// forward convolutions: 1 = banded tcgen05 kernel for inference (default; training
// forwards and inputs too wide for it take the per-tile one), 2 = per-tile tcgen05
// kernel, 0 = mma.sync kernel
int g_net_tc = 1;

// Dynamic shared memory of the tcgen05 kernel is exactly its slab and the
// weights (19 to 72 KB for 80-pixel-wide inputs), so up to four
// blocks share an SM: some stage their slab while others multiply. (Double-
// buffering the slab within a block measured slower: it halves the blocks per
// SM.) Images too wide for one slab (over ~200 KB) take the mma.sync kernel.
constexpr int kTcSmemMax = 200 * 1024;

template <int CIN, int COUT, int MODE>
bool conv_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias, int dil,
             int H, int W, long long total, void *out, int *fault, cudaStream_t st) {
  const int smem = tc_smem_bytes<CIN, COUT>(dil, W);
  if (smem > kTcSmemMax) return false;
  // the shared-memory limit is a per-device attribute of the kernel
  static uint64_t attr_set = 0;  // bit d: set on device d
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(attr_set >> dev & 1u)) {
    if (cudaFuncSetAttribute(conv_tc_kernel<CIN, COUT, MODE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kTcSmemMax) != cudaSuccess) {
      cudaGetLastError();  // not sticky: clear it, the mma.sync kernel runs instead
      return false;
    }
    if (dev < 64) attr_set |= 1ull << dev;
  }
  const int count = (int)(total / ((long long)H * W));
  const long long totalp = (long long)(H + 2 * dil) * (W + 2 * dil) * count;
  const long long tiles = (totalp + 127) / 128;
  const int per_sm = std::max(1, std::min(4, (227 * 1024) / (smem + 1024)));
  const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)per_sm * g_sms);
  conv_tc_kernel<CIN, COUT, MODE><<<grid, 128, smem, st>>>(in, wt, bias, dil, H, W, count, out,
                                                             fault);
  return true;
}

void init_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&g_sms, cudaDevAttrMultiProcessorCount, dev);
  if (g_sms <= 0) g_sms = 152;
}

template <int CIN, int COUT, int MODE>
void conv(const __nv_bfloat16 *in, const __nv_bfloat16 *wt, const float *bias, int dil, int H,
          int W, long long total, const __nv_bfloat16 *mask, void *out, int *fault,
          cudaStream_t st) {
  if (!g_sms) init_sms();
  if constexpr (MODE == kFwdRelu || MODE == kFwdLinearF32) {
    if (g_net_tc && conv_tc<CIN, COUT, MODE>(in, wt, bias, dil, H, W, total, out, fault, st))
      return;
  }
  const long long tiles = (total + 255) / 256;  // 64 pixels x 4 m-tiles per block tile
  const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)g_sms * 3);
  conv_mma_kernel<CIN, COUT, MODE><<<grid, 128, 0, st>>>(in, wt, bias, dil, H, W, total, mask,
                                                         out);
}

// Band height of one layer of the fused kernel: the tallest band whose two
// slabs fit the shared memory beside the largest layer's weights and whose
// tiles fit one accumulator's tensor-memory columns; 0 if none does (images
// too wide: the per-tile kernels run instead).
constexpr int kBandWeightsMax = 36 * 4 * 128;  // 32 -> 32 channels, 9 taps

template <int CIN, int COUT>
int band_rows(int dil, int H, int W, int *nsb_out) {
  const int Wp = W + 2 * kPad, soff = dil * Wp + dil;
  for (int bh = H; bh >= 1; --bh) {
    const int tiles = (bh * Wp + 127) / 128;
    if (tiles * COUT > kBandCols) continue;
    const int nsb = tiles * 128 + 2 * soff;
    if (2 * (CIN / 8) * nsb * 16 + kBandWeightsMax <= kBandSmem) {
      *nsb_out = nsb;
      return bh;
    }
  }
  return 0;
}

// The inference forward pass as one cooperative launch of net_forward_kernel:
// level planes in, the proposal (channel 0 of the last layer) written straight
// to `out`. Returns false, having launched nothing, when the images are too
// wide for it or the device cannot run the grid cooperatively.
bool forward_pp(bdis_net *n, const float *L3, const float *R3, int r_stride, int H, int W,
                int count, float *out, cudaStream_t st) {
  if (g_net_tc != 1) return false;
  BandNet net{};
  int nsb[6], bh[6];
  bh[0] = band_rows<16, 32>(kDil[0], H, W, &nsb[0]);
  for (int l = 1; l < 5; ++l) bh[l] = band_rows<32, 32>(kDil[l], H, W, &nsb[l]);
  bh[5] = band_rows<32, 16>(kDil[5], H, W, &nsb[5]);
  // Band heights. Small batches: bands of fewer rows, so that a layer's
  // bands spread over the SMs (a single 40x30 image would otherwise be two
  // bands on two SMs, the rest waiting at the grid barriers). Then the bands
  // of an image are made equal (30 rows: 15 + 15, not 21 + 9): blocks take
  // bands round robin, and unequal bands would give every other block all
  // the tall ones. A proposal does not depend on the band height: each
  // position's MMAs and epilogue are the same.
  const int per_image = (g_sms + count - 1) / count;  // bands wanted per image
  const int want = std::max(1, (H + per_image - 1) / per_image);
  int slab = 0;
  for (int l = 0; l < 6; ++l) {
    if (!bh[l]) return false;
    const int nb = (H + std::min(want, bh[l]) - 1) / std::min(want, bh[l]);
    const int even = (H + nb - 1) / nb;  // <= bh[l]: the limits still hold
    if (even < bh[l]) {
      const int Wp = W + 2 * kPad, soff = kDil[l] * Wp + kDil[l];
      bh[l] = even;
      nsb[l] = (even * Wp + 127) / 128 * 128 + 2 * soff;
    }
    slab = std::max(slab, (kCinP[l] / 8) * nsb[l] * 16);
  }
  const int smem = 2 * slab + kBandWeightsMax;
  static uint64_t attr_set = 0;  // bit d: the shared-memory limit is set on device d
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(attr_set >> dev & 1u)) {
    if (cudaFuncSetAttribute(net_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kBandSmem) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    if (dev < 64) attr_set |= 1ull << dev;
  }
  const __nv_bfloat16 *ins[6] = {n->x0pp, n->app[0], n->app[1], n->app[2], n->app[3], n->app[4]};
  for (int l = 0; l < 6; ++l) {
    net.layer[l].in = ins[l];
    net.layer[l].wt = n->wf[l];
    net.layer[l].bias = n->bias[l];
    net.layer[l].out = l < 5 ? (void *)n->app[l] : (void *)out;
    net.layer[l].dil = kDil[l];
    net.layer[l].BH = bh[l];
    net.layer[l].nsb = nsb[l];
  }
  net.L = L3;
  net.R = R3;
  net.r_stride = r_stride;
  net.H = H;
  net.W = W;
  net.count = count;
  net.slab_bytes = slab;
  net.sync = n->sync;
  net.fault = n->fault;
  if (cudaMemsetAsync(n->sync, 0, sizeof(unsigned), st) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // one block per SM, or one per band where a layer has fewer bands (a
  // single image): fewer blocks meet at each grid barrier and restage the
  // weights
  long long units = 1;
  for (int l = 0; l < 6; ++l)
    units = std::max(units, (long long)count * ((H + bh[l] - 1) / bh[l]));
  const unsigned grid = (unsigned)std::min<long long>(g_sms, units);
  void *args[] = {&net};
  if (cudaLaunchCooperativeKernel((const void *)net_forward_kernel, dim3(grid),
                                  dim3(kBandThreads), args, (size_t)smem, st) != cudaSuccess) {
    cudaGetLastError();  // not sticky: the per-tile kernels run instead
    return false;
  }
  return true;
}

cudaError_t forward(bdis_net *n, const float *L3, const float *R3, int r_stride, int H, int W,
                    long long total, cudaStream_t st) {
  pack_input_kernel<<<nblocks(total, 256), 256, 0, st>>>(L3, R3, r_stride, total, n->x0);
  conv<16, 32, kFwdRelu>(n->x0, n->wf[0], n->bias[0], kDil[0], H, W, total, nullptr, n->a[0],
                         n->fault, st);
  for (int l = 1; l < 5; ++l)
    conv<32, 32, kFwdRelu>(n->a[l - 1], n->wf[l], n->bias[l], kDil[l], H, W, total, nullptr,
                           n->a[l], n->fault, st);
  conv<32, 16, kFwdLinearF32>(n->a[4], n->wf[5], n->bias[5], kDil[5], H, W, total, nullptr,
                              n->z6, n->fault, st);
  return cudaGetLastError();
}

// Backward through all layers into the padded gradient buffers (zeroed here).
cudaError_t backward(bdis_net *n, int H, int W, long long total, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
    e = cudaMemsetAsync(n->dW[l], 0, sizeof(float) * kCoutP[l] * 9 * kCinP[l], st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n->db[l], 0, sizeof(float) * kCoutP[l], st);
  }
  if (e != cudaSuccess) return e;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, n->device);
  const unsigned wblocks = (unsigned)std::min<long long>((total + 63) / 64, (long long)sms * 4);
  // layer 6 (linear): gradient g6 of z6
  conv_wgrad_kernel<32, 16><<<wblocks, 128, 0, st>>>(n->a[4], n->g6, kDil[5], H, W, total,
                                                     n->dW[5], n->db[5]);
  // g5 = (W6^T g6) * relu'(a5)
  conv<16, 32, kBwdDataMasked>(n->g6, n->wb[5], nullptr, kDil[5], H, W, total, n->a[4],
                               n->gbuf[0], n->fault, st);
  int cur = 0;
  for (int l = 4; l >= 1; --l) {
    // gradient of layer l (0-based) output is gbuf[cur]; its input is a[l-1]
    conv_wgrad_kernel<32, 32><<<wblocks, 128, 0, st>>>(n->a[l - 1], n->gbuf[cur], kDil[l], H, W,
                                                       total, n->dW[l], n->db[l]);
    conv<32, 32, kBwdDataMasked>(n->gbuf[cur], n->wb[l], nullptr, kDil[l], H, W, total,
                                 n->a[l - 1], n->gbuf[cur ^ 1], n->fault, st);
    cur ^= 1;
  }
  conv_wgrad_kernel<16, 32><<<wblocks, 128, 0, st>>>(n->x0, n->gbuf[cur], kDil[0], H, W, total,
                                                     n->dW[0], n->db[0]);
  for (int l = 0; l < kLayers; ++l) {
    const int cnt = kCout[l] * 9 * kCin[l] + kCout[l];
    gather_grad_kernel<<<nblocks(cnt, 256), 256, 0, st>>>(n->dW[l], n->db[l], n->grad,
                                                          master_w_offset(l), kCin[l], kCout[l],
                                                          kCinP[l]);
  }
  return cudaGetLastError();
}

void net_release(bdis_net *n) {
  if (!n) return;
  net_free_acts(n);
  net_free_pp(n);
  cudaFree(n->w);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->grad);
  cudaFree(n->loss);
  cudaFree(n->fault);
  cudaFree(n->sync);
  for (int l = 0; l < kLayers; ++l) {
    cudaFree(n->wf[l]);
    cudaFree(n->wb[l]);
    cudaFree(n->bias[l]);
    cudaFree(n->dW[l]);
    cudaFree(n->db[l]);
  }
  delete n;
}

}  // namespace

namespace bdis {

bdis_status net_forward_on(bdis_net *n, const float *L, const float *R, int r_stride, int w,
                           int h, int count, float *out, cudaStream_t st) {
  const long long total = (long long)w * h * count;
  if (g_net_tc == 1) {
    if (!g_sms) init_sms();
    int nsb = 0;
    if (band_rows<32, 32>(4, h, w, &nsb) && band_rows<16, 32>(1, h, w, &nsb) &&
        band_rows<32, 16>(1, h, w, &nsb)) {
      bdis_status s = net_reserve_pp(n, h, w, count, st);
      if (s != BDIS_OK) return s;
      if (forward_pp(n, L, R, r_stride, h, w, count, out, st)) return record_cuda(cudaGetLastError());
    }
  }
  bdis_status s = net_reserve(n, total);
  if (s != BDIS_OK) return s;
  cudaError_t e = forward(n, L, R, r_stride, h, w, total, st);
  if (e == cudaSuccess) {
    take_channel0_kernel<<<nblocks(total, 256), 256, 0, st>>>(n->z6, total, out);
    e = cudaGetLastError();
  }
  return record_cuda(e);
}

}  // namespace bdis

extern "C" {

int bdis_net_weight_count(void) { return kMasterCount; }

void bdis_set_net_variant(int tensor_path) {
  g_net_tc = tensor_path < 0 ? 0 : (tensor_path > 2 ? 1 : tensor_path);
}

int bdis_get_net_variant(void) { return g_net_tc; }

bdis_status bdis_net_create(int device, const float *weights, bdis_net **out) {
  if (!out || !weights) return BDIS_E_INVALID_ARG;
  *out = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return bdis::record_cuda(e);
  bdis_net *n = new (std::nothrow) bdis_net();
  if (!n) return BDIS_E_NOMEM;
  n->device = device;
  auto alloc = [&](void **p, size_t bytes) {
    if (e == cudaSuccess) e = bdis::device_alloc(p, bytes);
  };
  const size_t wb = sizeof(float) * kMasterCount;
  alloc((void **)&n->w, wb);
  alloc((void **)&n->m, wb);
  alloc((void **)&n->v, wb);
  alloc((void **)&n->grad, wb);
  alloc((void **)&n->loss, sizeof(float));
  alloc((void **)&n->fault, sizeof(int));
  alloc((void **)&n->sync, sizeof(unsigned));
  for (int l = 0; l < kLayers; ++l) {
    alloc((void **)&n->wf[l], 2 * kCoutP[l] * 9 * kCinP[l]);
    if (l > 0) alloc((void **)&n->wb[l], 2 * kCoutP[l] * 9 * kCinP[l]);
    alloc((void **)&n->bias[l], sizeof(float) * kCoutP[l]);
    alloc((void **)&n->dW[l], sizeof(float) * kCoutP[l] * 9 * kCinP[l]);
    alloc((void **)&n->db[l], sizeof(float) * kCoutP[l]);
  }
  if (e == cudaSuccess) e = cudaMemcpy(n->w, weights, wb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(n->m, 0, wb);
  if (e == cudaSuccess) e = cudaMemset(n->v, 0, wb);
  if (e == cudaSuccess) e = cudaMemset(n->fault, 0, sizeof(int));
  if (e == cudaSuccess) e = pack_all(n, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaGetLastError();
    net_release(n);
    return e == cudaErrorMemoryAllocation ? BDIS_E_NOMEM : bdis::record_cuda(e);
  }
  *out = n;
  return BDIS_OK;
}

bdis_status bdis_net_forward(bdis_net *n, const float *L3, const float *R3, int r_stride,
                             int width, int height, int count, float *disparity, void *stream) {
  if (!n || !L3 || !R3 || !disparity || width < 1 || height < 1 || count < 1 ||
      (r_stride != 1 && r_stride != 2))
    return BDIS_E_INVALID_ARG;
  return bdis::net_forward_on(n, L3, R3, r_stride, width, height, count, disparity,
                              static_cast<cudaStream_t>(stream));
}

bdis_status bdis_net_gradient(bdis_net *n, const float *L3, const float *R3, int r_stride,
                              int width, int height, int count, const float *label,
                              float *loss_out, float *grad_out, void *stream) {
  if (!n || !L3 || !R3 || !label || width < 1 || height < 1 || count < 1 ||
      (r_stride != 1 && r_stride != 2))
    return BDIS_E_INVALID_ARG;
  const long long total = (long long)width * height * count;
  bdis_status s = net_reserve(n, total);
  if (s != BDIS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = forward(n, L3, R3, r_stride, height, width, total, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->loss, 0, sizeof(float), st);
  if (e == cudaSuccess) {
    loss_kernel<<<nblocks(total, 256), 256, 0, st>>>(n->z6, label, total, 1.f / (float)total,
                                                     n->g6, n->loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = backward(n, height, width, total, st);
  if (e == cudaSuccess && loss_out)
    e = cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad_out)
    e = cudaMemcpyAsync(grad_out, n->grad, sizeof(float) * kMasterCount, cudaMemcpyDeviceToHost,
                        st);
  if (e == cudaSuccess && (loss_out || grad_out)) e = cudaStreamSynchronize(st);
  return bdis::record_cuda(e);
}

bdis_status bdis_net_train_step(bdis_net *n, const float *L3, const float *R3, int r_stride,
                                int width, int height, int count, const float *label, float lr,
                                float *loss_out, void *stream) {
  bdis_status s = bdis_net_gradient(n, L3, R3, r_stride, width, height, count, label, nullptr,
                                    nullptr, stream);
  if (s != BDIS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  n->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)n->step), c2 = 1.f - powf(b2, (float)n->step);
  adam_kernel<<<nblocks(kMasterCount, 256), 256, 0, st>>>(n->w, n->m, n->v, n->grad, kMasterCount,
                                                          lr, b1, b2, 1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = pack_all(n, st);
  if (e == cudaSuccess && loss_out) {
    e = cudaMemcpyAsync(loss_out, n->loss, sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return bdis::record_cuda(e);
}

bdis_status bdis_net_get_weights(bdis_net *n, float *weights_out) {
  if (!n || !weights_out) return BDIS_E_INVALID_ARG;
  cudaError_t e = cudaSetDevice(n->device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(weights_out, n->w, sizeof(float) * kMasterCount, cudaMemcpyDeviceToHost);
  return bdis::record_cuda(e);
}

bdis_status bdis_net_status(bdis_net *n, void *stream) {
  if (!n) return BDIS_E_INVALID_ARG;
  int cur = -1;
  cudaError_t e = cudaGetDevice(&cur);
  if (e == cudaSuccess && cur != n->device) e = cudaSetDevice(n->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  int fault = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&fault, n->fault, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && fault) e = cudaMemset(n->fault, 0, sizeof(int));
  if (e != cudaSuccess) return bdis::record_cuda(e);
  if (fault) {
    bdis::set_last_error("proposal network: a forward pass's bounded wait ran out (its tile "
                         "was written as NaN)");
    return BDIS_E_TIMEOUT;
  }
  return BDIS_OK;
}

bdis_status bdis_net_inject_timeout(bdis_net *n) {
  if (!n) return BDIS_E_INVALID_ARG;
  const int one = 1;
  cudaError_t e = cudaSetDevice(n->device);
  if (e == cudaSuccess) e = cudaMemcpy(n->fault, &one, sizeof(int), cudaMemcpyHostToDevice);
  return bdis::record_cuda(e);
}

void bdis_net_destroy(bdis_net *n) {
  if (!n) return;
  cudaSetDevice(n->device);
  cudaDeviceSynchronize();
  net_release(n);
}

}  // extern "C"
