// search.cu -- patch-wise inverse search (Sec. 2.1, Eq. 1) with the Bayesian
// patch posterior (Sec. 2.2, Eqs. 3-4) and the patch tests, one kernel.
//
// Layout: one patch per group of G lanes (G = 4, 8, 16 or 32, the smallest
// power of two >= patch size), lane c owning column c of its patch and
// walking the rows. Per lane the template T and gradient g of its column stay
// in registers for the whole search; the right image is read with
// coalesced row loads (the G lanes of a group read consecutive pixels of one
// row) served mostly from L1/L2, since neighbouring patches overlap.
// Reductions over the patch are xor-butterflies inside the group.
//
// Arithmetic per patch (the method's own, Eq. 1 and Eq. 3):
//   - the valid set is a run of columns (rows are aligned), so its sums are
//     recomputed only when that run changes;
//   - with mean normalisation, sum g_n (R~_n - T_n) = sum g_c R~ - sum g_c T
//     where g_c is the gradient centred on the valid set, so an iteration is
//     two FMAs per pixel (interpolate, accumulate) and one group reduction;
//   - the window energies use two passes (mean, then squares) to keep the
//     saddle decisions well conditioned.
//
// Roofline: FP32/L1 bound. Algorithmic work per patch: ps^2 * (2*iters + 4*s)
// flops; unique DRAM bytes are only the level planes (12 B/px) plus 8 B per
// patch written.
#include "bdis_internal.cuh"

namespace bdis {
namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Split a sample position x - D into integer base and fraction computed from
// D alone (exact in float): x - D = (x + k) + t with t in [0, 1).
__device__ __forceinline__ void split_disp(float D, int &k, float &t) {
  float nd = fminf(fmaxf(-D, -1.0e7f), 1.0e7f);  // NaN -> bound, never in range
  float f = floorf(nd);
  k = (int)f;
  t = nd - f;
}

// Sample at (i0 + t) is inside [0, w-1].
__device__ __forceinline__ bool sample_ok(int i0, float t, int w) {
  return i0 >= 0 && (i0 < w - 1 || (i0 == w - 1 && t == 0.f));
}

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

template <int G>
__global__ void __launch_bounds__(128) search_kernel(const SearchArgs a) {
  const int lane = threadIdx.x & 31;
  const int c = lane & (G - 1);
  const unsigned gbits = (G == 32) ? kFull : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const long long gid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const bool live = gid < a.total;
  // Groups past the end redo the last patch (so every lane joins the
  // shuffles) and store nothing.
  const long long k = live ? gid : a.total - 1;
  const int b = (int)(k / a.np);
  const int kk = (int)(k - (long long)b * a.np);
  const int pj = kk / a.nx, pi = kk - (kk / a.nx) * a.nx;
  const int ps = a.ps, w = a.w;
  const int x0 = grid_origin(pi, a.nx, w, ps, a.stride);
  const int y0 = grid_origin(pj, a.ny, a.h, ps, a.stride);
  const bool act = c < ps;
  const int x = x0 + c;
  const float *Lp = a.L + (long long)b * a.plane;
  const float *Rp = a.R + (long long)b * a.plane;
  const float *Gp = a.G + (long long)b * a.plane;

  float T[G], g[G];
#pragma unroll
  for (int r = 0; r < G; ++r) {
    const bool in = act && r < ps;
    T[r] = in ? __ldg(Lp + (size_t)(y0 + r) * w + x) : 0.f;
    g[r] = in ? __ldg(Gp + (size_t)(y0 + r) * w + x) : 0.f;
  }

  // Coarse-to-fine start (Sec. 2.1): twice the coarser map at half the centre.
  float u0 = 0.f;
  if (a.coarse) {
    const float cx = (float)x0 + (ps - 1) * 0.5f, cy = (float)y0 + (ps - 1) * 0.5f;
    u0 = 2.f * bilinear_clamped(a.coarse + (long long)b * a.cplane, a.cw, a.ch, cx * 0.5f,
                                cy * 0.5f);
  }

  // ---- inverse-search iterations (Eq. 1)
  float D = u0;
  float last_step = 0.f;
  bool frozen = false, flat = false, have = false;
  unsigned prev = 0u;
  float gc[G];
#pragma unroll
  for (int r = 0; r < G; ++r) gc[r] = 0.f;
  float H = 0.f, gcT = 0.f;
  int n = 0;
  for (int it = 0; it < a.iters; ++it) {
    int kd;
    float t;
    split_disp(D, kd, t);
    const int i0 = x + kd;
    const bool v = act && sample_ok(i0, t, w);
    const unsigned m = __ballot_sync(kFull, v) & gbits;
    const bool need = !frozen && (!have || m != prev);
    if (__any_sync(kFull, need)) {
      // sums of the new valid set (normalised gradient, Hessian, template term)
      float sg = 0.f;
#pragma unroll
      for (int r = 0; r < G; ++r) sg += (v && r < ps) ? g[r] : 0.f;
      sg = group_sum<G>(sg);
      const int nn = ps * __popc(m);
      const float mg = (a.normalize && nn > 0) ? sg / (float)nn : 0.f;
      float hh = 0.f, ct = 0.f;
#pragma unroll
      for (int r = 0; r < G; ++r) {
        const float q = (v && r < ps) ? g[r] - mg : 0.f;
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
      const float *Rr = Rp + (size_t)y0 * w + i0;
      const int d1 = (i0 + 1 < w) ? 1 : 0;  // at the last column t == 0
#pragma unroll
      for (int r = 0; r < G; ++r) {
        if (r < ps) {
          const float r0 = __ldg(Rr + (size_t)r * w);
          const float r1 = __ldg(Rr + (size_t)r * w + d1);
          acc = fmaf(gc[r], fmaf(t, r1 - r0, r0), acc);
        }
      }
    }
    const float S = group_sum<G>(acc);
    if (!frozen) {
      last_step = (S - gcT) / H;
      D += last_step;
      // non-finite, or left the search range: no further steps (dropped below)
      if (!isfinite(D) || fabsf(D - u0) > (float)ps) frozen = true;
    }
  }

  // ---- Bayesian window (Eqs. 3-4) and patch tests
  const bool fin = isfinite(D);
  int kd;
  float t;
  split_disp(D, kd, t);
  const bool v0 = act && fin && sample_ok(x + kd, t, w);
  const int nvalid = ps * __popc(__ballot_sync(kFull, v0) & gbits);
  const int half = (a.s - 1) / 2;
  bool vc = act && fin;
  for (int i = 0; i < a.s; ++i) {
    split_disp(D + (float)(i - half) * a.step, kd, t);
    vc = vc && sample_ok(x + kd, t, w);
  }
  const int nc = ps * __popc(__ballot_sync(kFull, vc) & gbits);

  float Ec = 0.f, Eo = INFINITY, Emin = INFINITY, z = 0.f;
  const float inv_kappa = 1.f / a.kappa;
  const bool write = live && c == 0;
  const long long eoff = k * a.s;
  for (int i = 0; i < a.s; ++i) {
    split_disp(D + (float)(i - half) * a.step, kd, t);
    const int i0 = x + kd;
    const int d1 = (i0 + 1 < w) ? 1 : 0;
    float dres[G];
    float sd = 0.f;
#pragma unroll
    for (int r = 0; r < G; ++r) {
      dres[r] = 0.f;
      if (vc && r < ps) {
        const float *Rr = Rp + (size_t)(y0 + r) * w + i0;
        const float r0 = __ldg(Rr), r1 = __ldg(Rr + d1);
        dres[r] = fmaf(t, r1 - r0, r0) - T[r];
        sd += dres[r];
      }
    }
    float md = 0.f;
    if (a.normalize) {
      sd = group_sum<G>(sd);
      md = nc > 0 ? sd / (float)nc : 0.f;
    }
    float e = 0.f;
#pragma unroll
    for (int r = 0; r < G; ++r) {
      if (vc && r < ps) {
        const float q = dres[r] - md;
        e = fmaf(q, q, e);
      }
    }
    const float E = group_sum<G>(e);
    if (write && a.energies) a.energies[eoff + i] = E;
    if (i == half) Ec = E;
    else Eo = fminf(Eo, E);
    // streaming sum of exp(-(E_i - Emin) / kappa)
    if (E < Emin) {
      z = (Emin == INFINITY ? 0.f : z * expf(-(Emin - E) * inv_kappa)) + 1.f;
      Emin = E;
    } else {
      z += expf(-(E - Emin) * inv_kappa);
    }
  }

  uint8_t flags = flat ? kFlagFlat : 0;
  if (!fin || fabsf(D - u0) > (float)ps) flags |= kFlagDiverged;
  if (fabsf(last_step) > kConvergeTol) flags |= kFlagUnconverged;
  float post = 0.f;
  if (nc == 0) {
    flags |= kFlagEmpty;
  } else {
    post = expf(-(Ec - Emin) * inv_kappa) / z;
    if (a.s > 1 && Eo < Ec - kSaddleTau * fmaxf(Ec, 1.f)) flags |= kFlagSaddle;
  }
  if (nvalid < a.nmin_valid) flags |= kFlagGamma;
  const bool drop = (flags & kDropFlags) != 0;

  if (write) {
    a.d_star[k] = D;
    a.weight[k] = drop ? 0.f : post * (float)nvalid / (float)(ps * ps);
    if (a.u_init) a.u_init[k] = u0;
    if (a.posterior) a.posterior[k] = post;
    if (a.flags) a.flags[k] = flags;
    if (a.n_valid) a.n_valid[k] = nvalid;
  }
}

template <int G>
cudaError_t launch_g(const SearchArgs &a, cudaStream_t st) {
  const int threads = 128;
  const long long lanes = a.total * G;
  const unsigned blocks = (unsigned)((lanes + threads - 1) / threads);
  search_kernel<G><<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

void fill_search_args(SearchArgs &a, int w, int h, int count, const bdis_params &p) {
  a.w = w;
  a.h = h;
  a.plane = (long long)w * h;
  a.ps = p.patch_size;
  a.stride = grid_stride(p.patch_size, p.overlap);
  a.nx = grid_count(w, p.patch_size, a.stride);
  a.ny = grid_count(h, p.patch_size, a.stride);
  a.np = a.nx * a.ny;
  a.total = (long long)a.np * count;
  a.iters = p.iterations;
  a.s = p.window_samples;
  a.step = p.window_step;
  a.kappa = 2.f * p.sigma_r * p.sigma_r * (float)(p.window_samples * p.window_samples);
  a.nmin_valid = gamma_min_count(p.gamma, p.patch_size);
  a.normalize = p.normalize ? 1 : 0;
}

cudaError_t launch_search(const SearchArgs &a, cudaStream_t st) {
  if (a.total == 0) return cudaSuccess;
  if (a.ps <= 4) return launch_g<4>(a, st);
  if (a.ps <= 8) return launch_g<8>(a, st);
  if (a.ps <= 16) return launch_g<16>(a, st);
  return launch_g<32>(a, st);
}

}  // namespace bdis
