/*
 * bdis_oracle.c -- FP64 CPU oracle of Bayesian Dense Inverse Search (BDIS),
 * Song et al., "Bayesian dense inverse searching algorithm for real-time
 * stereo matching in minimally invasive surgery", arXiv 2106.07136.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * restatement of the method that the CUDA path is checked against. Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline leg
 * may build, load or call it. It shares no code, header or constant table
 * with the CUDA library.
 *
 * Everything is double precision and single threaded. Each function follows
 * one step of the method in the order the paper gives it:
 *   - image pyramid, coarse to fine (Sec. 2.1, Fig. 1);
 *   - patch-wise inverse-search Lucas-Kanade (Sec. 2.1, Eq. 1);
 *   - Bayesian patch posterior over a window of disparities (Sec. 2.2,
 *     Eqs. 3-4), with the saddle-point / convergence filter (Sec. 2.2) and
 *     the valid-pixel threshold gamma (Sec. 3, Sec. 3.2);
 *   - densification with the spatial Gaussian mask (Sec. 2.3, Eq. 5 and the
 *     combined pixel-wise posterior that follows it);
 *   - uncovered pixels are left unestimated (Sec. 3.2);
 *   - DIS mode: the paper's baseline fusion by inverse residual (Eq. 2).
 *
 * Where the paper leaves a detail open, the reading taken here is named at
 * the point of use (R1..R12); the same list is kept in the design notes.
 *
 * Parity status per function:
 *   orc_level_dim, orc_grid_*           pinned (closed-form counts)
 *   orc_downsample, orc_sobel_x         pinned (polynomial closed forms)
 *   orc_search_patch                    pinned (exact shifts, linear texture
 *                                        closed form, bisection fixed point,
 *                                        brute-force SSD, flat texture)
 *   orc_densify_level                   pinned (constant field, single and
 *                                        two-patch closed forms; DIS weights
 *                                        on an exact linear texture)
 *   orc_match                           pinned through the exact-shift and
 *                                        linear-texture pairs; on mixed
 *                                        scenes the result is "parity
 *                                        unpinned" beyond those invariants.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Parameters of the method. Names follow the paper's notation where it has
 * one (sigma_r, sigma_s, s = window_samples, gamma; Sec. 3). */
typedef struct {
    int patch_size;      /* side of the square patch, pixels (Sec. 1) */
    double overlap;      /* fraction of the patch shared with the next one */
    int iterations;      /* inverse-search iterations per patch and scale */
    int coarsest_scale;  /* pyramid level where the search starts */
    int finest_scale;    /* pyramid level where it ends */
    double sigma_r;      /* brightness std of the Boltzmann likelihood, Eq. 4 */
    double sigma_s;      /* spatial std of the Gaussian mask, Eq. 5 */
    int window_samples;  /* s: candidates in the Bayesian window, Eq. 3 */
    double window_step;  /* spacing of the candidates in pixels */
    double gamma;        /* minimum fraction of valid pixels in a patch */
    int normalize;       /* 1: patch mean normalisation (DIS default) */
    int fusion;          /* 0: BDIS (Eqs. 3-5), 1: DIS inverse-residual fusion (Eq. 2) */
} orc_params;

#define ORC_FUSION_BDIS 0
#define ORC_FUSION_DIS 1

/* Per-patch flags. Only FLAG_FLAT does not discard the patch. */
enum {
    ORC_FLAG_FLAT = 1,      /* no gradient energy: no update possible */
    ORC_FLAG_DIVERGED = 2,  /* |D* - u_init| > patch size, or non-finite */
    ORC_FLAG_SADDLE = 4,    /* D* is not the minimum of its window (Sec. 2.2) */
    ORC_FLAG_GAMMA = 8,     /* valid-pixel fraction below gamma (Sec. 3) */
    ORC_FLAG_EMPTY = 16,    /* no pixel valid at every window sample */
    ORC_FLAG_UNCONVERGED = 32 /* last update above ORC_CONVERGE_TOL (Sec. 3.2) */
};

/* Saddle tolerance (R7), flat-patch threshold (R5) and the largest final
 * update, in pixels, of a patch that counts as converged (R8). */
#define ORC_SADDLE_TAU 1e-6
#define ORC_FLAT_EPS 1e-4
#define ORC_CONVERGE_TOL 0.02
/* A patch whose update falls below this (px) has converged: no more steps. */
#define ORC_STEP_TOL 1e-4
#define ORC_SAME_SOLUTION 0.1 /* px of the level searched twice (R16) */

/* ---------------------------------------------------------------- geometry */

/* Size of pyramid level `level` along an axis of n pixels (R2: ceil halving). */
int orc_level_dim(int n, int level)
{
    for (int l = 0; l < level; ++l) n = (n + 1) / 2;
    return n;
}

/* Patch stride from size and overlap (R3): round(ps * (1 - overlap)), >= 1. */
int orc_grid_stride(int ps, double overlap)
{
    int s = (int)floor(ps * (1.0 - overlap) + 0.5);
    return s < 1 ? 1 : s;
}

/* Number of patch origins along an axis of n pixels (R3). */
int orc_grid_count(int n, int ps, int stride)
{
    if (n < ps) return 0;
    return (n - ps + stride - 1) / stride + 1;
}

/* Origin of patch i along an axis: i*stride, the last one moved to n - ps so
 * that the grid reaches the image border (R3). */
int orc_grid_origin(int i, int count, int n, int ps, int stride)
{
    return (i == count - 1) ? n - ps : i * stride;
}

/* --------------------------------------------------------------- pyramid */

/* Reflect-101 border: -1 -> 1, n -> n - 2 (R2). */
static int reflect101(int i, int n)
{
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

/* One pyramid step (Sec. 2.1: the images are resized to coarser scales).
 * R2: 5x5 binomial [1 4 6 4 1]/16 in each axis, reflect-101 border, keep the
 * even samples. dst is ceil(w/2) x ceil(h/2); dst(X, Y) sits on src(2X, 2Y). */
void orc_downsample(const double *src, int w, int h, double *dst)
{
    static const double b[5] = {1.0 / 16, 4.0 / 16, 6.0 / 16, 4.0 / 16, 1.0 / 16};
    int dw = (w + 1) / 2, dh = (h + 1) / 2;
    for (int Y = 0; Y < dh; ++Y)
        for (int X = 0; X < dw; ++X) {
            double acc = 0.0;
            for (int j = -2; j <= 2; ++j)
                for (int i = -2; i <= 2; ++i) {
                    int x = reflect101(2 * X + i, w);
                    int y = reflect101(2 * Y + j, h);
                    acc += b[i + 2] * b[j + 2] * src[(size_t)y * w + x];
                }
            dst[(size_t)Y * dw + X] = acc;
        }
}

/* Template gradient along x (Sec. 2.1: the inverse search takes the gradient
 * of the left patch only; stereo makes it one-dimensional). Sobel-x / 8 with a
 * reflect-101 border, so that a linear ramp of slope a gives exactly a. */
void orc_sobel_x(const double *img, int w, int h, double *gx)
{
    static const double s[3] = {1.0, 2.0, 1.0};
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double acc = 0.0;
            for (int j = -1; j <= 1; ++j) {
                int yy = reflect101(y + j, h);
                acc += s[j + 1] * (img[(size_t)yy * w + reflect101(x + 1, w)] -
                                   img[(size_t)yy * w + reflect101(x - 1, w)]);
            }
            gx[(size_t)y * w + x] = acc / 8.0;
        }
}

/* ------------------------------------------------------------- sampling */

/* Right image sampled at (xs, y) by linear interpolation along the row
 * (rows are aligned after rectification, Sec. 3). Valid iff 0 <= xs <= w-1. */
static double sample_row(const double *R, int w, int y, double xs, int *valid)
{
    if (!(xs >= 0.0 && xs <= (double)(w - 1))) {
        *valid = 0;
        return 0.0;
    }
    *valid = 1;
    int i0 = (int)floor(xs);
    if (i0 > w - 2) i0 = w - 2;
    double t = xs - i0;
    const double *row = R + (size_t)y * w;
    return (1.0 - t) * row[i0] + t * row[i0 + 1];
}

/* Bilinear read of a level map at real coordinates, clamped to the map. */
static double bilinear_clamped(const double *M, int w, int h, double x, double y)
{
    if (x < 0.0) x = 0.0;
    if (y < 0.0) y = 0.0;
    if (x > w - 1) x = w - 1;
    if (y > h - 1) y = h - 1;
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
    int y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double tx = x - x0, ty = y - y0;
    double top = (1.0 - tx) * M[(size_t)y0 * w + x0] + tx * M[(size_t)y0 * w + x1];
    double bot = (1.0 - tx) * M[(size_t)y1 * w + x0] + tx * M[(size_t)y1 * w + x1];
    return (1.0 - ty) * top + ty * bot;
}

/* ------------------------------------------------- inverse search, Eq. 1 */

typedef struct {
    double u_init;
    double d_star;
    double posterior;
    double weight;
    int flags;
    int n_valid;
    int steps; /* updates applied to D (R12: at most `iterations`) */
} orc_patch_result;

/* Inverse-search Lucas-Kanade for one patch (Sec. 2.1, Eq. 1), then the
 * Bayesian window (Sec. 2.2, Eqs. 3-4) and the patch tests.
 *
 * R1: D = -u >= 0 with I_l(x) ~ I_r(x - D). Linearising the template,
 *     I_r(x - D) - I_l(x) ~ g(x) (D_true - D), so each step is
 *     D <- D + sum g (R~ - T) / sum g^2 with the Hessian taken once from the
 *     left patch (the point of the inverse formulation).
 * R5: with normalize = 1, T, R~ and g are mean-subtracted over the pixels
 *     valid at the current D; the step is the Gauss-Newton step of the
 *     normalised objective. A patch whose Hessian is below ORC_FLAT_EPS per
 *     pixel (or with no valid pixel) is flat and gets no further update.
 * R8: a patch that moves more than ps from its start has left its search
 *     range and is abandoned there (no further steps, dropped); a patch
 *     whose last step is still above ORC_CONVERGE_TOL has not converged and
 *     is dropped (Sec. 3.2 discards the patches that do not converge).
 * R12: at most `iterations` steps; a patch stops early when it is flat, when
 *     it leaves its search range, or when its update falls below
 *     ORC_STEP_TOL (further steps would move it by less than that).
 * energies[] receives s values (may be NULL). */
void orc_search_patch(const double *L, const double *R, const double *G, int w, int h,
                      int x0, int y0, double u_init, const orc_params *p,
                      orc_patch_result *res, double *energies)
{
    (void)h;
    const int ps = p->patch_size;
    const int s = p->window_samples;
    double D = u_init;
    double last_step = 0.0;
    int flags = 0, steps = 0;

    for (int it = 0; it < p->iterations; ++it) {
        /* means over the valid pixels at the current D */
        double n = 0.0, sT = 0.0, sR = 0.0, sG = 0.0;
        for (int r = 0; r < ps; ++r)
            for (int c = 0; c < ps; ++c) {
                int x = x0 + c, y = y0 + r, ok;
                double Rs = sample_row(R, w, y, x - D, &ok);
                if (!ok) continue;
                n += 1.0;
                sT += L[(size_t)y * w + x];
                sR += Rs;
                sG += G[(size_t)y * w + x];
            }
        if (n == 0.0) {
            flags |= ORC_FLAG_FLAT;
            break;
        }
        double mT = 0.0, mR = 0.0, mG = 0.0;
        if (p->normalize) {
            mT = sT / n;
            mR = sR / n;
            mG = sG / n;
        }
        double H = 0.0, num = 0.0;
        for (int r = 0; r < ps; ++r)
            for (int c = 0; c < ps; ++c) {
                int x = x0 + c, y = y0 + r, ok;
                double Rs = sample_row(R, w, y, x - D, &ok);
                if (!ok) continue;
                double gn = G[(size_t)y * w + x] - mG;
                double res_px = (Rs - mR) - (L[(size_t)y * w + x] - mT);
                H += gn * gn;
                num += gn * res_px;
            }
        if (H <= ORC_FLAT_EPS * n) {
            flags |= ORC_FLAG_FLAT;
            break;
        }
        last_step = num / H;
        D += last_step;
        ++steps;
        if (!isfinite(D)) break;
        if (fabs(D - u_init) > (double)ps) break; /* R8: left the search range */
        if (fabs(last_step) < ORC_STEP_TOL) break; /* R12: converged */
    }

    /* R8: divergence and convergence */
    if (!isfinite(D) || fabs(D - u_init) > (double)ps) flags |= ORC_FLAG_DIVERGED;
    if (fabs(last_step) > ORC_CONVERGE_TOL) flags |= ORC_FLAG_UNCONVERGED;

    /* R9: pixels valid at D* (their right sample is inside the image) */
    int n_valid = 0;
    if (isfinite(D))
        for (int r = 0; r < ps; ++r)
            for (int c = 0; c < ps; ++c) {
                int ok;
                sample_row(R, w, y0 + r, x0 + c - D, &ok);
                n_valid += ok;
            }

    /* R6: Bayesian window P' = {D* + (i - (s-1)/2) * step}, energies over the
     * pixels valid at every sample so that they compare (Sec. 2.2). R8: a
     * patch that left its search range is dropped as diverged; its window is
     * not evaluated (posterior 0, no window flags). */
    const int diverged = (flags & ORC_FLAG_DIVERGED) != 0;
    double E[64];
    unsigned char common[32 * 32];
    int n_common = 0;
    for (int q = 0; q < ps * ps; ++q) common[q] = 0;
    if (!diverged) {
        for (int r = 0; r < ps; ++r)
            for (int c = 0; c < ps; ++c) {
                int all = 1;
                for (int i = 0; i < s; ++i) {
                    int ok;
                    double di = D + (i - (s - 1) / 2) * p->window_step;
                    sample_row(R, w, y0 + r, x0 + c - di, &ok);
                    all &= ok;
                }
                common[r * ps + c] = (unsigned char)all;
                n_common += all;
            }
    }
    for (int i = 0; i < 64; ++i) E[i] = 0.0;
    if (n_common == 0) {
        if (!diverged) flags |= ORC_FLAG_EMPTY;
    } else {
        for (int i = 0; i < s; ++i) {
            double di = D + (i - (s - 1) / 2) * p->window_step;
            double dres[32 * 32];
            double md = 0.0;
            for (int r = 0; r < ps; ++r)
                for (int c = 0; c < ps; ++c) {
                    if (!common[r * ps + c]) continue;
                    int ok;
                    double Rs = sample_row(R, w, y0 + r, x0 + c - di, &ok);
                    dres[r * ps + c] = Rs - L[(size_t)(y0 + r) * w + x0 + c];
                    md += dres[r * ps + c];
                }
            /* patch normalisation: subtract the residual mean (R5) */
            md = p->normalize ? md / n_common : 0.0;
            double e = 0.0;
            for (int q = 0; q < ps * ps; ++q)
                if (common[q]) e += (dres[q] - md) * (dres[q] - md);
            E[i] = e;
        }
    }

    /* Eq. 3 with Eq. 4 as likelihood: P = exp(-E_c / k) / sum_i exp(-E_i / k),
     * k = 2 sigma_r^2 s^2 (R6), evaluated relative to min E for range. */
    double post = 0.0;
    if (n_common > 0) {
        const int ic = (s - 1) / 2;
        const double kappa = 2.0 * p->sigma_r * p->sigma_r * (double)s * (double)s;
        double emin = E[0];
        for (int i = 1; i < s; ++i)
            if (E[i] < emin) emin = E[i];
        double z = 0.0;
        for (int i = 0; i < s; ++i) z += exp(-(E[i] - emin) / kappa);
        post = exp(-(E[ic] - emin) / kappa) / z;

        /* R7: saddle / convergence filter (Sec. 2.2): discard unless D* is the
         * minimum of its window, with a small relative tolerance; ties keep. */
        double eo = INFINITY;
        for (int i = 0; i < s; ++i)
            if (i != ic && E[i] < eo) eo = E[i];
        double tol = ORC_SADDLE_TAU * (E[ic] > 1.0 ? E[ic] : 1.0);
        if (s > 1 && eo < E[ic] - tol) flags |= ORC_FLAG_SADDLE;
    }

    /* R9: gamma test on the pixels valid at D* (Sec. 3) */
    if ((double)n_valid < p->gamma * (double)(ps * ps)) flags |= ORC_FLAG_GAMMA;

    int discard = flags & (ORC_FLAG_DIVERGED | ORC_FLAG_SADDLE | ORC_FLAG_GAMMA | ORC_FLAG_EMPTY |
                           ORC_FLAG_UNCONVERGED);
    res->u_init = u_init;
    res->d_star = D;
    res->posterior = post;
    /* Sec. 3.2: patches with invalid pixels get a lower probability (R9) */
    res->weight = discard ? 0.0 : post * (double)n_valid / (double)(ps * ps);
    if (p->fusion == ORC_FUSION_DIS) {
        /* R14: DIS fuses every patch (Eq. 2, all covering patches); a patch
         * that left its search range falls back to where it started. */
        if (flags & ORC_FLAG_DIVERGED) res->d_star = u_init;
        res->weight = 1.0;
    }
    res->flags = flags;
    res->n_valid = n_valid;
    res->steps = steps;
    if (energies)
        for (int i = 0; i < s; ++i) energies[i] = E[i];
}

/* Initial disparity of a patch (Sec. 2.1: a finer scale starts from the
 * optimised coarser one). R4: twice the coarse map, read bilinearly at half
 * the patch centre; zero at the coarsest searched level (coarse == NULL). */
double orc_patch_init(const double *coarse, int cw, int ch, int x0, int y0, int ps)
{
    if (!coarse) return 0.0;
    double cx = x0 + (ps - 1) / 2.0, cy = y0 + (ps - 1) / 2.0;
    return 2.0 * bilinear_clamped(coarse, cw, ch, cx / 2.0, cy / 2.0);
}

/* Search every patch of one level. Outputs are per patch, row-major over the
 * patch grid (ny x nx); any may be NULL. energies holds s values per patch;
 * steps the number of updates applied to each patch's D. */
void orc_search_level(const double *L, const double *R, const double *G, int w, int h,
                      const double *coarse, int cw, int ch, const orc_params *p,
                      double *u_init, double *d_star, double *posterior, double *weight,
                      int *flags, int *n_valid, double *energies, int *steps)
{
    const int ps = p->patch_size;
    const int stride = orc_grid_stride(ps, p->overlap);
    const int nx = orc_grid_count(w, ps, stride), ny = orc_grid_count(h, ps, stride);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            int x0 = orc_grid_origin(i, nx, w, ps, stride);
            int y0 = orc_grid_origin(j, ny, h, ps, stride);
            orc_patch_result res;
            double u0 = orc_patch_init(coarse, cw, ch, x0, y0, ps);
            orc_search_patch(L, R, G, w, h, x0, y0, u0, p, &res,
                             energies ? energies + (size_t)k * p->window_samples : NULL);
            if (u_init) u_init[k] = res.u_init;
            if (d_star) d_star[k] = res.d_star;
            if (posterior) posterior[k] = res.posterior;
            if (weight) weight[k] = res.weight;
            if (flags) flags[k] = res.flags;
            if (n_valid) n_valid[k] = res.n_valid;
            if (steps) steps[k] = res.steps;
        }
}

/* --------------------------------------------------------- densification */

/* Dense disparity of one level (Sec. 2.3): every kept patch k spreads D*_k
 * over its pixels with weight w_k * exp(-|x - c_k|^2 / (2 sigma_s^2)) (Eq. 5
 * times the patch posterior); each pixel takes the normalised weighted mean
 * over its covering patches (the normalised form of Eq. 2).
 * R10: a pixel with no kept covering patch is NaN at the finest searched
 * level (Sec. 3.2: not estimated); at coarser levels it carries the value
 * the patches of this level started from (0 at the coarsest searched level,
 * else twice the coarser map), so finer patches still get an initial value. */
void orc_densify_level(int w, int h, const orc_params *p, const double *d_star,
                       const double *weight, const double *coarse, int cw, int ch,
                       int is_finest, const double *L, const double *R, double *out)
{
    const int ps = p->patch_size;
    const int stride = orc_grid_stride(ps, p->overlap);
    const int nx = orc_grid_count(w, ps, stride), ny = orc_grid_count(h, ps, stride);
    const double two_s2 = 2.0 * p->sigma_s * p->sigma_s;
    double *num = (double *)calloc((size_t)w * h, sizeof(double));
    double *den = (double *)calloc((size_t)w * h, sizeof(double));
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            if (!(weight[k] > 0.0)) continue;
            int x0 = orc_grid_origin(i, nx, w, ps, stride);
            int y0 = orc_grid_origin(j, ny, h, ps, stride);
            double cx = x0 + (ps - 1) / 2.0, cy = y0 + (ps - 1) / 2.0;
            for (int r = 0; r < ps; ++r)
                for (int c = 0; c < ps; ++c) {
                    int x = x0 + c, y = y0 + r;
                    double wk;
                    if (p->fusion == ORC_FUSION_DIS) {
                        /* Eq. 2: inverse squared photometric residual of the
                         * patch's disparity at this pixel, floored at 1 (R14) */
                        int ok;
                        double Rs = sample_row(R, w, y, x - d_star[k], &ok);
                        if (!ok) continue;
                        double res_px = Rs - L[(size_t)y * w + x];
                        double r2 = res_px * res_px;
                        wk = weight[k] / (r2 > 1.0 ? r2 : 1.0);
                    } else {
                        double d2 = (x - cx) * (x - cx) + (y - cy) * (y - cy);
                        wk = weight[k] * exp(-d2 / two_s2);
                    }
                    num[(size_t)y * w + x] += wk * d_star[k];
                    den[(size_t)y * w + x] += wk;
                }
        }
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            size_t q = (size_t)y * w + x;
            if (den[q] > 0.0)
                out[q] = num[q] / den[q];
            else if (is_finest)
                out[q] = NAN;
            else if (!coarse)
                out[q] = 0.0;
            else
                out[q] = 2.0 * bilinear_clamped(coarse, cw, ch, x / 2.0, y / 2.0);
        }
    free(num);
    free(den);
}

/* R11: a map searched at level f > 0 is brought to full resolution by
 * bilinear reads at x / 2^f scaled by 2^f, over the finite neighbours with
 * positive weight; NaN where there is none. */
void orc_upsample(const double *M, int mw, int mh, int f, int w, int h, double *out)
{
    const double sc = ldexp(1.0, f);
    for (int y = 0; y < h; ++y)
        for (int x = 0; x < w; ++x) {
            double fx = x / sc, fy = y / sc;
            if (fx > mw - 1) fx = mw - 1;
            if (fy > mh - 1) fy = mh - 1;
            int x0 = (int)floor(fx), y0 = (int)floor(fy);
            int x1 = x0 + 1 < mw ? x0 + 1 : mw - 1;
            int y1 = y0 + 1 < mh ? y0 + 1 : mh - 1;
            double tx = fx - x0, ty = fy - y0;
            double wt[4] = {(1 - tx) * (1 - ty), tx * (1 - ty), (1 - tx) * ty, tx * ty};
            double v[4] = {M[(size_t)y0 * mw + x0], M[(size_t)y0 * mw + x1],
                           M[(size_t)y1 * mw + x0], M[(size_t)y1 * mw + x1]};
            double a = 0.0, b = 0.0;
            for (int q = 0; q < 4; ++q)
                if (wt[q] > 0.0 && isfinite(v[q])) {
                    a += wt[q] * v[q];
                    b += wt[q];
                }
            out[(size_t)y * w + x] = b > 0.0 ? sc * a / b : NAN;
        }
}

/* ------------------------------------------------------------ the method */

/* R16, the per-patch choice on the level searched twice: result a (searched
 * from the seed) is kept only if a is kept, it is not within
 * ORC_SAME_SOLUTION px of a kept result b (searched from the plain start;
 * that close, both found one solution and the plain one stands), and b is
 * dropped or has no higher posterior. Otherwise b's D* and weight overwrite
 * a's. use_a (may be NULL) receives 1 where a was kept, else 0. */
void orc_select_start(int np, double *d_a, double *w_a, const double *post_a,
                      const int *fl_a, const double *d_b, const double *w_b,
                      const double *post_b, const int *fl_b, int *use_a)
{
    const int drop = ORC_FLAG_DIVERGED | ORC_FLAG_SADDLE | ORC_FLAG_GAMMA | ORC_FLAG_EMPTY |
                     ORC_FLAG_UNCONVERGED;
    for (int k = 0; k < np; ++k) {
        int same = !(fl_a[k] & drop) && !(fl_b[k] & drop) &&
                   fabs(d_a[k] - d_b[k]) <= ORC_SAME_SOLUTION;
        int use_seed = !same && !(fl_a[k] & drop) && ((fl_b[k] & drop) || post_a[k] >= post_b[k]);
        if (!use_seed) {
            d_a[k] = d_b[k];
            w_a[k] = w_b[k];
        }
        if (use_a) use_a[k] = use_seed;
    }
}

int orc_match_warm(const double *left, const double *right, int w, int h, const orc_params *p,
                   const double *prev, double *out);
int orc_match_seeded(const double *left, const double *right, int w, int h,
                     const orc_params *p, const double *seed, int seed_level, int fallback,
                     double *out);
void orc_warm_map(const double *P, int w, int h, int level, double *out);

/* Full BDIS on one pair (Sec. 2, Fig. 1). left/right: w x h gray levels in
 * [0, 255] as doubles (row-major). out: w x h, NaN where not estimated.
 * Returns 0 on success, a negative value on bad arguments or no memory. */
int orc_match(const double *left, const double *right, int w, int h, const orc_params *p,
              double *out)
{
    return orc_match_warm(left, right, w, h, p, NULL, out);
}

int orc_match_warm(const double *left, const double *right, int w, int h, const orc_params *p,
                   const double *prev, double *out)
{
    return orc_match_seeded(left, right, w, h, p, prev, 0, 0, out);
}

int orc_match_seeded(const double *left, const double *right, int w, int h,
                     const orc_params *p, const double *seed, int seed_level, int fallback,
                     double *out)
{
    const int ps = p->patch_size;
    const int top = p->coarsest_scale, fin = p->finest_scale;
    if (ps < 2 || ps > 32 || top < fin || fin < 0 || top > 15 || p->iterations < 0 ||
        p->window_samples < 1 || p->window_samples > 63 || p->window_samples % 2 == 0 ||
        !(p->overlap >= 0.0 && p->overlap < 1.0) ||
        (p->fusion != ORC_FUSION_BDIS && p->fusion != ORC_FUSION_DIS))
        return -1;
    if (orc_level_dim(w, top) < ps || orc_level_dim(h, top) < ps) return -1;
    if (seed && (seed_level < 0 || seed_level > top)) return -1;

    int nl = top + 1;
    double **Lp = (double **)calloc(nl, sizeof(double *));
    double **Rp = (double **)calloc(nl, sizeof(double *));
    int *lw = (int *)calloc(nl, sizeof(int)), *lh = (int *)calloc(nl, sizeof(int));
    for (int l = 0; l < nl; ++l) {
        lw[l] = orc_level_dim(w, l);
        lh[l] = orc_level_dim(h, l);
        Lp[l] = (double *)malloc(sizeof(double) * lw[l] * lh[l]);
        Rp[l] = (double *)malloc(sizeof(double) * lw[l] * lh[l]);
    }
    memcpy(Lp[0], left, sizeof(double) * w * h);
    memcpy(Rp[0], right, sizeof(double) * w * h);
    for (int l = 0; l < top; ++l) {
        orc_downsample(Lp[l], lw[l], lh[l], Lp[l + 1]);
        orc_downsample(Rp[l], lw[l], lh[l], Rp[l + 1]);
    }

    double *coarse = NULL;
    int cw = 0, ch = 0;
    if (seed) {
        cw = orc_level_dim(w, top + 1);
        ch = orc_level_dim(h, top + 1);
        coarse = (double *)malloc(sizeof(double) * cw * ch);
        orc_warm_map(seed, orc_level_dim(w, seed_level), orc_level_dim(h, seed_level),
                     top + 1 - seed_level, coarse);
    }
    for (int l = top; l >= fin; --l) {
        int W = lw[l], H = lh[l];
        int stride = orc_grid_stride(ps, p->overlap);
        int np = orc_grid_count(W, ps, stride) * orc_grid_count(H, ps, stride);
        double *G = (double *)malloc(sizeof(double) * W * H);
        double *dst = (double *)malloc(sizeof(double) * np);
        double *wgt = (double *)malloc(sizeof(double) * np);
        double *dense = (double *)malloc(sizeof(double) * W * H);
        orc_sobel_x(Lp[l], W, H, G);
        const double *carry = coarse;
        if (seed && fallback && l == top) {
            /* R16: seeded and plain searches of the coarsest level, per-patch choice */
            double *post_a = (double *)malloc(sizeof(double) * np);
            double *dst_b = (double *)malloc(sizeof(double) * np);
            double *wgt_b = (double *)malloc(sizeof(double) * np);
            double *post_b = (double *)malloc(sizeof(double) * np);
            int *fl_a = (int *)malloc(sizeof(int) * np), *fl_b = (int *)malloc(sizeof(int) * np);
            orc_search_level(Lp[l], Rp[l], G, W, H, coarse, cw, ch, p, NULL, dst, post_a, wgt,
                             fl_a, NULL, NULL, NULL);
            orc_search_level(Lp[l], Rp[l], G, W, H, NULL, 0, 0, p, NULL, dst_b, post_b, wgt_b,
                             fl_b, NULL, NULL, NULL);
            orc_select_start(np, dst, wgt, post_a, fl_a, dst_b, wgt_b, post_b, fl_b, NULL);
            free(post_a);
            free(dst_b);
            free(wgt_b);
            free(post_b);
            free(fl_a);
            free(fl_b);
            carry = NULL; /* carried pixels keep the plain start */
        } else {
            orc_search_level(Lp[l], Rp[l], G, W, H, coarse, cw, ch, p, NULL, dst, NULL, wgt,
                             NULL, NULL, NULL, NULL);
        }
        orc_densify_level(W, H, p, dst, wgt, carry, carry ? cw : 0, carry ? ch : 0, l == fin,
                          Lp[l], Rp[l], dense);
        free(G);
        free(dst);
        free(wgt);
        free(coarse);
        coarse = dense;
        cw = W;
        ch = H;
    }
    if (fin == 0)
        memcpy(out, coarse, sizeof(double) * w * h);
    else
        orc_upsample(coarse, cw, ch, fin, w, h, out);
    free(coarse);
    for (int l = 0; l < nl; ++l) {
        free(Lp[l]);
        free(Rp[l]);
    }
    free(Lp);
    free(Rp);
    free(lw);
    free(lh);
    return 0;
}

/* R15 warm start: the map that seeds the coarsest searched level L from a
 * previous disparity P of the same scene (full size, NaN = not estimated).
 * With s = 2^(L+1), output pixel (X, Y) of level L+1 is the mean of the
 * finite values of P over the s x s block centred on full-size pixel
 * (sX, sY) (rows and columns sX - s/2 .. sX + s/2 - 1, clipped to the
 * image), divided by s; 0 where the block has no finite value. */
void orc_warm_map(const double *P, int w, int h, int level, double *out)
{
    const int s = 1 << level;
    const int mw = orc_level_dim(w, level), mh = orc_level_dim(h, level);
    for (int Y = 0; Y < mh; ++Y)
        for (int X = 0; X < mw; ++X) {
            double sum = 0.0;
            int n = 0;
            for (int y = Y * s - s / 2; y < Y * s + s / 2 + (s == 1); ++y)
                for (int x = X * s - s / 2; x < X * s + s / 2 + (s == 1); ++x) {
                    if (x < 0 || y < 0 || x >= w || y >= h) continue;
                    double v = P[(size_t)y * w + x];
                    if (!isfinite(v)) continue;
                    sum += v;
                    n++;
                }
            out[(size_t)Y * mw + X] = n ? sum / n / s : 0.0;
        }
}

/* The method with a warm start (R15): identical to orc_match except that the
 * coarsest searched level starts from orc_warm_map(prev) instead of 0 (its
 * patches' initial values and its carried pixels). prev NULL = orc_match. */
int orc_match_warm(const double *left, const double *right, int w, int h, const orc_params *p,
                   const double *prev, double *out);

/* R16 proposal start: `seed` is a disparity map at pyramid level seed_level
 * (values in that level's pixels, NaN allowed). Its block means seed the
 * coarsest searched level as in R15 (blocks of 2^(coarsest + 1 - seed_level)
 * pixels of the seed level). With fallback = 0 this is the warm start. With
 * fallback = 1 the coarsest level is searched twice, from the seed and from
 * the plain start (0); a patch keeps the seeded result only if it is kept,
 * differs from a kept plain result by more than ORC_SAME_SOLUTION pixels
 * (closer, the two searches found the same solution and the plain one
 * stands), and either the plain result is dropped or the seeded posterior is
 * at least the plain one; pixels of that level that no kept patch covers carry the plain
 * start, so a proposal that every patch rejects gives the plain method. */
int orc_match_seeded(const double *left, const double *right, int w, int h,
                     const orc_params *p, const double *seed, int seed_level, int fallback,
                     double *out);

/* uint8 entry: converts to gray levels as doubles (step 1 of the oracle). */
int orc_match_u8(const uint8_t *left, const uint8_t *right, int w, int h, const orc_params *p,
                 double *out)
{
    size_t n = (size_t)w * h;
    double *l = (double *)malloc(sizeof(double) * n), *r = (double *)malloc(sizeof(double) * n);
    for (size_t i = 0; i < n; ++i) {
        l[i] = left[i];
        r[i] = right[i];
    }
    int rc = orc_match(l, r, w, h, p, out);
    free(l);
    free(r);
    return rc;
}
