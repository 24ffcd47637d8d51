/*
 * ebof_oracle.c -- plain, slow FP64 CPU oracle of the event-to-flow path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file or the library built from it; only the tests, the smoke
 * check and the benchmark's CPU-baseline leg do.  It shares no code, header
 * or table with the CUDA library.
 *
 * Every function states the passage of the paper (Brebion, Moreau, Davoine,
 * "Real-Time Optical Flow for Vehicular Perception with Low- and
 * High-Resolution Event Cameras") that it follows.  Where the paper is
 * silent the reading taken is stated beside the code.  The frame-based flow
 * block (§III-D) leaves the choice of method open: the surfaces are meant to
 * be fed to an established frame-based flow method.  The one written here is
 * Dense Inverse Search
 * (Kroeger et al., ECCV 2016): image pyramid, per-patch inverse-compositional
 * Gauss-Newton, patch densification and variational refinement, with every
 * free constant fixed by the readings below.
 *
 * Arithmetic is double precision throughout; loops are the plain
 * definitions, in the paper's order, with no blocking or fusion.
 *
 * Parity pins (tests that tie this file to something other than itself) are
 * listed with each function.  The mutation switch `orc_mutation` plants one
 * deliberate mistake at a time so the tests can show that each pin catches
 * the mistake it guards against; it is 0 (no mistake) unless a test sets it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF_D 2147483647 /* squared distance of an image without edges */

int orc_mutation = 0; /* test-only planted mistake; 0 = none */

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* ---------------------------------------------------------------------------
 * §III-A: accumulation of one time window into a binary edge image.
 * A pixel is an edge pixel iff at least one event with t in the window
 * [t_begin, t_end) fell on it; polarity is ignored (§III-A).
 * Reading: the window is half open; events outside the image are dropped.
 * stats[0] = events given, [1] = events in the window, [2] = events outside
 * the window, [3] = in-window events outside the image.
 * ------------------------------------------------------------------------- */
void orc_edge_image(int W, int H, int64_t n, const uint16_t *x, const uint16_t *y,
                    const int64_t *t, int64_t t_begin, int64_t t_end, uint8_t *E,
                    int64_t *stats)
{
    int64_t in_win = 0, out_time = 0, out_img = 0;
    memset(E, 0, (size_t)W * (size_t)H);
    for (int64_t i = 0; i < n; ++i) {
        if (t[i] < t_begin || t[i] >= t_end) { ++out_time; continue; }
        ++in_win;
        if ((int)x[i] >= W || (int)y[i] >= H) { ++out_img; continue; }
        E[(size_t)y[i] * W + x[i]] = 1;
    }
    stats[0] = n; stats[1] = in_win; stats[2] = out_time; stats[3] = out_img;
}

/* Number of edge pixels among the direct neighbours of (px, py) in img.
 * conn = 4: the 4 direct neighbours named by Alg. 1 and Alg. 2;
 * conn = 8: the full 3x3 ring (used by the 3x3 isolated-pixel denoise).
 * Neighbours outside the image count as non-edge. */
static int edge_neighbours(const uint8_t *img, int W, int H, int px, int py, int conn)
{
    int c = 0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            if (conn == 4 && dx != 0 && dy != 0) continue;
            int qx = px + dx, qy = py + dy;
            if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
            c += img[(size_t)qy * W + qx] ? 1 : 0;
        }
    return c;
}

/* Alg. 1 (denoising, §III-B): an edge pixel of E whose count of edge
 * neighbours in E is below N_d stops being an edge pixel.  N_d = 0 disables
 * it.  Pins: hand cases (lone pixel, segment, order example), identity at
 * N_d = 0. */
void orc_denoise(int W, int H, const uint8_t *E, int conn, int n_d, uint8_t *Ed)
{
    memcpy(Ed, E, (size_t)W * H);
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            size_t p = (size_t)py * W + px;
            if (!E[p]) continue;
            int cnt = edge_neighbours(E, W, H, px, py, conn);
            int remove = (orc_mutation == 1) ? (cnt <= n_d) : (cnt < n_d);
            if (remove) Ed[p] = 0;
        }
}

/* Alg. 2 (filling, §III-B): a non-edge pixel of the DENOISED image whose
 * count of edge neighbours in that image reaches N_f becomes an edge pixel.
 * The count reads E_d, never E (the order argument of §III-B).  N_f above
 * the neighbourhood size (5 for 4-neighbours) disables it. */
void orc_fill(int W, int H, const uint8_t *Ed, int conn, int n_f, uint8_t *Edf)
{
    memcpy(Edf, Ed, (size_t)W * H);
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            size_t p = (size_t)py * W + px;
            if (Ed[p]) continue;
            if (edge_neighbours(Ed, W, H, px, py, conn) >= n_f) Edf[p] = 1;
        }
}

/* ---------------------------------------------------------------------------
 * §III-C: Euclidean distance transform.  d_Euc is a pixel's Euclidean
 * distance to its nearest edge pixel; the squared value is an integer and is
 * unique even when several edge pixels are equally close.
 * ------------------------------------------------------------------------- */

/* The definition itself: minimum over all edge pixels.  O(P * sites). */
void orc_edt_brute(int W, int H, const uint8_t *E, int32_t *D)
{
    int64_t nsites = 0;
    for (size_t p = 0; p < (size_t)W * H; ++p) nsites += E[p] ? 1 : 0;
    int *sx = (int *)malloc(sizeof(int) * (size_t)(nsites + 1));
    int *sy = (int *)malloc(sizeof(int) * (size_t)(nsites + 1));
    int64_t k = 0;
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px)
            if (E[(size_t)py * W + px]) { sx[k] = px; sy[k] = py; ++k; }
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int64_t best = ORC_INF_D;
            for (int64_t i = 0; i < nsites; ++i) {
                int64_t dx = px - sx[i], dy = py - sy[i];
                int64_t d = dx * dx + dy * dy;
                if (d < best) best = d;
            }
            D[(size_t)py * W + px] = (int32_t)best;
        }
    free(sx); free(sy);
}

/* The separable form the paper builds on (§III-C cites the separable exact
 * EDT of Coeurjolly et al.): first, per column, the distance g to the
 * nearest edge pixel of that column; then, per pixel,
 *     D(x, y) = min over columns x' of (x - x')^2 + g(x', y)^2,
 * evaluated here by scanning every column x' (no lower-envelope shortcut).
 * Columns without any edge pixel take no part.  An image without edge
 * pixels gives D = INT32_MAX everywhere (reading).  Pins: orc_edt_brute on
 * small images, scipy's exact EDT, the single-site closed form. */
void orc_edt_separable(int W, int H, const uint8_t *E, int32_t *D)
{
    int64_t *g = (int64_t *)malloc(sizeof(int64_t) * (size_t)W * H);
    const int64_t NONE = -1;
    for (int px = 0; px < W; ++px) {
        int64_t last = NONE; /* nearest edge row at or above */
        for (int py = 0; py < H; ++py) {
            if (E[(size_t)py * W + px]) last = py;
            g[(size_t)py * W + px] = (last == NONE) ? NONE : (py - last);
        }
        last = NONE; /* nearest edge row at or below */
        for (int py = H - 1; py >= 0; --py) {
            if (E[(size_t)py * W + px]) last = py;
            if (last != NONE) {
                int64_t d = last - py;
                int64_t *gp = &g[(size_t)py * W + px];
                if (*gp == NONE || d < *gp) *gp = d;
            }
        }
    }
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int64_t best = ORC_INF_D;
            for (int qx = 0; qx < W; ++qx) {
                int64_t gq = g[(size_t)py * W + qx];
                if (gq == NONE) continue;
                int64_t dx = px - qx;
                int64_t d = (orc_mutation == 2) ? (dx < 0 ? -dx : dx) + gq * gq
                                                : dx * dx + gq * gq;
                if (d < best) best = d;
            }
            D[(size_t)py * W + px] = (int32_t)best;
        }
    free(g);
}

/* Eq. 1: d_exp = 1 - exp(-d_Euc / alpha), d_Euc = sqrt(D).  An image without
 * edge pixels (D = INT32_MAX) gives the saturated value 1 (reading).
 * Pins: d_exp(0) = 0; Eq. 2 with eps = 1/255 gives d_exp(d_sat) = 254/255;
 * monotone in D. */
void orc_surface(int n, const int32_t *D, double alpha, double *S)
{
    for (int i = 0; i < n; ++i) {
        if (D[i] == ORC_INF_D) { S[i] = 1.0; continue; }
        double d = sqrt((double)D[i]);
        S[i] = (orc_mutation == 3) ? 1.0 - exp(-d * alpha) : 1.0 - exp(-d / alpha);
    }
}

/* The distance surfaces compared in the ablations of §IV-D (plotted beside
 * Eq. 1 in §III-C), as functions y(d) of the Euclidean distance d = sqrt(D):
 *   mode 0  d_exp = 1 - exp(-d / alpha)             (Eq. 1, the proposal)
 *   mode 1  DS_L   y = d                            (the plain distance)
 *   mode 2  DS_LB  y = min(d, d_sat)                (bounded at d_sat)
 *   mode 3  DS_Log y = ln(d + 1)
 * Reading S1: an image without edge pixels (D = INT32_MAX) gives
 * d_exp = 1 and, for the variants, y at the finite distance
 * d = sqrt(INT32_MAX), so every surface is a constant image there. */
void orc_surface_mode(int n, const int32_t *D, int mode, double alpha, double d_sat, double *Y)
{
    for (int i = 0; i < n; ++i) {
        const double d = sqrt((double)D[i]);
        if (mode == 0) {
            orc_surface(1, &D[i], alpha, &Y[i]);
        } else if (mode == 1) {
            Y[i] = d;
        } else if (mode == 2) {
            Y[i] = (orc_mutation == 10) ? fmax(d, d_sat) : fmin(d, d_sat);
        } else {
            Y[i] = log(d + 1.0);
        }
    }
}

/* Eq. 2: alpha = -d_sat / ln(eps).  Eq. 3 is its value at eps = 1/255. */
double orc_alpha_from_dsat(double d_sat, double eps) { return -d_sat / log(eps); }

/* ---------------------------------------------------------------------------
 * Frame-based flow block (§III-D), Dense Inverse Search.
 *
 * Readings (the paper and its flow method leave these open):
 *  F0  the flow runs on I = 255 * d_exp, the 8-bit coding of §III-C, so the
 *      densification weights below see intensities on a 0..255 scale;
 *  F1  pyramid level l+1 is the 2x2 box mean of level l, size floor(W/2) x
 *      floor(H/2); the number of levels is capped so that the smallest level
 *      still holds one patch; an image smaller than a patch gives zero flow;
 *  F2  patch origins per axis: min(k * stride, W_l - ps), k = 0..n-1 with
 *      n = ceil((W_l - ps) / stride) + 1, so the last patch is flush with
 *      the border; the patch centre is origin + (ps - 1) / 2;
 *  F3  flow maps the previous window (template I0) to the current one
 *      (query I1) in pixels per window; at the coarsest level every patch
 *      starts at 0, at finer levels at 2 * U_{l+1} sampled at the nearest
 *      coarse pixel (round half down of centre / 2, clamped to the image);
 *  F4  inverse-compositional Gauss-Newton on mean-normalised patches with a
 *      fixed iteration count, determinant guard 1e-6 * (ps^2)^2, a damped
 *      step (H + kappa * trace(H) * Id)^-1 b, and a reset to the start value
 *      when the patch drifts more than ps pixels;
 *  F5  densification weights 1 / max(1, |I1(x + u_i) - I0(x)|) over every
 *      patch whose square contains x;
 *  F6  variational refinement: normalised data and gradient-constancy
 *      terms and a smoothness term, robust weights Psi'(s^2) =
 *      1 / (2 sqrt(s^2 + eps^2)), eps = 1e-3, frozen at dU = 0 for each
 *      outer iteration; red-black SOR.
 * Derivatives everywhere are central differences with the index clamped to
 * the image (replicated border); samples off the pixel grid are bilinear
 * with the position clamped to the image.
 * ------------------------------------------------------------------------- */

/* Central difference along x / y with clamped indices. */
static double cdx(const double *F, int W, int x, int y)
{
    int xp = x + 1 < W ? x + 1 : W - 1, xm = x > 0 ? x - 1 : 0;
    return 0.5 * (F[(size_t)y * W + xp] - F[(size_t)y * W + xm]);
}
static double cdy(const double *F, int W, int H, int x, int y)
{
    int yp = y + 1 < H ? y + 1 : H - 1, ym = y > 0 ? y - 1 : 0;
    return 0.5 * (F[(size_t)yp * W + x] - F[(size_t)ym * W + x]);
}

/* Bilinear sample with the position clamped to [0, W-1] x [0, H-1]. */
static double bilinear(const double *I, int W, int H, double x, double y)
{
    if (x < 0) x = 0;
    if (x > W - 1) x = W - 1;
    if (y < 0) y = 0;
    if (y > H - 1) y = H - 1;
    int x0 = (int)floor(x), y0 = (int)floor(y);
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    double fx = x - x0, fy = y - y0;
    double a = I[(size_t)y0 * W + x0], b = I[(size_t)y0 * W + x1];
    double c = I[(size_t)y1 * W + x0], d = I[(size_t)y1 * W + x1];
    return (1 - fy) * ((1 - fx) * a + fx * b) + fy * ((1 - fx) * c + fx * d);
}

/* F1: one pyramid step, 2x2 box mean; output is (W/2) x (H/2), floored. */
void orc_downsample(int W, int H, const double *I, double *out)
{
    int Wc = W / 2, Hc = H / 2;
    for (int y = 0; y < Hc; ++y)
        for (int x = 0; x < Wc; ++x) {
            int sx = 2 * x;
            if (orc_mutation == 4 && 2 * x + 2 < W) sx = 2 * x + 1;
            double a = I[(size_t)(2 * y) * W + sx], b = I[(size_t)(2 * y) * W + sx + 1];
            double c = I[(size_t)(2 * y + 1) * W + sx], d = I[(size_t)(2 * y + 1) * W + sx + 1];
            out[(size_t)y * Wc + x] = 0.25 * (a + b + c + d);
        }
}

/* Image gradients: central differences, replicated border. */
void orc_gradients(int W, int H, const double *I, double *Ix, double *Iy)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double gx = cdx(I, W, x, y), gy = cdy(I, W, H, x, y);
            if (orc_mutation == 5) gx = -gx;
            Ix[(size_t)y * W + x] = gx;
            Iy[(size_t)y * W + x] = gy;
        }
}

/* F2: patch origins along one axis; returns their count (0 if ps > n). */
int orc_patch_origins(int n, int ps, int stride, int *origins)
{
    if (ps > n) return 0;
    int cnt = (n - ps + stride - 1) / stride + 1;
    for (int k = 0; k < cnt; ++k) {
        int o = k * stride;
        origins[k] = o < n - ps ? o : n - ps;
    }
    return cnt;
}

/* Number of pyramid levels used (F1): at most `levels`, and every used level
 * must hold one patch.  0 when the image itself is smaller than a patch. */
int orc_levels_used(int W, int H, int levels, int ps)
{
    int L = 0;
    while (L < levels && (W >> L) >= ps && (H >> L) >= ps) ++L;
    return L;
}

/* F3 + F4: inverse search of every patch at one level.
 * I0, I0x, I0y: previous-window level image and its gradients (template);
 * I1: current-window level image (query); Uc: dense flow of the next coarser
 * level (Wc x Hc, planar u then v) or NULL at the coarsest level.
 * up: patch flows, planar [2][npy][npx]; flags: 0 = searched, 1 = determinant
 * guard (kept its start value), 2 = reset after drifting more than ps.
 * The Gauss-Newton step solves (H + mu Id) Delta = b with mu = kappa *
 * trace(H): on an edge-like patch (the aperture problem) H is nearly
 * singular and the undamped step wanders along the edge; the damping keeps
 * that component near its start value and leaves well-textured patches
 * (eigenvalues of the same order) converging as before. */
void orc_patch_search(int W, int H, const double *I0, const double *I0x,
                      const double *I0y, const double *I1, const double *Uc,
                      int Wc, int Hc, int ps, int stride, int iters, double kappa,
                      double *up, uint8_t *flags)
{
    int *ox = (int *)malloc(sizeof(int) * (size_t)(W + 1));
    int *oy = (int *)malloc(sizeof(int) * (size_t)(H + 1));
    int npx = orc_patch_origins(W, ps, stride, ox);
    int npy = orc_patch_origins(H, ps, stride, oy);
    int n = ps * ps;
    double *T = (double *)malloc(sizeof(double) * n);
    double *gx = (double *)malloc(sizeof(double) * n);
    double *gy = (double *)malloc(sizeof(double) * n);
    double *w = (double *)malloc(sizeof(double) * n);
    size_t np = (size_t)npx * npy;
    for (int j = 0; j < npy; ++j)
        for (int i = 0; i < npx; ++i) {
            int x0 = ox[i], y0 = oy[j];
            /* F3: start value */
            double u0 = 0.0, v0 = 0.0;
            if (Uc) {
                int cx = clampi((2 * x0 + ps) / 4, 0, Wc - 1);
                int cy = clampi((2 * y0 + ps) / 4, 0, Hc - 1);
                u0 = 2.0 * Uc[(size_t)cy * Wc + cx];
                v0 = 2.0 * Uc[(size_t)Wc * Hc + (size_t)cy * Wc + cx];
            }
            /* F4: template, mean-normalised gradients, Hessian */
            double mT = 0, mgx = 0, mgy = 0;
            for (int q = 0; q < n; ++q) {
                size_t p = (size_t)(y0 + q / ps) * W + (x0 + q % ps);
                T[q] = I0[p]; gx[q] = I0x[p]; gy[q] = I0y[p];
                mT += T[q]; mgx += gx[q]; mgy += gy[q];
            }
            mT /= n; mgx /= n; mgy /= n;
            double h11 = 0, h12 = 0, h22 = 0;
            for (int q = 0; q < n; ++q) {
                gx[q] -= mgx; gy[q] -= mgy;
                h11 += gx[q] * gx[q]; h12 += gx[q] * gy[q]; h22 += gy[q] * gy[q];
            }
            double det = h11 * h22 - h12 * h12;
            size_t id = (size_t)j * npx + i;
            double mu = kappa * (h11 + h22);
            double a11 = h11 + mu, a22 = h22 + mu, adet = a11 * a22 - h12 * h12;
            if (det <= 1e-6 * (double)n * (double)n) {
                up[id] = u0; up[np + id] = v0; flags[id] = 1;
                continue;
            }
            double u = u0, v = v0;
            for (int it = 0; it < iters; ++it) {
                double mw = 0;
                for (int q = 0; q < n; ++q) {
                    w[q] = bilinear(I1, W, H, x0 + q % ps + u, y0 + q / ps + v);
                    mw += w[q];
                }
                mw /= n;
                double b1 = 0, b2 = 0;
                for (int q = 0; q < n; ++q) {
                    double r = (w[q] - mw) - (T[q] - mT);
                    b1 += gx[q] * r; b2 += gy[q] * r;
                }
                double du = (a22 * b1 - h12 * b2) / adet;
                double dv = (a11 * b2 - h12 * b1) / adet;
                if (orc_mutation == 6) { u += du; v += dv; }
                else { u -= du; v -= dv; }
            }
            flags[id] = 0;
            if (hypot(u - u0, v - v0) > ps) { u = u0; v = v0; flags[id] = 2; }
            up[id] = u; up[np + id] = v;
        }
    free(ox); free(oy); free(T); free(gx); free(gy); free(w);
}

/* F5: densification.  U(x) = sum_i lambda_i(x) u_i / sum_i lambda_i(x) over
 * the patches i whose square contains x, lambda_i(x) = 1 / max(1, |I1(x +
 * u_i) - I0(x)|).  U is planar [2][H][W]. */
void orc_densify(int W, int H, const double *I0, const double *I1, int ps,
                 int stride, const double *up, double *U)
{
    int *ox = (int *)malloc(sizeof(int) * (size_t)(W + 1));
    int *oy = (int *)malloc(sizeof(int) * (size_t)(H + 1));
    int npx = orc_patch_origins(W, ps, stride, ox);
    int npy = orc_patch_origins(H, ps, stride, oy);
    size_t np = (size_t)npx * npy, P = (size_t)W * H;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double nu = 0, nv = 0, den = 0;
            for (int j = 0; j < npy; ++j) {
                if (y < oy[j] || y >= oy[j] + ps) continue;
                for (int i = 0; i < npx; ++i) {
                    if (x < ox[i] || x >= ox[i] + ps) continue;
                    size_t id = (size_t)j * npx + i;
                    double u = up[id], v = up[np + id];
                    double r = bilinear(I1, W, H, x + u, y + v) - I0[(size_t)y * W + x];
                    if (orc_mutation == 7) r = I0[(size_t)y * W + x];
                    double lam = 1.0 / fmax(1.0, fabs(r));
                    nu += lam * u; nv += lam * v; den += lam;
                }
            }
            U[(size_t)y * W + x] = den > 0 ? nu / den : 0.0;
            U[P + (size_t)y * W + x] = den > 0 ? nv / den : 0.0;
        }
    free(ox); free(oy);
}

/* Robust penaliser derivative Psi'(s^2) = 1 / (2 sqrt(s^2 + eps^2)), eps = 1e-3. */
static double psi_prime(double s2) { return 1.0 / (2.0 * sqrt(s2 + 1e-6)); }
#define ZETA2 0.01 /* zeta = 0.1 in the constraint normalisation */

/* Planes of the linearised system of one outer iteration of F6, in the
 * order of orc_var_linearise's output Q [ORC_VQ][H][W]. */
enum { VQ_IX, VQ_IY, VQ_IXX, VQ_IXY, VQ_IYY, VQ_IZ, VQ_IXZ, VQ_IYZ, VQ_AD, VQ_AG, VQ_AS,
       ORC_VQ };

/* F6, first half of one outer iteration: warp I1 by U, take the derivatives
 * of the warped image and the constraint residuals, and the robust weights
 * frozen at dU = 0.
 *   I1w = I1(x + U) (bilinear, clamped), Iz = I1w - I0,
 *   Ix, Iy = central differences of I1w; Ixx, Ixy, Iyy = central
 *   differences of Ix (x, y) and Iy (y),
 *   Ixz = Ix - dI0/dx, Iyz = Iy - dI0/dy (I0x, I0y given),
 *   ad = delta nd Psi'(nd Iz^2),        nd = 1 / (Ix^2 + Iy^2 + zeta^2),
 *   ag = gamma ng Psi'(ng (Ixz^2 + Iyz^2)),
 *                        ng = 1 / (Ixx^2 + 2 Ixy^2 + Iyy^2 + zeta^2),
 *   ad = ag = 0 where x + U lies outside the image,
 *   as = alpha_s Psi'(|grad u|^2 + |grad v|^2), forward differences (0 at
 *   the last column / row).
 * The normalisations nd, ng follow Zimmer, Bruhn and Weickert (IJCV 2011):
 * the robust weights then measure a displacement rather than an intensity.
 * Output Q: the ORC_VQ planes in the VQ_* order.
 * Pins: closed-form derivative planes of a quadratic image warped by an
 * integer flow, dropped terms where the warp leaves the image, the weight
 * Psi'(0) of a constant flow. */
void orc_var_linearise(int W, int H, const double *I0, const double *I0x,
                       const double *I0y, const double *I1, const double *U,
                       double delta, double gamma, double alpha_s, double *Q)
{
    size_t P = (size_t)W * H;
    const double *u = U, *v = U + P;
    double *I1w = (double *)malloc(sizeof(double) * P);
    double *Ix = Q + VQ_IX * P, *Iy = Q + VQ_IY * P, *Ixx = Q + VQ_IXX * P,
           *Ixy = Q + VQ_IXY * P, *Iyy = Q + VQ_IYY * P, *Iz = Q + VQ_IZ * P,
           *Ixz = Q + VQ_IXZ * P, *Iyz = Q + VQ_IYZ * P, *ad = Q + VQ_AD * P,
           *ag = Q + VQ_AG * P, *as = Q + VQ_AS * P;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            I1w[p] = bilinear(I1, W, H, x + u[p], y + v[p]);
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            Ix[p] = cdx(I1w, W, x, y); Iy[p] = cdy(I1w, W, H, x, y);
        }
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            Ixx[p] = cdx(Ix, W, x, y);
            Ixy[p] = cdy(Ix, W, H, x, y);
            Iyy[p] = cdy(Iy, W, H, x, y);
            Iz[p] = I1w[p] - I0[p];
            Ixz[p] = Ix[p] - I0x[p];
            Iyz[p] = Iy[p] - I0y[p];
            /* constraint normalisation (reading F6) */
            double nd = 1.0 / (Ix[p] * Ix[p] + Iy[p] * Iy[p] + ZETA2);
            double ng = 1.0 / (Ixx[p] * Ixx[p] + 2.0 * Ixy[p] * Ixy[p] + Iyy[p] * Iyy[p] + ZETA2);
            ad[p] = delta * nd * psi_prime(nd * Iz[p] * Iz[p]);
            ag[p] = gamma * ng * psi_prime(ng * (Ixz[p] * Ixz[p] + Iyz[p] * Iyz[p]));
            double wx = x + u[p], wy = y + v[p];
            if (wx < 0 || wx > W - 1 || wy < 0 || wy > H - 1) { ad[p] = 0; ag[p] = 0; }
            double ux = x + 1 < W ? u[p + 1] - u[p] : 0.0;
            double uy = y + 1 < H ? u[p + W] - u[p] : 0.0;
            double vx = x + 1 < W ? v[p + 1] - v[p] : 0.0;
            double vy = y + 1 < H ? v[p + W] - v[p] : 0.0;
            as[p] = alpha_s * psi_prime(ux * ux + uy * uy + vx * vx + vy * vy);
        }
    free(I1w);
}

/* F6, second half: `sor` red-black SOR sweeps (relaxation omega) on the
 * linear system whose solution dU makes the quadratic energy
 *   sum_x  ad (Ix du + Iy dv + Iz)^2
 *        + ag ((Ixx du + Ixy dv + Ixz)^2 + (Ixy du + Iyy dv + Iyz)^2)
 *   + sum over 4-neighbour pairs (x, n) of w_xn (|(u + du)(n) - (u + du)(x)|^2
 *                                               + |(v + dv)(n) - (v + dv)(x)|^2),
 *   w_xn = (as(x) + as(n)) / 2,
 * stationary (its Euler-Lagrange equations): per pixel
 *   a11 du + a12 dv = r1,  a12 du + a22 dv = r2, with
 *   a11 = ad Ix^2 + ag (Ixx^2 + Ixy^2) + sum_n w_xn,
 *   a12 = ad Ix Iy + ag (Ixx Ixy + Ixy Iyy),
 *   a22 = ad Iy^2 + ag (Ixy^2 + Iyy^2) + sum_n w_xn,
 *   r1  = sum_n w_xn (u(n) + du(n) - u(x)) - ad Ix Iz - ag (Ixx Ixz + Ixy Iyz),
 *   r2  = sum_n w_xn (v(n) + dv(n) - v(x)) - ad Iy Iz - ag (Ixy Ixz + Iyy Iyz);
 * neighbours outside the image are dropped (Neumann border).  A sweep
 * updates the red pixels ((x + y) even) first, then the black ones, each in
 * raster order; inside a pixel du first, then dv with the new du.
 * Q: planes of orc_var_linearise; U: current flow [2][H][W]; dU [2][H][W]:
 * start values in, result out.
 * Pins: one sweep on a 2x2 grid worked by hand (tests/golden), and the
 * converged solution is the minimum of the energy above, differentiated
 * numerically. */
void orc_var_sor(int W, int H, const double *Q, const double *U, int sor, double omega,
                 double *dU)
{
    size_t P = (size_t)W * H;
    const double *u = U, *v = U + P;
    double *du = dU, *dv = dU + P;
    const double *Ix = Q + VQ_IX * P, *Iy = Q + VQ_IY * P, *Ixx = Q + VQ_IXX * P,
                 *Ixy = Q + VQ_IXY * P, *Iyy = Q + VQ_IYY * P, *Iz = Q + VQ_IZ * P,
                 *Ixz = Q + VQ_IXZ * P, *Iyz = Q + VQ_IYZ * P, *ad = Q + VQ_AD * P,
                 *ag = Q + VQ_AG * P, *as = Q + VQ_AS * P;
    for (int s = 0; s < sor; ++s)
        for (int k = 0; k < 2; ++k) {
            int colour = (orc_mutation == 13) ? 1 - k : k;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    if (((x + y) & 1) != colour) continue;
                    size_t p = (size_t)y * W + x;
                    double sw = 0, su = 0, sv = 0;
                    const int nx[4] = {x - 1, x + 1, x, x};
                    const int ny[4] = {y, y, y - 1, y + 1};
                    for (int e = 0; e < 4; ++e) {
                        if (nx[e] < 0 || ny[e] < 0 || nx[e] >= W || ny[e] >= H) continue;
                        size_t q = (size_t)ny[e] * W + nx[e];
                        double wn = 0.5 * (as[p] + as[q]);
                        sw += wn;
                        su += wn * (u[q] + du[q] - u[p]);
                        sv += wn * (v[q] + dv[q] - v[p]);
                    }
                    if (orc_mutation == 9) { su = 0; sv = 0; }
                    double a11 = ad[p] * Ix[p] * Ix[p] + ag[p] * (Ixx[p] * Ixx[p] + Ixy[p] * Ixy[p]) + sw;
                    double a12 = ad[p] * Ix[p] * Iy[p];
                    if (orc_mutation != 12) a12 += ag[p] * (Ixx[p] * Ixy[p] + Ixy[p] * Iyy[p]);
                    double a22 = ad[p] * Iy[p] * Iy[p] + ag[p] * (Ixy[p] * Ixy[p] + Iyy[p] * Iyy[p]) + sw;
                    double sd = (orc_mutation == 8) ? -1.0 : 1.0;
                    double r1 = su - sd * ad[p] * Ix[p] * Iz[p] - ag[p] * (Ixx[p] * Ixz[p] + Ixy[p] * Iyz[p]);
                    double r2 = sv - sd * ad[p] * Iy[p] * Iz[p] - ag[p] * (Ixy[p] * Ixz[p] + Iyy[p] * Iyz[p]);
                    if (a11 > 0) du[p] = (1 - omega) * du[p] + omega * (r1 - a12 * dv[p]) / a11;
                    if (a22 > 0) dv[p] = (1 - omega) * dv[p] + omega * (r2 - a12 * du[p]) / a22;
                }
        }
}

/* F6: variational refinement of the dense flow U (planar [2][H][W], in
 * place): `outer` fixed-point iterations, each one linearising at the
 * current U (orc_var_linearise), solving for dU from dU = 0 with `sor`
 * red-black SOR sweeps (orc_var_sor), then U += dU. */
void orc_variational(int W, int H, const double *I0, const double *I0x,
                     const double *I0y, const double *I1, double *U, int outer,
                     int sor, double delta, double gamma, double alpha_s,
                     double omega)
{
    size_t P = (size_t)W * H;
    double *Q = (double *)malloc(sizeof(double) * P * ORC_VQ);
    double *dU = (double *)malloc(sizeof(double) * P * 2);
    for (int k = 0; k < outer; ++k) {
        orc_var_linearise(W, H, I0, I0x, I0y, I1, U, delta, gamma, alpha_s, Q);
        memset(dU, 0, sizeof(double) * P * 2);
        orc_var_sor(W, H, Q, U, sor, omega, dU);
        for (size_t p = 0; p < 2 * P; ++p) U[p] += dU[p];
    }
    free(Q);
    free(dU);
}

/* Whole flow block: pyramids of both intensity images, then coarse to fine:
 * inverse search, densification, variational refinement.  I0, I1 are the
 * level-0 intensities (255 * d_exp) of the previous and current windows.
 * U_out: planar [2][H][W].  Returns the number of levels used. */
int orc_flow(int W, int H, const double *I0, const double *I1, int levels,
             int ps, int stride, int iters, double kappa, int var_outer, int var_sor,
             double delta, double gamma, double alpha_s, double omega,
             double *U_out)
{
    size_t P = (size_t)W * H;
    int L = orc_levels_used(W, H, levels, ps);
    memset(U_out, 0, sizeof(double) * 2 * P);
    if (L == 0) return 0;
    double *A[16], *B[16], *Ax[16], *Ay[16];
    int Wl[16], Hl[16];
    for (int l = 0; l < L; ++l) {
        Wl[l] = W >> l; Hl[l] = H >> l;
        size_t Pl = (size_t)Wl[l] * Hl[l];
        A[l] = (double *)malloc(sizeof(double) * Pl);
        B[l] = (double *)malloc(sizeof(double) * Pl);
        Ax[l] = (double *)malloc(sizeof(double) * Pl);
        Ay[l] = (double *)malloc(sizeof(double) * Pl);
        if (l == 0) {
            memcpy(A[0], I0, sizeof(double) * P);
            memcpy(B[0], I1, sizeof(double) * P);
        } else {
            orc_downsample(Wl[l - 1], Hl[l - 1], A[l - 1], A[l]);
            orc_downsample(Wl[l - 1], Hl[l - 1], B[l - 1], B[l]);
        }
        orc_gradients(Wl[l], Hl[l], A[l], Ax[l], Ay[l]);
    }
    double *Uc = NULL;
    int Wc = 0, Hc = 0;
    for (int l = L - 1; l >= 0; --l) {
        int w = Wl[l], h = Hl[l];
        int *tmp = (int *)malloc(sizeof(int) * (size_t)(w + h + 2));
        int npx = orc_patch_origins(w, ps, stride, tmp);
        int npy = orc_patch_origins(h, ps, stride, tmp);
        free(tmp);
        double *up = (double *)malloc(sizeof(double) * 2 * (size_t)npx * npy);
        uint8_t *fl = (uint8_t *)malloc((size_t)npx * npy);
        double *U = (double *)malloc(sizeof(double) * 2 * (size_t)w * h);
        orc_patch_search(w, h, A[l], Ax[l], Ay[l], B[l], Uc, Wc, Hc, ps, stride,
                         iters, kappa, up, fl);
        orc_densify(w, h, A[l], B[l], ps, stride, up, U);
        orc_variational(w, h, A[l], Ax[l], Ay[l], B[l], U, var_outer, var_sor,
                        delta, gamma, alpha_s, omega);
        free(up); free(fl);
        if (Uc) free(Uc);
        Uc = U; Wc = w; Hc = h;
    }
    memcpy(U_out, Uc, sizeof(double) * 2 * P);
    free(Uc);
    for (int l = 0; l < L; ++l) { free(A[l]); free(B[l]); free(Ax[l]); free(Ay[l]); }
    return L;
}

/* ---------------------------------------------------------------------------
 * Flow Warping Loss (§IV-C): each event of the window is moved back along
 * the flow to the window's start and accumulated with its polarity; the
 * sharper the resulting image, the better the flow.  FWL = var(I_comp) /
 * var(I_uncomp), the image variance taken over all W*H pixels.
 * Readings:
 *  W1  the flow U [2][H][W] is in pixels per window, so an event at time t
 *      moves by -U(x, y) * (t - t_begin) / (t_end - t_begin), U read at the
 *      event's own pixel; the reference time is t_begin;
 *  W2  each moved event votes its polarity (+1 / -1; +1 for every event when
 *      p is NULL) into the four pixels around its position with bilinear
 *      weights; votes falling outside the image are dropped; I_uncomp is the
 *      same image without moving the events (one vote at the event's pixel);
 *  W3  only events with t_begin <= t < t_end and x < W, y < H take part;
 *  W4  var(I) = mean(I^2) - mean(I)^2; FWL = 1 when var(I_uncomp) = 0.
 * ------------------------------------------------------------------------- */
void orc_iwe(int W, int H, int64_t n, const uint16_t *x, const uint16_t *y, const int64_t *t,
             const int8_t *p, int64_t t_begin, int64_t t_end, const double *U, double *img)
{
    const size_t P = (size_t)W * H;
    memset(img, 0, sizeof(double) * P);
    const double span = (double)(t_end - t_begin);
    for (int64_t i = 0; i < n; ++i) {
        if (t[i] < t_begin || t[i] >= t_end || x[i] >= W || y[i] >= H) continue;
        const double s = p ? (double)p[i] : 1.0;
        double xw = x[i], yw = y[i];
        if (U) {
            const double tau = span > 0 ? (double)(t[i] - t_begin) / span : 0.0;
            const size_t o = (size_t)y[i] * W + x[i];
            const double sg = (orc_mutation == 11) ? 1.0 : -1.0;
            xw += sg * U[o] * tau;
            yw += sg * U[P + o] * tau;
        }
        const double fx0 = floor(xw), fy0 = floor(yw);
        const double ax = xw - fx0, ay = yw - fy0;
        const long X0 = (long)fx0, Y0 = (long)fy0;
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                const long X = X0 + dx, Y = Y0 + dy;
                if (X < 0 || Y < 0 || X >= W || Y >= H) continue;
                const double w = (dx ? ax : 1.0 - ax) * (dy ? ay : 1.0 - ay);
                img[(size_t)Y * W + X] += s * w;
            }
    }
}

static double orc_variance(size_t n, const double *a)
{
    double m = 0.0, q = 0.0;
    for (size_t i = 0; i < n; ++i) { m += a[i]; q += a[i] * a[i]; }
    m /= (double)n;
    return q / (double)n - m * m;
}

/* out[0] = FWL, out[1] = var(I_comp), out[2] = var(I_uncomp). */
void orc_fwl(int W, int H, int64_t n, const uint16_t *x, const uint16_t *y, const int64_t *t,
             const int8_t *p, int64_t t_begin, int64_t t_end, const double *U, double *out)
{
    const size_t P = (size_t)W * H;
    double *ic = (double *)malloc(sizeof(double) * P);
    double *iu = (double *)malloc(sizeof(double) * P);
    orc_iwe(W, H, n, x, y, t, p, t_begin, t_end, U, ic);
    orc_iwe(W, H, n, x, y, t, p, t_begin, t_end, NULL, iu);
    out[1] = orc_variance(P, ic);
    out[2] = orc_variance(P, iu);
    out[0] = out[2] > 0.0 ? out[1] / out[2] : 1.0;
    free(ic);
    free(iu);
}
