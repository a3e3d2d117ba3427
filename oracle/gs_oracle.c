/*
 * gs_oracle.c -- plain FP64 CPU oracle for the differentiable 3D Gaussian
 * rasterizer of CG-SLAM (arXiv 2403.16095, Sec. 3.1-3.4).
 *
 * TEST INFRASTRUCTURE ONLY. The product (CUDA) path never links, loads or
 * calls this file; only the test-suite, the package smoke check and the CPU
 * baseline leg of the benchmark do. It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes (per frame, one camera, one world->camera pose [R|t]):
 *   - Gaussian activation (Eq. 1): s = exp(log_scale), q_hat = q/|q|,
 *     Sigma = R(q_hat) S S^T R(q_hat)^T, opacity = sigmoid(logit).
 *   - EWA projection (Eq. 2): Sigma_2d = J W Sigma W^T J^T + 0.3 I (low-pass
 *     dilation), conic = Sigma_2d^{-1}, centre mu_hat = (fx x/z + cx, fy y/z + cy).
 *   - Per pixel, with NO tiles: every Gaussian whose pixel rectangle holds the
 *     pixel and whose Mahalanobis distance q <= 9 is collected, the list is
 *     sorted by (depth z, index) and alpha-blended front to back
 *     (Eq. 3-5 colour, Eq. 6 alpha-blended depth, Eq. 7-8 median depth,
 *     Eq. 9 accumulated opacity, Eq. 10 depth uncertainty U, plus the blended
 *     per-Gaussian uncertainty nu).
 *   - The loss of Eq. 14/16/19 (L1 colour + L1 depth, optionally weighted per
 *     pixel by 1/(1 + nu_map/tau)) plus optional |U| (Eq. 11) and nu_map terms.
 *   - Its analytic adjoint in FP64: per pixel through the blend, per Gaussian
 *     through the projection to mean, log-scale, quaternion, opacity logit,
 *     colour and nu, and to the camera pose under a left se(3) perturbation
 *     T(xi) = Exp(xi) T, xi = (rho, phi) (Sec. 3.4 optimises the pose in its
 *     Lie algebra; the derivation is reconstructed here from first principles).
 *   - Tile binning by brute force (Sec. 3.1: visible Gaussians pre-sorted near
 *     to far), for the bit-exact tile-list comparison.
 *   - Central differences of a keyframe window's loss (Eq. 21) for every
 *     parameter of chosen Gaussians, re-blending only the pixels the perturbed
 *     Gaussian can reach, with the active-set check of each element.
 *   - The Adam step on the pose in the {so(3) | T} form (Sec. 3.4, Sec. 4).
 *
 * Readings where the paper is silent (prior-art values): near plane 0.2 m is a
 * camera input; dilation 0.3 px^2; alpha = min(0.99, opacity*G); entries with
 * alpha < 1/255 are skipped; blending stops BEFORE an entry that would take
 * the transmittance below 1e-4; footprint r = ceil(3 sqrt(lambda_max)); the
 * Jacobian uses x/z, y/z clamped to +-jclamp * (W/2)/fx (resp. H), gradient 0
 * through a clamped coordinate; pixel (i, j) has its centre at (i+.5, j+.5).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ types */
typedef struct {
    int n;
    const double *means, *log_scales, *quats, *opacity_logit, *colors, *nu;
} orc_scene;

typedef struct {
    int width, height;
    double fx, fy, cx, cy, znear;
} orc_cam;

typedef struct {
    double jclamp;  /* > 0: clamp x/z, y/z in J to +-jclamp * half-FOV tangent */
    double nu_cull; /* > 0: Gaussians with nu > nu_cull are culled            */
} orc_opts;

typedef struct {
    double w_color, w_depth, w_unc, w_nu, unc_tau;
    const double *target_color; /* [3][H][W]                            */
    const double *target_depth; /* [H][W]; also the sensor depth D of U */
    double w_align;             /* weight of L_align (Eq. 12)           */
    const unsigned char *mask;  /* [H][W] or NULL: only pixels with mask != 0 enter the loss
                                   (sampled comparisons; the 1/(HW) factor stays the image's) */
} orc_loss;

typedef struct { /* optional outputs; NULL members are skipped */
    double *color, *depth, *alpha, *unc, *nu_map, *median, *T_final; /* color [3][H][W] */
    int *n_contrib;
    double *margins; /* [6][H][W]: q-9, alpha-1/255, T'-1e-4, opacity*G-0.99, depth gap, T'-0.5 */
    int *dominant;      /* Gaussian with the largest blend weight (Sec. 3.2), -1 if none */
    double *dom_weight; /* that weight w = alpha T                                       */
    double *dom_margin; /* (w_max - second largest w) / w_max; +inf with < 2 entries     */
} orc_image;

typedef struct { /* gradient outputs; NULL members are skipped */
    double *means, *log_scales, *quats, *opacity_logit, *colors, *nu; /* [n][3|4|1] */
    double *g_mean2d, *g_conic, *g_opacity, *g_depth;                 /* per-Gaussian 2D */
    double *pose;                                                     /* [6] (rho, phi) */
} orc_grads;

/* per-Gaussian projection state, kept for the adjoint */
typedef struct {
    int valid;
    double qnorm, qn[4], s[3], R[3][3], Sig[3][3];
    double p[3];
    double ux, uy;    /* x/z and y/z after the optional clamp */
    int clx, cly;     /* clamp active */
    double J[2][3], T[2][3];
    double cov[3];    /* a, b, c of the dilated 2D covariance */
    double det, conic[3];
    double mu[2];
    double opac;
    int radius, rect[4];
} gproj;

static int g_threads = 0;
void orc_set_threads(int n) { g_threads = n; }
int orc_get_threads(void) {
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------- projection */
static void quat_rot(const double q[4], double R[3][3]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static void project_one(const orc_scene *sc, int i, const orc_cam *cam, const double *Tcw,
                        const orc_opts *op, gproj *g) {
    memset(g, 0, sizeof(*g));
    const double *q = sc->quats + 4 * i;
    g->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (!(g->qnorm > 0)) return;
    for (int k = 0; k < 4; ++k) g->qn[k] = q[k] / g->qnorm;
    quat_rot(g->qn, g->R);
    for (int k = 0; k < 3; ++k) g->s[k] = exp(sc->log_scales[3 * i + k]);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += g->R[a][k] * g->s[k] * g->s[k] * g->R[b][k];
            g->Sig[a][b] = acc;
        }
    const double *m = sc->means + 3 * i;
    for (int a = 0; a < 3; ++a)
        g->p[a] = Tcw[4 * a + 0] * m[0] + Tcw[4 * a + 1] * m[1] + Tcw[4 * a + 2] * m[2] + Tcw[4 * a + 3];
    double z = g->p[2];
    if (!(z > cam->znear)) return;
    if (op->nu_cull > 0 && sc->nu[i] > op->nu_cull) return;

    g->ux = g->p[0] / z;
    g->uy = g->p[1] / z;
    if (op->jclamp > 0) {
        double lx = op->jclamp * 0.5 * cam->width / cam->fx;
        double ly = op->jclamp * 0.5 * cam->height / cam->fy;
        if (g->ux < -lx) { g->ux = -lx; g->clx = 1; }
        if (g->ux > lx) { g->ux = lx; g->clx = 1; }
        if (g->uy < -ly) { g->uy = -ly; g->cly = 1; }
        if (g->uy > ly) { g->uy = ly; g->cly = 1; }
    }
    g->J[0][0] = cam->fx / z; g->J[0][1] = 0;            g->J[0][2] = -cam->fx * g->ux / z;
    g->J[1][0] = 0;           g->J[1][1] = cam->fy / z;  g->J[1][2] = -cam->fy * g->uy / z;
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            g->T[r][c] = g->J[r][0] * Tcw[0 * 4 + c] + g->J[r][1] * Tcw[1 * 4 + c] + g->J[r][2] * Tcw[2 * 4 + c];
    double C2[2][2];
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            double acc = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) acc += g->T[r][a] * g->Sig[a][b] * g->T[c][b];
            C2[r][c] = acc;
        }
    g->cov[0] = C2[0][0] + 0.3;
    g->cov[1] = C2[0][1];
    g->cov[2] = C2[1][1] + 0.3;
    g->det = g->cov[0] * g->cov[2] - g->cov[1] * g->cov[1];
    if (!(g->det > 0)) return;
    g->conic[0] = g->cov[2] / g->det;
    g->conic[1] = -g->cov[1] / g->det;
    g->conic[2] = g->cov[0] / g->det;
    g->mu[0] = cam->fx * g->p[0] / z + cam->cx;
    g->mu[1] = cam->fy * g->p[1] / z + cam->cy;

    double half = 0.5 * (g->cov[0] - g->cov[2]);
    double disc = half * half + g->cov[1] * g->cov[1];
    double lam = 0.5 * (g->cov[0] + g->cov[2]) + sqrt(disc > 0 ? disc : 0);
    g->radius = (int)ceil(3.0 * sqrt(lam));
    double r = g->radius;
    double x0 = ceil(g->mu[0] - 0.5 - r), x1 = floor(g->mu[0] - 0.5 + r);
    double y0 = ceil(g->mu[1] - 0.5 - r), y1 = floor(g->mu[1] - 0.5 + r);
    if (x0 < 0) x0 = 0;
    if (y0 < 0) y0 = 0;
    if (x1 > cam->width - 1) x1 = cam->width - 1;
    if (y1 > cam->height - 1) y1 = cam->height - 1;
    if (!(x0 <= x1 && y0 <= y1)) return;
    g->rect[0] = (int)x0; g->rect[1] = (int)y0; g->rect[2] = (int)x1; g->rect[3] = (int)y1;
    g->opac = 1.0 / (1.0 + exp(-sc->opacity_logit[i]));
    g->valid = 1;
}

static gproj *project_all(const orc_scene *sc, const orc_cam *cam, const double *Tcw, const orc_opts *op) {
    gproj *G = (gproj *)malloc(sizeof(gproj) * (size_t)(sc->n > 0 ? sc->n : 1));
    if (!G) return NULL;
#pragma omp parallel for schedule(static) num_threads(orc_get_threads())
    for (int i = 0; i < sc->n; ++i) project_one(sc, i, cam, Tcw, op, &G[i]);
    return G;
}

/* Exported stage view of the projection (per Gaussian). */
int orc_project(const orc_scene *sc, const orc_cam *cam, const double *Tcw, const orc_opts *op,
                double *mean2d, double *conic, double *depth, double *opacity, int *radius,
                int *rect, int *valid) {
    gproj *G = project_all(sc, cam, Tcw, op);
    if (!G) return -1;
    for (int i = 0; i < sc->n; ++i) {
        valid[i] = G[i].valid;
        mean2d[2 * i] = G[i].mu[0]; mean2d[2 * i + 1] = G[i].mu[1];
        for (int k = 0; k < 3; ++k) conic[3 * i + k] = G[i].conic[k];
        depth[i] = G[i].p[2];
        opacity[i] = G[i].opac;
        radius[i] = G[i].radius;
        for (int k = 0; k < 4; ++k) rect[4 * i + k] = G[i].valid ? G[i].rect[k] : (k < 2 ? 1 : 0);
    }
    free(G);
    return 0;
}

/* ----------------------------------------------------------- pixel lists */
typedef struct { double z; int idx; } zent;

static int zent_cmp(const void *a, const void *b) {
    const zent *x = (const zent *)a, *y = (const zent *)b;
    if (x->z < y->z) return -1;
    if (x->z > y->z) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* Row candidate lists: Gaussians whose rect spans each image row. */
typedef struct { int *off, *idx; } rowlists;

static int build_rows(const gproj *G, int n, int H, rowlists *rl) {
    rl->off = (int *)calloc((size_t)H + 1, sizeof(int));
    if (!rl->off) return -1;
    for (int i = 0; i < n; ++i)
        if (G[i].valid)
            for (int y = G[i].rect[1]; y <= G[i].rect[3]; ++y) rl->off[y + 1]++;
    for (int y = 0; y < H; ++y) rl->off[y + 1] += rl->off[y];
    rl->idx = (int *)malloc(sizeof(int) * (size_t)(rl->off[H] > 0 ? rl->off[H] : 1));
    int *cur = (int *)malloc(sizeof(int) * (size_t)H);
    if (!rl->idx || !cur) { free(cur); return -1; }
    memcpy(cur, rl->off, sizeof(int) * (size_t)H);
    for (int i = 0; i < n; ++i)
        if (G[i].valid)
            for (int y = G[i].rect[1]; y <= G[i].rect[3]; ++y) rl->idx[cur[y]++] = i;
    free(cur);
    return 0;
}

/* one contributing list entry, kept for the adjoint */
typedef struct { int k; double alpha, T, G, dx, dy; int clamped; } contrib;

typedef struct {
    double color[3], depth, alpha, unc, nu, median, T;
    int n;
    int med;  /* index (among the blended entries) of the median Gaussian, -1 if none */
    int dom;  /* dominant Gaussian: largest w, the first one in blend order on ties; -1 if none */
    double wmax, w2;  /* largest and second largest blend weight */
    double margin[6];
    uint64_t hash;
} pixout;

static uint64_t fnv(uint64_t h, uint64_t v) {
    for (int b = 0; b < 8; ++b) { h ^= (v >> (8 * b)) & 0xff; h *= 1099511628211ULL; }
    return h;
}

/* Blend one pixel's depth-sorted candidate list (Eq. 3-10). */
static void blend_pixel(const orc_scene *sc, const gproj *G, const zent *list, int nl, int px, int py,
                        double Dp, int has_D, pixout *o, contrib *cb) {
    memset(o, 0, sizeof(*o));
    o->med = -1;
    o->dom = -1;
    for (int k = 0; k < 6; ++k) o->margin[k] = INFINITY;
    o->hash = 1469598103934665603ULL;
    double T = 1.0;
    double prev_z = -1.0;
    for (int e = 0; e < nl; ++e) {
        int k = list[e].idx;
        const gproj *g = &G[k];
        double dx = px + 0.5 - g->mu[0], dy = py + 0.5 - g->mu[1];
        double q = g->conic[0] * dx * dx + 2.0 * g->conic[1] * dx * dy + g->conic[2] * dy * dy;
        double mq = fabs(q - 9.0) / 9.0;
        if (mq < o->margin[0]) o->margin[0] = mq;
        if (q > 9.0) continue;
        if (prev_z >= 0) {
            double mz = fabs(g->p[2] - prev_z) / g->p[2];
            if (mz < o->margin[4]) o->margin[4] = mz;
        }
        prev_z = g->p[2];
        double Gv = exp(-0.5 * q);
        double sg = g->opac * Gv;
        double mc = fabs(sg - 0.99) / 0.99;
        if (mc < o->margin[3]) o->margin[3] = mc;
        int clamped = sg >= 0.99;
        double a = clamped ? 0.99 : sg;
        double ma = fabs(a - 1.0 / 255.0) * 255.0;
        if (ma < o->margin[1]) o->margin[1] = ma;
        if (a < 1.0 / 255.0) continue;
        double Tn = T * (1.0 - a);
        double mt = fabs(Tn - 1e-4) / 1e-4;
        if (mt < o->margin[2]) o->margin[2] = mt;
        if (Tn < 1e-4) { o->hash = fnv(o->hash, 0xffffffffULL); break; }
        double mh = fabs(Tn - 0.5) / 0.5;
        if (mh < o->margin[5]) o->margin[5] = mh;
        double w = a * T;
        for (int c = 0; c < 3; ++c) o->color[c] += w * sc->colors[3 * k + c];
        o->depth += w * g->p[2];
        o->alpha += w;
        if (has_D) o->unc += w * (g->p[2] - Dp) * (g->p[2] - Dp);
        o->nu += w * sc->nu[k];
        if (T >= 0.5 && Tn < 0.5) { o->median = g->p[2]; o->med = o->n; }
        if (w > o->wmax) { o->w2 = o->wmax; o->wmax = w; o->dom = k; }
        else if (w > o->w2) o->w2 = w;
        if (cb) {
            contrib *c = &cb[o->n];
            c->k = k; c->alpha = a; c->T = T; c->G = Gv; c->dx = dx; c->dy = dy; c->clamped = clamped;
        }
        o->hash = fnv(o->hash, (uint64_t)k * 2u + (uint64_t)clamped);
        o->n++;
        T = Tn;
    }
    o->T = T;
}

/* Collect the candidates of pixel (px, py): rect-scatter mode uses the row
 * list, brute-force mode scans every Gaussian. Both test the same predicate. */
static int collect(const gproj *G, int n, const rowlists *rl, int px, int py, zent *buf) {
    int m = 0;
    if (rl) {
        for (int e = rl->off[py]; e < rl->off[py + 1]; ++e) {
            int k = rl->idx[e];
            if (px >= G[k].rect[0] && px <= G[k].rect[2]) { buf[m].z = G[k].p[2]; buf[m].idx = k; ++m; }
        }
    } else {
        for (int k = 0; k < n; ++k)
            if (G[k].valid && px >= G[k].rect[0] && px <= G[k].rect[2] && py >= G[k].rect[1] && py <= G[k].rect[3]) {
                buf[m].z = G[k].p[2]; buf[m].idx = k; ++m;
            }
    }
    qsort(buf, (size_t)m, sizeof(zent), zent_cmp);
    return m;
}

static void store_pixel(orc_image *im, int HW, int p, const pixout *o) {
    if (im->color) for (int c = 0; c < 3; ++c) im->color[c * HW + p] = o->color[c];
    if (im->depth) im->depth[p] = o->depth;
    if (im->alpha) im->alpha[p] = o->alpha;
    if (im->unc) im->unc[p] = o->unc;
    if (im->nu_map) im->nu_map[p] = o->nu;
    if (im->median) im->median[p] = o->median;
    if (im->T_final) im->T_final[p] = o->T;
    if (im->n_contrib) im->n_contrib[p] = o->n;
    if (im->margins) for (int k = 0; k < 6; ++k) im->margins[k * HW + p] = o->margin[k];
    if (im->dominant) im->dominant[p] = o->dom;
    if (im->dom_weight) im->dom_weight[p] = o->wmax;
    if (im->dom_margin) im->dom_margin[p] = o->n >= 2 ? (o->wmax - o->w2) / o->wmax : INFINITY;
}

/* ---------------------------------------------------------------- loss */
static double sgn(double v) { return v > 0 ? 1.0 : (v < 0 ? -1.0 : 0.0); }

/* per-pixel loss value and its gradient w.r.t. the 7 blended channels
 * (r, g, b, depth, opacity, U, nu_map) and, in g[7], the median depth. */
static double pixel_loss(const orc_loss *L, const pixout *o, int p, int HW, double g[8]) {
    double inv = 1.0 / HW;
    double m = L->unc_tau > 0 ? 1.0 / (1.0 + o->nu / L->unc_tau) : 1.0;
    double val = 0;
    for (int c = 0; c < 8; ++c) g[c] = 0;
    if (L->w_align != 0) { /* Eq. 12: |D_alpha - D_median| */
        double d = o->depth - o->median;
        val += inv * L->w_align * fabs(d);
        g[3] += inv * L->w_align * sgn(d);
        g[7] = -inv * L->w_align * sgn(d);
    }
    if (L->w_color != 0 && L->target_color)
        for (int c = 0; c < 3; ++c) {
            double d = o->color[c] - L->target_color[c * HW + p];
            val += inv * m * L->w_color * fabs(d);
            g[c] = inv * m * L->w_color * sgn(d);
        }
    if (L->w_depth != 0 && L->target_depth) {
        double d = o->depth - L->target_depth[p];
        val += inv * m * L->w_depth * fabs(d);
        g[3] += inv * m * L->w_depth * sgn(d);
    }
    if (L->w_unc != 0) { val += inv * L->w_unc * fabs(o->unc); g[5] = inv * L->w_unc * sgn(o->unc); }
    if (L->w_nu != 0) { val += inv * L->w_nu * o->nu; g[6] = inv * L->w_nu; }
    return val;
}

/* ---------------------------------------------------------------- render */
static int max_row_len(const rowlists *rl, int H, int n) {
    if (!rl) return n;
    int mx = 0;
    for (int y = 0; y < H; ++y) if (rl->off[y + 1] - rl->off[y] > mx) mx = rl->off[y + 1] - rl->off[y];
    return mx;
}

/* Full-image forward. mode 0 = brute force per pixel, 1 = rect-scatter. */
int orc_render(const orc_scene *sc, const orc_cam *cam, const double *Tcw, const orc_opts *op,
               const double *obs_depth, int mode, orc_image *im) {
    int W = cam->width, H = cam->height, HW = W * H;
    gproj *G = project_all(sc, cam, Tcw, op);
    if (!G) return -1;
    rowlists rl = {0, 0}, *prl = NULL;
    if (mode == 1) { if (build_rows(G, sc->n, H, &rl)) { free(G); return -1; } prl = &rl; }
    int cap = max_row_len(prl, H, sc->n);
    int err = 0;
#pragma omp parallel num_threads(orc_get_threads())
    {
        zent *buf = (zent *)malloc(sizeof(zent) * (size_t)(cap > 0 ? cap : 1));
        if (!buf) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(static)
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < W && buf; ++px) {
                int p = py * W + px;
                int m = collect(G, sc->n, prl, px, py, buf);
                pixout o;
                blend_pixel(sc, G, buf, m, px, py, obs_depth ? obs_depth[p] : 0, obs_depth != NULL, &o, NULL);
                store_pixel(im, HW, p, &o);
            }
        free(buf);
    }
    free(rl.off); free(rl.idx); free(G);
    return err ? -1 : 0;
}

/* Sampled forward: only the listed pixel indices (p = y*W + x); outputs are
 * indexed by sample position. mode 0 = brute force per pixel, 1 = candidates
 * from the row lists (rect-scatter), as in orc_render. */
int orc_render_pixels(const orc_scene *sc, const orc_cam *cam, const double *Tcw, const orc_opts *op,
                      const double *obs_depth, int n_pix, const int *pix, int mode, orc_image *im) {
    int W = cam->width, H = cam->height;
    gproj *G = project_all(sc, cam, Tcw, op);
    if (!G) return -1;
    rowlists rl = {0, 0}, *prl = NULL;
    if (mode == 1) { if (build_rows(G, sc->n, H, &rl)) { free(G); return -1; } prl = &rl; }
    int cap = max_row_len(prl, H, sc->n);
    int err = 0;
#pragma omp parallel num_threads(orc_get_threads())
    {
        zent *buf = (zent *)malloc(sizeof(zent) * (size_t)(cap > 0 ? cap : 1));
        if (!buf) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 8)
        for (int s = 0; s < n_pix; ++s) {
            if (!buf) continue;
            int p = pix[s], px = p % W, py = p / W;
            int m = collect(G, sc->n, prl, px, py, buf);
            pixout o;
            blend_pixel(sc, G, buf, m, px, py, obs_depth ? obs_depth[p] : 0, obs_depth != NULL, &o, NULL);
            store_pixel(im, n_pix, s, &o);
        }
        free(buf);
    }
    free(rl.off); free(rl.idx); free(G);
    return err ? -1 : 0;
}

/* Loss only (for central finite differences) plus a hash of every discrete
 * decision (membership, clamp, stop) so callers can detect active-set changes. */
int orc_loss_value(const orc_scene *sc, const orc_cam *cam, const double *Tcw, const orc_opts *op,
                   const orc_loss *L, double *loss_out, uint64_t *hash_out) {
    int W = cam->width, H = cam->height, HW = W * H;
    gproj *G = project_all(sc, cam, Tcw, op);
    if (!G) return -1;
    rowlists rl;
    if (build_rows(G, sc->n, H, &rl)) { free(G); return -1; }
    int cap = max_row_len(&rl, H, sc->n);
    double *row_loss = (double *)calloc((size_t)H, sizeof(double));
    uint64_t *row_hash = (uint64_t *)calloc((size_t)H, sizeof(uint64_t));
    int err = (!row_loss || !row_hash);
#pragma omp parallel num_threads(orc_get_threads())
    {
        zent *buf = (zent *)malloc(sizeof(zent) * (size_t)(cap > 0 ? cap : 1));
#pragma omp for schedule(static)
        for (int py = 0; py < H; ++py) {
            if (!buf || err) continue;
            double acc = 0;
            uint64_t h = 1469598103934665603ULL;
            for (int px = 0; px < W; ++px) {
                int p = py * W + px;
                if (L->mask && !L->mask[p]) continue;
                int m = collect(G, sc->n, &rl, px, py, buf);
                pixout o;
                double g[8];
                blend_pixel(sc, G, buf, m, px, py, L->target_depth ? L->target_depth[p] : 0,
                            L->target_depth != NULL, &o, NULL);
                acc += pixel_loss(L, &o, p, HW, g);
                h = fnv(h, o.hash);
            }
            row_loss[py] = acc;
            row_hash[py] = h;
        }
        free(buf);
    }
    double tot = 0;
    uint64_t h = 1469598103934665603ULL;
    for (int y = 0; y < H && !err; ++y) { tot += row_loss[y]; h = fnv(h, row_hash[y]); }
    *loss_out = tot;
    if (hash_out) *hash_out = h;
    free(row_loss); free(row_hash); free(rl.off); free(rl.idx); free(G);
    return err ? -1 : 0;
}

/* ------------------------------------------------------------- adjoint */
enum { A_MU0, A_MU1, A_CA, A_CB, A_CC, A_OP, A_Z, A_NU, A_R, A_G, A_B, A_N };

/* dL/dR(q_hat) -> dL/dq_hat using the partials of the rotation entries. */
static void rot_vjp(const double qn[4], double GR[3][3], double gq[4]) {
    double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
    double dw[3][3] = {{0, -z, y}, {z, 0, -x}, {-y, x, 0}};
    double dx[3][3] = {{0, y, z}, {y, -2 * x, -w}, {z, w, -2 * x}};
    double dy[3][3] = {{-2 * y, x, w}, {x, 0, z}, {-w, z, -2 * y}};
    double dz[3][3] = {{-2 * z, -w, x}, {w, -2 * z, y}, {x, y, 0}};
    gq[0] = gq[1] = gq[2] = gq[3] = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            gq[0] += 2 * GR[a][b] * dw[a][b];
            gq[1] += 2 * GR[a][b] * dx[a][b];
            gq[2] += 2 * GR[a][b] * dy[a][b];
            gq[3] += 2 * GR[a][b] * dz[a][b];
        }
}

/* Chain one Gaussian's 2D gradients back to its parameters and to the pose. */
static void chain_gaussian(const orc_scene *sc, int i, const orc_cam *cam, const double *Tcw,
                           const gproj *g, const double *a2, orc_grads *out, double pose_c[6]) {
    for (int k = 0; k < 6; ++k) pose_c[k] = 0;
    if (out->colors) for (int c = 0; c < 3; ++c) out->colors[3 * i + c] = a2[A_R + c];
    if (out->nu) out->nu[i] = a2[A_NU];
    if (out->opacity_logit) out->opacity_logit[i] = a2[A_OP] * g->opac * (1 - g->opac);

    /* conic (A,B,C) = (c, -b, a) / det  ->  (a, b, c) */
    double a = g->cov[0], b = g->cov[1], c = g->cov[2], det = g->det, d2 = det * det;
    double gA = a2[A_CA], gB = a2[A_CB], gC = a2[A_CC];
    double ga = gA * (-c * c / d2) + gB * (b * c / d2) + gC * (1.0 / det - a * c / d2);
    double gb = gA * (2 * b * c / d2) + gB * (-1.0 / det - 2 * b * b / d2) + gC * (2 * a * b / d2);
    double gc = gA * (1.0 / det - a * c / d2) + gB * (a * b / d2) + gC * (-a * a / d2);
    double G2[2][2] = {{ga, 0.5 * gb}, {0.5 * gb, gc}};

    /* Sigma_2d = T Sigma T^T, T = J W */
    double gT[2][3], gSig[3][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int s = 0; s < 2; ++s)
                for (int m = 0; m < 3; ++m) acc += 2 * G2[r][s] * g->T[s][m] * g->Sig[m][k];
            gT[r][k] = acc;
        }
    for (int u = 0; u < 3; ++u)
        for (int v = 0; v < 3; ++v) {
            double acc = 0;
            for (int r = 0; r < 2; ++r)
                for (int s = 0; s < 2; ++s) acc += g->T[r][u] * G2[r][s] * g->T[s][v];
            gSig[u][v] = acc;
        }
    double gJ[2][3], gW[3][3];
    for (int r = 0; r < 2; ++r)
        for (int m = 0; m < 3; ++m) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += gT[r][k] * Tcw[4 * m + k];
            gJ[r][m] = acc;
        }
    for (int m = 0; m < 3; ++m)
        for (int k = 0; k < 3; ++k) gW[m][k] = g->J[0][m] * gT[0][k] + g->J[1][m] * gT[1][k];

    /* p (camera-space mean) through J, mu_hat and the depth */
    double x = g->p[0], y = g->p[1], z = g->p[2];
    double fx = cam->fx, fy = cam->fy;
    double gp[3] = {0, 0, 0};
    gp[2] += gJ[0][0] * (-fx / (z * z)) + gJ[1][1] * (-fy / (z * z));
    if (g->clx) gp[2] += gJ[0][2] * (fx * g->ux / (z * z));
    else { gp[0] += gJ[0][2] * (-fx / (z * z)); gp[2] += gJ[0][2] * (2 * fx * x / (z * z * z)); }
    if (g->cly) gp[2] += gJ[1][2] * (fy * g->uy / (z * z));
    else { gp[1] += gJ[1][2] * (-fy / (z * z)); gp[2] += gJ[1][2] * (2 * fy * y / (z * z * z)); }
    gp[0] += a2[A_MU0] * fx / z;
    gp[2] += a2[A_MU0] * (-fx * x / (z * z));
    gp[1] += a2[A_MU1] * fy / z;
    gp[2] += a2[A_MU1] * (-fy * y / (z * z));
    gp[2] += a2[A_Z];

    if (out->means)
        for (int k = 0; k < 3; ++k)
            out->means[3 * i + k] = Tcw[0 * 4 + k] * gp[0] + Tcw[1 * 4 + k] * gp[1] + Tcw[2 * 4 + k] * gp[2];

    /* Sigma = M M^T with M = R diag(s) */
    double M[3][3], gM[3][3];
    for (int r = 0; r < 3; ++r) for (int k = 0; k < 3; ++k) M[r][k] = g->R[r][k] * g->s[k];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int m = 0; m < 3; ++m) acc += (gSig[r][m] + gSig[m][r]) * M[m][k];
            gM[r][k] = acc;
        }
    double gR[3][3];
    for (int r = 0; r < 3; ++r) for (int k = 0; k < 3; ++k) gR[r][k] = gM[r][k] * g->s[k];
    if (out->log_scales)
        for (int k = 0; k < 3; ++k) {
            double gs = 0;
            for (int r = 0; r < 3; ++r) gs += gM[r][k] * g->R[r][k];
            out->log_scales[3 * i + k] = gs * g->s[k];
        }
    if (out->quats) {
        double gqn[4];
        rot_vjp(g->qn, gR, gqn);
        double dot = 0;
        for (int k = 0; k < 4; ++k) dot += gqn[k] * g->qn[k];
        for (int k = 0; k < 4; ++k) out->quats[4 * i + k] = (gqn[k] - g->qn[k] * dot) / g->qnorm;
    }

    /* pose: left perturbation Exp(xi) T with xi = (rho, phi):
     *   dp = rho + phi x p,  dW = [phi]_x W.                               */
    pose_c[0] = gp[0]; pose_c[1] = gp[1]; pose_c[2] = gp[2];
    pose_c[3] = y * gp[2] - z * gp[1];
    pose_c[4] = z * gp[0] - x * gp[2];
    pose_c[5] = x * gp[1] - y * gp[0];
    for (int e = 0; e < 3; ++e) {
        double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        /* [e_k]_x */
        if (e == 0) { K[1][2] = -1; K[2][1] = 1; }
        if (e == 1) { K[0][2] = 1; K[2][0] = -1; }
        if (e == 2) { K[0][1] = -1; K[1][0] = 1; }
        double acc = 0;
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                double KW = K[r][0] * Tcw[0 * 4 + k] + K[r][1] * Tcw[1 * 4 + k] + K[r][2] * Tcw[2 * 4 + k];
                acc += gW[r][k] * KW;
            }
        pose_c[3 + e] += acc;
    }
}

/* Forward + loss + analytic adjoint for one frame. */
int orc_grad(const orc_scene *sc, const orc_cam *cam, const double *Tcw, const orc_opts *op,
             const orc_loss *L, orc_grads *out, double *loss_out) {
    int W = cam->width, H = cam->height, HW = W * H, n = sc->n;
    gproj *G = project_all(sc, cam, Tcw, op);
    if (!G) return -1;
    rowlists rl;
    if (build_rows(G, n, H, &rl)) { free(G); return -1; }
    /* compact visible ids so per-thread accumulators stay small */
    int *vid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int nv = 0;
    for (int i = 0; i < n; ++i) vid[i] = G[i].valid ? nv++ : -1;
    int cap = max_row_len(&rl, H, n);
    int nth = orc_get_threads();
    if (nth > 16) nth = 16;
    double *acc = (double *)calloc((size_t)nth * (size_t)(nv > 0 ? nv : 1) * A_N, sizeof(double));
    double *row_loss = (double *)calloc((size_t)H, sizeof(double));
    int err = (!vid || !acc || !row_loss);
#pragma omp parallel num_threads(nth)
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        double *A = acc + (size_t)t * (size_t)nv * A_N;
        zent *buf = (zent *)malloc(sizeof(zent) * (size_t)(cap > 0 ? cap : 1));
        contrib *cb = (contrib *)malloc(sizeof(contrib) * (size_t)(cap > 0 ? cap : 1));
#pragma omp for schedule(static)
        for (int py = 0; py < H; ++py) {
            if (!buf || !cb || err) continue;
            for (int px = 0; px < W; ++px) {
                int p = py * W + px;
                if (L->mask && !L->mask[p]) continue;
                int m = collect(G, n, &rl, px, py, buf);
                double Dp = L->target_depth ? L->target_depth[p] : 0;
                pixout o;
                double gch[8];
                blend_pixel(sc, G, buf, m, px, py, Dp, L->target_depth != NULL, &o, cb);
                row_loss[py] += pixel_loss(L, &o, p, HW, gch);
                double S[7] = {0, 0, 0, 0, 0, 0, 0};
                for (int e = o.n - 1; e >= 0; --e) {
                    const contrib *c = &cb[e];
                    int k = c->k;
                    const gproj *g = &G[k];
                    double f[7] = {sc->colors[3 * k], sc->colors[3 * k + 1], sc->colors[3 * k + 2], g->p[2], 1.0,
                                   (g->p[2] - Dp) * (g->p[2] - Dp), sc->nu[k]};
                    double w = c->alpha * c->T;
                    double dal = 0;
                    for (int ch = 0; ch < 7; ++ch) dal += gch[ch] * (c->T * f[ch] - S[ch] / (1.0 - c->alpha));
                    for (int ch = 0; ch < 7; ++ch) S[ch] += w * f[ch];
                    double *a = A + (size_t)vid[k] * A_N;
                    for (int ch = 0; ch < 3; ++ch) a[A_R + ch] += w * gch[ch];
                    a[A_NU] += w * gch[6];
                    a[A_Z] += w * (gch[3] + 2.0 * gch[5] * (g->p[2] - Dp));
                    if (e == o.med) a[A_Z] += gch[7];  /* D_median = z of this entry (Eq. 7) */
                    if (!c->clamped) {
                        double dpow = dal * g->opac * c->G;
                        a[A_OP] += dal * c->G;
                        a[A_MU0] += dpow * (g->conic[0] * c->dx + g->conic[1] * c->dy);
                        a[A_MU1] += dpow * (g->conic[1] * c->dx + g->conic[2] * c->dy);
                        a[A_CA] += dpow * (-0.5 * c->dx * c->dx);
                        a[A_CB] += dpow * (-c->dx * c->dy);
                        a[A_CC] += dpow * (-0.5 * c->dy * c->dy);
                    }
                }
            }
        }
        free(buf); free(cb);
    }
    if (!err) {
        /* reduce the per-thread accumulators in thread order */
        for (int t = 1; t < nth; ++t)
            for (size_t j = 0; j < (size_t)nv * A_N; ++j) acc[j] += acc[(size_t)t * nv * A_N + j];
        double *pc = (double *)calloc((size_t)(n > 0 ? n : 1) * 6, sizeof(double));
        err = !pc;
#pragma omp parallel for schedule(static) num_threads(orc_get_threads())
        for (int i = 0; i < n; ++i) {
            if (err) continue;
            double zero[A_N] = {0};
            const double *a2 = G[i].valid ? acc + (size_t)vid[i] * A_N : zero;
            if (G[i].valid) chain_gaussian(sc, i, cam, Tcw, &G[i], a2, out, pc + 6 * i);
            else {
                if (out->means) for (int k = 0; k < 3; ++k) out->means[3 * i + k] = 0;
                if (out->log_scales) for (int k = 0; k < 3; ++k) out->log_scales[3 * i + k] = 0;
                if (out->quats) for (int k = 0; k < 4; ++k) out->quats[4 * i + k] = 0;
                if (out->opacity_logit) out->opacity_logit[i] = 0;
                if (out->colors) for (int k = 0; k < 3; ++k) out->colors[3 * i + k] = 0;
                if (out->nu) out->nu[i] = 0;
            }
            if (out->g_mean2d) { out->g_mean2d[2 * i] = a2[A_MU0]; out->g_mean2d[2 * i + 1] = a2[A_MU1]; }
            if (out->g_conic) for (int k = 0; k < 3; ++k) out->g_conic[3 * i + k] = a2[A_CA + k];
            if (out->g_opacity) out->g_opacity[i] = a2[A_OP];
            if (out->g_depth) out->g_depth[i] = a2[A_Z];
        }
        if (out->pose && pc) {
            /* Neumaier-compensated sum over Gaussians in index order */
            for (int k = 0; k < 6; ++k) {
                double s = 0, comp = 0;
                for (int i = 0; i < n; ++i) {
                    double v = pc[6 * i + k], t2 = s + v;
                    comp += fabs(s) >= fabs(v) ? (s - t2) + v : (v - t2) + s;
                    s = t2;
                }
                out->pose[k] = s + comp;
            }
        }
        free(pc);
        double tot = 0;
        for (int y = 0; y < H; ++y) tot += row_loss[y];
        if (loss_out) *loss_out = tot;
    }
    free(acc); free(row_loss); free(vid); free(rl.off); free(rl.idx); free(G);
    return err ? -1 : 0;
}

/* ---------------------------------------- windowed central differences (O14) */
/* Per-pixel state the loss is smooth in: the blend decisions of the pixel
 * (membership, clamp, stop; o->hash), which entry is the median (Eq. 7-8: a
 * jump of D_median when T crosses 0.5 at another entry) and the sign of every
 * absolute-value residual of the loss (its kinks). Two evaluations with equal
 * states differ smoothly, so a central difference across them is a derivative
 * estimate. */
static uint64_t loss_state(const orc_loss *L, const pixout *o, int p, int HW) {
    uint64_t h = fnv(o->hash, (uint64_t)(int64_t)o->med), bits = 0;
    int b = 0;
    if (L->w_color != 0 && L->target_color)
        for (int c = 0; c < 3; ++c) {
            double d = o->color[c] - L->target_color[c * HW + p];
            bits |= (uint64_t)(d > 0 ? 1 : (d < 0 ? 2 : 3)) << (2 * b++);
        }
    if (L->w_depth != 0 && L->target_depth) {
        double d = o->depth - L->target_depth[p];
        bits |= (uint64_t)(d > 0 ? 1 : (d < 0 ? 2 : 3)) << (2 * b++);
    }
    if (L->w_unc != 0) bits |= (uint64_t)(o->unc > 0 ? 1 : (o->unc < 0 ? 2 : 3)) << (2 * b++);
    if (L->w_align != 0) {
        double d = o->depth - o->median;
        bits |= (uint64_t)(d > 0 ? 1 : (d < 0 ? 2 : 3)) << (2 * b++);
    }
    return fnv(h, bits);
}

/* The 15 scalar parameters of Gaussian i, in the order means (3), log-scales
 * (3), quaternion (4), opacity logit, colour (3), nu. */
static void params_of(const orc_scene *sc, int i, double v[15]) {
    for (int k = 0; k < 3; ++k) v[k] = sc->means[3 * i + k];
    for (int k = 0; k < 3; ++k) v[3 + k] = sc->log_scales[3 * i + k];
    for (int k = 0; k < 4; ++k) v[6 + k] = sc->quats[4 * i + k];
    v[10] = sc->opacity_logit[i];
    for (int k = 0; k < 3; ++k) v[11 + k] = sc->colors[3 * i + k];
    v[14] = sc->nu[i];
}

/* Central differences (L(x + h e) - L(x - h e)) / 2h of the window loss
 * sum_f L_f (Eq. 21: one keyframe window, each frame with its own pose and
 * loss) for all 15 parameters of each listed Gaussian.
 *
 * Perturbing Gaussian i changes only the pixels inside the union of its pixel
 * rects over the base and perturbed projections; every other pixel's list and
 * blend are identical, so its loss terms cancel. Per frame the full projection
 * and the row lists are built once; per (Gaussian, frame) the pixels of that
 * union are blended again for the base and the 30 perturbed variants, each
 * pixel's list drawn from the frame's row lists (index order kept, so the
 * (z, index) order is that of the full render). stable[s][k] = 0 when any
 * re-blended pixel's state (loss_state) under +h or -h differs from the base:
 * the active set changed, and the difference is not a derivative estimate. */
int orc_fd_window(const orc_scene *sc, int n_frames, const orc_cam *cams, const double *Tcw,
                  const orc_opts *op, const orc_loss *losses, int n_sel, const int *sel, double h,
                  double *fd, int *stable) {
    enum { NP = 15, NV = 31 };
    for (int e = 0; e < n_sel * NP; ++e) { fd[e] = 0; stable[e] = 1; }
    int err = 0;
    for (int f = 0; f < n_frames && !err; ++f) {
        const orc_cam *cam = &cams[f];
        const double *T = Tcw + 12 * f;
        const orc_loss *L = &losses[f];
        int W = cam->width, H = cam->height, HW = W * H;
        gproj *G = project_all(sc, cam, T, op);
        if (!G) return -1;
        rowlists rl;
        if (build_rows(G, sc->n, H, &rl)) { free(G); return -1; }
#pragma omp parallel num_threads(orc_get_threads())
        {
            int cap = 0;
            int *cand = NULL;
            gproj *lg = NULL;
            double *lcol = NULL, *lnu = NULL;
            zent *buf = NULL;
            uint64_t *base_state = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)W);
#pragma omp for schedule(dynamic, 1)
            for (int s = 0; s < n_sel; ++s) {
                if (err || !base_state) {
#pragma omp atomic write
                    err = 1;
                    continue;
                }
                int i = sel[s];
                double p0[NP], vc[NV][3], vn[NV];
                gproj gv[NV];
                params_of(sc, i, p0);
                /* variant 0: base; 1 + 2k: +h on parameter k; 2 + 2k: -h */
                int ux0 = W, uy0 = H, ux1 = -1, uy1 = -1;
                for (int v = 0; v < NV; ++v) {
                    double pv[NP];
                    memcpy(pv, p0, sizeof(pv));
                    if (v > 0) pv[(v - 1) / 2] += (v & 1) ? h : -h;
                    orc_scene one = {1, pv, pv + 3, pv + 6, pv + 10, pv + 11, pv + 14};
                    project_one(&one, 0, cam, T, op, &gv[v]);
                    for (int c = 0; c < 3; ++c) vc[v][c] = pv[11 + c];
                    vn[v] = pv[14];
                    if (gv[v].valid) {
                        if (gv[v].rect[0] < ux0) ux0 = gv[v].rect[0];
                        if (gv[v].rect[1] < uy0) uy0 = gv[v].rect[1];
                        if (gv[v].rect[2] > ux1) ux1 = gv[v].rect[2];
                        if (gv[v].rect[3] > uy1) uy1 = gv[v].rect[3];
                    }
                }
                if (ux1 < ux0) continue; /* culled in every variant: no pixel changes */
                double acc[NV];
                int moved[NV];
                for (int v = 0; v < NV; ++v) { acc[v] = 0; moved[v] = 0; }
                for (int y = uy0; y <= uy1; ++y) {
                    /* candidates of this row over [ux0, ux1], in index order, with a
                     * slot for Gaussian i at its index position */
                    int row_n = rl.off[y + 1] - rl.off[y] + 1;
                    if (row_n > cap) {
                        cap = row_n * 2;
                        cand = (int *)realloc(cand, sizeof(int) * (size_t)cap);
                        lg = (gproj *)realloc(lg, sizeof(gproj) * (size_t)cap);
                        lcol = (double *)realloc(lcol, sizeof(double) * 3 * (size_t)cap);
                        lnu = (double *)realloc(lnu, sizeof(double) * (size_t)cap);
                        buf = (zent *)realloc(buf, sizeof(zent) * (size_t)cap);
                        if (!cand || !lg || !lcol || !lnu || !buf) {
#pragma omp atomic write
                            err = 1;
                            break;
                        }
                    }
                    int nc = 0, slot = -1;
                    for (int e = rl.off[y]; e < rl.off[y + 1]; ++e) {
                        int j = rl.idx[e];
                        if (j == i) continue;
                        if (G[j].rect[2] < ux0 || G[j].rect[0] > ux1) continue;
                        if (slot < 0 && j > i) { slot = nc; cand[nc++] = i; }
                        cand[nc++] = j;
                    }
                    if (slot < 0) { slot = nc; cand[nc++] = i; }
                    for (int c = 0; c < nc; ++c) {
                        if (c == slot) continue;
                        int j = cand[c];
                        lg[c] = G[j];
                        for (int k = 0; k < 3; ++k) lcol[3 * c + k] = sc->colors[3 * j + k];
                        lnu[c] = sc->nu[j];
                    }
                    orc_scene lsc = {nc, NULL, NULL, NULL, NULL, lcol, lnu};
                    for (int v = 0; v < NV; ++v) {
                        lg[slot] = gv[v];
                        for (int k = 0; k < 3; ++k) lcol[3 * slot + k] = vc[v][k];
                        lnu[slot] = vn[v];
                        for (int x = ux0; x <= ux1; ++x) {
                            int p = y * W + x;
                            if (L->mask && !L->mask[p]) continue;
                            int m = collect(lg, nc, NULL, x, y, buf);
                            double Dp = L->target_depth ? L->target_depth[p] : 0;
                            pixout o;
                            double g8[8];
                            blend_pixel(&lsc, lg, buf, m, x, y, Dp, L->target_depth != NULL, &o, NULL);
                            double val = pixel_loss(L, &o, p, HW, g8);
                            uint64_t st = loss_state(L, &o, p, HW);
                            if (v == 0) base_state[x] = st;
                            else if (st != base_state[x]) moved[v] = 1;
                            acc[v] += val;
                        }
                    }
                }
                if (err) continue;
                for (int k = 0; k < NP; ++k) {
                    fd[s * NP + k] += (acc[1 + 2 * k] - acc[2 + 2 * k]) / (2.0 * h);
                    if (moved[1 + 2 * k] || moved[2 + 2 * k]) stable[s * NP + k] = 0;
                }
            }
            free(cand); free(lg); free(lcol); free(lnu); free(buf); free(base_state);
        }
        free(rl.off); free(rl.idx); free(G);
    }
    return err ? -1 : 0;
}

/* ------------------------------------------------------------- binning */
typedef struct { uint64_t key; uint32_t val; } kv;

static int kv_cmp(const void *a, const void *b) {
    const kv *x = (const kv *)a, *y = (const kv *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->val > y->val) - (x->val < y->val);
}

/* Brute-force tile binning of n records (records of frame f are
 * [f*n_per_frame, (f+1)*n_per_frame)). For every record and every tile of its
 * frame, the record is listed in the tile iff the tile's pixel square overlaps
 * the record's inclusive pixel rect (empty rect: x0 > x1). Pairs are ordered by
 * (global tile id, float bits of the depth, record index).
 * Returns the pair count P, or -1 if P > capacity (nothing written then). */
long long orc_bin_tiles(int n, int n_per_frame, const int *rect, const float *depth, int tile,
                        int n_frames, const int *tiles_x, const int *tiles_y, const int *tile_off,
                        long long capacity, uint64_t *keys, uint32_t *vals, uint32_t *ranges) {
    long long P = 0;
    for (int i = 0; i < n; ++i) {
        int f = i / n_per_frame;
        const int *r = rect + 4 * i;
        if (r[0] > r[2] || r[1] > r[3]) continue;
        for (int ty = 0; ty < tiles_y[f]; ++ty)
            for (int tx = 0; tx < tiles_x[f]; ++tx)
                if (tx * tile <= r[2] && tx * tile + tile - 1 >= r[0] && ty * tile <= r[3] &&
                    ty * tile + tile - 1 >= r[1])
                    ++P;
    }
    if (P > capacity) return -1;
    kv *buf = (kv *)malloc(sizeof(kv) * (size_t)(P > 0 ? P : 1));
    if (!buf) return -2;
    long long m = 0;
    for (int i = 0; i < n; ++i) {
        int f = i / n_per_frame;
        const int *r = rect + 4 * i;
        if (r[0] > r[2] || r[1] > r[3]) continue;
        uint32_t zb;
        memcpy(&zb, &depth[i], 4);
        for (int ty = 0; ty < tiles_y[f]; ++ty)
            for (int tx = 0; tx < tiles_x[f]; ++tx)
                if (tx * tile <= r[2] && tx * tile + tile - 1 >= r[0] && ty * tile <= r[3] &&
                    ty * tile + tile - 1 >= r[1]) {
                    uint64_t t = (uint64_t)(tile_off[f] + ty * tiles_x[f] + tx);
                    buf[m].key = (t << 32) | zb;
                    buf[m].val = (uint32_t)i;
                    ++m;
                }
    }
    qsort(buf, (size_t)P, sizeof(kv), kv_cmp);
    int n_tiles = tile_off[n_frames - 1] + tiles_x[n_frames - 1] * tiles_y[n_frames - 1];
    for (int t = 0; t < 2 * n_tiles; ++t) ranges[t] = 0;
    for (long long k = 0; k < P; ++k) {
        keys[k] = buf[k].key;
        vals[k] = buf[k].val;
        uint32_t t = (uint32_t)(buf[k].key >> 32);
        if (k == 0 || (uint32_t)(buf[k - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)k;
        if (k == P - 1 || (uint32_t)(buf[k + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(k + 1);
    }
    free(buf);
    return P;
}

/* ------------------------------------------------------- pose update */
/* One Adam step on the pose in the {so(3) | T} form of Sec. 3.4: the left
 * gradient (rho, phi) is converted to g_t = g_rho, g_R = g_phi - t x g_rho,
 * then R <- Exp(d_phi) R, t <- t + d_t with d = -lr * mhat / (sqrt(vhat)+eps).
 * state: R[9], t[3], m[6], v[6], step count. */
static void so3_exp(const double w[3], double R[3][3]) {
    double th = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double K[3][3] = {{0, -w[2], w[1]}, {w[2], 0, -w[0]}, {-w[1], w[0], 0}};
    double a, b;
    if (th < 1e-8) { a = 1.0 - th * th / 6.0; b = 0.5 - th * th / 24.0; }
    else { a = sin(th) / th; b = (1.0 - cos(th)) / (th * th); }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double KK = K[i][0] * K[0][j] + K[i][1] * K[1][j] + K[i][2] * K[2][j];
            R[i][j] = (i == j) + a * K[i][j] + b * KK;
        }
}

void orc_adam_step(double *state, const double grad[6], double lr_rot, double lr_trans, double beta1,
                   double beta2, double eps) {
    double *R = state, *t = state + 9, *m = state + 12, *v = state + 18;
    double step = state[24] + 1.0;
    state[24] = step;
    double g[6];
    g[0] = grad[0]; g[1] = grad[1]; g[2] = grad[2];
    g[3] = grad[3] - (t[1] * grad[2] - t[2] * grad[1]);
    g[4] = grad[4] - (t[2] * grad[0] - t[0] * grad[2]);
    g[5] = grad[5] - (t[0] * grad[1] - t[1] * grad[0]);
    double d[6];
    for (int k = 0; k < 6; ++k) {
        m[k] = beta1 * m[k] + (1 - beta1) * g[k];
        v[k] = beta2 * v[k] + (1 - beta2) * g[k] * g[k];
        double mh = m[k] / (1 - pow(beta1, step)), vh = v[k] / (1 - pow(beta2, step));
        d[k] = -(k < 3 ? lr_trans : lr_rot) * mh / (sqrt(vh) + eps);
    }
    double dR[3][3], Rn[3][3];
    so3_exp(d + 3, dR);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Rn[i][j] = dR[i][0] * R[0 * 3 + j] + dR[i][1] * R[1 * 3 + j] + dR[i][2] * R[2 * 3 + j];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) R[3 * i + j] = Rn[i][j];
    for (int k = 0; k < 3; ++k) t[k] += d[k];
}
