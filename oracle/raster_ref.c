/*
 * FP64 CPU oracle for the splatting part of the VBM fine-tuning step.
 * TEST INFRASTRUCTURE ONLY: called by the tests, by __graft_entry__.smoke()
 * and by the CPU-baseline leg of bench.py; never by the CUDA library, with
 * which it shares no code.
 *
 * Sec. 4.4 fine-tunes the Gaussians "as in" 3D Gaussian Splatting (3DGS):
 * EWA projection of each 3D Gaussian to a 2D conic, tile binning with a
 * depth order, front-to-back alpha compositing and the reverse-mode
 * derivative of all of it.  The paper fixes none of the constants; the
 * readings are the 3DGS ones, each named below:
 *   ZNEAR (camera field)  cull when camera-space z <= znear (0.2)
 *   FRUSTUM_GUARD 0.15    x/z, y/z clamped to the image extended by 15% per
 *                         side before the Jacobian (1.3 tan(fov/2) for a
 *                         centred principal point)
 *   DILATION 0.3          added to the diagonal of the 2D covariance
 *   EIG_FLOOR 0.1         lambda_max = mid + sqrt(max(0.1, mid^2 - det))
 *   RADIUS_SIGMAS 3       r = ceil(k sqrt(lambda_max)) pixels with
 *                         k = min(3, sqrt(2 ln(255 o))): the 3-sigma extent of
 *                         3DGS, shrunk to the ellipse outside which
 *                         o e^power < 1/255 (such pairs are skipped anyway, so
 *                         the image is unchanged); Gaussians with o < 1/255 can
 *                         never be composited and get no tiles
 *   ALPHA_MAX 0.99, ALPHA_MIN 1/255, T_MIN 1e-4 compositing cut-offs
 * Pixel (i, j) has its centre at (i + 1/2, j + 1/2); the image-plane mean is
 * (fx x/z + cx, fy y/z + cy).  A Gaussian's tile rectangle covers the tiles
 * containing u - r .. u + r (and v - r .. v + r), clamped to the image:
 *   x0 = clamp(floor((u - r) / TW), 0, TX), x1 = clamp(floor((u + r) / TW) + 1, 0, TX)
 * computed exactly as integer divisions of floor(u) -/+ r.  Of that
 * rectangle, a tile is listed only if some point of the rectangle of its
 * pixel centres can see alpha >= 1/255 (tile_min_q below, with a margin of
 * CULL_MARGIN in the log): a pixel of an unlisted tile would skip the splat
 * anyway, so images and gradients are those of the whole rectangle.
 * Order within a tile: ascending depth (camera z), ties by item index.
 *
 * Layouts (all row-major, double unless stated):
 *   params   P[14][n]: mean(3) log_scale(3) quat wxyz(4) opacity_logit(1) rgb(3)
 *   camera   19 doubles: R[9] t[3] fx fy cx cy znear width height
 *   proj     per item NPROJ doubles (enum below)
 *   splat    per item 6 doubles: u v A B C opacity (conic = inverse 2D cov)
 *   image    [V][3][H][W], per-pixel state [V][H][W]
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FRUSTUM_GUARD 0.15
#define DILATION 0.3
#define EIG_FLOOR 0.1
#define RADIUS_SIGMAS 3.0
#define ALPHA_MAX 0.99
#define ALPHA_MIN (1.0 / 255.0)
#define T_MIN 1e-4
#define COORD_CLAMP 1e7
#define CULL_MARGIN 1e-3

enum { CAM_R = 0, CAM_T = 9, CAM_FX = 12, CAM_FY, CAM_CX, CAM_CY, CAM_ZNEAR, CAM_W, CAM_H, CAM_N };

enum {
    PJ_U = 0, PJ_V, PJ_A, PJ_B, PJ_C, PJ_OPAC, PJ_DEPTH, PJ_RADIUS,
    PJ_X0, PJ_Y0, PJ_X1, PJ_Y1, PJ_TOUCHED,
    PJ_M_RADIUS,   /* distance of 3 sqrt(lambda_max) to the nearest integer      */
    PJ_M_RECT,     /* distance (px) of u -/+ r, v -/+ r to the nearest tile edge */
    PJ_M_CULL,     /* |z - znear|                                               */
    PJ_M_CLAMP,    /* distance of x/z, y/z to the frustum clamp limits           */
    PJ_M_OPAC,     /* |255 o - 1|: distance of the opacity to the 1/255 cut-off  */
    NPROJ
};

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static int64_t clampi(int64_t x, int64_t lo, int64_t hi) { return x < lo ? lo : (x > hi ? hi : x); }
static int64_t floordiv(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) q--; return q; }
static double dist_to_multiple(double x, double m) { double r = fmod(x, m); if (r < 0) r += m; return r < m - r ? r : m - r; }

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

typedef struct {
    double mu[3], s[3], qn[4], qnorm, R[3][3], Sig[3][3];
    double t[3], xzc, yzc, clampx, clampy;   /* clampx: 1 if x/z was clamped */
    double J00, J02, J11, J12, T0[3], T1[3];
    double a, b, c, det, opac;
    int culled;
} proj_state;

/* Forward EWA projection of Gaussian i for one camera (3DGS conventions). */
static void project_state(const double *P, int64_t n, int64_t i, const double *cam, proj_state *st)
{
    memset(st, 0, sizeof(*st));
    const double *Wm = cam + CAM_R;
    for (int k = 0; k < 3; k++) st->mu[k] = P[k * n + i];
    for (int k = 0; k < 3; k++) st->s[k] = exp(P[(3 + k) * n + i]);
    double q[4];
    for (int k = 0; k < 4; k++) q[k] = P[(6 + k) * n + i];
    st->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; k++) st->qn[k] = q[k] / st->qnorm;
    quat_to_rot(st->qn, st->R);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += st->R[a][k] * st->s[k] * st->s[k] * st->R[b][k];
            st->Sig[a][b] = acc;
        }
    for (int r = 0; r < 3; r++)
        st->t[r] = Wm[3 * r] * st->mu[0] + Wm[3 * r + 1] * st->mu[1] + Wm[3 * r + 2] * st->mu[2] + cam[CAM_T + r];
    st->opac = 1.0 / (1.0 + exp(-P[10 * n + i]));
    if (st->t[2] <= cam[CAM_ZNEAR]) { st->culled = 1; return; }
    double fx = cam[CAM_FX], fy = cam[CAM_FY], cx = cam[CAM_CX], cy = cam[CAM_CY];
    double Wi = cam[CAM_W], Hi = cam[CAM_H], tz = st->t[2];
    double xz = st->t[0] / tz, yz = st->t[1] / tz;
    double xlo = (-FRUSTUM_GUARD * Wi - cx) / fx, xhi = ((1 + FRUSTUM_GUARD) * Wi - cx) / fx;
    double ylo = (-FRUSTUM_GUARD * Hi - cy) / fy, yhi = ((1 + FRUSTUM_GUARD) * Hi - cy) / fy;
    st->xzc = clampd(xz, xlo, xhi);
    st->yzc = clampd(yz, ylo, yhi);
    st->clampx = (st->xzc != xz);
    st->clampy = (st->yzc != yz);
    st->J00 = fx / tz; st->J02 = -fx * st->xzc / tz;
    st->J11 = fy / tz; st->J12 = -fy * st->yzc / tz;
    for (int k = 0; k < 3; k++) {
        st->T0[k] = st->J00 * Wm[k] + st->J02 * Wm[6 + k];
        st->T1[k] = st->J11 * Wm[3 + k] + st->J12 * Wm[6 + k];
    }
    double a = 0, b = 0, c = 0;
    for (int p = 0; p < 3; p++)
        for (int q2 = 0; q2 < 3; q2++) {
            a += st->T0[p] * st->Sig[p][q2] * st->T0[q2];
            b += st->T0[p] * st->Sig[p][q2] * st->T1[q2];
            c += st->T1[p] * st->Sig[p][q2] * st->T1[q2];
        }
    st->a = a + DILATION; st->b = b; st->c = c + DILATION;
    st->det = st->a * st->c - st->b * st->b;
    if (st->det <= 0) st->culled = 1;
}

/* Projection of items: item it = (view of cam, Gaussian gidx[it]). */
/*
 * Binning tile test.  alpha = o e^(-q/2) >= 1/255 with q = A dx^2 + 2 B dx dy
 * + C dy^2 (dx = x - u, dy = y - v) means q <= 2 ln(255 o).  The smallest q
 * over the rectangle [x0, x1] x [y0, y1] of a tile's pixel centres is 0 if
 * (u, v) lies inside; else it lies on an edge, where the 1D minimiser along
 * the edge (dy = -(B / C) dx on a vertical edge, dx = -(B / A) dy on a
 * horizontal one) is clamped to the edge.  The tile is listed when that
 * minimum is <= tau = 2 (ln(255 o) + CULL_MARGIN).  Two copies: double for the
 * FP64 pipeline (all four edges: the plain definition), and float, operation
 * by operation, for checking a float32 implementation's lists bit for bit
 * from its own float32 splat records (bc = B / C and ba = B / A rounded to
 * float; compiled with -ffp-contract=off, so nothing is fused).  The float
 * copy follows that implementation in evaluating only the edges whose
 * half-planes exclude the centre (x0 if u < x0, x1 if u > x1, likewise in y):
 * the minimum of a convex quadratic over a box lies on such an edge (at a
 * point inside an edge the level set through it touches the edge from the far
 * side, where the centre lies; at a corner a line through the corner
 * separates the box from that level set, so the centre violates one of the
 * corner's two edges), and each kept edge is evaluated with the same
 * operations as in the four-edge form.
 */
static double tile_min_q(double u, double v, double A, double B, double C, double bc, double ba, double x0,
                         double x1, double y0, double y1)
{
    if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return 0.0;
    double best = INFINITY;
    for (int e = 0; e < 2; e++) {
        double dx = (e ? x1 : x0) - u;
        double dy = fmin(fmax(v - bc * dx, y0), y1) - v;
        double q = (A * dx) * dx + ((2.0 * B) * dx) * dy + (C * dy) * dy;
        best = fmin(best, q);
        double ey = (e ? y1 : y0) - v;
        double ex = fmin(fmax(u - ba * ey, x0), x1) - u;
        q = (A * ex) * ex + ((2.0 * B) * ex) * ey + (C * ey) * ey;
        best = fmin(best, q);
    }
    return best;
}

static float tile_min_q_f32(float u, float v, float A, float B, float C, float bc, float ba, float x0, float x1,
                            float y0, float y1)
{
    int left = u < x0, right = u > x1, below = v < y0, above = v > y1;
    if (!(left || right || below || above)) return 0.0f;
    float dx = (left ? x0 : x1) - u;
    float dy = fminf(fmaxf(v - bc * dx, y0), y1) - v;
    float qv = (A * dx) * dx + ((2.0f * B) * dx) * dy + (C * dy) * dy;
    float ey = (below ? y0 : y1) - v;
    float ex = fminf(fmaxf(u - ba * ey, x0), x1) - u;
    float qh = (A * ex) * ex + ((2.0f * B) * ex) * ey + (C * ey) * ey;
    return fminf(left || right ? qv : INFINITY, below || above ? qh : INFINITY);
}

/* The tile test, exported for the oracle's own tests. */
double orc_tile_min_q(double u, double v, double A, double B, double C, double x0, double x1, double y0, double y1)
{
    return tile_min_q(u, v, A, B, C, B / C, B / A, x0, x1, y0, y1);
}

/* Its float copy, exported likewise (bc, ba as the caller rounded them). */
float orc_tile_min_q_f32(float u, float v, float A, float B, float C, float bc, float ba, float x0, float x1,
                         float y0, float y1)
{
    return tile_min_q_f32(u, v, A, B, C, bc, ba, x0, x1, y0, y1);
}

/* Is tile (tx, ty) listed for a splat record sp = u v A B C bc ba tau? */
static int tile_listed(const double *sp, int tx, int ty, int tile_w, int tile_h, int W, int H)
{
    double x0 = tx * tile_w + 0.5, x1 = (tx * tile_w + tile_w < W ? tx * tile_w + tile_w : W) - 0.5;
    double y0 = ty * tile_h + 0.5, y1 = (ty * tile_h + tile_h < H ? ty * tile_h + tile_h : H) - 0.5;
    return tile_min_q(sp[0], sp[1], sp[2], sp[3], sp[4], sp[5], sp[6], x0, x1, y0, y1) <= sp[7];
}

static int tile_listed_f32(const float *sp, int tx, int ty, int tile_w, int tile_h, int W, int H)
{
    float x0 = (float)(tx * tile_w) + 0.5f;
    float x1 = (float)(tx * tile_w + tile_w < W ? tx * tile_w + tile_w : W) - 0.5f;
    float y0 = (float)(ty * tile_h) + 0.5f;
    float y1 = (float)(ty * tile_h + tile_h < H ? ty * tile_h + tile_h : H) - 0.5f;
    return tile_min_q_f32(sp[0], sp[1], sp[2], sp[3], sp[4], sp[5], sp[6], x0, x1, y0, y1) <= sp[7];
}

void orc_project(int64_t n_items, const int64_t *gidx, const double *P, int64_t n,
                 const double *cam, int tile_w, int tile_h, double *out)
{
    int64_t TX = ((int64_t)cam[CAM_W] + tile_w - 1) / tile_w;
    int64_t TY = ((int64_t)cam[CAM_H] + tile_h - 1) / tile_h;
    double xlo = (-FRUSTUM_GUARD * cam[CAM_W] - cam[CAM_CX]) / cam[CAM_FX];
    double xhi = ((1 + FRUSTUM_GUARD) * cam[CAM_W] - cam[CAM_CX]) / cam[CAM_FX];
    double ylo = (-FRUSTUM_GUARD * cam[CAM_H] - cam[CAM_CY]) / cam[CAM_FY];
    double yhi = ((1 + FRUSTUM_GUARD) * cam[CAM_H] - cam[CAM_CY]) / cam[CAM_FY];
    for (int64_t it = 0; it < n_items; it++) {
        double *o = out + it * NPROJ;
        memset(o, 0, NPROJ * sizeof(double));
        proj_state st;
        project_state(P, n, gidx[it], cam, &st);
        o[PJ_DEPTH] = st.t[2];
        o[PJ_OPAC] = st.opac;
        o[PJ_M_CULL] = fabs(st.t[2] - cam[CAM_ZNEAR]);
        o[PJ_M_OPAC] = fabs(255.0 * st.opac - 1.0);
        if (st.culled || st.opac < ALPHA_MIN) continue;
        o[PJ_A] = st.c / st.det;
        o[PJ_B] = -st.b / st.det;
        o[PJ_C] = st.a / st.det;
        double mid = 0.5 * (st.a + st.c);
        double disc = mid * mid - st.det;
        double lam1 = mid + sqrt(disc > EIG_FLOOR ? disc : EIG_FLOOR);
        double k = sqrt(2.0 * log(255.0 * st.opac));
        if (k > RADIUS_SIGMAS) k = RADIUS_SIGMAS;
        double rr = k * sqrt(lam1);
        double r = ceil(rr);
        o[PJ_RADIUS] = r;
        o[PJ_M_RADIUS] = fmin(rr - floor(rr), ceil(rr) - rr);
        double xz = st.t[0] / st.t[2], yz = st.t[1] / st.t[2];
        double u = cam[CAM_FX] * xz + cam[CAM_CX];
        double v = cam[CAM_FY] * yz + cam[CAM_CY];
        o[PJ_U] = u; o[PJ_V] = v;
        o[PJ_M_CLAMP] = fmin(fmin(fabs(xz - xlo), fabs(xz - xhi)), fmin(fabs(yz - ylo), fabs(yz - yhi)));
        int64_t ri = (int64_t)r;
        int64_t fu = (int64_t)floor(clampd(u, -COORD_CLAMP, COORD_CLAMP));
        int64_t fv = (int64_t)floor(clampd(v, -COORD_CLAMP, COORD_CLAMP));
        int64_t x0 = clampi(floordiv(fu - ri, tile_w), 0, TX);
        int64_t x1 = clampi(floordiv(fu + ri, tile_w) + 1, 0, TX);
        int64_t y0 = clampi(floordiv(fv - ri, tile_h), 0, TY);
        int64_t y1 = clampi(floordiv(fv + ri, tile_h) + 1, 0, TY);
        o[PJ_X0] = x0; o[PJ_X1] = x1; o[PJ_Y0] = y0; o[PJ_Y1] = y1;
        double sp[8] = {u, v, o[PJ_A], o[PJ_B], o[PJ_C], o[PJ_B] / o[PJ_C], o[PJ_B] / o[PJ_A],
                        2.0 * (log(255.0 * st.opac) + CULL_MARGIN)};
        int64_t listed = 0;
        for (int64_t ty = y0; ty < y1; ty++)
            for (int64_t tx = x0; tx < x1; tx++)
                listed += tile_listed(sp, (int)tx, (int)ty, tile_w, tile_h, (int)cam[CAM_W], (int)cam[CAM_H]);
        o[PJ_TOUCHED] = (double)listed;
        o[PJ_M_RECT] = fmin(fmin(dist_to_multiple(u - r, tile_w), dist_to_multiple(u + r, tile_w)),
                            fmin(dist_to_multiple(v - r, tile_h), dist_to_multiple(v + r, tile_h)));
    }
}

/* ---------------------------------------------------------------- binning */

typedef struct { int64_t tile; double depth; int64_t order; int32_t item; } pair_rec;

static int cmp_pair(const void *pa, const void *pb)
{
    const pair_rec *a = pa, *b = pb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->order < b->order ? -1 : (a->order > b->order);
}

/*
 * Emit one (global tile, item) pair per listed tile of each item's rectangle,
 * items in index order and tiles row-major, then sort by (tile, depth,
 * emission order).  global tile = view * TY * TX + ty * TX + tx.  A tile is
 * listed by the test above on the splat records sp64 (double) or sp32 (float)
 * [n][8] = u v A B C bc ba tau; with neither, every tile of the rectangle is.
 * Writes the sorted tiles and items and, per global tile, [start, end) into
 * ranges (2 ints).  Returns the number of pairs, or -1 if it exceeds capacity.
 */
static int listed(const double *sp64, const float *sp32, int64_t it, int tx, int ty, int tile_w, int tile_h,
                  int W, int H)
{
    if (sp64) return tile_listed(sp64 + 8 * it, tx, ty, tile_w, tile_h, W, H);
    if (sp32) return tile_listed_f32(sp32 + 8 * it, tx, ty, tile_w, tile_h, W, H);
    return 1;
}

int64_t orc_bin_sort(int64_t n_items, const int32_t *view_of, const int32_t *rect /* [n][4] x0 y0 x1 y1 */,
                     const double *depth, int TX, int TY, int n_views, int64_t capacity,
                     int64_t *tiles_out, int32_t *items_out, int32_t *ranges, const double *sp64,
                     const float *sp32, int tile_w, int tile_h, int W, int H)
{
    int64_t total = 0;
    for (int64_t it = 0; it < n_items; it++) {
        const int32_t *rc = rect + 4 * it;
        for (int ty = rc[1]; ty < rc[3]; ty++)
            for (int tx = rc[0]; tx < rc[2]; tx++) total += listed(sp64, sp32, it, tx, ty, tile_w, tile_h, W, H);
    }
    if (total > capacity) return -1;
    pair_rec *pr = (pair_rec *)malloc((size_t)(total > 0 ? total : 1) * sizeof(pair_rec));
    int64_t k = 0;
    for (int64_t it = 0; it < n_items; it++) {
        const int32_t *rc = rect + 4 * it;
        for (int ty = rc[1]; ty < rc[3]; ty++)
            for (int tx = rc[0]; tx < rc[2]; tx++) {
                if (!listed(sp64, sp32, it, tx, ty, tile_w, tile_h, W, H)) continue;
                pr[k].tile = (int64_t)view_of[it] * TY * TX + (int64_t)ty * TX + tx;
                pr[k].depth = depth[it];
                pr[k].order = k;
                pr[k].item = (int32_t)it;
                k++;
            }
    }
    qsort(pr, (size_t)total, sizeof(pair_rec), cmp_pair);
    int64_t n_tiles = (int64_t)n_views * TY * TX;
    for (int64_t t = 0; t < 2 * n_tiles; t++) ranges[t] = 0;
    for (int64_t p = 0; p < total; p++) {
        tiles_out[p] = pr[p].tile;
        items_out[p] = pr[p].item;
        if (p == 0 || pr[p - 1].tile != pr[p].tile) ranges[2 * pr[p].tile] = (int32_t)p;
        if (p == total - 1 || pr[p + 1].tile != pr[p].tile) ranges[2 * pr[p].tile + 1] = (int32_t)(p + 1);
    }
    free(pr);
    return total;
}

/* ----------------------------------------------------------- compositing */

typedef struct {
    const int32_t *ranges, *items;
    const double *splat, *color, *bg;
    int W, H, tw, th, TX, TY;
} scene_desc;

typedef struct { int32_t item; double alpha, T, G; int clamped; } contrib;

/*
 * Front-to-back compositing of one pixel over its tile's list (3DGS rules):
 * power = -1/2 (A dx^2 + C dy^2) - B dx dy with (dx, dy) = mean - pixel
 * centre; skip if power > 0; alpha = min(0.99, o e^power); skip if
 * alpha < 1/255; stop (without blending) once T (1 - alpha) < 1e-4; else
 * C += c alpha T, T *= 1 - alpha.  Fills the contributor list when given.
 * Returns the number of blended Gaussians; *last = 1-based list position of
 * the last blended one; *n_eval = list positions evaluated; *margin =
 * smallest relative distance of a decision to its cut-off.
 */
static int composite_pixel(const scene_desc *sd, int view, int px, int py, double Cout[3], double *Tout,
                           int32_t *last, int32_t *n_eval, double *margin, contrib *list)
{
    int64_t tile = (int64_t)view * sd->TY * sd->TX + (int64_t)(py / sd->th) * sd->TX + (px / sd->tw);
    int32_t start = sd->ranges[2 * tile], end = sd->ranges[2 * tile + 1];
    double pxc = px + 0.5, pyc = py + 0.5, T = 1.0, C[3] = {0, 0, 0}, m = INFINITY;
    int nc = 0;
    int32_t lastc = 0, ev = 0;
    for (int32_t p = start; p < end; p++) {
        int32_t it = sd->items[p];
        const double *s = sd->splat + 6 * (int64_t)it;
        double dx = s[0] - pxc, dy = s[1] - pyc;
        double power = -0.5 * (s[2] * dx * dx + s[4] * dy * dy) - s[3] * dx * dy;
        ev = p - start + 1;
        if (power > 0) continue;
        double G = exp(power);
        double raw = s[5] * G;
        m = fmin(m, fabs(raw / ALPHA_MIN - 1.0));
        double alpha = raw < ALPHA_MAX ? raw : ALPHA_MAX;
        if (alpha < ALPHA_MIN) continue;
        double testT = T * (1.0 - alpha);
        m = fmin(m, fabs(testT / T_MIN - 1.0));
        if (testT < T_MIN) break;
        const double *col = sd->color + 3 * (int64_t)it;
        for (int ch = 0; ch < 3; ch++) C[ch] += col[ch] * alpha * T;
        if (list) { list[nc].item = it; list[nc].alpha = alpha; list[nc].T = T; list[nc].G = G; list[nc].clamped = raw >= ALPHA_MAX; }
        nc++;
        T = testT;
        lastc = p - start + 1;
    }
    for (int ch = 0; ch < 3; ch++) Cout[ch] = C[ch] + T * sd->bg[ch];
    *Tout = T;
    if (last) *last = lastc;
    if (n_eval) *n_eval = ev;
    if (margin) *margin = m;
    return nc;
}

void orc_render(int n_views, int W, int H, int tile_w, int tile_h, const int32_t *ranges, const int32_t *items,
                const double *splat, const double *color, const double *bg,
                double *img, double *T_final, int32_t *n_contrib, int32_t *n_eval, double *margin,
                int32_t *n_blend)
{
    scene_desc sd = {ranges, items, splat, color, bg, W, H, tile_w, tile_h,
                     (W + tile_w - 1) / tile_w, (H + tile_h - 1) / tile_h};
    int64_t HW = (int64_t)H * W;
    for (int v = 0; v < n_views; v++)
        for (int py = 0; py < H; py++)
            for (int px = 0; px < W; px++) {
                double C[3], T, m;
                int32_t last, ev;
                int nb = composite_pixel(&sd, v, px, py, C, &T, &last, &ev, &m, NULL);
                int64_t pix = (int64_t)py * W + px;
                for (int ch = 0; ch < 3; ch++) img[((int64_t)v * 3 + ch) * HW + pix] = C[ch];
                T_final[v * HW + pix] = T;
                n_contrib[v * HW + pix] = last;
                if (n_eval) n_eval[v * HW + pix] = ev;
                if (margin) margin[v * HW + pix] = m;
                if (n_blend) n_blend[v * HW + pix] = nb;
            }
}

/*
 * Reverse-mode derivative of the composited image.  With contributors
 * k = 1..K (alpha_k, T_k = transmittance before k), C = sum_k c_k alpha_k T_k
 * + T_final bg and 1 - T_final as the alpha output:
 *   dC/dc_k     = alpha_k T_k
 *   dC/dalpha_k = c_k T_k - (S_k + T_final bg) / (1 - alpha_k),  S_k = sum_{m>k} c_m alpha_m T_m
 *   d(1-T_final)/dalpha_k = T_final / (1 - alpha_k)
 * then alpha = o G (zero derivative where the 0.99 clamp is active),
 * G = e^power.  Accumulates per item: du dv dA dB dC dopacity (g_splat[6])
 * and colour (g_color[3]).
 */
void orc_render_bwd(int n_views, int W, int H, int tile_w, int tile_h, const int32_t *ranges, const int32_t *items,
                    const double *splat, const double *color, const double *bg,
                    const double *dL_dimg, const double *dL_dalpha, double *g_splat, double *g_color,
                    int64_t max_list)
{
    scene_desc sd = {ranges, items, splat, color, bg, W, H, tile_w, tile_h,
                     (W + tile_w - 1) / tile_w, (H + tile_h - 1) / tile_h};
    int64_t HW = (int64_t)H * W;
    contrib *list = (contrib *)malloc((size_t)(max_list > 0 ? max_list : 1) * sizeof(contrib));
    for (int v = 0; v < n_views; v++)
        for (int py = 0; py < H; py++)
            for (int px = 0; px < W; px++) {
                double C[3], Tf;
                int nc = composite_pixel(&sd, v, px, py, C, &Tf, NULL, NULL, NULL, list);
                int64_t pix = (int64_t)py * W + px;
                double dC[3];
                for (int ch = 0; ch < 3; ch++) dC[ch] = dL_dimg[((int64_t)v * 3 + ch) * HW + pix];
                double dA_out = dL_dalpha ? dL_dalpha[v * HW + pix] : 0.0;
                double S[3] = {0, 0, 0};
                for (int k = nc - 1; k >= 0; k--) {
                    int32_t it = list[k].item;
                    const double *s = splat + 6 * (int64_t)it;
                    const double *col = color + 3 * (int64_t)it;
                    double al = list[k].alpha, T = list[k].T, G = list[k].G;
                    double dLda = dA_out * Tf / (1.0 - al);
                    for (int ch = 0; ch < 3; ch++) {
                        g_color[3 * (int64_t)it + ch] += al * T * dC[ch];
                        dLda += dC[ch] * (col[ch] * T - (S[ch] + Tf * bg[ch]) / (1.0 - al));
                    }
                    for (int ch = 0; ch < 3; ch++) S[ch] += col[ch] * al * T;
                    if (list[k].clamped) continue;
                    double o = s[5];
                    double dx = s[0] - (px + 0.5), dy = s[1] - (py + 0.5);
                    double dLdpow = dLda * o * G;
                    double *g = g_splat + 6 * (int64_t)it;
                    g[0] += dLdpow * (-(s[2] * dx + s[3] * dy));
                    g[1] += dLdpow * (-(s[4] * dy + s[3] * dx));
                    g[2] += dLdpow * (-0.5 * dx * dx);
                    g[3] += dLdpow * (-dx * dy);
                    g[4] += dLdpow * (-0.5 * dy * dy);
                    g[5] += dLda * G;
                }
            }
    free(list);
}

/* Brute force: every item of the view whose rectangle holds the pixel's tile,
 * sorted by (depth, item) per pixel, composited with the same rules. */
typedef struct { double depth; int32_t item; } dep_rec;
static int cmp_dep(const void *pa, const void *pb)
{
    const dep_rec *a = pa, *b = pb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->item < b->item ? -1 : (a->item > b->item);
}

void orc_render_brute(int n_views, int W, int H, int tile_w, int tile_h, int64_t n_items, const int32_t *view_of,
                      const int32_t *rect, const double *depth, const double *splat, const double *color,
                      const double *bg, double *img, double *T_final)
{
    int64_t HW = (int64_t)H * W;
    dep_rec *sel = (dep_rec *)malloc((size_t)(n_items > 0 ? n_items : 1) * sizeof(dep_rec));
    for (int v = 0; v < n_views; v++)
        for (int py = 0; py < H; py++)
            for (int px = 0; px < W; px++) {
                int tx = px / tile_w, ty = py / tile_h;
                int64_t m = 0;
                for (int64_t it = 0; it < n_items; it++) {
                    const int32_t *rc = rect + 4 * it;
                    if (view_of[it] == v && tx >= rc[0] && tx < rc[2] && ty >= rc[1] && ty < rc[3]) {
                        sel[m].depth = depth[it];
                        sel[m].item = (int32_t)it;
                        m++;
                    }
                }
                qsort(sel, (size_t)m, sizeof(dep_rec), cmp_dep);
                double T = 1.0, C[3] = {0, 0, 0};
                for (int64_t k = 0; k < m; k++) {
                    int32_t it = sel[k].item;
                    const double *s = splat + 6 * (int64_t)it;
                    double dx = s[0] - (px + 0.5), dy = s[1] - (py + 0.5);
                    double power = -0.5 * (s[2] * dx * dx + s[4] * dy * dy) - s[3] * dx * dy;
                    if (power > 0) continue;
                    double alpha = fmin(ALPHA_MAX, s[5] * exp(power));
                    if (alpha < ALPHA_MIN) continue;
                    double testT = T * (1.0 - alpha);
                    if (testT < T_MIN) break;
                    for (int ch = 0; ch < 3; ch++) C[ch] += color[3 * (int64_t)it + ch] * alpha * T;
                    T = testT;
                }
                int64_t pix = (int64_t)py * W + px;
                for (int ch = 0; ch < 3; ch++) img[((int64_t)v * 3 + ch) * HW + pix] = C[ch] + T * bg[ch];
                T_final[v * HW + pix] = T;
            }
    free(sel);
}

/* ------------------------------------------------------ projection backward */

/*
 * Chain rule from (du, dv, dA, dB, dC, dopacity) of item it to the 14
 * parameters of its Gaussian (out[14], overwritten).  Steps, reversing
 * project_state:
 *   conic (A, B, C) = (c, -b, a) / det of the dilated 2D covariance [[a, b], [b, c]];
 *   [[a, b], [b, c]] - 0.3 I = T Sigma T^T with T = J W (rows T0, T1);
 *   J = [[fx/z, 0, -fx xc/z], [0, fy/z, -fy yc/z]] with xc = clamp(x/z)
 *       (no derivative through a clamped coordinate);
 *   mean2D = (fx x/z + cx, fy y/z + cy);  t = W mu + t_cam;
 *   Sigma = M M^T, M = R(q/|q|) diag(exp(log_scale));  opacity = sigmoid(logit).
 */
void orc_project_bwd(const double *P, int64_t n, int64_t gi, const double *cam, const double *g6, double *out)
{
    for (int k = 0; k < 14; k++) out[k] = 0.0;
    proj_state st;
    project_state(P, n, gi, cam, &st);
    out[10] = g6[5] * st.opac * (1.0 - st.opac);
    if (st.culled) return;
    const double *Wm = cam + CAM_R;
    double fx = cam[CAM_FX], fy = cam[CAM_FY];
    double a = st.a, b = st.b, c = st.c, D = st.det, D2 = D * D;
    double dA = g6[2], dB = g6[3], dC = g6[4];
    double dLa = dA * (-c * c / D2) + dB * (b * c / D2) + dC * (-b * b / D2);
    double dLb = dA * (2 * b * c / D2) + dB * (-(a * c + b * b) / D2) + dC * (2 * a * b / D2);
    double dLc = dA * (-b * b / D2) + dB * (a * b / D2) + dC * (-a * a / D2);
    /* dL/dSigma (all nine entries treated as independent) */
    double GS[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            GS[i][j] = dLa * st.T0[i] * st.T0[j] + dLb * st.T0[i] * st.T1[j] + dLc * st.T1[i] * st.T1[j];
    double ST0[3], ST1[3];
    for (int i = 0; i < 3; i++) {
        ST0[i] = ST1[i] = 0;
        for (int j = 0; j < 3; j++) { ST0[i] += st.Sig[i][j] * st.T0[j]; ST1[i] += st.Sig[i][j] * st.T1[j]; }
    }
    double dT0[3], dT1[3];
    for (int i = 0; i < 3; i++) {
        dT0[i] = 2 * dLa * ST0[i] + dLb * ST1[i];
        dT1[i] = dLb * ST0[i] + 2 * dLc * ST1[i];
    }
    double dJ00 = 0, dJ02 = 0, dJ11 = 0, dJ12 = 0;
    for (int k = 0; k < 3; k++) {
        dJ00 += dT0[k] * Wm[k];
        dJ02 += dT0[k] * Wm[6 + k];
        dJ11 += dT1[k] * Wm[3 + k];
        dJ12 += dT1[k] * Wm[6 + k];
    }
    double tx = st.t[0], ty = st.t[1], tz = st.t[2];
    double dxc_dtx = st.clampx ? 0.0 : 1.0 / tz, dxc_dtz = st.clampx ? 0.0 : -tx / (tz * tz);
    double dyc_dty = st.clampy ? 0.0 : 1.0 / tz, dyc_dtz = st.clampy ? 0.0 : -ty / (tz * tz);
    double dt[3];
    dt[0] = g6[0] * fx / tz + dJ02 * (-fx / tz) * dxc_dtx;
    dt[1] = g6[1] * fy / tz + dJ12 * (-fy / tz) * dyc_dty;
    dt[2] = g6[0] * (-fx * tx / (tz * tz)) + g6[1] * (-fy * ty / (tz * tz))
          + dJ00 * (-fx / (tz * tz)) + dJ11 * (-fy / (tz * tz))
          + dJ02 * (fx * st.xzc / (tz * tz) - fx / tz * dxc_dtz)
          + dJ12 * (fy * st.yzc / (tz * tz) - fy / tz * dyc_dtz);
    for (int k = 0; k < 3; k++) out[k] = Wm[k] * dt[0] + Wm[3 + k] * dt[1] + Wm[6 + k] * dt[2];
    /* Sigma = M M^T, M = R diag(s) */
    double dM[3][3];
    for (int i = 0; i < 3; i++)
        for (int k = 0; k < 3; k++) {
            double acc = 0;
            for (int j = 0; j < 3; j++) acc += (GS[i][j] + GS[j][i]) * st.R[j][k] * st.s[k];
            dM[i][k] = acc;
        }
    double dR[3][3];
    for (int k = 0; k < 3; k++) {
        double ds = 0;
        for (int i = 0; i < 3; i++) { ds += dM[i][k] * st.R[i][k]; dR[i][k] = dM[i][k] * st.s[k]; }
        out[3 + k] = ds * st.s[k];
    }
    double w = st.qn[0], x = st.qn[1], y = st.qn[2], z = st.qn[3];
    double dq[4];
    dq[0] = 2 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    dq[1] = 2 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2 * x * dR[1][1] - w * dR[1][2]
                 + z * dR[2][0] + w * dR[2][1] - 2 * x * dR[2][2]);
    dq[2] = 2 * (-2 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2]
                 - w * dR[2][0] + z * dR[2][1] - 2 * y * dR[2][2]);
    dq[3] = 2 * (-2 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2 * z * dR[1][1]
                 + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    double dot = dq[0] * st.qn[0] + dq[1] * st.qn[1] + dq[2] * st.qn[2] + dq[3] * st.qn[3];
    for (int k = 0; k < 4; k++) out[6 + k] = (dq[k] - st.qn[k] * dot) / st.qnorm;
}

/* Batched projection backward: out[n_items][14]. */
void orc_project_bwd_items(int64_t n_items, const int64_t *gidx, const double *P, int64_t n, const double *cam,
                           const double *g_splat, double *out)
{
    for (int64_t it = 0; it < n_items; it++)
        orc_project_bwd(P, n, gidx[it], cam, g_splat + 6 * it, out + 14 * it);
}
