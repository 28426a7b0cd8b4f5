/*
 * pbr_oracle.c -- plain, slow, FP64 reference of the point-splat renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant with the CUDA path.
 *
 * What it computes (Zhang et al., "Differentiable Point-Based Radiance Fields
 * for Efficient View Synthesis", SIGGRAPH Asia 2022):
 *   - Sec. 3.1, Eq. 1 (projection): p = (M (R P + t))v, (x,y,z)v = (x/z, y/z).
 *   - Sec. 3.1, Eq. 3 (view direction): v = (R P + t) / |R P + t|.
 *   - Sec. 3.1, Eq. 4 (colour): c = sum_{l<=lmax} sum_m h_lm Y_lm(v).
 *   - Sec. 3.2, Eq. 5 (radial kernel): alpha = amplitude * exp(-|p-u|^2/(2 s^2)).
 *   - Sec. 3.2, Eqs. 6-7 (front-to-back blending after a z sort):
 *     I(u) = sum_i alpha_i prod_{k<i}(1-alpha_k) c_i.
 *   - Sec. 3.2, last paragraph: only points within a maximum distance of u.
 *   - Sec. 3.3: the model is trained end to end by gradient descent, so the
 *     adjoint of the above w.r.t. positions and SH coefficients is written
 *     out here by hand (chain rule, FP64), for checking against central
 *     finite differences.
 *
 * Form: for every pixel, every point is tested; the candidates are fully
 * sorted by depth; blending is done in double precision.  No tiles and no
 * shortcut other than the stated transmittance / count stop rule.
 *
 * Discrete decisions (culling, the cutoff test, the pixel bounding box, the
 * tile rectangle and the depth key) are taken in IEEE binary32 with
 * round-to-nearest and no contraction, in the operation order written below,
 * because the renderer under test works in fp32 and both sides must take
 * those integer decisions in the same precision.  This file must therefore be
 * compiled with -ffp-contract=off and without fast-math.
 *
 * Tile lists: a point is listed in a tile of its clamped pixel box when the
 * box spans more than 32 tiles, or else when the fp32 distance from the
 * splat centre to the tile's rectangle of pixel centres (clipped to the
 * image) is within the cutoff radius.
 *
 * Readings of points the paper leaves open (each one also listed in the
 * design notes of the repository):
 *   - the kernel normalisation 1/sqrt(2 pi r^2) is folded into a per-point
 *     amplitude o_i and alpha is clamped to alpha_max (<1);
 *   - the kernel acts in image space with s in pixels: s = fx * r / z
 *     (radius_mode 0) or s = r * min(W,H) / 2 (radius_mode 1);
 *   - the cutoff distance is cutoff_k * s;
 *   - real orthonormal SH, no Condon-Shortley phase, index l*l + l + m;
 *   - linear colour, no activation;
 *   - equal depths are ordered by point index; pixel centres at +0.5;
 *   - compositing stops after the point that brings T below t_eps, or after
 *     max_per_pixel composited points (0 = no count limit).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LMAX 8
#define ORC_KMAX ((ORC_LMAX + 1) * (ORC_LMAX + 1))

/* ------------------------------------------------------------------------ */
/* Public structures (mirrored by ctypes in oracle.py).                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    double fx, fy, cx, cy;
    double R[9]; /* row-major world->camera rotation */
    double t[3];
    int32_t width, height;
} orc_camera;

typedef struct {
    int32_t radius_mode;   /* 0: s = fx*r/z ; 1: s = r*min(W,H)/2 */
    int32_t dir_frame;     /* 0: camera-frame direction (Eq. 3) ; 1: world frame */
    double cutoff_k;
    double alpha_max;
    double t_eps;
    int32_t max_per_pixel; /* 0 = unlimited */
    double bg[3];
    double z_near;
    int32_t tile_w, tile_h;
    int32_t screen_fp32;   /* 1: blend with the fp32 screen position and s;
                              0: every continuous quantity in double */
} orc_opts;

/* Per (view, point) projection record, fp32 decisions + double geometry. */
typedef struct {
    int32_t visible;
    float z32, px32, py32, s32, rc32, rc2_32;
    int32_t px_lo, px_hi, py_lo, py_hi; /* clamped inclusive pixel box */
    int32_t tx_lo, tx_hi, ty_lo, ty_hi; /* inclusive tile box */
    int64_t ntiles;                     /* listed tiles (see block_mask) */
    double X[3];      /* camera-space position, double */
    double px, py, s; /* double screen position and kernel width */
    double dir[3];    /* unit view direction in the SH frame */
    double rgb[3];
} orc_rec;

/* ------------------------------------------------------------------------ */
/* Spherical harmonics from the closed form.                                */
/*                                                                          */
/* Y_l0  = K_l0 P_l(z)                                                      */
/* Y_lm  = sqrt2 K_lm Re((x+iy)^m)  d^m P_l/dz^m (z)      m > 0            */
/* Y_l-m = sqrt2 K_lm Im((x+iy)^m)  d^m P_l/dz^m (z)      m > 0            */
/* K_lm  = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!)                                */
/* On the unit sphere sin^m(theta) cos(m phi) = Re((x+iy)^m), so these are  */
/* the usual real SH (no Condon-Shortley phase) written as polynomials; the */
/* Legendre polynomials come from Bonnet's recurrence.                      */
/* ------------------------------------------------------------------------ */
static double g_leg[ORC_LMAX + 2][ORC_LMAX + 2]; /* g_leg[l][j]: coeff of z^j in P_l */
static int g_leg_ready = 0;

static void legendre_init(void)
{
    if (g_leg_ready) return;
    memset(g_leg, 0, sizeof(g_leg));
    g_leg[0][0] = 1.0;
    g_leg[1][1] = 1.0;
    for (int l = 1; l < ORC_LMAX + 1; ++l) {
        /* (l+1) P_{l+1} = (2l+1) z P_l - l P_{l-1} */
        for (int j = 0; j <= l + 1; ++j) {
            double a = (j >= 1) ? (2.0 * l + 1.0) * g_leg[l][j - 1] : 0.0;
            double b = (double)l * g_leg[l - 1][j];
            g_leg[l + 1][j] = (a - b) / (double)(l + 1);
        }
    }
    g_leg_ready = 1;
}

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

/* d^k P_l / dz^k evaluated at z */
static double legendre_deriv(int l, int k, double z)
{
    double acc = 0.0;
    for (int j = l; j >= k; --j) {
        double c = g_leg[l][j];
        for (int q = 0; q < k; ++q) c *= (double)(j - q);
        acc = acc * z + c;
    }
    /* Horner over the powers j-k; above loop folds in descending order */
    return acc;
}

/* Re and Im of (x + i y)^m for m = 0..mmax */
static void complex_powers(double x, double y, int mmax, double *re, double *im)
{
    re[0] = 1.0;
    im[0] = 0.0;
    for (int m = 1; m <= mmax; ++m) {
        re[m] = re[m - 1] * x - im[m - 1] * y;
        im[m] = re[m - 1] * y + im[m - 1] * x;
    }
}

/* Y[k] for k = 0..(deg+1)^2-1 at the point (x,y,z); optional Cartesian
 * gradient of the polynomial form, dY[k*3 + {0,1,2}]. */
static void sh_eval(int deg, const double v[3], double *Y, double *dY)
{
    legendre_init();
    double re[ORC_LMAX + 1], im[ORC_LMAX + 1];
    complex_powers(v[0], v[1], deg, re, im);
    const double pi = 3.14159265358979323846;
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int k = l * l + l + m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * pi) * factorial(l - am) / factorial(l + am));
            double scale = (m == 0) ? K : sqrt(2.0) * K;
            double Q = legendre_deriv(l, am, v[2]);
            double A = (m >= 0) ? re[am] : im[am];
            Y[k] = scale * A * Q;
            if (dY) {
                double dAx, dAy;
                if (am == 0) {
                    dAx = 0.0;
                    dAy = 0.0;
                } else if (m > 0) { /* A = Re(w^m) */
                    dAx = am * re[am - 1];
                    dAy = -am * im[am - 1];
                } else {            /* A = Im(w^m) */
                    dAx = am * im[am - 1];
                    dAy = am * re[am - 1];
                }
                double dQ = (am + 1 <= l) ? legendre_deriv(l, am + 1, v[2]) : 0.0;
                dY[k * 3 + 0] = scale * dAx * Q;
                dY[k * 3 + 1] = scale * dAy * Q;
                dY[k * 3 + 2] = scale * A * dQ;
            }
        }
    }
}

int orc_sh_eval(int deg, const double *dir, double *Y, double *dY)
{
    if (deg < 0 || deg > ORC_LMAX) return -1;
    legendre_init();
    sh_eval(deg, dir, Y, dY);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Projection and the fp32 decisions (Eq. 1, Eq. 3, Eq. 4).                 */
/* ------------------------------------------------------------------------ */
static uint32_t f32_bits(float f)
{
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}
/* Cutoff test of Sec. 3.2 at the centre of pixel (x, y), in fp32
 * round-to-nearest in the order the renderer fixes: u = (x + 0.5, y + 0.5),
 * d2 = (ux - px)^2 + (uy - py)^2 <= rc^2. */
static int pixel_included(const orc_rec *r, int x, int y)
{
    const float dx = ((float)x + 0.5f) - r->px32;
    const float dy = ((float)y + 0.5f) - r->py32;
    return dx * dx + dy * dy <= r->rc2_32;
}

/* Binning of Sec. 3.2: tile (tx, ty) lists the point-view iff some pixel of
 * the tile inside the image passes the cutoff test.  Returns the mask of
 * the tile's 8 x 8 pixel blocks holding such a pixel (bit by * (tile_w / 8)
 * + bx, blocks numbered row-major inside the tile), found by testing every
 * pixel of the tile; 0 = not listed. */
static uint32_t block_mask(const orc_rec *r, const orc_camera *cam, const orc_opts *o, int tx,
                           int ty)
{
    uint32_t m = 0;
    const int bpr = o->tile_w / 8;
    for (int y = ty * o->tile_h; y < (ty + 1) * o->tile_h && y < cam->height; ++y)
        for (int x = tx * o->tile_w; x < (tx + 1) * o->tile_w && x < cam->width; ++x)
            if (pixel_included(r, x, y))
                m |= 1u << (((y - ty * o->tile_h) / 8) * bpr + (x - tx * o->tile_w) / 8);
    return m;
}



static void project_point(const double *P, double radius, const orc_camera *cam,
                          const orc_opts *o, int deg, const double *sh, orc_rec *r)
{
    memset(r, 0, sizeof *r);
    /* fp32 decision path: X = ((R0 P0 + R1 P1) + R2 P2) + t, rounded per op */
    float Pf[3] = {(float)P[0], (float)P[1], (float)P[2]};
    float Rf[9], tf[3];
    for (int i = 0; i < 9; ++i) Rf[i] = (float)cam->R[i];
    for (int i = 0; i < 3; ++i) tf[i] = (float)cam->t[i];
    float Xf[3];
    for (int a = 0; a < 3; ++a) {
        float s = Rf[3 * a + 0] * Pf[0];
        s = s + Rf[3 * a + 1] * Pf[1];
        s = s + Rf[3 * a + 2] * Pf[2];
        Xf[a] = s + tf[a];
    }
    float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;
    float rf = (float)radius;
    float z = Xf[2];
    r->z32 = z;
    if (!(z > (float)o->z_near)) return; /* behind the near plane, or NaN */
    float px = fx * (Xf[0] / z) + cx;
    float py = fy * (Xf[1] / z) + cy;
    float s;
    if (o->radius_mode == 0) {
        s = (fx * rf) / z;
    } else {
        int mn = cam->width < cam->height ? cam->width : cam->height;
        s = (rf * (float)mn) * 0.5f;
    }
    float rc = (float)o->cutoff_k * s;
    float rc2 = rc * rc;
    r->px32 = px;
    r->py32 = py;
    r->s32 = s;
    r->rc32 = rc;
    r->rc2_32 = rc2;
    if (!(s > 0.0f)) return;
    float xlo = floorf(px - rc) - 1.0f;
    float xhi = ceilf(px + rc);
    float ylo = floorf(py - rc) - 1.0f;
    float yhi = ceilf(py + rc);
    float W1 = (float)(cam->width - 1), H1 = (float)(cam->height - 1);
    if (!(xhi >= 0.0f && xlo <= W1 && yhi >= 0.0f && ylo <= H1)) return;
    /* clamp in float before converting (values may be huge) */
    xlo = xlo < 0.0f ? 0.0f : xlo;
    ylo = ylo < 0.0f ? 0.0f : ylo;
    xhi = xhi > W1 ? W1 : xhi;
    yhi = yhi > H1 ? H1 : yhi;
    r->px_lo = (int)xlo;
    r->px_hi = (int)xhi;
    r->py_lo = (int)ylo;
    r->py_hi = (int)yhi;
    r->tx_lo = r->px_lo / o->tile_w;
    r->tx_hi = r->px_hi / o->tile_w;
    r->ty_lo = r->py_lo / o->tile_h;
    r->ty_hi = r->py_hi / o->tile_h;
    {
        int64_t nt = 0;
        for (int ty = r->ty_lo; ty <= r->ty_hi; ++ty)
            for (int tx = r->tx_lo; tx <= r->tx_hi; ++tx)
                nt += block_mask(r, cam, o, tx, ty) != 0;
        r->ntiles = nt;
    }
    if (r->ntiles == 0) return; /* no pixel centre within reach */
    r->visible = 1;

    /* double geometry (Eq. 1) */
    for (int a = 0; a < 3; ++a)
        r->X[a] = cam->R[3 * a] * P[0] + cam->R[3 * a + 1] * P[1] + cam->R[3 * a + 2] * P[2] + cam->t[a];
    r->px = cam->fx * r->X[0] / r->X[2] + cam->cx;
    r->py = cam->fy * r->X[1] / r->X[2] + cam->cy;
    if (o->radius_mode == 0) {
        r->s = cam->fx * radius / r->X[2];
    } else {
        int mn = cam->width < cam->height ? cam->width : cam->height;
        r->s = radius * (double)mn * 0.5;
    }
    /* view direction (Eq. 3) and colour (Eq. 4) */
    double nrm = sqrt(r->X[0] * r->X[0] + r->X[1] * r->X[1] + r->X[2] * r->X[2]);
    double vc[3] = {r->X[0] / nrm, r->X[1] / nrm, r->X[2] / nrm};
    if (o->dir_frame == 0) {
        memcpy(r->dir, vc, sizeof vc);
    } else { /* world frame: R^T v */
        for (int a = 0; a < 3; ++a)
            r->dir[a] = cam->R[a] * vc[0] + cam->R[3 + a] * vc[1] + cam->R[6 + a] * vc[2];
    }
    double Y[ORC_KMAX];
    sh_eval(deg, r->dir, Y, NULL);
    int K = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double c = 0.0;
        for (int k = 0; k < K; ++k) c += sh[k * 3 + ch] * Y[k];
        r->rgb[ch] = c;
    }
}

static int check_opts(const orc_opts *o)
{
    if (o->tile_w <= 0 || o->tile_h <= 0) return -1;
    if (!(o->alpha_max < 1.0)) return -1;
    return 0;
}

/* Records for every (view, point) pair: out[v*n + i]. */
int orc_preprocess(int64_t n, const double *pos, const double *sh, const double *radius, int deg,
                   int ncam, const orc_camera *cams, const orc_opts *o, orc_rec *out)
{
    if (check_opts(o) || deg < 0 || deg > 3) return -1;
    legendre_init();
    int K = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static) collapse(2)
    for (int v = 0; v < ncam; ++v)
        for (int64_t i = 0; i < n; ++i)
            project_point(pos + 3 * i, radius[i], &cams[v], o, deg, sh + (size_t)i * K * 3,
                          &out[(size_t)v * n + i]);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Tile binning: the set {(tile, pv) : block_mask(pv, tile) != 0} ordered  */
/* by (global tile id, fp32 depth bits, pv).  Global tile ids number the    */
/* tiles of view 0 row-major, then view 1, and so on; pv = v*n + i.         */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t tile;
    uint32_t zbits;
    uint32_t pv;
    uint32_t mask;
} bin_entry;

static int cmp_bin(const void *a, const void *b)
{
    const bin_entry *x = (const bin_entry *)a, *y = (const bin_entry *)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->zbits != y->zbits) return x->zbits < y->zbits ? -1 : 1;
    if (x->pv != y->pv) return x->pv < y->pv ? -1 : 1;
    return 0;
}

/* Returns the number of (tile, pv) pairs.  When keys/vals are non-NULL they
 * receive the sorted lists (capacity `cap`) -- the global tile id and the
 * point-view id of every pair in (tile, depth bits, point-view) order --
 * and `masks` (nullable) the pair's 8 x 8 block mask (block_mask); ranges
 * (2 per tile) receive [start, end) per global tile when non-NULL. */
int64_t orc_bin(int64_t n, int ncam, const orc_camera *cams, const orc_opts *o, const orc_rec *recs,
                uint32_t *keys, uint32_t *vals, uint8_t *masks, int64_t cap, uint32_t *ranges)
{
    int64_t total = 0;
    for (int64_t q = 0; q < (int64_t)ncam * n; ++q)
        if (recs[q].visible) total += recs[q].ntiles;
    if (!keys) return total;
    if (total > cap) return -1;
    bin_entry *e = (bin_entry *)malloc(sizeof(bin_entry) * (size_t)(total > 0 ? total : 1));
    if (!e) return -2;
    int64_t w = 0;
    uint32_t tile_base = 0;
    for (int v = 0; v < ncam; ++v) {
        int tx = (cams[v].width + o->tile_w - 1) / o->tile_w;
        int ty = (cams[v].height + o->tile_h - 1) / o->tile_h;
        for (int64_t i = 0; i < n; ++i) {
            const orc_rec *r = &recs[(size_t)v * n + i];
            if (!r->visible) continue;
            for (int y = r->ty_lo; y <= r->ty_hi; ++y)
                for (int x = r->tx_lo; x <= r->tx_hi; ++x) {
                    const uint32_t m = block_mask(r, &cams[v], o, x, y);
                    if (!m) continue;
                    e[w].tile = tile_base + (uint32_t)(y * tx + x);
                    e[w].zbits = f32_bits(r->z32);
                    e[w].pv = (uint32_t)((int64_t)v * n + i);
                    e[w].mask = m;
                    ++w;
                }
        }
        tile_base += (uint32_t)(tx * ty);
    }
    qsort(e, (size_t)total, sizeof(bin_entry), cmp_bin);
    for (int64_t q = 0; q < total; ++q) {
        keys[q] = e[q].tile;
        vals[q] = e[q].pv;
        if (masks) masks[q] = (uint8_t)e[q].mask;
    }
    if (ranges) {
        memset(ranges, 0, sizeof(uint32_t) * 2 * tile_base);
        for (int64_t q = 0; q < total; ++q) {
            uint32_t t = e[q].tile;
            if (q == 0 || e[q - 1].tile != t) ranges[2 * t] = (uint32_t)q;
            ranges[2 * t + 1] = (uint32_t)(q + 1);
        }
    }
    free(e);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Rendering (Eqs. 5-7) and its adjoint, per pixel, brute force.            */
/* ------------------------------------------------------------------------ */
typedef struct {
    uint32_t zbits;
    uint32_t idx;
} cand;

static int cmp_cand(const void *a, const void *b)
{
    const cand *x = (const cand *)a, *y = (const cand *)b;
    if (x->zbits != y->zbits) return x->zbits < y->zbits ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

typedef struct {
    double alpha, T, G, d2, dx, dy, s, amp;
    int clamped;
    uint32_t idx;
} blend_item;

/* Builds the ordered candidate list of pixel (x, y) in view v and blends it.
 * Writes rgb/T/count, and (when items != NULL) the per-point blend terms. */
static int blend_pixel(int64_t n, const orc_rec *vrec, const double *opacity, const orc_opts *o,
                       int x, int y, cand *buf, blend_item *items, double rgb[3], double *T_out)
{
    float ux = (float)x + 0.5f, uy = (float)y + 0.5f;
    int nc = 0;
    for (int64_t i = 0; i < n; ++i) {
        const orc_rec *r = &vrec[i];
        if (!r->visible) continue;
        float dx = ux - r->px32;
        float dy = uy - r->py32;
        float d2 = dx * dx + dy * dy;
        if (d2 <= r->rc2_32) {
            buf[nc].zbits = f32_bits(r->z32);
            buf[nc].idx = (uint32_t)i;
            ++nc;
        }
    }
    qsort(buf, (size_t)nc, sizeof(cand), cmp_cand);
    double C[3] = {0, 0, 0}, T = 1.0;
    int cnt = 0;
    for (int q = 0; q < nc; ++q) {
        const orc_rec *r = &vrec[buf[q].idx];
        double px = o->screen_fp32 ? (double)r->px32 : r->px;
        double py = o->screen_fp32 ? (double)r->py32 : r->py;
        double s = o->screen_fp32 ? (double)r->s32 : r->s;
        double dx = ((double)x + 0.5) - px, dy = ((double)y + 0.5) - py;
        double d2 = dx * dx + dy * dy;
        double G = exp(-d2 / (2.0 * s * s));
        double amp = opacity[buf[q].idx];
        double a = amp * G;
        int clamped = 0;
        if (a > o->alpha_max) {
            a = o->alpha_max;
            clamped = 1;
        }
        if (items) {
            blend_item *it = &items[cnt];
            it->alpha = a;
            it->T = T;
            it->G = G;
            it->d2 = d2;
            it->dx = dx;
            it->dy = dy;
            it->s = s;
            it->amp = amp;
            it->clamped = clamped;
            it->idx = buf[q].idx;
        }
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * a * r->rgb[ch];
        T *= (1.0 - a);
        ++cnt;
        if (T < o->t_eps) break;
        if (o->max_per_pixel > 0 && cnt >= o->max_per_pixel) break;
    }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch] + T * o->bg[ch];
    *T_out = T;
    return cnt;
}

/* pix: npix triples (view, x, y) or NULL for every pixel of every view (in
 * view order, row-major).  Outputs per selected pixel: rgb[3], T, count. */
int orc_render(int64_t n, const double *pos, const double *sh, const double *opacity,
               const double *radius, int deg, int ncam, const orc_camera *cams, const orc_opts *o,
               int64_t npix, const int32_t *pix, double *rgb, double *T_final, int32_t *count)
{
    if (check_opts(o) || deg < 0 || deg > 3) return -1;
    orc_rec *recs = (orc_rec *)malloc(sizeof(orc_rec) * (size_t)(ncam * n > 0 ? ncam * n : 1));
    if (!recs) return -2;
    orc_preprocess(n, pos, sh, radius, deg, ncam, cams, o, recs);
    int64_t total = npix;
    int64_t *vbase = (int64_t *)calloc((size_t)ncam + 1, sizeof(int64_t));
    for (int v = 0; v < ncam; ++v) vbase[v + 1] = vbase[v] + (int64_t)cams[v].width * cams[v].height;
    if (!pix) total = vbase[ncam];
    int err = 0;
#pragma omp parallel
    {
        cand *buf = (cand *)malloc(sizeof(cand) * (size_t)(n > 0 ? n : 1));
        if (!buf) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            if (!buf) continue;
            int v, x, y;
            if (pix) {
                v = pix[3 * q];
                x = pix[3 * q + 1];
                y = pix[3 * q + 2];
            } else {
                v = 0;
                while (q >= vbase[v + 1]) ++v;
                int64_t local = q - vbase[v];
                x = (int)(local % cams[v].width);
                y = (int)(local / cams[v].width);
            }
            double T;
            int c = blend_pixel(n, recs + (size_t)v * n, opacity, o, x, y, buf, NULL, rgb + 3 * q, &T);
            if (T_final) T_final[q] = T;
            if (count) count[q] = c;
        }
        free(buf);
    }
    free(vbase);
    free(recs);
    return err;
}

static void atomic_add(double *p, double v)
{
#pragma omp atomic
    *p += v;
}

/* Adjoint of orc_render for the loss L = sum_pixels g . I over the selected
 * pixels.  Outputs (overwritten): dpos[n,3], dsh[n,K,3], dopacity[n] and,
 * when non-NULL, the screen-space adjoint per (view, point):
 * g2d[(v*n+i)*7 + {dpx, dpy, ds, damp, dr, dg, db}]. */
int orc_backward(int64_t n, const double *pos, const double *sh, const double *opacity,
                 const double *radius, int deg, int ncam, const orc_camera *cams, const orc_opts *o,
                 int64_t npix, const int32_t *pix, const double *grad_rgb, double *dpos, double *dsh,
                 double *dopacity, double *g2d_out)
{
    if (check_opts(o) || deg < 0 || deg > 3) return -1;
    int K = (deg + 1) * (deg + 1);
    size_t npv = (size_t)ncam * (size_t)n;
    orc_rec *recs = (orc_rec *)malloc(sizeof(orc_rec) * (npv > 0 ? npv : 1));
    double *g2d = (double *)calloc((npv > 0 ? npv : 1) * 7, sizeof(double));
    if (!recs || !g2d) {
        free(recs);
        free(g2d);
        return -2;
    }
    orc_preprocess(n, pos, sh, radius, deg, ncam, cams, o, recs);
    int64_t *vbase = (int64_t *)calloc((size_t)ncam + 1, sizeof(int64_t));
    for (int v = 0; v < ncam; ++v) vbase[v + 1] = vbase[v] + (int64_t)cams[v].width * cams[v].height;
    int64_t total = pix ? npix : vbase[ncam];
#pragma omp parallel
    {
        cand *buf = (cand *)malloc(sizeof(cand) * (size_t)(n > 0 ? n : 1));
        blend_item *items = (blend_item *)malloc(sizeof(blend_item) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < total; ++q) {
            int v, x, y;
            if (pix) {
                v = pix[3 * q];
                x = pix[3 * q + 1];
                y = pix[3 * q + 2];
            } else {
                v = 0;
                while (q >= vbase[v + 1]) ++v;
                int64_t local = q - vbase[v];
                x = (int)(local % cams[v].width);
                y = (int)(local / cams[v].width);
            }
            const orc_rec *vrec = recs + (size_t)v * n;
            double rgb[3], T;
            int cnt = blend_pixel(n, vrec, opacity, o, x, y, buf, items, rgb, &T);
            const double *g = grad_rgb + 3 * q;
            /* S: sum over later points of alpha_k T_k (c_k . g) plus the
             * background term T_final (bg . g). */
            double S = T * (o->bg[0] * g[0] + o->bg[1] * g[1] + o->bg[2] * g[2]);
            for (int i = cnt - 1; i >= 0; --i) {
                const blend_item *it = &items[i];
                const orc_rec *r = &vrec[it->idx];
                double *gp = g2d + ((size_t)v * n + it->idx) * 7;
                double cg = r->rgb[0] * g[0] + r->rgb[1] * g[1] + r->rgb[2] * g[2];
                double w = it->alpha * it->T;
                for (int ch = 0; ch < 3; ++ch) atomic_add(&gp[4 + ch], w * g[ch]);
                double dalpha = it->T * cg - S / (1.0 - it->alpha);
                S += w * cg;
                if (!it->clamped) {
                    double s2 = it->s * it->s;
                    double aG = it->amp * it->G;
                    atomic_add(&gp[3], dalpha * it->G);
                    atomic_add(&gp[0], dalpha * aG * it->dx / s2);
                    atomic_add(&gp[1], dalpha * aG * it->dy / s2);
                    atomic_add(&gp[2], dalpha * aG * it->d2 / (s2 * it->s));
                }
            }
        }
        free(buf);
        free(items);
    }
    free(vbase);

    /* chain the screen-space adjoint back to the point parameters */
    memset(dpos, 0, sizeof(double) * 3 * (size_t)n);
    memset(dsh, 0, sizeof(double) * 3 * (size_t)K * (size_t)n);
    if (dopacity) memset(dopacity, 0, sizeof(double) * (size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int v = 0; v < ncam; ++v) {
            const orc_rec *r = &recs[(size_t)v * n + i];
            const double *gp = g2d + ((size_t)v * n + i) * 7;
            if (!r->visible) continue;
            const orc_camera *cam = &cams[v];
            double X0 = r->X[0], X1 = r->X[1], z = r->X[2];
            double dX[3] = {0, 0, 0};
            /* p = (fx X0/z + cx, fy X1/z + cy) */
            dX[0] += gp[0] * cam->fx / z;
            dX[2] -= gp[0] * cam->fx * X0 / (z * z);
            dX[1] += gp[1] * cam->fy / z;
            dX[2] -= gp[1] * cam->fy * X1 / (z * z);
            /* s = fx r / z */
            if (o->radius_mode == 0) dX[2] -= gp[2] * r->s / z;
            if (dopacity) dopacity[i] += gp[3];
            /* colour: c_ch = sum_k h[k][ch] Y_k(dir) */
            double Y[ORC_KMAX], dY[ORC_KMAX * 3];
            sh_eval(deg, r->dir, Y, dY);
            double ddir[3] = {0, 0, 0};
            for (int k = 0; k < K; ++k) {
                const double *h = sh + ((size_t)i * K + k) * 3;
                double *dh = dsh + ((size_t)i * K + k) * 3;
                double hg = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    dh[ch] += Y[k] * gp[4 + ch];
                    hg += h[ch] * gp[4 + ch];
                }
                for (int a = 0; a < 3; ++a) ddir[a] += hg * dY[k * 3 + a];
            }
            double dvc[3];
            if (o->dir_frame == 0) {
                memcpy(dvc, ddir, sizeof dvc);
            } else { /* dir = R^T vc  =>  d vc = R d dir */
                for (int a = 0; a < 3; ++a)
                    dvc[a] = cam->R[3 * a] * ddir[0] + cam->R[3 * a + 1] * ddir[1] + cam->R[3 * a + 2] * ddir[2];
            }
            double nrm = sqrt(X0 * X0 + X1 * X1 + z * z);
            double vc[3] = {X0 / nrm, X1 / nrm, z / nrm};
            double vd = vc[0] * dvc[0] + vc[1] * dvc[1] + vc[2] * dvc[2];
            for (int a = 0; a < 3; ++a) dX[a] += (dvc[a] - vc[a] * vd) / nrm;
            /* X = R P + t  =>  dP = R^T dX */
            for (int a = 0; a < 3; ++a)
                dpos[3 * i + a] += cam->R[a] * dX[0] + cam->R[3 + a] * dX[1] + cam->R[6 + a] * dX[2];
        }
    }
    if (g2d_out) memcpy(g2d_out, g2d, sizeof(double) * 7 * npv);
    free(g2d);
    free(recs);
    return 0;
}

/* Threads of the following OpenMP regions (timing on one core); n <= 0
 * leaves the default. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
    int nt = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        nt = omp_get_num_threads();
    }
#endif
    return nt;
}
