/*
 * splotch_oracle.c -- plain, slow FP64 CPU oracle for the Splotch per-frame
 * render ("GPU Accelerated Particle Visualization with Splotch", Rivi et al.).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the bench's CPU-baseline
 * leg do.  It shares no code, header, table or constant with the CUDA library.
 *
 * Everything is computed in double precision from the FP32 values the caller
 * stores (FP16-stored attributes arrive already widened to float, exactly).
 * No blocking, fusion or reordering beyond what the definitions state.
 *
 * What the render computes (all references are to the paper):
 *   Sec. 2 "Processing and Rasterization": normalise the colour scalar,
 *     roto-translate and project coordinates and smoothing lengths with the
 *     camera, mark particles that lie entirely outside the scene inactive,
 *     and assign RGB colour through a look-up table (palette).
 *   Eq. 2: each particle carries rho_p(x) = rho0 * exp(-|x-x_p|^2 / sigma^2),
 *     clipped to zero beyond chi*sigma (rays farther away are unaffected).
 *   Eq. 1 with E_p = A_p (Sec. 2): the result does not depend on particle
 *     order, so the image is the plain sum of per-particle contributions
 *     (additive, optically thin form); mode 1 applies the E=A solution
 *     I = 1 - exp(-S) per channel to that sum.
 *   Eq. 7: the screen radius r(p) is proportional to chi*sigma_p, to the
 *     screen transform (here f / z_c) and to the image size (folded into f).
 *   Sec. 4 classification: particles with r <= r_sml (= 0.5) fall inside a
 *     single pixel; only their location is computed, and the oracle deposits
 *     their emission once into that pixel.
 *   Eq. 1 in general (E_p != A_p, mode 2): the particles a ray crosses are
 *     taken one after the other from the far end towards the observer, and
 *     across particle p the solution of Eq. 1 is
 *     I -> I exp(-tau_p) + (E_p / A_p)(1 - exp(-tau_p)), tau_p = A_p w_p
 *     (see orc_render_absorb for the reading of E_p, A_p and the order).
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - sigma_p = sigma_per_h * h (default 1: sigma_p is the smoothing length);
 *   - chi is a parameter (default 3);
 *   - camera: look-at basis fwd = unit(target-eye), right = unit(fwd x up),
 *     upc = right x fwd; f = (H/2)/tan(fov_y/2); x_s = W/2 + f x_c/z_c,
 *     y_s = H/2 - f y_c/z_c (y grows downwards); pixel (i,j) has its centre
 *     at (i+1/2, j+1/2); sigma_s = sigma_p f / (z_c S_box); r = chi sigma_s;
 *   - inactive iff z_c <= z_near or the box [x_s-r,x_s+r]x[y_s-r,y_s+r]
 *     misses [0,W)x[0,H); a particle with a non-finite input (x, y, z, h, I,
 *     s) or a negative smoothing length is inactive as well;
 *   - palette: s' = clamp((s-s_min)/(s_max-s_min),0,1), u = s'(n-1),
 *     k = min(floor(u), n-2), colour = pal[k] + (u-k)(pal[k+1]-pal[k]);
 *     emission e = brightness * I * colour (I plays rho0 of Eq. 2);
 *   - point rule weight 1 at pixel (floor(x_s), floor(y_s));
 *   - the clip is inclusive: d^2 <= r^2;
 *   - colour components (Sec. 2: a vector quantity such as a velocity gives
 *     the R, G and B components directly): when per-particle components are
 *     given they replace the palette, e = brightness * I * (c_R, c_G, c_B);
 *   - logarithms of processed quantities (Sec. 2): optionally I is replaced by
 *     log10(I), and s by log10(s) before its normalisation (s_min, s_max are
 *     then in log units); a non-positive value makes the particle inactive.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double eye[3], target[3], up[3];
    double fov_y_deg;
    int width, height;
    double z_near;
} orc_camera;

typedef struct {
    double chi;          /* clip factor of Eq. 2 */
    double sigma_per_h;  /* sigma_p = sigma_per_h * h */
    double s_box;        /* S_box of Eq. 7 */
    double r_sml;        /* point-rule radius of Sec. 4 (0.5) */
    double brightness;   /* global emission scale */
    double s_min, s_max; /* colour-scalar normalisation (Sec. 4 footnote) */
    int mode;            /* 0: additive sum, 1: E=A map 1-exp(-S), 2: absorption */
    double absorption;   /* mode 2: A_p = absorption * brightness * I_p (> 0) */
    int log_flags;       /* 1: log10 of I, 2: log10 of s (before normalisation) */
    const float *cr, *cg, *cb;   /* per-particle colour components, or NULL (palette) */
} orc_params;

/* Class labels written by orc_project. */
#define ORC_INACTIVE (-2)
#define ORC_POINT 0
#define ORC_SPLAT 1

typedef struct {
    double right[3], upc[3], fwd[3];
    double eye[3];
    double f, half_w, half_h;
    int w, h;
    double z_near;
} orc_view;

static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static int unit3(double *a) {
    double n = sqrt(dot3(a, a));
    if (!(n > 0.0)) return -1;
    a[0] /= n; a[1] /= n; a[2] /= n;
    return 0;
}

/* Camera set-up: the roto-translation and projection of Sec. 2. */
static int make_view(const orc_camera *c, orc_view *v) {
    double fwd[3], right[3], upc[3];
    if (c->width <= 0 || c->height <= 0) return -1;
    if (!(c->fov_y_deg > 0.0 && c->fov_y_deg < 180.0)) return -1;
    for (int k = 0; k < 3; ++k) fwd[k] = c->target[k] - c->eye[k];
    if (unit3(fwd)) return -1;
    cross3(fwd, c->up, right);
    if (unit3(right)) return -1;
    cross3(right, fwd, upc);
    for (int k = 0; k < 3; ++k) {
        v->right[k] = right[k]; v->upc[k] = upc[k]; v->fwd[k] = fwd[k];
        v->eye[k] = c->eye[k];
    }
    v->w = c->width; v->h = c->height;
    v->half_w = 0.5 * c->width; v->half_h = 0.5 * c->height;
    v->f = v->half_h / tan(0.5 * c->fov_y_deg * M_PI / 180.0);
    v->z_near = c->z_near;
    return 0;
}

/* One particle's projected record. */
typedef struct {
    double xs, ys, sigma, r;
    double e[3];
    double zc;           /* camera depth */
    double ib;           /* brightness * intensity */
    int cls;
} orc_rec;

/* Palette look-up of Sec. 2 (linear interpolation, clamped). */
static void palette(const float *pal, int npal, const orc_params *q, double s,
                    double *c) {
    double den = q->s_max - q->s_min;
    double sn = den != 0.0 ? (s - q->s_min) / den : 0.0;
    if (sn < 0.0) sn = 0.0;
    if (sn > 1.0) sn = 1.0;
    if (npal == 1) {
        for (int k = 0; k < 3; ++k) c[k] = pal[k];
        return;
    }
    double u = sn * (npal - 1);
    int k0 = (int)floor(u);
    if (k0 > npal - 2) k0 = npal - 2;
    double t = u - k0;
    for (int k = 0; k < 3; ++k) {
        double a = pal[3 * k0 + k], b = pal[3 * (k0 + 1) + k];
        c[k] = a + t * (b - a);
    }
}

/* Rasterisation of one particle (Sec. 2; Eq. 7; Sec. 4 classes). */
static void project_one(const orc_view *v, const orc_params *q, const float *pal,
                        int npal, long p, double x, double y, double z, double hh,
                        double inten, double sc, orc_rec *o) {
    double d[3] = {x - v->eye[0], y - v->eye[1], z - v->eye[2]};
    double xc = dot3(v->right, d), yc = dot3(v->upc, d), zc = dot3(v->fwd, d);
    double col[3];
    o->cls = ORC_INACTIVE;
    o->xs = o->ys = o->sigma = o->r = 0.0;
    o->e[0] = o->e[1] = o->e[2] = 0.0;
    o->zc = zc;
    o->ib = q->brightness * inten;
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(hh) || !isfinite(inten) ||
        !isfinite(sc) || hh < 0.0)
        return;
    if (q->cr && (!isfinite(q->cr[p]) || !isfinite(q->cg[p]) || !isfinite(q->cb[p]))) return;
    if (!(zc > v->z_near)) return;
    if (q->log_flags & 1) {
        if (!(inten > 0.0)) return;
        inten = log10(inten);
        o->ib = q->brightness * inten;
    }
    if (q->log_flags & 2) {
        if (!(sc > 0.0)) return;
        sc = log10(sc);
    }
    o->xs = v->half_w + v->f * xc / zc;
    o->ys = v->half_h - v->f * yc / zc;
    o->sigma = q->sigma_per_h * hh * v->f / (zc * q->s_box);
    o->r = q->chi * o->sigma;
    if (q->cr) {
        col[0] = q->cr[p]; col[1] = q->cg[p]; col[2] = q->cb[p];
    } else {
        palette(pal, npal, q, sc, col);
    }
    for (int k = 0; k < 3; ++k) o->e[k] = q->brightness * inten * col[k];
    if (o->xs + o->r < 0.0 || o->xs - o->r >= v->w || o->ys + o->r < 0.0 ||
        o->ys - o->r >= v->h)
        return;
    o->cls = (o->r <= q->r_sml) ? ORC_POINT : ORC_SPLAT;
}

/* Add one projected particle to an H*W*3 double image (Eq. 2, point rule). */
static void splat_one(const orc_view *v, const orc_rec *p, double *img) {
    if (p->cls == ORC_POINT) {
        double fx = floor(p->xs), fy = floor(p->ys);
        if (fx < 0.0 || fy < 0.0 || fx >= v->w || fy >= v->h) return;
        long o = 3L * ((long)fy * v->w + (long)fx);
        for (int k = 0; k < 3; ++k) img[o + k] += p->e[k];
        return;
    }
    if (p->cls != ORC_SPLAT) return;
    /* pixel centres i+1/2 with |i+1/2-x_s| <= r */
    double i0 = ceil(p->xs - p->r - 0.5), i1 = floor(p->xs + p->r - 0.5);
    double j0 = ceil(p->ys - p->r - 0.5), j1 = floor(p->ys + p->r - 0.5);
    if (i0 < 0.0) i0 = 0.0;
    if (j0 < 0.0) j0 = 0.0;
    if (i1 > v->w - 1) i1 = v->w - 1;
    if (j1 > v->h - 1) j1 = v->h - 1;
    double r2 = p->r * p->r, s2 = p->sigma * p->sigma;
    for (long j = (long)j0; j <= (long)j1; ++j) {
        double dy = (j + 0.5) - p->ys;
        for (long i = (long)i0; i <= (long)i1; ++i) {
            double dx = (i + 0.5) - p->xs;
            double d2 = dx * dx + dy * dy;
            if (d2 <= r2) {
                double w = exp(-d2 / s2);
                long o = 3L * (j * v->w + i);
                for (int k = 0; k < 3; ++k) img[o + k] += p->e[k] * w;
            }
        }
    }
}

static void finish(const orc_params *q, double *img, long npx) {
    if (q->mode == 1)
        for (long k = 0; k < 3 * npx; ++k) img[k] = -expm1(-img[k]);
}

/* ---------------------------------------------------------------------- */
/* exported entry points                                                   */
/* ---------------------------------------------------------------------- */

int orc_view_info(const orc_camera *cam, double *out /* [13] */) {
    orc_view v;
    if (make_view(cam, &v)) return -1;
    for (int k = 0; k < 3; ++k) {
        out[k] = v.right[k]; out[3 + k] = v.upc[k]; out[6 + k] = v.fwd[k];
    }
    out[9] = v.f; out[10] = v.half_w; out[11] = v.half_h; out[12] = v.z_near;
    return 0;
}

/* Per-particle rasterisation records (Sec. 2, Eq. 7, Sec. 4 labels). */
int orc_project(long n, const float *x, const float *y, const float *z,
                const float *h, const float *inten, const float *s,
                const float *pal, int npal, const orc_camera *cam,
                const orc_params *q, double *xs, double *ys, double *sigma,
                double *r, double *e /* n*3 */, int *cls) {
    orc_view v;
    if (npal < 1 || make_view(cam, &v)) return -1;
    for (long p = 0; p < n; ++p) {
        orc_rec o;
        project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &o);
        xs[p] = o.xs; ys[p] = o.ys; sigma[p] = o.sigma; r[p] = o.r;
        for (int k = 0; k < 3; ++k) e[3 * p + k] = o.e[k];
        cls[p] = o.cls;
    }
    return 0;
}

/* Full image, particle-major.  nthreads > 1 gives each OpenMP thread its own
 * partial image over a contiguous chunk of particles and sums the partial
 * images afterwards (the MPI/OpenMP scheme of Sec. 2). */
static int render_absorb(long n, const float *x, const float *y, const float *z,
                         const float *h, const float *inten, const float *s,
                         const float *pal, int npal, const orc_view *v,
                         const orc_params *q, double *img, int pixel_major);

int orc_render(long n, const float *x, const float *y, const float *z,
               const float *h, const float *inten, const float *s,
               const float *pal, int npal, const orc_camera *cam,
               const orc_params *q, double *img, int nthreads) {
    orc_view v;
    if (npal < 1 || make_view(cam, &v)) return -1;
    if (q->mode == 2) return render_absorb(n, x, y, z, h, inten, s, pal, npal, &v, q, img, 0);
    long npx = (long)v.w * v.h;
    memset(img, 0, sizeof(double) * 3 * npx);
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
    if (nthreads > 1) {
        int nt = nthreads;
        double **part = (double **)calloc(nt, sizeof(double *));
        if (!part) return -2;
        for (int t = 0; t < nt; ++t) {
            part[t] = (double *)calloc(3 * npx, sizeof(double));
            if (!part[t]) {
                for (int u = 0; u < t; ++u) free(part[u]);
                free(part);
                return -2;
            }
        }
#pragma omp parallel num_threads(nt)
        {
            int t = omp_get_thread_num();
            int tn = omp_get_num_threads();
            long lo = n * t / tn, hi = n * (t + 1) / tn;
            for (long p = lo; p < hi; ++p) {
                orc_rec o;
                project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p],
                            s[p], &o);
                splat_one(&v, &o, part[t]);
            }
        }
        for (int t = 0; t < nt; ++t) {
            for (long k = 0; k < 3 * npx; ++k) img[k] += part[t][k];
            free(part[t]);
        }
        free(part);
        finish(q, img, npx);
        return 0;
    }
#endif
    for (long p = 0; p < n; ++p) {
        orc_rec o;
        project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &o);
        splat_one(&v, &o, img);
    }
    finish(q, img, npx);
    return 0;
}

/* Contribution of one projected particle to pixel (i, j), the pixel-major
 * formulation: no bounding box, only the rules themselves. */
static void pixel_term(const orc_rec *o, long i, long j, double *acc) {
    if (o->cls == ORC_POINT) {
        if (floor(o->xs) == (double)i && floor(o->ys) == (double)j)
            for (int k = 0; k < 3; ++k) acc[k] += o->e[k];
        return;
    }
    if (o->cls != ORC_SPLAT) return;
    double dx = (i + 0.5) - o->xs, dy = (j + 0.5) - o->ys;
    double d2 = dx * dx + dy * dy;
    if (d2 <= o->r * o->r) {
        double w = exp(-d2 / (o->sigma * o->sigma));
        for (int k = 0; k < 3; ++k) acc[k] += o->e[k] * w;
    }
}

/* Whole image, pixel-major brute force (every pixel against every particle).
 * For tiny scenes only: it pins the particle-major loop's bounding box. */
int orc_render_bruteforce(long n, const float *x, const float *y, const float *z,
                          const float *h, const float *inten, const float *s,
                          const float *pal, int npal, const orc_camera *cam,
                          const orc_params *q, double *img) {
    orc_view v;
    if (npal < 1 || make_view(cam, &v)) return -1;
    if (q->mode == 2) return render_absorb(n, x, y, z, h, inten, s, pal, npal, &v, q, img, 1);
    orc_rec *rec = (orc_rec *)malloc(sizeof(orc_rec) * (n > 0 ? n : 1));
    if (!rec) return -2;
    for (long p = 0; p < n; ++p)
        project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &rec[p]);
    for (long j = 0; j < v.h; ++j)
        for (long i = 0; i < v.w; ++i) {
            double acc[3] = {0.0, 0.0, 0.0};
            for (long p = 0; p < n; ++p) pixel_term(&rec[p], i, j, acc);
            for (int k = 0; k < 3; ++k) img[3 * (j * v.w + i) + k] = acc[k];
        }
    free(rec);
    finish(q, img, (long)v.w * v.h);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Eq. 1 with independent emission and absorption (mode 2)                 */
/* ---------------------------------------------------------------------- */
/*
 * Along the line of sight of a pixel the particles are crossed one after the
 * other.  Across particle p Eq. 1 has the solution
 *     I -> I exp(-tau_p) + (E_p / A_p) (1 - exp(-tau_p)),   tau_p = A_p w_p,
 * where w_p is the particle's clipped Gaussian weight of Eq. 2 at the pixel
 * (weight 1 at its pixel for a point particle), the line-integral factor being
 * folded into rho0 as in the additive form.  Readings (the paper gives no
 * formula for the coefficients):
 *   - emission E_p (RGB) is the additive form's emission, brightness * I_p *
 *     colour(s_p); absorption is grey, A_p = absorption * brightness * I_p
 *     (absorption > 0), so the source term E_p / A_p = colour(s_p) /
 *     absorption varies between particles and the order matters;
 *   - a particle with A_p <= 0 (I_p = 0, or a non-positive logarithm of I)
 *     emits nothing and absorbs nothing;
 *   - the ray starts with I = 0 behind the farthest particle and ends at the
 *     observer: particles are taken in decreasing camera depth z_c (FP64),
 *     equal depths in decreasing particle index (so that the ascending
 *     (z_c, index) order runs front to back);
 *   - with a constant palette equal to `absorption` in every channel E_p = A_p,
 *     and the result is the E=A map 1 - exp(-S) of mode 1.
 * pixel_major = 0: particle-major over the sorted particles, an H*W*3 image
 * updated in place; pixel_major = 1: every pixel sorts its own contributing
 * particles (the brute force of the tests).
 */
typedef struct {
    double key;
    long id;
} orc_depth;

static int cmp_back_to_front(const void *pa, const void *pb) {
    const orc_depth *a = (const orc_depth *)pa, *b = (const orc_depth *)pb;
    if (a->key != b->key) return a->key > b->key ? -1 : 1;
    if (a->id != b->id) return a->id > b->id ? -1 : 1;
    return 0;
}

/* Crossing of one particle with weight w by the ray of pixel value I[3]. */
static void cross_particle(const orc_rec *o, const orc_params *q, double w, double *I) {
    double A = q->absorption * o->ib;
    double tau = A * w;
    double keep = exp(-tau), gain = -expm1(-tau);
    for (int k = 0; k < 3; ++k) I[k] = I[k] * keep + (o->e[k] / A) * gain;
}

/* Weight of particle o at pixel (i, j): Eq. 2 clipped, or the point rule;
 * returns 0 where the particle does not reach the pixel. */
static double pixel_weight(const orc_rec *o, long i, long j) {
    if (o->cls == ORC_POINT)
        return floor(o->xs) == (double)i && floor(o->ys) == (double)j ? 1.0 : 0.0;
    if (o->cls != ORC_SPLAT) return 0.0;
    double dx = (i + 0.5) - o->xs, dy = (j + 0.5) - o->ys;
    double d2 = dx * dx + dy * dy;
    return d2 <= o->r * o->r ? exp(-d2 / (o->sigma * o->sigma)) : 0.0;
}

static int render_absorb(long n, const float *x, const float *y, const float *z,
                         const float *h, const float *inten, const float *s,
                         const float *pal, int npal, const orc_view *v,
                         const orc_params *q, double *img, int pixel_major) {
    if (!(q->absorption > 0.0)) return -1;
    long npx = (long)v->w * v->h;
    memset(img, 0, sizeof(double) * 3 * npx);
    orc_rec *rec = (orc_rec *)malloc(sizeof(orc_rec) * (n > 0 ? n : 1));
    orc_depth *ord = (orc_depth *)malloc(sizeof(orc_depth) * (n > 0 ? n : 1));
    if (!rec || !ord) {
        free(rec);
        free(ord);
        return -2;
    }
    long m = 0;
    for (long p = 0; p < n; ++p) {
        project_one(v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &rec[p]);
        if (rec[p].cls != ORC_INACTIVE && q->absorption * rec[p].ib > 0.0) {
            ord[m].key = rec[p].zc;
            ord[m].id = p;
            ++m;
        }
    }
    if (!pixel_major) {
        qsort(ord, (size_t)m, sizeof(orc_depth), cmp_back_to_front);
        for (long k = 0; k < m; ++k) {
            const orc_rec *o = &rec[ord[k].id];
            double i0, i1, j0, j1;
            if (o->cls == ORC_POINT) {
                i0 = i1 = floor(o->xs);
                j0 = j1 = floor(o->ys);
            } else {
                i0 = ceil(o->xs - o->r - 0.5); i1 = floor(o->xs + o->r - 0.5);
                j0 = ceil(o->ys - o->r - 0.5); j1 = floor(o->ys + o->r - 0.5);
            }
            if (i0 < 0.0) i0 = 0.0;
            if (j0 < 0.0) j0 = 0.0;
            if (i1 > v->w - 1) i1 = v->w - 1;
            if (j1 > v->h - 1) j1 = v->h - 1;
            for (long j = (long)j0; j <= (long)j1; ++j)
                for (long i = (long)i0; i <= (long)i1; ++i) {
                    double w = pixel_weight(o, i, j);
                    if (w > 0.0) cross_particle(o, q, w, img + 3 * (j * v->w + i));
                }
        }
    } else {
        orc_depth *hit = (orc_depth *)malloc(sizeof(orc_depth) * (m > 0 ? m : 1));
        if (!hit) {
            free(rec);
            free(ord);
            return -2;
        }
        for (long j = 0; j < v->h; ++j)
            for (long i = 0; i < v->w; ++i) {
                long c = 0;
                for (long k = 0; k < m; ++k)
                    if (pixel_weight(&rec[ord[k].id], i, j) > 0.0) hit[c++] = ord[k];
                qsort(hit, (size_t)c, sizeof(orc_depth), cmp_back_to_front);
                double *I = img + 3 * (j * v->w + i);
                for (long k = 0; k < c; ++k)
                    cross_particle(&rec[hit[k].id], q, pixel_weight(&rec[hit[k].id], i, j), I);
            }
        free(hit);
    }
    free(rec);
    free(ord);
    return 0;
}

/* Ambiguity mass B (per pixel and channel): the sum of |contributions| whose
 * inclusion, weight or pixel could legitimately flip when the same rules are
 * evaluated in FP32 instead of FP64:
 *   - the clip test, when |d - r| < 1e-5 r + 1e-6 px;
 *   - the point/splat class test, when |r - r_sml| < 1e-6 r_sml (both the
 *     point deposit and the whole splat are added);
 *   - the point pixel, when x_s or y_s lies within 1e-5 px of an integer (the
 *     deposit is added to every candidate pixel).
 * For mode 1 it is propagated through the map (derivative exp(-S) <= 1), so
 * the additive mass is an upper bound there too. */
static void add_mass(const orc_view *v, long i, long j, const double *e, double w,
                     double *B) {
    if (i < 0 || j < 0 || i >= v->w || j >= v->h) return;
    long o = 3L * (j * v->w + i);
    for (int k = 0; k < 3; ++k) B[o + k] += fabs(e[k]) * w;
}

static void ambiguity_one(const orc_view *v, const orc_params *q, const orc_rec *o,
                          double *B) {
    if (o->cls == ORC_INACTIVE) return;
    int class_amb = fabs(o->r - q->r_sml) < 1e-6 * q->r_sml;
    if (o->cls == ORC_POINT || class_amb) {
        /* candidate pixels: floor(x_s), and its left neighbour as well when
         * x_s sits within 1e-5 px of an integer (same for y) */
        double mx = floor(o->xs + 0.5), my = floor(o->ys + 0.5);
        int ax = fabs(o->xs - mx) < 1e-5, ay = fabs(o->ys - my) < 1e-5;
        double cx[2] = {ax ? mx - 1.0 : floor(o->xs), mx};
        double cy[2] = {ay ? my - 1.0 : floor(o->ys), my};
        if (class_amb || ax || ay)
            for (int a = 0; a < (ax ? 2 : 1); ++a)
                for (int b = 0; b < (ay ? 2 : 1); ++b)
                    add_mass(v, (long)cx[a], (long)cy[b], o->e, 1.0, B);
    }
    if (o->cls == ORC_SPLAT || class_amb) {
        double band = 1e-5 * o->r + 1e-6;
        double rr = o->r + band;
        double i0 = ceil(o->xs - rr - 0.5), i1 = floor(o->xs + rr - 0.5);
        double j0 = ceil(o->ys - rr - 0.5), j1 = floor(o->ys + rr - 0.5);
        if (i0 < 0.0) i0 = 0.0;
        if (j0 < 0.0) j0 = 0.0;
        if (i1 > v->w - 1) i1 = v->w - 1;
        if (j1 > v->h - 1) j1 = v->h - 1;
        for (long j = (long)j0; j <= (long)j1; ++j)
            for (long i = (long)i0; i <= (long)i1; ++i) {
                double dx = (i + 0.5) - o->xs, dy = (j + 0.5) - o->ys;
                double d = sqrt(dx * dx + dy * dy);
                if (class_amb ? d <= rr : fabs(d - o->r) < band)
                    add_mass(v, i, j, o->e, exp(-(d * d) / (o->sigma * o->sigma)), B);
            }
    }
}

static int near_tie_mass(long n, const float *x, const float *y, const float *z,
                         const float *h, const float *inten, const float *s, const float *pal,
                         int npal, const orc_view *v, const orc_params *q, double *B);

/* B image plus the number of particles whose class or point pixel is
 * ambiguous (clip-edge ambiguity is reported through B only).  In mode 2 B
 * also holds the near-tie mass (near_tie_mass): contributions of particles
 * whose depth lies within two FP32 ulps of another particle's that reaches
 * the same pixel. */
int orc_ambiguity(long n, const float *x, const float *y, const float *z,
                  const float *h, const float *inten, const float *s,
                  const float *pal, int npal, const orc_camera *cam,
                  const orc_params *q, double *B, long *n_amb_particles) {
    orc_view v;
    if (npal < 1 || make_view(cam, &v)) return -1;
    memset(B, 0, sizeof(double) * 3 * (long)v.w * v.h);
    /* mode 2: a contribution tau = A w that flips changes the pixel by at most
     * tau * max(E/A) = brightness * I * w * (largest palette value) in every
     * channel (the pixel value stays between 0 and the largest source term) */
    double pal_max = 0.0;
    for (long k = 0; k < 3L * npal; ++k) pal_max = fmax(pal_max, fabs((double)pal[k]));
    long cnt = 0;
    for (long p = 0; p < n; ++p) {
        orc_rec o;
        project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &o);
        if (o.cls == ORC_INACTIVE) continue;
        if (q->mode == 2)
            for (int k = 0; k < 3; ++k) o.e[k] = fabs(o.ib) * pal_max;
        int class_amb = fabs(o.r - q->r_sml) < 1e-6 * q->r_sml;
        int pix_amb = (o.cls == ORC_POINT) &&
                      (fabs(o.xs - floor(o.xs + 0.5)) < 1e-5 ||
                       fabs(o.ys - floor(o.ys + 0.5)) < 1e-5);
        if (class_amb || pix_amb) ++cnt;
        ambiguity_one(&v, q, &o, B);
    }
    if (n_amb_particles) *n_amb_particles = cnt;
    if (q->mode == 2) return near_tie_mass(n, x, y, z, h, inten, s, pal, npal, &v, q, B);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Selected pixels, pixel-major, with their ambiguity mass                 */
/* ---------------------------------------------------------------------- */

/* Ambiguity mass of one projected particle at pixel (i, j): the three rules
 * of ambiguity_one evaluated at one pixel.  e3 is the magnitude per channel
 * that a flipped contribution of weight 1 carries. */
static void pixel_ambiguity(const orc_params *q, const orc_rec *o, const double *e3, long i,
                            long j, double *B) {
    if (o->cls == ORC_INACTIVE) return;
    int class_amb = fabs(o->r - q->r_sml) < 1e-6 * q->r_sml;
    if (o->cls == ORC_POINT || class_amb) {
        double mx = floor(o->xs + 0.5), my = floor(o->ys + 0.5);
        int ax = fabs(o->xs - mx) < 1e-5, ay = fabs(o->ys - my) < 1e-5;
        int on_x = ax ? (i == (long)mx - 1 || i == (long)mx) : i == (long)floor(o->xs);
        int on_y = ay ? (j == (long)my - 1 || j == (long)my) : j == (long)floor(o->ys);
        if ((class_amb || ax || ay) && on_x && on_y)
            for (int k = 0; k < 3; ++k) B[k] += fabs(e3[k]);
    }
    if (o->cls == ORC_SPLAT || class_amb) {
        double band = 1e-5 * o->r + 1e-6, rr = o->r + band;
        double dx = (i + 0.5) - o->xs, dy = (j + 0.5) - o->ys;
        double d = sqrt(dx * dx + dy * dy);
        if (class_amb ? d <= rr : fabs(d - o->r) < band) {
            double w = exp(-(d * d) / (o->sigma * o->sigma));
            for (int k = 0; k < 3; ++k) B[k] += fabs(e3[k]) * w;
        }
    }
}

/* Mode 2: two absorbing particles whose FP64 depths lie this close together
 * (the smaller is at least the larger times 1 - 2^-22, i.e. within two FP32
 * ulps) may be crossed in either order by a renderer whose depth key is a
 * float.  The relation is monotone along sorted depths, so the particles
 * near one particle form a contiguous run around it in depth order. */
static int depth_near(double za, double zb) {
    double lo = za < zb ? za : zb, hi = za < zb ? zb : za;
    return lo >= hi * (1.0 - 0x1p-22);
}

/* Largest magnitude of a palette entry: in mode 2 a contribution tau = A w
 * moves a pixel by at most tau * max(E/A) = brightness * I * w * pal_max. */
static double palette_max(const float *pal, int npal) {
    double m = 0.0;
    for (long k = 0; k < 3L * npal; ++k) m = fmax(m, fabs((double)pal[k]));
    return m;
}

/* Mode 2 near-tie mass of a whole image: a contribution of particle p to a
 * pixel is ambiguous when another absorbing particle whose depth is near p's
 * (depth_near) also reaches that pixel: swapping two such particles changes
 * the pixel by at most g_1 g_2 |S_1 - S_2| <= the mass of either of them, and
 * permuting a run of them by at most the sum of the run's masses. */
static int near_tie_mass(long n, const float *x, const float *y, const float *z,
                         const float *h, const float *inten, const float *s, const float *pal,
                         int npal, const orc_view *v, const orc_params *q, double *B) {
    double pal_max = palette_max(pal, npal);
    orc_rec *rec = (orc_rec *)malloc(sizeof(orc_rec) * (n > 0 ? n : 1));
    orc_depth *ord = (orc_depth *)malloc(sizeof(orc_depth) * (n > 0 ? n : 1));
    if (!rec || !ord) {
        free(rec);
        free(ord);
        return -2;
    }
    long m = 0;
    for (long p = 0; p < n; ++p) {
        project_one(v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &rec[p]);
        if (rec[p].cls != ORC_INACTIVE && q->absorption * rec[p].ib > 0.0) {
            ord[m].key = rec[p].zc;
            ord[m].id = p;
            ++m;
        }
    }
    qsort(ord, (size_t)m, sizeof(orc_depth), cmp_back_to_front);
    for (long k = 0; k < m; ++k) {
        long a = k, b = k;
        while (a > 0 && depth_near(ord[a - 1].key, ord[k].key)) --a;
        while (b + 1 < m && depth_near(ord[b + 1].key, ord[k].key)) ++b;
        if (a == b) continue;
        const orc_rec *o = &rec[ord[k].id];
        double e3[3] = {fabs(o->ib) * pal_max, fabs(o->ib) * pal_max, fabs(o->ib) * pal_max};
        double i0, i1, j0, j1;
        if (o->cls == ORC_POINT) {
            i0 = i1 = floor(o->xs);
            j0 = j1 = floor(o->ys);
        } else {
            i0 = ceil(o->xs - o->r - 0.5); i1 = floor(o->xs + o->r - 0.5);
            j0 = ceil(o->ys - o->r - 0.5); j1 = floor(o->ys + o->r - 0.5);
        }
        if (i0 < 0.0) i0 = 0.0;
        if (j0 < 0.0) j0 = 0.0;
        if (i1 > v->w - 1) i1 = v->w - 1;
        if (j1 > v->h - 1) j1 = v->h - 1;
        for (long j = (long)j0; j <= (long)j1; ++j)
            for (long i = (long)i0; i <= (long)i1; ++i) {
                double w = pixel_weight(o, i, j);
                if (!(w > 0.0)) continue;
                int shared = 0;
                for (long t = a; t <= b && !shared; ++t)
                    if (t != k && pixel_weight(&rec[ord[t].id], i, j) > 0.0) shared = 1;
                if (shared) add_mass(v, i, j, e3, w, B);
            }
    }
    free(rec);
    free(ord);
    return 0;
}

/* One absorbing particle that reaches a selected pixel. */
typedef struct {
    double z, w;
    long id;
} orc_hit;

static int cmp_hit_back_to_front(const void *pa, const void *pb) {
    const orc_hit *a = (const orc_hit *)pa, *b = (const orc_hit *)pb;
    if (a->z != b->z) return a->z > b->z ? -1 : 1;
    if (a->id != b->id) return a->id > b->id ? -1 : 1;
    return 0;
}

/* Mode 2 at selected pixels: every pixel collects the absorbing particles
 * that reach it, sorts them from the farthest to the nearest (FP64 depth, then
 * decreasing index) and crosses them one after the other -- the pixel-major
 * branch of render_absorb, restricted to the selected pixels.  B (may be NULL)
 * receives the ambiguity mass: the rules of pixel_ambiguity with the mode-2
 * magnitude, plus the near-tie mass of near_tie_mass. */
static int pixels_absorb(long n, const float *x, const float *y, const float *z,
                         const float *h, const float *inten, const float *s, const float *pal,
                         int npal, const orc_view *v, const orc_params *q, long npix,
                         const int *px, const int *py, double *out, double *B, int nt) {
    if (!(q->absorption > 0.0)) return -1;
    double pal_max = palette_max(pal, npal);
    const long chunk = 16384;
    orc_rec *rec = (orc_rec *)malloc(sizeof(orc_rec) * chunk);
    orc_hit **hits = (orc_hit **)calloc((size_t)(npix > 0 ? npix : 1), sizeof(orc_hit *));
    long *cnt = (long *)calloc((size_t)(npix > 0 ? npix : 1), sizeof(long));
    long *cap = (long *)calloc((size_t)(npix > 0 ? npix : 1), sizeof(long));
    int err = 0;
    if (!rec || !hits || !cnt || !cap) err = 1;
    memset(out, 0, sizeof(double) * 3 * npix);
    if (B) memset(B, 0, sizeof(double) * 3 * npix);
    for (long lo = 0; lo < n && !err; lo += chunk) {
        long hi = lo + chunk < n ? lo + chunk : n;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt)
#endif
        for (long p = lo; p < hi; ++p)
            project_one(v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &rec[p - lo]);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 8) reduction(| : err)
#endif
        for (long k = 0; k < npix; ++k) {
            for (long p = lo; p < hi; ++p) {
                const orc_rec *o = &rec[p - lo];
                if (o->cls == ORC_INACTIVE) continue;
                if (B) {
                    double e3[3] = {fabs(o->ib) * pal_max, fabs(o->ib) * pal_max,
                                    fabs(o->ib) * pal_max};
                    pixel_ambiguity(q, o, e3, px[k], py[k], B + 3 * k);
                }
                if (!(q->absorption * o->ib > 0.0)) continue;
                double w = pixel_weight(o, px[k], py[k]);
                if (!(w > 0.0)) continue;
                if (cnt[k] == cap[k]) {
                    long nc = cap[k] ? 2 * cap[k] : 64;
                    orc_hit *g = (orc_hit *)realloc(hits[k], sizeof(orc_hit) * nc);
                    if (!g) {
                        err |= 1;
                        break;
                    }
                    hits[k] = g;
                    cap[k] = nc;
                }
                hits[k][cnt[k]].z = o->zc;
                hits[k][cnt[k]].w = w;
                hits[k][cnt[k]].id = p;
                cnt[k]++;
            }
        }
    }
    if (!err) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
#endif
        for (long k = 0; k < npix; ++k) {
            orc_hit *hk = hits[k];
            long c = cnt[k];
            qsort(hk, (size_t)c, sizeof(orc_hit), cmp_hit_back_to_front);
            double *I = out + 3 * k;
            for (long m = 0; m < c; ++m) {
                long id = hk[m].id;
                orc_rec o;
                project_one(v, q, pal, npal, id, x[id], y[id], z[id], h[id], inten[id], s[id], &o);
                cross_particle(&o, q, hk[m].w, I);
                if (B && ((m > 0 && depth_near(hk[m - 1].z, hk[m].z)) ||
                          (m + 1 < c && depth_near(hk[m + 1].z, hk[m].z))))
                    for (int ch = 0; ch < 3; ++ch) B[3 * k + ch] += fabs(o.ib) * pal_max * hk[m].w;
            }
        }
    }
    if (hits)
        for (long k = 0; k < npix; ++k) free(hits[k]);
    free(hits);
    free(cnt);
    free(cap);
    free(rec);
    return err ? -2 : 0;
}

/* Selected pixels, pixel-major: out[3*k..] = value of pixel (px[k], py[k]),
 * and (B not NULL) B[3*k..] = its ambiguity mass, the same as orc_ambiguity's
 * at that pixel.  Modes 0 and 1: particles are projected once per chunk;
 * threads own chunks and keep their own partial sums, summed at the end.
 * Mode 2: pixels_absorb. */
int orc_render_pixels(long n, const float *x, const float *y, const float *z,
                      const float *h, const float *inten, const float *s,
                      const float *pal, int npal, const orc_camera *cam,
                      const orc_params *q, long npix, const int *px,
                      const int *py, double *out, double *B, int nthreads) {
    orc_view v;
    if (npal < 1 || make_view(cam, &v)) return -1;
    for (long k = 0; k < npix; ++k)
        if (px[k] < 0 || py[k] < 0 || px[k] >= v.w || py[k] >= v.h) return -1;
    if (nthreads < 1) nthreads = 1;
    int nt = nthreads;
#ifndef _OPENMP
    nt = 1;
#endif
    if (q->mode == 2)
        return pixels_absorb(n, x, y, z, h, inten, s, pal, npal, &v, q, npix, px, py, out, B, nt);
    const long chunk = 16384;
    long nchunks = (n + chunk - 1) / chunk;
    memset(out, 0, sizeof(double) * 3 * npix);
    if (B) memset(B, 0, sizeof(double) * 3 * npix);
    double *part = (double *)calloc((size_t)nt * 3 * npix * (B ? 2 : 1) + 1, sizeof(double));
    if (!part) return -2;
    double *bpart = B ? part + (size_t)nt * 3 * npix : NULL;
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        orc_rec *rec = (orc_rec *)malloc(sizeof(orc_rec) * chunk);
        if (!rec) {
            err = 1;
        } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
            for (long c = 0; c < nchunks; ++c) {
                long lo = c * chunk, hi = lo + chunk < n ? lo + chunk : n;
                for (long p = lo; p < hi; ++p)
                    project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p],
                                inten[p], s[p], &rec[p - lo]);
                for (long k = 0; k < npix; ++k) {
                    double *acc = part + ((long)t * npix + k) * 3;
                    for (long p = 0; p < hi - lo; ++p)
                        pixel_term(&rec[p], px[k], py[k], acc);
                    if (bpart) {
                        double *bacc = bpart + ((long)t * npix + k) * 3;
                        for (long p = 0; p < hi - lo; ++p)
                            pixel_ambiguity(q, &rec[p], rec[p].e, px[k], py[k], bacc);
                    }
                }
            }
            free(rec);
        }
    }
    for (int t = 0; t < nt; ++t)
        for (long k = 0; k < 3 * npix; ++k) {
            out[k] += part[(long)t * 3 * npix + k];
            if (B) B[k] += bpart[(long)t * 3 * npix + k];
        }
    free(part);
    if (err) return -2;
    if (q->mode == 1)
        for (long k = 0; k < 3 * npix; ++k) out[k] = -expm1(-out[k]);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Tile-cost network: 32 -> 64 (ReLU) -> 1, FP64 reference.                */
/* Parameter vector layout: W1[64][32] row-major, b1[64], w2[64], b2.      */
/* ---------------------------------------------------------------------- */
#define ORC_MLP_IN 32
#define ORC_MLP_HID 64
#define ORC_MLP_NPARAM (ORC_MLP_HID * ORC_MLP_IN + 2 * ORC_MLP_HID + 1)

int orc_mlp_nparam(void) { return ORC_MLP_NPARAM; }

/* y[b] = w2 . relu(W1 x_b + b1) + b2 */
int orc_mlp_forward(const double *theta, long nb, const double *xin, double *yout) {
    const double *W1 = theta, *b1 = theta + ORC_MLP_HID * ORC_MLP_IN;
    const double *w2 = b1 + ORC_MLP_HID, *b2 = w2 + ORC_MLP_HID;
    for (long b = 0; b < nb; ++b) {
        double y = b2[0];
        for (int j = 0; j < ORC_MLP_HID; ++j) {
            double z = b1[j];
            for (int i = 0; i < ORC_MLP_IN; ++i) z += W1[j * ORC_MLP_IN + i] * xin[b * ORC_MLP_IN + i];
            if (z > 0.0) y += w2[j] * z;
        }
        yout[b] = y;
    }
    return 0;
}

/* Mean-squared-error loss L = (1/nb) sum_b (y_b - t_b)^2 and its gradient
 * with respect to every parameter (chain rule through the ReLU). */
double orc_mlp_loss_grad(const double *theta, long nb, const double *xin,
                         const double *target, double *grad) {
    const double *W1 = theta, *b1 = theta + ORC_MLP_HID * ORC_MLP_IN;
    const double *w2 = b1 + ORC_MLP_HID, *b2 = w2 + ORC_MLP_HID;
    double *gW1 = grad, *gb1 = grad + ORC_MLP_HID * ORC_MLP_IN;
    double *gw2 = gb1 + ORC_MLP_HID, *gb2 = gw2 + ORC_MLP_HID;
    double z[ORC_MLP_HID], loss = 0.0;
    memset(grad, 0, sizeof(double) * ORC_MLP_NPARAM);
    if (nb <= 0) return 0.0;
    for (long b = 0; b < nb; ++b) {
        const double *xb = xin + b * ORC_MLP_IN;
        double y = b2[0];
        for (int j = 0; j < ORC_MLP_HID; ++j) {
            double a = b1[j];
            for (int i = 0; i < ORC_MLP_IN; ++i) a += W1[j * ORC_MLP_IN + i] * xb[i];
            z[j] = a;
            if (a > 0.0) y += w2[j] * a;
        }
        double res = y - target[b];
        loss += res * res;
        double dy = 2.0 * res / nb;
        gb2[0] += dy;
        for (int j = 0; j < ORC_MLP_HID; ++j) {
            if (z[j] <= 0.0) continue;
            gw2[j] += dy * z[j];
            double dz = dy * w2[j];
            gb1[j] += dz;
            for (int i = 0; i < ORC_MLP_IN; ++i) gW1[j * ORC_MLP_IN + i] += dz * xb[i];
        }
    }
    return loss / nb;
}

/* One Adam step (Kingma & Ba, Algorithm 1) on every parameter; t >= 1. */
int orc_adam_step(double *theta, const double *grad, double *m, double *v,
                  long np, long t, double lr, double beta1, double beta2,
                  double eps) {
    double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
    for (long k = 0; k < np; ++k) {
        m[k] = beta1 * m[k] + (1.0 - beta1) * grad[k];
        v[k] = beta2 * v[k] + (1.0 - beta2) * grad[k] * grad[k];
        double mh = m[k] / c1, vh = v[k] / c2;
        theta[k] -= lr * mh / (sqrt(vh) + eps);
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Tile-cost features (the scheduler's input; no counterpart in the paper, */
/* which only notes that particles per tile vary and unbalance the work).  */
/* For an image cut into T x T tiles (the tiling of Eq. 8), a particle      */
/* belongs to tile t when its pixel-centre bounding box (the pixels with    */
/* |i+1/2-x_s| <= r and |j+1/2-y_s| <= r, cut to the image) meets t and the */
/* disc reaches the centre of a pixel of t (a tile whose pixel centres all  */
/* lie beyond r receives nothing, Eq. 2); a point-rule particle belongs to  */
/* the tile of its pixel.  Per tile:                                        */
/*   f[b]      = log1p(number of member particles with radius bin b)        */
/*   f[16 + b] = log1p(sum over those particles of the number of tile       */
/*               pixels inside their box, divided by area_scale)            */
/* with radius bin b = clamp(floor(log2(r / 0.5)), 0, 15) (0 for r < 1).    */
/* ---------------------------------------------------------------------- */
int orc_tile_features(long n, const float *x, const float *y, const float *z,
                      const float *h, const float *inten, const float *s,
                      const float *pal, int npal, const orc_camera *cam,
                      const orc_params *q, int tile, double area_scale,
                      double *feat) {
    orc_view v;
    if (npal < 1 || tile < 1 || !(area_scale > 0.0) || make_view(cam, &v)) return -1;
    long ntx = (v.w + tile - 1) / tile, nty = (v.h + tile - 1) / tile;
    double *cnt = (double *)calloc((size_t)ntx * nty * 16, sizeof(double));
    double *area = (double *)calloc((size_t)ntx * nty * 16, sizeof(double));
    if (!cnt || !area) {
        free(cnt); free(area);
        return -2;
    }
    for (long p = 0; p < n; ++p) {
        orc_rec o;
        project_one(&v, q, pal, npal, p, x[p], y[p], z[p], h[p], inten[p], s[p], &o);
        if (o.cls == ORC_INACTIVE) continue;
        int b = 0;
        if (o.r >= 1.0) {
            b = (int)floor(log2(o.r / 0.5));
            if (b > 15) b = 15;
        }
        double i0, i1, j0, j1;
        if (o.cls == ORC_POINT) {
            i0 = i1 = floor(o.xs);
            j0 = j1 = floor(o.ys);
        } else {
            i0 = ceil(o.xs - o.r - 0.5); i1 = floor(o.xs + o.r - 0.5);
            j0 = ceil(o.ys - o.r - 0.5); j1 = floor(o.ys + o.r - 0.5);
        }
        if (i0 < 0.0) i0 = 0.0;
        if (j0 < 0.0) j0 = 0.0;
        if (i1 > v.w - 1) i1 = v.w - 1;
        if (j1 > v.h - 1) j1 = v.h - 1;
        if (i0 > i1 || j0 > j1) continue;
        for (long ty = (long)j0 / tile; ty <= (long)j1 / tile; ++ty)
            for (long tx = (long)i0 / tile; tx <= (long)i1 / tile; ++tx) {
                double a0 = fmax(i0, (double)(tx * tile)), a1 = fmin(i1, (double)(tx * tile + tile - 1));
                double c0 = fmax(j0, (double)(ty * tile)), c1 = fmin(j1, (double)(ty * tile + tile - 1));
                if (o.cls == ORC_SPLAT) {
                    /* nearest pixel centre of the tile to the particle */
                    double ex = fmin(fmax(o.xs, tx * tile + 0.5), fmin((double)(tx * tile + tile), (double)v.w) - 0.5);
                    double ey = fmin(fmax(o.ys, ty * tile + 0.5), fmin((double)(ty * tile + tile), (double)v.h) - 0.5);
                    if ((ex - o.xs) * (ex - o.xs) + (ey - o.ys) * (ey - o.ys) > o.r * o.r) continue;
                }
                long t = ty * ntx + tx;
                cnt[t * 16 + b] += 1.0;
                area[t * 16 + b] += (a1 - a0 + 1.0) * (c1 - c0 + 1.0);
            }
    }
    for (long t = 0; t < ntx * nty; ++t)
        for (int b = 0; b < 16; ++b) {
            feat[t * 32 + b] = log1p(cnt[t * 16 + b]);
            feat[t * 32 + 16 + b] = log1p(area[t * 16 + b] / area_scale);
        }
    free(cnt);
    free(area);
    return 0;
}
