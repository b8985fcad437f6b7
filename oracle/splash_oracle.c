/*
 * FP64 CPU oracle for the Gaussian Splashing underwater rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, slow, obviously correct
 * statement of what the CUDA renderer computes. Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg load it; the product path
 * never does. It shares no code, header, table or constant with the CUDA
 * sources: no tiling, no sort keys, no telescoped colour, no fast math.
 *
 * Passages followed (Gaussian Splashing, arXiv 2411.19588):
 *  - Scene = N Gaussians theta_i = (mu_i, Sigma_i, c_i via SH, opacity):
 *    Sec. III-A.
 *  - Front-to-back alpha compositing over the depth-sorted Gaussians that
 *    affect a pixel, C = sum c_i alpha_i T_i, T_i = prod_{j<i} (1 - alpha_j):
 *    Eq. 1.
 *  - alpha_i = sigmoid(o_i) exp(-1/2 d^T Sigma2^{-1} d), evaluated in 2D with
 *    the affine (EWA) projection of the covariance: Eq. 2 and the sentence
 *    after it (Sec. III-A).
 *  - Water: the Sea-thru formation I = J e^{-beta_D z} + B_inf (1 - e^{-beta_B z})
 *    (Eq. 3, Eq. 4) folded into compositing (Eq. 5). This oracle states the
 *    per-Gaussian discretisation of that model: the direct signal of
 *    Gaussian i is attenuated by e^{-beta_D d_i}; backscatter
 *    B_inf (e^{-beta_B d_{i-1}} - e^{-beta_B d_i}) is accumulated over the
 *    water between consecutive Gaussians (d_0 = 0, the camera) and behind the
 *    last one out to z_far, each water segment weighted by the transmittance
 *    in front of it. With a single opaque surface this is exactly Eq. 4.
 *  - Expected depth z = sum d_i alpha_i T_i / sum alpha_i T_i: Eq. 6; the
 *    logistic map z01 = 2 / (1 + e^{-0.1 z}) - 1: Sec. IV-D.
 *
 * Readings where the paper is silent (3DGS conventions; listed in the design
 * notes): alpha clamped at 0.99; a Gaussian with alpha < 1/255 at a pixel is
 * skipped; a pixel stops before the Gaussian that would bring T below 1e-4;
 * a Gaussian takes part at a pixel only when d^T Sigma2^{-1} d <= 9 there;
 * 2D dilation +0.3 px^2; near plane z_near, Gaussians with z > z_far culled;
 * projection Jacobian with t_x/t_z and t_y/t_z clamped to 1.3x the half-FOV
 * tangent; colour = real SH (degree <= 3) + 0.5, clamped at 0; depth d_i is
 * the camera-frame z of the mean; ties in depth go to the lower index; an
 * empty pixel has depth z_far.
 *
 * Parity pins (tests, CPU only): beta = 0 reduces to plain compositing;
 * empty scene = pure backscatter; closed form at a single Gaussian's centre;
 * zero-alpha insertions are invisible; the telescoped identity; projection
 * against scipy rotations and a finite-difference projection Jacobian; SH
 * orthonormality; analytic gradients against central finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define A_MAX 0.99
#define A_MIN (1.0 / 255.0)
#define T_STOP 1e-4
#define Q_MAX 9.0
#define DILATE 0.3
#define JCLAMP 1.3

/* per-Gaussian fields written by oracle_project */
enum {
    P_VIS, P_X, P_Y, P_KA, P_KB, P_KC, P_SA, P_SB, P_SC, P_OPAC,
    P_COL, P_A = P_COL + 3, P_B = P_A + 3, P_D = P_B + 3, P_RAW,
    P_CULLM = P_RAW + 3, P_TX, P_TY, P_GMARG, NPROJ
};
/* per-pixel fields written by oracle_render */
enum {
    O_R, O_G, O_B, O_DEPTH, O_DEPTH01, O_TF, O_NCONTRIB, O_ACC, O_MARGIN,
    O_GMARGIN, O_TIE, O_NCAND, O_DSUM, O_NITER, O_NNEAR, NPIX
};
/* per-branch fields written by oracle_render_branches */
enum { B_R, B_G, B_B, B_DEPTH, B_DEPTH01, B_TF, B_NCONTRIB, B_VALID, NBF };

int oracle_nproj(void) { return NPROJ; }
int oracle_npix(void) { return NPIX; }

typedef struct {
    int W, H;
    double fx, fy, cx, cy;
    double R[9], t[3];
    double znear, zfar;
} cam_t;

static void cam_load(const double *c, cam_t *k)
{
    k->W = (int)c[0];
    k->H = (int)c[1];
    k->fx = c[2];
    k->fy = c[3];
    k->cx = c[4];
    k->cy = c[5];
    for (int r = 0; r < 3; r++) {
        for (int j = 0; j < 3; j++) k->R[3 * r + j] = c[6 + 4 * r + j];
        k->t[r] = c[6 + 4 * r + 3];
    }
    k->znear = c[18];
    k->zfar = c[19];
}

/* Real spherical harmonics of degree <= 3, orthonormal on the unit sphere
 * (no Condon-Shortley phase), index k = l^2 + l + m, written as harmonic
 * polynomials of the unit vector (x, y, z); dY holds their partial
 * derivatives with respect to x, y and z. */
static void sh_basis(int deg, const double *v, double *Y, double (*dY)[3])
{
    const double x = v[0], y = v[1], z = v[2], pi = M_PI;
    const int K = (deg + 1) * (deg + 1);
    for (int k = 0; k < K; k++) {
        Y[k] = 0.0;
        if (dY) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
    }
    Y[0] = 0.5 / sqrt(pi);
    if (deg >= 1) {
        const double k1 = sqrt(3.0 / (4.0 * pi));
        Y[1] = k1 * y;
        Y[2] = k1 * z;
        Y[3] = k1 * x;
        if (dY) {
            dY[1][1] = k1;
            dY[2][2] = k1;
            dY[3][0] = k1;
        }
    }
    if (deg >= 2) {
        const double ka = 0.5 * sqrt(15.0 / pi), kb = 0.25 * sqrt(5.0 / pi), kc = 0.25 * sqrt(15.0 / pi);
        Y[4] = ka * x * y;
        Y[5] = ka * y * z;
        Y[6] = kb * (2 * z * z - x * x - y * y);
        Y[7] = ka * x * z;
        Y[8] = kc * (x * x - y * y);
        if (dY) {
            dY[4][0] = ka * y; dY[4][1] = ka * x;
            dY[5][1] = ka * z; dY[5][2] = ka * y;
            dY[6][0] = -2 * kb * x; dY[6][1] = -2 * kb * y; dY[6][2] = 4 * kb * z;
            dY[7][0] = ka * z; dY[7][2] = ka * x;
            dY[8][0] = 2 * kc * x; dY[8][1] = -2 * kc * y;
        }
    }
    if (deg >= 3) {
        const double k9 = 0.25 * sqrt(35.0 / (2 * pi)), k10 = 0.5 * sqrt(105.0 / pi);
        const double k11 = 0.25 * sqrt(21.0 / (2 * pi)), k12 = 0.25 * sqrt(7.0 / pi);
        const double k14 = 0.25 * sqrt(105.0 / pi);
        Y[9] = k9 * y * (3 * x * x - y * y);
        Y[10] = k10 * x * y * z;
        Y[11] = k11 * y * (4 * z * z - x * x - y * y);
        Y[12] = k12 * z * (2 * z * z - 3 * x * x - 3 * y * y);
        Y[13] = k11 * x * (4 * z * z - x * x - y * y);
        Y[14] = k14 * z * (x * x - y * y);
        Y[15] = k9 * x * (x * x - 3 * y * y);
        if (dY) {
            dY[9][0] = k9 * 6 * x * y; dY[9][1] = k9 * (3 * x * x - 3 * y * y);
            dY[10][0] = k10 * y * z; dY[10][1] = k10 * x * z; dY[10][2] = k10 * x * y;
            dY[11][0] = k11 * (-2 * x * y); dY[11][1] = k11 * (4 * z * z - x * x - 3 * y * y); dY[11][2] = k11 * 8 * y * z;
            dY[12][0] = k12 * (-6 * x * z); dY[12][1] = k12 * (-6 * y * z); dY[12][2] = k12 * (6 * z * z - 3 * x * x - 3 * y * y);
            dY[13][0] = k11 * (4 * z * z - 3 * x * x - y * y); dY[13][1] = k11 * (-2 * x * y); dY[13][2] = k11 * 8 * x * z;
            dY[14][0] = k14 * 2 * x * z; dY[14][1] = -k14 * 2 * y * z; dY[14][2] = k14 * (x * x - y * y);
            dY[15][0] = k9 * (3 * x * x - 3 * y * y); dY[15][1] = k9 * (-6 * x * y);
        }
    }
}

int oracle_sh_basis(int deg, const double *dir, double *Y)
{
    if (deg < 0 || deg > 3) return -1;
    sh_basis(deg, dir, Y, NULL);
    return 0;
}

/* rotation matrix of the unit quaternion u = (w, x, y, z), row-major */
static void quat_rot(const double *u, double *R)
{
    const double w = u[0], x = u[1], y = u[2], z = u[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* dR/du_c for c = w, x, y, z */
static void quat_rot_grad(const double *u, double dR[4][9])
{
    const double w = u[0], x = u[1], y = u[2], z = u[3];
    const double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    const double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    const double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof Dw);
    memcpy(dR[1], Dx, sizeof Dx);
    memcpy(dR[2], Dy, sizeof Dy);
    memcpy(dR[3], Dz, sizeof Dz);
}

/* Everything the oracle knows about one projected Gaussian. */
typedef struct {
    int vis;
    double t[3];        /* camera-frame mean */
    double d;           /* depth: camera-frame z */
    double x, y;        /* projected centre, pixel units */
    double u[4], qn;    /* unit quaternion and |q| */
    double Rq[9];       /* Gaussian rotation */
    double s[3];        /* exp(log_scale) */
    double S3[9];       /* 3D covariance */
    double J[6];        /* 2x3 projection Jacobian (with clamps) */
    int clx, cly;       /* -1 / 0 / +1: which Jacobian clamp is active */
    double rxc, ryc;    /* clamped t_x/t_z, t_y/t_z */
    double U[6];        /* J * W */
    double S2[3];       /* 2D covariance a, b, c (dilated) */
    double K[3];        /* its inverse: q = K0 dx^2 + 2 K1 dx dy + K2 dy^2 */
    double opac;        /* sigmoid(logit) */
    double dir[3], vn;  /* unit view direction and |mu - camera centre| */
    double Y[16], dY[16][3];
    double raw[3], col[3];
    double a[3], b[3];  /* e^{-beta_D d}, e^{-beta_B d} */
    double cullm;       /* relative distance of z to the near/far planes */
    double gm;          /* relative distance to a gradient kink (clamps) */
} pg_t;

static void project_one(const cam_t *c, const double *mu, const double *ls, const double *q, double ologit,
                        const double *sh, int deg, const double *med, pg_t *g)
{
    memset(g, 0, sizeof *g);
    for (int r = 0; r < 3; r++)
        g->t[r] = c->R[3 * r] * mu[0] + c->R[3 * r + 1] * mu[1] + c->R[3 * r + 2] * mu[2] + c->t[r];
    const double tx = g->t[0], ty = g->t[1], tz = g->t[2];
    g->d = tz;
    g->cullm = fmin(fabs(tz - c->znear) / c->znear, fabs(tz - c->zfar) / c->zfar);
    g->vis = (tz > c->znear) && (tz <= c->zfar);
    if (!g->vis) return;

    /* 3D covariance Sigma = R S S^T R^T from scale and rotation */
    g->qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; k++) g->u[k] = q[k] / g->qn;
    quat_rot(g->u, g->Rq);
    for (int j = 0; j < 3; j++) g->s[j] = exp(ls[j]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += g->Rq[3 * i + k] * g->s[k] * g->s[k] * g->Rq[3 * j + k];
            g->S3[3 * i + j] = acc;
        }

    /* affine approximation of the pinhole projection at t (EWA) */
    const double limx = JCLAMP * 0.5 * c->W / c->fx, limy = JCLAMP * 0.5 * c->H / c->fy;
    const double rx = tx / tz, ry = ty / tz;
    g->clx = rx < -limx ? -1 : (rx > limx ? 1 : 0);
    g->cly = ry < -limy ? -1 : (ry > limy ? 1 : 0);
    g->rxc = g->clx ? g->clx * limx : rx;
    g->ryc = g->cly ? g->cly * limy : ry;
    g->J[0] = c->fx / tz; g->J[1] = 0;            g->J[2] = -c->fx * g->rxc / tz;
    g->J[3] = 0;          g->J[4] = c->fy / tz;   g->J[5] = -c->fy * g->ryc / tz;
    for (int a = 0; a < 2; a++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += g->J[3 * a + k] * c->R[3 * k + j];
            g->U[3 * a + j] = acc;
        }
    double S2[4];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double acc = 0;
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) acc += g->U[3 * a + i] * g->S3[3 * i + j] * g->U[3 * b + j];
            S2[2 * a + b] = acc;
        }
    g->S2[0] = S2[0] + DILATE;
    g->S2[1] = 0.5 * (S2[1] + S2[2]);
    g->S2[2] = S2[3] + DILATE;
    const double det = g->S2[0] * g->S2[2] - g->S2[1] * g->S2[1];
    g->K[0] = g->S2[2] / det;
    g->K[1] = -g->S2[1] / det;
    g->K[2] = g->S2[0] / det;
    g->x = c->fx * tx / tz + c->cx;
    g->y = c->fy * ty / tz + c->cy;
    g->opac = 1.0 / (1.0 + exp(-ologit));

    /* view-dependent colour from SH, direction from the camera centre */
    double cc[3];
    for (int j = 0; j < 3; j++) cc[j] = -(c->R[j] * c->t[0] + c->R[3 + j] * c->t[1] + c->R[6 + j] * c->t[2]);
    double v[3] = {mu[0] - cc[0], mu[1] - cc[1], mu[2] - cc[2]};
    g->vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int j = 0; j < 3; j++) g->dir[j] = v[j] / g->vn;
    sh_basis(deg, g->dir, g->Y, g->dY);
    const int K = (deg + 1) * (deg + 1);
    g->gm = INFINITY;
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.5;
        for (int k = 0; k < K; k++) acc += sh[3 * k + ch] * g->Y[k];
        g->raw[ch] = acc;
        g->col[ch] = acc > 0 ? acc : 0;
        g->gm = fmin(g->gm, fabs(acc));
        g->a[ch] = exp(-med[ch] * tz);
        g->b[ch] = exp(-med[3 + ch] * tz);
    }
    g->gm = fmin(g->gm, fabs(fabs(rx) - limx) / limx);
    g->gm = fmin(g->gm, fabs(fabs(ry) - limy) / limy);
}

static void project_all(const cam_t *c, int64_t n, const double *means, const double *ls, const double *quats,
                        const double *ologits, const double *sh, int deg, const double *med, pg_t *out, int nthreads)
{
    const int K = (deg + 1) * (deg + 1);
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t i = 0; i < n; i++)
        project_one(c, means + 3 * i, ls + 3 * i, quats + 4 * i, ologits[i], sh + 3 * K * i, deg, med, &out[i]);
}

int oracle_project(int64_t n, const double *means, const double *ls, const double *quats, const double *ologits,
                   const double *sh, int deg, const double *med, const double *cam, double *out, int nthreads)
{
    if (n < 0 || deg < 0 || deg > 3) return -1;
    cam_t c;
    cam_load(cam, &c);
    pg_t *P = (pg_t *)malloc(sizeof(pg_t) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(&c, n, means, ls, quats, ologits, sh, deg, med, P, nthreads);
    for (int64_t i = 0; i < n; i++) {
        double *o = out + (size_t)NPROJ * i;
        const pg_t *g = &P[i];
        memset(o, 0, sizeof(double) * NPROJ);
        o[P_VIS] = g->vis;
        o[P_D] = g->d;
        o[P_CULLM] = g->cullm;
        o[P_TX] = g->t[0];
        o[P_TY] = g->t[1];
        if (!g->vis) continue;
        o[P_X] = g->x; o[P_Y] = g->y;
        for (int k = 0; k < 3; k++) {
            o[P_KA + k] = g->K[k];
            o[P_SA + k] = g->S2[k];
            o[P_COL + k] = g->col[k];
            o[P_A + k] = g->a[k];
            o[P_B + k] = g->b[k];
            o[P_RAW + k] = g->raw[k];
        }
        o[P_OPAC] = g->opac;
        o[P_GMARG] = g->gm;
    }
    free(P);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* One pixel: which Gaussians take part, in which order.                  */

typedef struct { double d; int64_t id; double q, dx, dy; } cand_t;

static int cand_cmp(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    if (a->d < b->d) return -1;
    if (a->d > b->d) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

typedef struct { int64_t id; double alpha, araw, q, dx, dy, T; } contrib_t;

typedef struct {
    cand_t *cand;
    contrib_t *lst;
    int64_t cap;
} scratch_t;

static void scratch_reserve(scratch_t *s, int64_t need)
{
    if (need <= s->cap) return;
    int64_t cap = s->cap ? s->cap : 256;
    while (cap < need) cap *= 2;
    s->cand = (cand_t *)realloc(s->cand, sizeof(cand_t) * (size_t)cap);
    s->lst = (contrib_t *)realloc(s->lst, sizeof(contrib_t) * (size_t)cap);
    s->cap = cap;
}

/* The discrete decisions a pixel takes: the 3-sigma cut of a Gaussian, the
 * alpha < 1/255 skip, the transmittance stop, and the order of Gaussians
 * whose depths are equal at FP32 resolution. A renderer that evaluates the
 * same definition in FP32 may take a decision the other way when its FP64
 * quantity lies within rounding of the threshold; either outcome is then a
 * render of the definition at that precision. The oracle lists the decisions
 * of a pixel whose quantity lies within a relative distance `rel` of the
 * threshold ("near" decisions) and can evaluate the pixel under any
 * combination of their outcomes (a branch; branch 0 takes every decision as
 * FP64 does). For the order, the one alternative is the order of the FP32
 * depths, ties to the lower index. */
enum { D_CUT, D_SKIP, D_STOP, D_ORDER };
#define NEAR_MAX 4
#define NBR (1 << NEAR_MAX)
typedef struct { int kind; int64_t id; } decision_t;
typedef struct {
    double rel;              /* relative distance to a threshold counted as near */
    int n;                   /* near decisions found (may exceed NEAR_MAX) */
    decision_t d[NEAR_MAX];  /* the first NEAR_MAX of them, in walk order */
} near_t;
typedef struct { int n; decision_t d[NEAR_MAX]; } flips_t;

static int flipped(const flips_t *f, int kind, int64_t id)
{
    if (!f) return 0;
    for (int i = 0; i < f->n; i++)
        if (f->d[i].kind == kind && f->d[i].id == id) return 1;
    return 0;
}

static void note_near(near_t *nr, int kind, int64_t id, double dist)
{
    if (!nr || !(dist < nr->rel)) return;
    if (nr->n < NEAR_MAX) {
        nr->d[nr->n].kind = kind;
        nr->d[nr->n].id = id;
    }
    nr->n++;
}

/* the decisions a branch flips: bit i of b flips near decision i */
static void branch_flips(const near_t *nr, int64_t b, flips_t *f)
{
    f->n = 0;
    for (int i = 0; i < nr->n && i < NEAR_MAX; i++)
        if ((b >> i) & 1) f->d[f->n++] = nr->d[i];
}

static int cand_cmp_f32(const void *pa, const void *pb)
{
    const cand_t *a = (const cand_t *)pa, *b = (const cand_t *)pb;
    const float fa = (float)a->d, fb = (float)b->d;
    if (fa < fb) return -1;
    if (fa > fb) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

typedef struct {
    int64_t m;         /* contributors */
    int64_t ncand;     /* Gaussians within the 3-sigma ellipse */
    int64_t niter;     /* candidates walked, including the one that stopped the pixel */
    double Tf;         /* transmittance after the last contributor */
    double margin;     /* smallest relative distance to a discrete decision */
    double gmargin;    /* smallest relative distance to a gradient kink */
    int tie;           /* an FP32 depth sort would swap two alpha-valid neighbours */
} plist_t;

/* Collect, sort and walk the Gaussians at pixel centre (px, py) with the
 * skip and stop rules; the contributors land in s->lst. `fl` (may be NULL)
 * names the decisions taken the other way; `nr` (may be NULL) collects the
 * near decisions of this walk. */
static void pixel_list(const pg_t *P, const int64_t *vis, int64_t nvis, double px, double py, scratch_t *s,
                       plist_t *out, const flips_t *fl, near_t *nr)
{
    int64_t nc = 0;
    double mg = INFINITY, gm = INFINITY;
    if (nr) nr->n = 0;
    for (int64_t k = 0; k < nvis; k++) {
        const pg_t *g = &P[vis[k]];
        const double dx = px - g->x, dy = py - g->y;
        const double q = g->K[0] * dx * dx + 2.0 * g->K[1] * dx * dy + g->K[2] * dy * dy;
        const double dist = fabs(q - Q_MAX) / Q_MAX;
        mg = fmin(mg, dist);
        note_near(nr, D_CUT, vis[k], dist);
        int inside = q <= Q_MAX;
        if (flipped(fl, D_CUT, vis[k])) inside = !inside;
        if (inside) {
            scratch_reserve(s, nc + 1);
            s->cand[nc].d = g->d;
            s->cand[nc].id = vis[k];
            s->cand[nc].q = q;
            s->cand[nc].dx = dx;
            s->cand[nc].dy = dy;
            nc++;
        }
    }
    qsort(s->cand, (size_t)nc, sizeof(cand_t), flipped(fl, D_ORDER, -1) ? cand_cmp_f32 : cand_cmp);
    double T = 1.0, prev_d = -1.0;
    int64_t m = 0, it = 0, prev_id = -1;
    int tie = 0;
    for (int64_t k = 0; k < nc; k++) {
        const cand_t *cd = &s->cand[k];
        const pg_t *g = &P[cd->id];
        const double araw = g->opac * exp(-0.5 * cd->q);
        const double alpha = araw < A_MAX ? araw : A_MAX;
        it++;
        gm = fmin(gm, fabs(araw - A_MAX) / A_MAX);
        const double adist = fabs(alpha - A_MIN) / A_MIN;
        mg = fmin(mg, adist);
        note_near(nr, D_SKIP, cd->id, adist);
        int skip = alpha < A_MIN;
        if (flipped(fl, D_SKIP, cd->id)) skip = !skip;
        if (skip) continue;
        /* An FP32 depth orders two Gaussians like their exact depths unless
         * both round to the same float, where ties go to the lower index
         * (rounding is monotonic). Flag the pixel when that index order
         * disagrees with the exact depth order of two alpha-valid neighbours. */
        if (prev_id >= 0 && (float)cd->d == (float)prev_d && prev_id > cd->id) {
            if (!tie) note_near(nr, D_ORDER, -1, 0.0);
            tie = 1;
        }
        prev_d = cd->d;
        prev_id = cd->id;
        const double Tn = T * (1.0 - alpha);
        const double tdist = fabs(Tn - T_STOP) / T_STOP;
        mg = fmin(mg, tdist);
        note_near(nr, D_STOP, cd->id, tdist);
        int stop = Tn < T_STOP;
        if (flipped(fl, D_STOP, cd->id)) stop = !stop;
        if (stop) break;
        gm = fmin(gm, g->gm);
        contrib_t *c = &s->lst[m++];
        c->id = cd->id;
        c->alpha = alpha;
        c->araw = araw;
        c->q = cd->q;
        c->dx = cd->dx;
        c->dy = cd->dy;
        c->T = T;
        T = Tn;
    }
    out->m = m;
    out->ncand = nc;
    out->niter = it;
    out->Tf = T;
    out->margin = mg;
    out->gmargin = gm;
    out->tie = tie;
}

/* The water model on one ordered contributor list, as a sum over Gaussians
 * and water segments (the definition, not a telescoped form):
 *   C = sum_i c_i e^{-beta_D d_i} alpha_i T_i
 *     + B_inf sum_{i=1}^{m+1} T_i (e^{-beta_B d_{i-1}} - e^{-beta_B d_i}),
 * with d_0 = 0 (the camera) and d_{m+1} = z_far; also returns T after the
 * list and the depth sums D = sum d alpha T, A = sum alpha T (Eq. 6). */
static void composite_segments(int64_t m, const double *alpha, const double *col, const double *d,
                               const double *med, double zfar, double *rgb, double *Tf, double *Ds, double *As)
{
    double T = 1.0, dprev = 0.0, D = 0.0, A = 0.0;
    rgb[0] = rgb[1] = rgb[2] = 0.0;
    for (int64_t i = 0; i < m; i++) {
        for (int ch = 0; ch < 3; ch++) {
            const double direct = col[3 * i + ch] * exp(-med[ch] * d[i]) * alpha[i] * T;
            const double water = med[6 + ch] * T * (exp(-med[3 + ch] * dprev) - exp(-med[3 + ch] * d[i]));
            rgb[ch] += direct + water;
        }
        D += d[i] * alpha[i] * T;
        A += alpha[i] * T;
        T *= 1.0 - alpha[i];
        dprev = d[i];
    }
    for (int ch = 0; ch < 3; ch++)
        rgb[ch] += med[6 + ch] * T * (exp(-med[3 + ch] * dprev) - exp(-med[3 + ch] * zfar));
    *Tf = T;
    *Ds = D;
    *As = A;
}

int oracle_composite(int64_t m, const double *alpha, const double *col, const double *d, const double *med,
                     double zfar, double *out)
{
    if (m < 0) return -1;
    composite_segments(m, alpha, col, d, med, zfar, out, out + 3, out + 4, out + 5);
    return 0;
}

static double depth_of(double D, double A, double zfar) { return A > 0 ? D / A : zfar; }
static double logistic01(double z) { return 2.0 / (1.0 + exp(-0.1 * z)) - 1.0; }

static int64_t *visible_ids(const pg_t *P, int64_t n, int64_t *nvis)
{
    int64_t *vis = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        if (P[i].vis) vis[k++] = i;
    *nvis = k;
    return vis;
}

/* Per-thread buffers of one pixel's composite. */
typedef struct {
    scratch_t s;
    double *al, *co, *dd;
    int64_t acap;
} pixbuf_t;

static void pixbuf_free(pixbuf_t *b)
{
    free(b->s.cand);
    free(b->s.lst);
    free(b->al);
    free(b->co);
    free(b->dd);
}

/* Walk one pixel (with the flipped decisions `fl`, collecting near ones into
 * `nr`) and composite its contributors. res = r, g, b, depth, depth01, A, D. */
static void render_pixel(const pg_t *P, const int64_t *vis, int64_t nvis, const cam_t *c, const double *med,
                         int64_t p, const flips_t *fl, near_t *nr, pixbuf_t *b, plist_t *L, double *res)
{
    const double px = (double)(p % c->W) + 0.5, py = (double)(p / c->W) + 0.5;
    pixel_list(P, vis, nvis, px, py, &b->s, L, fl, nr);
    if (L->m > b->acap) {
        b->acap = L->m * 2;
        b->al = (double *)realloc(b->al, sizeof(double) * (size_t)b->acap);
        b->co = (double *)realloc(b->co, sizeof(double) * 3 * (size_t)b->acap);
        b->dd = (double *)realloc(b->dd, sizeof(double) * (size_t)b->acap);
    }
    for (int64_t i = 0; i < L->m; i++) {
        const pg_t *g = &P[b->s.lst[i].id];
        b->al[i] = b->s.lst[i].alpha;
        b->dd[i] = g->d;
        for (int ch = 0; ch < 3; ch++) b->co[3 * i + ch] = g->col[ch];
    }
    double Tf, D, A;
    composite_segments(L->m, b->al, b->co, b->dd, med, c->zfar, res, &Tf, &D, &A);
    res[3] = depth_of(D, A, c->zfar);
    res[4] = logistic01(res[3]);
    res[5] = A;
    res[6] = D;
}

/* Render every pixel (pix = NULL) or the npix listed linear pixel indices.
 * near_rel: the relative distance to a threshold that counts a decision as
 * near (the O_NNEAR field). */
/* Optional binning, a speed-up of the per-pixel candidate scan that leaves
 * every result unchanged: each visible Gaussian is listed in every
 * bin x bin block of pixels that its axis-aligned box |dx| <= sqrt(Qb Sxx),
 * |dy| <= sqrt(Qb Syy) meets, with Qb = 9 (1 + 4 near_rel) + 1e-9. The box
 * holds every point where q <= Qb, so a pixel's list holds every Gaussian
 * that can lie inside its 3-sigma ellipse or within near_rel of its edge, in
 * increasing index order like the unbinned scan. bin = 0: no binning. */
typedef struct {
    int bin, bx, by;
    int64_t *start, *ids;
} bins_t;

static int bins_build(const pg_t *P, const int64_t *vis, int64_t nvis, const cam_t *c, int bin, double near_rel,
                      bins_t *b)
{
    memset(b, 0, sizeof *b);
    if (bin <= 0) return 0;
    b->bin = bin;
    b->bx = (c->W + bin - 1) / bin;
    b->by = (c->H + bin - 1) / bin;
    const int64_t nb = (int64_t)b->bx * b->by;
    b->start = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    int64_t *fill = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    if (!b->start || !fill) return -2;
    const double Qb = Q_MAX * (1.0 + 4.0 * near_rel) + 1e-9;
    for (int pass = 0; pass < 2; pass++) {
        for (int64_t k = 0; k < nvis; k++) {
            const pg_t *g = &P[vis[k]];
            const double hx = sqrt(Qb * g->S2[0]), hy = sqrt(Qb * g->S2[2]);
            if (!(isfinite(hx) && isfinite(hy) && isfinite(g->x) && isfinite(g->y))) continue;
            /* pixel columns and rows whose centres lie in the box */
            const double fx0 = fmax(ceil(g->x - hx - 0.5), 0.0), fx1 = fmin(floor(g->x + hx - 0.5), c->W - 1.0);
            const double fy0 = fmax(ceil(g->y - hy - 0.5), 0.0), fy1 = fmin(floor(g->y + hy - 0.5), c->H - 1.0);
            if (fx0 > fx1 || fy0 > fy1) continue;
            const int tx0 = (int)fx0 / bin, tx1 = (int)fx1 / bin, ty0 = (int)fy0 / bin, ty1 = (int)fy1 / bin;
            for (int ty = ty0; ty <= ty1; ty++)
                for (int tx = tx0; tx <= tx1; tx++) {
                    const int64_t t = (int64_t)ty * b->bx + tx;
                    if (pass == 0)
                        b->start[t + 1]++;
                    else
                        b->ids[fill[t]++] = vis[k];
                }
        }
        if (pass == 0) {
            for (int64_t t = 0; t < nb; t++) b->start[t + 1] += b->start[t];
            b->ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(b->start[nb] > 0 ? b->start[nb] : 1));
            if (!b->ids) {
                free(fill);
                return -2;
            }
            memcpy(fill, b->start, sizeof(int64_t) * (size_t)nb);
        }
    }
    free(fill);
    return 0;
}

static void bins_free(bins_t *b)
{
    free(b->start);
    free(b->ids);
}

/* the Gaussians pixel p scans: every visible one, or its bin's list */
static void pixel_candidates(const bins_t *b, const int64_t *vis, int64_t nvis, const cam_t *c, int64_t p,
                             const int64_t **ids, int64_t *nids)
{
    if (b->bin <= 0) {
        *ids = vis;
        *nids = nvis;
        return;
    }
    const int64_t t = (p / c->W) / b->bin * b->bx + (p % c->W) / b->bin;
    *ids = b->ids + b->start[t];
    *nids = b->start[t + 1] - b->start[t];
}

int oracle_render(int64_t n, const double *means, const double *ls, const double *quats, const double *ologits,
                  const double *sh, int deg, const double *med, const double *cam, int64_t npix,
                  const int64_t *pix, double near_rel, int bin, double *out, int nthreads)
{
    if (n < 0 || deg < 0 || deg > 3) return -1;
    cam_t c;
    cam_load(cam, &c);
    if (!pix) npix = (int64_t)c.W * c.H;
    pg_t *P = (pg_t *)malloc(sizeof(pg_t) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(&c, n, means, ls, quats, ologits, sh, deg, med, P, nthreads);
    int64_t nvis;
    int64_t *vis = visible_ids(P, n, &nvis);
    bins_t bins;
    if (bins_build(P, vis, nvis, &c, bin, near_rel, &bins) != 0) return -2;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    {
        pixbuf_t b = {0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < npix; k++) {
            plist_t L;
            near_t nr = {near_rel, 0, {{0, 0}}};
            double res[7];
            const int64_t p = pix ? pix[k] : k;
            const int64_t *ids;
            int64_t nids;
            pixel_candidates(&bins, vis, nvis, &c, p, &ids, &nids);
            render_pixel(P, ids, nids, &c, med, p, NULL, &nr, &b, &L, res);
            double *o = out + (size_t)NPIX * k;
            o[O_R] = res[0];
            o[O_G] = res[1];
            o[O_B] = res[2];
            o[O_DEPTH] = res[3];
            o[O_DEPTH01] = res[4];
            o[O_TF] = L.Tf;
            o[O_NCONTRIB] = (double)L.m;
            o[O_ACC] = res[5];
            o[O_MARGIN] = L.margin;
            o[O_GMARGIN] = L.gmargin;
            o[O_TIE] = L.tie;
            o[O_NCAND] = (double)L.ncand;
            o[O_DSUM] = res[6];
            o[O_NITER] = (double)L.niter;
            o[O_NNEAR] = (double)nr.n;
        }
        pixbuf_free(&b);
    }
    bins_free(&bins);
    free(vis);
    free(P);
    return 0;
}

int oracle_nbranch(void) { return NBR; }
int oracle_nbf(void) { return NBF; }

/* Every branch of the listed pixels: out[k][b][NBF] for b < NBR. Branch b
 * takes near decision i the other way when bit i of b is set; B_VALID is 1
 * for the 2^k branches of a pixel with k <= NEAR_MAX near decisions (branch
 * 0 alone when it has more). */
int oracle_render_branches(int64_t n, const double *means, const double *ls, const double *quats,
                           const double *ologits, const double *sh, int deg, const double *med, const double *cam,
                           int64_t npix, const int64_t *pix, double near_rel, int bin, double *out, int nthreads)
{
    if (n < 0 || deg < 0 || deg > 3 || npix < 0 || (npix > 0 && !pix)) return -1;
    cam_t c;
    cam_load(cam, &c);
    pg_t *P = (pg_t *)malloc(sizeof(pg_t) * (size_t)(n > 0 ? n : 1));
    if (!P) return -2;
    project_all(&c, n, means, ls, quats, ologits, sh, deg, med, P, nthreads);
    int64_t nvis;
    int64_t *vis = visible_ids(P, n, &nvis);
    bins_t bins;
    if (bins_build(P, vis, nvis, &c, bin, near_rel, &bins) != 0) return -2;
    memset(out, 0, sizeof(double) * (size_t)npix * NBR * NBF);
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    {
        pixbuf_t b = {0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t k = 0; k < npix; k++) {
            plist_t L;
            near_t nr = {near_rel, 0, {{0, 0}}};
            double res[7];
            const int64_t *ids;
            int64_t nids;
            pixel_candidates(&bins, vis, nvis, &c, pix[k], &ids, &nids);
            render_pixel(P, ids, nids, &c, med, pix[k], NULL, &nr, &b, &L, res);
            const int64_t nb = nr.n <= NEAR_MAX ? ((int64_t)1 << nr.n) : 1;
            for (int64_t br = 0; br < nb; br++) {
                flips_t fl;
                branch_flips(&nr, br, &fl);
                render_pixel(P, ids, nids, &c, med, pix[k], &fl, NULL, &b, &L, res);
                double *o = out + ((size_t)k * NBR + (size_t)br) * NBF;
                o[B_R] = res[0];
                o[B_G] = res[1];
                o[B_B] = res[2];
                o[B_DEPTH] = res[3];
                o[B_DEPTH01] = res[4];
                o[B_TF] = L.Tf;
                o[B_NCONTRIB] = (double)L.m;
                o[B_VALID] = 1.0;
            }
        }
        pixbuf_free(&b);
    }
    bins_free(&bins);
    free(vis);
    free(P);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Backward: the adjoint of the definition above, in FP64.               */

/* per-Gaussian accumulators of the pixel pass */
enum { G_X, G_Y, G_KA, G_KB, G_KC, G_OP, G_COL, G_D = G_COL + 3, NGP };

int oracle_ngproj(void) { return NGP; }

static void atomic_add(double *p, double v)
{
#ifdef _OPENMP
#pragma omp atomic
#endif
    *p += v;
}

/* Adjoint of one pixel. G[0..2] = dL/dC, G[3] = dL/dz, G[4] = dL/dz01.
 * Accumulates into gp (per Gaussian) and gmed (9 medium parameters). */
static void pixel_backward(const pg_t *P, const contrib_t *lst, int64_t m, double Tf, const double *med, double zfar,
                           const double *G, double *gp, double *gmed)
{
    if (m == 0) {
        /* pure water: C = B_inf (1 - e^{-beta_B zfar}) */
        for (int ch = 0; ch < 3; ch++) {
            const double bf = exp(-med[3 + ch] * zfar);
            gmed[6 + ch] += G[ch] * (1.0 - bf);
            gmed[3 + ch] += G[ch] * med[6 + ch] * zfar * bf;
        }
        return;
    }
    double *T = (double *)malloc(sizeof(double) * (size_t)(m + 2)); /* T[k], k = 1..m+1 */
    double *bb = (double *)malloc(sizeof(double) * 3 * (size_t)(m + 2)); /* b_k per channel, k = 0..m+1 */
    for (int64_t k = 1; k <= m; k++) T[k] = lst[k - 1].T;
    T[m + 1] = Tf;
    for (int ch = 0; ch < 3; ch++) {
        bb[ch] = 1.0;
        for (int64_t k = 1; k <= m; k++) bb[3 * k + ch] = exp(-med[3 + ch] * P[lst[k - 1].id].d);
        bb[3 * (m + 1) + ch] = exp(-med[3 + ch] * zfar);
    }
    /* depth: z = D / A */
    double D = 0, A = 0;
    for (int64_t k = 1; k <= m; k++) {
        D += P[lst[k - 1].id].d * lst[k - 1].alpha * T[k];
        A += lst[k - 1].alpha * T[k];
    }
    double gD = 0, gA = 0;
    if (A > 0) {
        const double z = D / A, e = exp(-0.1 * z);
        const double gz = G[3] + G[4] * 0.2 * e / ((1 + e) * (1 + e));
        gD = gz / A;
        gA = -gz * D / (A * A);
    }
    /* medium: B_inf over all segments; beta_B through b_far */
    for (int ch = 0; ch < 3; ch++) {
        double segs = 0;
        for (int64_t k = 1; k <= m + 1; k++) segs += T[k] * (bb[3 * (k - 1) + ch] - bb[3 * k + ch]);
        gmed[6 + ch] += G[ch] * segs;
        const double bf = bb[3 * (m + 1) + ch];
        gmed[3 + ch] += G[ch] * (-med[6 + ch] * T[m + 1]) * (-zfar * bf);
    }
    for (int64_t i = 1; i <= m; i++) {
        const contrib_t *ci = &lst[i - 1];
        const pg_t *gi = &P[ci->id];
        double *gpi = gp + (size_t)NGP * ci->id;
        const double al = ci->alpha, Ti = T[i];
        /* sums over everything behind i, with T_k stripped of its (1 - alpha_i) factor */
        double S[3] = {0, 0, 0}, Sb[3] = {0, 0, 0}, SD = 0, SA = 0, Pk = Ti;
        for (int64_t k = i + 1; k <= m + 1; k++) {
            if (k <= m) {
                const contrib_t *ck = &lst[k - 1];
                const pg_t *gk = &P[ck->id];
                for (int ch = 0; ch < 3; ch++) S[ch] += gk->col[ch] * gk->a[ch] * ck->alpha * Pk;
                SD += gk->d * ck->alpha * Pk;
                SA += ck->alpha * Pk;
            }
            for (int ch = 0; ch < 3; ch++) Sb[ch] += Pk * (bb[3 * (k - 1) + ch] - bb[3 * k + ch]);
            if (k <= m) Pk *= 1.0 - lst[k - 1].alpha;
        }
        double galpha = 0, gd = 0;
        for (int ch = 0; ch < 3; ch++) {
            const double dCda = gi->col[ch] * gi->a[ch] * Ti - S[ch] - med[6 + ch] * Sb[ch];
            galpha += G[ch] * dCda;
            /* colour and attenuation of the direct signal */
            atomic_add(&gpi[G_COL + ch], G[ch] * gi->a[ch] * al * Ti);
            const double gaa = G[ch] * gi->col[ch] * al * Ti; /* dL/da_i */
            gmed[ch] += gaa * (-gi->d * gi->a[ch]);
            gd += gaa * (-med[ch] * gi->a[ch]);
            /* b_i borders water segments i (-T_i) and i+1 (+T_{i+1}) */
            const double gbb = G[ch] * med[6 + ch] * (T[i + 1] - T[i]);
            gmed[3 + ch] += gbb * (-gi->d * bb[3 * i + ch]);
            gd += gbb * (-med[3 + ch] * bb[3 * i + ch]);
        }
        galpha += gD * (gi->d * Ti - SD) + gA * (Ti - SA);
        gd += gD * al * Ti;
        atomic_add(&gpi[G_D], gd);
        /* alpha = min(0.99, opac e^{-q/2}) */
        if (ci->araw < A_MAX) {
            const double e = exp(-0.5 * ci->q);
            atomic_add(&gpi[G_OP], galpha * e);
            const double gq = galpha * (-0.5 * al);
            const double dx = ci->dx, dy = ci->dy;
            atomic_add(&gpi[G_KA], gq * dx * dx);
            atomic_add(&gpi[G_KB], gq * 2.0 * dx * dy);
            atomic_add(&gpi[G_KC], gq * dy * dy);
            /* dx = px - x: dq/dx = -(2 K0 dx + 2 K1 dy) */
            atomic_add(&gpi[G_X], gq * -(2.0 * gi->K[0] * dx + 2.0 * gi->K[1] * dy));
            atomic_add(&gpi[G_Y], gq * -(2.0 * gi->K[1] * dx + 2.0 * gi->K[2] * dy));
        }
    }
    free(T);
    free(bb);
}

/* Chain one Gaussian's projected-space gradient back to its parameters. */
static void gaussian_backward(const cam_t *c, const pg_t *g, const double *gp, const double *sh, int deg, double ologit,
                              double *gmu, double *gls, double *gq, double *go, double *gsh)
{
    const int K = (deg + 1) * (deg + 1);
    (void)ologit;
    /* opacity */
    *go = gp[G_OP] * g->opac * (1.0 - g->opac);
    /* colour = max(0, sum_k sh_k Y_k(dir) + 0.5) */
    double graw[3], gdir[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) graw[ch] = g->raw[ch] > 0 ? gp[G_COL + ch] : 0.0;
    for (int k = 0; k < K; k++)
        for (int ch = 0; ch < 3; ch++) {
            gsh[3 * k + ch] = graw[ch] * g->Y[k];
            for (int j = 0; j < 3; j++) gdir[j] += graw[ch] * sh[3 * k + ch] * g->dY[k][j];
        }
    const double dg = g->dir[0] * gdir[0] + g->dir[1] * gdir[1] + g->dir[2] * gdir[2];
    for (int j = 0; j < 3; j++) gmu[j] = (gdir[j] - g->dir[j] * dg) / g->vn;

    /* conic -> 2D covariance: dL/dSigma2 = -K (dL/dK) K, symmetric convention */
    const double Km[4] = {g->K[0], g->K[1], g->K[1], g->K[2]};
    const double Gk[4] = {gp[G_KA], 0.5 * gp[G_KB], 0.5 * gp[G_KB], gp[G_KC]};
    double tmp[4], GS[4];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) tmp[2 * a + b] = Km[2 * a] * Gk[b] + Km[2 * a + 1] * Gk[2 + b];
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) GS[2 * a + b] = -(tmp[2 * a] * Km[b] + tmp[2 * a + 1] * Km[2 + b]);
    /* Sigma2 = U Sigma3 U^T (+ dilation), U = J W */
    double G3[9], GU[6];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) acc += g->U[3 * a + i] * GS[2 * a + b] * g->U[3 * b + j];
            G3[3 * i + j] = acc;
        }
    /* dL/dU = 2 GS U Sigma3 (GS and Sigma3 symmetric) */
    for (int a = 0; a < 2; a++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int b = 0; b < 2; b++)
                for (int i = 0; i < 3; i++) acc += 2.0 * GS[2 * a + b] * g->U[3 * b + i] * g->S3[3 * i + j];
            GU[3 * a + j] = acc;
        }
    double GJ[6];
    for (int a = 0; a < 2; a++)
        for (int k = 0; k < 3; k++) {
            double acc = 0;
            for (int j = 0; j < 3; j++) acc += GU[3 * a + j] * c->R[3 * k + j];
            GJ[3 * a + k] = acc;
        }
    const double tx = g->t[0], ty = g->t[1], tz = g->t[2];
    double gt[3] = {0, 0, 0};
    gt[2] += GJ[0] * (-c->fx / (tz * tz)) + GJ[4] * (-c->fy / (tz * tz));
    if (g->clx == 0) {
        gt[0] += GJ[2] * (-c->fx / (tz * tz));
        gt[2] += GJ[2] * (2.0 * c->fx * tx / (tz * tz * tz));
    } else {
        gt[2] += GJ[2] * (c->fx * g->rxc / (tz * tz));
    }
    if (g->cly == 0) {
        gt[1] += GJ[5] * (-c->fy / (tz * tz));
        gt[2] += GJ[5] * (2.0 * c->fy * ty / (tz * tz * tz));
    } else {
        gt[2] += GJ[5] * (c->fy * g->ryc / (tz * tz));
    }
    /* Sigma3 = M M^T, M = Rq diag(s) */
    double GM[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += 2.0 * G3[3 * i + k] * g->Rq[3 * k + j] * g->s[j];
            GM[3 * i + j] = acc;
        }
    double GR[9];
    for (int j = 0; j < 3; j++) {
        double acc = 0;
        for (int i = 0; i < 3; i++) {
            acc += GM[3 * i + j] * g->Rq[3 * i + j];
            GR[3 * i + j] = GM[3 * i + j] * g->s[j];
        }
        gls[j] = acc * g->s[j];
    }
    double dR[4][9], gu[4];
    quat_rot_grad(g->u, dR);
    for (int k = 0; k < 4; k++) {
        double acc = 0;
        for (int e = 0; e < 9; e++) acc += GR[e] * dR[k][e];
        gu[k] = acc;
    }
    const double ug = g->u[0] * gu[0] + g->u[1] * gu[1] + g->u[2] * gu[2] + g->u[3] * gu[3];
    for (int k = 0; k < 4; k++) gq[k] = (gu[k] - g->u[k] * ug) / g->qn;
    /* projected centre and depth */
    gt[0] += gp[G_X] * c->fx / tz;
    gt[2] += gp[G_X] * (-c->fx * tx / (tz * tz));
    gt[1] += gp[G_Y] * c->fy / tz;
    gt[2] += gp[G_Y] * (-c->fy * ty / (tz * tz));
    gt[2] += gp[G_D];
    /* t = W mu + t0 */
    for (int j = 0; j < 3; j++) gmu[j] += c->R[j] * gt[0] + c->R[3 + j] * gt[1] + c->R[6 + j] * gt[2];
}

int oracle_backward(int64_t n, const double *means, const double *ls, const double *quats, const double *ologits,
                    const double *sh, int deg, const double *med, const double *cam, int64_t npix,
                    const int64_t *pix, const double *gout, const int64_t *branch, double near_rel, int bin,
                    double *g_means, double *g_ls, double *g_quats, double *g_ologits, double *g_sh, double *g_med,
                    double *g_proj, int nthreads)
{
    if (n < 0 || deg < 0 || deg > 3) return -1;
    cam_t c;
    cam_load(cam, &c);
    if (!pix) npix = (int64_t)c.W * c.H;
    const int K = (deg + 1) * (deg + 1);
    pg_t *P = (pg_t *)malloc(sizeof(pg_t) * (size_t)(n > 0 ? n : 1));
    double *gp = (double *)calloc((size_t)NGP * (size_t)(n > 0 ? n : 1), sizeof(double));
    if (!P || !gp) return -2;
    project_all(&c, n, means, ls, quats, ologits, sh, deg, med, P, nthreads);
    int64_t nvis;
    int64_t *vis = visible_ids(P, n, &nvis);
    bins_t bins;
    if (bins_build(P, vis, nvis, &c, bin, near_rel, &bins) != 0) return -2;
    double gmed_total[9] = {0};
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    {
        scratch_t s = {0};
        double gmed[9] = {0};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t k = 0; k < npix; k++) {
            const double *G = gout + 5 * k;
            if (G[0] == 0 && G[1] == 0 && G[2] == 0 && G[3] == 0 && G[4] == 0) continue;
            const int64_t p = pix ? pix[k] : k;
            const double px = (double)(p % c.W) + 0.5, py = (double)(p / c.W) + 0.5;
            plist_t L;
            const int64_t br = branch ? branch[k] : 0;
            const int64_t *ids;
            int64_t nids;
            pixel_candidates(&bins, vis, nvis, &c, p, &ids, &nids);
            if (br == 0) {
                pixel_list(P, ids, nids, px, py, &s, &L, NULL, NULL);
            } else {
                /* the branch's flips name near decisions of the FP64 walk */
                near_t nr = {near_rel, 0, {{0, 0}}};
                flips_t fl;
                pixel_list(P, ids, nids, px, py, &s, &L, NULL, &nr);
                branch_flips(&nr, br, &fl);
                pixel_list(P, ids, nids, px, py, &s, &L, &fl, NULL);
            }
            pixel_backward(P, s.lst, L.m, L.Tf, med, c.zfar, G, gp, gmed);
        }
#ifdef _OPENMP
#pragma omp critical
#endif
        for (int j = 0; j < 9; j++) gmed_total[j] += gmed[j];
        free(s.cand);
        free(s.lst);
    }
    for (int j = 0; j < 9; j++) g_med[j] = gmed_total[j];
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
#endif
    for (int64_t i = 0; i < n; i++) {
        double *gmu = g_means + 3 * i, *gl = g_ls + 3 * i, *gqq = g_quats + 4 * i, *gs = g_sh + 3 * K * i;
        const double *gpi = gp + (size_t)NGP * i;
        int any = 0;
        for (int j = 0; j < NGP; j++) any |= gpi[j] != 0.0;
        if (!P[i].vis || !any) {
            memset(gmu, 0, 3 * sizeof(double));
            memset(gl, 0, 3 * sizeof(double));
            memset(gqq, 0, 4 * sizeof(double));
            memset(gs, 0, 3 * (size_t)K * sizeof(double));
            g_ologits[i] = 0;
            continue;
        }
        gaussian_backward(&c, &P[i], gpi, sh + 3 * K * i, deg, ologits[i], gmu, gl, gqq, &g_ologits[i], gs);
    }
    if (g_proj) memcpy(g_proj, gp, sizeof(double) * (size_t)NGP * (size_t)n);
    bins_free(&bins);
    free(vis);
    free(gp);
    free(P);
    return 0;
}
