/*
 * fgs_oracle.c -- plain FP64 CPU oracle for one 3D Gaussian Splatting
 * optimisation step as Faster-GS (arXiv 2602.09999) describes it.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path, and the CUDA path
 * never calls it.
 *
 * Every value is computed in double precision from float32 inputs promoted
 * to double, so the oracle gives the exact-arithmetic result (up to double
 * rounding) for the very inputs the GPU path receives.  Loops follow the
 * definitions in the paper's order; there is no blocking or fusion beyond
 * what those definitions state.  OpenMP only splits independent outputs
 * (pixels, tiles, Gaussians) over threads; every floating-point sum runs
 * in a fixed order, so results do not depend on the thread count.
 *
 * Conventions (readings of the paper where it is silent):
 *  - quaternions are (w, x, y, z), Hamilton, normalised before use (Sec. 2.1)
 *  - camera axes are OpenCV (x right, y down, z forward); R is world->camera
 *  - pixel (u, v) is evaluated at its centre (u + 0.5, v + 0.5)
 *  - tiles are 16 x 16 pixels (Sec. 3.1)
 *  - SH are real, orthonormal, with the Condon-Shortley phase; coefficient
 *    k = l*l + l + m; sh_dc holds k = 0, sh_rest holds k = 1..15, [n,15,3]
 *  - colour = max(0, SH(dir) + 0.5) per channel (Sec. 2.1 "clipped to be
 *    positive"; the 0.5 offset is the 3DGS convention)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TILE 16
#define ORC_ALPHA_MIN (1.0 / 255.0)  /* tau_alpha, Sec. 3.2 "Splat Bounding" */
#define ORC_ALPHA_MAX 0.99           /* alpha clamp, Suppl. B.1 */
#define ORC_T_MIN 1e-4               /* early-stop transmittance, Suppl. B.1 */
#define ORC_QNORM_MIN 1e-4           /* degenerate quaternion, Suppl. B.1 */
#define ORC_DET_MIN 1e-6             /* degenerate 2D covariance, Suppl. B.1 */
#define ORC_DILATION 0.3             /* 2D low-pass filter, Suppl. C Eq. original_2dfilter */

typedef struct {
    double R[9];        /* world -> camera rotation, row-major */
    double t[3];        /* world -> camera translation */
    double fx, fy, cx, cy;
    int32_t width, height;
    double near_plane;
    double cam_pos[3];  /* camera centre in world space (for SH directions) */
    double time;        /* timestamp of the view (dynamic Gaussians) */
} orc_camera;

/* Dynamic Gaussians (Sec. 3.4, the conditional Gaussian in its
 * linear-velocity form): at time t the mean is mu + v (t - t0) and the
 * opacity is multiplied by the temporal marginal exp(-(t - t0)^2 /
 * (2 sigma_t^2)).  NULL (or velocity NULL) for static Gaussians. */
typedef struct {
    const double *velocity;  /* [n,3] */
    const double *t0;        /* [n] */
    double sigma_t;
} orc_motion;

/* Decision margins used to flag results that float32 may legitimately
 * decide the other way (all zero = pure FP64 decisions, nothing flagged). */
typedef struct {
    double rel;        /* relative margin for scalar threshold tests */
    double q_rel;      /* rounding of a quadratic form, relative to its error scale */
    double pos_rel;    /* error of mu2D relative to max(1, |mu2D|) (pixels) */
    double px;         /* absolute margin (pixels) for rectangle edges */
    double t_rel;      /* relative margin for the transmittance stop test */
    double depth_rel;  /* relative depth difference treated as a tie */
    double value_tol;  /* a pixel is flagged only if taking such a decision the other way
                          can move its value by more than this (0: any such decision) */
    int32_t tile_culling; /* 1: per-tile culling (Sec. 3.2); 0: whole rectangle */
} orc_margins;

/* per-Gaussian status bits */
#define ORC_VISIBLE 1
#define ORC_MARGINAL 2
/* per-instance flag bits */
#define ORC_KEEP 1
#define ORC_IMARGINAL 2

/* ---------------------------------------------------------------------- */
/* Spherical harmonics, degree <= 3                                        */
/* ---------------------------------------------------------------------- */

/* Real orthonormal SH with the Condon-Shortley phase, evaluated at a unit
 * direction d; Y[k] with k = l*l + l + m.  The normalisation constants are
 * the textbook ones written as square roots of rationals over pi. */
static void sh_basis(const double d[3], int degree, double Y[16], double dY[16][3])
{
    const double x = d[0], y = d[1], z = d[2];
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < 16; ++k) {
        Y[k] = 0.0;
        if (dY) dY[k][0] = dY[k][1] = dY[k][2] = 0.0;
    }
    Y[0] = 0.5 * sqrt(1.0 / pi);
    if (degree < 1) return;
    const double c1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (dY) {
        dY[1][1] = -c1;
        dY[2][2] = c1;
        dY[3][0] = -c1;
    }
    if (degree < 2) return;
    const double c2a = 0.5 * sqrt(15.0 / pi);
    const double c2b = 0.25 * sqrt(5.0 / pi);
    const double c2c = 0.25 * sqrt(15.0 / pi);
    /* on the unit sphere 3z^2 - 1 = 2z^2 - x^2 - y^2; the latter form is used */
    Y[4] = c2a * x * y;
    Y[5] = -c2a * y * z;
    Y[6] = c2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -c2a * x * z;
    Y[8] = c2c * (x * x - y * y);
    if (dY) {
        dY[4][0] = c2a * y;  dY[4][1] = c2a * x;
        dY[5][1] = -c2a * z; dY[5][2] = -c2a * y;
        dY[6][0] = -2.0 * c2b * x; dY[6][1] = -2.0 * c2b * y; dY[6][2] = 4.0 * c2b * z;
        dY[7][0] = -c2a * z; dY[7][2] = -c2a * x;
        dY[8][0] = 2.0 * c2c * x; dY[8][1] = -2.0 * c2c * y;
    }
    if (degree < 3) return;
    const double c3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double c3b = 0.5 * sqrt(105.0 / pi);
    const double c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double c3d = 0.25 * sqrt(7.0 / pi);
    const double c3e = 0.25 * sqrt(105.0 / pi);
    /* unit-sphere forms: 5z^2-1 = 4z^2-x^2-y^2 and z(5z^2-3) = z(2z^2-3x^2-3y^2) */
    Y[9] = -c3a * y * (3.0 * x * x - y * y);
    Y[10] = c3b * x * y * z;
    Y[11] = -c3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = c3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -c3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = c3e * z * (x * x - y * y);
    Y[15] = -c3a * x * (x * x - 3.0 * y * y);
    if (dY) {
        dY[9][0] = -c3a * 6.0 * x * y;
        dY[9][1] = -c3a * (3.0 * x * x - 3.0 * y * y);
        dY[10][0] = c3b * y * z; dY[10][1] = c3b * x * z; dY[10][2] = c3b * x * y;
        dY[11][0] = -c3c * (-2.0 * x * y);
        dY[11][1] = -c3c * (4.0 * z * z - x * x - 3.0 * y * y);
        dY[11][2] = -c3c * (8.0 * y * z);
        dY[12][0] = c3d * (-6.0 * x * z);
        dY[12][1] = c3d * (-6.0 * y * z);
        dY[12][2] = c3d * (6.0 * z * z - 3.0 * x * x - 3.0 * y * y);
        dY[13][0] = -c3c * (4.0 * z * z - 3.0 * x * x - y * y);
        dY[13][1] = -c3c * (-2.0 * x * y);
        dY[13][2] = -c3c * (8.0 * x * z);
        dY[14][0] = c3e * 2.0 * x * z; dY[14][1] = -c3e * 2.0 * y * z;
        dY[14][2] = c3e * (x * x - y * y);
        dY[15][0] = -c3a * (3.0 * x * x - 3.0 * y * y);
        dY[15][1] = -c3a * (-6.0 * x * y);
    }
}

/* Exported for tests: Y[16] at unit direction d. */
void orc_sh_basis(const double *d, int degree, double *Y, double *dY)
{
    double dYl[16][3];
    sh_basis(d, degree, Y, dY ? dYl : NULL);
    if (dY)
        for (int k = 0; k < 16; ++k)
            for (int a = 0; a < 3; ++a) dY[3 * k + a] = dYl[k][a];
}

/* ---------------------------------------------------------------------- */
/* Small helpers                                                          */
/* ---------------------------------------------------------------------- */

/* Rotation matrix of a unit quaternion (w, x, y, z), Hamilton convention. */
static void quat_to_rot(const double q[4], double Rq[9])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    Rq[0] = 1.0 - 2.0 * (y * y + z * z);
    Rq[1] = 2.0 * (x * y - w * z);
    Rq[2] = 2.0 * (x * z + w * y);
    Rq[3] = 2.0 * (x * y + w * z);
    Rq[4] = 1.0 - 2.0 * (x * x + z * z);
    Rq[5] = 2.0 * (y * z - w * x);
    Rq[6] = 2.0 * (x * z - w * y);
    Rq[7] = 2.0 * (y * z + w * x);
    Rq[8] = 1.0 - 2.0 * (x * x + y * y);
}

static double sigmoid(double w) { return 1.0 / (1.0 + exp(-w)); }

static int near_threshold(double value, double thr, double rel)
{
    return fabs(value - thr) <= rel * fabs(thr);
}

/* Everything the forward derives for one Gaussian in one view. */
typedef struct {
    int ok;               /* screen quantities computable (tz > 0 etc.) */
    int visible;          /* FP64 decision */
    int marginal;         /* some Gaussian-level decision within margin */
    double t[3];          /* camera-space mean */
    double qhat[4], qnorm;
    double Rq[9], s[3];
    double M[9];          /* Rq * S */
    double Sigma[9];      /* 3D covariance */
    double T2[6];         /* J * Rcam, 2x3 */
    double cov2[3];       /* Sigma2D (a, b, c) undilated */
    double det2;          /* det(Sigma2D), Cauchy-Binet */
    double covd[3];       /* dilated */
    double detd;
    double conic[3];
    double xy[2];
    double o;             /* opacity at the view's time */
    double obase;         /* sigmoid of the logit (o without the temporal factor) */
    double dtime;         /* t - t0 (dynamic Gaussians; 0 otherwise) */
    double vel[3];        /* velocity (dynamic Gaussians; 0 otherwise) */
    double k;             /* 2 ln(255 o) */
    double ext[2];        /* half extents sqrt(k * covd_ii) */
    int rect[4];          /* pixel rect u0, v0, u1, v1 (inclusive) */
    int rect_wide[4];     /* rect widened by the pixel margin */
    int rect_narrow[4];   /* rect narrowed by the pixel margin */
    int narrow_empty;
    double dir[3], dist;  /* view direction for SH */
    double rgb_raw[3];
    double rgb[3];
    uint8_t clamped[3];
    double depth;
} orc_gauss;

/* Eq. 1, Eq. 2, Sec. 2.1 activations, Sec. 3.2 bounds, Suppl. B.1
 * degeneracy tests, Suppl. C dilation.  Computes the per-Gaussian screen
 * state of Gaussian i for one camera. */
static void gauss_forward(const orc_camera *cam, int sh_degree, int64_t i,
                          const double *means, const double *log_scales, const double *quats,
                          const double *opacity_logits, const double *sh_dc, const double *sh_rest,
                          const orc_motion *mo, const orc_margins *mg, orc_gauss *g)
{
    memset(g, 0, sizeof(*g));
    double mu[3] = {means[3 * i], means[3 * i + 1], means[3 * i + 2]};
    double ptime = 1.0;  /* temporal marginal */
    if (mo && mo->velocity) {
        /* conditional mean mu + v (t - t0) and marginal exp(-(t - t0)^2 / (2 sigma_t^2)) */
        g->dtime = cam->time - mo->t0[i];
        for (int a = 0; a < 3; ++a) {
            g->vel[a] = mo->velocity[3 * i + a];
            mu[a] += g->vel[a] * g->dtime;
        }
        ptime = exp(-0.5 * g->dtime * g->dtime / (mo->sigma_t * mo->sigma_t));
    }
    const double *R = cam->R;
    int marginal = 0;
    int visible = 1;

    /* camera-space mean: mu_hat = W (mu, 1) */
    for (int r = 0; r < 3; ++r)
        g->t[r] = R[3 * r] * mu[0] + R[3 * r + 1] * mu[1] + R[3 * r + 2] * mu[2] + cam->t[r];
    const double tx = g->t[0], ty = g->t[1], tz = g->t[2];
    if (near_threshold(tz, cam->near_plane, mg->rel)) marginal = 1;
    if (tz <= cam->near_plane) visible = 0;
    if (tz <= 0.0) { g->ok = 0; g->visible = 0; g->marginal = marginal; return; }

    /* quaternion normalisation and degeneracy */
    double qn = 0.0;
    for (int a = 0; a < 4; ++a) qn += (double)quats[4 * i + a] * (double)quats[4 * i + a];
    qn = sqrt(qn);
    g->qnorm = qn;
    if (near_threshold(qn, ORC_QNORM_MIN, mg->rel)) marginal = 1;
    if (qn < ORC_QNORM_MIN) visible = 0;
    if (qn <= 0.0) { g->ok = 0; g->visible = 0; g->marginal = marginal; return; }
    for (int a = 0; a < 4; ++a) g->qhat[a] = quats[4 * i + a] / qn;
    quat_to_rot(g->qhat, g->Rq);

    /* Sigma = Rq S S^T Rq^T with S = diag(exp(log_scale)) */
    for (int a = 0; a < 3; ++a) g->s[a] = exp((double)log_scales[3 * i + a]);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) g->M[3 * r + c] = g->Rq[3 * r + c] * g->s[c];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += g->M[3 * r + k] * g->M[3 * c + k];
            g->Sigma[3 * r + c] = acc;
        }

    /* Eq. 2: J, T2 = J Rcam, Sigma2D = T2 Sigma T2^T */
    const double J[6] = {cam->fx / tz, 0.0, -cam->fx * tx / (tz * tz),
                         0.0, cam->fy / tz, -cam->fy * ty / (tz * tz)};
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            g->T2[3 * r + c] = J[3 * r] * R[c] + J[3 * r + 1] * R[3 + c] + J[3 * r + 2] * R[6 + c];
    double M2[6]; /* T2 M, so Sigma2D = M2 M2^T */
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 3; ++c)
            M2[3 * r + c] = g->T2[3 * r] * g->M[c] + g->T2[3 * r + 1] * g->M[3 + c] +
                            g->T2[3 * r + 2] * g->M[6 + c];
    g->cov2[0] = M2[0] * M2[0] + M2[1] * M2[1] + M2[2] * M2[2];
    g->cov2[1] = M2[0] * M2[3] + M2[1] * M2[4] + M2[2] * M2[5];
    g->cov2[2] = M2[3] * M2[3] + M2[4] * M2[4] + M2[5] * M2[5];
    /* det(M2 M2^T) = sum of squared 2x2 minors of M2 (Cauchy-Binet) */
    {
        const double m01 = M2[0] * M2[4] - M2[1] * M2[3];
        const double m02 = M2[0] * M2[5] - M2[2] * M2[3];
        const double m12 = M2[1] * M2[5] - M2[2] * M2[4];
        g->det2 = m01 * m01 + m02 * m02 + m12 * m12;
    }
    if (near_threshold(g->det2, ORC_DET_MIN, mg->rel)) marginal = 1;
    if (g->det2 < ORC_DET_MIN) visible = 0;

    /* dilation Sigma2D + 0.3 I and the conic (inverse) */
    g->covd[0] = g->cov2[0] + ORC_DILATION;
    g->covd[1] = g->cov2[1];
    g->covd[2] = g->cov2[2] + ORC_DILATION;
    g->detd = g->det2 + ORC_DILATION * (g->cov2[0] + g->cov2[2]) + ORC_DILATION * ORC_DILATION;
    g->conic[0] = g->covd[2] / g->detd;
    g->conic[1] = -g->covd[1] / g->detd;
    g->conic[2] = g->covd[0] / g->detd;

    /* Eq. 1 */
    g->xy[0] = cam->fx * tx / tz + cam->cx;
    g->xy[1] = cam->fy * ty / tz + cam->cy;

    /* opacity activation (times the temporal marginal); a Gaussian with
     * o < tau_alpha can never reach it */
    g->obase = sigmoid((double)opacity_logits[i]);
    g->o = g->obase * ptime;
    if (near_threshold(g->o, ORC_ALPHA_MIN, mg->rel)) marginal = 1;
    if (g->o < ORC_ALPHA_MIN) visible = 0;
    if (g->o <= ORC_ALPHA_MIN * (1.0 - mg->rel)) { g->ok = 0; g->visible = 0; g->marginal = marginal; return; }

    /* opacity-aware rectangle, Sec. 3.2: radicand * -2 ln(tau_alpha / o) */
    g->k = 2.0 * log(g->o / ORC_ALPHA_MIN);
    if (g->k < 0.0) g->k = 0.0;
    g->ext[0] = sqrt(g->k * g->covd[0]);
    g->ext[1] = sqrt(g->k * g->covd[2]);
    const int dims[2] = {cam->width, cam->height};
    int empty = 0, empty_wide = 0, empty_narrow = 0;
    for (int a = 0; a < 2; ++a) {
        /* pixel centres u + 0.5 inside [mu - ext, mu + ext] */
        const double lo = g->xy[a] - g->ext[a] - 0.5;
        const double hi = g->xy[a] + g->ext[a] - 0.5;
        int p0 = (int)ceil(lo), p1 = (int)floor(hi);
        int w0 = (int)ceil(lo - mg->px), w1 = (int)floor(hi + mg->px);
        int n0 = (int)ceil(lo + mg->px), n1 = (int)floor(hi - mg->px);
        if (p0 < 0) p0 = 0;
        if (p1 > dims[a] - 1) p1 = dims[a] - 1;
        if (w0 < 0) w0 = 0;
        if (w1 > dims[a] - 1) w1 = dims[a] - 1;
        if (n0 < 0) n0 = 0;
        if (n1 > dims[a] - 1) n1 = dims[a] - 1;
        if (p0 > p1) empty = 1;
        if (w0 > w1) empty_wide = 1;
        if (n0 > n1) empty_narrow = 1;
        g->rect[a] = p0; g->rect[2 + a] = p1;
        g->rect_wide[a] = w0; g->rect_wide[2 + a] = w1;
        g->rect_narrow[a] = n0; g->rect_narrow[2 + a] = n1;
    }
    g->narrow_empty = empty_narrow;
    if (empty) visible = 0;

    /* SH colour from the view direction, then +0.5 and clip at zero */
    for (int a = 0; a < 3; ++a) g->dir[a] = mu[a] - cam->cam_pos[a];
    g->dist = sqrt(g->dir[0] * g->dir[0] + g->dir[1] * g->dir[1] + g->dir[2] * g->dir[2]);
    for (int a = 0; a < 3; ++a) g->dir[a] /= g->dist;
    double Y[16];
    sh_basis(g->dir, sh_degree, Y, NULL);
    const int ncoef = (sh_degree + 1) * (sh_degree + 1);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = Y[0] * sh_dc[3 * i + ch];
        for (int kk = 1; kk < ncoef; ++kk) acc += Y[kk] * sh_rest[45 * i + 3 * (kk - 1) + ch];
        g->rgb_raw[ch] = acc + 0.5;
        g->clamped[ch] = g->rgb_raw[ch] < 0.0;
        g->rgb[ch] = g->clamped[ch] ? 0.0 : g->rgb_raw[ch];
    }
    g->depth = tz;
    g->ok = !empty_wide;
    g->visible = visible && g->ok;
    g->marginal = marginal;
}

/* Size of the float32 rounding error of q(d) = d^T C d, C = [[a, b], [b, c]]
 * positive definite, when C is held as its eigenvalues lb >= ls and the
 * angle of its eigenvectors: with u, w the offsets along the eigenvectors of
 * ls and lb, each eigenvalue carries a relative error of a few ulps, which
 * moves the form by that fraction of ls u^2 + lb w^2 = q, and the angle an
 * absolute error of a few ulps (radians), which moves it by that amount times
 * |dq/dangle| = 2 (lb - ls) |u w|.  (Held as the entries a, b, c instead, the
 * error would be a fraction of |a dx^2| + |2 b dx dy| + |c dy^2|, far larger
 * along a needle-like splat, where a c - b^2 cancels.) */
static double form_error_scale(double a, double b, double c, double dx, double dy)
{
    const double half = sqrt(0.25 * (a - c) * (a - c) + b * b);
    const double lb = 0.5 * (a + c) + half;
    const double ls = (a * c - b * b) / lb;
    /* unit eigenvector of lb: (b, lb - a) or (lb - c, b), whichever is longer */
    double ex = b, ey = lb - a;
    if (fabs(lb - c) + fabs(b) > fabs(ex) + fabs(ey)) { ex = lb - c; ey = b; }
    const double nrm = sqrt(ex * ex + ey * ey);
    double w = dx, u = dy;
    if (nrm > 0.0) {
        w = (ex * dx + ey * dy) / nrm;
        u = (ex * dy - ey * dx) / nrm;
    }
    return ls * u * u + lb * w * w + 2.0 * (lb - ls) * fabs(u * w);
}

/* Minimum of q(d) = d^T C d over the box [x0,x1] x [y0,y1] of offsets d,
 * for a positive definite C = [[a, b], [b, c]].  Zero if the origin is
 * inside; otherwise the minimum over the four edges, each a clamped 1D
 * quadratic.  Also returns, at the minimiser, the float32 error scale of the
 * form (form_error_scale) and |C d| (1-norm), its sensitivity to the
 * position of the mean. */
static double box_qmin(double a, double b, double c, double x0, double x1, double y0, double y1,
                       double *mag, double *grad)
{
    if (x0 <= 0.0 && 0.0 <= x1 && y0 <= 0.0 && 0.0 <= y1) { *mag = 0.0; *grad = 0.0; return 0.0; }
    double best = INFINITY, bmag = 0.0, bgrad = 0.0;
    const double xs[2] = {x0, x1}, ys[2] = {y0, y1};
    for (int e = 0; e < 2; ++e) {
        /* edge x = xs[e]: minimise over y */
        double X = xs[e];
        double Yv = -b * X / c;
        if (Yv < y0) Yv = y0;
        if (Yv > y1) Yv = y1;
        double q = a * X * X + 2.0 * b * X * Yv + c * Yv * Yv;
        if (q < best) {
            best = q;
            bmag = form_error_scale(a, b, c, X, Yv);
            bgrad = fabs(a * X + b * Yv) + fabs(b * X + c * Yv);
        }
        /* edge y = ys[e]: minimise over x */
        double Yf = ys[e];
        double Xv = -b * Yf / a;
        if (Xv < x0) Xv = x0;
        if (Xv > x1) Xv = x1;
        q = a * Xv * Xv + 2.0 * b * Xv * Yf + c * Yf * Yf;
        if (q < best) {
            best = q;
            bmag = form_error_scale(a, b, c, Xv, Yf);
            bgrad = fabs(a * Xv + b * Yf) + fabs(b * Xv + c * Yf);
        }
    }
    *mag = bmag;
    *grad = bgrad;
    return best;
}

/* Tile culling (Sec. 3.2 "Tile-based Culling", the per-tile maximum of the
 * Gaussian): a tile is kept iff the minimum of d^T conic d over the box of
 * the tile's pixel centres (clipped to the image) is <= k.
 * Returns instance flags (ORC_KEEP / ORC_IMARGINAL), 0 = not a candidate. */
static int tile_decision(const orc_camera *cam, const orc_gauss *g, const orc_margins *mg,
                         int tx, int ty)
{
    const double x_lo = tx * ORC_TILE + 0.5;
    double x_hi = tx * ORC_TILE + (ORC_TILE - 1) + 0.5;
    if (x_hi > cam->width - 0.5) x_hi = cam->width - 0.5;
    const double y_lo = ty * ORC_TILE + 0.5;
    double y_hi = ty * ORC_TILE + (ORC_TILE - 1) + 0.5;
    if (y_hi > cam->height - 0.5) y_hi = cam->height - 0.5;
    double mag, grad;
    const double qmin = box_qmin(g->conic[0], g->conic[1], g->conic[2], x_lo - g->xy[0],
                                 x_hi - g->xy[0], y_lo - g->xy[1], y_hi - g->xy[1], &mag, &grad);
    const int in_rect = !(g->rect[0] > g->rect[2] || g->rect[1] > g->rect[3]) &&
                        tx >= g->rect[0] / ORC_TILE && tx <= g->rect[2] / ORC_TILE &&
                        ty >= g->rect[1] / ORC_TILE && ty <= g->rect[3] / ORC_TILE;
    const int in_narrow = !g->narrow_empty &&
                          tx >= g->rect_narrow[0] / ORC_TILE && tx <= g->rect_narrow[2] / ORC_TILE &&
                          ty >= g->rect_narrow[1] / ORC_TILE && ty <= g->rect_narrow[3] / ORC_TILE;
    const int keep = g->visible && in_rect && (qmin <= g->k || !mg->tile_culling);
    const double pos_err = mg->pos_rel * fmax(1.0, fmax(fabs(g->xy[0]), fabs(g->xy[1])));
    const double slack = mg->q_rel * mag + mg->rel * g->k + 2.0 * pos_err * grad;
    const int marginal_cull = mg->tile_culling && fabs(qmin - g->k) <= slack;
    const int in_wide = qmin <= g->k + slack || !mg->tile_culling;
    int flags = 0;
    if (keep) flags |= ORC_KEEP;
    if ((g->marginal || marginal_cull || !in_narrow) && in_wide) flags |= ORC_IMARGINAL;
    if (!keep && !(flags & ORC_IMARGINAL)) return 0;
    return flags;
}

/* ---------------------------------------------------------------------- */
/* Forward: preprocessing and instance lists                              */
/* ---------------------------------------------------------------------- */

/* Per-Gaussian screen state for one camera.
 * Outputs (length n or multiples): xy[2n], conic[3n], opac[n], rgb[3n],
 * clamped[3n], depth[n], rect[4n] (pixel rect, inclusive), status[n]
 * (ORC_VISIBLE | ORC_MARGINAL), aux[8n] = (tz, qnorm, det2, o, k, ext_x,
 * ext_y, detd). */
int orc_preprocess(const orc_camera *cam, int64_t n, int sh_degree, const double *means, const double *log_scales, const double *quats, const double *opacity_logits, const double *sh_dc, const double *sh_rest, const orc_motion *mo, const orc_margins *mg, double *xy,
                   double *conic, double *opac, double *rgb, uint8_t *clamped, double *depth,
                   int32_t *rect, int32_t *status, double *aux)
{
    if (sh_degree < 0 || sh_degree > 3) return -1;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_gauss g;
        gauss_forward(cam, sh_degree, i, means, log_scales, quats, opacity_logits, sh_dc, sh_rest,
                      mo, mg, &g);
        xy[2 * i] = g.xy[0]; xy[2 * i + 1] = g.xy[1];
        for (int a = 0; a < 3; ++a) {
            conic[3 * i + a] = g.conic[a];
            rgb[3 * i + a] = g.rgb[a];
            clamped[3 * i + a] = g.clamped[a];
        }
        opac[i] = g.o;
        depth[i] = g.depth;
        for (int a = 0; a < 4; ++a) rect[4 * i + a] = g.ok ? g.rect_wide[a] : -1;
        status[i] = (g.visible ? ORC_VISIBLE : 0) | (g.marginal ? ORC_MARGINAL : 0) | (g.ok ? 4 : 0);
        aux[8 * i + 0] = g.t[2];
        aux[8 * i + 1] = g.qnorm;
        aux[8 * i + 2] = g.det2;
        aux[8 * i + 3] = g.o;
        aux[8 * i + 4] = g.k;
        aux[8 * i + 5] = g.ext[0];
        aux[8 * i + 6] = g.ext[1];
        aux[8 * i + 7] = g.detd;
    }
    return 0;
}

/* Number of candidate (Gaussian, tile) instances per Gaussian: every kept
 * instance plus every instance a float32 evaluation could keep. */
int orc_count_instances(const orc_camera *cam, int64_t n, int sh_degree, const double *means, const double *log_scales, const double *quats, const double *opacity_logits, const double *sh_dc, const double *sh_rest, const orc_motion *mo, const orc_margins *mg,
                        int64_t *counts)
{
    const int tiles_x = (cam->width + ORC_TILE - 1) / ORC_TILE;
    (void)tiles_x;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        orc_gauss g;
        gauss_forward(cam, sh_degree, i, means, log_scales, quats, opacity_logits, sh_dc, sh_rest,
                      mo, mg, &g);
        int64_t cnt = 0;
        if (g.ok && (g.visible || g.marginal)) {
            for (int ty = g.rect_wide[1] / ORC_TILE; ty <= g.rect_wide[3] / ORC_TILE; ++ty)
                for (int tx = g.rect_wide[0] / ORC_TILE; tx <= g.rect_wide[2] / ORC_TILE; ++tx)
                    if (tile_decision(cam, &g, mg, tx, ty)) ++cnt;
        }
        counts[i] = cnt;
    }
    return 0;
}

/* Emits the candidates at offsets[i] in ascending Gaussian id, tiles
 * row-major inside the rectangle: tile id, Gaussian id and flags. */
int orc_emit_instances(const orc_camera *cam, int64_t n, int sh_degree, const double *means, const double *log_scales, const double *quats, const double *opacity_logits, const double *sh_dc, const double *sh_rest, const orc_motion *mo, const orc_margins *mg,
                       const int64_t *offsets, int32_t *tile, int32_t *gid, uint8_t *flags)
{
    const int tiles_x = (cam->width + ORC_TILE - 1) / ORC_TILE;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n; ++i) {
        orc_gauss g;
        gauss_forward(cam, sh_degree, i, means, log_scales, quats, opacity_logits, sh_dc, sh_rest,
                      mo, mg, &g);
        if (!(g.ok && (g.visible || g.marginal))) continue;
        int64_t o = offsets[i];
        for (int ty = g.rect_wide[1] / ORC_TILE; ty <= g.rect_wide[3] / ORC_TILE; ++ty)
            for (int tx = g.rect_wide[0] / ORC_TILE; tx <= g.rect_wide[2] / ORC_TILE; ++tx) {
                const int f = tile_decision(cam, &g, mg, tx, ty);
                if (!f) continue;
                tile[o] = ty * tiles_x + tx;
                gid[o] = (int32_t)i;
                flags[o] = (uint8_t)f;
                ++o;
            }
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Blending (Eq. 3, Eq. 4, Suppl. B.1 clamp and early stop)               */
/* ---------------------------------------------------------------------- */

/* One pixel's walk over an ordered candidate list.  Blends the entries
 * flagged KEEP front to back, with the 3DGS rules: skip power > 0, alpha =
 * min(0.99, o G), skip alpha < 1/255, stop before blending an entry whose
 * T (1 - alpha) would fall below 1e-4.  Returns the number of kept entries
 * up to and including the last blended one, its list index, and flags the
 * pixel where a decision within the margins can move its value by more
 * than mg->value_tol:
 *  - whether entry j is blended (a culling candidate, the alpha >= 1/255
 *    test, a zero exponent): blending it or not changes the pixel by
 *    alpha T_j (c_j - R_j), R_j the colour behind it normalised by the
 *    transmittance behind it, known once the walk is done (later decisions
 *    held fixed);
 *  - the order of two blended entries with tied depths: swapping adjacent
 *    entries changes the pixel by T alpha_1 alpha_2 (c_1 - c_2);
 *  - the stop test, where the tested T (1 - alpha) lies within its float32
 *    error bound of 1e-4.  That bound is relative and grows along the walk:
 *    t_rel, plus (alpha slack + rounding) / (1 - alpha) for every blended
 *    factor 1 - alpha, plus alpha / (1 - alpha) for every uncertain blend
 *    decision before the test (taking one the other way scales all later T
 *    by 1 - alpha or its inverse).  Stopping at entry j instead of going on
 *    loses what the walk blended from j onwards and leaves T_j on the
 *    background: the oracle knows that change once the walk is done.
 *    Going on past the oracle's last test instead adds alpha T (c - bg) of
 *    that entry and at most T (1 - alpha)(1 + bound) times the largest
 *    |c - bg| of the list's later entries.
 * The 0.99 clamp leaves the value continuous; it is flagged only when every
 * decision is (value_tol = 0), for scenes that must avoid kinks.  More than
 * ORC_MAX_EVENTS blend decisions or ORC_MAX_STOPS stop tests near the
 * threshold in one pixel flag it as `hard` (effect not bounded);
 * `allowance` sums the bounded effects. */
#define ORC_MAX_EVENTS 64
#define ORC_MAX_STOPS 16
typedef struct {
    double C[3];
    double T;
    int64_t n_contrib;   /* position among KEEP entries, 1-based; 0 if none */
    int64_t last;        /* list index of the last blended entry, -1 if none */
    int amb;             /* a decision within the margins moves the value by > value_tol */
    int hard;            /* a decision whose effect is not bounded (stop test, overflow) */
    double allowance;    /* sum of the bounded effects of all such decisions */
} orc_pixel;

typedef struct {
    double T0, alpha, c[3], C_after[3], T_after;
} orc_event;

/* a stop test within its error bound: T and C before the entry, its alpha
 * and colour, whether the walk stopped there, and the bound */
typedef struct {
    double T0, alpha, c[3], C_before[3], bound;
    int stopped;
} orc_stop;

static double max_abs_diff3(const double *a, const double *b)
{
    double m = 0.0;
    for (int ch = 0; ch < 3; ++ch) m = fmax(m, fabs(a[ch] - b[ch]));
    return m;
}

/* One list entry at one pixel centre (Eq. 3 with the 3DGS rules): its
 * exponent, o G, alpha = min(0.99, o G), whether FP64 blends it (a kept
 * tile, power <= 0, alpha >= 1/255), the relative float32 error of o G
 * (slack), whether float32 may take the blend decision the other way
 * (uncertain) and whether o G lies within its error of the 0.99 clamp. */
typedef struct {
    double power, oG, alpha, slack;
    int keep, blend, uncertain, near_clamp;
} orc_entry;

static void entry_eval(double px, double py, int32_t g, uint8_t f, const double *xy,
                       const double *conic, const double *opac, const orc_margins *mg,
                       orc_entry *e)
{
    const int keep = f & ORC_KEEP;
    const double dx = px - xy[2 * g], dy = py - xy[2 * g + 1];
    const double qa = conic[3 * g] * dx * dx;
    const double qb = 2.0 * conic[3 * g + 1] * dx * dy;
    const double qc = conic[3 * g + 2] * dy * dy;
    const double power = -0.5 * (qa + qb + qc);
    const double oG = opac[g] * exp(power);
    /* relative float32 error of o G: opacity and exp rounding, the
     * rounding of the form (form_error_scale) and the position error of
     * mu2D */
    const double pos_err = mg->pos_rel * fmax(1.0, fmax(fabs(xy[2 * g]), fabs(xy[2 * g + 1])));
    const double grad = fabs(conic[3 * g] * dx + conic[3 * g + 1] * dy) +
                        fabs(conic[3 * g + 1] * dx + conic[3 * g + 2] * dy);
    const double mag = mg->q_rel > 0.0
                           ? form_error_scale(conic[3 * g], conic[3 * g + 1], conic[3 * g + 2], dx, dy)
                           : 0.0;
    const double slack = mg->rel + 0.5 * mg->q_rel * mag + pos_err * grad;
    /* is whether this entry is blended a decision float32 may take the other way? */
    int uncertain = 0;
    if (!keep || (f & ORC_IMARGINAL)) uncertain |= oG >= ORC_ALPHA_MIN * (1.0 - slack);
    if (keep) {
        uncertain |= fabs(power) <= 0.5 * mg->q_rel * mag + (mg->q_rel > 0.0 ? 1e-12 : 0.0);
        uncertain |= fabs(oG - ORC_ALPHA_MIN) <= ORC_ALPHA_MIN * slack;
    }
    e->power = power;
    e->oG = oG;
    e->alpha = oG < ORC_ALPHA_MAX ? oG : ORC_ALPHA_MAX;
    e->slack = slack;
    e->keep = keep;
    e->blend = keep && power <= 0.0 && e->alpha >= ORC_ALPHA_MIN;
    e->uncertain = uncertain;
    e->near_clamp = keep && fabs(oG - ORC_ALPHA_MAX) <= ORC_ALPHA_MAX * slack;
}

static void pixel_walk(double px, double py, int64_t start, int64_t end, const int32_t *list_gid,
                       const uint8_t *list_flags, const double *xy, const double *conic,
                       const double *opac, const double *rgb, const double *depth, const double *bg,
                       const orc_margins *mg, orc_pixel *out)
{
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int64_t pos = 0, n = 0, last = -1;
    int amb = 0, hard = 0;
    double allowance = 0.0;
    /* relative error bound of T as float32 computes it (zero without margins) */
    double t_err = 0.0;
    const double t_unit = mg->t_rel > 0.0 ? 0x1p-23 : 0.0;
    orc_event ev[ORC_MAX_EVENTS];
    int nev = 0;
    orc_stop st[ORC_MAX_STOPS];
    int nst = 0;
    int64_t j_stop = end;      /* the entry the walk stopped before, end if none */
    double prev_depth = -1.0, prev_T = 0.0, prev_alpha = 0.0;
    const double *prev_c = NULL;
    int have_prev = 0;
    for (int64_t j = start; j < end; ++j) {
        const int32_t g = list_gid[j];
        const uint8_t f = list_flags ? list_flags[j] : ORC_KEEP;
        orc_entry en;
        entry_eval(px, py, g, f, xy, conic, opac, mg, &en);
        if (en.keep) ++pos;
        const int uncertain = en.uncertain;
        const double slack = en.slack;
        /* the clamp: no effect on the value, a kink for derivatives; flagged
         * only when every decision is (value_tol = 0) */
        if (mg->value_tol <= 0.0 && en.near_clamp) amb = 1;
        const double alpha = en.alpha;
        const int blend = en.blend;
        /* this entry's blend decision taken the other way scales T by 1 - a */
        const double a_flip = alpha > ORC_ALPHA_MIN ? alpha : ORC_ALPHA_MIN;
        const double own_flip = uncertain && mg->t_rel > 0.0 ? a_flip / (1.0 - a_flip) : 0.0;
        double test = T;
        if (blend) {
            if (have_prev && fabs(depth[g] - prev_depth) <= mg->depth_rel * fabs(depth[g])) {
                const double effect = prev_T * prev_alpha * alpha * max_abs_diff3(prev_c, rgb + 3 * g);
                allowance += effect;
                if (effect > mg->value_tol || mg->value_tol <= 0.0) amb = 1;
            }
            test = T * (1.0 - alpha);
            const double eps = (alpha * slack + t_unit) / (1.0 - alpha);
            const double bound = mg->t_rel + t_err + eps + own_flip;
            if (fabs(test - ORC_T_MIN) <= ORC_T_MIN * bound) {
                amb = 1;
                if (nst == ORC_MAX_STOPS) {
                    hard = 1;
                } else {
                    orc_stop *sp = &st[nst++];
                    sp->T0 = T;
                    sp->alpha = alpha;
                    sp->bound = bound;
                    sp->stopped = test < ORC_T_MIN;
                    for (int ch = 0; ch < 3; ++ch) {
                        sp->c[ch] = rgb[3 * g + ch];
                        sp->C_before[ch] = C[ch];
                    }
                }
            }
            if (test < ORC_T_MIN) {
                j_stop = j;
                break;
            }
            t_err += eps;
        }
        t_err += own_flip;
        if (uncertain) {
            if (nev == ORC_MAX_EVENTS) {
                amb = hard = 1;
            } else {
                orc_event *e = &ev[nev++];
                e->T0 = T;
                e->alpha = alpha > ORC_ALPHA_MIN ? alpha : ORC_ALPHA_MIN;
                for (int ch = 0; ch < 3; ++ch) {
                    e->c[ch] = rgb[3 * g + ch];
                    e->C_after[ch] = C[ch] + (blend ? alpha * T * rgb[3 * g + ch] : 0.0);
                }
                e->T_after = blend ? test : T;
            }
        }
        if (!blend) continue;
        for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * rgb[3 * g + ch];
        prev_depth = depth[g];
        prev_T = T;
        prev_alpha = alpha;
        prev_c = rgb + 3 * g;
        have_prev = 1;
        T = test;
        n = pos;
        last = j;
    }
    /* effect of taking each uncertain blend decision the other way */
    for (int k = 0; k < nev; ++k) {
        const orc_event *e = &ev[k];
        double R[3];
        for (int ch = 0; ch < 3; ++ch) R[ch] = (C[ch] + T * bg[ch] - e->C_after[ch]) / e->T_after;
        const double effect = e->alpha * e->T0 * max_abs_diff3(e->c, R);
        allowance += effect;
        if (effect > mg->value_tol || mg->value_tol <= 0.0) amb = 1;
    }
    /* effect of each stop test near the threshold going the other way */
    double c_later = -1.0;     /* largest |c - bg| after the stop entry */
    for (int k = 0; k < nst; ++k) {
        const orc_stop *sp = &st[k];
        double effect;
        if (!sp->stopped) {
            effect = 0.0;
            for (int ch = 0; ch < 3; ++ch)
                effect = fmax(effect, fabs(C[ch] + T * bg[ch] - sp->C_before[ch] - sp->T0 * bg[ch]));
        } else {
            if (c_later < 0.0) {
                c_later = 0.0;
                for (int64_t j = j_stop + 1; j < end; ++j) {
                    const uint8_t f = list_flags ? list_flags[j] : ORC_KEEP;
                    if (f & ORC_KEEP) c_later = fmax(c_later, max_abs_diff3(rgb + 3 * list_gid[j], bg));
                }
            }
            effect = sp->alpha * sp->T0 * max_abs_diff3(sp->c, bg) +
                     sp->T0 * (1.0 - sp->alpha) * (1.0 + sp->bound) * c_later;
        }
        allowance += effect;
    }
    for (int ch = 0; ch < 3; ++ch) out->C[ch] = C[ch];
    out->T = T;
    out->n_contrib = n;
    out->last = last;
    out->amb = amb;
    out->hard = hard;
    out->allowance = allowance;
}

/* Tile-based forward.  ranges[2*t], ranges[2*t+1] delimit tile t's entries
 * in list_gid/list_flags (sorted by depth, then Gaussian id).
 * Outputs: image[3,H,W] = C + T bg, T_final[H,W], n_contrib[H,W],
 * last_gid[H,W] (-1 if none), ambiguous[H,W], hard[H,W] and allowance[H,W]
 * (see pixel_walk). */
int orc_blend_forward(int32_t width, int32_t height, const int64_t *ranges,
                      const int32_t *list_gid, const uint8_t *list_flags, const double *xy,
                      const double *conic, const double *opac, const double *rgb,
                      const double *depth, const double *bg, const orc_margins *mg, double *image,
                      double *T_final, int32_t *n_contrib, int32_t *last_gid, uint8_t *ambiguous,
                      uint8_t *hard, double *allowance)
{
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    const int64_t npix = (int64_t)width * height;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        const int u = (int)(p % width), v = (int)(p / width);
        const int t = (v / ORC_TILE) * tiles_x + (u / ORC_TILE);
        orc_pixel r;
        pixel_walk(u + 0.5, v + 0.5, ranges[2 * t], ranges[2 * t + 1], list_gid, list_flags, xy,
                   conic, opac, rgb, depth, bg, mg, &r);
        for (int ch = 0; ch < 3; ++ch) image[ch * npix + p] = r.C[ch] + r.T * bg[ch];
        T_final[p] = r.T;
        n_contrib[p] = (int32_t)r.n_contrib;
        last_gid[p] = r.last >= 0 ? list_gid[r.last] : -1;
        ambiguous[p] = (uint8_t)r.amb;
        hard[p] = (uint8_t)r.hard;
        allowance[p] = r.allowance;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Admissible decision paths of a pixel (a float32 evaluation's results)   */
/* ---------------------------------------------------------------------- */

/* Every result a float32 evaluation of one pixel's walk may legitimately
 * reach.  The pixel's candidates -- the entries FP64 blends and those whose
 * blend decision float32 may take the other way (entry_eval) -- are walked
 * front to back, and the walk branches at each decision float32 may take
 * either way:
 *  - an uncertain blend decision: the entry skipped, or blended with its
 *    FP64 alpha;
 *  - a stop test whose tested T (1 - alpha) lies within its float32 error
 *    bound of 1e-4: stopped before the entry, or the entry blended and on;
 *  - two consecutive candidates with depths tied within depth_rel: both
 *    orders (the sort may order them either way).
 * Every other decision is taken as FP64 takes it.  The error bound of the
 * tested T is pixel_walk's without its flip terms, since each branch takes
 * its decisions explicitly: t_rel plus (alpha slack + 2^-23) / (1 - alpha)
 * for every blended factor.  Each end of a walk is one admissible result:
 * C + T bg, T, and the last blended Gaussian.  One result means every
 * decision of the pixel is determined.  The walk gives up (overflow) beyond
 * max_paths results, or at three consecutive tied candidates. */
typedef struct {
    int32_t gid;
    int uncertain;
    double alpha, slack, depth, c[3];
} orc_cand;

typedef struct {
    orc_cand *seq;
    int64_t m;
    double bg[3];
    double t_rel, t_unit, depth_rel;
    int max_paths, npaths, overflow;
    double *val;  /* max_paths x 5: C + T bg (3), T, last blended Gaussian (-1: none) */
} orc_paths;

static void paths_emit(orc_paths *x, const double C[3], double T, int32_t last)
{
    if (x->npaths >= x->max_paths) {
        x->overflow = 1;
        return;
    }
    double *v = x->val + 5 * x->npaths++;
    for (int ch = 0; ch < 3; ++ch) v[ch] = C[ch] + T * x->bg[ch];
    v[3] = T;
    v[4] = (double)last;
}

static int cand_tied(const orc_paths *x, int64_t a, int64_t b)
{
    return x->depth_rel > 0.0 && fabs(x->seq[a].depth - x->seq[b].depth) <= x->depth_rel * fabs(x->seq[a].depth);
}

static void cand_swap(orc_paths *x, int64_t k)
{
    const orc_cand tmp = x->seq[k];
    x->seq[k] = x->seq[k + 1];
    x->seq[k + 1] = tmp;
}

/* Walks candidates k.. from transmittance T, colour C and the accumulated
 * error bound t_err of T; tie_done: the order of candidates k and k + 1 was
 * already branched on. */
static void paths_walk(orc_paths *x, int64_t k, double T, const double C_in[3], double t_err,
                       int32_t last, int tie_done)
{
    double C[3] = {C_in[0], C_in[1], C_in[2]};
    for (; k < x->m; ++k, tie_done = 0) {
        if (x->overflow) return;
        if (!tie_done && k + 1 < x->m && cand_tied(x, k, k + 1)) {
            if (k + 2 < x->m && (cand_tied(x, k + 1, k + 2) || cand_tied(x, k, k + 2))) {
                x->overflow = 1;
                return;
            }
            cand_swap(x, k);
            paths_walk(x, k, T, C, t_err, last, 1);
            cand_swap(x, k);
            if (x->overflow) return;
        }
        const orc_cand *e = &x->seq[k];
        if (e->uncertain) {
            paths_walk(x, k + 1, T, C, t_err, last, 0);  /* the entry skipped */
            if (x->overflow) return;
        }
        /* the entry blended: first the stop test */
        const double test = T * (1.0 - e->alpha);
        const double eps = (e->alpha * e->slack + x->t_unit) / (1.0 - e->alpha);
        const double bound = x->t_rel + t_err + eps;
        const int near = fabs(test - ORC_T_MIN) <= ORC_T_MIN * bound;
        if (test < ORC_T_MIN || near) {
            paths_emit(x, C, T, last);  /* stopped before the entry */
            if (!near) return;
        }
        for (int ch = 0; ch < 3; ++ch) C[ch] += e->alpha * T * e->c[ch];
        T = test;
        t_err += eps;
        last = e->gid;
    }
    paths_emit(x, C, T, last);
}

/* For every pixel of the tile-based forward (inputs as orc_blend_forward):
 * status[H,W] = 0 when the pixel has one admissible result (every decision
 * determined), 1 when it has several, 2 when their enumeration overflowed
 * (then only pixel_walk's allowance bounds the pixel).  The results of the
 * status-1 pixels are appended to path_pix (pixel index v W + u) and
 * path_val (5 per result, as paths_emit writes them), up to `cap` results in
 * all, in no particular order; *n_out receives the number of results there
 * were (when it exceeds cap, the call must be repeated with a larger cap).
 * Returns -1 when a scratch allocation fails. */
int orc_blend_paths(int32_t width, int32_t height, const int64_t *ranges, const int32_t *list_gid,
                    const uint8_t *list_flags, const double *xy, const double *conic,
                    const double *opac, const double *rgb, const double *depth, const double *bg,
                    const orc_margins *mg, int32_t max_paths, int64_t cap, uint8_t *status,
                    int64_t *n_out, int64_t *path_pix, double *path_val)
{
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    const int tiles_y = (height + ORC_TILE - 1) / ORC_TILE;
    const int64_t npix = (int64_t)width * height;
    int64_t longest = 1;
    for (int64_t t = 0; t < (int64_t)tiles_x * tiles_y; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > longest) longest = ranges[2 * t + 1] - ranges[2 * t];
    int64_t total = 0;
    int failed = 0;
#pragma omp parallel
    {
        orc_cand *seq = (orc_cand *)malloc(sizeof(orc_cand) * (size_t)longest);
        double *val = (double *)malloc(sizeof(double) * 5 * (size_t)(max_paths > 0 ? max_paths : 1));
        if (!seq || !val) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 64)
        for (int64_t p = 0; p < npix; ++p) {
            if (!seq || !val) continue;
            const int u = (int)(p % width), v = (int)(p / width);
            const int t = (v / ORC_TILE) * tiles_x + (u / ORC_TILE);
            const double px = u + 0.5, py = v + 0.5;
            orc_paths x;
            x.seq = seq;
            x.m = 0;
            for (int ch = 0; ch < 3; ++ch) x.bg[ch] = bg[ch];
            x.t_rel = mg->t_rel;
            x.t_unit = mg->t_rel > 0.0 ? 0x1p-23 : 0.0;
            x.depth_rel = mg->depth_rel;
            x.max_paths = max_paths;
            x.npaths = 0;
            x.overflow = 0;
            x.val = val;
            for (int64_t j = ranges[2 * t]; j < ranges[2 * t + 1]; ++j) {
                const int32_t g = list_gid[j];
                orc_entry en;
                entry_eval(px, py, g, list_flags ? list_flags[j] : ORC_KEEP, xy, conic, opac, mg, &en);
                if (!(en.blend || en.uncertain)) continue;
                orc_cand *c = &seq[x.m++];
                c->gid = g;
                c->uncertain = en.uncertain;
                c->alpha = en.alpha;
                c->slack = en.slack;
                c->depth = depth[g];
                for (int ch = 0; ch < 3; ++ch) c->c[ch] = rgb[3 * g + ch];
            }
            const double C0[3] = {0.0, 0.0, 0.0};
            paths_walk(&x, 0, 1.0, C0, 0.0, -1, 0);
            if (x.overflow) {
                status[p] = 2;
            } else if (x.npaths <= 1) {
                status[p] = 0;
            } else {
                status[p] = 1;
                int64_t off;
#pragma omp atomic capture
                {
                    off = total;
                    total += x.npaths;
                }
                for (int k = 0; k < x.npaths && off + k < cap; ++k) {
                    path_pix[off + k] = p;
                    for (int q = 0; q < 5; ++q) path_val[5 * (off + k) + q] = val[5 * k + q];
                }
            }
        }
        free(seq);
        free(val);
    }
    *n_out = total;
    return failed ? -1 : 0;
}

/* Brute-force twin: every pixel walks ONE list holding every visible
 * Gaussian ordered by (depth, id) -- no tiles, no bounds, no culling. */
int orc_blend_brute(int32_t width, int32_t height, int64_t count, const int32_t *order,
                    const double *xy, const double *conic, const double *opac, const double *rgb,
                    const double *depth, const double *bg, double *image, double *T_final,
                    int32_t *last_gid)
{
    const int64_t npix = (int64_t)width * height;
    const orc_margins none = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1};
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < npix; ++p) {
        const int u = (int)(p % width), v = (int)(p / width);
        orc_pixel r;
        pixel_walk(u + 0.5, v + 0.5, 0, count, order, NULL, xy, conic, opac, rgb, depth, bg, &none, &r);
        for (int ch = 0; ch < 3; ++ch) image[ch * npix + p] = r.C[ch] + r.T * bg[ch];
        T_final[p] = r.T;
        last_gid[p] = r.last >= 0 ? order[r.last] : -1;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Blend backward: the exact adjoint of Eq. 4 with the clamp (Suppl. B.1)  */
/* ---------------------------------------------------------------------- */

/* Per pixel, the blended fragments are listed front to back with their
 * alpha_i and T_i; S_i = sum_{j>i} alpha_j T_j c_j + T_final bg is formed
 * by an explicit suffix sum, so no division by (1 - alpha) chains is used.
 *   dC/dc_i     = alpha_i T_i
 *   dC/dalpha_i = T_i c_i - S_i / (1 - alpha_i)
 * alpha_i = min(0.99, o G): zero derivative where the clamp is active.
 *   dalpha/do = G, dalpha/dpower = o G
 *   power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), d = pixel - mu2D
 * Per-instance sums (9 values) are accumulated per tile in pixel order, then
 * summed per Gaussian in list order.  Outputs are accumulated (+=) into
 * dxy[2n], dconic[3n], dopac[n], drgb[3n]. */
int orc_blend_backward(int32_t width, int32_t height, int64_t n_inst, const int64_t *ranges,
                       const int32_t *list_gid, const uint8_t *list_flags, const double *xy,
                       const double *conic, const double *opac, const double *rgb,
                       const double *bg, const double *dL_dimage, double *dxy, double *dconic,
                       double *dopac, double *drgb)
{
    const int tiles_x = (width + ORC_TILE - 1) / ORC_TILE;
    const int tiles_y = (height + ORC_TILE - 1) / ORC_TILE;
    const int64_t npix = (int64_t)width * height;
    double *inst = (double *)calloc((size_t)(n_inst > 0 ? n_inst : 1) * 9, sizeof(double));
    if (!inst) return -2;
    int err = 0;
#pragma omp parallel
    {
        int64_t cap = 0;
        int64_t *fidx = NULL;
        double *fa = NULL, *fT = NULL, *fG = NULL, *fdx = NULL, *fdy = NULL;
        uint8_t *fclamp = NULL;
#pragma omp for schedule(dynamic, 1)
        for (int t = 0; t < tiles_x * tiles_y; ++t) {
            const int64_t start = ranges[2 * t], end = ranges[2 * t + 1];
            const int64_t len = end - start;
            if (len <= 0) continue;
            if (len > cap) {
                cap = len;
                fidx = (int64_t *)realloc(fidx, cap * sizeof(int64_t));
                fa = (double *)realloc(fa, cap * sizeof(double));
                fT = (double *)realloc(fT, cap * sizeof(double));
                fG = (double *)realloc(fG, cap * sizeof(double));
                fdx = (double *)realloc(fdx, cap * sizeof(double));
                fdy = (double *)realloc(fdy, cap * sizeof(double));
                fclamp = (uint8_t *)realloc(fclamp, cap);
                if (!fidx || !fa || !fT || !fG || !fdx || !fdy || !fclamp) {
#pragma omp atomic write
                    err = 1;
                    cap = 0;
                    continue;
                }
            }
            const int tx = t % tiles_x, ty = t / tiles_x;
            for (int v = ty * ORC_TILE; v < ty * ORC_TILE + ORC_TILE && v < height; ++v)
                for (int u = tx * ORC_TILE; u < tx * ORC_TILE + ORC_TILE && u < width; ++u) {
                    const int64_t p = (int64_t)v * width + u;
                    const double px = u + 0.5, py = v + 0.5;
                    /* forward walk, recording the blended fragments */
                    double T = 1.0;
                    int64_t nf = 0;
                    for (int64_t j = start; j < end; ++j) {
                        if (list_flags && !(list_flags[j] & ORC_KEEP)) continue;
                        const int32_t g = list_gid[j];
                        const double dx = px - xy[2 * g], dy = py - xy[2 * g + 1];
                        const double power = -0.5 * (conic[3 * g] * dx * dx +
                                                     2.0 * conic[3 * g + 1] * dx * dy +
                                                     conic[3 * g + 2] * dy * dy);
                        if (power > 0.0) continue;
                        const double G = exp(power);
                        const double oG = opac[g] * G;
                        const double alpha = oG < ORC_ALPHA_MAX ? oG : ORC_ALPHA_MAX;
                        if (alpha < ORC_ALPHA_MIN) continue;
                        const double test = T * (1.0 - alpha);
                        if (test < ORC_T_MIN) break;
                        fidx[nf] = j;
                        fa[nf] = alpha;
                        fT[nf] = T;
                        fG[nf] = G;
                        fdx[nf] = dx;
                        fdy[nf] = dy;
                        fclamp[nf] = oG >= ORC_ALPHA_MAX;
                        ++nf;
                        T = test;
                    }
                    const double gC[3] = {dL_dimage[p], dL_dimage[npix + p], dL_dimage[2 * npix + p]};
                    /* suffix sums S_i, walked back to front */
                    double S[3] = {T * bg[0], T * bg[1], T * bg[2]};
                    for (int64_t f = nf - 1; f >= 0; --f) {
                        const int64_t j = fidx[f];
                        const int32_t g = list_gid[j];
                        double *acc = inst + 9 * j;
                        const double a = fa[f], Ti = fT[f];
                        double dalpha = 0.0;
                        for (int ch = 0; ch < 3; ++ch) {
                            acc[6 + ch] += a * Ti * gC[ch];
                            dalpha += gC[ch] * (Ti * rgb[3 * g + ch] - S[ch] / (1.0 - a));
                        }
                        for (int ch = 0; ch < 3; ++ch) S[ch] += a * Ti * rgb[3 * g + ch];
                        if (fclamp[f]) continue;
                        const double dx = fdx[f], dy = fdy[f];
                        const double dpower = dalpha * opac[g] * fG[f];
                        acc[5] += dalpha * fG[f];                     /* d/d o */
                        acc[2] += dpower * (-0.5 * dx * dx);          /* d/d conic a */
                        acc[3] += dpower * (-dx * dy);                /* d/d conic b */
                        acc[4] += dpower * (-0.5 * dy * dy);          /* d/d conic c */
                        acc[0] += dpower * (conic[3 * g] * dx + conic[3 * g + 1] * dy);     /* mu x */
                        acc[1] += dpower * (conic[3 * g + 1] * dx + conic[3 * g + 2] * dy); /* mu y */
                    }
                }
        }
        free(fidx); free(fa); free(fT); free(fG); free(fdx); free(fdy); free(fclamp);
    }
    if (err) { free(inst); return -2; }
    for (int64_t j = 0; j < n_inst; ++j) {
        const int32_t g = list_gid[j];
        const double *acc = inst + 9 * j;
        dxy[2 * g] += acc[0]; dxy[2 * g + 1] += acc[1];
        dconic[3 * g] += acc[2]; dconic[3 * g + 1] += acc[3]; dconic[3 * g + 2] += acc[4];
        dopac[g] += acc[5];
        drgb[3 * g] += acc[6]; drgb[3 * g + 1] += acc[7]; drgb[3 * g + 2] += acc[8];
    }
    free(inst);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Preprocess backward: chain rule of Eq. 1, Eq. 2, Sigma = R S S^T R^T,    */
/* the dilation, the activations and the SH colour (Sec. 3.2 fused          */
/* activations), accumulated (+=) into the parameter gradients.             */
/* ---------------------------------------------------------------------- */
int orc_preprocess_backward(const orc_camera *cam, int64_t n, int sh_degree, const double *means, const double *log_scales, const double *quats, const double *opacity_logits, const double *sh_dc, const double *sh_rest, const double *dxy, const double *dconic,
                            const double *dopac, const double *drgb, double *g_means,
                            double *g_log_scales, double *g_quats, double *g_opacity,
                            double *g_sh_dc, double *g_sh_rest, const orc_motion *mo,
                            double *g_velocity, double *g_t0)
{
    const orc_margins none = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1};
    const double *R = cam->R;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_gauss g;
        gauss_forward(cam, sh_degree, i, means, log_scales, quats, opacity_logits, sh_dc, sh_rest,
                      mo, &none, &g);
        if (!g.visible) continue;
        const double tx = g.t[0], ty = g.t[1], tz = g.t[2];
        double dmu[3] = {0.0, 0.0, 0.0};
        double dt[3] = {0.0, 0.0, 0.0};

        /* opacity: o = sigmoid(w) p(t): do/dw = o (1 - sigmoid(w)),
         * do/dt0 = o (t - t0) / sigma_t^2 */
        g_opacity[i] += dopac[i] * g.o * (1.0 - g.obase);
        if (mo && mo->velocity) g_t0[i] += dopac[i] * g.o * g.dtime / (mo->sigma_t * mo->sigma_t);

        /* colour: rgb = max(0, sum_k Y_k(dir) sh_k + 0.5) */
        {
            double Y[16], dY[16][3];
            sh_basis(g.dir, sh_degree, Y, dY);
            const int ncoef = (sh_degree + 1) * (sh_degree + 1);
            double ddir[3] = {0.0, 0.0, 0.0};
            for (int ch = 0; ch < 3; ++ch) {
                if (g.clamped[ch]) continue;
                const double gc = drgb[3 * i + ch];
                g_sh_dc[3 * i + ch] += Y[0] * gc;
                for (int kk = 1; kk < ncoef; ++kk) {
                    const double coef = kk == 0 ? 0.0 : sh_rest[45 * i + 3 * (kk - 1) + ch];
                    g_sh_rest[45 * i + 3 * (kk - 1) + ch] += Y[kk] * gc;
                    for (int a = 0; a < 3; ++a) ddir[a] += coef * dY[kk][a] * gc;
                }
            }
            /* dir = v / |v|, v = mu - cam_pos: dv = (I - dir dir^T) ddir / |v| */
            const double dd = ddir[0] * g.dir[0] + ddir[1] * g.dir[1] + ddir[2] * g.dir[2];
            for (int a = 0; a < 3; ++a) dmu[a] += (ddir[a] - g.dir[a] * dd) / g.dist;
        }

        /* Eq. 1: mu2D = (fx tx / tz + cx, fy ty / tz + cy) */
        dt[0] += dxy[2 * i] * cam->fx / tz;
        dt[1] += dxy[2 * i + 1] * cam->fy / tz;
        dt[2] += -dxy[2 * i] * cam->fx * tx / (tz * tz) - dxy[2 * i + 1] * cam->fy * ty / (tz * tz);

        /* conic = inverse(Sigma2D + 0.3 I): dSigma = -conic Gs conic with
         * Gs the full symmetric gradient [[ga, gb/2], [gb/2, gc]] */
        const double ca = g.conic[0], cb = g.conic[1], cc = g.conic[2];
        const double ga = dconic[3 * i], gb = 0.5 * dconic[3 * i + 1], gc2 = dconic[3 * i + 2];
        /* P = conic * Gs */
        const double P00 = ca * ga + cb * gb, P01 = ca * gb + cb * gc2;
        const double P10 = cb * ga + cc * gb, P11 = cb * gb + cc * gc2;
        /* dS = -P * conic (symmetric) */
        const double dS00 = -(P00 * ca + P01 * cb);
        const double dS01 = -(P00 * cb + P01 * cc);
        const double dS11 = -(P10 * cb + P11 * cc);
        const double GS2[4] = {dS00, dS01, dS01, dS11}; /* full 2x2 gradient of Sigma2D */

        /* Sigma2D = T2 Sigma T2^T: dT2 = 2 GS2 T2 Sigma, dSigma = T2^T GS2 T2 */
        double T2S[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                T2S[3 * r + c] = g.T2[3 * r] * g.Sigma[c] + g.T2[3 * r + 1] * g.Sigma[3 + c] +
                                 g.T2[3 * r + 2] * g.Sigma[6 + c];
        double dT2[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                dT2[3 * r + c] = 2.0 * (GS2[2 * r] * T2S[c] + GS2[2 * r + 1] * T2S[3 + c]);
        double dSigma[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int p = 0; p < 2; ++p)
                    for (int q = 0; q < 2; ++q) acc += g.T2[3 * p + r] * GS2[2 * p + q] * g.T2[3 * q + c];
                dSigma[3 * r + c] = acc;
            }

        /* T2 = J Rcam: dJ = dT2 Rcam^T */
        double dJ[6];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c)
                dJ[3 * r + c] = dT2[3 * r] * R[3 * c] + dT2[3 * r + 1] * R[3 * c + 1] +
                                dT2[3 * r + 2] * R[3 * c + 2];
        /* J = [[fx/tz, 0, -fx tx/tz^2], [0, fy/tz, -fy ty/tz^2]] */
        const double tz2 = tz * tz, tz3 = tz2 * tz;
        dt[0] += dJ[2] * (-cam->fx / tz2);
        dt[1] += dJ[5] * (-cam->fy / tz2);
        dt[2] += dJ[0] * (-cam->fx / tz2) + dJ[2] * (2.0 * cam->fx * tx / tz3) +
                 dJ[4] * (-cam->fy / tz2) + dJ[5] * (2.0 * cam->fy * ty / tz3);

        /* t = Rcam mu(t) + tcam; mu(t) = mu + v (t - t0) */
        for (int a = 0; a < 3; ++a) dmu[a] += R[a] * dt[0] + R[3 + a] * dt[1] + R[6 + a] * dt[2];
        for (int a = 0; a < 3; ++a) g_means[3 * i + a] += dmu[a];
        if (mo && mo->velocity)
            for (int a = 0; a < 3; ++a) {
                g_velocity[3 * i + a] += dmu[a] * g.dtime;
                g_t0[i] -= dmu[a] * g.vel[a];
            }

        /* Sigma = M M^T, M = Rq S: dM = 2 dSigma M (dSigma symmetric) */
        double dM[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += (dSigma[3 * r + k] + dSigma[3 * k + r]) * g.M[3 * k + c];
                dM[3 * r + c] = acc;
            }
        double dRq[9];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) dRq[3 * r + c] = dM[3 * r + c] * g.s[c];
        for (int c = 0; c < 3; ++c) {
            double ds = 0.0;
            for (int r = 0; r < 3; ++r) ds += dM[3 * r + c] * g.Rq[3 * r + c];
            g_log_scales[3 * i + c] += ds * g.s[c]; /* s = exp(log s) */
        }
        /* Rq(qhat) -> qhat */
        const double w = g.qhat[0], x = g.qhat[1], y = g.qhat[2], z = g.qhat[3];
        const double *G = dRq;
        double dq[4];
        dq[0] = 2.0 * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
        dq[1] = 2.0 * (y * G[1] + z * G[2] + y * G[3] - 2.0 * x * G[4] - w * G[5] + z * G[6] +
                       w * G[7] - 2.0 * x * G[8]);
        dq[2] = 2.0 * (-2.0 * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] +
                       z * G[7] - 2.0 * y * G[8]);
        dq[3] = 2.0 * (-2.0 * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2.0 * z * G[4] +
                       y * G[5] + x * G[6] + y * G[7]);
        /* normalisation qhat = q / |q| */
        const double qd = w * dq[0] + x * dq[1] + y * dq[2] + z * dq[3];
        for (int a = 0; a < 4; ++a) g_quats[4 * i + a] += (dq[a] - g.qhat[a] * qd) / g.qnorm;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Loss: (1 - lambda) L1 + lambda (1 - SSIM), Suppl. A                      */
/* ---------------------------------------------------------------------- */

/* 1D Gaussian window, sigma 1.5, 11 taps, normalised to sum 1. */
static void ssim_window(double w[11])
{
    double s = 0.0;
    for (int i = 0; i < 11; ++i) {
        const double d = i - 5;
        w[i] = exp(-d * d / (2.0 * 1.5 * 1.5));
        s += w[i];
    }
    for (int i = 0; i < 11; ++i) w[i] /= s;
}

/* Separable 11x11 Gaussian blur of one H x W plane with zero padding. */
static void blur(const double *in, double *tmp, double *out, int H, int W, const double w[11])
{
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = -5; k <= 5; ++k) {
                const int xx = x + k;
                if (xx >= 0 && xx < W) acc += w[k + 5] * in[(int64_t)y * W + xx];
            }
            tmp[(int64_t)y * W + x] = acc;
        }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double acc = 0.0;
            for (int k = -5; k <= 5; ++k) {
                const int yy = y + k;
                if (yy >= 0 && yy < H) acc += w[k + 5] * tmp[(int64_t)yy * W + x];
            }
            out[(int64_t)y * W + x] = acc;
        }
}

/* loss = (1 - lambda) mean|img - tgt| + lambda (1 - mean SSIM), means over
 * the 3 H W values.  SSIM uses local statistics under the 11 x 11 window
 * (sigma 1.5), zero padding, C1 = 0.01^2, C2 = 0.03^2.  dL_dimg[3,H,W] is
 * written (not accumulated), scaled by grad_scale (1/B for a batch mean).
 * d|x|/dx is taken as 0 at x = 0. */
int orc_loss(int32_t H, int32_t W, const double *img, const double *tgt, double lambda,
             double grad_scale, double *loss_out, double *dL_dimg)
{
    const int64_t P = (int64_t)H * W;
    const double inv = 1.0 / (3.0 * (double)P);
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double w[11];
    ssim_window(w);
    double *buf = (double *)malloc(sizeof(double) * P * 13);
    if (!buf) return -2;
    double *x = buf, *y = buf + P, *tmp = buf + 2 * P, *mx = buf + 3 * P, *my = buf + 4 * P,
           *exx = buf + 5 * P, *eyy = buf + 6 * P, *exy = buf + 7 * P, *D0 = buf + 8 * P,
           *D1 = buf + 9 * P, *D2 = buf + 10 * P, *prod = buf + 11 * P, *rowsum = buf + 12 * P;
    double l1 = 0.0, ssim = 0.0;
    for (int ch = 0; ch < 3; ++ch) {
        for (int64_t p = 0; p < P; ++p) {
            x[p] = img[ch * P + p];
            y[p] = tgt[ch * P + p];
        }
        blur(x, tmp, mx, H, W, w);
        blur(y, tmp, my, H, W, w);
        for (int64_t p = 0; p < P; ++p) prod[p] = x[p] * x[p];
        blur(prod, tmp, exx, H, W, w);
        for (int64_t p = 0; p < P; ++p) prod[p] = y[p] * y[p];
        blur(prod, tmp, eyy, H, W, w);
        for (int64_t p = 0; p < P; ++p) prod[p] = x[p] * y[p];
        blur(prod, tmp, exy, H, W, w);
        /* per-pixel SSIM and its partial derivatives w.r.t. mu_x, the
         * variance and the covariance (holding the raw moments fixed) */
#pragma omp parallel for schedule(static)
        for (int yy = 0; yy < H; ++yy) {
            double rs = 0.0;
            for (int xx = 0; xx < W; ++xx) {
                const int64_t p = (int64_t)yy * W + xx;
                const double ux = mx[p], uy = my[p];
                const double vx = exx[p] - ux * ux, vy = eyy[p] - uy * uy, cxy = exy[p] - ux * uy;
                const double n1 = 2.0 * ux * uy + C1, n2 = 2.0 * cxy + C2;
                const double d1 = ux * ux + uy * uy + C1, d2 = vx + vy + C2;
                const double S = (n1 * n2) / (d1 * d2);
                rs += S;
                /* the partials of S = n1 n2 / (d1 d2), none divided by n1 or
                 * n2 (n2 = 2 cov + C2 vanishes where cov = -C2 / 2) */
                const double dS_dux = 2.0 * uy * n2 / (d1 * d2) - 2.0 * ux * S / d1;
                const double dS_dvx = -S / d2;
                const double dS_dcxy = 2.0 * n1 / (d1 * d2);
                /* vx = exx - ux^2 and cxy = exy - ux uy also depend on ux */
                D0[p] = dS_dux + dS_dvx * (-2.0 * ux) + dS_dcxy * (-uy);
                D1[p] = dS_dvx;   /* d/d exx */
                D2[p] = dS_dcxy;  /* d/d exy */
            }
            rowsum[yy] = rs;
        }
        for (int yy = 0; yy < H; ++yy) ssim += rowsum[yy];
        /* dSSIM/dx(p) = (w*D0)(p) + 2 x(p) (w*D1)(p) + y(p) (w*D2)(p) */
        blur(D0, tmp, mx, H, W, w);
        blur(D1, tmp, exx, H, W, w);
        blur(D2, tmp, exy, H, W, w);
        for (int yy = 0; yy < H; ++yy) {
            double rs = 0.0;
            for (int xx = 0; xx < W; ++xx) {
                const int64_t p = (int64_t)yy * W + xx;
                const double diff = x[p] - y[p];
                rs += fabs(diff);
                const double sgn = diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0);
                const double dssim = mx[p] + 2.0 * x[p] * exx[p] + y[p] * exy[p];
                dL_dimg[ch * P + p] =
                    grad_scale * inv * ((1.0 - lambda) * sgn - lambda * dssim);
            }
            l1 += rs;
        }
    }
    *loss_out = (1.0 - lambda) * l1 * inv + lambda * (1.0 - ssim * inv);
    free(buf);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Adam (Suppl. A: beta = (0.9, 0.999), eps = 1e-15; Sec. 3.3 "precisely   */
/* match the behavior of the PyTorch implementation"), step t >= 1.        */
/* ---------------------------------------------------------------------- */
int orc_adam(int64_t n, double *p, const double *g, double *m, double *v, double lr, double b1,
             double b2, double eps, int32_t step)
{
    if (step < 1) return -1;
    const double bc1 = 1.0 - pow(b1, step);
    const double bc2 = 1.0 - pow(b2, step);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        const double mhat = m[i] / bc1;
        const double vhat = v[i] / bc2;
        p[i] -= lr * mhat / (sqrt(vhat) + eps);
    }
    return 0;
}
