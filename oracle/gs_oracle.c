/*
 * gs_oracle.c — FP64 CPU oracle for Gaussian splatting with polynomial kernels
 * (arXiv 2603.18707, "From ex(p) to poly").
 *
 * TEST INFRASTRUCTURE ONLY: it checks the CUDA renderer and times a CPU
 * baseline. The renderer never links or calls it.
 *
 * What the paper defines is written out directly: the kernels (Eq. 1, 2, 6),
 * the culling thresholds (Eq. 3-5, App. B), the anti-aliasing normalisation
 * (Sec. 3.4) and front-to-back compositing (Sec. 2). What the paper takes
 * from 3DGS by citation (Sec. 2: EWA projection, SH colour, the 0.99 alpha
 * clamp, the 1e-4 transmittance stop, the 0.2 near plane, the 1.3 tan(fov/2)
 * Jacobian clamp) is written out the way 3DGS states it.
 *
 * Parity notes: the kernel values, radii, projection special cases,
 * anti-aliasing invariance, compositing and gradients are pinned by tests
 * against closed forms, brute force and finite differences. The fitted f'2 and
 * f3 coefficient VALUES are not printed in the paper: parity unpinned for them
 * (only their structure is pinned).
 */
#include "gs_oracle.h"

#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* Kernel math                                                                */
/* ------------------------------------------------------------------------- */

/* Polynomial order N of each kernel kind (Eq. 2); 0 for the exponential. */
int orc_order(int kind)
{
    switch (kind) {
    case ORC_POLY1: return 1;
    case ORC_POLY2CUT: return 2;
    case ORC_POLY3: return 3;
    default: return 0;
    }
}

/* sum_{i=0}^{N} c_i x^i, the polynomial inside the max of Eq. 2. */
double orc_poly(const double c[4], int order, double x)
{
    double sum = 0.0, xi = 1.0;
    for (int i = 0; i <= order; ++i) {
        sum += c[i] * xi;
        xi *= x;
    }
    return sum;
}

static double poly_deriv(const double c[4], int order, double x)
{
    double sum = 0.0, xi = 1.0;
    for (int i = 1; i <= order; ++i) {
        sum += i * c[i] * xi;
        xi *= x;
    }
    return sum;
}

/* Real roots of c3 x^3 + c2 x^2 + c1 x + c0' = 0 when the Cardano
 * discriminant is negative (three real roots): trigonometric form. */
static int cubic_three_real(double c3, double c2, double c1, double c0, double r[3])
{
    /* depressed cubic t^3 + p t + q with x = t - c2 / (3 c3) */
    double a = c2 / c3, b = c1 / c3, d = c0 / c3;
    double p = b - a * a / 3.0;
    double q = 2.0 * a * a * a / 27.0 - a * b / 3.0 + d;
    if (p >= 0.0) return 0;
    double m = 2.0 * sqrt(-p / 3.0);
    double arg = 3.0 * q / (p * m);
    if (arg > 1.0) arg = 1.0;
    if (arg < -1.0) arg = -1.0;
    double th = acos(arg) / 3.0;
    for (int k = 0; k < 3; ++k)
        r[k] = m * cos(th - 2.0 * M_PI * k / 3.0) - a / 3.0;
    return 3;
}

/*
 * Smallest real root x > 0 of sum c_i x^i = rhs; +INFINITY if there is none.
 * Order 1: Eq. 4 in quadric units (t^2 = (eps - o c0) / (o c1) with
 *          rhs = eps / o), Eq. 5 for rhs = 0.
 * Order 2: App. B quadratic formula.
 * Order 3: App. B Cardano formula (Delta0, Delta1, C, t_f3). Of the two signs
 *          of the inner square root (both yield the same real root) the one
 *          that avoids cancellation is taken. When Delta1^2 - 4 Delta0^3 < 0
 *          the cubic has three real roots and C is complex; the three real
 *          roots are then taken in trigonometric form.
 * "Taking the first root that is real and bigger than 0" (App. B).
 */
double orc_first_root(const double c[4], int order, double rhs)
{
    const double INF = INFINITY;
    double c0 = c[0] - rhs;
    if (order == 1) {
        if (c[1] == 0.0) return INF;
        double x = -c0 / c[1];
        return x > 0.0 ? x : INF;
    }
    if (order == 2) {
        double a = c[2], b = c[1];
        if (a == 0.0) {
            if (b == 0.0) return INF;
            double x = -c0 / b;
            return x > 0.0 ? x : INF;
        }
        double disc = b * b - 4.0 * a * c0;
        /* A discriminant that is negative only by rounding (the tangent f'2
         * fit has a double root) is taken as zero. */
        if (disc < 0.0 && -disc <= 64.0 * 2.220446049250313e-16 * (b * b + fabs(4.0 * a * c0)))
            disc = 0.0;
        if (disc < 0.0) return INF;
        double s = sqrt(disc);
        double r1 = (-b - s) / (2.0 * a);
        double r2 = (-b + s) / (2.0 * a);
        double best = INF;
        if (r1 > 0.0 && r1 < best) best = r1;
        if (r2 > 0.0 && r2 < best) best = r2;
        return best;
    }
    if (order == 3) {
        double c1 = c[1], c2 = c[2], c3 = c[3];
        if (c3 == 0.0) {
            double cc[4] = {c0, c1, c2, 0.0};
            return orc_first_root(cc, 2, 0.0);
        }
        double D0 = c2 * c2 - 3.0 * c3 * c1;
        double D1 = 2.0 * c2 * c2 * c2 - 9.0 * c3 * c2 * c1 + 27.0 * c3 * c3 * c0;
        double disc = D1 * D1 - 4.0 * D0 * D0 * D0;
        if (disc >= 0.0) {
            double s = sqrt(disc);
            double inner = (D1 >= 0.0) ? (D1 + s) / 2.0 : (D1 - s) / 2.0;
            double C = cbrt(inner);
            double x;
            if (C == 0.0)
                x = -c2 / (3.0 * c3); /* triple root */
            else
                x = -(c2 + C + D0 / C) / (3.0 * c3);
            return x > 0.0 ? x : INF;
        }
        double r[3];
        int n = cubic_three_real(c3, c2, c1, c0, r);
        double best = INF;
        for (int k = 0; k < n; ++k)
            if (r[k] > 0.0 && r[k] < best) best = r[k];
        return best;
    }
    return INF;
}

/* x0, the first root of the polynomial itself (eps = 0): the universal
 * support bound of Eq. 5 and App. B, and the cut point of Eq. 6. The
 * exponential never reaches zero: +INFINITY. */
double orc_universal_root(const orc_config *cfg)
{
    int n = orc_order(cfg->kind);
    if (n == 0) return INFINITY;
    return orc_first_root(cfg->c, n, 0.0);
}

/* k(x): Eq. 1 g(x) = exp(-x/2); Eq. 2 f_N(x) = max(sum c_i x^i, 0);
 * Eq. 6 f'_N(x) = sum c_i x^i for x < x0, else 0. */
double orc_kernel(const orc_config *cfg, double x0, double x)
{
    int n = orc_order(cfg->kind);
    if (cfg->kind == ORC_EXP) return exp(-0.5 * x);
    if (cfg->kind == ORC_POLY2CUT) return (x < x0) ? orc_poly(cfg->c, n, x) : 0.0;
    double p = orc_poly(cfg->c, n, x);
    return p > 0.0 ? p : 0.0;
}

/* dk/dx of the kernel above; 0 where the ReLU or the cut is inactive. */
double orc_kernel_deriv(const orc_config *cfg, double x0, double x)
{
    int n = orc_order(cfg->kind);
    if (cfg->kind == ORC_EXP) return -0.5 * exp(-0.5 * x);
    if (cfg->kind == ORC_POLY2CUT) return (x < x0) ? poly_deriv(cfg->c, n, x) : 0.0;
    return orc_poly(cfg->c, n, x) > 0.0 ? poly_deriv(cfg->c, n, x) : 0.0;
}

/*
 * Quadric threshold x_cut beyond which a splat of opacity o contributes
 * nothing; -1 when the splat has no pixel with alpha >= eps at all (culled).
 * Thresholds are in quadric units: the paper's radii t (in sigma) are sqrt(x).
 *   OPACITY, exp:   t_g^2 = 2 ln(o / eps)                  (Eq. 3)
 *   OPACITY, f1:    t_f1^2 = (eps - o c0) / (o c1)          (Eq. 4)
 *   OPACITY, f'2/f3: first root of sum c_i x^i = eps / o    (App. B); for f'2
 *                    also no further than the cut x0 of Eq. 6
 *   UNIVERSAL, poly: x0, the root at eps = 0                (Eq. 5, App. B)
 *   UNIVERSAL, exp:  -2 ln eps, the eps bound at o = 1      (Sec. 3.1, "3.3 sigma")
 *   LEGACY3:         9, the 3-sigma radius of 3DGS          (Sec. 2.1)
 * Only the OPACITY mode culls whole splats (o k(0) < eps).
 */
double orc_xcut(const orc_config *cfg, double x0, double o)
{
    int n = orc_order(cfg->kind);
    if (cfg->cull == ORC_CULL_LEGACY3) return 9.0;
    if (cfg->cull == ORC_CULL_UNIVERSAL) {
        if (cfg->kind == ORC_EXP) return -2.0 * log(cfg->eps);
        return x0;
    }
    double k0 = orc_kernel(cfg, x0, 0.0);
    if (!(o * k0 >= cfg->eps)) return -1.0;
    if (cfg->kind == ORC_EXP) return 2.0 * log(o / cfg->eps);
    if (cfg->kind == ORC_POLY1) return (cfg->eps - o * cfg->c[0]) / (o * cfg->c[1]);
    double r = orc_first_root(cfg->c, n, cfg->eps / o);
    if (cfg->kind == ORC_POLY2CUT && r > x0) r = x0;
    return r;
}

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics (3DGS colour model, degrees 0..3)                 */
/* ------------------------------------------------------------------------- */

/* Real SH basis Y_k(dir) for k < (degree+1)^2 in the order and sign
 * convention 3DGS uses (Condon-Shortley phase); dir must be unit length.
 * Constants are written from their closed forms. Returns the count. */
int orc_sh_basis(int degree, const double dir[3], double *Y)
{
    double x = dir[0], y = dir[1], z = dir[2];
    int k = 0;
    Y[k++] = 0.5 / sqrt(M_PI);
    if (degree < 1) return k;
    double c1 = sqrt(3.0 / (4.0 * M_PI));
    Y[k++] = -c1 * y;
    Y[k++] = c1 * z;
    Y[k++] = -c1 * x;
    if (degree < 2) return k;
    double xx = x * x, yy = y * y, zz = z * z;
    Y[k++] = 0.5 * sqrt(15.0 / M_PI) * x * y;
    Y[k++] = -0.5 * sqrt(15.0 / M_PI) * y * z;
    Y[k++] = 0.25 * sqrt(5.0 / M_PI) * (2.0 * zz - xx - yy);
    Y[k++] = -0.5 * sqrt(15.0 / M_PI) * x * z;
    Y[k++] = 0.25 * sqrt(15.0 / M_PI) * (xx - yy);
    if (degree < 3) return k;
    Y[k++] = -0.25 * sqrt(35.0 / (2.0 * M_PI)) * y * (3.0 * xx - yy);
    Y[k++] = 0.5 * sqrt(105.0 / M_PI) * x * y * z;
    Y[k++] = -0.25 * sqrt(21.0 / (2.0 * M_PI)) * y * (4.0 * zz - xx - yy);
    Y[k++] = 0.25 * sqrt(7.0 / M_PI) * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[k++] = -0.25 * sqrt(21.0 / (2.0 * M_PI)) * x * (4.0 * zz - xx - yy);
    Y[k++] = 0.25 * sqrt(105.0 / M_PI) * z * (xx - yy);
    Y[k++] = -0.25 * sqrt(35.0 / (2.0 * M_PI)) * x * (xx - 3.0 * yy);
    return k;
}

/* Gradient of each basis function with respect to dir (3 per function),
 * differentiated from the closed forms above. */
static void sh_basis_grad(int degree, const double dir[3], double (*G)[3])
{
    double x = dir[0], y = dir[1], z = dir[2];
    int k = 0;
    G[k][0] = G[k][1] = G[k][2] = 0.0; ++k;
    if (degree < 1) return;
    double c1 = sqrt(3.0 / (4.0 * M_PI));
    G[k][0] = 0; G[k][1] = -c1; G[k][2] = 0; ++k;
    G[k][0] = 0; G[k][1] = 0; G[k][2] = c1; ++k;
    G[k][0] = -c1; G[k][1] = 0; G[k][2] = 0; ++k;
    if (degree < 2) return;
    double a = 0.5 * sqrt(15.0 / M_PI), b = 0.25 * sqrt(5.0 / M_PI), e = 0.25 * sqrt(15.0 / M_PI);
    G[k][0] = a * y; G[k][1] = a * x; G[k][2] = 0; ++k;
    G[k][0] = 0; G[k][1] = -a * z; G[k][2] = -a * y; ++k;
    G[k][0] = -2 * b * x; G[k][1] = -2 * b * y; G[k][2] = 4 * b * z; ++k;
    G[k][0] = -a * z; G[k][1] = 0; G[k][2] = -a * x; ++k;
    G[k][0] = 2 * e * x; G[k][1] = -2 * e * y; G[k][2] = 0; ++k;
    if (degree < 3) return;
    double d0 = 0.25 * sqrt(35.0 / (2.0 * M_PI)), d1 = 0.5 * sqrt(105.0 / M_PI);
    double d2 = 0.25 * sqrt(21.0 / (2.0 * M_PI)), d3 = 0.25 * sqrt(7.0 / M_PI);
    double d5 = 0.25 * sqrt(105.0 / M_PI);
    double xx = x * x, yy = y * y, zz = z * z;
    /* -d0 y (3x^2 - y^2) */
    G[k][0] = -d0 * 6 * x * y; G[k][1] = -d0 * (3 * xx - 3 * yy); G[k][2] = 0; ++k;
    /* d1 x y z */
    G[k][0] = d1 * y * z; G[k][1] = d1 * x * z; G[k][2] = d1 * x * y; ++k;
    /* -d2 y (4z^2 - x^2 - y^2) */
    G[k][0] = -d2 * y * (-2 * x); G[k][1] = -d2 * (4 * zz - xx - 3 * yy); G[k][2] = -d2 * y * 8 * z; ++k;
    /* d3 z (2z^2 - 3x^2 - 3y^2) */
    G[k][0] = d3 * z * (-6 * x); G[k][1] = d3 * z * (-6 * y); G[k][2] = d3 * (6 * zz - 3 * xx - 3 * yy); ++k;
    /* -d2 x (4z^2 - x^2 - y^2) */
    G[k][0] = -d2 * (4 * zz - 3 * xx - yy); G[k][1] = -d2 * x * (-2 * y); G[k][2] = -d2 * x * 8 * z; ++k;
    /* d5 z (x^2 - y^2) */
    G[k][0] = d5 * z * 2 * x; G[k][1] = -d5 * z * 2 * y; G[k][2] = d5 * (xx - yy); ++k;
    /* -d0 x (x^2 - 3y^2) */
    G[k][0] = -d0 * (3 * xx - 3 * yy); G[k][1] = -d0 * x * (-6 * y); G[k][2] = 0; ++k;
}

/* ------------------------------------------------------------------------- */
/* Projection                                                                 */
/* ------------------------------------------------------------------------- */

/* Rotation matrix of a unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z); R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y); R[2][1] = 2 * (y * z + w * x); R[2][2] = 1 - 2 * (x * x + y * y);
}

/* Intermediate quantities of one splat's projection, kept for the reverse pass. */
typedef struct {
    double qn[4], qlen, R[3][3], M[3][3], Sigma[3][3];
    double t[3], txc, tyc;
    int clampx, clampy; /* -1, 0, +1: which side of the Jacobian clamp */
    double J[2][3], Tm[2][3];
    double cov[3], a, b, c, det0, det1;
    double campos[3], dir[3], dist;
} proj_state;

static void camera_rotation(const orc_camera *cam, double W[3][3], double tv[3])
{
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) W[i][j] = cam->viewmat[4 * i + j];
        tv[i] = cam->viewmat[4 * i + 3];
    }
}

/*
 * Project splat i (Eq. 1 notation): Sigma = R S S^T R^T, t = W mu + t_cam,
 * Sigma' = J W Sigma W^T J^T (EWA, 3DGS), + v I low-pass (Sec. 3.4),
 * rho = sqrt(|Sigma'| / |Sigma' + v I|) (Sec. 3.4, Eq. 7-9), o' = o rho,
 * conic = (Sigma' + v I)^-1, mu' = (fx tx/tz + cx, fy ty/tz + cy),
 * colour from real SH plus 0.5 clamped at 0 (3DGS), x_cut (Eq. 3-5, App. B)
 * and the tile rectangle around the support ellipse.
 */
static void project_one(int i, const double *means, const double *scales, const double *quats,
                        const double *opacities, const double *sh, int sh_degree,
                        const orc_camera *cam, const orc_config *cfg, double x0,
                        orc_splat2d *o, proj_state *st)
{
    memset(o, 0, sizeof(*o));
    memset(st, 0, sizeof(*st));
    const double *mu = means + 3 * i, *s = scales + 3 * i, *q = quats + 4 * i;
    double W[3][3], tv[3];
    camera_rotation(cam, W, tv);

    /* 3D covariance */
    st->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) st->qn[k] = q[k] / st->qlen;
    quat_to_rot(st->qn, st->R);
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) st->M[r][k] = st->R[r][k] * s[k];
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < 3; ++k) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) acc += st->M[r][m] * st->M[k][m];
            st->Sigma[r][k] = acc;
        }

    /* camera-space mean */
    for (int r = 0; r < 3; ++r) st->t[r] = W[r][0] * mu[0] + W[r][1] * mu[1] + W[r][2] * mu[2] + tv[r];
    o->depth = st->t[2];
    if (!(st->t[2] > cam->znear)) return; /* invisible */
    double tz = st->t[2];

    /* EWA Jacobian at the mean, tx/tz and ty/tz clamped to 1.3 tan(fov/2) */
    double limx = 1.3 * (0.5 * cam->width / cam->fx);
    double limy = 1.3 * (0.5 * cam->height / cam->fy);
    double ux = st->t[0] / tz, uy = st->t[1] / tz;
    st->clampx = (ux < -limx) ? -1 : (ux > limx ? 1 : 0);
    st->clampy = (uy < -limy) ? -1 : (uy > limy ? 1 : 0);
    st->txc = (st->clampx == 0 ? ux : st->clampx * limx) * tz;
    st->tyc = (st->clampy == 0 ? uy : st->clampy * limy) * tz;
    st->J[0][0] = cam->fx / tz; st->J[0][1] = 0.0; st->J[0][2] = -cam->fx * st->txc / (tz * tz);
    st->J[1][0] = 0.0; st->J[1][1] = cam->fy / tz; st->J[1][2] = -cam->fy * st->tyc / (tz * tz);
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            st->Tm[r][k] = st->J[r][0] * W[0][k] + st->J[r][1] * W[1][k] + st->J[r][2] * W[2][k];

    /* Sigma' = Tm Sigma Tm^T */
    double TS[2][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k)
            TS[r][k] = st->Tm[r][0] * st->Sigma[0][k] + st->Tm[r][1] * st->Sigma[1][k] + st->Tm[r][2] * st->Sigma[2][k];
    double S00 = TS[0][0] * st->Tm[0][0] + TS[0][1] * st->Tm[0][1] + TS[0][2] * st->Tm[0][2];
    double S01 = TS[0][0] * st->Tm[1][0] + TS[0][1] * st->Tm[1][1] + TS[0][2] * st->Tm[1][2];
    double S11 = TS[1][0] * st->Tm[1][0] + TS[1][1] * st->Tm[1][1] + TS[1][2] * st->Tm[1][2];
    st->cov[0] = S00; st->cov[1] = S01; st->cov[2] = S11;
    o->cov2d[0] = S00; o->cov2d[1] = S01; o->cov2d[2] = S11;

    /* low-pass and anti-aliasing normalisation */
    st->a = S00 + cfg->dilation; st->b = S01; st->c = S11 + cfg->dilation;
    st->det0 = S00 * S11 - S01 * S01;
    st->det1 = st->a * st->c - st->b * st->b;
    if (!(st->det1 > 0.0)) return;
    o->rho = 1.0;
    if (cfg->aa) o->rho = sqrt((st->det0 > 0.0 ? st->det0 : 0.0) / st->det1);
    o->opacity = opacities[i] * o->rho;
    o->conic[0] = st->c / st->det1;
    o->conic[1] = -st->b / st->det1;
    o->conic[2] = st->a / st->det1;
    o->mean2d[0] = cam->fx * st->t[0] / tz + cam->cx;
    o->mean2d[1] = cam->fy * st->t[1] / tz + cam->cy;

    /* view-dependent colour */
    for (int r = 0; r < 3; ++r) st->campos[r] = -(W[0][r] * tv[0] + W[1][r] * tv[1] + W[2][r] * tv[2]);
    double dv[3] = {mu[0] - st->campos[0], mu[1] - st->campos[1], mu[2] - st->campos[2]};
    st->dist = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int r = 0; r < 3; ++r) st->dir[r] = dv[r] / st->dist;
    double Y[16];
    int K = orc_sh_basis(sh_degree, st->dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += Y[k] * sh[((long long)i * K + k) * 3 + ch];
        o->color_raw[ch] = acc + 0.5;
        o->color[ch] = o->color_raw[ch] > 0.0 ? o->color_raw[ch] : 0.0;
    }

    /* support threshold and tile rectangle */
    o->xcut = orc_xcut(cfg, x0, o->opacity);
    if (o->xcut < 0.0) return; /* culled: no pixel reaches eps */
    o->visible = 1;
    double hx, hy;
    if (cfg->rect_mode == ORC_RECT_CIRCLE) {
        double mid = 0.5 * (st->a + st->c);
        double disc = mid * mid - st->det1;
        double lmax = mid + sqrt(disc > 0.0 ? disc : 0.0);
        hx = hy = sqrt(o->xcut * lmax);
    } else {
        hx = sqrt(o->xcut * st->a);
        hy = sqrt(o->xcut * st->c);
    }
    /* pixel columns whose centre x + 0.5 lies in [mu'x - hx, mu'x + hx] */
    double px0 = ceil(o->mean2d[0] - hx - 0.5), px1 = floor(o->mean2d[0] + hx - 0.5);
    double py0 = ceil(o->mean2d[1] - hy - 0.5), py1 = floor(o->mean2d[1] + hy - 0.5);
    if (px0 < 0) px0 = 0;
    if (py0 < 0) py0 = 0;
    if (px1 > cam->width - 1) px1 = cam->width - 1;
    if (py1 > cam->height - 1) py1 = cam->height - 1;
    if (px0 > px1 || py0 > py1) {
        o->tiles = 0;
        return;
    }
    o->rect[0] = (int)px0 / cfg->tile_w;
    o->rect[1] = (int)py0 / cfg->tile_h;
    o->rect[2] = (int)px1 / cfg->tile_w;
    o->rect[3] = (int)py1 / cfg->tile_h;
    o->tiles = (long long)(o->rect[2] - o->rect[0] + 1) * (o->rect[3] - o->rect[1] + 1);
}

void orc_project(int P, const double *means, const double *scales, const double *quats,
                 const double *opacities, const double *sh, int sh_degree,
                 const orc_camera *cam, const orc_config *cfg, orc_splat2d *out)
{
    double x0 = orc_universal_root(cfg);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < P; ++i) {
        proj_state st;
        project_one(i, means, scales, quats, opacities, sh, sh_degree, cam, cfg, x0, &out[i], &st);
    }
}

/* ------------------------------------------------------------------------- */
/* Compositing                                                                */
/* ------------------------------------------------------------------------- */

static const orc_splat2d *g_sort_s; /* qsort has no context argument */

static int cmp_depth_index(const void *pa, const void *pb)
{
    int a = *(const int *)pa, b = *(const int *)pb;
    double da = g_sort_s[a].depth, db = g_sort_s[b].depth;
    if (da < db) return -1;
    if (da > db) return 1;
    return (a > b) - (a < b);
}

/* Indices of the visible splats ordered by (depth, index). */
static int *sorted_visible(int P, const orc_splat2d *s, int *count)
{
    int *idx = (int *)malloc(sizeof(int) * (P > 0 ? P : 1));
    int n = 0;
    for (int i = 0; i < P; ++i)
        if (s[i].visible) idx[n++] = i;
    g_sort_s = s;
    qsort(idx, n, sizeof(int), cmp_depth_index);
    *count = n;
    return idx;
}

static double quadric(const orc_splat2d *s, double px, double py)
{
    double dx = px - s->mean2d[0], dy = py - s->mean2d[1];
    return s->conic[0] * dx * dx + 2.0 * s->conic[1] * dx * dy + s->conic[2] * dy * dy;
}

/*
 * One pixel, front to back over the given order (Sec. 2): alpha_i =
 * min(alpha_max, o'_i k(Q_i)); entries with alpha_i < eps are skipped; the walk
 * stops at the first entry whose T (1 - alpha) would fall below t_min, without
 * adding it; C = sum c_i alpha_i T_i, output C + T bg.
 * Returns the number of entries evaluated; *last = position + 1 of the last
 * contributing entry (0 if none).
 */
/* Diagnostic scale of the decision margin (pixels): an FP32 renderer holds
 * pixel coordinates up to 4096 to within 2.4e-4 px, so its alphas move as if
 * each splat were shifted by up to that much; 0.3 px times the margin's 1e-3
 * flip band is 3e-4 px. */
#define ORC_MARGIN_PX 0.3

static long long composite_pixel(const orc_splat2d *s, const int *order, long long n,
                                 const orc_config *cfg, double x0, double px, double py,
                                 const double bg[3], double out[3], double *Tout, long long *last,
                                 double *margin)
{
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    long long evaluated = n;
    double m = INFINITY;
    double tsens = 0.0; /* diagnostic: sum of |grad alpha| / (1 - alpha) over blended entries */
    *last = 0;
    for (long long j = 0; j < n; ++j) {
        const orc_splat2d *g = &s[order[j]];
        double Q = quadric(g, px, py);
        double alpha = g->opacity * orc_kernel(cfg, x0, Q);
        /* diagnostic only: distance of this entry's skip decision from its
         * threshold, relative to eps plus the change of alpha over
         * ORC_MARGIN_PX (|grad alpha| = o' |k'(Q)| |grad Q|) */
        double ga = 0.0;
        if (margin) {
            double dx = px - g->mean2d[0], dy = py - g->mean2d[1];
            double hx = g->conic[0] * dx + g->conic[1] * dy, hy = g->conic[1] * dx + g->conic[2] * dy;
            ga = g->opacity * fabs(orc_kernel_deriv(cfg, x0, Q)) * 2.0 * sqrt(hx * hx + hy * hy);
            double me = fabs(alpha - cfg->eps) / (cfg->eps + ORC_MARGIN_PX * ga);
            if (me < m) m = me;
        }
        if (alpha > cfg->alpha_max) alpha = cfg->alpha_max;
        if (alpha < cfg->eps) continue;
        double Tn = T * (1.0 - alpha);
        if (margin) {
            /* the stop decision: against t_min plus the change of T (1 - alpha)
             * over the same shift of this and every earlier blended entry */
            double ms = fabs(Tn - cfg->t_min) / (cfg->t_min + ORC_MARGIN_PX * (T * ga + Tn * tsens));
            if (ms < m) m = ms;
        }
        if (Tn < cfg->t_min) {
            evaluated = j + 1;
            break;
        }
        for (int ch = 0; ch < 3; ++ch) C[ch] += g->color[ch] * alpha * T;
        if (margin) tsens += ga / (1.0 - alpha);
        T = Tn;
        *last = j + 1;
    }
    for (int ch = 0; ch < 3; ++ch) out[ch] = C[ch] + T * bg[ch];
    *Tout = T;
    if (margin) *margin = m;
    return evaluated;
}

/* Untiled, unculled reference: every pixel walks every visible splat. */
void orc_render_untiled(int P, const orc_splat2d *s, const orc_camera *cam,
                        const orc_config *cfg, const double bg[3],
                        double *img, double *final_T, long long *n_contrib)
{
    int n;
    int *order = sorted_visible(P, s, &n);
    double x0 = orc_universal_root(cfg);
    int W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            long long p = (long long)y * W + x, last;
            double T;
            composite_pixel(s, order, n, cfg, x0, x + 0.5, y + 0.5, bg, img + 3 * p, &T, &last, NULL);
            if (final_T) final_T[p] = T;
            if (n_contrib) n_contrib[p] = last;
        }
    free(order);
}

/*
 * Tile-binned render: each tile walks only the splats whose rectangle
 * contains it, in (depth, index) order. With a conservative x_cut this equals
 * the untiled render exactly. tiles_sel lists the tile ids to render
 * (n_tiles_sel < 0: all tiles); pixels of other tiles are left untouched.
 * n_eval: entries evaluated per pixel; list_len: list length per tile;
 * margin (optional, diagnostic): per pixel, the smallest distance of any skip
 * (alpha vs eps) or stop (T (1 - alpha) vs t_min) decision from its
 * threshold, relative to the threshold plus the change the decided quantity
 * undergoes when the splats move by ORC_MARGIN_PX — pixels where a
 * lower-precision renderer may decide otherwise (below 1e-3: within 0.1 % of
 * the threshold, or within 3e-4 px of the boundary).
 */
void orc_render_tiled(int P, const orc_splat2d *s, const orc_camera *cam,
                      const orc_config *cfg, const double bg[3],
                      int n_tiles_sel, const int *tiles_sel,
                      double *img, double *final_T, long long *last_contrib,
                      long long *n_eval, long long *list_len, double *margin)
{
    int n;
    int *order = sorted_visible(P, s, &n);
    double x0 = orc_universal_root(cfg);
    int W = cam->width, H = cam->height;
    int tx = (W + cfg->tile_w - 1) / cfg->tile_w, ty = (H + cfg->tile_h - 1) / cfg->tile_h;
    int nsel = n_tiles_sel < 0 ? tx * ty : n_tiles_sel;
#pragma omp parallel for schedule(dynamic)
    for (int si = 0; si < nsel; ++si) {
        int tile = n_tiles_sel < 0 ? si : tiles_sel[si];
        int gx = tile % tx, gy = tile / tx;
        int *list = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
        long long m = 0;
        for (int j = 0; j < n; ++j) {
            const orc_splat2d *g = &s[order[j]];
            if (g->tiles > 0 && gx >= g->rect[0] && gx <= g->rect[2] && gy >= g->rect[1] && gy <= g->rect[3])
                list[m++] = order[j];
        }
        if (list_len) list_len[tile] = m;
        for (int y = gy * cfg->tile_h; y < (gy + 1) * cfg->tile_h && y < H; ++y)
            for (int x = gx * cfg->tile_w; x < (gx + 1) * cfg->tile_w && x < W; ++x) {
                long long p = (long long)y * W + x, last;
                double T;
                long long ev = composite_pixel(s, list, m, cfg, x0, x + 0.5, y + 0.5, bg, img + 3 * p, &T,
                                               &last, margin ? margin + p : NULL);
                if (final_T) final_T[p] = T;
                if (last_contrib) last_contrib[p] = last;
                if (n_eval) n_eval[p] = ev;
            }
        free(list);
    }
    free(order);
}

void orc_decisions(int P, const orc_splat2d *s, const orc_camera *cam,
                   const orc_config *cfg, unsigned long long *sig)
{
    int n;
    int *order = sorted_visible(P, s, &n);
    double x0 = orc_universal_root(cfg);
    int W = cam->width, H = cam->height;
#pragma omp parallel for schedule(dynamic)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            unsigned long long h = 1469598103934665603ull;
            double T = 1.0;
            for (int j = 0; j < n; ++j) {
                const orc_splat2d *g = &s[order[j]];
                double Q = quadric(g, x + 0.5, y + 0.5);
                double k = orc_kernel(cfg, x0, Q);
                double alpha = g->opacity * k;
                int state = 2;
                if (alpha > cfg->alpha_max) { alpha = cfg->alpha_max; state = 1; }
                if (alpha < cfg->eps) state = 0;
                if (state != 0 && T * (1.0 - alpha) < cfg->t_min) state = 3;
                h = (h ^ (unsigned long long)(order[j] * 8 + state)) * 1099511628211ull;
                if (state == 3) break;
                if (state != 0) T *= (1.0 - alpha);
            }
            sig[(long long)y * W + x] = h;
        }
    free(order);
}

/* ------------------------------------------------------------------------- */
/* Reverse pass                                                               */
/* ------------------------------------------------------------------------- */

/*
 * Analytic gradients of the untiled render with respect to the splat inputs
 * (means, scales, quaternions as given, opacities, SH) and the intermediate 2D
 * quantities. Kinks: ReLU / cut inactive -> 0; alpha clamped -> no gradient to
 * o' k; skipped or stopping entries contribute nothing; colour clamp inactive
 * -> 0. The paper modifies the backward of its Baseline for the ReLU
 * polynomial (Sec. 4.3); this is that derivative written out.
 */
void orc_render_backward(int P, const double *means, const double *scales,
                         const double *quats, const double *opacities, const double *sh,
                         int sh_degree, const orc_camera *cam, const orc_config *cfg,
                         const double bg[3], const double *dL_dimg,
                         double *d_means, double *d_scales, double *d_quats,
                         double *d_opacities, double *d_sh,
                         double *d_mean2d, double *d_conic, double *d_opacity2d,
                         double *d_color)
{
    int K = (sh_degree + 1) * (sh_degree + 1);
    double x0 = orc_universal_root(cfg);
    orc_splat2d *s = (orc_splat2d *)malloc(sizeof(orc_splat2d) * (P > 0 ? P : 1));
    proj_state *st = (proj_state *)malloc(sizeof(proj_state) * (P > 0 ? P : 1));
    for (int i = 0; i < P; ++i)
        project_one(i, means, scales, quats, opacities, sh, sh_degree, cam, cfg, x0, &s[i], &st[i]);

    memset(d_mean2d, 0, sizeof(double) * 2 * P);
    memset(d_conic, 0, sizeof(double) * 3 * P);
    memset(d_opacity2d, 0, sizeof(double) * P);
    memset(d_color, 0, sizeof(double) * 3 * P);

    int n;
    int *order = sorted_visible(P, s, &n);
    int W = cam->width, H = cam->height;
    int *cidx = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    double *calpha = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    double *cT = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
    int *cclamp = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));

    /* per pixel: forward walk recording contributors, then the reverse walk */
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double px = x + 0.5, py = y + 0.5;
            const double *g = dL_dimg + 3 * ((long long)y * W + x);
            /* a pixel with zero upstream gradient contributes nothing */
            if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
            double T = 1.0;
            int m = 0;
            for (int j = 0; j < n; ++j) {
                const orc_splat2d *sp = &s[order[j]];
                double Q = quadric(sp, px, py);
                double a = sp->opacity * orc_kernel(cfg, x0, Q);
                int clamped = 0;
                if (a > cfg->alpha_max) { a = cfg->alpha_max; clamped = 1; }
                if (a < cfg->eps) continue;
                double Tn = T * (1.0 - a);
                if (Tn < cfg->t_min) break;
                cidx[m] = order[j]; calpha[m] = a; cT[m] = T; cclamp[m] = clamped; ++m;
                T = Tn;
            }
            /* S = sum over later contributors of c alpha T, plus T_final bg */
            double S[3] = {T * bg[0], T * bg[1], T * bg[2]};
            for (int r = m - 1; r >= 0; --r) {
                int i = cidx[r];
                const orc_splat2d *sp = &s[i];
                double a = calpha[r], Ti = cT[r];
                double dalpha = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    d_color[3 * i + ch] += a * Ti * g[ch];
                    dalpha += g[ch] * (sp->color[ch] * Ti - S[ch] / (1.0 - a));
                }
                for (int ch = 0; ch < 3; ++ch) S[ch] += sp->color[ch] * a * Ti;
                if (cclamp[r]) continue;
                double dx = px - sp->mean2d[0], dy = py - sp->mean2d[1];
                double Q = sp->conic[0] * dx * dx + 2.0 * sp->conic[1] * dx * dy + sp->conic[2] * dy * dy;
                d_opacity2d[i] += orc_kernel(cfg, x0, Q) * dalpha;
                double dQ = sp->opacity * orc_kernel_deriv(cfg, x0, Q) * dalpha;
                d_conic[3 * i + 0] += dQ * dx * dx;
                d_conic[3 * i + 1] += dQ * 2.0 * dx * dy;
                d_conic[3 * i + 2] += dQ * dy * dy;
                d_mean2d[2 * i + 0] += -dQ * 2.0 * (sp->conic[0] * dx + sp->conic[1] * dy);
                d_mean2d[2 * i + 1] += -dQ * 2.0 * (sp->conic[1] * dx + sp->conic[2] * dy);
            }
        }
    free(cidx); free(calpha); free(cT); free(cclamp); free(order);

    /* per splat: chain through colour, AA, conic, EWA, covariance */
    double Wr[3][3], tv[3];
    camera_rotation(cam, Wr, tv);
    for (int i = 0; i < P; ++i) {
        double *dm = d_means + 3 * i, *ds = d_scales + 3 * i, *dq = d_quats + 4 * i;
        double *dsh = d_sh + (long long)i * K * 3;
        dm[0] = dm[1] = dm[2] = 0.0;
        ds[0] = ds[1] = ds[2] = 0.0;
        dq[0] = dq[1] = dq[2] = dq[3] = 0.0;
        d_opacities[i] = 0.0;
        for (int k = 0; k < K * 3; ++k) dsh[k] = 0.0;
        if (!s[i].visible) continue;
        const proj_state *p = &st[i];
        const double *s3 = scales + 3 * i;

        /* colour: c = max(sum_k Y_k sh_k + 0.5, 0) */
        double Y[16], GY[16][3];
        orc_sh_basis(sh_degree, p->dir, Y);
        sh_basis_grad(sh_degree, p->dir, GY);
        double draw[3], ddir[3] = {0.0, 0.0, 0.0};
        for (int ch = 0; ch < 3; ++ch) draw[ch] = s[i].color_raw[ch] > 0.0 ? d_color[3 * i + ch] : 0.0;
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) {
                dsh[k * 3 + ch] = Y[k] * draw[ch];
                double coeff = sh[((long long)i * K + k) * 3 + ch];
                for (int r = 0; r < 3; ++r) ddir[r] += GY[k][r] * coeff * draw[ch];
            }
        double dd = ddir[0] * p->dir[0] + ddir[1] * p->dir[1] + ddir[2] * p->dir[2];
        for (int r = 0; r < 3; ++r) dm[r] += (ddir[r] - p->dir[r] * dd) / p->dist;

        /* o' = o rho */
        double rho = s[i].rho;
        d_opacities[i] = rho * d_opacity2d[i];
        double drho = cfg->aa ? opacities[i] * d_opacity2d[i] : 0.0;

        /* conic = (Sigma' + vI)^-1 with entries (a, b, c) of Sigma' + vI */
        double a = p->a, b = p->b, c = p->c, det1 = p->det1;
        double dA = d_conic[3 * i + 0], dB = d_conic[3 * i + 1], dC = d_conic[3 * i + 2];
        double ddet1 = -(dA * c - dB * b + dC * a) / (det1 * det1);
        double da = dC / det1, db = -dB / det1, dc = dA / det1;
        double ddet0 = 0.0;
        if (cfg->aa && p->det0 > 0.0) {
            ddet0 = drho / (2.0 * sqrt(p->det0 * det1));
            ddet1 += -drho * rho / (2.0 * det1);
        }
        da += ddet1 * c; dc += ddet1 * a; db += -2.0 * b * ddet1;
        /* det0 = cov00 cov11 - cov01^2; the low-pass shifts a and c only */
        double dS00 = da + ddet0 * p->cov[2];
        double dS11 = dc + ddet0 * p->cov[0];
        double dS01 = db - 2.0 * p->cov[1] * ddet0;
        double G[2][2] = {{dS00, 0.5 * dS01}, {0.5 * dS01, dS11}};

        /* Sigma' = Tm Sigma Tm^T: dTm = 2 G Tm Sigma; dSigma = Tm^T G Tm */
        double TS[2][3], dTm[2][3], dSig[3][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                TS[r][k] = p->Tm[r][0] * p->Sigma[0][k] + p->Tm[r][1] * p->Sigma[1][k] + p->Tm[r][2] * p->Sigma[2][k];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k) dTm[r][k] = 2.0 * (G[r][0] * TS[0][k] + G[r][1] * TS[1][k]);
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int u = 0; u < 2; ++u)
                    for (int v = 0; v < 2; ++v) acc += p->Tm[u][r] * G[u][v] * p->Tm[v][k];
                dSig[r][k] = acc;
            }

        /* Tm = J W: dJ = dTm W^T */
        double dJ[2][3];
        for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 3; ++k)
                dJ[r][k] = dTm[r][0] * Wr[k][0] + dTm[r][1] * Wr[k][1] + dTm[r][2] * Wr[k][2];
        double tz = p->t[2], fx = cam->fx, fy = cam->fy;
        double dt[3] = {0.0, 0.0, 0.0};
        dt[2] += -fx / (tz * tz) * dJ[0][0] + 2.0 * fx * p->txc / (tz * tz * tz) * dJ[0][2]
                 - fy / (tz * tz) * dJ[1][1] + 2.0 * fy * p->tyc / (tz * tz * tz) * dJ[1][2];
        double dtxc = -fx / (tz * tz) * dJ[0][2], dtyc = -fy / (tz * tz) * dJ[1][2];
        double limx = 1.3 * (0.5 * cam->width / cam->fx), limy = 1.3 * (0.5 * cam->height / cam->fy);
        if (p->clampx == 0) dt[0] += dtxc; else dt[2] += p->clampx * limx * dtxc;
        if (p->clampy == 0) dt[1] += dtyc; else dt[2] += p->clampy * limy * dtyc;

        /* mu' = (fx tx / tz + cx, fy ty / tz + cy) */
        double dmx = d_mean2d[2 * i + 0], dmy = d_mean2d[2 * i + 1];
        dt[0] += fx / tz * dmx;
        dt[1] += fy / tz * dmy;
        dt[2] += -fx * p->t[0] / (tz * tz) * dmx - fy * p->t[1] / (tz * tz) * dmy;

        /* t = W mu + t_cam */
        for (int r = 0; r < 3; ++r) dm[r] += Wr[0][r] * dt[0] + Wr[1][r] * dt[1] + Wr[2][r] * dt[2];

        /* Sigma = M M^T, M = R diag(s): dM = (dSig + dSig^T) M */
        double dM[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int u = 0; u < 3; ++u) acc += (dSig[r][u] + dSig[u][r]) * p->M[u][k];
                dM[r][k] = acc;
            }
        double dR[3][3];
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) {
                ds[k] += dM[r][k] * p->R[r][k];
                dR[r][k] = dM[r][k] * s3[k];
            }
        /* R(q) for unit q = (w, x, y, z) */
        double w = p->qn[0], x = p->qn[1], y = p->qn[2], z = p->qn[3];
        double dqn[4];
        dqn[0] = 2.0 * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
        dqn[1] = 2.0 * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.0 * x * dR[1][1] - w * dR[1][2]
                        + z * dR[2][0] + w * dR[2][1] - 2.0 * x * dR[2][2]);
        dqn[2] = 2.0 * (-2.0 * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2]
                        - w * dR[2][0] + z * dR[2][1] - 2.0 * y * dR[2][2]);
        dqn[3] = 2.0 * (-2.0 * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.0 * z * dR[1][1]
                        + y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
        /* q_n = q / |q| */
        double dot = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * z;
        for (int k = 0; k < 4; ++k) dq[k] = (dqn[k] - p->qn[k] * dot) / p->qlen;
    }
    free(s);
    free(st);
}
