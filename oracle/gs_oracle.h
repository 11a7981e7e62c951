/*
 * gs_oracle.h — FP64 CPU oracle for Gaussian splatting with polynomial kernels
 * (Mueller, Winter, Steinberger, "From ex(p) to poly: Gaussian Splatting with
 * Polynomial Kernels", arXiv 2603.18707).
 *
 * TEST INFRASTRUCTURE. This library exists to check the CUDA renderer. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg load it; the
 * rendering library neither includes this header nor links this code, and this
 * code includes nothing from the rendering library.
 *
 * Every quantity is double precision. Functions are written as plain loops over
 * the definitions they cite, with no fusion or reordering beyond what those
 * definitions state.
 */
#ifndef GS_ORACLE_H
#define GS_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Kernel k(x) on the quadric x = Q(v). Sec. 3, Eq. 1 (exp), Eq. 2 (ReLU poly),
 * Eq. 6 (poly cut at its first root). */
enum { ORC_EXP = 0, ORC_POLY1 = 1, ORC_POLY2CUT = 2, ORC_POLY3 = 3 };

/* Culling radius. UNIVERSAL: opacity-free (Eq. 5; for exp the eps bound at
 * o = 1). OPACITY: per splat (Eq. 3, Eq. 4, App. B). LEGACY3: the 3-sigma
 * radius of the original 3DGS (Sec. 2.1). */
enum { ORC_CULL_UNIVERSAL = 0, ORC_CULL_OPACITY = 1, ORC_CULL_LEGACY3 = 2 };

/* Screen rectangle around the support ellipse: its axis-aligned bounding box,
 * or the square around the circle of radius sqrt(x_cut * lambda_max) (Sec. 2.1). */
enum { ORC_RECT_AABB = 0, ORC_RECT_CIRCLE = 1 };

typedef struct {
    double viewmat[16]; /* world -> camera, row-major; camera looks along +z, +y down */
    double fx, fy, cx, cy;
    int width, height;
    double znear;
} orc_camera;

typedef struct {
    int kind;          /* ORC_EXP .. ORC_POLY3 */
    double c[4];       /* polynomial coefficients c0..c3 (unused ones zero) */
    int cull;          /* ORC_CULL_* */
    double eps;        /* alpha threshold, 1/255 */
    double alpha_max;  /* alpha clamp, 0.99 */
    double t_min;      /* transmittance stop, 1e-4 */
    int aa;            /* 1: anti-aliasing normalisation of Sec. 3.4 */
    double dilation;   /* low-pass v added to the 2D covariance diagonal, 0.3 */
    int tile_w, tile_h;
    int rect_mode;     /* ORC_RECT_* */
} orc_config;

/* Per-splat record after projection (one per input splat). */
typedef struct {
    int visible;          /* 0: behind the near plane, or no pixel can reach eps */
    int pad_;
    double mean2d[2];     /* mu' in pixel coordinates */
    double cov2d[3];      /* Sigma' = J W Sigma W^T J^T as (a, b, c) before the low-pass */
    double conic[3];      /* (Sigma' + v I)^-1 as (A, B, C) */
    double rho;           /* AA normalisation factor (1 when AA is off) */
    double opacity;       /* o' = o * rho */
    double depth;         /* camera-space z */
    double color[3];      /* SH colour, clamped at 0 */
    double color_raw[3];  /* SH colour before the clamp */
    double xcut;          /* quadric threshold of the support */
    int rect[4];          /* tile range x0, y0, x1, y1 (inclusive) */
    long long tiles;      /* number of tiles in rect, 0 if empty */
} orc_splat2d;

/* ---- kernel math (Sec. 3, 3.1, 3.2, 3.3, App. B) ---- */
int    orc_order(int kind);
double orc_poly(const double c[4], int order, double x);
double orc_first_root(const double c[4], int order, double rhs);
double orc_universal_root(const orc_config *cfg);
double orc_kernel(const orc_config *cfg, double x0, double x);
double orc_kernel_deriv(const orc_config *cfg, double x0, double x);
double orc_xcut(const orc_config *cfg, double x0, double opacity);

/* ---- real spherical harmonics used by 3DGS for view-dependent colour ---- */
int  orc_sh_basis(int degree, const double dir[3], double *Y);

/* ---- projection (Eq. 1, Sec. 3.4; EWA and SH by reference to 3DGS) ---- */
void orc_project(int P, const double *means, const double *scales, const double *quats,
                 const double *opacities, const double *sh, int sh_degree,
                 const orc_camera *cam, const orc_config *cfg, orc_splat2d *out);

/* ---- compositing (Sec. 2, front-to-back alpha blending) ---- */
void orc_render_untiled(int P, const orc_splat2d *s, const orc_camera *cam,
                        const orc_config *cfg, const double bg[3],
                        double *img, double *final_T, long long *n_contrib);
void orc_render_tiled(int P, const orc_splat2d *s, const orc_camera *cam,
                      const orc_config *cfg, const double bg[3],
                      int n_tiles_sel, const int *tiles_sel,
                      double *img, double *final_T, long long *last_contrib,
                      long long *n_eval, long long *list_len, double *margin);

/* ---- analytic reverse pass (Sec. 4.3 ablation "Opt" rows need it) ---- */
void orc_render_backward(int P, const double *means, const double *scales,
                         const double *quats, const double *opacities, const double *sh,
                         int sh_degree, const orc_camera *cam, const orc_config *cfg,
                         const double bg[3], const double *dL_dimg,
                         double *d_means, double *d_scales, double *d_quats,
                         double *d_opacities, double *d_sh,
                         double *d_mean2d, double *d_conic, double *d_opacity2d,
                         double *d_color);

/* Per-pixel fingerprint of every discrete decision of the untiled render
 * (skip / clamp / stop per splat) — finite differences are only taken where it
 * does not change. */
void orc_decisions(int P, const orc_splat2d *s, const orc_camera *cam,
                   const orc_config *cfg, unsigned long long *sig);

#ifdef __cplusplus
}
#endif
#endif
