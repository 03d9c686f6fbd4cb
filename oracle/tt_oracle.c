/*
 * tt_oracle.c -- plain FP64 CPU oracle for the gradient-residual evaluation of
 * SAXS/WAXS tensor tomography with a real even-order spherical-harmonic basis
 * (Mumott, arXiv 2504.16446, Section "Methodology").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  It is used by tests/,
 * by __graft_entry__.smoke() and by the cpu_baseline leg of bench.py, and by
 * nothing else.  It shares no code, header, table or constant with the CUDA
 * library under paper_2504_16446_gb300/csrc, and the CUDA library never calls
 * it.
 *
 * Everything is double precision and single-threaded; loops follow the
 * paper's equations in the order they are written, with no blocking, fusion
 * or reordering.
 *
 * Conventions (the paper leaves these open; the readings are listed in the
 * design notes and pinned by tests/test_oracle_*.py):
 *   - Real SH, even l only, orthonormal on the sphere, no Condon-Shortley
 *     phase, polar axis +z, azimuth from +x towards +y.  Index order
 *     i = (l = 0, 2, 4, ...; m = -l..l).
 *   - R_s = R_beta(beta) R_alpha(alpha), right-handed rotations (Section
 *     "Methodology", goniometer paragraph).
 *   - Voxel (x,y,z) has sample-frame centre a*(x-(nx-1)/2, y-(ny-1)/2,
 *     z-(nz-1)/2); ray (j,k) is the line through b*(j-(nj-1)/2-dj)*j_s +
 *     b*(k-(nk-1)/2-dk)*k_s along p_s, with j_s = R_s^T j etc.  This is
 *     Eq. (real_space_geom) read with centred indices: a voxel is on the beam
 *     when its lab position has no j or k component.
 *   - Joseph's method (Section "Projectors and basis sets"): march the planes
 *     of the main axis m = argmax |p_s,t| (ties -> smallest t among axes
 *     within a relative 1e-12 of the maximum); bilinear interpolation of the
 *     four surrounding voxel centres on each plane, zero outside the volume;
 *     each plane contributes with the step length a/|p_s,m|.
 *   - Loss L = sum W (A c - I)^2 (Eq. opt_prob_general_form with a = 2 and
 *     per-datum weights), gradient 2 A^T (W (A c - I)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Problem description, mirroring the fields of the paper's data format
 * (Table "h5_format") and geometry vectors (Table "geometry_vectors"). */
typedef struct {
    int nx, ny, nz;          /* volume shape                                */
    int nj, nk;              /* raster-scan pixels per projection            */
    int n_proj;              /* number of projections s                     */
    int ell_max;             /* band limit (even)                           */
    int n_seg;               /* detector segments c                         */
    const double *inner_angle, *outer_angle;   /* alpha_s, beta_s [rad]    */
    const double *j_offset, *k_offset;         /* delta j, delta k [pixels] */
    const double *seg_start, *seg_end;         /* phi_c,start/end [rad]    */
    double two_theta;        /* scattering angle 2 theta [rad]              */
    double a;                /* voxel size                                  */
    double b;                /* raster step                                 */
    double p[3], j[3], k[3], q0[3], q90[3], alpha_axis[3], beta_axis[3];
} or_problem;

int or_num_coeffs(int ell_max) { return (ell_max + 1) * (ell_max + 2) / 2; }

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics (Section "Basis sets", SH)                       */
/* ------------------------------------------------------------------------ */

/* Unnormalised associated Legendre function P_l^m(x), m >= 0, WITHOUT the
 * Condon-Shortley phase, by the textbook three-term recurrence in l. */
static double assoc_legendre(int l, int m, double x)
{
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;                       /* P_m^m = (2m-1)!! s^m       */
    for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double pm1m = x * (2.0 * m + 1.0) * pmm; /* P_{m+1}^m                  */
    if (l == m + 1) return pm1m;
    double plm = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        plm = ((2.0 * ll - 1.0) * x * pm1m - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1m;
        pm1m = plm;
    }
    return plm;
}

/* N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) */
static double sh_norm(int l, int m)
{
    double ratio = 1.0;                     /* (l-m)!/(l+m)!              */
    for (int t = l - m + 1; t <= l + m; ++t) ratio /= (double)t;
    return sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
}

/* Y_i(q) for all even-l indices i at one unit direction q (need not be exactly
 * normalised; it is normalised here). */
static void sh_at(int ell_max, const double q[3], double *out)
{
    double r = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    double ct = q[2] / r;
    if (ct > 1.0) ct = 1.0;
    if (ct < -1.0) ct = -1.0;
    double phi = atan2(q[1], q[0]);
    int i = 0;
    for (int l = 0; l <= ell_max; l += 2) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double v = sh_norm(l, am) * assoc_legendre(l, am, ct);
            if (m > 0) v *= sqrt(2.0) * cos(am * phi);
            if (m < 0) v *= sqrt(2.0) * sin(am * phi);
            out[i++] = v;
        }
    }
}

void or_sh_eval(int ell_max, int n, const double *dirs, double *out)
{
    int K = or_num_coeffs(ell_max);
    for (int t = 0; t < n; ++t) sh_at(ell_max, dirs + 3 * t, out + (size_t)t * K);
}

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
void or_gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {   /* final derivative at the converged node */
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                double p2 = ((2.0 * l - 1.0) * z * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* ------------------------------------------------------------------------ */
/* Geometry (Section "Methodology": R_s = R_beta(beta) R_alpha(alpha))        */
/* ------------------------------------------------------------------------ */

/* Rodrigues rotation matrix about unit axis n by angle t (right-handed). */
void or_rotation(const double n_in[3], double t, double R[9])
{
    double nn = sqrt(n_in[0] * n_in[0] + n_in[1] * n_in[1] + n_in[2] * n_in[2]);
    double n[3] = {n_in[0] / nn, n_in[1] / nn, n_in[2] / nn};
    double c = cos(t), s = sin(t);
    double K[9] = {0, -n[2], n[1], n[2], 0, -n[0], -n[1], n[0], 0};
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            double kk = 0.0;
            for (int t2 = 0; t2 < 3; ++t2) kk += K[3 * r + t2] * K[3 * t2 + q];
            R[3 * r + q] = (r == q ? 1.0 : 0.0) + s * K[3 * r + q] + (1.0 - c) * kk;
        }
}

/* R_s = R_beta(beta_s) R_alpha(alpha_s), row-major. */
void or_projection_rotation(const or_problem *P, int s, double R[9])
{
    double Ra[9], Rb[9];
    or_rotation(P->alpha_axis, P->inner_angle[s], Ra);
    or_rotation(P->beta_axis, P->outer_angle[s], Rb);
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            double v = 0.0;
            for (int t = 0; t < 3; ++t) v += Rb[3 * r + t] * Ra[3 * t + q];
            R[3 * r + q] = v;
        }
}

/* v_s = R_s^T v */
static void rotate_back(const double R[9], const double v[3], double out[3])
{
    for (int q = 0; q < 3; ++q)
        out[q] = R[0 * 3 + q] * v[0] + R[1 * 3 + q] * v[1] + R[2 * 3 + q] * v[2];
}

/* Sample-frame unit vectors of projection s: rows p_s, j_s, k_s, q0_s, q90_s. */
void or_projection_frame(const or_problem *P, int s, double out[15])
{
    double R[9];
    or_projection_rotation(P, s, R);
    rotate_back(R, P->p, out + 0);
    rotate_back(R, P->j, out + 3);
    rotate_back(R, P->k, out + 6);
    rotate_back(R, P->q0, out + 9);
    rotate_back(R, P->q90, out + 12);
}

/* Main axis of a ray direction: argmax |d_t|, ties to the smallest t among
 * the axes within a relative 1e-12 of the maximum. */
int or_main_axis(const double d[3])
{
    double mx = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
    for (int t = 0; t < 3; ++t)
        if (fabs(d[t]) >= (1.0 - 1e-12) * mx) return t;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Basis matrix, Eq. (projection_matrix)                                     */
/* ------------------------------------------------------------------------ */

/* B[s][c][i] = 1/(phi_end-phi_start) * integral over the segment of
 * Y_i(R_s^T q(phi)) dphi, with q(phi) = cos(theta)(cos phi q0 + sin phi q90)
 * - sin(theta) p and theta = two_theta/2; one n_nodes-point Gauss-Legendre
 * rule per segment. */
void or_basis_matrix(const or_problem *P, int n_nodes, double *B)
{
    int K = or_num_coeffs(P->ell_max);
    double *x = (double *)malloc(sizeof(double) * n_nodes);
    double *w = (double *)malloc(sizeof(double) * n_nodes);
    double *y = (double *)malloc(sizeof(double) * K);
    or_gauss_legendre(n_nodes, x, w);
    double th = 0.5 * P->two_theta;
    for (int s = 0; s < P->n_proj; ++s) {
        double F[15];
        or_projection_frame(P, s, F);
        const double *ps = F + 0, *q0s = F + 9, *q90s = F + 12;
        for (int c = 0; c < P->n_seg; ++c) {
            double lo = P->seg_start[c], hi = P->seg_end[c];
            double half = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
            double *Bsc = B + ((size_t)s * P->n_seg + c) * K;
            for (int i = 0; i < K; ++i) Bsc[i] = 0.0;
            for (int t = 0; t < n_nodes; ++t) {
                double phi = mid + half * x[t];
                double q[3];
                for (int r = 0; r < 3; ++r)
                    q[r] = cos(th) * (cos(phi) * q0s[r] + sin(phi) * q90s[r]) - sin(th) * ps[r];
                sh_at(P->ell_max, q, y);
                /* (1/(hi-lo)) * half * sum w f = 0.5 * sum w f */
                for (int i = 0; i < K; ++i) Bsc[i] += 0.5 * w[t] * y[i];
            }
        }
    }
    free(x);
    free(w);
    free(y);
}

/* ------------------------------------------------------------------------ */
/* John transform by Joseph's method (Section "Projectors and basis sets"),  */
/* Eq. (real_space_geom) and Eq. (projection_operator)                       */
/* ------------------------------------------------------------------------ */

static size_t vox_index(const or_problem *P, const int xyz[3])
{
    return ((size_t)xyz[0] * P->ny + xyz[1]) * P->nz + xyz[2];
}

/* Calls visit(ctx, s, pixel, voxel, weight) for every (ray, tap) pair of the
 * Joseph discretisation; weight includes the step length a/|p_m|.  The
 * forward and adjoint below both use this single enumeration, so the adjoint
 * is the exact transpose by construction. */
typedef void (*visit_fn)(void *ctx, int s, size_t pix, size_t vox, double w);

static void joseph_enumerate(const or_problem *P, visit_fn visit, void *ctx)
{
    int N[3] = {P->nx, P->ny, P->nz};
    for (int s = 0; s < P->n_proj; ++s) {
        double F[15];
        or_projection_frame(P, s, F);
        const double *d = F + 0, *js = F + 3, *ks = F + 6;
        int m = or_main_axis(d);
        int u = (m == 0) ? 1 : 0;
        int v = (m == 2) ? 1 : 2;
        double step = P->a / fabs(d[m]);
        for (int j = 0; j < P->nj; ++j)
            for (int k = 0; k < P->nk; ++k) {
                double tj = P->b * (j - 0.5 * (P->nj - 1) - P->j_offset[s]);
                double tk = P->b * (k - 0.5 * (P->nk - 1) - P->k_offset[s]);
                double X0[3];
                for (int r = 0; r < 3; ++r) X0[r] = tj * js[r] + tk * ks[r];
                size_t pix = ((size_t)s * P->nj + j) * P->nk + k;
                for (int p = 0; p < N[m]; ++p) {
                    double Xm = P->a * (p - 0.5 * (N[m] - 1));
                    double t = (Xm - X0[m]) / d[m];
                    double fu = (X0[u] + t * d[u]) / P->a + 0.5 * (N[u] - 1);
                    double fv = (X0[v] + t * d[v]) / P->a + 0.5 * (N[v] - 1);
                    double iu = floor(fu), iv = floor(fv);
                    double wu = fu - iu, wv = fv - iv;
                    for (int du = 0; du <= 1; ++du)
                        for (int dv = 0; dv <= 1; ++dv) {
                            int tu = (int)iu + du, tv = (int)iv + dv;
                            if (tu < 0 || tu >= N[u] || tv < 0 || tv >= N[v]) continue;
                            double w = (du ? wu : 1.0 - wu) * (dv ? wv : 1.0 - wv);
                            int xyz[3];
                            xyz[m] = p;
                            xyz[u] = tu;
                            xyz[v] = tv;
                            visit(ctx, s, pix, vox_index(P, xyz), step * w);
                        }
                }
            }
    }
}

typedef struct { int K; const double *src; double *dst; } john_ctx;

static void fwd_visit(void *vctx, int s, size_t pix, size_t vox, double w)
{
    john_ctx *c = (john_ctx *)vctx;
    (void)s;
    for (int i = 0; i < c->K; ++i) c->dst[pix * c->K + i] += w * c->src[vox * c->K + i];
}

static void adj_visit(void *vctx, int s, size_t pix, size_t vox, double w)
{
    john_ctx *c = (john_ctx *)vctx;
    (void)s;
    for (int i = 0; i < c->K; ++i) c->dst[vox * c->K + i] += w * c->src[pix * c->K + i];
}

/* Y[s][j][k][i] = sum_xyz P_sjk,xyz c[x][y][z][i] for K channels. */
void or_john_forward(const or_problem *P, int K, const double *c, double *Y)
{
    memset(Y, 0, sizeof(double) * (size_t)P->n_proj * P->nj * P->nk * K);
    john_ctx ctx = {K, c, Y};
    joseph_enumerate(P, fwd_visit, &ctx);
}

/* g[x][y][z][i] = sum_sjk P_sjk,xyz Y[s][j][k][i]  (exact transpose). */
void or_john_adjoint(const or_problem *P, int K, const double *Y, double *g)
{
    memset(g, 0, sizeof(double) * (size_t)P->nx * P->ny * P->nz * K);
    john_ctx ctx = {K, Y, g};
    joseph_enumerate(P, adj_visit, &ctx);
}

/* ------------------------------------------------------------------------ */
/* Forward model, Eq. (forward_model): I_sjkc = sum_xyz P sum_i B_sci c_xyzi  */
/* ------------------------------------------------------------------------ */

void or_forward(const or_problem *P, const double *B, const double *c, double *I)
{
    int K = or_num_coeffs(P->ell_max), C = P->n_seg;
    size_t npix = (size_t)P->n_proj * P->nj * P->nk;
    double *Y = (double *)malloc(sizeof(double) * npix * K);
    or_john_forward(P, K, c, Y);
    for (size_t q = 0; q < npix; ++q) {
        int s = (int)(q / ((size_t)P->nj * P->nk));
        for (int cc = 0; cc < C; ++cc) {
            double v = 0.0;
            for (int i = 0; i < K; ++i) v += B[((size_t)s * C + cc) * K + i] * Y[q * K + i];
            I[q * C + cc] = v;
        }
    }
    free(Y);
}

/* Adjoint of the forward model: g = A^T R. */
void or_adjoint(const or_problem *P, const double *B, const double *R, double *g)
{
    int K = or_num_coeffs(P->ell_max), C = P->n_seg;
    size_t npix = (size_t)P->n_proj * P->nj * P->nk;
    double *Y = (double *)malloc(sizeof(double) * npix * K);
    for (size_t q = 0; q < npix; ++q) {
        int s = (int)(q / ((size_t)P->nj * P->nk));
        for (int i = 0; i < K; ++i) {
            double v = 0.0;
            for (int cc = 0; cc < C; ++cc) v += B[((size_t)s * C + cc) * K + i] * R[q * C + cc];
            Y[q * K + i] = v;
        }
    }
    or_john_adjoint(P, K, Y, g);
    free(Y);
}

/* Residual r = A c - I (Eq. residual), loss sum W r^2, gradient 2 A^T (W r).
 * W may be NULL (all ones).  Returns the loss; g may be NULL. */
double or_gradient_residual(const or_problem *P, const double *B, const double *c,
                            const double *I, const double *W, double *g)
{
    int C = P->n_seg;
    size_t n = (size_t)P->n_proj * P->nj * P->nk * C;
    double *r = (double *)malloc(sizeof(double) * n);
    or_forward(P, B, c, r);
    double loss = 0.0;
    for (size_t q = 0; q < n; ++q) {
        double w = W ? W[q] : 1.0;
        r[q] -= I[q];
        loss += w * r[q] * r[q];
        r[q] *= 2.0 * w;
    }
    if (g) or_adjoint(P, B, r, g);
    free(r);
    return loss;
}
