/*
 * UPSLAM hot-path ORACLE: a plain, slow, obviously-correct CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference arm may load this code.  The CUDA
 * library never calls it and shares no code, header, table or constant with it.
 *
 * It restates, step by step, what the paper's per-sweep path computes
 * (UPSLAM, arXiv 2101.00585):
 *   - Sec. III-A "Data Intake": the points are binned into a panoramic image, and a
 *     normal is the cross product of the vectors from a pixel's point to two
 *     image neighbours;
 *   - Sec. III-B "Motion Estimation", Eq. 1: point-to-plane ICP over projective
 *     correspondences C filtered by the similarity test Omega_{d,theta};
 *   - Sec. III-C "Keyframe Update": every keyframe pixel is carried over to the
 *     sweep image, gated by the same kind of similarity test, and averaged in
 *     with a per-pixel sample count saturated at 10; the registration quality
 *     is inliers / valid sweep measurements;
 *   - Sec. IV-F footnote: the ICP initial guess from a zero-velocity or a
 *     zero-acceleration motion prior.
 *
 * Arithmetic: values are FP64.  Where floating point decides an integer (the
 * pixel a point falls in, and the z-buffer winner), the decision is taken in
 * FP32 with one fixed sequence of IEEE round-to-nearest operations (no fused
 * multiply-add: build with -ffp-contract=off), because the GPU kernels take the
 * same decisions in FP32.  The similarity-filter and normal-validity thresholds
 * are evaluated in FP64 here; a GPU disagreement there is legitimate only at a
 * near-tie, which the parity tests check.
 *
 * Pins (tests/test_oracle_pins.py): atan error bound against FP64 atan2; pixel
 * bins against FP64 angular bounds by brute force; project/unproject round trip;
 * z-buffer winner as lexicographic minimum under permutation; analytic plane
 * normals from the ray caster; identity gives zero residual; a known rigid
 * perturbation is recovered; a single plane is degenerate; the Jacobian against
 * finite differences; the 6x6 solve against LAPACK; SE(3) exp against the
 * matrix exponential; brute-force association; the fusion closed form; the
 * motion prior against constant-twist trajectories built by the matrix
 * exponential.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared upslam_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>

/* ------------------------------------------------------------------ types */

typedef struct {
    int32_t rows, cols;
    float el_top; /* elevation of the top edge of row 0 (rad) */
    float s_az;   /* columns per radian of azimuth: cols / 2pi */
    float s_el;   /* rows per radian of elevation */
    float r_min, r_max;
} orc_pano;

typedef struct {
    float jump_rel, jump_abs; /* neighbour rejected if |r_nb - r| > jump_rel * r + jump_abs */
    float min_cross;          /* normal rejected if |a x b| < min_cross |a| |b| */
} orc_normal_params;

typedef struct {
    float d_max;         /* Omega: point distance threshold (m) */
    float cos_theta_max; /* Omega: minimum cosine between normals */
    int32_t max_iters;
    int32_t min_inliers;
    double eps_rot, eps_trans; /* convergence on |omega|, |v| of the update */
    double pivot_eps;          /* Cholesky pivot <= pivot_eps * max diag => degenerate */
    int32_t loss;              /* 0: squared residuals; 1: absolute residuals by IRLS */
    float loss_delta;          /* IRLS weight 1 / max(|r|, loss_delta) */
} orc_icp_params;

typedef struct {
    double A[21]; /* upper triangle of J^T J, row-major */
    double b[6];  /* J^T r */
    double sse;
    int64_t inliers, valid;
    int32_t status; /* 0 ok, 3 degenerate */
    int32_t converged;
    double xi[6]; /* the update solved for (omega, v) */
} orc_icp_stats;

typedef struct {
    float d_max, cos_theta_max;
    float w_max;
} orc_fuse_params;

#define ORC_PI_F 3.14159265358979323846f
#define ORC_HALF_PI_F 1.57079632679489661923f

/* ------------------------------------------------------------------ FP32 decision arithmetic */

/*
 * atan(t) for t in [0, 1] by the 8-term odd polynomial of Abramowitz & Stegun
 * 4.4.49 (|error| <= 2e-8 in exact arithmetic), evaluated by Horner in FP32.
 * atan2 is reduced to it by octant symmetry.  (0, 0) -> 0; -0 counts as +0.
 */
float orc_atan2p(float y, float x) {
    float ax = fabsf(x), ay = fabsf(y);
    float mx = ax > ay ? ax : ay;
    float mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    float t = mn / mx;
    float s = t * t;
    float p = 0.0028662257f;
    p = p * s + -0.0161657367f;
    p = p * s + 0.0429096138f;
    p = p * s + -0.0752896400f;
    p = p * s + 0.1065626393f;
    p = p * s + -0.1420889944f;
    p = p * s + 0.1999355085f;
    p = p * s + -0.3333314528f;
    p = p * s + 1.0f;
    float a = t * p;
    if (ay > ax) a = ORC_HALF_PI_F - a;
    if (x < 0.0f) a = ORC_PI_F - a;
    if (y < 0.0f) a = -a;
    return a;
}

/*
 * Pixel of an FP32 point in a panorama (Sec. III-A projection).  Returns 1 and
 * (row, col, range) when the range lies in [r_min, r_max] and the elevation
 * falls inside the panorama's rows; 0 otherwise.
 */
int orc_bin(float x, float y, float z, const orc_pano *pp, int32_t *row, int32_t *col, float *range) {
    float xy2 = x * x + y * y;
    float r = sqrtf(xy2 + z * z);
    if (!(r >= pp->r_min && r <= pp->r_max)) return 0;
    float rho = sqrtf(xy2);
    float az = orc_atan2p(y, x);
    float el = orc_atan2p(z, rho);
    float fc = (ORC_PI_F - az) * pp->s_az;
    float fr = (pp->el_top - el) * pp->s_el;
    if (!(fr >= 0.0f) || !(fr < (float)pp->rows)) return 0;
    int32_t v = (int32_t)floorf(fr);
    int32_t u = (int32_t)floorf(fc);
    if (v >= pp->rows) return 0;
    if (u >= pp->cols) u -= pp->cols;
    if (u < 0) u += pp->cols;
    *row = v;
    *col = u;
    *range = r;
    return 1;
}

/* p = R q + t with the pose rounded to FP32 and a fixed summation order */
void orc_xform_f32(const double *T, float qx, float qy, float qz, float *px, float *py, float *pz) {
    float r[12];
    for (int i = 0; i < 12; ++i) r[i] = (float)T[i];
    *px = ((r[0] * qx + r[1] * qy) + r[2] * qz) + r[3];
    *py = ((r[4] * qx + r[5] * qy) + r[6] * qz) + r[7];
    *pz = ((r[8] * qx + r[9] * qy) + r[10] * qz) + r[11];
}

/* q = R^T (s - t), FP32, fixed order */
void orc_xform_inv_f32(const double *T, float sx, float sy, float sz, float *qx, float *qy, float *qz) {
    float r[12];
    for (int i = 0; i < 12; ++i) r[i] = (float)T[i];
    float dx = sx - r[3], dy = sy - r[7], dz = sz - r[11];
    *qx = (r[0] * dx + r[4] * dy) + r[8] * dz;
    *qy = (r[1] * dx + r[5] * dy) + r[9] * dz;
    *qz = (r[2] * dx + r[6] * dy) + r[10] * dz;
}

/* FP64 elevation of the centre of row v and azimuth of the centre of column u */
static double row_el(const orc_pano *pp, int v) { return (double)pp->el_top - ((double)v + 0.5) / (double)pp->s_el; }
static double col_az(const orc_pano *pp, int u) { return 3.14159265358979323846 - ((double)u + 0.5) / (double)pp->s_az; }

/*
 * Pixel-centre direction tables: rowtab[2v] = cos(el_v), rowtab[2v+1] = sin(el_v),
 * coltab[2u] = cos(az_u), coltab[2u+1] = sin(az_u), each FP64 rounded to FP32.
 */
void orc_dir_table(const orc_pano *pp, float *rowtab, float *coltab) {
    for (int v = 0; v < pp->rows; ++v) {
        double e = row_el(pp, v);
        rowtab[2 * v] = (float)cos(e);
        rowtab[2 * v + 1] = (float)sin(e);
    }
    for (int u = 0; u < pp->cols; ++u) {
        double a = col_az(pp, u);
        coltab[2 * u] = (float)cos(a);
        coltab[2 * u + 1] = (float)sin(a);
    }
}

/* FP32 point at depth d along the centre of pixel (v, u), from the FP32 tables */
static void pixel_point_f32(const float *rowtab, const float *coltab, int v, int u, float d,
                            float *x, float *y, float *z) {
    float ce = rowtab[2 * v], se = rowtab[2 * v + 1], ca = coltab[2 * u], sa = coltab[2 * u + 1];
    *x = d * (ce * ca);
    *y = d * (ce * sa);
    *z = d * se;
}

/* FP64 direction through the centre of pixel (v, u) */
static void pixel_dir64(const orc_pano *pp, int v, int u, double dir[3]) {
    double e = row_el(pp, v), a = col_az(pp, u);
    dir[0] = cos(e) * cos(a);
    dir[1] = cos(e) * sin(a);
    dir[2] = sin(e);
}

/* ------------------------------------------------------------------ a1: projection + z-buffer */

/*
 * Bin every valid point (pts4[i].w != 0) into the panorama, optionally after the
 * transform T (FP32, as orc_xform_f32).  Each pixel keeps the point with the
 * smallest (range, index), i.e. the smallest 64-bit key (bits(range) << 32 | i).
 * Outputs depth[k] = range of the winner (0 if empty) and idx[k] = its index (-1).
 * Returns the number of points binned.
 */
int64_t orc_project(const float *pts4, int32_t n, const double *T, const orc_pano *pp,
                    float *depth, int32_t *idx) {
    int64_t npx = (int64_t)pp->rows * pp->cols;
    uint64_t *best = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(npx > 0 ? npx : 1));
    for (int64_t k = 0; k < npx; ++k) best[k] = UINT64_MAX;
    int64_t binned = 0;
    for (int32_t i = 0; i < n; ++i) {
        const float *p = pts4 + 4 * (int64_t)i;
        if (p[3] == 0.0f) continue;
        float x = p[0], y = p[1], z = p[2];
        if (T) orc_xform_f32(T, p[0], p[1], p[2], &x, &y, &z);
        int32_t v, u;
        float r;
        if (!orc_bin(x, y, z, pp, &v, &u, &r)) continue;
        ++binned;
        uint32_t rb;
        memcpy(&rb, &r, 4);
        uint64_t key = ((uint64_t)rb << 32) | (uint32_t)i;
        int64_t k = (int64_t)v * pp->cols + u;
        if (key < best[k]) best[k] = key;
    }
    for (int64_t k = 0; k < npx; ++k) {
        if (best[k] == UINT64_MAX) {
            depth[k] = 0.0f;
            idx[k] = -1;
        } else {
            uint32_t rb = (uint32_t)(best[k] >> 32);
            memcpy(&depth[k], &rb, 4);
            idx[k] = (int32_t)(best[k] & 0xffffffffu);
        }
    }
    free(best);
    return binned;
}

/* ------------------------------------------------------------------ a2: normals */

/* neighbour usable: valid and no depth discontinuity (decided in FP32) */
static int nb_ok(const float *pts4, const float *depth, int64_t k, int64_t kn, const orc_normal_params *np) {
    if (pts4[4 * kn + 3] == 0.0f) return 0;
    float d = depth[k], dn = depth[kn];
    float jump = fabsf(dn - d);
    float lim = np->jump_rel * d + np->jump_abs;
    return !(jump > lim);
}

/*
 * Per-pixel normal (Sec. III-A): n = a x b with a toward the right neighbour
 * (column + 1, wrapping) and b toward the neighbour below (row + 1); when one is
 * unusable the opposite neighbour is used with the vector's sign flipped.  The
 * normal is normalised and oriented toward the sensor (n . P < 0).
 * Inputs: pts4 [rows*cols] pixel points (w != 0 valid), depth [rows*cols].
 * Outputs: nrm [rows*cols*3] (zeros when invalid), valid [rows*cols], and, if
 * sin_ab is not NULL, |a x b| / (|a| |b|) per pixel: the conditioning of the
 * cross product (a tolerance for any lower-precision evaluation scales with
 * its inverse).
 */
void orc_normals(const float *pts4, const float *depth, const orc_pano *pp, const orc_normal_params *np,
                 double *nrm, uint8_t *valid, double *sin_ab) {
    int H = pp->rows, W = pp->cols;
    for (int v = 0; v < H; ++v) {
        for (int u = 0; u < W; ++u) {
            int64_t k = (int64_t)v * W + u;
            nrm[3 * k] = nrm[3 * k + 1] = nrm[3 * k + 2] = 0.0;
            valid[k] = 0;
            if (sin_ab) sin_ab[k] = 0.0;
            if (pts4[4 * k + 3] == 0.0f) continue;
            double P[3] = { pts4[4 * k], pts4[4 * k + 1], pts4[4 * k + 2] };
            double a[3], b[3];
            int64_t kr = (int64_t)v * W + (u + 1) % W, kl = (int64_t)v * W + (u + W - 1) % W;
            if (nb_ok(pts4, depth, k, kr, np)) {
                for (int c = 0; c < 3; ++c) a[c] = (double)pts4[4 * kr + c] - P[c];
            } else if (nb_ok(pts4, depth, k, kl, np)) {
                for (int c = 0; c < 3; ++c) a[c] = P[c] - (double)pts4[4 * kl + c];
            } else continue;
            if (v + 1 < H && nb_ok(pts4, depth, k, k + W, np)) {
                for (int c = 0; c < 3; ++c) b[c] = (double)pts4[4 * (k + W) + c] - P[c];
            } else if (v >= 1 && nb_ok(pts4, depth, k, k - W, np)) {
                for (int c = 0; c < 3; ++c) b[c] = P[c] - (double)pts4[4 * (k - W) + c];
            } else continue;
            double n[3] = { a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0] };
            double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            double na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
            double nb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
            if (sin_ab && na > 0.0 && nb > 0.0) sin_ab[k] = nn / (na * nb);
            if (!(nn >= (double)np->min_cross * na * nb) || nn == 0.0) continue;
            double s = (n[0] * P[0] + n[1] * P[1] + n[2] * P[2]) > 0.0 ? -1.0 / nn : 1.0 / nn;
            nrm[3 * k] = n[0] * s;
            nrm[3 * k + 1] = n[1] * s;
            nrm[3 * k + 2] = n[2] * s;
            valid[k] = 1;
        }
    }
}

/* ------------------------------------------------------------------ SE(3) and the 6x6 solve */

/* T <- exp(xi^) T, xi = (omega, v); Rodrigues rotation and the V matrix for the translation */
void orc_se3_exp_left(const double xi[6], double *T) {
    double w0 = xi[0], w1 = xi[1], w2 = xi[2];
    double th2 = w0 * w0 + w1 * w1 + w2 * w2, th = sqrt(th2);
    double A, B, C; /* sin(th)/th, (1-cos th)/th^2, (th - sin th)/th^3 */
    if (th < 1e-8) {
        A = 1.0 - th2 / 6.0;
        B = 0.5 - th2 / 24.0;
        C = 1.0 / 6.0 - th2 / 120.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    double W[9] = { 0, -w2, w1, w2, 0, -w0, -w1, w0, 0 };
    double W2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += W[3 * i + k] * W[3 * k + j];
            W2[3 * i + j] = s;
        }
    double R[9], V[9];
    for (int i = 0; i < 9; ++i) {
        double I = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = I + A * W[i] + B * W2[i];
        V[i] = I + B * W[i] + C * W2[i];
    }
    double te[3];
    for (int i = 0; i < 3; ++i) te[i] = V[3 * i] * xi[3] + V[3 * i + 1] * xi[4] + V[3 * i + 2] * xi[5];
    double Tn[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double s = 0;
            for (int k = 0; k < 3; ++k) s += R[3 * i + k] * T[4 * k + j];
            Tn[4 * i + j] = s;
        }
        double s = te[i];
        for (int k = 0; k < 3; ++k) s += R[3 * i + k] * T[4 * k + 3];
        Tn[4 * i + 3] = s;
    }
    memcpy(T, Tn, sizeof(Tn));
}

/*
 * Solve M x = rhs for a symmetric positive-definite 6x6 M given as its upper
 * triangle (21 values, row-major) by Cholesky M = L L^T.  Returns 0, or 3 when a
 * pivot falls to pivot_eps * max diagonal or below (rank-deficient geometry).
 */
int orc_solve6(const double *Aup, const double *rhs, double pivot_eps, double *x) {
    double M[36], L[36];
    int p = 0;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j) { M[6 * i + j] = Aup[p]; M[6 * j + i] = Aup[p]; ++p; }
    double dmax = 0;
    for (int i = 0; i < 6; ++i) if (M[7 * i] > dmax) dmax = M[7 * i];
    if (!(dmax > 0)) return 3;
    memset(L, 0, sizeof(L));
    for (int j = 0; j < 6; ++j) {
        double s = M[7 * j];
        for (int k = 0; k < j; ++k) s -= L[6 * j + k] * L[6 * j + k];
        if (!(s > pivot_eps * dmax)) return 3;
        double d = sqrt(s);
        L[7 * j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double t = M[6 * i + j];
            for (int k = 0; k < j; ++k) t -= L[6 * i + k] * L[6 * j + k];
            L[6 * i + j] = t / d;
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = rhs[i];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s / L[7 * i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s / L[7 * i];
    }
    return 0;
}

/* ------------------------------------------------------------------ a3: one Gauss-Newton ICP step */

/*
 * Projective correspondence of one keyframe pixel k = (v, u) under T (Eq. 1's set
 * C and filter Omega, Sec. III-B).  As in the keyframe update (Sec. III-C), the
 * keyframe pixel is carried over to the sweep's depth image: its point s1 = d_k dir_k
 * goes to the sweep frame by T^-1 and is binned (FP32 decision) into sweep pixel
 * j; s2 = P_j.  Returns 1 for an inlier and fills r = (T s2 - s1) . N(s1) and
 * J = d r / d xi for the left update T <- exp(xi^) T, xi = (omega, v).
 */
static int associate(const double *T, int v, int u, const float *kf_depth, const float *kf_nrm4,
                     const orc_pano *kp, const float *rowtab, const float *coltab, const float *sp4,
                     const float *sn4, const orc_pano *sw, const orc_icp_params *ip, double *r_out,
                     double J[6], int64_t *jpix) {
    int64_t k = (int64_t)v * kp->cols + u;
    float dk = kf_depth[k];
    const float *nk = kf_nrm4 + 4 * k;
    if (!(dk > 0.0f)) return 0;
    if (!(nk[0] * nk[0] + nk[1] * nk[1] + nk[2] * nk[2] > 0.25f)) return 0;
    float sx, sy, sz, qx, qy, qz;
    pixel_point_f32(rowtab, coltab, v, u, dk, &sx, &sy, &sz);
    orc_xform_inv_f32(T, sx, sy, sz, &qx, &qy, &qz);
    int32_t jv, ju;
    float rr;
    if (!orc_bin(qx, qy, qz, sw, &jv, &ju, &rr)) return 0;
    int64_t j = (int64_t)jv * sw->cols + ju;
    if (jpix) *jpix = j;
    const float *P = sp4 + 4 * j, *m = sn4 + 4 * j;
    if (P[3] == 0.0f || m[3] == 0.0f) return 0;
    double p[3], Rm[3], dir[3];
    for (int i = 0; i < 3; ++i) {
        p[i] = T[4 * i] * P[0] + T[4 * i + 1] * P[1] + T[4 * i + 2] * P[2] + T[4 * i + 3];
        Rm[i] = T[4 * i] * m[0] + T[4 * i + 1] * m[1] + T[4 * i + 2] * m[2];
    }
    pixel_dir64(kp, v, u, dir);
    double s1[3] = { dk * dir[0], dk * dir[1], dk * dir[2] };
    double n[3] = { nk[0], nk[1], nk[2] };
    double e[3] = { p[0] - s1[0], p[1] - s1[1], p[2] - s1[2] };
    double dist = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    if (!(dist <= (double)ip->d_max)) return 0;
    double cs = Rm[0] * n[0] + Rm[1] * n[1] + Rm[2] * n[2];
    if (!(cs >= (double)ip->cos_theta_max)) return 0;
    *r_out = e[0] * n[0] + e[1] * n[1] + e[2] * n[2];
    J[0] = p[1] * n[2] - p[2] * n[1];
    J[1] = p[2] * n[0] - p[0] * n[2];
    J[2] = p[0] * n[1] - p[1] * n[0];
    J[3] = n[0];
    J[4] = n[1];
    J[5] = n[2];
    return 1;
}

/*
 * Normal equations at T: A = sum w J^T J, b = sum w J^T r and sse = sum w r^2
 * over the inlier correspondences of all keyframe pixels; valid = sweep pixels
 * holding a point.  Eq. 1 prints the point-to-plane error inside |.|: with
 * loss 0 it is squared (w = 1, Gauss-Newton); with loss 1 the absolute error is
 * minimised by iteratively reweighted least squares, w = 1 / max(|r|, delta),
 * which makes w r^2 = |r| wherever |r| >= delta.
 * kf_depth [H*W], kf_nrm4 [H*W*4] (normal xyz, the 4th value unused);
 * sp4 / sn4 [Hs*Ws*4] sweep pixel points / normals (4th value != 0: valid).
 */
void orc_icp_normal_equations(const float *kf_depth, const float *kf_nrm4, const orc_pano *kp,
                              const float *sp4, const float *sn4, const orc_pano *sw, const double *T,
                              const orc_icp_params *ip, orc_icp_stats *st) {
    memset(st, 0, sizeof(*st));
    int64_t nsw = (int64_t)sw->rows * sw->cols;
    for (int64_t j = 0; j < nsw; ++j) st->valid += sp4[4 * j + 3] != 0.0f;
    float *rowtab = (float *)malloc(sizeof(float) * 2 * (size_t)kp->rows);
    float *coltab = (float *)malloc(sizeof(float) * 2 * (size_t)kp->cols);
    orc_dir_table(kp, rowtab, coltab);
    for (int v = 0; v < kp->rows; ++v) {
        for (int u = 0; u < kp->cols; ++u) {
            double r, J[6];
            if (!associate(T, v, u, kf_depth, kf_nrm4, kp, rowtab, coltab, sp4, sn4, sw, ip, &r, J, 0)) continue;
            double w = 1.0;
            if (ip->loss == 1) {
                double ar = fabs(r);
                w = 1.0 / (ar > (double)ip->loss_delta ? ar : (double)ip->loss_delta);
            }
            int p = 0;
            for (int a = 0; a < 6; ++a)
                for (int c = a; c < 6; ++c) st->A[p++] += w * J[a] * J[c];
            for (int a = 0; a < 6; ++a) st->b[a] += w * J[a] * r;
            st->sse += w * r * r;
            st->inliers += 1;
        }
    }
    free(rowtab);
    free(coltab);
}

/*
 * One Gauss-Newton step: normal equations at T, solve A xi = -b, T <- exp(xi^) T.
 * A degenerate system (too few inliers, or a Cholesky pivot at or below
 * pivot_eps * max diagonal) leaves T unchanged and sets status 3.
 */
int orc_icp_step(const float *kf_depth, const float *kf_nrm4, const orc_pano *kp, const float *sp4,
                 const float *sn4, const orc_pano *sw, double *T, const orc_icp_params *ip, orc_icp_stats *st) {
    orc_icp_normal_equations(kf_depth, kf_nrm4, kp, sp4, sn4, sw, T, ip, st);
    if (st->inliers < ip->min_inliers) { st->status = 3; return 3; }
    double nb[6];
    for (int i = 0; i < 6; ++i) nb[i] = -st->b[i];
    if (orc_solve6(st->A, nb, ip->pivot_eps, st->xi)) { st->status = 3; return 3; }
    orc_se3_exp_left(st->xi, T);
    double wn = sqrt(st->xi[0] * st->xi[0] + st->xi[1] * st->xi[1] + st->xi[2] * st->xi[2]);
    double vn = sqrt(st->xi[3] * st->xi[3] + st->xi[4] * st->xi[4] + st->xi[5] * st->xi[5]);
    st->converged = (wn < ip->eps_rot && vn < ip->eps_trans) ? 1 : 0;
    return 0;
}

/* residual of keyframe pixel (v, u) under T (finite-difference checks); 1 if an inlier */
int orc_icp_residual(int32_t v, int32_t u, const float *kf_depth, const float *kf_nrm4, const orc_pano *kp,
                     const float *sp4, const float *sn4, const orc_pano *sw, const double *T,
                     const orc_icp_params *ip, double *r, double *J, int64_t *jpix) {
    float *rowtab = (float *)malloc(sizeof(float) * 2 * (size_t)kp->rows);
    float *coltab = (float *)malloc(sizeof(float) * 2 * (size_t)kp->cols);
    orc_dir_table(kp, rowtab, coltab);
    int ok = associate(T, v, u, kf_depth, kf_nrm4, kp, rowtab, coltab, sp4, sn4, sw, ip, r, J, jpix);
    free(rowtab);
    free(coltab);
    return ok;
}

/* ------------------------------------------------------------------ a4: keyframe fusion */

/*
 * Keyframe update (Sec. III-C) with the keyframe-from-sweep pose T.
 *
 * Gather: each keyframe pixel k holding a sample (w_k > 0) is put at its FP32
 * point d_k * dir_k, taken into the sweep frame, and binned into the sweep
 * panorama.  If the sweep pixel j there holds a point with a normal, and the two
 * pass the similarity test (distance <= d_max and normal cosine >= cos_theta_max,
 * in the keyframe frame), the keyframe pixel averages in the sweep sample:
 *   d_k <- (w_k d_k + |T P_j|) / (w_k + 1),  n_k <- unit(w_k n_k + R m_j),
 *   w_k <- min(w_k + 1, w_max).
 * Hole fill: every sweep pixel with a point and a normal is projected (FP32, as
 * a1) into the keyframe; each keyframe pixel that was empty (w_k == 0) takes the
 * nearest such sample (smallest (range, sweep pixel index)): d = |T P_j|,
 * n = R m_j, w = 1.
 *
 * kf_depth [H*W], kf_nrm [H*W*3], kf_w [H*W] are FP64 state updated in place;
 * their FP32 roundings kf_depth_f32 (the values a keyframe stores) drive the
 * pixel decisions.  Returns the number of keyframe pixels averaged.
 */
int64_t orc_fuse(double *kf_depth, double *kf_nrm, double *kf_w, const orc_pano *kp,
                 const float *sp4, const float *sn4, const orc_pano *sw, const double *T,
                 const orc_fuse_params *fp, int64_t *n_filled) {
    int64_t H = kp->rows, W = kp->cols, npx = H * W;
    float *rowtab = (float *)malloc(sizeof(float) * 2 * (size_t)H);
    float *coltab = (float *)malloc(sizeof(float) * 2 * (size_t)W);
    orc_dir_table(kp, rowtab, coltab);
    /* pixels empty before this sweep (the gather never touches them) */
    uint8_t *was_empty = (uint8_t *)malloc((size_t)npx);
    for (int64_t k = 0; k < npx; ++k) was_empty[k] = kf_w[k] == 0.0;
    int64_t fused = 0;
    for (int64_t v = 0; v < H; ++v) {
        for (int64_t u = 0; u < W; ++u) {
            int64_t k = v * W + u;
            if (was_empty[k]) continue;
            float dk = (float)kf_depth[k];
            float sx, sy, sz, qx, qy, qz;
            pixel_point_f32(rowtab, coltab, (int)v, (int)u, dk, &sx, &sy, &sz);
            orc_xform_inv_f32(T, sx, sy, sz, &qx, &qy, &qz);
            int32_t jv, ju;
            float rr;
            if (!orc_bin(qx, qy, qz, sw, &jv, &ju, &rr)) continue;
            int64_t j = (int64_t)jv * sw->cols + ju;
            const float *P = sp4 + 4 * j, *m = sn4 + 4 * j;
            if (P[3] == 0.0f || m[3] == 0.0f) continue;
            double dir[3], s[3], p[3], Rm[3];
            pixel_dir64(kp, (int)v, (int)u, dir);
            for (int i = 0; i < 3; ++i) {
                s[i] = kf_depth[k] * dir[i];
                p[i] = T[4 * i] * P[0] + T[4 * i + 1] * P[1] + T[4 * i + 2] * P[2] + T[4 * i + 3];
                Rm[i] = T[4 * i] * m[0] + T[4 * i + 1] * m[1] + T[4 * i + 2] * m[2];
            }
            double e0 = p[0] - s[0], e1 = p[1] - s[1], e2 = p[2] - s[2];
            if (!(sqrt(e0 * e0 + e1 * e1 + e2 * e2) <= (double)fp->d_max)) continue;
            double *n = kf_nrm + 3 * k;
            if (!(Rm[0] * n[0] + Rm[1] * n[1] + Rm[2] * n[2] >= (double)fp->cos_theta_max)) continue;
            double w = kf_w[k];
            double dm = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
            kf_depth[k] = (w * kf_depth[k] + dm) / (w + 1.0);
            double nn[3] = { w * n[0] + Rm[0], w * n[1] + Rm[1], w * n[2] + Rm[2] };
            double l = sqrt(nn[0] * nn[0] + nn[1] * nn[1] + nn[2] * nn[2]);
            n[0] = nn[0] / l; n[1] = nn[1] / l; n[2] = nn[2] / l;
            kf_w[k] = (w + 1.0 < (double)fp->w_max) ? w + 1.0 : (double)fp->w_max;
            ++fused;
        }
    }
    /* hole fill: lexicographic minimum of (FP32 range bits, sweep pixel index) per empty pixel */
    uint64_t *best = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)npx);
    for (int64_t k = 0; k < npx; ++k) best[k] = UINT64_MAX;
    int64_t nsw = (int64_t)sw->rows * sw->cols;
    for (int64_t j = 0; j < nsw; ++j) {
        const float *P = sp4 + 4 * j, *m = sn4 + 4 * j;
        if (P[3] == 0.0f || m[3] == 0.0f) continue;
        float px, py, pz, r;
        orc_xform_f32(T, P[0], P[1], P[2], &px, &py, &pz);
        int32_t v, u;
        if (!orc_bin(px, py, pz, kp, &v, &u, &r)) continue;
        int64_t k = (int64_t)v * W + u;
        if (!was_empty[k]) continue;
        uint32_t rb;
        memcpy(&rb, &r, 4);
        uint64_t key = ((uint64_t)rb << 32) | (uint32_t)j;
        if (key < best[k]) best[k] = key;
    }
    int64_t filled = 0;
    for (int64_t k = 0; k < npx; ++k) {
        if (best[k] == UINT64_MAX) continue;
        int64_t j = (int64_t)(best[k] & 0xffffffffu);
        const float *P = sp4 + 4 * j, *m = sn4 + 4 * j;
        double p[3], Rm[3];
        for (int i = 0; i < 3; ++i) {
            p[i] = T[4 * i] * P[0] + T[4 * i + 1] * P[1] + T[4 * i + 2] * P[2] + T[4 * i + 3];
            Rm[i] = T[4 * i] * m[0] + T[4 * i + 1] * m[1] + T[4 * i + 2] * m[2];
        }
        kf_depth[k] = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        double l = sqrt(Rm[0] * Rm[0] + Rm[1] * Rm[1] + Rm[2] * Rm[2]);
        kf_nrm[3 * k] = Rm[0] / l; kf_nrm[3 * k + 1] = Rm[1] / l; kf_nrm[3 * k + 2] = Rm[2] / l;
        kf_w[k] = 1.0;
        ++filled;
    }
    if (n_filled) *n_filled = filled;
    free(best);
    free(was_empty);
    free(rowtab);
    free(coltab);
    return fused;
}

/* ------------------------------------------------------------------ keyframe mutual consistency */

/*
 * Sec. III-C: when switching keyframes, a mutual consistency check between
 * keyframes filters moving objects from the map.  The paper gives no rule.
 * Reading: a sample of keyframe A is inconsistent with keyframe B when B's rays
 * around it measured surfaces beyond it, i.e. B saw through the place where
 * A's sample sat.  A's sample s = d dir (FP32 table point) is taken into B's
 * frame by T_ab^-1 (T_ab = pose of B in A, rounded to FP32, fixed order as
 * orc_xform_inv_f32) and binned into B with the FP32 rule (pixel j, range r).
 * It is flagged when B holds a depth at j and every pixel of the 3 x 3
 * neighbourhood of j (columns wrapped, rows clipped) that holds a depth exceeds
 * lim = (rel * r + abs) + r, formed in FP32.  The neighbourhood keeps a
 * half-pixel misalignment of the two keyframes' ray grids at a silhouette edge
 * from reading as a see-through.  flag_a[k] = 1 for flagged samples of A, else
 * 0.  Returns the number flagged.
 */
int64_t orc_consistency_flags(const float *depth_a, const orc_pano *pa, const float *depth_b, const orc_pano *pb,
                              const double *T_ab, float rel, float abs_m, uint8_t *flag_a) {
    float *rowtab = (float *)malloc(sizeof(float) * 2 * (size_t)pa->rows);
    float *coltab = (float *)malloc(sizeof(float) * 2 * (size_t)pa->cols);
    orc_dir_table(pa, rowtab, coltab);
    int64_t n = 0;
    for (int v = 0; v < pa->rows; ++v) {
        for (int u = 0; u < pa->cols; ++u) {
            int64_t k = (int64_t)v * pa->cols + u;
            flag_a[k] = 0;
            float d = depth_a[k];
            if (!(d > 0.0f)) continue;
            float sx, sy, sz, qx, qy, qz;
            pixel_point_f32(rowtab, coltab, v, u, d, &sx, &sy, &sz);
            orc_xform_inv_f32(T_ab, sx, sy, sz, &qx, &qy, &qz);
            int32_t jv, ju;
            float r;
            if (!orc_bin(qx, qy, qz, pb, &jv, &ju, &r)) continue;
            if (!(depth_b[(int64_t)jv * pb->cols + ju] > 0.0f)) continue;
            float lim = (rel * r + abs_m) + r;
            int seen_through = 1;
            for (int dv = -1; dv <= 1 && seen_through; ++dv) {
                int vv = jv + dv;
                if (vv < 0 || vv >= pb->rows) continue;
                for (int du = -1; du <= 1; ++du) {
                    int uu = ju + du;
                    if (uu < 0) uu += pb->cols;
                    if (uu >= pb->cols) uu -= pb->cols;
                    float dn = depth_b[(int64_t)vv * pb->cols + uu];
                    if (dn > 0.0f && !(dn > lim)) {
                        seen_through = 0;
                        break;
                    }
                }
            }
            if (seen_through) {
                flag_a[k] = 1;
                ++n;
            }
        }
    }
    free(rowtab);
    free(coltab);
    return n;
}

/*
 * Inverse of a rigid pose in a fixed FP64 order: R' = R^T (exact) and
 * t'_i = -((R_0i t_0 + R_1i t_1) + R_2i t_2), so any implementation that
 * follows the same order obtains the same bits.
 */
void orc_pose_inv_fixed(const double *T, double *out) {
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) out[4 * i + j] = T[4 * j + i];
        out[4 * i + 3] = -((T[i] * T[3] + T[4 + i] * T[7]) + T[8 + i] * T[11]);
    }
}

/* ------------------------------------------------------------------ motion prior */

/*
 * Sec. IV-F footnote: the registration of a sweep starts from a motion prior,
 * zero velocity by default (the previous sweep's pose) or zero acceleration
 * (the previous pose carried on by the last inter-sweep motion).  Poses are
 * 3x4 [R | t] maps sweep -> keyframe, so the sweep-to-sweep motion is
 * M = T_prev^-1 T and the zero-acceleration guess is T_prev M.
 *
 * Reading: after each product the rotation is put back on SO(3) by
 * Gram-Schmidt on its rows (r0 normalised, r1 minus its r0 component then
 * normalised, r2 = r0 x r1), so that rounding cannot compound over a long
 * sequence.  Plain FP64 with sqrt and division.
 */
static void pose_mul34(const double *A, const double *B, double *C) {
    double t[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[4 * i + k] * B[4 * k + j];
            if (j == 3) s += A[4 * i + 3];
            t[4 * i + j] = s;
        }
    }
    memcpy(C, t, sizeof(t));
}

void orc_orthonormalise_rows(double *T) {
    double *r0 = T, *r1 = T + 4, *r2 = T + 8;
    double n0 = sqrt(r0[0] * r0[0] + r0[1] * r0[1] + r0[2] * r0[2]);
    for (int i = 0; i < 3; ++i) r0[i] /= n0;
    double d = r0[0] * r1[0] + r0[1] * r1[1] + r0[2] * r1[2];
    for (int i = 0; i < 3; ++i) r1[i] -= d * r0[i];
    double n1 = sqrt(r1[0] * r1[0] + r1[1] * r1[1] + r1[2] * r1[2]);
    for (int i = 0; i < 3; ++i) r1[i] /= n1;
    r2[0] = r0[1] * r1[2] - r0[2] * r1[1];
    r2[1] = r0[2] * r1[0] - r0[0] * r1[2];
    r2[2] = r0[0] * r1[1] - r0[1] * r1[0];
}

/* Initial guess: T_out = T_prev (M == NULL, zero velocity) or T_prev M re-orthonormalised. */
void orc_predict_pose(const double *T_prev, const double *M, double *T_out) {
    double t[12];
    if (!M) {
        memcpy(t, T_prev, sizeof(t));
    } else {
        pose_mul34(T_prev, M, t);
        orc_orthonormalise_rows(t);
    }
    memcpy(T_out, t, sizeof(t));
}

/* Last inter-sweep motion: M = T_prev^-1 T (T_prev^-1 = [R^T | -R^T t]), re-orthonormalised. */
void orc_update_motion(const double *T_prev, const double *T, double *M) {
    double inv[12], t[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) inv[4 * i + j] = T_prev[4 * j + i];
        inv[4 * i + 3] = -(T_prev[i] * T_prev[3] + T_prev[4 + i] * T_prev[7] + T_prev[8 + i] * T_prev[11]);
    }
    pose_mul34(inv, T, t);
    orc_orthonormalise_rows(t);
    memcpy(M, t, sizeof(t));
}
