/*
 * Analytic ray caster for the seeded synthetic lidar scenes.
 *
 * This is input generation only: it turns a procedural scene description into
 * exact ranges and surface normals along given rays.  It holds none of the
 * registration / fusion arithmetic, and both the CPU oracle and the CUDA path
 * consume what it produces.
 *
 * A scene is a flat array of primitives, SYNTH_PRIM_STRIDE doubles each, the
 * first double being the primitive type.  All arithmetic is FP64.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp raycast.c -o _raycast.so -lm
 */
#include <math.h>
#include <stdint.h>

#define SYNTH_PRIM_STRIDE 16

enum {
    PRIM_PLANE = 0,      /* c(3) n(3)                          infinite one-sided-agnostic plane   */
    PRIM_OBB = 1,        /* c(3) h(3) yaw                      solid box rotated about z           */
    PRIM_ROOM = 2,       /* lo(3) hi(3)                        interior of an axis-aligned box     */
    PRIM_VCYL = 3,       /* cx cy r z0 z1                      solid vertical cylinder             */
    PRIM_ARCH = 4,       /* c(3) yaw R L                       interior of a horizontal half-tube  */
    PRIM_HFIELD = 5      /* amp cell seed zbase                value-noise height field z = h(x,y) */
};

#define T_EPS 1e-6

typedef struct { double t; double n[3]; int id; } hit_t;

static void consider(hit_t *h, double t, double nx, double ny, double nz, int id) {
    if (t > T_EPS && t < h->t) { h->t = t; h->n[0] = nx; h->n[1] = ny; h->n[2] = nz; h->id = id; }
}

/* ---------------- primitives ---------------- */

static void hit_plane(const double *p, const double *o, const double *d, hit_t *h, int id) {
    double nx = p[4], ny = p[5], nz = p[6];
    double den = d[0] * nx + d[1] * ny + d[2] * nz;
    if (fabs(den) < 1e-12) return;
    double t = ((p[1] - o[0]) * nx + (p[2] - o[1]) * ny + (p[3] - o[2]) * nz) / den;
    if (den > 0) { nx = -nx; ny = -ny; nz = -nz; }
    consider(h, t, nx, ny, nz, id);
}

static void hit_obb(const double *p, const double *o, const double *d, hit_t *h, int id) {
    double c = cos(p[7]), s = sin(p[7]);
    /* ray into the box frame (rotate by -yaw about z) */
    double ox = o[0] - p[1], oy = o[1] - p[2], oz = o[2] - p[3];
    double lo[3] = { c * ox + s * oy, -s * ox + c * oy, oz };
    double ld[3] = { c * d[0] + s * d[1], -s * d[0] + c * d[1], d[2] };
    double he[3] = { p[4], p[5], p[6] };
    double tn = -1e300, tf = 1e300; int ax = -1; double sg = 0;
    for (int k = 0; k < 3; ++k) {
        if (fabs(ld[k]) < 1e-15) {
            if (lo[k] < -he[k] || lo[k] > he[k]) return;
            continue;
        }
        double t1 = (-he[k] - lo[k]) / ld[k], t2 = (he[k] - lo[k]) / ld[k];
        double s1 = -1.0;
        if (t1 > t2) { double tmp = t1; t1 = t2; t2 = tmp; s1 = 1.0; }
        if (t1 > tn) { tn = t1; ax = k; sg = s1; }
        if (t2 < tf) tf = t2;
    }
    if (tn > tf || tf <= T_EPS || ax < 0 || tn <= T_EPS) return;
    double ln[3] = { 0, 0, 0 }; ln[ax] = sg;
    consider(h, tn, c * ln[0] - s * ln[1], s * ln[0] + c * ln[1], ln[2], id);
}

static void hit_room(const double *p, const double *o, const double *d, hit_t *h, int id) {
    double tbest = 1e300; int ax = -1; double sg = 0;
    for (int k = 0; k < 3; ++k) {
        if (fabs(d[k]) < 1e-15) continue;
        double b = d[k] > 0 ? p[4 + k] : p[1 + k];
        double t = (b - o[k]) / d[k];
        if (t < tbest) { tbest = t; ax = k; sg = d[k] > 0 ? -1.0 : 1.0; }
    }
    if (ax < 0) return;
    double n[3] = { 0, 0, 0 }; n[ax] = sg;
    consider(h, tbest, n[0], n[1], n[2], id);
}

static void hit_vcyl(const double *p, const double *o, const double *d, hit_t *h, int id) {
    double fx = o[0] - p[1], fy = o[1] - p[2], r = p[3];
    double a = d[0] * d[0] + d[1] * d[1];
    if (a < 1e-15) return;
    double b = fx * d[0] + fy * d[1];
    double cc = fx * fx + fy * fy - r * r;
    if (cc <= 0) return; /* origin inside the trunk */
    double disc = b * b - a * cc;
    if (disc < 0) return;
    double t = (-b - sqrt(disc)) / a;
    double z = o[2] + t * d[2];
    if (z < p[4] || z > p[5]) return;
    double nx = (fx + t * d[0]) / r, ny = (fy + t * d[1]) / r;
    consider(h, t, nx, ny, 0.0, id);
}

static void hit_arch(const double *p, const double *o, const double *d, hit_t *h, int id) {
    /* local frame: u along the tube axis (yaw), w lateral, z up; origin at the axis start */
    double c = cos(p[4]), s = sin(p[4]), R = p[5], L = p[6];
    double ox = o[0] - p[1], oy = o[1] - p[2], oz = o[2] - p[3];
    double lu = c * ox + s * oy, lw = -s * ox + c * oy;
    double du = c * d[0] + s * d[1], dw = -s * d[0] + c * d[1], dz = d[2];
    double a = dw * dw + dz * dz;
    if (a < 1e-15) return;
    double b = lw * dw + oz * dz;
    double cc = lw * lw + oz * oz - R * R;
    double disc = b * b - a * cc;
    if (disc < 0) return;
    double sq = sqrt(disc);
    double roots[2] = { (-b - sq) / a, (-b + sq) / a };
    for (int k = 0; k < 2; ++k) {
        double t = roots[k];
        if (t <= T_EPS) continue;
        double zz = oz + t * dz, uu = lu + t * du, ww = lw + t * dw;
        if (zz < 0 || uu < 0 || uu > L) continue;
        /* normal of the tube surface, pointing toward the axis */
        double nw = -ww / R, nz = -zz / R;
        double nx = -s * nw, ny = c * nw;
        double dn = nx * d[0] + ny * d[1] + nz * d[2];
        if (dn > 0) { nx = -nx; ny = -ny; nz = -nz; }
        consider(h, t, nx, ny, nz, id);
        return;
    }
}

/* value noise on an integer lattice, hashed from the lattice coordinates and a seed */
static double lattice(int64_t i, int64_t j, uint64_t seed) {
    uint64_t x = (uint64_t)i * 0x9E3779B97F4A7C15ull ^ ((uint64_t)j * 0xC2B2AE3D27D4EB4Full) ^ seed;
    x ^= x >> 30; x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27; x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static double smooth(double f) { return f * f * (3.0 - 2.0 * f); }
static double dsmooth(double f) { return 6.0 * f * (1.0 - f); }

/* height and its gradient */
static double hfield(const double *p, double x, double y, double *gx, double *gy) {
    double amp = p[1], cell = p[2], zb = p[4];
    uint64_t seed = (uint64_t)p[3];
    double fx = x / cell, fy = y / cell;
    double ix = floor(fx), iy = floor(fy);
    double tx = fx - ix, ty = fy - iy;
    int64_t i = (int64_t)ix, j = (int64_t)iy;
    double v00 = lattice(i, j, seed), v10 = lattice(i + 1, j, seed);
    double v01 = lattice(i, j + 1, seed), v11 = lattice(i + 1, j + 1, seed);
    double sx = smooth(tx), sy = smooth(ty);
    double a = v00 + (v10 - v00) * sx, b = v01 + (v11 - v01) * sx;
    double hval = a + (b - a) * sy;
    if (gx) {
        double dsx = dsmooth(tx) / cell, dsy = dsmooth(ty) / cell;
        double dax = (v10 - v00) * dsx, dbx = (v11 - v01) * dsx;
        *gx = amp * (dax + (dbx - dax) * sy);
        *gy = amp * (b - a) * dsy;
    }
    return zb + amp * hval;
}

static void hit_hfield(const double *p, const double *o, const double *d, hit_t *h, int id, double tmax) {
    double amp = fabs(p[1]), zb = p[4];
    /* the surface lies in the slab |z - zb| <= amp */
    double t0 = 0, t1 = tmax;
    if (fabs(d[2]) > 1e-15) {
        double ta = (zb - amp - o[2]) / d[2], tb = (zb + amp - o[2]) / d[2];
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    } else if (o[2] > zb + amp || o[2] < zb - amp) return;
    if (t1 <= t0) return;
    if (t1 > h->t) t1 = h->t;
    double step = 0.2 * p[2];
    double tprev = t0;
    double fprev = o[2] + t0 * d[2] - hfield(p, o[0] + t0 * d[0], o[1] + t0 * d[1], 0, 0);
    if (fprev < 0) return;
    for (double t = t0 + step;; t += step) {
        if (t > t1) t = t1;
        double f = o[2] + t * d[2] - hfield(p, o[0] + t * d[0], o[1] + t * d[1], 0, 0);
        if (f < 0) {
            double a = tprev, b = t;
            for (int it = 0; it < 60; ++it) {
                double m = 0.5 * (a + b);
                double fm = o[2] + m * d[2] - hfield(p, o[0] + m * d[0], o[1] + m * d[1], 0, 0);
                if (fm < 0) b = m; else a = m;
            }
            double tt = 0.5 * (a + b), gx, gy;
            hfield(p, o[0] + tt * d[0], o[1] + tt * d[1], &gx, &gy);
            double nn = sqrt(gx * gx + gy * gy + 1.0);
            consider(h, tt, -gx / nn, -gy / nn, 1.0 / nn, id);
            return;
        }
        if (t >= t1) return;
        tprev = t;
    }
}

/*
 * Cast n rays from origin o (world) with unit directions d_world (n x 3).
 * t_out[i] = range of the nearest hit (or -1), n_out = world normal facing the
 * ray, id_out = primitive index (or -1).  Hits beyond tmax are dropped.
 */
int synth_cast(const double *prims, int nprims, const double *o, const double *dirs, int n,
               double tmax, double *t_out, double *n_out, int32_t *id_out) {
    #pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < n; ++i) {
        const double *d = dirs + 3 * (int64_t)i;
        hit_t h; h.t = tmax; h.n[0] = h.n[1] = h.n[2] = 0; h.id = -1;
        for (int k = 0; k < nprims; ++k) {
            const double *p = prims + (int64_t)SYNTH_PRIM_STRIDE * k;
            switch ((int)p[0]) {
                case PRIM_PLANE: hit_plane(p, o, d, &h, k); break;
                case PRIM_OBB: hit_obb(p, o, d, &h, k); break;
                case PRIM_ROOM: hit_room(p, o, d, &h, k); break;
                case PRIM_VCYL: hit_vcyl(p, o, d, &h, k); break;
                case PRIM_ARCH: hit_arch(p, o, d, &h, k); break;
                default: break;
            }
        }
        /* height fields last: their march is clipped at the nearest analytic hit */
        for (int k = 0; k < nprims; ++k) {
            const double *p = prims + (int64_t)SYNTH_PRIM_STRIDE * k;
            if ((int)p[0] == PRIM_HFIELD) hit_hfield(p, o, d, &h, k, tmax);
        }
        if (h.id < 0) { t_out[i] = -1.0; n_out[3 * (int64_t)i] = n_out[3 * (int64_t)i + 1] = n_out[3 * (int64_t)i + 2] = 0; }
        else {
            t_out[i] = h.t;
            n_out[3 * (int64_t)i] = h.n[0]; n_out[3 * (int64_t)i + 1] = h.n[1]; n_out[3 * (int64_t)i + 2] = h.n[2];
        }
        id_out[i] = h.id;
    }
    return 0;
}

/* terrain height lookup for placing trajectories and trunks on the ground */
double synth_hfield_height(const double *prim, double x, double y) {
    return hfield(prim, x, y, 0, 0);
}
