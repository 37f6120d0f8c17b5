// GPU version of the analytic ray caster (input generation only, FP32).
//
// Same primitives as raycast.c; used to make the many sweeps that training
// pairs for the pose-proposal network need.  One thread per ray, B sensor poses
// per launch.  Returns the range of the nearest hit (or -1).  Holds none of the
// registration or fusion arithmetic.
//
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -Xcompiler -fPIC -shared raycast_cuda.cu
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#define STRIDE 16

struct Hit {
    float t;
};

__device__ __forceinline__ void consider(Hit &h, float t) {
    if (t > 1e-4f && t < h.t) h.t = t;
}

__device__ void hit_plane(const float *p, const float *o, const float *d, Hit &h) {
    const float den = d[0] * p[4] + d[1] * p[5] + d[2] * p[6];
    if (fabsf(den) < 1e-9f) return;
    consider(h, ((p[1] - o[0]) * p[4] + (p[2] - o[1]) * p[5] + (p[3] - o[2]) * p[6]) / den);
}

__device__ void hit_obb(const float *p, const float *o, const float *d, Hit &h) {
    float s, c;
    sincosf(p[7], &s, &c);
    const float ox = o[0] - p[1], oy = o[1] - p[2], oz = o[2] - p[3];
    const float lo[3] = {c * ox + s * oy, -s * ox + c * oy, oz};
    const float ld[3] = {c * d[0] + s * d[1], -s * d[0] + c * d[1], d[2]};
    const float he[3] = {p[4], p[5], p[6]};
    float tn = -1e30f, tf = 1e30f;
    for (int k = 0; k < 3; ++k) {
        if (fabsf(ld[k]) < 1e-12f) {
            if (lo[k] < -he[k] || lo[k] > he[k]) return;
            continue;
        }
        float t1 = (-he[k] - lo[k]) / ld[k], t2 = (he[k] - lo[k]) / ld[k];
        if (t1 > t2) {
            const float tmp = t1;
            t1 = t2;
            t2 = tmp;
        }
        tn = fmaxf(tn, t1);
        tf = fminf(tf, t2);
    }
    if (tn > tf || tf <= 1e-4f || tn <= 1e-4f) return;
    consider(h, tn);
}

__device__ void hit_room(const float *p, const float *o, const float *d, Hit &h) {
    float tb = 1e30f;
    for (int k = 0; k < 3; ++k) {
        if (fabsf(d[k]) < 1e-12f) continue;
        const float b = d[k] > 0 ? p[4 + k] : p[1 + k];
        tb = fminf(tb, (b - o[k]) / d[k]);
    }
    if (tb < 1e29f) consider(h, tb);
}

__device__ void hit_vcyl(const float *p, const float *o, const float *d, Hit &h) {
    const float fx = o[0] - p[1], fy = o[1] - p[2], r = p[3];
    const float a = d[0] * d[0] + d[1] * d[1];
    if (a < 1e-12f) return;
    const float b = fx * d[0] + fy * d[1];
    const float cc = fx * fx + fy * fy - r * r;
    if (cc <= 0) return;
    const float disc = b * b - a * cc;
    if (disc < 0) return;
    const float t = (-b - sqrtf(disc)) / a;
    const float z = o[2] + t * d[2];
    if (z < p[4] || z > p[5]) return;
    consider(h, t);
}

__device__ void hit_arch(const float *p, const float *o, const float *d, Hit &h) {
    float s, c;
    sincosf(p[4], &s, &c);
    const float R = p[5], L = p[6];
    const float ox = o[0] - p[1], oy = o[1] - p[2], oz = o[2] - p[3];
    const float lu = c * ox + s * oy, lw = -s * ox + c * oy;
    const float du = c * d[0] + s * d[1], dw = -s * d[0] + c * d[1], dz = d[2];
    const float a = dw * dw + dz * dz;
    if (a < 1e-12f) return;
    const float b = lw * dw + oz * dz;
    const float cc = lw * lw + oz * oz - R * R;
    const float disc = b * b - a * cc;
    if (disc < 0) return;
    const float sq = sqrtf(disc);
    const float roots[2] = {(-b - sq) / a, (-b + sq) / a};
    for (int k = 0; k < 2; ++k) {
        const float t = roots[k];
        if (t <= 1e-4f) continue;
        const float zz = oz + t * dz, uu = lu + t * du;
        if (zz < 0 || uu < 0 || uu > L) continue;
        consider(h, t);
        return;
    }
}

__device__ float lattice(long long i, long long j, unsigned long long seed) {
    unsigned long long x = (unsigned long long)i * 0x9E3779B97F4A7C15ull ^ ((unsigned long long)j * 0xC2B2AE3D27D4EB4Full) ^ seed;
    x ^= x >> 30;
    x *= 0xBF58476D1CE4E5B9ull;
    x ^= x >> 27;
    x *= 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (float)((double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

__device__ float hfield(const float *p, float x, float y) {
    const float amp = p[1], cell = p[2], zb = p[4];
    const unsigned long long seed = (unsigned long long)p[3];
    const float fx = x / cell, fy = y / cell;
    const float ix = floorf(fx), iy = floorf(fy);
    const float tx = fx - ix, ty = fy - iy;
    const long long i = (long long)ix, j = (long long)iy;
    const float v00 = lattice(i, j, seed), v10 = lattice(i + 1, j, seed);
    const float v01 = lattice(i, j + 1, seed), v11 = lattice(i + 1, j + 1, seed);
    const float sx = tx * tx * (3.f - 2.f * tx), sy = ty * ty * (3.f - 2.f * ty);
    const float a = v00 + (v10 - v00) * sx, b = v01 + (v11 - v01) * sx;
    return zb + amp * (a + (b - a) * sy);
}

__device__ void hit_hfield(const float *p, const float *o, const float *d, Hit &h, float tmax) {
    const float amp = fabsf(p[1]), zb = p[4];
    float t0 = 0.f, t1 = tmax;
    if (fabsf(d[2]) > 1e-12f) {
        float ta = (zb - amp - o[2]) / d[2], tb = (zb + amp - o[2]) / d[2];
        if (ta > tb) {
            const float tmp = ta;
            ta = tb;
            tb = tmp;
        }
        t0 = fmaxf(t0, ta);
        t1 = fminf(t1, tb);
    } else if (o[2] > zb + amp || o[2] < zb - amp) {
        return;
    }
    if (t1 <= t0) return;
    t1 = fminf(t1, h.t);
    const float step = 0.2f * p[2];
    float tprev = t0;
    float fprev = o[2] + t0 * d[2] - hfield(p, o[0] + t0 * d[0], o[1] + t0 * d[1]);
    if (fprev < 0) return;
    for (int guard = 0; guard < 100000; ++guard) {
        float t = fminf(tprev + step, t1);
        const float f = o[2] + t * d[2] - hfield(p, o[0] + t * d[0], o[1] + t * d[1]);
        if (f < 0) {
            float a = tprev, b = t;
            for (int it = 0; it < 30; ++it) {
                const float m = 0.5f * (a + b);
                if (o[2] + m * d[2] - hfield(p, o[0] + m * d[0], o[1] + m * d[1]) < 0) b = m;
                else a = m;
            }
            consider(h, 0.5f * (a + b));
            return;
        }
        if (t >= t1) return;
        tprev = t;
    }
}

__global__ void cast_kernel(const float *__restrict__ prims, int nprims, const float *__restrict__ origins,
                            const float *__restrict__ rots, const float *__restrict__ dirs, int n, int B, float tmax,
                            float *__restrict__ t_out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)n * B) return;
    const int b = (int)(i / n), r = (int)(i % n);
    const float *R = rots + 9 * b;
    const float *ds = dirs + 3 * r;
    const float d[3] = {R[0] * ds[0] + R[1] * ds[1] + R[2] * ds[2], R[3] * ds[0] + R[4] * ds[1] + R[5] * ds[2],
                        R[6] * ds[0] + R[7] * ds[1] + R[8] * ds[2]};
    const float *o = origins + 3 * b;
    Hit h;
    h.t = tmax;
    int hf = -1;
    for (int k = 0; k < nprims; ++k) {
        const float *p = prims + STRIDE * k;
        switch ((int)p[0]) {
            case 0: hit_plane(p, o, d, h); break;
            case 1: hit_obb(p, o, d, h); break;
            case 2: hit_room(p, o, d, h); break;
            case 3: hit_vcyl(p, o, d, h); break;
            case 4: hit_arch(p, o, d, h); break;
            case 5: hf = k; break;
            default: break;
        }
    }
    if (hf >= 0) hit_hfield(prims + STRIDE * hf, o, d, h, tmax);
    t_out[i] = h.t < tmax ? h.t : -1.0f;
}

extern "C" int synth_cast_cuda(const float *d_prims, int nprims, const float *d_origins, const float *d_rots,
                               const float *d_dirs, int n, int B, float tmax, float *d_t, void *stream) {
    const long long total = (long long)n * B;
    if (total <= 0) return 0;
    cast_kernel<<<(unsigned)((total + 255) / 256), 256, 0, (cudaStream_t)stream>>>(d_prims, nprims, d_origins, d_rots,
                                                                                   d_dirs, n, B, tmax, d_t);
    return cudaPeekAtLastError() == cudaSuccess ? 0 : 1;
}
