// Keyframe update (UPSLAM Sec. III-C).
//
// With the optimised T, every keyframe pixel holding a sample is projected onto
// the sweep depth image (the same keyframe-to-sweep correspondence as the ICP
// step).  When the similarity gate keeps the pair, the pixel averages the sweep
// sample in with its sample count as weight, and the count saturates at w_max:
//   d <- (w d + |T s2|) / (w + 1),  n <- unit(w n + R m),  w <- min(w + 1, w_max).
// Empty keyframe pixels are filled from the sweep (hole fill): every sweep pixel
// with a point and a normal is binned into the keyframe with T; each empty
// pixel keeps its nearest sample via an atomicMin z-buffer on
// (bits(range) << 32 | sweep pixel index), then takes d = range, n = R m, w = 1.
//
// Launches:
//  1. fuse_main_kernel: CTAs [0, gk) average keyframe pixels in place; CTAs
//     [gk, gk + gs) run the hole-fill atomics.  The two touch disjoint pixels
//     (averaging only writes pixels with w > 0, hole fill only targets w == 0).
//  2. fuse_fill_kernel: each sweep pixel re-derives its key; the one whose key
//     won writes the pixel and resets the z-buffer word to all-ones.
// Both launches read the registration record first and do nothing unless the
// sweep was accepted (inliers / valid >= accept_quality, status OK).
//
// Roofline: the keyframe is streamed once in and once out: 4 + 16 B (FP32) or
// 4 + 8 B (FP16) each way per pixel, plus sweep gathers from L2.
#include "common.cuh"

namespace upslam {

struct FuseArgs {
    upslam_pano kp;
    float *kdepth;
    void *knw;
    int kprec;
    const float *kdirs;
    upslam_pano sp;
    const float4 *spix;
    const void *snrm;
    int sprec;
    float d_max2, cos_min, w_max, accept;
};

__device__ __forceinline__ bool accepted(const upslam_icp_stats *st, float accept) {
    if (!st) return true;
    if (st->status != UPSLAM_OK) return false;
    const long long valid = st->valid;
    return valid > 0 && (double)st->inliers >= (double)accept * (double)valid;
}

__global__ void __launch_bounds__(256) fuse_main_kernel(FuseArgs a, const double *pose, upslam_icp_stats *st,
                                                        unsigned long long *__restrict__ zbuf, int gk) {
    if (!accepted(st, a.accept)) return;
    const PoseF T = pose_to_f32(pose);
    if ((int)blockIdx.x < gk) {
        // averaging: each thread takes 4 pixels a CTA-width apart, issuing their keyframe loads together
        constexpr int kB = 4;
        const int npx = a.kp.rows * a.kp.cols;
        const int W = a.kp.cols;
        const int stride = gk * blockDim.x * kB;
        for (int base = blockIdx.x * blockDim.x * kB + threadIdx.x; base < npx; base += stride) {
            float4 n[kB];
            float d[kB];
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const int k = base + b * blockDim.x;
                n[b] = k < npx ? load_nw(a.knw, k, a.kprec) : make_float4(0.f, 0.f, 0.f, 0.f);
                d[b] = k < npx ? __ldg(a.kdepth + k) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const int k = base + b * blockDim.x;
                const float w = n[b].w;
                if (!(w > 0.0f)) continue;
                const int v = k / W, u = k - v * W;
                const float3 s = pixel_point(a.kdirs, a.kp.rows, v, u, d[b]);
                const float3 q = xform_inv(T, s.x, s.y, s.z);
                int jv, ju;
                float rr;
                if (!bin_point(q.x, q.y, q.z, a.sp, jv, ju, rr)) continue;
                const int j = jv * a.sp.cols + ju;
                const float4 P = __ldg(a.spix + j);
                const float4 m = load_nw(a.snrm, j, a.sprec);
                if (P.w == 0.0f || m.w == 0.0f) continue;
                const float *r = T.r;
                const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
                const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
                const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
                const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
                if (!(ex * ex + ey * ey + ez * ez <= a.d_max2)) continue;
                const float3 Rm = rotate(T, m.x, m.y, m.z);
                const float4 nk = n[b];
                if (!(Rm.x * nk.x + Rm.y * nk.y + Rm.z * nk.z >= a.cos_min)) continue;
                const float dm = sqrtf(px * px + py * py + pz * pz);
                const float inv = 1.0f / (w + 1.0f);
                a.kdepth[k] = (w * d[b] + dm) * inv;
                const float nx = w * nk.x + Rm.x, ny = w * nk.y + Rm.y, nz = w * nk.z + Rm.z;
                const float l = rsqrtf(nx * nx + ny * ny + nz * nz);
                const float wn = w + 1.0f < a.w_max ? w + 1.0f : a.w_max;
                store_nw(a.knw, k, a.kprec, make_float4(nx * l, ny * l, nz * l, wn));
            }
        }
    } else {
        const int ns = a.sp.rows * a.sp.cols;
        const int gs = gridDim.x - gk;
        for (int j = (blockIdx.x - gk) * blockDim.x + threadIdx.x; j < ns; j += gs * blockDim.x) {
            const float4 P = __ldg(a.spix + j);
            if (P.w == 0.0f) continue;
            const float4 m = load_nw(a.snrm, j, a.sprec);
            if (m.w == 0.0f) continue;
            const float3 p = xform(T, P.x, P.y, P.z);
            int v, u;
            float r;
            if (!bin_point(p.x, p.y, p.z, a.kp, v, u, r)) continue;
            const int k = v * a.kp.cols + u;
            if (load_nw(a.knw, k, a.kprec).w != 0.0f) continue;
            atomicMin(zbuf + k, ((unsigned long long)__float_as_uint(r) << 32) | (unsigned int)j);
        }
    }
}

__global__ void __launch_bounds__(256) fuse_fill_kernel(FuseArgs a, const double *pose, upslam_icp_stats *st,
                                                        unsigned long long *__restrict__ zbuf) {
    if (!accepted(st, a.accept)) return;
    const PoseF T = pose_to_f32(pose);
    const int ns = a.sp.rows * a.sp.cols;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
        const float4 P = __ldg(a.spix + j);
        if (P.w == 0.0f) continue;
        const float4 m = load_nw(a.snrm, j, a.sprec);
        if (m.w == 0.0f) continue;
        const float3 p = xform(T, P.x, P.y, P.z);
        int v, u;
        float r;
        if (!bin_point(p.x, p.y, p.z, a.kp, v, u, r)) continue;
        const int k = v * a.kp.cols + u;
        const unsigned long long key = ((unsigned long long)__float_as_uint(r) << 32) | (unsigned int)j;
        if (zbuf[k] != key) continue;
        zbuf[k] = kEmptyKey;
        const float3 Rm = rotate(T, m.x, m.y, m.z);
        const float l = 1.0f / sqrtf(Rm.x * Rm.x + Rm.y * Rm.y + Rm.z * Rm.z);
        a.kdepth[k] = r;
        store_nw(a.knw, k, a.kprec, make_float4(Rm.x * l, Rm.y * l, Rm.z * l, 1.0f));
    }
    if (st && blockIdx.x == 0 && threadIdx.x == 0) st->accepted = 1;
}

}  // namespace upslam

using namespace upslam;

extern "C" upslam_status upslam_fuse(const upslam_keyframe *kf, const upslam_sweep *sw, const double *d_pose12,
                                     const upslam_fuse_params *fp, upslam_icp_stats *d_stats, uint64_t *d_zbuf_kf,
                                     void *stream) {
    if (!kf || !sw || !fp || !d_pose12 || !d_zbuf_kf) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_pano_ok(&kf->pano) || !upslam_pano_ok(&sw->pano) || !kf->d_depth || !kf->d_nw || !kf->d_dirs ||
        !sw->d_pix || !sw->d_nrm)
        return UPSLAM_ERR_INVALID_ARG;
    if ((kf->precision != UPSLAM_F32 && kf->precision != UPSLAM_F16) ||
        (sw->nrm_precision != UPSLAM_F32 && sw->nrm_precision != UPSLAM_F16))
        return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_aligned(kf->d_nw, kf->precision == UPSLAM_F32 ? 16 : 8) || !upslam_aligned(d_zbuf_kf, 8) ||
        !upslam_aligned(sw->d_pix, 16) || !upslam_aligned(kf->d_dirs, 8))
        return UPSLAM_ERR_INVALID_ARG;
    if (!(fp->w_max >= 1.0f) || !(fp->d_max > 0.0f)) return UPSLAM_ERR_INVALID_ARG;
    FuseArgs a;
    a.kp = kf->pano;
    a.kdepth = kf->d_depth;
    a.knw = kf->d_nw;
    a.kprec = kf->precision;
    a.kdirs = kf->d_dirs;
    a.sp = sw->pano;
    a.spix = reinterpret_cast<const float4 *>(sw->d_pix);
    a.snrm = sw->d_nrm;
    a.sprec = sw->nrm_precision;
    a.d_max2 = fp->d_max * fp->d_max;
    a.cos_min = fp->cos_theta_max;
    a.w_max = fp->w_max;
    a.accept = fp->accept_quality;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *zb = reinterpret_cast<unsigned long long *>(d_zbuf_kf);
    const int64_t npx = (int64_t)kf->pano.rows * kf->pano.cols;
    const int64_t ns = (int64_t)sw->pano.rows * sw->pano.cols;
    const int gk = upslam_grid((npx + 3) / 4, 256, 8);
    const int gs = upslam_grid(ns, 256, 2);
    fuse_main_kernel<<<gk + gs, 256, 0, s>>>(a, d_pose12, d_stats, zb, gk);
    UPSLAM_CHECK_LAUNCH();
    fuse_fill_kernel<<<gs, 256, 0, s>>>(a, d_pose12, d_stats, zb);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}
