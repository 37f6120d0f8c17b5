// Keyframe update (UPSLAM Sec. III-C).
//
// With the optimised T, every keyframe pixel holding a sample is carried over to
// the sweep's depth image (the same keyframe-to-sweep correspondence as the ICP
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
//     (a pixel holds a sample exactly when its depth and count are positive;
//     averaging only writes such pixels, hole fill only targets depth 0).
//  2. fuse_fill_kernel: each sweep pixel re-derives its key; the one whose key
//     won writes the pixel and resets the z-buffer word to all-ones.  Launched as
//     a programmatic dependent of the first, so its CTAs are placed while the
//     first drains; it waits for the first's results before it reads anything.
// Both launches read the registration record first and do nothing unless the
// sweep was accepted (inliers / valid >= accept_quality, status OK).  The same
// per-pixel functions (common.cuh) serve the fused register + update launch.
//
// Roofline: the keyframe is streamed once in and once out: 4 + 16 B (FP32) or
// 4 + 8 B (FP16) each way per pixel, plus sweep gathers from L2.  Empty pixels
// are read only as far as their depth.
#include "common.cuh"

namespace upslam {

constexpr int kFuseB = 2;  // keyframe pixels per averaging thread and iteration

// Registration accepted?  Decided by one thread per CTA (in FP32, off the FP64 pipe) and broadcast.
__device__ __forceinline__ bool accepted(const upslam_icp_stats *st, float accept) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        if (!st) {
            ok = 1;
        } else {
            const long long valid = st->valid;
            ok = st->status == UPSLAM_OK && valid > 0 && (float)st->inliers >= accept * (float)valid;
        }
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(256) fuse_main_kernel(FuseView f, const double *pose, upslam_icp_stats *st, int gk) {
    pdl_release();  // the hole-fill write launch may place its CTAs while this grid drains
    if (!accepted(st, f.accept)) return;
    const PoseF T = cta_pose_f32(pose);
    if ((int)blockIdx.x < gk) {
        // averaging: each thread takes kB pixels a CTA-width apart, issuing their depth loads together,
        // then the normal and count of the pixels that hold a sample (an empty pixel has depth 0 and
        // count 0, so half a fresh keyframe is never read past its depth)
        const int npx = f.kp.rows * f.kp.cols;
        const int W = f.kp.cols;
        const int stride = gk * blockDim.x * kFuseB;
        for (int base = blockIdx.x * blockDim.x * kFuseB + threadIdx.x; base < npx; base += stride) {
            constexpr int kB = kFuseB;
            float4 n[kB];
            float d[kB];
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const int k = base + b * blockDim.x;
                d[b] = k < npx ? __ldg(f.kdepth + k) : 0.0f;
            }
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const int k = base + b * blockDim.x;
                n[b] = d[b] > 0.0f ? load_nw(f.knw, k, f.kprec) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const int k = base + b * blockDim.x;
                if (!(n[b].w > 0.0f)) continue;
                const int v = k / W;
                const float3 s = pixel_point(f.kdirs, f.kp.rows, v, k - v * W, d[b]);
                fuse_average(f, T, k, s, n[b], d[b]);
            }
        }
    } else {
        const int ns = f.sp.rows * f.sp.cols;
        const int gs = gridDim.x - gk;
        for (int j = (blockIdx.x - gk) * blockDim.x + threadIdx.x; j < ns; j += gs * blockDim.x) {
            int k;
            unsigned long long key;
            float r;
            float4 m;
            if (!holefill_key(f, T, j, k, key, r, m)) continue;
            if (__ldg(f.kdepth + k) > 0.0f) continue;  // a pixel holding a sample is averaged, not filled
            atomicMin(f.zbuf + k, key);
        }
    }
}

__global__ void __launch_bounds__(256) fuse_fill_kernel(FuseView f, const double *pose, upslam_icp_stats *st) {
    pdl_wait();  // the averaging and the z-buffer atomics have finished
    if (!accepted(st, f.accept)) return;
    const PoseF T = cta_pose_f32(pose);
    const int ns = f.sp.rows * f.sp.cols;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x) {
        int k;
        unsigned long long key;
        float r;
        float4 m;
        if (!holefill_key(f, T, j, k, key, r, m)) continue;
        if (__ldcg(f.zbuf + k) != key) continue;
        holefill_write(f, T, k, r, m);
    }
    if (st && blockIdx.x == 0 && threadIdx.x == 0) st->accepted = 1;
}

}  // namespace upslam

using namespace upslam;

bool upslam_fuse_view(const upslam_keyframe *kf, const upslam_sweep *sw, const upslam_fuse_params *fp,
                      uint64_t *d_zbuf_kf, FuseView &f) {
    if (!kf || !sw || !fp || !d_zbuf_kf) return false;
    if (!upslam_pano_ok(&kf->pano) || !upslam_pano_ok(&sw->pano) || !kf->d_depth || !kf->d_nw || !kf->d_dirs ||
        !sw->d_pix || !sw->d_nrm)
        return false;
    if ((kf->precision != UPSLAM_F32 && kf->precision != UPSLAM_F16) ||
        (sw->nrm_precision != UPSLAM_F32 && sw->nrm_precision != UPSLAM_F16))
        return false;
    if (!upslam_aligned(kf->d_nw, kf->precision == UPSLAM_F32 ? 16 : 8) || !upslam_aligned(d_zbuf_kf, 8) ||
        !upslam_aligned(sw->d_pix, 16) || !upslam_aligned(kf->d_dirs, 8))
        return false;
    if (!(fp->w_max >= 1.0f) || !(fp->d_max > 0.0f)) return false;
    f.kp = kf->pano;
    f.kdepth = kf->d_depth;
    f.knw = kf->d_nw;
    f.kprec = kf->precision;
    f.kdirs = kf->d_dirs;
    f.sp = sw->pano;
    f.spix = reinterpret_cast<const float4 *>(sw->d_pix);
    f.snrm = sw->d_nrm;
    f.sprec = sw->nrm_precision;
    f.d_max2 = fp->d_max * fp->d_max;
    f.cos_min = fp->cos_theta_max;
    f.w_max = fp->w_max;
    f.accept = fp->accept_quality;
    f.zbuf = reinterpret_cast<unsigned long long *>(d_zbuf_kf);
    return true;
}

extern "C" upslam_status upslam_fuse(const upslam_keyframe *kf, const upslam_sweep *sw, const double *d_pose12,
                                     const upslam_fuse_params *fp, upslam_icp_stats *d_stats, uint64_t *d_zbuf_kf,
                                     void *stream) {
    FuseView f;
    if (!d_pose12 || !upslam_fuse_view(kf, sw, fp, d_zbuf_kf, f)) return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npx = (int64_t)kf->pano.rows * kf->pano.cols;
    const int64_t ns = (int64_t)sw->pano.rows * sw->pano.cols;
    const int gk = upslam_grid((npx + kFuseB - 1) / kFuseB, 256, 8);
    const int gs = upslam_grid(ns, 256, 2);
    fuse_main_kernel<<<gk + gs, 256, 0, s>>>(f, d_pose12, d_stats, gk);
    UPSLAM_CHECK_LAUNCH();
    if (!launch_dependent(fuse_fill_kernel, dim3(gs), dim3(256), 0, s, f, d_pose12, d_stats)) return UPSLAM_ERR_CUDA;
    return UPSLAM_OK;
}
