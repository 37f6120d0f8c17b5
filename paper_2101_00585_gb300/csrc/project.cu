// Spherical projection with a deterministic z-buffer (UPSLAM Sec. III-A).
//
// Pass 1 bins every valid point with the FP32 rule of upslam.h and does an
// atomicMin of its 64-bit key (bits(range) << 32 | index) into the pixel's
// z-buffer word.  Positive IEEE floats order like their bit patterns, so the
// minimum key is the nearest point, ties going to the smaller index: the
// winner does not depend on thread order.  Pass 2 decodes each word, gathers
// the winner's point, and resets the word to all-ones so the scratch buffer is
// ready for the next sweep without a separate clear.
//
// Roofline: HBM-bound streaming.  Pass 1 reads 16 B per point and touches one
// 8 B word in L2 per binned point; pass 2 reads 8 B and writes 8 + 4 + 4 + 16 B
// per pixel (z-buffer reset, depth, index, point) plus a 16 B point gather.
#include "common.cuh"

namespace upslam {

__global__ void pano_dirs_kernel(upslam_pano pp, float *dirs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < pp.rows) {
        const double e = (double)pp.el_top - ((double)i + 0.5) / (double)pp.s_el;
        double s, c;
        sincos(e, &s, &c);
        dirs[2 * i] = (float)c;
        dirs[2 * i + 1] = (float)s;
    } else if (i < pp.rows + pp.cols) {
        const int u = i - pp.rows;
        const double a = 3.14159265358979323846 - ((double)u + 0.5) / (double)pp.s_az;
        double s, c;
        sincos(a, &s, &c);
        dirs[2 * pp.rows + 2 * u] = (float)c;
        dirs[2 * pp.rows + 2 * u + 1] = (float)s;
    }
}

template <bool kPose>
__global__ void __launch_bounds__(256) project_kernel(const float4 *__restrict__ pts, int n, const double *pose,
                                                      upslam_pano pp, unsigned long long *__restrict__ zbuf) {
    pdl_release();  // the resolve launch may place its CTAs while this grid drains
    if (!kPose) {
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
            project_point(pts, i, pp, zbuf);
        return;
    }
    const PoseF T = cta_pose_f32(pose);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = __ldg(pts + i);
        if (p.w == 0.0f) continue;
        const float3 q = xform(T, p.x, p.y, p.z);
        int v, u;
        float r;
        if (!bin_point(q.x, q.y, q.z, pp, v, u, r)) continue;
        const unsigned long long key = ((unsigned long long)__float_as_uint(r) << 32) | (unsigned int)i;
        atomicMin(zbuf + (size_t)v * pp.cols + u, key);
    }
}

__global__ void __launch_bounds__(256) resolve_kernel(const float4 *__restrict__ pts, int npx,
                                                      unsigned long long *__restrict__ zbuf, float *__restrict__ depth,
                                                      int *__restrict__ idx, float4 *__restrict__ pix) {
    pdl_wait();  // every point of the projection has reached the z-buffer
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x)
        resolve_pixel<false>(pts, k, zbuf, depth, idx, pix);
}

__global__ void __launch_bounds__(256) unproject_kernel(const float *__restrict__ depth, upslam_pano pp,
                                                        const float *__restrict__ dirs, float4 *__restrict__ pix) {
    const int npx = pp.rows * pp.cols;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x) {
        const float d = depth[k];
        if (d > 0.0f) {
            const float3 p = pixel_point(dirs, pp.rows, k / pp.cols, k % pp.cols, d);
            pix[k] = make_float4(p.x, p.y, p.z, 1.0f);
        } else {
            pix[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

}  // namespace upslam

using namespace upslam;

extern "C" size_t upslam_pano_dirs_floats(const upslam_pano *pp) {
    if (!upslam_pano_ok(pp)) return 0;
    return 2 * (size_t)pp->rows + 2 * (size_t)pp->cols;
}

extern "C" upslam_status upslam_pano_dirs(const upslam_pano *pp, float *d_dirs, void *stream) {
    if (!upslam_pano_ok(pp) || !d_dirs || !upslam_aligned(d_dirs, 8)) return UPSLAM_ERR_INVALID_ARG;
    const int n = pp->rows + pp->cols;
    pano_dirs_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(*pp, d_dirs);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_project(const float *d_pts, int32_t n, const double *d_pose12, const upslam_pano *pp,
                                        uint64_t *d_zbuf, float *d_depth, int32_t *d_idx, float *d_pix,
                                        void *stream) {
    if (!upslam_pano_ok(pp) || n < 0 || (n > 0 && !d_pts) || !d_zbuf || !d_depth || !d_idx)
        return UPSLAM_ERR_INVALID_ARG;
    if ((d_pts && !upslam_aligned(d_pts, 16)) || !upslam_aligned(d_zbuf, 8) || (d_pix && !upslam_aligned(d_pix, 16)))
        return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *zb = reinterpret_cast<unsigned long long *>(d_zbuf);
    if (n > 0) {
        const int g = upslam_grid(n, 256);
        if (d_pose12)
            project_kernel<true><<<g, 256, 0, s>>>(reinterpret_cast<const float4 *>(d_pts), n, d_pose12, *pp, zb);
        else
            project_kernel<false><<<g, 256, 0, s>>>(reinterpret_cast<const float4 *>(d_pts), n, nullptr, *pp, zb);
        UPSLAM_CHECK_LAUNCH();
    }
    const int npx = pp->rows * pp->cols;
    if (!launch_dependent(resolve_kernel, dim3(upslam_grid(npx, 256)), dim3(256), 0, s,
                          reinterpret_cast<const float4 *>(d_pts), npx, zb, d_depth, d_idx,
                          reinterpret_cast<float4 *>(d_pix)))
        return UPSLAM_ERR_CUDA;
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_unproject(const float *d_depth, const upslam_pano *pp, const float *d_dirs,
                                          float *d_pix, void *stream) {
    if (!upslam_pano_ok(pp) || !d_depth || !d_dirs || !d_pix || !upslam_aligned(d_pix, 16) ||
        !upslam_aligned(d_dirs, 8))
        return UPSLAM_ERR_INVALID_ARG;
    const int npx = pp->rows * pp->cols;
    unproject_kernel<<<upslam_grid(npx, 256), 256, 0, (cudaStream_t)stream>>>(d_depth, *pp, d_dirs,
                                                                           reinterpret_cast<float4 *>(d_pix));
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}
