// Loop-closure grid search (UPSLAM Sec. III-C): a few hundred candidate poses
// each get a cheap projective score on a subsampled keyframe, and the winner
// is then refined by ICP at full resolution.
//
// The check is the ICP association of the registration kernels (keyframe pixel
// -> sweep pixel under T^-1 with the FP32 binning rule, filter Omega on the
// point distance and the normal angle) over the keyframe pixels (stride i,
// stride j); a candidate scores its number of inliers.  The best candidate is
// the first one with the largest score.
//
// grid_score_kernel: each CTA takes a slice of the sampled keyframe pixels and
// kCand candidates; a sample's depth, normal and point are loaded once and
// tested against every candidate of the CTA.  Counts leave the CTA as one
// 64-bit integer atomic per candidate, so the scores do not depend on the order
// in which CTAs finish.  grid_best_kernel picks the winner and copies its pose.
//
// Roofline: per candidate a sample costs an L2 gather of 32 B (16 B in FP16) of
// sweep data; the sampled keyframe (20 B per sample) is read once per CTA
// column, i.e. n / kCand times, mostly from L2.  The work is gather- and
// ALU-bound (the binning rule), not HBM-bound.
#include "common.cuh"

namespace upslam {

constexpr int kGridThreads = 256;
constexpr int kCand = 8;  // candidates per CTA

struct GridArgs {
    upslam_pano kp;
    const float *kdepth;
    const void *knw;
    int kprec;
    const float *kdirs;
    upslam_pano sp;
    const float4 *spix;
    const void *snrm;
    int sprec;
    float d_max2, cos_min;
    int stride, rows_s, cols_s;  // sampled grid: rows_s x cols_s pixels (stride v, stride u)
    const double *poses;         // [n][12]
    int n;
    unsigned long long *scores;  // [n], zeroed by the host before the launch
};

__global__ void __launch_bounds__(kGridThreads) grid_score_kernel(GridArgs g) {
    pdl_release();  // the arg-max launch may place its CTA while this grid drains
    __shared__ float Ts[kCand][12];
    const int c0 = blockIdx.y * kCand;
    const int nc = min(kCand, g.n - c0);
    if (threadIdx.x < kCand * 12) {
        const int c = threadIdx.x / 12, i = threadIdx.x % 12;
        Ts[c][i] = c < nc ? (float)__ldg(g.poses + (size_t)(c0 + c) * 12 + i) : 0.0f;
    }
    __syncthreads();
    unsigned cnt[kCand];
#pragma unroll
    for (int c = 0; c < kCand; ++c) cnt[c] = 0;
    const int ms = g.rows_s * g.cols_s;
    for (int m = blockIdx.x * kGridThreads + threadIdx.x; m < ms; m += gridDim.x * kGridThreads) {
        const int vs = m / g.cols_s;
        const int v = vs * g.stride, u = (m - vs * g.cols_s) * g.stride;
        const int k = v * g.kp.cols + u;
        const float d = __ldg(g.kdepth + k);
        if (!(d > 0.0f)) continue;
        const float4 n4 = load_nw(g.knw, k, g.kprec);
        if (!(__fadd_rn(__fadd_rn(__fmul_rn(n4.x, n4.x), __fmul_rn(n4.y, n4.y)), __fmul_rn(n4.z, n4.z)) > 0.25f))
            continue;
        const float3 s = pixel_point(g.kdirs, g.kp.rows, v, u, d);
#pragma unroll
        for (int c = 0; c < kCand; ++c) {
            if (c >= nc) break;
            PoseF T;
#pragma unroll
            for (int i = 0; i < 12; ++i) T.r[i] = Ts[c][i];
            const float3 q = xform_inv(T, s.x, s.y, s.z);
            int jv, ju;
            float rr;
            if (!bin_point(q.x, q.y, q.z, g.sp, jv, ju, rr)) continue;
            const int j = jv * g.sp.cols + ju;
            const float4 P = __ldg(g.spix + j);
            const float4 mm = load_nw(g.snrm, j, g.sprec);
            if (P.w == 0.0f || mm.w == 0.0f) continue;
            const float *r = T.r;
            const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
            const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
            const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
            const float3 Rm = rotate(T, mm.x, mm.y, mm.z);
            const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
            const bool ok = (ex * ex + ey * ey + ez * ez <= g.d_max2) &&
                            (Rm.x * n4.x + Rm.y * n4.y + Rm.z * n4.z >= g.cos_min);
            cnt[c] += ok ? 1u : 0u;
        }
    }
    __shared__ unsigned cta[kCand];
    if (threadIdx.x < kCand) cta[threadIdx.x] = 0;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kCand; ++c) {
        const unsigned w = __reduce_add_sync(0xffffffffu, cnt[c]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&cta[c], w);
    }
    __syncthreads();
    if (threadIdx.x < nc && cta[threadIdx.x]) atomicAdd(g.scores + c0 + threadIdx.x, (unsigned long long)cta[threadIdx.x]);
}

// One CTA: the first candidate with the largest score, and (optionally) its pose.
__global__ void __launch_bounds__(1024) grid_best_kernel(const unsigned long long *scores, int n, const double *poses,
                                                         int *best, double *best_pose) {
    pdl_wait();  // every score is in
    __shared__ unsigned long long ws[32];
    __shared__ int wi[32];
    __shared__ int win;
    unsigned long long bs = 0;
    int bi = n;  // beyond every index: loses every tie
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long s = scores[i];
        if (s > bs || (s == bs && i < bi)) {
            bs = s;
            bi = i;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long s = __shfl_xor_sync(0xffffffffu, bs, o);
        const int i = __shfl_xor_sync(0xffffffffu, bi, o);
        if (s > bs || (s == bs && i < bi)) {
            bs = s;
            bi = i;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        ws[warp] = bs;
        wi[warp] = bi;
    }
    __syncthreads();
    if (warp == 0) {
        bs = lane < nw ? ws[lane] : 0;
        bi = lane < nw ? wi[lane] : n;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long s = __shfl_xor_sync(0xffffffffu, bs, o);
            const int i = __shfl_xor_sync(0xffffffffu, bi, o);
            if (s > bs || (s == bs && i < bi)) {
                bs = s;
                bi = i;
            }
        }
        if (lane == 0) {
            win = bi < n ? bi : 0;
            *best = win;
        }
    }
    __syncthreads();
    if (best_pose && threadIdx.x < 12) best_pose[threadIdx.x] = poses[(size_t)win * 12 + threadIdx.x];
}

// poses[i] = exp(xi_i^) * center (left update, FP64), xi_i = (omega, v) in FP32.
__global__ void grid_candidates_kernel(const double *center, const float *xi, int n, double *poses) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double T[12], x[6];
#pragma unroll
    for (int k = 0; k < 12; ++k) T[k] = __ldg(center + k);
#pragma unroll
    for (int k = 0; k < 6; ++k) x[k] = (double)__ldg(xi + (size_t)i * 6 + k);
    se3_exp_left(x, T);
#pragma unroll
    for (int k = 0; k < 12; ++k) poses[(size_t)i * 12 + k] = T[k];
}

}  // namespace upslam

using namespace upslam;

extern "C" upslam_status upslam_grid_candidates(const double *d_center12, const float *d_xi, int32_t n,
                                                double *d_poses, void *stream) {
    if (!d_center12 || !d_xi || !d_poses || n < 0) return UPSLAM_ERR_INVALID_ARG;
    if (n == 0) return UPSLAM_OK;
    grid_candidates_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_center12, d_xi, n, d_poses);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_grid_score(const upslam_keyframe *kf, const upslam_sweep *sw, const double *d_poses,
                                           int32_t n, int32_t stride, const upslam_icp_params *ip,
                                           uint64_t *d_scores, int32_t *d_best, double *d_best_pose12,
                                           void *stream) {
    if (!kf || !sw || !d_poses || !ip || !d_scores || !d_best || n <= 0 || stride < 1) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_pano_ok(&kf->pano) || !upslam_pano_ok(&sw->pano) || !kf->d_depth || !kf->d_nw || !kf->d_dirs ||
        !sw->d_pix || !sw->d_nrm)
        return UPSLAM_ERR_INVALID_ARG;
    if ((kf->precision != UPSLAM_F32 && kf->precision != UPSLAM_F16) ||
        (sw->nrm_precision != UPSLAM_F32 && sw->nrm_precision != UPSLAM_F16))
        return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_aligned(kf->d_nw, kf->precision == UPSLAM_F32 ? 16 : 8) || !upslam_aligned(sw->d_pix, 16) ||
        !upslam_aligned(kf->d_dirs, 8) || !upslam_aligned(d_scores, 8) || !upslam_aligned(d_poses, 8))
        return UPSLAM_ERR_INVALID_ARG;
    if (!(ip->d_max > 0.0f)) return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GridArgs g;
    g.kp = kf->pano;
    g.kdepth = kf->d_depth;
    g.knw = kf->d_nw;
    g.kprec = kf->precision;
    g.kdirs = kf->d_dirs;
    g.sp = sw->pano;
    g.spix = reinterpret_cast<const float4 *>(sw->d_pix);
    g.snrm = sw->d_nrm;
    g.sprec = sw->nrm_precision;
    g.d_max2 = ip->d_max * ip->d_max;
    g.cos_min = ip->cos_theta_max;
    g.stride = stride;
    g.rows_s = (kf->pano.rows + stride - 1) / stride;
    g.cols_s = (kf->pano.cols + stride - 1) / stride;
    g.poses = d_poses;
    g.n = n;
    g.scores = reinterpret_cast<unsigned long long *>(d_scores);
    if (cudaMemsetAsync(d_scores, 0, (size_t)n * sizeof(uint64_t), s) != cudaSuccess) return UPSLAM_ERR_CUDA;
    const int64_t ms = (int64_t)g.rows_s * g.cols_s;
    const int cand_blocks = (n + kCand - 1) / kCand;
    // enough sample slices that the launch covers every SM about four times over
    int xb = (int)((4LL * upslam_sm_count() + cand_blocks - 1) / cand_blocks);
    const int xb_max = (int)((ms + kGridThreads - 1) / kGridThreads);
    xb = xb < 1 ? 1 : (xb > xb_max ? xb_max : xb);
    if (cand_blocks > 65535) return UPSLAM_ERR_INVALID_ARG;
    grid_score_kernel<<<dim3(xb, cand_blocks), kGridThreads, 0, s>>>(g);
    UPSLAM_CHECK_LAUNCH();
    if (!launch_dependent(grid_best_kernel, dim3(1), dim3(1024), 0, s, (const unsigned long long *)g.scores, n,
                          (const double *)d_poses, d_best, d_best_pose12))
        return UPSLAM_ERR_CUDA;
    return UPSLAM_OK;
}
