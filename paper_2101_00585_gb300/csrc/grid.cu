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
// grid_score_kernel: CTA (x, y) scores candidates [32 y, 32 y + 32) on the
// sampled keyframe pixels of column x.  The sampled grid is dealt to the CTA
// columns in slices of kGridSlice pixels (slice s to column s mod gridDim.x),
// so that every column holds rows of every elevation band.  Each round the CTA
// loads kGridChunk of its pixels, every thread a few, all loads in flight, and
// compacts the ones that hold a sample (depth > 0, normal longer than 1/2) into
// shared memory as keyframe point and normal.  Then every warp walks the staged
// samples, one sample per step for the whole warp (a shared-memory broadcast),
// and lane c scores candidate 32 y + c against it: no lane idles on an empty
// pixel, and a lane keeps its candidate's pose and count in registers.  Counts
// leave the CTA as one 64-bit integer atomic per candidate, so the scores do
// not depend on the order in which CTAs finish.  grid_best_kernel picks the
// winner and copies its pose.
//
// Roofline: per candidate a sample costs an L2 gather of 32 B (16 B in FP16) of
// sweep data; the sampled keyframe (20 B per sample) is read once per CTA
// row, i.e. n / 32 times, mostly from L2.  The work is bound by instruction
// issue (the FP32 binning rule), not by HBM.
#include "common.cuh"

namespace upslam {

constexpr int kGridThreads = 256;
constexpr int kGridWarps = kGridThreads / 32;
constexpr int kCand = 32;         // candidates per CTA: one per lane
constexpr int kGridSlice = 64;    // sampled pixels dealt to a CTA column at a time
constexpr int kGridChunk = 1024;  // sampled pixels staged per round
constexpr int kGridPer = kGridChunk / kGridThreads;

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

// Sampled pixel m of round r, thread slot i (kGridPer per thread), or -1 past the grid.
__device__ __forceinline__ int grid_pixel(const GridArgs &g, int r, int i) {
    const int p = i * kGridThreads + threadIdx.x;  // 0 .. kGridChunk - 1
    const long long slice = ((long long)r * (kGridChunk / kGridSlice) + p / kGridSlice) * gridDim.x + blockIdx.x;
    const long long m = slice * kGridSlice + (p % kGridSlice);
    return m < (long long)g.rows_s * g.cols_s ? (int)m : -1;
}

__global__ void __launch_bounds__(kGridThreads) grid_score_kernel(GridArgs g, int rounds) {
    pdl_release();  // the arg-max launch may place its CTA while this grid drains
    __shared__ float sx[kGridChunk], sy[kGridChunk], sz[kGridChunk];
    __shared__ float snx[kGridChunk], sny[kGridChunk], snz[kGridChunk];
    __shared__ int staged[2];  // round r counts into slot r & 1; the other slot is reset for round r + 1
    __shared__ unsigned cta[kCand];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c0 = blockIdx.y * kCand;
    const int nc = min(kCand, g.n - c0);
    const bool mine = lane < nc;  // this lane's candidate exists
    PoseF T;
#pragma unroll
    for (int i = 0; i < 12; ++i) T.r[i] = mine ? (float)__ldg(g.poses + (size_t)(c0 + lane) * 12 + i) : 0.0f;
    if (threadIdx.x < kCand) cta[threadIdx.x] = 0;
    if (threadIdx.x == 0) staged[0] = 0;
    unsigned cnt = 0;
    for (int r = 0; r < rounds; ++r) {
        __syncthreads();  // the previous round's samples are consumed, and its count read by every thread
        if (threadIdx.x == 0) staged[(r + 1) & 1] = 0;
        // stage: every depth of the round in flight, then the normals of the pixels that hold a sample
        int k[kGridPer];
        float d[kGridPer];
        float4 n4[kGridPer];
#pragma unroll
        for (int i = 0; i < kGridPer; ++i) {
            const int m = grid_pixel(g, r, i);
            k[i] = -1;
            if (m >= 0) {
                const int vs = m / g.cols_s;
                const int v = vs * g.stride, u = (m - vs * g.cols_s) * g.stride;
                k[i] = v * g.kp.cols + u;
            }
            d[i] = k[i] >= 0 ? __ldg(g.kdepth + k[i]) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < kGridPer; ++i)
            n4[i] = d[i] > 0.0f ? load_nw(g.knw, k[i], g.kprec) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int i = 0; i < kGridPer; ++i) {
            const float nn = __fadd_rn(__fadd_rn(__fmul_rn(n4[i].x, n4[i].x), __fmul_rn(n4[i].y, n4[i].y)),
                                       __fmul_rn(n4[i].z, n4[i].z));
            const bool has = d[i] > 0.0f && nn > 0.25f;
            const unsigned b = __ballot_sync(0xffffffffu, has);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(&staged[r & 1], __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (has) {
                const int e = base + __popc(b & ((1u << lane) - 1u));
                const int v = k[i] / g.kp.cols;
                const float3 s = pixel_point(g.kdirs, g.kp.rows, v, k[i] - v * g.kp.cols, d[i]);
                sx[e] = s.x;
                sy[e] = s.y;
                sz[e] = s.z;
                snx[e] = n4[i].x;
                sny[e] = n4[i].y;
                snz[e] = n4[i].z;
            }
        }
        __syncthreads();
        // score: the warp takes one staged sample per step, lane c against candidate c0 + c
        const int ns = staged[r & 1];
        if (mine) {
            for (int e = warp; e < ns; e += kGridWarps) {
                const float3 s = make_float3(sx[e], sy[e], sz[e]);
                const float3 q = xform_inv(T, s.x, s.y, s.z);
                int jv, ju;
                float rr;
                if (!bin_point(q.x, q.y, q.z, g.sp, jv, ju, rr)) continue;
                const int j = jv * g.sp.cols + ju;
                const float4 P = __ldg(g.spix + j);
                const float4 mm = load_nw(g.snrm, j, g.sprec);
                if (P.w == 0.0f || mm.w == 0.0f) continue;
                const float *R = T.r;
                const float px = fmaf(R[0], P.x, fmaf(R[1], P.y, fmaf(R[2], P.z, R[3])));
                const float py = fmaf(R[4], P.x, fmaf(R[5], P.y, fmaf(R[6], P.z, R[7])));
                const float pz = fmaf(R[8], P.x, fmaf(R[9], P.y, fmaf(R[10], P.z, R[11])));
                const float3 Rm = rotate(T, mm.x, mm.y, mm.z);
                const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
                const bool ok = (ex * ex + ey * ey + ez * ez <= g.d_max2) &&
                                (Rm.x * snx[e] + Rm.y * sny[e] + Rm.z * snz[e] >= g.cos_min);
                cnt += ok ? 1u : 0u;
            }
        }
    }
    if (mine && cnt) atomicAdd(&cta[lane], cnt);
    __syncthreads();
    if (threadIdx.x < nc && cta[threadIdx.x])
        atomicAdd(g.scores + c0 + threadIdx.x, (unsigned long long)cta[threadIdx.x]);
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
    const int64_t cand_blocks = (n + kCand - 1) / kCand;  // CTA rows of kCand candidates
    if (cand_blocks > 65535) return UPSLAM_ERR_INVALID_ARG;
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
    // enough CTA columns that the launch covers every SM about four times over, each column at least one
    // slice; every column then stages its slices kGridChunk pixels per round
    const int64_t slices = (ms + kGridSlice - 1) / kGridSlice;
    int64_t xb = (4LL * upslam_sm_count() + cand_blocks - 1) / cand_blocks;
    xb = xb < 1 ? 1 : (xb > slices ? slices : xb);
    const int64_t per_round = (int64_t)xb * (kGridChunk / kGridSlice);
    const int rounds = (int)((slices + per_round - 1) / per_round);
    grid_score_kernel<<<dim3((unsigned)xb, (unsigned)cand_blocks), kGridThreads, 0, s>>>(g, rounds);
    UPSLAM_CHECK_LAUNCH();
    if (!launch_dependent(grid_best_kernel, dim3(1), dim3(1024), 0, s, (const unsigned long long *)g.scores, n,
                          (const double *)d_poses, d_best, d_best_pose12))
        return UPSLAM_ERR_CUDA;
    return UPSLAM_OK;
}
