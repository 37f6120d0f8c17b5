// Point-to-plane ICP over projective correspondences (UPSLAM Sec. III-B, Eq. 1).
//
// Correspondences run from keyframe to sweep, as in the keyframe update of
// Sec. III-C: every keyframe pixel holding a sample is put at s1 = d * dir,
// taken into the sweep frame by T^-1 and binned into the sweep panorama; the
// sweep pixel's point s2 and normal m complete the pair.  Omega keeps it when
// |T s2 - s1| <= d_max and (R m) . N(s1) >= cos(theta_max).  Each inlier adds
// J^T J and J^T r with r = (T s2 - s1) . N(s1) and J = [p x N, N] (p = T s2,
// left update T <- exp(xi^) T).
//
// Reduction: FP32 per thread -> warp shuffles -> compensated FP32 per CTA ->
// compensated FP32 over CTAs in a fixed order (deterministic) -> FP64.  The CTA
// that arrives last solves the 6x6 system with an FP64 square-root-free
// Cholesky (L D L^T) and applies the SE(3) exponential in FP64.
//
// Two launch forms:
//  * icp_step_kernel: one Gauss-Newton step, "last CTA done" ticket.
//  * icp_persistent_kernel: all iterations in one cooperative launch; each
//    step ends at a grid barrier whose last arriver solves and then releases
//    the others through a generation counter.  Every wait is bounded by a
//    clock64 budget and reports UPSLAM_ERR_TIMEOUT instead of hanging.
//
// Roofline: per step the keyframe is streamed once (4 B depth + 16 B or 8 B
// normal/weight per pixel) and each correspondence gathers 32 B (16 B in FP16)
// of sweep data that stays resident in L2.
#include <mutex>

#include "common.cuh"

namespace upslam {

constexpr int kIcpThreads = 256;
constexpr int kIcpWarps = kIcpThreads / 32;
// Per-CTA partial: 28 FP32 sums and their Neumaier compensations, then the
// inlier and valid counts as integers (64 words = 256 bytes per CTA).
constexpr int kSlots = 64;
constexpr size_t kCtrlBytes = 256;
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at 2 GHz

struct IcpArgs {
    upslam_pano kp;
    const float *kdepth;
    const void *knw;
    int kprec;
    const float *kdirs;
    upslam_pano sp;
    const float4 *spix;
    const void *snrm;
    int sprec;
    float d_max2;
    float cos_min;
};

struct IcpCtrl {
    unsigned int arrive;  // CTAs arrived at the current barrier
    unsigned int gen;     // barrier generation (monotonic across launches)
    unsigned int ticket;  // single-step "last CTA" ticket
    int valid;            // sweep pixels with a point (persistent form, step 0)
};

__device__ __forceinline__ void accumulate_pixel(const IcpArgs &a, const PoseF &T, int k, float acc[28], int &inl) {
    const float d = __ldg(a.kdepth + k);
    if (!(d > 0.0f)) return;
    const float4 n = load_nw(a.knw, k, a.kprec);
    if (!(__fadd_rn(__fadd_rn(__fmul_rn(n.x, n.x), __fmul_rn(n.y, n.y)), __fmul_rn(n.z, n.z)) > 0.25f)) return;
    const int W = a.kp.cols;
    const int v = k / W, u = k - v * W;
    const float3 s = pixel_point(a.kdirs, a.kp.rows, v, u, d);
    const float3 q = xform_inv(T, s.x, s.y, s.z);
    int jv, ju;
    float rr;
    if (!bin_point(q.x, q.y, q.z, a.sp, jv, ju, rr)) return;
    const int j = jv * a.sp.cols + ju;
    const float4 P = __ldg(a.spix + j);
    if (P.w == 0.0f) return;
    const float4 m = load_nw(a.snrm, j, a.sprec);
    if (m.w == 0.0f) return;
    const float *r = T.r;
    const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
    const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
    const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
    const float3 Rm = rotate(T, m.x, m.y, m.z);
    const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
    if (!(ex * ex + ey * ey + ez * ez <= a.d_max2)) return;
    if (!(Rm.x * n.x + Rm.y * n.y + Rm.z * n.z >= a.cos_min)) return;
    const float res = ex * n.x + ey * n.y + ez * n.z;
    float J[6];
    J[0] = py * n.z - pz * n.y;
    J[1] = pz * n.x - px * n.z;
    J[2] = px * n.y - py * n.x;
    J[3] = n.x;
    J[4] = n.y;
    J[5] = n.z;
    int p = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int c = i; c < 6; ++c) acc[p++] += J[i] * J[c];
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[21 + i] += J[i] * res;
    acc[27] += res * res;
    inl += 1;
}

// Warp shuffles, then the CTA's warps summed (compensated FP32) into its partial record.
__device__ __forceinline__ void cta_partial(float acc[28], int inl, int valid, float *partial, float (*sh)[32],
                                            int (*shi)[2]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < 28; ++i) {
        const float s = warp_sum(acc[i]);
        if (lane == 0) sh[warp][i] = s;
    }
    const int si = __reduce_add_sync(0xffffffffu, inl);
    const int sv = __reduce_add_sync(0xffffffffu, valid);
    if (lane == 0) {
        shi[warp][0] = si;
        shi[warp][1] = sv;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        float t = 0.0f, c = 0.0f;
        for (int w = 0; w < kIcpWarps; ++w) kadd(t, c, sh[w][threadIdx.x]);
        partial[threadIdx.x] = t;
        partial[28 + threadIdx.x] = c;
    } else if (threadIdx.x < 30) {
        int t = 0;
        for (int w = 0; w < kIcpWarps; ++w) t += shi[w][threadIdx.x - 28];
        reinterpret_cast<int *>(partial)[56 + threadIdx.x - 28] = t;
    }
}

// Sum the CTA partials in a fixed order (compensated FP32, then FP64), solve,
// update the pose and the stats.  Run by every thread of the CTA that arrived last.
__device__ void finalize(const float *partials, int nparts, double *pose, const upslam_icp_params &ip,
                         upslam_icp_stats *st, int valid_override, int step_index, float (*sh)[32], int (*shi)[2],
                         double *tot) {
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    __shared__ float shc[kIcpWarps][32];
    __shared__ long long shn[kIcpWarps][2];
    if (lane < 28) {
        float t = 0.0f, c = 0.0f;
        for (int b = grp; b < nparts; b += kIcpWarps) {
            const float *pb = partials + (size_t)b * kSlots;
            kadd(t, c, __ldcg(pb + lane));
            c += __ldcg(pb + 28 + lane);
        }
        sh[grp][lane] = t;
        shc[grp][lane] = c;
    } else if (lane < 30) {
        long long t = 0;
        for (int b = grp; b < nparts; b += kIcpWarps)
            t += __ldcg(reinterpret_cast<const int *>(partials + (size_t)b * kSlots) + 56 + lane - 28);
        shn[grp][lane - 28] = t;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        float t = 0.0f, c = 0.0f;
        for (int g = 0; g < kIcpWarps; ++g) {
            kadd(t, c, sh[g][threadIdx.x]);
            c += shc[g][threadIdx.x];
        }
        tot[threadIdx.x] = (double)t + (double)c;
    } else if (threadIdx.x < 30) {
        long long t = 0;
        for (int g = 0; g < kIcpWarps; ++g) t += shn[g][threadIdx.x - 28];
        tot[threadIdx.x] = (double)t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const long long inliers = (long long)tot[28];
        const long long valid = valid_override >= 0 ? valid_override : (long long)tot[29];
        double xi[6] = {0, 0, 0, 0, 0, 0};
        int status = UPSLAM_OK, conv = 0;
        if (inliers < ip.min_inliers) {
            status = UPSLAM_ERR_DEGENERATE;
        } else {
            double rhs[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) rhs[i] = -tot[21 + i];
            if (!solve6(tot, rhs, ip.pivot_eps, xi)) {
                status = UPSLAM_ERR_DEGENERATE;
#pragma unroll
                for (int i = 0; i < 6; ++i) xi[i] = 0.0;
            } else {
                double T[12];
#pragma unroll
                for (int i = 0; i < 12; ++i) T[i] = __ldcg(pose + i);
                se3_exp_left(xi, T);
#pragma unroll
                for (int i = 0; i < 12; ++i) pose[i] = T[i];
                const double wn2 = xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2];
                const double vn2 = xi[3] * xi[3] + xi[4] * xi[4] + xi[5] * xi[5];
                conv = (wn2 < ip.eps_rot * ip.eps_rot && vn2 < ip.eps_trans * ip.eps_trans) ? 1 : 0;
            }
        }
#pragma unroll
        for (int i = 0; i < 6; ++i) st->xi[i] = xi[i];
        st->status = status;
        st->converged = conv;
        st->iters = step_index + 1;
        st->accepted = 0;
        st->inliers = inliers;
        st->valid = valid;
    }
    // the rest of the record is written by other threads, off the solver's path
    if (threadIdx.x >= 32 && threadIdx.x < 32 + 28) {
        const int i = threadIdx.x - 32;
        if (i < 21) st->A[i] = tot[i];
        else if (i < 27) st->b[i - 21] = tot[i];
        else st->sse = tot[27];
    }
}

__device__ __forceinline__ int count_valid(const IcpArgs &a) {
    int c = 0;
    const int ns = a.sp.rows * a.sp.cols;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ns; j += gridDim.x * blockDim.x)
        c += __ldg(&a.spix[j].w) != 0.0f;
    return c;
}

__global__ void __launch_bounds__(kIcpThreads) icp_step_kernel(IcpArgs a, double *pose, upslam_icp_params ip,
                                                               upslam_icp_stats *st, IcpCtrl *ctrl,
                                                               float *partials) {
    __shared__ float sh[kIcpWarps][32];
    __shared__ int shi[kIcpWarps][2];
    __shared__ double tot[32];
    __shared__ int last;
    const PoseF T = pose_to_f32_cg(pose);
    float acc[28];
#pragma unroll
    for (int i = 0; i < 28; ++i) acc[i] = 0.0f;
    int inl = 0;
    const int npx = a.kp.rows * a.kp.cols;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x)
        accumulate_pixel(a, T, k, acc, inl);
    const int valid = count_valid(a);
    cta_partial(acc, inl, valid, partials + (size_t)blockIdx.x * kSlots, sh, shi);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    finalize(partials, gridDim.x, pose, ip, st, -1, 0, sh, shi, tot);
    if (threadIdx.x == 0) {
        __threadfence();
        ctrl->ticket = 0;
    }
}

__global__ void __launch_bounds__(kIcpThreads) icp_persistent_kernel(IcpArgs a, double *pose, upslam_icp_params ip,
                                                                     upslam_icp_stats *st, IcpCtrl *ctrl,
                                                                     float *partials) {
    __shared__ float sh[kIcpWarps][32];
    __shared__ int shi[kIcpWarps][2];
    __shared__ double tot[32];
    __shared__ float pose_s[12];
    __shared__ int flag;  // 1 = last arriver, 2 = stop, 3 = timeout
    const int npx = a.kp.rows * a.kp.cols;
    unsigned int my_gen = 0;
    if (threadIdx.x == 0) my_gen = *((volatile unsigned int *)&ctrl->gen);
    for (int it = 0; it < ip.max_iters; ++it) {
        if (threadIdx.x < 12) pose_s[threadIdx.x] = (float)__ldcg(pose + threadIdx.x);
        __syncthreads();
        PoseF T;
#pragma unroll
        for (int i = 0; i < 12; ++i) T.r[i] = pose_s[i];
        float acc[28];
#pragma unroll
        for (int i = 0; i < 28; ++i) acc[i] = 0.0f;
        int inl = 0;
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x)
            accumulate_pixel(a, T, k, acc, inl);
        const int valid = it == 0 ? count_valid(a) : 0;
        cta_partial(acc, inl, valid, partials + (size_t)blockIdx.x * kSlots, sh, shi);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            flag = atomicAdd(&ctrl->arrive, 1u) == gridDim.x - 1 ? 1 : 0;
        }
        __syncthreads();
        if (flag == 1) {
            __threadfence();
            // the valid count is summed at step 0 and kept for the later steps
            finalize(partials, gridDim.x, pose, ip, st, it == 0 ? -1 : __ldcg(&ctrl->valid), it, sh, shi, tot);
            if (threadIdx.x == 0) {
                if (it == 0) ctrl->valid = (int)st->valid;
                __threadfence();
                ctrl->arrive = 0;
                __threadfence();
                atomicAdd(&ctrl->gen, 1u);
            }
        } else if (threadIdx.x == 0) {
            const long long t0 = clock64();
            int timed_out = 0;
            while (*((volatile unsigned int *)&ctrl->gen) == my_gen) {
                if (clock64() - t0 > kWaitCycles) {
                    timed_out = 1;
                    break;
                }
                __nanosleep(64);
            }
            if (timed_out) {
                st->status = UPSLAM_ERR_TIMEOUT;
                flag = 3;
            }
            __threadfence();
        }
        if (threadIdx.x == 0) ++my_gen;
        __syncthreads();
        if (flag == 3) return;
        if (threadIdx.x == 0) {
            const int status = *((volatile int *)&st->status);
            const int conv = *((volatile int *)&st->converged);
            flag = (status != UPSLAM_OK || conv) ? 2 : 0;
        }
        __syncthreads();
        if (flag == 2) return;
    }
}

static IcpArgs make_args(const upslam_keyframe *kf, const upslam_sweep *sw, const upslam_icp_params *ip) {
    IcpArgs a;
    a.kp = kf->pano;
    a.kdepth = kf->d_depth;
    a.knw = kf->d_nw;
    a.kprec = kf->precision;
    a.kdirs = kf->d_dirs;
    a.sp = sw->pano;
    a.spix = reinterpret_cast<const float4 *>(sw->d_pix);
    a.snrm = sw->d_nrm;
    a.sprec = sw->nrm_precision;
    a.d_max2 = ip->d_max * ip->d_max;
    a.cos_min = ip->cos_theta_max;
    return a;
}

static bool views_ok(const upslam_keyframe *kf, const upslam_sweep *sw) {
    if (!kf || !sw || !upslam_pano_ok(&kf->pano) || !upslam_pano_ok(&sw->pano)) return false;
    if (!kf->d_depth || !kf->d_nw || !kf->d_dirs || !sw->d_pix || !sw->d_nrm) return false;
    if ((kf->precision != UPSLAM_F32 && kf->precision != UPSLAM_F16) ||
        (sw->nrm_precision != UPSLAM_F32 && sw->nrm_precision != UPSLAM_F16))
        return false;
    if (!upslam_aligned(kf->d_nw, kf->precision == UPSLAM_F32 ? 16 : 8) ||
        !upslam_aligned(sw->d_nrm, sw->nrm_precision == UPSLAM_F32 ? 16 : 8) || !upslam_aligned(sw->d_pix, 16) ||
        !upslam_aligned(kf->d_dirs, 8))
        return false;
    return true;
}

static int max_ctas() { return upslam_sm_count() * 8; }

}  // namespace upslam

using namespace upslam;

extern "C" size_t upslam_icp_workspace_bytes(const upslam_keyframe *kf) {
    (void)kf;
    return kCtrlBytes + (size_t)max_ctas() * kSlots * sizeof(float);
}

static upslam_status icp_common_checks(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                       const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                       size_t ws_bytes) {
    if (!views_ok(kf, sw) || !d_pose12 || !ip || !d_stats || !d_ws) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_aligned(d_ws, 256) || ws_bytes < upslam_icp_workspace_bytes(kf)) return UPSLAM_ERR_INVALID_ARG;
    if (!(ip->d_max > 0.0f) || ip->max_iters < 0 || ip->min_inliers < 0) return UPSLAM_ERR_INVALID_ARG;
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_icp_step(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                         const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                         size_t ws_bytes, void *stream) {
    const upslam_status chk = icp_common_checks(kf, sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    const IcpArgs a = make_args(kf, sw, ip);
    const int64_t npx = (int64_t)kf->pano.rows * kf->pano.cols;
    const int grid = upslam_grid(npx, kIcpThreads, 8);
    IcpCtrl *ctrl = reinterpret_cast<IcpCtrl *>(d_ws);
    float *partials = reinterpret_cast<float *>(reinterpret_cast<char *>(d_ws) + kCtrlBytes);
    icp_step_kernel<<<grid, kIcpThreads, 0, (cudaStream_t)stream>>>(a, d_pose12, *ip, d_stats, ctrl, partials);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_icp(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                    const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                    size_t ws_bytes, void *stream) {
    const upslam_status chk = icp_common_checks(kf, sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    if (ip->max_iters == 0) return UPSLAM_OK;
    IcpArgs a = make_args(kf, sw, ip);
    int dev = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return UPSLAM_ERR_UNSUPPORTED;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, icp_persistent_kernel, kIcpThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return UPSLAM_ERR_UNSUPPORTED;
    if (per_sm > 4) per_sm = 4;
    int grid = upslam_sm_count() * per_sm;
    if (grid > max_ctas()) grid = max_ctas();
    IcpCtrl *ctrl = reinterpret_cast<IcpCtrl *>(d_ws);
    float *partials = reinterpret_cast<float *>(reinterpret_cast<char *>(d_ws) + kCtrlBytes);
    upslam_icp_params ipc = *ip;
    void *args[] = {&a, &d_pose12, &ipc, &d_stats, &ctrl, &partials};
    if (cudaLaunchCooperativeKernel((const void *)icp_persistent_kernel, dim3(grid), dim3(kIcpThreads), args, 0,
                                    (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    return UPSLAM_OK;
}

// ----------------------------------------------------------------------------- allocation-free variant
//
// upslam_icp_noalloc runs the same persistent kernel as upslam_icp, but its
// workspace is this file-scope device array instead of caller memory.  The
// array is part of the library image: every GPU that loads the library holds
// it until the process exits.  Host code must not hand the symbol itself to a
// kernel (on the host it only names a stand-in); the device address is looked
// up once per device with cudaGetSymbolAddress.

namespace upslam {

constexpr int kNoAllocMaxCtas = 2048;
constexpr size_t kNoAllocBytes = kCtrlBytes + (size_t)kNoAllocMaxCtas * kSlots * sizeof(float);  // 512.25 KiB

static __device__ __align__(256) unsigned char g_icp_noalloc_ws[kNoAllocBytes];

static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up on first use).
static upslam_status noalloc_scratch(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_icp_noalloc_ws) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return UPSLAM_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return UPSLAM_OK;
}

}  // namespace upslam

extern "C" size_t upslam_icp_noalloc_capacity_bytes(void) { return kNoAllocBytes; }

extern "C" upslam_status upslam_icp_noalloc(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                            const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *stream) {
    if (!views_ok(kf, sw) || !d_pose12 || !ip || !d_stats) return UPSLAM_ERR_INVALID_ARG;
    if (!(ip->d_max > 0.0f) || ip->max_iters < 0 || ip->min_inliers < 0) return UPSLAM_ERR_INVALID_ARG;
    if (ip->max_iters == 0) return UPSLAM_OK;
    int dev = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return UPSLAM_ERR_UNSUPPORTED;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, icp_persistent_kernel, kIcpThreads, 0) != cudaSuccess ||
        per_sm < 1)
        return UPSLAM_ERR_UNSUPPORTED;
    if (per_sm > 4) per_sm = 4;
    int grid = upslam_sm_count() * per_sm;
    if (grid > max_ctas()) grid = max_ctas();
    // the scratch a launch of this grid needs must fit the fixed array
    if (kCtrlBytes + (size_t)grid * kSlots * sizeof(float) > kNoAllocBytes) return UPSLAM_ERR_CAPACITY;
    void *ws = nullptr;
    const upslam_status st = noalloc_scratch(&ws);
    if (st != UPSLAM_OK) return st;
    // the barrier counters must start at zero; the per-CTA sums are written before they are read
    if (cudaMemsetAsync(ws, 0, kCtrlBytes, (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    IcpArgs a = make_args(kf, sw, ip);
    IcpCtrl *ctrl = reinterpret_cast<IcpCtrl *>(ws);
    float *partials = reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + kCtrlBytes);
    upslam_icp_params ipc = *ip;
    void *args[] = {&a, &d_pose12, &ipc, &d_stats, &ctrl, &partials};
    if (cudaLaunchCooperativeKernel((const void *)icp_persistent_kernel, dim3(grid), dim3(kIcpThreads), args, 0,
                                    (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    return UPSLAM_OK;
}
