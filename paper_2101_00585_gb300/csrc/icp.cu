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
// The 6x6 system is solved with an FP64 square-root-free Cholesky (L D L^T)
// and the SE(3) exponential is applied in FP64.
//
// Two launch forms:
//  * icp_step_kernel: one Gauss-Newton step.  FP32 per thread -> warp shuffles
//    -> compensated FP32 per CTA -> compensated FP32 over CTAs in a fixed order
//    (deterministic) -> FP64; the CTA that arrives last ("last CTA done"
//    ticket) solves.
//  * icp_tile_kernel: all iterations in one cooperative launch, one CTA per SM,
//    the CTA's keyframe samples staged in shared memory once.  Each step's sums
//    are exact fixed-point integers that every CTA adds into global words; the
//    same words carry an arrival count, so one poll of them is both the grid
//    barrier and the read of the totals.  Every CTA then solves the identical
//    system itself.  Every wait is bounded by a clock64 budget and reports
//    UPSLAM_ERR_TIMEOUT instead of hanging.
//
// Roofline: icp_step_kernel streams the keyframe once per step (4 B depth +
// 16 B or 8 B normal/weight per pixel); icp_tile_kernel streams it once per
// launch.  Each correspondence gathers 32 B (16 B in FP16) of sweep data that
// stays resident in L2.
#include <mutex>
#include <string.h>

#include "common.cuh"

namespace upslam {

constexpr int kIcpThreads = 256;
constexpr int kIcpWarps = kIcpThreads / 32;
// Per-CTA partial: 28 FP32 sums and their Neumaier compensations, then the
// inlier and valid counts as integers (64 words = 256 bytes per CTA).
constexpr int kSlots = 64;
constexpr size_t kCtrlBytes = 36864;  // IcpCtrl, then the tiled form's exact accumulators
constexpr size_t kAccOffset = 256;    // three buffers of kFxWords accumulators
constexpr int kFxWords = 86;          // 28 sums x 3 chunks, inliers, valid
// 64-bit words from one accumulator to the next: each sits on its own 128-byte L2 line, so the
// adds and polls of 152 CTAs spread over many L2 slices instead of queueing on six lines
constexpr int kAccStride = 16;
// Each CTA adds into every accumulator of a step exactly once: its partial (a CTA's partial lies
// in (-2^36, 2^36): 16 warps of chunks below 2^32) plus kFxBias, which makes the addend positive,
// plus one arrival unit in bits 48-63.  With at most kFxMaxCtas CTAs the low 48 bits never carry
// into the count, so a word holds its whole total exactly when its count equals the grid size.
constexpr unsigned long long kFxBias = 1ull << 36;
constexpr unsigned long long kFxCount = 1ull << 48;
constexpr int kFxMaxCtas = 2048;
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at 2 GHz
// the exact accumulators sit after IcpCtrl inside the control block that every call clears
static_assert(kAccOffset + 3 * (size_t)kFxWords * kAccStride * sizeof(unsigned long long) <= kCtrlBytes,
              "three accumulator buffers fit the control block");
static_assert((long long)kFxMaxCtas * 2 * (long long)kFxBias <= (long long)kFxCount,
              "the biased partials of the largest grid stay below the count field");

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
    int l1;            // 1: absolute error by IRLS (weights 1 / max(|r|, loss_delta)); 0: squared error
    float loss_delta;
    float d_max2_fine;  // the gate of steps coarse_iters, coarse_iters + 1, ... (coarse_iters > 0)
    int coarse_iters;
    long long wait_cycles;  // budget of every grid-barrier wait (clock64 cycles)
    int withhold;           // test support: CTA 0 does not arrive at the first Gauss-Newton barrier
};

// Square root of the IRLS weight of residual r: each correspondence enters the
// normal equations as (s J, s r), so J^T J, J^T r and r^2 carry w = s^2.  The
// loss is a template parameter, so the squared-error kernels carry no trace of it.
template <int L1>
__device__ __forceinline__ float irls_scale(const IcpArgs &a, float r) {
    return L1 ? rsqrtf(fmaxf(fabsf(r), a.loss_delta)) : 1.0f;
}

// Motion prior folded into the persistent launch (upslam_register).
struct PriorArgs {
    const double *prev;  // previous sweep's pose in the keyframe (mode >= 1)
    const double *motion;  // last inter-sweep motion (mode 2)
    double *motion_out;  // if set: prev^-1 * registered pose
    double *prev_out;    // if set: the registered pose
    int mode;            // 0: start from *pose, 1: zero velocity, 2: constant velocity
};

// Sweep front end folded into the register + update launch (upslam_track_scan):
// projection with the z-buffer, resolve and normals of the sweep (Sec. III-A),
// each phase ending at a grid barrier.
struct FrontArgs {
    const float4 *pts;          // scan points (x, y, z, valid)
    int n;                      // points
    unsigned long long *zbuf;   // sweep z-buffer, all ones at rest (left so)
    float *depth;               // sweep depth [rows * cols]
    int *idx;                   // winner index [rows * cols]
    float4 *pix;                // winner point [rows * cols]
    void *nrm;                  // sweep normals (nrm_prec)
    int nrm_prec;
    upslam_normal_params np;
    int on;
};

struct IcpCtrl {
    unsigned int arrive;               // unused by the current kernels (kept zero)
    unsigned int gen;                  // unused by the current kernels (kept zero)
    unsigned int ticket;               // single-step "last CTA" ticket
    int valid;                         // unused by the current kernels (kept zero)
    unsigned long long arrive64;       // persistent form: CTA arrivals, monotonic across launches
};
static_assert(sizeof(IcpCtrl) <= kAccOffset, "the control words end before the exact accumulators");

template <int L1>
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
    const float4 P = __ldcg(a.spix + j);
    if (P.w == 0.0f) return;
    const float4 m = load_nw_cg(a.snrm, j, a.sprec);
    if (m.w == 0.0f) return;
    const float *r = T.r;
    const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
    const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
    const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
    const float3 Rm = rotate(T, m.x, m.y, m.z);
    const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
    if (!(ex * ex + ey * ey + ez * ez <= a.d_max2)) return;
    if (!(Rm.x * n.x + Rm.y * n.y + Rm.z * n.z >= a.cos_min)) return;
    const float r0 = ex * n.x + ey * n.y + ez * n.z;
    const float w = irls_scale<L1>(a, r0);
    const float res = r0 * w;
    float J[6];
    J[0] = (py * n.z - pz * n.y) * w;
    J[1] = (pz * n.x - px * n.z) * w;
    J[2] = (px * n.y - py * n.x) * w;
    J[3] = n.x * w;
    J[4] = n.y * w;
    J[5] = n.z * w;
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

// Warp reduce-scatter, then the CTA's warps summed (compensated FP32) into its partial record.
__device__ __forceinline__ void cta_partial(float acc[28], int inl, int valid, float *partial, float (*sh)[32],
                                            int (*shi)[2]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = i < 28 ? acc[i] : 0.0f;
    const float s = warp_reduce_scatter(v);  // lane i: the warp's sum of acc[i]
    if (lane < 28) sh[warp][lane] = s;
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
        c += __ldcg(&a.spix[j].w) != 0.0f;
    return c;
}

template <int L1>
__global__ void __launch_bounds__(kIcpThreads) icp_step_kernel(IcpArgs a, double *pose, upslam_icp_params ip,
                                                               upslam_icp_stats *st, IcpCtrl *ctrl,
                                                               float *partials) {
    __shared__ float sh[kIcpWarps][32];
    __shared__ int shi[kIcpWarps][2];
    __shared__ double tot[32];
    __shared__ int last;
    const PoseF T = cta_pose_f32(pose, true);
    float acc[28];
#pragma unroll
    for (int i = 0; i < 28; ++i) acc[i] = 0.0f;
    int inl = 0;
    const int npx = a.kp.rows * a.kp.cols;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x)
        accumulate_pixel<L1>(a, T, k, acc, inl);
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

// ----------------------------------------------------------------------------- tiled persistent form
//
// One CTA of 512 threads per SM.  The keyframe is cut into slices of 64
// pixels dealt round-robin to the CTAs (samples only occupy the rows the sensor
// sees, so contiguous ranges would leave most CTAs idle; and short slices mix
// every azimuth into every CTA, where chunks of whole row quarters or eighths
// would give each CTA one azimuth sector).  Before the first step each CTA
// streams its slices once from HBM and stages every pixel that
// holds a sample (depth > 0, unit normal) into shared memory as its FP32 point
// s = d * dir and normal n, compacted in pixel order (a block-wide ballot
// prefix, so the order and therefore the sums are deterministic).  Every
// Gauss-Newton step then reads the staged points from shared memory and gathers
// only the sweep pixel each one lands in.  Units beyond the shared-memory
// capacity are read from global memory each step.

constexpr int kTileThreads = 512;
constexpr int kTileWarps = kTileThreads / 32;
// keyframe units (kTileThreads pixels) staged per memory round trip: a 512x2048 keyframe deals 14 units
// to each of 152 CTAs, so each half of the front end's staging is one round trip (8 spills registers)
constexpr int kStageGroup = 7;
// The keyframe is dealt to the CTAs in slices of kSlice pixels, slice s to CTA s mod gridDim, and a
// CTA walks its slices in units of kTileThreads pixels (one per thread).  The fine interleave evens
// the CTAs' sample counts, whatever rows of the panorama hold samples.
constexpr int kSlice = 64;
constexpr int kUnitSlices = kTileThreads / kSlice;

// The sweep pixel a staged keyframe point lands in: its point and normal,
// gathered from L2, and whether the point binned at all.
struct SweepHit {
    float4 P, m;
    bool binned;
};

__device__ __forceinline__ SweepHit gather_entry(const IcpArgs &a, const PoseF &T, float3 s) {
    const float3 q = xform_inv(T, s.x, s.y, s.z);
    int jv = 0, ju = 0;
    float rr;
    SweepHit h;
    h.binned = bin_point(q.x, q.y, q.z, a.sp, jv, ju, rr);
    const int j = h.binned ? jv * a.sp.cols + ju : 0;
    h.P = __ldcg(a.spix + j);
    h.m = load_nw_cg(a.snrm, j, a.sprec);
    return h;
}

// One staged correspondence, branch-free: a rejected pair contributes zeros.
template <int L1>
__device__ __forceinline__ void accumulate_entry(const IcpArgs &a, const PoseF &T, float3 s, float3 n,
                                                 const SweepHit &h, float acc[28], int &inl) {
    const float4 P = h.P, m = h.m;
    bool ok = h.binned && P.w != 0.0f && m.w != 0.0f;
    const float *r = T.r;
    const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
    const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
    const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
    const float3 Rm = rotate(T, m.x, m.y, m.z);
    const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
    ok = ok && (ex * ex + ey * ey + ez * ez <= a.d_max2) && (Rm.x * n.x + Rm.y * n.y + Rm.z * n.z >= a.cos_min);
    const float r0 = ex * n.x + ey * n.y + ez * n.z;
    const float w = ok ? irls_scale<L1>(a, r0) : 0.0f;
    const float res = r0 * w;
    float J[6];
    J[0] = (py * n.z - pz * n.y) * w;
    J[1] = (pz * n.x - px * n.z) * w;
    J[2] = (px * n.y - py * n.x) * w;
    J[3] = n.x * w;
    J[4] = n.y * w;
    J[5] = n.z * w;
    int p = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int c = i; c < 6; ++c) {
            acc[p] = fmaf(J[i], J[c], acc[p]);
            ++p;
        }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[21 + i] = fmaf(J[i], res, acc[21 + i]);
    acc[27] = fmaf(res, res, acc[27]);
    inl += ok ? 1 : 0;
}

// The CTA's contribution to one step's sums, exact: each warp's 28 sums (warp
// reduce-scatter) go into shared 64-bit integer accumulators as fixed-point
// chunks, the inlier and valid counts as integers.
__device__ __forceinline__ void tile_fx(float acc[28], int inl, int valid, unsigned long long *fxs) {
    const int lane = threadIdx.x & 31;
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = i < 28 ? acc[i] : 0.0f;
    const float s = warp_reduce_scatter(v);  // lane i: the warp's sum of acc[i]
    if (lane < 28) {
        long long c[3];
        fx_chunks(s, c);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            if (c[k]) atomicAdd(fxs + 3 * lane + k, (unsigned long long)c[k]);
    }
    const int si = __reduce_add_sync(0xffffffffu, inl);
    const int sv = __reduce_add_sync(0xffffffffu, valid);
    if (lane == 0) {
        if (si) atomicAdd(fxs + 84, (unsigned long long)si);
        if (sv) atomicAdd(fxs + 85, (unsigned long long)sv);
    }
}

// Grid barrier on a monotonic 64-bit arrival counter, called by one thread per
// CTA after a __syncthreads.  The release add publishes everything the CTA
// wrote before the barrier; the polls are relaxed loads, and one acquire fence
// after the last makes every other CTA's writes visible (the caller's next
// __syncthreads extends both to the whole CTA).  False when the count has not
// reached target after `budget` cycles (the caller reports UPSLAM_ERR_TIMEOUT).
__device__ __forceinline__ void grid_arrive(unsigned long long *ctr) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
}

__device__ __forceinline__ bool grid_wait(unsigned long long *ctr, unsigned long long target, long long budget) {
    const long long t0 = clock64();
    unsigned long long v;
    for (;;) {
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        if (v >= target) break;
        if (clock64() - t0 > budget) return false;
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    return true;
}

__device__ __forceinline__ bool grid_arrive_wait(unsigned long long *ctr, unsigned long long target,
                                                 long long budget) {
    grid_arrive(ctr);
    return grid_wait(ctr, target, budget);
}

// Split-phase grid barrier: the CTA arrives (after everything it wrote), does other work,
// then waits.  cta_grid_arrive must be reached by the whole CTA; so must cta_grid_await.
__device__ __forceinline__ void cta_grid_arrive(IcpCtrl *ctrl) {
    __syncthreads();
    if (threadIdx.x == 0) grid_arrive(&ctrl->arrive64);
}

__device__ __forceinline__ bool cta_grid_await(IcpCtrl *ctrl, unsigned long long target, upslam_icp_stats *st,
                                               int *flag_s, long long budget) {
    __syncthreads();
    if (threadIdx.x == 0) {
        *flag_s = 0;
        if (!grid_wait(&ctrl->arrive64, target, budget)) {
            *flag_s = 3;
            st->status = UPSLAM_ERR_TIMEOUT;
        }
    }
    __syncthreads();
    return *flag_s != 3;
}

// The tiled persistent kernel.  Each step: accumulate the CTA's staged (and
// spilled) correspondences, publish the CTA record (double-buffered by step
// parity), arrive at a grid barrier (a monotonic 64-bit arrival counter), then
// every CTA sums all records and solves redundantly: identical arithmetic on
// identical data gives every CTA the same pose, so no CTA waits for another
// to broadcast it.  CTA 0 writes the pose and the record at the end.  L1: the IRLS
// reading of Eq. 1; KF16: the keyframe stores FP16 normals and counts.
template <int L1, int KF16>
__global__ void __launch_bounds__(kTileThreads, 1)
    icp_tile_kernel(IcpArgs a, double *pose, upslam_icp_params ip, upslam_icp_stats *st, IcpCtrl *ctrl,
                    float *partials, int cap, PriorArgs pr, FuseView fz, int fuse_on, FrontArgs fr) {
    // staged samples, structure of arrays of length cap (a multiple of 4): the point s = d * dir, the
    // normal and count (FP32 keyframes: three floats and the count; FP16 keyframes: the keyframe's own four
    // halves, which lose nothing) and the pixel index.  The depth is read again from the keyframe when the
    // update averages a sample (no step writes it before then).
    extern __shared__ float stage[];
    constexpr bool kf16 = KF16 != 0;
    float *sx = stage, *sy = stage + cap, *sz = stage + 2 * cap;
    float *snx = stage + 3 * cap, *sny = stage + 4 * cap, *snz = stage + 5 * cap, *sw8 = stage + 6 * cap;
    uint2 *snh = reinterpret_cast<uint2 *>(stage + 3 * cap);
    int *sk = reinterpret_cast<int *>(stage + (kf16 ? 5 : 7) * cap);
    auto staged_nw = [&](int e) -> float4 {
        if (!kf16) return make_float4(snx[e], sny[e], snz[e], sw8[e]);
        const uint2 h = snh[e];
        const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&h.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&h.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    };
    __shared__ double tot[32];
    __shared__ long long totn[2];
    __shared__ unsigned long long fxs[kFxWords];
    __shared__ int gbm_s;
    __shared__ double Tsh[12];
    __shared__ double Tprev[12], Tmot[12];
    __shared__ float Tf[12];
    __shared__ int acc_ok_s;
    __shared__ double xi_sh[6];
    __shared__ int wcnt[2][kStageGroup][kTileWarps];
    __shared__ int flag, status_s, conv_s, valid_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npx = a.kp.rows * a.kp.cols;
    const int nslices = (npx + kSlice - 1) / kSlice;
    const int W = a.kp.cols;
    const unsigned long long G = gridDim.x;
    unsigned long long base = 0;
    if (threadIdx.x == 0) {
        base = (*((volatile unsigned long long *)&ctrl->arrive64) / G) * G;
        gbm_s = (int)((base / G) % 3ull);
    }
    // exact step sums: barrier number j (counted over the whole workspace's life) owns buffer
    // j mod 3, and only the Gauss-Newton steps' barriers add into theirs.  CTA 0 clears buffer
    // j - 1 once it has passed barrier j (every CTA has then finished reading it, and nobody adds
    // into it before barrier j + 1 has passed).  So at a launch's start only the buffer of the
    // last barrier before it can hold sums, and the launch's first barrier clears it.
    unsigned long long *const acc_base =
        reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(ctrl) + kAccOffset);
    auto acc_buf = [&](unsigned long long j) {
        return acc_base + (size_t)((gbm_s + j) % 3ull) * kFxWords * kAccStride;
    };
    auto clear_buf = [&](unsigned long long *b) {  // one warp
        for (int i = lane; i < kFxWords; i += 32) b[(size_t)i * kAccStride] = 0ull;
    };
    auto clear_prev = [&](unsigned long long j) {  // after passing barrier j; warp 1 of CTA 0
        if (blockIdx.x == 0 && warp == 1) clear_buf(acc_buf(j + 2));  // = buffer j - 1
    };
    if (pr.mode == 0) {
        if (threadIdx.x < 12) Tsh[threadIdx.x] = __ldcg(pose + threadIdx.x);
    } else if (warp == 0) {
        // initial guess from the motion prior: T0 = prev (zero velocity) or prev * motion
        if (lane < 12) {
            Tprev[lane] = __ldcg(pr.prev + lane);
            Tmot[lane] = pr.mode == 2 ? __ldcg(pr.motion + lane) : 0.0;
        }
        __syncwarp();
        if (pr.mode == 2) {
            warp_pose_mul(Tprev, Tmot, Tsh);
            if (lane == 0) orthonormalise_rows(Tsh);
        } else if (lane < 12) {
            Tsh[lane] = Tprev[lane];
        }
        __syncwarp();
    }

    // ---- stage the CTA's slices into shared memory (once per launch), a unit of
    // eight slices (one pixel per thread) at a time.  kStageGroup units are loaded
    // together (one memory round trip for the group) and compacted with one
    // barrier: the per-warp counts are double-buffered by group parity.  A unit
    // that no longer fits is left, with every later unit of this CTA, to the
    // global-memory path.
    const int my_slices = (int)blockIdx.x < nslices ? (nslices - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int my_units = (my_slices + kUnitSlices - 1) / kUnitSlices;
    const int my_groups = (my_units + kStageGroup - 1) / kStageGroup;
    // this thread's pixel of the CTA's unit u; false past the panorama
    auto unit_pixel = [&](int u, int &k) -> bool {
        const int s = (u * kUnitSlices + (int)threadIdx.x / kSlice) * (int)gridDim.x + (int)blockIdx.x;
        k = s * kSlice + ((int)threadIdx.x & (kSlice - 1));
        return s < nslices && k < npx;
    };
    int staged = 0, spill_u = my_units, par = 0;
    bool spilled = false;
    auto stage_groups = [&](int g_begin, int g_end) {
        for (int gi = g_begin; gi < g_end && !spilled; ++gi, par ^= 1) {
            const int u0 = gi * kStageGroup;
            float dg[kStageGroup];
            // FP16 keyframes hold a unit in three registers (the depth and the keyframe's four halves as
            // stored; the direction tables are read at the commit, for samples only), which leaves the
            // kernel room below its register limit; FP32 keyframes hold the normal, count and directions
            float4 ng[kStageGroup];
            uint2 hg[kStageGroup];
            float2 eg[kStageGroup], ag[kStageGroup];
#pragma unroll
            for (int g = 0; g < kStageGroup; ++g) {
                int k;
                const bool in = unit_pixel(u0 + g, k);
                dg[g] = 0.0f;
                ng[g] = make_float4(0.f, 0.f, 0.f, 0.f);
                hg[g] = make_uint2(0u, 0u);
                eg[g] = ag[g] = make_float2(0.f, 0.f);
                if (in) {
                    dg[g] = __ldg(a.kdepth + k);
                    if (!kf16) {
                        const int v = k / W;
                        eg[g] = __ldg(reinterpret_cast<const float2 *>(a.kdirs) + v);
                        ag[g] = __ldg(reinterpret_cast<const float2 *>(a.kdirs + 2 * a.kp.rows) + (k - v * W));
                    }
                }
            }
            // the normal and count only where the depth holds a sample (empty pixels have depth 0)
#pragma unroll
            for (int g = 0; g < kStageGroup; ++g) {
                int k;
                unit_pixel(u0 + g, k);
                if (dg[g] > 0.0f) {
                    if (kf16) hg[g] = __ldg(reinterpret_cast<const uint2 *>(a.knw) + k);
                    else ng[g] = load_nw(a.knw, k, a.kprec);
                }
            }
            unsigned bal[kStageGroup];
#pragma unroll
            for (int g = 0; g < kStageGroup; ++g) {
                float4 n4 = ng[g];
                if (kf16) {
                    const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&hg[g].x));
                    const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&hg[g].y));
                    n4 = make_float4(lo.x, lo.y, hi.x, hi.y);
                }
                const bool ok = dg[g] > 0.0f && __fadd_rn(__fadd_rn(__fmul_rn(n4.x, n4.x), __fmul_rn(n4.y, n4.y)),
                                                          __fmul_rn(n4.z, n4.z)) > 0.25f;
                bal[g] = __ballot_sync(0xffffffffu, ok);
                if (lane == 0) wcnt[par][g][warp] = __popc(bal[g]);
            }
            __syncthreads();
            // every thread derives the same offsets and totals from the counts
            int fit = kStageGroup;
            int off[kStageGroup];
            int total = staged;
#pragma unroll
            for (int g = 0; g < kStageGroup; ++g) {
                // the warps' counts, scanned across lanes 0..15: the count before this warp, and the group's
                const int c = lane < kTileWarps ? wcnt[par][g][lane] : 0;
                int incl = c;
#pragma unroll
                for (int d = 1; d < kTileWarps; d <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += v;
                }
                const int before = __shfl_sync(0xffffffffu, incl - c, warp);
                const int o = total + before;
                total += __shfl_sync(0xffffffffu, incl, kTileWarps - 1);
                off[g] = o + __popc(bal[g] & ((1u << lane) - 1u));
                if (fit == kStageGroup && total > cap) fit = g;
                if (fit == kStageGroup) staged = total;
            }
#pragma unroll
            for (int g = 0; g < kStageGroup; ++g) {
                if (g >= fit || !((bal[g] >> lane) & 1u)) continue;
                int k;
                unit_pixel(u0 + g, k);
                const int slot = off[g];
                const float d = dg[g];
                float2 e = eg[g], az = ag[g];
                if (kf16) {  // direction-table entries (small, cached) read for samples only
                    const int v = k / W;
                    e = __ldg(reinterpret_cast<const float2 *>(a.kdirs) + v);
                    az = __ldg(reinterpret_cast<const float2 *>(a.kdirs + 2 * a.kp.rows) + (k - v * W));
                }
                sx[slot] = __fmul_rn(d, __fmul_rn(e.x, az.x));
                sy[slot] = __fmul_rn(d, __fmul_rn(e.x, az.y));
                sz[slot] = __fmul_rn(d, e.y);
                if (kf16) {
                    snh[slot] = hg[g];  // the halves the keyframe holds
                } else {
                    snx[slot] = ng[g].x;
                    sny[slot] = ng[g].y;
                    snz[slot] = ng[g].z;
                    sw8[slot] = ng[g].w;
                }
                sk[slot] = k;
            }
            if (fit < kStageGroup) {  // uniform across the CTA: the counts are shared
                spill_u = u0 + fit;
                spilled = true;
            }
        }
    };

    // ---- sweep front end (upslam_track_scan): project; arrive; stage the first half of
    // the keyframe while the other CTAs finish projecting; wait; resolve the z-buffer and
    // form the normals from it in one pass; arrive; stage the rest; wait; reset the words.
    // The keyframe does not depend on the sweep, so its loads fill both barrier waits.
    unsigned long long nbar = 0;  // grid barriers passed before the Gauss-Newton steps
    if (fr.on) {
        const int ns = a.sp.rows * a.sp.cols;
        const int stride = gridDim.x * kTileThreads;
        // (warps 1.. project while warp 0 forms the motion prior above)
        if (warp > 0) {
            const int pstride = gridDim.x * (kTileThreads - 32);
            for (int i = blockIdx.x * (kTileThreads - 32) + threadIdx.x - 32; i < fr.n; i += pstride)
                project_point(fr.pts, i, a.sp, fr.zbuf);
        }
        cta_grid_arrive(ctrl);
        stage_groups(0, my_groups / 2);
        if (!cta_grid_await(ctrl, base + G * ++nbar, st, &flag, a.wait_cycles)) return;
        clear_prev(nbar);
        const PixZbuf zb{fr.pts, fr.zbuf};
        for (int k = blockIdx.x * kTileThreads + threadIdx.x; k < ns; k += stride) {
            resolve_pixel<true, false>(fr.pts, k, fr.zbuf, fr.depth, fr.idx, fr.pix);
            store_nw(fr.nrm, k, fr.nrm_prec, normal_pixel(zb, a.sp, fr.np, k));
        }
        cta_grid_arrive(ctrl);
        stage_groups(my_groups / 2, my_groups);
        if (!cta_grid_await(ctrl, base + G * ++nbar, st, &flag, a.wait_cycles)) return;
        // (the buffer before this barrier belongs to the front end's first barrier: never added into)
        for (int k = blockIdx.x * kTileThreads + threadIdx.x; k < ns; k += stride) fr.zbuf[k] = kEmptyKey;
    } else {
        stage_groups(0, my_groups);
        __syncthreads();
    }

    // convergence thresholds, squared once per launch (read by warp 0 only)
    const double er2 = warp == 0 ? ip.eps_rot * ip.eps_rot : 0.0, et2 = warp == 0 ? ip.eps_trans * ip.eps_trans : 0.0;
    int it = 0;
    for (; it < ip.max_iters; ++it) {
        // the pose in FP32: converted once per CTA (FP64 conversions are slow on GB300), read by all
        if (threadIdx.x < 12) Tf[threadIdx.x] = (float)Tsh[threadIdx.x];
        if (threadIdx.x < kFxWords) fxs[threadIdx.x] = 0ull;
        __syncthreads();
        PoseF T;
#pragma unroll
        for (int i = 0; i < 12; ++i) T.r[i] = Tf[i];
        float acc[28];
#pragma unroll
        for (int i = 0; i < 28; ++i) acc[i] = 0.0f;
        int inl = 0;
        // this step's Omega distance gate (coarse-to-fine when coarse_iters > 0)
        IcpArgs as = a;
        if (a.coarse_iters > 0 && it >= a.coarse_iters) as.d_max2 = a.d_max2_fine;
        // Software-pipelined: the gathers of a thread's next entry are issued
        // before the current one is reduced, so each L2 round trip overlaps
        // the previous entry's arithmetic.  The entries are still summed in
        // the same order.
        if (threadIdx.x < staged) {
            SweepHit h = gather_entry(as, T, make_float3(sx[threadIdx.x], sy[threadIdx.x], sz[threadIdx.x]));
            for (int e = threadIdx.x; e < staged; e += kTileThreads) {
                const int e1 = min(e + kTileThreads, staged - 1);  // the last prefetch repeats an entry, unused
                const SweepHit h1 = gather_entry(as, T, make_float3(sx[e1], sy[e1], sz[e1]));
                const float4 n4 = staged_nw(e);
                accumulate_entry<L1>(as, T, make_float3(sx[e], sy[e], sz[e]), make_float3(n4.x, n4.y, n4.z), h, acc,
                                     inl);
                h = h1;
            }
        }
        for (int u = spill_u; u < my_units; ++u) {
            int k;
            if (unit_pixel(u, k)) accumulate_pixel<L1>(as, T, k, acc, inl);
        }
        const int valid = it == 0 ? count_valid(a) : 0;
        tile_fx(acc, inl, valid, fxs);
        __syncthreads();
        const unsigned long long jb = nbar + (unsigned long long)(it + 1);  // this step's barrier
        unsigned long long *const buf = acc_buf(jb);
        // (test support: with `withhold`, CTA 0 skips its first contribution, so no CTA's wait can end)
        if (!(a.withhold && it == 0 && blockIdx.x == 0)) {
            if (threadIdx.x < kFxWords) {
                const unsigned long long v = fxs[threadIdx.x] + kFxBias + kFxCount;
                asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(buf + (size_t)threadIdx.x * kAccStride),
                             "l"(v)
                             : "memory");
            } else if (threadIdx.x == kTileThreads - 32) {
                grid_arrive(&ctrl->arrive64);  // keeps the barrier count that the later phases wait on
            }
        }
        if (warp == 0) {
            // wait until every CTA has added into every word: the last loads hold the step's totals
            // (lane i < 28 reads sum i's three chunks, lane 28 the inlier and valid counts)
            // (lanes past the last word re-read it)
            unsigned long long w[3];
            const long long t0 = clock64();
            bool late = false;
            for (;;) {
                bool done = true;
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];"
                                 : "=l"(w[k])
                                 : "l"(buf + (size_t)min(3 * lane + k, kFxWords - 1) * kAccStride)
                                 : "memory");
                    done = done && (w[k] >> 48) == G;
                }
                if (__all_sync(0xffffffffu, done)) break;
                if (__any_sync(0xffffffffu, clock64() - t0 > a.wait_cycles)) {
                    late = true;
                    break;
                }
            }
            if (lane == 0) {
                flag = late ? 3 : 0;
                if (late) st->status = UPSLAM_ERR_TIMEOUT;
            }
            // (no fence here: the solve reads nothing but these words, and a fence would cost the
            // critical path about 800 cycles; warp 1 of CTA 0 takes the fences that the clearing needs)
            if (blockIdx.x == 0) asm volatile("bar.arrive 1, 64;" ::: "memory");  // warp 1 may clear
            if (!late) {
                const long long off = (long long)G * (long long)kFxBias;
                if (lane < 28) {
                    tot[lane] = fx_value((long long)(w[0] & (kFxCount - 1)) - off,
                                         (long long)(w[1] & (kFxCount - 1)) - off,
                                         (long long)(w[2] & (kFxCount - 1)) - off);
                } else if (lane == 28) {
                    totn[0] = (long long)(w[0] & (kFxCount - 1)) - off;
                    totn[1] = (long long)(w[1] & (kFxCount - 1)) - off;
                }
                __syncwarp();
                const long long inliers = totn[0];
                double xi[6] = {0, 0, 0, 0, 0, 0};
                int status = UPSLAM_OK, conv = 0;
                if (inliers < ip.min_inliers) {
                    status = UPSLAM_ERR_DEGENERATE;
                } else {
                    if (!warp_solve6(tot, ip.pivot_eps, xi)) {
                        status = UPSLAM_ERR_DEGENERATE;
#pragma unroll
                        for (int i = 0; i < 6; ++i) xi[i] = 0.0;
                    } else {
                        warp_se3_update(xi, Tsh);
                        conv = warp_converged(xi, er2, et2) ? 1 : 0;
                    }
                }
                if (lane == 0) {
                    status_s = status;
                    conv_s = conv;
                    if (it == 0) valid_s = (int)totn[1];
#pragma unroll
                    for (int i = 0; i < 6; ++i) xi_sh[i] = xi[i];
                }
            }
        } else if (warp == 1 && blockIdx.x == 0) {
            // every CTA has added into this step's buffer, so every CTA has read the previous one:
            // clear that one.  The first fence orders the clearing after warp 0's observation of
            // those adds; the second orders the zeros before CTA 0's next contribution, which every
            // CTA must observe before it can add into the cleared buffer again.  Both run while
            // warp 0 solves.
            asm volatile("bar.sync 1, 64;" ::: "memory");
            if (*((volatile int *)&flag) != 3) {
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
                clear_buf(acc_buf(jb + 2));
                asm volatile("fence.acq_rel.gpu;" ::: "memory");
            }
        }
        __syncthreads();
        if (flag == 3) return;
        if (status_s != UPSLAM_OK || conv_s) {
            ++it;
            break;
        }
    }
    // the motion update M = T_prev^-1 T, by warp 0 of CTA 0
    auto publish_motion = [&]() {
        if (blockIdx.x == 0 && warp == 0 && pr.mode != 0 && pr.motion_out) {
            warp_pose_inv(Tprev, Tmot);
            double M[12];
            warp_pose_mul(Tmot, Tsh, Tmot);
            if (lane == 0) {
                for (int i = 0; i < 12; ++i) M[i] = Tmot[i];
                orthonormalise_rows(M);
                for (int i = 0; i < 12; ++i) pr.motion_out[i] = M[i];
            }
        }
    };
    // ---- keyframe update with the registered pose (Sec. III-C), gated by the
    // registration quality: every CTA holds the same totals, so all take the same decision.
    int accepted_flag = 0;
    if (fuse_on) {
        if (threadIdx.x == 0) {
            acc_ok_s = status_s == UPSLAM_OK && valid_s > 0 && (float)totn[0] >= fz.accept * (float)valid_s;
        }
        if (threadIdx.x < 12) Tf[threadIdx.x] = (float)Tsh[threadIdx.x];
        __syncthreads();
        const bool acc_ok = acc_ok_s != 0;
        accepted_flag = acc_ok ? 1 : 0;
        PoseF T;
#pragma unroll
        for (int i = 0; i < 12; ++i) T.r[i] = Tf[i];
        const int ns = fz.sp.rows * fz.sp.cols;
        // warp 0 of CTA 0 forms the motion update meanwhile; the other threads take its share
        const int ex = (pr.mode != 0 && pr.motion_out) ? 32 : 0;
        publish_motion();
        if (acc_ok) {
            // average the staged samples straight from shared memory, spilled units from global memory
            const int e0 = blockIdx.x == 0 ? (int)threadIdx.x - ex : (int)threadIdx.x;
            const int es = blockIdx.x == 0 ? kTileThreads - ex : kTileThreads;
            for (int e = e0; e >= 0 && e < staged; e += es)
                fuse_average(fz, T, sk[e], make_float3(sx[e], sy[e], sz[e]), staged_nw(e), fz.kdepth[sk[e]]);
            for (int u = spill_u; u < my_units; ++u) {
                int k;
                if (!unit_pixel(u, k)) continue;
                const float4 n4 = load_nw(fz.knw, k, fz.kprec);
                if (!(n4.w > 0.0f)) continue;
                const float d = __ldg(fz.kdepth + k);
                const int v = k / W;
                fuse_average(fz, T, k, pixel_point(fz.kdirs, fz.kp.rows, v, k - v * W, d), n4, d);
            }
            // hole fill, first pass: z-buffer atomics into empty keyframe pixels
            for (int j = (int)(blockIdx.x * kTileThreads + threadIdx.x) - ex; j >= 0 && j < ns;
                 j += (int)(gridDim.x * kTileThreads) - ex) {
                int k;
                unsigned long long key;
                float r;
                float4 m;
                if (!holefill_key(fz, T, j, k, key, r, m)) continue;
                if (load_nw(fz.knw, k, fz.kprec).w != 0.0f) continue;
                atomicMin(fz.zbuf + k, key);
            }
        }
        // one more grid barrier (every CTA arrives, accepted or not)
        __syncthreads();
        if (threadIdx.x == 0) {
            flag = 0;
            if (!grid_arrive_wait(&ctrl->arrive64, base + G * (nbar + (unsigned long long)(it + 1)), a.wait_cycles)) {
                flag = 3;
                st->status = UPSLAM_ERR_TIMEOUT;
            }
        }
        __syncthreads();
        if (flag == 3) return;
        clear_prev(nbar + (unsigned long long)(it + 1));
        if (acc_ok) {
            // hole fill, second pass: the winning sweep pixel writes the keyframe pixel
            for (int j = blockIdx.x * kTileThreads + threadIdx.x; j < ns; j += gridDim.x * kTileThreads) {
                int k;
                unsigned long long key;
                float r;
                float4 m;
                if (!holefill_key(fz, T, j, k, key, r, m)) continue;
                if (__ldcg(fz.zbuf + k) != key) continue;
                holefill_write(fz, T, k, r, m);
            }
        }
    }
    // CTA 0 publishes the pose, the motion update (already, when the keyframe update ran) and the
    // record of the last linearisation
    if (!fuse_on) publish_motion();
    if (blockIdx.x == 0 && pr.prev_out && threadIdx.x < 12) pr.prev_out[threadIdx.x] = Tsh[threadIdx.x];
    if (blockIdx.x == 0) {
        if (threadIdx.x < 12) pose[threadIdx.x] = Tsh[threadIdx.x];
        if (threadIdx.x < 21) st->A[threadIdx.x] = tot[threadIdx.x];
        else if (threadIdx.x < 27) st->b[threadIdx.x - 21] = tot[threadIdx.x];
        else if (threadIdx.x == 27) st->sse = tot[27];
        else if (threadIdx.x == 28) st->inliers = totn[0];
        else if (threadIdx.x == 29) st->valid = valid_s;
        else if (threadIdx.x == 30) {
            st->status = status_s;
            st->converged = conv_s;
            st->iters = it;
            st->accepted = accepted_flag;
        } else if (threadIdx.x >= 32 && threadIdx.x < 38) {
            st->xi[threadIdx.x - 32] = xi_sh[threadIdx.x - 32];
        }
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
    a.l1 = ip->loss == UPSLAM_LOSS_L1 ? 1 : 0;
    a.loss_delta = ip->loss_delta;
    a.d_max2_fine = ip->d_max_fine * ip->d_max_fine;
    a.coarse_iters = ip->coarse_iters;
    a.wait_cycles = kWaitCycles;
    a.withhold = 0;
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


// Launch the tiled persistent kernel: one CTA per SM, the keyframe slice staged
// in as much dynamic shared memory as the slice needs (up to the opt-in limit).
static upslam_status launch_tile(const IcpArgs &a, double *pose, const upslam_icp_params *ip, upslam_icp_stats *st,
                                 void *ws, size_t ws_bytes, cudaStream_t stream, PriorArgs pr = PriorArgs{},
                                 const FuseView *fz = nullptr, const FrontArgs *front = nullptr) {
    int dev = 0, coop = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return UPSLAM_ERR_CUDA;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return UPSLAM_ERR_UNSUPPORTED;
    // per device and kernel variant: the kernel's static shared memory, recorded when its dynamic
    // limit is raised (once, so later calls under stream capture change no attribute); any host
    // thread may call, so the flags are atomic (the release store publishes static_smem)
    static std::atomic<bool> attr_set[4][64];
    static size_t static_smem[4][64] = {{0}};
    if (dev < 0 || dev >= 64) return UPSLAM_ERR_UNSUPPORTED;
    const int var = (a.l1 ? 1 : 0) + (a.kprec == UPSLAM_F16 ? 2 : 0);
    const void *const kernels[4] = {(const void *)icp_tile_kernel<0, 0>, (const void *)icp_tile_kernel<1, 0>,
                                    (const void *)icp_tile_kernel<0, 1>, (const void *)icp_tile_kernel<1, 1>};
    const void *fn = kernels[var];
    const size_t reserve = 1024;
    if (!attr_set[var][dev].load(std::memory_order_acquire)) {
        static std::mutex mu;
        std::lock_guard<std::mutex> lock(mu);
        if (!attr_set[var][dev].load(std::memory_order_relaxed)) {
            cudaFuncAttributes fa;
            if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return UPSLAM_ERR_CUDA;
            const int dyn_max = optin - (int)fa.sharedSizeBytes - (int)reserve;
            if (dyn_max <= 0 ||
                cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess)
                return UPSLAM_ERR_UNSUPPORTED;
            static_smem[var][dev] = fa.sharedSizeBytes;
            attr_set[var][dev].store(true, std::memory_order_release);
        }
    }
    const int grid = upslam_sm_count();
    if (grid > kFxMaxCtas) return UPSLAM_ERR_UNSUPPORTED;
    const int64_t npx = (int64_t)a.kp.rows * a.kp.cols;
    const int64_t nslices = (npx + kSlice - 1) / kSlice;
    const int64_t per = (nslices + grid - 1) / grid * kSlice;  // most pixels one CTA can stage
    // each staged sample: point (3), normal and count (4 floats, or 4 halves for an FP16 keyframe), pixel index
    const int64_t kWords = a.kprec == UPSLAM_F16 ? 6 : 8;
    const int64_t cap_max =
        (((int64_t)optin - (int64_t)static_smem[var][dev] - (int64_t)reserve) / (kWords * (int64_t)sizeof(float))) &
        ~(int64_t)3;
    const int64_t per4 = (per + 3) & ~(int64_t)3;
    const int cap = (int)(per4 < cap_max ? (per4 > 0 ? per4 : 4) : cap_max);
    const size_t dyn = (size_t)cap * kWords * sizeof(float);
    if (kCtrlBytes + 2 * (size_t)grid * kSlots * sizeof(float) > ws_bytes) return UPSLAM_ERR_CAPACITY;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTileThreads, dyn) != cudaSuccess ||
        per_sm < 1)
        return UPSLAM_ERR_UNSUPPORTED;
    IcpCtrl *ctrl = reinterpret_cast<IcpCtrl *>(ws);
    float *partials = reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + kCtrlBytes);
    IcpArgs ac = a;
    upslam_icp_params ipc = *ip;
    int capc = cap;
    PriorArgs prc = pr;
    FuseView fzc;
    int fuse_on = 0;
    if (fz) {
        fzc = *fz;
        fuse_on = 1;
    } else {
        memset(&fzc, 0, sizeof(fzc));
    }
    FrontArgs frc;
    if (front) {
        frc = *front;
    } else {
        memset(&frc, 0, sizeof(frc));
    }
    void *args[] = {&ac, &pose, &ipc, &st, &ctrl, &partials, &capc, &prc, &fzc, &fuse_on, &frc};
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTileThreads), args, dyn, stream) !=
        cudaSuccess) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    return UPSLAM_OK;
}

}  // namespace upslam

using namespace upslam;

extern "C" size_t upslam_icp_workspace_bytes(const upslam_keyframe *kf) {
    (void)kf;
    return kCtrlBytes + 2 * (size_t)max_ctas() * kSlots * sizeof(float);
}

static upslam_status icp_common_checks(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                       const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                       size_t ws_bytes) {
    if (!views_ok(kf, sw) || !d_pose12 || !ip || !d_stats || !d_ws) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_aligned(d_ws, 256) || ws_bytes < upslam_icp_workspace_bytes(kf)) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_icp_params_ok(ip)) return UPSLAM_ERR_INVALID_ARG;
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
    if (a.l1)
        icp_step_kernel<1><<<grid, kIcpThreads, 0, (cudaStream_t)stream>>>(a, d_pose12, *ip, d_stats, ctrl, partials);
    else
        icp_step_kernel<0><<<grid, kIcpThreads, 0, (cudaStream_t)stream>>>(a, d_pose12, *ip, d_stats, ctrl, partials);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_icp(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                    const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                    size_t ws_bytes, void *stream) {
    const upslam_status chk = icp_common_checks(kf, sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    if (ip->max_iters == 0) return UPSLAM_OK;
    return launch_tile(make_args(kf, sw, ip), d_pose12, ip, d_stats, d_ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" upslam_status upslam_icp_wait_probe(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_pose12,
                                               const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                               size_t ws_bytes, long long wait_cycles, void *stream) {
    const upslam_status chk = icp_common_checks(kf, sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    if (ip->max_iters < 1 || wait_cycles < 1000 || wait_cycles > kWaitCycles) return UPSLAM_ERR_INVALID_ARG;
    IcpArgs a = make_args(kf, sw, ip);
    a.wait_cycles = wait_cycles;
    a.withhold = 1;
    return launch_tile(a, d_pose12, ip, d_stats, d_ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" upslam_status upslam_register(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_prev,
                                         double *d_motion, double *d_pose12, int32_t prior,
                                         const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                         size_t ws_bytes, void *stream) {
    const upslam_status chk = icp_common_checks(kf, sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    if (prior < 0 || prior > 2 || (prior >= 1 && !d_prev) || (prior == 2 && !d_motion)) return UPSLAM_ERR_INVALID_ARG;
    if (ip->max_iters == 0) return UPSLAM_OK;
    PriorArgs pr;
    pr.prev = d_prev;
    pr.motion = d_motion;
    pr.motion_out = prior >= 1 ? d_motion : nullptr;
    pr.prev_out = prior >= 1 ? d_prev : nullptr;
    pr.mode = prior;
    return launch_tile(make_args(kf, sw, ip), d_pose12, ip, d_stats, d_ws, ws_bytes, (cudaStream_t)stream, pr);
}

bool upslam_fuse_view(const upslam_keyframe *kf, const upslam_sweep *sw, const upslam_fuse_params *fp,
                      uint64_t *d_zbuf_kf, FuseView &f);

extern "C" upslam_status upslam_track(const upslam_keyframe *kf, const upslam_sweep *sw, double *d_prev,
                                      double *d_motion, double *d_pose12, int32_t prior,
                                      const upslam_icp_params *ip, const upslam_fuse_params *fp,
                                      upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes, uint64_t *d_zbuf_kf,
                                      void *stream) {
    const upslam_status chk = icp_common_checks(kf, sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    if (prior < 0 || prior > 2 || (prior >= 1 && !d_prev) || (prior == 2 && !d_motion)) return UPSLAM_ERR_INVALID_ARG;
    FuseView f;
    if (!upslam_fuse_view(kf, sw, fp, d_zbuf_kf, f)) return UPSLAM_ERR_INVALID_ARG;
    if (ip->max_iters < 1) return UPSLAM_ERR_INVALID_ARG;
    PriorArgs pr;
    pr.prev = d_prev;
    pr.motion = d_motion;
    pr.motion_out = prior >= 1 ? d_motion : nullptr;
    pr.prev_out = prior >= 1 ? d_prev : nullptr;
    pr.mode = prior;
    return launch_tile(make_args(kf, sw, ip), d_pose12, ip, d_stats, d_ws, ws_bytes, (cudaStream_t)stream, pr, &f);
}

extern "C" upslam_status upslam_track_scan(const upslam_keyframe *kf, const float *d_pts4, int32_t n_pts,
                                           const upslam_sweep_buffers *sb, const upslam_normal_params *np,
                                           double *d_prev, double *d_motion, double *d_pose12, int32_t prior,
                                           const upslam_icp_params *ip, const upslam_fuse_params *fp,
                                           upslam_icp_stats *d_stats, void *d_ws, size_t ws_bytes,
                                           uint64_t *d_zbuf_kf, void *stream) {
    if (!sb || !np || n_pts < 0 || (n_pts > 0 && !d_pts4) || !sb->d_zbuf || !sb->d_depth || !sb->d_idx ||
        !sb->d_pix || !sb->d_nrm)
        return UPSLAM_ERR_INVALID_ARG;
    if ((d_pts4 && !upslam_aligned(d_pts4, 16)) || !upslam_aligned(sb->d_zbuf, 8) || !upslam_aligned(sb->d_pix, 16))
        return UPSLAM_ERR_INVALID_ARG;
    upslam_sweep sw;
    sw.pano = sb->pano;
    sw.d_pix = sb->d_pix;
    sw.d_nrm = sb->d_nrm;
    sw.nrm_precision = sb->nrm_precision;
    const upslam_status chk = icp_common_checks(kf, &sw, d_pose12, ip, d_stats, d_ws, ws_bytes);
    if (chk != UPSLAM_OK) return chk;
    if (prior < 0 || prior > 2 || (prior >= 1 && !d_prev) || (prior == 2 && !d_motion)) return UPSLAM_ERR_INVALID_ARG;
    FuseView f;
    if (!upslam_fuse_view(kf, &sw, fp, d_zbuf_kf, f)) return UPSLAM_ERR_INVALID_ARG;
    if (ip->max_iters < 1) return UPSLAM_ERR_INVALID_ARG;
    PriorArgs pr;
    pr.prev = d_prev;
    pr.motion = d_motion;
    pr.motion_out = prior >= 1 ? d_motion : nullptr;
    pr.prev_out = prior >= 1 ? d_prev : nullptr;
    pr.mode = prior;
    FrontArgs fr;
    fr.pts = reinterpret_cast<const float4 *>(d_pts4);
    fr.n = n_pts;
    fr.zbuf = reinterpret_cast<unsigned long long *>(sb->d_zbuf);
    fr.depth = sb->d_depth;
    fr.idx = sb->d_idx;
    fr.pix = reinterpret_cast<float4 *>(sb->d_pix);
    fr.nrm = sb->d_nrm;
    fr.nrm_prec = sb->nrm_precision;
    fr.np = *np;
    fr.on = 1;
    return launch_tile(make_args(kf, &sw, ip), d_pose12, ip, d_stats, d_ws, ws_bytes, (cudaStream_t)stream, pr, &f,
                       &fr);
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

// A launch needs the control block plus two 64-float records per CTA (one CTA per SM), so the
// array's record count fixes the largest device it serves: 2048 records = 1024 CTAs, and
// 36864 + 2048 * 64 * 4 = 561152 bytes (548 KiB).
constexpr int kNoAllocMaxRecords = 2048;
constexpr int kNoAllocMaxCtas = kNoAllocMaxRecords / 2;
constexpr size_t kNoAllocBytes = kCtrlBytes + (size_t)kNoAllocMaxRecords * kSlots * sizeof(float);
static_assert(kNoAllocBytes == 561152, "the documented capacity of the allocation-free scratch");
static_assert(kCtrlBytes + 2 * (size_t)kNoAllocMaxCtas * kSlots * sizeof(float) <= kNoAllocBytes,
              "the largest accepted grid fits the array");

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
    if (!upslam_icp_params_ok(ip)) return UPSLAM_ERR_INVALID_ARG;
    if (ip->max_iters == 0) return UPSLAM_OK;
    // the scratch a launch on this device needs (two records per SM) must fit the fixed array
    if (upslam_sm_count() > kNoAllocMaxCtas) return UPSLAM_ERR_CAPACITY;
    void *ws = nullptr;
    const upslam_status st = noalloc_scratch(&ws);
    if (st != UPSLAM_OK) return st;
    // the barrier counters must start at zero; the per-CTA sums are written before they are read
    if (cudaMemsetAsync(ws, 0, kCtrlBytes, (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    return launch_tile(make_args(kf, sw, ip), d_pose12, ip, d_stats, ws, kNoAllocBytes, (cudaStream_t)stream);
}
