// Batched persistent ICP: many registration problems in one cooperative launch.
//
// A batch is one sweep registered against n_kf keyframes of mixed sizes, with
// n_hyp initial-pose hypotheses per keyframe (problem p = kf * n_hyp + h).  The
// paper evaluates several hundred candidate transforms when it searches for a
// loop closure (Sec. III-C, grid search); here every candidate is a full
// Gauss-Newton ICP problem (Sec. III-B, Eq. 1), all advancing in lockstep.
//
// Prologue (once): every CTA takes the keyframe chunks q = blockIdx, +grid, ...
// of each keyframe and compacts the pixels holding a sample into its own
// entry lists in the workspace (FP32 point d*dir and normal, structure of
// arrays), so later steps touch samples only.
//
// Each step:
//  1. every active problem (keyframe kf, hypothesis h) is one work item: one warp
//     evaluates all of this CTA's staged samples of kf under h, keeps the sums
//     in registers, reduces them once across the warp and stores them to the
//     problem's accumulator in shared memory (no two warps add into one
//     accumulator, so the result does not depend on timing);
//  2. every CTA writes one record (29 sums) per problem; grid barrier;
//  3. problem p is owned by CTA p mod grid: its warps sum the records of p in
//     a fixed order (compensated FP32), and the CTA's warps then solve up to
//     one owned problem each, side by side, in FP64 (L D L^T, SE(3) exp) and
//     write the pose, the record and the active flag; grid barrier;
//  4. every CTA reloads the poses and flags of the active problems.
// The launch ends when no problem is active or after max_iters steps.
// Grid barriers are a monotonic 64-bit arrival counter with a clock64 budget.
#include <string.h>

#include "common.cuh"

namespace upslam {

constexpr int kBatchMaxProblems = 1024;
constexpr int kBatchMaxKf = 256;
constexpr long long kBatchWaitCycles = 8000000000ll;  // about 4 s at 2 GHz
constexpr int kRecWords = 32;

struct BatchCtrl {
    unsigned long long arrive;
    int valid;  // sweep pixels holding a point
    int pad;
};

struct BatchArgs {
    const upslam_keyframe *kfs;  // device array [n_kf]
    int n_kf, n_hyp, n_prob;
    upslam_pano sp;
    const float4 *spix;
    const void *snrm;
    int sprec;
    float d_max2, cos_min;
    float d_max2_fine;        // the gate from step ip.coarse_iters on (when ip.coarse_iters > 0)
    int l1;                   // 1: absolute error by IRLS, weights 1 / max(|r|, loss_delta)
    float loss_delta;
    double *poses;            // [n_prob][12] in/out
    upslam_icp_stats *stats;  // [n_prob]
    int *active;              // [n_prob] workspace flags
    float *poses_f;           // [n_prob][12] FP32 copies written by each problem's owner
    float *entries;           // per keyframe, its samples as [6][rows*cols] floats (structure of arrays)
    int *counts;              // [n_kf][grid] samples each CTA found in its chunks of each keyframe
    float *records;           // [n_prob][grid][kRecWords]
    BatchCtrl *ctrl;
    upslam_icp_params ip;
    int chunk;  // pixels per chunk (a multiple of blockDim)
};

__device__ __forceinline__ bool grid_wait(BatchCtrl *ctrl, unsigned long long target) {
    const long long t0 = clock64();
    while (*((volatile unsigned long long *)&ctrl->arrive) < target) {
        if (clock64() - t0 > kBatchWaitCycles) return false;
        __nanosleep(32);
    }
    return true;
}

// A staged keyframe sample's correspondence: the sweep pixel it bins into under the hypothesis,
// that pixel's point and normal (gathered from L2), and whether it binned at all.
struct BatchHit {
    float4 P, m;
    bool binned;
};

__device__ __forceinline__ BatchHit batch_gather(const BatchArgs &a, const float *ent, int cap, const PoseF &Tp, int q,
                                                 float3 &s, float3 &n) {
    s = make_float3(ent[q], ent[cap + q], ent[2 * cap + q]);
    n = make_float3(ent[3 * cap + q], ent[4 * cap + q], ent[5 * cap + q]);
    const float3 qq = xform_inv(Tp, s.x, s.y, s.z);
    int jv = 0, ju = 0;
    float rr;
    BatchHit h;
    h.binned = bin_point(qq.x, qq.y, qq.z, a.sp, jv, ju, rr);
    const int j = h.binned ? jv * a.sp.cols + ju : 0;
    h.P = __ldg(a.spix + j);
    h.m = load_nw(a.snrm, j, a.sprec);
    return h;
}

// One correspondence of Eq. 1 under the problem's pose, branch-free (a rejected pair adds zeros):
// Omega with the step's squared distance gate, r = (T s2 - s1) . n, J = [p x n, n], IRLS weight.
__device__ __forceinline__ void batch_accumulate(const BatchArgs &a, const PoseF &Tp, float gate2, float3 s, float3 n,
                                                 const BatchHit &h, float acc[28], int &inl) {
    const float4 P = h.P, m = h.m;
    bool ok = h.binned && P.w != 0.0f && m.w != 0.0f;
    const float *r = Tp.r;
    const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
    const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
    const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
    const float3 Rm = rotate(Tp, m.x, m.y, m.z);
    const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
    ok = ok && (ex * ex + ey * ey + ez * ez <= gate2) && (Rm.x * n.x + Rm.y * n.y + Rm.z * n.z >= a.cos_min);
    const float r0 = ex * n.x + ey * n.y + ez * n.z;
    // square root of the IRLS weight (1 for the squared error); 0 for an outlier
    const float w = ok ? (a.l1 ? rsqrtf(fmaxf(fabsf(r0), a.loss_delta)) : 1.0f) : 0.0f;
    const float res = r0 * w;
    float J[6];
    J[0] = (py * n.z - pz * n.y) * w;
    J[1] = (pz * n.x - px * n.z) * w;
    J[2] = (px * n.y - py * n.x) * w;
    J[3] = n.x * w;
    J[4] = n.y * w;
    J[5] = n.z * w;
    int c = 0;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int k2 = i; k2 < 6; ++k2) {
            acc[c] = fmaf(J[i], J[k2], acc[c]);
            ++c;
        }
#pragma unroll
    for (int i = 0; i < 6; ++i) acc[21 + i] = fmaf(J[i], res, acc[21 + i]);
    acc[27] = fmaf(res, res, acc[27]);
    inl += ok ? 1 : 0;
}

constexpr int kPx = 8;  // keyframe pixels per thread in flight in the prologue

// Keyframe pixel k as a sample: it holds one when its depth is positive and its normal unit (the test of the
// single-problem launch); the normal is read only where the depth holds a sample.
__device__ __forceinline__ bool kf_sample(const upslam_keyframe &K, int k, float d, float4 &n4) {
    n4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!(d > 0.0f)) return false;
    n4 = load_nw(K.d_nw, k, K.precision);
    return __fadd_rn(__fadd_rn(__fmul_rn(n4.x, n4.x), __fmul_rn(n4.y, n4.y)), __fmul_rn(n4.z, n4.z)) > 0.25f;
}

__global__ void __launch_bounds__(512, 1) icp_batched_kernel(BatchArgs a) {
    extern __shared__ float smem[];
    float *acc = smem;                                 // [n_prob][kRecWords]
    float *pose_f = acc + a.n_prob * kRecWords;        // [n_prob][12]
    int *act = reinterpret_cast<int *>(pose_f + a.n_prob * 12);  // [n_prob]
    __shared__ long long kf_base[kBatchMaxKf];              // float offset of a keyframe's sample arrays
    __shared__ int kf_cap[kBatchMaxKf];                      // its pixels: the length of each array
    __shared__ int kf_lo[kBatchMaxKf], kf_hi[kBatchMaxKf];   // this CTA's slice of its samples
    __shared__ int kf_wb[kBatchMaxKf];                       // where this CTA's own samples go
    __shared__ int wcnt[32];
    __shared__ int pcnt[2][kPx][16];
    __shared__ int flag_s, any_active;
    __shared__ double totq[16][32];   // step sums of the problems being solved, one per warp
    __shared__ double Tsh[16][12];    // their poses
    __shared__ int pown[16];
    __shared__ float shs[16][32], shc[16][32];
    __shared__ float wpart[16][32];   // per-warp totals when warps share a problem
    const int T = blockDim.x, nw = T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned long long G = gridDim.x;
    unsigned long long base = 0;
    if (threadIdx.x == 0) {
        base = (*((volatile unsigned long long *)&a.ctrl->arrive) / G) * G;
        flag_s = 0;
    }
    // ---- prologue, once per launch: the keyframe samples.  Keyframe chunks are dealt to CTAs round-robin,
    // the deal rotated from one keyframe to the next (the samples sit in a band of rows: without the
    // rotation the same CTAs would take one chunk more of every keyframe of a size).
    //  (1) every CTA counts the samples in its chunks of each keyframe;
    //  (2) after a grid barrier, it writes them to the keyframe's sample arrays behind those of the CTAs
    //      before it, in pixel order, so the arrays are the same on every launch;
    //  (3) after a second barrier, each CTA takes an equal slice of every keyframe's samples for the steps.
    // A thread keeps kPx pixels in flight, and reads a normal only where the depth holds a sample.
    if (threadIdx.x == 0) {
        long long o = 0;
        for (int kf = 0; kf < a.n_kf; ++kf) {
            const int npx = a.kfs[kf].pano.rows * a.kfs[kf].pano.cols;
            kf_base[kf] = o;
            kf_cap[kf] = npx;
            o += 6ll * npx;
        }
    }
    __syncthreads();
    for (int pass = 0; pass < 2 && !flag_s; ++pass) {
        for (int kf = 0; kf < a.n_kf; ++kf) {
            const upslam_keyframe K = a.kfs[kf];
            const int npx = kf_cap[kf], W = K.pano.cols;
            const int nch = (npx + a.chunk - 1) / a.chunk;
            const int rot = (int)(((long long)kf * 61) % gridDim.x);
            const int c0 = ((int)blockIdx.x - rot + (int)gridDim.x) % (int)gridDim.x;
            float *E = a.entries + kf_base[kf];
            // this CTA's pixels as blocks of T: chunk c0 + m * grid holds blocks m * bpc .. m * bpc + bpc - 1,
            // taken kPx blocks at a time in that order
            const int bpc = a.chunk / T;
            const int nmine = c0 < nch ? ((nch - 1 - c0) / (int)gridDim.x + 1) * bpc : 0;
            int mine = 0, run = pass == 1 ? kf_wb[kf] : 0, par = 0;
            for (int b0 = 0; b0 < nmine; b0 += kPx, par ^= 1) {
                {
                    float d[kPx];
                    float4 n4[kPx];
                    bool ok[kPx];
                    int kk[kPx];
#pragma unroll
                    for (int i = 0; i < kPx; ++i) {
                        const int b = b0 + i;
                        kk[i] = -1;
                        if (b < nmine) {
                            const int k = (c0 + (b / bpc) * (int)gridDim.x) * a.chunk + (b % bpc) * T + threadIdx.x;
                            kk[i] = k < npx ? k : -1;
                        }
                        d[i] = kk[i] >= 0 ? __ldg(K.d_depth + kk[i]) : 0.0f;
                    }
#pragma unroll
                    for (int i = 0; i < kPx; ++i) ok[i] = kf_sample(K, kk[i], d[i], n4[i]);
                    if (pass == 0) {
#pragma unroll
                        for (int i = 0; i < kPx; ++i) mine += ok[i] ? 1 : 0;
                        continue;
                    }
                    // positions in pixel order: ballots per pixel slot, counts per warp, double-buffered
                    unsigned bal[kPx];
#pragma unroll
                    for (int i = 0; i < kPx; ++i) {
                        bal[i] = __ballot_sync(0xffffffffu, ok[i]);
                        if (lane == 0) pcnt[par][i][warp] = __popc(bal[i]);
                    }
                    __syncthreads();
                    int o = run;
#pragma unroll
                    for (int i = 0; i < kPx; ++i) {
                        int before = 0, tot = 0;
                        for (int w = 0; w < nw; ++w) {
                            const int cw = pcnt[par][i][w];
                            before += w < warp ? cw : 0;
                            tot += cw;
                        }
                        if (ok[i]) {
                            const int slot = o + before + __popc(bal[i] & ((1u << lane) - 1u));
                            const int k = kk[i];
                            const int v = k / W;
                            const float3 sp = pixel_point(K.d_dirs, K.pano.rows, v, k - v * W, d[i]);
                            E[slot] = sp.x;
                            E[npx + slot] = sp.y;
                            E[2 * npx + slot] = sp.z;
                            E[3 * npx + slot] = n4[i].x;
                            E[4 * npx + slot] = n4[i].y;
                            E[5 * npx + slot] = n4[i].z;
                        }
                        o += tot;
                    }
                    run = o;
                }
            }
            if (pass == 0) {
                mine = __reduce_add_sync(0xffffffffu, mine);
                if (lane == 0) wcnt[warp] = mine;
                __syncthreads();
                if (threadIdx.x == 0) {
                    int t = 0;
                    for (int w = 0; w < nw; ++w) t += wcnt[w];
                    a.counts[(size_t)kf * gridDim.x + blockIdx.x] = t;
                }
                __syncthreads();
            }
        }
        // grid barrier: the counts (after pass 0), the sample arrays (after pass 1)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.ctrl->arrive, 1ull);
            flag_s = grid_wait(a.ctrl, base + G * (unsigned long long)(pass + 1)) ? 0 : 1;
            __threadfence();
        }
        __syncthreads();
        if (pass == 0 && !flag_s) {
            // where this CTA's samples go, and its slice of each keyframe's samples
            for (int kf = threadIdx.x; kf < a.n_kf; kf += T) {
                const int *ck = a.counts + (size_t)kf * gridDim.x;
                int before = 0, tot = 0;
                for (int c = 0; c < (int)gridDim.x; ++c) {
                    const int v = __ldcg(ck + c);
                    before += c < (int)blockIdx.x ? v : 0;
                    tot += v;
                }
                kf_wb[kf] = before;
                kf_lo[kf] = (int)((long long)tot * blockIdx.x / gridDim.x);
                kf_hi[kf] = (int)((long long)tot * (blockIdx.x + 1) / gridDim.x);
            }
            __syncthreads();
        }
    }
    // sweep pixels holding a point (for the registration quality)
    {
        int c = 0;
        const int ns = a.sp.rows * a.sp.cols;
        for (int j = blockIdx.x * T + threadIdx.x; j < ns; j += gridDim.x * T) c += __ldg(&a.spix[j].w) != 0.0f;
        c = __reduce_add_sync(0xffffffffu, c);
        if (lane == 0 && c) atomicAdd(&a.ctrl->valid, c);
    }
    for (int p = threadIdx.x; p < a.n_prob; p += T) {
        act[p] = 1;
        for (int i = 0; i < 12; ++i) pose_f[p * 12 + i] = (float)__ldcg(a.poses + (size_t)p * 12 + i);
    }
    __syncthreads();

    int it = 0;
    for (; it < a.ip.max_iters && !flag_s; ++it) {
        // this step's Omega distance gate (coarse-to-fine when coarse_iters > 0)
        const float gate2 = (a.ip.coarse_iters > 0 && it >= a.ip.coarse_iters) ? a.d_max2_fine : a.d_max2;
        for (int i = threadIdx.x; i < a.n_prob * kRecWords; i += T) acc[i] = 0.0f;
        __syncthreads();
        // ---- 1. accumulate.  A work item is one problem p = (keyframe kf, hypothesis h) over every
        // sample this CTA staged for kf.  One warp takes an item (items dealt round-robin to the
        // warps), keeps the 28 sums and the inlier count per lane in registers, reduces them once
        // (reduce-scatter) and stores the totals to p's accumulator.  No two warps add into one
        // accumulator, so the sums do not depend on timing.  With fewer problems than warps, `split`
        // warps share a problem (each takes every split-th group of 32 samples) and their totals are
        // added in warp order.  Each lane bins and gathers its next sample before it reduces the
        // current one, so the L2 round trips overlap the arithmetic.
        const int split = a.n_prob < nw ? nw / a.n_prob : 1;
        for (int item = warp; item < a.n_prob * split; item += nw) {
            const int p = item / split, part = item - p * split;
            if (!act[p]) continue;
            const int kf = p / a.n_hyp;
            const int lo = kf_lo[kf], hi = kf_hi[kf], capk = kf_cap[kf];
            const float *E = a.entries + kf_base[kf];
            PoseF Tp;
#pragma unroll
            for (int i = 0; i < 12; ++i) Tp.r[i] = pose_f[p * 12 + i];
            float accr[28];
#pragma unroll
            for (int i = 0; i < 28; ++i) accr[i] = 0.0f;
            int inl = 0;
            const int stride = 32 * split;
            int e = lo + part * 32 + lane;
            if (e < hi) {
                float3 sc, nc;
                BatchHit hc = batch_gather(a, E, capk, Tp, e, sc, nc);
                for (; e < hi; e += stride) {
                    float3 sn = sc, nn = nc;
                    BatchHit hn = hc;
                    if (e + stride < hi) hn = batch_gather(a, E, capk, Tp, e + stride, sn, nn);
                    batch_accumulate(a, Tp, gate2, sc, nc, hc, accr, inl);
                    sc = sn;
                    nc = nn;
                    hc = hn;
                }
            }
            float v[32];
#pragma unroll
            for (int i = 0; i < 28; ++i) v[i] = accr[i];
            v[28] = (float)inl;
            v[29] = v[30] = v[31] = 0.0f;
            const float sum = warp_reduce_scatter(v);
            if (lane < 29) {
                if (split == 1) acc[p * kRecWords + lane] = sum;
                else wpart[item][lane] = sum;  // items < nw here
            }
        }
        __syncthreads();
        if (split > 1) {
            for (int i = threadIdx.x; i < a.n_prob * 29; i += T) {
                const int p = i / 29, l = i - p * 29;
                if (!act[p]) continue;
                float t = 0.0f;
                for (int q = 0; q < split; ++q) t += wpart[p * split + q][l];
                acc[p * kRecWords + l] = t;
            }
        }
        __syncthreads();
        // ---- 2. publish this CTA's record of every active problem
        for (int i = threadIdx.x; i < a.n_prob * kRecWords; i += T) {
            const int p = i / kRecWords;
            if (act[p]) a.records[((size_t)p * gridDim.x + blockIdx.x) * kRecWords + (i % kRecWords)] = acc[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.ctrl->arrive, 1ull);
            flag_s = grid_wait(a.ctrl, base + G * (2ull * it + 3ull)) ? 0 : 1;
            __threadfence();
        }
        __syncthreads();
        if (flag_s) break;
        // ---- 3. the problems this CTA owns (p = blockIdx.x + j * grid), up to one per warp at a
        // time: all warps sum each problem's records over the CTAs in a fixed order (compensated
        // FP32), then the warps solve their problems side by side in FP64 and publish them.
        for (int p0 = blockIdx.x; p0 < a.n_prob; p0 += (int)gridDim.x * nw) {
            int n_own = 0;
            for (int j = 0; j < nw; ++j) {
                const int p = p0 + j * (int)gridDim.x;
                if (p >= a.n_prob) break;
                if (!act[p]) continue;
                float s = 0.0f, c = 0.0f;
                for (int b = warp; b < (int)gridDim.x; b += nw) {
                    const float x = __ldcg(a.records + ((size_t)p * gridDim.x + b) * kRecWords + lane);
                    kadd(s, c, x);
                }
                shs[warp][lane] = s;
                shc[warp][lane] = c;
                __syncthreads();
                if (threadIdx.x < 29) {
                    float t = 0.0f, cc = 0.0f;
                    for (int w = 0; w < nw; ++w) {
                        kadd(t, cc, shs[w][threadIdx.x]);
                        cc += shc[w][threadIdx.x];
                    }
                    totq[n_own][threadIdx.x] = (double)t + (double)cc;
                }
                if (threadIdx.x < 12) Tsh[n_own][threadIdx.x] = __ldcg(a.poses + (size_t)p * 12 + threadIdx.x);
                if (threadIdx.x == 0) pown[n_own] = p;
                __syncthreads();
                ++n_own;
            }
            if (warp < n_own) {
                const int p = pown[warp];
                const double *tq = totq[warp];
                double *Tw = Tsh[warp];
                const long long inliers = (long long)(tq[28] + 0.5);
                double xi[6] = {0, 0, 0, 0, 0, 0};
                int status = UPSLAM_OK, conv = 0;
                if (inliers < a.ip.min_inliers) {
                    status = UPSLAM_ERR_DEGENERATE;
                } else if (!warp_solve6(tq, a.ip.pivot_eps, xi)) {
                    status = UPSLAM_ERR_DEGENERATE;
#pragma unroll
                    for (int i = 0; i < 6; ++i) xi[i] = 0.0;
                } else {
                    warp_se3_update(xi, Tw);
                    conv = warp_converged(xi, a.ip.eps_rot * a.ip.eps_rot, a.ip.eps_trans * a.ip.eps_trans) ? 1 : 0;
                }
                upslam_icp_stats *st = a.stats + p;
                if (lane < 12) {
                    a.poses[(size_t)p * 12 + lane] = Tw[lane];
                    a.poses_f[(size_t)p * 12 + lane] = (float)Tw[lane];
                }
                if (lane < 21) st->A[lane] = tq[lane];
                else if (lane < 27) st->b[lane - 21] = tq[lane];
                if (lane < 6) st->xi[lane] = xi[lane];
                if (lane == 0) {
                    st->sse = tq[27];
                    st->inliers = inliers;
                    st->valid = *((volatile int *)&a.ctrl->valid);
                    st->status = status;
                    st->converged = conv;
                    st->iters = it + 1;
                    st->accepted = 0;
                    a.active[p] = (status == UPSLAM_OK && !conv) ? 1 : 0;
                }
            }
            __syncthreads();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(&a.ctrl->arrive, 1ull);
            flag_s = grid_wait(a.ctrl, base + G * (2ull * it + 4ull)) ? 0 : 1;
            __threadfence();
            any_active = 0;
        }
        __syncthreads();
        if (flag_s) break;
        // ---- 4. reload poses and flags
        for (int p = threadIdx.x; p < a.n_prob; p += T) {
            if (!act[p]) continue;
            const int still = __ldcg(a.active + p);
            act[p] = still;
            if (still) {
                any_active = 1;
                // the owner's FP32 copy: no FP64 conversion here (slow on GB300)
                for (int i = 0; i < 12; ++i) pose_f[p * 12 + i] = __ldcg(a.poses_f + (size_t)p * 12 + i);
            }
        }
        __syncthreads();
        if (!any_active) break;
    }
    if (flag_s && threadIdx.x == 0) {
        for (int p = blockIdx.x; p < a.n_prob; p += gridDim.x) a.stats[p].status = UPSLAM_ERR_TIMEOUT;
    }
}

}  // namespace upslam

using namespace upslam;

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace: control block, active flags, FP32 poses, per-CTA records, the per-(keyframe, CTA) sample counts,
// then every keyframe's sample arrays (6 floats per pixel: the worst case of a keyframe full of samples).
static size_t batch_ws_layout(const upslam_keyframe *kfs, int32_t n_kf, int32_t n_prob, int grid,
                              size_t *off_active, size_t *off_records, size_t *off_counts, size_t *off_entries,
                              size_t *off_posef) {
    size_t o = 256;  // control block
    *off_active = o;
    o = align256(o + (size_t)n_prob * sizeof(int));
    *off_posef = o;
    o = align256(o + (size_t)n_prob * 12 * sizeof(float));
    *off_records = o;
    o = align256(o + (size_t)n_prob * grid * kRecWords * sizeof(float));
    *off_counts = o;
    o = align256(o + (size_t)n_kf * grid * sizeof(int));
    *off_entries = o;
    size_t px = 0;
    for (int i = 0; i < n_kf; ++i) px += (size_t)kfs[i].pano.rows * kfs[i].pano.cols;
    o = align256(o + 6 * px * sizeof(float));
    return o;
}

static int batch_chunk(const upslam_batch_tiles *tiles) { return tiles ? tiles->chunk : 512; }
static int batch_threads(const upslam_batch_tiles *tiles) { return tiles ? tiles->threads : 512; }

extern "C" size_t upslam_icp_batched_workspace_bytes(const upslam_keyframe *kfs, int32_t n_kf, int32_t n_hyp,
                                                     const upslam_batch_tiles *tiles) {
    if (!kfs || n_kf <= 0 || n_hyp <= 0) return 0;
    (void)tiles;
    size_t a, r, c, e, f;
    return batch_ws_layout(kfs, n_kf, n_kf * n_hyp, upslam_sm_count(), &a, &r, &c, &e, &f);
}

extern "C" upslam_status upslam_icp_batched(const upslam_keyframe *d_kfs, const upslam_keyframe *kfs, int32_t n_kf,
                                            const upslam_sweep *sw, int32_t n_hyp, double *d_poses,
                                            const upslam_icp_params *ip, upslam_icp_stats *d_stats, void *d_ws,
                                            size_t ws_bytes, const upslam_batch_tiles *tiles, void *stream) {
    if (!d_kfs || !kfs || n_kf <= 0 || n_kf > kBatchMaxKf || n_hyp <= 0 || !sw || !d_poses || !ip || !d_stats ||
        !d_ws)
        return UPSLAM_ERR_INVALID_ARG;
    const int n_prob = n_kf * n_hyp;
    if (n_prob > kBatchMaxProblems) return UPSLAM_ERR_CAPACITY;
    if (!upslam_pano_ok(&sw->pano) || !sw->d_pix || !sw->d_nrm || !upslam_aligned(sw->d_pix, 16) ||
        (sw->nrm_precision != UPSLAM_F32 && sw->nrm_precision != UPSLAM_F16))
        return UPSLAM_ERR_INVALID_ARG;
    for (int i = 0; i < n_kf; ++i) {
        const upslam_keyframe &K = kfs[i];
        if (!upslam_pano_ok(&K.pano) || !K.d_depth || !K.d_nw || !K.d_dirs ||
            (K.precision != UPSLAM_F32 && K.precision != UPSLAM_F16))
            return UPSLAM_ERR_INVALID_ARG;
    }
    const int threads = batch_threads(tiles), chunk = batch_chunk(tiles);
    if ((threads != 256 && threads != 512) || chunk < threads || chunk % threads) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_icp_params_ok(ip) || ip->max_iters < 1 || !upslam_aligned(d_ws, 256)) return UPSLAM_ERR_INVALID_ARG;
    int dev = 0, coop = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (!coop) return UPSLAM_ERR_UNSUPPORTED;
    const int grid = upslam_sm_count();
    size_t off_active, off_records, off_counts, off_entries, off_posef;
    const size_t need = batch_ws_layout(kfs, n_kf, n_prob, grid, &off_active, &off_records, &off_counts, &off_entries,
                                        &off_posef);
    if (ws_bytes < need) return UPSLAM_ERR_INVALID_ARG;
    const size_t dyn = (size_t)n_prob * (kRecWords + 12) * sizeof(float) + (size_t)n_prob * sizeof(int);
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, icp_batched_kernel) != cudaSuccess) return UPSLAM_ERR_CUDA;
    if ((int)(dyn + fa.sharedSizeBytes) > optin) return UPSLAM_ERR_CAPACITY;
    // raise the dynamic shared-memory limit once per device, so that a later call made while a
    // stream is being captured into a CUDA graph issues no attribute change
    static std::atomic<int> smem_raised[64];
    if (dev < 0 || dev >= 64) return UPSLAM_ERR_UNSUPPORTED;
    if (!smem_raised[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(icp_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes) != cudaSuccess)
            return UPSLAM_ERR_UNSUPPORTED;
        smem_raised[dev].store(1, std::memory_order_release);
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, icp_batched_kernel, threads, dyn) != cudaSuccess ||
        per_sm < 1)
        return UPSLAM_ERR_UNSUPPORTED;
    char *ws = reinterpret_cast<char *>(d_ws);
    // control block: valid counter must start at zero each call (arrivals are monotonic)
    if (cudaMemsetAsync(ws + offsetof(BatchCtrl, valid), 0, sizeof(int), (cudaStream_t)stream) != cudaSuccess)
        return UPSLAM_ERR_CUDA;
    BatchArgs a;
    a.kfs = d_kfs;
    a.n_kf = n_kf;
    a.n_hyp = n_hyp;
    a.n_prob = n_prob;
    a.sp = sw->pano;
    a.spix = reinterpret_cast<const float4 *>(sw->d_pix);
    a.snrm = sw->d_nrm;
    a.sprec = sw->nrm_precision;
    a.d_max2 = ip->d_max * ip->d_max;
    a.d_max2_fine = ip->d_max_fine * ip->d_max_fine;
    a.cos_min = ip->cos_theta_max;
    a.l1 = ip->loss == UPSLAM_LOSS_L1 ? 1 : 0;
    a.loss_delta = ip->loss_delta;
    a.poses = d_poses;
    a.stats = d_stats;
    a.active = reinterpret_cast<int *>(ws + off_active);
    a.poses_f = reinterpret_cast<float *>(ws + off_posef);
    a.entries = reinterpret_cast<float *>(ws + off_entries);
    a.counts = reinterpret_cast<int *>(ws + off_counts);
    a.records = reinterpret_cast<float *>(ws + off_records);
    a.ctrl = reinterpret_cast<BatchCtrl *>(ws);
    a.ip = *ip;
    a.chunk = chunk;
    void *args[] = {&a};
    if (cudaLaunchCooperativeKernel((const void *)icp_batched_kernel, dim3(grid), dim3(threads), args, dyn,
                                    (cudaStream_t)stream) != cudaSuccess) {
        (void)cudaGetLastError();
        return UPSLAM_ERR_CUDA;
    }
    return UPSLAM_OK;
}
