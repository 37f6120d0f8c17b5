// Keyframe mutual consistency check (UPSLAM Sec. III-C: whenever it switches
// keyframes, a mutual consistency check between keyframes filters moving
// objects from the map).
//
// A sample of keyframe A is flagged when keyframe B saw through it: the sample
// s = d dir (FP32 table point) is taken into B's frame by T_ab^-1 (T_ab = pose of
// B in A, rounded to FP32) and binned into B with the FP32 rule (pixel j, range
// r); B must hold a depth at j, and every depth-holding pixel of the 3 x 3
// neighbourhood of j (columns wrapped, rows clipped) must lie beyond
// lim = (rel * r + abs) + r (FP32, round-to-nearest, this order).  B's samples
// are checked against A the same way with T_ba = T_ab^-1, formed in FP64 in the
// fixed order R' = R^T, t'_i = -((R_0i t_0 + R_1i t_1) + R_2i t_2).  Every
// decision is FP32 with the same operations as any checker, so the flags are
// exact.
//
// Launches: consistency_flags_kernel (CTAs [0, ga) check A, the rest check B,
// both against the unmodified depths) writes one flag byte per pixel;
// consistency_apply_kernel then empties the flagged pixels (depth 0, normal and
// count 0) and counts them.
//
// Roofline: per sample the source depth (4 B) is streamed, the flag written
// (1 B) and up to 9 depths of the other keyframe gathered (mostly L1/L2 hits);
// the apply pass reads the flags and writes 4 + 16 (or 8) B per flagged pixel.
#include "common.cuh"

namespace upslam {

struct ConsSide {
    upslam_pano pp;
    float *depth;
    void *nw;
    int prec;
    const float *dirs;
};

// The CTA's FP32 pose: T (forward) or its fixed-order inverse.
__device__ __forceinline__ PoseF cta_pose_or_inverse(const double *T, bool inverse) {
    __shared__ float ps[12];
    __syncthreads();
    if (threadIdx.x < 12) {
        const int i = threadIdx.x / 4, j = threadIdx.x % 4;
        double v;
        if (!inverse) {
            v = T[threadIdx.x];
        } else if (j < 3) {
            v = T[4 * j + i];
        } else {
            v = -__dadd_rn(__dadd_rn(__dmul_rn(T[i], T[3]), __dmul_rn(T[4 + i], T[7])), __dmul_rn(T[8 + i], T[11]));
        }
        ps[threadIdx.x] = (float)v;
    }
    __syncthreads();
    PoseF p;
#pragma unroll
    for (int i = 0; i < 12; ++i) p.r[i] = ps[i];
    return p;
}

__device__ __forceinline__ bool seen_through(const ConsSide &src, const ConsSide &dst, const PoseF &T, int k,
                                             float rel, float abs_m) {
    const float d = __ldg(src.depth + k);
    if (!(d > 0.0f)) return false;
    const int W = src.pp.cols;
    const int v = k / W;
    const float3 s = pixel_point(src.dirs, src.pp.rows, v, k - v * W, d);
    const float3 q = xform_inv(T, s.x, s.y, s.z);
    int jv, ju;
    float r;
    if (!bin_point(q.x, q.y, q.z, dst.pp, jv, ju, r)) return false;
    const int Wd = dst.pp.cols;
    if (!(__ldg(dst.depth + jv * Wd + ju) > 0.0f)) return false;
    const float lim = __fadd_rn(__fadd_rn(__fmul_rn(rel, r), abs_m), r);
#pragma unroll
    for (int dv = -1; dv <= 1; ++dv) {
        const int vv = jv + dv;
        if (vv < 0 || vv >= dst.pp.rows) continue;
#pragma unroll
        for (int du = -1; du <= 1; ++du) {
            int uu = ju + du;
            uu = uu < 0 ? uu + Wd : (uu >= Wd ? uu - Wd : uu);
            const float dn = __ldg(dst.depth + vv * Wd + uu);
            if (dn > 0.0f && !(dn > lim)) return false;
        }
    }
    return true;
}

__global__ void __launch_bounds__(256) consistency_flags_kernel(ConsSide a, ConsSide b, const double *T_ab, float rel,
                                                                float abs_m, unsigned char *flags_a,
                                                                unsigned char *flags_b, int ga) {
    pdl_release();  // the removal launch may place its CTAs while this grid drains
    const bool side_a = (int)blockIdx.x < ga;
    const PoseF T = cta_pose_or_inverse(T_ab, !side_a);
    const ConsSide &src = side_a ? a : b;
    const ConsSide &dst = side_a ? b : a;
    unsigned char *flags = side_a ? flags_a : flags_b;
    const int g0 = side_a ? 0 : ga, gn = side_a ? ga : (int)gridDim.x - ga;
    const int npx = src.pp.rows * src.pp.cols;
    for (int k = ((int)blockIdx.x - g0) * blockDim.x + threadIdx.x; k < npx; k += gn * blockDim.x)
        flags[k] = seen_through(src, dst, T, k, rel, abs_m) ? 1 : 0;
}

__global__ void __launch_bounds__(256) consistency_apply_kernel(ConsSide a, ConsSide b, const unsigned char *flags_a,
                                                                const unsigned char *flags_b, int ga,
                                                                unsigned long long *removed) {
    pdl_wait();  // every flag is written
    const bool side_a = (int)blockIdx.x < ga;
    const ConsSide &src = side_a ? a : b;
    const unsigned char *flags = side_a ? flags_a : flags_b;
    const int g0 = side_a ? 0 : ga, gn = side_a ? ga : (int)gridDim.x - ga;
    const int npx = src.pp.rows * src.pp.cols;
    unsigned n = 0;
    for (int k = ((int)blockIdx.x - g0) * blockDim.x + threadIdx.x; k < npx; k += gn * blockDim.x) {
        if (!flags[k]) continue;
        src.depth[k] = 0.0f;
        store_nw(src.nw, k, src.prec, make_float4(0.f, 0.f, 0.f, 0.f));
        ++n;
    }
    n = __reduce_add_sync(0xffffffffu, n);
    if (removed && (threadIdx.x & 31) == 0 && n) atomicAdd(removed + (side_a ? 0 : 1), (unsigned long long)n);
}

static bool side_ok(const upslam_keyframe *kf) {
    return kf && upslam_pano_ok(&kf->pano) && kf->d_depth && kf->d_nw && kf->d_dirs &&
           (kf->precision == UPSLAM_F32 || kf->precision == UPSLAM_F16) &&
           upslam_aligned(kf->d_nw, kf->precision == UPSLAM_F32 ? 16 : 8) && upslam_aligned(kf->d_dirs, 8);
}

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace upslam

using namespace upslam;

extern "C" size_t upslam_consistency_workspace_bytes(const upslam_keyframe *kf_a, const upslam_keyframe *kf_b) {
    if (!kf_a || !kf_b || !upslam_pano_ok(&kf_a->pano) || !upslam_pano_ok(&kf_b->pano)) return 0;
    return align256((size_t)kf_a->pano.rows * kf_a->pano.cols) + align256((size_t)kf_b->pano.rows * kf_b->pano.cols);
}

extern "C" upslam_status upslam_keyframe_consistency(const upslam_keyframe *kf_a, const upslam_keyframe *kf_b,
                                                     const double *d_T_ab12, float rel, float abs_m, void *d_ws,
                                                     size_t ws_bytes, int64_t *d_removed2, void *stream) {
    if (!side_ok(kf_a) || !side_ok(kf_b) || !d_T_ab12 || !d_ws || !upslam_aligned(d_ws, 256)) return UPSLAM_ERR_INVALID_ARG;
    if (kf_a->d_depth == kf_b->d_depth || kf_a->d_nw == kf_b->d_nw) return UPSLAM_ERR_INVALID_ARG;
    if (!(rel >= 0.0f) || !(abs_m >= 0.0f) || ws_bytes < upslam_consistency_workspace_bytes(kf_a, kf_b))
        return UPSLAM_ERR_INVALID_ARG;
    if (d_removed2 && !upslam_aligned(d_removed2, 8)) return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ConsSide a{kf_a->pano, kf_a->d_depth, kf_a->d_nw, kf_a->precision, kf_a->d_dirs};
    ConsSide b{kf_b->pano, kf_b->d_depth, kf_b->d_nw, kf_b->precision, kf_b->d_dirs};
    unsigned char *flags_a = reinterpret_cast<unsigned char *>(d_ws);
    unsigned char *flags_b = flags_a + align256((size_t)kf_a->pano.rows * kf_a->pano.cols);
    const int64_t na = (int64_t)kf_a->pano.rows * kf_a->pano.cols, nb = (int64_t)kf_b->pano.rows * kf_b->pano.cols;
    const int ga = upslam_grid(na, 256, 4), gb = upslam_grid(nb, 256, 4);
    if (d_removed2 && cudaMemsetAsync(d_removed2, 0, 2 * sizeof(int64_t), s) != cudaSuccess) return UPSLAM_ERR_CUDA;
    consistency_flags_kernel<<<ga + gb, 256, 0, s>>>(a, b, d_T_ab12, rel, abs_m, flags_a, flags_b, ga);
    UPSLAM_CHECK_LAUNCH();
    if (!launch_dependent(consistency_apply_kernel, dim3(ga + gb), dim3(256), 0, s, a, b,
                          (const unsigned char *)flags_a, (const unsigned char *)flags_b, ga,
                          reinterpret_cast<unsigned long long *>(d_removed2)))
        return UPSLAM_ERR_CUDA;
    return UPSLAM_OK;
}
