// Per-pixel normals (UPSLAM Sec. III-A): the cross product of the vectors from
// a pixel's point to two image neighbours.
//
// a points toward column + 1 (wrapping around the panorama), b toward row + 1.
// A neighbour is unusable when it holds no point or its range jumps by more
// than jump_rel * r + jump_abs (decided in FP32 with the same round-to-nearest
// operations as any checker); the opposite neighbour then replaces it with the
// vector's sign flipped.  The normal is normalised and oriented toward the
// sensor.  Roofline: streaming, 20 B read + 16 B (8 B in FP16) written per pixel;
// neighbour reads hit L1/L2.
#include "common.cuh"

namespace upslam {

__device__ __forceinline__ bool nb_ok(const float4 *pix, const float *depth, int k, int kn, float d,
                                      const upslam_normal_params &np) {
    if (__ldg(&pix[kn].w) == 0.0f) return false;
    const float dn = __ldg(depth + kn);
    const float jump = fabsf(__fsub_rn(dn, d));
    const float lim = __fadd_rn(__fmul_rn(np.jump_rel, d), np.jump_abs);
    return !(jump > lim);
}

__global__ void __launch_bounds__(256) normals_kernel(const float4 *__restrict__ pix, const float *__restrict__ depth,
                                                      upslam_pano pp, upslam_normal_params np, void *nrm,
                                                      int precision) {
    const int H = pp.rows, W = pp.cols, npx = H * W;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x) {
        const float4 c = __ldg(pix + k);
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c.w != 0.0f) {
            const int v = k / W, u = k - v * W;
            const float d = __ldg(depth + k);
            const int kr = v * W + (u + 1 == W ? 0 : u + 1);
            const int kl = v * W + (u == 0 ? W - 1 : u - 1);
            float3 a, b;
            bool ok = true;
            if (nb_ok(pix, depth, k, kr, d, np)) {
                const float4 q = __ldg(pix + kr);
                a = make_float3(q.x - c.x, q.y - c.y, q.z - c.z);
            } else if (nb_ok(pix, depth, k, kl, d, np)) {
                const float4 q = __ldg(pix + kl);
                a = make_float3(c.x - q.x, c.y - q.y, c.z - q.z);
            } else {
                ok = false;
            }
            if (ok) {
                if (v + 1 < H && nb_ok(pix, depth, k, k + W, d, np)) {
                    const float4 q = __ldg(pix + k + W);
                    b = make_float3(q.x - c.x, q.y - c.y, q.z - c.z);
                } else if (v >= 1 && nb_ok(pix, depth, k, k - W, d, np)) {
                    const float4 q = __ldg(pix + k - W);
                    b = make_float3(c.x - q.x, c.y - q.y, c.z - q.z);
                } else {
                    ok = false;
                }
            }
            if (ok) {
                float3 n = make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
                const float nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
                const float na = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
                const float nb = sqrtf(b.x * b.x + b.y * b.y + b.z * b.z);
                if (nn >= np.min_cross * na * nb && nn > 0.0f) {
                    float s = 1.0f / nn;
                    if (n.x * c.x + n.y * c.y + n.z * c.z > 0.0f) s = -s;
                    out = make_float4(n.x * s, n.y * s, n.z * s, 1.0f);
                }
            }
        }
        store_nw(nrm, k, precision, out);
    }
}

}  // namespace upslam

using namespace upslam;

extern "C" upslam_status upslam_normals(const float *d_pix, const float *d_depth, const upslam_pano *pp,
                                        const upslam_normal_params *np, void *d_nrm, int32_t nrm_precision,
                                        void *stream) {
    if (!upslam_pano_ok(pp) || !np || !d_pix || !d_depth || !d_nrm || !upslam_aligned(d_pix, 16))
        return UPSLAM_ERR_INVALID_ARG;
    if (nrm_precision != UPSLAM_F32 && nrm_precision != UPSLAM_F16) return UPSLAM_ERR_INVALID_ARG;
    if (!upslam_aligned(d_nrm, nrm_precision == UPSLAM_F32 ? 16 : 8)) return UPSLAM_ERR_INVALID_ARG;
    const int npx = pp->rows * pp->cols;
    normals_kernel<<<upslam_grid(npx, 256), 256, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float4 *>(d_pix), d_depth, *pp, *np, d_nrm, nrm_precision);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}
