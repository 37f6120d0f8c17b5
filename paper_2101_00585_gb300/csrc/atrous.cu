// Edge-avoiding a-trous smoothing of a normal image (UPSLAM Sec. III-A: normals
// from neighbour cross products carry much noise and are smoothed by a filter
// that stops at edges, the a-trous wavelet filter of Dammertz et al. 2010;
// Sec. III-B: the smoothing helps ICP converge).
//
// Level l (step s = 2^l) sets every valid pixel p to the normalised sum over the
// 5 x 5 taps q = p + s (dy, dx), dy, dx in -2..2, of
//     h(dy) h(dx) exp(-|N_p - N_q|^2 / sigma_n^2 - (N_p . (P_q - P_p))^2 / (sigma_x |P_p|)^2) N_q,
// h = [1, 4, 6, 4, 1] / 16, over valid taps only; columns wrap (the panorama is
// a full turn), rows outside the image are skipped, invalid pixels stay invalid.
// The levels run as one launch each, ping-ponging between the output and a
// scratch image so the last level lands in the output.  CTAs of 64 threads
// spread a 64x1024 image's 1024 CTAs evenly over the SMs, and 128 registers
// let each thread keep more of its 50 tap loads in flight.
//
// Roofline: per level a pixel reads its own point and normal once from HBM or
// L2 (16 + 16 B in FP32, 16 + 8 B in FP16) and writes its normal (16 / 8 B); the
// 24 other taps are neighbours' data, served by L1/L2.
#include "common.cuh"

namespace upslam {

template <int PREC>
__global__ void __launch_bounds__(64, 8) atrous_kernel(upslam_pano pp, const float4 *__restrict__ pix, const void *nin,
                                                      void *nout, int step, float inv_sn2, float inv_sx2) {
    pdl_wait();     // the previous level's output is complete
    pdl_release();  // and the next level may place its CTAs
    const int W = pp.cols, H = pp.rows, npx = H * W;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= npx) return;
    const float4 n0 = load_nw(nin, k, PREC);
    if (n0.w == 0.0f) {
        store_nw(nout, k, PREC, make_float4(0.f, 0.f, 0.f, 0.f));
        return;
    }
    const float h[5] = {0.0625f, 0.25f, 0.375f, 0.25f, 0.0625f};
    const int v = k / W, u = k - v * W;
    const float4 P = __ldg(pix + k);
    const float inv_scale2 = inv_sx2 / (P.x * P.x + P.y * P.y + P.z * P.z);
    float ax = 0.0f, ay = 0.0f, az = 0.0f;
    // Branch-free taps: a row outside the image reads the pixel's own row instead and an invalid tap is
    // read anyway, both then dropped, so every load of the 25 taps can be in flight at once.
#pragma unroll
    for (int dy = -2; dy <= 2; ++dy) {
        const int vq = v + dy * step;
        const bool row_ok = vq >= 0 && vq < H;
        const int vr = row_ok ? vq : v;
#pragma unroll
        for (int dx = -2; dx <= 2; ++dx) {
            int uq = u + dx * step;
            uq = uq < 0 ? uq + W : (uq >= W ? uq - W : uq);
            const int q = vr * W + uq;
            const float4 n = load_nw(nin, q, PREC);
            const float4 Q = __ldg(pix + q);
            const float ex = n0.x - n.x, ey = n0.y - n.y, ez = n0.z - n.z;
            const float dn2 = ex * ex + ey * ey + ez * ez;
            const float dpl = n0.x * (Q.x - P.x) + n0.y * (Q.y - P.y) + n0.z * (Q.z - P.z);
            const float w = h[dy + 2] * h[dx + 2] * __expf(-(dn2 * inv_sn2 + dpl * dpl * inv_scale2));
            // selected, not multiplied: an invalid tap's contents are unspecified
            const bool ok = row_ok && n.w != 0.0f;
            ax += ok ? w * n.x : 0.0f;
            ay += ok ? w * n.y : 0.0f;
            az += ok ? w * n.z : 0.0f;
        }
    }
    const float l = rsqrtf(ax * ax + ay * ay + az * az);
    store_nw(nout, k, PREC, make_float4(ax * l, ay * l, az * l, 1.0f));
}

}  // namespace upslam

using namespace upslam;

extern "C" upslam_status upslam_atrous_normals(const upslam_pano *pp, const float *d_pix, const void *d_nrm_in,
                                               void *d_nrm_out, void *d_tmp, int32_t precision,
                                               const upslam_atrous_params *ap, void *stream) {
    if (!pp || !ap || !d_pix || !d_nrm_in || !d_nrm_out || !upslam_pano_ok(pp)) return UPSLAM_ERR_INVALID_ARG;
    if (precision != UPSLAM_F32 && precision != UPSLAM_F16) return UPSLAM_ERR_INVALID_ARG;
    if (ap->levels < 0 || ap->levels > 6 || !(ap->sigma_n > 0.0f) || !(ap->sigma_x > 0.0f))
        return UPSLAM_ERR_INVALID_ARG;
    if ((1 << ap->levels) > pp->cols) return UPSLAM_ERR_INVALID_ARG;  // taps reach at most 2^levels columns away
    if (ap->levels >= 2 && !d_tmp) return UPSLAM_ERR_INVALID_ARG;
    const size_t esz = precision == UPSLAM_F32 ? 16 : 8;
    if (!upslam_aligned(d_pix, 16) || !upslam_aligned(d_nrm_in, esz) || !upslam_aligned(d_nrm_out, esz) ||
        (d_tmp && !upslam_aligned(d_tmp, esz)))
        return UPSLAM_ERR_INVALID_ARG;
    if (d_nrm_in == d_nrm_out || d_nrm_in == d_tmp || (d_tmp && d_tmp == d_nrm_out)) return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npx = (int64_t)pp->rows * pp->cols;
    if (ap->levels == 0)
        return cudaMemcpyAsync(d_nrm_out, d_nrm_in, (size_t)npx * esz, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                   ? UPSLAM_OK
                   : UPSLAM_ERR_CUDA;
    const float inv_sn2 = 1.0f / (ap->sigma_n * ap->sigma_n), inv_sx2 = 1.0f / (ap->sigma_x * ap->sigma_x);
    const float4 *pix = reinterpret_cast<const float4 *>(d_pix);
    const int blocks = (int)((npx + 63) / 64);
    // level l writes out when levels - 1 - l is even, so the last level lands in the output
    const void *src = d_nrm_in;
    for (int l = 0; l < ap->levels; ++l) {
        void *dst = ((ap->levels - 1 - l) % 2 == 0) ? d_nrm_out : d_tmp;
        if (l == 0) {
            if (precision == UPSLAM_F32)
                atrous_kernel<UPSLAM_F32><<<blocks, 64, 0, s>>>(*pp, pix, src, dst, 1 << l, inv_sn2, inv_sx2);
            else
                atrous_kernel<UPSLAM_F16><<<blocks, 64, 0, s>>>(*pp, pix, src, dst, 1 << l, inv_sn2, inv_sx2);
            UPSLAM_CHECK_LAUNCH();
        } else {
            // later levels overlap the previous level's tail (each waits for its input first)
            const bool ok = precision == UPSLAM_F32
                                ? launch_dependent(atrous_kernel<UPSLAM_F32>, dim3(blocks), dim3(64), 0, s, *pp, pix,
                                                   src, dst, 1 << l, inv_sn2, inv_sx2)
                                : launch_dependent(atrous_kernel<UPSLAM_F16>, dim3(blocks), dim3(64), 0, s, *pp, pix,
                                                   src, dst, 1 << l, inv_sn2, inv_sx2);
            if (!ok) return UPSLAM_ERR_CUDA;
        }
        src = dst;
    }
    return UPSLAM_OK;
}
