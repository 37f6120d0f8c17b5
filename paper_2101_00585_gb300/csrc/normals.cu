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

__global__ void __launch_bounds__(256) normals_kernel(const float4 *__restrict__ pix, const float *__restrict__ depth,
                                                      upslam_pano pp, upslam_normal_params np, void *nrm,
                                                      int precision) {
    const int npx = pp.rows * pp.cols;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npx; k += gridDim.x * blockDim.x)
        store_nw(nrm, k, precision, normal_pixel(PixArrays<false>{pix, depth}, pp, np, k));
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
