// Motion prior for the ICP initial guess (UPSLAM Sec. IV-F footnote: a zero
// velocity prior by default, a zero acceleration prior as the alternative).
//
// Kept on the device so a whole sweep can run without a host round trip:
//   predict:        T0 = T_prev * M   (M = identity for the zero-velocity prior)
//   update motion:  M  = T_prev^-1 * T
// Rotations are re-orthonormalised (Gram-Schmidt on the rows) after every
// product so rounding cannot compound from sweep to sweep.  FP64, one thread,
// no FP64 division or square root.
#include "common.cuh"

namespace upslam {

__device__ void mul34(const double *A, const double *B, double *C) {
    double t[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) t[4 * i + j] = A[4 * i] * B[j] + A[4 * i + 1] * B[4 + j] + A[4 * i + 2] * B[8 + j];
        t[4 * i + 3] = A[4 * i] * B[3] + A[4 * i + 1] * B[7] + A[4 * i + 2] * B[11] + A[4 * i + 3];
    }
    for (int i = 0; i < 12; ++i) C[i] = t[i];
}

__device__ void inv34(const double *A, double *B) {
    double t[12];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t[4 * i + j] = A[4 * j + i];
    for (int i = 0; i < 3; ++i) t[4 * i + 3] = -(t[4 * i] * A[3] + t[4 * i + 1] * A[7] + t[4 * i + 2] * A[11]);
    for (int i = 0; i < 12; ++i) B[i] = t[i];
}

__device__ void orthonormalise(double *T) { orthonormalise_rows(T); }

__global__ void predict_kernel(const double *T_prev, const double *M, double *T_out) {
    double t[12];
    if (M) {
        mul34(T_prev, M, t);
        orthonormalise(t);
    } else {
        for (int i = 0; i < 12; ++i) t[i] = T_prev[i];
    }
    for (int i = 0; i < 12; ++i) T_out[i] = t[i];
}

__global__ void motion_kernel(const double *T_prev, const double *T, double *M) {
    double inv[12], t[12];
    inv34(T_prev, inv);
    mul34(inv, T, t);
    orthonormalise(t);
    for (int i = 0; i < 12; ++i) M[i] = t[i];
}

}  // namespace upslam

using namespace upslam;

extern "C" upslam_status upslam_predict_pose(const double *d_T_prev, const double *d_motion, double *d_T_out,
                                             void *stream) {
    if (!d_T_prev || !d_T_out) return UPSLAM_ERR_INVALID_ARG;
    predict_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_T_prev, d_motion, d_T_out);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_update_motion(const double *d_T_prev, const double *d_T, double *d_motion,
                                              void *stream) {
    if (!d_T_prev || !d_T || !d_motion) return UPSLAM_ERR_INVALID_ARG;
    motion_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_T_prev, d_T, d_motion);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

namespace upslam {

__global__ void se3_exp_batch_kernel(const float *xi, int n, double *poses) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[6], T[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    for (int k = 0; k < 6; ++k) x[k] = (double)xi[6 * i + k];
    se3_exp_left(x, T);
    for (int k = 0; k < 12; ++k) poses[12 * i + k] = T[k];
}

}  // namespace upslam

extern "C" upslam_status upslam_se3_exp(const float *d_xi, int32_t n, double *d_poses, void *stream) {
    if (!d_xi || !d_poses || n < 0) return UPSLAM_ERR_INVALID_ARG;
    if (n == 0) return UPSLAM_OK;
    se3_exp_batch_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(d_xi, n, d_poses);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}
