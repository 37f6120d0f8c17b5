// Device-side building blocks shared by the UPSLAM kernels (sm_103a).
//
// The FP32 functions here implement the binning rule stated in upslam.h with
// explicit round-to-nearest intrinsics, so no multiply-add is ever contracted
// into an FMA: the pixel a point falls in, and therefore every z-buffer winner
// and every projective correspondence, is a bit-exact function of the inputs.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/upslam.h"

namespace upslam {

constexpr float kPiF = 3.14159265358979323846f;
constexpr float kHalfPiF = 1.57079632679489661923f;
constexpr unsigned long long kEmptyKey = 0xffffffffffffffffull;
constexpr int kNumSums = 29;  // 21 (J^T J) + 6 (J^T r) + sse + inliers

// ----------------------------------------------------------------------------- FP32 decisions

// atan2 reduced by octant symmetry to atan(t), t in [0, 1], with the odd
// polynomial of Abramowitz & Stegun 4.4.49 (|error| <= 2e-8 before rounding).
__device__ __forceinline__ float atan2p(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = ax > ay ? ax : ay;
    const float mn = ax > ay ? ay : ax;
    if (mx == 0.0f) return 0.0f;
    const float t = __fdiv_rn(mn, mx);
    const float s = __fmul_rn(t, t);
    float p = 0.0028662257f;
    p = __fadd_rn(__fmul_rn(p, s), -0.0161657367f);
    p = __fadd_rn(__fmul_rn(p, s), 0.0429096138f);
    p = __fadd_rn(__fmul_rn(p, s), -0.0752896400f);
    p = __fadd_rn(__fmul_rn(p, s), 0.1065626393f);
    p = __fadd_rn(__fmul_rn(p, s), -0.1420889944f);
    p = __fadd_rn(__fmul_rn(p, s), 0.1999355085f);
    p = __fadd_rn(__fmul_rn(p, s), -0.3333314528f);
    p = __fadd_rn(__fmul_rn(p, s), 1.0f);
    float a = __fmul_rn(t, p);
    if (ay > ax) a = __fsub_rn(kHalfPiF, a);
    if (x < 0.0f) a = __fsub_rn(kPiF, a);
    if (y < 0.0f) a = -a;
    return a;
}

// Pixel (row, col) and range of an FP32 point; false when outside the panorama.
__device__ __forceinline__ bool bin_point(float x, float y, float z, const upslam_pano &pp, int &row, int &col,
                                          float &r) {
    const float xy2 = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
    r = __fsqrt_rn(__fadd_rn(xy2, __fmul_rn(z, z)));
    if (!(r >= pp.r_min && r <= pp.r_max)) return false;
    const float rho = __fsqrt_rn(xy2);
    const float az = atan2p(y, x);
    const float el = atan2p(z, rho);
    const float fc = __fmul_rn(__fsub_rn(kPiF, az), pp.s_az);
    const float fr = __fmul_rn(__fsub_rn(pp.el_top, el), pp.s_el);
    if (!(fr >= 0.0f) || !(fr < (float)pp.rows)) return false;
    row = (int)floorf(fr);
    col = (int)floorf(fc);
    if (row >= pp.rows) return false;
    if (col >= pp.cols) col -= pp.cols;
    if (col < 0) col += pp.cols;
    return true;
}

// Pose rounded to FP32, row-major [R | t].
struct PoseF {
    float r[12];
};

__device__ __forceinline__ PoseF pose_to_f32(const double *T) {
    PoseF p;
#pragma unroll
    for (int i = 0; i < 12; ++i) p.r[i] = (float)T[i];
    return p;
}

// The CTA's pose in FP32, converted once: threads 0..11 convert one entry each
// into shared memory and every thread reads the FP32 copy.  (An FP64 -> FP32
// conversion issues on GB300's FP64 pipe; converting per thread would cost
// every warp twelve slow instructions.)  Must be reached by the whole CTA.
__device__ __forceinline__ PoseF cta_pose_f32(const double *T, bool through_l2 = false) {
    __shared__ float ps[12];
    __syncthreads();
    if (threadIdx.x < 12) ps[threadIdx.x] = (float)(through_l2 ? __ldcg(T + threadIdx.x) : T[threadIdx.x]);
    __syncthreads();
    PoseF p;
#pragma unroll
    for (int i = 0; i < 12; ++i) p.r[i] = ps[i];
    return p;
}

// Pose read through L2 only (never a stale L1 line): for poses other CTAs rewrite.
__device__ __forceinline__ PoseF pose_to_f32_cg(const double *T) {
    PoseF p;
#pragma unroll
    for (int i = 0; i < 12; ++i) p.r[i] = (float)__ldcg(T + i);
    return p;
}

// p = R q + t, fixed order ((r0 x + r1 y) + r2 z) + t0, no contraction.
__device__ __forceinline__ float3 xform(const PoseF &T, float qx, float qy, float qz) {
    const float *r = T.r;
    float3 p;
    p.x = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[0], qx), __fmul_rn(r[1], qy)), __fmul_rn(r[2], qz)), r[3]);
    p.y = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[4], qx), __fmul_rn(r[5], qy)), __fmul_rn(r[6], qz)), r[7]);
    p.z = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r[8], qx), __fmul_rn(r[9], qy)), __fmul_rn(r[10], qz)), r[11]);
    return p;
}

// q = R^T (s - t), fixed order.
__device__ __forceinline__ float3 xform_inv(const PoseF &T, float sx, float sy, float sz) {
    const float *r = T.r;
    const float dx = __fsub_rn(sx, r[3]), dy = __fsub_rn(sy, r[7]), dz = __fsub_rn(sz, r[11]);
    float3 q;
    q.x = __fadd_rn(__fadd_rn(__fmul_rn(r[0], dx), __fmul_rn(r[4], dy)), __fmul_rn(r[8], dz));
    q.y = __fadd_rn(__fadd_rn(__fmul_rn(r[1], dx), __fmul_rn(r[5], dy)), __fmul_rn(r[9], dz));
    q.z = __fadd_rn(__fadd_rn(__fmul_rn(r[2], dx), __fmul_rn(r[6], dy)), __fmul_rn(r[10], dz));
    return q;
}

// Rotation only (values, FMA allowed).
__device__ __forceinline__ float3 rotate(const PoseF &T, float x, float y, float z) {
    const float *r = T.r;
    return make_float3(r[0] * x + r[1] * y + r[2] * z, r[4] * x + r[5] * y + r[6] * z,
                       r[8] * x + r[9] * y + r[10] * z);
}

// FP32 point of pixel (v, u) at depth d from the direction table: d * (ce*ca, ce*sa, se).
__device__ __forceinline__ float3 pixel_point(const float *dirs, int rows, int v, int u, float d) {
    const float2 e = __ldg(reinterpret_cast<const float2 *>(dirs) + v);
    const float2 a = __ldg(reinterpret_cast<const float2 *>(dirs + 2 * rows) + u);
    return make_float3(__fmul_rn(d, __fmul_rn(e.x, a.x)), __fmul_rn(d, __fmul_rn(e.x, a.y)), __fmul_rn(d, e.y));
}

// ----------------------------------------------------------------------------- storage helpers

__device__ __forceinline__ float4 load_nw(const void *base, int64_t k, int precision) {
    if (precision == UPSLAM_F32) return __ldg(reinterpret_cast<const float4 *>(base) + k);
    const uint2 raw = __ldg(reinterpret_cast<const uint2 *>(base) + k);
    const __half2 a = *reinterpret_cast<const __half2 *>(&raw.x);
    const __half2 b = *reinterpret_cast<const __half2 *>(&raw.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// Same load, through L2 only (for data rewritten during the kernel's lifetime by other CTAs).
__device__ __forceinline__ float4 load_nw_cg(const void *base, int64_t k, int precision) {
    if (precision == UPSLAM_F32) return __ldcg(reinterpret_cast<const float4 *>(base) + k);
    const uint2 raw = __ldcg(reinterpret_cast<const uint2 *>(base) + k);
    const __half2 a = *reinterpret_cast<const __half2 *>(&raw.x);
    const __half2 b = *reinterpret_cast<const __half2 *>(&raw.y);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

__device__ __forceinline__ void store_nw(void *base, int64_t k, int precision, float4 v) {
    if (precision == UPSLAM_F32) {
        reinterpret_cast<float4 *>(base)[k] = v;
        return;
    }
    const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
    uint2 raw;
    raw.x = *reinterpret_cast<const unsigned int *>(&a);
    raw.y = *reinterpret_cast<const unsigned int *>(&b);
    reinterpret_cast<uint2 *>(base)[k] = raw;
}

// ----------------------------------------------------------------------------- reductions

// Warp reduce-scatter: lane L ends with the sum over the warp's lanes of v[L]
// (32 values per lane, 31 shuffles in all; v is overwritten).
__device__ __forceinline__ float warp_reduce_scatter(float v[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = upper ? v[i] : v[i + o];
            const float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// ----------------------------------------------------------------------------- FP64 solve
//
// GB300 runs FP64 at a small fraction of its FP32 rate, and a dependent FP64
// FMA costs tens of cycles (a division an order of magnitude more), so the
// solve is written for a short dependency chain: fully unrolled (every value
// in a register), no FP64 division or square root on the critical path.

// FP64 helpers that stay off the FP64 pipe.  Comparisons, maxima, sign flips
// and format changes work on the bit patterns with integer instructions: for
// doubles that are not NaN, the signed 64-bit order of the bit patterns of
// non-negative values is their numeric order.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool dfinite(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ double dneg(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ull);
}

// Exact FP32 -> FP64 widening: the exponent is rebiased (+896) and the
// mantissa shifted into place with integer instructions.  Zero, subnormal,
// infinite and NaN inputs take the conversion instruction.
__device__ __forceinline__ double f2d(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const unsigned m = b & 0x7fffffu;
    return __hiloint2double((int)((b & 0x80000000u) | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// 1/d for a positive d.  The FP32 seed is d's exponent and top 23 mantissa bits
// (truncation: relative error below 2^-23), formed and widened back with integer
// instructions; one FP64 Newton step then leaves a relative error below 2^-44,
// far below the FP32 accumulation error of the normal equations.  d outside
// [2^-126, 2^126) takes an FP64 division.
__device__ __forceinline__ double rcp64(double d) {
    const int hi = __double2hiint(d), lo = __double2loint(d);
    const int e = ((hi >> 20) & 0x7ff) - (1023 - 127);
    if (hi < 0 || e < 1 || e > 252) return 1.0 / d;
    const float f = __int_as_float((e << 23) | ((hi & 0xfffff) << 3) | (int)((unsigned)lo >> 29));
    const int rb = __float_as_int(__frcp_rn(f));  // normal: f in [2^-126, 2^126)
    const int m = rb & 0x7fffff;
    const double x = __hiloint2double((((rb >> 23) & 0xff) + (1023 - 127)) << 20 | (m >> 3), m << 29);
    return fma(x, fma(-d, x, 1.0), x);
}

// sin(t)/t, (1 - cos t)/t^2, (t - sin t)/t^3 from t^2: Taylor series (truncation
// below 1e-18 for t <= 0.25), sincos otherwise.
__device__ __forceinline__ void se3_coeffs(double th2, double &A, double &B, double &C) {
    if (th2 <= 0.0625) {
        A = fma(th2, fma(th2, fma(th2, fma(th2, fma(th2, fma(th2, 1.0 / 6227020800.0, -1.0 / 39916800.0),
                                                    1.0 / 362880.0), -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0), 1.0);
        B = fma(th2, fma(th2, fma(th2, fma(th2, fma(th2, fma(th2, 1.0 / 87178291200.0, -1.0 / 479001600.0),
                                                    1.0 / 3628800.0), -1.0 / 40320.0), 1.0 / 720.0), -1.0 / 24.0), 0.5);
        C = fma(th2, fma(th2, fma(th2, fma(th2, fma(th2, fma(th2, 1.0 / 1307674368000.0, -1.0 / 6227020800.0),
                                                    1.0 / 39916800.0), -1.0 / 362880.0), 1.0 / 5040.0), -1.0 / 120.0),
                1.0 / 6.0);
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(th, &sn, &cs);
        A = sn / th;
        B = (1.0 - cs) / th2;
        C = (th - sn) / (th2 * th);
    }
}

// T <- exp(xi^) T (left update), xi = (omega, v): Rodrigues rotation
// R = I + A W + B W^2 and translation V v with V = I + B W + C W^2, where
// W = [omega]_x and W^2 = omega omega^T - |omega|^2 I.
__device__ __forceinline__ void se3_exp_left(const double xi[6], double T[12]) {
    const double w0 = xi[0], w1 = xi[1], w2 = xi[2];
    const double th2 = fma(w0, w0, fma(w1, w1, w2 * w2));
    double A, B, C;
    se3_coeffs(th2, A, B, C);
    const double W[9] = {0.0, -w2, w1, w2, 0.0, -w0, -w1, w0, 0.0};
    const double om[3] = {w0, w1, w2};
    double R[9], V[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double W2 = fma(om[i], om[j], i == j ? -th2 : 0.0);
            const double I = i == j ? 1.0 : 0.0;
            R[3 * i + j] = fma(A, W[3 * i + j], fma(B, W2, I));
            V[3 * i + j] = fma(B, W[3 * i + j], fma(C, W2, I));
        }
    double Tn[12];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j)
            Tn[4 * i + j] = fma(R[3 * i], T[j], fma(R[3 * i + 1], T[4 + j], R[3 * i + 2] * T[8 + j]));
        const double te = fma(V[3 * i], xi[3], fma(V[3 * i + 1], xi[4], V[3 * i + 2] * xi[5]));
        Tn[4 * i + 3] = fma(R[3 * i], T[3], fma(R[3 * i + 1], T[7], fma(R[3 * i + 2], T[11], te)));
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) T[i] = Tn[i];
}

// Solve M x = rhs for the symmetric positive-definite 6x6 M given by its
// row-major upper triangle, by the square-root-free Cholesky factorisation
// M = L D L^T (elimination on the upper triangle, then back substitution).
// Returns false when a pivot D_j <= pivot_eps * max diagonal (the same
// quantity a square-root Cholesky compares before its square root).
__device__ __forceinline__ bool solve6(const double *Aup, const double *rhs, double pivot_eps, double *x) {
    double U[6][6];
    double y[6], r[6];
    {
        int p = 0;
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = i; j < 6; ++j) U[i][j] = Aup[p++];
    }
    double dmax = U[0][0];
#pragma unroll
    for (int i = 1; i < 6; ++i) dmax = fmax(dmax, U[i][i]);
    if (!(dmax > 0.0)) return false;
    const double lim = pivot_eps * dmax;
#pragma unroll
    for (int i = 0; i < 6; ++i) y[i] = rhs[i];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double d = U[j][j];
        if (!(d > lim) || !(d > 1e-300)) return false;
        r[j] = rcp64(d);
#pragma unroll
        for (int i = j + 1; i < 6; ++i) {
            const double l = U[j][i] * r[j];  // M symmetric: row j, column i of the reduced matrix
#pragma unroll
            for (int k = i; k < 6; ++k) U[i][k] = fma(-l, U[j][k], U[i][k]);
            y[i] = fma(-l, y[j], y[i]);
        }
    }
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
#pragma unroll
        for (int k = i + 1; k < 6; ++k) s = fma(-U[i][k], x[k], s);
        x[i] = s * r[i];
    }
    return true;
}

// 1/sqrt(x) for a positive normal x: FP32 seed, two FP64 Newton steps.
__device__ __forceinline__ double rsqrt64(double x) {
    double y = (double)rsqrtf((float)x);
    const double hx = 0.5 * x;
    y = y * fma(-hx * y, y, 1.5);
    y = y * fma(-hx * y, y, 1.5);
    return y;
}

// Gram-Schmidt on the rows of the rotation of a 3x4 pose (FP64, one thread).
__device__ __forceinline__ void orthonormalise_rows(double *T) {
    double *r0 = T, *r1 = T + 4, *r2 = T + 8;
    double n = rsqrt64(fma(r0[0], r0[0], fma(r0[1], r0[1], r0[2] * r0[2])));
    r0[0] *= n;
    r0[1] *= n;
    r0[2] *= n;
    const double d = fma(r0[0], r1[0], fma(r0[1], r1[1], r0[2] * r1[2]));
    r1[0] = fma(-d, r0[0], r1[0]);
    r1[1] = fma(-d, r0[1], r1[1]);
    r1[2] = fma(-d, r0[2], r1[2]);
    n = rsqrt64(fma(r1[0], r1[0], fma(r1[1], r1[1], r1[2] * r1[2])));
    r1[0] *= n;
    r1[1] *= n;
    r1[2] *= n;
    r2[0] = r0[1] * r1[2] - r0[2] * r1[1];
    r2[1] = r0[2] * r1[0] - r0[0] * r1[2];
    r2[2] = r0[0] * r1[1] - r0[1] * r1[0];
}

// C = A B for 3x4 poses on one warp: lane e < 12 computes entry e.  C may alias an input: every
// lane reads its operands before any lane writes.
__device__ __forceinline__ void warp_pose_mul(const double *A, const double *B, double *C) {
    const int lane = threadIdx.x & 31;
    const int i = lane < 12 ? lane / 4 : 0, j = lane < 12 ? lane % 4 : 0;
    const double v =
        fma(A[4 * i], B[j], fma(A[4 * i + 1], B[4 + j], fma(A[4 * i + 2], B[8 + j], j == 3 ? A[4 * i + 3] : 0.0)));
    __syncwarp();
    if (lane < 12) C[lane] = v;
    __syncwarp();
}

// C = A^-1 = [R^T | -R^T t] on one warp.
__device__ __forceinline__ void warp_pose_inv(const double *A, double *C) {
    const int lane = threadIdx.x & 31;
    const int i = lane < 12 ? lane / 4 : 0, j = lane < 12 ? lane % 4 : 0;
    const double v = j < 3 ? A[4 * j + i] : -fma(A[i], A[3], fma(A[4 + i], A[7], A[8 + i] * A[11]));
    __syncwarp();
    if (lane < 12) C[lane] = v;
    __syncwarp();
}

// Neumaier-compensated FP32 accumulation: (s, c) holds s + c.
__device__ __forceinline__ void kadd(float &s, float &c, float v) {
    const float t = s + v;
    c += fabsf(s) >= fabsf(v) ? (s - t) + v : (v - t) + s;
    s = t;
}

// Lane of the upper-triangle element (i, k), i <= k, in row-major order (0..20).
__device__ __forceinline__ int uidx(int i, int k) { return i * 6 - (i * (i - 1)) / 2 + (k - i); }

// d's mantissa as a double in [1, 2) (its exponent field set to the bias) and its unbiased exponent.
__device__ __forceinline__ double dmant(double d) {
    return __longlong_as_double((__double_as_longlong(d) & ~(0x7ffLL << 52)) | (1023LL << 52));
}
__device__ __forceinline__ int dexpo(double d) { return ((__double2hiint(d) >> 20) & 0x7ff) - 1023; }

// x * 2^-e by exponent arithmetic (exact for normal results); zero stays zero, results below the
// normal range become signed zero and above it signed infinity.
__device__ __forceinline__ double dscale2(double x, int e) {
    const long long b = __double_as_longlong(x);
    const int ef = (int)((b >> 52) & 0x7ff);
    if (ef == 0) return x;
    const int en = ef - e;
    const long long sign = b & (long long)0x8000000000000000ull;
    if (en <= 0) return __longlong_as_double(sign);
    if (en >= 0x7ff) return __longlong_as_double(sign | (0x7ffLL << 52));
    return __longlong_as_double((b & ~(0x7ffLL << 52)) | ((long long)en << 52));
}

// FP64 solve of A xi = -b for the symmetric 6x6 A (the square-root-free Cholesky
// factorisation A = L D L^T, i.e. symmetric Gaussian elimination), spread over the
// lanes of one warp: lanes 0..20 hold the upper triangle of A (lane uidx(i, k)),
// lanes 21..26 the right-hand side.  GB300 issues an FP64 warp instruction every
// 64 cycles whatever its active lanes, so independent work goes across lanes and
// the elimination is division-free: step j replaces every later row by
//     row <- mant(D_j) row - (L_jrow 2^-exp(D_j)) row_j,
// i.e. the Schur complement scaled by D_j / 2^exp(D_j) in [1, 2), with the power
// of two taken off by exponent arithmetic: one multiply and one multiply-add per
// step and no reciprocal on the chain.  Row j then holds F_j times the standard
// pivot row (F_j = prod_{m<j} mant(D_m) < 2^j), so the pivot test uses
// D_j / F_j, and the back substitution, which the common factor of a row does
// not change, scales every row by its reciprocal pivot in one instruction and
// then takes one multiply-add per unknown.  Comparisons, maxima and sign flips
// are integer instructions on the bit patterns.  Every lane returns the same xi.
// False when a standard pivot D_j / F_j <= max(pivot_eps * max diagonal, 1e-300),
// a pivot is not finite, or the solution is not finite.
__device__ __forceinline__ bool warp_solve6(const double *tot, double pivot_eps, double xi[6]) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool is_u = lane < 21, is_y = lane >= 21 && lane < 27;
    int li = -1, lk = -1;
    if (is_u) {
        int i = 0, rem = lane;
        while (rem >= 6 - i) {
            rem -= 6 - i;
            ++i;
        }
        li = i;
        lk = i + rem;
    } else if (is_y) {
        li = lane - 21;
        lk = 6;
    }
    const double t = (is_u || is_y) ? tot[lane] : 0.0;
    double u = is_y ? dneg(t) : t;
    long long dm = dbits(tot[0]);
#pragma unroll
    for (int i = 1; i < 6; ++i) dm = max(dm, dbits(tot[uidx(i, i)]));
    if (!(dm > 0) || !dfinite(__longlong_as_double(dm))) return false;
    const double lim = __longlong_as_double(max(dbits(pivot_eps * __longlong_as_double(dm)), dbits(1e-300)));
    double piv[6], mnt[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double d = __shfl_sync(full, u, uidx(j, j));
        const bool act = li > j;
        const int src_l = act ? uidx(j, li) : lane;
        const int src_k = act ? (is_u ? uidx(j, lk) : 21 + j) : lane;
        const double ujl = __shfl_sync(full, u, src_l);
        const double ujk = __shfl_sync(full, u, src_k);
        piv[j] = d;
        mnt[j] = dmant(d);
        if (act) u = fma(-dscale2(ujl, dexpo(d)), ujk, mnt[j] * u);
    }
    // pivot test on the standard pivots D_j / F_j: lane j < 6 forms F_j = prod_{m<j} mant(D_m)
    double F = 1.0;
#pragma unroll
    for (int m = 0; m < 5; ++m) F = m < lane ? F * mnt[m] : F;
    const int jl = lane < 6 ? lane : 0;
    double pj = piv[0];
#pragma unroll
    for (int j = 1; j < 6; ++j) pj = jl == j ? piv[j] : pj;
    const bool bad = lane < 6 && (!dfinite(pj) || !(dbits(pj) > dbits(lim * F)));
    if (__any_sync(full, bad)) return false;
    // back substitution: lane (i, k) -> S_ik / D_i, lane 21 + i -> y_i / D_i
    double di = piv[0];
#pragma unroll
    for (int j = 1; j < 6; ++j) di = li == j ? piv[j] : di;
    double v = li >= 0 ? u * rcp64(di) : 0.0;
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        const double x = __shfl_sync(full, v, 21 + i);
        xi[i] = x;
        if (i > 0) {
            const bool act = is_y && li < i;
            const double lmi = __shfl_sync(full, v, act ? uidx(li, i) : lane);
            if (act) v = fma(-lmi, x, v);
        }
    }
    bool fin = true;
#pragma unroll
    for (int i = 0; i < 6; ++i) fin = fin && dfinite(xi[i]);
    return fin;
}

// (-1)^n / (2n + 1 + c)!: the n-th Taylor coefficient in t^2 of sin(t)/t (c = 0),
// (1 - cos t)/t^2 (c = 1) and (t - sin t)/t^3 (c = 2).
__device__ __forceinline__ double se3_taylor_coef(int n, int c) {
    constexpr double k[6][3] = {
        {1.0, 1.0 / 2.0, 1.0 / 6.0},
        {-1.0 / 6.0, -1.0 / 24.0, -1.0 / 120.0},
        {1.0 / 120.0, 1.0 / 720.0, 1.0 / 5040.0},
        {-1.0 / 5040.0, -1.0 / 40320.0, -1.0 / 362880.0},
        {1.0 / 362880.0, 1.0 / 3628800.0, 1.0 / 39916800.0},
        {-1.0 / 39916800.0, -1.0 / 479001600.0, -1.0 / 6227020800.0},
    };
    return c == 0 ? k[n][0] : (c == 1 ? k[n][1] : k[n][2]);
}

// T <- exp(xi^) T on one warp: lanes 0..2 evaluate the coefficients A, B, C;
// lanes 0..8 the rotation R = I + A W + B W^2 and lanes 9..17 V = I + B W + C W^2
// (one matrix entry each); then, in the same three multiply-adds, lanes 0..11
// each compose one entry of R T and lanes 12..14 one entry of V v, which the
// translation lanes add.  The series is cut where its remainder (below the
// first omitted term) is under 5e-17 relative: degree 3 in t^2 for t^2 <= 2^-9,
// degree 4 for t^2 <= 2^-6, degree 5 for t^2 <= 1/16, sincos beyond.
// T lives in shared memory (12 doubles) and is updated in place; xi is the same in every lane.
__device__ __forceinline__ void warp_se3_update(const double xi[6], double *T) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const double w0 = xi[0], w1 = xi[1], w2 = xi[2];
    const double th2 = fma(w0, w0, fma(w1, w1, w2 * w2));
    const long long tb = dbits(th2);
    const int c = lane < 3 ? lane : 0;
    double coef;
    if (tb <= dbits(0.001953125)) {
        coef = fma(th2, fma(th2, fma(th2, se3_taylor_coef(3, c), se3_taylor_coef(2, c)), se3_taylor_coef(1, c)),
                   se3_taylor_coef(0, c));
    } else if (tb <= dbits(0.015625)) {
        coef = fma(th2,
                   fma(th2, fma(th2, fma(th2, se3_taylor_coef(4, c), se3_taylor_coef(3, c)), se3_taylor_coef(2, c)),
                       se3_taylor_coef(1, c)),
                   se3_taylor_coef(0, c));
    } else if (tb <= dbits(0.0625)) {
        double p = se3_taylor_coef(5, c);
#pragma unroll
        for (int n = 4; n >= 0; --n) p = fma(th2, p, se3_taylor_coef(n, c));
        coef = p;
    } else {
        double A, B, C;
        se3_coeffs(th2, A, B, C);
        coef = lane == 0 ? A : (lane == 1 ? B : C);
    }
    const double A = __shfl_sync(full, coef, 0), B = __shfl_sync(full, coef, 1), C = __shfl_sync(full, coef, 2);
    // one entry of R (lanes 0..8) or V (lanes 9..17)
    const int e = lane < 9 ? lane : (lane < 18 ? lane - 9 : 0);
    const int ei = e / 3, ek = e - 3 * (e / 3);
    const double om_i = ei == 0 ? w0 : (ei == 1 ? w1 : w2);
    const double om_k = ek == 0 ? w0 : (ek == 1 ? w1 : w2);
    // W = [omega]_x: W[i][k] = -eps_ikl omega_l
    double Wik = 0.0;
    if (ei == 0 && ek == 1) Wik = dneg(w2);
    if (ei == 0 && ek == 2) Wik = w1;
    if (ei == 1 && ek == 0) Wik = w2;
    if (ei == 1 && ek == 2) Wik = dneg(w0);
    if (ei == 2 && ek == 0) Wik = dneg(w1);
    if (ei == 2 && ek == 1) Wik = w0;
    const double W2 = fma(om_i, om_k, ei == ek ? dneg(th2) : 0.0);
    const double c1 = lane < 9 ? A : B, c2 = lane < 9 ? B : C;
    const double ent = fma(c1, Wik, fma(c2, W2, ei == ek ? 1.0 : 0.0));
    // lanes 0..11: (R T)(i, j), i = lane / 4, j = lane % 4; lanes 12..14: (V v)(lane - 12)
    const bool comp = lane < 12, tv = lane >= 12 && lane < 15;
    const int oi = comp ? lane / 4 : (tv ? lane - 12 : 0), oj = comp ? lane % 4 : 0;
    const int src = tv ? 9 + 3 * oi : 3 * oi;
    const double M0 = __shfl_sync(full, ent, src), M1 = __shfl_sync(full, ent, src + 1),
                 M2 = __shfl_sync(full, ent, src + 2);
    const double X0 = tv ? xi[3] : T[oj], X1 = tv ? xi[4] : T[4 + oj], X2 = tv ? xi[5] : T[8 + oj];
    const double o = fma(M0, X0, fma(M1, X1, M2 * X2));
    const double te = __shfl_sync(full, o, 12 + oi);
    const double out = oj == 3 ? o + te : o;
    __syncwarp();
    if (lane < 12) T[lane] = out;
    __syncwarp();
}

// Convergence test on one warp: |omega|^2 < er2 and |v|^2 < et2 (lane 0 takes
// the rotation, lane 1 the translation, in the same instructions).
__device__ __forceinline__ bool warp_converged(const double xi[6], double er2, double et2) {
    const int lane = threadIdx.x & 31;
    const bool tr = lane == 1;
    const double a = tr ? xi[3] : xi[0], b = tr ? xi[4] : xi[1], c = tr ? xi[5] : xi[2];
    const double n2 = fma(a, a, fma(b, b, c * c));
    const bool below = dbits(n2) < dbits(tr ? et2 : er2);
    return (__ballot_sync(0xffffffffu, below) & 3u) == 3u;
}

// ----------------------------------------------------------------------------- exact order-free sums
//
// A float v is held as the integer X = v * 2^48 (truncated toward zero below 2^-48, saturated
// at |v| = 2^47) split into three chunks X = c0 + c1 2^32 + c2 2^64 with |c_k| < 2^32.  Chunks
// add into 64-bit integers with no carry between them for up to 2^31 terms, so a sum of floats
// formed this way is exact and does not depend on the order of the additions (integer atomics
// from any number of CTAs give every reader the same bits).

__device__ __forceinline__ void fx_chunks(float v, long long c[3]) {
    const unsigned b = __float_as_uint(v);
    int e = (int)((b >> 23) & 0xffu);
    unsigned long long m = b & 0x7fffffu;
    if (e == 0xff) m = 0;  // infinities and NaN do not enter a sum
    if (e) m |= 0x800000u;
    else e = 1;
    int sh = e - 150 + 48;  // X = m * 2^sh
    if (sh > 71) sh = 71;   // saturate: |X| < 2^95
    unsigned long long lo, hi;
    if (sh < 0) {
        lo = sh > -32 ? (m >> -sh) : 0ull;
        hi = 0ull;
    } else if (sh < 64) {
        lo = m << sh;
        hi = sh > 40 ? (m >> (64 - sh)) : 0ull;
    } else {
        lo = 0ull;
        hi = m << (sh - 64);
    }
    const long long sgn = (b >> 31) ? -1 : 1;
    c[0] = sgn * (long long)(lo & 0xffffffffull);
    c[1] = sgn * (long long)(lo >> 32);
    c[2] = sgn * (long long)hi;
}

// (s0 + s1 2^32 + s2 2^64) * 2^-48 as the nearest double (ties to even), integer instructions only.
__device__ __forceinline__ double fx_value(long long s0, long long s1, long long s2) {
    const __int128 x = (__int128)s0 + ((__int128)s1 << 32) + ((__int128)s2 << 64);
    if (x == 0) return 0.0;
    const bool neg = x < 0;
    const unsigned __int128 mag = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
    const unsigned long long h = (unsigned long long)(mag >> 64), l = (unsigned long long)mag;
    const int nbits = h ? 128 - __clzll((long long)h) : 64 - __clzll((long long)l);
    unsigned long long mant;
    int top = nbits;  // the value is mant * 2^(top - 53)
    if (nbits <= 53) {
        mant = l << (53 - nbits);
    } else {
        const int sh = nbits - 53;
        mant = (unsigned long long)(mag >> sh);
        const unsigned __int128 rem = mag & ((((unsigned __int128)1) << sh) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) ++mant;
        if (mant >> 53) {
            mant >>= 1;
            ++top;
        }
    }
    const long long ebits = (long long)(top - 1 - 48 + 1023);
    const long long bits = (neg ? (long long)0x8000000000000000ull : 0ll) | (ebits << 52) |
                           (long long)(mant & 0xfffffffffffffull);
    return __longlong_as_double(bits);
}

// ----------------------------------------------------------------------------- sweep front end (Sec. III-A)
//
// The per-point and per-pixel bodies of projection, resolve and normals, shared by
// the standalone kernels and the fused register launch so both give the same bits.
// kCg selects L2-only loads for data that the same launch wrote earlier (the
// read-only cache path is only for data no launch writes while it runs).

template <bool kCg, typename T>
__device__ __forceinline__ T ld_front(const T *p) {
    return kCg ? __ldcg(p) : __ldg(p);
}

// Pass 1 of the z-buffer: the point's key (bits(range) << 32 | index) into its pixel.
__device__ __forceinline__ void project_point(const float4 *pts, int i, const upslam_pano &pp,
                                              unsigned long long *zbuf) {
    const float4 p = __ldg(pts + i);
    if (p.w == 0.0f) return;
    int v, u;
    float r;
    if (!bin_point(p.x, p.y, p.z, pp, v, u, r)) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(r) << 32) | (unsigned int)i;
    atomicMin(zbuf + (size_t)v * pp.cols + u, key);
}

// Pass 2: decode the pixel's word into depth / index / point and (kReset) reset the word.
template <bool kCg, bool kReset = true>
__device__ __forceinline__ void resolve_pixel(const float4 *pts, int k, unsigned long long *zbuf, float *depth,
                                              int *idx, float4 *pix) {
    const unsigned long long key = kCg ? __ldcg(zbuf + k) : zbuf[k];
    if (key == kEmptyKey) {
        depth[k] = 0.0f;
        idx[k] = -1;
        if (pix) pix[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        if (kReset) zbuf[k] = kEmptyKey;
        const int i = (int)(key & 0xffffffffull);
        depth[k] = __uint_as_float((unsigned int)(key >> 32));
        idx[k] = i;
        if (pix) {
            const float4 p = __ldg(pts + i);
            pix[k] = make_float4(p.x, p.y, p.z, 1.0f);
        }
    }
}

// Pixel data for the normals, read from the resolved arrays (point with validity in .w, range).
template <bool kCg>
struct PixArrays {
    const float4 *pix;
    const float *depth;
    __device__ __forceinline__ float4 point(int k) const { return ld_front<kCg>(pix + k); }
    __device__ __forceinline__ float range(int k) const { return ld_front<kCg>(depth + k); }
};

// The same data decoded straight from the z-buffer words (winner index and range in the key),
// before any resolve pass has run: a pixel's normal can then be formed in the pass that resolves it.
struct PixZbuf {
    const float4 *pts;
    const unsigned long long *zbuf;
    __device__ __forceinline__ float4 point(int k) const {
        const unsigned long long key = __ldcg(zbuf + k);
        if (key == kEmptyKey) return make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 p = __ldg(pts + (int)(key & 0xffffffffull));
        return make_float4(p.x, p.y, p.z, 1.0f);
    }
    __device__ __forceinline__ float range(int k) const {
        const unsigned long long key = __ldcg(zbuf + k);
        return key == kEmptyKey ? 0.0f : __uint_as_float((unsigned int)(key >> 32));
    }
};

// Normal of pixel k: a toward column + 1 (wrapping), b toward row + 1, each replaced by the
// opposite neighbour with the sign flipped when unusable; n = a x b, normalised, toward the
// sensor; (0, 0, 0, 0) when there is none.  A neighbour is usable when it holds a point and its
// range is within jump_rel * d + jump_abs of the pixel's (FP32, round to nearest).
template <typename Acc>
__device__ __forceinline__ float4 normal_pixel(const Acc &px, const upslam_pano &pp, const upslam_normal_params &np,
                                               int k) {
    const int H = pp.rows, W = pp.cols;
    const int v = k / W, u = k - v * W;
    const int kr = v * W + (u + 1 == W ? 0 : u + 1);
    const int kl = v * W + (u == 0 ? W - 1 : u - 1);
    const int kd = v + 1 < H ? k + W : k, ku = v >= 1 ? k - W : k;  // (past the edge: k, unused)
    // every pixel the normal may use, read before any test, so the reads overlap
    const float4 c = px.point(k), qr = px.point(kr), ql = px.point(kl), qd = px.point(kd), qu = px.point(ku);
    const float d = px.range(k), dr = px.range(kr), dl = px.range(kl), dd = px.range(kd), du = px.range(ku);
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (c.w == 0.0f) return out;
    const float lim = __fadd_rn(__fmul_rn(np.jump_rel, d), np.jump_abs);
    auto usable = [&](const float4 &q, float dn) { return q.w != 0.0f && !(fabsf(__fsub_rn(dn, d)) > lim); };
    float3 a, b;
    if (usable(qr, dr)) {
        a = make_float3(qr.x - c.x, qr.y - c.y, qr.z - c.z);
    } else if (usable(ql, dl)) {
        a = make_float3(c.x - ql.x, c.y - ql.y, c.z - ql.z);
    } else {
        return out;
    }
    if (v + 1 < H && usable(qd, dd)) {
        b = make_float3(qd.x - c.x, qd.y - c.y, qd.z - c.z);
    } else if (v >= 1 && usable(qu, du)) {
        b = make_float3(c.x - qu.x, c.y - qu.y, c.z - qu.z);
    } else {
        return out;
    }
    const float3 n = make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
    const float nn = sqrtf(n.x * n.x + n.y * n.y + n.z * n.z);
    const float na = sqrtf(a.x * a.x + a.y * a.y + a.z * a.z);
    const float nb = sqrtf(b.x * b.x + b.y * b.y + b.z * b.z);
    if (nn >= np.min_cross * na * nb && nn > 0.0f) {
        float s = 1.0f / nn;
        if (n.x * c.x + n.y * c.y + n.z * c.z > 0.0f) s = -s;
        out = make_float4(n.x * s, n.y * s, n.z * s, 1.0f);
    }
    return out;
}

// ----------------------------------------------------------------------------- keyframe update pieces

// Everything one keyframe update reads and writes.
struct FuseView {
    upslam_pano kp;
    float *kdepth;
    void *knw;
    int kprec;
    const float *kdirs;
    upslam_pano sp;
    const float4 *spix;
    const void *snrm;
    int sprec;
    float d_max2, cos_min, w_max, accept;
    unsigned long long *zbuf;
};

// Average the sweep sample that keyframe pixel k (point s, normal + count nk,
// depth d, nk.w > 0) projects onto into the pixel, if the similarity gate keeps
// the pair (Sec. III-C).  Shared by upslam_fuse and the fused register+update.
__device__ __forceinline__ void fuse_average(const FuseView &f, const PoseF &T, int k, float3 s, float4 nk, float d) {
    const float w = nk.w;
    const float3 q = xform_inv(T, s.x, s.y, s.z);
    int jv, ju;
    float rr;
    if (!bin_point(q.x, q.y, q.z, f.sp, jv, ju, rr)) return;
    const int j = jv * f.sp.cols + ju;
    const float4 P = __ldcg(f.spix + j);
    const float4 m = load_nw_cg(f.snrm, j, f.sprec);
    if (P.w == 0.0f || m.w == 0.0f) return;
    const float *r = T.r;
    const float px = fmaf(r[0], P.x, fmaf(r[1], P.y, fmaf(r[2], P.z, r[3])));
    const float py = fmaf(r[4], P.x, fmaf(r[5], P.y, fmaf(r[6], P.z, r[7])));
    const float pz = fmaf(r[8], P.x, fmaf(r[9], P.y, fmaf(r[10], P.z, r[11])));
    const float ex = px - s.x, ey = py - s.y, ez = pz - s.z;
    if (!(fmaf(ex, ex, fmaf(ey, ey, ez * ez)) <= f.d_max2)) return;
    const float3 Rm = rotate(T, m.x, m.y, m.z);
    if (!(fmaf(Rm.x, nk.x, fmaf(Rm.y, nk.y, Rm.z * nk.z)) >= f.cos_min)) return;
    const float dm = sqrtf(fmaf(px, px, fmaf(py, py, pz * pz)));
    const float inv = 1.0f / (w + 1.0f);
    f.kdepth[k] = fmaf(w, d, dm) * inv;
    const float nx = fmaf(w, nk.x, Rm.x), ny = fmaf(w, nk.y, Rm.y), nz = fmaf(w, nk.z, Rm.z);
    const float l = rsqrtf(fmaf(nx, nx, fmaf(ny, ny, nz * nz)));
    const float wn = w + 1.0f < f.w_max ? w + 1.0f : f.w_max;
    store_nw(f.knw, k, f.kprec, make_float4(nx * l, ny * l, nz * l, wn));
}

// Hole fill, first pass for sweep pixel j: its z-buffer key into the empty
// keyframe pixel it lands on.  Returns false when it lands on no empty pixel.
__device__ __forceinline__ bool holefill_key(const FuseView &f, const PoseF &T, int j, int &k,
                                             unsigned long long &key, float &range, float4 &m) {
    const float4 P = __ldcg(f.spix + j);
    m = load_nw_cg(f.snrm, j, f.sprec);  // read with the point (unused when the point is empty)
    if (P.w == 0.0f) return false;
    if (m.w == 0.0f) return false;
    const float3 p = xform(T, P.x, P.y, P.z);
    int v, u;
    if (!bin_point(p.x, p.y, p.z, f.kp, v, u, range)) return false;
    k = v * f.kp.cols + u;
    key = ((unsigned long long)__float_as_uint(range) << 32) | (unsigned int)j;
    return true;
}

// Hole fill, second pass: the winning sweep pixel writes the keyframe pixel
// (d = range, n = unit(R m), w = 1) and resets its z-buffer word.
__device__ __forceinline__ void holefill_write(const FuseView &f, const PoseF &T, int k, float range, float4 m) {
    f.zbuf[k] = 0xffffffffffffffffull;
    const float3 Rm = rotate(T, m.x, m.y, m.z);
    const float l = rsqrtf(fmaf(Rm.x, Rm.x, fmaf(Rm.y, Rm.y, Rm.z * Rm.z)));
    f.kdepth[k] = range;
    store_nw(f.knw, k, f.kprec, make_float4(Rm.x * l, Rm.y * l, Rm.z * l, 1.0f));
}

// ----------------------------------------------------------------------------- programmatic dependent launch
//
// Where one entry point runs several kernels in a row, the later ones are launched with
// launch_dependent: their CTAs may be placed while the kernel before them drains, and each runs
// pdl_wait() before it reads anything (the wait returns once the previous grid has finished and its
// writes are visible).  A kernel lets its successor start early with pdl_release(); without it the
// successor starts at its end, as an ordinary launch would.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

}  // namespace upslam

// ----------------------------------------------------------------------------- host helpers

#define UPSLAM_CHECK_LAUNCH()                                     \
    do {                                                          \
        if (cudaPeekAtLastError() != cudaSuccess) {               \
            (void)cudaGetLastError();                             \
            return UPSLAM_ERR_CUDA;                               \
        }                                                         \
    } while (0)

// A launch that may overlap the previous kernel on the stream (the kernel must call pdl_wait()
// before it reads that kernel's results).  False when the launch fails.
template <typename... KArgs, typename... Args>
static inline bool launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                    Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kernel, args...) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return true;
}

static inline bool upslam_pano_ok(const upslam_pano *pp) {
    return pp && pp->rows > 0 && pp->cols > 0 && (int64_t)pp->rows * pp->cols < (int64_t(1) << 31) &&
           pp->s_az > 0.0f && pp->s_el > 0.0f && pp->r_max >= pp->r_min;
}

static inline bool upslam_aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

static inline bool upslam_icp_params_ok(const upslam_icp_params *ip) {
    return ip && ip->d_max > 0.0f && ip->max_iters >= 0 && ip->min_inliers >= 0 &&
           (ip->loss == UPSLAM_LOSS_L2 || (ip->loss == UPSLAM_LOSS_L1 && ip->loss_delta > 0.0f)) &&
           ip->coarse_iters >= 0 && (ip->coarse_iters == 0 || ip->d_max_fine > 0.0f);
}

// Multiprocessor count of the current device, cached per device ordinal.  Any host thread may call
// the library, so the cache is atomic (every writer stores the same value).
static inline int upslam_sm_count() {
    static std::atomic<int> cache[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    int sms = cache[dev].load(std::memory_order_relaxed);
    if (sms == 0) {
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
        cache[dev].store(sms, std::memory_order_relaxed);
    }
    return sms;
}

// Grid for a grid-stride loop over `work` items: enough CTAs to fill every SM
// several times over, never more than the work needs.
static inline int upslam_grid(int64_t work, int threads, int per_sm = 8) {
    const int64_t want = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)upslam_sm_count() * per_sm;
    return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}
