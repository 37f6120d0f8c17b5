// Pose-proposal network: BF16 tensor-core training and inference kernels.
//
// Not in the paper: a learned initial guess for ICP under large motion.  A small
// network reads a keyframe/sweep pair downsampled to 64 x 256 (depth and normal
// of each, 8 channels) and predicts the relative pose xi = (omega, v); ICP
// (Sec. III-B) refines it, and a residual gate falls back to the plain prior.
//
//   x0 [B, 64, 256, 8] --conv3x3/s2+ReLU--> [B,32,128,32] --> [B,16,64,64]
//      --> [B,8,32,128] --> [B,4,16,128] --mean--> [B,128] --linear--> [B,6]
//
// Convolutions are GEMMs over im2col columns (reduction index (ky*3+kx)*Cin+ci):
//   forward  Y[M,N]  = cols[M,K] . W[N,K]^T          (+ bias, ReLU, BF16 out)
//   dW[N,K] += dY[M,N]^T . cols[M,K]                 (split-K, FP32 atomics)
//   dcols    = dY[M,N] . W[N,K]  -> col2im -> x ReLU mask -> dY of the layer below
// The GEMM is one kernel: 64x64x32 CTA tiles, four warps of 32x32, BF16
// operands staged in shared memory, mma.sync.m16n8k16 with FP32 accumulators.
// Parameters live as one FP32 master array (w0 b0 w1 b1 w2 b2 w3 b3 wf bf,
// weights [C_out][3][3][C_in], head [6][128]); BF16 copies of the conv weights
// (K padded to a multiple of 32) are what the GEMMs read.
#include <string.h>

#include "common.cuh"

namespace upslam {

constexpr int kCnnCh[5] = {8, 32, 64, 128, 128};
constexpr int kCnnH = 64, kCnnW = 256;

__host__ __device__ constexpr int cnn_k(int l) { return 9 * (l == 0 ? 8 : (l == 1 ? 32 : (l == 2 ? 64 : 128))); }
__host__ __device__ constexpr int cnn_kp(int l) { return (cnn_k(l) + 31) / 32 * 32; }
__host__ __device__ constexpr int cnn_co(int l) { return l == 0 ? 32 : (l == 1 ? 64 : 128); }

// ----------------------------------------------------------------------------- GEMM

enum { EPI_BIAS_RELU_BF16 = 0, EPI_F32 = 1, EPI_F32_ATOMIC = 2 };

struct GemmArgs {
    const __nv_bfloat16 *A;
    long long sam, sak;  // A(m, k) = A[m * sam + k * sak]
    const __nv_bfloat16 *B;
    long long sbn, sbk;  // B(n, k) = B[n * sbn + k * sbk]
    int M, N, K;
    int k_split;  // K per grid.z slice (multiple of 32)
    void *C;
    long long ldc;
    const float *bias;
};

__device__ __forceinline__ void mma_bf16(float c[4], const unsigned a[4], const unsigned b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int EPI>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
    constexpr int BM = 64, BN = 64, BK = 32, LD = BK + 8;
    __shared__ __align__(16) __nv_bfloat16 As[BM][LD];
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][LD];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kbeg = blockIdx.z * g.k_split, kend = min(g.K, kbeg + g.k_split);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int grp = lane >> 2, tg = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.0f;
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // stage the A and B tiles (generic strides; 8-wide vector loads when K is contiguous and aligned)
        if (g.sak == 1 && (g.sam % 8) == 0 && k0 + BK <= kend) {
            for (int i = tid; i < BM * (BK / 8); i += 128) {
                const int r = i / (BK / 8), c8 = (i % (BK / 8)) * 8;
                const int m = m0 + r;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (m < g.M) v = *reinterpret_cast<const uint4 *>(g.A + (long long)m * g.sam + k0 + c8);
                *reinterpret_cast<uint4 *>(&As[r][c8]) = v;
            }
        } else if (g.sam == 1 && (g.sak % 8) == 0 && m0 + BM <= g.M && k0 + BK <= kend) {
            // M contiguous: 8 consecutive rows of one column per 16-byte load, transposed into the tile
            for (int i = tid; i < (BM / 8) * BK; i += 128) {
                const int c = i / (BM / 8), r8 = (i % (BM / 8)) * 8;
                const uint4 v = *reinterpret_cast<const uint4 *>(g.A + (long long)(k0 + c) * g.sak + m0 + r8);
                const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) As[r8 + q][c] = e[q];
            }
        } else {
            for (int i = tid; i < BM * BK; i += 128) {
                const int r = i / BK, c = i % BK;
                const int m = m0 + r, k = k0 + c;
                As[r][c] = (m < g.M && k < kend) ? g.A[(long long)m * g.sam + (long long)k * g.sak] : zero;
            }
        }
        if (g.sbk == 1 && (g.sbn % 8) == 0 && k0 + BK <= kend) {
            for (int i = tid; i < BN * (BK / 8); i += 128) {
                const int r = i / (BK / 8), c8 = (i % (BK / 8)) * 8;
                const int n = n0 + r;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (n < g.N) v = *reinterpret_cast<const uint4 *>(g.B + (long long)n * g.sbn + k0 + c8);
                *reinterpret_cast<uint4 *>(&Bs[r][c8]) = v;
            }
        } else if (g.sbn == 1 && (g.sbk % 8) == 0 && n0 + BN <= g.N && k0 + BK <= kend) {
            // N contiguous: 8 consecutive columns of one k per 16-byte load, transposed into the tile
            for (int i = tid; i < (BN / 8) * BK; i += 128) {
                const int c = i / (BN / 8), r8 = (i % (BN / 8)) * 8;
                const uint4 v = *reinterpret_cast<const uint4 *>(g.B + (long long)(k0 + c) * g.sbk + n0 + r8);
                const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) Bs[r8 + q][c] = e[q];
            }
        } else {
            for (int i = tid; i < BN * BK; i += 128) {
                const int r = i / BK, c = i % BK;
                const int n = n0 + r, k = k0 + c;
                Bs[r][c] = (n < g.N && k < kend) ? g.B[(long long)n * g.sbn + (long long)k * g.sbk] : zero;
            }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + grp;
                af[i][0] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * tg]);
                af[i][1] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * tg]);
                af[i][2] = *reinterpret_cast<const unsigned *>(&As[r][kk + 2 * tg + 8]);
                af[i][3] = *reinterpret_cast<const unsigned *>(&As[r + 8][kk + 2 * tg + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + grp;
                bf[j][0] = *reinterpret_cast<const unsigned *>(&Bs[n][kk + 2 * tg]);
                bf[j][1] = *reinterpret_cast<const unsigned *>(&Bs[n][kk + 2 * tg + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    // epilogue: acc[i][j][c] is row wm + i*16 + grp (+8 for c >= 2), column wn + j*8 + 2*tg + (c & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = m0 + wm + i * 16 + grp + (c >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * tg + (c & 1);
                if (m >= g.M || n >= g.N) continue;
                const float v = acc[i][j][c];
                if (EPI == EPI_BIAS_RELU_BF16) {
                    reinterpret_cast<__nv_bfloat16 *>(g.C)[(long long)m * g.ldc + n] =
                        __float2bfloat16(fmaxf(v + g.bias[n], 0.0f));
                } else if (EPI == EPI_F32) {
                    reinterpret_cast<float *>(g.C)[(long long)m * g.ldc + n] = v;
                } else {
                    atomicAdd(reinterpret_cast<float *>(g.C) + (long long)m * g.ldc + n, v);
                }
            }
}

// ----------------------------------------------------------------------------- layout kernels

// [B,H,W,C] BF16 -> [B*H/2*W/2, Kp] BF16 columns of a 3x3 stride-2 pad-1 convolution (zero K padding).
__global__ void im2col_kernel(const __nv_bfloat16 *__restrict__ x, int B, int H, int W, int C, int Kp,
                              __nv_bfloat16 *__restrict__ cols) {
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)B * Ho * Wo * Kp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % Kp);
        const long long m = i / Kp;
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (k < 9 * C) {
            const int ci = k % C, tap = k / C, ky = tap / 3, kx = tap % 3;
            const int ox = (int)(m % Wo), oy = (int)((m / Wo) % Ho), b = (int)(m / ((long long)Wo * Ho));
            const int y = 2 * oy + ky - 1, xx = 2 * ox + kx - 1;
            if (y >= 0 && y < H && xx >= 0 && xx < W) v = x[(((long long)b * H + y) * W + xx) * C + ci];
        }
        cols[i] = v;
    }
}

// Adjoint of im2col followed by the ReLU mask of the layer's input (activation > 0):
// dy_in[b,y,x,c] = (x_in > 0) * sum over the (output pixel, tap) pairs that read (y, x) of dcols.
__global__ void col2im_mask_kernel(const float *__restrict__ dcols, int B, int H, int W, int C, int Kp,
                                   const __nv_bfloat16 *__restrict__ x_in, __nv_bfloat16 *__restrict__ dy_in) {
    const int Ho = H / 2, Wo = W / 2;
    const long long total = (long long)B * H * W * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const int xx = (int)((i / C) % W), y = (int)((i / ((long long)C * W)) % H);
        const int b = (int)(i / ((long long)C * W * H));
        float s = 0.0f;
        if (__bfloat162float(x_in[i]) > 0.0f) {
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int t = y + 1 - ky;
                if (t < 0 || (t & 1) || (t >> 1) >= Ho) continue;
                const int oy = t >> 1;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int u = xx + 1 - kx;
                    if (u < 0 || (u & 1) || (u >> 1) >= Wo) continue;
                    const int ox = u >> 1;
                    const long long m = ((long long)b * Ho + oy) * Wo + ox;
                    s += dcols[m * Kp + (ky * 3 + kx) * C + c];
                }
            }
        }
        dy_in[i] = __float2bfloat16(s);
    }
}

// Global mean over [B, HW, C] (BF16) -> g [B, C] (FP32), then the linear head out = g W^T + b.
__global__ void pool_head_kernel(const __nv_bfloat16 *__restrict__ x, int B, int HW, int C, const float *wf,
                                 const float *bf, float *g, float *out) {
    const int b = blockIdx.x;
    __shared__ float gs[128];
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.0f;
        for (int p = 0; p < HW; ++p) s += __bfloat162float(x[((long long)b * HW + p) * C + c]);
        gs[c] = s / HW;
        g[b * C + c] = s / HW;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        float o = bf[threadIdx.x];
        for (int c = 0; c < C; ++c) o += wf[threadIdx.x * C + c] * gs[c];
        out[b * 6 + threadIdx.x] = o;
    }
}

// Loss and the head's backward: dout = 2 w (out - t) / B; d wf += dout^T g; d bf += dout;
// dy4 = (dout wf) / HW broadcast over the last feature map, masked by its ReLU.
__global__ void head_backward_kernel(const float *out, const float *target, const float *w6, int B, const float *g,
                                     const float *wf, const __nv_bfloat16 *__restrict__ x4, int HW, int C,
                                     float *dwf, float *dbf, __nv_bfloat16 *__restrict__ dy4, float *loss) {
    const int b = blockIdx.x;
    __shared__ float dout[6], dg[128];
    if (threadIdx.x < 6) {
        const float diff = out[b * 6 + threadIdx.x] - target[b * 6 + threadIdx.x];
        dout[threadIdx.x] = 2.0f * w6[threadIdx.x] * diff / B;
        atomicAdd(loss, w6[threadIdx.x] * diff * diff / B);
        atomicAdd(dbf + threadIdx.x, dout[threadIdx.x]);
    }
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.0f;
        for (int i = 0; i < 6; ++i) {
            s += dout[i] * wf[i * C + c];
            atomicAdd(dwf + i * C + c, dout[i] * g[b * C + c]);
        }
        dg[c] = s / HW;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < HW * C; i += blockDim.x) {
        const long long idx = (long long)b * HW * C + i;
        dy4[idx] = __float2bfloat16(__bfloat162float(x4[idx]) > 0.0f ? dg[i % C] : 0.0f);
    }
}

// Column sums of dy [M, N] (BF16) added to db [N] (FP32).
__global__ void bias_grad_kernel(const __nv_bfloat16 *__restrict__ dy, int M, int N, float *db) {
    for (int col = threadIdx.x; col < N; col += blockDim.x) {
        float s = 0.0f;
        for (int m = blockIdx.x; m < M; m += gridDim.x) s += __bfloat162float(dy[(long long)m * N + col]);
        atomicAdd(db + col, s);
    }
}

// FP32 master weights -> BF16 conv weights with K padded to a multiple of 32.
__global__ void pack_weights_kernel(const float *w, int N, int K, int Kp, __nv_bfloat16 *wb) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * Kp; i += gridDim.x * blockDim.x) {
        const int n = i / Kp, k = i % Kp;
        wb[i] = __float2bfloat16(k < K ? w[n * K + k] : 0.0f);
    }
}

// Padded FP32 weight gradient [N][Kp] -> the master layout [N][K], added.
__global__ void unpad_grad_kernel(const float *gp, int N, int K, int Kp, float *gw) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N * K; i += gridDim.x * blockDim.x) {
        const int n = i / K, k = i % K;
        gw[i] += gp[n * Kp + k];
    }
}

// Adam (Kingma & Ba) on the FP32 master parameters, bias-corrected.
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Downsample a panorama (depth + normal with validity in .w) to out_rows x out_cols cells:
// channels (mean depth / depth_scale, mean nx, ny, nz) over the cell's valid pixels, 0 where none.
__global__ void downsample_kernel(const float *__restrict__ depth, const void *nrm, int prec, int H, int W, int oh,
                                  int ow, float depth_scale, __nv_bfloat16 *__restrict__ out, int c_stride,
                                  int c_off) {
    const int cell = blockIdx.x * blockDim.x + threadIdx.x;
    if (cell >= oh * ow) return;
    const int cy = cell / ow, cx = cell % ow;
    const int bh = H / oh, bw = W / ow;
    float sd = 0.f, sx = 0.f, sy = 0.f, sz = 0.f;
    int n = 0;
    for (int y = cy * bh; y < (cy + 1) * bh; ++y)
        for (int x = cx * bw; x < (cx + 1) * bw; ++x) {
            const int k = y * W + x;
            const float d = depth[k];
            const float4 v = load_nw(nrm, k, prec);
            if (d > 0.0f && v.w != 0.0f && (v.x != 0.0f || v.y != 0.0f || v.z != 0.0f)) {
                sd += d;
                sx += v.x;
                sy += v.y;
                sz += v.z;
                ++n;
            }
        }
    const float inv = n ? 1.0f / n : 0.0f;
    __nv_bfloat16 *o = out + (long long)cell * c_stride + c_off;
    o[0] = __float2bfloat16(sd * inv / depth_scale);
    o[1] = __float2bfloat16(sx * inv);
    o[2] = __float2bfloat16(sy * inv);
    o[3] = __float2bfloat16(sz * inv);
}

// ----------------------------------------------------------------------------- host side

struct CnnLayout {
    size_t off_w[4], off_b[4], off_wf, off_bf, count;
};

static CnnLayout cnn_layout() {
    CnnLayout L;
    size_t o = 0;
    for (int l = 0; l < 4; ++l) {
        L.off_w[l] = o;
        o += (size_t)cnn_co(l) * cnn_k(l);
        L.off_b[l] = o;
        o += cnn_co(l);
    }
    L.off_wf = o;
    o += 6 * 128;
    L.off_bf = o;
    o += 6;
    L.count = o;
    return L;
}

struct CnnWs {
    __nv_bfloat16 *wb[4];
    __nv_bfloat16 *act[4];  // outputs of the four conv layers
    __nv_bfloat16 *cols;
    __nv_bfloat16 *dy[4];
    float *dcols, *dwpad, *g, *out;
};

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t cnn_ws_layout(int B, CnnWs *w, char *base) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + o : nullptr;
        o = align_up(o + bytes);
        return p;
    };
    int H = kCnnH, W = kCnnW;
    size_t max_cols = 0, max_dcols = 0, max_dw = 0;
    for (int l = 0; l < 4; ++l) {
        const size_t M = (size_t)B * (H / 2) * (W / 2);
        if (w) w->wb[l] = reinterpret_cast<__nv_bfloat16 *>(take((size_t)cnn_co(l) * cnn_kp(l) * 2));
        else take((size_t)cnn_co(l) * cnn_kp(l) * 2);
        void *a = take(M * cnn_co(l) * 2);
        void *d = take(M * cnn_co(l) * 2);
        if (w) {
            w->act[l] = reinterpret_cast<__nv_bfloat16 *>(a);
            w->dy[l] = reinterpret_cast<__nv_bfloat16 *>(d);
        }
        max_cols = max_cols > M * cnn_kp(l) ? max_cols : M * cnn_kp(l);
        max_dcols = max_dcols > M * cnn_kp(l) ? max_dcols : M * cnn_kp(l);
        max_dw = max_dw > (size_t)cnn_co(l) * cnn_kp(l) ? max_dw : (size_t)cnn_co(l) * cnn_kp(l);
        H /= 2;
        W /= 2;
    }
    void *c = take(max_cols * 2);
    void *dc = take(max_dcols * 4);
    void *dw = take(max_dw * 4);
    void *g = take((size_t)B * 128 * 4);
    void *out = take((size_t)B * 6 * 4);
    if (w) {
        w->cols = reinterpret_cast<__nv_bfloat16 *>(c);
        w->dcols = reinterpret_cast<float *>(dc);
        w->dwpad = reinterpret_cast<float *>(dw);
        w->g = reinterpret_cast<float *>(g);
        w->out = reinterpret_cast<float *>(out);
    }
    return o;
}

static int grid1d(long long n, int t = 256) {
    const long long b = (n + t - 1) / t;
    const long long cap = (long long)upslam_sm_count() * 16;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

template <int EPI>
static void gemm(const GemmArgs &g0, cudaStream_t s, int splits = 1) {
    GemmArgs g = g0;
    const int per = ((g.K + splits - 1) / splits + 31) / 32 * 32;
    g.k_split = per;
    dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, (g.K + per - 1) / per);
    gemm_bf16_kernel<EPI><<<grid, 128, 0, s>>>(g);
}

}  // namespace upslam

using namespace upslam;

extern "C" size_t upslam_cnn_param_count(void) { return cnn_layout().count; }

extern "C" size_t upslam_cnn_workspace_bytes(int32_t batch) {
    if (batch <= 0) return 0;
    return cnn_ws_layout(batch, nullptr, nullptr);
}

extern "C" upslam_status upslam_cnn_forward(const float *d_params, const void *d_x, int32_t batch, float *d_out,
                                            void *d_ws, size_t ws_bytes, void *stream) {
    if (!d_params || !d_x || !d_out || !d_ws || batch <= 0 || !upslam_aligned(d_ws, 256) ||
        ws_bytes < upslam_cnn_workspace_bytes(batch) || !upslam_aligned(d_x, 16))
        return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CnnWs w;
    cnn_ws_layout(batch, &w, reinterpret_cast<char *>(d_ws));
    const CnnLayout L = cnn_layout();
    const __nv_bfloat16 *x = reinterpret_cast<const __nv_bfloat16 *>(d_x);
    int H = kCnnH, W = kCnnW;
    for (int l = 0; l < 4; ++l) {
        const int C = kCnnCh[l], N = cnn_co(l), K = cnn_k(l), Kp = cnn_kp(l);
        pack_weights_kernel<<<grid1d((long long)N * Kp), 256, 0, s>>>(d_params + L.off_w[l], N, K, Kp, w.wb[l]);
        const long long M = (long long)batch * (H / 2) * (W / 2);
        im2col_kernel<<<grid1d(M * Kp), 256, 0, s>>>(x, batch, H, W, C, Kp, w.cols);
        GemmArgs g;
        g.A = w.cols;
        g.sam = Kp;
        g.sak = 1;
        g.B = w.wb[l];
        g.sbn = Kp;
        g.sbk = 1;
        g.M = (int)M;
        g.N = N;
        g.K = Kp;
        g.C = w.act[l];
        g.ldc = N;
        g.bias = d_params + L.off_b[l];
        gemm<EPI_BIAS_RELU_BF16>(g, s);
        x = w.act[l];
        H /= 2;
        W /= 2;
    }
    pool_head_kernel<<<batch, 128, 0, s>>>(w.act[3], batch, H * W, 128, d_params + L.off_wf, d_params + L.off_bf, w.g,
                                           d_out);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_cnn_backward(const float *d_params, const void *d_x, int32_t batch,
                                             const float *d_out, const float *d_target, const float *d_wloss6,
                                             float *d_grads, float *d_loss, void *d_ws, size_t ws_bytes,
                                             void *stream) {
    if (!d_params || !d_x || !d_out || !d_target || !d_wloss6 || !d_grads || !d_loss || !d_ws || batch <= 0 ||
        !upslam_aligned(d_ws, 256) || !upslam_aligned(d_x, 16) || ws_bytes < upslam_cnn_workspace_bytes(batch))
        return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CnnWs w;
    cnn_ws_layout(batch, &w, reinterpret_cast<char *>(d_ws));
    const CnnLayout L = cnn_layout();
    if (cudaMemsetAsync(d_grads, 0, L.count * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(d_loss, 0, sizeof(float), s) != cudaSuccess)
        return UPSLAM_ERR_CUDA;
    // head: loss, d wf, d bf, and the gradient entering the last feature map (masked by its ReLU)
    head_backward_kernel<<<batch, 128, 0, s>>>(d_out, d_target, d_wloss6, batch, w.g, d_params + L.off_wf, w.act[3],
                                               4 * 16, 128, d_grads + L.off_wf, d_grads + L.off_bf, w.dy[3], d_loss);
    int Hs[4], Ws[4];
    {
        int H = kCnnH, W = kCnnW;
        for (int l = 0; l < 4; ++l) {
            Hs[l] = H;
            Ws[l] = W;
            H /= 2;
            W /= 2;
        }
    }
    for (int l = 3; l >= 0; --l) {
        const int C = kCnnCh[l], N = cnn_co(l), K = cnn_k(l), Kp = cnn_kp(l);
        const int H = Hs[l], W = Ws[l];
        const long long M = (long long)batch * (H / 2) * (W / 2);
        const __nv_bfloat16 *xin = l == 0 ? reinterpret_cast<const __nv_bfloat16 *>(d_x) : w.act[l - 1];
        im2col_kernel<<<grid1d(M * Kp), 256, 0, s>>>(xin, batch, H, W, C, Kp, w.cols);
        // d W (padded layout) = dY^T cols, split over the M reduction
        if (cudaMemsetAsync(w.dwpad, 0, (size_t)N * Kp * sizeof(float), s) != cudaSuccess) return UPSLAM_ERR_CUDA;
        GemmArgs gw;
        gw.A = w.dy[l];
        gw.sam = 1;
        gw.sak = N;
        gw.B = w.cols;
        gw.sbn = 1;
        gw.sbk = Kp;
        gw.M = N;
        gw.N = Kp;
        gw.K = (int)M;
        gw.C = w.dwpad;
        gw.ldc = Kp;
        gw.bias = nullptr;
        const int tiles = ((N + 63) / 64) * ((Kp + 63) / 64);
        int splits = (upslam_sm_count() * 4 + tiles - 1) / tiles;
        if ((long long)splits * 256 > M) splits = (int)((M + 255) / 256);
        gemm<EPI_F32_ATOMIC>(gw, s, splits < 1 ? 1 : splits);
        unpad_grad_kernel<<<grid1d((long long)N * K), 256, 0, s>>>(w.dwpad, N, K, Kp, d_grads + L.off_w[l]);
        bias_grad_kernel<<<upslam_sm_count() * 2, 128, 0, s>>>(w.dy[l], (int)M, N, d_grads + L.off_b[l]);
        if (l > 0) {
            // d cols = dY W, then col2im with the input activation's ReLU mask
            GemmArgs gd;
            gd.A = w.dy[l];
            gd.sam = N;
            gd.sak = 1;
            gd.B = w.wb[l];
            gd.sbn = 1;
            gd.sbk = Kp;
            gd.M = (int)M;
            gd.N = Kp;
            gd.K = N;
            gd.C = w.dcols;
            gd.ldc = Kp;
            gd.bias = nullptr;
            gemm<EPI_F32>(gd, s);
            col2im_mask_kernel<<<grid1d((long long)batch * H * W * C), 256, 0, s>>>(w.dcols, batch, H, W, C, Kp,
                                                                                    w.act[l - 1], w.dy[l - 1]);
        }
    }
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_cnn_adam(float *d_params, const float *d_grads, float *d_m, float *d_v, int32_t step,
                                         float lr, void *stream) {
    if (!d_params || !d_grads || !d_m || !d_v || step < 1) return UPSLAM_ERR_INVALID_ARG;
    const long long n = (long long)cnn_layout().count;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    adam_kernel<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(d_params, d_grads, d_m, d_v, n, lr, b1, b2, 1e-8f, c1,
                                                            c2);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_downsample(const float *d_depth, const void *d_nrm, int32_t precision,
                                           const upslam_pano *pp, int32_t out_rows, int32_t out_cols,
                                           float depth_scale, void *d_out, int32_t c_stride, int32_t c_off,
                                           void *stream) {
    if (!d_depth || !d_nrm || !pp || !upslam_pano_ok(pp) || !d_out || out_rows <= 0 || out_cols <= 0 ||
        pp->rows % out_rows || pp->cols % out_cols || c_stride < c_off + 4 || c_off < 0 || !(depth_scale > 0.0f) ||
        (precision != UPSLAM_F32 && precision != UPSLAM_F16))
        return UPSLAM_ERR_INVALID_ARG;
    const int cells = out_rows * out_cols;
    downsample_kernel<<<(cells + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        d_depth, d_nrm, precision, pp->rows, pp->cols, out_rows, out_cols, depth_scale,
        reinterpret_cast<__nv_bfloat16 *>(d_out), c_stride, c_off);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}
