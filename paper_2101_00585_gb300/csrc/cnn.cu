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
// Each convolution is a GEMM whose im2col operand (reduction index
// f = (ky*3+kx)*Cin+ci over pixel p) is gathered straight from the NHWC
// activation while it is staged, so no column matrix is ever stored:
//   forward  Y[p, n]  = sum_f cols(p, f) W[n, f]        (+ bias, ReLU, BF16 out)
//   dW[n, f]         += sum_p cols(p, f) dY[p, n]       (split over p, FP32 red)
//   dX[p', c]         = (x > 0) sum over the taps t that read input pixel p'
//                       of sum_n dY[p_t, n] W[n, t C + c]  (one GEMM per parity
//                       class of p', ReLU mask and BF16 store in the epilogue)
// All three run on one persistent kernel on the fifth-generation tensor cores
// (tcgen05.mma, FP32 accumulators in tensor memory); see gemm_tc_kernel.
// Parameters live as one FP32 master array (w0 b0 w1 b1 w2 b2 w3 b3 wf bf,
// weights [C_out][3][3][C_in], head [6][128]); BF16 copies of the conv weights
// are what the GEMMs read.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "common.cuh"

namespace upslam {

constexpr int kCnnCh[5] = {8, 32, 64, 128, 128};
constexpr int kCnnH = 64, kCnnW = 256;

__host__ __device__ constexpr int cnn_k(int l) { return 9 * (l == 0 ? 8 : (l == 1 ? 32 : (l == 2 ? 64 : 128))); }
__host__ __device__ constexpr int cnn_co(int l) { return l == 0 ? 32 : (l == 1 ? 64 : 128); }

// ----------------------------------------------------------------------------- tcgen05 GEMM
//
// C(m, n) = sum_k A(m, k) B(n, k).  Work is cut into units of one 128 x BN
// output tile and one slice of K (split-K; for the data gradient, one parity
// class); each persistent CTA walks the units blockIdx.x, blockIdx.x +
// gridDim.x, ... and, inside each, K in steps of 64, through a ring of S
// shared-memory stages shared by three warp roles (gemm_tc_kernel):
//   * one producer thread issues each step's TMA tensor-map loads (coordinates
//     outside the tensor read zeros), running ahead across unit boundaries;
//   * one thread issues the step's tcgen05.mma.kind::f16 (BF16 in, FP32
//     accumulate, K = 16 each) into one of two tensor-memory accumulators;
//   * epilogue warps read a finished accumulator with tcgen05.ld while the
//     next unit's MMAs fill the other one.
// Operand tiles are R rows (along M or N) x 64 (along K), written by TMA with
// a 128-, 64- or 32-byte swizzle and read through matching UMMA descriptors
// (K-major or MN-major; instruction descriptor bits 15/16 say which).  The
// im2col operands are the taps of a 3x3 stride-2 pad-1 convolution over an
// NHWC activation [B][H][W][C] (H, W, C powers of two), x[b][2oy+ky-1][2ox+kx-1][c],
// loaded as boxes that step 2 along W and H; the 8-channel first layer is read
// as a space-to-depth convolution instead (below).
// Every wait is bounded; a wait that gives up sets *err and the CTA stops.

enum { EPI_BIAS_RELU_BF16 = 0, EPI_F32_RED_T = 1, EPI_DGRAD_MASK_BF16 = 2 };
enum {
    LD_DY_TAPS_K = 4,   // TMA: dY rows of one tap (data gradient)
    LD_W_TAPS_MN = 5,   // TMA: W per tap, MN-major (data gradient)
    LD_IM2COL_KT = 6,   // TMA: im2col of an input with C >= 64, one tap's 64 channels per K step (forward)
    LD_DENSE_KT = 7,    // TMA: weights [N][K], K-major (forward)
    LD_IM2COL_MNT = 8,  // TMA: im2col of an input with C >= 64, MN-major (weight gradient)
    LD_DENSE_MNT = 9,   // TMA: dY [P][N], MN-major (weight gradient)
    LD_IM2COL_KT32 = 10,  // TMA: as LD_IM2COL_KT for C = 32 (two taps per K step, 64-byte swizzle)
    LD_IM2COL_MNT32 = 11,  // TMA: as LD_IM2COL_MNT for C = 32 (64-byte swizzle)
    LD_S2D_KT = 12,        // TMA: the 8-channel input as a 2x2 space-to-depth convolution (forward)
    LD_S2D_MNT = 13,       // TMA: the same, MN-major (weight gradient)
    LD_DENSE_MNT32 = 14    // TMA: dY [P][32], MN-major, 64-byte swizzle (weight gradient, N = 32)
};

// The first layer (C = 8) as a space-to-depth convolution.  Input pixels (2Y + dy, 2X + dx) form the
// 32-channel pixel (Y, X) with channel 16 dy + 8 dx + c, and the 3x3 stride-2 pad-1 convolution becomes a
// 2x2 stride-1 one over taps (ty, tx) at (oy + ty - 1, ox + tx - 1): feature f = 32 (2 ty + tx) + 16 dy +
// 8 dx + c carries the weight of tap (ky, kx) = (2 ty + dy - 1, 2 tx + dx - 1) and channel c, and is zero
// where ky or kx is -1 (56 of the 128 features).  No copy is made: the NHWC input read as [B][H][W/2][16]
// (pairs of pixels along W) gives, for one dy, 16 of a feature's 32 channels in one 32-byte box row.
// The first 16 features (tap (0, 0), dy = 0) are all unused, so the weight gradient reads its feature of
// ones (the bias gradient) there.
constexpr int kS2dK = 128;
__host__ __device__ inline int s2d_feature_source(int f) {  // the 3x3 feature of f, or -1
    const int tap = f >> 5, dy = (f >> 4) & 1, dx = (f >> 3) & 1, c = f & 7;
    const int ky = 2 * (tap >> 1) + dy - 1, kx = 2 * (tap & 1) + dx - 1;
    return ky < 0 || kx < 0 ? -1 : (3 * ky + kx) * 8 + c;
}

// Channels per im2col TMA box: 64 (128-byte swizzle) or 32 (64-byte swizzle).
template <int LD>
constexpr int tma_cb() { return LD == LD_IM2COL_KT32 || LD == LD_IM2COL_MNT32 ? 32 : 64; }

struct TcOperand {
    const __nv_bfloat16 *p;
    long long ld;    // dense and LD_W_TAPS_MN: elements between consecutive a
    int rows;        // extent along M (operand A) or N (operand B)
    int hs, ws, cs;  // im2col: log2 of the input's H, W, C; LD_DY_TAPS_K: log2 of dY's H, W, C
    int ones_row;    // weight gradient: feature index whose every element reads 1 (or -1: none)
    int kf;          // im2col: number of features (9 C)
    int nb;          // im2col and LD_DY_TAPS_K: number of images (a chunk loaded at image nb reads zeros)
};

// An appended feature of ones makes the weight-gradient GEMM also produce the bias gradient
// sum_p dY[p][n]; its source is this box of 64 pixels by 64 features, feature 0 = 1.
struct OnesBox {
    unsigned short v[64 * 64];
    constexpr OnesBox() : v() {
        for (int i = 0; i < 64; ++i) v[64 * i] = 0x3F80;
    }
};
static __device__ __align__(1024) const OnesBox kOnesBox;

struct TcGemm {
    TcOperand a, b;
    int M, N, K;
    int k_split;      // K per unit (multiple of 64)
    int mt, nt, units;
    void *C;
    long long ldc;    // EPI_F32_RED_T: C[n * ldc + m]; otherwise C[m * ldc + n]
    const float *bias;
    const __nv_bfloat16 *mask;  // EPI_DGRAD_MASK_BF16: the layer input, whose ReLU masks dX
    float *db;                  // EPI_F32_RED_T with a ones row: the bias gradient it feeds
    unsigned long long timeout_ns;  // limit of every mbarrier wait (global-timer nanoseconds)
    int withhold;  // test support: the MMA thread does not signal its first accumulator as full
    int s2d;       // EPI_F32_RED_T: row m is feature m of the space-to-depth first layer
};

constexpr int kTcBM = 128, kTcBK = 64;
constexpr unsigned kTcWaitIters = 1u << 26;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// UMMA shared-memory descriptor (start, leading and stride byte offsets) for a tile written by TMA with a
// swizzle (layout type in bits 61-63: 2 = 128-byte, 4 = 64-byte, 6 = 32-byte; tile aligned to the swizzle
// atom).  K-major: rows of one swizzle width, 8-row groups `sbo` apart, the leading offset unused.  MN-major:
// rows along K of one swizzle width, 8-row K groups `sbo` apart, atoms along M/N `lbo` apart.
__device__ __forceinline__ unsigned long long umma_desc_sw(unsigned addr, unsigned lbo, unsigned sbo, unsigned type) {
    return (unsigned long long)((addr >> 4) & 0x3FFFu) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((unsigned long long)type << 61);
}

__device__ __forceinline__ void mbar_expect_tx(unsigned mbar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// One TMA tile load of a 4-D tensor map into shared memory, completing on mbar (transaction bytes).
__device__ __forceinline__ void tma_load4(unsigned dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          unsigned mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}],"
        " [%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}

// The data gradient of a 3x3 stride-2 pad-1 convolution, without the column matrix: an input pixel
// (y, x) = (2i + py, 2j + px) is read by the taps ky = 1 (py = 0) or ky in {0, 2} (py = 1), and likewise kx,
// from output pixel ((y + 1 - ky) / 2, (x + 1 - kx) / 2).  Parity class q = 2 py + px has
// taps(q) = (1 + py)(1 + px) taps; its GEMM runs over i, j (M = B H/2 W/2) with k = t N + n (tap t of the
// class, output channel n):  dX(y, x, c) = sum_k dY(oy_t, ox_t, n) W[n][(3 ky_t + kx_t) C + c].
__device__ __forceinline__ int class_taps(int q) { return (1 + (q >> 1)) * (1 + (q & 1)); }
__device__ __forceinline__ void class_tap(int q, int t, int &ky, int &kx) {
    const int py = q >> 1, px = q & 1;
    const int ty = px ? (t >> 1) : t, tx = px ? (t & 1) : 0;
    ky = py ? 2 * ty : 1;
    kx = px ? 2 * tx : 1;
}

// Warps: 0-3 epilogue, 4 the TMA producer (one thread), 5 the MMA issue (one thread).
constexpr int kTcThreads = 32 * 6;

struct TcUnit {
    int r0a, r0b, kbeg, kend, nkt, cls;
};

// Unit u: output tile (and class, for the data gradient) and its slice of K.
template <int EPI, int BN>
__device__ __forceinline__ TcUnit tc_unit(const TcGemm &g, int u) {
    TcUnit t;
    if (EPI == EPI_DGRAD_MASK_BF16) {
        // the four classes of one row tile are consecutive units, so neighbouring CTAs write both halves of
        // each output line at about the same time; the class order rotates with the tile (by a function of the
        // tile alone, so the four units still cover the four classes) so that each CTA's units, gridDim.x
        // apart, cycle through the classes and their 1, 2, 2 or 4 taps of work
        const int tile = u >> 2;
        t.cls = ((u & 3) + (int)((4ll * tile) / gridDim.x)) & 3;
        t.r0a = tile * kTcBM;
        t.r0b = 0;
        t.kbeg = 0;
        t.kend = class_taps(t.cls) * g.K;
    } else {
        const int nt = u % g.nt, rest = u / g.nt;
        t.cls = 0;
        t.r0a = (rest % g.mt) * kTcBM;
        t.r0b = nt * BN;
        t.kbeg = (rest / g.mt) * g.k_split;
        t.kend = min(g.K, t.kbeg + g.k_split);
    }
    t.nkt = (t.kend - t.kbeg + kTcBK - 1) / kTcBK;
    return t;
}

// TMA loads of the A operand of one K step (tensor maps built on the host; coordinates past the tensor read as
// zeros).  The data gradient's:
//   A, LD_DY_TAPS_K: class pixels (b, i, j) from t.r0a by (tap, n) from k0: one box [128 rows][128 B] in the
//     128-byte-swizzled K-major layout (SBO 1024; an MMA's 16 k start 32 bytes further along the row); a tap's
//     offset pixels past dY read zeros;
//   B, LD_W_TAPS_MN, at stage + 16 KB: per 64 channels one box [64 k][128 B] (128-byte swizzle), or for
//     BN = 32 one box [64 k][64 B] (64-byte swizzle).
// The im2col operands of the forward and the weight gradient follow in the function's branches.
template <int LA>
__device__ __forceinline__ void tc_tma_a(unsigned stage, unsigned mbar, const TcOperand &a, const CUtensorMap *ma,
                                         const CUtensorMap *mo, const TcUnit &t, int k0) {
    if (LA == LD_S2D_KT || LA == LD_S2D_MNT) {
        // boxes of 16 features (one dy of a tap: 32-byte rows, 32-byte swizzle) over the NHWC input read as
        // [B][H][W/2][16], at (X, y) = (ox + tx - 1, 2 (oy + ty - 1) + dy); padding reads zeros.  Forward:
        // rows = 128 output pixels from t.r0a, the K step's 64 features = 4 boxes [128][32 B] 4 KB apart.
        // Weight gradient: k = 64 output pixels from k0, rows = the 128 features as 8 boxes [64][32 B] 2 KB
        // apart, the first box the feature of ones.
        constexpr bool FWD = LA == LD_S2D_KT;
        const int wo = a.ws - 1, ho = a.hs - 1;
        const int p0 = FWD ? t.r0a : k0;
        const int ox0 = p0 & ((1 << wo) - 1), oy0 = (p0 >> wo) & ((1 << ho) - 1), b0 = p0 >> (wo + ho);
#pragma unroll 1
        for (int h = 0; h < (FWD ? 4 : 8); ++h) {
            const int f = (FWD ? k0 : t.r0a) + 16 * h;
            const unsigned dst = stage + h * (FWD ? 4096 : 2048);
            if (!FWD && f == a.ones_row) {
                tma_load4(dst, mo, 0, 0, 0, 0, mbar);
                continue;
            }
            const int tap = f >> 5, dy = (f >> 4) & 1;
            tma_load4(dst, ma, 0, ox0 + (tap & 1) - 1, 2 * (oy0 + (tap >> 1) - 1) + dy, b0, mbar);
        }
        return;
    }
    if (LA == LD_IM2COL_MNT || LA == LD_IM2COL_MNT32) {
        // k: 64 pixels from k0; rows: features t.r0a.. as boxes of CB channels, [64 k][2 CB bytes] each, 128 CB
        // bytes apart (the appended feature of ones from mo; features past it read zeros from image nb)
        constexpr int CB = tma_cb<LA>();
        const int wo = a.ws - 1, ho = a.hs - 1;
        const int ox0 = k0 & ((1 << wo) - 1), oy0 = (k0 >> wo) & ((1 << ho) - 1), b0 = k0 >> (wo + ho);
#pragma unroll 1
        for (int h = 0; h < kTcBM / CB; ++h) {
            const int f = t.r0a + CB * h;
            if (f == a.ones_row) {
                tma_load4(stage + h * CB * 128, mo, 0, 0, 0, 0, mbar);
                continue;
            }
            int c0 = 0, c1 = 0, c2 = 0, c3 = a.nb;
            if (f < a.kf) {
                const int tap = f >> a.cs, ky = tap / 3, kx = tap - 3 * ky;
                c0 = f & ((1 << a.cs) - 1);
                c1 = 2 * ox0 + kx - 1;
                c2 = 2 * oy0 + ky - 1;
                c3 = b0;
            }
            tma_load4(stage + h * CB * 128, ma, c0, c1, c2, c3, mbar);
        }
        return;
    }
    if (LA == LD_IM2COL_KT || LA == LD_IM2COL_KT32) {
        // rows: 128 output pixels from t.r0a (whole output rows); k: 64 features as boxes of CB channels of one
        // tap ([128 rows][2 CB bytes], 8 KB apart when CB = 32), each stepping 2 along W and H from
        // (2 ox0 + kx - 1, 2 oy0 + ky - 1); the padding and features past 9 C read zeros
        constexpr int CB = tma_cb<LA>();
        const int wo = a.ws - 1, ho = a.hs - 1;
        const int ox0 = t.r0a & ((1 << wo) - 1), oy0 = (t.r0a >> wo) & ((1 << ho) - 1), b0 = t.r0a >> (wo + ho);
#pragma unroll 1
        for (int h = 0; h < kTcBK / CB; ++h) {
            const int f = k0 + CB * h;
            int c0 = 0, c1 = 0, c2 = 0, c3 = a.nb;
            if (f < a.kf) {
                const int tap = f >> a.cs, ky = tap / 3, kx = tap - 3 * ky;
                c0 = f & ((1 << a.cs) - 1);
                c1 = 2 * ox0 + kx - 1;
                c2 = 2 * oy0 + ky - 1;
                c3 = b0;
            }
            tma_load4(stage + h * 8192, ma, c0, c1, c2, c3, mbar);
        }
        return;
    }
    int ky, kx;
    class_tap(t.cls, k0 >> a.cs, ky, kx);
    const int doy = ((t.cls >> 1) + 1 - ky) >> 1, dox = ((t.cls & 1) + 1 - kx) >> 1;
    const int j0 = t.r0a & ((1 << a.ws) - 1), i0 = (t.r0a >> a.ws) & ((1 << a.hs) - 1), b0 = t.r0a >> (a.ws + a.hs);
    const int n0 = k0 & ((1 << a.cs) - 1);
    tma_load4(stage, ma, n0, j0 + dox, i0 + doy, b0, mbar);
}

template <int LB, int BN>
__device__ __forceinline__ void tc_tma_b(unsigned sb, unsigned mbar, const TcOperand &b, const CUtensorMap *mb,
                                         const TcUnit &t, int k0) {
    if (LB == LD_DENSE_KT) {
        // weights [N][K]: BN rows from t.r0b by 64 k from k0, one 128-byte-swizzled box
        tma_load4(sb, mb, k0, t.r0b, 0, 0, mbar);
        return;
    }
    if (LB == LD_DENSE_MNT32) {
        // dY [P][32]: k = 64 pixels from k0, rows = the 32 channels, one 64-byte-swizzled box
        tma_load4(sb, mb, t.r0b, k0, 0, 0, mbar);
        return;
    }
    if (LB == LD_DENSE_MNT) {
        // dY [P][N]: k = 64 pixels from k0, rows = channels from t.r0b in 64-channel boxes 8 KB apart
#pragma unroll 1
        for (int h = 0; h < BN / 64; ++h) tma_load4(sb + h * 8192, mb, t.r0b + 64 * h, k0, 0, 0, mbar);
        return;
    }
    // W[n][(3 ky + kx) C + c]: k = (tap, n) from k0, rows = c from t.r0b; boxes of 64 n by 64 c (32 c when
    // BN = 32), swizzled rows along k, one box per 64 channels
    int ky, kx;
    class_tap(t.cls, k0 >> b.cs, ky, kx);
    const int n0 = k0 & ((1 << b.cs) - 1);
#pragma unroll 1
    for (int h = 0; h < (BN + 63) / 64; ++h)
        tma_load4(sb + h * 8192, mb, (3 * ky + kx) * b.rows + t.r0b + 64 * h, n0, 0, 0, mbar);
}

// Stages that fit in about 100 KB of shared memory (two CTAs per SM), at most 8.
template <int BN>
constexpr int tc_stages() {
    return 102400 / ((kTcBM + BN) * kTcBK * 2) < 8 ? 102400 / ((kTcBM + BN) * kTcBK * 2) : 8;
}
template <int BN>
constexpr int tc_smem_bytes() { return tc_stages<BN>() * (kTcBM + BN) * kTcBK * 2; }


struct TcSync {
    unsigned long long full[8];   // producers -> MMA: a stage's copies landed (4 warp arrivals)
    unsigned long long empty[8];  // MMA -> producers: the stage's MMAs are done (tcgen05.commit)
    unsigned long long accf[2];   // MMA -> epilogue: an accumulator buffer holds a finished tile
    unsigned long long acce[2];   // epilogue -> MMA: the buffer has been read (4 warp arrivals)
    unsigned tmem_base;
    int abort;
};

__device__ __forceinline__ void mbar_init(unsigned mbar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// Bounded wait for the phase of the given parity: gives up early once another role has aborted, and aborts
// the CTA (error word set) after kTcTimeoutNs of global time.  (A suspend-time hint on try_wait, letting
// waiting warps sleep, measured no different from polling.)
constexpr unsigned long long kTcTimeoutNs = 2000000000ull;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity, volatile int *abort, int *err,
                                        unsigned long long timeout_ns) {
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63) {
            if (*abort) return false;
            const unsigned long long t = global_ns();
            if (t0 == 0) {
                t0 = t;
            } else if (t - t0 > timeout_ns) {
                *abort = 1;
                atomicExch(err, 1);
                return false;
            }
        }
    }
}

// The epilogue of one 128 x BN tile from tensor-memory columns [acc, acc + BN): warp w owns rows 32w..32w+31.
// sbias: the forward bias of the tile's BN columns, staged in shared memory.
template <int EPI, int BN>
__device__ __forceinline__ void tc_epilogue(const TcGemm &g, const TcUnit &cur, unsigned acc, int warp, int lane,
                                            const float *sbias) {
    const int m = cur.r0a + warp * 32 + lane;
    long long pix = 0;
    // the mask of up to 32 columns is loaded before the accumulator is read; wider tiles load the rest per group
    constexpr int PF = EPI == EPI_DGRAD_MASK_BF16 ? (BN < 32 ? BN : 32) / 8 : 1;
    uint4 xm[PF];
    if (EPI == EPI_DGRAD_MASK_BF16) {
        // row m = (b, i, j) of class cur.cls -> input pixel (b, 2i + py, 2j + px); its mask is loaded first
        const int hs = g.a.hs, ws = g.a.ws;
        const int j2 = m & ((1 << ws) - 1), i2 = (m >> ws) & ((1 << hs) - 1), b = m >> (ws + hs);
        pix = ((((long long)b << (hs + 1)) + 2 * i2 + (cur.cls >> 1)) << (ws + 1)) + 2 * j2 + (cur.cls & 1);
#pragma unroll
        for (int q = 0; q < PF; ++q)
            xm[q] = (m < g.M && cur.r0b + 8 * q < g.N)
                        ? __ldg(reinterpret_cast<const uint4 *>(g.mask + pix * g.ldc + cur.r0b + 8 * q))
                        : make_uint4(0, 0, 0, 0);
    }
    constexpr int CW = BN < 32 ? BN : 32;  // columns per tensor-memory wait
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += CW) {
        unsigned v[CW];
#pragma unroll
        for (int q = 0; q < CW / 8; ++q)
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(v[8 * q]), "=r"(v[8 * q + 1]), "=r"(v[8 * q + 2]), "=r"(v[8 * q + 3]), "=r"(v[8 * q + 4]),
                  "=r"(v[8 * q + 5]), "=r"(v[8 * q + 6]), "=r"(v[8 * q + 7])
                : "r"(acc + ((unsigned)(warp * 32) << 16) + (unsigned)(c0 + 8 * q)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (m >= g.M) continue;
#pragma unroll
        for (int q = 0; q < CW / 8; ++q) {
            const int n = cur.r0b + c0 + 8 * q;
            const unsigned *w = v + 8 * q;
            if (n >= g.N) continue;
            if (EPI == EPI_BIAS_RELU_BF16) {
                uint4 o;
                unsigned *ow = &o.x;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int c = c0 + 8 * q + 2 * jj;
                    const __nv_bfloat162 h =
                        __floats2bfloat162_rn(fmaxf(__uint_as_float(w[2 * jj]) + sbias[c], 0.0f),
                                              fmaxf(__uint_as_float(w[2 * jj + 1]) + sbias[c + 1], 0.0f));
                    ow[jj] = *reinterpret_cast<const unsigned *>(&h);
                }
                *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(g.C) + (long long)m * g.ldc + n) = o;
            } else if (EPI == EPI_DGRAD_MASK_BF16) {
                const uint4 mq = (c0 + 8 * q) / 8 < PF
                                     ? xm[((c0 + 8 * q) / 8) % PF]
                                     : __ldg(reinterpret_cast<const uint4 *>(g.mask + pix * g.ldc + n));
                const __nv_bfloat162 *xh = reinterpret_cast<const __nv_bfloat162 *>(&mq);
                uint4 o;
                unsigned *ow = &o.x;
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const float2 xv = __bfloat1622float2(xh[jj]);
                    const __nv_bfloat162 h =
                        __floats2bfloat162_rn(xv.x > 0.0f ? __uint_as_float(w[2 * jj]) : 0.0f,
                                              xv.y > 0.0f ? __uint_as_float(w[2 * jj + 1]) : 0.0f);
                    ow[jj] = *reinterpret_cast<const unsigned *>(&h);
                }
                *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(g.C) + pix * g.ldc + n) = o;
            } else if (m == g.a.ones_row) {
                // the appended feature of ones: sum_p dY[p][n], the bias gradient
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                    if (n + jj < g.N) atomicAdd(g.db + n + jj, __uint_as_float(w[jj]));
            } else {
                // (the space-to-depth first layer: its feature m is 3x3 feature s2d_feature_source(m), or unused)
                const int mc = g.s2d ? s2d_feature_source(m) : m;
                if (mc < 0) continue;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj)
                    if (n + jj < g.N)
                        atomicAdd(reinterpret_cast<float *>(g.C) + (long long)(n + jj) * g.ldc + mc,
                                  __uint_as_float(w[jj]));
            }
        }
    }
}

// Warp-specialised persistent GEMM, two CTAs per SM.  One producer thread (warp 4) issues each step's TMA
// loads into the S-stage ring, announcing the step's bytes on its full barrier; the MMA thread (warp 5, lane 0)
// waits for full, issues the stage's MMAs into one of two tensor-memory accumulators and commits them to the
// stage's empty barrier, and after a unit's last step to the accumulator's full barrier; the epilogue warps
// (0-3) drain one accumulator while the MMAs of the next unit fill the other, then arrive on its empty barrier.
template <int EPI, int BN, int LA, int LB>
__global__ void __launch_bounds__(kTcThreads, 2)
    gemm_tc_kernel(TcGemm g, int *err, const __grid_constant__ CUtensorMap tma_a,
                   const __grid_constant__ CUtensorMap tma_b, const __grid_constant__ CUtensorMap tma_one) {
    constexpr int S = tc_stages<BN>();
    static_assert(S >= 2 && S <= 8, "stage ring");
    constexpr int kA = kTcBM * kTcBK * 2, kStage = (kTcBM + BN) * kTcBK * 2;
    constexpr unsigned kTxBytes = (unsigned)kStage;  // TMA boxes are written in full (zeros outside)
    constexpr bool A_MN = LA == LD_IM2COL_MNT || LA == LD_IM2COL_MNT32 || LA == LD_S2D_MNT;
    constexpr bool B_MN = LB == LD_W_TAPS_MN || LB == LD_DENSE_MNT || LB == LD_DENSE_MNT32;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) TcSync sy;
    __shared__ float sbias[EPI == EPI_BIAS_RELU_BF16 ? BN : 1];
    const unsigned smem0 = smem_u32(tc_smem);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &sy.abort;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sy.tmem_base)),
                     "r"(2 * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < S; ++i) {
            mbar_init(smem_u32(&sy.full[i]), 1);
            mbar_init(smem_u32(&sy.empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&sy.accf[i]), 1);
            mbar_init(smem_u32(&sy.acce[i]), 4);
        }
        sy.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = sy.tmem_base;

    if (warp == 4) {
        // ---- producer (one thread)
        const bool tma_thread = lane == 0;
        int it = 0;
        bool ok = true;
        if (tma_thread) {
            for (int u = blockIdx.x; ok && u < g.units; u += gridDim.x) {
                const TcUnit t = tc_unit<EPI, BN>(g, u);
                for (int k = 0; k < t.nkt; ++k, ++it) {
                    const int st = it % S;
                    if (it >= S && !tc_wait(smem_u32(&sy.empty[st]), (unsigned)(((it / S) - 1) & 1), abort, err, g.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    const unsigned stage = smem0 + st * kStage, fb = smem_u32(&sy.full[st]);
                    const int k0 = t.kbeg + k * kTcBK;
                    mbar_expect_tx(fb, kTxBytes);
                    tc_tma_a<LA>(stage, fb, g.a, &tma_a, &tma_one, t, k0);
                    tc_tma_b<LB, BN>(stage + kA, fb, g.b, &tma_b, t, k0);
                }
            }
        }
        if (tma_thread && !ok) {
            // let the loads already issued land before the CTA's shared memory goes away
            for (int j = it > S ? it - S : 0; j < it; ++j)
                for (unsigned w = 0; w < kTcWaitIters; ++w) {
                    unsigned done;
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                        " selp.u32 %0, 1, 0, p;\n}\n"
                        : "=r"(done)
                        : "r"(smem_u32(&sy.full[j % S])), "r"((unsigned)((j / S) & 1))
                        : "memory");
                    if (done) break;
                }
        }
        __syncwarp();
    } else if (warp == 5) {
        // ---- MMA issue
        if (lane == 0) {
            // instruction descriptor: FP32 accumulator, BF16 A and B, majors, N = BN, M = 128
            const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((A_MN ? 1u : 0u) << 15) |
                                   ((B_MN ? 1u : 0u) << 16) | ((unsigned)(BN >> 3) << 17) |
                                   ((unsigned)(kTcBM >> 4) << 24);
            int it = 0, uc = 0;
            unsigned last_bar = 0, last_par = 0;
            bool ok = true;
            for (int u = blockIdx.x; ok && u < g.units; u += gridDim.x, ++uc) {
                const TcUnit t = tc_unit<EPI, BN>(g, u);
                const int b = uc & 1;
                if (uc >= 2 && !tc_wait(smem_u32(&sy.acce[b]), (unsigned)(((uc >> 1) - 1) & 1), abort, err, g.timeout_ns)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned acc = tmem + (unsigned)(b * BN);
                for (int k = 0; k < t.nkt; ++k, ++it) {
                    const int st = it % S;
                    if (!tc_wait(smem_u32(&sy.full[st]), (unsigned)((it / S) & 1), abort, err, g.timeout_ns)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const unsigned a0 = smem0 + st * kStage, b0 = a0 + kA;
                    const int k0 = t.kbeg + k * kTcBK;
                    const int nk = min(kTcBK / 16, (t.kend - k0 + 15) / 16);
                    for (int kk = 0; kk < nk; ++kk) {
                        // TMA tiles: A K-major 128-byte swizzle (an MMA's 16 k start 32 bytes along the row); B
                        // MN-major, 128-byte swizzle (BN >= 64: 8-row K groups 1024 B apart, 64-channel atoms
                        // 8 KB apart) or 64-byte swizzle (BN = 32: K groups 512 B apart); an MMA spans two K groups
                        const unsigned long long ad =
                            LA == LD_IM2COL_MNT ? umma_desc_sw(a0 + kk * 2048, 8192, 1024, 2)
                            // 64-byte swizzle: MN-major 8-row K groups 512 B apart, 32-feature atoms 4 KB apart;
                            // K-major: two 64-byte-row sub-tiles 8 KB apart, an MMA's 16 k 32 bytes along the row
                            : LA == LD_IM2COL_MNT32 ? umma_desc_sw(a0 + kk * 1024, 4096, 512, 4)
                            : LA == LD_IM2COL_KT32  ? umma_desc_sw(a0 + (kk >> 1) * 8192 + (kk & 1) * 32, 16, 512, 4)
                            // 32-byte swizzle: K-major, one [128][32 B] box per MMA (8-row groups 256 B
                            // apart); MN-major, 8-row K groups 256 B apart, 16-feature atoms 2 KB apart
                            : LA == LD_S2D_KT  ? umma_desc_sw(a0 + kk * 4096, 16, 256, 6)
                            : LA == LD_S2D_MNT ? umma_desc_sw(a0 + kk * 512, 2048, 256, 6)
                                                  : umma_desc_sw(a0 + kk * 32, 16, 1024, 2);
                        const unsigned long long bd =
                            LB == LD_DENSE_KT    ? umma_desc_sw(b0 + kk * 32, 16, 1024, 2)
                            : LB == LD_DENSE_MNT ? umma_desc_sw(b0 + kk * 2048, 8192, 1024, 2)
                            : LB == LD_DENSE_MNT32 ? umma_desc_sw(b0 + kk * 1024, 512, 512, 4)
                            : BN == 32           ? umma_desc_sw(b0 + kk * 1024, 512, 512, 4)
                                                 : umma_desc_sw(b0 + kk * 2048, 8192, 1024, 2);
                        const unsigned accum = (k > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                    tc_commit(smem_u32(&sy.empty[st]));
                    last_bar = smem_u32(&sy.empty[st]);
                    last_par = (unsigned)((it / S) & 1);
                }
                if (!ok) break;
                if (!(g.withhold && uc == 0)) tc_commit(smem_u32(&sy.accf[b]));
            }
            // after an abort (or with a withheld signal, which nothing else waits out), let the MMAs already
            // issued finish before the accumulators are freed
            if ((!ok || g.withhold) && last_bar) {
                for (unsigned w = 0; w < kTcWaitIters; ++w) {
                    unsigned done;
                    asm volatile(
                        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                        " selp.u32 %0, 1, 0, p;\n}\n"
                        : "=r"(done)
                        : "r"(last_bar), "r"(last_par)
                        : "memory");
                    if (done) break;
                }
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue
        if (EPI == EPI_BIAS_RELU_BF16) {
            // the forward tile spans all N (BN = N, one column tile): its bias is staged once per CTA, which
            // took the epilogue from 2.2 to 0.6 us per 128 x 32 tile (per-element bias loads before)
            for (int c = threadIdx.x; c < BN; c += 128) sbias[c] = c < g.N ? __ldg(g.bias + c) : 0.0f;
            asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
        }
        int uc = 0;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x, ++uc) {
            const TcUnit t = tc_unit<EPI, BN>(g, u);
            const int b = uc & 1;
            if (!tc_wait(smem_u32(&sy.accf[b]), (unsigned)((uc >> 1) & 1), abort, err, g.timeout_ns)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_epilogue<EPI, BN>(g, t, tmem + (unsigned)(b * BN), warp, lane, sbias);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sy.acce[b]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN) : "memory");
}

// ----------------------------------------------------------------------------- layout kernels

// Global mean over [B, HW, C = 128] (BF16) -> g [B, C] (FP32), then the linear head out = g W^T + b.
// 128 threads per sample: thread t sums channels 8 (t % 16) .. + 7 over pixels t / 16, t / 16 + 8, ... with
// 16-byte loads; the eight partial sums of each channel are folded in shared memory.
__global__ void __launch_bounds__(128) pool_head_kernel(const __nv_bfloat16 *__restrict__ x, int B, int HW, int C,
                                                        const float *wf, const float *bf, float *g, float *out) {
    const int b = blockIdx.x, t = threadIdx.x, c8 = (t & 15) * 8, p0 = t >> 4;
    __shared__ float part[8][128];
    __shared__ float gs[128];
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int p = p0; p < HW; p += 8) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(x + ((long long)b * HW + p) * C + c8));
        const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 f = __bfloat1622float2(h[q]);
            acc[2 * q] += f.x;
            acc[2 * q + 1] += f.y;
        }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) part[p0][c8 + q] = acc[q];
    __syncthreads();
    float sum = 0.0f;
#pragma unroll
    for (int r = 0; r < 8; ++r) sum += part[r][t];
    gs[t] = sum / HW;
    g[b * C + t] = sum / HW;
    __syncthreads();
    if (t < 6) {
        float o = bf[t];
        for (int c = 0; c < C; ++c) o += wf[t * C + c] * gs[c];
        out[b * 6 + t] = o;
    }
}

// Loss and the head's backward for kHeadB samples per block (C = 128 threads):
// dout = 2 w (out - t) / B; loss += sum w (out - t)^2 / B; d bf += dout; d wf += dout^T g (summed over the
// block's samples before one atomic per weight); dg[b][c] = (dout wf)[c] / HW, the gradient of every pixel
// of the last feature map before its ReLU mask.
constexpr int kHeadB = 8;
__global__ void __launch_bounds__(128) head_backward_kernel(const float *out, const float *target, const float *w6,
                                                            int B, const float *g, const float *wf, int HW,
                                                            float *dwf, float *dbf, float *dg, float *loss) {
    constexpr int C = 128;
    const int b0 = blockIdx.x * kHeadB;
    __shared__ float dout[kHeadB][6];
    __shared__ float lsum;
    const int t = threadIdx.x;
    if (t == 0) lsum = 0.0f;
    __syncthreads();
    if (t < kHeadB * 6) {
        const int j = t / 6, i = t % 6, b = b0 + j;
        float d = 0.0f, l = 0.0f;
        if (b < B) {
            const float diff = out[b * 6 + i] - target[b * 6 + i];
            d = 2.0f * w6[i] * diff / B;
            l = w6[i] * diff * diff / B;
        }
        dout[j][i] = d;
        atomicAdd(&lsum, l);
    }
    __syncthreads();
    if (t == 0) atomicAdd(loss, lsum);
    if (t < 6) {
        float sb = 0.0f;
        for (int j = 0; j < kHeadB; ++j) sb += dout[j][t];
        atomicAdd(dbf + t, sb);
    }
    float sw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int j = 0; j < kHeadB && b0 + j < B; ++j) {
        const float gv = g[(b0 + j) * C + t];
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            sw[i] += dout[j][i] * gv;
            s += dout[j][i] * wf[i * C + t];
        }
        dg[(b0 + j) * C + t] = s / HW;
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) atomicAdd(dwf + i * C + t, sw[i]);
}

// dy4[b][p][c] = (x4[b][p][c] > 0) * dg[b][c], 8 channels per thread (C = 128).
__global__ void __launch_bounds__(256) head_dy_kernel(const float *__restrict__ dg, const __nv_bfloat16 *__restrict__ x4,
                                                      int B, int HW, __nv_bfloat16 *__restrict__ dy4) {
    const int total = B * HW * 16;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int c = (i & 15) << 3, pix = i >> 4, b = pix / HW;
        const uint4 xm = __ldg(reinterpret_cast<const uint4 *>(x4) + i);
        const float4 lo = __ldg(reinterpret_cast<const float4 *>(dg + b * 128 + c));
        const float4 hi = __ldg(reinterpret_cast<const float4 *>(dg + b * 128 + c) + 1);
        const float v[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
        const __nv_bfloat162 *xh = reinterpret_cast<const __nv_bfloat162 *>(&xm);
        uint4 o;
        unsigned *ow = &o.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 xv = __bfloat1622float2(xh[q]);
            const __nv_bfloat162 h =
                __floats2bfloat162_rn(xv.x > 0.0f ? v[2 * q] : 0.0f, xv.y > 0.0f ? v[2 * q + 1] : 0.0f);
            ow[q] = *reinterpret_cast<const unsigned *>(&h);
        }
        reinterpret_cast<uint4 *>(dy4)[i] = o;
    }
}

// FP32 master conv weights [N][K] -> the BF16 copy the GEMMs read.
// The four layers' FP32 master weights -> their BF16 copies, in one launch.
struct PackArgs {
    const float *src[4];
    __nv_bfloat16 *dst[4];
    int n[4];
};
__global__ void pack_weights_kernel(PackArgs a) {
    const int total = a.n[0] + a.n[1] + a.n[2] + a.n[3];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        int l = 0, k = i;
        while (k >= a.n[l]) k -= a.n[l++];
        if (l == 0) {
            // the first layer in the space-to-depth order: row n, feature f (zero where unused)
            const int n = k / kS2dK, src = s2d_feature_source(k - n * kS2dK);
            a.dst[0][k] = __float2bfloat16(src < 0 ? 0.0f : a.src[0][n * cnn_k(0) + src]);
        } else {
            a.dst[l][k] = __float2bfloat16(a.src[l][k]);
        }
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
    __nv_bfloat16 *dy[4];
    float *g, *dg, *out;
    int *err;               // nonzero once a tensor-core wait gave up
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
    for (int l = 0; l < 4; ++l) {
        const size_t M = (size_t)B * (H / 2) * (W / 2);
        void *wb = take((size_t)cnn_co(l) * (l == 0 ? kS2dK : cnn_k(l)) * 2);  // the GEMM's weight layout
        void *a = take(M * cnn_co(l) * 2);
        void *d = take(M * cnn_co(l) * 2);
        if (w) {
            w->wb[l] = reinterpret_cast<__nv_bfloat16 *>(wb);
            w->act[l] = reinterpret_cast<__nv_bfloat16 *>(a);
            w->dy[l] = reinterpret_cast<__nv_bfloat16 *>(d);
        }
        H /= 2;
        W /= 2;
    }
    void *g = take((size_t)B * 128 * 4);
    void *dg = take((size_t)B * 128 * 4);
    void *out = take((size_t)B * 6 * 4);
    void *err = take(256);
    if (w) {
        w->g = reinterpret_cast<float *>(g);
        w->dg = reinterpret_cast<float *>(dg);
        w->out = reinterpret_cast<float *>(out);
        w->err = reinterpret_cast<int *>(err);
    }
    return o;
}

static int grid1d(long long n, int t = 256) {
    const long long b = (n + t - 1) / t;
    const long long cap = (long long)upslam_sm_count() * 16;
    return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

static int ilog2(int v) {
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// The operands of the layer whose input is [B][H][W][C].
static TcOperand op_im2col(const __nv_bfloat16 *x, int H, int W, int C) {
    TcOperand o;
    o.p = x;
    o.ld = 0;
    o.rows = 0;
    o.hs = ilog2(H);
    o.ws = ilog2(W);
    o.cs = ilog2(C);
    o.ones_row = -1;
    o.kf = 9 * C;
    o.nb = 0;
    return o;
}

static TcOperand op_dense(const __nv_bfloat16 *x, long long ld) {
    TcOperand o;
    o.p = x;
    o.ld = ld;
    o.rows = 0;
    o.hs = o.ws = o.cs = 0;
    o.ones_row = -1;
    o.kf = 0;
    o.nb = 0;
    return o;
}

// ----------------------------------------------------------------------------- tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder() {
    // looked up once per process (a driver entry point is the same for every device); atomic since
    // any host thread may call, and every writer stores the same pointer
    static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> cached{nullptr};
    PFN_cuTensorMapEncodeTiled_v12000 fn = cached.load(std::memory_order_acquire);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess) {
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
            cached.store(fn, std::memory_order_release);
        }
    }
    return fn;
}

// A 4-D BF16 tensor map: dims innermost first, byte strides of dims 1..3, box and element strides; out-of-range
// elements read as zeros.
static bool tmap4(CUtensorMap *m, const void *base, unsigned long long d0, unsigned long long d1, unsigned long long d2,
                  unsigned long long d3, unsigned long long s1, unsigned long long s2, unsigned long long s3,
                  const unsigned box[4], const unsigned estr[4],
                  CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t dims[4] = {d0, d1, d2, d3};
    const cuuint64_t strides[3] = {s1, s2, s3};
    const cuuint32_t bx[4] = {box[0], box[1], box[2], box[3]}, es[4] = {estr[0], estr[1], estr[2], estr[3]};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(base), dims, strides, bx, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dY [B][Ho][Wo][N] in boxes of 128 consecutive pixels by 64 channels (one 128-byte row per pixel), written
// with the 128-byte swizzle: one request per pixel row instead of eight.
static bool tmap_dy_tiles(CUtensorMap *m, const TcOperand &o) {
    const int Ho = 1 << o.hs, Wo = 1 << o.ws, N = 1 << o.cs;
    const int wb = Wo < 128 ? Wo : 128, hb = Ho < 128 / wb ? Ho : 128 / wb, nb = 128 / (wb * hb);
    const unsigned box[4] = {64u, (unsigned)wb, (unsigned)hb, (unsigned)nb}, estr[4] = {1, 1, 1, 1};
    return tmap4(m, o.p, N, Wo, Ho, o.nb, 2ull * N, 2ull * N * Wo, 2ull * N * Wo * Ho, box, estr,
                 CU_TENSOR_MAP_SWIZZLE_128B);
}

// An NHWC input [B][H][W][C] (C >= cb) seen by a 3x3 stride-2 convolution: boxes of 128 consecutive output
// pixels (128 for the forward, 64 for the weight gradient; whole output rows or part of one) by cb channels
// (64 or 32), stepping 2 along W and H, written with the 128-byte or 64-byte swizzle.
static bool tmap_im2col_wide(CUtensorMap *m, const TcOperand &o, int pix, int cb) {
    const int H = 1 << o.hs, W = 1 << o.ws, C = 1 << o.cs, Ho = H / 2, Wo = W / 2;
    const int wb = Wo < pix ? Wo : pix, hb = Ho < pix / wb ? Ho : pix / wb, nb = pix / (wb * hb);
    const unsigned box[4] = {(unsigned)cb, 2u * wb, 2u * hb, (unsigned)nb}, estr[4] = {1, 2, 2, 1};
    return tmap4(m, o.p, C, W, H, o.nb, 2ull * C, 2ull * C * W, 2ull * C * W * H, box, estr,
                 cb == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
}

// The 8-channel input [B][H][W][8] read as [B][H][W/2][16] for the space-to-depth first layer: boxes of `pix`
// consecutive pairs of pixels along one row (16 BF16, 32 bytes each), written with the 32-byte swizzle.
static bool tmap_s2d(CUtensorMap *m, const TcOperand &o, int pix) {
    const int H = 1 << o.hs, W = 1 << o.ws, C = 1 << o.cs;
    const unsigned box[4] = {16u, (unsigned)pix, 1u, 1u}, estr[4] = {1, 1, 1, 1};
    return tmap4(m, o.p, 16, W / 2, H, o.nb, 32ull, 2ull * C * W, 2ull * C * W * H, box, estr,
                 CU_TENSOR_MAP_SWIZZLE_32B);
}

// A row-major matrix [rows][cols] (cols contiguous) in boxes of `box_rows` rows by `box_cols` columns.
static bool tmap_matrix(CUtensorMap *m, const void *p, long long rows, long long cols, int box_rows, int box_cols,
                        CUtensorMapSwizzle swz) {
    const unsigned box[4] = {(unsigned)box_cols, (unsigned)box_rows, 1, 1}, estr[4] = {1, 1, 1, 1};
    return tmap4(m, p, cols, rows, 1, 1, 2ull * cols, 2ull * cols * rows, 2ull * cols * rows, box, estr, swz);
}

// The ones box's device address, per device (host code must not take the symbol itself as an address).
static const void *ones_box_address() {
    static std::atomic<const void *> addr[64];  // any host thread may call; writers store the same address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    const void *a = addr[dev].load(std::memory_order_acquire);
    if (!a) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, kOnesBox) != cudaSuccess) return nullptr;
        a = p;
        addr[dev].store(a, std::memory_order_release);
    }
    return a;
}

// C(m, n) = sum_k A(m, k) B(n, k) on the tensor cores, K cut into `splits` slices (rounded to 64).
// False when a tensor map cannot be built (nothing is launched then).
template <int EPI, int BN, int LA, int LB>
static bool gemm(TcGemm g, int *err, cudaStream_t s, int splits = 1) {
    constexpr int smem = tc_smem_bytes<BN>();
    // the dynamic shared-memory limit is a per-device attribute: raised once on each device (atomic
    // flags, since any host thread may call)
    static std::atomic<bool> attr[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    if (!attr[dev].load(std::memory_order_acquire)) {
        if (cudaFuncSetAttribute(gemm_tc_kernel<EPI, BN, LA, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem) != cudaSuccess)
            return false;
        attr[dev].store(true, std::memory_order_release);
    }
    if (g.timeout_ns == 0) g.timeout_ns = kTcTimeoutNs;
    g.a.rows = g.M;
    g.b.rows = g.N;
    g.k_split = ((g.K + splits - 1) / splits + kTcBK - 1) / kTcBK * kTcBK;
    const int z = (g.K + g.k_split - 1) / g.k_split;
    g.mt = (g.M + kTcBM - 1) / kTcBM;
    g.nt = (g.N + BN - 1) / BN;
    g.units = EPI == EPI_DGRAD_MASK_BF16 ? 4 * g.mt : g.mt * g.nt * z;  // four parity classes
    CUtensorMap ma, mb, mo;
    memset(&mo, 0, sizeof(mo));
    constexpr int CB = tma_cb<LA>();
    constexpr CUtensorMapSwizzle kSwzA = CB == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
    if (LA == LD_S2D_KT) {
        // forward of the first layer: the input in 128-pixel boxes, the weights [N][128] in BN-row boxes
        if (!tmap_s2d(&ma, g.a, kTcBM) || !tmap_matrix(&mb, g.b.p, g.N, g.b.ld, BN, 64, CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
    } else if (LA == LD_S2D_MNT) {
        // weight gradient of the first layer: the input in 64-pixel boxes, dY [P][32] in 64-pixel boxes, the
        // feature of ones from the constant box (its first 16 columns)
        const void *ones = ones_box_address();
        if (!ones || !tmap_s2d(&ma, g.a, kTcBK) ||
            !tmap_matrix(&mb, g.b.p, g.K, g.b.ld, kTcBK, 32, CU_TENSOR_MAP_SWIZZLE_64B) ||
            !tmap_matrix(&mo, ones, 64, 64, 64, 16, CU_TENSOR_MAP_SWIZZLE_32B))
            return false;
    } else if (LA == LD_IM2COL_MNT || LA == LD_IM2COL_MNT32) {
        // weight gradient with C >= 32: the input in 64-pixel boxes of CB channels, dY [P][N] in 64-pixel boxes
        // of 64 channels, the appended feature of ones from a constant box
        const void *ones = ones_box_address();
        if (!ones || !tmap_im2col_wide(&ma, g.a, kTcBK, CB) ||
            !tmap_matrix(&mb, g.b.p, g.K, g.b.ld, kTcBK, 64, CU_TENSOR_MAP_SWIZZLE_128B) ||
            !tmap_matrix(&mo, ones, 64, 64, 64, CB, kSwzA))
            return false;
    } else if (LA == LD_IM2COL_KT || LA == LD_IM2COL_KT32) {
        // forward with C >= 32: the input in 128-pixel boxes of CB channels, the weights [N][9 C] in BN-row boxes
        if (!tmap_im2col_wide(&ma, g.a, kTcBM, CB) ||
            !tmap_matrix(&mb, g.b.p, g.N, g.b.ld, BN, 64, CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
    } else {
        // data gradient: dY in 128-pixel tiles, W [N_out][9 C] in 64-row boxes
        const bool narrow = BN < 64;
        if (!tmap_dy_tiles(&ma, g.a) ||
            !tmap_matrix(&mb, g.b.p, 1 << g.b.cs, g.b.ld, kTcBK, narrow ? 32 : 64,
                         narrow ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B))
            return false;
    }
    const int cap = 2 * upslam_sm_count();  // persistent: two CTAs per SM
    gemm_tc_kernel<EPI, BN, LA, LB><<<g.units < cap ? g.units : cap, kTcThreads, smem, s>>>(g, err, ma, mb, mo);
    return true;
}

}  // namespace upslam

using namespace upslam;

extern "C" size_t upslam_cnn_param_count(void) { return cnn_layout().count; }

extern "C" size_t upslam_cnn_workspace_bytes(int32_t batch) {
    if (batch <= 0) return 0;
    return cnn_ws_layout(batch, nullptr, nullptr);
}

extern "C" size_t upslam_cnn_workspace_layout(int32_t batch, size_t *offsets16) {
    if (batch <= 0 || !offsets16) return 0;
    CnnWs w;
    char *const base = reinterpret_cast<char *>(256);  // any non-null base: offsets are relative to it
    const size_t total = cnn_ws_layout(batch, &w, base);
    auto off = [&](const void *p) { return (size_t)(reinterpret_cast<const char *>(p) - base); };
    for (int l = 0; l < 4; ++l) {
        offsets16[l] = off(w.wb[l]);
        offsets16[4 + l] = off(w.act[l]);
        offsets16[8 + l] = off(w.dy[l]);
    }
    offsets16[12] = off(w.g);
    offsets16[13] = off(w.dg);
    offsets16[14] = off(w.out);
    offsets16[15] = off(w.err);
    return total;
}

extern "C" size_t upslam_cnn_error_offset(int32_t batch) {
    if (batch <= 0) return 0;
    return cnn_ws_layout(batch, nullptr, nullptr) - 256;  // the last block of the layout
}

// The forward pass; timeout_ns / withhold (test support) go to the first layer's GEMM.
static upslam_status cnn_forward(const float *d_params, const void *d_x, int32_t batch, float *d_out, void *d_ws,
                                 size_t ws_bytes, void *stream, unsigned long long timeout_ns, int withhold) {
    if (!d_params || !d_x || !d_out || !d_ws || batch <= 0 || !upslam_aligned(d_ws, 256) ||
        ws_bytes < upslam_cnn_workspace_bytes(batch) || !upslam_aligned(d_x, 16))
        return UPSLAM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CnnWs w;
    cnn_ws_layout(batch, &w, reinterpret_cast<char *>(d_ws));
    const CnnLayout L = cnn_layout();
    const __nv_bfloat16 *x = reinterpret_cast<const __nv_bfloat16 *>(d_x);
    PackArgs pk;
    int n_w = 0;
    for (int l = 0; l < 4; ++l) {
        pk.src[l] = d_params + L.off_w[l];
        pk.dst[l] = w.wb[l];
        pk.n[l] = cnn_co(l) * (l == 0 ? kS2dK : cnn_k(l));
        n_w += pk.n[l];
    }
    pack_weights_kernel<<<grid1d(n_w), 256, 0, s>>>(pk);
    int H = kCnnH, W = kCnnW;
    for (int l = 0; l < 4; ++l) {
        const int C = kCnnCh[l], N = cnn_co(l), K = l == 0 ? kS2dK : cnn_k(l);
        TcGemm g{};
        g.a = op_im2col(x, H, W, C);
        g.a.nb = batch;
        g.b = op_dense(w.wb[l], K);
        g.M = batch * (H / 2) * (W / 2);
        g.N = N;
        g.K = K;
        g.C = w.act[l];
        g.ldc = N;
        g.bias = d_params + L.off_b[l];
        if (l == 0) {
            g.timeout_ns = timeout_ns;
            g.withhold = withhold;
        }
        // the staged-bias epilogue needs one column tile: BN = N
        // layers with C >= 32 load through TMA (128- or 64-byte swizzle); the 8-channel input as the 2x2
        // space-to-depth convolution (32-byte swizzle)
        const bool ok = C >= 64   ? gemm<EPI_BIAS_RELU_BF16, 128, LD_IM2COL_KT, LD_DENSE_KT>(g, w.err, s)
                        : C == 32 ? gemm<EPI_BIAS_RELU_BF16, 64, LD_IM2COL_KT32, LD_DENSE_KT>(g, w.err, s)
                                  : gemm<EPI_BIAS_RELU_BF16, 32, LD_S2D_KT, LD_DENSE_KT>(g, w.err, s);
        if (!ok) return UPSLAM_ERR_CUDA;
        x = w.act[l];
        H /= 2;
        W /= 2;
    }
    pool_head_kernel<<<batch, 128, 0, s>>>(w.act[3], batch, H * W, 128, d_params + L.off_wf, d_params + L.off_bf, w.g,
                                           d_out);
    UPSLAM_CHECK_LAUNCH();
    return UPSLAM_OK;
}

extern "C" upslam_status upslam_cnn_forward(const float *d_params, const void *d_x, int32_t batch, float *d_out,
                                            void *d_ws, size_t ws_bytes, void *stream) {
    return cnn_forward(d_params, d_x, batch, d_out, d_ws, ws_bytes, stream, 0, 0);
}

extern "C" upslam_status upslam_cnn_forward_wait_probe(const float *d_params, const void *d_x, int32_t batch,
                                                       float *d_out, void *d_ws, size_t ws_bytes,
                                                       unsigned long long timeout_ns, void *stream) {
    if (timeout_ns < 1000 || timeout_ns > kTcTimeoutNs) return UPSLAM_ERR_INVALID_ARG;
    return cnn_forward(d_params, d_x, batch, d_out, d_ws, ws_bytes, stream, timeout_ns, 1);
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
    head_backward_kernel<<<(batch + kHeadB - 1) / kHeadB, 128, 0, s>>>(d_out, d_target, d_wloss6, batch, w.g,
                                                                       d_params + L.off_wf, 4 * 16,
                                                                       d_grads + L.off_wf, d_grads + L.off_bf, w.dg,
                                                                       d_loss);
    head_dy_kernel<<<grid1d((long long)batch * 64 * 16), 256, 0, s>>>(w.dg, w.act[3], batch, 4 * 16, w.dy[3]);
    const int sms = upslam_sm_count();
    for (int l = 3; l >= 0; --l) {
        const int C = kCnnCh[l], N = cnn_co(l), K = cnn_k(l);
        const int H = kCnnH >> l, W = kCnnW >> l;
        const int P = batch * (H / 2) * (W / 2);
        const __nv_bfloat16 *xin = l == 0 ? reinterpret_cast<const __nv_bfloat16 *>(d_x) : w.act[l - 1];
        // dW[n][f] += sum_p cols(p, f) dY[p][n]: M = f (im2col, MN-major), N = n (dY, MN-major), K = p;
        // an appended feature f = K of ones yields db[n] = sum_p dY[p][n] in the same GEMM
        TcGemm gw{};
        gw.a = op_im2col(xin, H, W, C);
        gw.a.nb = batch;
        gw.a.ones_row = K;
        gw.db = d_grads + L.off_b[l];
        gw.b = op_dense(w.dy[l], N);
        gw.M = K + 1;
        gw.N = N;
        gw.K = P;
        gw.C = d_grads + L.off_w[l];
        gw.ldc = K;
        gw.bias = nullptr;
        // enough slices for two CTAs per SM, each at least 16 K tiles deep
        const int tiles = (K + 1 + kTcBM - 1) / kTcBM;
        const int ktiles = (P + kTcBK - 1) / kTcBK;
        int splits = (2 * sms + tiles - 1) / tiles;
        if (splits > ktiles / 16) splits = ktiles / 16;
        if (splits < 1) splits = 1;
        // layers with C >= 32 load through TMA (128- or 64-byte swizzle); the 8-channel input as the 2x2
        // space-to-depth convolution, its 128 features one M tile with the feature of ones at 0 (unused there)
        if (C == 8) {
            gw.M = kS2dK;
            gw.a.ones_row = 0;
            gw.s2d = 1;
        }
        const bool okw = C >= 64   ? gemm<EPI_F32_RED_T, 128, LD_IM2COL_MNT, LD_DENSE_MNT>(gw, w.err, s, splits)
                         : C == 32 ? gemm<EPI_F32_RED_T, 64, LD_IM2COL_MNT32, LD_DENSE_MNT>(gw, w.err, s, splits)
                                   : gemm<EPI_F32_RED_T, 32, LD_S2D_MNT, LD_DENSE_MNT32>(gw, w.err, s, splits);
        if (!okw) return UPSLAM_ERR_CUDA;
        if (l > 0) {
            // dY of the layer below = its ReLU mask x sum over the taps that read each input pixel of dY W,
            // one GEMM per parity class of the input pixels (no column matrix)
            TcGemm gd{};
            gd.a = op_dense(w.dy[l], N);
            gd.a.nb = batch;
            gd.a.hs = ilog2(H / 2);
            gd.a.ws = ilog2(W / 2);
            gd.a.cs = ilog2(N);
            gd.b = op_dense(w.wb[l], K);
            gd.b.cs = ilog2(N);
            gd.M = P;
            gd.N = C;
            gd.K = N;  // per tap
            gd.C = w.dy[l - 1];
            gd.ldc = C;
            gd.mask = w.act[l - 1];
            const bool okd = C == 32   ? gemm<EPI_DGRAD_MASK_BF16, 32, LD_DY_TAPS_K, LD_W_TAPS_MN>(gd, w.err, s)
                             : C == 64 ? gemm<EPI_DGRAD_MASK_BF16, 64, LD_DY_TAPS_K, LD_W_TAPS_MN>(gd, w.err, s)
                                       : gemm<EPI_DGRAD_MASK_BF16, 128, LD_DY_TAPS_K, LD_W_TAPS_MN>(gd, w.err, s);
            if (!okd) return UPSLAM_ERR_CUDA;
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
