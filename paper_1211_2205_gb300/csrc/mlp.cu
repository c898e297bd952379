// Learned order-8 closure: the per-cell perceptron 38 -> 128 -> 128 -> 9
// (tanh hidden layers) on the tensor cores (BF16 operands, FP32
// accumulation), its training kernels, and its use inside the step.
//
// Network input at a cell centre: the 36 moments of order <= 7 averaged to
// the centre from their own staggered grid, divided by their RMS s, then
// log(1 + sigma_a), log(1 + sigma_s0).  Output y (9 values) times s gives the
// order-8 moments R_8^{8,6,4,2,0}, I_8^{8,6,4,2} at the centre; R_8^m are
// written at the cell centres (grid G11), I_8^m at the points of G22 as the
// mean of the four surrounding centres.  The closed system is the P_8 system
// of section 3 with the order-8 components frozen in the even passes and set
// by the network before every odd half-step, so the order-7 rows see
// predicted order-8 moments instead of the zero of the P_7 truncation.
//
// Inference (k_forward, k_closure): one warp per 16 samples with the
// activations in registers (see warp_mlp).  Training (k_loss_grad): one CTA
// of 8 warps per tile of 128 samples, activations and their gradients in
// shared memory (the weight gradients contract over the samples).  Both
// use mma.sync m16n8k16 with fragments loaded by ldmatrix from padded
// shared-memory rows (no bank conflicts).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <utility>

#include "closure_features.cuh"
#include "internal.h"
#include "mlp.h"
#include "pdl.h"

namespace starmap {
namespace mlp {

namespace {

constexpr int ROWS = 128;          // samples per tile
constexpr int WARPS = 8;           // 16 samples per warp
constexpr int THREADS = WARPS * 32;
constexpr int KX = 48;             // input width rounded up to the mma k (16)
constexpr int LDO = 24;            // padded row of dY (16 used)

struct Smem {
    Packed w;
    __nv_bfloat16 X[ROWS * LDX];
    __nv_bfloat16 H1[ROWS * LDH];
    __nv_bfloat16 H2[ROWS * LDH];
};
// backward buffers behind Smem (training kernel only)
struct SmemBack {
    __nv_bfloat16 dY[ROWS * LDO];
    __nv_bfloat16 dZ2[ROWS * LDH];
    __nv_bfloat16 dZ1[ROWS * LDH];
    float wloss[WARPS];
};
static_assert(sizeof(Packed) % 16 == 0, "packed weights must keep 16-byte rows");
static_assert(sizeof(Smem) % 16 == 0, "shared layout must keep 16-byte rows");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(su32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(su32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(su32(p)));
}
// D += A (16x16 bf16, row-major) * B (16x8 bf16, column-major), FP32 accumulate
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// A fragment: 16x16 tile at (r0, c0) of a row-major matrix
__device__ __forceinline__ void frag_a(uint32_t (&a)[4], const __nv_bfloat16* M, int ld, int r0, int c0, int lane) {
    ldsm_x4(a, M + (r0 + (lane & 15)) * ld + c0 + (lane >> 4) * 8);
}
// B fragments of the two 8-column tiles n0, n0 + 8 at k0, from a matrix
// stored [n][k] (a weight matrix [out][in]): b[0..1] tile n0, b[2..3] tile n0 + 8
__device__ __forceinline__ void frag_b_nk(uint32_t (&b)[4], const __nv_bfloat16* W, int ld, int n0, int k0, int lane) {
    const int n = n0 + (lane & 7) + ((lane >> 4) << 3);
    const int k = k0 + ((lane >> 3) & 1) * 8;
    ldsm_x4(b, W + n * ld + k);
}
// B fragment of one 8-column tile from a matrix stored [k][n]
__device__ __forceinline__ void frag_b_kn(uint32_t (&b)[2], const __nv_bfloat16* M, int ld, int k0, int n0, int lane) {
    const int k = k0 + (lane & 7) + ((lane >> 3) & 1) * 8;
    ldsm_x2_t(b, M + k * ld + n0);
}
// A fragment of the tile (m0, k0) of A = S^T, S stored [k][m]
__device__ __forceinline__ void frag_a_t(uint32_t (&a)[4], const __nv_bfloat16* S, int ld, int m0, int k0, int lane) {
    const int k = k0 + (lane & 7) + ((lane >> 4) << 3);
    const int m = m0 + ((lane >> 3) & 1) * 8;
    ldsm_x4_t(a, S + k * ld + m);
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// Hidden-layer activation of two pre-activations: rounded to BF16, then
// the hardware tanh on the BF16 pair (the result is the packed BF16 pair
// the next layer consumes).  Training and inference share it, so a trained
// network is evaluated with the function it was trained on.
__device__ __forceinline__ uint32_t act2(float lo, float hi) {
    const uint32_t x = pack_bf16(lo, hi);
    uint32_t y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

__device__ void load_weights(Packed& dst, const Packed* src) {
    const uint4* s = reinterpret_cast<const uint4*>(src);
    uint4* d = reinterpret_cast<uint4*>(&dst);
    for (int i = threadIdx.x; i < (int)(sizeof(Packed) / 16); i += blockDim.x) d[i] = s[i];
}

// Hidden layer of this warp's 16 rows: Hout = tanh(A W^T + b), 128 outputs.
__device__ void dense_tanh(const __nv_bfloat16* A, int lda, int kdim, const __nv_bfloat16* W, int ldw,
                           const float* bias, __nv_bfloat16* Hout, int warp, int lane) {
    const int r0 = warp * 16;
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll 1
    for (int nb = 0; nb < HID; nb += 32) {
        float acc[4][4];
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
#pragma unroll 2
        for (int k0 = 0; k0 < kdim; k0 += 16) {
            uint32_t a[4], b01[4], b23[4];
            frag_a(a, A, lda, r0, k0, lane);
            frag_b_nk(b01, W, ldw, nb, k0, lane);
            frag_b_nk(b23, W, ldw, nb + 16, k0, lane);
            mma16816(acc[0], a, b01[0], b01[1]);
            mma16816(acc[1], a, b01[2], b01[3]);
            mma16816(acc[2], a, b23[0], b23[1]);
            mma16816(acc[3], a, b23[2], b23[3]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int c = nb + t * 8 + 2 * tg;
            const float bl = bias[c], bh = bias[c + 1];
            *reinterpret_cast<uint32_t*>(Hout + (r0 + g) * LDH + c) = act2(acc[t][0] + bl, acc[t][1] + bh);
            *reinterpret_cast<uint32_t*>(Hout + (r0 + g + 8) * LDH + c) = act2(acc[t][2] + bl, acc[t][3] + bh);
        }
    }
}

// Output layer of this warp's rows: y = H2 W3^T + b3 in registers.  y[t][e]:
// tile t (columns 8t..8t+7), e = 0,1 row g columns 2tg, 2tg+1; e = 2,3 row g+8.
__device__ void dense_out(const Smem& S, int warp, int lane, float (&y)[2][4]) {
    const int r0 = warp * 16;
    const int tg = lane & 3;
#pragma unroll
    for (int t = 0; t < 2; ++t) y[t][0] = y[t][1] = y[t][2] = y[t][3] = 0.f;
#pragma unroll 2
    for (int k0 = 0; k0 < HID; k0 += 16) {
        uint32_t a[4], b[4];
        frag_a(a, S.H2, LDH, r0, k0, lane);
        frag_b_nk(b, S.w.W3, LDH, 0, k0, lane);
        mma16816(y[0], a, b[0], b[1]);
        mma16816(y[1], a, b[2], b[3]);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int c = t * 8 + 2 * tg;
        y[t][0] += S.w.b3[c]; y[t][1] += S.w.b3[c + 1];
        y[t][2] += S.w.b3[c]; y[t][3] += S.w.b3[c + 1];
    }
}

// The three layers of one tile whose inputs sit in S.X.
__device__ __forceinline__ void network(Smem& S, int warp, int lane, float (&y)[2][4]) {
    dense_tanh(S.X, LDX, KX, S.w.W1, LDX, S.w.b1, S.H1, warp, lane);
    __syncwarp();
    dense_tanh(S.H1, LDH, HID, S.w.W2, LDH, S.w.b2, S.H2, warp, lane);
    __syncwarp();
    dense_out(S, warp, lane, y);
}

// Stage rows row0.. of X (FP32 [M][38]) into S.X as BF16, zero-padded.
__device__ void stage_inputs(Smem& S, const float* __restrict__ X, const int* __restrict__ idx, long row0, long M) {
    for (int i = threadIdx.x; i < ROWS * LDX; i += THREADS) {
        const int r = i / LDX, c = i % LDX;
        const long m = row0 + r;
        float v = 0.f;
        if (m < M && c < NIN) {
            const long src = idx ? (long)idx[m] : m;
            v = X[src * NIN + c];
        }
        S.X[i] = __float2bfloat16_rn(v);
    }
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

// ------------------------------------------------ register-resident inference
// One warp evaluates the network for 32 samples (two 16-row blocks) with
// the activations in registers: each layer's accumulator fragments become,
// after bias and activation, the A fragments of the next layer (the m16n8
// accumulator layout of two adjacent 8-column tiles is the m16k16 A
// layout).  Layers are computed 16 output columns at a time, so every
// weight fragment read from shared memory serves both row blocks.  The
// inputs come from a per-warp shared tile of 32 rows (ldmatrix).  Warps run
// independent persistent loops, so the input gathers of some warps overlap
// the tensor work of others.
constexpr int IW = 8;                   // warps per inference CTA
constexpr int ITHREADS = IW * 32;
constexpr int IROWS = 32;               // samples per warp and tile

struct InferSmem {
    Packed w;
    __nv_bfloat16 X[IW][IROWS * LDX];  // per-warp input tile
    float scale[IW][IROWS];
};

// Bias + activation of accumulator pair (tile 2np, 2np + 1) into A fragments
__device__ __forceinline__ void act_frag(uint32_t (&h)[4], const float (&a0)[4], const float (&a1)[4], const float* bias,
                                         int np, int tg) {
    const float2 bA = *reinterpret_cast<const float2*>(bias + np * 16 + 2 * tg);
    const float2 bB = *reinterpret_cast<const float2*>(bias + np * 16 + 8 + 2 * tg);
    h[0] = act2(a0[0] + bA.x, a0[1] + bA.y);
    h[1] = act2(a0[2] + bA.x, a0[3] + bA.y);
    h[2] = act2(a1[0] + bB.x, a1[1] + bB.y);
    h[3] = act2(a1[2] + bB.x, a1[3] + bB.y);
}

// y[mb][t][e]: row block mb, output tile t (columns 8t..8t+7); e = 0, 1:
// row g, columns 2tg, 2tg+1; e = 2, 3: row g + 8.
__device__ __forceinline__ void warp_mlp32(const Packed& W, const __nv_bfloat16* Xs, float (&y)[2][2][4], int lane) {
    const int tg = lane & 3;
    uint32_t h1[2][8][4];
    {
        uint32_t xa[2][3][4];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int kb = 0; kb < 3; ++kb) frag_a(xa[mb][kb], Xs, LDX, 16 * mb, 16 * kb, lane);
#pragma unroll
        for (int np = 0; np < 8; ++np) {
            float acc[2][2][4] = {};
#pragma unroll
            for (int kb = 0; kb < 3; ++kb) {
                uint32_t b[4];
                frag_b_nk(b, W.W1, LDX, np * 16, kb * 16, lane);
#pragma unroll
                for (int mb = 0; mb < 2; ++mb) {
                    mma16816(acc[mb][0], xa[mb][kb], b[0], b[1]);
                    mma16816(acc[mb][1], xa[mb][kb], b[2], b[3]);
                }
            }
#pragma unroll
            for (int mb = 0; mb < 2; ++mb) act_frag(h1[mb][np], acc[mb][0], acc[mb][1], W.b1, np, tg);
        }
    }
    uint32_t h2[2][8][4];
#pragma unroll
    for (int np = 0; np < 8; ++np) {
        float acc[2][2][4] = {};
#pragma unroll
        for (int kb = 0; kb < 8; ++kb) {
            uint32_t b[4];
            frag_b_nk(b, W.W2, LDH, np * 16, kb * 16, lane);
#pragma unroll
            for (int mb = 0; mb < 2; ++mb) {
                mma16816(acc[mb][0], h1[mb][kb], b[0], b[1]);
                mma16816(acc[mb][1], h1[mb][kb], b[2], b[3]);
            }
        }
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) act_frag(h2[mb][np], acc[mb][0], acc[mb][1], W.b2, np, tg);
    }
#pragma unroll
    for (int mb = 0; mb < 2; ++mb)
#pragma unroll
        for (int t = 0; t < 2; ++t) y[mb][t][0] = y[mb][t][1] = y[mb][t][2] = y[mb][t][3] = 0.f;
#pragma unroll
    for (int kb = 0; kb < 8; ++kb) {
        uint32_t b[4];
        frag_b_nk(b, W.W3, LDH, 0, kb * 16, lane);
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            mma16816(y[mb][0], h2[mb][kb], b[0], b[1]);
            mma16816(y[mb][1], h2[mb][kb], b[2], b[3]);
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float2 bo = *reinterpret_cast<const float2*>(W.b3 + t * 8 + 2 * tg);
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
            y[mb][t][0] += bo.x; y[mb][t][1] += bo.y;
            y[mb][t][2] += bo.x; y[mb][t][3] += bo.y;
        }
    }
}

// Row of output element (mb, e) within a warp tile, and its output column (t, e).
__device__ __forceinline__ int out_row(int mb, int e, int lane) { return 16 * mb + (lane >> 2) + 8 * (e >> 1); }
__device__ __forceinline__ int out_col(int t, int e, int lane) { return 8 * t + 2 * (lane & 3) + (e & 1); }

__global__ void __launch_bounds__(ITHREADS, 1) k_forward(const float* __restrict__ X, long M,
                                                         const Packed* __restrict__ P, float* __restrict__ Y) {
    extern __shared__ __align__(128) unsigned char raw[];
    InferSmem& S = *reinterpret_cast<InferSmem*>(raw);
    load_weights(S.w, P);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __nv_bfloat16* Xs = S.X[warp];
    const long tiles = (M + IROWS - 1) / IROWS;
    for (long tile = (long)blockIdx.x * IW + warp; tile < tiles; tile += (long)gridDim.x * IW) {
        const long m0 = tile * IROWS;
        // the tile's rows are contiguous in X: coalesced copy into the tile
        for (int i = lane; i < IROWS * LDX; i += 32) {
            const int r = i / LDX, c = i % LDX;
            const long m = m0 + r;
            Xs[i] = __float2bfloat16_rn(m < M && c < NIN ? X[m * NIN + c] : 0.f);
        }
        __syncwarp();
        float y[2][2][4];
        warp_mlp32(S.w, Xs, y, lane);
        __syncwarp();
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const long m = m0 + out_row(mb, e, lane);
                    const int o = out_col(t, e, lane);
                    if (m < M && o < NOUT) Y[m * NOUT + o] = y[mb][t][e];
                }
    }
}

// Loss sum_{s,o} (y - t)^2 / (B 9) and its gradient over one tile of 128
// samples; the CTA writes its partial sums to part[blockIdx.x][NPARAM + 1].
__global__ void __launch_bounds__(THREADS) k_loss_grad(const float* __restrict__ X, const float* __restrict__ T,
                                                       const int* __restrict__ idx, long B,
                                                       const Packed* __restrict__ P, float* __restrict__ part) {
    extern __shared__ __align__(128) unsigned char raw[];
    Smem& S = *reinterpret_cast<Smem*>(raw);
    SmemBack& D = *reinterpret_cast<SmemBack*>(raw + sizeof(Smem));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tg = lane & 3;
    const int r0 = warp * 16;
    float* out = part + (long)blockIdx.x * (NPARAM + 1);
    load_weights(S.w, P);
    const long row0 = (long)blockIdx.x * ROWS;
    stage_inputs(S, X, idx, row0, B);
    __syncthreads();
    float y[2][4];
    network(S, warp, lane, y);
    // dY = 2 (y - t) / (B 9) on valid samples and outputs, else 0
    const float inv = 2.f / (float)(B * NOUT);
    float lsum = 0.f;
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = r0 + g + 8 * h;
            const long m = row0 + r;
            float d[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int c = t * 8 + 2 * tg + e;
                float v = 0.f;
                if (m < B && c < NOUT) {
                    const long src = idx ? (long)idx[m] : m;
                    const float rr = y[t][2 * h + e] - T[src * NOUT + c];
                    lsum += rr * rr;
                    v = inv * rr;
                }
                d[e] = v;
            }
            *reinterpret_cast<uint32_t*>(D.dY + r * LDO + t * 8 + 2 * tg) = pack_bf16(d[0], d[1]);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) D.wloss[warp] = lsum / (float)(B * NOUT);
    __syncwarp();
    // dZ2 = (dY W3) * (1 - H2^2), K = 16 outputs (9 used)
    {
        uint32_t a[4];
        frag_a(a, D.dY, LDO, r0, 0, lane);
#pragma unroll 4
        for (int nb = 0; nb < HID; nb += 8) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t b[2];
            frag_b_kn(b, S.w.W3, LDH, 0, nb, lane);
            mma16816(acc, a, b[0], b[1]);
            const int c = nb + 2 * tg;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                const float h0 = __bfloat162float(S.H2[r * LDH + c]), h1 = __bfloat162float(S.H2[r * LDH + c + 1]);
                *reinterpret_cast<uint32_t*>(D.dZ2 + r * LDH + c) =
                    pack_bf16(acc[2 * h] * (1.f - h0 * h0), acc[2 * h + 1] * (1.f - h1 * h1));
            }
        }
    }
    __syncwarp();
    // dZ1 = (dZ2 W2) * (1 - H1^2), K = 128
    {
#pragma unroll 1
        for (int nb = 0; nb < HID; nb += 8) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int k0 = 0; k0 < HID; k0 += 16) {
                uint32_t a[4], b[2];
                frag_a(a, D.dZ2, LDH, r0, k0, lane);
                frag_b_kn(b, S.w.W2, LDH, k0, nb, lane);
                mma16816(acc, a, b[0], b[1]);
            }
            const int c = nb + 2 * tg;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = r0 + g + 8 * h;
                const float h0 = __bfloat162float(S.H1[r * LDH + c]), h1 = __bfloat162float(S.H1[r * LDH + c + 1]);
                *reinterpret_cast<uint32_t*>(D.dZ1 + r * LDH + c) =
                    pack_bf16(acc[2 * h] * (1.f - h0 * h0), acc[2 * h + 1] * (1.f - h1 * h1));
            }
        }
    }
    __syncthreads();
    // weight gradients over the tile's samples (K = 128): warp w owns rows
    // 16w..16w+15 of dW2 and dW1; warp 0 also the rows of dW3.
    {
        const int m0 = r0;
#pragma unroll 1
        for (int nb = 0; nb < HID; nb += 8) {               // dW2[o][i] = sum_s dZ2[s][o] H1[s][i]
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int k0 = 0; k0 < ROWS; k0 += 16) {
                uint32_t a[4], b[2];
                frag_a_t(a, D.dZ2, LDH, m0, k0, lane);
                frag_b_kn(b, S.H1, LDH, k0, nb, lane);
                mma16816(acc, a, b[0], b[1]);
            }
            float* o = out + OFF_W2;
            const int c = nb + 2 * tg;
            o[(m0 + g) * HID + c] = acc[0];
            o[(m0 + g) * HID + c + 1] = acc[1];
            o[(m0 + g + 8) * HID + c] = acc[2];
            o[(m0 + g + 8) * HID + c + 1] = acc[3];
        }
#pragma unroll 1
        for (int nb = 0; nb < KX; nb += 8) {                // dW1[o][i] = sum_s dZ1[s][o] X[s][i]
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int k0 = 0; k0 < ROWS; k0 += 16) {
                uint32_t a[4], b[2];
                frag_a_t(a, D.dZ1, LDH, m0, k0, lane);
                frag_b_kn(b, S.X, LDX, k0, nb, lane);
                mma16816(acc, a, b[0], b[1]);
            }
            float* o = out + OFF_W1;
            const int c = nb + 2 * tg;
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (c + (e & 1) < NIN) o[(m0 + g + 8 * (e >> 1)) * NIN + c + (e & 1)] = acc[e];
        }
        if (warp == 0) {
#pragma unroll 1
            for (int nb = 0; nb < HID; nb += 8) {           // dW3[o][i] = sum_s dY[s][o] H2[s][i]
                float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
                for (int k0 = 0; k0 < ROWS; k0 += 16) {
                    uint32_t a[4], b[2];
                    frag_a_t(a, D.dY, LDO, 0, k0, lane);
                    frag_b_kn(b, S.H2, LDH, k0, nb, lane);
                    mma16816(acc, a, b[0], b[1]);
                }
                float* o = out + OFF_W3;
                const int c = nb + 2 * tg;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = g + 8 * (e >> 1);
                    if (row < NOUT) o[row * HID + c + (e & 1)] = acc[e];
                }
            }
        }
    }
    // bias gradients: column sums of dZ1, dZ2, dY over the tile
    for (int c = threadIdx.x; c < HID; c += THREADS) {
        float s1 = 0.f, s2 = 0.f;
        for (int r = 0; r < ROWS; ++r) {
            s1 += __bfloat162float(D.dZ1[r * LDH + c]);
            s2 += __bfloat162float(D.dZ2[r * LDH + c]);
        }
        out[OFF_B1 + c] = s1;
        out[OFF_B2 + c] = s2;
    }
    if (threadIdx.x < NOUT) {
        float s3 = 0.f;
        for (int r = 0; r < ROWS; ++r) s3 += __bfloat162float(D.dY[r * LDO + threadIdx.x]);
        out[OFF_B3 + threadIdx.x] = s3;
    }
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int w = 0; w < WARPS; ++w) l += D.wloss[w];
        out[NPARAM] = l;
    }
}

// grad[i] = sum over CTAs of part[cta][i], i <= NPARAM (the last entry is the loss)
__global__ void k_reduce_grad(const float* __restrict__ part, long nblk, float* __restrict__ grad,
                              float* __restrict__ loss) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= NPARAM; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (long b = 0; b < nblk; ++b) s += part[b * (NPARAM + 1) + i];
        if (i < NPARAM) grad[i] = s;
        else if (loss) *loss = s;
    }
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters; c1, c2 are the
// bias corrections 1 - beta^t.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// FP32 parameters -> BF16 weights in the padded layout, FP32 biases.
__global__ void k_pack(const float* __restrict__ params, Packed* __restrict__ P) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int i = tid; i < HID * LDX; i += stride) {
        const int o = i / LDX, c = i % LDX;
        P->W1[i] = __float2bfloat16_rn(c < NIN ? params[OFF_W1 + o * NIN + c] : 0.f);
    }
    for (int i = tid; i < HID * LDH; i += stride) {
        const int o = i / LDH, c = i % LDH;
        P->W2[i] = __float2bfloat16_rn(c < HID ? params[OFF_W2 + o * HID + c] : 0.f);
    }
    for (int i = tid; i < OUTP * LDH; i += stride) {
        const int o = i / LDH, c = i % LDH;
        P->W3[i] = __float2bfloat16_rn(o < NOUT && c < HID ? params[OFF_W3 + o * HID + c] : 0.f);
    }
    for (int i = tid; i < HID; i += stride) { P->b1[i] = params[OFF_B1 + i]; P->b2[i] = params[OFF_B2 + i]; }
    for (int i = tid; i < OUTP; i += stride) P->b3[i] = i < NOUT ? params[OFF_B3 + i] : 0.f;
}

// ------------------------------------------------------------ closure glue
// (cell features: closure_features.cuh)

// Training samples: X[m][38] (FP32), scale[m], and (tgt not NULL) the
// order-8 moments at the centre divided by the scale.
template <class T>
__global__ void __launch_bounds__(256) k_samples(const ClosureArgs<T> A, float* __restrict__ X,
                                                 float* __restrict__ scale, float* __restrict__ tgt) {
    const int nx = A.nx, ny = A.ny;
    const long M = (long)nx * ny;
    for (long m = blockIdx.x * (long)blockDim.x + threadIdx.x; m < M; m += (long)gridDim.x * blockDim.x) {
        const int ix = (int)(m % nx), iy = (int)(m / nx);
        const Stencil o = stencil(ix, iy, nx, ny, A.p[0], A.p[1], A.pitch);
        float f[NMOM], s, inv;
        features36<T>(A.col, o, true, f, s, inv);
#pragma unroll
        for (int c = 0; c < NMOM; ++c) X[m * NIN + c] = f[c];
        X[m * NIN + NMOM] = A.lsa[m];
        X[m * NIN + NMOM + 1] = A.lss[m];
        scale[m] = s;
        if (tgt) {
            float t[NOUT];
            gather8<T>(A.col, o, t, std::make_integer_sequence<int, NOUT>{});
#pragma unroll
            for (int k = 0; k < NOUT; ++k) tgt[m * NOUT + k] = t[k] * inv;
        }
    }
}

constexpr int PAD_ROWS_F = 128;         // input rows are written up to a whole number of 128-row tiles

// Closure inputs of every cell as padded BF16 rows xg[m][LDX] (columns 38..
// LDX-1 zero; rows up to a whole number of 128-row tiles) and the scale
// sc[m]: one thread per cell, exactly the features of k_samples (the
// training samples), rounded to BF16.
template <class T>
__global__ void __launch_bounds__(256) k_closure_features(const ClosureArgs<T> A, __nv_bfloat16* __restrict__ xg,
                                                          float* __restrict__ sc) {
    const int nx = A.nx, ny = A.ny;
    const int M = nx * ny;
    const int Mpad = (M + PAD_ROWS_F - 1) / PAD_ROWS_F * PAD_ROWS_F;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < Mpad; m += gridDim.x * blockDim.x) {
        const bool ok = m < M;
        const int ix = ok ? m % nx : 0, iy = ok ? m / nx : 0;
        const Stencil o = stencil(ix, iy, nx, ny, A.p[0], A.p[1], A.pitch);
        float f[NMOM], scale, inv;
        features36<T>(A.col, o, ok, f, scale, inv);
        uint32_t w[LDX / 2];
#pragma unroll
        for (int c = 0; c < NMOM / 2; ++c) w[c] = pack_bf16(f[2 * c], f[2 * c + 1]);
        w[NMOM / 2] = pack_bf16(ok ? A.lsa[m] : 0.f, ok ? A.lss[m] : 0.f);
#pragma unroll
        for (int c = NIN / 2; c < LDX / 2; ++c) w[c] = 0u;
        uint4* row = reinterpret_cast<uint4*>(xg + (long)m * LDX);
#pragma unroll
        for (int q = 0; q < LDX / 8; ++q) row[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        sc[m] = scale;
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(su32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Closure prediction from the input rows: persistent warps, each
// double-buffering its 32-row tiles with cp.async, network in registers,
// s * y written out: R_8^m straight to G11 (with their ghost copies), the
// centre values of I_8^m to ctr[o][M] for the node averaging of
// k_closure_nodes.
struct ClosureSmem {
    Packed w;
    __nv_bfloat16 X[IW][2][IROWS * LDX];
};

template <class T>
__global__ void __launch_bounds__(ITHREADS, 1) k_closure_mlp(const ClosureArgs<T> A, const Packed* __restrict__ P,
                                                             const __nv_bfloat16* __restrict__ xg,
                                                             const float* __restrict__ sc, float* __restrict__ ctr) {
    extern __shared__ __align__(128) unsigned char raw[];
    ClosureSmem& S = *reinterpret_cast<ClosureSmem*>(raw);
    load_weights(S.w, P);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = A.nx, ny = A.ny;
    const int M = nx * ny;
    const int tiles = (M + IROWS - 1) / IROWS;
    const long Pp = A.pitch;
    constexpr int CHUNKS = IROWS * LDX * 2 / 16;      // 16-byte pieces of a tile
    auto issue = [&](int tile, int buf) {
        const char* src = reinterpret_cast<const char*>(xg + (long)tile * IROWS * LDX);
        char* dst = reinterpret_cast<char*>(S.X[warp][buf]);
        for (int i = lane; i < CHUNKS; i += 32) cp_async16(dst + 16 * i, src + 16 * i);
        cp_async_commit();
    };
    const int stride = gridDim.x * IW;
    int tile = blockIdx.x * IW + warp;
    if (tile < tiles) issue(tile, 0);
    for (int k = 0; tile < tiles; tile += stride, k ^= 1) {
        if (tile + stride < tiles) issue(tile + stride, k ^ 1);
        else cp_async_commit();
        cp_async_wait1();
        __syncwarp();
        float scl[2][2];
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int h = 0; h < 2; ++h) scl[mb][h] = __ldg(sc + tile * IROWS + out_row(mb, 2 * h, lane));
        float y[2][2][4];
        warp_mlp32(S.w, S.X[warp][k], y, lane);
#pragma unroll
        for (int mb = 0; mb < 2; ++mb)
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int m = tile * IROWS + out_row(mb, e, lane);
                    const int o = out_col(t, e, lane);
                    if (m >= M || o >= NOUT) continue;
                    const float val = scl[mb][e >> 1] * y[mb][t][e];
                    if (A.slot[NMOM + o].x != 0) { ctr[(long)o * M + m] = val; continue; }
                    const int ix = m % nx, iy = m / nx;
                    T* c = A.g[0].base + (long)A.slot[NMOM + o].y * A.g[0].cstride;
                    const T tv = (T)val;
                    c[(long)(iy + 1) * Pp + ix] = tv;
                    // ghost copies: periodic -1 <- n-1, n <- 0; extrapolation -1 <- 0, n <- n-1
                    if (ix == (A.p[0] ? nx - 1 : 0)) c[(long)(iy + 1) * Pp - 1] = tv;
                    if (ix == (A.p[0] ? 0 : nx - 1)) c[(long)(iy + 1) * Pp + nx] = tv;
                    if (iy == (A.p[1] ? ny - 1 : 0)) c[ix] = tv;
                    if (iy == (A.p[1] ? 0 : ny - 1)) c[(long)(ny + 1) * Pp + ix] = tv;
                }
        __syncwarp();
    }
}

// I_8^m at the points of G22: mean of the four surrounding cell centres.
// Node k of an axis lies between cells k + p - 1 and k + p (wrapped when
// periodic, clamped to the boundary cell for extrapolation); ghost copies
// only on periodic axes (extrapolation node axes are never read outside).
// One thread per node; the outputs on G22 come as a list (their centre
// values and their point (0, 0)), all loads before the first store.
template <class T>
struct NodeJobs {
    int count;
    const float* src[NOUT];     // centre values of the output, [ny][nx]
    T* dst[NOUT];               // its component on G22
};

template <class T>
__global__ void __launch_bounds__(256) k_closure_nodes(const ClosureArgs<T> A, const NodeJobs<T> J) {
    pdl_trigger();
    pdl_wait();                         // the centre values are written
    const int gnx = A.g[3].nx, gny = A.g[3].ny;
    const int nx = A.nx, ny = A.ny;
    const long Pp = A.pitch;
    // (cells below 2^31, checked by the caller, so nodes below 2^32)
    const unsigned nodes = (unsigned)gnx * (unsigned)gny;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < nodes; i += gridDim.x * blockDim.x) {
        const int ky = (int)(i / (unsigned)gnx), kx = (int)(i - (unsigned)ky * (unsigned)gnx);
        int cy0 = ky + A.p[1] - 1, cy1 = ky + A.p[1];
        if (A.p[1]) { cy0 = cy0 < 0 ? ny - 1 : cy0; cy1 = cy1 == ny ? 0 : cy1; }
        else { cy0 = max(cy0, 0); cy1 = min(cy1, ny - 1); }
        int cx0 = kx + A.p[0] - 1, cx1 = kx + A.p[0];
        if (A.p[0]) { cx0 = cx0 < 0 ? nx - 1 : cx0; cx1 = cx1 == nx ? 0 : cx1; }
        else { cx0 = max(cx0, 0); cx1 = min(cx1, nx - 1); }
        const int a = cy0 * nx + cx0, b = cy0 * nx + cx1, c = cy1 * nx + cx0, d = cy1 * nx + cx1;
        float v[NOUT];
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
            if (j >= J.count) break;
            const float* s = J.src[j];
            v[j] = 0.25f * ((s[a] + s[b]) + (s[c] + s[d]));
        }
        const long row = (long)(ky + 1) * Pp;
#pragma unroll
        for (int j = 0; j < NOUT; ++j) {
            if (j >= J.count) break;
            T* dd = J.dst[j];
            const T tv = (T)v[j];
            dd[row + kx] = tv;
            if (A.p[0]) {
                if (kx == gnx - 1) dd[row - 1] = tv;
                if (kx == 0) dd[row + gnx] = tv;
            }
            if (A.p[1]) {
                if (ky == gny - 1) dd[kx] = tv;
                if (ky == 0) dd[(long)(gny + 1) * Pp + kx] = tv;
            }
        }
    }
}

// Training-input noise: Xn[m][c] = X[m][c] + sigma g(seed, m NIN + c) for
// c < cols, a copy of X[m][c] otherwise.  g is a standard normal from a
// counter-based stream: the SplitMix64 finaliser (Steele, Lea & Flood 2014)
// of seed * golden + counter gives two 32-bit uniforms in (0, 1), turned
// into one normal by the Box-Muller transform (Box & Muller 1958).
__host__ __device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_perturb(const float* X, float* Xn, long total, int cols, float sigma,
                          unsigned long long seed) {
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        float v = X[e];
        if ((int)(e % NIN) < cols) {
            const unsigned long long z = splitmix64(seed * 0x9e3779b97f4a7c15ull + (unsigned long long)e);
            const float u1 = ((float)(unsigned)(z >> 32) + 0.5f) * 2.3283064365386963e-10f;   // (0, 1)
            const float u2 = ((float)(unsigned)(z & 0xffffffffu) + 0.5f) * 2.3283064365386963e-10f;
            v += sigma * sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
        }
        Xn[e] = v;
    }
}

// Sample order for an epoch: out[i] = index[perm(i)] (index NULL: perm(i))
// for a keyed pseudo-random permutation of [0, count).  perm is a balanced
// four-round Feistel network on the smallest even number of bits 2h with
// 2^(2h) >= count (round function: the SplitMix64 finaliser of the key, the
// round and the right half, keeping h bits), restricted to [0, count) by
// cycle walking — applying it again until the value falls inside, which
// stays a bijection and ends within the cycle through i (Black & Rogaway
// 2002, "Ciphers with arbitrary finite domains"); with 2^(2h) < 4 count a
// walk takes fewer than four rounds of the network on average.
__device__ __forceinline__ unsigned long long feistel(unsigned long long x, int h, unsigned long long key) {
    const unsigned long long mask = (1ull << h) - 1;
    unsigned long long L = x >> h, R = x & mask;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const unsigned long long F = splitmix64(key ^ ((unsigned long long)(r + 1) * 0xd1b54a32d192ed03ull) ^ R) & mask;
        const unsigned long long nl = R;
        R = L ^ F;
        L = nl;
    }
    return (L << h) | R;
}

__global__ void k_shuffle(const int* __restrict__ index, long count, int h, unsigned long long key, int* __restrict__ out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        unsigned long long x = (unsigned long long)i;
        do x = feistel(x, h, key); while (x >= (unsigned long long)count);
        out[i] = index ? index[x] : (int)x;
    }
}

int status(cudaError_t e) { return e == cudaSuccess ? 0 : -4; }

template <class K>
int set_smem(K kernel, size_t bytes, bool& done) {
    if (done) return 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return -4;
    done = true;
    return 0;
}

constexpr size_t SMEM_FWD = sizeof(InferSmem);
constexpr size_t SMEM_TRAIN = sizeof(Smem) + sizeof(SmemBack);
static_assert(SMEM_TRAIN <= 227 * 1024, "training tile exceeds shared memory");

}  // namespace

long grad_blocks(long B) { return (B + ROWS - 1) / ROWS; }

int pack(const float* params, Packed* P, void* stream) {
    k_pack<<<64, 256, 0, (cudaStream_t)stream>>>(params, P);
    return status(cudaGetLastError());
}

int forward(const float* X, long M, const Packed* P, float* Y, void* stream) {
    if (M <= 0) return 0;
    static bool attr = false;
    if (set_smem(k_forward, SMEM_FWD, attr)) return -4;
    long blocks = (M + IROWS * IW - 1) / (IROWS * IW);
    if (blocks > sm_count()) blocks = sm_count();
    k_forward<<<(unsigned)blocks, ITHREADS, SMEM_FWD, (cudaStream_t)stream>>>(X, M, P, Y);
    return status(cudaGetLastError());
}

int loss_grad(const float* X, const float* T, const int* idx, long B, const Packed* P, float* part, float* grad,
              float* loss, int engine, int* err, void* stream) {
    if (B <= 0) return 0;
    const long blocks = grad_blocks(B);
    if (engine == ENGINE_TCGEN05) {
        if (loss_grad_tc(X, T, idx, B, P, part, err, stream)) return -4;
    } else {
        static bool attr = false;
        if (set_smem(k_loss_grad, SMEM_TRAIN, attr)) return -4;
        k_loss_grad<<<(unsigned)blocks, THREADS, SMEM_TRAIN, (cudaStream_t)stream>>>(X, T, idx, B, P, part);
        if (cudaGetLastError() != cudaSuccess) return -4;
    }
    k_reduce_grad<<<(NPARAM + 1 + 255) / 256, 256, 0, (cudaStream_t)stream>>>(part, blocks, grad, loss);
    return status(cudaGetLastError());
}

int shuffle(const int* index, long count, unsigned long long seed, int* out, void* stream) {
    if (count <= 0) return 0;
    int h = 1;
    while ((1ll << (2 * h)) < count) ++h;
    long blocks = (count + 255) / 256;
    if (blocks > 32L * sm_count()) blocks = 32L * sm_count();
    k_shuffle<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(index, count, h, splitmix64(seed), out);
    return status(cudaGetLastError());
}

int perturb(const float* X, float* Xn, long M, int cols, float sigma, unsigned long long seed, void* stream) {
    const long total = M * NIN;
    if (total <= 0) return 0;
    long blocks = (total + 255) / 256;
    if (blocks > 32L * sm_count()) blocks = 32L * sm_count();
    k_perturb<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(X, Xn, total, cols, sigma, seed);
    return status(cudaGetLastError());
}

int adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps, long step,
         void* stream) {
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)step));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)step));
    k_adam<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return status(cudaGetLastError());
}

template <class T>
int samples(const ClosureArgs<T>& A, float* X, float* scale, float* tgt, void* stream) {
    const long M = (long)A.nx * A.ny;
    if (M <= 0) return 0;
    long blocks = (M + 255) / 256;
    if (blocks > 16L * sm_count()) blocks = 16L * sm_count();
    k_samples<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(A, X, scale, tgt);
    return status(cudaGetLastError());
}

// input rows are padded to whole 128-row tiles (the tcgen05 network's M)
constexpr int PAD_ROWS = 128;

long closure_scratch_floats(long M) {
    const long Mpad = (M + PAD_ROWS - 1) / PAD_ROWS * PAD_ROWS;
    return Mpad * LDX / 2 + Mpad + (long)NOUT * M;      // BF16 input rows, scales, I_8 centre values
}

template <class T>
int closure(const ClosureArgs<T>& A, const Packed* P, float* scratch, int engine, int* err, void* stream) {
    static bool attr = false;
    if (set_smem(k_closure_mlp<T>, sizeof(ClosureSmem), attr)) return -4;
    const long M = (long)A.nx * A.ny;
    if (M <= 0) return 0;
    if (M > 0x7fff0000L) return -8;
    const long tiles = (M + IROWS - 1) / IROWS;
    const long Mpad = (M + PAD_ROWS - 1) / PAD_ROWS * PAD_ROWS;
    __nv_bfloat16* xg = reinterpret_cast<__nv_bfloat16*>(scratch);
    float* sc = scratch + Mpad * LDX / 2;
    float* ctr = sc + Mpad;
    if (engine == ENGINE_TCGEN05) {
        if (closure_tc<T>(A, P, ctr, sc, err, stream)) return -4;
    } else {
        long fb = (Mpad + 255) / 256;      // the features kernel covers the padded rows too
        if (fb > 32L * sm_count()) fb = 32L * sm_count();
        k_closure_features<T><<<(unsigned)fb, 256, 0, (cudaStream_t)stream>>>(A, xg, sc);
        if (cudaGetLastError() != cudaSuccess) return -4;
        long blocks = (tiles + IW - 1) / IW;
        if (blocks > sm_count()) blocks = sm_count();
        k_closure_mlp<T><<<(unsigned)blocks, ITHREADS, sizeof(ClosureSmem), (cudaStream_t)stream>>>(A, P, xg, sc, ctr);
        if (cudaGetLastError() != cudaSuccess) return -4;
    }
    if (A.g[3].nx > 0 && A.g[3].ny > 0) {
        NodeJobs<T> J;
        J.count = 0;
        for (int o = 0; o < NOUT; ++o)
            if (A.slot[NMOM + o].x == 3) {
                J.src[J.count] = ctr + (long)o * M;
                J.dst[J.count] = A.g[3].base + (long)A.slot[NMOM + o].y * A.g[3].cstride;
                ++J.count;
            }
        const long nodes = (long)A.g[3].nx * A.g[3].ny;
        long blocks = (nodes + 255) / 256;
        if (blocks > 64L * sm_count()) blocks = 64L * sm_count();
        if (J.count > 0 && launch_pdl(k_closure_nodes<T>, dim3((unsigned)blocks), dim3(256), 0, (cudaStream_t)stream,
                                      true, A, J) != cudaSuccess)
            return -4;
    }
    return status(cudaGetLastError());
}

template int samples<float>(const ClosureArgs<float>&, float*, float*, float*, void*);
template int samples<double>(const ClosureArgs<double>&, float*, float*, float*, void*);
template int closure<float>(const ClosureArgs<float>&, const Packed*, float*, int, int*, void*);
template int closure<double>(const ClosureArgs<double>&, const Packed*, float*, int, int*, void*);

}  // namespace mlp
}  // namespace starmap
