// The closure network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Operands live in shared memory in the canonical K-major layout without
// swizzle: 8-row x 16-byte core matrices; an M x K (or N x K) operand stores
// element (r, k) at
//     (k / 8) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2  bytes,
// LBO = (rows / 8) * 128 (core matrices adjacent along M/N are 128 bytes
// apart = SBO, along K LBO apart).  A tile is 128 samples.  One elected
// thread of a 4-warp group issues the layer's tcgen05.mma (M = 128, K = 16
// per instruction, BF16 x BF16 -> FP32) into the group's 128-column TMEM
// accumulator and commits it to the group's mbarrier; the group's 4 warps
// then read the accumulator with tcgen05.ld (thread = row = TMEM lane), add
// the bias, apply the shared activation (tanh.approx.bf16x2 of the
// BF16-rounded pre-activation) and write the next layer's operand back to
// shared memory.  Layers: 38(48) -> 128 (3 MMAs), 128 -> 128 (8 MMAs),
// 128 -> 16 (9 used, 8 MMAs with N = 16).
//
// Three kernels, one CTA per SM each:
//  - k_forward_tc (inference on given input rows): five groups, each staging
//    its own tiles, sharing four TMEM accumulators (a group loading its
//    inputs holds none);
//  - k_closure_tc (the fused closure): one producer group gathers each
//    tile's cell features from the moment grids into the input buffer of the
//    consumer group that runs the tile's network; full / empty mbarriers
//    hand the buffers back and forth, so the gather's memory latency hides
//    behind the other tiles' tensor and activation work;
//  - k_loss_grad_tc (training): the loss and every parameter gradient of a
//    tile of samples, the backward contractions reading the same natural
//    buffers MN-major (see the training section below).
// Every wait is bounded; on expiry the kernel raises the error flag, skips
// the rest, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "closure_features.cuh"
#include "internal.h"
#include "mlp.h"
#include "pdl.h"

namespace starmap {
namespace mlp {

namespace {

constexpr int TM = 128;                  // samples per tile (MMA M)
constexpr int GROUPS = 5;                // independent 4-warp groups per CTA, one tile each
constexpr int SLOTS = 4;                 // 128-column TMEM accumulators, shared by the groups
constexpr int GWARPS = 4;
constexpr int GTHREADS = GWARPS * 32;    // one thread per tile row (= TMEM lane)
constexpr int TC_THREADS = GROUPS * GTHREADS;
constexpr int KX_TC = 48;                // input width padded to the MMA K step
constexpr int BIAS_COL = NIN;            // first of the three input columns carrying layer 0's bias
static_assert(BIAS_COL + 3 <= KX_TC, "the bias columns fit in the padding");
constexpr int XC_BYTES = (KX_TC / 8) * (TM / 8) * 128;       // 12288
constexpr int W1_BYTES = (KX_TC / 8) * (HID / 8) * 128;      // 12288
constexpr int W2_BYTES = (HID / 8) * (HID / 8) * 128;        // 32768
constexpr int W3_BYTES = (HID / 8) * (OUTP / 8) * 128;       // 4096
constexpr int H_BYTES = (HID / 8) * (TM / 8) * 128;          // 32768
constexpr int TMEM_COLS = SLOTS * 128;   // one 128-column accumulator per slot
constexpr int CONSUMERS = 4;             // closure kernel: network groups (one accumulator each)
constexpr int PRODUCERS = 2;             // closure kernel: feature-gathering groups
constexpr int CL_THREADS = (CONSUMERS + PRODUCERS) * GTHREADS;
static_assert(CONSUMERS % PRODUCERS == 0, "each consumer is fed by one producer");
static_assert(CONSUMERS * 128 <= TMEM_COLS, "one accumulator per consumer group");
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;
static_assert(XC_BYTES <= H_BYTES, "the input operand fits in the hidden operand's buffer");

// A group's operand buffer: the layer-0 input (canonical, K = 48) at its
// start, overwritten by the hidden activations once layer 0's MMAs are done.
struct TcGroup {
    alignas(128) unsigned char h[H_BYTES];
};
struct TcSmem {
    alignas(1024) unsigned char w1[W1_BYTES];
    alignas(128) unsigned char w2[W2_BYTES];
    alignas(128) unsigned char w3[W3_BYTES];
    TcGroup grp[GROUPS];
    alignas(16) float b1[HID];
    alignas(16) float b2[HID];
    alignas(16) float b3[OUTP];
    alignas(8) uint64_t mbar[GROUPS];
    uint32_t tmem;
    int abort[GROUPS];
    int slot[GROUPS];                    // TMEM slot a group holds from its first MMA to its output
    int free_slots;                      // bit s: slot s is free
};
static_assert(sizeof(TcSmem) <= 227 * 1024, "forward kernel shared memory");

// Closure kernel: per consumer group its hidden operand h and its input
// buffer x (written by the producer group); full[c] completes when the
// producer has written consumer c's next tile (one arrival per producer
// thread), empty[c] when consumer c's layer-0 MMAs have read it.
struct ClSmem {
    alignas(128) unsigned char w1[W1_BYTES];
    alignas(128) unsigned char w2[W2_BYTES];
    alignas(128) unsigned char w3[W3_BYTES];
    alignas(128) unsigned char h[CONSUMERS][H_BYTES];
    alignas(128) unsigned char x[CONSUMERS][XC_BYTES];
    alignas(16) float b1[HID];
    alignas(16) float b2[HID];
    alignas(16) float b3[OUTP];
    alignas(8) uint64_t mma[CONSUMERS];
    alignas(8) uint64_t full[CONSUMERS];
    alignas(8) uint64_t empty[CONSUMERS];
    uint32_t tmem;
    int abort;                           // a wait expired: every role stops at its next wait
    int stop[CONSUMERS];                 // a consumer group's verdict, set by its leader
};
static_assert(sizeof(ClSmem) <= 227 * 1024, "closure kernel shared memory");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// byte offset of element (r, k) of a canonical K-major operand with `rows` rows
__device__ __forceinline__ uint32_t canon(int r, int k, int rows) {
    return (uint32_t)((k >> 3) * (rows >> 3) * 128 + (r >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// barrier of one 128-thread group (ids 1..GROUPS; 0 is __syncthreads)
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(GTHREADS) : "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}
// 32 consecutive columns of this warp's 32 lanes in one load
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// 32 consecutive columns of this warp's 32 lanes in one store
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
          "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
          "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
          "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// The waiting thread is suspended until the phase completes or about 0.1 ms
// pass, so a wait issues a handful of instructions rather than a busy loop.
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(bar)), "r"(parity), "r"(100000u) : "memory");
    return ok != 0;
}
// bounded wait for the MMA commit of the given phase; false on expiry
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    while (!mbar_test(bar, parity))
        if (gtime() - t0 > TC_WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
    return true;
}

__device__ __forceinline__ uint32_t pack_bf16_tc(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
// the activation of the mma.sync kernels, bit for bit
__device__ __forceinline__ uint32_t act2_tc(float lo, float hi) {
    const uint32_t x = pack_bf16_tc(lo, hi);
    uint32_t y;
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}
// accumulator pair + bias pair in one packed FP32 add (each half rounded
// exactly as a scalar add), then the activation
__device__ __forceinline__ uint32_t bias_act2_tc(uint32_t a_lo, uint32_t a_hi, float b_lo, float b_hi) {
    unsigned long long a, b, s;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "r"(a_lo), "r"(a_hi));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(b_lo), "f"(b_hi));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(s) : "l"(a), "l"(b));
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(s));
    return act2_tc(lo, hi);
}

__device__ __forceinline__ void cp_async16_tc(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}

// Weights (row-major padded BF16 of Packed) into the canonical layouts,
// 16-byte pieces by cp.async (no register round trip); the caller waits.
//
// Layer 0's bias rides in the MMA: input columns BIAS_COL .. BIAS_COL + 2
// (padding beyond the NIN features) hold 1.0, and W1's row n holds there the
// three BF16 parts hi + mid + lo of b1[n] (each part the BF16 rounding of
// what the previous parts leave, so their sum is b1[n] to FP32 precision).
template <class Sm>
__device__ void load_weights_tc(Sm& S, const Packed* P) {
    const uint32_t w1 = su32(S.w1), w2 = su32(S.w2), w3 = su32(S.w3);
    const int nt = (int)blockDim.x;
    for (int i = threadIdx.x; i < HID * (KX_TC / 8); i += nt) {         // W1: 128 rows x 6 chunks
        const int n = i / (KX_TC / 8), c = i % (KX_TC / 8);
        if (8 * c + 8 <= BIAS_COL) {
            cp_async16_tc(w1 + canon(n, 8 * c, HID), P->W1 + n * LDX + 8 * c);
            continue;
        }
        __nv_bfloat16 e[8];
        const float b = P->b1[n];
        const __nv_bfloat16 hi = __float2bfloat16_rn(b);
        const float r1 = b - __bfloat162float(hi);
        const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
        const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int col = 8 * c + j;
            e[j] = col < BIAS_COL ? P->W1[n * LDX + col]
                 : col == BIAS_COL ? hi : col == BIAS_COL + 1 ? mid : col == BIAS_COL + 2 ? lo
                 : __float2bfloat16_rn(0.f);
        }
        *reinterpret_cast<uint4*>(S.w1 + canon(n, 8 * c, HID)) = *reinterpret_cast<const uint4*>(e);
    }
    for (int i = threadIdx.x; i < HID * (HID / 8); i += nt) {           // W2: 128 rows x 16 chunks
        const int n = i / (HID / 8), c = i % (HID / 8);
        cp_async16_tc(w2 + canon(n, 8 * c, HID), P->W2 + n * LDH + 8 * c);
    }
    for (int i = threadIdx.x; i < OUTP * (HID / 8); i += nt) {          // W3: 16 rows x 16 chunks
        const int n = i / (HID / 8), c = i % (HID / 8);
        cp_async16_tc(w3 + canon(n, 8 * c, OUTP), P->W3 + n * LDH + 8 * c);
    }
    for (int i = threadIdx.x; i < HID; i += nt) { S.b1[i] = P->b1[i]; S.b2[i] = P->b2[i]; }
    for (int i = threadIdx.x; i < OUTP; i += nt) S.b3[i] = P->b3[i];
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Per-thread view of its group: group g, row (TMEM lane) and the lane
// quarter's TMEM address (column 0; the group's slot adds 128 per slot).
struct GroupCtx {
    int g, row;
    uint32_t tlane;
    bool leader;
};

__device__ __forceinline__ GroupCtx group_ctx(const TcSmem& S) {
    GroupCtx c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    c.g = warp / GWARPS;
    c.row = 32 * (warp % GWARPS) + lane;
    c.tlane = S.tmem + ((uint32_t)(32 * (warp % GWARPS)) << 16);
    c.leader = (threadIdx.x % GTHREADS) == 0;
    return c;
}

// The leader takes a free TMEM slot (bounded spin: a slot is released by a
// group that holds it, which never waits for another group); false and the
// error flag on expiry.
__device__ bool slot_take(int* free_slots, int* slot, int* err) {
    volatile int* mask = free_slots;
    const unsigned long long t0 = gtime();
    for (;;) {
        const int m = *mask;
        if (m != 0) {
            const int s = __ffs(m) - 1;
            if (atomicCAS(free_slots, m, m & ~(1 << s)) == m) {
                __threadfence_block();          // acquire: the last holder's reads are done
                *slot = s;
                return true;
            }
            continue;
        }
        if (gtime() - t0 > TC_WAIT_NS) {
            atomicExch(err, 1);
            return false;
        }
        __nanosleep(64);
    }
}

// One layer's MMAs of a tile: A (canonical; K = 48 for layer 0, else 128)
// at shared address a0, the layer's weights as B, into the accumulator at
// TMEM address dcol (lane 0, the accumulator's first column).  The K steps
// advance both descriptors' start address (bits 0-13, in 16-byte units) by
// the bytes of two core-matrix columns; shared memory is below 2^18 bytes,
// so the field does not carry.
template <class Sm>
__device__ __forceinline__ void issue_layer(const Sm& S, int layer, uint32_t dcol, uint32_t a0, bool onto = false) {
    const uint64_t ad = sdesc(a0, (TM / 8) * 128, 128);
    constexpr uint64_t ASTEP = (2 * (TM / 8) * 128) >> 4;
    if (layer == 0) {
        const uint64_t bd = sdesc(su32(S.w1), (HID / 8) * 128, 128);
#pragma unroll
        for (int kk = 0; kk < KX_TC / 16; ++kk)
            mma_f16(dcol, ad + kk * ASTEP, bd + kk * ((2 * (HID / 8) * 128) >> 4), idesc(TM, HID), kk > 0);
    } else if (layer == 1) {
        const uint64_t bd = sdesc(su32(S.w2), (HID / 8) * 128, 128);
#pragma unroll
        for (int kk = 0; kk < HID / 16; ++kk)
            mma_f16(dcol, ad + kk * ASTEP, bd + kk * ((2 * (HID / 8) * 128) >> 4), idesc(TM, HID), onto || kk > 0);
    } else {
        const uint64_t bd = sdesc(su32(S.w3), (OUTP / 8) * 128, 128);
#pragma unroll
        for (int kk = 0; kk < HID / 16; ++kk)
            mma_f16(dcol, ad + kk * ASTEP, bd + kk * ((2 * (OUTP / 8) * 128) >> 4), idesc(TM, OUTP), kk > 0);
    }
}

// Bias + activation of a hidden layer for the thread's row: accumulator
// (tacc: the thread's lane, first column) -> row `row` of the next layer's
// A operand h.
// bias == nullptr: the bias is already in the accumulator (layer 0).
// prefill != nullptr: once a 32-column block is read, it is overwritten with
// prefill (the next layer's bias; that layer's MMAs then accumulate onto it)
__device__ __forceinline__ void epilogue_layer(unsigned char* h, uint32_t tacc, const float* bias, int row,
                                               const float* prefill = nullptr) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t v[32];
        tmem_ld32(tacc + (uint32_t)(32 * q), v);
        tmem_wait_ld();
#pragma unroll
        for (int cb = 0; cb < 32; cb += 16) {
            uint32_t w[8];
            if (bias) {
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const float4 b = *reinterpret_cast<const float4*>(bias + 32 * q + cb + 2 * e);
                    w[e] = bias_act2_tc(v[cb + 2 * e], v[cb + 2 * e + 1], b.x, b.y);
                    w[e + 1] = bias_act2_tc(v[cb + 2 * e + 2], v[cb + 2 * e + 3], b.z, b.w);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    w[e] = act2_tc(__uint_as_float(v[cb + 2 * e]), __uint_as_float(v[cb + 2 * e + 1]));
            }
            *reinterpret_cast<uint4*>(h + canon(row, 32 * q + cb, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(h + canon(row, 32 * q + cb + 8, TM)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        if (prefill) {
            uint32_t b[32];
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
                const uint4 t = *reinterpret_cast<const uint4*>(prefill + 32 * q + e);
                b[e] = t.x; b[e + 1] = t.y; b[e + 2] = t.z; b[e + 3] = t.w;
            }
            tmem_st32(tacc + (uint32_t)(32 * q), b);
        }
    }
    if (prefill) tmem_wait_st();
}

// The three layers of the group's tile (inputs at the start of its operand
// buffer); the leader first takes a TMEM slot, which the group keeps until
// slot_give.  On return the output accumulator (columns 0..15 of the slot)
// is in TMEM.  Returns false if a wait expired.
__device__ bool tile_network(TcSmem& S, const GroupCtx& c, uint32_t& ph, int* err) {
    TcGroup& G = S.grp[c.g];
    if (c.leader && !slot_take(&S.free_slots, &S.slot[c.g], err)) S.abort[c.g] = 1;
    for (int layer = 0; layer < 3; ++layer) {
        if (c.leader && !S.abort[c.g]) {
            fence_after();
            issue_layer(S, layer, S.tmem + (uint32_t)(128 * S.slot[c.g]), su32(G.h));
            mma_commit(&S.mbar[c.g]);
            if (!mbar_wait(&S.mbar[c.g], ph & 1, err)) S.abort[c.g] = 1;
        }
        ++ph;
        group_sync(c.g);
        if (S.abort[c.g]) return false;
        fence_after();
        if (layer == 2) return true;
        epilogue_layer(G.h, c.tlane + (uint32_t)(128 * S.slot[c.g]), layer == 0 ? nullptr : S.b2, c.row);
        fence_async_smem();
        fence_before();
        group_sync(c.g);
    }
    return true;
}

// Output of the group's tile (thread = row): y[0..15] from TMEM + b3.
__device__ __forceinline__ void tile_output(const TcSmem& S, const GroupCtx& c, float (&y)[16]) {
    uint32_t v[16];
    tmem_ld16(c.tlane + (uint32_t)(128 * S.slot[c.g]), v);
    tmem_wait_ld();
#pragma unroll
    for (int o = 0; o < 16; ++o) y[o] = __uint_as_float(v[o]) + S.b3[o];
}

// After the group's last TMEM read of a tile: the slot goes back to the pool.
__device__ __forceinline__ void slot_give(TcSmem& S, const GroupCtx& c) {
    fence_before();
    group_sync(c.g);
    if (c.leader) {
        __threadfence_block();              // release: the group's TMEM reads precede the hand-back
        atomicOr(&S.free_slots, 1 << S.slot[c.g]);
    }
}

__device__ void tc_setup(TcSmem& S, const Packed* P) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x < GROUPS) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.mbar[threadIdx.x])) : "memory");
        S.abort[threadIdx.x] = 0;
        S.slot[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) S.free_slots = (1 << SLOTS) - 1;
    if (threadIdx.x == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_weights_tc(S, P);
    asm volatile("cp.async.wait_all;" ::: "memory");
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

__device__ void tc_teardown(TcSmem& S) {
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(TMEM_COLS) : "memory");
    }
}

__device__ __forceinline__ void mbar_arrive_tc(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}

// Bounded wait on a phase of a closure-kernel barrier: false (and the error
// flag) on expiry, or as soon as another role of the CTA has given up.
__device__ bool cl_wait(int* abort_flag, uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = gtime();
    volatile int* abort = abort_flag;
    while (!mbar_test(bar, parity)) {
        if (*abort) return false;
        if (gtime() - t0 > TC_WAIT_NS) {
            *abort = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

__device__ void cl_setup(ClSmem& S, const Packed* P) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x < CONSUMERS) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.mma[threadIdx.x])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&S.full[threadIdx.x])), "r"(GTHREADS)
                     : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.empty[threadIdx.x])) : "memory");
        S.stop[threadIdx.x] = 0;
    }
    if (threadIdx.x == 0) {
        S.abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_weights_tc(S, P);
    asm volatile("cp.async.wait_all;" ::: "memory");
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

// Fused closure evaluation.  CTA b takes a contiguous run of the 128-cell
// tiles (tiles / grid or one more: the runs differ by at most one tile, so
// no SM carries a round of tiles more than the others); the k-th tile of
// the run belongs to consumer group k mod 4 and producer group k mod 2.  A
// producer group (one thread per cell) gathers its tiles in turn: the
// inputs of its cell, exactly the features of the training sampler, into
// the consumer's input buffer as BF16, and the feature scale s to scl[m],
// once the consumer has released the buffer.  A consumer group runs the
// network on its tiles and writes s * y: R_8^m straight to G11 (with their
// ghost copies), the centre values of I_8^m to ctr[o][M] for the node
// averaging.  Every consumer's tiles come from one producer in order, so
// each barrier phase is waited on at most one phase ahead.
template <class T>
__global__ void __launch_bounds__(CL_THREADS, 1) k_closure_tc(const ClosureArgs<T> A, const Packed* __restrict__ P,
                                                              float* __restrict__ ctr, float* __restrict__ scl,
                                                              int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    ClSmem& S = *reinterpret_cast<ClSmem*>(raw);
    cl_setup(S, P);
    // weights, TMEM and the column table come from host-written data; the
    // state is read below, after the previous kernel of the stream is done
    pdl_trigger();
    pdl_wait();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = warp / GWARPS, row = 32 * (warp % GWARPS) + lane;
    const int nx = A.nx, ny = A.ny;
    const int M = nx * ny;
    const int tiles = (M + TM - 1) / TM;
    const long Pp = A.pitch;
    const int per = tiles / (int)gridDim.x, extra = tiles % (int)gridDim.x;
    const int t0 = (int)blockIdx.x * per + min((int)blockIdx.x, extra);
    const int n = per + ((int)blockIdx.x < extra ? 1 : 0);
    if (g >= CONSUMERS) {
        // producer p: tiles p, p + PRODUCERS, ... of the run, tile k into consumer k mod 4's buffer
        for (int k = g - CONSUMERS; k < n; k += PRODUCERS) {
            const int c = k % CONSUMERS, use = k / CONSUMERS;
            if (use > 0 && !cl_wait(&S.abort, &S.empty[c], (uint32_t)(use - 1) & 1, err)) break;
            const int m = (t0 + k) * TM + row;
            const bool ok = m < M;
            const int ix = ok ? m % nx : 0, iy = ok ? m / nx : 0;
            float f[NMOM], s, inv;
            features36<T>(A.col, stencil(ix, iy, nx, ny, A.p[0], A.p[1], Pp), ok, f, s, inv);
            const float la = ok ? A.lsa[m] : 0.f, ls = ok ? A.lss[m] : 0.f;
            uint32_t w[KX_TC / 2];
#pragma unroll
            for (int q = 0; q < NMOM / 2; ++q) w[q] = pack_bf16_tc(f[2 * q], f[2 * q + 1]);
            w[NMOM / 2] = pack_bf16_tc(la, ls);
#pragma unroll
            for (int q = NMOM / 2 + 1; q < KX_TC / 2; ++q) w[q] = 0u;
            w[BIAS_COL / 2] = pack_bf16_tc(1.f, 1.f);         // the bias columns
            w[BIAS_COL / 2 + 1] = pack_bf16_tc(1.f, 0.f);
#pragma unroll
            for (int q = 0; q < KX_TC / 8; ++q)
                *reinterpret_cast<uint4*>(S.x[c] + canon(row, 8 * q, TM)) =
                    make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
            if (ok) scl[m] = s;
            fence_async_smem();             // the rows are read by the tensor cores (async proxy)
            mbar_arrive_tc(&S.full[c]);
        }
    } else {
        // consumer g: tiles g, g + 4, ... of the run
        const bool leader = (threadIdx.x % GTHREADS) == 0;
        const uint32_t dcol = S.tmem + (uint32_t)(128 * g);
        const uint32_t tacc = dcol + ((uint32_t)(32 * (warp % GWARPS)) << 16);
        uint32_t ph = 0;
        for (int k = g, use = 0; k < n; k += CONSUMERS, ++use) {
            const int m = (t0 + k) * TM + row;
            float s = 0.f;                  // the cell's feature scale, loaded once the tile is produced
            for (int layer = 0; layer < 3; ++layer) {
                if (leader) {
                    bool ok = layer > 0 || cl_wait(&S.abort, &S.full[g], (uint32_t)use & 1, err);
                    if (ok) {
                        fence_after();
                        issue_layer(S, layer, dcol, su32(layer == 0 ? S.x[g] : S.h[g]), layer == 1);
                        mma_commit(&S.mma[g]);
                        ok = cl_wait(&S.abort, &S.mma[g], ph & 1, err);
                        if (ok && layer == 0) mbar_arrive_tc(&S.empty[g]);   // the input buffer is read
                    }
                    if (!ok) S.stop[g] = 1;
                }
                ++ph;
                group_sync(g);
                if (S.stop[g]) break;
                fence_after();
                if (layer == 0 && m < M) s = scl[m];
                if (layer == 2) break;
                // layer 0's epilogue leaves b2 in the accumulator for layer 1 to add onto
                epilogue_layer(S.h[g], tacc, nullptr, row, layer == 0 ? S.b2 : nullptr);
                fence_async_smem();
                fence_before();
                group_sync(g);
            }
            if (S.stop[g]) break;
            // output: s * (y + b3), y from the accumulator's first 16 columns
            uint32_t v[16];
            tmem_ld16(tacc, v);
            tmem_wait_ld();
            if (m < M) {
                const int iy = m / nx, ix = m - iy * nx;
                const long at = (long)(iy + 1) * Pp + ix;     // the cell on G11, ghost row/column offsets below
                const bool gw = ix == (A.p[0] ? nx - 1 : 0), ge = ix == (A.p[0] ? 0 : nx - 1);
                const bool gs = iy == (A.p[1] ? ny - 1 : 0), gn = iy == (A.p[1] ? 0 : ny - 1);
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const float val = s * (__uint_as_float(v[o]) + S.b3[o]);
                    if (A.slot[NMOM + o].x != 0) { ctr[(long)o * M + m] = val; continue; }
                    T* cc = const_cast<T*>(A.col[NMOM + o]);
                    const T tv = (T)val;
                    cc[at] = tv;
                    if (gw) cc[at - 1 - ix] = tv;
                    if (ge) cc[at - ix + nx] = tv;
                    if (gs) cc[ix] = tv;
                    if (gn) cc[(long)(ny + 1) * Pp + ix] = tv;
                }
            }
            fence_before();                 // the accumulator is read before the next tile's MMAs
            group_sync(g);
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(TMEM_COLS) : "memory");
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_forward_tc(const float* __restrict__ X, long M,
                                                              const Packed* __restrict__ P, float* __restrict__ Y,
                                                              int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(raw);
    tc_setup(S, P);
    const GroupCtx c = group_ctx(S);
    const int t = threadIdx.x % GTHREADS;
    const long tiles = (M + TM - 1) / TM;
    uint32_t ph = 0;
    const long per = tiles / (long)gridDim.x, extra = tiles % (long)gridDim.x;
    const long t0 = (long)blockIdx.x * per + min((long)blockIdx.x, extra);
    const long t1 = t0 + per + ((long)blockIdx.x < extra ? 1 : 0);
    for (long tile = t0 + c.g; tile < t1; tile += GROUPS) {
        TcGroup& G = S.grp[c.g];
        // FP32 rows -> BF16 canonical (two columns per step)
        for (int i = t; i < TM * (KX_TC / 2); i += GTHREADS) {
            const int r = i / (KX_TC / 2), col = 2 * (i % (KX_TC / 2));
            const long m = tile * TM + r;
            float a = 0.f, b = 0.f;
            if (m < M && col < NIN) { a = X[m * NIN + col]; b = X[m * NIN + col + 1]; }
            if (col == BIAS_COL) a = b = 1.f;              // the bias columns
            if (col == BIAS_COL + 2) a = 1.f;
            *reinterpret_cast<uint32_t*>(G.h + canon(r, col, TM)) = pack_bf16_tc(a, b);
        }
        fence_async_smem();
        group_sync(c.g);
        if (!tile_network(S, c, ph, err)) break;
        float y[16];
        tile_output(S, c, y);
        const long m = tile * TM + c.row;
        if (m < M)
#pragma unroll
            for (int o = 0; o < NOUT; ++o) Y[m * NOUT + o] = y[o];
        slot_give(S, c);
    }
    tc_teardown(S);
}

// Self-test of the network kernels' bounded waits, with no tensor work: the
// closure kernel's wait and the forward / training kernels' wait for an
// mbarrier phase that nothing completes, and a request for a TMEM slot while
// every slot is held.  All must give up and raise the flag.
__global__ void k_tc_wait_selftest(int* err, int* result) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag, free_slots, slot;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
        free_slots = 0;
        slot = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool waited = cl_wait(&abort_flag, &bar, 0, err);
        const bool took = slot_take(&free_slots, &slot, err);
        const bool plain = mbar_wait(&bar, 0, err);
        result[0] = waited ? 1 : 0;
        result[1] = took ? 1 : 0;
        result[2] = abort_flag;
        result[3] = plain ? 1 : 0;
    }
}

// ------------------------------------------------------------------ training
// One CTA per tile of 128 samples computes the loss and every parameter
// gradient with tcgen05: forward (3 layers), dH2 = dY W3, dH1 = dZ2 W2 and
// the weight gradients dW3^T = H2^T dY, dW2 = dZ2^T H1, dW1 = dZ1^T X, which
// contract over the samples.  Every operand stays in its natural layout (one
// sample per row, as the forward layers and the epilogues write it); where a
// contraction needs it the other way round, the MMA reads it as an MN-major
// operand (transpose bit of the instruction descriptor).  The bias gradients
// b1 and b2 come out of the same MMAs: X and H1 carry a column of ones, so
// dW1 and dW2 gain a column sum_s dZ[s][o].
constexpr int TR_THREADS = 256;          // two warps per TMEM lane quarter, each one half of the columns
constexpr int H1K = HID + 16;            // H1 columns: the hidden values, a ones column, zeros
constexpr int H1_BYTES = (H1K / 8) * (TM / 8) * 128;        // 36864
constexpr int DY_BYTES = (OUTP / 8) * (TM / 8) * 128;       // 4096
constexpr int ONES_X = NIN;              // X column holding 1: b1's gradient in dW1's column NIN
constexpr int ONES_H = HID;              // H1 column holding 1: b2's gradient in dW2's column HID
constexpr uint32_t TC_ACC = 0;           // TMEM: forward accumulators, then dH2, then dH1 (128 columns)
constexpr uint32_t TC_DW3 = 128;         // dW3^T (16 columns)
constexpr uint32_t TC_DW2 = 256;         // dW2 and b2's gradient (144 columns)
constexpr uint32_t TC_DW1 = 400;         // dW1 and b1's gradient (48 columns)
static_assert(TC_DW1 + KX_TC <= TMEM_COLS, "the training accumulators fit in TMEM");
// Layout order matters for nothing but keeps every operand's MN-major
// reading inside the CTA's allocation: the buffers read that way (W3, dY,
// X, H1, H2) are followed by at least 32 KB of the others.
struct TrSmem {
    alignas(128) unsigned char w1[W1_BYTES];    // W1 [o][i], K = 48
    alignas(128) unsigned char w2[W2_BYTES];    // W2 [o][i]
    alignas(128) unsigned char w3[W3_BYTES];    // W3 [o (16)][i]
    alignas(128) unsigned char dy[DY_BYTES];    // dY [s][o (16)]
    alignas(128) unsigned char x[XC_BYTES];     // X [s][48]
    alignas(128) unsigned char h1[H1_BYTES];    // H1 [s][144], later dZ1 in its first 128 columns
    alignas(128) unsigned char h2[H_BYTES];     // H2 [s][128], later dZ2
    alignas(16) float b1[HID];
    alignas(16) float b2[HID];
    alignas(16) float b3[OUTP];
    float wloss[TR_THREADS / 32];
    float wb3[GWARPS][OUTP];
    alignas(8) uint64_t bar;
    uint32_t tmem;
    int stop;
};
static_assert(sizeof(TrSmem) <= 227 * 1024, "training kernel shared memory");

// instruction descriptor with the operands' majorness: ta / tb = 1 reads A / B MN-major
__host__ __device__ constexpr uint32_t idesc_t(int m, int n, int ta, int tb) {
    return idesc(m, n) | ((uint32_t)ta << 15) | ((uint32_t)tb << 16);
}
// K-major reading of a natural buffer of `rows` rows: core matrices 128 bytes
// apart along the rows, (rows / 8) * 128 apart along K; a K step of 16 is
// two of the latter
__device__ __forceinline__ uint64_t kdesc(uint32_t a, int rows) { return sdesc(a, (rows / 8) * 128, 128); }
__device__ __forceinline__ uint64_t kstep(int rows) { return (uint64_t)((2 * (rows / 8) * 128) >> 4); }
// MN-major reading of the same buffer (the contraction runs over its rows):
// along K (the rows) core matrices are 128 bytes apart, along M/N (the
// buffer's columns) (rows / 8) * 128; a K step of 16 rows advances 256 bytes
__device__ __forceinline__ uint64_t mdesc(uint32_t a, int rows) { return sdesc(a, 128, (rows / 8) * 128); }
constexpr uint64_t MSTEP = 256 >> 4;

__device__ __forceinline__ void mma_k(uint32_t d, uint64_t a, uint64_t as, uint64_t b, uint64_t bs, uint32_t id,
                                      int ksteps) {
    for (int kk = 0; kk < ksteps; ++kk) mma_f16(d, a + kk * as, b + kk * bs, id, kk > 0);
}

// Thread 0 commits the MMAs it issued and waits for them; every thread then
// learns whether to stop.  Returns false if a wait expired.
__device__ __forceinline__ bool tr_sync_mma(TrSmem& S, uint32_t& ph, int* err) {
    if (threadIdx.x == 0) {
        mma_commit(&S.bar);
        if (!mbar_wait(&S.bar, ph & 1, err)) S.stop = 1;
    }
    ++ph;
    __syncthreads();
    fence_after();
    return S.stop == 0;
}
// Before the next MMAs read what the threads wrote: generic -> async proxy,
// TMEM reads ordered before the MMAs that overwrite the columns.
__device__ __forceinline__ void tr_publish() {
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

// dZ = dH * (1 - H^2) for the thread's row and 64 columns starting at c0:
// dH from TMEM, H (BF16) read from and dZ written over the natural buffer
__device__ __forceinline__ void tanh_backward(unsigned char* buf, uint32_t tacc, int row, int c0) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        uint32_t v[32];
        tmem_ld32(tacc + (uint32_t)(c0 + 32 * q), v);
        tmem_wait_ld();
#pragma unroll
        for (int cb = 0; cb < 32; cb += 8) {
            uint4* at = reinterpret_cast<uint4*>(buf + canon(row, c0 + 32 * q + cb, TM));
            const uint4 hv = *at;
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&hw[e]);
                const float h0 = __low2float(h), h1 = __high2float(h);
                w[e] = pack_bf16_tc(__uint_as_float(v[cb + 2 * e]) * (1.f - h0 * h0),
                                    __uint_as_float(v[cb + 2 * e + 1]) * (1.f - h1 * h1));
            }
            *at = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

__global__ void __launch_bounds__(TR_THREADS, 1) k_loss_grad_tc(const float* __restrict__ X, const float* __restrict__ T,
                                                                const int* __restrict__ idx, long B,
                                                                const Packed* __restrict__ P, float* __restrict__ part,
                                                                int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    TrSmem& S = *reinterpret_cast<TrSmem*>(raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp % GWARPS, half = warp / GWARPS;
    const int row = 32 * quarter + lane;                 // TMEM lane: a sample, or an output / input index
    const long row0 = (long)blockIdx.x * TM;
    float* out = part + (long)blockIdx.x * (NPARAM + 1);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.stop = 0;
    }
    if (warp == 0)
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem)),
                     "r"(TMEM_COLS) : "memory");
    // weights (natural layouts; Packed's padding columns are zero)
    {
        const uint32_t w1 = su32(S.w1), w2 = su32(S.w2), w3 = su32(S.w3);
        for (int i = threadIdx.x; i < HID * (KX_TC / 8); i += TR_THREADS) {
            const int n = i / (KX_TC / 8), c = i % (KX_TC / 8);
            cp_async16_tc(w1 + canon(n, 8 * c, HID), P->W1 + n * LDX + 8 * c);
        }
        for (int i = threadIdx.x; i < HID * (HID / 8); i += TR_THREADS) {
            const int n = i / (HID / 8), c = i % (HID / 8);
            cp_async16_tc(w2 + canon(n, 8 * c, HID), P->W2 + n * LDH + 8 * c);
        }
        for (int i = threadIdx.x; i < OUTP * (HID / 8); i += TR_THREADS) {
            const int n = i / (HID / 8), c = i % (HID / 8);
            cp_async16_tc(w3 + canon(n, 8 * c, OUTP), P->W3 + n * LDH + 8 * c);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int i = threadIdx.x; i < HID; i += TR_THREADS) { S.b1[i] = P->b1[i]; S.b2[i] = P->b2[i]; }
        if (threadIdx.x < OUTP) S.b3[threadIdx.x] = P->b3[threadIdx.x];
    }
    // inputs: sample rows (gathered through idx), a ones column, zeros; H1's
    // ones column and zeros behind it
    {
        const int r = threadIdx.x % TM, side = threadIdx.x / TM;        // half a row each
        const long m = row0 + r;
        const bool ok = m < B;
        const float* xs = X + (ok ? (idx ? (long)idx[m] : m) : 0) * NIN;
#pragma unroll
        for (int c = 3 * side; c < 3 * side + 3; ++c) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float v[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int col = 8 * c + 2 * e + h;
                    v[h] = col < NIN ? (ok ? xs[col] : 0.f) : col == ONES_X ? 1.f : 0.f;
                }
                w[e] = pack_bf16_tc(v[0], v[1]);
            }
            *reinterpret_cast<uint4*>(S.x + canon(r, 8 * c, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        const uint32_t one = pack_bf16_tc(1.f, 0.f);
        *reinterpret_cast<uint4*>(S.h1 + canon(r, HID + 8 * side, TM)) =
            side == 0 ? make_uint4(one, 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    }
    // the targets of the thread's sample (rows of the output epilogue), loaded
    // now so that their latency hides behind the forward layers
    float tgt[NOUT];
    {
        const long m = row0 + row;
        const bool valid = half == 0 && m < B;
        const float* ts = T + (valid ? (idx ? (long)idx[m] : m) : 0) * NOUT;
#pragma unroll
        for (int o = 0; o < NOUT; ++o) tgt[o] = valid ? ts[o] : 0.f;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    fence_before();
    tr_publish();
    const uint32_t tm = S.tmem;
    const uint32_t tl = tm + ((uint32_t)(32 * quarter) << 16);      // this warp's lane quarter, column 0
    uint32_t ph = 0;
    bool ok = true;
    // ---- forward: Z1 = X W1^T, H1 = tanh(Z1 + b1)
    if (threadIdx.x == 0) mma_k(tm + TC_ACC, kdesc(su32(S.x), TM), kstep(TM), kdesc(su32(S.w1), HID), kstep(HID),
                                idesc(TM, HID), KX_TC / 16);
    ok = tr_sync_mma(S, ph, err);
    if (ok) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c0 = 64 * half + 32 * q;
            uint32_t v[32];
            tmem_ld32(tl + TC_ACC + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int cb = 0; cb < 32; cb += 8) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = bias_act2_tc(v[cb + 2 * e], v[cb + 2 * e + 1], S.b1[c0 + cb + 2 * e], S.b1[c0 + cb + 2 * e + 1]);
                *reinterpret_cast<uint4*>(S.h1 + canon(row, c0 + cb, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tr_publish();
        // Z2 = H1 W2^T, H2 = tanh(Z2 + b2)
        if (threadIdx.x == 0) mma_k(tm + TC_ACC, kdesc(su32(S.h1), TM), kstep(TM), kdesc(su32(S.w2), HID), kstep(HID),
                                    idesc(TM, HID), HID / 16);
        ok = tr_sync_mma(S, ph, err);
    }
    if (ok) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c0 = 64 * half + 32 * q;
            uint32_t v[32];
            tmem_ld32(tl + TC_ACC + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int cb = 0; cb < 32; cb += 8) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    w[e] = bias_act2_tc(v[cb + 2 * e], v[cb + 2 * e + 1], S.b2[c0 + cb + 2 * e], S.b2[c0 + cb + 2 * e + 1]);
                *reinterpret_cast<uint4*>(S.h2 + canon(row, c0 + cb, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tr_publish();
        // Y = H2 W3^T (+ b3 below)
        if (threadIdx.x == 0) mma_k(tm + TC_ACC, kdesc(su32(S.h2), TM), kstep(TM), kdesc(su32(S.w3), OUTP), kstep(OUTP),
                                    idesc(TM, OUTP), HID / 16);
        ok = tr_sync_mma(S, ph, err);
    }
    if (ok) {
        // dY = 2 (y - t) / (B 9) on the tile's samples and the 9 outputs, else 0;
        // the loss and b3's gradient (column sums of the BF16 dY) per warp
        const float inv = 2.f / (float)(B * NOUT);
        if (half == 0) {
            uint32_t v[16];
            tmem_ld16(tl + TC_ACC, v);
            tmem_wait_ld();
            const bool valid = row0 + row < B;
            float lsum = 0.f, d[OUTP];
#pragma unroll
            for (int o = 0; o < OUTP; ++o) {
                d[o] = 0.f;
                if (valid && o < NOUT) {
                    const float rr = __uint_as_float(v[o]) + S.b3[o] - tgt[o];
                    lsum += rr * rr;
                    d[o] = inv * rr;
                }
            }
            uint32_t w[OUTP / 2];
#pragma unroll
            for (int e = 0; e < OUTP / 2; ++e) w[e] = pack_bf16_tc(d[2 * e], d[2 * e + 1]);
            *reinterpret_cast<uint4*>(S.dy + canon(row, 0, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(S.dy + canon(row, 8, TM)) = make_uint4(w[4], w[5], w[6], w[7]);
#pragma unroll
            for (int o = 0; o < NOUT; ++o) {
                const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162*>(&w[o / 2]);
                float c = (o & 1) ? __high2float(pr) : __low2float(pr);
#pragma unroll
                for (int sh = 16; sh > 0; sh >>= 1) c += __shfl_xor_sync(0xffffffffu, c, sh);
                if (lane == 0) S.wb3[quarter][o] = c;
            }
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, sh);
            if (lane == 0) S.wloss[quarter] = lsum / (float)(B * NOUT);
        }
        tr_publish();
        // dH2 = dY W3 (K = 16 outputs; W3 read MN-major) and dW3^T = H2^T dY
        // (M = inputs, N = outputs, K = samples; both read MN-major)
        if (threadIdx.x == 0) {
            mma_k(tm + TC_ACC, kdesc(su32(S.dy), TM), kstep(TM), mdesc(su32(S.w3), OUTP), MSTEP, idesc_t(TM, HID, 0, 1), 1);
            mma_k(tm + TC_DW3, mdesc(su32(S.h2), TM), MSTEP, mdesc(su32(S.dy), TM), MSTEP, idesc_t(HID, OUTP, 1, 1),
                  TM / 16);
        }
        ok = tr_sync_mma(S, ph, err);
    }
    if (ok) {
        // dZ2 = dH2 (1 - H2^2) over H2; dW3 from its transpose (lane = input)
        tanh_backward(S.h2, tl + TC_ACC, row, 64 * half);
        if (half == 1) {
            uint32_t v[16];
            tmem_ld16(tl + TC_DW3, v);
            tmem_wait_ld();
#pragma unroll
            for (int o = 0; o < NOUT; ++o) out[OFF_W3 + o * HID + row] = __uint_as_float(v[o]);
        }
        tr_publish();
        // dH1 = dZ2 W2 (W2 read MN-major) and dW2 = dZ2^T [H1 | 1]
        // (M = outputs, N = inputs and the ones column, K = samples)
        if (threadIdx.x == 0) {
            mma_k(tm + TC_ACC, kdesc(su32(S.h2), TM), kstep(TM), mdesc(su32(S.w2), HID), MSTEP, idesc_t(TM, HID, 0, 1),
                  HID / 16);
            mma_k(tm + TC_DW2, mdesc(su32(S.h2), TM), MSTEP, mdesc(su32(S.h1), TM), MSTEP, idesc_t(HID, H1K, 1, 1),
                  TM / 16);
        }
        ok = tr_sync_mma(S, ph, err);
    }
    if (ok) {
        // dZ1 = dH1 (1 - H1^2) over H1's first 128 columns; dW2 and b2's gradient
        tanh_backward(S.h1, tl + TC_ACC, row, 64 * half);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int c0 = 64 * half + 32 * q;
            uint32_t v[32];
            tmem_ld32(tl + TC_DW2 + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) out[OFF_W2 + row * HID + c0 + e] = __uint_as_float(v[e]);
        }
        if (half == 0) {
            uint32_t v[16];
            tmem_ld16(tl + TC_DW2 + (uint32_t)ONES_H, v);
            tmem_wait_ld();
            out[OFF_B2 + row] = __uint_as_float(v[0]);
        }
        tr_publish();
        // dW1 = dZ1^T [X | 1] (M = outputs, N = the 48 input columns, K = samples)
        if (threadIdx.x == 0)
            mma_k(tm + TC_DW1, mdesc(su32(S.h1), TM), MSTEP, mdesc(su32(S.x), TM), MSTEP, idesc_t(HID, KX_TC, 1, 1),
                  TM / 16);
        ok = tr_sync_mma(S, ph, err);
    }
    if (ok) {
        if (half == 0) {
            uint32_t v[32];
            tmem_ld32(tl + TC_DW1, v);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e) out[OFF_W1 + row * NIN + e] = __uint_as_float(v[e]);
        } else {
            uint32_t v[16];
            tmem_ld16(tl + TC_DW1 + 32u, v);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < NIN - 32; ++e) out[OFF_W1 + row * NIN + 32 + e] = __uint_as_float(v[e]);
            out[OFF_B1 + row] = __uint_as_float(v[ONES_X - 32]);
        }
        if (threadIdx.x < NOUT) {
            float c = 0.f;
            for (int q = 0; q < GWARPS; ++q) c += S.wb3[q][threadIdx.x];
            out[OFF_B3 + threadIdx.x] = c;
        }
        if (threadIdx.x == 0) {
            float l = 0.f;
            for (int q = 0; q < GWARPS; ++q) l += S.wloss[q];
            out[NPARAM] = l;
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(TMEM_COLS) : "memory");
    }
}

int sms_tc() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

template <class K>
int smem_attr(K kernel, bool& done) {
    if (done) return 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem)) != cudaSuccess)
        return -4;
    done = true;
    return 0;
}

}  // namespace

size_t tc_smem_bytes() { return sizeof(TcSmem); }

int tc_wait_selftest(int* gave_up) {
    int* d = nullptr;
    if (cudaMalloc(&d, 5 * sizeof(int)) != cudaSuccess) return -4;
    int h[5] = {0, -1, -1, -1, -1};
    cudaError_t e = cudaMemcpy(d, h, 5 * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_tc_wait_selftest<<<1, 32>>>(d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, 5 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return -4;
    *gave_up = (h[0] == 1 && h[1] == 0 && h[2] == 0 && h[3] == 1 && h[4] == 0) ? 1 : 0;
    return 0;
}

int loss_grad_tc(const float* X, const float* T, const int* idx, long B, const Packed* P, float* part, int* err,
                 void* stream) {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_loss_grad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TrSmem)) !=
            cudaSuccess)
            return -4;
        attr = true;
    }
    const long blocks = (B + TM - 1) / TM;
    k_loss_grad_tc<<<(unsigned)blocks, TR_THREADS, sizeof(TrSmem), (cudaStream_t)stream>>>(X, T, idx, B, P, part, err);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

int forward_tc(const float* X, long M, const Packed* P, float* Y, int* err, void* stream) {
    if (M <= 0) return 0;
    static bool attr = false;
    if (smem_attr(k_forward_tc, attr)) return -4;
    long blocks = (M + TM * GROUPS - 1) / (TM * GROUPS);
    if (blocks > sms_tc()) blocks = sms_tc();
    k_forward_tc<<<(unsigned)blocks, TC_THREADS, sizeof(TcSmem), (cudaStream_t)stream>>>(X, M, P, Y, err);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <class T>
int closure_tc(const ClosureArgs<T>& A, const Packed* P, float* ctr, float* scl, int* err, void* stream) {
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_closure_tc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ClSmem)) !=
            cudaSuccess)
            return -4;
        attr = true;
    }
    const long M = (long)A.nx * A.ny;
    if (M <= 0) return 0;
    long blocks = (M + TM * CONSUMERS - 1) / (TM * CONSUMERS);
    if (blocks > sms_tc()) blocks = sms_tc();
    const cudaError_t e = launch_pdl(k_closure_tc<T>, dim3((unsigned)blocks), dim3(CL_THREADS), sizeof(ClSmem),
                                     (cudaStream_t)stream, true, A, P, ctr, scl, err);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template int closure_tc<float>(const ClosureArgs<float>&, const Packed*, float*, float*, int*, void*);
template int closure_tc<double>(const ClosureArgs<double>&, const Packed*, float*, float*, int*, void*);

}  // namespace mlp
}  // namespace starmap
