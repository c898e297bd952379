// The closure network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One CTA per SM: four independent groups of 4 warps, each owning a tile of
// 128 samples at a time (its own TMEM columns, operand buffers, mbarrier and
// named barrier; the weights are shared).  Operands live in shared
// memory in the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices; an M x K (or N x K) operand stores element (r, k) at
//     (k / 8) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2  bytes,
// LBO = (rows / 8) * 128 (core matrices adjacent along M/N are 128 bytes
// apart = SBO, along K LBO apart).  One elected thread issues the layer's
// tcgen05.mma (M = 128, K = 16 per instruction, BF16 x BF16 -> FP32) into the
// group's 128-column TMEM accumulator and commits it to the group's
// mbarrier; the group's 4 warps then read the accumulator with tcgen05.ld
// (thread = row = TMEM lane), add the bias, apply the shared activation
// (tanh.approx.bf16x2 of the BF16-rounded pre-activation) and write the
// next layer's operand back to shared memory.  Layers: 38(48) -> 128
// (3 MMAs), 128 -> 128 (8 MMAs), 128 -> 16 (9 used, 8 MMAs with N = 16).
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
constexpr int GROUPS = 4;                // independent 4-warp groups per CTA, one tile each
constexpr int GWARPS = 4;
constexpr int GTHREADS = GWARPS * 32;    // one thread per tile row (= TMEM lane)
constexpr int TC_THREADS = GROUPS * GTHREADS;
constexpr int KX_TC = 48;                // input width padded to the MMA K step
constexpr int XC_BYTES = (KX_TC / 8) * (TM / 8) * 128;       // 12288
constexpr int W1_BYTES = (KX_TC / 8) * (HID / 8) * 128;      // 12288
constexpr int W2_BYTES = (HID / 8) * (HID / 8) * 128;        // 32768
constexpr int W3_BYTES = (HID / 8) * (OUTP / 8) * 128;       // 4096
constexpr int H_BYTES = (HID / 8) * (TM / 8) * 128;          // 32768
constexpr int TMEM_COLS = 512;           // 128 accumulator columns per group
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

struct TcGroup {
    alignas(128) unsigned char x[XC_BYTES];
    alignas(128) unsigned char h[H_BYTES];
};
struct TcSmem {
    alignas(1024) unsigned char w1[W1_BYTES];
    alignas(128) unsigned char w2[W2_BYTES];
    alignas(128) unsigned char w3[W3_BYTES];
    TcGroup grp[GROUPS];
    float b1[HID], b2[HID], b3[OUTP];
    alignas(8) uint64_t mbar[GROUPS];
    uint32_t tmem;
    int abort[GROUPS];
};
static_assert(sizeof(TcSmem) <= 227 * 1024, "tile groups must fit in shared memory");

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
__device__ __forceinline__ uint32_t idesc(int m, int n) {
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
// 64 consecutive columns of this warp's 32 lanes in one load
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
          "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
          "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
          "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(su32(bar)), "r"(parity) : "memory");
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

__device__ __forceinline__ void cp_async16_tc(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
}

// Weights (row-major padded BF16 of Packed) into the canonical layouts,
// 16-byte pieces by cp.async (no register round trip); the caller waits.
__device__ void load_weights_tc(TcSmem& S, const Packed* P) {
    const uint32_t w1 = su32(S.w1), w2 = su32(S.w2), w3 = su32(S.w3);
    for (int i = threadIdx.x; i < HID * (KX_TC / 8); i += TC_THREADS) {         // W1: 128 rows x 6 chunks
        const int n = i / (KX_TC / 8), c = i % (KX_TC / 8);
        cp_async16_tc(w1 + canon(n, 8 * c, HID), P->W1 + n * LDX + 8 * c);
    }
    for (int i = threadIdx.x; i < HID * (HID / 8); i += TC_THREADS) {           // W2: 128 rows x 16 chunks
        const int n = i / (HID / 8), c = i % (HID / 8);
        cp_async16_tc(w2 + canon(n, 8 * c, HID), P->W2 + n * LDH + 8 * c);
    }
    for (int i = threadIdx.x; i < OUTP * (HID / 8); i += TC_THREADS) {          // W3: 16 rows x 16 chunks
        const int n = i / (HID / 8), c = i % (HID / 8);
        cp_async16_tc(w3 + canon(n, 8 * c, OUTP), P->W3 + n * LDH + 8 * c);
    }
    for (int i = threadIdx.x; i < HID; i += TC_THREADS) { S.b1[i] = P->b1[i]; S.b2[i] = P->b2[i]; }
    for (int i = threadIdx.x; i < OUTP; i += TC_THREADS) S.b3[i] = P->b3[i];
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Per-thread view of its group: group g, row (TMEM lane) and TMEM base.
struct GroupCtx {
    int g, row;
    uint32_t tacc;                      // this thread's lane quarter, the group's columns
    bool leader;
};

__device__ __forceinline__ GroupCtx group_ctx(const TcSmem& S) {
    GroupCtx c;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    c.g = warp / GWARPS;
    c.row = 32 * (warp % GWARPS) + lane;
    c.tacc = S.tmem + ((uint32_t)(32 * (warp % GWARPS)) << 16) + (uint32_t)(128 * c.g);
    c.leader = (threadIdx.x % GTHREADS) == 0;
    return c;
}

// The three layers of the group's tile (inputs in its x buffer); on return
// the output accumulator (columns 0..15 of the group) is in TMEM.  Returns
// false if a wait expired.
__device__ bool tile_network(TcSmem& S, const GroupCtx& c, uint32_t& ph, int* err) {
    TcGroup& G = S.grp[c.g];
    const uint32_t dcol = S.tmem + (uint32_t)(128 * c.g);     // lane 0 of the group's accumulator
    const uint32_t id128 = idesc(TM, HID), id16 = idesc(TM, OUTP);
    for (int layer = 0; layer < 3; ++layer) {
        if (c.leader) {
            fence_after();
            if (layer == 0) {
                const uint32_t a0 = su32(G.x), b0 = su32(S.w1);
                for (int kk = 0; kk < KX_TC / 16; ++kk)
                    mma_f16(dcol, sdesc(a0 + kk * 2 * (TM / 8) * 128, (TM / 8) * 128, 128),
                            sdesc(b0 + kk * 2 * (HID / 8) * 128, (HID / 8) * 128, 128), id128, kk > 0);
            } else {
                const uint32_t a0 = su32(G.h), b0 = su32(layer == 1 ? S.w2 : S.w3);
                const int nb = layer == 1 ? HID : OUTP;
                for (int kk = 0; kk < HID / 16; ++kk)
                    mma_f16(dcol, sdesc(a0 + kk * 2 * (TM / 8) * 128, (TM / 8) * 128, 128),
                            sdesc(b0 + kk * 2 * (nb / 8) * 128, (nb / 8) * 128, 128), layer == 1 ? id128 : id16,
                            kk > 0);
            }
            mma_commit(&S.mbar[c.g]);
            if (!mbar_wait(&S.mbar[c.g], ph & 1, err)) S.abort[c.g] = 1;
        }
        ++ph;
        group_sync(c.g);
        if (S.abort[c.g]) return false;
        fence_after();
        if (layer == 2) return true;
        // bias + activation: accumulator -> next layer's A operand in G.h
        const float* bias = layer == 0 ? S.b1 : S.b2;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t v[64];
            tmem_ld64(c.tacc + (uint32_t)(64 * half), v);
            tmem_wait_ld();
#pragma unroll
            for (int cb = 0; cb < 64; cb += 16) {
                uint32_t w[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int col = 64 * half + cb + 2 * e;
                    w[e] = act2_tc(__uint_as_float(v[cb + 2 * e]) + bias[col],
                                   __uint_as_float(v[cb + 2 * e + 1]) + bias[col + 1]);
                }
                *reinterpret_cast<uint4*>(G.h + canon(c.row, 64 * half + cb, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4*>(G.h + canon(c.row, 64 * half + cb + 8, TM)) = make_uint4(w[4], w[5], w[6], w[7]);
            }
        }
        fence_async_smem();
        fence_before();
        group_sync(c.g);
    }
    return true;
}

// Output of the group's tile (thread = row): y[0..15] from TMEM + b3.
__device__ __forceinline__ void tile_output(const TcSmem& S, const GroupCtx& c, float (&y)[16]) {
    uint32_t v[16];
    tmem_ld16(c.tacc, v);
    tmem_wait_ld();
#pragma unroll
    for (int o = 0; o < 16; ++o) y[o] = __uint_as_float(v[o]) + S.b3[o];
}

__device__ void tc_setup(TcSmem& S, const Packed* P) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x < GROUPS) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.mbar[threadIdx.x])) : "memory");
        S.abort[threadIdx.x] = 0;
    }
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

// Fused closure evaluation: four groups per CTA work on their own tiles of
// 128 cells (the CTA's contiguous run of tiles, group g taking every fourth
// from the g-th; the runs of the CTAs differ by at most one tile, so no SM
// carries a round of tiles more than the others).  Each
// thread of a group gathers the inputs of its cell (exactly the features
// of the training sampler) into the group's operand buffer, the group runs
// the network, and the thread writes s * y: R_8^m straight to G11 (with
// their ghost copies), the centre values of I_8^m to ctr[o][M] for the node
// averaging.  While one group gathers or waits for its MMAs, the others
// run their epilogues, so load, tensor and MUFU latencies overlap.
template <class T>
__global__ void __launch_bounds__(TC_THREADS, 1) k_closure_tc(const ClosureArgs<T> A, const Packed* __restrict__ P,
                                                              float* __restrict__ ctr, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(raw);
    __shared__ const T* colp[NMOM];
    column_table(A, colp, NMOM);
    tc_setup(S, P);                         // ends with a CTA barrier: colp is visible
    // weights, TMEM and the column table come from host-written data; the
    // state is read below, after the previous kernel of the stream is done
    pdl_trigger();
    pdl_wait();
    const GroupCtx c = group_ctx(S);
    const int nx = A.nx, ny = A.ny;
    const int M = nx * ny;
    const int tiles = (M + TM - 1) / TM;
    const long Pp = A.pitch;
    uint32_t ph = 0;
    // CTA b takes a contiguous run of tiles/grid or one more tiles (the
    // runs differ by at most one tile), its groups every GROUPS-th of them
    const int per = tiles / (int)gridDim.x, extra = tiles % (int)gridDim.x;
    const int t0 = (int)blockIdx.x * per + min((int)blockIdx.x, extra);
    const int t1 = t0 + per + ((int)blockIdx.x < extra ? 1 : 0);
    for (int tile = t0 + c.g; tile < t1; tile += GROUPS) {
        TcGroup& G = S.grp[c.g];
        const int m = tile * TM + c.row;
        const bool ok = m < M;
        const int ix = ok ? m % nx : 0, iy = ok ? m / nx : 0;
        float f[NMOM], s, inv;
        features36<T>(colp, stencil(ix, iy, nx, ny, A.p[0], A.p[1], Pp), ok, f, s, inv);
        {
            const float la = ok ? A.lsa[m] : 0.f, ls = ok ? A.lss[m] : 0.f;
            uint32_t w[KX_TC / 2];
#pragma unroll
            for (int q = 0; q < NMOM / 2; ++q) w[q] = pack_bf16_tc(f[2 * q], f[2 * q + 1]);
            w[NMOM / 2] = pack_bf16_tc(la, ls);
#pragma unroll
            for (int q = NMOM / 2 + 1; q < KX_TC / 2; ++q) w[q] = 0u;
#pragma unroll
            for (int q = 0; q < KX_TC / 8; ++q)
                *reinterpret_cast<uint4*>(G.x + canon(c.row, 8 * q, TM)) =
                    make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
        }
        fence_async_smem();
        group_sync(c.g);
        if (!tile_network(S, c, ph, err)) break;
        float y[16];
        tile_output(S, c, y);
        if (ok) {
#pragma unroll
            for (int o = 0; o < NOUT; ++o) {
                const float val = s * y[o];
                if (A.slot[NMOM + o].x != 0) { ctr[(long)o * M + m] = val; continue; }
                T* cc = A.g[0].base + (long)A.slot[NMOM + o].y * A.g[0].cstride;
                const T tv = (T)val;
                cc[(long)(iy + 1) * Pp + ix] = tv;
                if (ix == (A.p[0] ? nx - 1 : 0)) cc[(long)(iy + 1) * Pp - 1] = tv;
                if (ix == (A.p[0] ? 0 : nx - 1)) cc[(long)(iy + 1) * Pp + nx] = tv;
                if (iy == (A.p[1] ? ny - 1 : 0)) cc[ix] = tv;
                if (iy == (A.p[1] ? 0 : ny - 1)) cc[(long)(ny + 1) * Pp + ix] = tv;
            }
        }
        fence_before();
        group_sync(c.g);
    }
    tc_teardown(S);
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
            *reinterpret_cast<uint32_t*>(G.x + canon(r, col, TM)) = pack_bf16_tc(a, b);
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
        fence_before();
        group_sync(c.g);
    }
    tc_teardown(S);
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
int closure_tc(const ClosureArgs<T>& A, const Packed* P, float* ctr, int* err, void* stream) {
    static bool attr = false;
    if (smem_attr(k_closure_tc<T>, attr)) return -4;
    const long M = (long)A.nx * A.ny;
    if (M <= 0) return 0;
    long blocks = (M + TM * GROUPS - 1) / (TM * GROUPS);
    if (blocks > sms_tc()) blocks = sms_tc();
    const cudaError_t e = launch_pdl(k_closure_tc<T>, dim3((unsigned)blocks), dim3(TC_THREADS), sizeof(TcSmem),
                                     (cudaStream_t)stream, true, A, P, ctr, err);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template int closure_tc<float>(const ClosureArgs<float>&, const Packed*, float*, int*, void*);
template int closure_tc<double>(const ClosureArgs<double>&, const Packed*, float*, int*, void*);

}  // namespace mlp
}  // namespace starmap
