// The closure network on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// One CTA (8 warps) owns 128 samples at a time.  Operands live in shared
// memory in the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices; an M x K (or N x K) operand stores element (r, k) at
//     (k / 8) * LBO + (r / 8) * 128 + (r % 8) * 16 + (k % 8) * 2  bytes,
// LBO = (rows / 8) * 128 (core matrices adjacent along M/N are 128 bytes
// apart = SBO, along K LBO apart).  One elected thread issues the layer's
// tcgen05.mma (M = 128, K = 16 per instruction, BF16 x BF16 -> FP32) into a
// 128-column TMEM accumulator and commits it to an mbarrier; all 8 warps
// then read the accumulator with tcgen05.ld (warp w: lanes 32 (w % 4)..,
// columns 64 (w / 4)..), add the bias, apply the shared activation
// (tanh.approx.bf16x2 of the BF16-rounded pre-activation) and write the
// next layer's operand back to shared memory.  Layers: 38(48) -> 128
// (3 MMAs), 128 -> 128 (8 MMAs), 128 -> 16 (9 used, 8 MMAs with N = 16).
// Every wait is bounded; on expiry the kernel raises the error flag, skips
// the rest, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "mlp.h"

namespace starmap {
namespace mlp {

namespace {

constexpr int TM = 128;                  // samples per tile (MMA M)
constexpr int TC_THREADS = 256;
constexpr int KX_TC = 48;                // input width padded to the MMA K step
constexpr int XC_BYTES = (KX_TC / 8) * (TM / 8) * 128;       // 12288
constexpr int W1_BYTES = (KX_TC / 8) * (HID / 8) * 128;      // 12288
constexpr int W2_BYTES = (HID / 8) * (HID / 8) * 128;        // 32768
constexpr int W3_BYTES = (HID / 8) * (OUTP / 8) * 128;       // 4096
constexpr int H_BYTES = (HID / 8) * (TM / 8) * 128;          // 32768
// TMEM columns per CTA and CTAs per SM.  Sized generously: an operand
// descriptor read with leading and stride offsets swapped would span up to
// 15 * 2048 + 256 bytes past its start; the shared layout below keeps that
// inside this CTA's allocation (OVERREAD), and 512 columns cover any N.
constexpr int TMEM_COLS = 512;
constexpr int TC_MINB = 1;
constexpr int OVERREAD = 15 * 2048 + 256;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;

struct TcSmem {
    alignas(1024) unsigned char w1[W1_BYTES];
    alignas(128) unsigned char w2[W2_BYTES];
    alignas(128) unsigned char w3[W3_BYTES];
    alignas(128) unsigned char x[2][XC_BYTES];
    alignas(128) unsigned char h[H_BYTES];
    float b1[HID], b2[HID], b3[OUTP];
    alignas(8) uint64_t mbar;
    uint32_t tmem;
    int abort;
    unsigned char guard[OVERREAD];       // never accessed by the kernel's own code
};

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

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
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

// Weights (row-major padded BF16 of Packed) into the canonical layouts.
__device__ void load_weights_tc(TcSmem& S, const Packed* P) {
    for (int i = threadIdx.x; i < HID * (KX_TC / 8); i += TC_THREADS) {         // W1: 128 rows x 6 chunks
        const int n = i / (KX_TC / 8), c = i % (KX_TC / 8);
        *reinterpret_cast<uint4*>(S.w1 + canon(n, 8 * c, HID)) = *reinterpret_cast<const uint4*>(P->W1 + n * LDX + 8 * c);
    }
    for (int i = threadIdx.x; i < HID * (HID / 8); i += TC_THREADS) {           // W2: 128 rows x 16 chunks
        const int n = i / (HID / 8), c = i % (HID / 8);
        *reinterpret_cast<uint4*>(S.w2 + canon(n, 8 * c, HID)) = *reinterpret_cast<const uint4*>(P->W2 + n * LDH + 8 * c);
    }
    for (int i = threadIdx.x; i < OUTP * (HID / 8); i += TC_THREADS) {          // W3: 16 rows x 16 chunks
        const int n = i / (HID / 8), c = i % (HID / 8);
        *reinterpret_cast<uint4*>(S.w3 + canon(n, 8 * c, OUTP)) = *reinterpret_cast<const uint4*>(P->W3 + n * LDH + 8 * c);
    }
    for (int i = threadIdx.x; i < HID; i += TC_THREADS) { S.b1[i] = P->b1[i]; S.b2[i] = P->b2[i]; }
    for (int i = threadIdx.x; i < OUTP; i += TC_THREADS) S.b3[i] = P->b3[i];
}

// The three layers of the tile whose inputs sit in S.x[buf]; on return the
// output accumulator (columns 0..15) is in TMEM and `ph` has advanced.
// Returns false if a wait expired.
__device__ bool tile_network(TcSmem& S, int buf, uint32_t& ph, int* err) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane;            // TMEM lane = sample row of this thread
    const int col0 = 64 * (warp >> 2);                  // this warp's column half
    const uint32_t tm = S.tmem;
    const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
    const uint32_t id128 = idesc(TM, HID), id16 = idesc(TM, OUTP);
    for (int layer = 0; layer < 3; ++layer) {
        // issue the layer
        if (threadIdx.x == 0) {
            fence_after();
            if (layer == 0) {
                const uint32_t a0 = su32(S.x[buf]), b0 = su32(S.w1);
                for (int kk = 0; kk < KX_TC / 16; ++kk)
                    mma_f16(tm, sdesc(a0 + kk * 2 * (TM / 8) * 128, (TM / 8) * 128, 128),
                            sdesc(b0 + kk * 2 * (HID / 8) * 128, (HID / 8) * 128, 128), id128, kk > 0);
            } else if (layer == 1) {
                const uint32_t a0 = su32(S.h), b0 = su32(S.w2);
                for (int kk = 0; kk < HID / 16; ++kk)
                    mma_f16(tm, sdesc(a0 + kk * 2 * (TM / 8) * 128, (TM / 8) * 128, 128),
                            sdesc(b0 + kk * 2 * (HID / 8) * 128, (HID / 8) * 128, 128), id128, kk > 0);
            } else {
                const uint32_t a0 = su32(S.h), b0 = su32(S.w3);
                for (int kk = 0; kk < HID / 16; ++kk)
                    mma_f16(tm, sdesc(a0 + kk * 2 * (TM / 8) * 128, (TM / 8) * 128, 128),
                            sdesc(b0 + kk * 2 * (OUTP / 8) * 128, (OUTP / 8) * 128, 128), id16, kk > 0);
            }
            mma_commit(&S.mbar);
        }
        const bool ok = mbar_wait(&S.mbar, ph & 1, err);
        ++ph;
        if (!ok) S.abort = 1;
        __syncthreads();
        if (S.abort) return false;
        fence_after();
        if (layer == 2) return true;
        // bias + activation: accumulator -> next layer's A operand in S.h
        const float* bias = layer == 0 ? S.b1 : S.b2;
#pragma unroll
        for (int cb = 0; cb < 64; cb += 16) {
            uint32_t v[16];
            tmem_ld16(tm + tlane + (uint32_t)(col0 + cb), v);
            tmem_wait_ld();
            uint32_t w[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int c = col0 + cb + 2 * e;
                w[e] = act2_tc(__uint_as_float(v[2 * e]) + bias[c], __uint_as_float(v[2 * e + 1]) + bias[c + 1]);
            }
            *reinterpret_cast<uint4*>(S.h + canon(row, col0 + cb, TM)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4*>(S.h + canon(row, col0 + cb + 8, TM)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
        fence_async_smem();
        fence_before();
        __syncthreads();
    }
    return true;
}

// Output of the tile (warps 0..3; thread = row): y[0..15] from TMEM + b3.
__device__ __forceinline__ void tile_output(const TcSmem& S, float (&y)[16]) {
    const int warp = threadIdx.x >> 5;
    uint32_t v[16];
    tmem_ld16(S.tmem + ((uint32_t)(32 * (warp & 3)) << 16), v);
    tmem_wait_ld();
#pragma unroll
    for (int o = 0; o < 16; ++o) y[o] = __uint_as_float(v[o]) + S.b3[o];
}

__device__ void tc_setup(TcSmem& S, const Packed* P) {
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&S.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        S.abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&S.tmem)),
                     "r"(TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_weights_tc(S, P);
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

// Input rows (BF16, LDX per row) of tile t into S.x[buf] (canonical), cp.async.
__device__ __forceinline__ void issue_rows(TcSmem& S, int buf, const __nv_bfloat16* xg, long row0) {
    const uint32_t base = su32(S.x[buf]);
    for (int i = threadIdx.x; i < TM * (KX_TC / 8); i += TC_THREADS) {
        const int r = i / (KX_TC / 8), c = i % (KX_TC / 8);
        cp_async16_tc(base + canon(r, 8 * c, TM), xg + (row0 + r) * LDX + 8 * c);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <class T>
__global__ void __launch_bounds__(TC_THREADS, TC_MINB) k_closure_mlp_tc(const ClosureArgs<T> A, const Packed* __restrict__ P,
                                                                  const __nv_bfloat16* __restrict__ xg,
                                                                  const float* __restrict__ sc,
                                                                  float* __restrict__ ctr, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(raw);
    tc_setup(S, P);
    const int nx = A.nx, ny = A.ny;
    const int M = nx * ny;
    const int tiles = (M + TM - 1) / TM;
    const long Pp = A.pitch;
    uint32_t ph = 0;
    int buf = 0;
    int tile = blockIdx.x;
    if (tile < tiles) issue_rows(S, 0, xg, (long)tile * TM);
    for (; tile < tiles; tile += gridDim.x, buf ^= 1) {
        if (tile + (int)gridDim.x < tiles) issue_rows(S, buf ^ 1, xg, (long)(tile + gridDim.x) * TM);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        fence_async_smem();
        __syncthreads();
        if (!tile_network(S, buf, ph, err)) break;
        if (threadIdx.x < TM) {
            float y[16];
            tile_output(S, y);
            const int m = tile * TM + threadIdx.x;
            if (m < M) {
                const float s = sc[m];
                const int ix = m % nx, iy = m / nx;
#pragma unroll
                for (int o = 0; o < NOUT; ++o) {
                    const float val = s * y[o];
                    if (A.slot[NMOM + o].x != 0) { ctr[(long)o * M + m] = val; continue; }
                    T* c = A.g[0].base + (long)A.slot[NMOM + o].y * A.g[0].cstride;
                    const T tv = (T)val;
                    c[(long)(iy + 1) * Pp + ix] = tv;
                    if (ix == (A.p[0] ? nx - 1 : 0)) c[(long)(iy + 1) * Pp - 1] = tv;
                    if (ix == (A.p[0] ? 0 : nx - 1)) c[(long)(iy + 1) * Pp + nx] = tv;
                    if (iy == (A.p[1] ? ny - 1 : 0)) c[ix] = tv;
                    if (iy == (A.p[1] ? 0 : ny - 1)) c[(long)(ny + 1) * Pp + ix] = tv;
                }
            }
        }
        fence_before();
        __syncthreads();
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    tc_teardown(S);
}

__global__ void __launch_bounds__(TC_THREADS, TC_MINB) k_forward_tc(const float* __restrict__ X, long M,
                                                              const Packed* __restrict__ P, float* __restrict__ Y,
                                                              int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char raw[];
    TcSmem& S = *reinterpret_cast<TcSmem*>(raw);
    tc_setup(S, P);
    const long tiles = (M + TM - 1) / TM;
    uint32_t ph = 0;
    for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // FP32 rows -> BF16 canonical (two columns per thread step)
        for (int i = threadIdx.x; i < TM * (KX_TC / 2); i += TC_THREADS) {
            const int r = i / (KX_TC / 2), c = 2 * (i % (KX_TC / 2));
            const long m = tile * TM + r;
            float a = 0.f, b = 0.f;
            if (m < M && c < NIN) { a = X[m * NIN + c]; b = X[m * NIN + c + 1]; }
            *reinterpret_cast<uint32_t*>(S.x[0] + canon(r, c, TM)) = pack_bf16_tc(a, b);
        }
        fence_async_smem();
        __syncthreads();
        if (!tile_network(S, 0, ph, err)) break;
        if (threadIdx.x < TM) {
            float y[16];
            tile_output(S, y);
            const long m = tile * TM + threadIdx.x;
            if (m < M)
#pragma unroll
                for (int o = 0; o < NOUT; ++o) Y[m * NOUT + o] = y[o];
        }
        fence_before();
        __syncthreads();
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
    long blocks = (M + TM - 1) / TM;
    if (blocks > (long)TC_MINB * sms_tc()) blocks = (long)TC_MINB * sms_tc();
    k_forward_tc<<<(unsigned)blocks, TC_THREADS, sizeof(TcSmem), (cudaStream_t)stream>>>(X, M, P, Y, err);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template <class T>
int closure_mlp_tc(const ClosureArgs<T>& A, const Packed* P, const __nv_bfloat16* xg, const float* sc, float* ctr,
                   int* err, void* stream) {
    static bool attr = false;
    if (smem_attr(k_closure_mlp_tc<T>, attr)) return -4;
    const long M = (long)A.nx * A.ny;
    if (M <= 0) return 0;
    long blocks = (M + TM - 1) / TM;
    if (blocks > (long)TC_MINB * sms_tc()) blocks = (long)TC_MINB * sms_tc();
    k_closure_mlp_tc<T><<<(unsigned)blocks, TC_THREADS, sizeof(TcSmem), (cudaStream_t)stream>>>(A, P, xg, sc, ctr, err);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

template int closure_mlp_tc<float>(const ClosureArgs<float>&, const Packed*, const __nv_bfloat16*, const float*, float*,
                                   int*, void*);
template int closure_mlp_tc<double>(const ClosureArgs<double>&, const Packed*, const __nv_bfloat16*, const float*,
                                    float*, int*, void*);

}  // namespace mlp
}  // namespace starmap
