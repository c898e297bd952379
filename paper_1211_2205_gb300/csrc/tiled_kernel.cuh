// Tiled half-step pass for the 2D real P_N system in FP32 (sm_103a).
//
// One CTA owns a TX x TY tile of point indices, shared by the four staggered
// grids (section 4.1); each consumer thread owns PX points of one row.  A
// pass updates the components of one parity (odd l: grids G21 (R) and G12
// (I); even l: G11 (R) and G22 (I)) from the half-grid differences
// (eq. central_differences) of the other parity, weighted by -Mx/dx and
// -My/dy, followed by the exact sub-step u <- a u + b (W + q)
// (eq. sub_step_solution).
//
// Streaming by moment order.  Input components of order l' are visited in
// the paper's real order (m' = l', l'-2, ...; R then I).  Writing m = l - 2q,
// Lemma 2 says input (l', q') reaches only the outputs
//     (l'-1, q'-1), (l'-1, q'), (l'+1, q'), (l'+1, q'+1)
// of the same kind through Mx and of the other kind through My.  So while
// the inputs of order l' stream by in increasing q', register windows per
// kind hold the accumulators W of the two previous-order and the two
// next-order targets in reach:
//   * a previous-order target is complete once input q'+1 has been seen and
//     is finalised right there (its old value arrives through the ring);
//   * a next-order target has received all contributions of this order once
//     input q'+1 has been seen; its partial sum goes to a per-thread slice of
//     shared memory and comes back when order l'+2 streams by.
// Every input value is read from HBM once, every output read and written
// once; the differences of an input are formed once per point.
//
// Data movement: one producer warp walks a host-built stage list and issues
// the TMA boxes (cp.async.bulk.tensor.3d) of each stage into a ring of
// shared-memory stages guarded by mbarriers (full: transaction bytes, empty:
// one arrival per consumer warp).  A stage is one step of the consumer loop:
// slots for the R and I input of (l', q') and the R and I output finalised
// there.  Input boxes are BX x (TY+1) (one-point halo, x start aligned to 16
// bytes); output boxes TX x TY.  Boundary conditions live in ghost cells,
// which the finalising thread writes with each boundary value.  Every wait
// is bounded: on expiry the kernel raises an error flag, waits (bounded) for
// its copies in flight, and returns.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace starmap {
namespace tiled {

constexpr int PX = 2;                   // points per consumer thread (along x)
constexpr int TX = 32 * PX;             // tile width
constexpr int TY = 8;                   // tile height (one consumer warp per row)
constexpr int VEC = 4;                  // 16 bytes of FP32: TMA x alignment
constexpr int BX = TX + VEC;            // input box width (halo + alignment)
constexpr int BYI = TY + 1;             // input box height (halo)
constexpr int IN_BYTES = BX * BYI * 4;
constexpr int OUT_BYTES = TX * TY * 4;
constexpr int SLOT = ((IN_BYTES + 127) / 128) * 128;   // slot stride in bytes
constexpr int SLOTS_PER_STAGE = 4;      // input R, input I, output R, output I
constexpr int STAGE_BYTES = SLOT * SLOTS_PER_STAGE;
constexpr int NSTAGES = 6;              // stages in the ring
constexpr int CONSUMER_WARPS = TY;
constexpr int CONSUMERS = CONSUMER_WARPS * 32;
constexpr int THREADS = CONSUMERS + 32;
constexpr int MAXN = 63;
constexpr int RING_OFF = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded waits: 2 s

struct OutGrid {
    float* base;        // point (0,0) of component 0
    long cstride;       // elements between components
    const float* coef;  // decay coefficients [cls][4][ny][nx]
    int nx, ny;
};

struct Params {
    CUtensorMap maps[4];        // input R, input I, output R, output I
    OutGrid out[2];             // output grids: R, I
    long pitch;
    int p[2];
    int tiles_x;
    int N, P;                   // moment order, pass parity (1 odd, 0 even)
    int which;                  // 0 half-step coefficients, 1 full-step
    int nclasses;               // 2 = isotropic (class 0: l = 0, 1: l >= 1), else class = l
    int nstages, nin, nfin;
    const int4* stages;         // per stage: component (in its grid) of slot 0..3, -1 if absent
    const float4* coef;         // per input: cx Pm, P0, N0, Np, cy Pm, P0, N0, Np, each twice
    const longlong2* fin;       // per finalise event: (element offset | class << 48, source array or 0)
    int* err;                   // bounded-wait failure flag
    int smem_coef_off, smem_fin_off, smem_part_off;   // byte offsets in dynamic smem
};

__host__ __device__ constexpr int nq_of(int l) { return l < 0 ? 0 : l / 2 + 1; }
__host__ __device__ constexpr bool has_imag(int l, int q) { return l - 2 * q >= 1; }

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Wait for a barrier phase with a time limit; on expiry raise the CTA's
// abort flag and the global error flag.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (global_ns() - t0 > WAIT_NS) {
            *abort_flag = 1;
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Offsets of the right / upper neighbour of the staggered outputs read from
// the input grid of kind k (0 = R, 1 = I) in pass P.
__device__ __forceinline__ void input_shift(int P, int k, int px, int py, int& sx, int& sy) {
    // input grids: odd pass (P=1) R -> G11, I -> G22; even pass R -> G21, I -> G12
    const int g = P == 1 ? (k == 0 ? 0 : 3) : (k == 0 ? 1 : 2);
    const bool xnode = g & 1, ynode = g & 2;
    sx = xnode ? 1 - px : px;
    sy = ynode ? 1 - py : py;
}

// Packed pair of FP32 values (point A in the low half, point B in the high
// half) and the f32x2 arithmetic of sm_100-family parts.
typedef unsigned long long f2;
__device__ __forceinline__ f2 f2_make(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_split(f2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 f2_fma(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 f2_sub(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 lds2(const float* p) { return *reinterpret_cast<const f2*>(p); }

// x-differences of points A (column c) and B (column c + 1) of one box row:
// right operands at columns c, c + 1, left operands at c - 1, c.  The pair
// load starts at the even column of the two.
__device__ __forceinline__ f2 diff_x(const float* row, int c, bool c_even) {
    if (c_even) {
        const f2 P = lds2(row + c);                 // v[c], v[c+1]
        const float Q = row[c - 1];
        float lo, hi;
        f2_split(P, lo, hi);
        return f2_sub(P, f2_make(Q, lo));
    }
    const f2 P = lds2(row + c - 1);                 // v[c-1], v[c]
    const float Q = row[c + 1];
    float lo, hi;
    f2_split(P, lo, hi);
    return f2_sub(f2_make(hi, Q), P);
}

__global__ void __launch_bounds__(THREADS, 1) k_tiled_pass(const __grid_constant__ Params prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NSTAGES;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NSTAGES);
    unsigned char* ring = smem + RING_OFF;
    const float4* s_coef = reinterpret_cast<const float4*>(smem + prm.smem_coef_off);
    const longlong2* s_fin = reinterpret_cast<const longlong2*>(smem + prm.smem_fin_off);
    f2* s_part = reinterpret_cast<f2*>(smem + prm.smem_part_off);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x;
    const int x0 = (tile % prm.tiles_x) * TX;
    const int y0 = (tile / prm.tiles_x) * TY;

    if (tid == 0) {
        for (int r = 0; r < NSTAGES; ++r) {
            mbar_init(&full[r], 1);
            mbar_init(&empty[r], CONSUMER_WARPS);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    // stage the coefficient and finalise tables in shared memory
    {
        float4* c = reinterpret_cast<float4*>(smem + prm.smem_coef_off);
        for (int i = tid; i < 4 * prm.nin; i += THREADS) c[i] = __ldg(prm.coef + i);
        longlong2* f = reinterpret_cast<longlong2*>(smem + prm.smem_fin_off);
        for (int i = tid; i < prm.nfin; i += THREADS) f[i] = __ldg(prm.fin + i);
    }
    __syncthreads();

    int sxR, syR, sxI, syI;
    input_shift(prm.P, 0, prm.p[0], prm.p[1], sxR, syR);
    input_shift(prm.P, 1, prm.p[0], prm.p[1], sxI, syI);

    // --------------------------------------------------------- producer
    if (warp == CONSUMER_WARPS) {
        if (lane == 0) {
            // box origins in tensor coordinates (x' = x + VEC, row = y + 1)
            const int bxR = x0 + (sxR == 0 ? 0 : VEC), byR = y0 + (syR == 0 ? -1 : 0) + 1;
            const int bxI = x0 + (sxI == 0 ? 0 : VEC), byI = y0 + (syI == 0 ? -1 : 0) + 1;
            int issued = 0;
            bool ok = true;
            for (int s = 0; s < prm.nstages; ++s) {
                const int r = s % NSTAGES;
                if (s >= NSTAGES && !wait_bounded(&empty[r], ((s / NSTAGES) - 1) & 1, abort_flag, prm.err)) {
                    ok = false;
                    break;
                }
                const int4 st = __ldg(prm.stages + s);
                const uint32_t bytes = (st.x >= 0 ? IN_BYTES : 0) + (st.y >= 0 ? IN_BYTES : 0) +
                                       (st.z >= 0 ? OUT_BYTES : 0) + (st.w >= 0 ? OUT_BYTES : 0);
                unsigned char* base = ring + r * STAGE_BYTES;
                fence_proxy_async();
                mbar_expect_tx(&full[r], bytes);
                if (st.x >= 0) tma_load_3d(base, &prm.maps[0], bxR, byR, st.x, &full[r]);
                if (st.y >= 0) tma_load_3d(base + SLOT, &prm.maps[1], bxI, byI, st.y, &full[r]);
                if (st.z >= 0) tma_load_3d(base + 2 * SLOT, &prm.maps[2], x0 + VEC, y0 + 1, st.z, &full[r]);
                if (st.w >= 0) tma_load_3d(base + 3 * SLOT, &prm.maps[3], x0 + VEC, y0 + 1, st.w, &full[r]);
                ++issued;
            }
            if (!ok) {
                // aborted: wait (bounded) for the copies still in flight
                for (int s = issued - 1; s >= 0 && s >= issued - NSTAGES; --s) {
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait(&full[s % NSTAGES], (s / NSTAGES) & 1))
                        if (global_ns() - t0 > WAIT_NS) break;
                }
            }
        }
        return;
    }

    // --------------------------------------------------------- consumers
    // this thread owns points A = (x0 + 2 lane, y) and B = A + (1, 0)
    const int gy = y0 + warp;
    const int gxA = x0 + 2 * lane;
    // float offsets, inside a stage, of the difference operands
    int rxR, cxR, uR, rxI, cxI, uI;          // x: row start, column of A's right operand; y: up pair
    bool evR, evI;
    {
        const int bxsR = sxR == 0 ? -VEC : 0, oyR = syR == 0 ? -1 : 0;
        const int bxsI = sxI == 0 ? -VEC : 0, oyI = syI == 0 ? -1 : 0;
        rxR = (warp - oyR) * BX;
        cxR = 2 * lane + sxR - bxsR;
        evR = (cxR & 1) == 0;
        uR = (warp + syR - oyR) * BX + (2 * lane - bxsR);
        rxI = SLOT / 4 + (warp - oyI) * BX;
        cxI = 2 * lane + sxI - bxsI;
        evI = (cxI & 1) == 0;
        uI = SLOT / 4 + (warp + syI - oyI) * BX + (2 * lane - bxsI);
    }
    // output kinds k = 0 (R), 1 (I)
    float* pptr[2];                           // point A in component 0 of the output grid
    bool inA[2], inB[2], both[2], bndAny[2];
    long cidxA[2];
    f2 ca2[2][2], cb2[2][2];                  // decay pairs by class (isotropic)
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const OutGrid& G = prm.out[k];
        const int g = prm.P == 1 ? (k == 0 ? 1 : 2) : (k == 0 ? 0 : 3);
        const bool xnode = g & 1, ynode = g & 2;
        const long plane = (long)G.nx * G.ny;
        inA[k] = gxA < G.nx && gy < G.ny;
        inB[k] = gxA + 1 < G.nx && gy < G.ny;
        both[k] = inA[k] && inB[k];
        pptr[k] = G.base + (long)(gy + 1) * prm.pitch + gxA;
        cidxA[k] = (long)gy * G.nx + gxA;
        bool bnd = false;
        for (int pt = 0; pt < 2; ++pt) {
            const int gx = gxA + pt;
            if (prm.p[0]) bnd |= (gx == G.nx - 1) || (gx == 0);
            else if (!xnode) bnd |= (gx == 0) || (gx == G.nx - 1);
            if (prm.p[1]) bnd |= (gy == G.ny - 1) || (gy == 0);
            else if (!ynode) bnd |= (gy == 0) || (gy == G.ny - 1);
        }
        bndAny[k] = bnd && (inA[k] || inB[k]);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f};
            if (prm.nclasses == 2 && G.coef != nullptr) {
                const float* cf = G.coef + (long)c * 4 * plane + cidxA[k];
                if (inA[k]) { a[0] = __ldg(cf + 2 * prm.which * plane); b[0] = __ldg(cf + (2 * prm.which + 1) * plane); }
                if (inB[k]) { a[1] = __ldg(cf + 2 * prm.which * plane + 1); b[1] = __ldg(cf + (2 * prm.which + 1) * plane + 1); }
            }
            ca2[k][c] = f2_make(a[0], a[1]);
            cb2[k][c] = f2_make(b[0], b[1]);
        }
    }

    int s = 0, ii = 0, e = 0;
    bool alive = true;
    auto stage_ptr = [&]() -> const float* {
        const int r = s % NSTAGES;
        if (alive) alive = wait_bounded(&full[r], (s / NSTAGES) & 1, abort_flag, prm.err);
        return reinterpret_cast<const float*>(ring + r * STAGE_BYTES);
    };
    auto stage_done = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s % NSTAGES]);
        ++s;
    };
    auto part = [&](int q, int k) -> f2& { return s_part[(q * 2 + k) * CONSUMERS + tid]; };
    // write one point (and its boundary copies) of output kind k
    auto store_point = [&](int k, float* dst, int gx, float v) {
        const OutGrid& G = prm.out[k];
        const int g = prm.P == 1 ? (k == 0 ? 1 : 2) : (k == 0 ? 0 : 3);
        const bool xnode = g & 1, ynode = g & 2;
        *dst = v;
        int xa = -2, xb = -2, ya = -2, yb = -2;
        if (prm.p[0]) { if (gx == G.nx - 1) xa = -1; if (gx == 0) xb = G.nx; }
        else if (!xnode) { if (gx == 0) xa = -1; if (gx == G.nx - 1) xb = G.nx; }
        if (prm.p[1]) { if (gy == G.ny - 1) ya = -1; if (gy == 0) yb = G.ny; }
        else if (!ynode) { if (gy == 0) ya = -1; if (gy == G.ny - 1) yb = G.ny; }
        float* row = dst - gx;
        if (xa != -2) row[xa] = v;
        if (xb != -2) row[xb] = v;
        float* col = dst - (long)(gy + 1) * prm.pitch;
        if (ya != -2) col[(long)(ya + 1) * prm.pitch] = v;
        if (yb != -2) col[(long)(yb + 1) * prm.pitch] = v;
    };
    // finalise output kind k (slot 2 + k of stage t) of order L with sums W
    auto finalize = [&](const float* t, int k, int L, f2 W) {
        const longlong2 f = s_fin[e];                 // (element offset of the component, source pointer)
        ++e;
        const f2 u = lds2(t + (2 + k) * (SLOT / 4) + warp * TX + 2 * lane);
        f2 aa, bb;
        if (prm.nclasses == 2) {
            aa = L == 0 ? ca2[k][0] : ca2[k][1];
            bb = L == 0 ? cb2[k][0] : cb2[k][1];
        } else {
            const long plane = (long)prm.out[k].nx * prm.out[k].ny;
            const long cls = (long)(f.x >> 48);
            const float* cf = prm.out[k].coef + cls * 4 * plane + cidxA[k];
            float a0 = inA[k] ? __ldg(cf + 2 * prm.which * plane) : 0.f;
            float b0 = inA[k] ? __ldg(cf + (2 * prm.which + 1) * plane) : 0.f;
            float a1 = inB[k] ? __ldg(cf + 2 * prm.which * plane + 1) : 0.f;
            float b1 = inB[k] ? __ldg(cf + (2 * prm.which + 1) * plane + 1) : 0.f;
            aa = f2_make(a0, a1);
            bb = f2_make(b0, b1);
        }
        const float* qs = reinterpret_cast<const float*>(f.y);
        if (qs != nullptr) {
            const float q0 = inA[k] ? __ldg(qs + cidxA[k]) : 0.f;
            const float q1 = inB[k] ? __ldg(qs + cidxA[k] + 1) : 0.f;
            W = f2_add(W, f2_make(q0, q1));
        }
        const f2 v = f2_fma(aa, u, f2_mul(bb, W));
        if (!alive) return;
        float* dst = pptr[k] + (f.x & 0xFFFFFFFFFFFFll);
        if (both[k] && !bndAny[k]) {
            *reinterpret_cast<f2*>(dst) = v;
        } else {
            float v0, v1;
            f2_split(v, v0, v1);
            if (inA[k]) store_point(k, dst, gxA, v0);
            if (inB[k]) store_point(k, dst + 1, gxA + 1, v1);
        }
    };

    const int N = prm.N;
    const int first = 1 - prm.P;              // first input order: even l' for the odd pass
    int last_in = first;
    const f2 zero = 0ull;
    for (int lp = first; lp <= N && alive; lp += 2) {
        last_in = lp;
        const int nq = nq_of(lp);
        const int nqp = nq_of(lp - 1);                    // previous-order targets
        const int nqn = lp + 1 <= N ? nq_of(lp + 1) : 0;  // next-order targets
        f2 PcR = zero, PcI = zero, NcR = zero, NcI = zero;
        for (int q = 0; q < nq && alive; ++q) {
            const bool inI = has_imag(lp, q);
            // partial sums of a previous-order target exist once order
            // lp - 2 has streamed by (not for the first input order)
            const bool ldP = q < nqp && lp > first;
            f2 PnR = ldP ? part(q, 0) : zero;
            f2 PnI = (ldP && has_imag(lp - 1, q)) ? part(q, 1) : zero;
            f2 NnR = zero, NnI = zero;
            const float* t = stage_ptr();
            {
                // input R: d_x feeds R targets, d_y feeds I targets
                const float4* c = s_coef + 4 * ii;
                ++ii;
                const float4 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
                const f2 dx = diff_x(t + rxR, cxR, evR);
                const f2 dy = f2_sub(lds2(t + uR), lds2(t + uR - BX));
                PcR = f2_fma(f2_make(c0.x, c0.y), dx, PcR);
                PnR = f2_fma(f2_make(c0.z, c0.w), dx, PnR);
                NcR = f2_fma(f2_make(c1.x, c1.y), dx, NcR);
                NnR = f2_fma(f2_make(c1.z, c1.w), dx, NnR);
                PcI = f2_fma(f2_make(c2.x, c2.y), dy, PcI);
                PnI = f2_fma(f2_make(c2.z, c2.w), dy, PnI);
                NcI = f2_fma(f2_make(c3.x, c3.y), dy, NcI);
                NnI = f2_fma(f2_make(c3.z, c3.w), dy, NnI);
            }
            if (inI) {
                // input I: d_x feeds I targets, d_y feeds R targets
                const float4* c = s_coef + 4 * ii;
                ++ii;
                const float4 c0 = c[0], c1 = c[1], c2 = c[2], c3 = c[3];
                const f2 dx = diff_x(t + rxI, cxI, evI);
                const f2 dy = f2_sub(lds2(t + uI), lds2(t + uI - BX));
                PcI = f2_fma(f2_make(c0.x, c0.y), dx, PcI);
                PnI = f2_fma(f2_make(c0.z, c0.w), dx, PnI);
                NcI = f2_fma(f2_make(c1.x, c1.y), dx, NcI);
                NnI = f2_fma(f2_make(c1.z, c1.w), dx, NnI);
                PcR = f2_fma(f2_make(c2.x, c2.y), dy, PcR);
                PnR = f2_fma(f2_make(c2.z, c2.w), dy, PnR);
                NcR = f2_fma(f2_make(c3.x, c3.y), dy, NcR);
                NnR = f2_fma(f2_make(c3.z, c3.w), dy, NnR);
            }
            if (q >= 1 && q - 1 < nqp) {
                finalize(t, 0, lp - 1, PcR);
                if (has_imag(lp - 1, q - 1)) finalize(t, 1, lp - 1, PcI);
            }
            stage_done();
            if (q < nqn) {
                part(q, 0) = NcR;
                if (has_imag(lp + 1, q)) part(q, 1) = NcI;
            }
            PcR = PnR; PcI = PnI; NcR = NnR; NcI = NnI;
        }
        if (alive && nq - 1 < nqp) {
            // tail stage: the last previous-order target
            const float* t = stage_ptr();
            finalize(t, 0, lp - 1, PcR);
            if (has_imag(lp - 1, nq - 1)) finalize(t, 1, lp - 1, PcI);
            stage_done();
        }
        if (nq < nqn) {
            part(nq, 0) = NcR;
            if (has_imag(lp + 1, nq)) part(nq, 1) = NcI;
        }
    }
    // outputs of the order above the last input order have no further inputs
    const int L = last_in + 1;
    if (L <= N) {
        for (int q = 0; q < nq_of(L) && alive; ++q) {
            const bool hi = has_imag(L, q);
            const f2 WR = part(q, 0);
            const f2 WI = hi ? part(q, 1) : zero;
            const float* t = stage_ptr();
            finalize(t, 0, L, WR);
            if (hi) finalize(t, 1, L, WI);
            stage_done();
        }
    }
}

}  // namespace tiled
}  // namespace starmap
