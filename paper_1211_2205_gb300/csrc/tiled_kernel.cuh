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
constexpr int NSTAGES = 8;              // stages in the ring (power of two)
constexpr int CONSUMER_WARPS = 2 * TY;  // one warp per tile row and output kind (R, I)
constexpr int CONSUMERS = CONSUMER_WARPS * 32;
constexpr int PRODUCER_WARPS = 2;       // independent TMA issue streams (even / odd stages)
constexpr int THREADS = CONSUMERS + 32 * PRODUCER_WARPS;
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
    const float4* coef[2];      // per output kind K, per q step: (cx Pm, cx P0, cx N0, cx Np) of the
                                // input of kind K and (cy Pm, cy P0, cy N0, cy Np) of the other
                                // input, each value twice (f32x2 operands); zero if absent
    const int2* fin[2];         // per output kind K, per finalising stage: (element offset of the
                                // component, or -1 if absent; source slot or -1)
    const float* const* srcs;   // source arrays by slot
    int* err;                   // bounded-wait failure flag
    int smem_coef_off[2], smem_fin_off[2], smem_part_off, smem_stage_off;   // byte offsets in dynamic smem
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
__device__ __forceinline__ f2 zero2() { return 0ull; }

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
    f2* s_part = reinterpret_cast<f2*>(smem + prm.smem_part_off);
    const int4* s_stages = reinterpret_cast<const int4*>(smem + prm.smem_stage_off);

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
    // stage the coefficient, finalise and stage tables in shared memory
    for (int k = 0; k < 2; ++k) {
        float4* c = reinterpret_cast<float4*>(smem + prm.smem_coef_off[k]);
        for (int i = tid; i < 4 * prm.nin; i += THREADS) c[i] = __ldg(prm.coef[k] + i);
        int2* f = reinterpret_cast<int2*>(smem + prm.smem_fin_off[k]);
        for (int i = tid; i < prm.nfin; i += THREADS) f[i] = __ldg(prm.fin[k] + i);
    }
    {
        int4* st = reinterpret_cast<int4*>(smem + prm.smem_stage_off);
        for (int i = tid; i < prm.nstages; i += THREADS) st[i] = __ldg(prm.stages + i);
    }
    __syncthreads();

    int sxR, syR, sxI, syI;
    input_shift(prm.P, 0, prm.p[0], prm.p[1], sxR, syR);
    input_shift(prm.P, 1, prm.p[0], prm.p[1], sxI, syI);

    // --------------------------------------------------------- producer
    // Producer warp pw owns the stages s = pw (mod PRODUCER_WARPS).  Its
    // lane 0 waits for the slot to drain and arms the barrier with the
    // stage's byte count; lanes 0..3 then issue the (up to) four boxes.
    if (warp >= CONSUMER_WARPS) {
        const int pw = warp - CONSUMER_WARPS;
        const int bxR = x0 + (sxR == 0 ? 0 : VEC), byR = y0 + (syR == 0 ? -1 : 0) + 1;
        const int bxI = x0 + (sxI == 0 ? 0 : VEC), byI = y0 + (syI == 0 ? -1 : 0) + 1;
        // box origin of this lane's slot (tensor coordinates x' = x + VEC, row = y + 1)
        const int bx = lane == 0 ? bxR : lane == 1 ? bxI : x0 + VEC;
        const int by = lane == 0 ? byR : lane == 1 ? byI : y0 + 1;
        const CUtensorMap* map = &prm.maps[lane & 3];
        int last = -1;
        bool ok = true;
        for (int s = pw; s < prm.nstages; s += PRODUCER_WARPS) {
            const int r = s & (NSTAGES - 1);
            const int4 st = s_stages[s];
            if (lane == 0) {
                if (s >= NSTAGES && !wait_bounded(&empty[r], ((s / NSTAGES) - 1) & 1, abort_flag, prm.err)) ok = false;
                if (ok) {
                    const uint32_t bytes = (st.x >= 0 ? IN_BYTES : 0) + (st.y >= 0 ? IN_BYTES : 0) +
                                           (st.z >= 0 ? OUT_BYTES : 0) + (st.w >= 0 ? OUT_BYTES : 0);
                    mbar_expect_tx(&full[r], bytes);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            const int comp = lane == 0 ? st.x : lane == 1 ? st.y : lane == 2 ? st.z : st.w;
            if (lane < 4 && comp >= 0)
                tma_load_3d(ring + r * STAGE_BYTES + lane * SLOT, map, bx, by, comp, &full[r]);
            last = s;
        }
        if (!ok && lane == 0) {
            // aborted: wait (bounded) for this warp's copies still in flight
            for (int s = last; s >= 0 && s > last - NSTAGES; s -= PRODUCER_WARPS) {
                const unsigned long long t0 = global_ns();
                while (!mbar_try_wait(&full[s & (NSTAGES - 1)], (s / NSTAGES) & 1))
                    if (global_ns() - t0 > WAIT_NS) break;
            }
        }
        return;
    }

    // --------------------------------------------------------- consumers
    // Warp w handles tile row w % TY for the targets of kind K = w / TY
    // (0: R outputs, 1: I outputs), at points A = (x0 + 2 lane, y) and
    // B = A + (1, 0).  Targets of kind K take d_x of the inputs of kind K
    // (through Mx) and d_y of the inputs of the other kind (through My).
    const int K = warp / TY;
    const int row = warp % TY;
    const int gy = y0 + row;
    const int gxA = x0 + 2 * lane;
    // float offsets, inside a stage, of the difference operands: d_x from the
    // input of kind K (slot K), d_y from the input of kind 1 - K (slot 1 - K)
    int rx, cx, uy;
    bool ev;
    {
        const int sxK = K == 0 ? sxR : sxI;
        const int syO = K == 0 ? syI : syR;
        const int syK = K == 0 ? syR : syI;
        const int sxO = K == 0 ? sxI : sxR;
        const int bxsK = sxK == 0 ? -VEC : 0, oyK = syK == 0 ? -1 : 0;
        const int bxsO = sxO == 0 ? -VEC : 0, oyO = syO == 0 ? -1 : 0;
        rx = K * (SLOT / 4) + (row - oyK) * BX;
        cx = 2 * lane + sxK - bxsK;
        ev = (cx & 1) == 0;
        uy = (1 - K) * (SLOT / 4) + (row + syO - oyO) * BX + (2 * lane - bxsO);
    }
    // the output grid of kind K
    const OutGrid& G = prm.out[K];
    const int gK = prm.P == 1 ? (K == 0 ? 1 : 2) : (K == 0 ? 0 : 3);
    const bool xnode = gK & 1, ynode = gK & 2;
    const long plane = (long)G.nx * G.ny;
    const bool inA = gxA < G.nx && gy < G.ny;
    const bool inB = gxA + 1 < G.nx && gy < G.ny;
    float* const pptr = G.base + (long)(gy + 1) * prm.pitch + gxA;   // point A in component 0
    const long cidxA = (long)gy * G.nx + gxA;
    bool bnd = false;
    for (int pt = 0; pt < 2; ++pt) {
        const int gx = gxA + pt;
        if (prm.p[0]) bnd |= (gx == G.nx - 1) || (gx == 0);
        else if (!xnode) bnd |= (gx == 0) || (gx == G.nx - 1);
        if (prm.p[1]) bnd |= (gy == G.ny - 1) || (gy == 0);
        else if (!ynode) bnd |= (gy == 0) || (gy == G.ny - 1);
    }
    const bool fast = inA && inB && !bnd;     // plain paired store
    f2 ca2[2], cb2[2];                         // decay pairs by class (isotropic)
    for (int c = 0; c < 2; ++c) {
        float a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f};
        if (prm.nclasses == 2 && G.coef != nullptr) {
            const float* cf = G.coef + (long)c * 4 * plane + cidxA;
            if (inA) { a[0] = __ldg(cf + 2 * prm.which * plane); b[0] = __ldg(cf + (2 * prm.which + 1) * plane); }
            if (inB) { a[1] = __ldg(cf + 2 * prm.which * plane + 1); b[1] = __ldg(cf + (2 * prm.which + 1) * plane + 1); }
        }
        ca2[c] = f2_make(a[0], a[1]);
        cb2[c] = f2_make(b[0], b[1]);
    }

    static_assert((NSTAGES & (NSTAGES - 1)) == 0, "ring depth must be a power of two");
    // walking pointers into this kind's tables and this thread's partial sums
    const ulonglong2* cp = reinterpret_cast<const ulonglong2*>(smem + prm.smem_coef_off[K]);
    const int2* fp = reinterpret_cast<const int2*>(smem + prm.smem_fin_off[K]);
    f2* const pp = s_part + tid;
    const unsigned char* const ring_c = ring;
    const int uoff = (2 + K) * (SLOT / 4) + row * TX + 2 * lane;    // old value inside a stage
    int s = 0;
    bool alive = true;
    auto stage_ptr = [&]() -> const float* {
        const int r = s & (NSTAGES - 1);
        if (alive) alive = wait_bounded(&full[r], (s / NSTAGES) & 1, abort_flag, prm.err);
        return reinterpret_cast<const float*>(ring_c + r * STAGE_BYTES);
    };
    auto stage_done = [&]() {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s & (NSTAGES - 1)]);
        ++s;
    };
    // write one point (and its boundary copies)
    auto store_point = [&](float* dst, int gx, float v) {
        *dst = v;
        int xa = -2, xb = -2, ya = -2, yb = -2;
        if (prm.p[0]) { if (gx == G.nx - 1) xa = -1; if (gx == 0) xb = G.nx; }
        else if (!xnode) { if (gx == 0) xa = -1; if (gx == G.nx - 1) xb = G.nx; }
        if (prm.p[1]) { if (gy == G.ny - 1) ya = -1; if (gy == 0) yb = G.ny; }
        else if (!ynode) { if (gy == 0) ya = -1; if (gy == G.ny - 1) yb = G.ny; }
        float* rw = dst - gx;
        if (xa != -2) rw[xa] = v;
        if (xb != -2) rw[xb] = v;
        float* col = dst - (long)(gy + 1) * prm.pitch;
        if (ya != -2) col[(long)(ya + 1) * prm.pitch] = v;
        if (yb != -2) col[(long)(yb + 1) * prm.pitch] = v;
    };
    // decay pair (a, b) of the outputs of order L
    f2 aL = zero2(), bL = zero2();
    auto set_order = [&](int L) {
        if (prm.nclasses == 2) {
            aL = L == 0 ? ca2[0] : ca2[1];
            bL = L == 0 ? cb2[0] : cb2[1];
        } else {
            const float* cf = G.coef + (long)L * 4 * plane + cidxA;
            float a0 = inA ? __ldg(cf + 2 * prm.which * plane) : 0.f;
            float b0 = inA ? __ldg(cf + (2 * prm.which + 1) * plane) : 0.f;
            float a1 = inB ? __ldg(cf + 2 * prm.which * plane + 1) : 0.f;
            float b1 = inB ? __ldg(cf + (2 * prm.which + 1) * plane + 1) : 0.f;
            aL = f2_make(a0, a1);
            bL = f2_make(b0, b1);
        }
    };
    // finalise this warp's output of the current finalising stage (slot 2 + K)
    auto finalize = [&](const float* t, f2 W) {
        const int2 f = *fp;
        fp += 1;
        const f2 u = lds2(t + uoff);
        if (f.y >= 0) {
            const float* qs = prm.srcs[f.y];
            const float q0 = inA ? __ldg(qs + cidxA) : 0.f;
            const float q1 = inB ? __ldg(qs + cidxA + 1) : 0.f;
            W = f2_add(W, f2_make(q0, q1));
        }
        const f2 v = f2_fma(aL, u, f2_mul(bL, W));
        if (f.x < 0 || !alive) return;
        float* dst = pptr + f.x;
        if (fast) {
            *reinterpret_cast<f2*>(dst) = v;
        } else {
            float v0, v1;
            f2_split(v, v0, v1);
            if (inA) store_point(dst, gxA, v0);
            if (inB) store_point(dst + 1, gxA + 1, v1);
        }
    };
    // accumulate a q step into the four targets of kind K in reach: d_x of
    // the input of kind K (slot K), d_y of the other input (slot 1 - K);
    // a missing I input has zero coefficients and its differences masked
    auto accumulate = [&](const float* t, bool inI, f2& Pc, f2& Pn, f2& Nc, f2& Nn) {
        const ulonglong2 xa = cp[0], xb = cp[1], ya = cp[2], yb = cp[3];
        cp += 4;
        f2 dx = diff_x(t + rx, cx, ev);
        f2 dy = f2_sub(lds2(t + uy), lds2(t + uy - BX));
        if (!inI) {
            if (K == 1) dx = zero2(); else dy = zero2();
        }
        Pc = f2_fma(xa.x, dx, Pc);
        Pn = f2_fma(xa.y, dx, Pn);
        Nc = f2_fma(xb.x, dx, Nc);
        Nn = f2_fma(xb.y, dx, Nn);
        Pc = f2_fma(ya.x, dy, Pc);
        Pn = f2_fma(ya.y, dy, Pn);
        Nc = f2_fma(yb.x, dy, Nc);
        Nn = f2_fma(yb.y, dy, Nn);
    };

    const int N = prm.N;
    const int first = 1 - prm.P;              // first input order: even l' for the odd pass
    int last_in = first;
    for (int lp = first; lp <= N && alive; lp += 2) {
        last_in = lp;
        const int nq = nq_of(lp);
        const int nqp = nq_of(lp - 1);                    // previous-order targets
        const int nqn = lp + 1 <= N ? nq_of(lp + 1) : 0;  // next-order targets
        const int nqload = lp > first ? nqp : 0;          // previous-order partial sums exist once order lp - 2 passed
        set_order(lp - 1);
        f2 Pc = zero2(), Nc = zero2();
        // one q step: (Pc, Nc) carried in, (Pn, Nn) started here
        auto qstep = [&](int q, f2& Pc_, f2& Nc_, f2& Pn_, f2& Nn_) {
            Pn_ = q < nqload ? pp[q * CONSUMERS] : zero2();
            Nn_ = zero2();
            const float* t = stage_ptr();
            accumulate(t, has_imag(lp, q), Pc_, Pn_, Nc_, Nn_);
            if (q >= 1 && q - 1 < nqp) finalize(t, Pc_);
            stage_done();
            if (q < nqn) pp[q * CONSUMERS] = Nc_;
        };
        int q = 0;
        f2 Pn, Nn;
        for (; q + 1 < nq && alive; q += 2) {
            qstep(q, Pc, Nc, Pn, Nn);
            qstep(q + 1, Pn, Nn, Pc, Nc);
        }
        if (q < nq && alive) {
            qstep(q, Pc, Nc, Pn, Nn);
            Pc = Pn; Nc = Nn;
        }
        if (alive && nq - 1 < nqp) {
            // tail stage: the last previous-order target
            const float* t = stage_ptr();
            finalize(t, Pc);
            stage_done();
        }
        if (nq < nqn) pp[nq * CONSUMERS] = Nc;
    }
    // outputs of the order above the last input order have no further inputs
    const int L = last_in + 1;
    if (L <= N) {
        set_order(L);
        for (int q = 0; q < nq_of(L) && alive; ++q) {
            const f2 W = pp[q * CONSUMERS];
            const float* t = stage_ptr();
            finalize(t, W);
            stage_done();
        }
    }
}

}  // namespace tiled
}  // namespace starmap
