// Tiled half-step pass for the 2D real P_N system in FP32 (sm_103a).
//
// One CTA owns a TX x TY tile of point indices, shared by the four staggered
// grids (section 4.1); each consumer thread owns a pair of points in each of
// RW rows of the tile.  A
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
// bytes); output boxes TX x TY.  Boundary conditions live in ghost cells
// (section 4.2), which a separate refresh kernel rewrites after the pass
// (the boundary tiles would otherwise wait on scattered single-value
// stores).  Every wait is bounded: on expiry the kernel raises an error
// flag, waits (bounded) for its copies in flight, and returns.
//
// The file is compiled once per tile height: STARMAP_TILED_NS names the
// namespace, STARMAP_TILED_TY the tile height, STARMAP_TILED_RW the rows per
// consumer warp and STARMAP_TILED_MINB the CTAs per SM the launch bounds ask
// for (10 rows, two per warp, one CTA per SM, for large N: a warp's fixed
// cost per step (barrier wait, table reads, release) is spread over four
// points; 5 rows, one per warp, two CTAs per SM, so that one CTA's setup,
// fill and drain overlap the other's streaming when a tile has few stages).
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pdl.h"

#ifndef STARMAP_TILED_NS
#define STARMAP_TILED_NS tiled
#define STARMAP_TILED_TY 10
#define STARMAP_TILED_MINB 1
#define STARMAP_TILED_RW 2
#endif

namespace starmap {
namespace STARMAP_TILED_NS {

constexpr int PX = 1;                   // point pairs per consumer thread along x
constexpr int TX = 64 * PX;             // tile width
constexpr int TY = STARMAP_TILED_TY;    // tile height
constexpr int RW = STARMAP_TILED_RW;    // tile rows per consumer warp
constexpr int RSTEP = TY / RW;          // rows between the rows of one warp
constexpr int PP = PX * RW;             // point pairs per consumer thread: pair j of lane l covers
                                        // x = x0 + 64 (j % PX) + 2 l, +1 in row row0 + RSTEP (j / PX)
static_assert(TY % RW == 0, "the rows of a tile split evenly over the warps");
constexpr int MINB = STARMAP_TILED_MINB;
constexpr int VEC = 4;                  // 16 bytes of FP32: TMA x alignment
constexpr int BX = TX + VEC;            // input box width (halo + alignment)
constexpr int BYI = TY + 1;             // input box height (halo)
constexpr int IN_BYTES = BX * BYI * 4;
constexpr int OUT_BYTES = TX * TY * 4;
constexpr int IN_SLOT = ((IN_BYTES + 127) / 128) * 128;    // slot strides in bytes
constexpr int OUT_SLOT = ((OUT_BYTES + 127) / 128) * 128;
// a stage (one consumer step) holds the input R, input I, output R, output I boxes
constexpr int STAGE_BYTES = 2 * IN_SLOT + 2 * OUT_SLOT;
__host__ __device__ constexpr int slot_off(int slot) { return slot < 2 ? slot * IN_SLOT : 2 * IN_SLOT + (slot - 2) * OUT_SLOT; }
constexpr int MAX_STAGES = 15;          // ring depth limit (the host fills the shared memory up to it)
constexpr int CONSUMER_WARPS = 2 * RSTEP;   // per output kind (R, I), one warp per RW rows
constexpr int CONSUMERS = CONSUMER_WARPS * 32;
constexpr int PRODUCER_WARPS = 2;       // independent TMA issue streams (stage s mod 2)
constexpr int THREADS = CONSUMERS + 32 * PRODUCER_WARPS;
constexpr int MAXN = 63;
constexpr int RING_OFF = 256;           // full[MAX_STAGES], empty[MAX_STAGES], abort flag
static_assert(2 * MAX_STAGES * 8 + 4 <= RING_OFF, "barriers fit before the ring");
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
    int nring;                  // stages in the ring (2 .. MAX_STAGES)
    int top;                    // highest output order finalised: N, or N - 1 when every order-N
                                // component is frozen (a closure sets them)
    const int4* stages;         // per stage: component (in its grid) of slot 0..3, -1 if absent
    const float4* coef[2];      // per output kind K, per q step: (cx Pm, cx P0, cx N0, cx Np) of the
                                // input of kind K and (cy Pm, cy P0, cy N0, cy Np) of the other
                                // input; zero if absent
    const int2* fin[2];         // per output kind K, per finalising stage: (element offset of the
                                // component / 32, or -1 if absent; source slot or -1)
    const float* const* srcs;   // source arrays by slot
    int* err;                   // bounded-wait failure flag
    int smem_coef_off[2], smem_fin_off[2], smem_part_off, smem_stage_off;   // byte offsets in dynamic smem
    const float* pf_src[2];     // per output kind: the source array its finalisations read, if it
                                // has exactly one (prefetched into L2 with the decay pairs), else null
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
__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// float offsets of point pair j from pair 0 inside an input box / an output box
__host__ __device__ constexpr int in_off(int j) { return (j / PX) * RSTEP * BX + 64 * (j % PX); }
__host__ __device__ constexpr int out_off(int j) { return (j / PX) * RSTEP * TX + 64 * (j % PX); }

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

// Tiles t0, t0 + tstride, ... < tend of one pass, through one continuous
// pipeline: the producers walk a global stage index over all of them (the
// first stages of the next tile are in flight while the consumers finish
// the current one), the consumers step through the tiles in the same order.
// maps: the pass's four tensor maps (in parameter or global memory: TMA
// reads them from there); prm: everything else.  first_call: the CTA's
// first call (a later call invalidates and re-initialises the barriers; the
// caller synchronises the CTA in between).
__device__ __forceinline__ void tiled_tiles(const Params& prm, const CUtensorMap* maps, int t0, int tstride, int tend,
                                            bool first_call) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + MAX_STAGES;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + MAX_STAGES);
    const int NR = prm.nring;
    unsigned char* ring = smem + RING_OFF;
    f2* s_part = reinterpret_cast<f2*>(smem + prm.smem_part_off);
    const int4* s_stages = reinterpret_cast<const int4*>(smem + prm.smem_stage_off);

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ntl = t0 < tend ? (tend - t0 + tstride - 1) / tstride : 0;

    // warm the TMA descriptor cache while the barriers and tables are set up
    if (warp == CONSUMER_WARPS && lane < 4)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(maps + lane)) : "memory");
    if (tid == 0) {
        for (int r = 0; r < MAX_STAGES; ++r) {      // every barrier: a batch's items differ in depth
            if (!first_call) {
                mbar_inval(&full[r]);
                mbar_inval(&empty[r]);
            }
            mbar_init(&full[r], 1);
            mbar_init(&empty[r], CONSUMER_WARPS);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    // stage the coefficient, finalise and stage tables in shared memory
    for (int k = 0; k < 2; ++k) {
        float4* c = reinterpret_cast<float4*>(smem + prm.smem_coef_off[k]);
        for (int i = tid; i < 2 * prm.nin; i += THREADS) c[i] = __ldg(prm.coef[k] + i);
        int2* f = reinterpret_cast<int2*>(smem + prm.smem_fin_off[k]);
        for (int i = tid; i < prm.nfin; i += THREADS) f[i] = __ldg(prm.fin[k] + i);
    }
    {
        int4* st = reinterpret_cast<int4*>(smem + prm.smem_stage_off);
        for (int i = tid; i < prm.nstages; i += THREADS) st[i] = __ldg(prm.stages + i);
    }
    __syncthreads();
    if (first_call) {
        // everything above reads host-written data only; the state is read
        // and written below, after the previous kernel of the stream is done
        pdl_trigger();
        pdl_wait();
    }

    int sxR, syR, sxI, syI;
    input_shift(prm.P, 0, prm.p[0], prm.p[1], sxR, syR);
    input_shift(prm.P, 1, prm.p[0], prm.p[1], sxI, syI);

    // --------------------------------------------------------- producer
    // Producer warp pw owns the global stages G = pw (mod PRODUCER_WARPS)
    // over all of the CTA's tiles (stage k of tile t is G = t * nstages + k,
    // ring slot G mod nring).  Lane 0 waits for the slot to drain and arms
    // its barrier with the byte count; lanes 0..3 then issue the (up to) four
    // boxes, lane = slot.
    if (warp >= CONSUMER_WARPS) {
        const int pw = warp - CONSUMER_WARPS;
        const int slot = lane & 3;
        const CUtensorMap* map = maps + slot;
        const int nst = prm.nstages;
        const int total = ntl * nst;        // the host keeps this below 2^31
        int last = -1;
        bool ok = true;
        // G = pw, pw + PRODUCER_WARPS, ...: stage k of local tile tl, ring
        // slot r, ring round u (all advanced incrementally)
        int k = pw, tl = 0, r = pw, u = 0;
        while (k >= nst && nst > 0) { k -= nst; ++tl; }
        int tile_at = -1, bx = 0, by = 0;
        bool entered = false;   // this warp has just issued its first stage of tile tl
        for (int G = pw; G < total; G += PRODUCER_WARPS) {
            entered = tl != tile_at;
            if (tl != tile_at) {
                // box origin of this lane's slot in tile tl (tensor coordinates x' = x + VEC, row = y + 1)
                tile_at = tl;
                const int tile = t0 + tl * tstride;
                const int x0 = (tile % prm.tiles_x) * TX, y0 = (tile / prm.tiles_x) * TY;
                const int bxR = x0 + (sxR == 0 ? 0 : VEC), byR = y0 + (syR == 0 ? -1 : 0) + 1;
                const int bxI = x0 + (sxI == 0 ? 0 : VEC), byI = y0 + (syI == 0 ? -1 : 0) + 1;
                bx = slot == 0 ? bxR : slot == 1 ? bxI : x0 + VEC;
                by = slot == 0 ? byR : slot == 1 ? byI : y0 + 1;
            }
            int4 st = make_int4(-1, -1, -1, -1);
            if (lane < 4) st = s_stages[k];
            const int comp = slot == 0 ? st.x : slot == 1 ? st.y : slot == 2 ? st.z : st.w;
            const uint32_t mine = lane < 4 && comp >= 0 ? (slot < 2 ? IN_BYTES : OUT_BYTES) : 0u;
            uint32_t bytes = mine;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            if (lane == 0) {
                if (u > 0 && !wait_bounded(&empty[r], (u - 1) & 1, abort_flag, prm.err)) ok = false;
                if (ok) mbar_expect_tx(&full[r], bytes);
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            if (mine != 0u) tma_load_3d(ring + r * STAGE_BYTES + slot_off(slot), map, bx, by, comp, &full[r]);
            if (entered && tl > 0 && pw == 0 && prm.nclasses == 2) {
                // the decay pairs (and the source) of this tile (not the first: there
                // the consumers load them at once) into L2 while the consumers finish
                // the previous tiles; lane = (kind, class, plane a / b, half row of 32)
                const int tile = t0 + tl * tstride;
                const int x0 = (tile % prm.tiles_x) * TX, y0 = (tile / prm.tiles_x) * TY;
                const int kind = lane >> 4, c = (lane >> 3) & 1, ab = (lane >> 2) & 1, hx = lane & 1;
                const OutGrid& Gk = prm.out[kind];
                const int x = x0 + 32 * hx;
                if (x < Gk.nx) {
                    const long plane = (long)Gk.nx * Gk.ny;
                    // lanes with bit 1 clear: decay pairs; lanes 2 + 16 kind (+1): the kind's source
                    const float* base = ((lane >> 1) & 1) == 0
                        ? (Gk.coef != nullptr ? Gk.coef + ((long)c * 4 + 2 * prm.which + ab) * plane + x : nullptr)
                        : ((lane & 12) == 0 && prm.pf_src[kind] != nullptr ? prm.pf_src[kind] + x : nullptr);
                    if (base != nullptr)
                        for (int y = y0; y < y0 + TY && y < Gk.ny; ++y)
                            asm volatile("prefetch.global.L2 [%0];" ::"l"(base + (long)y * Gk.nx));
                }
            }
            last = G;
            k += PRODUCER_WARPS;
            while (k >= nst) { k -= nst; ++tl; }
            r += PRODUCER_WARPS;
            if (r >= NR) { r -= NR; ++u; }
        }
        if (!ok && lane == 0) {
            // aborted: wait (bounded) for this warp's copies still in flight
            for (int G = last; G >= 0 && G > last - NR; G -= PRODUCER_WARPS) {
                const unsigned long long tw = global_ns();
                while (!mbar_try_wait(&full[G % NR], (G / NR) & 1))
                    if (global_ns() - tw > WAIT_NS) break;
            }
        }
        return;
    }

    // --------------------------------------------------------- consumers
    // Warp w handles the tile rows row0 + RSTEP i (row0 = w % RSTEP, i < RW)
    // for the targets of kind K = w / RSTEP (0: R outputs, 1: I outputs), at
    // the point pairs j = 0..PP-1: A_j = (x0 + 64 (j % PX) + 2 lane,
    // y0 + row0 + RSTEP (j / PX)), B_j = A_j + (1, 0).  Targets of kind K
    // take d_x of the inputs of kind K (through Mx) and d_y of the inputs of
    // the other kind (through My).
    const int K = warp / RSTEP;
    const int row = warp % RSTEP;
    int s = 0;                  // global consumer step (= stage) over the CTA's tiles
    int ring_r = 0;             // its ring slot and barrier phase
    uint32_t ring_ph = 0;
    bool alive = true;
    // the output grid of kind K
    const OutGrid& G = prm.out[K];
    const long plane = (long)G.nx * G.ny;
    for (int tl = 0; tl < ntl && alive; ++tl) {
        const int tile = t0 + tl * tstride;
        const int x0 = (tile % prm.tiles_x) * TX, y0 = (tile / prm.tiles_x) * TY;
        // float offsets, inside a step, of the difference operands of pair 0
        // (pair j sits in_off(j) floats further): d_x from the input of kind K (slot
        // K), d_y from the input of kind 1 - K (slot 1 - K)
        int rx, cx, uy;
        bool ev;
        {
            const int sxK = K == 0 ? sxR : sxI;
            const int syO = K == 0 ? syI : syR;
            const int syK = K == 0 ? syR : syI;
            const int sxO = K == 0 ? sxI : sxR;
            const int bxsK = sxK == 0 ? -VEC : 0, oyK = syK == 0 ? -1 : 0;
            const int bxsO = sxO == 0 ? -VEC : 0, oyO = syO == 0 ? -1 : 0;
            rx = slot_off(K) / 4 + (row - oyK) * BX;
            cx = 2 * lane + sxK - bxsK;
            ev = (cx & 1) == 0;
            uy = slot_off(1 - K) / 4 + (row + syO - oyO) * BX + (2 * lane - bxsO);
        }
        bool inA[PP], inB[PP], pair[PP];
        float* pptr[PP];          // point A_j in component 0
        long cidxA[PP];
        f2 ca2[PP][2], cb2[PP][2];  // decay pairs by class (isotropic)
    #pragma unroll
        for (int j = 0; j < PP; ++j) {
            const int gx = x0 + 64 * (j % PX) + 2 * lane;
            const int gy = y0 + row + RSTEP * (j / PX);
            inA[j] = gx < G.nx && gy < G.ny;
            inB[j] = gx + 1 < G.nx && gy < G.ny;
            pptr[j] = G.base + (long)(gy + 1) * prm.pitch + gx;
            cidxA[j] = (long)gy * G.nx + gx;
            pair[j] = inA[j] && inB[j];
            for (int c = 0; c < 2; ++c) {
                float a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f};
                if (prm.nclasses == 2 && G.coef != nullptr) {
                    const float* cf = G.coef + (long)c * 4 * plane + cidxA[j];
                    if (inA[j]) { a[0] = __ldg(cf + 2 * prm.which * plane); b[0] = __ldg(cf + (2 * prm.which + 1) * plane); }
                    if (inB[j]) { a[1] = __ldg(cf + 2 * prm.which * plane + 1); b[1] = __ldg(cf + (2 * prm.which + 1) * plane + 1); }
                }
                ca2[j][c] = f2_make(a[0], a[1]);
                cb2[j][c] = f2_make(b[0], b[1]);
            }
        }

        // walking pointers into this kind's tables and this thread's partial sums
        const float4* cp = reinterpret_cast<const float4*>(smem + prm.smem_coef_off[K]);
        const int2* fp = reinterpret_cast<const int2*>(smem + prm.smem_fin_off[K]);
        f2* const pp = s_part + tid;            // entry (q, j) at pp[(q * PP + j) * CONSUMERS]
        const int uoff = slot_off(2 + K) / 4 + row * TX + 2 * lane;    // old value of pair 0 inside a step
        // consumer step s is stage s (ring slot ring_r, phase ring_ph): its
        // barrier is awaited before the step and released after it
        auto stage_ptr = [&]() -> const float* {
            if (alive) alive = wait_bounded(&full[ring_r], ring_ph, abort_flag, prm.err);
            return reinterpret_cast<const float*>(ring + ring_r * STAGE_BYTES);
        };
        auto stage_done = [&]() {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[ring_r]);
            ++s;
            if (++ring_r == NR) { ring_r = 0; ring_ph ^= 1u; }
        };
        // decay pairs (a, b) of the outputs of order L
        f2 aL[PP], bL[PP];
        auto set_order = [&](int L) {
    #pragma unroll
            for (int j = 0; j < PP; ++j) {
                if (prm.nclasses == 2) {
                    aL[j] = L == 0 ? ca2[j][0] : ca2[j][1];
                    bL[j] = L == 0 ? cb2[j][0] : cb2[j][1];
                } else {
                    const float* cf = G.coef + (long)L * 4 * plane + cidxA[j];
                    const float a0 = inA[j] ? __ldg(cf + 2 * prm.which * plane) : 0.f;
                    const float b0 = inA[j] ? __ldg(cf + (2 * prm.which + 1) * plane) : 0.f;
                    const float a1 = inB[j] ? __ldg(cf + 2 * prm.which * plane + 1) : 0.f;
                    const float b1 = inB[j] ? __ldg(cf + (2 * prm.which + 1) * plane + 1) : 0.f;
                    aL[j] = f2_make(a0, a1);
                    bL[j] = f2_make(b0, b1);
                }
            }
        };
        // finalise this warp's output of the current finalising step (slot 2 + K)
        auto finalize = [&](const float* t, const f2 (&W)[PP]) {
            const int2 f = *fp;
            fp += 1;
    #pragma unroll
            for (int j = 0; j < PP; ++j) {
                const f2 u = lds2(t + uoff + out_off(j));
                f2 w = W[j];
                if (f.y >= 0) {
                    const float* qs = prm.srcs[f.y];
                    const float q0 = inA[j] ? __ldg(qs + cidxA[j]) : 0.f;
                    const float q1 = inB[j] ? __ldg(qs + cidxA[j] + 1) : 0.f;
                    w = f2_add(w, f2_make(q0, q1));
                }
                const f2 v = f2_fma(aL[j], u, f2_mul(bL[j], w));
                if (f.x < 0 || !alive) continue;
                float* dst = pptr[j] + 32 * (long)f.x;            // 64-bit: states beyond 2^31 values
                // the pair with one 8-byte store; only a ragged right edge
                // stores A alone
                if (pair[j]) {
                    *reinterpret_cast<f2*>(dst) = v;
                } else if (inA[j]) {
                    float v0, v1;
                    f2_split(v, v0, v1);
                    *dst = v0;
                }
            }
        };
        // accumulate a q step into the four targets of kind K in reach: d_x of
        // the input of kind K (slot K), d_y of the other input (slot 1 - K);
        // a missing I input has zero coefficients and its differences masked
        auto accumulate = [&](const float* t, bool inI, f2 (&Pc)[PP], f2 (&Pn)[PP], f2 (&Nc)[PP], f2 (&Nn)[PP]) {
            // each coefficient as an f32x2 pair (the same value for both points)
            const float4 cxv = cp[0], cyv = cp[1];
            cp += 2;
            const f2 xPm = f2_make(cxv.x, cxv.x), xP0 = f2_make(cxv.y, cxv.y);
            const f2 xN0 = f2_make(cxv.z, cxv.z), xNp = f2_make(cxv.w, cxv.w);
            const f2 yPm = f2_make(cyv.x, cyv.x), yP0 = f2_make(cyv.y, cyv.y);
            const f2 yN0 = f2_make(cyv.z, cyv.z), yNp = f2_make(cyv.w, cyv.w);
    #pragma unroll
            for (int j = 0; j < PP; ++j) {
                f2 dx = diff_x(t + rx + in_off(j), cx, ev);
                f2 dy = f2_sub(lds2(t + uy + in_off(j)), lds2(t + uy + in_off(j) - BX));
                if (!inI) {
                    if (K == 1) dx = zero2(); else dy = zero2();
                }
                Pc[j] = f2_fma(xPm, dx, Pc[j]);
                Pn[j] = f2_fma(xP0, dx, Pn[j]);
                Nc[j] = f2_fma(xN0, dx, Nc[j]);
                Nn[j] = f2_fma(xNp, dx, Nn[j]);
                Pc[j] = f2_fma(yPm, dy, Pc[j]);
                Pn[j] = f2_fma(yP0, dy, Pn[j]);
                Nc[j] = f2_fma(yN0, dy, Nc[j]);
                Nn[j] = f2_fma(yNp, dy, Nn[j]);
            }
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
            f2 Pc[PP], Nc[PP], Pn[PP], Nn[PP];
    #pragma unroll
            for (int j = 0; j < PP; ++j) { Pc[j] = zero2(); Nc[j] = zero2(); }
            // one q step: (Pc, Nc) carried in, (Pn, Nn) started here
            auto qstep = [&](int q, f2 (&Pc_)[PP], f2 (&Nc_)[PP], f2 (&Pn_)[PP], f2 (&Nn_)[PP]) {
    #pragma unroll
                for (int j = 0; j < PP; ++j) {
                    Pn_[j] = q < nqload ? pp[(q * PP + j) * CONSUMERS] : zero2();
                    Nn_[j] = zero2();
                }
                const float* t = stage_ptr();
                accumulate(t, has_imag(lp, q), Pc_, Pn_, Nc_, Nn_);
                if (q >= 1 && q - 1 < nqp) finalize(t, Pc_);
                stage_done();
                if (q < nqn) {
    #pragma unroll
                    for (int j = 0; j < PP; ++j) pp[(q * PP + j) * CONSUMERS] = Nc_[j];
                }
            };
            int q = 0;
            for (; q + 1 < nq && alive; q += 2) {
                qstep(q, Pc, Nc, Pn, Nn);
                qstep(q + 1, Pn, Nn, Pc, Nc);
            }
            if (q < nq && alive) {
                qstep(q, Pc, Nc, Pn, Nn);
    #pragma unroll
                for (int j = 0; j < PP; ++j) { Pc[j] = Pn[j]; Nc[j] = Nn[j]; }
            }
            if (alive && nq - 1 < nqp) {
                // tail step: the last previous-order target
                const float* t = stage_ptr();
                finalize(t, Pc);
                stage_done();
            }
            if (nq < nqn) {
    #pragma unroll
                for (int j = 0; j < PP; ++j) pp[(nq * PP + j) * CONSUMERS] = Nc[j];
            }
        }
        // outputs of the order above the last input order have no further inputs
        const int L = last_in + 1;
        if (L <= prm.top) {
            set_order(L);
            for (int q = 0; q < nq_of(L) && alive; ++q) {
                f2 W[PP];
    #pragma unroll
                for (int j = 0; j < PP; ++j) W[j] = pp[(q * PP + j) * CONSUMERS];
                const float* t = stage_ptr();
                finalize(t, W);
                stage_done();
            }
        }
        // every tile consumes exactly the stages the producers issue for it
        if (alive && s != (tl + 1) * prm.nstages) {
            alive = false;
            atomicExch(prm.err, 1);
        }
    }
}

// Single-instance pass: a persistent grid; CTA b takes tiles b, b + gridDim.x,
// ... (raster order).  The CTAs then work on one contiguous band of tiles
// at any time, so the halo rows that vertically adjacent tiles share come
// from DRAM once, and each CTA's pipeline runs on across its tiles.
__global__ void __launch_bounds__(THREADS, MINB) k_tiled_pass(const __grid_constant__ Params prm, int ntiles) {
    tiled_tiles(prm, prm.maps, blockIdx.x, gridDim.x, ntiles, true);
}

// Batched pass: CTA b runs items[off[b]] .. items[off[b + 1] - 1], each a
// strided run of tiles of one instance, (instance, first tile, tile count,
// tile stride), streamed through one pipeline.  Instance i's
// parameters for parity P and coefficient set `which` are
// prms[(2 i + P) * 2 + which] in global memory; the CTA copies them to
// shared memory and hands TMA the tensor maps of the global copy.
__global__ void __launch_bounds__(THREADS, MINB) k_tiled_batch(const Params* __restrict__ prms,
                                                            const int4* __restrict__ items,
                                                            const int* __restrict__ off, int P, int which) {
    __shared__ Params s_prm;
    const int begin = off[blockIdx.x], end = off[blockIdx.x + 1];
    for (int it = begin; it < end; ++it) {
        const int4 item = items[it];
        const Params* g = prms + (2 * item.x + P) * 2 + which;
        if (it != begin) __syncthreads();             // previous run done with s_prm and the barriers
        {
            const uint4* src = reinterpret_cast<const uint4*>(g);
            uint4* dst = reinterpret_cast<uint4*>(&s_prm);
            for (int i = threadIdx.x; i < (int)(sizeof(Params) / 16); i += blockDim.x) dst[i] = src[i];
        }
        __syncthreads();
        tiled_tiles(s_prm, g->maps, item.y, item.w, item.y + (item.z - 1) * item.w + 1, it == begin);
    }
}

}  // namespace STARMAP_TILED_NS
}  // namespace starmap
