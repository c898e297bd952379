// Tiled half-step pass for the 2D real P_N system in FP32 (sm_103a).
//
// One CTA owns a TX x TY tile of point indices, shared by the four staggered
// grids (section 4.1).  A pass updates the components of one parity (odd l:
// grids G21 (R) and G12 (I); even l: G11 (R) and G22 (I)) from the half-grid
// differences (eq. central_differences) of the other parity, weighted by
// -Mx/dx and -My/dy, followed by the exact sub-step u <- a u + b (W + q)
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
// Data movement: one producer warp walks a host-built item list and issues
// one TMA box (cp.async.bulk.tensor.3d) per item into a ring of shared-memory
// slots guarded by mbarriers (full: transaction bytes, empty: one arrival per
// consumer warp).  Input boxes are BX x (TY+1) (one-point halo, x start
// aligned to 16 bytes); output boxes TX x TY.  Boundary conditions live in
// ghost cells, which the finalising thread writes with each boundary value.
// Every wait is bounded: on expiry the kernel raises an error flag, waits
// (bounded) for its copies in flight, and returns.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace starmap {
namespace tiled {

constexpr int TX = 32;                  // tile width (one warp per row)
constexpr int TY = 8;                   // tile height (one consumer warp per row)
constexpr int VEC = 4;                  // 16 bytes of FP32: TMA x alignment
constexpr int BX = TX + VEC;            // input box width (halo + alignment)
constexpr int BYI = TY + 1;             // input box height (halo)
constexpr int IN_BYTES = BX * BYI * 4;  // 1296
constexpr int OUT_BYTES = TX * TY * 4;  // 1024
constexpr int SLOT = 1408;              // slot stride in bytes, multiple of 128
constexpr int GROUP = 4;                // items per mbarrier stage
constexpr int NSTAGES = 8;              // stages in the ring
constexpr int NSLOTS = GROUP * NSTAGES;
constexpr int CONSUMER_WARPS = TY;
constexpr int CONSUMERS = CONSUMER_WARPS * 32;
constexpr int THREADS = CONSUMERS + 32;
constexpr int MAXN = 63;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // bounded waits: 2 s

// item codes: bits 30..31 = map (0 input R, 1 input I, 2 output R, 3 output I),
// bits 0..29 = component index inside its grid
constexpr uint32_t ITEM_MAP_SHIFT = 30;

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
    int nitems, nin, nfin;
    const uint32_t* items;      // TMA item stream
    const float4* coef;         // per input: (cx Pm, P0, N0, Np), (cy Pm, P0, N0, Np)
    const int2* fin;            // per finalise event: (component index in grid, class)
    const float* const* src;    // per finalise event: source array or null
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
__device__ __forceinline__ void input_shift(int P, int k, const int p[2], int& sx, int& sy) {
    // input grids: odd pass (P=1) R -> G11, I -> G22; even pass R -> G21, I -> G12
    const int g = P == 1 ? (k == 0 ? 0 : 3) : (k == 0 ? 1 : 2);
    const bool xnode = g & 1, ynode = g & 2;
    sx = xnode ? 1 - p[0] : p[0];
    sy = ynode ? 1 - p[1] : p[1];
}

__global__ void __launch_bounds__(THREADS, 2) k_tiled_pass(const __grid_constant__ Params prm) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + NSTAGES;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + NSTAGES);
    float* ring = reinterpret_cast<float*>(smem + 256);
    float4* s_coef = reinterpret_cast<float4*>(smem + prm.smem_coef_off);
    int2* s_fin = reinterpret_cast<int2*>(smem + prm.smem_fin_off);
    float* s_part = reinterpret_cast<float*>(smem + prm.smem_part_off);

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
    for (int i = tid; i < 2 * prm.nin; i += THREADS) s_coef[i] = __ldg(prm.coef + i);
    for (int i = tid; i < prm.nfin; i += THREADS) s_fin[i] = __ldg(prm.fin + i);
    __syncthreads();

    int sx[2], sy[2];
    input_shift(prm.P, 0, prm.p, sx[0], sy[0]);
    input_shift(prm.P, 1, prm.p, sx[1], sy[1]);

    // --------------------------------------------------------- producer
    if (warp == CONSUMER_WARPS) {
        if (lane == 0) {
            int issued_stages = 0;
            bool ok = true;
            for (int s = 0; s * GROUP < prm.nitems; ++s) {
                const int r = s % NSTAGES;
                if (s >= NSTAGES && !wait_bounded(&empty[r], ((s / NSTAGES) - 1) & 1, abort_flag, prm.err)) {
                    ok = false;
                    break;
                }
                const int i0 = s * GROUP, i1 = min(prm.nitems, i0 + GROUP);
                uint32_t bytes = 0;
                for (int i = i0; i < i1; ++i) bytes += (__ldg(prm.items + i) >> ITEM_MAP_SHIFT) < 2 ? IN_BYTES : OUT_BYTES;
                fence_proxy_async();
                mbar_expect_tx(&full[r], bytes);
                for (int i = i0; i < i1; ++i) {
                    const uint32_t code = __ldg(prm.items + i);
                    const int map = code >> ITEM_MAP_SHIFT;
                    const int comp = code & ((1u << ITEM_MAP_SHIFT) - 1);
                    float* dst = ring + (size_t)(i % NSLOTS) * (SLOT / 4);
                    if (map < 2) {
                        // x' = x + VEC; start VEC early when the left neighbour is needed
                        const int bx = x0 + (sx[map] == 0 ? 0 : VEC);
                        const int by = y0 + (sy[map] == 0 ? -1 : 0) + 1;
                        tma_load_3d(dst, &prm.maps[map], bx, by, comp, &full[r]);
                    } else {
                        tma_load_3d(dst, &prm.maps[map], x0 + VEC, y0 + 1, comp, &full[r]);
                    }
                }
                ++issued_stages;
            }
            if (!ok) {
                // aborted: wait (bounded) for the copies still in flight
                for (int s = issued_stages - 1; s >= 0 && s >= issued_stages - NSTAGES; --s) {
                    const unsigned long long t0 = global_ns();
                    while (!mbar_try_wait(&full[s % NSTAGES], (s / NSTAGES) & 1))
                        if (global_ns() - t0 > WAIT_NS) break;
                }
            }
        }
        return;
    }

    // --------------------------------------------------------- consumers
    const int gx = x0 + lane, gy = y0 + warp;
    // smem offsets of the difference operands inside an input box of kind k
    int dxr[2], dyu[2];
    for (int k = 0; k < 2; ++k) {
        const int bxs = sx[k] == 0 ? -VEC : 0;       // box x start relative to x0
        const int oy = sy[k] == 0 ? -1 : 0;          // box y start relative to y0
        dxr[k] = (warp - oy) * BX + (lane + sx[k] - bxs);
        dyu[k] = (warp + sy[k] - oy) * BX + (lane - bxs);
    }
    // output grids (kind 0 = R, 1 = I)
    bool inr[2];
    long row_off[2], cidx[2], plane[2];
    int gxa[2], gxb[2], gya[2], gyb[2];
    float ca[2][2], cb[2][2];
    for (int k = 0; k < 2; ++k) {
        const OutGrid& G = prm.out[k];
        const int g = prm.P == 1 ? (k == 0 ? 1 : 2) : (k == 0 ? 0 : 3);
        const bool xnode = g & 1, ynode = g & 2;
        inr[k] = gx < G.nx && gy < G.ny;
        row_off[k] = (long)(gy + 1) * prm.pitch + gx;
        plane[k] = (long)G.nx * G.ny;
        cidx[k] = (long)gy * G.nx + gx;
        int xa = -2, xb = -2, ya = -2, yb = -2;
        if (prm.p[0]) { if (gx == G.nx - 1) xa = -1; if (gx == 0) xb = G.nx; }
        else if (!xnode) { if (gx == 0) xa = -1; if (gx == G.nx - 1) xb = G.nx; }
        if (prm.p[1]) { if (gy == G.ny - 1) ya = -1; if (gy == 0) yb = G.ny; }
        else if (!ynode) { if (gy == 0) ya = -1; if (gy == G.ny - 1) yb = G.ny; }
        gxa[k] = xa; gxb[k] = xb; gya[k] = ya; gyb[k] = yb;
        for (int c = 0; c < 2; ++c) {
            ca[k][c] = 0.f;
            cb[k][c] = 0.f;
            if (inr[k] && prm.nclasses == 2 && G.coef != nullptr) {
                const float* cf = G.coef + (long)c * 4 * plane[k] + cidx[k];
                ca[k][c] = __ldg(cf + 2 * prm.which * plane[k]);
                cb[k][c] = __ldg(cf + (2 * prm.which + 1) * plane[k]);
            }
        }
    }

    int it = 0, ii = 0, e = 0;
    bool alive = true;
    auto acquire = [&](int i) -> const float* {
        if (i % GROUP == 0 && alive)
            alive = wait_bounded(&full[(i / GROUP) % NSTAGES], ((i / GROUP) / NSTAGES) & 1, abort_flag, prm.err);
        return ring + (size_t)(i % NSLOTS) * (SLOT / 4);
    };
    auto release = [&](int i) {
        if (i % GROUP == GROUP - 1 || i == prm.nitems - 1) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[(i / GROUP) % NSTAGES]);
        }
    };
    auto part = [&](int q, int k) -> float& { return s_part[(q * 2 + k) * CONSUMERS + tid]; };
    auto finalize = [&](int k, int L, float W) {
        const float* t = acquire(it);
        const int2 f = s_fin[e];
        float aa, bb;
        if (prm.nclasses == 2) {
            aa = ca[k][L == 0 ? 0 : 1];
            bb = cb[k][L == 0 ? 0 : 1];
        } else {
            const float* cf = prm.out[k].coef + (long)f.y * 4 * plane[k] + cidx[k];
            aa = inr[k] ? __ldg(cf + 2 * prm.which * plane[k]) : 0.f;
            bb = inr[k] ? __ldg(cf + (2 * prm.which + 1) * plane[k]) : 0.f;
        }
        const float u = t[warp * TX + lane];
        const float* qs = prm.src[e];
        if (qs != nullptr && inr[k]) W += __ldg(qs + cidx[k]);
        const float v = fmaf(aa, u, bb * W);
        if (inr[k] && alive) {
            float* comp = prm.out[k].base + (long)f.x * prm.out[k].cstride;
            comp[row_off[k]] = v;
            const long rowb = row_off[k] - gx;
            if (gxa[k] != -2) comp[rowb + gxa[k]] = v;
            if (gxb[k] != -2) comp[rowb + gxb[k]] = v;
            const long colb = row_off[k] - (long)(gy + 1) * prm.pitch;
            if (gya[k] != -2) comp[colb + (long)(gya[k] + 1) * prm.pitch] = v;
            if (gyb[k] != -2) comp[colb + (long)(gyb[k] + 1) * prm.pitch] = v;
        }
        release(it);
        ++it;
        ++e;
    };

    const int N = prm.N;
    const int first = 1 - prm.P;              // first input order: even l' for the odd pass
    int last_in = first;
    for (int lp = first; lp <= N && alive; lp += 2) {
        last_in = lp;
        const int nq = nq_of(lp);
        const int nqp = nq_of(lp - 1);                    // previous-order targets
        const int nqn = lp + 1 <= N ? nq_of(lp + 1) : 0;  // next-order targets
        float PcR = 0.f, PcI = 0.f, NcR = 0.f, NcI = 0.f;
        for (int q = 0; q < nq && alive; ++q) {
            float PnR = 0.f, PnI = 0.f, NnR = 0.f, NnI = 0.f;
            // partial sums of a previous-order target exist once order
            // lp - 2 has streamed by (not for the first input order)
            if (q < nqp && lp > first) {
                PnR = part(q, 0);
                if (has_imag(lp - 1, q)) PnI = part(q, 1);
            }
            // input R (k = 0) then I (k = 1, only for m' >= 1):
            // d_x feeds targets of the same kind, d_y those of the other kind
            {
                const float* t = acquire(it);
                const float dx = t[dxr[0]] - t[dxr[0] - 1];
                const float dy = t[dyu[0]] - t[dyu[0] - BX];
                const float4 c0 = s_coef[2 * ii], c1 = s_coef[2 * ii + 1];
                release(it);
                ++it;
                ++ii;
                PcR = fmaf(c0.x, dx, PcR); PnR = fmaf(c0.y, dx, PnR);
                NcR = fmaf(c0.z, dx, NcR); NnR = fmaf(c0.w, dx, NnR);
                PcI = fmaf(c1.x, dy, PcI); PnI = fmaf(c1.y, dy, PnI);
                NcI = fmaf(c1.z, dy, NcI); NnI = fmaf(c1.w, dy, NnI);
            }
            if (has_imag(lp, q)) {
                const float* t = acquire(it);
                const float dx = t[dxr[1]] - t[dxr[1] - 1];
                const float dy = t[dyu[1]] - t[dyu[1] - BX];
                const float4 c0 = s_coef[2 * ii], c1 = s_coef[2 * ii + 1];
                release(it);
                ++it;
                ++ii;
                PcI = fmaf(c0.x, dx, PcI); PnI = fmaf(c0.y, dx, PnI);
                NcI = fmaf(c0.z, dx, NcI); NnI = fmaf(c0.w, dx, NnI);
                PcR = fmaf(c1.x, dy, PcR); PnR = fmaf(c1.y, dy, PnR);
                NcR = fmaf(c1.z, dy, NcR); NnR = fmaf(c1.w, dy, NnR);
            }
            if (q >= 1 && q - 1 < nqp) {
                finalize(0, lp - 1, PcR);
                if (has_imag(lp - 1, q - 1)) finalize(1, lp - 1, PcI);
            }
            if (q < nqn) {
                part(q, 0) = NcR;
                if (has_imag(lp + 1, q)) part(q, 1) = NcI;
            }
            PcR = PnR; PcI = PnI; NcR = NnR; NcI = NnI;
        }
        if (alive && nq - 1 < nqp) {
            finalize(0, lp - 1, PcR);
            if (has_imag(lp - 1, nq - 1)) finalize(1, lp - 1, PcI);
        }
        if (nq < nqn) {
            part(nq, 0) = NcR;
            if (has_imag(lp + 1, nq)) part(nq, 1) = NcI;
        }
    }
    // outputs of the order above the last input order have no further inputs
    const int L = last_in + 1;
    if (L <= N && alive) {
        for (int q = 0; q < nq_of(L) && alive; ++q) {
            finalize(0, L, part(q, 0));
            if (has_imag(L, q)) finalize(1, L, part(q, 1));
        }
    }
}

}  // namespace tiled
}  // namespace starmap
