// Temporally fused step of the merged schedule (FP32, 2D, sm_103a): one
// launch applies the full even update E_dt (the fused even pair) and then
// the full odd update O_dt (two merged odd halves), tile by tile, so that
// a step reads the state once and writes it once (eq.
// solution_operator_full_step, the odd-half merge of section 5.8).
//
// The odd update of a tile needs the NEW even values on the tile plus one
// point on one side per axis (the staggered differences of eq.
// central_differences).  So each CTA runs two machines on the same tile:
//   * E computes the new even values on a window of its own, per output
//     kind (G11 and G22): 64 x 6 points placed so that they cover what the
//     odd update of the tile reads (the side is fixed by the staggering and
//     the boundary type, and the stencil then never reaches further than
//     the existing one-point boundary copies).  It writes them to the even
//     grids of the OTHER buffer set (the new state); neighbouring windows
//     overlap and write the same values bit for bit.
//   * O updates the 62 x 5 odd points of the tile from those new even
//     values, loading them back by TMA (they are still in L2), reading the
//     old odd values from the current set and writing the other set.
// O waits for E per stage: every E consumer warp publishes how many stages
// it has completed (after its stores and a generic-to-async proxy fence),
// and O's producer issues a stage only when every E warp has completed the
// E stage that finalises the stage's inputs.  Both machines stream the
// moment orders exactly like the two-pass kernel (same stage lists,
// coefficient rows and finalise tables), so every point sees the same
// arithmetic in the same order: the fused step equals the two passes bit
// for bit.
//
// Buffers: the current set is read only (old even for E's decay term, old
// odd for E's differences and O's decay term); the other set is written.
// The caller refreshes the new odd grids' boundary copies after the launch
// (E writes the new even values' copies that O reads itself).
//
// Every wait is bounded (2 s): on expiry the CTA raises the error flag,
// waits (bounded) for its own copies in flight and returns.

namespace starmap {
namespace fused {

using tiled::f2;
using tiled::f2_make;
using tiled::f2_split;
using tiled::f2_fma;
using tiled::f2_sub;
using tiled::f2_add;
using tiled::f2_mul;
using tiled::lds2;
using tiled::zero2;
using tiled::diff_x;
using tiled::mbar_init;
using tiled::fence_mbar_init;
using tiled::mbar_expect_tx;
using tiled::mbar_arrive;
using tiled::mbar_try_wait;
using tiled::global_ns;
using tiled::tma_load_3d;
using tiled::wait_bounded;
using tiled::input_shift;
using tiled::nq_of;
using tiled::has_imag;
using tiled::OutGrid;

constexpr int TXO = 62;                 // odd outputs per tile row
constexpr int TYO = 5;                  // odd tile rows
constexpr int TYE = TYO + 1;            // even window rows
constexpr int CW = 64;                  // points per computed row (32 lanes x 2)
constexpr int VEC = 4;                  // 16 bytes of FP32: TMA x alignment
constexpr int BXI = 72;                 // input box width (both machines)
constexpr int BYI = TYO + 2;            // input box rows: y0 - 1 .. y0 + TYO
constexpr int BXO = 68;                 // old-output box width (a window starts 0 or 2 past its box)
constexpr int IN_SLOT = ((BXI * BYI * 4 + 127) / 128) * 128;
constexpr int EOUT_SLOT = ((BXO * TYE * 4 + 127) / 128) * 128;
constexpr int OOUT_SLOT = ((BXO * TYO * 4 + 127) / 128) * 128;
constexpr int E_STAGE = 2 * IN_SLOT + 2 * EOUT_SLOT;
constexpr int O_STAGE = 2 * IN_SLOT + 2 * OOUT_SLOT;
constexpr int E_WARPS = 2 * TYE;        // per output kind, one warp per window row
constexpr int O_WARPS = 2 * TYO;
constexpr int E_CONS = E_WARPS * 32;
constexpr int O_CONS = O_WARPS * 32;
constexpr int E_PROD = E_WARPS + O_WARPS;   // warp index of E's producer
constexpr int O_PROD = E_PROD + 1;
constexpr int THREADS = (O_PROD + 1) * 32;
constexpr int MAXR = 12;                // ring stages per machine, at most
// barrier area: E full/empty, O full/empty, abort flag, E warps' progress, O warps' progress
constexpr int BAR_BYTES = 4 * MAXR * 8 + 4 + 4 * E_WARPS + 4 * O_WARPS;
constexpr int RING_OFF = ((BAR_BYTES + 127) / 128) * 128;
constexpr unsigned long long WAIT_NS = 2000000000ull;
constexpr int PUBLISH = 8;              // E stages between progress publications
// E may run at most LEAD of its stages ahead of what O has consumed, so that
// O's loads of the new even values and of the old odd values (which E read
// shortly before) find them in L2
constexpr int LEAD = 32;

struct Machine {
    CUtensorMap maps[4];        // input R, input I, old output R, old output I
    OutGrid out[2];             // new values of output kind R, I (the other buffer set)
    int nstages, nin, nfin, nring;
    const int4* stages;
    const float4* coef[2];
    const int2* fin[2];
    int smem_coef_off[2], smem_fin_off[2], smem_stage_off, smem_part_off, ring_off;
};

struct FusedParams {
    Machine m[2];               // 0: even update E, 1: odd update O
    const int* odep;            // per O stage: E stages of the same tile complete before its loads
    int smem_odep_off;
    long pitch;
    int p[2];
    int tiles_x;
    int N;
    int nclasses;
    const float* const* srcs;
    int* err;
};

__host__ __device__ constexpr int floor4(int v) { return v >= 0 ? v & ~3 : -((-v + 3) & ~3); }

// Tile geometry of one machine and output kind: window origin (first
// computed point) and the origins of the input boxes and of the kind's
// old-output box.
struct Geo {
    int wx, wy;                 // window origin
    int bx, by;                 // both input boxes
    int ox, oy;                 // old-output box of this kind
};

__device__ __forceinline__ Geo geometry(int E, int K, int x0, int y0, int px, int py) {
    Geo g;
    if (E) {
        // the odd update reads even kind K at shifts (sx - 1, sx) and (sy - 1, sy)
        int sx, sy;
        input_shift(1, K, px, py, sx, sy);
        g.wx = x0 - 2 * (1 - sx);           // covers x0 + sx - 1 .. x0 + TXO - 1 + sx, even origin
        g.wy = y0 + sy - 1;                 // covers y0 + sy - 1 .. y0 + TYO - 1 + sy
        g.bx = floor4(x0 - 2);              // inputs: columns x0 - 3 .. x0 + 64 at most
        g.by = y0 - 1;
    } else {
        g.wx = x0;
        g.wy = y0;
        g.bx = floor4(x0 - 1);              // columns x0 - 1 .. x0 + 64
        g.by = y0 - 1;
    }
    g.ox = g.wx & ~3;                       // the window origin is even: 0 or 2 past the box
    g.oy = g.wy;
    return g;
}

__device__ __forceinline__ int wrap_or_clamp(int v, int n, int periodic) {
    if (periodic) return v < 0 ? v + n : (v >= n ? v - n : v);
    return v < 0 ? 0 : (v >= n ? n - 1 : v);
}

// One CTA: tiles t0, t0 + tstride, ... < tend, both machines.
__device__ __forceinline__ void fused_tiles(const FusedParams& prm, int t0, int tstride, int tend) {
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* efull = reinterpret_cast<uint64_t*>(smem);
    uint64_t* eempty = efull + MAXR;
    uint64_t* ofull = eempty + MAXR;
    uint64_t* oempty = ofull + MAXR;
    volatile int* abort_flag = reinterpret_cast<volatile int*>(oempty + MAXR);
    volatile int* eprog = abort_flag + 1;
    volatile int* oprog = eprog + E_WARPS;      // in E stages: the E stage each O warp's last stage needed

    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int ntl = t0 < tend ? (tend - t0 + tstride - 1) / tstride : 0;
    const int px = prm.p[0], py = prm.p[1];

    if (warp == E_PROD && lane < 4)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(prm.m[0].maps + lane)) : "memory");
    if (warp == O_PROD && lane < 4)
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(prm.m[1].maps + lane)) : "memory");
    if (tid == 0) {
        for (int r = 0; r < MAXR; ++r) {
            mbar_init(&efull[r], 1);
            mbar_init(&eempty[r], E_WARPS);
            mbar_init(&ofull[r], 1);
            mbar_init(&oempty[r], O_WARPS);
        }
        *abort_flag = 0;
        for (int w = 0; w < E_WARPS; ++w) eprog[w] = 0;
        for (int w = 0; w < O_WARPS; ++w) oprog[w] = 0;
        fence_mbar_init();
    }
    for (int M = 0; M < 2; ++M) {
        const Machine& m = prm.m[M];
        for (int k = 0; k < 2; ++k) {
            float4* c = reinterpret_cast<float4*>(smem + m.smem_coef_off[k]);
            for (int i = tid; i < 2 * m.nin; i += THREADS) c[i] = __ldg(m.coef[k] + i);
            int2* f = reinterpret_cast<int2*>(smem + m.smem_fin_off[k]);
            for (int i = tid; i < m.nfin; i += THREADS) f[i] = __ldg(m.fin[k] + i);
        }
        int4* st = reinterpret_cast<int4*>(smem + m.smem_stage_off);
        for (int i = tid; i < m.nstages; i += THREADS) st[i] = __ldg(m.stages + i);
    }
    {
        int* od = reinterpret_cast<int*>(smem + prm.smem_odep_off);
        for (int i = tid; i < prm.m[1].nstages; i += THREADS) od[i] = __ldg(prm.odep + i);
    }
    __syncthreads();
    // everything above reads host-written data; the state only below
    pdl_trigger();
    pdl_wait();

    // --------------------------------------------------------- producers
    if (warp >= E_PROD) {
        const int E = warp == E_PROD ? 1 : 0;
        const Machine& m = prm.m[E ? 0 : 1];
        uint64_t* full = E ? efull : ofull;
        uint64_t* empty = E ? eempty : oempty;
        unsigned char* ring = smem + m.ring_off;
        const int SB = E ? E_STAGE : O_STAGE;
        const int OUTB = E ? BXO * TYE * 4 : BXO * TYO * 4;
        const int OUTSLOT = E ? EOUT_SLOT : OOUT_SLOT;
        const int slot = lane & 3;
        const CUtensorMap* map = m.maps + slot;
        const int4* s_stages = reinterpret_cast<const int4*>(smem + m.smem_stage_off);
        const int* s_odep = reinterpret_cast<const int*>(smem + prm.smem_odep_off);
        const int nst = m.nstages;
        const int nste = prm.m[0].nstages;
        const int NR = m.nring;
        const int total = ntl * nst;
        int last = -1;
        bool ok = true;
        int k = 0, tl = 0, r = 0, u = 0, tile_at = -1, bx = 0, by = 0;
        for (int G = 0; G < total; ++G) {
            if (tl != tile_at) {
                tile_at = tl;
                const int tile = t0 + tl * tstride;
                const int x0 = (tile % prm.tiles_x) * TXO, y0 = (tile / prm.tiles_x) * TYO;
                if (slot < 2) {
                    const Geo g = geometry(E, 0, x0, y0, px, py);
                    bx = g.bx;
                    by = g.by;
                } else {
                    const Geo g = geometry(E, slot - 2, x0, y0, px, py);
                    bx = g.ox;
                    by = g.oy;
                }
            }
            int4 st = make_int4(-1, -1, -1, -1);
            if (lane < 4) st = s_stages[k];
            const int comp = slot == 0 ? st.x : slot == 1 ? st.y : slot == 2 ? st.z : st.w;
            const uint32_t mine = lane < 4 && comp >= 0 ? (slot < 2 ? (uint32_t)(BXI * BYI * 4) : (uint32_t)OUTB) : 0u;
            uint32_t bytes = mine;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(0xffffffffu, bytes, o);
            if (E && ok && G >= LEAD) {
                // keep E within LEAD stages of what O has consumed
                const int need = G - LEAD;
                const unsigned long long tw = global_ns();
                for (;;) {
                    int v = lane < O_WARPS ? oprog[lane] : 0x7fffffff;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
                    if (v >= need) break;
                    if (*abort_flag) { ok = false; break; }
                    if (global_ns() - tw > WAIT_NS) {
                        if (lane == 0) { *abort_flag = 1; atomicExch(prm.err, 1); }
                        ok = false;
                        break;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            }
            if (!E && ok) {
                // the odd stage's inputs are new even values: wait until every
                // E warp has completed the E stage that finalises them
                const int need = tl * nste + s_odep[k];
                const unsigned long long tw = global_ns();
                for (;;) {
                    int v = lane < E_WARPS ? eprog[lane] : 0x7fffffff;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
                    if (v >= need) break;
                    if (*abort_flag) { ok = false; break; }
                    if (global_ns() - tw > WAIT_NS) {
                        if (lane == 0) { *abort_flag = 1; atomicExch(prm.err, 1); }
                        ok = false;
                        break;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                // the generic-proxy stores of the E warps, seen by the TMA loads below
                asm volatile("fence.proxy.async.global;" ::: "memory");
            }
            if (lane == 0 && ok) {
                if (u > 0 && !wait_bounded(&empty[r], (u - 1) & 1, abort_flag, prm.err)) ok = false;
                if (ok) mbar_expect_tx(&full[r], bytes);
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            if (mine != 0u) {
                const int off = slot < 2 ? slot * IN_SLOT : 2 * IN_SLOT + (slot - 2) * OUTSLOT;
                // tensor coordinates: x' = x + VEC (a multiple of 4: x is), row = y + 1
                tma_load_3d(ring + r * SB + off, map, bx + VEC, by + 1, comp, &full[r]);
            }
            last = G;
            if (++k == nst) { k = 0; ++tl; }
            if (++r == NR) { r = 0; ++u; }
        }
        if (!ok && lane == 0) {
            for (int G = last; G >= 0 && G > last - NR; --G) {
                const unsigned long long tw = global_ns();
                while (!mbar_try_wait(&full[G % NR], (G / NR) & 1))
                    if (global_ns() - tw > WAIT_NS) break;
            }
        }
        return;
    }

    // --------------------------------------------------------- consumers
    const int E = warp < E_WARPS ? 1 : 0;
    const int lw = E ? warp : warp - E_WARPS;           // warp index inside the machine
    const int RPK = E ? TYE : TYO;                      // warps (rows) per output kind
    const int K = lw / RPK;
    const int row = lw % RPK;
    const Machine& m = prm.m[E ? 0 : 1];
    uint64_t* full = E ? efull : ofull;
    uint64_t* empty = E ? eempty : oempty;
    const unsigned char* ring = smem + m.ring_off;
    const int SB = E ? E_STAGE : O_STAGE;
    const int OUTSLOT = E ? EOUT_SLOT : OOUT_SLOT;
    const int NR = m.nring;
    const int ncons = E ? E_CONS : O_CONS;
    const int ctid = E ? tid : tid - E_CONS;            // thread index inside the machine
    const int* s_odep = reinterpret_cast<const int*>(smem + prm.smem_odep_off);
    f2* const pp = reinterpret_cast<f2*>(smem + m.smem_part_off) + ctid;
    int sxR, syR, sxI, syI;
    input_shift(E ? 0 : 1, 0, px, py, sxR, syR);
    input_shift(E ? 0 : 1, 1, px, py, sxI, syI);
    const OutGrid& G = m.out[K];
    const long plane = (long)G.nx * G.ny;
    const bool xnode = E ? (K == 1) : (K == 0);          // G22 / G21 have node columns
    const bool ynode = K == 1;                           // G22 / G12 have node rows
    int s = 0, ring_r = 0;
    uint32_t ring_ph = 0;
    bool alive = true;
    for (int tl = 0; tl < ntl && alive; ++tl) {
        const int tile = t0 + tl * tstride;
        const int x0 = (tile % prm.tiles_x) * TXO, y0 = (tile / prm.tiles_x) * TYO;
        const Geo g = geometry(E, K, x0, y0, px, py);
        const int gx = g.wx + 2 * lane, gy = g.wy + row;   // point A; B = A + (1, 0)
        // offsets inside a stage: d_x from the input of kind K (slot K), d_y
        // from the input of kind 1 - K (slot 1 - K), old value (slot 2 + K)
        const int sxK = K == 0 ? sxR : sxI;
        const int syO = K == 0 ? syI : syR;
        const int rx = K * IN_SLOT / 4 + (gy - g.by) * BXI;
        const int cx = gx + sxK - g.bx;                   // right operand of point A
        const bool ev = (cx & 1) == 0;
        const int uy = (1 - K) * IN_SLOT / 4 + (gy + syO - g.by) * BXI + (gx - g.bx);
        const int uoff = (2 * IN_SLOT + K * OUTSLOT) / 4 + (gy - g.oy) * BXO + (gx - g.ox);
        // which points are stored, and where their coefficients sit
        bool stA, stB, plain;
        long cA, cB;
        {
            auto keep = [&](int x, int y) -> bool {
                const bool ix = x >= 0 && x < G.nx, iy = y >= 0 && y < G.ny;
                if (!E) return ix && iy && x - x0 < TXO;
                if (ix && iy) return true;
                if (px && (x == -1 || x == G.nx) && iy) return true;     // periodic: the wrapped point
                if (py && (y == -1 || y == G.ny) && ix) return true;
                return false;
            };
            stA = keep(gx, gy);
            stB = keep(gx + 1, gy);
            // both inside the grid and neither a boundary point with a copy to write
            auto copy = [&](int x) -> bool {
                return E && ((!px && !xnode && (x == 0 || x == G.nx - 1)) ||
                             (!py && !ynode && (gy == 0 || gy == G.ny - 1)));
            };
            plain = stA && stB && gx >= 0 && gx + 1 < G.nx && gy >= 0 && gy < G.ny && !copy(gx) && !copy(gx + 1);
            const int yw = wrap_or_clamp(gy, G.ny, py);
            cA = (long)yw * G.nx + wrap_or_clamp(gx, G.nx, px);
            cB = (long)yw * G.nx + wrap_or_clamp(gx + 1, G.nx, px);
        }
        const long apos = (long)(gy + 1) * prm.pitch + gx;         // point A inside a component
        f2 ca2[2], cb2[2];
        for (int c = 0; c < 2; ++c) {
            float a[2] = {0.f, 0.f}, b[2] = {0.f, 0.f};
            if (prm.nclasses == 2 && G.coef != nullptr) {
                const float* cf = G.coef + (long)c * 4 * plane;
                a[0] = __ldg(cf + 2 * plane + cA); b[0] = __ldg(cf + 3 * plane + cA);
                a[1] = __ldg(cf + 2 * plane + cB); b[1] = __ldg(cf + 3 * plane + cB);
            }
            ca2[c] = f2_make(a[0], a[1]);
            cb2[c] = f2_make(b[0], b[1]);
        }
        const float4* cp = reinterpret_cast<const float4*>(smem + m.smem_coef_off[K]);
        const int2* fp = reinterpret_cast<const int2*>(smem + m.smem_fin_off[K]);
        auto stage_ptr = [&]() -> const float* {
            if (alive) alive = wait_bounded(&full[ring_r], ring_ph, abort_flag, prm.err);
            return reinterpret_cast<const float*>(ring + ring_r * SB);
        };
        const int tile_end = (tl + 1) * m.nstages;
        auto stage_done = [&]() {
            // E publishes its progress every PUBLISH stages and at the tile's
            // end, after a generic-to-async proxy fence over its stores (a
            // fence waits for them: one per stage would stall the warp)
            const bool publish = E && ((s + 1) % PUBLISH == 0 || s + 1 == tile_end);
            if (publish) asm volatile("fence.proxy.async.global;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&empty[ring_r]);
                if (publish) {
                    __threadfence_block();
                    eprog[lw] = s + 1;
                }
                if (!E) oprog[lw] = tl * prm.m[0].nstages + s_odep[s - tl * m.nstages];
            }
            ++s;
            if (++ring_r == NR) { ring_r = 0; ring_ph ^= 1u; }
        };
        f2 aL, bL;
        auto set_order = [&](int L) {
            if (prm.nclasses == 2) {
                aL = L == 0 ? ca2[0] : ca2[1];
                bL = L == 0 ? cb2[0] : cb2[1];
            } else {
                const float* cf = G.coef + (long)L * 4 * plane;
                aL = f2_make(__ldg(cf + 2 * plane + cA), __ldg(cf + 2 * plane + cB));
                bL = f2_make(__ldg(cf + 3 * plane + cA), __ldg(cf + 3 * plane + cB));
            }
        };
        auto put = [&](float* comp, int x, int y, float v) { comp[(long)(y + 1) * prm.pitch + x] = v; };
        auto finalize = [&](const float* t, f2 W) {
            const int2 f = *fp;
            fp += 1;
            const f2 uo = lds2(t + uoff);
            f2 w = W;
            if (f.y >= 0) {
                const float* qs = prm.srcs[f.y];
                w = f2_add(w, f2_make(__ldg(qs + cA), __ldg(qs + cB)));
            }
            const f2 v = f2_fma(aL, uo, f2_mul(bL, w));
            if (f.x < 0 || !alive) return;
            float* comp0 = G.base + 32 * (long)f.x;          // 64-bit: states beyond 2^31 values
            if (plain) {
                *reinterpret_cast<f2*>(comp0 + apos) = v;     // gx is even: an 8-byte store
                return;
            }
            float v0, v1;
            f2_split(v, v0, v1);
            const float vv[2] = {v0, v1};
            const bool stv[2] = {stA, stB};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (!stv[q]) continue;
                const int x = gx + q;
                put(comp0, x, gy, vv[q]);
                if (E && x >= 0 && x < G.nx && gy >= 0 && gy < G.ny) {
                    // extrapolation boundaries of a cell axis: the boundary copy
                    if (!px && !xnode) {
                        if (x == 0) put(comp0, -1, gy, vv[q]);
                        if (x == G.nx - 1) put(comp0, G.nx, gy, vv[q]);
                    }
                    if (!py && !ynode) {
                        if (gy == 0) put(comp0, x, -1, vv[q]);
                        if (gy == G.ny - 1) put(comp0, x, G.ny, vv[q]);
                    }
                }
            }
        };
        auto accumulate = [&](const float* t, bool inI, f2& Pc, f2& Pn, f2& Nc, f2& Nn) {
            const float4 cxv = cp[0], cyv = cp[1];
            cp += 2;
            const f2 xPm = f2_make(cxv.x, cxv.x), xP0 = f2_make(cxv.y, cxv.y);
            const f2 xN0 = f2_make(cxv.z, cxv.z), xNp = f2_make(cxv.w, cxv.w);
            const f2 yPm = f2_make(cyv.x, cyv.x), yP0 = f2_make(cyv.y, cyv.y);
            const f2 yN0 = f2_make(cyv.z, cyv.z), yNp = f2_make(cyv.w, cyv.w);
            f2 dx = diff_x(t + rx, cx, ev);
            f2 dy = f2_sub(lds2(t + uy), lds2(t + uy - BXI));
            if (!inI) {
                if (K == 1) dx = zero2(); else dy = zero2();
            }
            Pc = f2_fma(xPm, dx, Pc);
            Pn = f2_fma(xP0, dx, Pn);
            Nc = f2_fma(xN0, dx, Nc);
            Nn = f2_fma(xNp, dx, Nn);
            Pc = f2_fma(yPm, dy, Pc);
            Pn = f2_fma(yP0, dy, Pn);
            Nc = f2_fma(yN0, dy, Nc);
            Nn = f2_fma(yNp, dy, Nn);
        };

        const int N = prm.N;
        const int first = E;                      // the even update streams the odd orders 1, 3, ...
        int last_in = first;
        for (int lp = first; lp <= N && alive; lp += 2) {
            last_in = lp;
            const int nq = nq_of(lp);
            const int nqp = nq_of(lp - 1);
            const int nqn = lp + 1 <= N ? nq_of(lp + 1) : 0;
            const int nqload = lp > first ? nqp : 0;
            set_order(lp - 1);
            f2 Pc = zero2(), Nc = zero2(), Pn, Nn;
            auto qstep = [&](int q, f2& Pc_, f2& Nc_, f2& Pn_, f2& Nn_) {
                Pn_ = q < nqload ? pp[q * ncons] : zero2();
                Nn_ = zero2();
                const float* t = stage_ptr();
                accumulate(t, has_imag(lp, q), Pc_, Pn_, Nc_, Nn_);
                if (q >= 1 && q - 1 < nqp) finalize(t, Pc_);
                stage_done();
                if (q < nqn) pp[q * ncons] = Nc_;
            };
            int q = 0;
            for (; q + 1 < nq && alive; q += 2) {
                qstep(q, Pc, Nc, Pn, Nn);
                qstep(q + 1, Pn, Nn, Pc, Nc);
            }
            if (q < nq && alive) {
                qstep(q, Pc, Nc, Pn, Nn);
                Pc = Pn;
                Nc = Nn;
            }
            if (alive && nq - 1 < nqp) {
                const float* t = stage_ptr();
                finalize(t, Pc);
                stage_done();
            }
            if (nq < nqn) pp[nq * ncons] = Nc;
        }
        const int L = last_in + 1;
        if (L <= N) {
            set_order(L);
            for (int q = 0; q < nq_of(L) && alive; ++q) {
                const f2 W = pp[q * ncons];
                const float* t = stage_ptr();
                finalize(t, W);
                stage_done();
            }
        }
        if (alive && s != (tl + 1) * m.nstages) {
            alive = false;
            atomicExch(prm.err, 1);
        }
    }
}

// Persistent grid: CTA b takes tiles b, b + gridDim.x, ... (raster order).
__global__ void __launch_bounds__(THREADS, 1) k_fused_step(const __grid_constant__ FusedParams prm, int ntiles) {
    fused_tiles(prm, blockIdx.x, gridDim.x, ntiles);
}

}  // namespace fused
}  // namespace starmap
