// Host side of the tiled half-step pass: TMA descriptors and the per-pass
// tables (item stream, coefficient rows, finalise events), built by walking
// the same loop the consumer threads walk.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "internal.h"
#include "tiled.h"
// the kernels, once per tile height (namespaces tiled: 10 rows, two per
// consumer warp; tiled5: 5 rows, one per consumer warp)
#include "tiled_kernel.cuh"
#undef STARMAP_TILED_NS
#undef STARMAP_TILED_TY
#undef STARMAP_TILED_MINB
#undef STARMAP_TILED_RW
#define STARMAP_TILED_NS tiled5
#define STARMAP_TILED_TY 5
#define STARMAP_TILED_MINB 2
#define STARMAP_TILED_RW 1
#include "tiled_kernel.cuh"
// the temporally fused step (even then odd update per tile, one launch)
#include "fused_kernel.cuh"

namespace starmap {

using namespace tiled;   // constants and types common to both tile heights

static_assert(sizeof(tiled::Params) == sizeof(tiled5::Params), "both tile heights share the parameter layout");
static_assert(tiled::TX == tiled5::TX && tiled::BX == tiled5::BX, "both tile heights share the tile width");

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3D map over one grid: x' = x + VEC (x = -VEC .. pitch-VEC-1), memory row
// y + 1, component; box (bx, by, 1).  The base address is 16-byte aligned
// (state rows start 128-byte aligned, VEC floats before them).
bool encode_grid_map(CUtensorMap* map, void* base, long pitch, long rows, int K, int bx, int by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)rows, (cuuint64_t)(K > 0 ? K : 1)};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * rows * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    void* addr = (char*)base - VEC * 4;
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, addr, dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// index of (l, m, imag) in the real ordering of eq. transformation
int comp_index(int l, int m, int imag) {
    return l * (l + 1) / 2 + (m > 0 ? 2 * ((l - m) / 2) + imag : l);
}

bool exists(int N, int L, int q, int imag) {
    if (L < 0 || L > N || q < 0 || q >= nq_of(L)) return false;
    return imag ? has_imag(L, q) : true;
}

struct PassTables {
    std::vector<int4> stages;             // slot components: in R, in I, out R, out I (-1 absent)
    std::vector<float> coef;              // nin x 16 (each coefficient twice, for f32x2)
    std::vector<int2> fin;                // (local, class)
    std::vector<int> fin_comp;            // global component per finalise event
    int nin = 0;
    int top = 0;                          // highest output order finalised
};

// Orders up to this use the 5-row tiles by default (few stages per tile:
// two CTAs per SM hide each other's setup, fill and drain).
constexpr int SHORT_TILE_MAX_N = 3;

// Per tile height: rows, input box rows, threads, consumer threads, point
// pairs per consumer thread, bytes of a ring stage.
struct Variant { int ty, byi, threads, consumers, pp, stage_bytes; };
const Variant kVariant[2] = {
    {tiled::TY, tiled::BYI, tiled::THREADS, tiled::CONSUMERS, tiled::PP, tiled::STAGE_BYTES},
    {tiled5::TY, tiled5::BYI, tiled5::THREADS, tiled5::CONSUMERS, tiled5::PP, tiled5::STAGE_BYTES}};
static_assert(tiled::MAX_STAGES == tiled5::MAX_STAGES && tiled::RING_OFF == tiled5::RING_OFF,
              "both tile heights share the barrier area");
// Ring depth: as many stages as the shared memory allows, at most RING_DEPTH
// (measured with 6, 9, 12 and 15 stages: 9 is best or level at every order
// and grid tried; 15 costs 5 % at N = 13..15), at least MIN_RING.
constexpr int RING_DEPTH = 9;
constexpr int MIN_RING = 4;
static_assert(RING_DEPTH <= MAX_STAGES, "the barrier area holds the ring");

}  // namespace

struct TiledPlan {
    TiledGeometry geo;
    std::string err;
    int N = 0;
    void* coef[4] = {nullptr, nullptr, nullptr, nullptr};
    int nclasses = 2;
    int* err_dev = nullptr;
    CUtensorMap maps_in[4], maps_out[4];
    PassTables tab[2];
    void* dev_stages[2] = {nullptr, nullptr};
    void* dev_coef[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [P][K]
    void* dev_fin[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    void* dev_src = nullptr;
    int tiles_x = 0, tiles_y = 0;
    int variant = 0;                      // 0: 10-row tiles, 1: 5-row tiles
    int sms = 1;
    int ctas_per_sm = 1;                  // resident CTAs per SM the tables allow (<= the variant's)
    int smem_bytes[2] = {0, 0};
    int nring[2] = {0, 0};                // ring stages per parity
    Params prm[2][2];                     // [P][which]
    bool ready = false;
    // temporally fused step
    bool fused = false;
    void* base1[4] = {nullptr, nullptr, nullptr, nullptr};   // the second buffer set
    fused::FusedParams fprm[2];           // [dir]: 0 set 0 -> set 1, 1 set 1 -> set 0
    void* dev_odep = nullptr;
    int fsmem = 0;
    int ftiles_x = 0, ftiles_y = 0;
    bool fready = false;
};

namespace {

void free_tables(TiledPlan* pl) {
    for (int P = 0; P < 2; ++P) {
        if (pl->dev_stages[P]) cudaFree(pl->dev_stages[P]);
        pl->dev_stages[P] = nullptr;
        for (int K = 0; K < 2; ++K) {
            if (pl->dev_coef[P][K]) cudaFree(pl->dev_coef[P][K]);
            if (pl->dev_fin[P][K]) cudaFree(pl->dev_fin[P][K]);
            pl->dev_coef[P][K] = pl->dev_fin[P][K] = nullptr;
        }
    }
    if (pl->dev_src) cudaFree(pl->dev_src);
    pl->dev_src = nullptr;
    if (pl->dev_odep) cudaFree(pl->dev_odep);
    pl->dev_odep = nullptr;
    pl->fready = false;
}

template <class V>
bool upload(void** dst, const std::vector<V>& v) {
    size_t bytes = std::max<size_t>(1, v.size()) * sizeof(V);
    if (dev_alloc(dst, bytes) != cudaSuccess) return false;
    if (!v.empty() && cudaMemcpy(*dst, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice) != cudaSuccess) return false;
    return true;
}

// Walk the consumer loop of pass P and emit its tables.
bool build_pass(TiledPlan* pl, const SystemMatrices& sys, const std::vector<int>& comp_class,
                const std::vector<char>& frozen, int P, double dx, double dy, PassTables& t, std::string& err) {
    const int N = pl->N, n = sys.ncomp;
    t = PassTables();
    // a frozen top order has no finalising stages at all (no data, no work)
    bool top_frozen = true;
    for (int j = 0; j < n; ++j)
        if (sys.moms[j].l == N && !frozen[j]) top_frozen = false;
    t.top = top_frozen ? N - 1 : N;
    const int gin[2] = {P == 1 ? 0 : 1, P == 1 ? 3 : 2};
    const int gout[2] = {P == 1 ? 1 : 0, P == 1 ? 2 : 3};
    auto local_of = [&](int L, int q, int imag, int grid_expected, int& local) -> bool {
        const int j = comp_index(L, L - 2 * q, imag);
        const Moment& m = sys.moms[j];
        if (m.l != L || m.m != L - 2 * q || (int)m.imag != imag || m.grid != grid_expected) return false;
        local = m.local;
        return true;
    };
    long covered = 0;
    auto coef_of = [&](const std::vector<double>& M, int L, int q, int imag, int k, double h) -> float {
        if (!exists(N, L, q, imag)) return 0.f;
        const int j = comp_index(L, L - 2 * q, imag);
        const double v = M[(size_t)j * n + k];
        if (v != 0.0) ++covered;
        return (float)(-v / h);
    };
    int4 cur = make_int4(-1, -1, -1, -1);
    auto emit_input = [&](int lp, int q, int imag) -> bool {
        int local;
        if (!local_of(lp, q, imag, gin[imag], local)) return false;
        if (imag) cur.y = local; else cur.x = local;
        const int k = comp_index(lp, lp - 2 * q, imag);
        // targets Pm (lp-1, q-1), P0 (lp-1, q), N0 (lp+1, q), Np (lp+1, q+1)
        const int TL[4] = {lp - 1, lp - 1, lp + 1, lp + 1};
        const int TQ[4] = {q - 1, q, q, q + 1};
        float row[16];
        for (int s = 0; s < 4; ++s) {
            row[2 * s] = row[2 * s + 1] = coef_of(sys.Mx, TL[s], TQ[s], imag, k, dx);          // same kind, Mx
            row[8 + 2 * s] = row[8 + 2 * s + 1] = coef_of(sys.My, TL[s], TQ[s], 1 - imag, k, dy);  // other kind, My
        }
        t.coef.insert(t.coef.end(), row, row + 16);
        ++t.nin;
        return true;
    };
    auto emit_fin = [&](int L, int q, int imag) -> bool {
        int local;
        if (!local_of(L, q, imag, gout[imag], local)) return false;
        const int j = comp_index(L, L - 2 * q, imag);
        // a frozen output is not finalised: its old value is not loaded either
        if (!frozen[j]) { if (imag) cur.w = local; else cur.z = local; }
        t.fin.push_back(make_int2(local, comp_class[j]));
        t.fin_comp.push_back(j);
        return true;
    };
    // a finalising stage carries entries for both kinds; absent I gets a placeholder
    auto emit_fin_pair = [&](int L, int q) -> bool {
        if (!emit_fin(L, q, 0)) return false;
        if (has_imag(L, q)) return emit_fin(L, q, 1);
        t.fin.push_back(make_int2(-1, 0));
        t.fin_comp.push_back(-1);
        return true;
    };
    // a q step carries coefficient rows for both kinds; absent I gets zeros
    auto emit_input_pair = [&](int lp, int q) -> bool {
        if (!emit_input(lp, q, 0)) return false;
        if (has_imag(lp, q)) return emit_input(lp, q, 1);
        t.coef.insert(t.coef.end(), 16, 0.f);
        return true;
    };
    auto close_stage = [&]() {
        t.stages.push_back(cur);
        cur = make_int4(-1, -1, -1, -1);
    };
    // the stages of the consumer loop (see k_tiled_pass)
    const int first = 1 - P;
    int last_in = first;
    bool ok = true;
    for (int lp = first; lp <= N && ok; lp += 2) {
        last_in = lp;
        const int nq = nq_of(lp), nqp = nq_of(lp - 1);
        for (int q = 0; q < nq && ok; ++q) {
            ok = ok && emit_input_pair(lp, q);
            if (q >= 1 && q - 1 < nqp) ok = ok && emit_fin_pair(lp - 1, q - 1);
            close_stage();
        }
        if (ok && nq - 1 < nqp) {
            ok = ok && emit_fin_pair(lp - 1, nq - 1);
            close_stage();
        }
    }
    const int L = last_in + 1;
    if (ok && L <= t.top)
        for (int q = 0; q < nq_of(L) && ok; ++q) {
            ok = ok && emit_fin_pair(L, q);
            close_stage();
        }
    if (!ok) { err = "moment placement differs from the tiled kernel's"; return false; }
    // every component of the output parity is finalised exactly once
    long nout = 0;
    for (int j = 0; j < n; ++j) nout += (sys.moms[j].l % 2 == P && sys.moms[j].l <= t.top);
    long nreal = 0;
    for (int c : t.fin_comp) nreal += c >= 0;
    if (nreal != nout) { err = "tiled schedule does not cover every output"; return false; }
    // every nonzero coupling between the two parities is covered
    long total = 0;
    for (int j = 0; j < n; ++j) {
        if (sys.moms[j].l % 2 != P) continue;
        for (int k = 0; k < n; ++k)
            if (sys.moms[k].l % 2 != P)
                total += (sys.Mx[(size_t)j * n + k] != 0.0) + (sys.My[(size_t)j * n + k] != 0.0);
    }
    if (covered != total) { err = "coupling pattern differs from the tiled kernel's structure"; return false; }
    return true;
}

// Parameters of the fused step, both directions, from the pass tables.
int build_fused(TiledPlan* pl) {
    pl->fready = false;
    if (!pl->fused || !pl->ready) return 0;
    const PassTables& te = pl->tab[0];
    const PassTables& to = pl->tab[1];
    if (te.top != pl->N || to.top != pl->N) { pl->err = "the fused step has no frozen components"; return -8; }
    // odep: the O stage's even inputs are finalised at these E stages
    std::vector<int> fin_at[2];
    for (int k = 0; k < 2; ++k) fin_at[k].assign(pl->geo.K[k == 0 ? 0 : 3] + 1, -1);
    for (size_t s = 0; s < te.stages.size(); ++s) {
        if (te.stages[s].z >= 0) fin_at[0][te.stages[s].z] = (int)s;
        if (te.stages[s].w >= 0) fin_at[1][te.stages[s].w] = (int)s;
    }
    std::vector<int> odep(to.stages.size());
    int run = 0;
    for (size_t k = 0; k < to.stages.size(); ++k) {
        const int4 st = to.stages[k];
        if (st.x >= 0) {
            if (fin_at[0][st.x] < 0) { pl->err = "fused step: an even input is never finalised"; return -8; }
            run = std::max(run, fin_at[0][st.x] + 1);
        }
        if (st.y >= 0) {
            if (fin_at[1][st.y] < 0) { pl->err = "fused step: an even input is never finalised"; return -8; }
            run = std::max(run, fin_at[1][st.y] + 1);
        }
        odep[k] = run;
    }
    if (pl->dev_odep) cudaFree(pl->dev_odep);
    pl->dev_odep = nullptr;
    if (!upload(&pl->dev_odep, odep)) { pl->err = "uploading the fused tables failed"; return -4; }
    // shared memory: barriers, two rings, both machines' tables, odep, partial sums
    auto al16 = [](int v) { return (v + 15) & ~15; };
    int tab = 0;
    int coef_rel[2][2], fin_rel[2][2], stage_rel[2], part_rel[2];
    for (int M = 0; M < 2; ++M) {
        const Params& q = pl->prm[M == 0 ? 0 : 1][1];
        for (int K = 0; K < 2; ++K) {
            coef_rel[M][K] = tab;
            tab = al16(tab + q.nin * 2 * (int)sizeof(float4));
            fin_rel[M][K] = tab;
            tab = al16(tab + q.nfin * (int)sizeof(int2));
        }
        stage_rel[M] = tab;
        tab = al16(tab + q.nstages * (int)sizeof(int4));
    }
    const int odep_rel = tab;
    tab = al16(tab + (int)odep.size() * (int)sizeof(int));
    part_rel[0] = tab;
    tab += nq_of(pl->N) * fused::E_CONS * 8;
    part_rel[1] = tab;
    tab += nq_of(pl->N) * fused::O_CONS * 8;
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int avail = maxsm - fused::RING_OFF - tab;
    int depth = std::min(8, avail / (fused::E_STAGE + fused::O_STAGE));
    if (depth < 3) { pl->err = "the fused step needs more shared memory than the device offers at this order"; return -8; }
    const int ering = fused::RING_OFF, oring = ering + depth * fused::E_STAGE;
    const int tables = oring + depth * fused::O_STAGE;
    pl->fsmem = tables + tab;
    if (cudaFuncSetAttribute(fused::k_fused_step, cudaFuncAttributeMaxDynamicSharedMemorySize, pl->fsmem) != cudaSuccess) {
        pl->err = "cudaFuncSetAttribute (fused step) failed";
        return -4;
    }
    int nxmax = 0, nymax = 0;
    for (int g = 0; g < 4; ++g) { nxmax = std::max(nxmax, pl->geo.nx[g]); nymax = std::max(nymax, pl->geo.ny[g]); }
    pl->ftiles_x = (nxmax + fused::TXO - 1) / fused::TXO;
    pl->ftiles_y = (nymax + fused::TYO - 1) / fused::TYO;
    const int geven[2] = {0, 3}, godd[2] = {1, 2};
    for (int dir = 0; dir < 2; ++dir) {
        void* cur[4];
        void* nxt[4];
        for (int g = 0; g < 4; ++g) {
            cur[g] = dir == 0 ? pl->geo.base[g] : pl->base1[g];
            nxt[g] = dir == 0 ? pl->base1[g] : pl->geo.base[g];
        }
        fused::FusedParams& fp = pl->fprm[dir];
        std::memset(&fp, 0, sizeof(fp));
        const long rows = pl->geo.rows, pitch = pl->geo.pitch;
        bool ok = true;
        for (int k = 0; k < 2; ++k) {
            // E: odd inputs of the current set, old even outputs of the current set
            ok = ok && encode_grid_map(&fp.m[0].maps[k], cur[godd[k]], pitch, rows, pl->geo.K[godd[k]], fused::BXI, fused::BYI);
            ok = ok && encode_grid_map(&fp.m[0].maps[2 + k], cur[geven[k]], pitch, rows, pl->geo.K[geven[k]], fused::BXO, fused::TYE);
            // O: new even inputs of the other set, old odd outputs of the current set
            ok = ok && encode_grid_map(&fp.m[1].maps[k], nxt[geven[k]], pitch, rows, pl->geo.K[geven[k]], fused::BXI, fused::BYI);
            ok = ok && encode_grid_map(&fp.m[1].maps[2 + k], cur[godd[k]], pitch, rows, pl->geo.K[godd[k]], fused::BXO, fused::TYO);
        }
        if (!ok) { pl->err = "cuTensorMapEncodeTiled failed (fused step)"; return -4; }
        for (int M = 0; M < 2; ++M) {
            const int P = M == 0 ? 0 : 1;
            const Params& q = pl->prm[P][1];
            fused::Machine& m = fp.m[M];
            for (int k = 0; k < 2; ++k) {
                const int g = M == 0 ? geven[k] : godd[k];
                m.out[k].base = (float*)nxt[g];
                m.out[k].cstride = pl->geo.cstride[g];
                m.out[k].coef = (const float*)pl->coef[g];
                m.out[k].nx = pl->geo.nx[g];
                m.out[k].ny = pl->geo.ny[g];
                m.coef[k] = q.coef[k];
                m.fin[k] = q.fin[k];
                m.smem_coef_off[k] = tables + coef_rel[M][k];
                m.smem_fin_off[k] = tables + fin_rel[M][k];
            }
            m.nstages = q.nstages;
            m.nin = q.nin;
            m.nfin = q.nfin;
            m.nring = depth;
            m.stages = q.stages;
            m.smem_stage_off = tables + stage_rel[M];
            m.smem_part_off = tables + part_rel[M];
            m.ring_off = M == 0 ? ering : oring;
        }
        fp.odep = (const int*)pl->dev_odep;
        fp.smem_odep_off = tables + odep_rel;
        fp.pitch = pitch;
        fp.p[0] = pl->geo.p[0];
        fp.p[1] = pl->geo.p[1];
        fp.tiles_x = pl->ftiles_x;
        fp.N = pl->N;
        fp.nclasses = pl->nclasses;
        fp.srcs = (const float* const*)pl->dev_src;
        fp.err = pl->err_dev;
    }
    pl->fready = true;
    return 0;
}

}  // namespace

int tiled_schedule(int N, int P, bool frozen_top, double dx, double dy, std::vector<int>& stages,
                   std::vector<float>& coef, std::vector<int>& fin, std::string& err) {
    if (N < 1 || N > MAXN || (P != 0 && P != 1)) { err = "schedule needs 1 <= N <= 63 and parity 0 or 1"; return -1; }
    SystemMatrices sys;
    if (!build_system(0, N, sys, err)) return -1;
    TiledPlan plan;
    plan.N = N;
    std::vector<int> cls(sys.ncomp, 0);
    std::vector<char> frozen(sys.ncomp, 0);
    for (int j = 0; j < sys.ncomp; ++j) frozen[j] = frozen_top && sys.moms[j].l == N;
    PassTables t;
    if (!build_pass(&plan, sys, cls, frozen, P, dx, dy, t, err)) return -8;
    // local indices of the stage slots back to global components
    std::vector<int> inv(4 * (sys.ncomp + 1), -1);
    for (int j = 0; j < sys.ncomp; ++j) inv[sys.moms[j].grid * (sys.ncomp + 1) + sys.moms[j].local] = j;
    const int grid_of_slot[4] = {P == 1 ? 0 : 1, P == 1 ? 3 : 2, P == 1 ? 1 : 0, P == 1 ? 2 : 3};
    stages.clear();
    for (const int4& st : t.stages) {
        const int v[4] = {st.x, st.y, st.z, st.w};
        for (int k = 0; k < 4; ++k) stages.push_back(v[k] < 0 ? -1 : inv[grid_of_slot[k] * (sys.ncomp + 1) + v[k]]);
    }
    coef = t.coef;
    fin = t.fin_comp;
    return 0;
}

bool tiled_supported(int system, int N, int precision) {
    return system == 0 && precision == 1 && N >= 1 && N <= MAXN && encode_fn() != nullptr;
}

int tiled_create(const TiledGeometry& geo, TiledPlan** out) {
    *out = nullptr;
    TiledPlan* pl = new TiledPlan();
    pl->geo = geo;
    pl->N = geo.N;
    *out = pl;
    if (geo.N < 1 || geo.N > MAXN) { pl->err = "tiled kernel supports 1 <= N <= 63"; return -8; }
    pl->variant = geo.variant == 1 ? 1 : 0;
    const Variant& V = kVariant[pl->variant];
    for (int g = 0; g < 4; ++g) {
        if (!encode_grid_map(&pl->maps_in[g], geo.base[g], geo.pitch, geo.rows, geo.K[g], BX, V.byi) ||
            !encode_grid_map(&pl->maps_out[g], geo.base[g], geo.pitch, geo.rows, geo.K[g], TX, V.ty)) {
            pl->err = "cuTensorMapEncodeTiled failed";
            return -4;
        }
    }
    int nxmax = 0, nymax = 0;
    for (int g = 0; g < 4; ++g) { nxmax = std::max(nxmax, geo.nx[g]); nymax = std::max(nymax, geo.ny[g]); }
    pl->tiles_x = (nxmax + TX - 1) / TX;
    pl->tiles_y = (nymax + V.ty - 1) / V.ty;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&pl->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || pl->sms < 1) pl->sms = 1;
    }
    if (dev_alloc(&pl->err_dev, sizeof(int)) != cudaSuccess || cudaMemset(pl->err_dev, 0, sizeof(int)) != cudaSuccess) {
        pl->err = "cudaMalloc error flag failed";
        return -4;
    }
    return 0;
}

int tiled_update(TiledPlan* pl, const SystemMatrices& sys, const std::vector<int>& comp_class,
                 const std::vector<int>& src_slot, const std::vector<void*>& src_dev,
                 const std::vector<char>& frozen, double dx, double dy) {
    free_tables(pl);
    pl->ready = false;
    {
        std::vector<const float*> sp(src_dev.size());
        for (size_t i = 0; i < src_dev.size(); ++i) sp[i] = (const float*)src_dev[i];
        if (!upload(&pl->dev_src, sp)) { pl->err = "uploading the source table failed"; return -4; }
    }
    const int gin[2][2] = {{1, 2}, {0, 3}};
    const int gout[2][2] = {{0, 3}, {1, 2}};
    for (int P = 0; P < 2; ++P) {
        PassTables& t = pl->tab[P];
        if (!build_pass(pl, sys, comp_class, frozen, P, dx, dy, t, pl->err)) return -8;
        // per output kind K: coefficient rows (x part of the kind-K input,
        // y part of the other input) and finalise entries (offset, source slot)
        // (each value once: the kernel pairs it for f32x2 itself)
        const size_t nsteps = t.coef.size() / 32;
        std::vector<float> ck[2];
        for (int K = 0; K < 2; ++K) {
            ck[K].resize(nsteps * 8);
            for (size_t k = 0; k < nsteps; ++k) {
                const float* rowK = t.coef.data() + 32 * k + 16 * K;
                const float* rowO = t.coef.data() + 32 * k + 16 * (1 - K);
                for (int q = 0; q < 4; ++q) {
                    ck[K][8 * k + q] = rowK[2 * q];            // Mx of the kind-K input, targets Pm P0 N0 Np
                    ck[K][8 * k + 4 + q] = rowO[8 + 2 * q];    // My of the other input
                }
            }
        }
        std::vector<int2> fk[2];
        for (size_t e = 0; e + 1 < t.fin.size() + 1; e += 2) {
            for (int K = 0; K < 2; ++K) {
                const int comp = t.fin_comp[e + K];
                if (comp < 0 || frozen[comp]) { fk[K].push_back(make_int2(-1, -1)); continue; }
                // the component's element offset in units of 32 (pitch, and so the
                // component stride, is a multiple of 32): 2^36 values per grid
                const int g = gout[P][K];
                const long long off = (long long)t.fin[e + K].x * pl->geo.cstride[g];
                if (pl->geo.cstride[g] % 32 != 0 || off / 32 > 0x7fffffffll) {
                    pl->err = "state too large for the tiled kernel's offsets";
                    return -8;
                }
                fk[K].push_back(make_int2((int)(off / 32), src_slot[comp]));
            }
        }
        for (int K = 0; K < 2; ++K)
            if (!upload(&pl->dev_coef[P][K], ck[K]) || !upload(&pl->dev_fin[P][K], fk[K])) {
                pl->err = "uploading the tiled tables failed";
                return -4;
            }
        if (!upload(&pl->dev_stages[P], t.stages)) {
            pl->err = "uploading the tiled tables failed";
            return -4;
        }
        // shared memory: barriers, ring, coefficient rows, finalise events,
        // partial sums; the ring takes what the variant's CTAs per SM leave,
        // up to RING_DEPTH stages (a deeper ring keeps more loads in flight:
        // 9 stages instead of 6 made the P_39 1024^2 pass 7 % faster)
        const Variant& V = kVariant[pl->variant];
        int tables = 0;
        int coef_rel[2], fin_rel[2];
        for (int K = 0; K < 2; ++K) {
            coef_rel[K] = tables;
            tables += (int)(ck[K].size() * sizeof(float));
            tables = (tables + 15) & ~15;
            fin_rel[K] = tables;
            tables += (int)(fk[K].size() * sizeof(int2));
            tables = (tables + 15) & ~15;
        }
        const int stage_rel = tables;
        tables += (int)(t.stages.size() * sizeof(int4));
        tables = (tables + 15) & ~15;
        const int part_rel = tables;
        tables += nq_of(pl->N) * V.pp * V.consumers * 8;    // pp pairs of partial sums per consumer thread and q
        int dev = 0, maxsm = 0, persm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&persm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        // per-CTA budget: the variant's CTAs per SM (1 KB reserved per CTA),
        // less the batch kernel's static parameter copy; where the tables of
        // a high order do not leave room for the ring, one CTA per SM
        auto ring_for = [&](int minb) {
            const int budget = std::min(maxsm, persm / minb - 1024) - (int)sizeof(Params) - 256;
            return std::min(RING_DEPTH, (budget - RING_OFF - tables) / V.stage_bytes);
        };
        int minb = tiled_ctas_per_sm(pl->variant);
        int nring = ring_for(minb);
        if (nring < MIN_RING && minb > 1) {
            minb = 1;
            nring = ring_for(1);
        }
        if (nring < MIN_RING) { pl->err = "tiled kernel needs more shared memory than the device offers"; return -8; }
        pl->ctas_per_sm = P == 0 ? minb : std::min(pl->ctas_per_sm, minb);
        const int ring_end = RING_OFF + nring * V.stage_bytes;
        const int coef_off[2] = {ring_end + coef_rel[0], ring_end + coef_rel[1]};
        const int fin_off[2] = {ring_end + fin_rel[0], ring_end + fin_rel[1]};
        const int stage_off = ring_end + stage_rel, part_off = ring_end + part_rel;
        pl->smem_bytes[P] = ring_end + tables;
        pl->nring[P] = nring;
        const int need = std::max(pl->smem_bytes[0], pl->smem_bytes[1]);
        const cudaError_t fe = pl->variant
            ? cudaFuncSetAttribute(tiled5::k_tiled_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, need)
            : cudaFuncSetAttribute(tiled::k_tiled_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
        if (fe != cudaSuccess) {
            pl->err = "cudaFuncSetAttribute failed";
            return -4;
        }
        for (int w = 0; w < 2; ++w) {
            Params& prm = pl->prm[P][w];
            std::memset(&prm, 0, sizeof(prm));
            for (int k = 0; k < 2; ++k) {
                prm.maps[k] = pl->maps_in[gin[P][k]];
                prm.maps[2 + k] = pl->maps_out[gout[P][k]];
                const int g = gout[P][k];
                prm.out[k].base = (float*)pl->geo.base[g];
                prm.out[k].cstride = pl->geo.cstride[g];
                prm.out[k].coef = (const float*)pl->coef[g];
                prm.out[k].nx = pl->geo.nx[g];
                prm.out[k].ny = pl->geo.ny[g];
            }
            prm.pitch = pl->geo.pitch;
            prm.p[0] = pl->geo.p[0];
            prm.p[1] = pl->geo.p[1];
            prm.tiles_x = pl->tiles_x;
            prm.N = pl->N;
            prm.P = P;
            prm.which = w;
            prm.nclasses = pl->nclasses;
            prm.nstages = (int)t.stages.size();
            prm.nin = (int)nsteps;
            prm.nfin = (int)fk[0].size();
            prm.nring = nring;
            prm.top = t.top;
            prm.stages = (const int4*)pl->dev_stages[P];
            for (int K = 0; K < 2; ++K) {
                prm.coef[K] = (const float4*)pl->dev_coef[P][K];
                prm.fin[K] = (const int2*)pl->dev_fin[P][K];
                prm.smem_coef_off[K] = coef_off[K];
                prm.smem_fin_off[K] = fin_off[K];
            }
            prm.srcs = (const float* const*)pl->dev_src;
            prm.err = pl->err_dev;
            prm.smem_part_off = part_off;
            prm.smem_stage_off = stage_off;
            for (int K = 0; K < 2; ++K) {
                int slot = -1;
                bool one = true;
                for (const int2& f : fk[K])
                    if (f.y >= 0) {
                        if (slot >= 0 && f.y != slot) one = false;
                        slot = f.y;
                    }
                prm.pf_src[K] = slot >= 0 && one ? (const float*)src_dev[slot] : nullptr;
            }
        }
    }
    pl->ready = true;
    return build_fused(pl);
}

void tiled_set_coef(TiledPlan* pl, int g, void* coef, int nclasses) {
    if (!pl) return;
    pl->coef[g] = coef;
    pl->nclasses = nclasses;
    for (int P = 0; P < 2; ++P)
        for (int w = 0; w < 2; ++w) {
            Params& prm = pl->prm[P][w];
            prm.nclasses = nclasses;
            for (int k = 0; k < 2; ++k) {
                const int gout = P == 1 ? (k == 0 ? 1 : 2) : (k == 0 ? 0 : 3);
                if (gout == g) prm.out[k].coef = (const float*)coef;
            }
        }
    for (int dir = 0; dir < 2; ++dir) {
        pl->fprm[dir].nclasses = nclasses;
        for (int M = 0; M < 2; ++M)
            for (int k = 0; k < 2; ++k) {
                const int gout = M == 0 ? (k == 0 ? 0 : 3) : (k == 0 ? 1 : 2);
                if (gout == g) pl->fprm[dir].m[M].out[k].coef = (const float*)coef;
            }
    }
}

int tiled_fused_setup(TiledPlan* pl, void* const base1[4]) {
    if (!pl) return -7;
    if (pl->variant != 0 && pl->variant != 1) return -8;
    for (int g = 0; g < 4; ++g) pl->base1[g] = base1[g];
    pl->fused = true;
    return pl->ready ? build_fused(pl) : 0;
}

bool tiled_fused_ready(TiledPlan* pl) { return pl && pl->fused && pl->fready; }

int tiled_fused_step(TiledPlan* pl, int dir, void* stream) {
    if (!pl || !pl->fready) { if (pl) pl->err = "fused step not prepared"; return -7; }
    const int ntiles = pl->ftiles_x * pl->ftiles_y;
    if (ntiles <= 0) return 0;
    const int grid = std::min(ntiles, pl->sms);
    if ((long long)((ntiles + grid - 1) / grid) * pl->fprm[dir].m[0].nstages > 0x7fffffffll) {
        pl->err = "too many pipeline stages per CTA for the fused step";
        return -8;
    }
    fused::k_fused_step<<<grid, fused::THREADS, pl->fsmem, (cudaStream_t)stream>>>(pl->fprm[dir & 1], ntiles);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        pl->err = std::string("fused step launch: ") + cudaGetErrorString(e);
        return -4;
    }
    return 0;
}

// Pipeline stages per CTA below which a pass overlaps its kernel boundaries
// (programmatic dependent launch): 512^2 passes gain 3-5 us each, while the
// 1 ms passes of P_39 at 1024^2 lost about 1 % with the early-launched
// dependents resident beside them.
constexpr long long OVERLAP_MAX_STAGES = 1000;

bool tiled_overlap(TiledPlan* pl, bool odd) {
    if (!pl || !pl->ready) return false;
    const int ntiles = pl->tiles_x * pl->tiles_y;
    const int grid = std::max(1, std::min(ntiles, pl->sms * pl->ctas_per_sm));
    return (long long)((ntiles + grid - 1) / grid) * pl->prm[odd ? 1 : 0][0].nstages < OVERLAP_MAX_STAGES;
}

int tiled_pass(TiledPlan* pl, bool odd, int which, void* stream) {
    if (!pl->ready) { pl->err = "tiled tables not built"; return -7; }
    const int P = odd ? 1 : 0;
    const int ntiles = pl->tiles_x * pl->tiles_y;
    if (ntiles <= 0) return 0;
    // persistent grid: every resident CTA slot, at most one per tile
    const int grid = std::min(ntiles, pl->sms * pl->ctas_per_sm);
    if ((long long)((ntiles + grid - 1) / grid) * pl->prm[P][which].nstages > 0x7fffffffll) {
        pl->err = "too many pipeline stages per CTA for the tiled kernel";
        return -8;
    }
    // short passes: programmatic dependent launch, the CTAs stage their
    // tables while the previous kernel of the stream finishes
    const bool pdl = tiled_overlap(pl, odd);
    cudaError_t e;
    if (pl->variant) {
        tiled5::Params q;
        std::memcpy(&q, &pl->prm[P][which], sizeof(q));
        e = launch_pdl(tiled5::k_tiled_pass, dim3(grid), dim3(tiled5::THREADS), (size_t)pl->smem_bytes[P],
                       (cudaStream_t)stream, pdl, q, ntiles);
    } else {
        e = launch_pdl(tiled::k_tiled_pass, dim3(grid), dim3(tiled::THREADS), (size_t)pl->smem_bytes[P],
                       (cudaStream_t)stream, pdl, pl->prm[P][which], ntiles);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        pl->err = std::string("tiled pass launch: ") + cudaGetErrorString(e);
        return -4;
    }
    return 0;
}

int tiled_poll(TiledPlan* pl, void* stream) {
    int flag = 0;
    if (cudaMemcpyAsync(&flag, pl->err_dev, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        pl->err = "reading the tiled kernel's error flag failed";
        return -4;
    }
    if (flag) {
        pl->err = "a bounded wait in the tiled kernel gave up";
        cudaMemsetAsync(pl->err_dev, 0, sizeof(int), (cudaStream_t)stream);
        return -6;
    }
    return 0;
}

const char* tiled_error(TiledPlan* p) { return p ? p->err.c_str() : "tiled kernel unavailable"; }

size_t tiled_params_bytes() { return sizeof(Params); }

int tiled_export_params(TiledPlan* pl, void* host4) {
    if (!pl || !pl->ready) return -7;
    Params* d = static_cast<Params*>(host4);
    for (int P = 0; P < 2; ++P)
        for (int w = 0; w < 2; ++w) d[2 * P + w] = pl->prm[P][w];
    return 0;
}

int tiled_smem_bytes(TiledPlan* pl, int P) { return pl ? pl->smem_bytes[P] : 0; }

void tiled_tile_grid(TiledPlan* pl, int* tx, int* ty) {
    *tx = pl ? pl->tiles_x : 0;
    *ty = pl ? pl->tiles_y : 0;
}

int tiled_stage_count(TiledPlan* pl, int P) { return pl ? (int)pl->tab[P].stages.size() : 0; }

int tiled_variant(TiledPlan* pl) { return pl ? pl->variant : 0; }

namespace {
// One CTA waits, through the passes' own bounded wait, for the phase of an
// mbarrier that nothing arrives at: the wait must give up and raise the flag.
__global__ void k_wait_selftest(int* err, int* result) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) *result = wait_bounded(&bar, 0, &abort_flag, err) ? 1 : 0;
}
}  // namespace

int tiled_wait_selftest(int* gave_up) {
    int *d = nullptr;
    if (dev_alloc(&d, 2 * sizeof(int)) != cudaSuccess) return -4;
    int h[2] = {0, -1};
    cudaError_t e = cudaMemcpy(d, h, 2 * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>(d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h, d, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return -4;
    *gave_up = (h[0] == 1 && h[1] == 0) ? 1 : 0;
    return 0;
}

int tiled_default_variant(int N) { return N <= SHORT_TILE_MAX_N ? 1 : 0; }

int tiled_ctas_per_sm(int variant) { return variant ? tiled5::MINB : tiled::MINB; }

int tiled_batch_prepare(int smem_bytes, int variant) {
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (smem_bytes + (int)sizeof(Params) > maxsm) return -8;
    const cudaError_t e = variant
        ? cudaFuncSetAttribute(tiled5::k_tiled_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes)
        : cudaFuncSetAttribute(tiled::k_tiled_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    return e == cudaSuccess ? 0 : -4;
}

int tiled_batch_pass(const void* params, const void* items, const int* off, int P, int which, int grid,
                     int smem_bytes, int variant, void* stream) {
    if (grid <= 0) return 0;
    if (variant)
        tiled5::k_tiled_batch<<<grid, tiled5::THREADS, smem_bytes, (cudaStream_t)stream>>>(
            static_cast<const tiled5::Params*>(params), static_cast<const int4*>(items), off, P, which);
    else
        tiled::k_tiled_batch<<<grid, tiled::THREADS, smem_bytes, (cudaStream_t)stream>>>(
            static_cast<const tiled::Params*>(params), static_cast<const int4*>(items), off, P, which);
    return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

void tiled_destroy(TiledPlan* p) {
    if (!p) return;
    free_tables(p);
    if (p->err_dev) cudaFree(p->err_dev);
    delete p;
}

}  // namespace starmap
