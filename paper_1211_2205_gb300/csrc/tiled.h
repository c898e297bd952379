// Interface of the tiled (TMA-staged, order-streamed) half-step kernel.
#pragma once
#include <string>
#include <vector>

#include "host_math.h"

namespace starmap {

struct TiledPlan;

struct TiledGeometry {
    void* base[4];
    long cstride[4];
    int nx[4], ny[4], K[4];
    long pitch, rows;
    int p[2];
    int N;
    int variant = 0;                   // tile height: 0 = 10 rows (one CTA per SM), 1 = 5 rows (two per SM)
};

// Tile height the tiled kernel uses for order N when nothing else decides.
int tiled_default_variant(int N);

bool tiled_supported(int system, int N, int precision);
// Host only: the stage list of pass P (parity of its outputs) as global
// components (4 per stage: input R, input I, output R, output I; -1 absent),
// its coefficient rows (16 floats per input, each value twice) and the
// component finalised at each finalising event (-1: absent I).
int tiled_schedule(int N, int P, bool frozen_top, double dx, double dy, std::vector<int>& stages,
                   std::vector<float>& coef, std::vector<int>& fin, std::string& err);
int tiled_create(const TiledGeometry& geo, TiledPlan** out);
// frozen[j] != 0: component j is read but never written (closure moments)
int tiled_update(TiledPlan* plan, const SystemMatrices& sys, const std::vector<int>& comp_class,
                 const std::vector<int>& src_slot, const std::vector<void*>& src_dev,
                 const std::vector<char>& frozen, double dx, double dy);
void tiled_set_coef(TiledPlan* plan, int g, void* coef, int nclasses);
int tiled_pass(TiledPlan* plan, bool odd, int which, void* stream);
// Whether the pass is launched with programmatic dependent launch (so its
// boundary refresh should be too): only for short passes, where the kernel
// boundary is a visible share of the pass.
bool tiled_overlap(TiledPlan* plan, bool odd);
// Temporally fused step: one launch applies the full even update and then
// the full odd update, tile by tile (fused_kernel.cuh), reading one buffer
// set and writing the other.  base1: the second set's grid bases (the same
// layout as the first).  The fused parameters follow every table rebuild.
int tiled_fused_setup(TiledPlan* plan, void* const base1[4]);
bool tiled_fused_ready(TiledPlan* plan);
// dir 0: set 0 -> set 1; dir 1: set 1 -> set 0.  The caller refreshes the
// boundary copies of the written odd grids afterwards.
int tiled_fused_step(TiledPlan* plan, int dir, void* stream);
// Read and clear the bounded-wait failure flag (synchronises the stream).
int tiled_poll(TiledPlan* plan, void* stream);
const char* tiled_error(TiledPlan* plan);
void tiled_destroy(TiledPlan* plan);

// Batched passes over several plans (one persistent launch per pass).
size_t tiled_params_bytes();
// Copy the plan's four pass parameter blocks (index 2 P + which) to host4
// (the passes leave the boundary copies to a separate refresh).
int tiled_export_params(TiledPlan* plan, void* host4);
int tiled_smem_bytes(TiledPlan* plan, int P);
void tiled_tile_grid(TiledPlan* plan, int* tiles_x, int* tiles_y);
int tiled_stage_count(TiledPlan* plan, int P);
int tiled_variant(TiledPlan* plan);
// Self-test of the bounded wait (an mbarrier nothing arrives at); *gave_up = 1
// when the wait expired and raised the flag as it must.
int tiled_wait_selftest(int* gave_up);
// Resident CTAs per SM the kernels of a tile height are built for.
int tiled_ctas_per_sm(int variant);
// Allow the batch kernel of the given tile height smem_bytes of dynamic shared memory.
int tiled_batch_prepare(int smem_bytes, int variant);
// items: device array of int4 (instance, first tile, tile count, stride),
// each the tiles first, first + stride, ... of one instance; CTA b runs
// items off[b] .. off[b + 1] - 1 (off: grid + 1 device ints); params: device array
// of 4 * instances parameter blocks (instance i, parity P, which at
// 4 i + 2 P + which).
int tiled_batch_pass(const void* params, const void* items, const int* off, int P, int which, int grid,
                     int smem_bytes, int variant, void* stream);

}  // namespace starmap
