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
};

bool tiled_supported(int system, int N, int precision);
int tiled_create(const TiledGeometry& geo, TiledPlan** out);
// frozen[j] != 0: component j is read but never written (closure moments)
int tiled_update(TiledPlan* plan, const SystemMatrices& sys, const std::vector<int>& comp_class,
                 const std::vector<int>& src_slot, const std::vector<void*>& src_dev,
                 const std::vector<char>& frozen, double dx, double dy);
void tiled_set_coef(TiledPlan* plan, int g, void* coef, int nclasses);
int tiled_pass(TiledPlan* plan, bool odd, int which, void* stream);
// Read and clear the bounded-wait failure flag (synchronises the stream).
int tiled_poll(TiledPlan* plan, void* stream);
const char* tiled_error(TiledPlan* plan);
void tiled_destroy(TiledPlan* plan);

}  // namespace starmap
