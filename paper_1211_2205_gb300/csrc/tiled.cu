// Tiled half-step kernel (placeholder until implemented).
#include "tiled.h"

namespace starmap {

struct TiledPlan { std::string err; };

bool tiled_supported(int, int, int) { return false; }
int tiled_create(const TiledGeometry&, TiledPlan** out) { *out = nullptr; return -8; }
int tiled_update(TiledPlan*, const SystemMatrices&, const std::vector<int>&, const std::vector<int>&,
                 const std::vector<void*>&, double, double) { return -8; }
void tiled_set_coef(TiledPlan*, int, void*, int) {}
int tiled_pass(TiledPlan*, bool, int, void*) { return -8; }
const char* tiled_error(TiledPlan* p) { return p ? p->err.c_str() : "tiled kernel unavailable"; }
void tiled_destroy(TiledPlan* p) { delete p; }

}  // namespace starmap
