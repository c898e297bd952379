// Cell features of the learned closure, shared by the training sampler,
// the mma.sync closure path and the fused tcgen05 closure kernel (so all
// three see bit-identical inputs).
#pragma once
#include <cuda_runtime.h>

#include <utility>

#include "internal.h"
#include "mlp.h"

namespace starmap {
namespace mlp {

constexpr float EMPTY = 1e-30f;    // largest moment magnitude of an empty cell

// Offsets (elements from point (0, 0) of a component) of the stencil of
// cell (ix, iy) on each grid type: the cell itself (G11), the nodes west /
// east of it (G21), south / north (G12) and the four corners (G22).  Node i
// of an axis lies between cells i + p - 1 and i + p; node -1 of a periodic
// axis is node n - 1, indexed directly (the corner boundary copies of a
// grid are not maintained).
struct Stencil {
    long c, w, e, s, n, sw, se, nw, ne;
};

__device__ __forceinline__ Stencil stencil(int ix, int iy, int nx, int ny, int px, int py, long P) {
    const int xw = ix - px < 0 ? nx - 1 : ix - px, xe = ix - px + 1;
    const int ys = iy - py < 0 ? ny - 1 : iy - py, yn = iy - py + 1;
    const long rc = (long)(iy + 1) * P, rs = (long)(ys + 1) * P, rn = (long)(yn + 1) * P;
    return Stencil{rc + ix, rc + xw, rc + xe, rs + ix, rn + ix, rs + xw, rs + xe, rn + xw, rn + xe};
}

// Value of a component on grid G averaged to the cell centre: the point
// itself, the mean of two nodes, or of four.
template <class T, int G>
__device__ __forceinline__ float centre(const T* c, const Stencil& o) {
    if constexpr (G == 0) return (float)c[o.c];
    else if constexpr (G == 1) return 0.5f * ((float)c[o.w] + (float)c[o.e]);
    else if constexpr (G == 2) return 0.5f * ((float)c[o.s] + (float)c[o.n]);
    else return 0.25f * (((float)c[o.sw] + (float)c[o.se]) + ((float)c[o.nw] + (float)c[o.ne]));
}

template <class T, int... J>
__device__ __forceinline__ void gather(const T* const* colp, const Stencil& o, float* f, std::integer_sequence<int, J...>) {
    ((f[J] = centre<T, grid_of(J)>(colp[J], o)), ...);
}
template <class T, int... J>
__device__ __forceinline__ void gather8(const T* const* colp, const Stencil& o, float* f, std::integer_sequence<int, J...>) {
    ((f[J] = centre<T, grid_of(NMOM + J)>(colp[NMOM + J], o)), ...);
}

// The 36 moment features of a cell (order <= 7 averaged to the centre and
// divided by their RMS s), s and 1/s.  A cell whose largest moment
// magnitude is at most EMPTY counts as empty: features 0, s = 0, 1/s = 0.
// Otherwise the RMS is formed relative to the largest magnitude, so that
// squares of tiny far-field values do not underflow in FP32.
template <class T>
__device__ __forceinline__ void features36(const T* const* colp, const Stencil& o, bool ok, float (&f)[NMOM],
                                           float& scale, float& inv) {
    gather<T>(colp, o, f, std::make_integer_sequence<int, NMOM>{});
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < NMOM; ++j) {
        f[j] = ok ? f[j] : 0.f;
        mx = fmaxf(mx, fabsf(f[j]));
    }
    scale = 0.f;
    inv = 0.f;
    if (mx > EMPTY) {
        const float im = 1.f / mx;
        float ss = 0.f;
#pragma unroll
        for (int j = 0; j < NMOM; ++j) ss += (f[j] * im) * (f[j] * im);
        scale = mx * sqrtf(ss / (float)NMOM);
        inv = 1.f / scale;
    }
#pragma unroll
    for (int j = 0; j < NMOM; ++j) f[j] *= inv;
}

}  // namespace mlp
}  // namespace starmap
