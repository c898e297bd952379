// Internal device-side data structures of the StaRMAP stepper.
//
// Memory layout of the state (one allocation per grid g = G11, G21, G12, G22):
//   component k, point (x, y), -1 <= x <= nx_g, -1 <= y <= ny_g, lives at
//     base_g + k*cstride + (y + 1)*pitch + x
//   where base_g is 128-byte aligned, pitch is a multiple of 32 elements and
//   pitch >= nxmax + 6.  The ghost column x = -1 therefore sits in the last
//   padding element of the previous memory row, and x = nx_g in the padding
//   of the same row; the ghost rows are memory rows 0 and ny_g + 1.  A pad of
//   LEAD elements precedes base_g so that x = -1 of the first row is valid.
// Boundary conditions (section 4.2) live entirely in the ghost cells: after
// every pass the kernel that wrote a boundary point also writes its copies
//   periodic:                 ghost -1 <- u(n-1), ghost n <- u(0)
//   extrapolation, cell axis: ghost -1 <- u(0),   ghost n <- u(n-1)
//   extrapolation, node axis: none (the n+1 nodes are never read outside)
// so that every half-grid difference (eq. central_differences) reads two
// plain neighbours.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdint>

namespace starmap {

// Every device allocation of the library goes through dev_alloc, so that a
// test can make the n-th following one fail (starmap_debug_fail_allocation)
// and check that each error path returns a status and leaves the process
// usable.  The countdown is process-wide.
std::atomic<int>& alloc_fail_countdown();
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
    std::atomic<int>& c = alloc_fail_countdown();
    int n = c.load();
    while (n > 0 && !c.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(reinterpret_cast<void**>(p), bytes);
}

constexpr int LEAD = 32;          // elements before base_g
constexpr int MAXC = 4;           // couplings per direction per row (Lemma 2)

template <class T>
struct GridDev {
    T* base = nullptr;            // point (0, 0) of component 0
    long cstride = 0;             // elements between components
    int nx = 0, ny = 0, K = 0;    // points and components of this grid
    T* coef = nullptr;            // decay coefficients [cls][4][ny][nx]
};

// One output component of the gather pass.
struct GatherOut {
    int grid, local, cls, src;
    int nxt, nyt;
    int xin[MAXC], yin[MAXC];
};
template <class T>
struct GatherCoef { T cx[MAXC], cy[MAXC]; };

template <class T>
struct GatherArgs {
    GridDev<T> g[4];
    long pitch;
    int p[2];                     // periodicity flags p_x, p_y
    int out_grid;                 // grid updated by this launch
    int begin, end;               // range of output components in outs[]
    int which;                    // 0: half-step coefficients, 1: full step
    const GatherOut* outs;
    const GatherCoef<T>* coefs;
    T* const* src;                // source arrays [ny][nx] by slot
};

template <class T>
struct GhostArgs {
    GridDev<T> g;
    long pitch;
    int grid;                     // grid number (its x / y type)
    int p[2];
    int kbegin, kend;             // components to refresh
};

// Boundary copies of every component of the two output grids of a pass.
template <class T>
struct GhostPassArgs {
    GridDev<T> g[2];
    int grid[2];                  // grid numbers (their x / y type)
    long pitch;
    int p[2];
};

// Boundary copies of one FP32 component, one entry of a batched refresh
// (comp points at the component's first interior value, as GridDev::base).
struct GhostJob {
    float* comp;
    long pitch;
    int nx, ny;
    int grid;                     // grid number (its x / y type)
    int px, py;                   // periodic in x / y
    int pad;
};

template <class T>
struct ReduceArgs {
    GridDev<T> g[4];
    long pitch;
    double cell;                  // dx * dy
    int row0 = 1;                 // memory row of y = 0 counted from base (1: ghost row first)
};

// launchers (kernels_gather.cu)
template <class T> int launch_gather_pass(const GatherArgs<T>& a, void* stream);
template <class T> int launch_fill_ghosts(const GhostArgs<T>& a, void* stream);
// overlap: programmatic dependent launch (after a short tiled pass)
template <class T> int launch_fill_ghosts_pass(const GhostPassArgs<T>& a, void* stream, bool overlap);
int launch_fill_ghosts_jobs(const GhostJob* jobs, int njobs, void* stream);
template <class T> int launch_reduce(const ReduceArgs<T>& a, double* partials, int nblocks,
                                     double* result, void* stream);
template <class T> int launch_axpby(T* out, const T* x, const T* y, double alpha, double beta,
                                    size_t n, void* stream);

}  // namespace starmap
