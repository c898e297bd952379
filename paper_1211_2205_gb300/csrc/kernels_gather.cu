// Gather kernel of the half-step pass and small helper kernels.
//
// k_gather_pass updates every output component of one grid at one point per
// thread: W = sum_k cx_k (u_k(right) - u_k(left)) + sum_k cy_k (u_k(up) -
// u_k(down)) with cx = -Mx[j][k]/dx, cy = -My[j][k]/dy (the weighted sparse
// sum of section 5.5 over eq. central_differences), then the exact sub-step
// u <- a u + b (W + q) (eq. sub_step_solution with a = exp(-c tau),
// b = tau E(-c tau), tau = dt/2 for a half-step, dt for the fused even pair
// or a merged odd pair).  It serves FP64 runs, the slab system and any N.
#include <cuda_runtime.h>

#include <algorithm>

#include "internal.h"
#include "pdl.h"

namespace starmap {

namespace {

// Write u at point (x, y) of a component and its boundary copies.
template <class T>
__device__ __forceinline__ void store_point(T* comp, long pitch, int x, int y, int nx, int ny,
                                            bool xnode, bool ynode, int px, int py, T v) {
    comp[(long)(y + 1) * pitch + x] = v;
    int gxa = -2, gxb = -2;
    if (px) { if (x == nx - 1) gxa = -1; if (x == 0) gxb = nx; }
    else if (!xnode) { if (x == 0) gxa = -1; if (x == nx - 1) gxb = nx; }
    if (gxa != -2) comp[(long)(y + 1) * pitch + gxa] = v;
    if (gxb != -2) comp[(long)(y + 1) * pitch + gxb] = v;
    int gya = -2, gyb = -2;
    if (py) { if (y == ny - 1) gya = -1; if (y == 0) gyb = ny; }
    else if (!ynode) { if (y == 0) gya = -1; if (y == ny - 1) gyb = ny; }
    if (gya != -2) comp[(long)(gya + 1) * pitch + x] = v;
    if (gyb != -2) comp[(long)(gyb + 1) * pitch + x] = v;
}

// Corner boundary copy t (0: (-1,-1), 1: (nx,-1), 2: (-1,ny), 3: (nx,ny)):
// where both axes keep a copy on that side, the x rule applied to the y
// copy.  The passes never read corners; the fused step's even update does
// at the points it adds beyond a periodic edge next to a corner.
template <class T>
__device__ __forceinline__ void corner_ghost(T* comp, long pitch, int nx, int ny, bool xnode, bool ynode,
                                             int px, int py, int t) {
    const bool hx = px || !xnode, hy = py || !ynode;
    if (!hx || !hy) return;
    const bool right = t & 1, top = t & 2;
    const int gx = right ? nx : -1, gy = top ? ny : -1;
    const int sx = right ? (px ? 0 : nx - 1) : (px ? nx - 1 : 0);
    const int sy = top ? (py ? 0 : ny - 1) : (py ? ny - 1 : 0);
    comp[(long)(gy + 1) * pitch + gx] = comp[(long)(sy + 1) * pitch + sx];
}

// Boundary copies of one component as independent items.  A column copy
// lands in a 32-byte sector that holds nothing else of use, so the item
// that writes it stores the sector whole (fewer partial stores, which make
// DRAM read the sector first):
//   items [0, ny)                row y's gap [nx, pitch): the sector holding
//                                nx (the interior values in it kept, row y's
//                                right copy at nx, zero padding) and the row's
//                                last sector (row y + 1's left copy at
//                                pitch - 1, zero padding)
//   items [.., + 2 nx)           rows -1 and ny (where the y axis keeps copies)
//   4 items                      single stores: row 0's left copy and the
//                                corners (-1,-1), (nx,-1), (nx,ny); the corner
//                                (-1,ny) is row ny - 1's gap
// Only padding lies between nx and pitch - 1 (pitch >= nx + 6); the copies
// follow the rules of store_point, corners those of corner_ghost.
// (Reading the boundary values costs a 128-byte line each from DRAM: one
// line per row and side is what bounds this kernel.)
__device__ __forceinline__ void store_sector(float* dst, const float (&v)[8]) {
    reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void store_sector(double* dst, const double (&v)[4]) {
    reinterpret_cast<double2*>(dst)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(dst)[1] = make_double2(v[2], v[3]);
}

template <class T>
__host__ __device__ __forceinline__ int ghost_items(int nx, int ny, bool hx, bool hy) {
    return (hx ? ny : 0) + (hy ? 2 * nx : 0) + 4;
}

template <class T>
__device__ __forceinline__ void ghost_item(T* comp, long pitch, int nx, int ny, bool xnode, bool ynode,
                                           int px, int py, int i) {
    constexpr int EPS = 32 / (int)sizeof(T);         // elements per 32-byte sector
    const bool hx = px || !xnode, hy = py || !ynode;
    const int xl = px ? nx - 1 : 0, xr = px ? 0 : nx - 1;          // sources of the left / right copies
    const int ylo = py ? ny - 1 : 0, yhi = py ? 0 : ny - 1;        // sources of rows -1 and ny
    auto at = [&](int x, int y) -> T& { return comp[(long)(y + 1) * pitch + x]; };
    if (hx) {
        if (i < ny) {
            const int y = i;
            T* row = &at(0, y);
            const int a0 = nx & ~(EPS - 1), b0 = (int)pitch - EPS;
            T sa[EPS];
#pragma unroll
            for (int e = 0; e < EPS; ++e) {
                const int x = a0 + e;
                sa[e] = x < nx ? row[x] : (x == nx ? row[xr] : T(0));
            }
            // left copy of row y + 1 (for the last row: the corner (-1, ny))
            const T left = y + 1 < ny ? at(xl, y + 1) : (hy ? at(xl, yhi) : T(0));
            if (a0 == b0) {
                sa[EPS - 1] = left;
            } else {
                T sb[EPS];
#pragma unroll
                for (int e = 0; e < EPS; ++e) sb[e] = T(0);
                sb[EPS - 1] = left;
                store_sector(row + b0, sb);
            }
            store_sector(row + a0, sa);
            return;
        }
        i -= ny;
    }
    if (hy) {
        if (i < nx) { at(i, -1) = at(i, ylo); return; }
        if (i < 2 * nx) { at(i - nx, ny) = at(i - nx, yhi); return; }
        i -= 2 * nx;
    }
    if (i == 0) { if (hx) at(-1, 0) = at(xl, 0); return; }
    if (!hx || !hy) return;
    if (i == 1) at(-1, -1) = at(xl, ylo);
    else if (i == 2) at(nx, -1) = at(xr, ylo);
    else if (i == 3) at(nx, ny) = at(xr, yhi);
}

template <class T>
__global__ void k_gather_pass(const GatherArgs<T> A) {
    const int g = A.out_grid;
    const GridDev<T>& G = A.g[g];
    const int ix = blockIdx.x * blockDim.x + threadIdx.x;
    const int iy = blockIdx.y;
    if (ix >= G.nx || iy >= G.ny) return;
    const bool xnode = (g & 1) != 0, ynode = (g & 2) != 0;
    const int xg = g ^ 1, yg = g ^ 2;                  // partner grids
    const long pitch = A.pitch;
    // right / upper neighbour index in the partner grid (eq. central_differences)
    const int xr = ix + (xnode ? A.p[0] : 1 - A.p[0]);
    const int yu = iy + (ynode ? A.p[1] : 1 - A.p[1]);
    const long o_r = (long)(iy + 1) * pitch + xr;
    const long o_u = (long)(yu + 1) * pitch + ix;
    const long o_self = (long)(iy + 1) * pitch + ix;
    const long cidx = (long)iy * G.nx + ix;
    const long plane = (long)G.nx * G.ny;
    const T* Xb = A.g[xg].base;
    const T* Yb = A.g[yg].base;
    const long cxs = A.g[xg].cstride, cys = A.g[yg].cstride;
    for (int t = A.begin + (int)blockIdx.z; t < A.end; t += (int)gridDim.z) {
        const GatherOut o = A.outs[t];
        const GatherCoef<T> c = A.coefs[t];
        T w = T(0);
        for (int k = 0; k < o.nxt; ++k) {
            const T* b = Xb + (long)o.xin[k] * cxs;
            w += c.cx[k] * (b[o_r] - b[o_r - 1]);
        }
        for (int k = 0; k < o.nyt; ++k) {
            const T* b = Yb + (long)o.yin[k] * cys;
            w += c.cy[k] * (b[o_u] - b[o_u - pitch]);
        }
        if (o.src >= 0) w += A.src[o.src][cidx];
        const T* cf = G.coef + (long)o.cls * 4 * plane + cidx;
        const T a = cf[(2 * A.which) * plane];
        const T bb = cf[(2 * A.which + 1) * plane];
        T* comp = G.base + (long)o.local * G.cstride;
        const T v = a * comp[o_self] + bb * w;
        store_point(comp, pitch, ix, iy, G.nx, G.ny, xnode, ynode, A.p[0], A.p[1], v);
    }
}

// Refresh the boundary copies of components [kbegin, kend) of one grid.
template <class T>
__global__ void k_fill_ghosts(const GhostArgs<T> A) {
    const GridDev<T>& G = A.g;
    const long per = 2L * G.nx + 2L * G.ny;
    const long total = per * (A.kend - A.kbegin);
    const bool xnode = (A.grid & 1) != 0, ynode = (A.grid & 2) != 0;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int k = A.kbegin + (int)(t / per);
        long r = t % per;
        int x, y;
        if (r < G.nx) { x = (int)r; y = 0; }
        else if (r < 2L * G.nx) { x = (int)(r - G.nx); y = G.ny - 1; }
        else if (r < 2L * G.nx + G.ny) { x = 0; y = (int)(r - 2L * G.nx); }
        else { x = G.nx - 1; y = (int)(r - 2L * G.nx - G.ny); }
        T* comp = G.base + (long)k * G.cstride;
        const T v = comp[(long)(y + 1) * A.pitch + x];
        store_point(comp, A.pitch, x, y, G.nx, G.ny, xnode, ynode, A.p[0], A.p[1], v);
    }
    const long corners = 4L * (A.kend - A.kbegin);
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < corners; t += (long)gridDim.x * blockDim.x)
        corner_ghost(G.base + (long)(A.kbegin + t / 4) * G.cstride, A.pitch, G.nx, G.ny, xnode, ynode, A.p[0], A.p[1],
                     (int)(t % 4));
}

// Boundary copies after a pass whose kernel left them out: blockIdx.y runs
// over the components of both output grids, threads over the four
// boundary lines of the component (rows y = 0 and ny - 1, columns x = 0
// and nx - 1), each point re-stored with its copies (store_point).
template <class T>
__global__ void k_fill_ghosts_pass(const GhostPassArgs<T> A) {
    pdl_trigger();
    pdl_wait();                         // the pass that wrote these components is done
    const int c = blockIdx.y;
    const int which = c < A.g[0].K ? 0 : 1;
    const GridDev<T>& G = A.g[which];
    const int k = which ? c - A.g[0].K : c;
    const bool xnode = (A.grid[which] & 1) != 0, ynode = (A.grid[which] & 2) != 0;
    T* comp = G.base + (long)k * G.cstride;
    const int nx = G.nx, ny = G.ny;
    const int items = ghost_items<T>(nx, ny, A.p[0] || !xnode, A.p[1] || !ynode);
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < items; r += gridDim.x * blockDim.x)
        ghost_item(comp, A.pitch, nx, ny, xnode, ynode, A.p[0], A.p[1], r);
}

// Batched refresh: block b re-stores the boundary points of component
// jobs[b] with their copies.
__global__ void k_fill_ghosts_jobs(const GhostJob* __restrict__ jobs) {
    const GhostJob J = jobs[blockIdx.x];
    const bool xnode = (J.grid & 1) != 0, ynode = (J.grid & 2) != 0;
    const int nx = J.nx, ny = J.ny;
    const int items = ghost_items<float>(nx, ny, J.px || !xnode, J.py || !ynode);
    for (int r = threadIdx.x; r < items; r += blockDim.x)
        ghost_item(J.comp, J.pitch, nx, ny, xnode, ynode, J.px, J.py, r);
}

// Deterministic FP64 reduction: per-block partials (mass, sum of squares,
// non-finite count) over all rows of all grids, then one block sums them in
// a fixed order.
template <class T>
__global__ void k_reduce_partials(const ReduceArgs<T> A, double* partials) {
    __shared__ double sh[3][256];
    double mass = 0.0, sq = 0.0, bad = 0.0;
    long rows_total = 0;
    for (int g = 0; g < 4; ++g) rows_total += (long)A.g[g].K * A.g[g].ny;
    for (long r = blockIdx.x; r < rows_total; r += gridDim.x) {
        long rr = r;
        int g = 0;
        while (rr >= (long)A.g[g].K * A.g[g].ny) { rr -= (long)A.g[g].K * A.g[g].ny; ++g; }
        const GridDev<T>& G = A.g[g];
        const int k = (int)(rr / G.ny), y = (int)(rr % G.ny);
        const T* row = G.base + (long)k * G.cstride + (long)(y + A.row0) * A.pitch;
        for (int x = threadIdx.x; x < G.nx; x += blockDim.x) {
            const double v = (double)row[x];
            if (!isfinite(v)) { bad += 1.0; continue; }
            sq += v * v;
            if (g == 0 && k == 0) mass += v;
        }
    }
    sh[0][threadIdx.x] = mass;
    sh[1][threadIdx.x] = sq;
    sh[2][threadIdx.x] = bad;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) partials[blockIdx.x * 3 + q] = sh[q][0];
}

__global__ void k_reduce_final(const double* partials, int nblocks, double cell, double* out) {
    __shared__ double sh[3][256];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int q = 0; q < 3; ++q) acc[q] += partials[b * 3 + q];
    for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0] * cell;
        out[1] = sqrt(sh[1][0] * cell);
        out[2] = sh[2][0];
    }
}

template <class T>
__global__ void k_axpby(T* out, const T* x, const T* y, double alpha, double beta, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (T)(alpha * (double)x[i] + beta * (double)y[i]);
}

int status_of(cudaError_t e) { return e == cudaSuccess ? 0 : -4; }

}  // namespace

static int sm_count_gather() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    }
    return n;
}

template <class T>
int launch_gather_pass(const GatherArgs<T>& a, void* stream) {
    const GridDev<T>& G = a.g[a.out_grid];
    if (a.end <= a.begin || G.nx == 0 || G.ny == 0) return 0;
    dim3 block(128);
    // one thread per point walks the grid's outputs; on a small grid the
    // outputs are dealt over blockIdx.z as well (output t to slice (t - begin)
    // mod z), so that about two waves of threads fill the GPU
    const long threads = (long)((G.nx + 127) / 128) * 128 * G.ny;
    const long want = 2L * 2048 * sm_count_gather();
    long z = threads >= want ? 1 : (want + threads - 1) / threads;
    if (z > a.end - a.begin) z = a.end - a.begin;
    if (z > 64) z = 64;
    dim3 grid((G.nx + 127) / 128, G.ny, (unsigned)z);
    k_gather_pass<T><<<grid, block, 0, (cudaStream_t)stream>>>(a);
    return status_of(cudaGetLastError());
}

template <class T>
int launch_fill_ghosts(const GhostArgs<T>& a, void* stream) {
    if (a.kend <= a.kbegin || a.g.nx == 0) return 0;
    long total = (2L * a.g.nx + 2L * a.g.ny) * (a.kend - a.kbegin);
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_fill_ghosts<T><<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return status_of(cudaGetLastError());
}

template <class T>
int launch_fill_ghosts_pass(const GhostPassArgs<T>& a, void* stream, bool overlap) {
    const int K = a.g[0].K + a.g[1].K;
    if (K <= 0) return 0;
    const int len = std::max(ghost_items<T>(a.g[0].nx, a.g[0].ny, true, true), ghost_items<T>(a.g[1].nx, a.g[1].ny, true, true));
    const dim3 grid((len + 255) / 256, K);
    const cudaError_t e = launch_pdl(k_fill_ghosts_pass<T>, grid, dim3(256), 0, (cudaStream_t)stream, overlap, a);
    return status_of(e != cudaSuccess ? e : cudaGetLastError());
}

int launch_fill_ghosts_jobs(const GhostJob* jobs, int njobs, void* stream) {
    if (njobs <= 0) return 0;
    k_fill_ghosts_jobs<<<njobs, 256, 0, (cudaStream_t)stream>>>(jobs);
    return status_of(cudaGetLastError());
}

template <class T>
int launch_reduce(const ReduceArgs<T>& a, double* partials, int nblocks, double* result, void* stream) {
    k_reduce_partials<T><<<nblocks, 256, 0, (cudaStream_t)stream>>>(a, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return status_of(e);
    k_reduce_final<<<1, 256, 0, (cudaStream_t)stream>>>(partials, nblocks, a.cell, result);
    return status_of(cudaGetLastError());
}

template <class T>
int launch_axpby(T* out, const T* x, const T* y, double alpha, double beta, size_t n, void* stream) {
    if (n == 0) return 0;
    size_t blocks = (n + 255) / 256;
    if (blocks > 65536) blocks = 65536;
    k_axpby<T><<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out, x, y, alpha, beta, n);
    return status_of(cudaGetLastError());
}

template int launch_gather_pass<float>(const GatherArgs<float>&, void*);
template int launch_gather_pass<double>(const GatherArgs<double>&, void*);
template int launch_fill_ghosts<float>(const GhostArgs<float>&, void*);
template int launch_fill_ghosts<double>(const GhostArgs<double>&, void*);
template int launch_fill_ghosts_pass<float>(const GhostPassArgs<float>&, void*, bool);
template int launch_fill_ghosts_pass<double>(const GhostPassArgs<double>&, void*, bool);
template int launch_reduce<float>(const ReduceArgs<float>&, double*, int, double*, void*);
template int launch_reduce<double>(const ReduceArgs<double>&, double*, int, double*, void*);
template int launch_axpby<float>(float*, const float*, const float*, double, double, size_t, void*);
template int launch_axpby<double>(double*, const double*, const double*, double, double, size_t, void*);

}  // namespace starmap
