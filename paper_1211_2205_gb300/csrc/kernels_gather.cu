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
    for (int t = A.begin; t < A.end; ++t) {
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
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < 2 * (nx + ny); r += gridDim.x * blockDim.x) {
        int x, y;
        if (r < nx) { x = r; y = 0; }
        else if (r < 2 * nx) { x = r - nx; y = ny - 1; }
        else if (r < 2 * nx + ny) { x = 0; y = r - 2 * nx; }
        else { x = nx - 1; y = r - 2 * nx - ny; }
        const T v = comp[(long)(y + 1) * A.pitch + x];
        store_point(comp, A.pitch, x, y, nx, ny, xnode, ynode, A.p[0], A.p[1], v);
    }
    if (blockIdx.x == 0 && threadIdx.x < 4) corner_ghost(comp, A.pitch, nx, ny, xnode, ynode, A.p[0], A.p[1], threadIdx.x);
}

// Batched refresh: block b re-stores the boundary points of component
// jobs[b] with their copies.
__global__ void k_fill_ghosts_jobs(const GhostJob* __restrict__ jobs) {
    const GhostJob J = jobs[blockIdx.x];
    const bool xnode = (J.grid & 1) != 0, ynode = (J.grid & 2) != 0;
    const int nx = J.nx, ny = J.ny;
    for (int r = threadIdx.x; r < 2 * (nx + ny); r += blockDim.x) {
        int x, y;
        if (r < nx) { x = r; y = 0; }
        else if (r < 2 * nx) { x = r - nx; y = ny - 1; }
        else if (r < 2 * nx + ny) { x = 0; y = r - 2 * nx; }
        else { x = nx - 1; y = r - 2 * nx - ny; }
        const float v = J.comp[(long)(y + 1) * J.pitch + x];
        store_point(J.comp, J.pitch, x, y, nx, ny, xnode, ynode, J.px, J.py, v);
    }
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

template <class T>
int launch_gather_pass(const GatherArgs<T>& a, void* stream) {
    const GridDev<T>& G = a.g[a.out_grid];
    if (a.end <= a.begin || G.nx == 0 || G.ny == 0) return 0;
    dim3 block(128);
    dim3 grid((G.nx + 127) / 128, G.ny);
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
    const int len = 2 * std::max(a.g[0].nx + a.g[0].ny, a.g[1].nx + a.g[1].ny);
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
