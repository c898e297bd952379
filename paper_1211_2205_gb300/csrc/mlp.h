// Internal interface of the learned order-8 closure (network kernels and the
// closure evaluation inside the step).
#pragma once
#include <cuda_bf16.h>

#include <cstddef>

#include "internal.h"

namespace starmap {
namespace mlp {

constexpr int NMOM = 36;          // moments of order <= 7
constexpr int NIN = NMOM + 2;     // + log(1 + sigma_a), log(1 + sigma_s0)
constexpr int HID = 128;
constexpr int NOUT = 9;           // moments of order 8
constexpr int OUTP = 16;          // output rows padded to two 8-wide tiles
constexpr int LDX = 56;           // padded row of X and W1 (bf16 elements)
constexpr int LDH = 136;          // padded row of H1, H2, W2, W3

// Grid of components 0..44 of P_8 in the real ordering of section 3 (per
// order l: R_l^l, I_l^l, R_l^(l-2), ..., R_l^0): R with even l on G11 (0),
// R with odd l on G21 (1), I with odd l on G12 (2), I with even l on G22
// (3), as the placement of section 4.1 puts them.  The closure kernels are
// unrolled over this table; the host checks it against its own placement.
constexpr int GRID45[45] = {0, 1, 2, 0, 3, 0, 1, 2, 1, 2, 0, 3, 0, 3, 0, 1, 2, 1, 2, 1, 2, 0, 3,
                            0, 3, 0, 3, 0, 1, 2, 1, 2, 1, 2, 1, 2, 0, 3, 0, 3, 0, 3, 0, 3, 0};
constexpr int grid_of(int j) { return GRID45[j]; }

// FP32 parameter vector: W1[128][38], b1[128], W2[128][128], b2[128], W3[9][128], b3[9]
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + HID * NIN;
constexpr int OFF_W2 = OFF_B1 + HID;
constexpr int OFF_B2 = OFF_W2 + HID * HID;
constexpr int OFF_W3 = OFF_B2 + HID;
constexpr int OFF_B3 = OFF_W3 + NOUT * HID;
constexpr int NPARAM = OFF_B3 + NOUT;        // 22665

// BF16 weights in the padded layout the kernels stage into shared memory.
struct alignas(16) Packed {
    __nv_bfloat16 W1[HID * LDX];
    __nv_bfloat16 W2[HID * LDH];
    __nv_bfloat16 W3[OUTP * LDH];
    float b1[HID], b2[HID], b3[OUTP];
};

template <class T>
struct ClosureArgs {
    GridDev<T> g[4];
    long pitch;
    int p[2];
    int nx, ny;                   // cells (points of G11)
    int2 slot[NMOM + NOUT];       // (grid, local) of components 0..44 of P_8
    const T* col[NMOM + NOUT];    // point (0, 0) of each of those components (kernel parameters:
                                  // the same for every thread, read without a shared-memory table)
    const float* lsa;             // log(1 + sigma_a) at the cell centres [ny][nx]
    const float* lss;             // log(1 + sigma_s0)
};

int pack(const float* params, Packed* P, void* stream);
int forward(const float* X, long M, const Packed* P, float* Y, void* stream);
// Per-CTA partial gradients (and losses) of the mean squared error over the
// B samples idx[0..B) (idx NULL: samples 0..B); part holds
// blocks(B) x (NPARAM + 1) floats, reduced into grad[NPARAM], loss[1].
// engine: ENGINE_MMA_SYNC (mma.sync tiles) or ENGINE_TCGEN05 (tcgen05 tiles;
// err: device flag raised by a bounded wait).
int loss_grad(const float* X, const float* T, const int* idx, long B, const Packed* P, float* part, float* grad,
              float* loss, int engine, int* err, void* stream);
long grad_blocks(long B);
int adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float eps, long step,
         void* stream);
// Xn = X with N(0, sigma^2) noise on the first `cols` of the NIN inputs of
// each of the M rows (counter-based: the same seed gives the same noise).
int perturb(const float* X, float* Xn, long M, int cols, float sigma, unsigned long long seed, void* stream);
// out[i] = index[perm(i)] (index NULL: perm(i)), perm a keyed pseudo-random
// permutation of [0, count) (count < 2^31); the same seed, the same order.
int shuffle(const int* index, long count, unsigned long long seed, int* out, void* stream);
template <class T> int samples(const ClosureArgs<T>& A, float* X, float* scale, float* tgt, void* stream);
// Closure evaluation (features, network, order-8 moments written to G11 and
// G22); scratch holds closure_scratch_floats(n_x n_y) floats; n_x n_y must
// stay below 2^31 (else -8).  engine: ENGINE_MMA_SYNC or ENGINE_TCGEN05;
// err: device flag raised by a bounded wait of the tcgen05 kernel.
constexpr int ENGINE_MMA_SYNC = 0;
constexpr int ENGINE_TCGEN05 = 1;
long closure_scratch_floats(long M);
template <class T>
int closure(const ClosureArgs<T>& A, const Packed* P, float* scratch, int engine, int* err, void* stream);

// tcgen05 network (mlp_tc.cu)
size_t tc_smem_bytes();
// Self-test of the network kernels' bounded waits (the closure kernel's and
// the forward / training kernels' waits on an mbarrier phase nothing
// completes, a TMEM slot request with every slot held): *gave_up = 1 when
// every wait expired and raised the flag as it must.
int tc_wait_selftest(int* gave_up);
int forward_tc(const float* X, long M, const Packed* P, float* Y, int* err, void* stream);
// per-tile partial loss and gradients of loss_grad on tcgen05 (same layout of part)
int loss_grad_tc(const float* X, const float* T, const int* idx, long B, const Packed* P, float* part, int* err,
                 void* stream);
// fused features + network + order-8 output on tcgen05 (I_8 centre values to
// ctr; scl: n_x n_y floats for the cells' feature scales)
template <class T>
int closure_tc(const ClosureArgs<T>& A, const Packed* P, float* ctr, float* scl, int* err, void* stream);

}  // namespace mlp
}  // namespace starmap
