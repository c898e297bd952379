// C ABI of the closure network object: FP32 master parameters, Adam state,
// BF16 packed copy, and the scratch of the gradient reduction.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "internal.h"
#include "mlp.h"
#include "../../include/starmap.h"

using namespace starmap;

namespace {
thread_local std::string g_mlp_create_error;
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;
}

struct starmap_mlp_s {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    float* params = nullptr;       // FP32 master parameters
    float* m = nullptr;            // Adam first moment
    float* v = nullptr;            // Adam second moment
    float* grad = nullptr;         // gradient of the last train step
    mlp::Packed* packed = nullptr; // BF16 copy used by the kernels
    float* part = nullptr;         // per-tile partial gradients
    long part_tiles = 0;
    long steps = 0;
    int engine = mlp::ENGINE_MMA_SYNC;
    int* flag = nullptr;           // bounded-wait flag of the tcgen05 network
    std::string err;
};

namespace {

int mfail(starmap_mlp_t* n, int code, const std::string& msg) {
    if (n) n->err = msg; else g_mlp_create_error = msg;
    return code;
}

#define MCK(call, what)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return mfail(net, e_ == cudaErrorMemoryAllocation ? STARMAP_E_NOMEM : STARMAP_E_CUDA, \
                         std::string(what) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

void mrelease(starmap_mlp_t* n) {
    cudaFree(n->params);
    cudaFree(n->m);
    cudaFree(n->v);
    cudaFree(n->grad);
    cudaFree(n->packed);
    cudaFree(n->part);
    cudaFree(n->flag);
    if (n->own_stream && n->stream) cudaStreamDestroy(n->stream);
}

int check_params(starmap_mlp_t* net, const float* params, size_t count) {
    if (!params || count != (size_t)mlp::NPARAM) return mfail(net, STARMAP_E_ARG, "parameters need STARMAP_MLP_PARAMS floats");
    for (size_t i = 0; i < count; ++i)
        if (!std::isfinite(params[i])) return mfail(net, STARMAP_E_NONFINITE, "parameters contain NaN or Inf");
    return STARMAP_OK;
}

int load(starmap_mlp_t* net, const float* params) {
    MCK(cudaMemcpyAsync(net->params, params, (size_t)mlp::NPARAM * sizeof(float), cudaMemcpyHostToDevice, net->stream),
        "upload parameters");
    MCK(cudaMemsetAsync(net->m, 0, (size_t)mlp::NPARAM * sizeof(float), net->stream), "reset optimiser");
    MCK(cudaMemsetAsync(net->v, 0, (size_t)mlp::NPARAM * sizeof(float), net->stream), "reset optimiser");
    if (mlp::pack(net->params, net->packed, net->stream)) MCK(cudaGetLastError(), "pack");
    MCK(cudaStreamSynchronize(net->stream), "load parameters");
    net->steps = 0;
    return STARMAP_OK;
}

int ensure_part(starmap_mlp_t* net, long tiles) {
    if (tiles <= net->part_tiles) return STARMAP_OK;
    if (net->part) {
        MCK(cudaStreamSynchronize(net->stream), "grow scratch");
        cudaFree(net->part);
        net->part = nullptr;
        net->part_tiles = 0;
    }
    MCK(dev_alloc(&net->part, (size_t)tiles * (mlp::NPARAM + 1) * sizeof(float)), "cudaMalloc gradient scratch");
    net->part_tiles = tiles;
    return STARMAP_OK;
}

}  // namespace

extern "C" {

int starmap_mlp_create(const float* params, size_t count, void* cuda_stream, starmap_mlp_t** out) {
    if (!out) return mfail(nullptr, STARMAP_E_ARG, "out is NULL");
    *out = nullptr;
    if (int rc = check_params(nullptr, params, count)) return rc;
    starmap_mlp_t* net = new (std::nothrow) starmap_mlp_t();
    if (!net) return mfail(nullptr, STARMAP_E_NOMEM, "host allocation failed");
    auto bail = [&](int rc) {
        std::string m = net->err;
        mrelease(net);
        delete net;
        g_mlp_create_error = m;
        return rc;
    };
    cudaError_t e;
    if (cuda_stream) {
        net->stream = (cudaStream_t)cuda_stream;
    } else {
        e = cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(mfail(net, STARMAP_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
        net->own_stream = true;
    }
    const size_t pb = (size_t)mlp::NPARAM * sizeof(float);
    float** bufs[4] = {&net->params, &net->m, &net->v, &net->grad};
    for (float** b : bufs) {
        e = dev_alloc(b, pb);
        if (e != cudaSuccess) return bail(mfail(net, STARMAP_E_NOMEM, "cudaMalloc parameters"));
    }
    e = dev_alloc(&net->packed, sizeof(mlp::Packed));
    if (e != cudaSuccess) return bail(mfail(net, STARMAP_E_NOMEM, "cudaMalloc packed weights"));
    e = dev_alloc(&net->flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(net->flag, 0, sizeof(int));
    if (e != cudaSuccess) return bail(mfail(net, STARMAP_E_NOMEM, "cudaMalloc error flag"));
    if (int rc = load(net, params)) return bail(rc);
    *out = net;
    return STARMAP_OK;
}

void starmap_mlp_destroy(starmap_mlp_t* net) {
    if (!net) return;
    if (net->stream) cudaStreamSynchronize(net->stream);
    mrelease(net);
    delete net;
}

const char* starmap_mlp_last_error(const starmap_mlp_t* net) {
    return net ? net->err.c_str() : g_mlp_create_error.c_str();
}

int starmap_mlp_get_params(starmap_mlp_t* net, float* params, size_t count) {
    if (!net) return STARMAP_E_ARG;
    if (!params || count != (size_t)mlp::NPARAM) return mfail(net, STARMAP_E_ARG, "parameters need STARMAP_MLP_PARAMS floats");
    MCK(cudaMemcpyAsync(params, net->params, count * sizeof(float), cudaMemcpyDeviceToHost, net->stream), "download parameters");
    MCK(cudaStreamSynchronize(net->stream), "download parameters");
    return STARMAP_OK;
}

int starmap_mlp_set_params(starmap_mlp_t* net, const float* params, size_t count) {
    if (!net) return STARMAP_E_ARG;
    if (int rc = check_params(net, params, count)) return rc;
    return load(net, params);
}

int starmap_mlp_forward(starmap_mlp_t* net, const float* X, size_t M, float* Y) {
    if (!net) return STARMAP_E_ARG;
    if (M == 0) return STARMAP_OK;
    if (!X || !Y) return mfail(net, STARMAP_E_ARG, "X and Y must be device pointers");
    const int rc = net->engine == mlp::ENGINE_TCGEN05 ? mlp::forward_tc(X, (long)M, net->packed, Y, net->flag, net->stream)
                                                      : mlp::forward(X, (long)M, net->packed, Y, net->stream);
    if (rc) MCK(cudaGetLastError(), "forward");
    return STARMAP_OK;
}

int starmap_mlp_loss_grad(starmap_mlp_t* net, const float* X, const float* T, const int32_t* idx, size_t B,
                          float* grad, float* loss) {
    if (!net) return STARMAP_E_ARG;
    if (B == 0 || !X || !T || !grad) return mfail(net, STARMAP_E_ARG, "loss_grad needs B > 0 and X, T, grad");
    if (int rc = ensure_part(net, mlp::grad_blocks((long)B))) return rc;
    if (mlp::loss_grad(X, T, idx, (long)B, net->packed, net->part, grad, loss, net->engine, net->flag, net->stream))
        MCK(cudaGetLastError(), "loss_grad");
    return STARMAP_OK;
}

int starmap_mlp_train_step(starmap_mlp_t* net, const float* X, const float* T, const int32_t* idx, size_t B, float lr,
                           float* loss) {
    if (!net) return STARMAP_E_ARG;
    if (!(lr > 0.f) || !std::isfinite(lr)) return mfail(net, STARMAP_E_ARG, "learning rate must be positive");
    if (int rc = starmap_mlp_loss_grad(net, X, T, idx, B, net->grad, loss)) return rc;
    net->steps += 1;
    if (mlp::adam(net->params, net->grad, net->m, net->v, mlp::NPARAM, lr, ADAM_B1, ADAM_B2, ADAM_EPS, net->steps,
                  net->stream))
        MCK(cudaGetLastError(), "adam");
    if (mlp::pack(net->params, net->packed, net->stream)) MCK(cudaGetLastError(), "pack");
    return STARMAP_OK;
}

int starmap_mlp_perturb_inputs(starmap_mlp_t* net, const float* X, float* Xn, size_t M, int cols, float sigma,
                               unsigned long long seed) {
    if (!net) return STARMAP_E_ARG;
    if (M == 0) return STARMAP_OK;
    if (!X || !Xn || cols < 0 || cols > mlp::NIN || !(sigma >= 0.f) || !std::isfinite(sigma))
        return mfail(net, STARMAP_E_ARG, "perturb_inputs needs X, Xn, 0 <= cols <= 38 and a finite sigma >= 0");
    if (mlp::perturb(X, Xn, (long)M, cols, sigma, seed, net->stream)) MCK(cudaGetLastError(), "perturb");
    return STARMAP_OK;
}

int starmap_mlp_shuffle(starmap_mlp_t* net, const int32_t* index, size_t count, unsigned long long seed,
                        int32_t* out) {
    if (!net) return STARMAP_E_ARG;
    if (count == 0) return STARMAP_OK;
    if (!out || count > 0x7fffffffu) return mfail(net, STARMAP_E_ARG, "shuffle needs an output and fewer than 2^31 samples");
    if (mlp::shuffle(index, (long)count, seed, out, net->stream)) MCK(cudaGetLastError(), "shuffle");
    return STARMAP_OK;
}

long starmap_mlp_steps(const starmap_mlp_t* net) { return net ? net->steps : 0; }

int starmap_mlp_sync(starmap_mlp_t* net) {
    if (!net) return STARMAP_E_ARG;
    MCK(cudaStreamSynchronize(net->stream), "sync");
    int flag = 0;
    MCK(cudaMemcpy(&flag, net->flag, sizeof(int), cudaMemcpyDeviceToHost), "read error flag");
    if (flag) {
        cudaMemset(net->flag, 0, sizeof(int));
        return mfail(net, STARMAP_E_TIMEOUT, "a bounded wait in the tcgen05 network gave up");
    }
    return STARMAP_OK;
}

int starmap_mlp_set_engine(starmap_mlp_t* net, int engine) {
    if (!net) return STARMAP_E_ARG;
    if (engine != STARMAP_MLP_ENGINE_MMA_SYNC && engine != STARMAP_MLP_ENGINE_TCGEN05)
        return mfail(net, STARMAP_E_ARG, "unknown network engine");
    net->engine = engine == STARMAP_MLP_ENGINE_TCGEN05 ? mlp::ENGINE_TCGEN05 : mlp::ENGINE_MMA_SYNC;
    return STARMAP_OK;
}

}  // extern "C"
