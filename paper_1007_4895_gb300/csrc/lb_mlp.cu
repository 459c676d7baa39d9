/*
 * lb_mlp.cu -- learned interface placement.
 *
 * Sec. 2.2 leaves the switching criterion open (it lists local Knudsen numbers and the
 * B parameter from the literature). This file adds a small network that predicts, per
 * node, whether the high-order set is needed:
 *   features (8, from the node's own populations): Pi^neq_xx / rho, Pi^neq_xy / rho,
 *     Pi^neq_yy / rho, q_x / rho, q_y / rho, wall distance / H, local Kn (Eq. (KN)),
 *     gradient-length Knudsen number Kn |grad rho| / rho;
 *   label (for training): 1 when more than a threshold of the node's non-equilibrium
 *     part lies beyond what a second-order Hermite expansion carries (what a low-order
 *     node can hold, Sec. 2.2), measured on a high-order run;
 *   network: 8 -> 64 -> 64 -> 1, GELU (erf form) hidden layers, sigmoid output.
 * Training runs here in FP32 (forward, backward, weight gradients, Adam: one kernel
 * each); inference uses BF16 weights with FP32 accumulation. Parameter layout:
 * W1 [64][8], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1] (4801 values).
 */
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "lb_mlp.h"

namespace lbm {

constexpr int NF = 8, NH = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NF, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == 4801, "parameter count");

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.0f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float a)
{
    return 0.5f * (1.0f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

/* Forward pass of a mini-batch: sample b uses column idx[b] of X [NF][n]; keeps the
 * pre-activations and activations for the backward pass. One thread per sample. */
__global__ void fwd_kernel(const float *__restrict__ th, const float *__restrict__ norm, const float *__restrict__ X,
                           long long n, const int *__restrict__ idx, int B, float *xn, float *a1, float *h1, float *a2,
                           float *h2, float *pout)
{
    __shared__ float s[NPARAM];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) s[k] = th[k];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long long c = idx ? idx[b] : b;
    float x[NF];
    for (int f = 0; f < NF; ++f) {
        x[f] = (X[(long long)f * n + c] - norm[f]) / norm[NF + f];
        xn[(size_t)b * NF + f] = x[f];
    }
    float hh[NH];
    for (int i = 0; i < NH; ++i) {
        float t = s[OFF_B1 + i];
        for (int f = 0; f < NF; ++f) t = fmaf(s[OFF_W1 + i * NF + f], x[f], t);
        a1[(size_t)b * NH + i] = t;
        hh[i] = gelu(t);
        h1[(size_t)b * NH + i] = hh[i];
    }
    float z = s[OFF_B3];
    for (int i = 0; i < NH; ++i) {
        float t = s[OFF_B2 + i];
        for (int k = 0; k < NH; ++k) t = fmaf(s[OFF_W2 + i * NH + k], hh[k], t);
        a2[(size_t)b * NH + i] = t;
        const float g = gelu(t);
        h2[(size_t)b * NH + i] = g;
        z = fmaf(s[OFF_W3 + i], g, z);
    }
    pout[b] = 1.0f / (1.0f + expf(-z));
}

/* Backward pass through the activations: dz = (p - y) / B, then dA2 and dA1 per sample. */
__global__ void bwd_kernel(const float *__restrict__ th, const float *__restrict__ Y, const int *__restrict__ idx, int B,
                           const float *a1, const float *a2, const float *pout, float *dz, float *da1, float *da2,
                           double *loss_acc)
{
    __shared__ float s[NPARAM];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) s[k] = th[k];
    __syncthreads();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const long long c = idx ? idx[b] : b;
    const float y = Y[c], p = pout[b];
    const float g = (p - y) / (float)B;
    dz[b] = g;
    if (loss_acc) {
        const double pc = fmin(fmax((double)p, 1e-30), 1.0 - 1e-7);
        atomicAdd(loss_acc, -((double)y * log(pc) + (1.0 - (double)y) * log(1.0 - pc)) / (double)B);
    }
    float d2[NH];
    for (int i = 0; i < NH; ++i) {
        d2[i] = g * s[OFF_W3 + i] * gelu_grad(a2[(size_t)b * NH + i]);
        da2[(size_t)b * NH + i] = d2[i];
    }
    for (int k = 0; k < NH; ++k) {
        float t = 0.0f;
        for (int i = 0; i < NH; ++i) t = fmaf(d2[i], s[OFF_W2 + i * NH + k], t);
        da1[(size_t)b * NH + k] = t * gelu_grad(a1[(size_t)b * NH + k]);
    }
}

/* Weight gradients, one thread per parameter, summed over the batch in sample order. */
__global__ void wgrad_kernel(int B, const float *xn, const float *h1, const float *h2, const float *dz, const float *da1,
                             const float *da2, float *grad)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    float t = 0.0f;
    if (k < OFF_B1) {
        const int i = k / NF, f = k % NF;
        for (int b = 0; b < B; ++b) t = fmaf(da1[(size_t)b * NH + i], xn[(size_t)b * NF + f], t);
    } else if (k < OFF_W2) {
        const int i = k - OFF_B1;
        for (int b = 0; b < B; ++b) t += da1[(size_t)b * NH + i];
    } else if (k < OFF_B2) {
        const int i = (k - OFF_W2) / NH, j = (k - OFF_W2) % NH;
        for (int b = 0; b < B; ++b) t = fmaf(da2[(size_t)b * NH + i], h1[(size_t)b * NH + j], t);
    } else if (k < OFF_W3) {
        const int i = k - OFF_B2;
        for (int b = 0; b < B; ++b) t += da2[(size_t)b * NH + i];
    } else if (k < OFF_B3) {
        const int i = k - OFF_W3;
        for (int b = 0; b < B; ++b) t = fmaf(dz[b], h2[(size_t)b * NH + i], t);
    } else {
        for (int b = 0; b < B; ++b) t += dz[b];
    }
    grad[k] = t;
}

/* Adam (Kingma & Ba), bias-corrected, step t >= 1. */
__global__ void adam_kernel(float *th, float *m, float *v, const float *g, int t, float lr, float b1, float b2, float eps)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPARAM) return;
    const float mk = b1 * m[k] + (1.0f - b1) * g[k];
    const float vk = b2 * v[k] + (1.0f - b2) * g[k] * g[k];
    m[k] = mk;
    v[k] = vk;
    const float mh = mk / (1.0f - powf(b1, (float)t)), vh = vk / (1.0f - powf(b2, (float)t));
    th[k] -= lr * mh / (sqrtf(vh) + eps);
}

/* BF16 copy of the weights used by inference. */
__global__ void to_bf16_kernel(const float *th, __nv_bfloat16 *wb)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < NPARAM) wb[k] = __float2bfloat16_rn(th[k]);
}

/* Inference: BF16 weights (held in shared memory as float), FP32 accumulation; one
 * thread per node; X [NF][n] raw features, out p [n]. */
__global__ void infer_kernel(const __nv_bfloat16 *__restrict__ wb, const float *__restrict__ norm,
                             const float *__restrict__ X, long long n, float *__restrict__ p)
{
    __shared__ float s[NPARAM];
    __shared__ float nm[2 * NF];
    for (int k = threadIdx.x; k < NPARAM; k += blockDim.x) s[k] = __bfloat162float(wb[k]);
    if (threadIdx.x < 2 * NF) nm[threadIdx.x] = norm[threadIdx.x];
    __syncthreads();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    float x[NF];
    bool ok = true;
    for (int f = 0; f < NF; ++f) {
        x[f] = (X[(long long)f * n + c] - nm[f]) / nm[NF + f];
        ok = ok && isfinite(x[f]);
    }
    if (!ok) {
        p[c] = nanf("");
        return;
    }
    float hh[NH];
    for (int i = 0; i < NH; ++i) {
        float t = s[OFF_B1 + i];
        for (int f = 0; f < NF; ++f) t = fmaf(s[OFF_W1 + i * NF + f], x[f], t);
        hh[i] = gelu(t);
    }
    float z = s[OFF_B3];
    for (int i = 0; i < NH; ++i) {
        float t = s[OFF_B2 + i];
        for (int k = 0; k < NH; ++k) t = fmaf(s[OFF_W2 + i * NH + k], hh[k], t);
        z = fmaf(s[OFF_W3 + i], gelu(t), z);
    }
    p[c] = 1.0f / (1.0f + expf(-z));
}

}  // namespace lbm

/* ------------------------------------------------------------------ host -- */

struct lb_mlp {
    float *th = nullptr, *m = nullptr, *v = nullptr, *g = nullptr, *norm = nullptr;
    __nv_bfloat16 *wb = nullptr;
    int cap = 0;   /* batch capacity of the activation buffers */
    float *xn = nullptr, *a1 = nullptr, *h1 = nullptr, *a2 = nullptr, *h2 = nullptr, *p = nullptr, *dz = nullptr,
          *da1 = nullptr, *da2 = nullptr;
    int *idx = nullptr;
    double *loss = nullptr;
    int t = 0;
    lb_opts opts{};
    cudaStream_t stream = nullptr;
    std::vector<void *> owned;
};

namespace {

void *mlp_alloc(lb_mlp *M, size_t bytes)
{
    void *ptr = nullptr;
    if (M->opts.alloc && M->opts.free) ptr = M->opts.alloc(bytes, M->opts.alloc_user);
    else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) M->owned.push_back(ptr);
    return ptr;
}

void mlp_free_all(lb_mlp *M)
{
    if (M->stream) cudaStreamSynchronize(M->stream);
    for (void *ptr : M->owned) {
        if (M->opts.alloc && M->opts.free) M->opts.free(ptr, M->opts.alloc_user);
        else cudaFree(ptr);
    }
    M->owned.clear();
}

int mlp_err(int code, const std::string &msg)
{
    lbk::set_last_error(msg);
    return code;
}

int ensure_batch(lb_mlp *M, int B)
{
    if (B <= M->cap) return LB_OK;
    /* grow the activation buffers (old ones stay owned until destroy) */
    const size_t b = (size_t)B;
    M->xn = (float *)mlp_alloc(M, b * lbm::NF * 4);
    M->a1 = (float *)mlp_alloc(M, b * lbm::NH * 4);
    M->h1 = (float *)mlp_alloc(M, b * lbm::NH * 4);
    M->a2 = (float *)mlp_alloc(M, b * lbm::NH * 4);
    M->h2 = (float *)mlp_alloc(M, b * lbm::NH * 4);
    M->da1 = (float *)mlp_alloc(M, b * lbm::NH * 4);
    M->da2 = (float *)mlp_alloc(M, b * lbm::NH * 4);
    M->p = (float *)mlp_alloc(M, b * 4);
    M->dz = (float *)mlp_alloc(M, b * 4);
    M->idx = (int *)mlp_alloc(M, b * 4);
    if (!M->xn || !M->a1 || !M->h1 || !M->a2 || !M->h2 || !M->da1 || !M->da2 || !M->p || !M->dz || !M->idx)
        return mlp_err(LB_ERR_NOMEM, "lb_mlp: device allocation failed");
    M->cap = B;
    return LB_OK;
}

/* forward + backward + weight gradients of one batch (samples idx_host, or the first B) */
int batch_grad(lb_mlp *M, const float *x, const float *y, int64_t n, const int *idx_dev, int B, bool want_loss)
{
    const int T = 128, nb = (B + T - 1) / T;
    if (want_loss && cudaMemsetAsync(M->loss, 0, sizeof(double), M->stream) != cudaSuccess)
        return mlp_err(LB_ERR_CUDA, "lb_mlp: memset failed");
    lbm::fwd_kernel<<<nb, T, 0, M->stream>>>(M->th, M->norm, x, (long long)n, idx_dev, B, M->xn, M->a1, M->h1, M->a2,
                                             M->h2, M->p);
    lbm::bwd_kernel<<<nb, T, 0, M->stream>>>(M->th, y, idx_dev, B, M->a1, M->a2, M->p, M->dz, M->da1, M->da2,
                                             want_loss ? M->loss : nullptr);
    lbm::wgrad_kernel<<<(lbm::NPARAM + 127) / 128, 128, 0, M->stream>>>(B, M->xn, M->h1, M->h2, M->dz, M->da1, M->da2,
                                                                        M->g);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : mlp_err(LB_ERR_CUDA, std::string("lb_mlp: ") + cudaGetErrorString(e));
}

}  // namespace

namespace lbk {

int mlp_infer_dev(lb_mlp *M, const float *x, int64_t n, float *p, void *stream)
{
    lbm::infer_kernel<<<(unsigned)((n + 127) / 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(M->wb, M->norm, x,
                                                                                                   (long long)n, p);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : mlp_err(LB_ERR_CUDA, std::string("lb_mlp_infer: ") + cudaGetErrorString(e));
}

}  // namespace lbk

extern "C" {

int lb_mlp_create(const float *params, const float norm[16], const lb_opts *opts, lb_mlp **out)
{
    if (!params || !norm || !opts || !out) return mlp_err(LB_ERR_INVALID, "lb_mlp_create: null argument");
    for (int f = 0; f < lbm::NF; ++f)
        if (!(norm[lbm::NF + f] > 0.0f)) return mlp_err(LB_ERR_INVALID, "lb_mlp_create: feature scales must be positive");
    lb_mlp *M = new lb_mlp();
    M->opts = *opts;
    M->stream = static_cast<cudaStream_t>(opts->stream);
    M->th = (float *)mlp_alloc(M, lbm::NPARAM * 4);
    M->m = (float *)mlp_alloc(M, lbm::NPARAM * 4);
    M->v = (float *)mlp_alloc(M, lbm::NPARAM * 4);
    M->g = (float *)mlp_alloc(M, lbm::NPARAM * 4);
    M->wb = (__nv_bfloat16 *)mlp_alloc(M, lbm::NPARAM * 2);
    M->norm = (float *)mlp_alloc(M, 2 * lbm::NF * 4);
    M->loss = (double *)mlp_alloc(M, 256);
    if (!M->th || !M->m || !M->v || !M->g || !M->wb || !M->norm || !M->loss) {
        mlp_free_all(M);
        delete M;
        return mlp_err(LB_ERR_NOMEM, "lb_mlp_create: device allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(M->th, params, lbm::NPARAM * 4, cudaMemcpyHostToDevice, M->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(M->norm, norm, 2 * lbm::NF * 4, cudaMemcpyHostToDevice, M->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, lbm::NPARAM * 4, M->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->v, 0, lbm::NPARAM * 4, M->stream);
    if (e == cudaSuccess) {
        lbm::to_bf16_kernel<<<(lbm::NPARAM + 255) / 256, 256, 0, M->stream>>>(M->th, M->wb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
    if (e != cudaSuccess) {
        mlp_free_all(M);
        delete M;
        return mlp_err(LB_ERR_CUDA, std::string("lb_mlp_create: ") + cudaGetErrorString(e));
    }
    *out = M;
    return LB_OK;
}

int lb_mlp_grad(lb_mlp *M, const float *x, const float *y, int64_t n, float *grad, double *loss)
{
    if (!M || !x || !y || !grad || n < 1 || n > (1 << 20)) return mlp_err(LB_ERR_INVALID, "lb_mlp_grad: bad argument");
    if (int e = ensure_batch(M, (int)n)) return e;
    if (int e = batch_grad(M, x, y, n, nullptr, (int)n, true)) return e;
    cudaError_t ce = cudaMemcpyAsync(grad, M->g, lbm::NPARAM * 4, cudaMemcpyDeviceToHost, M->stream);
    double l = 0.0;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&l, M->loss, sizeof(double), cudaMemcpyDeviceToHost, M->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(M->stream);
    if (ce != cudaSuccess) return mlp_err(LB_ERR_CUDA, std::string("lb_mlp_grad: ") + cudaGetErrorString(ce));
    if (loss) *loss = l;
    return LB_OK;
}

int lb_mlp_train(lb_mlp *M, const float *x, const float *y, int64_t n, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, double *last_epoch_loss)
{
    if (!M || !x || !y || n < 1 || epochs < 1 || batch < 1 || batch > 65536 || !(lr > 0.0f))
        return mlp_err(LB_ERR_INVALID, "lb_mlp_train: bad argument");
    if (int e = ensure_batch(M, batch)) return e;
    std::vector<int> perm((size_t)n);
    for (int64_t k = 0; k < n; ++k) perm[(size_t)k] = (int)k;
    std::mt19937_64 rng(seed);
    double eloss = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t k = n - 1; k > 0; --k) std::swap(perm[(size_t)k], perm[(size_t)(rng() % (uint64_t)(k + 1))]);
        eloss = 0.0;
        int nbat = 0;
        for (int64_t s0 = 0; s0 < n; s0 += batch) {
            const int B = (int)std::min<int64_t>(batch, n - s0);
            if (cudaMemcpyAsync(M->idx, perm.data() + s0, (size_t)B * 4, cudaMemcpyHostToDevice, M->stream) != cudaSuccess)
                return mlp_err(LB_ERR_CUDA, "lb_mlp_train: copy failed");
            const bool last_epoch = ep == epochs - 1;
            if (int e = batch_grad(M, x, y, n, M->idx, B, last_epoch)) return e;
            M->t += 1;
            lbm::adam_kernel<<<(lbm::NPARAM + 127) / 128, 128, 0, M->stream>>>(M->th, M->m, M->v, M->g, M->t, lr, 0.9f,
                                                                              0.999f, 1e-8f);
            if (last_epoch) {
                double l = 0.0;
                if (cudaMemcpyAsync(&l, M->loss, sizeof(double), cudaMemcpyDeviceToHost, M->stream) != cudaSuccess ||
                    cudaStreamSynchronize(M->stream) != cudaSuccess)
                    return mlp_err(LB_ERR_CUDA, "lb_mlp_train: copy failed");
                eloss += l * B;
                ++nbat;
            }
        }
        (void)nbat;
        /* the copy above waits; keep perm alive until the last batch's upload finished */
        if (cudaStreamSynchronize(M->stream) != cudaSuccess) return mlp_err(LB_ERR_CUDA, "lb_mlp_train: sync failed");
    }
    lbm::to_bf16_kernel<<<(lbm::NPARAM + 255) / 256, 256, 0, M->stream>>>(M->th, M->wb);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(M->stream) != cudaSuccess)
        return mlp_err(LB_ERR_CUDA, "lb_mlp_train: kernel failed");
    if (last_epoch_loss) *last_epoch_loss = eloss / (double)n;
    return LB_OK;
}

int lb_mlp_adam_step(lb_mlp *M, const float *x, const float *y, int64_t n, float lr)
{
    if (!M || !x || !y || n < 1 || n > (1 << 20)) return mlp_err(LB_ERR_INVALID, "lb_mlp_adam_step: bad argument");
    if (int e = ensure_batch(M, (int)n)) return e;
    if (int e = batch_grad(M, x, y, n, nullptr, (int)n, false)) return e;
    M->t += 1;
    lbm::adam_kernel<<<(lbm::NPARAM + 127) / 128, 128, 0, M->stream>>>(M->th, M->m, M->v, M->g, M->t, lr, 0.9f, 0.999f,
                                                                      1e-8f);
    lbm::to_bf16_kernel<<<(lbm::NPARAM + 255) / 256, 256, 0, M->stream>>>(M->th, M->wb);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(M->stream) != cudaSuccess)
        return mlp_err(LB_ERR_CUDA, "lb_mlp_adam_step: kernel failed");
    return LB_OK;
}

int lb_mlp_get_params(lb_mlp *M, float *params)
{
    if (!M || !params) return mlp_err(LB_ERR_INVALID, "lb_mlp_get_params: null argument");
    if (cudaMemcpyAsync(params, M->th, lbm::NPARAM * 4, cudaMemcpyDeviceToHost, M->stream) != cudaSuccess ||
        cudaStreamSynchronize(M->stream) != cudaSuccess)
        return mlp_err(LB_ERR_CUDA, "lb_mlp_get_params: copy failed");
    return LB_OK;
}

int lb_mlp_infer(lb_mlp *M, const float *x, int64_t n, float *p)
{
    if (!M || !x || !p || n < 1) return mlp_err(LB_ERR_INVALID, "lb_mlp_infer: bad argument");
    if (int e = lbk::mlp_infer_dev(M, x, n, p, M->stream)) return e;
    return cudaStreamSynchronize(M->stream) == cudaSuccess ? LB_OK : mlp_err(LB_ERR_CUDA, "lb_mlp_infer: sync failed");
}

void lb_mlp_destroy(lb_mlp *M)
{
    if (!M) return;
    mlp_free_all(M);
    delete M;
}

}  // extern "C"
