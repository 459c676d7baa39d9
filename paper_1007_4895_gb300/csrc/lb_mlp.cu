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

#include <algorithm>
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

/* Inference on the tensor cores: mma.sync m16n8k16 with BF16 operands and FP32
 * accumulation. A warp takes 16 nodes at a time. Layer 1 is the 16 x 16 (8 features,
 * zero-padded) by 16 x 64 product; its GELU outputs are rounded to BF16 and, because
 * the accumulator fragment of two neighbouring 8-column output tiles has exactly the
 * element layout of one 16-wide operand fragment, feed layer 2 from registers; layer 2's
 * GELU outputs meet W3 in FP32 (a dot product over the 64 hidden units, finished across
 * the four lanes that share a row). The weight fragments are built in shared memory
 * once per block. A node with a non-finite feature gets p = NaN. */
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t pack_bf16_raw(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<const uint32_t *>(&v);
}

__global__ void __launch_bounds__(128) infer_mma_kernel(const __nv_bfloat16 *__restrict__ wb,
                                                        const float *__restrict__ norm,
                                                        const float *__restrict__ X, long long n,
                                                        float *__restrict__ p)
{
    /* operand fragments of the weights: B[k][n] of layer 1 is W1[n][k] (k < 8, zero
     * above), of layer 2 W2[n][k]; fragment register r of lane l holds the rows
     * 2 (l % 4) + {0, 1} (+ 8 for r = 1) of column l / 4 */
    __shared__ uint32_t w1f[8][32][2];
    __shared__ uint32_t w2f[4][8][32][2];
    __shared__ float b1s[NH], b2s[NH], w3s[NH], nm[2 * NF], b3s;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.0f);
    for (int k = threadIdx.x; k < 8 * 32; k += blockDim.x) {
        const int nt = k / 32, l = k % 32, col = 8 * nt + l / 4, row = 2 * (l % 4);
        w1f[nt][l][0] = pack_bf16_raw(wb[OFF_W1 + col * NF + row], wb[OFF_W1 + col * NF + row + 1]);
        w1f[nt][l][1] = pack_bf16_raw(zero, zero);
    }
    for (int k = threadIdx.x; k < 4 * 8 * 32; k += blockDim.x) {
        const int kt = k / 256, nt = (k / 32) % 8, l = k % 32;
        const int col = 8 * nt + l / 4, row = 16 * kt + 2 * (l % 4);
        const __nv_bfloat16 *w = wb + OFF_W2 + col * NH;
        w2f[kt][nt][l][0] = pack_bf16_raw(w[row], w[row + 1]);
        w2f[kt][nt][l][1] = pack_bf16_raw(w[row + 8], w[row + 9]);
    }
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        b1s[k] = __bfloat162float(wb[OFF_B1 + k]);
        b2s[k] = __bfloat162float(wb[OFF_B2 + k]);
        w3s[k] = __bfloat162float(wb[OFF_W3 + k]);
    }
    if (threadIdx.x < 2 * NF) nm[threadIdx.x] = norm[threadIdx.x];
    if (threadIdx.x == 0) b3s = __bfloat162float(wb[OFF_B3]);
    __syncthreads();

    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const long long tiles = (n + 15) / 16;
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < tiles; t += stride) {
        const long long r0 = 16 * t + g, r1 = r0 + 8;   /* the two nodes (rows) of this lane */
        /* layer-1 operand: normalised features 2q, 2q + 1 of both rows (columns 8..15 zero) */
        float x[2][2];
        bool ok0 = true, ok1 = true;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int f = 2 * q + e;
            x[0][e] = r0 < n ? (X[(long long)f * n + r0] - nm[f]) / nm[NF + f] : 0.0f;
            x[1][e] = r1 < n ? (X[(long long)f * n + r1] - nm[f]) / nm[NF + f] : 0.0f;
            ok0 = ok0 && isfinite(x[0][e]);
            ok1 = ok1 && isfinite(x[1][e]);
        }
        /* a node is usable when all eight features are finite: the four lanes of a row
         * hold two each */
        const unsigned m0 = __ballot_sync(0xffffffffu, !ok0), m1 = __ballot_sync(0xffffffffu, !ok1);
        const unsigned qm = 0xfu << (4 * g);
        ok0 = !(m0 & qm);
        ok1 = !(m1 & qm);
        if (!ok0) x[0][0] = x[0][1] = 0.0f;
        if (!ok1) x[1][0] = x[1][1] = 0.0f;
        const uint32_t a1[4] = {pack_bf16(x[0][0], x[0][1]), pack_bf16(x[1][0], x[1][1]), 0u, 0u};
        /* layer 1 -> GELU -> BF16 operand fragments of layer 2 */
        uint32_t a2[4][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            const uint32_t b[2] = {w1f[nt][lane][0], w1f[nt][lane][1]};
            mma_bf16(c, a1, b);
            const int col = 8 * nt + 2 * q;
            const float h00 = gelu(c[0] + b1s[col]), h01 = gelu(c[1] + b1s[col + 1]);
            const float h10 = gelu(c[2] + b1s[col]), h11 = gelu(c[3] + b1s[col + 1]);
            const int kt = nt >> 1, hi = (nt & 1) * 2;
            a2[kt][hi] = pack_bf16(h00, h01);
            a2[kt][hi + 1] = pack_bf16(h10, h11);
        }
        /* layer 2 -> GELU -> W3 dot product */
        float z0 = 0.0f, z1 = 0.0f;
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int kt = 0; kt < 4; ++kt) {
                const uint32_t b[2] = {w2f[kt][nt][lane][0], w2f[kt][nt][lane][1]};
                mma_bf16(c, a2[kt], b);
            }
            const int col = 8 * nt + 2 * q;
            z0 = fmaf(gelu(c[0] + b2s[col]), w3s[col], z0);
            z0 = fmaf(gelu(c[1] + b2s[col + 1]), w3s[col + 1], z0);
            z1 = fmaf(gelu(c[2] + b2s[col]), w3s[col], z1);
            z1 = fmaf(gelu(c[3] + b2s[col + 1]), w3s[col + 1], z1);
        }
        z0 += __shfl_xor_sync(0xffffffffu, z0, 1);
        z0 += __shfl_xor_sync(0xffffffffu, z0, 2);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 1);
        z1 += __shfl_xor_sync(0xffffffffu, z1, 2);
        if (q == 0) {
            if (r0 < n) p[r0] = ok0 ? 1.0f / (1.0f + expf(-(z0 + b3s))) : nanf("");
            if (r1 < n) p[r1] = ok1 ? 1.0f / (1.0f + expf(-(z1 + b3s))) : nanf("");
        }
    }
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
    /* four warps per block, up to 8 blocks per SM resident (152 SMs): each warp walks
     * its 16-node tiles with a grid stride */
    const long long tiles = (n + 15) / 16;
    const unsigned blocks = (unsigned)std::min<long long>((tiles + 3) / 4, 152LL * 8);
    lbm::infer_mma_kernel<<<blocks, 128, 0, static_cast<cudaStream_t>(stream)>>>(M->wb, M->norm, x, (long long)n, p);
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
