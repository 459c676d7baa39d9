/*
 * lb_noalloc.cu -- the mass / residual reduction for callers that cannot allocate device
 * memory.
 *
 * Some callers cannot call cudaMalloc or any allocating routine: code running inside a
 * memory budget fixed by its host application, or code whose allocator is owned by
 * another framework and not reachable from C. For them lb_reduce_fields_noalloc does
 * the work of the
 * lb_reductions kernel on fields the caller already owns, and keeps everything else it
 * needs in one fixed scratch array that lives in this file:
 *   - per-block FP64 partial sums and the completion counter of the two-stage
 *     deterministic reduction;
 *   - the velocity field of the previous call (the residual compares against it).
 * The array is a file-scope __device__ variable: every GPU that loads the library holds
 * it until the process exits. Host code never dereferences its name (on the host it is
 * only a stand-in); the device address is looked up once per device with
 * cudaGetSymbolAddress, with that device current, on the first call made on it.
 * Every call is synchronous (it reads its result back to the host and waits for the
 * stream), so it must not be called while its stream is being captured.
 */
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/lb.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = (LB_NOALLOC_MAX_NODES + kThreads - 1) / kThreads;

struct NoallocScratch {
    double part[kMaxBlocks][4];               /* per-block partial sums */
    double result[4];                         /* mass, residual, non-finite count, nodes */
    unsigned int counter;                     /* blocks finished in the current call */
    unsigned int pad[63];
    double uprev[LB_NOALLOC_MAX_NODES][2];    /* velocity of the previous call */
};

__device__ __align__(256) NoallocScratch g_noalloc_scratch;

std::mutex g_mu;
NoallocScratch *g_dev_ptr[64] = {};   /* device address of the array, per device */

/* Same sums as the lb_reductions kernel, over caller-owned fields: per node rho, u and
 * u_prev (the previous call's velocity, kept in the scratch array); warp shuffles, then
 * shared memory, then one partial per block; the last block adds the partials in block
 * order and resets the counter. restart != 0 compares with u = 0. */
__global__ void noalloc_reduce_kernel(const double *rho, const double *ux, const double *uy, long long n, int restart,
                                      NoallocScratch *scr)
{
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double r = rho[i], u = ux[i], v = uy[i];
        if (!isfinite(r) || !isfinite(u) || !isfinite(v)) {
            acc[3] = 1.0;
        } else {
            const double pu = restart ? 0.0 : scr->uprev[i][0], pv = restart ? 0.0 : scr->uprev[i][1];
            acc[0] = r;
            acc[1] = (u - pu) * (u - pu) + (v - pv) * (v - pv);
            acc[2] = u * u + v * v;
        }
        /* every node keeps this call's velocity, a non-finite one included, so that the
         * next call never compares with a velocity older than the previous call */
        scr->uprev[i][0] = u;
        scr->uprev[i][1] = v;
    }
    for (int m = 0; m < 4; ++m)
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_down_sync(0xffffffffu, acc[m], o);
    __shared__ double sh[kThreads / 32][4];
    __shared__ bool last;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (lane == 0)
        for (int m = 0; m < 4; ++m) sh[warp][m] = acc[m];
    __syncthreads();
    if (threadIdx.x == 0) {
        double b[4] = {0.0, 0.0, 0.0, 0.0};
        for (int w = 0; w < kThreads / 32; ++w)
            for (int m = 0; m < 4; ++m) b[m] += sh[w][m];
        for (int m = 0; m < 4; ++m) scr->part[blockIdx.x][m] = b[m];
        __threadfence();
        last = (atomicAdd(&scr->counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (unsigned b = 0; b < gridDim.x; ++b)
            for (int m = 0; m < 4; ++m) t[m] += __ldcg(&scr->part[b][m]);   /* other blocks' partials, from L2 */
        scr->result[0] = t[0];
        scr->result[1] = t[2] > 0.0 ? sqrt(t[1] / t[2]) : 0.0;
        scr->result[2] = t[3];
        scr->result[3] = (double)n;
        scr->counter = 0u;
    }
}

/* Device address of the scratch array on the current device, looked up once per
 * device; 0 on success, else a CUDA error code (or -1). */
int scratch_ptr(NoallocScratch **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return -1;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return (int)e ? (int)e : -1;
        }
        g_dev_ptr[dev] = static_cast<NoallocScratch *>(p);
    }
    *out = g_dev_ptr[dev];
    return 0;
}

}  // namespace

namespace lbk {
void set_last_error(const std::string &msg);   /* read back by lb_last_error() */
}

namespace {
int fail_na(int code, const std::string &msg)
{
    lbk::set_last_error("lb_reduce_fields_noalloc: " + msg);
    return code;
}
}  // namespace

extern "C" int lb_reduce_fields_noalloc(const double *rho, const double *ux, const double *uy, int64_t n,
                                        int32_t restart, void *stream, double out[4])
{
    if (!rho || !ux || !uy || !out) return fail_na(LB_ERR_INVALID, "null argument");
    if (n < 1 || n > LB_NOALLOC_MAX_NODES)
        return fail_na(LB_ERR_INVALID, "n = " + std::to_string(n) + " is outside 1 .. " +
                                           std::to_string(LB_NOALLOC_MAX_NODES) + " (the size of its fixed scratch array)");
    NoallocScratch *scr = nullptr;
    if (int e = scratch_ptr(&scr))
        return fail_na(LB_ERR_CUDA, std::string("cannot locate the scratch array on the current device: ") +
                                        (e > 0 ? cudaGetErrorString((cudaError_t)e) : "no usable current device"));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    /* the completion counter must start at zero: clear it (a previous call that failed
     * part-way could have left it set) */
    cudaError_t ce = cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned int), st);
    const int blocks = (int)((n + kThreads - 1) / kThreads);
    if (ce == cudaSuccess) {
        noalloc_reduce_kernel<<<blocks, kThreads, 0, st>>>(rho, ux, uy, (long long)n, restart ? 1 : 0, scr);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(out, scr->result, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) return fail_na(LB_ERR_CUDA, cudaGetErrorString(ce));
    if (out[2] > 0.0) return fail_na(LB_ERR_DIVERGED, "non-finite density or velocity");
    return LB_OK;
}
