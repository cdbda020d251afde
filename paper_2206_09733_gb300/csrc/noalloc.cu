// Quadrature diagnostics that allocate nothing.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA stream
// capture is active (allocation is prohibited there), code inside a host
// framework that owns every byte of device memory through its own pool, or
// real-time loops where an allocation and its implicit synchronisation are
// not allowed.  hs3d_diagnostics keeps its per-block partial sums in scratch
// owned by the mesh; this variant takes every input from the caller and keeps
// the partial sums in a fixed file-scope device array instead.
//
// The array lives in every device that loads the library, until the process
// exits.  Host code may not pass the array's name to a kernel (on the host it
// is only a stand-in symbol): its device address is looked up once per device
// with cudaGetSymbolAddress and that pointer is passed.
#include <mutex>

#include "api_internal.h"

namespace hs3d {

// Capacity: one partial-sum slot (7 doubles, padded to 8) per 2048 nodes.
constexpr int kStaticSlots = 4096;
constexpr int kStaticNodesPerSlot = 2048;
constexpr long long kStaticMaxNodes = (long long)kStaticSlots * kStaticNodesPerSlot;   // 8,388,608
constexpr int kStaticThreads = 256;

static __device__ __align__(256) double g_static_partials[kStaticSlots * 8];

struct Weights {
    double w[kMaxn];
};

static __device__ void block_sum7_static(double v[7], double *sm)
{
    for (int k = 0; k < 7; ++k) sm[k * kStaticThreads + threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kStaticThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 7; ++k)
                sm[k * kStaticThreads + threadIdx.x] += sm[k * kStaticThreads + threadIdx.x + w];
        __syncthreads();
    }
    for (int k = 0; k < 7; ++k) v[k] = sm[k * kStaticThreads];
}

__global__ void __launch_bounds__(kStaticThreads)
k_diag_partial_static(int n, long long E, double g, const double *__restrict__ J, const double *__restrict__ u,
                      const double *__restrict__ dudt, Weights W, double *partials)
{
    __shared__ double sm[7 * kStaticThreads];
    const int n3 = n * n * n;
    const long long total = E * n3;
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    const long long begin = blockIdx.x * per, end = min(total, begin + per);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (long long t = begin + threadIdx.x; t < end; t += blockDim.x) {
        const long long e = t / n3;
        const int p = (int)(t - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const double wq = J[e * n3 + p] * W.w[i] * W.w[j] * W.w[k];
        const double *U = u + e * 5 * n3 + p;
        if (dudt) {
            const double *R = dudt + e * 5 * n3 + p;
            double uu[5], r[5];
            for (int v = 0; v < 5; ++v) {
                uu[v] = U[v * n3];
                r[v] = R[v * n3];
                acc[v] += wq * r[v];
            }
            double ir = 1.0 / uu[0];
            double v1 = uu[1] * ir, v2 = uu[2] * ir, v3 = uu[3] * ir;
            double vv = v1 * v1 + v2 * v2 + v3 * v3;
            double pr = (g - 1.0) * (uu[4] - 0.5 * uu[0] * vv);
            double s = log(pr) - g * log(uu[0]);
            double rp = (g - 1.0) * uu[0] / pr;
            double w[5] = {g - s - 0.5 * rp * vv, rp * v1, rp * v2, rp * v3, -rp};
            for (int v = 0; v < 5; ++v) {
                double tv = wq * w[v] * r[v];
                acc[5] += tv;
                acc[6] += fabs(tv);
            }
        } else {
            for (int v = 0; v < 5; ++v) acc[v] += wq * U[v * n3];
        }
    }
    block_sum7_static(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) partials[blockIdx.x * 8 + k] = acc[k];
}

__global__ void __launch_bounds__(kStaticThreads) k_diag_final_static(const double *partials, int nblocks, double *out)
{
    __shared__ double sm[7 * kStaticThreads];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 7; ++k) acc[k] += partials[b * 8 + k];
    block_sum7_static(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) out[k] = acc[k];
}

// Device address of g_static_partials, looked up once per device.
static double *static_partials_ptr(int dev, cudaError_t &err)
{
    static std::mutex mu;
    static double *ptrs[64] = {};
    err = cudaSuccess;
    if (dev < 0 || dev >= 64) {
        err = cudaErrorInvalidDevice;
        return nullptr;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!ptrs[dev]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_static_partials);
        if (err != cudaSuccess) return nullptr;
        ptrs[dev] = (double *)p;
    }
    return ptrs[dev];
}

}  // namespace hs3d

using namespace hs3d;

extern "C" hs3d_status hs3d_diagnostics_noalloc(int N, int64_t E, double gamma, int nodes, const double *J,
                                                const double *u, const double *dudt, double *out, void *stream)
{
    if (N < 1 || N > kMaxN) return fail(HS3D_ERR_INVALID, "N=%d outside 1..%d", N, kMaxN);
    if (nodes != HS3D_NODES_LOBATTO && nodes != HS3D_NODES_GAUSS) return fail(HS3D_ERR_INVALID, "bad nodes %d", nodes);
    if (E < 1) return fail(HS3D_ERR_INVALID, "E must be >= 1");
    if (!(gamma > 1.0)) return fail(HS3D_ERR_INVALID, "gamma must be > 1");
    if (!J || !u || !out) return fail(HS3D_ERR_INVALID, "J, u and out must not be NULL");
    const long long n3 = (long long)(N + 1) * (N + 1) * (N + 1);
    const long long total = (long long)E * n3;
    if (total > kStaticMaxNodes)
        return fail(HS3D_ERR_INVALID,
                    "E*(N+1)^3 = %lld nodes exceeds the static scratch capacity of %lld nodes "
                    "(%d partial-sum slots of %d nodes); use hs3d_diagnostics",
                    total, kStaticMaxNodes, kStaticSlots, kStaticNodesPerSlot);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "no CUDA device");
    double *partials = static_partials_ptr(dev, e);
    if (!partials) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
    // same partition as hs3d_diagnostics: one block per 2048 nodes
    long long nb = (total + kStaticNodesPerSlot - 1) / kStaticNodesPerSlot;
    int nblocks = (int)(nb < 1 ? 1 : nb);
    Weights W{};
    // the quadrature weights of the mesh's solution nodes (Gauss-Lobatto or Gauss-Legendre)
    const Ops &o = host_ops(N, nodes);
    for (int k = 0; k <= N; ++k) W.w[k] = o.w[k];
    cudaStream_t s = (cudaStream_t)stream;
    k_diag_partial_static<<<nblocks, kStaticThreads, 0, s>>>(N + 1, E, gamma, J, u, dudt, W, partials);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_diag_final_static<<<1, kStaticThreads, 0, s>>>(partials, nblocks, out);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "static diagnostics launch");
}
