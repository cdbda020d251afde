// Reductions: the time-step rule and the quadrature diagnostics.
//
// Time step (the paper names explicit RK3 with a CFL condition, Sec. 3.7, but
// gives no formula; this library uses)
//   dt_c = cfl * 2 / (n * max_nodes sum_d (|Ja^d.v| + c |Ja^d|)/J)
//   dt_v = 12 / (n^4 * max_nodes (mu/rho) sum_d (|Ja^d|/J)^2)      (Navier-Stokes)
//   dt   = min(dt_c, dt_v), clipped to reach t_final exactly.
// The maxima are taken with atomicMax on the bit patterns of non-negative
// doubles, which is exact and order-independent.
//
// Diagnostics: per-block partial sums of J w_i w_j w_k f in a fixed
// partition, then one block sums the partials in a fixed tree order, so the
// result does not depend on scheduling.
#include <math.h>

#include "internal.cuh"

namespace hs3d {

template <int N>
__global__ void __launch_bounds__(256) k_lambda(const __grid_constant__ Batch b, int ns)
{
    constexpr int n = N + 1, n3 = n * n * n;
    __shared__ double s_lc[256], s_lv[256];
    __shared__ const Item *s_it[256];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double lc = 0.0, lv = 0.0;
    const Item *itp = nullptr;
    if (t < b.total_elems * n3) {
        const long long ge = t / n3;
        const int p = (int)(t - ge * n3);
        itp = &find_item_elem(b, ge);
        const Item &it = *itp;
        const int e = (int)(ge - it.elem_begin);
        const double *U = it.u + (size_t)e * 5 * n3 + p;
        double rho = U[0], ir = 1.0 / rho;
        double v1 = U[n3] * ir, v2 = U[2 * n3] * ir, v3 = U[3 * n3] * ir;
        double pr = (it.gamma - 1.0) * (U[4 * n3] - 0.5 * rho * (v1 * v1 + v2 * v2 + v3 * v3));
        if (!(rho > 0.0) || !(pr > 0.0)) {
            it.clk->bad = 1;
        } else {
            double c = sqrt(it.gamma * pr * ir);
            const double *JA = it.Ja + (size_t)e * 9 * n3 + p;
            double iJ = it.invJ[(size_t)e * n3 + p];
            double sv = 0.0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                double a1 = JA[(d * 3) * n3], a2 = JA[(d * 3 + 1) * n3], a3 = JA[(d * 3 + 2) * n3];
                double an = sqrt(a1 * a1 + a2 * a2 + a3 * a3);
                lc += (fabs(a1 * v1 + a2 * v2 + a3 * v3) + c * an) * iJ;
                sv += (an * iJ) * (an * iJ);
            }
            if (ns) lv = it.mu * sv * ir;
        }
    }
    s_lc[threadIdx.x] = lc;
    s_lv[threadIdx.x] = lv;
    s_it[threadIdx.x] = itp;
    __syncthreads();
    // runs of equal items: the first thread of each run reduces it
    if (itp && (threadIdx.x == 0 || s_it[threadIdx.x - 1] != itp)) {
        double mc = lc, mv = lv;
        for (int k = threadIdx.x + 1; k < blockDim.x && s_it[k] == itp; ++k) {
            mc = fmax(mc, s_lc[k]);
            mv = fmax(mv, s_lv[k]);
        }
        atomicMax(&itp->clk->lam_c, (unsigned long long)__double_as_longlong(mc));
        if (ns) atomicMax(&itp->clk->lam_v, (unsigned long long)__double_as_longlong(mv));
    }
}

// One thread per item: dt from the maxima (mode 0) or the fixed dt (mode 1),
// clipped at t_final; advances the clock and resets the maxima.
__global__ void k_dt_finalize(const __grid_constant__ Batch b, int n, int mode)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.nitems) return;
    const Item &it = (b.nitems == 1) ? b.single : b.items[i];
    Clock *c = it.clk;
    double lc = __longlong_as_double((long long)c->lam_c);
    double lv = __longlong_as_double((long long)c->lam_v);
    c->lam_c = 0ull;
    c->lam_v = 0ull;
    // a solve that has reached its stopping rule takes no further step
    if (c->done || (c->t_final > 0.0 && c->t >= c->t_final) || (c->nsteps > 0 && c->step >= c->nsteps)) {
        c->done = 1;
        c->dt = 0.0;
        return;
    }
    double dt;
    if (b.dt_fixed > 0.0) {
        dt = b.dt_fixed;
    } else if (c->dt_fixed > 0.0) {
        dt = c->dt_fixed;
    } else {
        dt = it.cfl * 2.0 / (n * lc);
        if (lv > 0.0) {
            double n4 = (double)n * n * n * n;
            double dtv = 12.0 / (n4 * lv);
            dt = fmin(dt, dtv);
        }
    }
    if (!(dt > 0.0) || c->bad) {   // NaN or non-physical state
        c->bad = 1;
        c->done = 1;
        c->dt = 0.0;
        return;
    }
    bool last = false;
    if (c->t_final > 0.0 && c->t + dt >= c->t_final) {
        dt = c->t_final - c->t;
        last = true;
    }
    c->dt = dt;
    c->t = last ? c->t_final : c->t + dt;
    c->step += 1;
}

// dt only (no clock update): writes the rule's dt to out and resets the maxima.
__global__ void k_dt_value(Clock *c, int n, double cfl, double *out)
{
    double lc = __longlong_as_double((long long)c->lam_c);
    double lv = __longlong_as_double((long long)c->lam_v);
    c->lam_c = 0ull;
    c->lam_v = 0ull;
    double dt = cfl * 2.0 / (n * lc);
    if (lv > 0.0) dt = fmin(dt, 12.0 / ((double)n * n * n * n * lv));
    *out = dt;
}

cudaError_t launch_lambda(int N, int physics, const Batch &b, cudaStream_t s)
{
    int n3 = (N + 1) * (N + 1) * (N + 1);
    long long total = b.total_elems * n3;
    if (total == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((total + 255) / 256);
    int ns = physics == HS3D_NS;
    switch (N) {
        case 1: k_lambda<1><<<blocks, 256, 0, s>>>(b, ns); break;
        case 2: k_lambda<2><<<blocks, 256, 0, s>>>(b, ns); break;
        case 3: k_lambda<3><<<blocks, 256, 0, s>>>(b, ns); break;
        case 4: k_lambda<4><<<blocks, 256, 0, s>>>(b, ns); break;
        case 5: k_lambda<5><<<blocks, 256, 0, s>>>(b, ns); break;
        case 6: k_lambda<6><<<blocks, 256, 0, s>>>(b, ns); break;
        case 7: k_lambda<7><<<blocks, 256, 0, s>>>(b, ns); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_dt_finalize(int N, const Batch &b, int mode, cudaStream_t s)
{
    if (mode == 2) {   // dt value of a single item into b.single.out
        k_dt_value<<<1, 1, 0, s>>>(b.single.clk, N + 1, b.single.cfl, b.single.out);
        return cudaGetLastError();
    }
    unsigned blocks = (unsigned)((b.nitems + 127) / 128);
    k_dt_finalize<<<blocks, 128, 0, s>>>(b, N + 1, mode);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ diagnostics

constexpr int kDiagThreads = 256;

int diagnostics_blocks(int N, int E)
{
    long long total = (long long)E * (N + 1) * (N + 1) * (N + 1);
    long long blocks = (total + kDiagThreads * 8 - 1) / (kDiagThreads * 8);
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// Fixed-order block reduction of 7 values per thread.
__device__ void block_sum7(double v[7], double *sm)
{
    for (int k = 0; k < 7; ++k) sm[k * kDiagThreads + threadIdx.x] = v[k];
    __syncthreads();
    for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int k = 0; k < 7; ++k) sm[k * kDiagThreads + threadIdx.x] += sm[k * kDiagThreads + threadIdx.x + w];
        __syncthreads();
    }
    for (int k = 0; k < 7; ++k) v[k] = sm[k * kDiagThreads];
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(int n, Item it, const double *__restrict__ dudt,
                                                                const Ops *__restrict__ ops, double *partials)
{
    __shared__ double sm[7 * kDiagThreads];
    const int n3 = n * n * n;
    const long long total = (long long)it.E * n3;
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    const long long begin = blockIdx.x * per, end = min(total, begin + per);
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    const double g = it.gamma;
    for (long long t = begin + threadIdx.x; t < end; t += blockDim.x) {
        const long long e = t / n3;
        const int p = (int)(t - e * n3);
        const int i = p % n, j = (p / n) % n, k = p / (n * n);
        const double wq = it.J[e * n3 + p] * ops->w[i] * ops->w[j] * ops->w[k];
        const double *U = it.u + e * 5 * n3 + p;
        if (dudt) {
            const double *R = dudt + e * 5 * n3 + p;
            double u[5], r[5];
            for (int v = 0; v < 5; ++v) {
                u[v] = U[v * n3];
                r[v] = R[v * n3];
                acc[v] += wq * r[v];
            }
            double ir = 1.0 / u[0];
            double v1 = u[1] * ir, v2 = u[2] * ir, v3 = u[3] * ir;
            double vv = v1 * v1 + v2 * v2 + v3 * v3;
            double pr = (g - 1.0) * (u[4] - 0.5 * u[0] * vv);
            double s = log(pr) - g * log(u[0]);
            double rp = (g - 1.0) * u[0] / pr;
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
    block_sum7(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) partials[blockIdx.x * 7 + k] = acc[k];
}

__global__ void __launch_bounds__(kDiagThreads) k_diag_final(const double *partials, int nblocks, double *out)
{
    __shared__ double sm[7 * kDiagThreads];
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int k = 0; k < 7; ++k) acc[k] += partials[b * 7 + k];
    block_sum7(acc, sm);
    if (threadIdx.x == 0)
        for (int k = 0; k < 7; ++k) out[k] = acc[k];
}

cudaError_t launch_diagnostics(int N, const Item &it, const double *dudt, double *partials, int nblocks, double *out,
                               cudaStream_t s)
{
    const Ops *ops = device_ops(N);
    if (!ops) return cudaErrorMemoryAllocation;
    k_diag_partial<<<nblocks, kDiagThreads, 0, s>>>(N + 1, it, dudt, ops, partials);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_diag_final<<<1, kDiagThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace hs3d
