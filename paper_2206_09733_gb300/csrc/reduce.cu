// Reductions: the time-step rule and the quadrature diagnostics.
//
// Time step (the paper names explicit RK3 with a CFL condition, Sec. 3.7, but
// gives no formula; this library uses)
//   dt_c = cfl * 8 / (n^2 * max_nodes sum_d (|Ja^d.v| + c |Ja^d|)/J)
//          (the RK3 stability limit of the DGSEM operator shrinks like 1/n^2)
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
#include "lowmach.cuh"
#include "physics.cuh"

namespace hs3d {

template <typename R>
__device__ __forceinline__ const R *lambda_metric(const Item &it);
template <>
__device__ __forceinline__ const double *lambda_metric<double>(const Item &it) { return it.Ja; }
template <>
__device__ __forceinline__ const float *lambda_metric<float>(const Item &it) { return it.Jaf; }

template <int N, typename R>
__global__ void __launch_bounds__(256) k_lambda(const __grid_constant__ Batch b, int ns, int slot)
{
    constexpr int n = N + 1, n3 = n * n * n;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double lc = 0.0, lv = 0.0;
    bool active = false;
    const Item *itp = nullptr;
    if (t < b.total_elems * n3) {
        const long long ge = t / n3;
        const int p = (int)(t - ge * n3);
        itp = &find_item_elem(b, ge);
        const Item &it = *itp;
        const int e = (int)(ge - it.elem_begin);
        const double *U = it.u + (size_t)e * 5 * n3 + p;
        double u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = U[v * n3];
        const Phys<R> P = phys_of<R>(it);
        Prim<R> q;
        if constexpr (sizeof(R) == 8) {
            q = prim_from_u<R>(u, P.gm1);
        } else {
            // the mixed path's dt pass also writes the FP32 shadow of the state
            float us[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) us[v] = d2f_rn(u[v]);
            // the pass before a run also leaves each element's reference state
            if (it.anc && p == anchor_node(n)) write_anchor(it, e, u);
            if (it.uf) {
                float *S = it.uf + (size_t)e * 5 * n3 + p;
#pragma unroll
                for (int v = 0; v < 5; ++v) S[v * n3] = us[v];
            }
            q = prim_from_f(us, P.gm1);
        }
        if (!(q.rho > (R)0) || !(q.p > (R)0)) {
            it.clk->bad = 1;
        } else {
            const R c = sqrt(P.gamma * q.p / q.rho);
            const R *JA = lambda_metric<R>(it) + (size_t)e * 9 * n3 + p;
            R iJ;
            if constexpr (sizeof(R) == 8) iJ = it.invJ[(size_t)e * n3 + p];
            else iJ = it.invJf[(size_t)e * n3 + p];
            R sc = (R)0, sv = (R)0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const R a1 = JA[(d * 3) * n3], a2 = JA[(d * 3 + 1) * n3], a3 = JA[(d * 3 + 2) * n3];
                const R an = sqrt(a1 * a1 + a2 * a2 + a3 * a3);
                sc += (fabs(a1 * q.v1 + a2 * q.v2 + a3 * q.v3) + c * an) * iJ;
                sv += (an * iJ) * (an * iJ);
            }
            lc = widen<R>(sc);
            if (ns) lv = widen<R>(P.mu * sv / q.rho);
            active = true;
        }
    }
    unsigned long long *dc = nullptr, *dv = nullptr;
    if (active) {
        dc = &itp->clk->lam[slot][0];
        dv = ns ? &itp->clk->lam[slot][1] : nullptr;
    }
    warp_max_to_clock(dc, dv, lc, lv, active);
}

// One thread per item: dt from the maxima in clock slot `slot` (or the fixed
// dt), clipped at t_final; advances the clock and resets both maxima slots.
__global__ void k_dt_finalize(const __grid_constant__ Batch b, int n, int slot)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.nitems) return;
    const Item &it = (b.nitems == 1) ? b.single : b.items[i];
    Clock *c = it.clk;
    double lc = __longlong_as_double((long long)c->lam[slot][0]);
    double lv = __longlong_as_double((long long)c->lam[slot][1]);
    c->lam[0][0] = c->lam[0][1] = c->lam[1][0] = c->lam[1][1] = 0ull;
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
        dt = it.cfl * it.kc / ((double)n * n * lc);
        if (lv > 0.0) {
            double n4 = (double)n * n * n * n;
            double dtv = it.kv / (n4 * lv);
            dt = fmin(dt, dtv);
        }
    }
    if (!(dt > 0.0) || c->bad) {   // NaN or non-physical state (or a failed device wait)
        if (!c->bad) c->bad = 1;
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
__global__ void k_dt_value(Clock *c, int n, double cfl, double kc, double kv, double *out)
{
    double lc = __longlong_as_double((long long)c->lam[0][0]);
    double lv = __longlong_as_double((long long)c->lam[0][1]);
    c->lam[0][0] = 0ull;
    c->lam[0][1] = 0ull;
    double dt = cfl * kc / ((double)n * n * lc);
    if (lv > 0.0) dt = fmin(dt, kv / ((double)n * n * n * n * lv));
    *out = dt;
}

cudaError_t launch_lambda(int N, int prec, int physics, const Batch &b, int slot, cudaStream_t s)
{
    int n3 = (N + 1) * (N + 1) * (N + 1);
    long long total = b.total_elems * n3;
    if (total == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((total + 255) / 256);
    int ns = physics == HS3D_NS;
#define HS3D_LAM(K)                                                                                 \
    case K:                                                                                         \
        if (prec == HS3D_FP64) k_lambda<K, double><<<blocks, 256, 0, s>>>(b, ns, slot);             \
        else k_lambda<K, float><<<blocks, 256, 0, s>>>(b, ns, slot);                                \
        break;
    switch (N) {
        HS3D_LAM(1) HS3D_LAM(2) HS3D_LAM(3) HS3D_LAM(4) HS3D_LAM(5) HS3D_LAM(6) HS3D_LAM(7)
        default: return cudaErrorInvalidValue;
    }
#undef HS3D_LAM
    return cudaGetLastError();
}

// n from n^3 (n <= 8).
__device__ __forceinline__ int cbrt_int(int n3) { return n3 <= 8 ? 2 : n3 <= 27 ? 3 : n3 <= 64 ? 4 : n3 <= 125 ? 5 : n3 <= 216 ? 6 : n3 <= 343 ? 7 : 8; }

// FP32 shadow of every item's state (where it has one) and the reference
// state of every element (mixed path), one thread per node.
__global__ void __launch_bounds__(256) k_shadow(const __grid_constant__ Batch b, int n3)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= b.total_elems * n3) return;
    const long long ge = t / n3;
    const int p = (int)(t - ge * n3);
    const Item &it = find_item_elem(b, ge);
    const size_t idx = (size_t)(ge - it.elem_begin) * 5 * n3 + p;
    if (it.anc && p == anchor_node(cbrt_int(n3))) {
        double u[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = it.u[idx + (size_t)v * n3];
        write_anchor(it, (int)(ge - it.elem_begin), u);
    }
    if (!it.uf) return;
#pragma unroll
    for (int v = 0; v < 5; ++v) it.uf[idx + (size_t)v * n3] = d2f_rn(it.u[idx + (size_t)v * n3]);
}

cudaError_t launch_shadow(int N, const Batch &b, cudaStream_t s)
{
    const int n3 = (N + 1) * (N + 1) * (N + 1);
    const long long total = b.total_elems * n3;
    if (total == 0) return cudaSuccess;
    if (b.nitems == 1 && !b.single.uf && !b.single.anc) return cudaSuccess;   // nothing to write on this path
    k_shadow<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(b, n3);
    return cudaGetLastError();
}

cudaError_t launch_dt_finalize(int N, const Batch &b, int mode, int slot, cudaStream_t s)
{
    if (mode == 2) {   // dt value of a single item into b.single.out
        k_dt_value<<<1, 1, 0, s>>>(b.single.clk, N + 1, b.single.cfl, b.single.kc, b.single.kv, b.single.out);
        return cudaGetLastError();
    }
    unsigned blocks = (unsigned)((b.nitems + 127) / 128);
    cudaError_t e = launch_pdl(k_dt_finalize, blocks, 128, 0, s, b, N + 1, slot);
    if (e != cudaSuccess) return e;
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
    const Ops *ops = device_ops(N, it.gauss ? HS3D_NODES_GAUSS : HS3D_NODES_LOBATTO);
    if (!ops) return cudaErrorMemoryAllocation;
    k_diag_partial<<<nblocks, kDiagThreads, 0, s>>>(N + 1, it, dudt, ops, partials);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    k_diag_final<<<1, kDiagThreads, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace hs3d
