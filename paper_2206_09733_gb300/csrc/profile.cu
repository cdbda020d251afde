// Instrumentation entry points: per-kernel timing of one RK step and
// FMA-chain measurements of the FP64 / FP32 arithmetic peaks.
#include <string.h>

#include "api_internal.h"
#include "lowmach.cuh"
#include "physics.cuh"

namespace hs3d {

// Independent FMA chains per thread, long enough to hide the pipe latency.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_chain(T *out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)12345.678) out[threadIdx.x] = s;   // keep the chains alive
}

template <typename T>
static double fma_tflops(int sms, int iters, cudaStream_t s, cudaError_t &err)
{
    T *out = nullptr;
    err = cudaMalloc(&out, 256 * sizeof(T));
    if (err != cudaSuccess) return 0.0;
    int blocks = sms * 8;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chain<T><<<blocks, 256, 0, s>>>(out, iters / 4, (T)0.999, (T)0.001);   // warm-up
    cudaEventRecord(e0, s);
    k_fma_chain<T><<<blocks, 256, 0, s>>>(out, iters, (T)0.999, (T)0.001);
    cudaEventRecord(e1, s);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    double flops = 2.0 * 8.0 * (double)iters * blocks * 256.0;
    return flops / (ms * 1e-3) / 1e12;
}

// Compare the integer-pipe conversions with the hardware ones on n inputs:
// counts[0] = d2f_rn(x) differs bitwise from __double2float_rn(x) for x in
// the normal FP32 range or NaN/infinite, counts[1] = f2d_exact(f) differs from
// (double)f for f = __double2float_rn(x), counts[2] = inputs below the FP32
// normal range (flushed to zero by d2f_rn by design).
__global__ void k_check_rounding(const double *in, long long n, unsigned long long *counts)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = in[i];
    const float hw = __double2float_rn(x);
    const float sw = d2f_rn(x);
    const bool tiny = fabs(x) < 1.1754943508222875e-38 && x != 0.0;
    if (tiny) {
        atomicAdd(&counts[2], 1ull);
    } else {
        const bool both_nan = (hw != hw) && (sw != sw);
        if (!both_nan && __float_as_int(hw) != __float_as_int(sw)) atomicAdd(&counts[0], 1ull);
    }
    if (hw == hw && fabsf(hw) >= 1.17549435e-38f) {
        const double a = f2d_exact(hw), b = (double)hw;
        if (__double_as_longlong(a) != __double_as_longlong(b)) atomicAdd(&counts[1], 1ull);
    }
    const double ax = fabs(x);
    if (ax >= 5.293955920339377e-23 && ax < 1.7014118346046923e38) {   // 2^-74 .. 2^127
        float hi, lo;
        ff_split(x, hi, lo);
        const float ref = __double2float_rn(x - (double)hi);
        if (__float_as_int(lo) != __float_as_int(ref) && !(lo == 0.0f && ref == 0.0f)) atomicAdd(&counts[3], 1ull);
    }
}

}  // namespace hs3d

using namespace hs3d;

extern "C" hs3d_status hs3d_check_rounding(const double *in, int64_t n, unsigned long long *counts, void *stream)
{
    if (!in || !counts || n < 0) return fail(HS3D_ERR_INVALID, "bad arguments");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), s);
    if (e == cudaSuccess && n > 0) {
        k_check_rounding<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, n, counts);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "rounding check");
}

extern "C" {

hs3d_status hs3d_alu_peaks(double *tflops_out, void *stream)
{
    if (!tflops_out) return fail(HS3D_ERR_INVALID, "tflops_out is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    cudaStream_t s = (cudaStream_t)stream;
    tflops_out[0] = fma_tflops<double>(sms, 1 << 12, s, e);
    if (e == cudaSuccess) tflops_out[1] = fma_tflops<float>(sms, 1 << 16, s, e);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "fma chain kernel");
}

hs3d_status hs3d_rk3_step_profiled(const hs3d_mesh *m, const hs3d_solver_cfg *c, double *u, double *g, double dt,
                                   double *ms_out, void *stream)
{
    if (!m || !ms_out) return fail(HS3D_ERR_INVALID, "mesh or ms_out is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK) st = check_mesh_cfg(m, c);
    if (st != HS3D_OK) return st;
    if (!u || !g || u == g) return fail(HS3D_ERR_INVALID, "bad u/g");
    cudaStream_t s = (cudaStream_t)stream;
    const int ns = rk_stages(c->time_scheme);
    const int NEV = 2 + 3 * 5;
    cudaEvent_t ev[NEV];
    for (int k = 0; k < NEV; ++k) cudaEventCreate(&ev[k]);
    Batch b = single_batch(make_item(m, c, u, g, nullptr));
    b.dt_fixed = dt > 0.0 ? dt : 0.0;
    cudaError_t e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess && !(dt > 0.0)) e = launch_lambda(m->N, c->precision, c->physics, b, 0, s);
    else if (e == cudaSuccess && c->precision != HS3D_FP64) e = launch_shadow(m->N, b, s);
    if (e == cudaSuccess) e = launch_dt_finalize(m->N, b, 0, 0, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    int k = 2;
    for (int stage = 0; stage < ns && e == cudaSuccess; ++stage) {
        if (c->physics == HS3D_NS) e = launch_grad(m->N, c->precision, b, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k++], s);
        if (e == cudaSuccess) e = launch_face(m->N, c->precision, c->physics, c->surface_flux, b, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k++], s);
        if (e == cudaSuccess)
            e = launch_volume(m->N, c->precision, c->physics, c->volume_form, c->time_scheme, b, stage,
                              stage == ns - 1 ? 1 : -1, s);
        if (e == cudaSuccess) e = cudaEventRecord(ev[k++], s);
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[k - 1]);
    if (e == cudaSuccess) {
        float t;
        memset(ms_out, 0, sizeof(double) * 5);
        cudaEventElapsedTime(&t, ev[0], ev[1]);
        ms_out[0] = t;
        for (int stage = 0; stage < ns; ++stage) {
            for (int part = 0; part < 3; ++part) {
                cudaEventElapsedTime(&t, ev[1 + stage * 3 + part], ev[2 + stage * 3 + part]);
                ms_out[1 + part] += t;
            }
        }
        cudaEventElapsedTime(&t, ev[0], ev[k - 1]);
        ms_out[4] = t;
    }
    for (int j = 0; j < NEV; ++j) cudaEventDestroy(ev[j]);
    if (e != cudaSuccess) {
        cont_forget(m, nullptr);
        return cuda_fail(e, "profiled step");
    }
    cont_set(m, u, c);
    return HS3D_OK;
}

}  // extern "C"
