// Element-kernel dispatch: launch shape table, low-storage RK coefficients,
// and the choice of the per-volume-form kernel family (volume_<form>.cu,
// all instantiated from volume_kernel.cuh).
#include "internal.cuh"

namespace hs3d {

template <int FORM>
cudaError_t launch_volume_form(int N, int prec, int physics, const Batch &b, int stage, double rkA, double rkB,
                               int lam_slot, cudaStream_t s);
template <int FORM>
cudaError_t prepare_volume_form(int N);
template <int FORM>
cudaError_t launch_volume_dev_form(int N, int physics, const Batch &b, int stage, double rkA, double rkB,
                                   int lam_slot, cudaStream_t s);
template <int FORM>
cudaError_t prepare_volume_dev_form(int N);

// Low-storage Runge-Kutta schemes of Sec. 3.7, stage k: g <- A_k g + dt R,
// u <- u + B_k g.  Williamson (1980) three-stage third order; Carpenter and
// Kennedy (1994) five-stage fourth order (NASA TM 109112, their fourth-order
// 2N-storage solution).
static const double kRK3A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double kRK3B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
static const double kRK4A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double kRK4B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                2277821191437.0 / 14882151754819.0};

int rk_stages(int scheme) { return scheme == HS3D_TIME_RK4 ? 5 : 3; }

void rk_coeffs(int scheme, int k, double *A, double *B)
{
    const bool four = scheme == HS3D_TIME_RK4;
    *A = four ? kRK4A[k] : kRK3A[k];
    *B = four ? kRK4B[k] : kRK3B[k];
}

// Tuned elements per CTA by (N, precision FP64 / mixed, kernel).
static int g_epb[kMaxn + 1][2][2] = {};

// (HS3D_MIXED_TC runs the MIXED32 kernels and shares their slot)
static int prec_slot(int prec) { return prec == HS3D_FP64 ? 0 : 1; }

int tuned_elems_per_block(int N, int prec, int which) { return g_epb[N][prec_slot(prec)][which]; }

int elems_per_block_p(int N, int prec, int which)
{
    int v = g_epb[N][prec_slot(prec)][which];
    if (v > 0) return v;
    int n3 = (N + 1) * (N + 1) * (N + 1);
    int e = 256 / n3;
    return e < 1 ? 1 : e;
}

void set_elems_per_block_p(int N, int prec, int which, int epb) { g_epb[N][prec_slot(prec)][which] = epb; }

cudaError_t prepare_volume(int N)
{
    cudaError_t e = prepare_volume_form<HS3D_VOL_STANDARD>(N);
    if (e == cudaSuccess) e = prepare_volume_form<HS3D_VOL_EC>(N);
    if (e == cudaSuccess) e = prepare_volume_form<HS3D_VOL_KG>(N);
    if (e == cudaSuccess) e = prepare_volume_form<HS3D_VOL_PIROZZOLI>(N);
    if (e == cudaSuccess) e = prepare_volume_form<HS3D_VOL_DUCROS>(N);
    if (e == cudaSuccess) e = prepare_volume_form<HS3D_VOL_MORINISHI>(N);
    if (e == cudaSuccess) e = prepare_volume_form<HS3D_VOL_IR>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_STANDARD>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_EC>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_KG>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_PIROZZOLI>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_DUCROS>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_MORINISHI>(N);
    if (e == cudaSuccess) e = prepare_volume_dev_form<HS3D_VOL_IR>(N);
    return e;
}

cudaError_t launch_volume(int N, int prec, int physics, int form, int scheme, const Batch &b, int stage, int lam_slot,
                          cudaStream_t s)
{
    double A = 0.0, B = 0.0;
    if (stage >= 0) {
        if (stage >= rk_stages(scheme)) return cudaErrorInvalidValue;
        rk_coeffs(scheme, stage, &A, &B);
    }
    if (b.gauss) {
        if (form != HS3D_VOL_STANDARD) return cudaErrorInvalidValue;
        return launch_volume_gauss(N, prec, physics, b, stage, A, B, lam_slot, s);
    }
    if (prec != HS3D_FP64) {
        // mixed path: FP32 flux arithmetic on deviations (volume_dev.cuh)
        switch (form) {
            case HS3D_VOL_STANDARD:
                return launch_volume_dev_form<HS3D_VOL_STANDARD>(N, physics, b, stage, A, B, lam_slot, s);
            case HS3D_VOL_EC: return launch_volume_dev_form<HS3D_VOL_EC>(N, physics, b, stage, A, B, lam_slot, s);
            case HS3D_VOL_KG: return launch_volume_dev_form<HS3D_VOL_KG>(N, physics, b, stage, A, B, lam_slot, s);
            case HS3D_VOL_PIROZZOLI:
                return launch_volume_dev_form<HS3D_VOL_PIROZZOLI>(N, physics, b, stage, A, B, lam_slot, s);
            case HS3D_VOL_DUCROS: return launch_volume_dev_form<HS3D_VOL_DUCROS>(N, physics, b, stage, A, B, lam_slot, s);
            case HS3D_VOL_MORINISHI:
                return launch_volume_dev_form<HS3D_VOL_MORINISHI>(N, physics, b, stage, A, B, lam_slot, s);
            case HS3D_VOL_IR: return launch_volume_dev_form<HS3D_VOL_IR>(N, physics, b, stage, A, B, lam_slot, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (form) {
        case HS3D_VOL_STANDARD:
            return launch_volume_form<HS3D_VOL_STANDARD>(N, prec, physics, b, stage, A, B, lam_slot, s);
        case HS3D_VOL_EC: return launch_volume_form<HS3D_VOL_EC>(N, prec, physics, b, stage, A, B, lam_slot, s);
        case HS3D_VOL_KG: return launch_volume_form<HS3D_VOL_KG>(N, prec, physics, b, stage, A, B, lam_slot, s);
        case HS3D_VOL_PIROZZOLI:
            return launch_volume_form<HS3D_VOL_PIROZZOLI>(N, prec, physics, b, stage, A, B, lam_slot, s);
        case HS3D_VOL_DUCROS:
            return launch_volume_form<HS3D_VOL_DUCROS>(N, prec, physics, b, stage, A, B, lam_slot, s);
        case HS3D_VOL_MORINISHI:
            return launch_volume_form<HS3D_VOL_MORINISHI>(N, prec, physics, b, stage, A, B, lam_slot, s);
        case HS3D_VOL_IR: return launch_volume_form<HS3D_VOL_IR>(N, prec, physics, b, stage, A, B, lam_slot, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs3d
