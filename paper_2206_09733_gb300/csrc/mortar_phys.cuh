// Point functions of the mortar kernels (mortar.cu, aniso.cu): primitive
// and BR1 gradient variables of a conservative state, and the inviscid
// numerical flux at a mortar point (the conforming face kernel's flux
// functions).
#pragma once

#include "internal.cuh"
#include "mortar.cuh"
#include "physics.cuh"

namespace hs3d {

template <typename R>
__device__ __forceinline__ Prim<R> mortar_prim(const R u[5], R gm1)
{
    if constexpr (sizeof(R) == 8) return prim_from_u<double>((const double *)u, gm1);
    else return prim_from_f((const float *)u, gm1);
}

// BR1 gradient variables q = (v1, v2, v3, T), T = p/rho, of the state
// u[0], u[stride], ..., u[4 stride].
template <typename R>
__device__ __forceinline__ void mortar_q(const R *u, R gm1, R q[4], int stride = 1)
{
    R c[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) c[v] = u[v * stride];
    const Prim<R> w = mortar_prim(c, gm1);
    q[0] = w.v1;
    q[1] = w.v2;
    q[2] = w.v3;
    q[3] = w.p / w.rho;
}

// Inviscid numerical flux times the face scale, from the two conservative
// states at a mortar point (the same flux functions as the conforming face
// kernel).
template <typename R>
__device__ __forceinline__ void mortar_riemann(int flux, const R ul[5], const R ur[5], const MortarPhys<R> &P, R s1,
                                               R s2, R s3, R fs[5])
{
    const Prim<R> qL = mortar_prim(ul, P.gm1), qR = mortar_prim(ur, P.gm1);
    if (flux == HS3D_FLUX_EC) {
        flux_ec(ec_node(qL), ec_node(qR), P.hg, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_LF) {
        flux_lf(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_RUSANOV) {
        flux_rusanov(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_MATRIX) {
        flux_matrix(qL, qR, P.gamma, P.hg, s1, s2, s3, fs);
    } else {
        const R a[5] = {qL.rho, (R)0, (R)0, (R)0, qL.E};
        const R c[5] = {qR.rho, (R)0, (R)0, (R)0, qR.E};
        if (flux == HS3D_FLUX_LDROE) flux_ldroe(qL, a, qR, c, P.gamma, s1, s2, s3, fs);
        else flux_roe(qL, a, qR, c, P.gamma, s1, s2, s3, fs);
    }
}

}  // namespace hs3d
