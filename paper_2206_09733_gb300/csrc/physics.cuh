// Point-wise physics of the compressible Euler / Navier-Stokes equations,
// templated on the arithmetic type R (double, or float in the mixed path).
//
//   conserved u = (rho, rho v, rho e), p = (gamma-1)(rho e - rho|v|^2/2)
//   Euler flux F_e.a = (rho v.a, rho v v.a + p a, (rho e + p) v.a)      (Sec. 3.2)
//   viscous flux with tau = mu(grad v + grad v^T) - 2/3 mu I div v and the
//   heat flux kappa grad T                                             (Sec. 3.2, Eq. viscousfluxes)
//   surface fluxes Lax-Friedrichs, Roe, central EC (Sec. 3.3 list)
//   two-point fluxes of the split forms (Sec. 3.5): Chandrashekar,
//   Kennedy-Gruber, Pirozzoli, Ducros
#pragma once

#include <cuda_runtime.h>

#include "../../include/hs3d.h"

namespace hs3d {

template <typename R>
struct Prim {
    R rho, v1, v2, v3, p, E;   // E = rho e, the conserved total energy
};

// FP64 -> FP32 with round-to-nearest-even, on the integer pipe.  On this GPU
// every FP64-pipe instruction (conversions included) costs as much issue
// bandwidth as ~64 FP32 ones, so the mixed path rounds its FP64 inputs with
// bit operations on the IEEE-754 encodings instead: sign kept; the 52-bit
// significand cut to 23 bits, rounding on the 29 dropped bits (ties to even,
// a carry may step into the exponent); exponent rebased from 1023 to 127.
// Results below the smallest normal FP32 are flushed to signed zero (the
// state never holds such values), above the largest become infinity, NaN
// stays NaN.
__device__ __forceinline__ float d2f_rn(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu);
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rest = lo & 0x1fffffffu;
    const int ef = e - 1023 + 127;
    if (e == 0x7ff) return __int_as_float((int)(sign | 0x7f800000u | ((m | rest) ? 0x400000u : 0u)));
    if (ef <= 0) return __int_as_float((int)sign);
    if (ef >= 255) return __int_as_float((int)(sign | 0x7f800000u));
    unsigned r = ((unsigned)ef << 23) | m;
    if (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) r += 1u;
    return __int_as_float((int)(sign | r));
}

// FP32 -> FP64 (exact) on the integer pipe; FP32 subnormals become zero.
__device__ __forceinline__ double f2d_exact(float x);
template <typename R>
__device__ __forceinline__ double widen(R x);
template <>
__device__ __forceinline__ double widen<double>(double x) { return x; }
template <>
__device__ __forceinline__ double widen<float>(float x) { return f2d_exact(x); }
template <typename R>
__device__ __forceinline__ R narrow(double x);
template <>
__device__ __forceinline__ double narrow<double>(double x) { return x; }
template <>
__device__ __forceinline__ float narrow<float>(double x) { return d2f_rn(x); }

__device__ __forceinline__ double f2d_exact(float x)
{
    const unsigned b = (unsigned)__float_as_int(x);
    const unsigned sign = b & 0x80000000u;
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned m = b & 0x7fffffu;
    unsigned hi;
    if (e == 0) hi = sign;
    else if (e == 0xff) hi = sign | 0x7ff00000u | (m >> 3);
    else hi = sign | ((e - 127u + 1023u) << 20) | (m >> 3);
    const unsigned lo = (e == 0) ? 0u : (m << 29);
    return __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
}

// Primitive variables from the FP64 conserved state.  FP64 path: in FP64.
// Mixed path: the state is rounded to FP32 once (d2f_rn) and the primitives
// computed in FP32 (at Mach 0.1, rho e / p ~ 2.5, so the subtraction loses no
// more than rounding p itself to FP32 would).
template <typename R>
__device__ __forceinline__ Prim<R> prim_from_u(const double u[5], R gm1);

template <>
__device__ __forceinline__ Prim<double> prim_from_u<double>(const double u[5], double gm1)
{
    double ir = 1.0 / u[0];
    double v1 = u[1] * ir, v2 = u[2] * ir, v3 = u[3] * ir;
    Prim<double> q;
    q.rho = u[0];
    q.v1 = v1;
    q.v2 = v2;
    q.v3 = v3;
    q.p = gm1 * (u[4] - 0.5 * (u[1] * v1 + u[2] * v2 + u[3] * v3));
    q.E = u[4];
    return q;
}

// Primitive variables from a state already rounded to FP32.
__device__ __forceinline__ Prim<float> prim_from_f(const float uf[5], float gm1)
{
    const float r = uf[0], m1 = uf[1], m2 = uf[2], m3 = uf[3], E = uf[4];
    const float ir = __frcp_rn(r);
    Prim<float> q;
    q.rho = r;
    q.v1 = m1 * ir;
    q.v2 = m2 * ir;
    q.v3 = m3 * ir;
    q.p = gm1 * (E - 0.5f * (m1 * q.v1 + m2 * q.v2 + m3 * q.v3));
    q.E = E;
    return q;
}

template <>
__device__ __forceinline__ Prim<float> prim_from_u<float>(const double u[5], float gm1)
{
    const float uf[5] = {d2f_rn(u[0]), d2f_rn(u[1]), d2f_rn(u[2]), d2f_rn(u[3]), d2f_rn(u[4])};
    return prim_from_f(uf, gm1);
}

template <typename R>
__device__ __forceinline__ R rsqrt_(R x);
template <>
__device__ __forceinline__ double rsqrt_<double>(double x) { return 1.0 / sqrt(x); }
template <>
__device__ __forceinline__ float rsqrt_<float>(float x) { return rsqrtf(x); }

template <typename R>
__device__ __forceinline__ R log_(R x);
template <>
__device__ __forceinline__ double log_<double>(double x) { return log(x); }
template <>
__device__ __forceinline__ float log_<float>(float x) { return logf(x); }

// Euler flux dotted with a (any vector); E = rho e.
template <typename R>
__device__ __forceinline__ void euler_flux(const Prim<R> &q, R E, R a1, R a2, R a3, R f[5])
{
    R va = q.v1 * a1 + q.v2 * a2 + q.v3 * a3;
    R m = q.rho * va;
    f[0] = m;
    f[1] = m * q.v1 + q.p * a1;
    f[2] = m * q.v2 + q.p * a2;
    f[3] = m * q.v3 + q.p * a3;
    f[4] = (E + q.p) * va;
}

// Viscous flux dotted with a.  G[v*3 + c] = d q_v / d x_c for q = (v1,v2,v3,T).
template <typename R>
__device__ __forceinline__ void visc_flux(const Prim<R> &q, const R G[12], R mu, R kappa, R a1, R a2, R a3,
                                          R f[5])
{
    R div = G[0] + G[4] + G[8];
    R l = (R)(2.0 / 3.0) * mu * div;
    R t11 = mu * (G[0] + G[0]) - l;
    R t22 = mu * (G[4] + G[4]) - l;
    R t33 = mu * (G[8] + G[8]) - l;
    R t12 = mu * (G[1] + G[3]);
    R t13 = mu * (G[2] + G[6]);
    R t23 = mu * (G[5] + G[7]);
    R s1 = t11 * a1 + t12 * a2 + t13 * a3;
    R s2 = t12 * a1 + t22 * a2 + t23 * a3;
    R s3 = t13 * a1 + t23 * a2 + t33 * a3;
    f[0] = (R)0;
    f[1] = s1;
    f[2] = s2;
    f[3] = s3;
    f[4] = q.v1 * s1 + q.v2 * s2 + q.v3 * s3 + kappa * (G[9] * a1 + G[10] * a2 + G[11] * a3);
}

// Lax-Friedrichs flux times the face scale s = |Sn|, Sn the scaled normal
// pointing from L to R:  s [ (F_L + F_R).n/2 - lambda (u_R - u_L)/2 ],
// lambda = max(|v_L.n| + c_L, |v_R.n| + c_R).
template <typename R>
__device__ __forceinline__ void flux_lf(const Prim<R> &L, const R uL[5], const Prim<R> &Rr, const R uR[5], R gamma,
                                        R s1, R s2, R s3, R f[5])
{
    R s = sqrt(s1 * s1 + s2 * s2 + s3 * s3);
    R fl[5], fr[5];
    euler_flux(L, uL[4], s1, s2, s3, fl);
    euler_flux(Rr, uR[4], s1, s2, s3, fr);
    R vnL = fabs(L.v1 * s1 + L.v2 * s2 + L.v3 * s3) + s * sqrt(gamma * L.p / L.rho);
    R vnR = fabs(Rr.v1 * s1 + Rr.v2 * s2 + Rr.v3 * s3) + s * sqrt(gamma * Rr.p / Rr.rho);
    R lam = fmax(vnL, vnR);    // = s * lambda
#pragma unroll
    for (int v = 0; v < 5; ++v) f[v] = (R)0.5 * (fl[v] + fr[v]) - (R)0.5 * lam * (uR[v] - uL[v]);
}

// Roe flux times the face scale (Roe 1981, sqrt(rho)-weighted averages, no
// entropy fix): s [ (F_L + F_R).n/2 - sum_k |lambda_k| alpha_k r_k / 2 ].
template <typename R>
__device__ __forceinline__ void flux_roe(const Prim<R> &L, const R uL[5], const Prim<R> &Rr, const R uR[5], R gamma,
                                         R s1, R s2, R s3, R f[5])
{
    R s = sqrt(s1 * s1 + s2 * s2 + s3 * s3);
    R is = (R)1 / s;
    R n1 = s1 * is, n2 = s2 * is, n3 = s3 * is;
    R fl[5], fr[5];
    euler_flux(L, uL[4], s1, s2, s3, fl);
    euler_flux(Rr, uR[4], s1, s2, s3, fr);
    R sl = sqrt(L.rho), sr = sqrt(Rr.rho);
    R iw = (R)1 / (sl + sr);
    R HL = (uL[4] + L.p) / L.rho, HR = (uR[4] + Rr.p) / Rr.rho;
    R vt1 = (sl * L.v1 + sr * Rr.v1) * iw;
    R vt2 = (sl * L.v2 + sr * Rr.v2) * iw;
    R vt3 = (sl * L.v3 + sr * Rr.v3) * iw;
    R Ht = (sl * HL + sr * HR) * iw;
    R q2 = vt1 * vt1 + vt2 * vt2 + vt3 * vt3;
    R c2 = (gamma - (R)1) * (Ht - (R)0.5 * q2);
    R ct = sqrt(c2);
    R ic2 = (R)1 / c2;
    R rt = sl * sr;
    R vnt = vt1 * n1 + vt2 * n2 + vt3 * n3;
    R dr = Rr.rho - L.rho, dp = Rr.p - L.p;
    R d1 = Rr.v1 - L.v1, d2 = Rr.v2 - L.v2, d3 = Rr.v3 - L.v3;
    R dvn = d1 * n1 + d2 * n2 + d3 * n3;
    R a1 = (dp - rt * ct * dvn) * (R)0.5 * ic2;
    R a5 = (dp + rt * ct * dvn) * (R)0.5 * ic2;
    R a2 = dr - dp * ic2;
    R sh1 = rt * (d1 - dvn * n1), sh2 = rt * (d2 - dvn * n2), sh3 = rt * (d3 - dvn * n3);
    R l1 = fabs(vnt - ct) * a1, l2 = fabs(vnt), l5 = fabs(vnt + ct) * a5;
    R W0 = l1 + l2 * a2 + l5;
    R W1 = l1 * (vt1 - ct * n1) + l2 * (a2 * vt1 + sh1) + l5 * (vt1 + ct * n1);
    R W2 = l1 * (vt2 - ct * n2) + l2 * (a2 * vt2 + sh2) + l5 * (vt2 + ct * n2);
    R W3 = l1 * (vt3 - ct * n3) + l2 * (a2 * vt3 + sh3) + l5 * (vt3 + ct * n3);
    R W4 = l1 * (Ht - ct * vnt) + l2 * (a2 * (R)0.5 * q2 + vt1 * sh1 + vt2 * sh2 + vt3 * sh3) + l5 * (Ht + ct * vnt);
    R hs = (R)0.5 * s;
    f[0] = (R)0.5 * (fl[0] + fr[0]) - hs * W0;
    f[1] = (R)0.5 * (fl[1] + fr[1]) - hs * W1;
    f[2] = (R)0.5 * (fl[2] + fr[2]) - hs * W2;
    f[3] = (R)0.5 * (fl[3] + fr[3]) - hs * W3;
    f[4] = (R)0.5 * (fl[4] + fr[4]) - hs * W4;
}

template <typename R>
struct LogMeanEps;
template <>
struct LogMeanEps<double> {
    static constexpr double v = 1e-4;
};
template <>
struct LogMeanEps<float> {
    static constexpr float v = 1e-2f;
};

template <typename R>
__device__ __forceinline__ R rcp_(R x);
template <>
__device__ __forceinline__ double rcp_<double>(double x) { return 1.0 / x; }
template <>
__device__ __forceinline__ float rcp_<float>(float x) { return __frcp_rn(x); }

// Per-node quantities the Chandrashekar flux uses.
template <typename R>
struct ECNode {
    R rho, v1, v2, v3, beta, lrho, lbeta;
};

template <typename R>
__device__ __forceinline__ ECNode<R> ec_node(const Prim<R> &q)
{
    ECNode<R> z;
    z.rho = q.rho;
    z.v1 = q.v1;
    z.v2 = q.v2;
    z.v3 = q.v3;
    z.beta = q.rho / ((R)2 * q.p);
    z.lrho = log_(q.rho);
    z.lbeta = log_(z.beta);
    return z;
}

// Chandrashekar's entropy-conservative, kinetic-energy-preserving flux dotted
// with a:  beta = rho/(2p), rho^ and beta^ logarithmic means, {.} arithmetic
// means, p~ = {rho}/(2{beta}),
//   f_rho = rho^ {v}.a,  f_m = f_rho {v} + p~ a,
//   f_E = f_rho (1/(2(gamma-1) beta^) - {|v|^2}/2) + {v}.f_m.
// Logarithmic mean L(a,b) = (a-b)/(ln a - ln b) with the logarithms taken per
// node; near a = b (u = ((a-b)/(a+b))^2 below LogMeanEps) the Ismail-Roe
// series L = (a+b)/(2F), F = 1 + u/3 + u^2/5 + u^3/7, is used: for rho^ as
// (a+b)/2 times the series of 1/F to the same order (1 - u/3 - 4u^2/45 -
// 44u^3/945), for 1/beta^ directly as 2F/(a+b).  Only the two reciprocals
// 1/(rho_L+rho_R) and 1/(beta_L+beta_R) are needed on that branch;
// hg = 1/(2(gamma-1)).
template <typename R>
__device__ __forceinline__ void flux_ec(const ECNode<R> &L, const ECNode<R> &Rr, R hg, R a1, R a2, R a3, R f[5])
{
    const R srho = L.rho + Rr.rho, sbeta = L.beta + Rr.beta;
    const R irho = rcp_(srho), ibeta = rcp_(sbeta);
    const R dr = L.rho - Rr.rho;
    const R fr = dr * irho, ur = fr * fr;
    R rho_ln;
    if (ur < LogMeanEps<R>::v)
        rho_ln = (R)0.5 * srho * ((R)1 - ur * ((R)(1.0 / 3.0) + ur * ((R)(4.0 / 45.0) + ur * (R)(44.0 / 945.0))));
    else
        rho_ln = dr / (L.lrho - Rr.lrho);
    const R db = L.beta - Rr.beta;
    const R fb = db * ibeta, ub = fb * fb;
    R ibeta_ln;
    if (ub < LogMeanEps<R>::v)
        ibeta_ln = (R)2 * ibeta * ((R)1 + ub * ((R)(1.0 / 3.0) + ub * ((R)0.2 + ub * (R)(1.0 / 7.0))));
    else
        ibeta_ln = (L.lbeta - Rr.lbeta) / db;
    const R m1 = (R)0.5 * (L.v1 + Rr.v1), m2 = (R)0.5 * (L.v2 + Rr.v2), m3 = (R)0.5 * (L.v3 + Rr.v3);
    const R v2 =
        (R)0.5 * ((L.v1 * L.v1 + L.v2 * L.v2 + L.v3 * L.v3) + (Rr.v1 * Rr.v1 + Rr.v2 * Rr.v2 + Rr.v3 * Rr.v3));
    const R pt = (R)0.5 * srho * ibeta;
    const R fm = rho_ln * (m1 * a1 + m2 * a2 + m3 * a3);
    f[0] = fm;
    f[1] = fm * m1 + pt * a1;
    f[2] = fm * m2 + pt * a2;
    f[3] = fm * m3 + pt * a3;
    f[4] = fm * (hg * ibeta_ln - (R)0.5 * v2) + m1 * f[1] + m2 * f[2] + m3 * f[3];
}

// ------------------------------------------------------------------ split forms
//
// Per-node inputs of the two-point fluxes, kSplitSlots values per node:
//   EC         rho, v1, v2, v3, beta = rho/(2p), ln rho, ln beta
//   KG         rho, v1, v2, v3, p, e = (rho e)/rho
//   PIROZZOLI  rho, v1, v2, v3, p, h = (rho e + p)/rho
//   DUCROS     rho, v1, v2, v3, p, rho e + p
// (the average-product forms leave the seventh slot unused).
constexpr int kSplitSlots = 7;

template <int FORM, typename R>
__device__ __forceinline__ void split_node(const Prim<R> &q, R z[kSplitSlots])
{
    z[0] = q.rho;
    z[1] = q.v1;
    z[2] = q.v2;
    z[3] = q.v3;
    if constexpr (FORM == HS3D_VOL_EC) {
        const ECNode<R> c = ec_node(q);
        z[4] = c.beta;
        z[5] = c.lrho;
        z[6] = c.lbeta;
    } else {
        z[4] = q.p;
        if constexpr (FORM == HS3D_VOL_KG) z[5] = q.E / q.rho;
        else if constexpr (FORM == HS3D_VOL_PIROZZOLI) z[5] = (q.E + q.p) / q.rho;
        else z[5] = q.E + q.p;
        z[6] = (R)0;
    }
}

// Average-product two-point fluxes dotted with a = (a1, a2, a3), {x} = (x_L + x_R)/2,
// v_a = v.a, m = {rho}{v_a}:
//   KG         (m, m{v} + {p}a, m{e} + {p}{v_a})
//   PIROZZOLI  (m, m{v} + {p}a, m{h})
//   DUCROS     ({rho}{v_a}, {rho v}{v_a} + {p}a, {rho e + p}{v_a})
template <int FORM, typename R>
__device__ __forceinline__ void flux_avg_product(const R *L, const R *Rr, R a1, R a2, R a3, R f[5])
{
    const R h = (R)0.5;
    const R vaL = L[1] * a1 + L[2] * a2 + L[3] * a3;
    const R vaR = Rr[1] * a1 + Rr[2] * a2 + Rr[3] * a3;
    const R va = h * (vaL + vaR);
    const R rho = h * (L[0] + Rr[0]);
    const R pav = h * (L[4] + Rr[4]);
    const R m = rho * va;
    f[0] = m;
    if constexpr (FORM == HS3D_VOL_DUCROS) {
        f[1] = h * (L[0] * L[1] + Rr[0] * Rr[1]) * va + pav * a1;
        f[2] = h * (L[0] * L[2] + Rr[0] * Rr[2]) * va + pav * a2;
        f[3] = h * (L[0] * L[3] + Rr[0] * Rr[3]) * va + pav * a3;
        f[4] = h * (L[5] + Rr[5]) * va;
    } else {
        f[1] = m * (h * (L[1] + Rr[1])) + pav * a1;
        f[2] = m * (h * (L[2] + Rr[2])) + pav * a2;
        f[3] = m * (h * (L[3] + Rr[3])) + pav * a3;
        if constexpr (FORM == HS3D_VOL_KG) f[4] = m * (h * (L[5] + Rr[5])) + pav * va;
        else f[4] = m * (h * (L[5] + Rr[5]));
    }
}

template <int FORM, typename R>
__device__ __forceinline__ void split_pair(const R *L, const R *Rr, R hg, R a1, R a2, R a3, R f[5])
{
    if constexpr (FORM == HS3D_VOL_EC) {
        const ECNode<R> zl = {L[0], L[1], L[2], L[3], L[4], L[5], L[6]};
        const ECNode<R> zr = {Rr[0], Rr[1], Rr[2], Rr[3], Rr[4], Rr[5], Rr[6]};
        flux_ec(zl, zr, hg, a1, a2, a3, f);
    } else {
        flux_avg_product<FORM>(L, Rr, a1, a2, a3, f);
    }
}

}  // namespace hs3d
