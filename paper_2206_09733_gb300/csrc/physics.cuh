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
    // branch-free: the normal-range result is formed unconditionally and the
    // out-of-range cases are selected afterwards
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const unsigned e = (hi >> 20) & 0x7ffu;
    // exponent and the top 23 significand bits, rebased by (1023 - 127) << 23;
    // modulo 2^32 this is exact whenever the FP32 exponent is in range
    unsigned r = __funnelshift_l(lo, hi, 3) - (896u << 23);
    // round to nearest even on the 29 dropped bits: +1 above half, and at
    // exactly half when r is odd
    r += ((lo & 0x1fffffffu) + (r & 1u) + 0x0fffffffu) >> 29;
    const unsigned special = 0x7f800000u | ((e == 0x7ffu && ((hi & 0xfffffu) | lo)) ? 0x400000u : 0u);
    r = (e >= 1151u) ? special : r;   // FP32 exponent >= 255: infinity (NaN for NaN)
    r = (e <= 896u) ? 0u : r;         // FP32 exponent <= 0: signed zero
    return __uint_as_float((hi & 0x80000000u) | r);
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
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    // exponent and significand shifted into the FP64 layout, exponent rebased
    // by (1023 - 127) << 20; infinity and NaN keep the all-ones exponent
    unsigned hi = ((b & 0x7fffffffu) >> 3) + (896u << 20);
    hi = (e == 0xffu) ? (0x7ff00000u | ((b & 0x7fffffu) >> 3)) : hi;
    hi = (e == 0u) ? 0u : hi;
    const unsigned lo = (e == 0u) ? 0u : (b << 29);
    return __hiloint2double((int)((b & 0x80000000u) | hi), (int)lo);
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
    const float ir = __fdividef(1.0f, r);
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

// Rusanov flux times the face scale: as LF with the speed bound
// lambda = max(|v_L.n|, |v_R.n|) + max(c_L, c_R).
template <typename R>
__device__ __forceinline__ void flux_rusanov(const Prim<R> &L, const R uL[5], const Prim<R> &Rr, const R uR[5],
                                             R gamma, R s1, R s2, R s3, R f[5])
{
    R s = sqrt(s1 * s1 + s2 * s2 + s3 * s3);
    R fl[5], fr[5];
    euler_flux(L, uL[4], s1, s2, s3, fl);
    euler_flux(Rr, uR[4], s1, s2, s3, fr);
    R vn = fmax(fabs(L.v1 * s1 + L.v2 * s2 + L.v3 * s3), fabs(Rr.v1 * s1 + Rr.v2 * s2 + Rr.v3 * s3));
    R c = fmax(sqrt(gamma * L.p / L.rho), sqrt(gamma * Rr.p / Rr.rho));
    R lam = vn + s * c;        // = s * lambda
#pragma unroll
    for (int v = 0; v < 5; ++v) f[v] = (R)0.5 * (fl[v] + fr[v]) - (R)0.5 * lam * (uR[v] - uL[v]);
}

// Roe flux times the face scale (Roe 1981, sqrt(rho)-weighted averages, no
// entropy fix): s [ (F_L + F_R).n/2 - sum_k |lambda_k| alpha_k r_k / 2 ].
// zvel scales the velocity jump seen by the dissipation (1: Roe; the
// low-dissipation variant passes min(1, max Mach)).
template <typename R>
__device__ __forceinline__ void flux_roe(const Prim<R> &L, const R uL[5], const Prim<R> &Rr, const R uR[5], R gamma,
                                         R s1, R s2, R s3, R f[5], R zvel = (R)1)
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
    if (zvel != (R)1) {
        d1 *= zvel;
        d2 *= zvel;
        d3 *= zvel;
    }
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

// Low-dissipation Roe (L2Roe, Osswald et al. 2016): Roe with the velocity
// jump of the dissipation scaled by z = min(1, max(M_L, M_R)), M = |v|/c.
template <typename R>
__device__ __forceinline__ void flux_ldroe(const Prim<R> &L, const R uL[5], const Prim<R> &Rr, const R uR[5], R gamma,
                                           R s1, R s2, R s3, R f[5])
{
    const R mL = (L.v1 * L.v1 + L.v2 * L.v2 + L.v3 * L.v3) * L.rho / (gamma * L.p);
    const R mR = (Rr.v1 * Rr.v1 + Rr.v2 * Rr.v2 + Rr.v3 * Rr.v3) * Rr.rho / (gamma * Rr.p);
    const R z = fmin((R)1, sqrt(fmax(mL, mR)));
    flux_roe(L, uL, Rr, uR, gamma, s1, s2, s3, f, z);
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
// FP32: the hardware approximate reciprocal (at most 2 ulp, no IEEE fix-up
// path), well inside the rounding the FP32 flux arithmetic makes anyway.
template <>
__device__ __forceinline__ float rcp_<float>(float x) { return __fdividef(1.0f, x); }

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
    R irho, ibeta;
    if constexpr (sizeof(R) == 8) {
        // FP64: one division for both reciprocals (the FP64 pipe bounds this path)
        const R inv = (R)1 / (srho * sbeta);
        irho = sbeta * inv;
        ibeta = srho * inv;
    } else {
        irho = rcp_(srho);
        ibeta = rcp_(sbeta);
    }
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

// Logarithmic mean of a, b > 0 from their logarithms, and its reciprocal:
// the Ismail-Roe series in u = ((a-b)/(a+b))^2 below LogMeanEps (as in
// flux_ec), (a-b)/(ln a - ln b) above.
template <typename R>
__device__ __forceinline__ R ln_mean(R a, R b, R la, R lb)
{
    const R s = a + b, d = a - b, fr = d * rcp_(s), u = fr * fr;
    if (u < LogMeanEps<R>::v)
        return (R)0.5 * s * ((R)1 - u * ((R)(1.0 / 3.0) + u * ((R)(4.0 / 45.0) + u * (R)(44.0 / 945.0))));
    return d / (la - lb);
}

template <typename R>
__device__ __forceinline__ R inv_ln_mean(R a, R b, R la, R lb)
{
    const R s = a + b, d = a - b, is = rcp_(s), fr = d * is, u = fr * fr;
    if (u < LogMeanEps<R>::v) return (R)2 * is * ((R)1 + u * ((R)(1.0 / 3.0) + u * ((R)0.2 + u * (R)(1.0 / 7.0))));
    return (la - lb) / d;
}

// Entropy-stable flux with matrix dissipation (Winters, Derigs, Gassner and
// Walch 2017), times the face scale: Chandrashekar's flux minus
// (s/2) sum_k |lambda_k| T_k r_k (r_k . [[w]]), w the entropy variables
// ((gamma - s)/(gamma-1) - rho|v|^2/(2p), rho v/p, -rho/p), with the scaled
// eigenvectors at rho^ = ln-mean rho, p^ = {rho}/(2{beta}), v^ = {v},
// v2^ = 2|{v}|^2 - {|v|^2}, a^ = sqrt(gamma p^/rho^),
// h^ = gamma/(2(gamma-1) beta^ln) + v2^/2:
//   acoustic r = [1, v^ -+ a^ n, h^ -+ a^ v^.n], T = rho^/(2 gamma)
//   entropy  r = [1, v^, v2^/2],                T = rho^ (gamma-1)/gamma
//   shear    (I - n n^T) projection of [[w_m]] + v^ [[w_E]],  T = p^.
// The entropy-variable jump uses ln p - gamma ln rho = (1-gamma) ln rho -
// ln beta - ln 2 from the per-node logarithms of rho and beta.
template <typename R>
__device__ __forceinline__ void flux_matrix(const Prim<R> &L, const Prim<R> &Rr, R gamma, R hg, R s1, R s2, R s3,
                                            R f[5])
{
    const ECNode<R> zl = ec_node(L), zr = ec_node(Rr);
    flux_ec(zl, zr, hg, s1, s2, s3, f);
    const R s = sqrt(s1 * s1 + s2 * s2 + s3 * s3);
    const R is = rcp_(s);
    const R n1 = s1 * is, n2 = s2 * is, n3 = s3 * is;
    const R rho_h = ln_mean(zl.rho, zr.rho, zl.lrho, zr.lrho);
    const R ib_ln = inv_ln_mean(zl.beta, zr.beta, zl.lbeta, zr.lbeta);
    const R p_h = (R)0.5 * (zl.rho + zr.rho) * rcp_(zl.beta + zr.beta);
    const R v1 = (R)0.5 * (L.v1 + Rr.v1), v2 = (R)0.5 * (L.v2 + Rr.v2), v3 = (R)0.5 * (L.v3 + Rr.v3);
    const R qL = L.v1 * L.v1 + L.v2 * L.v2 + L.v3 * L.v3, qR = Rr.v1 * Rr.v1 + Rr.v2 * Rr.v2 + Rr.v3 * Rr.v3;
    const R v2h = (R)2 * (v1 * v1 + v2 * v2 + v3 * v3) - (R)0.5 * (qL + qR);
    const R a_h = sqrt(gamma * p_h / rho_h);
    const R h_h = gamma * hg * ib_ln + (R)0.5 * v2h;
    const R vn = v1 * n1 + v2 * n2 + v3 * n3;
    // [[w]]: (gamma-1) [[ln rho]] + [[ln beta]] enters w_0 through 2 hg = 1/(gamma-1)
    R dw[5];
    dw[0] = (zr.lrho - zl.lrho) + (R)2 * hg * (zr.lbeta - zl.lbeta) - (zr.beta * qR - zl.beta * qL);
    dw[1] = (R)2 * (zr.beta * Rr.v1 - zl.beta * L.v1);
    dw[2] = (R)2 * (zr.beta * Rr.v2 - zl.beta * L.v2);
    dw[3] = (R)2 * (zr.beta * Rr.v3 - zl.beta * L.v3);
    dw[4] = (R)-2 * (zr.beta - zl.beta);
    const R r1[5] = {(R)1, v1 - a_h * n1, v2 - a_h * n2, v3 - a_h * n3, h_h - a_h * vn};
    const R r5[5] = {(R)1, v1 + a_h * n1, v2 + a_h * n2, v3 + a_h * n3, h_h + a_h * vn};
    const R c1 = dw[0] + r1[1] * dw[1] + r1[2] * dw[2] + r1[3] * dw[3] + r1[4] * dw[4];
    const R c5 = dw[0] + r5[1] * dw[1] + r5[2] * dw[2] + r5[3] * dw[3] + r5[4] * dw[4];
    const R c2 = dw[0] + v1 * dw[1] + v2 * dw[2] + v3 * dw[3] + (R)0.5 * v2h * dw[4];
    const R T15 = rho_h / ((R)2 * gamma), T2 = rho_h * (gamma - (R)1) / gamma;
    const R k1 = fabs(vn - a_h) * T15 * c1, k5 = fabs(vn + a_h) * T15 * c5;
    const R l2 = fabs(vn);
    const R k2 = l2 * T2 * c2;
    const R q1 = dw[1] + v1 * dw[4], q2 = dw[2] + v2 * dw[4], q3 = dw[3] + v3 * dw[4];
    const R qn = q1 * n1 + q2 * n2 + q3 * n3;
    const R ks = l2 * p_h;
    const R P1 = ks * (q1 - qn * n1), P2 = ks * (q2 - qn * n2), P3 = ks * (q3 - qn * n3);
    const R hs = (R)0.5 * s;
    f[0] -= hs * (k1 + k2 + k5);
    f[1] -= hs * (k1 * r1[1] + k2 * v1 + k5 * r5[1] + P1);
    f[2] -= hs * (k1 * r1[2] + k2 * v2 + k5 * r5[2] + P2);
    f[3] -= hs * (k1 * r1[3] + k2 * v3 + k5 * r5[3] + P3);
    f[4] -= hs * (k1 * r1[4] + k2 * (R)0.5 * v2h + k5 * r5[4] + v1 * P1 + v2 * P2 + v3 * P3);
}

// ------------------------------------------------------------------ split forms
//
// Per-node inputs of the two-point fluxes, kSplitSlots values per node:
//   EC         rho, v1, v2, v3, beta = rho/(2p), ln rho, ln beta
//   KG         rho, v1, v2, v3, p, e = (rho e)/rho
//   PIROZZOLI  rho, v1, v2, v3, p, h = (rho e + p)/rho
//   DUCROS     rho, v1, v2, v3, p, rho e + p
//   MORINISHI  rho, v1, v2, v3, p, |v|^2/2
//   IR         z1 = sqrt(rho/p), z1 v1, z1 v2, z1 v3, z5 = sqrt(rho p), ln z1, ln z5
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
    } else if constexpr (FORM == HS3D_VOL_IR) {
        const R z1 = sqrt(q.rho / q.p), z5 = sqrt(q.rho * q.p);
        z[0] = z1;
        z[1] = z1 * q.v1;
        z[2] = z1 * q.v2;
        z[3] = z1 * q.v3;
        z[4] = z5;
        z[5] = log_(z1);
        z[6] = log_(z5);
    } else if constexpr (FORM == HS3D_VOL_MORINISHI) {
        z[4] = q.p;
        z[5] = (R)0.5 * (q.v1 * q.v1 + q.v2 * q.v2 + q.v3 * q.v3);
        z[6] = (R)0;
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

// Morinishi: ({rho v_a}, {rho v_a}{v} + {p}a, {rho v_a}{|v|^2/2} + gamma/(gamma-1){p v_a}).
template <typename R>
__device__ __forceinline__ void flux_morinishi(const R *L, const R *Rr, R hg, R a1, R a2, R a3, R f[5])
{
    const R h = (R)0.5;
    const R vaL = L[1] * a1 + L[2] * a2 + L[3] * a3;
    const R vaR = Rr[1] * a1 + Rr[2] * a2 + Rr[3] * a3;
    const R m = h * (L[0] * vaL + Rr[0] * vaR);
    const R pav = h * (L[4] + Rr[4]);
    f[0] = m;
    f[1] = m * (h * (L[1] + Rr[1])) + pav * a1;
    f[2] = m * (h * (L[2] + Rr[2])) + pav * a2;
    f[3] = m * (h * (L[3] + Rr[3])) + pav * a3;
    f[4] = m * (h * (L[5] + Rr[5])) + ((R)1 + (R)2 * hg) * (h * (L[4] * vaL + Rr[4] * vaR));
}

// Ismail-Roe entropy-conservative flux from the parameter vector
// z = sqrt(rho/p)(1, v, p): rho^ = {z1} z5^ln, v^ = {z_v}/{z1}, p1^ = {z5}/{z1},
// p2^ = (gamma+1)/(2 gamma) z5^ln/z1^ln + (gamma-1)/(2 gamma) {z5}/{z1},
// h^ = gamma p2^/((gamma-1) rho^) + |v^|^2/2;
// f = (rho^ v^.a, rho^ v^.a v^ + p1^ a, rho^ v^.a h^).
template <typename R>
__device__ __forceinline__ void flux_ir(const R *L, const R *Rr, R gamma, R hg, R a1, R a2, R a3, R f[5])
{
    const R h = (R)0.5;
    const R z1a = h * (L[0] + Rr[0]), z5a = h * (L[4] + Rr[4]);
    const R iz1a = rcp_(z1a);
    const R z5ln = ln_mean(L[4], Rr[4], L[6], Rr[6]);
    const R iz1ln = inv_ln_mean(L[0], Rr[0], L[5], Rr[5]);
    const R rho = z1a * z5ln;
    const R v1 = h * (L[1] + Rr[1]) * iz1a, v2 = h * (L[2] + Rr[2]) * iz1a, v3 = h * (L[3] + Rr[3]) * iz1a;
    const R p1 = z5a * iz1a;
    const R ig = rcp_(gamma);
    const R p2 = h * ((gamma + (R)1) * ig) * z5ln * iz1ln + h * ((gamma - (R)1) * ig) * p1;
    const R hh = (R)2 * hg * gamma * p2 / rho + h * (v1 * v1 + v2 * v2 + v3 * v3);
    const R m = rho * (v1 * a1 + v2 * a2 + v3 * a3);
    f[0] = m;
    f[1] = m * v1 + p1 * a1;
    f[2] = m * v2 + p1 * a2;
    f[3] = m * v3 + p1 * a3;
    f[4] = m * hh;
}

template <int FORM, typename R>
__device__ __forceinline__ void split_pair(const R *L, const R *Rr, R gamma, R hg, R a1, R a2, R a3, R f[5])
{
    if constexpr (FORM == HS3D_VOL_EC) {
        const ECNode<R> zl = {L[0], L[1], L[2], L[3], L[4], L[5], L[6]};
        const ECNode<R> zr = {Rr[0], Rr[1], Rr[2], Rr[3], Rr[4], Rr[5], Rr[6]};
        flux_ec(zl, zr, hg, a1, a2, a3, f);
    } else if constexpr (FORM == HS3D_VOL_MORINISHI) {
        flux_morinishi(L, Rr, hg, a1, a2, a3, f);
    } else if constexpr (FORM == HS3D_VOL_IR) {
        flux_ir(L, Rr, gamma, hg, a1, a2, a3, f);
    } else {
        flux_avg_product<FORM>(L, Rr, a1, a2, a3, f);
    }
}

}  // namespace hs3d
