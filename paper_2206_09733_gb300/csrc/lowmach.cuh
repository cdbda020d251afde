// FP32 flux arithmetic on deviations from a reference state (the mixed
// path's formulation).
//
// Why: at low Mach number the residual is a small difference of large
// fluxes.  The total enthalpy H ~ c^2/(gamma-1) multiplies the mass flux in
// the energy equation, so the energy residual contains H * div(rho v), a
// near-cancellation of O(1) terms amplified by H (~250 at Mach 0.1), and the
// momentum residual contains grad p with p ~ 1/(gamma Ma^2).  Rounding the
// state alone to FP32 (exact arithmetic afterwards) moves the residual of the
// 16^3 Mach 0.1 Taylor-Green vortex by ~5e-4 relative; the FP32 flux
// arithmetic made it ~1e-2.
//
// What: every element picks a reference ("anchor") state ubar, the state at
// its centre node rounded to FP32.  Deviations u - ubar are formed in FP64
// and rounded once, so their FP32 rounding error is relative to the
// deviation, not to the state.  The fluxes are evaluated as F(u) - F(ubar)
// from these deviations with formulas that never form a large quantity and
// then subtract another (below).  F(ubar) itself is dropped: a constant
// physical flux has zero volume term by the discrete metric identity
// sum_d D_d Ja^d = 0, and the surface terms use flux jumps formed by the face
// kernel, in which it cancels.  The energy flux is split as
//   F_E - F_E(ubar) = Hbar (F_rho - F_rho(ubar)) + rest,
// so that the energy volume term is Hbar * (mass volume term) + V[rest], and
// the mass volume term, whose error Hbar multiplies, is the conservative
// divergence sum_d D_d (Ja^d . m') of the momentum deviation m' (exact by the
// same identity), evaluated in float-float (pairs of FP32 numbers, ~44 bits)
// from the FP64 deviation and an FP32 low part of the metric terms.  The
// split forms' mass flux differs from that conservative divergence by a pair
// remainder that is a product of two small differences and stays in FP32.
//
// All identities are exact in exact arithmetic (the method is unchanged); only
// the rounding moves.  The formulas cover the standard volume form, the
// Chandrashekar entropy-conservative split form and every surface flux; the
// other split forms evaluate their two-point flux from full FP32 primitive
// variables and subtract F(ubar) (exact, with the plain FP32 accuracy).
#pragma once

#include <math.h>

#include "internal.cuh"
#include "physics.cuh"

namespace hs3d {

// ------------------------------------------------------------------ float-float

// s + e = a + b exactly (Knuth's two-sum; no assumption on |a|, |b|).
__host__ __device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// (sh, sl) += (ah + al) * (bh + bl): the head product exactly (fma residual),
// the cross terms and the low parts in FP32, the head sum by two-sum.  The
// pair is left unnormalised; its value is sh + sl.
__host__ __device__ __forceinline__ void ff_fma(float &sh, float &sl, float ah, float al, float bh, float bl)
{
    const float p = ah * bh;
    float pe = fmaf(ah, bh, -p);
    pe = fmaf(ah, bl, fmaf(al, bh, pe));
    float s, e;
    two_sum(sh, p, s, e);
    sh = s;
    sl += e + pe;
}

// (sh, sl) = (ah + al) * (bh + bl): ff_fma into a zero pair (the first term
// of a sum), bitwise the same, without the two-sum.
__host__ __device__ __forceinline__ void ff_mul(float &sh, float &sl, float ah, float al, float bh, float bl)
{
    sh = ah * bh;
    const float pe = fmaf(ah, bh, -sh);
    sl = fmaf(ah, bl, fmaf(al, bh, pe));
}

// FP64 -> FP32 (round to nearest even) of the deviations: the integer-pipe
// rounding d2f_rn (the hardware conversion, one FP64-pipe instruction each,
// measured 3-20% slower in all three deviation kernels).
__device__ __forceinline__ float dev_round(double x) { return d2f_rn(x); }

// FP64 -> (hi, lo) with hi = x rounded to FP32 (d2f_rn) and lo = x - hi
// rounded to FP32 (ff_lo), with no FP64 instruction: x - hi is exactly the integer
// R = (the 29 significand bits the rounding drops) - (2^29 if it rounded
// up), |R| <= 2^28, times 2^(e - 1075) (e the biased FP64 exponent of x), so
// lo is the integer-to-float conversion of R (round to nearest) scaled by that
// power of two, with the sign of x.  Equal to d2f_rn(x - (double)hi) for
// |x| >= 2^-74 (below, lo is flushed to zero; hi is already zero below the
// FP32 normal range).
__device__ __forceinline__ float ff_lo(double x)
{
    const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
    const unsigned e = (h >> 20) & 0x7ffu;
    const unsigned t = __funnelshift_l(l, h, 3);   // the kept bits, as d2f_rn truncates them
    const unsigned dropped = l & 0x1fffffffu;
    const unsigned up = (dropped + (t & 1u) + 0x0fffffffu) >> 29;   // d2f_rn's rounding increment
    const int R = (int)dropped - (int)(up << 29);
    const float scale = (e >= 949u && e <= 1202u) ? __int_as_float((int)(e - 948u) << 23) : 0.0f;
    const float mag = __int2float_rn(R) * scale;
    return (h & 0x80000000u) ? -mag : mag;
}

__device__ __forceinline__ void ff_split(double x, float &hi, float &lo)
{
    hi = d2f_rn(x);
    lo = ff_lo(x);
}

// ------------------------------------------------------------------ anchor

// Reference state of an element (or of a face).  Its primitive values rho,
// v, p are FP32 numbers near the node's; its conserved values are formed
// from them in FP64 so that the identities the deviation formulas rely on
// hold exactly: m = rho v (a product of two FP32 numbers is exact in FP64)
// and E = p/(gamma-1) + rho|v|^2/2 with the FP32 (gamma-1) of the kernels, so
// that (gamma-1)(E - m.v/2) is p.  H (an FP32 number near (E + p)/rho) is
// carried with rH = E + p - H rho, and the entropy-conservative flux's energy
// factor with cK = hg/beta + |v|^2/2 + p/rho - H, hg = 1/(2(gamma-1)) taken
// to ~2^-48 (hg + hglo), so that the one-point and the two-point fluxes share
// one reference flux F(ubar) and agree at u_i = u_m.
struct Anchor {
    float rho, m1, m2, m3, E;
    float v1, v2, v3, p, beta, H;
    float rbeta, rH, cK;
    float ib, pr;   // 1/beta and p/rho, factors of the flux formulas
};

// uc: the FP64 state at the anchor node; ad receives the FP64 conserved anchor.
__device__ __forceinline__ Anchor make_anchor(const double uc[5], float gm1, float hg, float hglo, double igm1,
                                              double ad[5])
{
    Anchor A;
    A.rho = d2f_rn(uc[0]);
    const float mf1 = d2f_rn(uc[1]), mf2 = d2f_rn(uc[2]), mf3 = d2f_rn(uc[3]), Ef = d2f_rn(uc[4]);
    const float ir = 1.0f / A.rho;
    A.v1 = mf1 * ir;
    A.v2 = mf2 * ir;
    A.v3 = mf3 * ir;
    A.p = gm1 * (Ef - 0.5f * (mf1 * A.v1 + mf2 * A.v2 + mf3 * A.v3));
    const double r = f2d_exact(A.rho), v1 = f2d_exact(A.v1), v2 = f2d_exact(A.v2), v3 = f2d_exact(A.v3);
    const double vv = fma(v1, v1, fma(v2, v2, v3 * v3));
    ad[0] = r;
    ad[1] = r * v1;
    ad[2] = r * v2;
    ad[3] = r * v3;
    ad[4] = fma(0.5 * r, vv, f2d_exact(A.p) * igm1);
    A.m1 = d2f_rn(ad[1]);
    A.m2 = d2f_rn(ad[2]);
    A.m3 = d2f_rn(ad[3]);
    A.E = d2f_rn(ad[4]);
    A.beta = A.rho / (2.0f * A.p);
    A.rbeta = fmaf(-2.0f * A.p, A.beta, A.rho);
    A.ib = __fdividef(1.0f, A.beta);
    A.pr = A.p * __fdividef(1.0f, A.rho);
    // H = hg/beta + |v|^2/2 + p/rho in FP32, every rounding residual into cK
    const float x = hg / A.beta;
    const float e1 = (fmaf(-x, A.beta, hg) + hglo) / A.beta;
    const float z = d2f_rn(0.5 * vv);
    const float e2 = d2f_rn(0.5 * vv - f2d_exact(z));
    const float y = A.p * ir;
    const float e3 = fmaf(-y, A.rho, A.p) * ir;
    float s1, t1, t2;
    two_sum(x, z, s1, t1);
    two_sum(s1, y, A.H, t2);
    A.cK = e1 + e2 + e3 + (t1 + t2);
    A.rH = d2f_rn(ad[4] + fma(-f2d_exact(A.H), r, f2d_exact(A.p)));
    return A;
}

// Reference state of a face for fluxes of the "central + dissipation" kind,
// which use only F(u_R) - F(u_L) and jumps: the minus side's state u_L is the
// reference (its deviation is zero, u_R's is the jump u_R - u_L formed in
// FP64), and its values rounded to FP32 serve as the coefficients of the
// deviation formulas, whose results are then accurate relative to the jump.
__device__ __forceinline__ Anchor make_anchor_face(const double uc[5], float gm1, double ad[5])
{
    Anchor A;
    A.rho = d2f_rn(uc[0]);
    A.m1 = d2f_rn(uc[1]);
    A.m2 = d2f_rn(uc[2]);
    A.m3 = d2f_rn(uc[3]);
    A.E = d2f_rn(uc[4]);
    const float ir = __fdividef(1.0f, A.rho);
    A.v1 = A.m1 * ir;
    A.v2 = A.m2 * ir;
    A.v3 = A.m3 * ir;
    A.p = gm1 * (A.E - 0.5f * (A.m1 * A.v1 + A.m2 * A.v2 + A.m3 * A.v3));
    A.beta = 0.5f * A.rho * __fdividef(1.0f, A.p);
    A.H = (A.E + A.p) * ir;
    A.ib = __fdividef(1.0f, A.beta);
    A.pr = A.p * __fdividef(1.0f, A.rho);
    A.rbeta = 0.0f;
    A.rH = 0.0f;
    A.cK = 0.0f;
    ad[0] = f2d_exact(A.rho);
    ad[1] = f2d_exact(A.m1);
    ad[2] = f2d_exact(A.m2);
    ad[3] = f2d_exact(A.m3);
    ad[4] = f2d_exact(A.E);
    return A;
}

// An element's reference state as the mixed kernels keep it in HBM (one
// record per element, Item::anc): the FP64 conserved values and the FP32
// Anchor.  The element kernel's centre-node thread rewrites it after each RK
// stage from the updated state (the priming passes before the first stage),
// so the next kernels load it instead of building it: any FP32 state near
// the element's serves, as long as every thread of one kernel launch uses
// the same one.
struct AnchorRec {
    double ad[5];
    Anchor a;
    float Elo;   // ad[4] - a.E rounded to FP32 (a.E is ad[4] rounded)
    float pad;
};
static_assert(sizeof(AnchorRec) == 112, "AnchorRec layout");

// Every thread of an element loads its record (seven 16-byte loads, the
// same addresses across the element: broadcast from L1).
__device__ __forceinline__ AnchorRec load_anchor(const void *anc, int e)
{
    AnchorRec r;
    const float4 *src = (const float4 *)((const AnchorRec *)anc + e);
    float4 *dst = (float4 *)&r;
#pragma unroll
    for (int k = 0; k < 7; ++k) dst[k] = __ldg(src + k);
    return r;
}

// Centre node of an element of n^3 nodes: its state becomes the reference.
__host__ __device__ constexpr int anchor_node(int n) { return (n / 2) * (1 + n + n * n); }

__device__ __forceinline__ void write_anchor(const Item &it, int e, const double u[5])
{
    AnchorRec r;
    r.a = make_anchor(u, it.gm1f, it.hgf, it.hglof, it.igm1f, r.ad);
    r.Elo = d2f_rn(r.ad[4] - f2d_exact(r.a.E));
    r.pad = 0.0f;
    ((AnchorRec *)it.anc)[e] = r;
}

// u - ad for an FP64 value u and a reference value given as an FP32 pair
// (h, l), with no FP64 arithmetic: u = uh + ul + r (uh = u rounded to FP32,
// ul = ff_lo(u), |r| <= 2^-48 |u|), then (uh - h) + (ul - l) in FP32: the
// deviation within ~1.5 ulp of its FP32 rounding, plus 2^-48 |u|.  uh is the
// hardware conversion (one FP64-pipe instruction, where the integer-pipe
// d2f_rn measured slower: the gradient kernel that uses this is ALU-bound).
__device__ __forceinline__ float dev_one(double u, float h, float l)
{
    return (__double2float_rn(u) - h) + (ff_lo(u) - l);
}

// ------------------------------------------------------------------ deviations of one node

// A node's state as deviations from the anchor plus the full FP32 values the
// flux formulas multiply them with.
struct Dev {
    float dr, dm1, dm2, dm3, dE;   // conserved deviations
    float dv1, dv2, dv3, dp;       // primitive deviations v - vbar, p - pbar
    float rho, v1, v2, v3, p;      // full values (FP32)
};

// The conserved deviations are formed in FP64 (five subtractions) and
// rounded once; the primitive deviations follow in FP32 (exact identities,
// mbar = rhobar vbar):
//   v' = (m' - vbar rho')/rho,
//   p' = (gamma-1)(E' - (m'.v + mbar.v')/2)     (m.v - mbar.vbar = m'.v + mbar.v').
__device__ __forceinline__ Dev make_dev_f(float dr, float dm1, float dm2, float dm3, float dE, const Anchor &A,
                                         float gm1)
{
    Dev d;
    d.dr = dr;
    d.dm1 = dm1;
    d.dm2 = dm2;
    d.dm3 = dm3;
    d.dE = dE;
    d.rho = A.rho + dr;
    const float ir = __fdividef(1.0f, d.rho);
    d.dv1 = fmaf(-A.v1, dr, dm1) * ir;
    d.dv2 = fmaf(-A.v2, dr, dm2) * ir;
    d.dv3 = fmaf(-A.v3, dr, dm3) * ir;
    d.v1 = A.v1 + d.dv1;
    d.v2 = A.v2 + d.dv2;
    d.v3 = A.v3 + d.dv3;
    const float mv = dm1 * d.v1 + dm2 * d.v2 + dm3 * d.v3 + (A.m1 * d.dv1 + A.m2 * d.dv2 + A.m3 * d.dv3);
    d.dp = gm1 * (dE - 0.5f * mv);
    d.p = A.p + d.dp;
    return d;
}

// make_dev from the record's FP32 values alone: the conserved reference values
// as FP32 pairs, rho (exact), m = rho v (a product of two FP32 numbers: its
// rounding a.m and the FMA residual) and E (a.E and Elo).
__device__ __forceinline__ Dev make_dev_rec(const double u[5], const Anchor &A, float Elo, float gm1)
{
    return make_dev_f(dev_one(u[0], A.rho, 0.0f), dev_one(u[1], A.m1, fmaf(A.rho, A.v1, -A.m1)),
                      dev_one(u[2], A.m2, fmaf(A.rho, A.v2, -A.m2)), dev_one(u[3], A.m3, fmaf(A.rho, A.v3, -A.m3)),
                      dev_one(u[4], A.E, Elo), A, gm1);
}

__device__ __forceinline__ Dev make_dev(const double u[5], const double ad[5], const Anchor &A, float gm1)
{
    return make_dev_f(dev_round(u[0] - ad[0]), dev_round(u[1] - ad[1]), dev_round(u[2] - ad[2]),
                      dev_round(u[3] - ad[3]), dev_round(u[4] - ad[4]), A, gm1);
}

// Primitive variables of the node in FP32 (for wave speeds and the
// viscous flux).
__device__ __forceinline__ Prim<float> dev_prim(const Dev &d, const Anchor &A)
{
    Prim<float> q;
    q.rho = d.rho;
    q.v1 = d.v1;
    q.v2 = d.v2;
    q.v3 = d.v3;
    q.p = d.p;
    q.E = A.E + d.dE;
    return q;
}

// H - Hbar = (E' + p' - Hbar rho' + rH)/rho.
__device__ __forceinline__ float dev_dH(const Dev &d, const Anchor &A)
{
    return (d.dE + d.dp - A.H * d.dr + A.rH) * __fdividef(1.0f, d.rho);
}

// beta - betabar = (rho' - 2 p' betabar + rbeta)/(2p).
__device__ __forceinline__ float dev_dbeta(const Dev &d, const Anchor &A)
{
    return (d.dr - 2.0f * d.dp * A.beta + A.rbeta) * __fdividef(0.5f, d.p);
}

// ------------------------------------------------------------------ one-point flux deviation

// (F(u) - F(ubar)).a for the Euler flux, all five components accurate
// relative to the deviation:
//   mass      m'.a
//   momentum  m'_c v.a + mbar_c v'.a + p' a_c
//   energy    Hbar m'.a + (H - Hbar) m.a
__device__ __forceinline__ void dflux_euler(const Dev &d, const Anchor &A, float a1, float a2, float a3, float f[5])
{
    const float ma_d = d.dm1 * a1 + d.dm2 * a2 + d.dm3 * a3;
    const float va = d.v1 * a1 + d.v2 * a2 + d.v3 * a3;
    const float dva = d.dv1 * a1 + d.dv2 * a2 + d.dv3 * a3;
    const float ma = (A.m1 * a1 + A.m2 * a2 + A.m3 * a3) + ma_d;
    f[0] = ma_d;
    f[1] = d.dm1 * va + A.m1 * dva + d.dp * a1;
    f[2] = d.dm2 * va + A.m2 * dva + d.dp * a2;
    f[3] = d.dm3 * va + A.m3 * dva + d.dp * a3;
    f[4] = A.H * ma_d + dev_dH(d, A) * ma;
}

// The standard volume form's FP32 fluxes: momentum as above and the energy
// remainder (H - Hbar) m.a (the Hbar m'.a part enters through the mass
// volume term).
__device__ __forceinline__ void dflux_euler_rest(const Dev &d, const Anchor &A, float dH, float a1, float a2, float a3,
                                                 float f[4])
{
    const float ma_d = d.dm1 * a1 + d.dm2 * a2 + d.dm3 * a3;
    const float va = d.v1 * a1 + d.v2 * a2 + d.v3 * a3;
    const float dva = d.dv1 * a1 + d.dv2 * a2 + d.dv3 * a3;
    const float ma = (A.m1 * a1 + A.m2 * a2 + A.m3 * a3) + ma_d;
    f[0] = d.dm1 * va + A.m1 * dva + d.dp * a1;
    f[1] = d.dm2 * va + A.m2 * dva + d.dp * a2;
    f[2] = d.dm3 * va + A.m3 * dva + d.dp * a3;
    f[3] = dH * ma;
}

// ------------------------------------------------------------------ Chandrashekar flux on deviations

// Per-node inputs of the deviation form of the Chandrashekar flux: rho',
// v', beta' (the logarithms of the logarithmic-mean branch, taken only for
// jumps of more than ~20%, are formed where that branch is taken).
struct ECDev {
    float dr, dv1, dv2, dv3, db;
    float q;   // |v|^2 - |vbar|^2 = v'.(v + vbar)
};

__device__ __forceinline__ ECDev ec_dev(const Dev &d, const Anchor &A)
{
    ECDev z;
    z.dr = d.dr;
    z.dv1 = d.dv1;
    z.dv2 = d.dv2;
    z.dv3 = d.dv3;
    z.db = dev_dbeta(d, A);
    z.q = d.dv1 * (d.v1 + A.v1) + d.dv2 * (d.v2 + A.v2) + d.dv3 * (d.v3 + A.v3);
    return z;
}

// Output of the deviation Chandrashekar flux dotted with A (= Ja_i + Ja_m in
// the volume, the scaled normal on a face):
//   frho   f_rho - Fbar_rho (FP32; the face kernel's mass component)
//   rmass  f_rho - (m_i.a_i + m_m.a_m) without the -(m_i - m_m).(a_i - a_m)/2
//          term (the volume kernel adds that term; see k_volume)
//   fm     f_m - Fbar_m
//   rest   f_E - Fbar_E - H_ec frho, H_ec = K + pbar/rhobar = A.H
// With rho^ = ln-mean rho, beta^ = ln-mean beta, p~ = {rho}/(2{beta}),
// K = hg/beta^ - {|v|^2}/2 + |{v}|^2:
//   f_rho = rho^ {v}.A,  f_m = f_rho {v} + p~ A,  f_E = f_rho K + p~ {v}.A,
// and at ubar  Fbar_rho = rhobar vbar.A, Kbar = hg/betabar + |vbar|^2/2,
//   f_rho - Fbar_rho = (rho^ - rhobar){v}.A + rhobar {v'}.A
//   f_m - Fbar_m     = (f_rho - Fbar_rho){v} + Fbar_rho {v'} + (p~ - pbar) A
//   rest             = [(p~ - pbar) - (pbar/rhobar)(rho^ - rhobar)] {v}.A + f_rho (K - Kbar),
// Kbar = H - pbar/rhobar, so that K - Kbar = hg (1/beta^ - 1/betabar) - ({|v|^2} - |vbar|^2)/2
// + (|{v}|^2 - |vbar|^2) + cK
// where every bracket is formed from deviations:
//   rho^ - {rho}   = -{rho} u (1/3 + u(4/45 + u 44/945))     (series, u < eps)
//   1/beta^ - 1/betabar = -(beta'_i + beta'_m)/(s_beta betabar) + (2/s_beta) u (1/3 + u(1/5 + u/7))
//   p~ - pbar      = ({rho'} - pbar(beta'_i + beta'_m) + rbeta)/s_beta
//   {|v|^2} - |vbar|^2 = (v'_i.(v_i + vbar) + v'_m.(v_m + vbar))/2,  |{v}|^2 - |vbar|^2 = {v'}.({v} + vbar)
// (logarithmic branch for u >= eps: the means themselves, then the subtraction).
__device__ __forceinline__ void dflux_ec(const ECDev &L, const ECDev &Rr, const Anchor &A, float hg, float a1,
                                         float a2, float a3, float &frho, float &rmass, float fm[3], float &rest)
{
    const float rL = A.rho + L.dr, rR = A.rho + Rr.dr;
    const float bL = A.beta + L.db, bR = A.beta + Rr.db;
    const float sr = rL + rR, sb = bL + bR;
    const float isr = __fdividef(1.0f, sr), isb = __fdividef(1.0f, sb);
    const float dr = L.dr - Rr.dr, db = L.db - Rr.db;
    const float fr = dr * isr, ur = fr * fr;
    const float rbar_m = 0.5f * (L.dr + Rr.dr);   // {rho'}
    const float fb = db * isb, ub = fb * fb;
    // rho^ - {rho} and 1/beta^ - 1/betabar on the series branch, replaced by the
    // logarithmic form where the jump is large; the common case is the series,
    // and a warp vote keeps the logarithms off the warps that need none
    float rh_m = -0.5f * sr * ur * ((1.0f / 3.0f) + ur * ((4.0f / 45.0f) + ur * (44.0f / 945.0f)));
    float ibd = -(L.db + Rr.db) * isb * A.ib +
                2.0f * isb * ub * ((1.0f / 3.0f) + ub * (0.2f + ub * (1.0f / 7.0f)));
    const bool log_r = !(ur < LogMeanEps<float>::v), log_b = !(ub < LogMeanEps<float>::v);
    if (__any_sync(__activemask(), log_r || log_b)) {
        if (log_r) rh_m = __fdividef(dr, logf(rL) - logf(rR)) - 0.5f * sr;
        if (log_b) ibd = __fdividef(logf(bL) - logf(bR), db) - A.ib;
    }
    const float rhd = rbar_m + rh_m;               // rho^ - rhobar
    const float dv1 = 0.5f * (L.dv1 + Rr.dv1), dv2 = 0.5f * (L.dv2 + Rr.dv2), dv3 = 0.5f * (L.dv3 + Rr.dv3);
    const float mv1 = A.v1 + dv1, mv2 = A.v2 + dv2, mv3 = A.v3 + dv3;
    const float va = mv1 * a1 + mv2 * a2 + mv3 * a3;
    const float vda = dv1 * a1 + dv2 * a2 + dv3 * a3;
    const float Fbr = A.m1 * a1 + A.m2 * a2 + A.m3 * a3;   // rhobar vbar.A
    frho = rhd * va + A.rho * vda;
    // rho^{v} - {m} = (rho^ - {rho}){v} - (rho_i - rho_m)(v_i - v_m)/4
    {
        const float ddv1 = L.dv1 - Rr.dv1, ddv2 = L.dv2 - Rr.dv2, ddv3 = L.dv3 - Rr.dv3;
        rmass = rh_m * va - 0.25f * dr * (ddv1 * a1 + ddv2 * a2 + ddv3 * a3);
    }
    const float ptd = (rbar_m - A.p * (L.db + Rr.db) + A.rbeta) * isb;
    fm[0] = frho * mv1 + Fbr * dv1 + ptd * a1;
    fm[1] = frho * mv2 + Fbr * dv2 + ptd * a2;
    fm[2] = frho * mv3 + Fbr * dv3 + ptd * a3;
    const float q2d = 0.5f * (L.q + Rr.q);
    const float m2d = dv1 * (mv1 + A.v1) + dv2 * (mv2 + A.v2) + dv3 * (mv3 + A.v3);
    const float Kd = hg * ibd - 0.5f * q2d + m2d + A.cK;
    rest = (ptd - A.pr * rhd) * va + (Fbr + frho) * Kd;
}

// dflux_ec at u_i = u_m (the diagonal pair of the volume term): the
// logarithmic means are the values themselves (u = 0 on the series branch),
// rho^ - rhobar = rho', 1/beta^ - 1/betabar = -beta'/(beta betabar),
// p~ - pbar = (rho' - 2 pbar beta' + rbeta)/(2 beta), {v} = v; the same
// algebra as the general function with these values, in fewer operations.
__device__ __forceinline__ void dflux_ec_diag(const ECDev &z, const Anchor &A, float hg, float a1, float a2, float a3,
                                              float fm[3], float &rest)
{
    const float b = A.beta + z.db;
    const float ib = __fdividef(1.0f, b);
    const float ibd = -z.db * ib * A.ib;
    const float v1 = A.v1 + z.dv1, v2 = A.v2 + z.dv2, v3 = A.v3 + z.dv3;
    const float va = v1 * a1 + v2 * a2 + v3 * a3;
    const float vda = z.dv1 * a1 + z.dv2 * a2 + z.dv3 * a3;
    const float Fbr = A.m1 * a1 + A.m2 * a2 + A.m3 * a3;
    const float frho = z.dr * va + A.rho * vda;
    const float ptd = (z.dr - 2.0f * A.p * z.db + A.rbeta) * 0.5f * ib;
    fm[0] = frho * v1 + Fbr * z.dv1 + ptd * a1;
    fm[1] = frho * v2 + Fbr * z.dv2 + ptd * a2;
    fm[2] = frho * v3 + Fbr * z.dv3 + ptd * a3;
    const float Kd = hg * ibd + 0.5f * z.q + A.cK;
    rest = (ptd - A.pr * z.dr) * va + (Fbr + frho) * Kd;
}

}  // namespace hs3d
