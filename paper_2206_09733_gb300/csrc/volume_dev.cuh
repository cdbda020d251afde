// Element kernel of the mixed path: volume term + surface lifting + Jacobian
// scaling + RK stage, FP32 flux arithmetic on deviations (lowmach.cuh).
//
// Strong form of Eq. NS5 (Sec. 3.3) on Gauss-Lobatto nodes, per element,
// du/dt = -(V + S)/J, with the element's reference state ubar (its centre
// node):
//   standard form (Sec. 3.3)   V = sum_d D_d Ja^d.(F(u) - F(ubar) - F_v)
//   Chandrashekar split form (Sec. 3.5)
//                              V = sum_d sum_m D_im (F#(u_i,u_m) - F(ubar)).(Ja_i + Ja_m) - sum_d D_d (Ja^d.F_v)
//   other split forms          V = sum_d sum_m D_im F#(u_i,u_m).(Ja_i + Ja_m) - sum_d D_d (Ja^d.F_v)
// (F(ubar) has no volume term: sum_d D_d Ja^d = 0).  For the standard and
// Chandrashekar forms the mass and energy rows are split as
//   V_rho = C + (split form: sum_d sum_m D_im e_im),   C = sum_d D_d (Ja^d.m')
//   V_E   = Hbar V_rho + V[rest]
// where C, the conservative divergence of the momentum deviation m', is
// contracted in float-float (the FP64 deviation split into two FP32 numbers,
// Ja = Jaf + Jalo, D = Df + Dlo), e_im = (rho^{v} - {m}).(Ja_i + Ja_m)
// - (m_i - m_m).(Ja_i - Ja_m)/2 is the split form's mass flux minus the
// conservative one (a product of small differences, FP32), and rest is the
// energy flux beyond Hbar times the mass flux (FP32).
//   surface   the face kernel's per-side jumps: S = (1/w) G_L on the +d face,
//             -(1/w) G_R on the -d face (G = F* - F(u_side).Sn); on a mesh
//             with per-element degrees (face6) the mortar flux F* and the own
//             FP32 flux: S = (1/w)(F* - F_own) and (1/w)(F_own - F*).
// followed by the residual store or one low-storage RK stage in FP64, and
// after the last stage the dt maxima of the updated state.
//
// One thread per node, epb elements per CTA.  The six face blocks, 1/J and
// (standard form) the RK register g reach shared memory by bulk copies on
// the TMA engine (an even number of nodes per direction) or per-thread
// cp.async, issued at the start and awaited before the surface term.
#pragma once

#include <stddef.h>

#include "internal.cuh"
#include "lowmach.cuh"
#include "physics.cuh"

namespace hs3d {

template <int FORM>
constexpr bool dev_lowmach()
{
    return FORM == HS3D_VOL_STANDARD || FORM == HS3D_VOL_EC;
}

template <int N>
constexpr int dev_threads()
{
    constexpr int t = ((N + 1) * (N + 1) * (N + 1) > 256) ? (N + 1) * (N + 1) * (N + 1) : 256;
    return (t + 31) & ~31;
}

// Staged floats per node:
//   standard   [d][4] FP32 fluxes (momentum, energy rest), [d][hi, lo] of Ja^d.m'      18
//   EC         rho', v'(3), beta', |v|^2 - |vbar|^2, m'(3), Ja - Ja_centre [d][3],
//              [d][hi, lo] of Ja^d.m', NS: [d][4] viscous contravariant fluxes      24 (+12)
//   other      7 two-point inputs, Jaf [d][3], NS: [d][4] viscous fluxes             16 (+12)
template <int FORM, bool NS>
constexpr int dev_per_node()
{
    return (FORM == HS3D_VOL_STANDARD) ? 18 : (FORM == HS3D_VOL_EC ? 24 : 16) + (NS ? 12 : 0);
}

template <int FORM, bool NS>
constexpr int dev_visc_off()
{
    return FORM == HS3D_VOL_EC ? 24 : 16;
}

// Per-element block of shared memory, 36 floats: the element's reference
// state record, copied in by the element's first seven threads before a
// barrier at the start (FP64 conserved values [0, 10), the FP32 Anchor
// [10, 26)), and the centre node's metric terms (EC, [26, 35)).  Read from
// shared memory, the record holds no registers while the node's inputs are
// in flight.
constexpr int kDevElemBlock = 36;
static_assert(sizeof(Anchor) == 16 * sizeof(float) && offsetof(AnchorRec, a) == 10 * sizeof(float),
              "reference-state record layout");

// Byte offset of the RK staging block (16-byte aligned): D, Dlo, per-element
// blocks, per-node staging, face blocks, pair buffers (split forms).
template <int N, bool NS, int FORM>
__host__ __device__ constexpr size_t dev_rk_offset(int epb)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr size_t pairs = (FORM == HS3D_VOL_STANDARD) ? 0 : (size_t)5 * (n / 2) * n3;
    const size_t fl = 2 * ((n2 + 3) & ~3) + (size_t)epb * kDevElemBlock + (size_t)epb * dev_per_node<FORM, NS>() * n3 +
                      (size_t)epb * 30 * n2 + (size_t)epb * pairs;
    return (sizeof(float) * fl + 15) & ~(size_t)15;
}

// RK staging: standard form g [epb][5 n3] (FP32), then 1/J [epb][n3] (FP32).
template <int N, bool NS, int FORM>
__host__ __device__ constexpr size_t dev_smem_bytes(int epb)
{
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    constexpr bool SG = (FORM == HS3D_VOL_STANDARD);
    return dev_rk_offset<N, NS, FORM>(epb) + (size_t)epb * n3 * ((SG ? 20 : 0) + 4);
}

// The node's FP64 state read again after the pair phase instead of being
// kept in registers across it (an L2 hit; registers are the kernel's
// limit): a load the compiler does not merge with the first one.
__device__ __forceinline__ double reload_state(const double *ptr)
{
    double x;
    asm volatile("ld.global.f64 %0, [%1];" : "=d"(x) : "l"(ptr));
    return x;
}

template <int n>
__device__ __forceinline__ int dev_line_node(int d, int idx, int ta, int tb)
{
    if (d == 0) return idx + n * (ta + n * tb);
    if (d == 1) return ta + n * (idx + n * tb);
    return ta + n * (tb + n * idx);
}

// Minimum resident CTAs asked of the compiler (its register budget), for
// CTAs of up to 256 threads: the split forms 4 (64 registers; with about
// 55 KB of shared memory per CTA, 4 are resident; ~56 bytes of spills per
// thread, and still 8-12% faster than 3 CTAs at 80 registers, 16^3 and 32^3
// N = 3, EC and KG); the standard form 5 up to N = 3 (48 registers, ~50
// bytes of spills: -4% at 64^3 N = 3) and 4 above (no spills; 5 measured
// +3% at N = 4).
template <int N, int FORM>
constexpr int dev_min_blocks()
{
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    if (n3 > 256) return 2;
    return (FORM == HS3D_VOL_STANDARD && n3 <= 64) ? 5 : 4;
}

// One tile (epb elements) of the element kernel; returns true on the
// thread that initialised its element's bulk-copy barrier.  MORT: the items
// take their face fluxes from the mortar kernels (Item::face6).
template <int N, bool NS, int FORM, bool MORT>
__device__ __forceinline__ bool volume_dev_tile(const Batch &b, const Ops *__restrict__ ops, int stage, double rkA,
                                                double rkB, int lam_slot, int epb, long long tile,
                                                unsigned long long *bulk_bar)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr bool STD = (FORM == HS3D_VOL_STANDARD);
    constexpr bool EC = (FORM == HS3D_VOL_EC);
    constexpr bool LM = dev_lowmach<FORM>();
    constexpr int PER = dev_per_node<FORM, NS>();
    constexpr int VOFF = dev_visc_off<FORM, NS>();
    constexpr int KP = n / 2;
    constexpr bool BULK = (n % 2 == 0);
    constexpr int D2 = (n2 + 3) & ~3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sD = (float *)smem_raw;
    float *sDl = sD + D2;
    float *selem = sDl + D2;
    float *sbuf = selem + (size_t)epb * kDevElemBlock;
    float *sface = sbuf + (size_t)epb * PER * n3;
    float *spair = sface + (size_t)epb * 30 * n2;
    float *sG = (float *)(smem_raw + dev_rk_offset<N, NS, FORM>(epb));
    float *sIJ = (float *)(sG + (STD ? (size_t)epb * 5 * n3 : 0));
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        sD[t] = ops->Df[t];
        sDl[t] = ops->Dlo[t];
    }
    const int le = threadIdx.x / n3, p = threadIdx.x - le * n3;
    const long long ge = tile * epb + le;
    bool valid = le < epb && ge < b.total_elems;
    const Item *itp = nullptr;
    int e = 0;
    if (valid) {
        itp = &find_item_elem(b, ge);
        e = (int)(ge - itp->elem_begin);
        if (itp->clk && itp->clk->done) valid = false;
    }
    const bool armed = BULK && valid && p == 0;
    float *S = sbuf + (size_t)le * PER * n3;
    float *F6 = sface + (size_t)le * 30 * n2;
    float *PB = spair + (size_t)le * 5 * KP * n3;
    double *AD = (double *)(selem + (size_t)le * kDevElemBlock);     // reference state, FP64 conserved
    Anchor *ANC = (Anchor *)(selem + (size_t)le * kDevElemBlock + 10);
    float *CEN = selem + (size_t)le * kDevElemBlock + 26;            // centre metric terms (EC)
    const int ijk[3] = {p % n, (p / n) % n, p / n2};
    constexpr int pc = anchor_node(n);   // centre node: the element's reference state

    double u[5];
    if (valid) {
        if constexpr (n3 > 256) {
            // N = 7: the element's metric terms and gradients toward L2 ahead of
            // their per-thread loads (-3% at 24^3; at N = 3 it measured +1-2%)
            prefetch_l2_block(itp->Jaf + (size_t)e * 9 * n3, sizeof(float) * 9 * n3, p, n3);
            if (LM) prefetch_l2_block(itp->Jalo + (size_t)e * 9 * n3, sizeof(float) * 9 * n3, p, n3);
            if (NS) prefetch_l2_block((const float *)itp->grad + (size_t)e * 12 * n3, sizeof(float) * 12 * n3, p, n3);
        }
        const double *U = itp->u + (size_t)e * 5 * n3;
#pragma unroll
        for (int v = 0; v < 5; ++v) u[v] = U[v * n3 + p];
        // the element's reference state, left by the pass before, into its shared
        // block (its first 26 floats: the record's padding would overwrite CEN)
        if (p < 7) {
            const float4 x = __ldg((const float4 *)((const AnchorRec *)itp->anc + e) + p);
            float *blk = selem + (size_t)le * kDevElemBlock;
            if (p < 6) ((float4 *)blk)[p] = x;
            else ((float2 *)blk)[12] = make_float2(x.x, x.y);
        }
        // the thread that initialises the element's barrier is the one that arms it
        // and issues the copies; the others poll it only after the staging barrier
        if (BULK && p == 0) mbar_init(bulk_bar + le, 1);
    }
    __syncthreads();
    float V[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    float Ch = 0.0f, Cl = 0.0f;   // float-float C (low-Mach forms)
    float Hb = 0.0f;
    if (valid) {
        const Item &it = *itp;
        const Nbrs nb = elem_nbrs(e, it.ex, it.ey, it.ez);
        // face blocks of this element's side of its six faces, 1/J, g
        {
            const float *gf = (const float *)it.g;   // the RK register: FP32 on this path
            const float *FS = (const float *)it.fstar;
            size_t blk[6];
#pragma unroll
            for (int slot = 0; slot < 6; ++slot) {
                const int d = slot >> 1;
                if (MORT) blk[slot] = ((size_t)slot * it.E + e) * 5 * n2;
                else if (slot & 1) blk[slot] = (((size_t)d * it.E + e) * 2 + 0) * 5 * n2;
                else blk[slot] = (((size_t)d * it.E + nb.m[d]) * 2 + 1) * 5 * n2;
            }
            if constexpr (BULK) {
                if (p == 0) {
                    unsigned long long *bar = bulk_bar + le;
                    constexpr unsigned fb = 5 * n2 * 4, gb = 5 * n3 * 4, jb = n3 * 4;
                    mbar_arrive_expect_tx(bar, 6 * fb + jb + (STD && stage > 0 ? gb : 0));
#pragma unroll
                    for (int slot = 0; slot < 6; ++slot) bulk_g2s(F6 + slot * 5 * n2, FS + blk[slot], fb, bar);
                    bulk_g2s(sIJ + (size_t)le * n3, it.invJf + (size_t)e * n3, jb, bar);
                    if (STD && stage > 0) bulk_g2s(sG + (size_t)le * 5 * n3, gf + (size_t)e * 5 * n3, gb, bar);
                }
            } else {
#pragma unroll
                for (int slot = 0; slot < 6; ++slot) cp_async_block<float>(F6 + slot * 5 * n2, FS + blk[slot], 5 * n2, p, n3);
                cp_async_block<float>(sIJ + (size_t)le * n3, it.invJf + (size_t)e * n3, n3, p, n3);
                if (STD && stage > 0) cp_async_block<float>(sG + (size_t)le * 5 * n3, gf + (size_t)e * 5 * n3, 5 * n3, p, n3);
            }
            if constexpr (!STD) {
                if (stage > 0) prefetch_l2_block(gf + (size_t)e * 5 * n3, sizeof(float) * 5 * n3, p, n3);
            }
        }
        const float gm1 = it.gm1f, hg = it.hgf;
        const Anchor A = *ANC;
        double ad[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) ad[v] = AD[v];
        Hb = A.H;
        // momentum deviations as FP32 pairs (hi: the deviation rounded once; lo: the rest)
        float mh[3], ml[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) ff_split(u[1 + c] - ad[1 + c], mh[c], ml[c]);
        const Dev dv = make_dev_f(dev_round(u[0] - ad[0]), mh[0], mh[1], mh[2], dev_round(u[4] - ad[4]), A, gm1);
        const Prim<float> q = dev_prim(dv, A);
        float ja[9];
        const float *JA = it.Jaf + (size_t)e * 9 * n3;
#pragma unroll
        for (int k = 0; k < 9; ++k) ja[k] = JA[k * n3 + p];
        float G[12];
        if (NS) {
            const float *Gp = (const float *)it.grad + (size_t)e * 12 * n3 + p;
#pragma unroll
            for (int k = 0; k < 12; ++k) G[k] = Gp[k * n3];
        }
        if constexpr (LM) {
            // Ja^d.m' in float-float: m' = (mh, ml) from the FP64 deviation,
            // Ja = Jaf + Jalo
            const float *JL = it.Jalo + (size_t)e * 9 * n3;
            constexpr int WOFF = STD ? 12 : 18;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float wh = 0.0f, wl = 0.0f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (c == 0) ff_mul(wh, wl, ja[d * 3], JL[(d * 3) * n3 + p], mh[0], ml[0]);
                    else ff_fma(wh, wl, ja[d * 3 + c], JL[(d * 3 + c) * n3 + p], mh[c], ml[c]);
                }
                S[(WOFF + 2 * d) * n3 + p] = wh;
                S[(WOFF + 2 * d + 1) * n3 + p] = wl;
            }
        }
        if constexpr (STD) {
            const float dH = dev_dH(dv, A);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                float f[4];
                dflux_euler_rest(dv, A, dH, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], f);
                if (NS) {
                    float fv[5];
                    visc_flux(q, G, it.muf, it.kappaf, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fv);
#pragma unroll
                    for (int v = 0; v < 4; ++v) f[v] -= fv[v + 1];
                }
#pragma unroll
                for (int v = 0; v < 4; ++v) S[(d * 4 + v) * n3 + p] = f[v];
            }
        } else if constexpr (EC) {
            const ECDev z = ec_dev(dv, A);
            S[0 * n3 + p] = z.dr;
            S[1 * n3 + p] = z.dv1;
            S[2 * n3 + p] = z.dv2;
            S[3 * n3 + p] = z.dv3;
            S[4 * n3 + p] = z.db;
            S[5 * n3 + p] = z.q;
            S[6 * n3 + p] = dv.dm1;
            S[7 * n3 + p] = dv.dm2;
            S[8 * n3 + p] = dv.dm3;
            // metric terms as deviations from the centre node's, accurate to FP32
            // relative to the deviation (their differences enter e_im)
            const float *JL = it.Jalo + (size_t)e * 9 * n3;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float jc = JA[k * n3 + pc], jlc = JL[k * n3 + pc];
                S[(9 + k) * n3 + p] = (ja[k] - jc) + (JL[k * n3 + p] - jlc);
                if (p == 0) CEN[k] = jc;
            }
            // the diagonal pair (i, i), nonzero on the boundary nodes only
            // (D_ii = 0 inside): the same two-point function as every other pair,
            // so that the reference flux dropped is the same; its mass remainder
            // e_ii is zero (the conservative part carries F_rho(u_i))
            // (D from the operator table: shared memory is not yet synchronised)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (ijk[d] == 0 || ijk[d] == N) {
                    const float dd = ops->Df[ijk[d] * n + ijk[d]];
                    float fm[3], rest;
                    dflux_ec_diag(z, A, hg, 2.0f * ja[d * 3], 2.0f * ja[d * 3 + 1], 2.0f * ja[d * 3 + 2], fm, rest);
                    V[1] += dd * fm[0];
                    V[2] += dd * fm[1];
                    V[3] += dd * fm[2];
                    V[4] += dd * rest;
                }
                if (NS) {
                    float fv[5];
                    visc_flux(q, G, it.muf, it.kappaf, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fv);
#pragma unroll
                    for (int v = 0; v < 4; ++v) S[(VOFF + d * 4 + v) * n3 + p] = fv[v + 1];
                }
            }
        } else {
            // other split forms: full FP32 two-point flux inputs
            float z[kSplitSlots];
            split_node<FORM>(q, z);
#pragma unroll
            for (int k = 0; k < kSplitSlots; ++k) S[k * n3 + p] = z[k];
#pragma unroll
            for (int k = 0; k < 9; ++k) S[(7 + k) * n3 + p] = ja[k];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float dd = 2.0f * ops->Df[ijk[d] * n + ijk[d]];
                float fe[5];
                euler_flux(q, q.E, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fe);
#pragma unroll
                for (int v = 0; v < 5; ++v) V[v] += dd * fe[v];
                if (NS) {
                    float fv[5];
                    visc_flux(q, G, it.muf, it.kappaf, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fv);
#pragma unroll
                    for (int v = 0; v < 4; ++v) S[(VOFF + d * 4 + v) * n3 + p] = fv[v + 1];
                }
            }
        }
    }
    if constexpr (!BULK) cp_async_wait_all();
    __syncthreads();

    if constexpr (STD) {
        if (valid) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int stride = (d == 0) ? 1 : (d == 1) ? n : n2;
                const int base = p - ijk[d] * stride;
                const float *Drow = sD + ijk[d] * n;
                const float *Dlrow = sDl + ijk[d] * n;
#pragma unroll
                for (int m = 0; m < n; ++m) {
                    const float Dm = Drow[m];
                    const int pm = base + m * stride;
#pragma unroll
                    for (int v = 0; v < 4; ++v) V[v + 1] += Dm * S[(d * 4 + v) * n3 + pm];
                    if (d == 0 && m == 0) ff_mul(Ch, Cl, Dm, Dlrow[m], S[(12 + 2 * d) * n3 + pm], S[(13 + 2 * d) * n3 + pm]);
                    else ff_fma(Ch, Cl, Dm, Dlrow[m], S[(12 + 2 * d) * n3 + pm], S[(13 + 2 * d) * n3 + pm]);
                }
            }
        }
    } else {
        const float hg = valid ? itp->hgf : 0.0f;
        const float gam = valid ? itp->gammaf : 0.0f;
        Anchor A{};
        if (EC && valid) A = *ANC;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int sd = (d == 0) ? 1 : (d == 1) ? n : n2;
            // N = 3: the x- and y-lines of a 64-thread element lie inside one warp,
            // so their pair fluxes go to the partner node by warp shuffles (no pair
            // buffer, no barrier); z-lines span two warps and take the shared-memory
            // pair buffer below
            const bool shfl = n == 4 && d < 2;
            if (shfl) {
                const int x = ijk[d];
                const int lane = threadIdx.x & 31;
                const float *Drow = sD + x * n;
                const float *DA = S + (9 + d * 3) * n3;   // Chandrashekar form: metric deviations
                const float *SJ = S + (7 + d * 3) * n3;   // other split forms: metric terms
                ECDev za{};
                float dma[3] = {0.0f, 0.0f, 0.0f}, da[3] = {0.0f, 0.0f, 0.0f};
                float c1 = 0.0f, c2 = 0.0f, c3 = 0.0f;
                float zo[kSplitSlots];
#pragma unroll
                for (int q = 0; q < kSplitSlots; ++q) zo[q] = 0.0f;
                if (valid) {
                    if constexpr (EC) {
                        za = {S[p], S[n3 + p], S[2 * n3 + p], S[3 * n3 + p], S[4 * n3 + p], S[5 * n3 + p]};
                        dma[0] = S[6 * n3 + p];
                        dma[1] = S[7 * n3 + p];
                        dma[2] = S[8 * n3 + p];
                        da[0] = DA[p];
                        da[1] = DA[n3 + p];
                        da[2] = DA[2 * n3 + p];
                        c1 = 2.0f * CEN[d * 3];
                        c2 = 2.0f * CEN[d * 3 + 1];
                        c3 = 2.0f * CEN[d * 3 + 2];
                    } else {
#pragma unroll
                        for (int q = 0; q < kSplitSlots; ++q) zo[q] = S[q * n3 + p];
                        c1 = SJ[p];
                        c2 = SJ[n3 + p];
                        c3 = SJ[2 * n3 + p];
                    }
                }
#pragma unroll
                for (int k = 1; k <= KP; ++k) {
                    // this node's thread evaluates the pair (x, x + k mod n) (for k = n/2 the
                    // lower half of the line only) and receives the pair (x - k mod n, x)
                    const bool own = !(2 * k == n && x >= KP);
                    const bool recv = !(2 * k == n && x < KP);
                    float fp[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
                    if (valid && own) {
                        const int xm = (x + k < n) ? x + k : x + k - n;
                        const int c = p + (xm - x) * sd;
                        if constexpr (EC) {
                            const ECDev zc = {S[c], S[n3 + c], S[2 * n3 + c], S[3 * n3 + c], S[4 * n3 + c], S[5 * n3 + c]};
                            const float dc[3] = {DA[c], DA[n3 + c], DA[2 * n3 + c]};
                            float frho, rmass, fm[3], rest;
                            dflux_ec(za, zc, A, hg, c1 + da[0] + dc[0], c2 + da[1] + dc[1], c3 + da[2] + dc[2], frho,
                                     rmass, fm, rest);
                            const float dm1 = dma[0] - S[6 * n3 + c], dm2 = dma[1] - S[7 * n3 + c],
                                        dm3 = dma[2] - S[8 * n3 + c];
                            fp[0] = rmass - 0.5f * (dm1 * (da[0] - dc[0]) + dm2 * (da[1] - dc[1]) + dm3 * (da[2] - dc[2]));
                            fp[1] = fm[0];
                            fp[2] = fm[1];
                            fp[3] = fm[2];
                            fp[4] = rest;
                        } else {
                            float zc[kSplitSlots];
#pragma unroll
                            for (int q = 0; q < kSplitSlots; ++q) zc[q] = S[q * n3 + c];
                            split_pair<FORM>(zo, zc, gam, hg, c1 + SJ[c], c2 + SJ[n3 + c], c3 + SJ[2 * n3 + c], fp);
                        }
                        const float Dm = Drow[xm];
#pragma unroll
                        for (int v = 0; v < 5; ++v) V[v] += Dm * fp[v];
                    }
                    const int xs = (x >= k) ? x - k : x - k + n;
                    const int src = lane + (xs - x) * sd;
                    float fr[5];
#pragma unroll
                    for (int v = 0; v < 5; ++v) fr[v] = __shfl_sync(0xffffffffu, fp[v], src);
                    if (valid && recv) {
                        const float Dm = Drow[xs];
#pragma unroll
                        for (int v = 0; v < 5; ++v) V[v] += Dm * fr[v];
                    }
                }
                if (valid) {
                    const int base = p - x * sd;
                    const float *Dlrow = sDl + x * n;
#pragma unroll
                    for (int m = 0; m < n; ++m) {
                        const float Dm = Drow[m];
                        const int pm = base + m * sd;
                        if (NS) {
#pragma unroll
                            for (int v = 0; v < 4; ++v) V[v + 1] -= Dm * S[(VOFF + d * 4 + v) * n3 + pm];
                        }
                        if constexpr (EC) {
                            if (d == 0 && m == 0) ff_mul(Ch, Cl, Dm, Dlrow[m], S[(18 + 2 * d) * n3 + pm], S[(19 + 2 * d) * n3 + pm]);
                            else ff_fma(Ch, Cl, Dm, Dlrow[m], S[(18 + 2 * d) * n3 + pm], S[(19 + 2 * d) * n3 + pm]);
                        }
                    }
                }
                continue;
            }
            if (valid) {
                // the thread of node a (index x along d) evaluates the pairs (x, x + k mod n)
                // of its line: consecutive threads read consecutive nodes, without the
                // shared-memory bank conflicts of a line-major assignment (the k = n/2
                // pairs then occupy half of each warp's lanes; measured at 16^3 N = 3:
                // -6% for this kernel; the FP64 kernel, bound by its FP64 pipe, keeps the
                // line-major assignment, for which this measured +8%)
                const int x = ijk[d];
                const int a = p;
                if constexpr (EC) {
                    const ECDev za = {S[a], S[n3 + a], S[2 * n3 + a], S[3 * n3 + a], S[4 * n3 + a], S[5 * n3 + a]};
                    const float dma[3] = {S[6 * n3 + a], S[7 * n3 + a], S[8 * n3 + a]};
                    const float *DA = S + (9 + d * 3) * n3;
                    const float da[3] = {DA[a], DA[n3 + a], DA[2 * n3 + a]};
                    const float c1 = 2.0f * CEN[d * 3], c2 = 2.0f * CEN[d * 3 + 1], c3 = 2.0f * CEN[d * 3 + 2];
#pragma unroll
                    for (int k = 1; k <= KP; ++k) {
                        if (2 * k == n && x >= KP) break;
                        const int xm = (x + k < n) ? x + k : x + k - n;
                        const int c = a + (xm - x) * sd;
                        const ECDev zc = {S[c], S[n3 + c], S[2 * n3 + c], S[3 * n3 + c], S[4 * n3 + c], S[5 * n3 + c]};
                        const float dc[3] = {DA[c], DA[n3 + c], DA[2 * n3 + c]};
                        float frho, rmass, fm[3], rest;
                        dflux_ec(za, zc, A, hg, c1 + da[0] + dc[0], c2 + da[1] + dc[1], c3 + da[2] + dc[2], frho, rmass,
                                 fm, rest);
                        const float dm1 = dma[0] - S[6 * n3 + c], dm2 = dma[1] - S[7 * n3 + c], dm3 = dma[2] - S[8 * n3 + c];
                        const float em = rmass - 0.5f * (dm1 * (da[0] - dc[0]) + dm2 * (da[1] - dc[1]) + dm3 * (da[2] - dc[2]));
                        PB[(0 * KP + k - 1) * n3 + p] = em;
                        PB[(1 * KP + k - 1) * n3 + p] = fm[0];
                        PB[(2 * KP + k - 1) * n3 + p] = fm[1];
                        PB[(3 * KP + k - 1) * n3 + p] = fm[2];
                        PB[(4 * KP + k - 1) * n3 + p] = rest;
                    }
                } else {
                    float za[kSplitSlots];
#pragma unroll
                    for (int k = 0; k < kSplitSlots; ++k) za[k] = S[k * n3 + a];
                    const float *SJ = S + (7 + d * 3) * n3;
                    const float j1 = SJ[a], j2 = SJ[n3 + a], j3 = SJ[2 * n3 + a];
#pragma unroll
                    for (int k = 1; k <= KP; ++k) {
                        if (2 * k == n && x >= KP) break;
                        const int xm = (x + k < n) ? x + k : x + k - n;
                        const int c = a + (xm - x) * sd;
                        float zc[kSplitSlots];
#pragma unroll
                        for (int qq = 0; qq < kSplitSlots; ++qq) zc[qq] = S[qq * n3 + c];
                        float fs[5];
                        split_pair<FORM>(za, zc, gam, hg, j1 + SJ[c], j2 + SJ[n3 + c], j3 + SJ[2 * n3 + c], fs);
#pragma unroll
                        for (int v = 0; v < 5; ++v) PB[(v * KP + k - 1) * n3 + p] = fs[v];
                    }
                }
            }
            __syncthreads();
            if (valid) {
                const int i = ijk[d];
                const int base = p - i * sd;
                const float *Drow = sD + i * n;
                const float *Dlrow = sDl + i * n;
#pragma unroll
                for (int m = 0; m < n; ++m) {
                    const float Dm = Drow[m];
                    if (m != i) {
                        const int k = (m > i) ? m - i : m - i + n;
                        int slot, x;
                        if (2 * k < n) {
                            slot = k;
                            x = i;
                        } else if (2 * k > n) {
                            slot = n - k;
                            x = m;
                        } else {
                            slot = KP;
                            x = (i < KP) ? i : m;
                        }
                        // (the pair sits with the thread of its node x, in slot k - 1)
                        const float *F = PB + (slot - 1) * n3 + base + x * sd;
#pragma unroll
                        for (int v = 0; v < 5; ++v) V[v] += Dm * F[v * KP * n3];
                    }
                    const int pm = base + m * sd;
                    if (NS) {
#pragma unroll
                        for (int v = 0; v < 4; ++v) V[v + 1] -= Dm * S[(VOFF + d * 4 + v) * n3 + pm];
                    }
                    if constexpr (EC) {
                        if (d == 0 && m == 0) ff_mul(Ch, Cl, Dm, Dlrow[m], S[(18 + 2 * d) * n3 + pm], S[(19 + 2 * d) * n3 + pm]);
                        else ff_fma(Ch, Cl, Dm, Dlrow[m], S[(18 + 2 * d) * n3 + pm], S[(19 + 2 * d) * n3 + pm]);
                    }
                }
            }
            // (after the last direction the pair buffer is not written again)
            if (d < 2) __syncthreads();
        }
    }
    if constexpr (BULK) {
        if (valid && !mbar_wait(bulk_bar + le, 0, kBulkWaitPolls)) {
#pragma unroll
            for (int v = 0; v < 5; ++v) V[v] = NAN;
            if (itp->clk) itp->clk->bad = 2;
        }
    }
    double lc = 0.0, lv = 0.0;
    bool lam_active = false;
    if (valid) {
    const Item &it = *itp;
    // the epilogue's global inputs, issued before the surface term so that their
    // latency overlaps it: the FP64 state (not kept in registers across the pair
    // phase), dt and the RK register's previous value (split forms; the standard
    // form has it in shared memory)
    float *Gp = (float *)it.g + (size_t)e * 5 * n3 + p;
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = reload_state(it.u + (size_t)e * 5 * n3 + v * n3 + p);
    double dtv = 0.0;
    float gprev[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (stage >= 0) {
        dtv = it.clk->dt;
        if (!STD && stage > 0) {
#pragma unroll
            for (int v = 0; v < 5; ++v) gprev[v] = Gp[v * n3];
        }
    }
    const float iw = ops->iw0f;
    // volume rows: mass = C (+ the split form's remainder), energy = Hbar mass + rest
    float Vr = V[0];
    if constexpr (LM) {
        Vr = (Ch + Cl) + V[0];
        V[4] += Hb * Vr;
    }
    V[0] = Vr;
    // surface term
    float own[3][5];
    bool need_own = false;
    if constexpr (MORT) {
        // mortar flux minus the own FP32 flux (full values)
#pragma unroll
        for (int d = 0; d < 3; ++d) need_own |= (ijk[d] == 0 || ijk[d] == N);
        if (need_own) {
            const Anchor A = *ANC;
            double ad[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) ad[v] = AD[v];
            const Prim<float> q = dev_prim(make_dev(u, ad, A, it.gm1f), A);
            float G[12];
            if (NS) {
                const float *Gp = (const float *)it.grad + (size_t)e * 12 * n3 + p;
#pragma unroll
                for (int k = 0; k < 12; ++k) G[k] = Gp[k * n3];
            }
            const float *JA = it.Jaf + (size_t)e * 9 * n3 + p;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                if (ijk[d] != 0 && ijk[d] != N) continue;
                const float a1 = JA[(d * 3) * n3], a2 = JA[(d * 3 + 1) * n3], a3 = JA[(d * 3 + 2) * n3];
                euler_flux(q, q.E, a1, a2, a3, own[d]);
                if (NS) {
                    float fv[5];
                    visc_flux(q, G, it.muf, it.kappaf, a1, a2, a3, fv);
#pragma unroll
                    for (int v = 1; v < 5; ++v) own[d][v] -= fv[v];
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        if (ijk[d] != N && ijk[d] != 0) continue;
        const int ta = (d == 0) ? ijk[1] : ijk[0];
        const int tb = (d == 2) ? ijk[1] : ijk[2];
        const int ab = ta + n * tb;
        const bool plus = ijk[d] == N;
        const float *F = F6 + (2 * d + (plus ? 1 : 0)) * 5 * n2 + ab;
        if constexpr (MORT) {
#pragma unroll
            for (int v = 0; v < 5; ++v) V[v] += plus ? iw * (F[v * n2] - own[d][v]) : iw * (own[d][v] - F[v * n2]);
        } else {
#pragma unroll
            for (int v = 0; v < 5; ++v) V[v] += plus ? iw * F[v * n2] : -iw * F[v * n2];
        }
    }
    // residual store or RK stage (FP64 accumulation), then the dt maxima
    const float ijf = sIJ[(size_t)le * n3 + p];
    if (stage < 0) {
        double *O = it.out + (size_t)e * 5 * n3 + p;
#pragma unroll
        for (int v = 0; v < 5; ++v) O[v * n3] = f2d_exact(-V[v] * ijf);
    } else {
        // the register g holds FP32 increments (dt R is an FP32 quantity here);
        // the state accumulates in FP64: u <- u + B g, one FP64 FMA a variable
        const float sdt = d2f_rn(dtv) * ijf;
        const float rkAf = d2f_rn(rkA);
        double *Up = it.u + (size_t)e * 5 * n3 + p;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float inc = -V[v] * sdt;
            float gv;
            if (stage == 0) gv = inc;
            else gv = fmaf(rkAf, STD ? sG[(size_t)le * 5 * n3 + v * n3 + p] : gprev[v], inc);
            Gp[v * n3] = gv;
            u[v] = fma(rkB, f2d_exact(gv), u[v]);
            Up[v * n3] = u[v];
        }
        float nf[5];
        if (it.uf || lam_slot >= 0) {
#pragma unroll
            for (int v = 0; v < 5; ++v) nf[v] = d2f_rn(u[v]);
        }
        if (it.uf) {
            float *Sp = it.uf + (size_t)e * 5 * n3 + p;
#pragma unroll
            for (int v = 0; v < 5; ++v) Sp[v * n3] = nf[v];
        }
        // the reference state of the next stage (every thread of this element
        // has read the current one: barriers lie in between)
        if (p == pc && it.anc) write_anchor(it, e, u);
        if (lam_slot >= 0) {
            const Prim<float> qn = prim_from_f(nf, it.gm1f);
            if (!(qn.rho > 0.0f) || !(qn.p > 0.0f)) {
                it.clk->bad = 1;
            } else {
                const float c = sqrtf(it.gammaf * qn.p / qn.rho);
                const float *JA = it.Jaf + (size_t)e * 9 * n3 + p;
                float sc = 0.0f, sv = 0.0f;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const float a1 = JA[(d * 3) * n3], a2 = JA[(d * 3 + 1) * n3], a3 = JA[(d * 3 + 2) * n3];
                    const float an = sqrtf(a1 * a1 + a2 * a2 + a3 * a3);
                    sc += (fabsf(a1 * qn.v1 + a2 * qn.v2 + a3 * qn.v3) + c * an) * ijf;
                    sv += (an * ijf) * (an * ijf);
                }
                lc = f2d_exact(sc);
                lv = NS ? f2d_exact(it.muf * sv / qn.rho) : 0.0;
                lam_active = true;
            }
        }
    }
    }
    if (lam_slot >= 0 && stage >= 0) {
        unsigned long long *dc = nullptr, *dvp = nullptr;
        if (lam_active) {
            dc = &itp->clk->lam[lam_slot][0];
            dvp = NS ? &itp->clk->lam[lam_slot][1] : nullptr;
        }
        warp_max_to_clock(dc, dvp, lc, lv, lam_active);
    }
    return armed;
}

// The tile as a separate function for the persistent loop (inlined into a
// loop, its values were hoisted across iterations and spilled).
template <int N, bool NS, int FORM>
__device__ __noinline__ bool volume_dev_tile_call(const Batch &b, const Ops *__restrict__ ops, int stage, double rkA,
                                                  double rkB, int lam_slot, int epb, long long tile,
                                                  unsigned long long *bulk_bar)
{
    return volume_dev_tile<N, NS, FORM, false>(b, ops, stage, rkA, rkB, lam_slot, epb, tile, bulk_bar);
}

// The element kernel: a CTA per tile, or (PERSIST, Batch::persistent) a
// persistent grid whose CTAs walk the tiles with a stride of the grid size,
// reusing their shared memory; a tile's element barriers are invalidated
// before the next tile initialises them again.
template <int N, bool NS, int FORM, bool PERSIST, bool MORT = false>
__global__ void __launch_bounds__(dev_threads<N>(), dev_min_blocks<N, FORM>())
k_volume_dev(const __grid_constant__ Batch b, const Ops *__restrict__ ops, int stage, double rkA, double rkB,
             int lam_slot, int epb, long long ntiles)
{
    pdl_wait();
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    constexpr bool BULK = ((N + 1) % 2 == 0);
    __shared__ unsigned long long bulk_bar[BULK ? 256 / (n3 < 256 ? n3 : 256) : 1];
    if constexpr (!PERSIST) {
        volume_dev_tile<N, NS, FORM, MORT>(b, ops, stage, rkA, rkB, lam_slot, epb, blockIdx.x, bulk_bar);
    } else {
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const bool armed =
                volume_dev_tile_call<N, NS, FORM>(b, ops, stage, rkA, rkB, lam_slot, epb, tile, bulk_bar);
            if (tile + gridDim.x >= ntiles) break;   // (uniform across the CTA)
            __syncthreads();
            if (armed) mbar_inval(bulk_bar + threadIdx.x / n3);
        }
    }
}

// ------------------------------------------------------------------ launch (one volume form)

template <int N, bool NS, int FORM>
static cudaError_t vol_dev_launch2(const Batch &b, int stage, double rkA, double rkB, int lam_slot, cudaStream_t s)
{
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    int epb = elems_per_block_p(N, HS3D_MIXED32, 1);
    if (epb * n3 > dev_threads<N>()) epb = dev_threads<N>() / n3;
    if (epb < 1) epb = 1;
    const int threads = ((epb * n3) + 31) & ~31;
    const size_t smem = dev_smem_bytes<N, NS, FORM>(epb);
    const unsigned blocks = (unsigned)((b.total_elems + epb - 1) / epb);
    const Ops *ops = device_ops(N);
    if (!ops) return cudaErrorMemoryAllocation;
    if (b.persistent && !b.mortar) {
        const unsigned grid = persistent_grid(k_volume_dev<N, NS, FORM, true>, threads, smem, blocks);
        return launch_pdl(k_volume_dev<N, NS, FORM, true>, grid, threads, smem, s, b, ops, stage, rkA, rkB,
                          stage >= 0 ? lam_slot : -1, epb, (long long)blocks);
    }
    if (b.mortar)
        return launch_pdl(k_volume_dev<N, NS, FORM, false, true>, blocks, threads, smem, s, b, ops, stage, rkA, rkB,
                          stage >= 0 ? lam_slot : -1, epb, (long long)blocks);
    return launch_pdl(k_volume_dev<N, NS, FORM, false>, blocks, threads, smem, s, b, ops, stage, rkA, rkB,
                      stage >= 0 ? lam_slot : -1, epb, (long long)blocks);
}

template <int FORM>
cudaError_t launch_volume_dev_form(int N, int physics, const Batch &b, int stage, double rkA, double rkB, int lam_slot,
                                   cudaStream_t s)
{
    if (b.total_elems == 0) return cudaSuccess;
#define HS3D_VDN(K)                                                                                       \
    case K:                                                                                               \
        return physics == HS3D_NS ? vol_dev_launch2<K, true, FORM>(b, stage, rkA, rkB, lam_slot, s)       \
                                  : vol_dev_launch2<K, false, FORM>(b, stage, rkA, rkB, lam_slot, s);
    switch (N) {
        HS3D_VDN(1) HS3D_VDN(2) HS3D_VDN(3) HS3D_VDN(4) HS3D_VDN(5) HS3D_VDN(6) HS3D_VDN(7)
    }
#undef HS3D_VDN
    return cudaErrorInvalidValue;
}

template <typename K>
static cudaError_t prep_vol_dev_kernel(K kernel)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int N, int FORM>
static cudaError_t prep_vol_dev_n()
{
    cudaError_t e = prep_vol_dev_kernel(k_volume_dev<N, false, FORM, false>);
    if (e == cudaSuccess) e = prep_vol_dev_kernel(k_volume_dev<N, true, FORM, false>);
    if (e == cudaSuccess) e = prep_vol_dev_kernel(k_volume_dev<N, false, FORM, true>);
    if (e == cudaSuccess) e = prep_vol_dev_kernel(k_volume_dev<N, true, FORM, true>);
    if (e == cudaSuccess) e = prep_vol_dev_kernel(k_volume_dev<N, false, FORM, false, true>);
    if (e == cudaSuccess) e = prep_vol_dev_kernel(k_volume_dev<N, true, FORM, false, true>);
    return e;
}

template <int FORM>
cudaError_t prepare_volume_dev_form(int N)
{
    switch (N) {
        case 1: return prep_vol_dev_n<1, FORM>();
        case 2: return prep_vol_dev_n<2, FORM>();
        case 3: return prep_vol_dev_n<3, FORM>();
        case 4: return prep_vol_dev_n<4, FORM>();
        case 5: return prep_vol_dev_n<5, FORM>();
        case 6: return prep_vol_dev_n<6, FORM>();
        case 7: return prep_vol_dev_n<7, FORM>();
    }
    return cudaErrorInvalidValue;
}

#define HS3D_VOLUME_DEV_FORM_TU(FORM)                                                                          \
    template cudaError_t launch_volume_dev_form<FORM>(int, int, const Batch &, int, double, double, int,        \
                                                      cudaStream_t);                                            \
    template cudaError_t prepare_volume_dev_form<FORM>(int);

}  // namespace hs3d
