// Element kernel: volume term + surface lifting + Jacobian scaling + RK stage.
// (Template shared by the per-volume-form translation units volume_*.cu.)
//
// Strong form of Eq. NS5 (Sec. 3.3) on Gauss-Lobatto nodes, per element:
//   du/dt = -(V + S)/J
//   standard form   V = sum_d D_d F~^d,   F~^d = Ja^d . (F_e - F_v)
//   split form      V = sum_d sum_m D_im F#(u_i, u_m).(Ja^d_i + Ja^d_m) - sum_d D_d (Ja^d . F_v)
//                   with a symmetric two-point flux F# (Sec. 3.5): Chandrashekar,
//                   Kennedy-Gruber, Pirozzoli, Ducros, Morinishi or Ismail-Roe
//   surface         S = (1/w_end) (F^* - F~^d_in) on the +d face, (1/w_0)(-F^* + F~^d_in) on the -d face
//                   F^* the face flux computed once per face by k_face
// followed either by the residual store or by one low-storage RK stage
// (Sec. 3.7) g <- A_k g + dt R, u <- u + B_k g in FP64, with the stage's A_k,
// B_k passed by the host (Williamson RK3 or Carpenter-Kennedy RK4).  After
// the last stage the kernel also reduces the dt maxima of the updated state (the time
// step rule's input for the next step) so that no separate pass over the
// state is needed between steps.
//
// One thread per node, `epb` elements per CTA (a kernel argument; the
// tensor-core variant pads the CTA to whole warps).  The element's
// contravariant fluxes (standard form) or its per-node two-point-flux inputs
// (split form) are staged in shared memory.  The six face-flux blocks of the
// element (contiguous 5n^2 chunks) and, on the mixed path, its 1/J (standard
// form also u and g) are copied into shared memory at the start — by
// cp.async.bulk copies on the TMA engine counted on a per-element mbarrier
// when every block is a multiple of 16 bytes (an even number of nodes per
// direction), else by per-thread cp.async — so the surface term and the RK
// update read no global memory they could have waited for.
#pragma once

#include "internal.cuh"
#include "physics.cuh"

namespace hs3d {

// Largest CTA of the element kernel: 256 threads, or one element when it has
// more nodes, rounded up to whole warps (the tensor-core contraction needs
// complete warps; threads beyond the CTA's elements only join it).
template <int N>
constexpr int vol_threads()
{
    constexpr int t = ((N + 1) * (N + 1) * (N + 1) > 256) ? (N + 1) * (N + 1) * (N + 1) : 256;
    return (t + 31) & ~31;
}

// Minimum resident CTAs per SM asked of the compiler: the mixed path is
// latency bound, so its register budget is capped (64 per thread with
// 256- or 512-thread CTAs) to keep more warps resident; the FP64 path is
// bound by the FP64 pipe and keeps its registers.
template <int N, typename R>
constexpr int vol_min_blocks()
{
    return sizeof(R) == 4 ? (((N + 1) * (N + 1) * (N + 1) <= 256) ? 4 : 2) : 1;
}

// Number of R values staged per node.
template <int FORM, bool NS>
constexpr int vol_smem_per_node()
{
    return is_standard(FORM) ? 15 : (16 + (NS ? 15 : 0));
}

// Index of the 5 n^2 face-flux block of face `slot` of element e: the +d
// face's own block d E + e or the -d neighbour's d E + owner (conforming
// mesh), or the element's own per-face block slot E + e (face6).
__device__ __forceinline__ size_t face_block(const Item &it, int slot, int d, int owner, int e)
{
    return it.face6 ? (size_t)slot * it.E + e : (size_t)d * it.E + owner;
}

// Node with index `idx` along direction d on the line with tangential indices (ta, tb).
template <int n>
__device__ __forceinline__ int line_node(int d, int idx, int ta, int tb)
{
    if (d == 0) return idx + n * (ta + n * tb);
    if (d == 1) return ta + n * (idx + n * tb);
    return ta + n * (tb + n * idx);
}

template <typename R>
__device__ __forceinline__ const R *metric_ptr(const Item &it);
template <>
__device__ __forceinline__ const double *metric_ptr<double>(const Item &it) { return it.Ja; }
template <>
__device__ __forceinline__ const float *metric_ptr<float>(const Item &it) { return it.Jaf; }

// Residual store or RK stage of one node from V (volume + surface sum), then,
// after the last stage (lam_slot >= 0), the dt maxima of the updated state.
// u holds the FP64 state on the FP64 path (loaded here on the mixed path).
// Mixed path: sU and sG, when given, are the element's FP64 u and g
// blocks (5 n3 each) and sIJ its 1/J (FP32), staged in shared memory by
// asynchronous copies at the start of the kernel (g only for stage > 0).
template <typename R, bool NS>
__device__ __forceinline__ void node_update(const Item &it, int e, int p, int n3, const R V[5], double u[5],
                                            int stage, double rkA, double rkB, int lam_slot, double &lc, double &lv,
                                            bool &lam_active, const double *sU = nullptr, const double *sG = nullptr,
                                            const float *sIJ = nullptr)
{
    if constexpr (sizeof(R) == 4) {
        // the FP64 state is needed only for the RK accumulation
        if (stage >= 0) {
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = sU ? sU[v * n3 + p] : it.u[(size_t)e * 5 * n3 + p + v * n3];
        }
    }

    float nf[5];   // mixed path: FP32 shadow of the updated state
    if constexpr (sizeof(R) == 8) {
        const double ij = it.invJ[(size_t)e * n3 + p];
        if (stage < 0) {
            double *O = it.out + (size_t)e * 5 * n3 + p;
#pragma unroll
            for (int v = 0; v < 5; ++v) O[v * n3] = -(double)V[v] * ij;
        } else {
            const double dt = it.clk->dt;
            const double A = rkA, B = rkB;
            double *Gp = it.g + (size_t)e * 5 * n3 + p;
            double *Up = it.u + (size_t)e * 5 * n3 + p;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const double r = -(double)V[v] * ij;
                const double gv = (stage == 0) ? dt * r : A * Gp[v * n3] + dt * r;
                Gp[v * n3] = gv;
                u[v] = u[v] + B * gv;
                Up[v * n3] = u[v];
            }
        }
    } else {
        // mixed path: the increment dt R = -dt V / J is formed in FP32; the
        // register g holds FP32 increments ([E][5][n3] floats in the first half
        // of the caller's buffer) and the state accumulates in FP64 (one FP64
        // FMA per variable).
        const float ijf = sIJ ? sIJ[p] : it.invJf[(size_t)e * n3 + p];
        if (stage < 0) {
            double *O = it.out + (size_t)e * 5 * n3 + p;
#pragma unroll
            for (int v = 0; v < 5; ++v) O[v * n3] = f2d_exact(-(float)V[v] * ijf);
        } else {
            const float sdt = d2f_rn(it.clk->dt) * ijf;
            const float A = d2f_rn(rkA);
            const double B = rkB;
            float *Gp = (float *)it.g + (size_t)e * 5 * n3 + p;
            double *Up = it.u + (size_t)e * 5 * n3 + p;
            float *Sp = it.uf + (size_t)e * 5 * n3 + p;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                const float inc = -(float)V[v] * sdt;
                const float gv = (stage == 0) ? inc : fmaf(A, Gp[v * n3], inc);
                Gp[v * n3] = gv;
                u[v] = fma(B, f2d_exact(gv), u[v]);
                Up[v * n3] = u[v];
                nf[v] = d2f_rn(u[v]);
                Sp[v * n3] = nf[v];
            }
        }
    }
    if (stage >= 0) {
        if (lam_slot >= 0) {
            // dt maxima of the updated state (same rule as k_lambda, in R)
            const Phys<R> P = phys_of<R>(it);
            Prim<R> qn;
            if constexpr (sizeof(R) == 8) qn = prim_from_u<R>(u, P.gm1);
            else qn = prim_from_f(nf, P.gm1);
            if (!(qn.rho > (R)0) || !(qn.p > (R)0)) {
                it.clk->bad = 1;
            } else {
                const R c = sqrt(P.gamma * qn.p / qn.rho);
                R iJ;
                if constexpr (sizeof(R) == 8) iJ = it.invJ[(size_t)e * n3 + p];
                else iJ = sIJ ? sIJ[p] : it.invJf[(size_t)e * n3 + p];
                R sc = (R)0, sv = (R)0;
                const R *JA = metric_ptr<R>(it) + (size_t)e * 9 * n3 + p;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    const R a1 = JA[(d * 3) * n3], a2 = JA[(d * 3 + 1) * n3], a3 = JA[(d * 3 + 2) * n3];
                    const R an = sqrt(a1 * a1 + a2 * a2 + a3 * a3);
                    sc += (fabs(a1 * qn.v1 + a2 * qn.v2 + a3 * qn.v3) + c * an) * iJ;
                    sv += (an * iJ) * (an * iJ);
                }
                lc = widen<R>(sc);
                lv = NS ? widen<R>(P.mu * sv / qn.rho) : 0.0;
                lam_active = true;
            }
        }
    }
}

// Byte offsets in the element kernel's dynamic shared memory: D, the
// per-node staging of epb elements, their face-flux blocks, the split-form
// pair buffers, then (mixed path) the staged RK block [epb][u, g][5 n3]
// FP64 followed by [epb][n3] FP32 1/J, 16-byte aligned.
template <int N, typename R, bool NS, int FORM>
__host__ __device__ constexpr size_t rk_stage_offset(int epb)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    // split forms: pair fluxes [5][n/2][n3]
    constexpr size_t pairs = !is_standard(FORM) ? (size_t)5 * (n / 2) * n3 : 0;
    const size_t b = sizeof(R) * (((n * n + 1) & ~1) + (size_t)epb * vol_smem_per_node<FORM, NS>() * n3 +
                                  (size_t)epb * 30 * n2 + (size_t)epb * pairs);
    return (b + 15) & ~(size_t)15;
}

// Whether the mixed element kernel stages the RK register g and the FP64
// state u (40 bytes of shared memory per node each).  Measured: the
// bandwidth-bound standard form gains from them (64^3 N = 3: -12%); the
// split forms, whose resident CTAs are limited by shared memory, do not
// (16^3 N = 3 EC: 8% faster without g, a further 2% without u), so they
// read u and g where the RK update uses them.
template <int N, typename R, bool NS, int FORM>
__host__ __device__ constexpr bool rk_stage_g()
{
    return is_standard(FORM);
}

template <int N, typename R, bool NS, int FORM>
__host__ __device__ constexpr bool rk_stage_u()
{
    return is_standard(FORM);
}

template <int N, typename R, bool NS, int FORM>
__host__ __device__ constexpr size_t vol_smem_bytes(int epb)
{
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    constexpr int rkw = (rk_stage_u<N, R, NS, FORM>() ? 5 : 0) + (rk_stage_g<N, R, NS, FORM>() ? 5 : 0);
    return rk_stage_offset<N, R, NS, FORM>(epb) + (sizeof(R) == 4 ? (size_t)epb * n3 * (rkw * 8 + 4) : 0);
}

template <int N, typename R, bool NS, int FORM>
__global__ void __launch_bounds__(vol_threads<N>(), vol_min_blocks<N, R>())
k_volume(const __grid_constant__ Batch b, const Ops *__restrict__ ops, int stage, double rkA, double rkB, int lam_slot,
         int epb)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr int PER = vol_smem_per_node<FORM, NS>();
    constexpr int FACEVALS = 6 * 5 * n2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sD = (R *)smem_raw;
    R *sbuf = sD + ((n * n + 1) & ~1);
    R *sface = sbuf + (size_t)epb * PER * n3;
    // mixed path: the FP64 state and register and 1/J of the RK update, staged
    // at the start so that their loads overlap the volume and surface work
    constexpr bool STAGE_RK = sizeof(R) == 4;
    // with an even number of nodes per direction every staged block is a
    // multiple of 16 bytes at 16-byte aligned addresses: one thread per element
    // moves them with bulk copies (TMA engine) counted on the element's mbarrier
    constexpr bool BULK = STAGE_RK && (n % 2 == 0);
    constexpr bool STAGE_U = rk_stage_u<N, R, NS, FORM>();
    constexpr bool STAGE_G = rk_stage_g<N, R, NS, FORM>();
    constexpr int RKW = (STAGE_U ? 5 : 0) + (STAGE_G ? 5 : 0);   // staged FP64 values per node
    constexpr int GOFF = STAGE_U ? 5 : 0;                          // g's plane offset in the block
    __shared__ unsigned long long bulk_bar[BULK ? 256 / (n3 < 256 ? n3 : 256) : 1];
    double *sRK = (double *)(smem_raw + rk_stage_offset<N, R, NS, FORM>(epb));
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = ops_D<R>(ops, t);
    const int le = threadIdx.x / n3, p = threadIdx.x - le * n3;
    const long long ge = blockIdx.x * (long long)epb + le;
    bool valid = le < epb && ge < b.total_elems;   // (threads past the CTA's elements: warp padding)
    const Item *itp = nullptr;
    int e = 0;
    if (valid) {
        itp = &find_item_elem(b, ge);
        e = (int)(ge - itp->elem_begin);
        if (itp->clk && itp->clk->done) valid = false;
    }
    R *S = sbuf + (size_t)le * PER * n3;
    R *F6 = sface + (size_t)le * FACEVALS;
    const int ijk[3] = {p % n, (p / n) % n, p / n2};

    double u[5];
    R V[5] = {(R)0, (R)0, (R)0, (R)0, (R)0};
    const R iw = ops_iw0<R>(ops);
    Prim<R> q;   // kept across the barrier: the surface term recomputes the own flux from it
    if (valid) {
        const Item &it = *itp;
        const Nbrs nb = elem_nbrs(e, it.ex, it.ey, it.ez);
        // the six face-flux blocks of this element (slot 2d+1: the +d face,
        // own index; slot 2d: the -d face, owned by the -d neighbour) go to
        // shared memory by asynchronous copies, waited for before the barrier
        if constexpr (BULK) {
            if (p == 0) {
                unsigned long long *bar = bulk_bar + le;
                constexpr unsigned fb = 5 * n2 * sizeof(R), ub = 5 * n3 * 8, jb = n3 * 4;
                mbar_init(bar, 1);
                mbar_arrive_expect_tx(bar, 6 * fb + (stage >= 0 ? (STAGE_U ? ub : 0) + (STAGE_G && stage > 0 ? ub : 0) + jb
                                                               : 0));
                const R *FS = (const R *)it.fstar;
#pragma unroll
                for (int slot = 0; slot < 6; ++slot) {
                    const int d = slot >> 1;
                    const int owner = (slot & 1) ? e : nb.m[d];
                    bulk_g2s(F6 + slot * 5 * n2, FS + face_block(it, slot, d, owner, e) * 5 * n2, fb, bar);
                }
                if (stage >= 0) {
                    double *mine = sRK + (size_t)le * RKW * n3;
                    if (STAGE_U) bulk_g2s(mine, it.u + (size_t)e * 5 * n3, ub, bar);
                    if (STAGE_G && stage > 0) bulk_g2s(mine + GOFF * n3, it.g + (size_t)e * 5 * n3, ub, bar);
                    bulk_g2s((float *)(sRK + (size_t)epb * RKW * n3) + (size_t)le * n3, it.invJf + (size_t)e * n3, jb,
                             bar);
                }
            }
        } else if constexpr (sizeof(R) == 4) {
            const R *FS = (const R *)it.fstar;
#pragma unroll
            for (int slot = 0; slot < 6; ++slot) {
                const int d = slot >> 1;
                const int owner = (slot & 1) ? e : nb.m[d];
                cp_async_block<R>(F6 + slot * 5 * n2, FS + face_block(it, slot, d, owner, e) * 5 * n2, 5 * n2, p, n3);
            }
        }
        if constexpr (STAGE_RK && !(STAGE_U && STAGE_G)) {
            // the RK operands read where they are used: their lines are
            // requested into L2 now, so the late loads do not wait on DRAM
            if (stage >= 0) {
                if (!STAGE_U) prefetch_l2_block(it.u + (size_t)e * 5 * n3, sizeof(double) * 5 * n3, p, n3);
                if (!STAGE_G && stage > 0) prefetch_l2_block(it.g + (size_t)e * 5 * n3, sizeof(double) * 5 * n3, p, n3);
            }
        }
        if constexpr (STAGE_RK && !BULK) {
            if (stage >= 0) {
                double *mine = sRK + (size_t)le * RKW * n3;
                if (STAGE_U) cp_async_block<double>(mine, it.u + (size_t)e * 5 * n3, 5 * n3, p, n3);
                if (STAGE_G && stage > 0)
                    cp_async_block<double>(mine + GOFF * n3, it.g + (size_t)e * 5 * n3, 5 * n3, p, n3);
                cp_async_block<float>((float *)(sRK + (size_t)epb * RKW * n3) + (size_t)le * n3,
                                      it.invJf + (size_t)e * n3, n3, p, n3);
            }
        }
        const size_t node = (size_t)e * 5 * n3 + p;
        const Phys<R> P = phys_of<R>(it);
        R ja[9];
        const R *JA = metric_ptr<R>(it) + (size_t)e * 9 * n3 + p;
#pragma unroll
        for (int k = 0; k < 9; ++k) ja[k] = JA[k * n3];
        if constexpr (sizeof(R) == 8) {
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = it.u[node + v * n3];
            q = prim_from_u<R>(u, P.gm1);
        } else {
            // the FP32 shadow carries exactly the rounded state the fluxes use
            float us[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) us[v] = it.uf[node + v * n3];
            q = prim_from_f(us, P.gm1);
        }
        R G[12];
        if (NS) {
            const R *Gp = (const R *)it.grad + (size_t)e * 12 * n3 + p;
#pragma unroll
            for (int k = 0; k < 12; ++k) G[k] = Gp[k * n3];
        }
        if constexpr (sizeof(R) == 8) {   // (the mixed path issued its face copies above)
            const R *FS = (const R *)it.fstar;
#pragma unroll
            for (int slot = 0; slot < 6; ++slot) {
                const int d = slot >> 1;
                const int owner = (slot & 1) ? e : nb.m[d];
                cp_async_block<R>(F6 + slot * 5 * n2, FS + face_block(it, slot, d, owner, e) * 5 * n2, 5 * n2, p, n3);
            }
        }
        // contravariant fluxes at this node; for the split form the diagonal
        // two-point term F#(u_i,u_i).(2 Ja_i) = 2 Ja_i.F_e(u_i) goes straight
        // into V so that no flux is held across the barrier
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            R fe[5], fv[5] = {(R)0, (R)0, (R)0, (R)0, (R)0};
            euler_flux(q, q.E, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fe);
            if (NS) visc_flux(q, G, P.mu, P.kappa, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fv);
            R own[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) own[v] = NS ? fe[v] - fv[v] : fe[v];
            if (is_standard(FORM)) {
#pragma unroll
                for (int v = 0; v < 5; ++v) S[(d * 5 + v) * n3 + p] = own[v];
            } else {
                const R dii = (R)2 * ops_D<R>(ops, ijk[d] * n + ijk[d]);
#pragma unroll
                for (int v = 0; v < 5; ++v) V[v] += dii * fe[v];
                if (NS) {
#pragma unroll
                    for (int v = 0; v < 5; ++v) S[(16 + d * 5 + v) * n3 + p] = fv[v];
                }
            }
        }
        if (!is_standard(FORM)) {
            R z[kSplitSlots];
            split_node<FORM>(q, z);
#pragma unroll
            for (int k = 0; k < kSplitSlots; ++k) S[k * n3 + p] = z[k];
#pragma unroll
            for (int k = 0; k < 9; ++k) S[(7 + k) * n3 + p] = ja[k];
        }
    }
    cp_async_wait_all();
    __syncthreads();

    double lc = 0.0, lv = 0.0;
    bool lam_active = false;
    if constexpr (is_standard(FORM)) {
        if (valid) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const int stride = (d == 0) ? 1 : (d == 1) ? n : n2;
                const int base = p - ijk[d] * stride;
                const R *Drow = sD + ijk[d] * n;
#pragma unroll
                for (int m = 0; m < n; ++m) {
                    const R Dm = Drow[m];
#pragma unroll
                    for (int v = 0; v < 5; ++v) V[v] += Dm * S[(d * 5 + v) * n3 + base + m * stride];
                }
            }
        }
    } else {
        // Split form.  F#(u_i,u_m).(Ja_i + Ja_m) is symmetric in (i, m), so
        // each pair of nodes on a line is evaluated once and shared through
        // shared memory.  Pair thread t = x n^2 + l (x a position along the
        // line, l = ta + n tb the line) evaluates the pairs (x, x + k mod n)
        // for k = 1 .. n/2, the half-way pair k = n/2 of an even n only for
        // x < n/2: every pair of the line exactly once, with no index search,
        // and the threads with the extra pair grouped in the lower warps.
        // Then every node sums D_im times the fluxes of its line.
        constexpr int KP = n / 2;
        R *PB = sface + (size_t)epb * FACEVALS + (size_t)le * 5 * KP * n3;
        const R hg = valid ? phys_of<R>(*itp).hg : (R)0;
        const R gam = valid ? phys_of<R>(*itp).gamma : (R)0;
#pragma unroll 1
        for (int d = 0; d < 3; ++d) {
            const int sd = (d == 0) ? 1 : (d == 1) ? n : n2;   // node stride along d
            if (valid) {
                const int x = p / n2, l = p - x * n2;
                const int ta = l % n, tb = l / n;
                const int a = x * sd + ta * ((d == 0) ? n : 1) + tb * ((d == 2) ? n : n2);
                R za[kSplitSlots];
#pragma unroll
                for (int k = 0; k < kSplitSlots; ++k) za[k] = S[k * n3 + a];
                const R *SJ = S + (7 + d * 3) * n3;
                const R j1 = SJ[a], j2 = SJ[n3 + a], j3 = SJ[2 * n3 + a];
#pragma unroll
                for (int k = 1; k <= KP; ++k) {
                    if (2 * k == n && x >= KP) break;
                    const int xm = (x + k < n) ? x + k : x + k - n;
                    const int c = a + (xm - x) * sd;
                    R zc[kSplitSlots];
#pragma unroll
                    for (int q = 0; q < kSplitSlots; ++q) zc[q] = S[q * n3 + c];
                    R fs[5];
                    split_pair<FORM>(za, zc, gam, hg, j1 + SJ[c], j2 + SJ[n3 + c], j3 + SJ[2 * n3 + c], fs);
#pragma unroll
                    for (int v = 0; v < 5; ++v) PB[(v * KP + k - 1) * n3 + p] = fs[v];
                }
            }
            __syncthreads();
            if (valid) {
                const int i = ijk[d];
                const int ta = (d == 0) ? ijk[1] : ijk[0];
                const int tb = (d == 2) ? ijk[1] : ijk[2];
                const int l = ta + n * tb;
                const int base = p - i * sd;
                const R *Drow = sD + i * n;
#pragma unroll
                for (int m = 0; m < n; ++m) {
                    const R Dm = Drow[m];
                    if (m != i) {
                        // the pair (i, m) sits with pair thread x n^2 + l in slot k - 1
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
                        const R *F = PB + (slot - 1) * n3 + x * n2 + l;
#pragma unroll
                        for (int v = 0; v < 5; ++v) V[v] += Dm * F[v * KP * n3];
                    }
                    if (NS) {
                        const int pm = base + m * sd;
#pragma unroll
                        for (int v = 1; v < 5; ++v) V[v] -= Dm * S[(16 + d * 5 + v) * n3 + pm];
                    }
                }
            }
            __syncthreads();
        }
    }
    if constexpr (BULK) {
        // the face fluxes and the RK operands staged by the bulk copies; a wait
        // that runs out of polls poisons the result (NaN) and flags the solve
        if (valid && !mbar_wait(bulk_bar + le, 0, kBulkWaitPolls)) {
#pragma unroll
            for (int v = 0; v < 5; ++v) V[v] = (R)NAN;
            if (itp->clk) itp->clk->bad = 2;
        }
    }
    if (valid) {
        const Item &it = *itp;
        // surface term (1/w)(F* - own) on the +d face, (1/w)(own - F*) on the
        // -d face: the difference is formed first (it is small where the large
        // fluxes nearly cancel), with the own flux Ja^d.(F_e - F_v) re-read
        // (standard form) or recomputed from the node's state (split form)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (ijk[d] != N && ijk[d] != 0) continue;
            const int ta = (d == 0) ? ijk[1] : ijk[0];
            const int tb = (d == 2) ? ijk[1] : ijk[2];
            const int ab = ta + n * tb;
            R own[5];
            if (is_standard(FORM)) {
#pragma unroll
                for (int v = 0; v < 5; ++v) own[v] = S[(d * 5 + v) * n3 + p];
            } else {
                euler_flux(q, q.E, S[(7 + d * 3) * n3 + p], S[(8 + d * 3) * n3 + p], S[(9 + d * 3) * n3 + p], own);
                if (NS) {
#pragma unroll
                    for (int v = 1; v < 5; ++v) own[v] -= S[(16 + d * 5 + v) * n3 + p];
                }
            }
            if (ijk[d] == N) {
                const R *F = F6 + (2 * d + 1) * 5 * n2 + ab;
#pragma unroll
                for (int v = 0; v < 5; ++v) V[v] += iw * (F[v * n2] - own[v]);
            } else {
                const R *F = F6 + (2 * d) * 5 * n2 + ab;
#pragma unroll
                for (int v = 0; v < 5; ++v) V[v] += iw * (own[v] - F[v * n2]);
            }
        }
        if constexpr (STAGE_RK) {
            if (stage >= 0)
                node_update<R, NS>(it, e, p, n3, V, u, stage, rkA, rkB, lam_slot, lc, lv, lam_active,
                                   STAGE_U ? sRK + (size_t)le * RKW * n3 : nullptr,
                                   STAGE_G ? sRK + (size_t)le * RKW * n3 + GOFF * n3 : nullptr,
                                   (const float *)(sRK + (size_t)epb * RKW * n3) + le * n3);
            else
                node_update<R, NS>(it, e, p, n3, V, u, stage, rkA, rkB, lam_slot, lc, lv, lam_active);
        } else {
            node_update<R, NS>(it, e, p, n3, V, u, stage, rkA, rkB, lam_slot, lc, lv, lam_active);
        }
    }
    if (lam_slot >= 0 && stage >= 0) {
        unsigned long long *dc = nullptr, *dv = nullptr;
        if (lam_active) {
            dc = &itp->clk->lam[lam_slot][0];
            dv = NS ? &itp->clk->lam[lam_slot][1] : nullptr;
        }
        warp_max_to_clock(dc, dv, lc, lv, lam_active);
    }
}

// ------------------------------------------------------------------ launch (one volume form)

template <int N, typename R, bool NS, int FORM>
static cudaError_t vol_launch2(const Batch &b, int stage, double rkA, double rkB, int lam_slot, cudaStream_t s)
{
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    int epb = elems_per_block_p(N, sizeof(R) == 4 ? HS3D_MIXED32 : HS3D_FP64, 1);
    int threads = epb * n3;
    if (threads > vol_threads<N>()) {
        epb = vol_threads<N>() / n3;
        threads = epb * n3;
    }
    const size_t smem = vol_smem_bytes<N, R, NS, FORM>(epb);
    unsigned blocks = (unsigned)((b.total_elems + epb - 1) / epb);
    const Ops *ops = device_ops(N);
    if (!ops) return cudaErrorMemoryAllocation;
    k_volume<N, R, NS, FORM><<<blocks, threads, smem, s>>>(b, ops, stage, rkA, rkB, stage >= 0 ? lam_slot : -1, epb);
    return cudaGetLastError();
}

template <int FORM>
cudaError_t launch_volume_form(int N, int prec, int physics, const Batch &b, int stage, double rkA, double rkB,
                               int lam_slot, cudaStream_t s)
{
    if (b.total_elems == 0) return cudaSuccess;
#define HS3D_VOLN(K)                                                                                          \
    case K:                                                                                                   \
        if (prec != HS3D_FP64) return cudaErrorInvalidValue;                                                  \
        return physics == HS3D_NS ? vol_launch2<K, double, true, FORM>(b, stage, rkA, rkB, lam_slot, s)       \
                                  : vol_launch2<K, double, false, FORM>(b, stage, rkA, rkB, lam_slot, s);
    switch (N) {
        HS3D_VOLN(1) HS3D_VOLN(2) HS3D_VOLN(3) HS3D_VOLN(4) HS3D_VOLN(5) HS3D_VOLN(6) HS3D_VOLN(7)
    }
#undef HS3D_VOLN
    return cudaErrorInvalidValue;
}

template <int N, int FORM>
static cudaError_t prep_vol_n()
{
    const int big = 220 * 1024;
    cudaError_t e = cudaSuccess;
#define HS3D_ATTR(R, NS)                                                                                      \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(k_volume<N, R, NS, FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
    if (e == cudaSuccess)                                                                                     \
        e = cudaFuncSetAttribute(k_volume<N, R, NS, FORM>, cudaFuncAttributePreferredSharedMemoryCarveout,    \
                                 cudaSharedmemCarveoutMaxShared);
    HS3D_ATTR(double, false)
    HS3D_ATTR(double, true)
#undef HS3D_ATTR
    return e;
}

template <int FORM>
cudaError_t prepare_volume_form(int N)
{
    switch (N) {
        case 1: return prep_vol_n<1, FORM>();
        case 2: return prep_vol_n<2, FORM>();
        case 3: return prep_vol_n<3, FORM>();
        case 4: return prep_vol_n<4, FORM>();
        case 5: return prep_vol_n<5, FORM>();
        case 6: return prep_vol_n<6, FORM>();
        case 7: return prep_vol_n<7, FORM>();
    }
    return cudaErrorInvalidValue;
}

// Each volume_<form>.cu instantiates the two entry points for its form.
#define HS3D_VOLUME_FORM_TU(FORM)                                                                               \
    template cudaError_t launch_volume_form<FORM>(int, int, int, const Batch &, int, double, double, int,        \
                                                  cudaStream_t);                                                 \
    template cudaError_t prepare_volume_form<FORM>(int);

}  // namespace hs3d
