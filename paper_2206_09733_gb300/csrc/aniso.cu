// Anisotropic per-element degrees (Sec. 3.6: the order may differ per
// element and per reference direction, P_x, P_y, P_z), FP64.
//
// Element e has n_d = P_d + 1 Gauss-Lobatto nodes along d; node (i, j, k) is
// i + n_x (j + n_y k) and its state block [5][n_x n_y n_z] starts at off[e]
// (elements in mesh order).  Geometry: the element map is the degree-Ngeo
// interpolant (Ngeo = max(1, floor(Pmin/2)), Pmin over elements and
// directions) of the box map at the element's own nodes (built on the host,
// the free-stream rule of p-non-conforming faces), and the curl-form metric
// terms use each direction's own derivative matrix (k_ageo).
//
// A stage is
//   [k_amortar<0> -> k_agrad]   (Navier-Stokes: BR1 interface values, gradients)
//   k_amortar<1> -> k_avol      (face fluxes; volume + surface + 1/J + RK stage)
// The face between L (its +d face, tangential degrees (P_L[d0], P_L[d1]))
// and R (its -d face) carries a mortar of degree M_k = max(P_L[dk], P_R[dk])
// in each tangential direction k: both sides' traces (and gradients) are
// interpolated to the mortar points, the flux (or the BR1 value) is formed
// there with the face metric of a side whose tangential degrees are the
// mortar's (L first, then R; when neither is, L's face metric interpolated,
// exact since it has degree <= Pmin per direction), and each side receives
// its L2 projection, direction by direction (Kopriva et al. 2002, the method
// Sec. 3.6 names).  Each element face's result goes to its own block of the
// face arrays (fstar, qhat), at the face-node offset fnoff[6e + slot].
//
// Kernels take one element (or one face) per CTA.  Elements are launched in
// classes by node count (kAnisoClass), so a CTA has at most twice the threads
// its element needs; the work is FP64 and per node, as in the oracle, with
// no symmetry or sum factorisation beyond it: this path is for coverage of
// the anisotropic discretisation, the isotropic meshes keep their
// specialised kernels.
#include <math.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "aniso.cuh"
#include "api_internal.h"
#include "ic.cuh"
#include "mortar.cuh"
#include "mortar_phys.cuh"
#include "physics.cuh"

namespace hs3d {

namespace {

// ------------------------------------------------------------------ device helpers

struct AShape {
    int n[3];
    int n3;
};

__device__ __forceinline__ AShape ashape(const int *P3, int e)
{
    AShape s;
    s.n[0] = P3[3 * e] + 1;
    s.n[1] = P3[3 * e + 1] + 1;
    s.n[2] = P3[3 * e + 2] + 1;
    s.n3 = s.n[0] * s.n[1] * s.n[2];
    return s;
}

__device__ __forceinline__ int astride(const AShape &s, int d) { return d == 0 ? 1 : d == 1 ? s.n[0] : s.n[0] * s.n[1]; }

// tangential directions of face direction d, in increasing order
__device__ __forceinline__ void aface_dirs(int d, int &d0, int &d1)
{
    d0 = (d == 0) ? 1 : 0;
    d1 = (d == 2) ? 1 : 2;
}

// node of an element with index `end` along d and tangential indices (ta, tb)
__device__ __forceinline__ int aface_node(const AShape &s, int d, int end, int ta, int tb)
{
    int idx[3];
    int d0, d1;
    aface_dirs(d, d0, d1);
    idx[d] = end;
    idx[d0] = ta;
    idx[d1] = tb;
    return idx[0] + s.n[0] * (idx[1] + s.n[1] * idx[2]);
}

// sum_m D_d[i_d][m] f[node with index m along d] (f in shared memory)
__device__ __forceinline__ double aderiv(const AOps *ops, const AShape &s, const double *f, int p, const int ijk[3],
                                         int d)
{
    const int nd = s.n[d], st = astride(s, d);
    const double *Drow = ops->D[nd - 1] + ijk[d] * nd;
    const int base = p - ijk[d] * st;
    double acc = 0.0;
    for (int m = 0; m < nd; ++m) acc += Drow[m] * f[base + m * st];
    return acc;
}

struct APhys {
    double gamma, gm1, hg, mu, kappa;
    int physics, flux, form;
};

APhys aphys(const hs3d_solver_cfg *c)
{
    APhys P;
    P.gamma = c->gamma;
    P.gm1 = c->gamma - 1.0;
    P.hg = 0.5 / P.gm1;
    P.mu = c->physics == HS3D_NS ? 1.0 / c->Re : 0.0;
    P.kappa = c->physics == HS3D_NS ? P.mu * c->gamma / ((c->gamma - 1.0) * c->Pr) : 0.0;
    P.physics = c->physics;
    P.flux = c->surface_flux;
    P.form = c->volume_form;
    return P;
}

// ------------------------------------------------------------------ geometry

// J, 1/J and the curl-form metric terms (Kopriva 2006) of every element from
// its node coordinates X (already in place), each derivative along d with the
// derivative matrix of the element's degree in d.
__global__ void __launch_bounds__(512) k_ageo(const int *__restrict__ elems, const int *__restrict__ P3, const long long *__restrict__ noff,
                       const AOps *__restrict__ ops, const double *__restrict__ Xall, double *__restrict__ Jaall,
                       double *__restrict__ Jall, double *__restrict__ invJall)
{
    extern __shared__ double sm[];
    const int e = elems[blockIdx.x];
    const AShape s = ashape(P3, e);
    const int n3 = s.n3, p = threadIdx.x;
    const bool live = p < n3;
    double *sX = sm;             // [3][n3]
    double *sT = sm + 3 * n3;    // [2][n3]
    const long long nb = noff[e];
    const double *X = Xall + 3 * nb;
    int ijk[3] = {0, 0, 0};
    double x[3] = {0, 0, 0};
    if (live) {
        ijk[0] = p % s.n[0];
        ijk[1] = (p / s.n[0]) % s.n[1];
        ijk[2] = p / (s.n[0] * s.n[1]);
        for (int c = 0; c < 3; ++c) x[c] = sX[c * n3 + p] = X[(size_t)c * n3 + p];
    }
    __syncthreads();
    double a[3][3] = {};   // a[d][c] = dX_c / dxi_d
    if (live)
        for (int d = 0; d < 3; ++d)
            for (int c = 0; c < 3; ++c) a[d][c] = aderiv(ops, s, sX + c * n3, p, ijk, d);
    if (live) {
        const double Jp = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) +
                          a[0][1] * (a[1][2] * a[2][0] - a[1][0] * a[2][2]) +
                          a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
        Jall[nb + p] = Jp;
        invJall[nb + p] = 1.0 / Jp;
    }
    double *Ja = Jaall + 9 * nb;
    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        for (int c = 0; c < 3; ++c) {
            const int m = (c + 1) % 3, l = (c + 2) % 3;
            __syncthreads();
            if (live) {
                sT[p] = x[l] * a[i1][m];
                sT[n3 + p] = x[l] * a[i2][m];
            }
            __syncthreads();
            if (live) Ja[(size_t)(i * 3 + c) * n3 + p] = aderiv(ops, s, sT, p, ijk, i2) - aderiv(ops, s, sT + n3, p, ijk, i1);
        }
    }
}

// ------------------------------------------------------------------ initial state

__global__ void __launch_bounds__(512) k_ainit(const int *__restrict__ elems, const int *__restrict__ P3, const long long *__restrict__ noff,
                        const double *__restrict__ Xall, hs3d_ic ic, double Lx, double Ly, double *__restrict__ u)
{
    const int e = elems[blockIdx.x];
    const AShape s = ashape(P3, e);
    const int p = threadIdx.x;
    if (p >= s.n3) return;
    const long long nb = noff[e];
    const double *X = Xall + 3 * nb;
    double w[5];
    ic_point(ic, Lx, Ly, X[p], X[s.n3 + p], X[2 * s.n3 + p], w);
    double *ue = u + 5 * nb;
    for (int v = 0; v < 5; ++v) ue[(size_t)v * s.n3 + p] = w[v];
}

// ------------------------------------------------------------------ dt maxima

// Per node: lam_c = sum_d n_d^2 (|Ja^d.v| + c |Ja^d|)/J and
// lam_v = (mu/rho) sum_d n_d^4 (|Ja^d|/J)^2 (each direction's resolution
// inside the sum), reduced to the clock's slot as bit patterns.
__device__ __forceinline__ void alam_node(const AShape &s, const double *Ja, int p, double iJ, const Prim<double> &q,
                                          const APhys &P, double &lc, double &lv)
{
    const double c = sqrt(P.gamma * q.p / q.rho);
    double sc = 0.0, sv = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double a1 = Ja[(size_t)(d * 3) * s.n3 + p], a2 = Ja[(size_t)(d * 3 + 1) * s.n3 + p],
                     a3 = Ja[(size_t)(d * 3 + 2) * s.n3 + p];
        const double an = sqrt(a1 * a1 + a2 * a2 + a3 * a3);
        const double n2 = (double)s.n[d] * s.n[d];
        sc += n2 * (fabs(a1 * q.v1 + a2 * q.v2 + a3 * q.v3) + c * an) * iJ;
        sv += n2 * n2 * (an * iJ) * (an * iJ);
    }
    lc = sc;
    lv = P.physics == HS3D_NS ? P.mu * sv / q.rho : 0.0;
}

__global__ void __launch_bounds__(512) k_alambda(const int *__restrict__ elems, const int *__restrict__ P3,
                          const long long *__restrict__ noff, const double *__restrict__ Jaall,
                          const double *__restrict__ invJall, const double *__restrict__ u, APhys P, Clock *clk,
                          int slot)
{
    const int e = elems[blockIdx.x];
    const AShape s = ashape(P3, e);
    const int p = threadIdx.x;
    const bool live = p < s.n3;
    double lc = 0.0, lv = 0.0;
    if (live) {
        const long long nb = noff[e];
        double w[5];
        for (int v = 0; v < 5; ++v) w[v] = u[5 * nb + (size_t)v * s.n3 + p];
        const Prim<double> q = prim_from_u<double>(w, P.gm1);
        if (!(q.rho > 0.0) || !(q.p > 0.0)) clk->bad = 1;
        else alam_node(s, Jaall + 9 * nb, p, invJall[nb + p], q, P, lc, lv);
    }
    warp_max_to_clock(&clk->lam[slot][0], P.physics == HS3D_NS ? &clk->lam[slot][1] : nullptr, lc, lv, live);
}

// ------------------------------------------------------------------ mortar faces

// One face per CTA of 64 threads (at most 8 x 8 mortar points).
//   MODE 0: q* = (q(u_L) + q(u_R))/2 at the mortar points -> qhat of both sides (4 values);
//   MODE 1: s F*(u_L, u_R; n) - (F_v(L) + F_v(R)).Sn/2 -> fstar of both sides (5 values,
//           oriented along +d).
constexpr int kAFaceThreads = 64;

template <int MODE, bool NS>
__global__ void __launch_bounds__(kAFaceThreads) k_amortar(const AFace *__restrict__ faces, const int *__restrict__ P3,
                                                           const long long *__restrict__ noff,
                                                           const long long *__restrict__ fnoff,
                                                           const double *__restrict__ u,
                                                           const double *__restrict__ grad,
                                                           const double *__restrict__ Jaall,
                                                           const MortarOps *__restrict__ mo, APhys P,
                                                           double *__restrict__ out)
{
    constexpr int NV = (MODE == 1 && NS) ? 17 : 5;   // conservative state (+ 12 gradients) per trace point
    constexpr int NO = MODE == 0 ? 4 : 5;
    __shared__ double tr[2][NV][kAFaceThreads];
    __shared__ double sn[2][3][kAFaceThreads];
    __shared__ double fm[NO][kAFaceThreads];
    const AFace F = faces[blockIdx.x];
    const int d = F.d, p = threadIdx.x;
    int d0, d1;
    aface_dirs(d, d0, d1);
    const int eS[2] = {F.eL, F.eR};
    AShape sh[2];
    int S0[2], S1[2];
    for (int k = 0; k < 2; ++k) {
        sh[k] = ashape(P3, eS[k]);
        S0[k] = sh[k].n[d0] - 1;
        S1[k] = sh[k].n[d1] - 1;
    }
    const int M0 = S0[0] > S0[1] ? S0[0] : S0[1], M1 = S1[0] > S1[1] ? S1[0] : S1[1];
    const int nm0 = M0 + 1, nM2 = nm0 * (M1 + 1);

    // 1. both sides' traces (and face metric) on their own face points
    for (int k = 0; k < 2; ++k) {
        const int ns0 = S0[k] + 1, f2 = ns0 * (S1[k] + 1);
        if (p < f2) {
            const int node = aface_node(sh[k], d, k == 0 ? sh[k].n[d] - 1 : 0, p % ns0, p / ns0);
            const long long nb = noff[eS[k]];
            const int n3 = sh[k].n3;
            for (int v = 0; v < 5; ++v) tr[k][v][p] = u[5 * nb + (size_t)v * n3 + node];
            if constexpr (MODE == 1 && NS)
                for (int q = 0; q < 12; ++q) tr[k][5 + q][p] = grad[12 * nb + (size_t)q * n3 + node];
            if constexpr (MODE == 1)
                for (int c = 0; c < 3; ++c) sn[k][c][p] = Jaall[9 * nb + (size_t)(d * 3 + c) * n3 + node];
        }
    }
    __syncthreads();

    // 2. the mortar function at this thread's mortar point (a, b)
    if (p < nM2) {
        const int a = p % nm0, b = p / nm0;
        double w[2][NV];
        for (int k = 0; k < 2; ++k) {
            const int ns0 = S0[k] + 1, ns1 = S1[k] + 1;
            const double *I0 = mo->Pi[S0[k]][M0] + a * ns0;   // identity rows when S == M
            const double *I1 = mo->Pi[S1[k]][M1] + b * ns1;
            for (int v = 0; v < NV; ++v) {
                double acc = 0.0;
                for (int j = 0; j < ns1; ++j) {
                    double r = 0.0;
                    for (int i = 0; i < ns0; ++i) r += I0[i] * tr[k][v][i + ns0 * j];
                    acc += I1[j] * r;
                }
                w[k][v] = acc;
            }
        }
        if constexpr (MODE == 0) {
            double qL[4], qR[4];
            mortar_q(w[0], P.gm1, qL);
            mortar_q(w[1], P.gm1, qR);
            for (int v = 0; v < 4; ++v) fm[v][p] = 0.5 * (qL[v] + qR[v]);
        } else {
            // face metric at the mortar point
            double s3[3];
            const int hk = (S0[0] == M0 && S1[0] == M1) ? 0 : (S0[1] == M0 && S1[1] == M1) ? 1 : -1;
            if (hk >= 0) {
                for (int c = 0; c < 3; ++c) s3[c] = sn[hk][c][p];
            } else {
                const int ns0 = S0[0] + 1, ns1 = S1[0] + 1;
                const double *I0 = mo->Pi[S0[0]][M0] + a * ns0;
                const double *I1 = mo->Pi[S1[0]][M1] + b * ns1;
                for (int c = 0; c < 3; ++c) {
                    double acc = 0.0;
                    for (int j = 0; j < ns1; ++j) {
                        double r = 0.0;
                        for (int i = 0; i < ns0; ++i) r += I0[i] * sn[0][c][i + ns0 * j];
                        acc += I1[j] * r;
                    }
                    s3[c] = acc;
                }
            }
            const MortarPhys<double> mp{P.gamma, P.gm1, P.hg, P.mu, P.kappa};
            double fs[5];
            mortar_riemann<double>(P.flux, w[0], w[1], mp, s3[0], s3[1], s3[2], fs);
            if constexpr (NS) {
                double fl[5], fr[5];
                const Prim<double> pL = mortar_prim(w[0], P.gm1), pR = mortar_prim(w[1], P.gm1);
                visc_flux(pL, &w[0][5], P.mu, P.kappa, s3[0], s3[1], s3[2], fl);
                visc_flux(pR, &w[1][5], P.mu, P.kappa, s3[0], s3[1], s3[2], fr);
                for (int v = 1; v < 5; ++v) fs[v] -= 0.5 * (fl[v] + fr[v]);
            }
            for (int v = 0; v < 5; ++v) fm[v][p] = fs[v];
        }
    }
    __syncthreads();

    // 3. each side's L2 projection onto its own face points, into its face block
    for (int k = 0; k < 2; ++k) {
        const int ns0 = S0[k] + 1, f2 = ns0 * (S1[k] + 1);
        if (p < f2) {
            const int a = p % ns0, b = p / ns0;
            const double *P0 = mo->P[S0[k]][M0] + a * nm0;   // identity rows when S == M
            const double *P1 = mo->P[S1[k]][M1] + b * (M1 + 1);
            const int slot = 2 * d + (k == 0 ? 1 : 0);
            double *dst = out + (size_t)NO * fnoff[6 * eS[k] + slot] + p;
            for (int v = 0; v < NO; ++v) {
                double acc = 0.0;
                for (int j = 0; j <= M1; ++j) {
                    double r = 0.0;
                    for (int i = 0; i < nm0; ++i) r += P0[i] * fm[v][i + nm0 * j];
                    acc += P1[j] * r;
                }
                dst[(size_t)v * f2] = acc;
            }
        }
    }
}

// ------------------------------------------------------------------ BR1 gradients

// J grad q_c = sum_d D_d (Ja^d_c q) + sum_faces (q*_e - q_in) (+-Ja^d_c)/w_end,
// q = (v1, v2, v3, T), q*_e from the mortar kernel; grad [12][n3] at 12 noff[e].
__global__ void __launch_bounds__(512) k_agrad(const int *__restrict__ elems, const int *__restrict__ P3, const long long *__restrict__ noff,
                        const long long *__restrict__ fnoff, const AOps *__restrict__ ops,
                        const double *__restrict__ u, const double *__restrict__ Jaall,
                        const double *__restrict__ invJall, const double *__restrict__ qhat, APhys P,
                        double *__restrict__ gradall)
{
    extern __shared__ double sm[];
    const int e = elems[blockIdx.x];
    const AShape s = ashape(P3, e);
    const int n3 = s.n3, p = threadIdx.x;
    const bool live = p < n3;
    double *sq = sm;            // [4][n3]
    double *sJ = sm + 4 * n3;   // [9][n3]
    const long long nb = noff[e];
    double qp[4] = {0, 0, 0, 0};
    int ijk[3] = {0, 0, 0};
    if (live) {
        ijk[0] = p % s.n[0];
        ijk[1] = (p / s.n[0]) % s.n[1];
        ijk[2] = p / (s.n[0] * s.n[1]);
        mortar_q(u + 5 * nb + p, P.gm1, qp, n3);
        for (int v = 0; v < 4; ++v) sq[v * n3 + p] = qp[v];
        for (int k = 0; k < 9; ++k) sJ[k * n3 + p] = Jaall[9 * nb + (size_t)k * n3 + p];
    }
    __syncthreads();
    if (!live) return;
    double G[12];
    for (int v = 0; v < 4; ++v)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int d = 0; d < 3; ++d) {
                const int nd = s.n[d], st = astride(s, d);
                const double *Drow = ops->D[nd - 1] + ijk[d] * nd;
                const int base = p - ijk[d] * st;
                const double *Jc = sJ + (d * 3 + c) * n3, *qv = sq + v * n3;
                for (int m = 0; m < nd; ++m) acc += Drow[m] * (Jc[base + m * st] * qv[base + m * st]);
            }
            G[v * 3 + c] = acc;
        }
    for (int d = 0; d < 3; ++d) {
        for (int side = -1; side <= 1; side += 2) {
            const int at = side > 0 ? s.n[d] - 1 : 0;
            if (ijk[d] != at) continue;
            int d0, d1;
            aface_dirs(d, d0, d1);
            const int f2 = s.n[d0] * s.n[d1];
            const int slot = 2 * d + (side > 0 ? 1 : 0);
            const double *qs = qhat + (size_t)4 * fnoff[6 * e + slot] + ijk[d0] + s.n[d0] * ijk[d1];
            const double iw = ops->iw0[s.n[d] - 1];
            for (int v = 0; v < 4; ++v) {
                const double jump = qs[(size_t)v * f2] - qp[v];
                for (int c = 0; c < 3; ++c) G[v * 3 + c] += jump * side * sJ[(d * 3 + c) * n3 + p] * iw;
            }
        }
    }
    const double iJ = invJall[nb + p];
    double *Gout = gradall + 12 * nb + p;
    for (int k = 0; k < 12; ++k) Gout[(size_t)k * n3] = G[k] * iJ;
}

// ------------------------------------------------------------------ volume + surface + RK

// du/dt = -(V + S)/J at every node; V the standard or split-form volume term
// (each direction with its own D), S = sum_faces (+-F*_e - (F_e - F_v)(in).(+-Ja^d))/w_end.
// stage < 0: du/dt into out; else the low-storage RK stage with coefficients
// (A, B) and the clock's dt, and (lam_slot >= 0) the new state's dt maxima.
template <bool NS, int FORM>
__global__ void __launch_bounds__(512) k_avol(const int *__restrict__ elems, const int *__restrict__ P3, const long long *__restrict__ noff,
                       const long long *__restrict__ fnoff, const AOps *__restrict__ ops, double *__restrict__ u,
                       double *__restrict__ g, double *__restrict__ out, const double *__restrict__ Jaall,
                       const double *__restrict__ invJall, const double *__restrict__ gradall,
                       const double *__restrict__ fstar, APhys P, Clock *clk, int stage, double rkA, double rkB,
                       int lam_slot)
{
    constexpr bool STD = FORM == HS3D_VOL_STANDARD;
    extern __shared__ double sm[];
    const int e = elems[blockIdx.x];
    const AShape s = ashape(P3, e);
    const int n3 = s.n3, p = threadIdx.x;
    // (a finished or failed run's clock stops its stages, not a residual evaluation)
    const bool live = p < n3 && (stage < 0 || !(clk->done));
    // shared: standard: the directional flux F~^d [5][n3];
    //         split: the pair inputs [kSplitSlots][n3], Ja^d [3][n3], (NS) F_v.Ja^d [4][n3]
    double *sF = sm;
    double *sZ = sm;
    double *sA = sm + kSplitSlots * n3;
    double *sV = sA + 3 * n3;
    const long long nb = noff[e];
    const double *Ja = Jaall + 9 * nb;
    int ijk[3] = {0, 0, 0};
    double w[5] = {0, 0, 0, 0, 0}, G[12] = {};
    Prim<double> q{};
    if (live) {
        ijk[0] = p % s.n[0];
        ijk[1] = (p / s.n[0]) % s.n[1];
        ijk[2] = p / (s.n[0] * s.n[1]);
        for (int v = 0; v < 5; ++v) w[v] = u[5 * nb + (size_t)v * n3 + p];
        q = prim_from_u<double>(w, P.gm1);
        if (NS)
            for (int k = 0; k < 12; ++k) G[k] = gradall[12 * nb + (size_t)k * n3 + p];
        if constexpr (!STD) {
            double z[kSplitSlots];
            split_node<FORM>(q, z);
            for (int k = 0; k < kSplitSlots; ++k) sZ[k * n3 + p] = z[k];
        }
    }
    double R[5] = {0, 0, 0, 0, 0};
    double own[3][5];   // (F_e - F_v).Ja^d at this node, for the surface term
    for (int d = 0; d < 3; ++d) {
        double a[3] = {0, 0, 0};
        if (live) {
            for (int c = 0; c < 3; ++c) a[c] = Ja[(size_t)(d * 3 + c) * n3 + p];
            double fe[5], fv[5] = {0, 0, 0, 0, 0};
            euler_flux(q, q.E, a[0], a[1], a[2], fe);
            if (NS) visc_flux(q, G, P.mu, P.kappa, a[0], a[1], a[2], fv);
            for (int v = 0; v < 5; ++v) own[d][v] = fe[v] - fv[v];
        }
        __syncthreads();   // the previous direction's shared values are consumed
        if (live) {
            if constexpr (STD) {
                for (int v = 0; v < 5; ++v) sF[v * n3 + p] = own[d][v];
            } else {
                for (int c = 0; c < 3; ++c) sA[c * n3 + p] = a[c];
                if (NS) {
                    double fv[5];
                    visc_flux(q, G, P.mu, P.kappa, a[0], a[1], a[2], fv);
                    for (int v = 1; v < 5; ++v) sV[(v - 1) * n3 + p] = fv[v];
                }
            }
        }
        __syncthreads();
        if (live) {
            const int nd = s.n[d], st = astride(s, d);
            const double *Drow = ops->D[nd - 1] + ijk[d] * nd;
            const int base = p - ijk[d] * st;
            if constexpr (STD) {
                for (int v = 0; v < 5; ++v) {
                    double acc = 0.0;
                    for (int m = 0; m < nd; ++m) acc += Drow[m] * sF[v * n3 + base + m * st];
                    R[v] += acc;
                }
            } else {
                // sum_m 2 D_im F#(u_i, u_m).(Ja_i + Ja_m)/2, the diagonal included
                double zi[kSplitSlots];
                for (int k = 0; k < kSplitSlots; ++k) zi[k] = sZ[k * n3 + p];
                for (int m = 0; m < nd; ++m) {
                    const int pm = base + m * st;
                    double zm[kSplitSlots];
                    for (int k = 0; k < kSplitSlots; ++k) zm[k] = sZ[k * n3 + pm];
                    double fs[5];
                    split_pair<FORM>(zi, zm, P.gamma, P.hg, a[0] + sA[pm], a[1] + sA[n3 + pm], a[2] + sA[2 * n3 + pm],
                                     fs);
                    for (int v = 0; v < 5; ++v) R[v] += Drow[m] * fs[v];
                }
                if (NS)
                    for (int v = 1; v < 5; ++v) {
                        double acc = 0.0;
                        for (int m = 0; m < nd; ++m) acc += Drow[m] * sV[(v - 1) * n3 + base + m * st];
                        R[v] -= acc;
                    }
            }
        }
    }
    double lc = 0.0, lv = 0.0;
    bool active = false;
    if (live) {
        // surface term
        for (int d = 0; d < 3; ++d) {
            for (int side = -1; side <= 1; side += 2) {
                const int at = side > 0 ? s.n[d] - 1 : 0;
                if (ijk[d] != at) continue;
                int d0, d1;
                aface_dirs(d, d0, d1);
                const int f2 = s.n[d0] * s.n[d1];
                const int slot = 2 * d + (side > 0 ? 1 : 0);
                const double *fs = fstar + (size_t)5 * fnoff[6 * e + slot] + ijk[d0] + s.n[d0] * ijk[d1];
                const double iw = ops->iw0[s.n[d] - 1];
                for (int v = 0; v < 5; ++v) R[v] += (side * fs[(size_t)v * f2] - side * own[d][v]) * iw;
            }
        }
        const double iJ = invJall[nb + p];
        if (stage < 0) {
            for (int v = 0; v < 5; ++v) out[5 * nb + (size_t)v * n3 + p] = -R[v] * iJ;
        } else {
            const double dt = clk->dt;
            double *gp = g + 5 * nb + p, *up = u + 5 * nb + p;
            for (int v = 0; v < 5; ++v) {
                const double r = -R[v] * iJ;
                const double gv = (stage == 0) ? dt * r : rkA * gp[(size_t)v * n3] + dt * r;
                gp[(size_t)v * n3] = gv;
                w[v] = w[v] + rkB * gv;
                up[(size_t)v * n3] = w[v];
            }
            if (lam_slot >= 0) {
                const Prim<double> qn = prim_from_u<double>(w, P.gm1);
                if (!(qn.rho > 0.0) || !(qn.p > 0.0)) clk->bad = 1;
                else {
                    alam_node(s, Ja, p, iJ, qn, P, lc, lv);
                    active = true;
                }
            }
        }
    }
    // (one call site: the warp reduction needs every lane)
    if (lam_slot >= 0 && stage >= 0)
        warp_max_to_clock(active ? &clk->lam[lam_slot][0] : nullptr,
                          active && P.physics == HS3D_NS ? &clk->lam[lam_slot][1] : nullptr, lc, lv, active);
}

// ------------------------------------------------------------------ diagnostics

// part[e][0..4] = sum_nodes J w_i w_j w_k f_v (f = dudt, else u), part[e][5]
// = sum J www (w . dudt), part[e][6] = sum |J www w_v dudt_v| (entropy
// variables w = dS/du, S = -rho s); a fixed-order tree over the nodes.
__global__ void __launch_bounds__(512) k_adiag(const int *__restrict__ elems, const int *__restrict__ P3, const long long *__restrict__ noff,
                        const double *__restrict__ wts, const double *__restrict__ Jall, const double *__restrict__ u,
                        const double *__restrict__ dudt, double gamma, double *__restrict__ part)
{
    extern __shared__ double sm[];   // [7][blockDim]
    const int e = elems[blockIdx.x];
    const AShape s = ashape(P3, e);
    const int p = threadIdx.x, T = blockDim.x;
    double val[7] = {0, 0, 0, 0, 0, 0, 0};
    if (p < s.n3) {
        const int i = p % s.n[0], j = (p / s.n[0]) % s.n[1], k = p / (s.n[0] * s.n[1]);
        const long long nb = noff[e];
        const double wq = Jall[nb + p] * wts[(s.n[0] - 1) * kMaxn + i] * wts[(s.n[1] - 1) * kMaxn + j] *
                          wts[(s.n[2] - 1) * kMaxn + k];
        const double *f = (dudt ? dudt : u) + 5 * nb + p;
        for (int v = 0; v < 5; ++v) val[v] = wq * f[(size_t)v * s.n3];
        if (dudt) {
            double w[5];
            for (int v = 0; v < 5; ++v) w[v] = u[5 * nb + (size_t)v * s.n3 + p];
            const Prim<double> q = prim_from_u<double>(w, gamma - 1.0);
            // entropy variables w = dS/du of S = -rho s, s = ln p - gamma ln rho
            const double sent = log(q.p) - gamma * log(q.rho);
            const double rp = (gamma - 1.0) * q.rho / q.p;
            const double ev[5] = {gamma - sent - 0.5 * rp * (q.v1 * q.v1 + q.v2 * q.v2 + q.v3 * q.v3), rp * q.v1,
                                  rp * q.v2, rp * q.v3, -rp};
            for (int v = 0; v < 5; ++v) {
                const double t = wq * ev[v] * f[(size_t)v * s.n3];
                val[5] += t;
                val[6] += fabs(t);
            }
        }
    }
    for (int k = 0; k < 7; ++k) sm[k * T + p] = val[k];
    __syncthreads();
    for (int h = T / 2; h > 0; h >>= 1) {
        if (p < h)
            for (int k = 0; k < 7; ++k) sm[k * T + p] += sm[k * T + p + h];
        __syncthreads();
    }
    if (p < 7) part[(size_t)e * 7 + p] = sm[p * T];
}

// out[k] = sum_e part[e][k] in a fixed order (256 strided partial sums, then a tree)
__global__ void k_adiag_final(const double *__restrict__ part, int E, double *__restrict__ out)
{
    __shared__ double sm[7][256];
    const int p = threadIdx.x;
    for (int k = 0; k < 7; ++k) {
        double acc = 0.0;
        for (int e = p; e < E; e += 256) acc += part[(size_t)e * 7 + k];
        sm[k][p] = acc;
    }
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (p < h)
            for (int k = 0; k < 7; ++k) sm[k][p] += sm[k][p + h];
        __syncthreads();
    }
    if (p < 7) out[p] = sm[p][0];
}

// ------------------------------------------------------------------ host tables

const AOps *device_aops()
{
    static std::mutex mu;
    static std::vector<AOps *> per_device;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)per_device.size() <= dev) per_device.resize(dev + 1, nullptr);
    if (per_device[dev]) return per_device[dev];
    AOps h;
    memset(&h, 0, sizeof h);
    for (int N = 1; N <= kMaxN; ++N) {
        const Ops &o = host_ops(N);
        const int n = N + 1;
        for (int t = 0; t < n * n; ++t) h.D[N][t] = o.D[t];
        h.iw0[N] = 1.0 / o.w[0];
    }
    AOps *d = nullptr;
    if (cudaMalloc(&d, sizeof(AOps)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, &h, sizeof(AOps), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    per_device[dev] = d;
    return d;
}

// Gauss-Lobatto weights of every degree [kMaxn][kMaxn] (device copy; row N-1... indexed by n - 1).
const double *device_aweights()
{
    static std::mutex mu;
    static std::vector<double *> per_device;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)per_device.size() <= dev) per_device.resize(dev + 1, nullptr);
    if (per_device[dev]) return per_device[dev];
    double h[kMaxn * kMaxn] = {0};
    for (int N = 1; N <= kMaxN; ++N) {
        const Ops &o = host_ops(N);
        for (int i = 0; i <= N; ++i) h[N * kMaxn + i] = o.w[i];
    }
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof h) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    per_device[dev] = d;
    return d;
}

void lagrange_at(int n, const double *x, double y, double *l)
{
    for (int j = 0; j < n; ++j) {
        double v = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) v *= (y - x[k]) / (x[j] - x[k]);
        l[j] = v;
    }
}

// The box map (affine position plus amp (L_c/2pi) sin sin sin of it, angles
// over [-pi, pi]) at reference point r of element e.
void abox_point(const AnisoMesh *a, int e, const double r[3], double X[3])
{
    const int Ed[3] = {a->ex, a->ey, a->ez};
    const int ab[3] = {e % a->ex, (e / a->ex) % a->ey, e / (a->ex * a->ey)};
    double x0[3], th[3];
    for (int c = 0; c < 3; ++c) {
        const double L = a->hi[c] - a->lo[c];
        x0[c] = a->lo[c] + (L / Ed[c]) * (ab[c] + 0.5 * (r[c] + 1.0));
        th[c] = -M_PI + 2.0 * M_PI * (x0[c] - a->lo[c]) / L;
    }
    const double sn = sin(th[0]) * sin(th[1]) * sin(th[2]);
    for (int c = 0; c < 3; ++c) X[c] = x0[c] + a->amp * ((a->hi[c] - a->lo[c]) / (2.0 * M_PI)) * sn;
}

// Node coordinates [3][n3] of element e: the degree-Ngeo interpolant of the
// box map at the element's own nodes, direction by direction.
void anodes(const AnisoMesh *a, int e, double *X)
{
    const int G = a->Ngeo, ng = G + 1;
    const Ops &og = host_ops(G);
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = a->P3[3 * e + d] + 1;
    const int n3 = n[0] * n[1] * n[2];
    std::vector<double> Xg(3 * ng * ng * ng);
    for (int k = 0; k < ng; ++k)
        for (int j = 0; j < ng; ++j)
            for (int i = 0; i < ng; ++i) {
                const double r[3] = {og.xi[i], og.xi[j], og.xi[k]};
                double x[3];
                abox_point(a, e, r, x);
                for (int c = 0; c < 3; ++c) Xg[(size_t)c * ng * ng * ng + i + ng * (j + ng * k)] = x[c];
            }
    double L[3][kMaxn][kMaxn];
    for (int d = 0; d < 3; ++d) {
        const Ops &on = host_ops(n[d] - 1);
        for (int t = 0; t < n[d]; ++t) lagrange_at(ng, og.xi, on.xi[t], L[d][t]);
    }
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < n[2]; ++k)
            for (int j = 0; j < n[1]; ++j)
                for (int i = 0; i < n[0]; ++i) {
                    double acc = 0.0;
                    for (int kk = 0; kk < ng; ++kk)
                        for (int jj = 0; jj < ng; ++jj)
                            for (int ii = 0; ii < ng; ++ii)
                                acc += L[2][k][kk] * L[1][j][jj] * L[0][i][ii] *
                                       Xg[(size_t)c * ng * ng * ng + ii + ng * (jj + ng * kk)];
                    X[(size_t)c * n3 + i + n[0] * (j + n[1] * k)] = acc;
                }
}

// fn(class threads, number of elements, element list) for every non-empty class
template <class F>
cudaError_t for_classes(const AnisoMesh *a, F fn)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kAnisoClasses && e == cudaSuccess; ++k) {
        const int cnt = a->cls_begin[k + 1] - a->cls_begin[k];
        if (cnt > 0) e = fn(kAnisoClass[k], cnt, a->cls_elems + a->cls_begin[k]);
    }
    return e;
}

// Shared memory of the element kernels per thread slot (doubles): the volume
// kernel's standard form 5, split forms kSplitSlots + 3 + 4; the gradient 13.
template <int FORM>
constexpr size_t avol_smem_per() { return FORM == HS3D_VOL_STANDARD ? 5 : (kSplitSlots + 3 + 4); }
constexpr size_t kAGradSmemPer = 13;

template <class K>
cudaError_t allow_smem(K kernel, size_t bytes)
{
    return bytes > 48 * 1024 ? cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes)
                             : cudaSuccess;
}

// (set once at mesh set-up: not a stream operation, but kept out of captured launches)
template <bool NS>
cudaError_t allow_avol_smem(size_t T)
{
    cudaError_t e = allow_smem(k_avol<NS, HS3D_VOL_STANDARD>, sizeof(double) * avol_smem_per<HS3D_VOL_STANDARD>() * T);
    if (e == cudaSuccess) e = allow_smem(k_avol<NS, HS3D_VOL_EC>, sizeof(double) * avol_smem_per<HS3D_VOL_EC>() * T);
    if (e == cudaSuccess) e = allow_smem(k_avol<NS, HS3D_VOL_KG>, sizeof(double) * avol_smem_per<HS3D_VOL_KG>() * T);
    if (e == cudaSuccess)
        e = allow_smem(k_avol<NS, HS3D_VOL_PIROZZOLI>, sizeof(double) * avol_smem_per<HS3D_VOL_PIROZZOLI>() * T);
    if (e == cudaSuccess)
        e = allow_smem(k_avol<NS, HS3D_VOL_DUCROS>, sizeof(double) * avol_smem_per<HS3D_VOL_DUCROS>() * T);
    if (e == cudaSuccess)
        e = allow_smem(k_avol<NS, HS3D_VOL_MORINISHI>, sizeof(double) * avol_smem_per<HS3D_VOL_MORINISHI>() * T);
    if (e == cudaSuccess) e = allow_smem(k_avol<NS, HS3D_VOL_IR>, sizeof(double) * avol_smem_per<HS3D_VOL_IR>() * T);
    return e;
}

template <bool NS, int FORM>
cudaError_t launch_avol(const AnisoMesh *a, const APhys &P, double *u, double *g, double *out, int stage, double A,
                        double B, int lam_slot, cudaStream_t s)
{
    const AOps *ops = device_aops();
    if (!ops) return cudaErrorMemoryAllocation;
    return for_classes(a, [&](int T, int cnt, const int *els) {
        const size_t smem = sizeof(double) * avol_smem_per<FORM>() * T;
        k_avol<NS, FORM><<<cnt, T, smem, s>>>(els, a->dP3, a->dnoff, a->dfnoff, ops, u, g, out, a->Ja, a->invJ,
                                              a->grad, a->fstar, P, a->clk, stage, A, B, lam_slot);
        return cudaGetLastError();
    });
}

template <bool NS>
cudaError_t launch_avol_form(const AnisoMesh *a, const APhys &P, double *u, double *g, double *out, int stage,
                             double A, double B, int lam_slot, cudaStream_t s)
{
    switch (P.form) {
        case HS3D_VOL_STANDARD: return launch_avol<NS, HS3D_VOL_STANDARD>(a, P, u, g, out, stage, A, B, lam_slot, s);
        case HS3D_VOL_EC: return launch_avol<NS, HS3D_VOL_EC>(a, P, u, g, out, stage, A, B, lam_slot, s);
        case HS3D_VOL_KG: return launch_avol<NS, HS3D_VOL_KG>(a, P, u, g, out, stage, A, B, lam_slot, s);
        case HS3D_VOL_PIROZZOLI: return launch_avol<NS, HS3D_VOL_PIROZZOLI>(a, P, u, g, out, stage, A, B, lam_slot, s);
        case HS3D_VOL_DUCROS: return launch_avol<NS, HS3D_VOL_DUCROS>(a, P, u, g, out, stage, A, B, lam_slot, s);
        case HS3D_VOL_MORINISHI: return launch_avol<NS, HS3D_VOL_MORINISHI>(a, P, u, g, out, stage, A, B, lam_slot, s);
        case HS3D_VOL_IR: return launch_avol<NS, HS3D_VOL_IR>(a, P, u, g, out, stage, A, B, lam_slot, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// ------------------------------------------------------------------ host API

void aniso_free(AnisoMesh *a)
{
    if (!a) return;
    void *ptrs[] = {a->dP3, a->dnoff, a->doff, a->dfnoff, a->cls_elems, a->faces, a->X, a->Ja, a->J, a->invJ,
                    a->grad, a->fstar, a->qhat, a->diag_part, a->clk, a->clkp, a->one};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete a;
}

hs3d_status aniso_build(const hs3d_mesh_desc *desc, const int *degree3, AnisoMesh **out)
{
    *out = nullptr;
    const long long E = (long long)desc->ex * desc->ey * desc->ez;
    AnisoMesh *a = new (std::nothrow) AnisoMesh();
    if (!a) return fail(HS3D_ERR_NOMEM, "host allocation failed");
    a->ex = desc->ex;
    a->ey = desc->ey;
    a->ez = desc->ez;
    a->E = (int)E;
    for (int c = 0; c < 3; ++c) {
        a->lo[c] = desc->lo[c];
        a->hi[c] = desc->hi[c];
    }
    a->amp = desc->perturb_amp;
    a->P3.assign(degree3, degree3 + 3 * E);
    a->Pmin = 99;
    a->Pmax = 0;
    for (int v : a->P3) {
        a->Pmin = v < a->Pmin ? v : a->Pmin;
        a->Pmax = v > a->Pmax ? v : a->Pmax;
    }
    a->Ngeo = a->Pmin / 2 >= 1 ? a->Pmin / 2 : 1;
    a->off.assign(E + 1, 0);
    a->noff.assign(E + 1, 0);
    a->fnoff.assign(6 * E + 1, 0);
    std::vector<int> cls[kAnisoClasses];
    for (long long e = 0; e < E; ++e) {
        const int n[3] = {a->P3[3 * e] + 1, a->P3[3 * e + 1] + 1, a->P3[3 * e + 2] + 1};
        const int n3 = n[0] * n[1] * n[2];
        a->noff[e + 1] = a->noff[e] + n3;
        a->off[e + 1] = 5 * a->noff[e + 1];
        for (int d = 0; d < 3; ++d) {
            const int d0 = d == 0 ? 1 : 0, d1 = d == 2 ? 1 : 2;
            for (int side = 0; side < 2; ++side)
                a->fnoff[6 * e + 2 * d + side + 1] = a->fnoff[6 * e + 2 * d + side] + n[d0] * n[d1];
        }
        int k = 0;
        while (kAnisoClass[k] < n3) ++k;
        cls[k].push_back((int)e);
    }
    std::vector<int> elems;
    for (int k = 0; k < kAnisoClasses; ++k) {
        a->cls_begin[k] = (int)elems.size();
        elems.insert(elems.end(), cls[k].begin(), cls[k].end());
    }
    a->cls_begin[kAnisoClasses] = (int)elems.size();
    std::vector<AFace> faces;
    faces.reserve(3 * E);
    for (long long e = 0; e < E; ++e) {
        const int ab[3] = {(int)(e % a->ex), (int)((e / a->ex) % a->ey), (int)(e / ((long long)a->ex * a->ey))};
        const int Ed[3] = {a->ex, a->ey, a->ez};
        for (int d = 0; d < 3; ++d) {
            int c[3] = {ab[0], ab[1], ab[2]};
            c[d] = (c[d] + 1) % Ed[d];
            faces.push_back(AFace{(int)e, c[0] + a->ex * (c[1] + a->ey * c[2]), d});
        }
    }
    const long long nodes = a->noff[E], fnodes = a->fnoff[6 * E];
    std::vector<double> X(3 * (size_t)nodes);
    for (long long e = 0; e < E; ++e) anodes(a, (int)e, X.data() + 3 * a->noff[e]);
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&a->dP3, sizeof(int) * 3 * E},
        {(void **)&a->dnoff, sizeof(long long) * (E + 1)},
        {(void **)&a->doff, sizeof(long long) * (E + 1)},
        {(void **)&a->dfnoff, sizeof(long long) * (6 * E + 1)},
        {(void **)&a->cls_elems, sizeof(int) * E},
        {(void **)&a->faces, sizeof(AFace) * 3 * E},
        {(void **)&a->X, sizeof(double) * 3 * nodes},
        {(void **)&a->Ja, sizeof(double) * 9 * nodes},
        {(void **)&a->J, sizeof(double) * nodes},
        {(void **)&a->invJ, sizeof(double) * nodes},
        {(void **)&a->grad, sizeof(double) * 12 * nodes},
        {(void **)&a->fstar, sizeof(double) * 5 * fnodes},
        {(void **)&a->qhat, sizeof(double) * 4 * fnodes},
        {(void **)&a->diag_part, sizeof(double) * 7 * E},
        {(void **)&a->clk, sizeof(Clock)},
        {(void **)&a->clkp, sizeof(Clock *)},
        {(void **)&a->one, sizeof(int)},
    };
    cudaError_t e = cudaSuccess;
    for (auto &al : allocs) {
        if (e == cudaSuccess) e = cudaMalloc(al.p, al.bytes);
        if (e == cudaSuccess) a->bytes += al.bytes;
    }
    const int one = 1;
    static_assert(sizeof(long long) == sizeof(int64_t), "offset layout");
    if (e == cudaSuccess) e = cudaMemcpy(a->dP3, a->P3.data(), sizeof(int) * 3 * E, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a->dnoff, a->noff.data(), sizeof(long long) * (E + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a->doff, a->off.data(), sizeof(long long) * (E + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(a->dfnoff, a->fnoff.data(), sizeof(long long) * (6 * E + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a->cls_elems, elems.data(), sizeof(int) * E, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a->faces, faces.data(), sizeof(AFace) * 3 * E, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a->X, X.data(), sizeof(double) * 3 * nodes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(a->clk, 0, sizeof(Clock));
    if (e == cudaSuccess) e = cudaMemcpy(a->clkp, &a->clk, sizeof(Clock *), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(a->one, &one, sizeof(int), cudaMemcpyHostToDevice);
    const AOps *ops = device_aops();
    if (e == cudaSuccess && (!ops || !device_aweights() || !device_mortar_ops())) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
        e = for_classes(a, [&](int T, int cnt, const int *els) {
            k_ageo<<<cnt, T, sizeof(double) * 5 * T>>>(els, a->dP3, a->dnoff, ops, a->X, a->Ja, a->J, a->invJ);
            return cudaGetLastError();
        });
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    const size_t Tmax = kAnisoClass[kAnisoClasses - 1];
    if (e == cudaSuccess) e = allow_avol_smem<false>(Tmax);
    if (e == cudaSuccess) e = allow_avol_smem<true>(Tmax);
    if (e == cudaSuccess) e = allow_smem(k_agrad, sizeof(double) * kAGradSmemPer * Tmax);
    if (e != cudaSuccess) {
        cudaGetLastError();
        aniso_free(a);
        return cuda_fail(e, "anisotropic mesh set-up");
    }
    *out = a;
    return HS3D_OK;
}

cudaError_t aniso_stage(const AnisoMesh *a, const hs3d_solver_cfg *c, double *u, double *g, double *out, int stage,
                        int lam_slot, cudaStream_t s)
{
    const APhys P = aphys(c);
    const MortarOps *mo = device_mortar_ops();
    const AOps *ops = device_aops();
    if (!mo || !ops) return cudaErrorMemoryAllocation;
    const bool ns = c->physics == HS3D_NS;
    const int nf = 3 * a->E;
    cudaError_t e = cudaSuccess;
    if (ns) {
        k_amortar<0, true><<<nf, kAFaceThreads, 0, s>>>(a->faces, a->dP3, a->dnoff, a->dfnoff, u, a->grad, a->Ja, mo,
                                                        P, a->qhat);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = for_classes(a, [&](int T, int cnt, const int *els) {
                const size_t smem = sizeof(double) * kAGradSmemPer * T;
                k_agrad<<<cnt, T, smem, s>>>(els, a->dP3, a->dnoff, a->dfnoff, ops, u, a->Ja, a->invJ, a->qhat, P,
                                             a->grad);
                return cudaGetLastError();
            });
    }
    if (e == cudaSuccess) {
        if (ns)
            k_amortar<1, true><<<nf, kAFaceThreads, 0, s>>>(a->faces, a->dP3, a->dnoff, a->dfnoff, u, a->grad, a->Ja,
                                                            mo, P, a->fstar);
        else
            k_amortar<1, false><<<nf, kAFaceThreads, 0, s>>>(a->faces, a->dP3, a->dnoff, a->dfnoff, u, a->grad, a->Ja,
                                                             mo, P, a->fstar);
        e = cudaGetLastError();
    }
    double A = 0.0, B = 0.0;
    if (stage >= 0) rk_coeffs(c->time_scheme, stage, &A, &B);
    if (e == cudaSuccess)
        e = ns ? launch_avol_form<true>(a, P, u, g, out, stage, A, B, lam_slot, s)
               : launch_avol_form<false>(a, P, u, g, out, stage, A, B, lam_slot, s);
    return e;
}

cudaError_t aniso_step(const AnisoMesh *a, const hs3d_solver_cfg *c, double *u, double *g, double dt, bool fresh,
                       cudaStream_t s)
{
    const APhys P = aphys(c);
    cudaError_t e = cudaSuccess;
    if (fresh && !(dt > 0.0))
        e = for_classes(a, [&](int T, int cnt, const int *els) {
            k_alambda<<<cnt, T, 0, s>>>(els, a->dP3, a->dnoff, a->Ja, a->invJ, u, P, a->clk, 0);
            return cudaGetLastError();
        });
    // the maxima already carry n_d^2 (n_d^4): the p-mesh finalize with n = 1
    if (e == cudaSuccess)
        e = launch_pdt_finalize(a->clkp, a->one, 1, c->cfl, 8.0, 12.0, fresh ? 0 : 1, dt > 0.0 ? dt : 0.0, s);
    const int ns = rk_stages(c->time_scheme);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) e = aniso_stage(a, c, u, g, nullptr, k, k == ns - 1 ? 1 : -1, s);
    return e;
}

cudaError_t aniso_init_state(const AnisoMesh *a, const hs3d_ic &ic, double *u, cudaStream_t s)
{
    return for_classes(a, [&](int T, int cnt, const int *els) {
        k_ainit<<<cnt, T, 0, s>>>(els, a->dP3, a->dnoff, a->X, ic, a->hi[0] - a->lo[0], a->hi[1] - a->lo[1], u);
        return cudaGetLastError();
    });
}

cudaError_t aniso_diagnostics(const AnisoMesh *a, const hs3d_solver_cfg *c, const double *u, const double *dudt,
                              double *out, cudaStream_t s)
{
    const double *wts = device_aweights();
    if (!wts) return cudaErrorMemoryAllocation;
    cudaError_t e = for_classes(a, [&](int T, int cnt, const int *els) {
        k_adiag<<<cnt, T, sizeof(double) * 7 * T, s>>>(els, a->dP3, a->dnoff, wts, a->J, u, dudt, c->gamma,
                                                       a->diag_part);
        return cudaGetLastError();
    });
    if (e == cudaSuccess) {
        k_adiag_final<<<1, 256, 0, s>>>(a->diag_part, a->E, out);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace hs3d
