// Mortar coupling of elements of different polynomial degree (Sec. 3.6).
//
// A mesh whose elements carry their own degree runs the element kernels once
// per degree (one bucket of elements per degree, Item::face6 set); what
// couples the buckets are the faces.  Every face between an element L (its
// +d face, degree N_L) and its +d neighbour R (its -d face, degree N_R)
// carries a mortar of degree N_M = max(N_L, N_R) on the Gauss-Lobatto points
// of that degree (the mortar method of Kopriva et al. 2002 that Sec. 3.6
// names; it does not keep entropy stability, as the section notes):
//   1. the conservative traces of both sides (and for the viscous flux their
//      BR1 gradients) are interpolated to the mortar points,
//        f_M(a, b) = sum_j I_b,j sum_i I_a,i f(i, j),  I = l_i^(N_s)(xi_a^(N_M));
//   2. at every mortar point either the BR1 interface value
//      q* = (q(u_L) + q(u_R))/2 (k_mortar<MODE 0>) or the face flux
//      s F*(u_L, u_R; n) - (F_v(L) + F_v(R)).Sn/2 (MODE 1) is formed, with the
//      face metric Sn = Ja^d of the side of degree N_M (of L on a tie);
//   3. each side receives the L2 projection of the mortar function onto its
//      degree, P = M_s^-1 S (M_s[i][k] = int l_i l_k, S[i][j] = int l_i^s l_j^M,
//      exact integrals), in both face directions; the side of degree N_M
//      receives the mortar values.
// Equal degrees make every matrix the identity: the conforming face.
//
// Faces are grouped by mortar degree; a CTA holds several faces of one
// degree, one thread per mortar point.  Faces of two equal degrees take a
// barrier-free variant (k_mortar_conf) with the same arithmetic.  The per-bucket pointers live in a
// small device table (MortarSide); the operators of every degree pair in
// MortarOps.
#include <math.h>

#include <mutex>
#include <vector>

#include "internal.cuh"
#include "mortar.cuh"
#include "physics.cuh"
#include "mortar_phys.cuh"

namespace hs3d {

// ------------------------------------------------------------------ operators (host)

// Lagrange basis of the nodes x[0..n) at y.
static void lagrange_basis(int n, const double *x, double y, double *l)
{
    for (int j = 0; j < n; ++j) {
        double v = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) v *= (y - x[k]) / (x[j] - x[k]);
        l[j] = v;
    }
}

// Interpolation Ns -> Nm (nm x ns) and the exact L2 projection Nm -> Ns
// (ns x nm) on the Gauss-Lobatto points.  The projection solves
// M_s P = S with the symmetric positive definite mass matrix M_s factored by
// Cholesky; both integrals use Nm + 1 Gauss-Legendre points (exact for the
// degree Ns + Nm <= 2 Nm products).
static void build_pair(int Ns, int Nm, double *Pi, double *P)
{
    const int ns = Ns + 1, nm = Nm + 1;
    const Ops &os = host_ops(Ns), &om = host_ops(Nm);
    if (Ns == Nm) {
        for (int a = 0; a < ns; ++a)
            for (int i = 0; i < ns; ++i) Pi[a * ns + i] = P[a * ns + i] = (a == i) ? 1.0 : 0.0;
        return;
    }
    for (int a = 0; a < nm; ++a) lagrange_basis(ns, os.xi, om.xi[a], Pi + a * ns);
    const Ops &og = host_ops(Nm, HS3D_NODES_GAUSS);
    double M[kMaxn * kMaxn] = {0}, S[kMaxn * kMaxn] = {0};
    for (int q = 0; q < nm; ++q) {
        double ls[kMaxn], lm[kMaxn];
        lagrange_basis(ns, os.xi, og.xi[q], ls);
        lagrange_basis(nm, om.xi, og.xi[q], lm);
        for (int i = 0; i < ns; ++i) {
            for (int k = 0; k < ns; ++k) M[i * ns + k] += og.w[q] * ls[i] * ls[k];
            for (int j = 0; j < nm; ++j) S[i * nm + j] += og.w[q] * ls[i] * lm[j];
        }
    }
    // M = C C^T (C lower triangular), then C y = S, C^T P = y, column by column
    double Cl[kMaxn * kMaxn] = {0};
    for (int i = 0; i < ns; ++i)
        for (int k = 0; k <= i; ++k) {
            double s = M[i * ns + k];
            for (int r = 0; r < k; ++r) s -= Cl[i * ns + r] * Cl[k * ns + r];
            Cl[i * ns + k] = (i == k) ? sqrt(s) : s / Cl[k * ns + k];
        }
    for (int j = 0; j < nm; ++j) {
        double y[kMaxn];
        for (int i = 0; i < ns; ++i) {
            double s = S[i * nm + j];
            for (int r = 0; r < i; ++r) s -= Cl[i * ns + r] * y[r];
            y[i] = s / Cl[i * ns + i];
        }
        for (int i = ns - 1; i >= 0; --i) {
            double s = y[i];
            for (int r = i + 1; r < ns; ++r) s -= Cl[r * ns + i] * P[r * nm + j];
            P[i * nm + j] = s / Cl[i * ns + i];
        }
    }
}

const MortarOps &host_mortar_ops()
{
    static MortarOps mo;
    static std::once_flag once;
    std::call_once(once, [] {
        for (int s = 1; s <= kMaxN; ++s)
            for (int m = s; m <= kMaxN; ++m) {
                build_pair(s, m, mo.Pi[s][m], mo.P[s][m]);
                for (int k = 0; k < kMaxn * kMaxn; ++k) {
                    mo.Pif[s][m][k] = (float)mo.Pi[s][m][k];
                    mo.Pf[s][m][k] = (float)mo.P[s][m][k];
                }
            }
    });
    return mo;
}

const MortarOps *device_mortar_ops()
{
    static std::mutex mu;
    static std::vector<MortarOps *> per_dev;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1, nullptr);
    if (!per_dev[dev]) {
        MortarOps *d = nullptr;
        if (cudaMalloc(&d, sizeof(MortarOps)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaMemcpy(d, &host_mortar_ops(), sizeof(MortarOps), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(d);
            cudaGetLastError();
            return nullptr;
        }
        per_dev[dev] = d;
    }
    return per_dev[dev];
}

// ------------------------------------------------------------------ device helpers

template <typename R>
__device__ __forceinline__ const R *mo_interp(const MortarOps *mo, int Ns, int Nm);
template <>
__device__ __forceinline__ const double *mo_interp<double>(const MortarOps *mo, int Ns, int Nm) { return mo->Pi[Ns][Nm]; }
template <>
__device__ __forceinline__ const float *mo_interp<float>(const MortarOps *mo, int Ns, int Nm) { return mo->Pif[Ns][Nm]; }
template <typename R>
__device__ __forceinline__ const R *mo_proj(const MortarOps *mo, int Ns, int Nm);
template <>
__device__ __forceinline__ const double *mo_proj<double>(const MortarOps *mo, int Ns, int Nm) { return mo->P[Ns][Nm]; }
template <>
__device__ __forceinline__ const float *mo_proj<float>(const MortarOps *mo, int Ns, int Nm) { return mo->Pf[Ns][Nm]; }

// Node of an element of n nodes per direction with index `end` along d and
// tangential indices (ta, tb) (increasing direction order).
__device__ __forceinline__ int mortar_face_node(int n, int d, int end, int ta, int tb)
{
    if (d == 0) return end + n * (ta + n * tb);
    if (d == 1) return ta + n * (end + n * tb);
    return ta + n * (tb + n * end);
}

// ------------------------------------------------------------------ the face kernel

// Faces are grouped by mortar degree NM (a template parameter): a CTA holds
// FPC faces of P = (NM+1)^2 threads each, thread p of a face owning mortar
// point (a, b) = (p mod (NM+1), p div (NM+1)).  Interpolation and projection
// are separable: a first pass along the face's first direction, shared by
// the face's threads through shared memory, then the second pass per point.
//   MODE 0: BR1 interface values, written as qhat = 2 q*_s - q_s (4 values)
//           to each side's qhat6 block;
//   MODE 1: face fluxes (5 values) to each side's fstar block (both oriented
//           along +d).
template <typename R, bool NS, int MODE, int NM>
struct MortarShape {
    static constexpr int nM = NM + 1, P = nM * nM;
    static constexpr int NV = (MODE == 1 && NS) ? 17 : 5;         // values per trace point
    static constexpr int TARGET = 128;                             // threads per CTA aimed at
    static constexpr int FPC = TARGET / P >= 1 ? TARGET / P : 1;  // faces per CTA
    static constexpr int THREADS = FPC * P;
    // shared values per face: two sides' traces, the first-pass buffer, the mortar result
    static constexpr int PER_FACE = 2 * NV * P + NV * P + 5 * P;
    // resident CTAs per SM asked of the register allocator (FP32): 8 (64
    // registers) where that spills nothing, 6 for the viscous flux, whose
    // two sides' state and gradients (34 values) are live at once
    // (measured at 32^3, degrees 2..5: 0.6% faster than no cap; asking for
    // the maximum shared-memory carveout as well made the step 6% slower --
    // the trace gathers go through L1)
    static constexpr int MIN_BLOCKS = sizeof(R) == 8 ? 1 : ((MODE == 1 && NS) ? 6 : 8);
};

template <typename R, bool NS, int MODE, int NM>
__global__ void __launch_bounds__(MortarShape<R, NS, MODE, NM>::THREADS, MortarShape<R, NS, MODE, NM>::MIN_BLOCKS)
k_mortar(const MortarFace *__restrict__ faces, int nfaces, const MortarSide *__restrict__ sides,
         const double *__restrict__ u, const MortarOps *__restrict__ mo, int flux, MortarPhys<R> Ph)
{
    using S = MortarShape<R, NS, MODE, NM>;
    constexpr int nM = S::nM, P = S::P, NV = S::NV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int q = threadIdx.x / P, p = threadIdx.x - q * P;
    const int f = blockIdx.x * S::FPC + q;
    const bool live = f < nfaces;
    R *tr = (R *)smem_raw + (size_t)q * S::PER_FACE;   // [2][NV][P]
    R *T = tr + 2 * NV * P;                            // [NV][P]
    R *fm = T + NV * P;                                // [5][P]
    const int a = p % nM, b = p / nM;
    MortarFace F{};
    int Nside[2] = {NM, NM};
    if (live) {
        F = faces[f];
        Nside[0] = sides[F.bL].N;
        Nside[1] = sides[F.bR].N;
    }
    const int d = F.d;

    // 1. traces of both sides on their own face points: L's +d face, R's -d face
    if (live) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const MortarSide &SD = sides[s ? F.bR : F.bL];
            const int ns = SD.N + 1, n3 = ns * ns * ns;
            const int le = s ? F.lR : F.lL;
            if (p < ns * ns) {
                const int node = mortar_face_node(ns, d, s ? 0 : SD.N, p % ns, p / ns);
                R *dst = tr + s * NV * P + p;
                if constexpr (sizeof(R) == 8) {
                    const double *src = u + SD.base + (size_t)le * 5 * n3 + node;
#pragma unroll
                    for (int v = 0; v < 5; ++v) dst[v * P] = src[(size_t)v * n3];
                } else {
                    const float *src = SD.uf + (size_t)le * 5 * n3 + node;
#pragma unroll
                    for (int v = 0; v < 5; ++v) dst[v * P] = src[(size_t)v * n3];
                }
                if constexpr (MODE == 1 && NS) {
                    const R *G = (const R *)SD.grad + (size_t)le * 12 * n3 + node;
#pragma unroll
                    for (int k = 0; k < 12; ++k) dst[(5 + k) * P] = G[(size_t)k * n3];
                }
            }
        }
    }
    __syncthreads();

    // 2. both sides at this thread's mortar point (registers)
    R w[2][NV];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int Ns = Nside[s], ns = Ns + 1;
        const R *src = tr + s * NV * P;
        // (nM ns <= P entries: at most one per thread; loops unrolled to nM with
        // the side's ns as a predicate)
        if (Ns < NM && p < nM * ns) {
            const R *I = mo_interp<R>(mo, Ns, NM);   // [nM][ns]
            // first pass: T[v][a' + nM j] = sum_i I[a'][i] f[v][i + ns j]
            const int ap = p % nM, j = p / nM;
            R row[nM];
#pragma unroll
            for (int i = 0; i < nM; ++i) row[i] = i < ns ? I[ap * ns + i] : (R)0;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                R acc = (R)0;
#pragma unroll
                for (int i = 0; i < nM; ++i)
                    if (i < ns) acc += row[i] * src[v * P + i + ns * j];
                T[v * P + p] = acc;
            }
        }
        __syncthreads();   // (uniform: every thread of the CTA reaches it for both sides)
        if (Ns < NM) {
            const R *I = mo_interp<R>(mo, Ns, NM);
            R col[nM];
#pragma unroll
            for (int j = 0; j < nM; ++j) col[j] = j < ns ? I[b * ns + j] : (R)0;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                R acc = (R)0;
#pragma unroll
                for (int j = 0; j < nM; ++j)
                    if (j < ns) acc += col[j] * T[v * P + a + nM * j];
                w[s][v] = acc;
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) w[s][v] = src[v * P + p];
        }
        __syncthreads();   // T is reused by the other side
    }

    // 3. the mortar function at this point
    if (live) {
        if constexpr (MODE == 0) {
            R qL[4], qR[4];
            mortar_q(w[0], Ph.gm1, qL);
            mortar_q(w[1], Ph.gm1, qR);
#pragma unroll
            for (int v = 0; v < 4; ++v) fm[v * P + p] = (R)0.5 * (qL[v] + qR[v]);
        } else {
            // face metric of the side of degree NM (L on a tie), at its own face point (a, b)
            const bool useL = Nside[0] >= Nside[1];
            const MortarSide &H = sides[useL ? F.bL : F.bR];
            const int n3h = nM * nM * nM;
            const int node = mortar_face_node(nM, d, useL ? NM : 0, a, b);
            const R *JA = (const R *)(sizeof(R) == 8 ? (const void *)H.Ja : (const void *)H.Jaf) +
                          ((size_t)(useL ? F.lL : F.lR) * 9 + d * 3) * n3h + node;
            const R s1 = JA[0], s2 = JA[n3h], s3 = JA[2 * (size_t)n3h];
            R fs[5];
            mortar_riemann<R>(flux, w[0], w[1], Ph, s1, s2, s3, fs);
            if constexpr (NS) {
                R fl[5], fr[5];
                const Prim<R> pL = mortar_prim(w[0], Ph.gm1), pR = mortar_prim(w[1], Ph.gm1);
                visc_flux(pL, &w[0][5], Ph.mu, Ph.kappa, s1, s2, s3, fl);
                visc_flux(pR, &w[1][5], Ph.mu, Ph.kappa, s1, s2, s3, fr);
#pragma unroll
                for (int v = 1; v < 5; ++v) fs[v] -= (R)0.5 * (fl[v] + fr[v]);
            }
#pragma unroll
            for (int v = 0; v < 5; ++v) fm[v * P + p] = fs[v];
        }
    }
    __syncthreads();

    // 4. projection onto each side and the write to its own face block
    constexpr int NOUT = MODE == 0 ? 4 : 5;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int Ns = Nside[s], ns = Ns + 1, n2 = ns * ns;
        if (Ns < NM && p < ns * nM) {
            const R *Pr = mo_proj<R>(mo, Ns, NM);   // [ns][nM]
            // first pass: T[v][a' + ns j] = sum_i Pr[a'][i] fm[v][i + nM j]
            const int ap = p % ns, j = p / ns;
            R row[nM];
#pragma unroll
            for (int i = 0; i < nM; ++i) row[i] = Pr[ap * nM + i];
#pragma unroll
            for (int v = 0; v < NOUT; ++v) {
                R acc = (R)0;
#pragma unroll
                for (int i = 0; i < nM; ++i) acc += row[i] * fm[v * P + i + nM * j];
                T[v * P + p] = acc;
            }
        }
        __syncthreads();
        if (live && p < n2) {
            const int ap = p % ns, bp = p / ns;
            R val[5];
            if (Ns < NM) {
                const R *Pr = mo_proj<R>(mo, Ns, NM);
                R col[nM];
#pragma unroll
                for (int j = 0; j < nM; ++j) col[j] = Pr[bp * nM + j];
#pragma unroll
                for (int v = 0; v < NOUT; ++v) {
                    R acc = (R)0;
#pragma unroll
                    for (int j = 0; j < nM; ++j) acc += col[j] * T[v * P + ap + ns * j];
                    val[v] = acc;
                }
            } else {
#pragma unroll
                for (int v = 0; v < NOUT; ++v) val[v] = fm[v * P + p];
            }
            const MortarSide &SD = sides[s ? F.bR : F.bL];
            const int slot = s ? 2 * d : 2 * d + 1;
            const int le = s ? F.lR : F.lL;
            if constexpr (MODE == 0) {
                R qin[4];
                mortar_q(tr + s * NV * P + p, Ph.gm1, qin, P);
                R *dst = (R *)SD.qhat6 + ((size_t)slot * SD.E + le) * 4 * n2 + p;
#pragma unroll
                for (int v = 0; v < 4; ++v) dst[v * n2] = (R)2 * val[v] - qin[v];
            } else {
                R *dst = (R *)SD.fstar6 + ((size_t)slot * SD.E + le) * 5 * n2 + p;
#pragma unroll
                for (int v = 0; v < 5; ++v) dst[v * n2] = val[v];
            }
        }
        __syncthreads();   // T is reused by the other side
    }
}

// Faces whose two sides have the same degree N: the mortar is the face
// itself and interpolation and projection are identities, so each thread
// takes one face point, gathers both traces into registers, forms the same
// interface value or flux as k_mortar and writes it to both sides' blocks --
// no shared memory, no barriers.  Several faces per CTA.
template <typename R, bool NS, int MODE, int N>
__global__ void __launch_bounds__(128) k_mortar_conf(const MortarFace *__restrict__ faces, int nfaces,
                                                     const MortarSide *__restrict__ sides, const double *__restrict__ u,
                                                     int flux, MortarPhys<R> Ph)
{
    constexpr int n = N + 1, P = n * n, n3 = P * n;
    constexpr int FPC = 128 / P >= 1 ? 128 / P : 1;
    constexpr int NV = (MODE == 1 && NS) ? 17 : 5;
    const int q = threadIdx.x / P, p = threadIdx.x - q * P;
    const int f = blockIdx.x * FPC + q;
    if (q >= FPC || f >= nfaces) return;
    const MortarFace F = faces[f];
    const int d = F.d;
    const MortarSide &SL = sides[F.bL], &SR = sides[F.bR];
    R w[2][NV];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const MortarSide &SD = s ? SR : SL;
        const int le = s ? F.lR : F.lL;
        const int node = mortar_face_node(n, d, s ? 0 : N, p % n, p / n);
        if constexpr (sizeof(R) == 8) {
            const double *src = u + SD.base + (size_t)le * 5 * n3 + node;
#pragma unroll
            for (int v = 0; v < 5; ++v) w[s][v] = src[(size_t)v * n3];
        } else {
            const float *src = SD.uf + (size_t)le * 5 * n3 + node;
#pragma unroll
            for (int v = 0; v < 5; ++v) w[s][v] = src[(size_t)v * n3];
        }
        if constexpr (MODE == 1 && NS) {
            const R *G = (const R *)SD.grad + (size_t)le * 12 * n3 + node;
#pragma unroll
            for (int k = 0; k < 12; ++k) w[s][5 + k] = G[(size_t)k * n3];
        }
    }
    if constexpr (MODE == 0) {
        R qL[4], qR[4], qs[4];
        mortar_q(w[0], Ph.gm1, qL);
        mortar_q(w[1], Ph.gm1, qR);
#pragma unroll
        for (int v = 0; v < 4; ++v) qs[v] = (R)0.5 * (qL[v] + qR[v]);
        R *dL = (R *)SL.qhat6 + ((size_t)(2 * d + 1) * SL.E + F.lL) * 4 * P + p;
        R *dR = (R *)SR.qhat6 + ((size_t)(2 * d) * SR.E + F.lR) * 4 * P + p;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            dL[v * P] = (R)2 * qs[v] - qL[v];
            dR[v * P] = (R)2 * qs[v] - qR[v];
        }
    } else {
        const int node = mortar_face_node(n, d, N, p % n, p / n);
        const R *JA = (const R *)(sizeof(R) == 8 ? (const void *)SL.Ja : (const void *)SL.Jaf) +
                      ((size_t)F.lL * 9 + d * 3) * n3 + node;
        const R s1 = JA[0], s2 = JA[n3], s3 = JA[2 * (size_t)n3];
        R fs[5];
        mortar_riemann<R>(flux, w[0], w[1], Ph, s1, s2, s3, fs);
        if constexpr (NS) {
            R fl[5], fr[5];
            const Prim<R> pL = mortar_prim(w[0], Ph.gm1), pR = mortar_prim(w[1], Ph.gm1);
            visc_flux(pL, &w[0][5], Ph.mu, Ph.kappa, s1, s2, s3, fl);
            visc_flux(pR, &w[1][5], Ph.mu, Ph.kappa, s1, s2, s3, fr);
#pragma unroll
            for (int v = 1; v < 5; ++v) fs[v] -= (R)0.5 * (fl[v] + fr[v]);
        }
        R *dL = (R *)SL.fstar6 + ((size_t)(2 * d + 1) * SL.E + F.lL) * 5 * P + p;
        R *dR = (R *)SR.fstar6 + ((size_t)(2 * d) * SR.E + F.lR) * 5 * P + p;
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            dL[v * P] = fs[v];
            dR[v * P] = fs[v];
        }
    }
}

template <typename R, bool NS, int MODE, int N>
static cudaError_t conf_group(const MortarFace *faces, int nfaces, const MortarSide *sides, const double *u, int flux,
                              const MortarPhys<R> &P, cudaStream_t s)
{
    constexpr int n2 = (N + 1) * (N + 1);
    constexpr int FPC = 128 / n2 >= 1 ? 128 / n2 : 1;
    const unsigned blocks = (unsigned)((nfaces + FPC - 1) / FPC);
    k_mortar_conf<R, NS, MODE, N><<<blocks, FPC * n2, 0, s>>>(faces, nfaces, sides, u, flux, P);
    return cudaGetLastError();
}

template <typename R, bool NS, int MODE, int NM>
static cudaError_t mortar_group(const MortarFace *faces, int nfaces, const MortarSide *sides, const double *u,
                                const MortarOps *mo, int flux, const MortarPhys<R> &P, cudaStream_t s)
{
    using S = MortarShape<R, NS, MODE, NM>;
    const size_t smem = sizeof(R) * (size_t)S::FPC * S::PER_FACE;
    static bool attr = false;   // (idempotent; raced writes store the same value)
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mortar<R, NS, MODE, NM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const unsigned blocks = (unsigned)((nfaces + S::FPC - 1) / S::FPC);
    k_mortar<R, NS, MODE, NM><<<blocks, S::THREADS, smem, s>>>(faces, nfaces, sides, u, mo, flux, P);
    return cudaGetLastError();
}

template <typename R, bool NS, int MODE>
static cudaError_t mortar_mode(const MortarFace *faces, const int *group_begin, int only, const MortarSide *sides,
                               const double *u, const MortarOps *mo, int flux, const MortarPhys<R> &P, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
#define HS3D_MG(K)                                                                                                \
    if (e == cudaSuccess && (only < 0 || only == K) && group_begin[K + 1] > group_begin[K])                       \
        e = mortar_group<R, NS, MODE, K>(faces + group_begin[K], group_begin[K + 1] - group_begin[K], sides, u, mo, \
                                         flux, P, s);
    HS3D_MG(1) HS3D_MG(2) HS3D_MG(3) HS3D_MG(4) HS3D_MG(5) HS3D_MG(6) HS3D_MG(7)
#undef HS3D_MG
#define HS3D_CG(K)                                                                                                 \
    if (e == cudaSuccess && (only < 0 || only == kMaxn + K) && group_begin[kMaxn + K + 1] > group_begin[kMaxn + K]) \
        e = conf_group<R, NS, MODE, K>(faces + group_begin[kMaxn + K],                                             \
                                       group_begin[kMaxn + K + 1] - group_begin[kMaxn + K], sides, u, flux, P, s);
    HS3D_CG(1) HS3D_CG(2) HS3D_CG(3) HS3D_CG(4) HS3D_CG(5) HS3D_CG(6) HS3D_CG(7)
#undef HS3D_CG
    return e;
}

cudaError_t launch_mortar(int prec, int physics, int mode, int flux, const MortarFace *faces, const int *group_begin,
                          int only, const MortarSide *sides, const double *u, const MortarPhys<double> &P,
                          cudaStream_t s)
{
    const MortarOps *mo = device_mortar_ops();
    if (!mo) return cudaErrorMemoryAllocation;
    const bool ns = physics == HS3D_NS;
    if (prec == HS3D_FP64) {
        if (mode == 0) return mortar_mode<double, true, 0>(faces, group_begin, only, sides, u, mo, flux, P, s);
        if (ns) return mortar_mode<double, true, 1>(faces, group_begin, only, sides, u, mo, flux, P, s);
        return mortar_mode<double, false, 1>(faces, group_begin, only, sides, u, mo, flux, P, s);
    }
    const MortarPhys<float> Pf{(float)P.gamma, (float)P.gm1, (float)P.hg, (float)P.mu, (float)P.kappa};
    if (mode == 0) return mortar_mode<float, true, 0>(faces, group_begin, only, sides, u, mo, flux, Pf, s);
    if (ns) return mortar_mode<float, true, 1>(faces, group_begin, only, sides, u, mo, flux, Pf, s);
    return mortar_mode<float, false, 1>(faces, group_begin, only, sides, u, mo, flux, Pf, s);
}

// ------------------------------------------------------------------ time step

// dt of a mesh with per-element degrees: the conforming rule per degree
// bucket (its own n, its maxima in clock slot `slot`), minimised over the
// buckets; every bucket's clock then carries the same dt, t and step count,
// and its maxima are reset.  One thread.
__global__ void k_pdt_finalize(Clock *const *clks, const int *nb_n, int nb, double cfl, double kc, double kv, int slot,
                               double dt_fixed)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double dt = dt_fixed > 0.0 ? dt_fixed : INFINITY;
    int bad = 0;
    for (int i = 0; i < nb; ++i) {
        Clock *c = clks[i];
        const double lc = __longlong_as_double((long long)c->lam[slot][0]);
        const double lv = __longlong_as_double((long long)c->lam[slot][1]);
        if (c->bad) bad = c->bad;
        if (dt_fixed > 0.0) continue;
        const double n = nb_n[i];
        double dti = cfl * kc / (n * n * lc);
        if (lv > 0.0) dti = fmin(dti, kv / (n * n * n * n * lv));
        dt = fmin(dt, dti);
    }
    if (!(dt > 0.0) || !(dt < INFINITY)) bad = bad ? bad : 1;
    for (int i = 0; i < nb; ++i) {
        Clock *c = clks[i];
        c->lam[0][0] = c->lam[0][1] = c->lam[1][0] = c->lam[1][1] = 0ull;
        if (bad) {
            c->bad = bad;
            c->done = 1;
            c->dt = 0.0;
            continue;
        }
        c->dt = dt;
        c->t += dt;
        c->step += 1;
    }
}

cudaError_t launch_pdt_finalize(Clock *const *clks, const int *nb_n, int nb, double cfl, double kc, double kv,
                                int slot, double dt_fixed, cudaStream_t s)
{
    k_pdt_finalize<<<1, 1, 0, s>>>(clks, nb_n, nb, cfl, kc, kv, slot, dt_fixed);
    return cudaGetLastError();
}

}  // namespace hs3d
