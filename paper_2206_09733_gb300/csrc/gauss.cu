// Kernels for Gauss-Legendre solution nodes (Sec. 3.3 allows Gauss as well as
// Gauss-Lobatto quadrature points).  The nodes exclude the element boundary,
// so every face value is an interpolation along the line of nodes normal to
// the face, u(side) = sum_j l_j(side) u_j with l_j(+-1) the Lagrange basis at
// the end points, and the surface term lifts onto every node of that line:
//
//   face kernel   F* from the interpolated conserved traces of the two
//                 elements (and, for Navier-Stokes, the interpolated BR1
//                 gradients), with the face metric of the minus-side element;
//   BR1 gradients J grad q_c = sum_d D_d (Ja^d_c q)
//                   + sum_faces (l_i(side)/w_i) side [q* Sf_c - (Ja^d_c q)(side)],
//                 q* = (q(u_in(side)) + q(u_out(side)))/2, Sf the face metric;
//   element       du/dt = -(1/J)[ sum_d D_d F~^d
//                   + sum_faces (l_i(side)/w_i) side (F* - F~^d(side)) ],
//                 F~^d(side) the element's own contravariant flux interpolated
//                 to the face, then the RK stage as on Gauss-Lobatto nodes.
// Only the standard volume term exists here: the split forms rest on the
// summation-by-parts property with boundary nodes.  The per-face-point
// quantities (traces, lifted differences) are formed once per face point by
// the element's threads in shared memory and then read by every node of the
// line.
#include "volume_kernel.cuh"

namespace hs3d {

// Node along direction d with index idx and tangential indices (ta, tb).
template <int n>
__device__ __forceinline__ int gline(int d, int idx, int ta, int tb)
{
    if (d == 0) return idx + n * (ta + n * tb);
    if (d == 1) return ta + n * (idx + n * tb);
    return ta + n * (tb + n * idx);
}

// Interpolated conserved trace of element-local node line (d, ta, tb) at the
// end `plus` from global memory: FP64 path from u, mixed path from the FP32
// shadow.
template <int n, typename R>
__device__ __forceinline__ void trace_u(const Item &it, const Ops *ops, int e, int d, int plus, int ta, int tb,
                                        R out[5])
{
    constexpr int n3 = n * n * n;
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v] = (R)0;
#pragma unroll
    for (int j = 0; j < n; ++j) {
        const R l = plus ? ops_rb<R>(ops, j) : ops_lb<R>(ops, j);
        const size_t idx = (size_t)e * 5 * n3 + gline<n>(d, j, ta, tb);
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            R x;
            if constexpr (sizeof(R) == 8) x = it.u[idx + (size_t)v * n3];
            else x = it.uf[idx + (size_t)v * n3];
            out[v] += l * x;
        }
    }
}

template <typename R>
__device__ __forceinline__ Prim<R> prim_of(const R u[5], R gm1);
template <>
__device__ __forceinline__ Prim<double> prim_of<double>(const double u[5], double gm1)
{
    return prim_from_u<double>(u, gm1);
}
template <>
__device__ __forceinline__ Prim<float> prim_of<float>(const float u[5], float gm1)
{
    return prim_from_f(u, gm1);
}

// ------------------------------------------------------------------ faces

template <int N, typename R, bool NS>
__global__ void __launch_bounds__(256) k_face_gauss(const __grid_constant__ Batch b, const Ops *__restrict__ ops,
                                                    int flux)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= b.total_faces * n2) return;
    const long long gf = t / n2;
    const int ab = (int)(t - gf * n2);
    const Item &it = find_item_face(b, gf);
    if (it.clk && it.clk->done) return;
    const int E = it.E;
    // element-major walk over the faces (as k_face), storage f = d*E + eL
    const int lf = (int)(gf - it.face_begin);
    const int eL = lf / 3;
    const int d = lf - 3 * eL;
    const int f = d * E + eL;
    const int eR = nbr_plus(eL, d, it.ex, it.ey, it.ez);
    const int ta = ab % n, tb = ab / n;
    const Phys<R> P = phys_of<R>(it);
    R ul[5], ur[5];
    trace_u<n, R>(it, ops, eL, d, 1, ta, tb, ul);
    trace_u<n, R>(it, ops, eR, d, 0, ta, tb, ur);
    const Prim<R> qL = prim_of<R>(ul, P.gm1), qR = prim_of<R>(ur, P.gm1);
    R s1, s2, s3;
    if constexpr (sizeof(R) == 8) {
        const double *Fn = it.fn + (size_t)f * 3 * n2 + ab;
        s1 = Fn[0];
        s2 = Fn[n2];
        s3 = Fn[2 * n2];
    } else {
        const float *Fn = it.fnf + (size_t)f * 3 * n2 + ab;
        s1 = Fn[0];
        s2 = Fn[n2];
        s3 = Fn[2 * n2];
    }
    R fs[5];
    if (flux == HS3D_FLUX_EC) {
        flux_ec(ec_node(qL), ec_node(qR), P.hg, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_LF) {
        flux_lf(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_RUSANOV) {
        flux_rusanov(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_MATRIX) {
        flux_matrix(qL, qR, P.gamma, P.hg, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_LDROE) {
        flux_ldroe(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else {
        flux_roe(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    }
    if (NS) {
        R gl[12], gr[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            gl[k] = (R)0;
            gr[k] = (R)0;
        }
        const R *GL = (const R *)it.grad + (size_t)eL * 12 * n3;
        const R *GR = (const R *)it.grad + (size_t)eR * 12 * n3;
#pragma unroll
        for (int j = 0; j < n; ++j) {
            const R lr = ops_rb<R>(ops, j), ll = ops_lb<R>(ops, j);
            const int pj = gline<n>(d, j, ta, tb);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                gl[k] += lr * GL[k * n3 + pj];
                gr[k] += ll * GR[k * n3 + pj];
            }
        }
        R fl[5], fr[5];
        visc_flux(qL, gl, P.mu, P.kappa, s1, s2, s3, fl);
        visc_flux(qR, gr, P.mu, P.kappa, s1, s2, s3, fr);
#pragma unroll
        for (int v = 1; v < 5; ++v) fs[v] -= (R)0.5 * (fl[v] + fr[v]);
    }
    R *out = (R *)it.fstar + (size_t)f * 5 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) out[v * n2] = fs[v];
}

// ------------------------------------------------------------------ BR1 gradients

template <int N>
constexpr int gauss_threads()
{
    return ((N + 1) * (N + 1) * (N + 1) > 256) ? (N + 1) * (N + 1) * (N + 1) : 256;
}

template <int N>
constexpr int grad_gauss_per_elem()
{
    return 18 * (N + 1) * (N + 1) * (N + 1) + 72 * (N + 1) * (N + 1);
}

template <typename R>
__device__ __forceinline__ const R *gmetric(const Item &it);
template <>
__device__ __forceinline__ const double *gmetric<double>(const Item &it) { return it.Ja; }
template <>
__device__ __forceinline__ const float *gmetric<float>(const Item &it) { return it.Jaf; }

template <typename R>
__device__ __forceinline__ const R *gnormal(const Item &it);
template <>
__device__ __forceinline__ const double *gnormal<double>(const Item &it) { return it.fn; }
template <>
__device__ __forceinline__ const float *gnormal<float>(const Item &it) { return it.fnf; }

// Shared memory per element: u [5][n3], q [4][n3], Ja [9][n3], lifted face
// differences [6 faces][12][n2] (slot 2d: the -d face, 2d+1: the +d face).
template <int N, typename R>
__global__ void __launch_bounds__(gauss_threads<N>())
k_grad_gauss(const __grid_constant__ Batch b, const Ops *__restrict__ ops)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr int PER = grad_gauss_per_elem<N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sD = (R *)smem_raw;
    R *sE = sD + ((n * n + 1) & ~1);
    const int epb = blockDim.x / n3;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = ops_D<R>(ops, t);
    const int le = threadIdx.x / n3, p = threadIdx.x - le * n3;
    const long long ge = blockIdx.x * (long long)epb + le;
    bool valid = ge < b.total_elems;
    const Item *itp = nullptr;
    int e = 0;
    if (valid) {
        itp = &find_item_elem(b, ge);
        e = (int)(ge - itp->elem_begin);
        if (itp->clk && itp->clk->done) valid = false;
    }
    R *su = sE + (size_t)le * PER;
    R *sq = su + 5 * n3;
    R *sja = sq + 4 * n3;
    R *slift = sja + 9 * n3;
    if (valid) {
        const Item &it = *itp;
        const R gm1 = phys_of<R>(it).gm1;
        R uu[5];
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            if constexpr (sizeof(R) == 8) uu[v] = it.u[(size_t)e * 5 * n3 + p + (size_t)v * n3];
            else uu[v] = it.uf[(size_t)e * 5 * n3 + p + (size_t)v * n3];
            su[v * n3 + p] = uu[v];
        }
        const Prim<R> qp = prim_of<R>(uu, gm1);
        sq[0 * n3 + p] = qp.v1;
        sq[1 * n3 + p] = qp.v2;
        sq[2 * n3 + p] = qp.v3;
        sq[3 * n3 + p] = qp.p / qp.rho;
        const R *JA = gmetric<R>(it) + (size_t)e * 9 * n3 + p;
#pragma unroll
        for (int k = 0; k < 9; ++k) sja[k * n3 + p] = JA[k * n3];
    }
    __syncthreads();
    if (valid) {
        // face points: q* from both interpolated traces, minus the
        // interpolated products Ja^d_c q, times the face metric
        const Item &it = *itp;
        const R gm1 = phys_of<R>(it).gm1;
        const Nbrs nbs = elem_nbrs(e, it.ex, it.ey, it.ez);
        for (int t = p; t < 6 * n2; t += n3) {
            const int slot = t / n2, ab = t - slot * n2;
            const int d = slot >> 1, plus = slot & 1;
            const int ta = ab % n, tb = ab / n;
            const int nb = nbr_of_slot(nbs, slot);
            R uo[5], un[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) uo[v] = (R)0;
#pragma unroll
            for (int j = 0; j < n; ++j) {
                const R l = plus ? ops_rb<R>(ops, j) : ops_lb<R>(ops, j);
                const int pj = gline<n>(d, j, ta, tb);
#pragma unroll
                for (int v = 0; v < 5; ++v) uo[v] += l * su[v * n3 + pj];
            }
            trace_u<n, R>(it, ops, nb, d, plus ? 0 : 1, ta, tb, un);
            const Prim<R> po = prim_of<R>(uo, gm1), pn = prim_of<R>(un, gm1);
            const R qs[4] = {(R)0.5 * (po.v1 + pn.v1), (R)0.5 * (po.v2 + pn.v2), (R)0.5 * (po.v3 + pn.v3),
                             (R)0.5 * (po.p / po.rho + pn.p / pn.rho)};
            // own face metric: this face's normal, held by its minus-side element
            const int owner = plus ? e : nb;
            const R *Sf = gnormal<R>(it) + ((size_t)d * it.E + owner) * 3 * n2 + ab;
            const R sf[3] = {Sf[0], Sf[n2], Sf[2 * n2]};
            const R sg = plus ? (R)1 : (R)-1;
            // interpolated products (Ja^d_c q_v)(+-1): line node by line node,
            // each node's 3 metric terms and 4 variables read once
            R jq[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) jq[k] = (R)0;
#pragma unroll
            for (int j = 0; j < n; ++j) {
                const R l = plus ? ops_rb<R>(ops, j) : ops_lb<R>(ops, j);
                const int pj = gline<n>(d, j, ta, tb);
                R jac[3], qv[4];
#pragma unroll
                for (int c = 0; c < 3; ++c) jac[c] = sja[(d * 3 + c) * n3 + pj];
#pragma unroll
                for (int v = 0; v < 4; ++v) qv[v] = sq[v * n3 + pj];
#pragma unroll
                for (int v = 0; v < 4; ++v)
#pragma unroll
                    for (int c = 0; c < 3; ++c) jq[v * 3 + c] += l * (jac[c] * qv[v]);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    slift[(slot * 12 + v * 3 + c) * n2 + ab] = sg * (qs[v] * sf[c] - jq[v * 3 + c]);
        }
    }
    __syncthreads();
    if (!valid) return;
    const Item &it = *itp;
    const int ijk[3] = {p % n, (p / n) % n, p / n2};
    R acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = (R)0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int stride = (d == 0) ? 1 : (d == 1) ? n : n2;
        const int base = p - ijk[d] * stride;
        const R *Drow = sD + ijk[d] * n;
#pragma unroll
        for (int m = 0; m < n; ++m) {
            const int pm = base + m * stride;
            const R Dm = Drow[m];
            const R a1 = Dm * sja[(d * 3 + 0) * n3 + pm], a2 = Dm * sja[(d * 3 + 1) * n3 + pm],
                    a3 = Dm * sja[(d * 3 + 2) * n3 + pm];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const R qv = sq[v * n3 + pm];
                acc[v * 3 + 0] += a1 * qv;
                acc[v * 3 + 1] += a2 * qv;
                acc[v * 3 + 2] += a3 * qv;
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int i = ijk[d];
        const int ta = (d == 0) ? ijk[1] : ijk[0];
        const int tb = (d == 2) ? ijk[1] : ijk[2];
        const int ab = ta + n * tb;
        const R wp = ops_rbw<R>(ops, i), wm = ops_lbw<R>(ops, i);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            acc[k] += wp * slift[((2 * d + 1) * 12 + k) * n2 + ab] + wm * slift[((2 * d) * 12 + k) * n2 + ab];
    }
    R ij;
    if constexpr (sizeof(R) == 8) ij = it.invJ[(size_t)e * n3 + p];
    else ij = it.invJf[(size_t)e * n3 + p];
    R *G = (R *)it.grad + (size_t)e * 12 * n3 + p;
#pragma unroll
    for (int k = 0; k < 12; ++k) G[k * n3] = acc[k] * ij;
}

// ------------------------------------------------------------------ element kernel (standard form)

// Shared memory per element: contravariant fluxes [15][n3], face fluxes then
// lifted differences [6][5][n2].
template <int N, typename R, bool NS>
__global__ void __launch_bounds__(gauss_threads<N>(), vol_min_blocks<N, R>())
k_volume_gauss(const __grid_constant__ Batch b, const Ops *__restrict__ ops, int stage, double rkA, double rkB,
               int lam_slot)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr int FACEVALS = 6 * 5 * n2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *sD = (R *)smem_raw;
    const int epb = blockDim.x / n3;
    R *sbuf = sD + ((n * n + 1) & ~1);
    R *sface = sbuf + (size_t)epb * 15 * n3;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = ops_D<R>(ops, t);
    const int le = threadIdx.x / n3, p = threadIdx.x - le * n3;
    const long long ge = blockIdx.x * (long long)epb + le;
    bool valid = ge < b.total_elems;
    const Item *itp = nullptr;
    int e = 0;
    if (valid) {
        itp = &find_item_elem(b, ge);
        e = (int)(ge - itp->elem_begin);
        if (itp->clk && itp->clk->done) valid = false;
    }
    R *S = sbuf + (size_t)le * 15 * n3;
    R *F6 = sface + (size_t)le * FACEVALS;
    const int ijk[3] = {p % n, (p / n) % n, p / n2};
    double u[5];
    if (valid) {
        const Item &it = *itp;
        const R *FS = (const R *)it.fstar;
        const Nbrs nb = elem_nbrs(e, it.ex, it.ey, it.ez);
#pragma unroll
        for (int slot = 0; slot < 6; ++slot) {
            const int d = slot >> 1;
            const int owner = (slot & 1) ? e : nb.m[d];
            cp_async_block<R>(F6 + slot * 5 * n2, FS + ((size_t)d * it.E + owner) * 5 * n2, 5 * n2, p, n3);
        }
        const size_t node = (size_t)e * 5 * n3 + p;
        const Phys<R> P = phys_of<R>(it);
        R ja[9];
        const R *JA = metric_ptr<R>(it) + (size_t)e * 9 * n3 + p;
#pragma unroll
        for (int k = 0; k < 9; ++k) ja[k] = JA[k * n3];
        Prim<R> q;
        if constexpr (sizeof(R) == 8) {
#pragma unroll
            for (int v = 0; v < 5; ++v) u[v] = it.u[node + v * n3];
            q = prim_from_u<R>(u, P.gm1);
        } else {
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
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            R fe[5], fv[5] = {(R)0, (R)0, (R)0, (R)0, (R)0};
            euler_flux(q, q.E, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fe);
            if (NS) visc_flux(q, G, P.mu, P.kappa, ja[d * 3], ja[d * 3 + 1], ja[d * 3 + 2], fv);
#pragma unroll
            for (int v = 0; v < 5; ++v) S[(d * 5 + v) * n3 + p] = NS ? fe[v] - fv[v] : fe[v];
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (valid) {
        // face points: side (F* - F~^d(side)), in place of F*
        for (int t = p; t < 6 * n2; t += n3) {
            const int slot = t / n2, ab = t - slot * n2;
            const int d = slot >> 1, plus = slot & 1;
            const int ta = ab % n, tb = ab / n;
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                R own = (R)0;
#pragma unroll
                for (int j = 0; j < n; ++j) {
                    const R l = plus ? ops_rb<R>(ops, j) : ops_lb<R>(ops, j);
                    own += l * S[(d * 5 + v) * n3 + gline<n>(d, j, ta, tb)];
                }
                R *Fp = F6 + (slot * 5 + v) * n2 + ab;
                *Fp = plus ? (*Fp - own) : (own - *Fp);
            }
        }
    }
    __syncthreads();
    double lc = 0.0, lv = 0.0;
    bool lam_active = false;
    if (valid) {
        R V[5] = {(R)0, (R)0, (R)0, (R)0, (R)0};
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
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int i = ijk[d];
            const int ta = (d == 0) ? ijk[1] : ijk[0];
            const int tb = (d == 2) ? ijk[1] : ijk[2];
            const int ab = ta + n * tb;
            const R wp = ops_rbw<R>(ops, i), wm = ops_lbw<R>(ops, i);
#pragma unroll
            for (int v = 0; v < 5; ++v)
                V[v] += wp * F6[((2 * d + 1) * 5 + v) * n2 + ab] + wm * F6[((2 * d) * 5 + v) * n2 + ab];
        }
        node_update<R, NS>(*itp, e, p, n3, V, u, stage, rkA, rkB, lam_slot, lc, lv, lam_active);
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

// ------------------------------------------------------------------ launchers

template <int N, typename R>
static cudaError_t face_gauss(int physics, int flux, const Batch &b, cudaStream_t s)
{
    constexpr int n2 = (N + 1) * (N + 1);
    const long long total = b.total_faces * n2;
    if (total == 0) return cudaSuccess;
    const Ops *ops = device_ops(N, HS3D_NODES_GAUSS);
    if (!ops) return cudaErrorMemoryAllocation;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    if (physics == HS3D_NS) k_face_gauss<N, R, true><<<blocks, 256, 0, s>>>(b, ops, flux);
    else k_face_gauss<N, R, false><<<blocks, 256, 0, s>>>(b, ops, flux);
    return cudaGetLastError();
}

template <int N>
static int gauss_epb(int prec, int which)
{
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    int epb = elems_per_block_p(N, prec, which);
    if (epb * n3 > gauss_threads<N>()) epb = gauss_threads<N>() / n3;
    return epb < 1 ? 1 : epb;
}

template <int N, typename R>
static cudaError_t grad_gauss(const Batch &b, cudaStream_t s)
{
    constexpr int n = N + 1, n3 = n * n * n;
    if (b.total_elems == 0) return cudaSuccess;
    const int epb = gauss_epb<N>(sizeof(R) == 4 ? HS3D_MIXED32 : HS3D_FP64, 0);
    const size_t smem = sizeof(R) * (((n * n + 1) & ~1) + (size_t)epb * grad_gauss_per_elem<N>());
    const unsigned blocks = (unsigned)((b.total_elems + epb - 1) / epb);
    const Ops *ops = device_ops(N, HS3D_NODES_GAUSS);
    if (!ops) return cudaErrorMemoryAllocation;
    k_grad_gauss<N, R><<<blocks, epb * n3, smem, s>>>(b, ops);
    return cudaGetLastError();
}

template <int N, typename R, bool NS>
static cudaError_t volume_gauss(const Batch &b, int stage, double rkA, double rkB, int lam_slot, cudaStream_t s)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    if (b.total_elems == 0) return cudaSuccess;
    const int epb = gauss_epb<N>(sizeof(R) == 4 ? HS3D_MIXED32 : HS3D_FP64, 1);
    const size_t smem = sizeof(R) * (((n * n + 1) & ~1) + (size_t)epb * (15 * n3 + 30 * n2));
    const unsigned blocks = (unsigned)((b.total_elems + epb - 1) / epb);
    const Ops *ops = device_ops(N, HS3D_NODES_GAUSS);
    if (!ops) return cudaErrorMemoryAllocation;
    k_volume_gauss<N, R, NS><<<blocks, epb * n3, smem, s>>>(b, ops, stage, rkA, rkB, stage >= 0 ? lam_slot : -1);
    return cudaGetLastError();
}

template <int N>
static cudaError_t prep_gauss_n()
{
    const int big = 220 * 1024;
    cudaError_t e = cudaSuccess;
#define HS3D_ATTR(K)                                                                                   \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, big); \
    if (e == cudaSuccess)                                                                              \
        e = cudaFuncSetAttribute(K, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    HS3D_ATTR((k_grad_gauss<N, double>))
    HS3D_ATTR((k_grad_gauss<N, float>))
    HS3D_ATTR((k_volume_gauss<N, double, false>))
    HS3D_ATTR((k_volume_gauss<N, double, true>))
    HS3D_ATTR((k_volume_gauss<N, float, false>))
    HS3D_ATTR((k_volume_gauss<N, float, true>))
#undef HS3D_ATTR
    return e;
}

#define HS3D_GSWITCH(CALL)                         \
    switch (N) {                                   \
        case 1: return CALL(1);                    \
        case 2: return CALL(2);                    \
        case 3: return CALL(3);                    \
        case 4: return CALL(4);                    \
        case 5: return CALL(5);                    \
        case 6: return CALL(6);                    \
        case 7: return CALL(7);                    \
    }                                              \
    return cudaErrorInvalidValue;

cudaError_t prepare_gauss(int N)
{
#define C_(K) prep_gauss_n<K>()
    HS3D_GSWITCH(C_)
#undef C_
}

cudaError_t launch_face_gauss(int N, int prec, int physics, int flux, const Batch &b, cudaStream_t s)
{
#define C_(K) (prec == HS3D_FP64 ? face_gauss<K, double>(physics, flux, b, s) : face_gauss<K, float>(physics, flux, b, s))
    HS3D_GSWITCH(C_)
#undef C_
}

cudaError_t launch_grad_gauss(int N, int prec, const Batch &b, cudaStream_t s)
{
#define C_(K) (prec == HS3D_FP64 ? grad_gauss<K, double>(b, s) : grad_gauss<K, float>(b, s))
    HS3D_GSWITCH(C_)
#undef C_
}

cudaError_t launch_volume_gauss(int N, int prec, int physics, const Batch &b, int stage, double rkA, double rkB,
                                int lam_slot, cudaStream_t s)
{
#define C_(K)                                                                                                  \
    (prec == HS3D_FP64                                                                                         \
         ? (physics == HS3D_NS ? volume_gauss<K, double, true>(b, stage, rkA, rkB, lam_slot, s)                \
                               : volume_gauss<K, double, false>(b, stage, rkA, rkB, lam_slot, s))              \
         : (physics == HS3D_NS ? volume_gauss<K, float, true>(b, stage, rkA, rkB, lam_slot, s)                 \
                               : volume_gauss<K, float, false>(b, stage, rkA, rkB, lam_slot, s)))
    HS3D_GSWITCH(C_)
#undef C_
}

#undef HS3D_GSWITCH

}  // namespace hs3d
