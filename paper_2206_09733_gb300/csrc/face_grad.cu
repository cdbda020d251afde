// Face Riemann solve and BR1 gradients.
//
// k_face: one thread per face node.  Gathers the two traces (Gauss-Lobatto
// nodes include the element boundary, so the trace is the boundary node
// itself), computes the inviscid numerical flux (LF, Roe, central EC,
// Rusanov, low-dissipation Roe or entropy-stable matrix dissipation,
// Sec. 3.3) times the face scale and, for Navier-Stokes, subtracts the BR1
// viscous flux (F_v(L) + F_v(R)).Sn/2.  Each face is solved once; both
// elements read the result (with opposite sign on the -d side).
//
// k_grad: BR1 gradients of q = (v1, v2, v3, T), T = p/rho (Bassi & Rebay 1997):
//   J grad q_c = sum_d D_d (Ja^d_c q) + sum_faces (1/w_end) (q* - q_in) (+-Ja^d_c),
//   q* = (q_in + q_out)/2.  Element per thread group, node per thread.
#include "internal.cuh"
#include "physics.cuh"

namespace hs3d {

// Index of the node with index `end` along direction d and tangential (ta, tb).
template <int n>
__device__ __forceinline__ int face_node(int d, int end, int ta, int tb)
{
    if (d == 0) return end + n * (ta + n * tb);
    if (d == 1) return ta + n * (end + n * tb);
    return ta + n * (tb + n * end);
}

// Primitive variables of node `idx` (element base + node) of an item: FP64
// path from u, mixed path from the FP32 shadow uf.
template <typename R>
__device__ __forceinline__ Prim<R> load_prim(const Item &it, size_t idx, int n3, R gm1);
template <>
__device__ __forceinline__ Prim<double> load_prim<double>(const Item &it, size_t idx, int n3, double gm1)
{
    double u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = it.u[idx + (size_t)v * n3];
    return prim_from_u<double>(u, gm1);
}
template <>
__device__ __forceinline__ Prim<float> load_prim<float>(const Item &it, size_t idx, int n3, float gm1)
{
    float u[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) u[v] = it.uf[idx + (size_t)v * n3];
    return prim_from_f(u, gm1);
}

template <int N, typename R, bool NS>
__global__ void __launch_bounds__(256) k_face(const __grid_constant__ Batch b, int flux)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= b.total_faces * n2) return;
    const long long gf = t / n2;
    const int ab = (int)(t - gf * n2);
    const Item &it = find_item_face(b, gf);
    if (it.clk && it.clk->done) return;
    const int E = it.E;
    // threads walk the faces element-major (the three +d faces of element 0,
    // then of element 1, ...), so that the state sectors an element's faces
    // share (every xi and eta trace sector holds nodes of both ends) are
    // fetched from DRAM once and then hit in L2; storage stays f = d*E + eL
    const int lf = (int)(gf - it.face_begin);
    const int eL = lf / 3;
    const int d = lf - 3 * eL;
    const int f = d * E + eL;
    const int eR = nbr_plus(eL, d, it.ex, it.ey, it.ez);
    const int ta = ab % n, tb = ab / n;
    const int pL = face_node<n>(d, N, ta, tb), pR = face_node<n>(d, 0, ta, tb);
    
    const Phys<R> P = phys_of<R>(it);
    const size_t iL = (size_t)eL * 5 * n3 + pL, iR = (size_t)eR * 5 * n3 + pR;
    const Prim<R> qL = load_prim<R>(it, iL, n3, P.gm1), qR = load_prim<R>(it, iR, n3, P.gm1);
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
        // conserved traces: the FP32 shadow on the mixed path (flux arithmetic
        // in FP32 throughout); on the FP64 path the jump is formed from u
        R ul[5], ur[5];
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                ul[v] = it.uf[iL + (size_t)v * n3];
                ur[v] = it.uf[iR + (size_t)v * n3];
            }
        } else {
            double uL[5], uR[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                uL[v] = it.u[iL + (size_t)v * n3];
                uR[v] = it.u[iR + (size_t)v * n3];
            }
            ul[0] = qL.rho; ul[1] = narrow<R>(uL[1]); ul[2] = narrow<R>(uL[2]); ul[3] = narrow<R>(uL[3]); ul[4] = qL.E;
#pragma unroll
            for (int v = 0; v < 5; ++v) ur[v] = ul[v] + narrow<R>(uR[v] - uL[v]);
        }
        flux_lf(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_RUSANOV) {
        R ul[5], ur[5];
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                ul[v] = it.uf[iL + (size_t)v * n3];
                ur[v] = it.uf[iR + (size_t)v * n3];
            }
        } else {
            double uL[5], uR[5];
#pragma unroll
            for (int v = 0; v < 5; ++v) {
                uL[v] = it.u[iL + (size_t)v * n3];
                uR[v] = it.u[iR + (size_t)v * n3];
            }
            ul[0] = qL.rho; ul[1] = narrow<R>(uL[1]); ul[2] = narrow<R>(uL[2]); ul[3] = narrow<R>(uL[3]); ul[4] = qL.E;
#pragma unroll
            for (int v = 0; v < 5; ++v) ur[v] = ul[v] + narrow<R>(uR[v] - uL[v]);
        }
        flux_rusanov(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    } else if (flux == HS3D_FLUX_MATRIX) {
        flux_matrix(qL, qR, P.gamma, P.hg, s1, s2, s3, fs);
    } else {
        const R ul[5] = {qL.rho, (R)0, (R)0, (R)0, qL.E};
        const R ur[5] = {qR.rho, (R)0, (R)0, (R)0, qR.E};
        if (flux == HS3D_FLUX_LDROE) flux_ldroe(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
        else flux_roe(qL, ul, qR, ur, P.gamma, s1, s2, s3, fs);
    }
    if (NS) {
        const R *GL = (const R *)it.grad + (size_t)eL * 12 * n3 + pL;
        const R *GR = (const R *)it.grad + (size_t)eR * 12 * n3 + pR;
        R gl[12], gr[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            gl[k] = GL[k * n3];
            gr[k] = GR[k * n3];
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
constexpr int grad_threads()
{
    return ((N + 1) * (N + 1) * (N + 1) > 256) ? (N + 1) * (N + 1) * (N + 1) : 256;
}

template <typename R>
__device__ __forceinline__ void grad_vars(const Prim<R> &q, R out[4])
{
    out[0] = q.v1;
    out[1] = q.v2;
    out[2] = q.v3;
    out[3] = q.p / q.rho;
}

template <typename R>
__device__ __forceinline__ const R *grad_metric(const Item &it);
template <>
__device__ __forceinline__ const double *grad_metric<double>(const Item &it) { return it.Ja; }
template <>
__device__ __forceinline__ const float *grad_metric<float>(const Item &it) { return it.Jaf; }

// Shared memory per element: q [4][n3], Ja [9][n3], neighbour traces of q
// [6 faces][4][n2] (slot 2d: the -d face, slot 2d+1: the +d face).  The
// neighbour traces are gathered by all threads of the element before the
// barrier, so the lifting reads no global memory.
// Shared-memory words per element of k_grad: q (or, on the bulk path, the
// staged FP32 state whose first four planes then hold q), Ja, neighbour traces.
template <int N, typename R>
constexpr bool grad_bulk()
{
    return sizeof(R) == 4 && (N + 1) % 2 == 0;
}
template <int N, typename R>
constexpr int grad_per_elem()
{
    return ((grad_bulk<N, R>() ? 5 : 4) + 9) * (N + 1) * (N + 1) * (N + 1) + 24 * (N + 1) * (N + 1);
}

template <int N, typename R>
__global__ void __launch_bounds__(grad_threads<N>()) k_grad(const __grid_constant__ Batch b, const Ops *__restrict__ ops)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    // mixed path with an even number of nodes per direction: the element's
    // FP32 state and metric terms arrive in shared memory by bulk copies
    // (TMA engine, one thread per element, counted on the element's
    // mbarrier) while its threads gather the neighbour traces
    constexpr bool BULK = grad_bulk<N, R>();
    constexpr int QW = BULK ? 5 : 4;
    constexpr int PER_ELEM = grad_per_elem<N, R>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ unsigned long long bulk_bar[BULK ? 256 / (n3 < 256 ? n3 : 256) : 1];
    R *sD = (R *)smem_raw;                      // n*n
    R *sE = sD + ((n * n + 1) & ~1);            // [epb][PER_ELEM]
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
    R *q = sE + (size_t)le * PER_ELEM;
    R *ja = q + QW * n3;
    R *qn = ja + 9 * n3;
    R qin[4];
    if constexpr (BULK) {
        // the element's barrier is initialised before any of its threads polls it
        if (valid && p == 0) mbar_init(bulk_bar + le, 1);
        __syncthreads();
    }
    if (valid) {
        const Item &it = *itp;
        const R gm1 = phys_of<R>(it).gm1;
        if constexpr (BULK) {
            if (p == 0) {
                unsigned long long *bar = bulk_bar + le;
                mbar_arrive_expect_tx(bar, 14 * n3 * 4);
                bulk_g2s(q, it.uf + (size_t)e * 5 * n3, 5 * n3 * 4, bar);
                bulk_g2s(ja, it.Jaf + (size_t)e * 9 * n3, 9 * n3 * 4, bar);
            }
        }
        // neighbour traces of q: all loads of this thread's face points first
        // (the loop is unrolled to its fixed trip count), then the conversions
        constexpr int IT = (6 * n2 + n3 - 1) / n3;
        if (it.face6) {
            // mesh with per-element degrees: the mortar kernel left 2 q*_e - q_in
#pragma unroll
            for (int k = 0; k < IT; ++k) {
                const int t = p + k * n3;
                if (t < 6 * n2) {
                    const int slot = t / n2, ab = t - slot * n2;
                    const R *src = (const R *)it.qhat6 + ((size_t)slot * it.E + e) * 4 * n2 + ab;
#pragma unroll
                    for (int v = 0; v < 4; ++v) qn[(slot * 4 + v) * n2 + ab] = src[v * n2];
                }
            }
        }
        const Nbrs nbs = elem_nbrs(e, it.ex, it.ey, it.ez);
        const R *st;
        if constexpr (sizeof(R) == 4) st = it.uf;
        else st = it.u;
        R raw[IT][5];
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            if (it.face6) break;
            const int t = p + k * n3;
            if (t < 6 * n2) {
                const int slot = t / n2, ab = t - slot * n2;
                const int d = slot >> 1, plus = slot & 1;
                const int pn = face_node<n>(d, plus ? 0 : N, ab % n, ab / n);
                const R *src = st + (size_t)nbr_of_slot(nbs, slot) * 5 * n3 + pn;
#pragma unroll
                for (int v = 0; v < 5; ++v) raw[k][v] = src[v * n3];
            }
        }
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            if (it.face6) break;
            const int t = p + k * n3;
            if (t < 6 * n2) {
                const int slot = t / n2, ab = t - slot * n2;
                R g4[4];
                if constexpr (sizeof(R) == 4) grad_vars(prim_from_f(raw[k], gm1), g4);
                else grad_vars(prim_from_u<R>(raw[k], gm1), g4);
#pragma unroll
                for (int v = 0; v < 4; ++v) qn[(slot * 4 + v) * n2 + ab] = g4[v];
            }
        }
        if constexpr (BULK) {
            float us[5];
            if (mbar_wait(bulk_bar + le, 0, kBulkWaitPolls)) {
#pragma unroll
                for (int v = 0; v < 5; ++v) us[v] = q[v * n3 + p];
            } else {
                // a wait that ran out of polls poisons the gradients and flags the solve
#pragma unroll
                for (int v = 0; v < 5; ++v) us[v] = NAN;
                if (it.clk) it.clk->bad = 2;
            }
            grad_vars(prim_from_f(us, gm1), qin);
        } else {
            grad_vars(load_prim<R>(it, (size_t)e * 5 * n3 + p, n3, gm1), qin);
            const R *JA = grad_metric<R>(it) + (size_t)e * 9 * n3 + p;
#pragma unroll
            for (int k = 0; k < 9; ++k) ja[k * n3 + p] = JA[k * n3];
        }
        // (on the bulk path this overwrites the staged state at this node only)
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v * n3 + p] = qin[v];
    }
    __syncthreads();
    if (!valid) return;
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
            const R a1 = Dm * ja[(d * 3 + 0) * n3 + pm], a2 = Dm * ja[(d * 3 + 1) * n3 + pm],
                    a3 = Dm * ja[(d * 3 + 2) * n3 + pm];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const R qv = q[v * n3 + pm];
                acc[v * 3 + 0] += a1 * qv;
                acc[v * 3 + 1] += a2 * qv;
                acc[v * 3 + 2] += a3 * qv;
            }
        }
    }
    // surface lifting of the BR1 jumps (q* - q_in) = (q_out - q_in)/2
    const Item &it = *itp;
    const R iw = ops_iw0<R>(ops);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int ta = (d == 0) ? ijk[1] : ijk[0];
        const int tb = (d == 2) ? ijk[1] : ijk[2];
        const int ab = ta + n * tb;
#pragma unroll
        for (int plus = 0; plus < 2; ++plus) {
            if (ijk[d] != (plus ? N : 0)) continue;
            const R sg = plus ? (R)1 : (R)-1;
            const R n1 = sg * ja[(d * 3 + 0) * n3 + p], n2_ = sg * ja[(d * 3 + 1) * n3 + p],
                    n3_ = sg * ja[(d * 3 + 2) * n3 + p];
            const int slot = 2 * d + plus;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const R j = (R)0.5 * (qn[(slot * 4 + v) * n2 + ab] - qin[v]) * iw;
                acc[v * 3 + 0] += j * n1;
                acc[v * 3 + 1] += j * n2_;
                acc[v * 3 + 2] += j * n3_;
            }
        }
    }
    R ij;
    if constexpr (sizeof(R) == 8) ij = it.invJ[(size_t)e * n3 + p];
    else ij = it.invJf[(size_t)e * n3 + p];
    R *G = (R *)it.grad + (size_t)e * 12 * n3 + p;
#pragma unroll
    for (int k = 0; k < 12; ++k) G[k * n3] = acc[k] * ij;
}

// ------------------------------------------------------------------ launchers

template <int N, typename R>
static cudaError_t face_launch(int physics, int flux, const Batch &b, cudaStream_t s)
{
    constexpr int n2 = (N + 1) * (N + 1);
    long long total = b.total_faces * n2;
    if (total == 0) return cudaSuccess;
    unsigned blocks = (unsigned)((total + 255) / 256);
    if (physics == HS3D_NS) k_face<N, R, true><<<blocks, 256, 0, s>>>(b, flux);
    else k_face<N, R, false><<<blocks, 256, 0, s>>>(b, flux);
    return cudaGetLastError();
}

template <int N, typename R>
static cudaError_t grad_launch(const Batch &b, cudaStream_t s)
{
    constexpr int n = N + 1, n3 = n * n * n;
    if (b.total_elems == 0) return cudaSuccess;
    int epb = elems_per_block_p(N, sizeof(R) == 4 ? HS3D_MIXED32 : HS3D_FP64, 0);
    if (epb * n3 > grad_threads<N>()) epb = grad_threads<N>() / n3;
    int threads = epb * n3;
    size_t smem = sizeof(R) * (((n * n + 1) & ~1) + (size_t)epb * grad_per_elem<N, R>());
    unsigned blocks = (unsigned)((b.total_elems + epb - 1) / epb);
    const Ops *ops = device_ops(N);
    if (!ops) return cudaErrorMemoryAllocation;
    k_grad<N, R><<<blocks, threads, smem, s>>>(b, ops);
    return cudaGetLastError();
}

template <int N>
static cudaError_t prep_grad()
{
    cudaError_t e = cudaFuncSetAttribute(k_grad<N, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_grad<N, double>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = prepare_grad_dev(N);
    return e;
}

#define HS3D_SWITCH_N(CALL_N)                 \
    switch (N) {                              \
        case 1: return CALL_N(1);             \
        case 2: return CALL_N(2);             \
        case 3: return CALL_N(3);             \
        case 4: return CALL_N(4);             \
        case 5: return CALL_N(5);             \
        case 6: return CALL_N(6);             \
        case 7: return CALL_N(7);             \
        default: return cudaErrorInvalidValue; \
    }

cudaError_t prepare_grad(int N)
{
#define P(K) prep_grad<K>()
    HS3D_SWITCH_N(P)
#undef P
}

cudaError_t launch_face(int N, int prec, int physics, int flux, const Batch &b, cudaStream_t s)
{
    if (b.gauss) return launch_face_gauss(N, prec, physics, flux, b, s);
    if (prec != HS3D_FP64) return launch_face_dev(N, physics, flux, b, s);
#define F64(K) face_launch<K, double>(physics, flux, b, s)
    HS3D_SWITCH_N(F64)
#undef F64
}

cudaError_t launch_grad(int N, int prec, const Batch &b, cudaStream_t s)
{
    if (b.gauss) return launch_grad_gauss(N, prec, b, s);
    if (prec != HS3D_FP64) return launch_grad_dev(N, b, s);
#define G64(K) grad_launch<K, double>(b, s)
    HS3D_SWITCH_N(G64)
#undef G64
}

}  // namespace hs3d
