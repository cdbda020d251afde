// BR1 gradients of the mixed path (FP32 arithmetic on deviations).
//
//   J grad q_c = sum_d D_d (Ja^d_c q) + sum_faces (1/w_end) (q* - q_in) (+-Ja^d_c),
//   q = (v1, v2, v3, T), T = p/rho, q* = (q_in + q_out)/2           (Bassi & Rebay 1997)
//
// The element's reference state ubar (its centre node, lowmach.cuh) turns the
// FP64 state into deviations, and q into q - qbar: the constant qbar drops
// out of the volume term by the discrete metric identity and out of every
// jump, so T' = T - Tbar = (p' - Tbar rho' + rT)/rho (rT = pbar - Tbar rhobar)
// keeps its accuracy relative to the temperature fluctuation instead of to
// T ~ 1/(gamma Ma^2).  The neighbours' traces are read in FP64 and made
// deviations from the same reference, so the lifted jumps are accurate.
// On a mesh with per-element degrees (Item::face6) the mortar kernel supplies
// 2 q*_e - q_in in full FP32 values; it is made a deviation by subtracting qbar.
//
// One thread per node, epb elements per CTA; the element's FP32 metric terms
// arrive in shared memory by one bulk copy (TMA engine) per element when the
// block is a multiple of 16 bytes (an even number of nodes per direction),
// else by per-thread loads.
#include "internal.cuh"
#include "lowmach.cuh"
#include "physics.cuh"

namespace hs3d {

template <int N>
constexpr int grad_dev_threads()
{
    return ((N + 1) * (N + 1) * (N + 1) > 256) ? (N + 1) * (N + 1) * (N + 1) : 256;
}

// Shared-memory floats per element: metric terms [9][n3], q' [4][n3],
// neighbour-trace deviations [6][4][n2].
template <int N>
constexpr int grad_dev_per_elem()
{
    return 13 * (N + 1) * (N + 1) * (N + 1) + 24 * (N + 1) * (N + 1);
}

template <int n>
__device__ __forceinline__ int gd_face_node(int d, int end, int ta, int tb)
{
    if (d == 0) return end + n * (ta + n * tb);
    if (d == 1) return ta + n * (end + n * tb);
    return ta + n * (tb + n * end);
}

// Velocity and temperature deviations of a node.
__device__ __forceinline__ void grad_dev_vars(const Dev &d, const Anchor &A, float Tb, float rT, float q[4])
{
    q[0] = d.dv1;
    q[1] = d.dv2;
    q[2] = d.dv3;
    q[3] = (d.dp - Tb * d.dr + rT) * __fdividef(1.0f, d.rho);
}

// One tile (epb elements) of the gradient kernel; returns true on the thread
// that initialised its element's bulk-copy barrier.
template <int N>
__device__ __forceinline__ bool grad_dev_tile(const Batch &b, const Ops *__restrict__ ops, long long tile,
                                              unsigned long long *bulk_bar)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    constexpr bool BULK = (n % 2 == 0);
    constexpr int PER = grad_dev_per_elem<N>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *sD = (float *)smem_raw;
    float *sE = sD + ((n * n + 3) & ~3);
    const int epb = blockDim.x / n3;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) sD[t] = ops->Df[t];
    const int le = threadIdx.x / n3, p = threadIdx.x - le * n3;
    const long long ge = tile * epb + le;
    bool valid = ge < b.total_elems;
    const Item *itp = nullptr;
    int e = 0;
    if (valid) {
        itp = &find_item_elem(b, ge);
        e = (int)(ge - itp->elem_begin);
        if (itp->clk && itp->clk->done) valid = false;
    }
    const bool armed = BULK && valid && p == 0;
    float *ja = sE + (size_t)le * PER;
    float *q = ja + 9 * n3;
    float *qn = q + 4 * n3;
    float qin[4];
    if (valid) {
        const Item &it = *itp;
        double uo[5];
        const double *U = it.u + (size_t)e * 5 * n3;
#pragma unroll
        for (int v = 0; v < 5; ++v) uo[v] = U[v * n3 + p];
        // the element's reference state, left by the pass before
        const AnchorRec R = load_anchor(it.anc, e);
        if constexpr (BULK) {
            // one thread initialises, arms and fills the element's barrier; the
            // others poll it only after the block barrier below
            if (p == 0) {
                unsigned long long *bar = bulk_bar + le;
                mbar_init(bar, 1);
                mbar_arrive_expect_tx(bar, 9 * n3 * 4);
                bulk_g2s(ja, it.Jaf + (size_t)e * 9 * n3, 9 * n3 * 4, bar);
            }
        }
        const float gm1 = it.gm1f;
        const Anchor A = R.a;
        const float Tb = A.p * __fdividef(1.0f, A.rho);
        const float rT = fmaf(-Tb, A.rho, A.p);
        constexpr int IT = (6 * n2 + n3 - 1) / n3;
        if (it.face6) {
            // 2 q*_e - q_in from the mortar kernel, full FP32 values -> deviations
#pragma unroll
            for (int k = 0; k < IT; ++k) {
                const int t = p + k * n3;
                if (t < 6 * n2) {
                    const int slot = t / n2, ab = t - slot * n2;
                    const float *src = (const float *)it.qhat6 + ((size_t)slot * it.E + e) * 4 * n2 + ab;
                    qn[(slot * 4 + 0) * n2 + ab] = src[0] - A.v1;
                    qn[(slot * 4 + 1) * n2 + ab] = src[n2] - A.v2;
                    qn[(slot * 4 + 2) * n2 + ab] = src[2 * n2] - A.v3;
                    qn[(slot * 4 + 3) * n2 + ab] = src[3 * n2] - Tb;
                }
            }
        } else {
            // neighbour traces in FP64: all loads first, then the deviations
            const Nbrs nbs = elem_nbrs(e, it.ex, it.ey, it.ez);
            double raw[IT][5];
#pragma unroll
            for (int k = 0; k < IT; ++k) {
                const int t = p + k * n3;
                if (t < 6 * n2) {
                    const int slot = t / n2, ab = t - slot * n2;
                    const int d = slot >> 1, plus = slot & 1;
                    const int pn = gd_face_node<n>(d, plus ? 0 : N, ab % n, ab / n);
                    const double *src = it.u + (size_t)nbr_of_slot(nbs, slot) * 5 * n3 + pn;
#pragma unroll
                    for (int v = 0; v < 5; ++v) raw[k][v] = src[v * n3];
                }
            }
#pragma unroll
            for (int k = 0; k < IT; ++k) {
                const int t = p + k * n3;
                if (t < 6 * n2) {
                    const int slot = t / n2, ab = t - slot * n2;
                    float g4[4];
                    grad_dev_vars(make_dev_rec(raw[k], A, R.Elo, gm1), A, Tb, rT, g4);
#pragma unroll
                    for (int v = 0; v < 4; ++v) qn[(slot * 4 + v) * n2 + ab] = g4[v];
                }
            }
        }
        grad_dev_vars(make_dev_rec(uo, A, R.Elo, gm1), A, Tb, rT, qin);
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v * n3 + p] = qin[v];
        if constexpr (!BULK) {
            const float *JA = it.Jaf + (size_t)e * 9 * n3 + p;
#pragma unroll
            for (int k = 0; k < 9; ++k) ja[k * n3 + p] = JA[k * n3];
        }
    }
    __syncthreads();
    if (!valid) return armed;
    if constexpr (BULK) {
        if (!mbar_wait(bulk_bar + le, 0, kBulkWaitPolls)) {
            // a wait that ran out of polls poisons the gradients and flags the solve
#pragma unroll
            for (int v = 0; v < 4; ++v) qin[v] = NAN;
            if (itp->clk) itp->clk->bad = 2;
        }
    }
    const int ijk[3] = {p % n, (p / n) % n, p / n2};
    float acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int stride = (d == 0) ? 1 : (d == 1) ? n : n2;
        const int base = p - ijk[d] * stride;
        const float *Drow = sD + ijk[d] * n;
#pragma unroll
        for (int m = 0; m < n; ++m) {
            const int pm = base + m * stride;
            const float Dm = Drow[m];
            const float a1 = Dm * ja[(d * 3 + 0) * n3 + pm], a2 = Dm * ja[(d * 3 + 1) * n3 + pm],
                        a3 = Dm * ja[(d * 3 + 2) * n3 + pm];
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float qv = q[v * n3 + pm];
                acc[v * 3 + 0] += a1 * qv;
                acc[v * 3 + 1] += a2 * qv;
                acc[v * 3 + 2] += a3 * qv;
            }
        }
    }
    // surface lifting of the BR1 jumps (q* - q_in) = (q_out - q_in)/2
    const Item &it = *itp;
    const float iw = ops->iw0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const int ta = (d == 0) ? ijk[1] : ijk[0];
        const int tb = (d == 2) ? ijk[1] : ijk[2];
        const int ab = ta + n * tb;
#pragma unroll
        for (int plus = 0; plus < 2; ++plus) {
            if (ijk[d] != (plus ? N : 0)) continue;
            const float sg = plus ? 1.0f : -1.0f;
            const float n1 = sg * ja[(d * 3 + 0) * n3 + p], n2_ = sg * ja[(d * 3 + 1) * n3 + p],
                        n3_ = sg * ja[(d * 3 + 2) * n3 + p];
            const int slot = 2 * d + plus;
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                const float j = 0.5f * (qn[(slot * 4 + v) * n2 + ab] - qin[v]) * iw;
                acc[v * 3 + 0] += j * n1;
                acc[v * 3 + 1] += j * n2_;
                acc[v * 3 + 2] += j * n3_;
            }
        }
    }
    const float ij = it.invJf[(size_t)e * n3 + p];
    float *G = (float *)it.grad + (size_t)e * 12 * n3 + p;
#pragma unroll
    for (int k = 0; k < 12; ++k) G[k * n3] = acc[k] * ij;
    return armed;
}

template <int N>
__device__ __noinline__ bool grad_dev_tile_call(const Batch &b, const Ops *__restrict__ ops, long long tile,
                                                unsigned long long *bulk_bar)
{
    return grad_dev_tile<N>(b, ops, tile, bulk_bar);
}

// The gradient kernel: a CTA per tile, or (PERSIST, Batch::persistent) a
// persistent grid walking the tiles (as k_volume_dev).
template <int N, bool PERSIST>
__global__ void __launch_bounds__(grad_dev_threads<N>()) k_grad_dev(const __grid_constant__ Batch b,
                                                                    const Ops *__restrict__ ops, long long ntiles)
{
    pdl_wait();
    constexpr int n3 = (N + 1) * (N + 1) * (N + 1);
    constexpr bool BULK = ((N + 1) % 2 == 0);
    __shared__ unsigned long long bulk_bar[BULK ? 256 / (n3 < 256 ? n3 : 256) : 1];
    if constexpr (!PERSIST) {
        grad_dev_tile<N>(b, ops, blockIdx.x, bulk_bar);
    } else {
        for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const bool armed = grad_dev_tile_call<N>(b, ops, tile, bulk_bar);
            if (tile + gridDim.x >= ntiles) break;   // (uniform across the CTA)
            __syncthreads();
            if (armed) mbar_inval(bulk_bar + threadIdx.x / n3);
        }
    }
}

template <int N>
static cudaError_t grad_dev_launch(const Batch &b, cudaStream_t s)
{
    constexpr int n = N + 1, n3 = n * n * n;
    if (b.total_elems == 0) return cudaSuccess;
    int epb = elems_per_block_p(N, HS3D_MIXED32, 0);
    if (epb * n3 > grad_dev_threads<N>()) epb = grad_dev_threads<N>() / n3;
    const int threads = epb * n3;
    const size_t smem = sizeof(float) * (((n * n + 3) & ~3) + (size_t)epb * grad_dev_per_elem<N>());
    const unsigned blocks = (unsigned)((b.total_elems + epb - 1) / epb);
    const Ops *ops = device_ops(N);
    if (!ops) return cudaErrorMemoryAllocation;
    cudaError_t e;
    if (b.persistent) {
        const unsigned grid = persistent_grid(k_grad_dev<N, true>, threads, smem, blocks);
        e = launch_pdl(k_grad_dev<N, true>, grid, threads, smem, s, b, ops, (long long)blocks);
    } else {
        e = launch_pdl(k_grad_dev<N, false>, blocks, threads, smem, s, b, ops, (long long)blocks);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int N, bool PERSIST>
static cudaError_t grad_dev_prep_one()
{
    cudaError_t e =
        cudaFuncSetAttribute(k_grad_dev<N, PERSIST>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_grad_dev<N, PERSIST>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

template <int N>
static cudaError_t grad_dev_prep()
{
    cudaError_t e = grad_dev_prep_one<N, false>();
    if (e == cudaSuccess) e = grad_dev_prep_one<N, true>();
    return e;
}

cudaError_t launch_grad_dev(int N, const Batch &b, cudaStream_t s)
{
    switch (N) {
        case 1: return grad_dev_launch<1>(b, s);
        case 2: return grad_dev_launch<2>(b, s);
        case 3: return grad_dev_launch<3>(b, s);
        case 4: return grad_dev_launch<4>(b, s);
        case 5: return grad_dev_launch<5>(b, s);
        case 6: return grad_dev_launch<6>(b, s);
        case 7: return grad_dev_launch<7>(b, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t prepare_grad_dev(int N)
{
    switch (N) {
        case 1: return grad_dev_prep<1>();
        case 2: return grad_dev_prep<2>();
        case 3: return grad_dev_prep<3>();
        case 4: return grad_dev_prep<4>();
        case 5: return grad_dev_prep<5>();
        case 6: return grad_dev_prep<6>();
        case 7: return grad_dev_prep<7>();
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs3d
