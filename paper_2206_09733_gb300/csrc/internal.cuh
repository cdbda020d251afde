// Internal definitions shared by the hs3d CUDA translation units.
//
// Data layout in HBM (all element-major so that one element is one contiguous
// block and every warp load of a node-indexed field is coalesced):
//   u, g, dudt  double [E][5][n3]             conserved variables
//   uf          float  [E][5][n3]              FP32 shadow of u (mixed path): d2f_rn of u
//   Ja          double [E][3(d)][3(c)][n3]     Ja^d_c = J dxi_d/dx_c (curl form)
//   Jaf         float  [E][3(d)][3(c)][n3]     the same, rounded once for the FP32 flux arithmetic
//   invJ        double [E][n3]                 1/J (and an FP32 copy invJf)
//   fn          double [3(d)][E][3(c)][n2]     scaled normal Ja^d of face (d, e) taken
//                                              from element e on its +d face
//   fstar       R      [3(d)][E][5][n2]        numerical flux minus viscous flux, times
//                                              the face scale, for face (d, e)
//   grad        R      [E][12][n3]             BR1 gradients of (v1,v2,v3,T), [v*3 + c]
// Face f = d*E + e is the face between element e and its +d neighbour.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hs3d.h"

namespace hs3d {

constexpr int kMaxN = 7;
constexpr int kMaxn = kMaxN + 1;

__host__ __device__ constexpr bool is_standard(int form) { return form == HS3D_VOL_STANDARD; }

// Per-solve device clock: dt rule inputs and the simulated time.
struct Clock {
    // Bits of the max convective / viscous rates (non-negative doubles), two
    // slots: [0] filled by k_lambda before a single step, [1] filled by the
    // last RK stage of the previous step (or by k_lambda before a run).
    unsigned long long lam[2][2];
    double dt;                  // dt of the current step
    double t;                   // simulated time after the current step
    double t_final;             // > 0: clip dt so that t reaches t_final exactly
    double dt_fixed;            // > 0: use this dt
    long long step;             // steps taken
    long long nsteps;           // > 0: stop after this many steps
    int done;                   // no more steps for this solve
    int bad;                    // 1: non-physical state seen (rho <= 0, p <= 0, NaN);
                                // 2: a device-side wait for a bulk copy ran out of polls
};

// One solve (mesh + state) inside a launch.
struct Item {
    const double *Ja;
    const float *Jaf;       // FP32 copy of Ja (the mixed path rounds Ja to FP32 anyway)
    const float *Jalo;      // Ja - Jaf rounded to FP32: Jaf + Jalo carries Ja to ~2^-48 (mixed path's
                            // float-float mass divergence)
    const double *invJ;
    const float *invJf;     // FP32 copy of 1/J
    const double *fn;
    const float *fnf;       // FP32 copy of fn
    const double *J;       // for diagnostics
    double *u;
    float *uf;              // FP32 shadow of u, or nullptr: read by the kernels that take FP32
                            // traces (mortars, Gauss-Legendre nodes); written by the kernel that
                            // writes u, or by a shadow/priming pass
    double *g;
    double *out;            // residual output (residual mode)
    void *fstar;            // R [3][E][5][n2] (face6: [6][E][5][n2], see below)
    void *grad;             // R [E][12][n3]
    // face6 != 0 (one degree bucket of a mesh with per-element degrees): the
    // element's six face fluxes are its own blocks fstar[slot][e], slot 2d
    // the -d face and 2d+1 the +d face, each already projected onto this
    // element's face; the BR1 gradient kernel reads, instead of the
    // neighbour's trace, qhat6[slot][e][4][n2] = 2 q*_e - q_in (q*_e the
    // mortar interface value projected onto this face), so that its lifting
    // (q_out - q_in)/2 = q*_e - q_in is unchanged
    const void *qhat6;
    int face6;
    void *anc;              // mixed path: one reference-state record per element (AnchorRec), or nullptr
    Clock *clk;
    int ex, ey, ez;
    int E;
    long long elem_begin;   // first element of this item in the launch
    long long face_begin;   // first face of this item in the launch (3E faces per item)
    double gamma, mu, kappa, cfl;
    double kc, kv;          // dt-rule constants of the node family (convective, viscous)
    int gauss;              // Gauss-Legendre solution nodes
    double gm1, hg;                          // gamma - 1, 1/(2(gamma - 1))
    float gammaf, gm1f, hgf, muf, kappaf;    // the same constants rounded once for the FP32 path
    float hglof;            // 1/(2 gm1f) - hgf: hgf + hglof is the reciprocal of the FP32 (gamma-1) to ~2^-48
    double igm1f;           // 1/gm1f in FP64
};

// Physical constants of an item in the arithmetic type R (no per-thread
// FP64 arithmetic or conversion in the FP32 path).
template <typename R>
struct Phys {
    R gamma, gm1, hg, mu, kappa;
};
template <typename R>
__device__ __forceinline__ Phys<R> phys_of(const Item &it);
template <>
__device__ __forceinline__ Phys<double> phys_of<double>(const Item &it)
{
    return Phys<double>{it.gamma, it.gm1, it.hg, it.mu, it.kappa};
}
template <>
__device__ __forceinline__ Phys<float> phys_of<float>(const Item &it)
{
    return Phys<float>{it.gammaf, it.gm1f, it.hgf, it.muf, it.kappaf};
}

struct Batch {
    Item single;            // used when nitems == 1
    const Item *items;      // device array when nitems > 1
    int nitems;
    long long total_elems;
    long long total_faces;
    double dt_fixed;        // > 0: every item steps with this dt
    int gauss;              // every item on Gauss-Legendre nodes (items of a batch share the node family)
    // work table (nitems > 1, optional): item of every element of the batch, items[elem_item[ge]],
    // instead of a binary search over the items' first elements
    const int *elem_item;
    // 1: the element, gradient and face kernels run a persistent grid (as many CTAs as fit at
    // once) whose CTAs walk the tiles with a stride of the grid size
    int persistent;
    // 1: every item takes its face fluxes from the mortar kernels (Item::face6, meshes with
    // per-element degrees), 0: none does; the element kernel has an instantiation for each
    int mortar;
};

// 1-D operators on the Gauss-Lobatto nodes for one N.
// 1-D operators of one degree N on the solution nodes (Gauss-Lobatto, or
// Gauss-Legendre with the boundary interpolation written out).
struct Ops {
    double D[kMaxn * kMaxn];   // D[i*n + m] = l_m'(xi_i)
    double w[kMaxn];
    double xi[kMaxn];
    float Df[kMaxn * kMaxn];
    float Dlo[kMaxn * kMaxn];  // D - Df rounded to FP32 (float-float contractions)
    double iw0;                // 1/w_0 = 1/w_N (Gauss-Lobatto surface lifting factor)
    float iw0f;
    int gauss;                 // 1: Gauss-Legendre nodes
    double lb[kMaxn], rb[kMaxn];     // l_j(-1), l_j(+1)
    double lbw[kMaxn], rbw[kMaxn];   // l_j(-1)/w_j, l_j(+1)/w_j
    float lbf[kMaxn], rbf[kMaxn], lbwf[kMaxn], rbwf[kMaxn];
    double IL[kMaxn * kMaxn];  // IL[t*n + s]: Gauss-Lobatto basis function s at solution node t
};

template <typename R>
__device__ __forceinline__ R ops_D(const Ops *o, int k);
template <>
__device__ __forceinline__ double ops_D<double>(const Ops *o, int k) { return o->D[k]; }
template <>
__device__ __forceinline__ float ops_D<float>(const Ops *o, int k) { return o->Df[k]; }
template <typename R>
__device__ __forceinline__ R ops_iw0(const Ops *o);
template <>
__device__ __forceinline__ double ops_iw0<double>(const Ops *o) { return o->iw0; }
template <>
__device__ __forceinline__ float ops_iw0<float>(const Ops *o) { return o->iw0f; }

template <typename R>
__device__ __forceinline__ R ops_lb(const Ops *o, int j) { if constexpr (sizeof(R) == 8) return o->lb[j]; else return o->lbf[j]; }
template <typename R>
__device__ __forceinline__ R ops_rb(const Ops *o, int j) { if constexpr (sizeof(R) == 8) return o->rb[j]; else return o->rbf[j]; }
template <typename R>
__device__ __forceinline__ R ops_lbw(const Ops *o, int j) { if constexpr (sizeof(R) == 8) return o->lbw[j]; else return o->lbwf[j]; }
template <typename R>
__device__ __forceinline__ R ops_rbw(const Ops *o, int j) { if constexpr (sizeof(R) == 8) return o->rbw[j]; else return o->rbwf[j]; }

// Host side.  nodes: HS3D_NODES_LOBATTO or HS3D_NODES_GAUSS.
const Ops &host_ops(int N, int nodes = HS3D_NODES_LOBATTO);   // computed once per (N, nodes)
const Ops *device_ops(int N, int nodes = HS3D_NODES_LOBATTO); // device copy, once per (device, N, nodes)

// Locate the item holding global element ge (binary search on elem_begin).
__device__ __forceinline__ const Item &find_item_elem(const Batch &b, long long ge)
{
    if (b.nitems == 1) return b.single;
    if (b.elem_item) return b.items[b.elem_item[ge]];
    int lo = 0, hi = b.nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (b.items[mid].elem_begin <= ge) lo = mid; else hi = mid - 1;
    }
    return b.items[lo];
}

__device__ __forceinline__ const Item &find_item_face(const Batch &b, long long gf)
{
    if (b.nitems == 1) return b.single;
    if (b.elem_item) return b.items[b.elem_item[gf / 3]];   // (face_begin = 3 elem_begin)
    int lo = 0, hi = b.nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (b.items[mid].face_begin <= gf) lo = mid; else hi = mid - 1;
    }
    return b.items[lo];
}

// Max-reduce non-negative rates over the lanes of a warp that share the same
// clock (threads map to consecutive nodes and an item's elements are
// consecutive, so each group is a contiguous run of lanes) and add them to
// that clock slot with one atomic per group.  All 32 lanes must call this.
__device__ __forceinline__ void warp_max_to_clock(unsigned long long *dst_c, unsigned long long *dst_v, double lc,
                                                  double lv, bool active)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    unsigned long long key = active ? (unsigned long long)dst_c : 0ull;
    unsigned peers = __match_any_sync(full, key);
    const int first = __ffs(peers) - 1;
    const int last = 31 - __clz(peers);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        double oc = __shfl_down_sync(full, lc, off);
        double ov = __shfl_down_sync(full, lv, off);
        if (lane + off <= last) {
            lc = fmax(lc, oc);
            lv = fmax(lv, ov);
        }
    }
    if (active && lane == first) {
        atomicMax(dst_c, (unsigned long long)__double_as_longlong(lc));
        if (dst_v) atomicMax(dst_v, (unsigned long long)__double_as_longlong(lv));
    }
}

// Programmatic dependent launch: a kernel launched by launch_pdl may be
// scheduled while the kernel before it in the stream drains (its CTAs take
// the SMs that the other's last CTAs free); it calls pdl_wait() before it
// reads or writes anything, which returns once that kernel has completed
// and its memory is visible.  (A no-op for a kernel launched without the
// attribute.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// CTAs of a persistent grid: as many as are resident at once (occupancy x
// SMs), at most `tiles`.
template <typename K>
inline unsigned persistent_grid(K kernel, int threads, size_t smem, unsigned tiles)
{
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) {
        cudaGetLastError();
        return tiles;
    }
    const unsigned long long cap = (unsigned long long)per * sms;
    return tiles < cap ? tiles : (unsigned)cap;
}

// Asynchronous global->shared copies (cp.async, sm_80+): the copies are
// issued without staging through registers and waited for once.
__device__ __forceinline__ void cp_async_16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Ask L2 to fetch the cache lines of [p, p + bytes) ahead of their use; each
// of `nthreads` threads (index tid) prefetches every nthreads-th line.
__device__ __forceinline__ void prefetch_l2_block(const void *p, size_t bytes, int tid, int nthreads)
{
    const uintptr_t a0 = (uintptr_t)p & ~(uintptr_t)127, a1 = ((uintptr_t)p + bytes - 1) & ~(uintptr_t)127;
    const int lines = (int)((a1 - a0) >> 7) + 1;
    for (int t = tid; t < lines; t += nthreads)
        asm volatile("prefetch.global.L2 [%0];\n" ::"l"((const void *)(a0 + ((uintptr_t)t << 7))));
}

// Bulk asynchronous copies on the TMA engine (cp.async.bulk, sm_90+): one
// thread moves a whole contiguous block (16-byte aligned addresses, size a
// multiple of 16 bytes); completion is counted in bytes on an mbarrier in
// shared memory (phase 0 completes once the arrival and all announced
// bytes have landed).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async (TMA) proxy
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Wait for phase `parity` of the barrier, at most `limit` polls (each poll
// may suspend the thread for a hardware-defined interval).  Returns false
// when the limit ran out.
// Invalidate a barrier whose copies have all completed, so that the same
// shared-memory word can be initialised again (the next tile of a
// persistent CTA).
__device__ __forceinline__ void mbar_inval(unsigned long long *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit)
{
    const unsigned a = smem_u32(bar);
    for (long long i = 0; i < limit; ++i) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// Poll limit of the element kernels' bulk-copy waits: far beyond any copy's
// duration (the copies are a few kilobytes), yet bounded.
constexpr long long kBulkWaitPolls = 1LL << 22;

// Copy `count` contiguous values of type R from global to shared memory with
// the widest cp.async both addresses allow (16 bytes when the byte count and
// both addresses are multiples of 16), spread over `nthreads` threads.
template <typename R>
__device__ __forceinline__ void cp_async_block(R *dst, const R *src, int count, int tid, int nthreads)
{
    const int bytes = count * (int)sizeof(R);
    if ((bytes & 15) == 0 && (((uintptr_t)dst | (uintptr_t)src) & 15) == 0) {
        const int chunks = bytes >> 4;
        for (int c = tid; c < chunks; c += nthreads)
            cp_async_16((char *)dst + 16 * c, (const char *)src + 16 * c);
    } else {
        for (int c = tid; c < count; c += nthreads) {
            if (sizeof(R) == 8) cp_async_8(dst + c, src + c);
            else cp_async_4(dst + c, src + c);
        }
    }
}

// Element neighbour across direction d (+1 side), periodic.  Element e of
// the ex x ey x ez box has coordinates a = e mod ex, b = (e / ex) mod ey,
// c = e / (ex ey): two integer divisions.
__device__ __forceinline__ int nbr_plus(int e, int d, int ex, int ey, int ez)
{
    const int q = e / ex, a = e - q * ex;
    const int c = q / ey, b = q - c * ey;
    if (d == 0) return (a + 1 == ex) ? e - (ex - 1) : e + 1;
    if (d == 1) return (b + 1 == ey) ? e - (ey - 1) * ex : e + ex;
    return (c + 1 == ez) ? e - (ez - 1) * ex * ey : e + ex * ey;
}

__device__ __forceinline__ int nbr_minus(int e, int d, int ex, int ey, int ez)
{
    const int q = e / ex, a = e - q * ex;
    const int c = q / ey, b = q - c * ey;
    if (d == 0) return (a == 0) ? e + (ex - 1) : e - 1;
    if (d == 1) return (b == 0) ? e + (ey - 1) * ex : e - ex;
    return (c == 0) ? e + (ez - 1) * ex * ey : e - ex * ey;
}

// All six neighbours of element e: m[d] across its -d face, p[d] across its
// +d face (one pair of divisions for the six).
struct Nbrs {
    int m[3], p[3];
};
__device__ __forceinline__ Nbrs elem_nbrs(int e, int ex, int ey, int ez)
{
    const int q = e / ex, a = e - q * ex;
    const int c = q / ey, b = q - c * ey;
    const int sz = ex * ey;
    Nbrs r;
    r.m[0] = (a == 0) ? e + (ex - 1) : e - 1;
    r.p[0] = (a + 1 == ex) ? e - (ex - 1) : e + 1;
    r.m[1] = (b == 0) ? e + (ey - 1) * ex : e - ex;
    r.p[1] = (b + 1 == ey) ? e - (ey - 1) * ex : e + ex;
    r.m[2] = (c == 0) ? e + (ez - 1) * sz : e - sz;
    r.p[2] = (c + 1 == ez) ? e - (ez - 1) * sz : e + sz;
    return r;
}

// Neighbour across face slot s = 2d (the -d face) or 2d + 1 (the +d face),
// for a run-time slot (a select chain, so that Nbrs stays in registers).
__device__ __forceinline__ int nbr_of_slot(const Nbrs &r, int s)
{
    return s == 0 ? r.m[0] : s == 1 ? r.p[0] : s == 2 ? r.m[1] : s == 3 ? r.p[1] : s == 4 ? r.m[2] : r.p[2];
}

// Launch helpers implemented in the .cu files (return cudaError_t of the launch).
cudaError_t launch_geometry(int N, int nodes, const double *node_xyz_dev, int ex, int ey, int ez, const double *lo,
                            const double *hi, double amp, double *X, double *Ja, float *Jaf, double *J, double *invJ,
                            float *invJf, double *fn, float *fnf, cudaStream_t s);
cudaError_t launch_init_state(int N, int E, const double *X, const hs3d_ic &ic, const double *lo, const double *hi,
                              double *u, cudaStream_t s);
cudaError_t launch_lambda(int N, int prec, int physics, const Batch &b, int slot, cudaStream_t s);
// Write the FP32 shadow uf of every item's state (mixed path, when no dt pass does it).
cudaError_t launch_shadow(int N, const Batch &b, cudaStream_t s);
// mode 0: advance every item's clock using lambda slot `slot`; mode 2: dt value of b.single into b.single.out
cudaError_t launch_dt_finalize(int N, const Batch &b, int mode, int slot, cudaStream_t s);
cudaError_t launch_grad(int N, int prec, const Batch &b, cudaStream_t s);
cudaError_t launch_face(int N, int prec, int physics, int flux, const Batch &b, cudaStream_t s);
// stage -1: residual into out; 0..rk_stages(scheme)-1: RK stage of `scheme`; lam_slot >= 0 (last
// stage only): also accumulate the dt maxima of the updated state into that clock slot
cudaError_t launch_volume(int N, int prec, int physics, int form, int scheme, const Batch &b, int stage, int lam_slot,
                          cudaStream_t s);
// Gauss-Legendre node kernels (gauss.cu); launch_face/grad/volume route batches with b.gauss to them.
cudaError_t launch_face_gauss(int N, int prec, int physics, int flux, const Batch &b, cudaStream_t s);
cudaError_t launch_grad_gauss(int N, int prec, const Batch &b, cudaStream_t s);
cudaError_t launch_volume_gauss(int N, int prec, int physics, const Batch &b, int stage, double rkA, double rkB,
                                int lam_slot, cudaStream_t s);
cudaError_t prepare_gauss(int N);
// Mixed path on Gauss-Lobatto nodes: FP32 flux arithmetic on deviations from
// a per-element reference state (face_dev.cu, grad_dev.cu, volume_dev.cuh).
cudaError_t launch_face_dev(int N, int physics, int flux, const Batch &b, cudaStream_t s);
cudaError_t launch_grad_dev(int N, const Batch &b, cudaStream_t s);
cudaError_t prepare_grad_dev(int N);
// Ja - Jaf rounded to FP32, one thread per value.
cudaError_t launch_metric_lo(const double *Ja, const float *Jaf, float *Jalo, long long count, cudaStream_t s);
// Low-storage RK schemes (HS3D_TIME_*): stage count and the stage's (A_k, B_k).
int rk_stages(int scheme);
void rk_coeffs(int scheme, int k, double *A, double *B);
cudaError_t launch_diagnostics(int N, const Item &it, const double *dudt, double *partials, int nblocks, double *out,
                               cudaStream_t s);
int diagnostics_blocks(int N, int E);

// One-time per-N set-up that must not happen inside a stream capture
// (shared-memory attributes, operator tables).
cudaError_t prepare_kernels(int N);
cudaError_t prepare_volume(int N);
cudaError_t prepare_grad(int N);

// Elements per block for the element kernels (threads = epb * n^3), per
// (N, precision 0 = FP64 / 1 = mixed, kernel: 0 = BR1 gradient, 1 = volume);
// the autotuner's choice if one was made, else 256 threads' worth.
int elems_per_block_p(int N, int prec, int which);
int tuned_elems_per_block(int N, int prec, int which);   // 0 if untuned
void set_elems_per_block_p(int N, int prec, int which, int epb);
void tune_cache_load();

}  // namespace hs3d
