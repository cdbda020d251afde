// Internal definitions shared by the hs3d CUDA translation units.
//
// Data layout in HBM (all element-major so that one element is one contiguous
// block and every warp load of a node-indexed field is coalesced):
//   u, g, dudt  double [E][5][n3]             conserved variables
//   Ja          double [E][3(d)][3(c)][n3]     Ja^d_c = J dxi_d/dx_c (curl form)
//   invJ        double [E][n3]                 1/J
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

// Per-solve device clock: dt rule inputs and the simulated time.
struct Clock {
    unsigned long long lam_c;   // bits of max convective rate (non-negative double)
    unsigned long long lam_v;   // bits of max viscous rate
    double dt;                  // dt of the current step
    double t;                   // simulated time after the current step
    double t_final;             // > 0: clip dt so that t reaches t_final exactly
    double dt_fixed;            // > 0: use this dt
    long long step;             // steps taken
    long long nsteps;           // > 0: stop after this many steps
    int done;                   // no more steps for this solve
    int bad;                    // non-physical state seen (rho <= 0, p <= 0, NaN)
};

// One solve (mesh + state) inside a launch.
struct Item {
    const double *Ja;
    const double *invJ;
    const double *fn;
    const double *J;       // for diagnostics
    double *u;
    double *g;
    double *out;            // residual output (residual mode)
    void *fstar;            // R [3][E][5][n2]
    void *grad;             // R [E][12][n3]
    Clock *clk;
    int ex, ey, ez;
    int E;
    long long elem_begin;   // first element of this item in the launch
    long long face_begin;   // first face of this item in the launch (3E faces per item)
    double gamma, mu, kappa, cfl;
};

struct Batch {
    Item single;            // used when nitems == 1
    const Item *items;      // device array when nitems > 1
    int nitems;
    long long total_elems;
    long long total_faces;
    double dt_fixed;        // > 0: every item steps with this dt
};

// 1-D operators on the Gauss-Lobatto nodes for one N.
struct Ops {
    double D[kMaxn * kMaxn];   // D[i*n + m] = l_m'(xi_i)
    double w[kMaxn];
    double xi[kMaxn];
    float Df[kMaxn * kMaxn];
};

// Host side.
const Ops &host_ops(int N);        // computed once per N
const Ops *device_ops(int N);      // device copy (cudaMalloc'd once per device and N)

// Locate the item holding global element ge (binary search on elem_begin).
__device__ __forceinline__ const Item &find_item_elem(const Batch &b, long long ge)
{
    if (b.nitems == 1) return b.single;
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
    int lo = 0, hi = b.nitems - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (b.items[mid].face_begin <= gf) lo = mid; else hi = mid - 1;
    }
    return b.items[lo];
}

// Element neighbour across direction d (+1 side), periodic.
__device__ __forceinline__ int nbr_plus(int e, int d, int ex, int ey, int ez)
{
    int a = e % ex, b = (e / ex) % ey, c = e / (ex * ey);
    if (d == 0) a = (a + 1 == ex) ? 0 : a + 1;
    else if (d == 1) b = (b + 1 == ey) ? 0 : b + 1;
    else c = (c + 1 == ez) ? 0 : c + 1;
    return a + ex * (b + ey * c);
}

__device__ __forceinline__ int nbr_minus(int e, int d, int ex, int ey, int ez)
{
    int a = e % ex, b = (e / ex) % ey, c = e / (ex * ey);
    if (d == 0) a = (a == 0) ? ex - 1 : a - 1;
    else if (d == 1) b = (b == 0) ? ey - 1 : b - 1;
    else c = (c == 0) ? ez - 1 : c - 1;
    return a + ex * (b + ey * c);
}

// Launch helpers implemented in the .cu files (return cudaError_t of the launch).
cudaError_t launch_geometry(int N, const double *node_xyz_dev, int ex, int ey, int ez, const double *lo,
                            const double *hi, double amp, double *X, double *Ja, double *J, double *invJ,
                            double *fn, cudaStream_t s);
cudaError_t launch_init_state(int N, int E, const double *X, const hs3d_ic &ic, const double *lo, const double *hi,
                              double *u, cudaStream_t s);
cudaError_t launch_lambda(int N, int physics, const Batch &b, cudaStream_t s);
cudaError_t launch_dt_finalize(int N, const Batch &b, int mode, cudaStream_t s);
cudaError_t launch_grad(int N, int prec, const Batch &b, cudaStream_t s);
cudaError_t launch_face(int N, int prec, int physics, int flux, const Batch &b, cudaStream_t s);
cudaError_t launch_volume(int N, int prec, int physics, int form, const Batch &b, int stage, cudaStream_t s);
cudaError_t launch_diagnostics(int N, const Item &it, const double *dudt, double *partials, int nblocks, double *out,
                               cudaStream_t s);
int diagnostics_blocks(int N, int E);

// One-time per-N set-up that must not happen inside a stream capture
// (shared-memory attributes, operator tables).
cudaError_t prepare_kernels(int N);
cudaError_t prepare_volume(int N);
cudaError_t prepare_grad(int N);

// Elements per block for the element kernels (threads = epb * n^3);
// which = 0: BR1 gradient kernel, 1: volume kernel.
int elems_per_block(int N, int which);
void set_elems_per_block(int N, int which, int epb);

}  // namespace hs3d
