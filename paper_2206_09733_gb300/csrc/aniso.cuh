// Meshes whose elements carry their own degree in each reference direction
// (Sec. 3.6: P_x, P_y, P_z per element, anisotropic p-adaptation), coupled by
// mortars whose degree is chosen per tangential direction: shared
// declarations of aniso.cu (kernels, tables) and pmesh.cu (host API).
#pragma once

#include <stdint.h>

#include <vector>

#include "hs3d.h"
#include "internal.cuh"

namespace hs3d {

// One face of the mesh: the +d face of element eL, shared with its +d
// neighbour eR (its -d face).
struct AFace {
    int eL, eR, d;
};

// Derivative matrices and end weights of every Gauss-Lobatto degree 1..kMaxN
// (device copy): D[N][i*(N+1) + m], iw0[N] = 1/w_0.
struct AOps {
    double D[kMaxn][kMaxn * kMaxn];
    double iw0[kMaxn];
};

// Elements are launched in classes of node count: class k holds the
// elements with kAnisoClass[k-1] < n_x n_y n_z <= kAnisoClass[k], one CTA of
// kAnisoClass[k] threads each (thread t owns node t).
constexpr int kAnisoClasses = 5;
constexpr int kAnisoClass[kAnisoClasses] = {32, 64, 128, 256, 512};

struct AnisoMesh {
    int ex = 0, ey = 0, ez = 0, E = 0, Pmin = 0, Pmax = 0, Ngeo = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, amp = 0.0;
    std::vector<int> P3;              // [3E] degree of element e along d at 3e + d
    std::vector<int64_t> off;         // [E+1] state offsets (doubles): element e's [5][nodes] at off[e]
    std::vector<int64_t> noff;        // [E+1] node offsets
    std::vector<int64_t> fnoff;       // [6E+1] face-node offsets, face slot s = 2d (-d) or 2d+1 (+d)
    int cls_begin[kAnisoClasses + 1] = {0};
    // device
    int *dP3 = nullptr;
    long long *dnoff = nullptr, *doff = nullptr, *dfnoff = nullptr;
    int *cls_elems = nullptr;         // element ids, class by class
    AFace *faces = nullptr;           // [3E]
    double *X = nullptr, *Ja = nullptr, *J = nullptr, *invJ = nullptr;
    double *grad = nullptr;           // [12 nodes]
    double *fstar = nullptr;          // [5 face nodes]: mortar flux projected onto each element face
    double *qhat = nullptr;           // [4 face nodes]: BR1 interface value on each element face
    double *diag_part = nullptr;      // [E][7]
    Clock *clk = nullptr;
    Clock **clkp = nullptr;           // device table of the one clock (the p-mesh dt finalize reads it)
    int *one = nullptr;               // device int 1 (that finalize's n)
    size_t bytes = 0;
};

hs3d_status aniso_build(const hs3d_mesh_desc *desc, const int *degree3, AnisoMesh **out);
void aniso_free(AnisoMesh *a);
// one residual (stage < 0, into out) or RK stage (g, the clock's dt); lam_slot >= 0: the stage
// also reduces the updated state's dt maxima into that clock slot
cudaError_t aniso_stage(const AnisoMesh *a, const hs3d_solver_cfg *c, double *u, double *g, double *out, int stage,
                        int lam_slot, cudaStream_t s);
// one RK step: dt from clock slot 0 after a fresh dt pass (fresh) or slot 1, or dt > 0 as given
cudaError_t aniso_step(const AnisoMesh *a, const hs3d_solver_cfg *c, double *u, double *g, double dt, bool fresh,
                       cudaStream_t s);
cudaError_t aniso_init_state(const AnisoMesh *a, const hs3d_ic &ic, double *u, cudaStream_t s);
cudaError_t aniso_diagnostics(const AnisoMesh *a, const hs3d_solver_cfg *c, const double *u, const double *dudt,
                              double *out, cudaStream_t s);

}  // namespace hs3d
