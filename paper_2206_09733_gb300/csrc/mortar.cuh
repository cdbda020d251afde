// Mortar coupling of elements of different degree: shared declarations of
// mortar.cu (kernels) and pmesh.cu (host API).
#pragma once

#include "internal.cuh"

namespace hs3d {

// Interpolation to the mortar and L2 projection back, for every pair of
// degrees Ns <= Nm (Gauss-Lobatto points):
//   Pi[Ns][Nm][a (Nm+1) ... ]: row a (mortar point), column i (face point): l_i^(Ns)(xi_a^(Nm))
//   P [Ns][Nm][i (Nm+1) + j]:  row i (face point), column j (mortar point)
// with FP32 copies for the mixed path.
struct MortarOps {
    double Pi[kMaxn][kMaxn][kMaxn * kMaxn];
    double P[kMaxn][kMaxn][kMaxn * kMaxn];
    float Pif[kMaxn][kMaxn][kMaxn * kMaxn];
    float Pf[kMaxn][kMaxn][kMaxn * kMaxn];
};

const MortarOps &host_mortar_ops();
const MortarOps *device_mortar_ops();

// One face of a mesh with per-element degrees: the +d face of an element
// (bucket bL, index lL within it) shared with its +d neighbour (bucket bR,
// index lR).  The face table is sorted into groups by mortar degree
// max(N_L, N_R) (on a mesh of one degree: the conforming groups, see
// launch_mortar).
struct MortarFace {
    int bL, lL, bR, lR, d;
};

// One degree bucket as the face kernel sees it.
struct MortarSide {
    int N, E;
    long long base;        // offset of the bucket's first element in the caller's state (doubles)
    const float *uf;       // FP32 shadow of the bucket's state [E][5][n3] (mixed path)
    const void *grad;      // BR1 gradients [E][12][n3] (R)
    const double *Ja;      // [E][9][n3]
    const float *Jaf;
    void *fstar6;          // face fluxes [6][E][5][n2] (R)
    void *qhat6;           // BR1 interface values [6][E][4][n2] (R)
};

template <typename R>
struct MortarPhys {
    R gamma, gm1, hg, mu, kappa;
};

// mode 0: BR1 interface values; mode 1: face fluxes.  group_begin (HOST,
// 2 kMaxn + 1 ints): faces of mortar degree NM taken by k_mortar are
// faces[group_begin[NM] .. group_begin[NM + 1]); faces between two elements
// of degree N taken by the barrier-free conforming kernel are
// faces[group_begin[kMaxn + N] .. group_begin[kMaxn + N + 1]).  only >= 0:
// launch that group alone (else every non-empty group, in order).
cudaError_t launch_mortar(int prec, int physics, int mode, int flux, const MortarFace *faces, const int *group_begin,
                          int only, const MortarSide *sides, const double *u, const MortarPhys<double> &P,
                          cudaStream_t s);
cudaError_t launch_pdt_finalize(Clock *const *clks, const int *nb_n, int nb, double cfl, double kc, double kv,
                                int slot, double dt_fixed, cudaStream_t s);

}  // namespace hs3d
