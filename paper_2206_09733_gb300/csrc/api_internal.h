// Host-side internals shared by api.cu and server.cu.
#pragma once

#include <stdarg.h>

#include <mutex>

#include "internal.cuh"

struct hs3d_mesh {
    int ex = 0, ey = 0, ez = 0, N = 0, n = 0, n2 = 0, n3 = 0;
    int E = 0;
    int nodes = HS3D_NODES_LOBATTO;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, amp = 0.0;
    int device = 0;
    double *X = nullptr, *Ja = nullptr, *J = nullptr, *invJ = nullptr, *fn = nullptr;
    float *Jaf = nullptr, *invJf = nullptr;
    float *Jalo = nullptr;          // Ja - Jaf in FP32 (the mixed path's float-float mass divergence)
    float *uf = nullptr;            // FP32 shadow of the state being stepped, only where FP32 traces are
                                    // read (Gauss-Legendre nodes; the degree buckets of a p-mesh)
    float *fnf = nullptr;
    void *anc = nullptr;            // mixed path: reference state of each element (112 bytes each)
    void *fstar = nullptr;          // scratch, sized for FP64
    void *grad = nullptr;           // scratch, sized for FP64
    hs3d::Clock *clk = nullptr;
    double *diag_partials = nullptr;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;  // private stream for set-up and graph capture
    // graph cache of hs3d_rk3_run: the two most recently used (cfg, u, g, dt)
    struct GraphSlot {
        cudaGraphExec_t exec = nullptr;
        const double *u = nullptr;
        const double *g = nullptr;
        double dt = 0.0;
        hs3d_solver_cfg cfg{};
        unsigned long long used = 0;
    };
    std::mutex mu;
    GraphSlot gslot[2];
    unsigned long long gtick = 0;
    // continuation record (under mu): the state and configuration the last
    // hs3d_rk3_step / hs3d_rk3_run advanced; clock slot 1 then holds that
    // state's dt maxima and uf its FP32 shadow, so hs3d_rk3_run with dt < 0
    // may skip the priming pass.  Cleared by anything that rewrites either.
    const double *cont_u = nullptr;
    hs3d_solver_cfg cont_cfg{};
};

namespace hs3d {

bool same_cfg(const hs3d_solver_cfg &a, const hs3d_solver_cfg &b);
void cont_set(const hs3d_mesh *m, const double *u, const hs3d_solver_cfg *c);
void cont_forget(const hs3d_mesh *m, const double *u_written);   // nullptr: forget unconditionally

hs3d_status fail(hs3d_status st, const char *fmt, ...);
hs3d_status cuda_fail(cudaError_t e, const char *what);
hs3d_status validate_cfg(const hs3d_solver_cfg *c);
hs3d_status check_ptr(const void *p, const char *name);   // non-NULL and 16-byte aligned
hs3d_status validate_desc(const hs3d_mesh_desc *d);
hs3d_status mesh_build(const hs3d_mesh_desc *desc, hs3d_mesh **out);
void mesh_free(hs3d_mesh *m);
size_t mesh_bytes(int N, long long E, int nodes);
hs3d_status check_mesh_cfg(const hs3d_mesh *m, const hs3d_solver_cfg *c);
Item make_item(const hs3d_mesh *m, const hs3d_solver_cfg *c, const double *u, double *g, double *out);
Batch single_batch(const Item &it);
cudaError_t enqueue_stage(int N, const hs3d_solver_cfg *c, const Batch &b, int stage, int lam_slot, cudaStream_t s);
cudaError_t enqueue_rk3_step(int N, const hs3d_solver_cfg *c, Batch b, double dt, int fresh_lambda, cudaStream_t s);
cudaError_t prime_lambda(int N, const hs3d_solver_cfg *c, const Batch &b, Clock *clk, cudaStream_t s);

}  // namespace hs3d
