// Autotuner for the element kernels' launch shape.
//
// The BR1-gradient and element (volume) kernels run one thread per node with
// `epb` elements per CTA.  hs3d_autotune times every admissible epb (the CTA
// must stay within the kernel's thread bound and shared-memory limit) for
// the given mesh and configuration on scratch copies of a smooth state (the
// element kernel as a middle RK stage, with its own clock and a tiny dt, so
// that the timed launches move the bytes of a real step), and keeps the
// fastest per (N, precision, kernel).  Choices
// persist across processes in a small JSON file when HS3D_TUNE_CACHE names
// one: it is read on first use and rewritten after each tuning.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <string>

#include "api_internal.h"

namespace hs3d {

static std::mutex g_tune_mu;
static bool g_cache_loaded = false;

static std::string cache_path()
{
    const char *p = getenv("HS3D_TUNE_CACHE");
    return p ? std::string(p) : std::string();
}

// Cache format: {"N<N>_p<prec>_k<which>": epb, ...}
static void load_cache_locked()
{
    if (g_cache_loaded) return;
    g_cache_loaded = true;
    std::string path = cache_path();
    if (path.empty()) return;
    FILE *f = fopen(path.c_str(), "r");
    if (!f) return;
    char buf[8192];
    size_t len = fread(buf, 1, sizeof buf - 1, f);
    fclose(f);
    buf[len] = 0;
    const char *s = buf;
    while ((s = strchr(s, '"')) != nullptr) {
        int N = 0, prec = 0, which = 0, epb = 0;
        if (sscanf(s, "\"N%d_p%d_k%d\": %d", &N, &prec, &which, &epb) == 4 && N >= 1 && N <= kMaxN && epb >= 1 &&
            epb <= 64 && prec >= 0 && prec <= 2 && (which == 0 || which == 1))
            set_elems_per_block_p(N, prec, which, epb);
        s = strchr(s + 1, '"');
        if (s) ++s;
    }
}

static void save_cache_locked()
{
    std::string path = cache_path();
    if (path.empty()) return;
    std::string tmp = path + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{");
    bool first = true;
    for (int N = 1; N <= kMaxN; ++N)
        for (int prec = 0; prec < 2; ++prec)
            for (int which = 0; which < 2; ++which) {
                int v = tuned_elems_per_block(N, prec, which);
                if (v <= 0) continue;
                fprintf(f, "%s\"N%d_p%d_k%d\": %d", first ? "" : ", ", N, prec, which, v);
                first = false;
            }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), path.c_str());
}

void tune_cache_load()
{
    std::lock_guard<std::mutex> g(g_tune_mu);
    load_cache_locked();
}

// Time `reps` launches of the gradient kernel, or of the element kernel as
// RK stage 1 (reads and writes u and g), with a given epb.
static float time_kernels(hs3d_mesh *m, const hs3d_solver_cfg *c, const Batch &b, int which, int reps, cudaStream_t s,
                          cudaError_t &err)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    err = cudaSuccess;
    // one untimed launch (also surfaces launch errors for this shape)
    if (which == 0) err = launch_grad(m->N, c->precision, b, s);
    else err = launch_volume(m->N, c->precision, c->physics, c->volume_form, c->time_scheme, b, 1, -1, s);
    if (err == cudaSuccess) err = cudaEventRecord(e0, s);
    for (int r = 0; r < reps && err == cudaSuccess; ++r) {
        if (which == 0) err = launch_grad(m->N, c->precision, b, s);
        else err = launch_volume(m->N, c->precision, c->physics, c->volume_form, c->time_scheme, b, 1, -1, s);
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, s);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / reps;
}

}  // namespace hs3d

using namespace hs3d;

extern "C" hs3d_status hs3d_autotune(const hs3d_mesh *mc, const hs3d_solver_cfg *c, int *choice_out, void *stream)
{
    hs3d_mesh *m = const_cast<hs3d_mesh *>(mc);
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK) st = check_mesh_cfg(m, c);
    if (st != HS3D_OK) return st;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_cache_locked();
    cudaStream_t s = (cudaStream_t)stream;
    size_t sz = sizeof(double) * (size_t)m->E * 5 * m->n3;
    double *u = nullptr, *g = nullptr;
    Clock *clk = nullptr;
    cudaError_t e = cudaMalloc(&u, sz);
    if (e == cudaSuccess) e = cudaMalloc(&g, sz);
    if (e == cudaSuccess) e = cudaMalloc(&clk, sizeof(Clock));
    if (e != cudaSuccess) {
        if (u) cudaFree(u);
        if (g) cudaFree(g);
        cudaGetLastError();
        return cuda_fail(e, "autotune scratch");
    }
    // the stages advance the scratch state by dt = 1e-12 (|A_1| < 1 keeps g bounded)
    Clock hclk{};
    hclk.dt = 1e-12;
    e = cudaMemsetAsync(g, 0, sz, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(clk, &hclk, sizeof(Clock), cudaMemcpyHostToDevice, s);
    // a smooth state on this mesh: the Taylor-Green field (any positive state would do)
    hs3d_ic ic{HS3D_IC_TGV, c->gamma, 0.3, 0.0, 0.0, 0.0, 0.0};
    if (e == cudaSuccess) e = launch_init_state(m->N, m->E, m->X, ic, m->lo, m->hi, u, s);
    Item it = make_item(m, c, u, g, nullptr);
    it.clk = clk;
    Batch b = single_batch(it);
    // the face fluxes the volume kernel reads: one face pass
    cont_forget(m, nullptr);   // the trial launches rewrite the mesh's FP32 shadow
    if (e == cudaSuccess && c->precision != HS3D_FP64) e = launch_shadow(m->N, b, s);
    if (e == cudaSuccess && c->physics == HS3D_NS) e = launch_grad(m->N, c->precision, b, s);
    if (e == cudaSuccess) e = launch_face(m->N, c->precision, c->physics, c->surface_flux, b, s);
    int best[2] = {0, 0};
    const int n3 = m->n3;
    const int maxthreads = n3 > 256 ? n3 : 256;
    const int reps = m->E >= 4096 ? 5 : 20;
    for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
        if (which == 0 && c->physics != HS3D_NS) continue;
        float best_ms = 1e30f;
        const int keep = tuned_elems_per_block(m->N, c->precision, which);
        for (int epb = 1; epb * n3 <= maxthreads && e == cudaSuccess; epb *= 2) {
            set_elems_per_block_p(m->N, c->precision, which, epb);
            float ms = time_kernels(m, c, b, which, reps, s, e);
            if (e != cudaSuccess) {
                // a shape the device cannot launch (shared memory): not a candidate
                if (e == cudaErrorInvalidValue || e == cudaErrorInvalidConfiguration) {
                    cudaGetLastError();
                    e = cudaSuccess;
                }
                continue;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best[which] = epb;
            }
        }
        set_elems_per_block_p(m->N, c->precision, which, best[which] ? best[which] : keep);
    }
    cudaStreamSynchronize(s);
    cudaFree(u);
    cudaFree(g);
    cudaFree(clk);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    save_cache_locked();
    if (choice_out) {
        choice_out[0] = elems_per_block_p(m->N, c->precision, 0);
        choice_out[1] = elems_per_block_p(m->N, c->precision, 1);
    }
    return HS3D_OK;
}
