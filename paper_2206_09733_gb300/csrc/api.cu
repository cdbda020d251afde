// C-ABI of the hs3d library: meshes, residual, RK3 steps, dt, diagnostics.
// The serving entry points live in server.cu.
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>

#include "api_internal.h"

namespace hs3d {

static thread_local std::string t_err;

hs3d_status fail(hs3d_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

hs3d_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? HS3D_ERR_NOMEM : HS3D_ERR_CUDA, "%s: %s (%s)", what,
                cudaGetErrorString(e), cudaGetErrorName(e));
}

cudaError_t prepare_kernels(int N)
{
    tune_cache_load();
    if (!device_ops(N)) return cudaErrorMemoryAllocation;
    cudaError_t e = prepare_volume(N);
    if (e == cudaSuccess) e = prepare_grad(N);
    if (e == cudaSuccess) e = prepare_gauss(N);
    return e;
}

hs3d_status validate_cfg(const hs3d_solver_cfg *c)
{
    if (!c) return fail(HS3D_ERR_INVALID, "cfg is NULL");
    if (c->physics != HS3D_EULER && c->physics != HS3D_NS) return fail(HS3D_ERR_INVALID, "bad physics %d", c->physics);
    if (c->surface_flux < HS3D_FLUX_LF || c->surface_flux > HS3D_FLUX_MATRIX)
        return fail(HS3D_ERR_INVALID, "bad surface_flux %d", c->surface_flux);
    if (c->volume_form < HS3D_VOL_STANDARD || c->volume_form > HS3D_VOL_IR)
        return fail(HS3D_ERR_INVALID, "bad volume_form %d", c->volume_form);
    if (c->time_scheme != HS3D_TIME_RK3 && c->time_scheme != HS3D_TIME_RK4)
        return fail(HS3D_ERR_INVALID, "bad time_scheme %d", c->time_scheme);
    if (c->precision != HS3D_FP64 && c->precision != HS3D_MIXED32 && c->precision != HS3D_MIXED_TC)
        return fail(HS3D_ERR_UNSUPPORTED, "unsupported precision %d", c->precision);
    if (!(c->gamma > 1.0)) return fail(HS3D_ERR_INVALID, "gamma must be > 1");
    if (c->physics == HS3D_NS && (!(c->Re > 0.0) || !(c->Pr > 0.0)))
        return fail(HS3D_ERR_INVALID, "Re and Pr must be > 0 for Navier-Stokes");
    return HS3D_OK;
}

hs3d_status validate_desc(const hs3d_mesh_desc *d)
{
    if (!d) return fail(HS3D_ERR_INVALID, "mesh desc is NULL");
    if (d->N < 1 || d->N > kMaxN) return fail(HS3D_ERR_UNSUPPORTED, "N=%d outside 1..%d", d->N, kMaxN);
    if (d->ex < 1 || d->ey < 1 || d->ez < 1) return fail(HS3D_ERR_INVALID, "element counts must be >= 1");
    long long E = (long long)d->ex * d->ey * d->ez;
    long long n3 = (long long)(d->N + 1) * (d->N + 1) * (d->N + 1);
    if (E * 12 * n3 > 0x7fffffffLL) return fail(HS3D_ERR_UNSUPPORTED, "mesh too large for 32-bit node indexing");
    for (int c = 0; c < 3; ++c) {
        if (!(d->hi[c] > d->lo[c])) return fail(HS3D_ERR_INVALID, "hi must exceed lo");
        if (!d->periodic[c]) return fail(HS3D_ERR_UNSUPPORTED, "only periodic boxes are supported");
    }
    if (!(d->perturb_amp >= 0.0 && d->perturb_amp <= 0.2))
        return fail(HS3D_ERR_INVALID, "perturb_amp must lie in [0, 0.2]");
    if (d->nodes != HS3D_NODES_LOBATTO && d->nodes != HS3D_NODES_GAUSS)
        return fail(HS3D_ERR_INVALID, "bad nodes %d", d->nodes);
    return HS3D_OK;
}

size_t mesh_bytes(int N, long long E, int nodes)
{
    long long n = N + 1, n2 = n * n, n3 = n2 * n;
    // X, Ja, J, 1/J in FP64; Jaf, Jalo, 1/J in FP32 (+ the FP32 shadow on Gauss-Legendre nodes); face normals
    size_t geo = sizeof(double) * (size_t)E * n3 * (3 + 9 + 1 + 1) +
                 sizeof(float) * (size_t)E * n3 * (19 + (nodes == HS3D_NODES_GAUSS ? 5 : 0)) +
                 (sizeof(double) + sizeof(float)) * 3 * (size_t)E * 3 * n2;
    size_t scratch = sizeof(double) * (3 * (size_t)E * 5 * n2 + (size_t)E * 12 * n3);
    // Gauss-Legendre meshes hold Gauss-Lobatto temporaries while they are built
    size_t build = (nodes == HS3D_NODES_GAUSS) ? sizeof(double) * ((size_t)E * 21 * n3 + 9 * (size_t)E * n2) : 0;
    return geo + scratch + build + sizeof(Clock) + 4096 * 7 * sizeof(double);
}

hs3d_status check_mesh_cfg(const hs3d_mesh *m, const hs3d_solver_cfg *c)
{
    if (m->nodes == HS3D_NODES_GAUSS && c->volume_form != HS3D_VOL_STANDARD)
        return fail(HS3D_ERR_UNSUPPORTED,
                    "split volume forms need Gauss-Lobatto nodes (summation-by-parts with boundary nodes)");
    return HS3D_OK;
}

static hs3d_status mesh_alloc(hs3d_mesh *m)
{
    long long E = m->E, n3 = m->n3, n2 = m->n2;
    struct {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&m->X, sizeof(double) * E * 3 * n3},
        {(void **)&m->Ja, sizeof(double) * E * 9 * n3},
        {(void **)&m->Jaf, sizeof(float) * E * 9 * n3},
        {(void **)&m->Jalo, sizeof(float) * E * 9 * n3},
        {(void **)&m->J, sizeof(double) * E * n3},
        {(void **)&m->invJ, sizeof(double) * E * n3},
        {(void **)&m->invJf, sizeof(float) * E * n3},
        {(void **)&m->uf, m->nodes == HS3D_NODES_GAUSS ? sizeof(float) * E * 5 * n3 : 0},
        {(void **)&m->fn, sizeof(double) * 3 * E * 3 * n2},
        {(void **)&m->fnf, sizeof(float) * 3 * E * 3 * n2},
        {(void **)&m->anc, (size_t)112 * E},
        {(void **)&m->fstar, sizeof(double) * 3 * E * 5 * n2},
        {(void **)&m->grad, sizeof(double) * E * 12 * n3},
        {(void **)&m->clk, sizeof(Clock)},
        {(void **)&m->diag_partials, sizeof(double) * 4096 * 7},
    };
    for (auto &a : allocs) {
        if (a.bytes == 0) continue;
        cudaError_t e = cudaMalloc(a.p, a.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_fail(e, "cudaMalloc of mesh arrays");
        }
        m->bytes += a.bytes;
    }
    return HS3D_OK;
}

void mesh_free(hs3d_mesh *m)
{
    if (!m) return;
    for (auto &gs : m->gslot)
        if (gs.exec) cudaGraphExecDestroy(gs.exec);
    void *ptrs[] = {m->X,  m->Ja,  m->Jaf,   m->Jalo, m->J,   m->invJ,          m->invJf,
                    m->uf, m->fn,  m->fnf,   m->anc,  m->fstar, m->grad, m->clk, m->diag_partials};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

hs3d_status mesh_build(const hs3d_mesh_desc *desc, hs3d_mesh **out)
{
    hs3d_status st = validate_desc(desc);
    if (st != HS3D_OK) return st;
    hs3d_mesh *m = new (std::nothrow) hs3d_mesh();
    if (!m) return fail(HS3D_ERR_NOMEM, "host allocation failed");
    m->ex = desc->ex;
    m->ey = desc->ey;
    m->ez = desc->ez;
    m->N = desc->N;
    m->n = desc->N + 1;
    m->n2 = m->n * m->n;
    m->n3 = m->n2 * m->n;
    m->E = desc->ex * desc->ey * desc->ez;
    for (int c = 0; c < 3; ++c) {
        m->lo[c] = desc->lo[c];
        m->hi[c] = desc->hi[c];
    }
    m->amp = desc->perturb_amp;
    m->nodes = desc->nodes;
    cudaError_t e = cudaGetDevice(&m->device);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "no CUDA device");
    }
    e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "cudaStreamCreate");
    }
    st = mesh_alloc(m);
    if (st != HS3D_OK) {
        mesh_free(m);
        return st;
    }
    e = prepare_kernels(m->N);
    if (e != cudaSuccess) {
        mesh_free(m);
        return cuda_fail(e, "kernel preparation");
    }
    double *xyz_dev = nullptr;
    if (desc->node_xyz) {
        size_t bytes = sizeof(double) * (size_t)m->E * 3 * m->n3;
        e = cudaMalloc(&xyz_dev, bytes);
        if (e == cudaSuccess) e = cudaMemcpyAsync(xyz_dev, desc->node_xyz, bytes, cudaMemcpyHostToDevice, m->stream);
        if (e != cudaSuccess) {
            if (xyz_dev) cudaFree(xyz_dev);
            mesh_free(m);
            return cuda_fail(e, "uploading node_xyz");
        }
    }
    if (!device_ops(m->N, m->nodes)) {
        if (xyz_dev) cudaFree(xyz_dev);
        mesh_free(m);
        return fail(HS3D_ERR_NOMEM, "operator tables");
    }
    e = launch_geometry(m->N, m->nodes, xyz_dev, m->ex, m->ey, m->ez, m->lo, m->hi, m->amp, m->X, m->Ja, m->Jaf, m->J, m->invJ,
                        m->invJf, m->fn, m->fnf, m->stream);
    if (e == cudaSuccess) e = launch_metric_lo(m->Ja, m->Jaf, m->Jalo, (long long)m->E * 9 * m->n3, m->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(m->clk, 0, sizeof(Clock), m->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (xyz_dev) cudaFree(xyz_dev);
    if (e != cudaSuccess) {
        mesh_free(m);
        return cuda_fail(e, "geometry kernel");
    }
    *out = m;
    return HS3D_OK;
}

Item make_item(const hs3d_mesh *m, const hs3d_solver_cfg *c, const double *u, double *g, double *out)
{
    Item it{};
    it.Ja = m->Ja;
    it.Jaf = m->Jaf;
    it.Jalo = m->Jalo;
    it.invJ = m->invJ;
    it.invJf = m->invJf;
    it.fn = m->fn;
    it.fnf = m->fnf;
    it.J = m->J;
    it.u = const_cast<double *>(u);
    it.uf = m->uf;
    it.anc = m->anc;
    it.g = g;
    it.out = out;
    it.fstar = m->fstar;
    it.grad = m->grad;
    it.clk = m->clk;
    it.ex = m->ex;
    it.ey = m->ey;
    it.ez = m->ez;
    it.E = m->E;
    it.elem_begin = 0;
    it.face_begin = 0;
    it.gamma = c ? c->gamma : 1.4;
    it.mu = (c && c->physics == HS3D_NS) ? 1.0 / c->Re : 0.0;
    it.kappa = (c && c->physics == HS3D_NS) ? it.mu * c->gamma / ((c->gamma - 1.0) * c->Pr) : 0.0;
    it.cfl = c ? c->cfl : 0.5;
    it.gauss = m->nodes == HS3D_NODES_GAUSS;
    it.kc = it.gauss ? 3.0 : 8.0;    // dt rule: cfl kc / (n^2 lambda_c), kv / (n^4 lambda_v)
    it.kv = it.gauss ? 4.0 : 12.0;
    it.gm1 = it.gamma - 1.0;
    it.hg = 0.5 / it.gm1;
    it.gammaf = (float)it.gamma;
    it.gm1f = (float)it.gm1;
    it.hgf = (float)it.hg;
    it.igm1f = 1.0 / (double)it.gm1f;
    it.hglof = (float)(0.5 * it.igm1f - (double)it.hgf);
    it.muf = (float)it.mu;
    it.kappaf = (float)it.kappa;
    return it;
}

Batch single_batch(const Item &it)
{
    Batch b{};
    b.single = it;
    b.items = nullptr;
    b.nitems = 1;
    b.total_elems = it.E;
    b.total_faces = 3LL * it.E;
    b.dt_fixed = 0.0;
    b.gauss = it.gauss;
    b.mortar = it.face6 ? 1 : 0;
    return b;
}

// Residual of a batch: [BR1 gradients] -> faces -> volume/lift/scale (+ RK stage).
cudaError_t enqueue_stage(int N, const hs3d_solver_cfg *c, const Batch &b, int stage, int lam_slot, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (c->physics == HS3D_NS) e = launch_grad(N, c->precision, b, s);
    if (e == cudaSuccess) e = launch_face(N, c->precision, c->physics, c->surface_flux, b, s);
    if (e == cudaSuccess) e = launch_volume(N, c->precision, c->physics, c->volume_form, c->time_scheme, b, stage, lam_slot, s);
    return e;
}

// One low-storage RK step (scheme c->time_scheme) of a batch.  The dt maxima come from clock slot 0 filled by a
// fresh k_lambda pass (fresh_lambda != 0, a single step on a state the caller
// may have changed), or from slot 1, filled by the previous step's last
// stage (or by prime_lambda before the first step of a run).  The last stage
// always refills slot 1 for the next step.
cudaError_t enqueue_rk3_step(int N, const hs3d_solver_cfg *c, Batch b, double dt, int fresh_lambda, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    b.dt_fixed = dt > 0.0 ? dt : 0.0;
    int slot = fresh_lambda ? 0 : 1;
    if (fresh_lambda && !(dt > 0.0)) e = launch_lambda(N, c->precision, c->physics, b, 0, s);
    else if (fresh_lambda && c->precision != HS3D_FP64) e = launch_shadow(N, b, s);
    if (e == cudaSuccess) e = launch_dt_finalize(N, b, 0, slot, s);
    const int ns = rk_stages(c->time_scheme);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) e = enqueue_stage(N, c, b, k, k == ns - 1 ? 1 : -1, s);
    return e;
}

// Fill clock slot 1 from the current state (before the first step of a run).
cudaError_t prime_lambda(int N, const hs3d_solver_cfg *c, const Batch &b, Clock *clk, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    if (clk) e = cudaMemsetAsync(&clk->lam[1][0], 0, sizeof(clk->lam[1]), s);
    if (e == cudaSuccess) e = launch_lambda(N, c->precision, c->physics, b, 1, s);
    return e;
}

bool same_cfg(const hs3d_solver_cfg &k, const hs3d_solver_cfg &c)
{
    // field-wise: the struct has padding
    return k.physics == c.physics && k.surface_flux == c.surface_flux && k.volume_form == c.volume_form &&
           k.precision == c.precision && k.gamma == c.gamma && k.Re == c.Re && k.Pr == c.Pr && k.Ma == c.Ma &&
           k.cfl == c.cfl && k.time_scheme == c.time_scheme;
}

void cont_set(const hs3d_mesh *mc, const double *u, const hs3d_solver_cfg *c)
{
    hs3d_mesh *m = const_cast<hs3d_mesh *>(mc);
    std::lock_guard<std::mutex> lock(m->mu);
    m->cont_u = u;
    m->cont_cfg = *c;
}

// A call rewrote the FP32 shadow or the clock for state u_written: the
// continuation record survives only if it is the same state.
void cont_forget(const hs3d_mesh *mc, const double *u_written)
{
    hs3d_mesh *m = const_cast<hs3d_mesh *>(mc);
    std::lock_guard<std::mutex> lock(m->mu);
    if (!u_written || u_written != m->cont_u) m->cont_u = nullptr;
}

hs3d_status check_ptr(const void *p, const char *name)
{
    if (!p) return fail(HS3D_ERR_INVALID, "%s is NULL", name);
    if (((uintptr_t)p) % 16) return fail(HS3D_ERR_INVALID, "%s is not 16-byte aligned", name);
    return HS3D_OK;
}

}  // namespace hs3d

using namespace hs3d;

extern "C" {

const char *hs3d_last_error(void) { return t_err.c_str(); }

const char *hs3d_version(void) { return "hs3d 0.1 (sm_103a)"; }

hs3d_status hs3d_mesh_create(const hs3d_mesh_desc *desc, hs3d_mesh **out)
{
    if (!out) return fail(HS3D_ERR_INVALID, "out is NULL");
    *out = nullptr;
    return mesh_build(desc, out);
}

void hs3d_mesh_destroy(hs3d_mesh *mesh) { mesh_free(mesh); }

hs3d_status hs3d_mesh_info(const hs3d_mesh *m, int64_t *E, int *N, size_t *bytes)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    if (E) *E = m->E;
    if (N) *N = m->N;
    if (bytes) *bytes = m->bytes;
    return HS3D_OK;
}

hs3d_status hs3d_mesh_geometry(const hs3d_mesh *m, double *X, double *Ja, double *J, void *stream)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    size_t en = (size_t)m->E * m->n3;
    cudaError_t e = cudaSuccess;
    if (X) e = cudaMemcpyAsync(X, m->X, sizeof(double) * en * 3, cudaMemcpyDeviceToDevice, s);
    if (Ja && e == cudaSuccess) e = cudaMemcpyAsync(Ja, m->Ja, sizeof(double) * en * 9, cudaMemcpyDeviceToDevice, s);
    if (J && e == cudaSuccess) e = cudaMemcpyAsync(J, m->J, sizeof(double) * en, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "geometry copy");
}

hs3d_status hs3d_init_state(const hs3d_mesh *m, const hs3d_ic *ic, double *u, void *stream)
{
    if (!m || !ic) return fail(HS3D_ERR_INVALID, "mesh or ic is NULL");
    hs3d_status st = check_ptr(u, "u");
    if (st != HS3D_OK) return st;
    if (ic->kind != HS3D_IC_VORTEX && ic->kind != HS3D_IC_TGV) return fail(HS3D_ERR_INVALID, "bad ic kind");
    if (!(ic->gamma > 1.0)) return fail(HS3D_ERR_INVALID, "ic gamma must be > 1");
    if (ic->kind == HS3D_IC_TGV && !(ic->Ma > 0.0)) return fail(HS3D_ERR_INVALID, "TGV needs Ma > 0");
    {   // the state itself is rewritten
        hs3d_mesh *mm = const_cast<hs3d_mesh *>(m);
        std::lock_guard<std::mutex> lock(mm->mu);
        if (mm->cont_u == u) mm->cont_u = nullptr;
    }
    cudaError_t e = launch_init_state(m->N, m->E, m->X, *ic, m->lo, m->hi, u, (cudaStream_t)stream);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "init_state");
}

hs3d_status hs3d_residual(const hs3d_mesh *m, const hs3d_solver_cfg *c, const double *u, double *dudt, void *stream)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK) st = check_mesh_cfg(m, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK) st = check_ptr(dudt, "dudt");
    if (st != HS3D_OK) return st;
    if ((const void *)u == (const void *)dudt) return fail(HS3D_ERR_INVALID, "u and dudt must differ");
    Item it = make_item(m, c, u, nullptr, dudt);
    it.clk = nullptr;
    cudaError_t e = cudaSuccess;
    if (c->precision != HS3D_FP64) {
        cont_forget(m, u);
        e = launch_shadow(m->N, single_batch(it), (cudaStream_t)stream);
    }
    if (e == cudaSuccess) e = enqueue_stage(m->N, c, single_batch(it), -1, -1, (cudaStream_t)stream);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "residual launch");
}

hs3d_status hs3d_rk3_step(const hs3d_mesh *m, const hs3d_solver_cfg *c, double *u, double *g, double dt, void *stream)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK) st = check_mesh_cfg(m, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK) st = check_ptr(g, "g");
    if (st != HS3D_OK) return st;
    if (u == g) return fail(HS3D_ERR_INVALID, "u and g must differ");
    Item it = make_item(m, c, u, g, nullptr);
    cudaError_t e = enqueue_rk3_step(m->N, c, single_batch(it), dt > 0.0 ? dt : 0.0, 1, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cont_forget(m, nullptr);
        return cuda_fail(e, "rk3 step launch");
    }
    cont_set(m, u, c);
    return HS3D_OK;
}

hs3d_status hs3d_rk3_run(const hs3d_mesh *mc, const hs3d_solver_cfg *c, double *u, double *g, double dt, int nsteps,
                         void *stream)
{
    hs3d_mesh *m = const_cast<hs3d_mesh *>(mc);
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK) st = check_mesh_cfg(m, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK) st = check_ptr(g, "g");
    if (st != HS3D_OK) return st;
    if (u == g) return fail(HS3D_ERR_INVALID, "u and g must differ");
    if (nsteps < 0) return fail(HS3D_ERR_INVALID, "nsteps < 0");
    if (nsteps == 0) return HS3D_OK;
    std::lock_guard<std::mutex> lock(m->mu);
    // dt < 0: continue from the previous step on this mesh when it advanced this
    // same state and configuration (the graph is the one of dt = 0)
    const bool cont = dt < 0.0 && m->cont_u == u && same_cfg(m->cont_cfg, *c);
    if (dt < 0.0) dt = 0.0;
    // a cached graph for exactly these arguments
    hs3d_mesh::GraphSlot *slot = nullptr;
    for (auto &gs : m->gslot)
        if (gs.exec && gs.u == u && gs.g == g && gs.dt == dt && same_cfg(gs.cfg, *c)) slot = &gs;
    cudaError_t e = cudaSuccess;
    if (!slot) {
        // capture into the empty or least recently used slot
        slot = &m->gslot[0];
        for (auto &gs : m->gslot)
            if (!gs.exec || (slot->exec && gs.used < slot->used)) slot = &gs;
        if (slot->exec) {
            cudaGraphExecDestroy(slot->exec);
            slot->exec = nullptr;
        }
        Item it = make_item(m, c, u, g, nullptr);
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_rk3_step(m->N, c, single_batch(it), dt, 0, m->stream);
            e = cudaStreamEndCapture(m->stream, &graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&slot->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            slot->exec = nullptr;
            cudaGetLastError();
            return cuda_fail(e, "graph capture");
        }
        slot->u = u;
        slot->g = g;
        slot->dt = dt;
        slot->cfg = *c;
    }
    slot->used = ++m->gtick;
    if (!cont) {
        Item it = make_item(m, c, u, g, nullptr);
        if (!(dt > 0.0)) e = prime_lambda(m->N, c, single_batch(it), m->clk, (cudaStream_t)stream);
        else if (c->precision != HS3D_FP64) e = launch_shadow(m->N, single_batch(it), (cudaStream_t)stream);
    }
    for (int k = 0; k < nsteps && e == cudaSuccess; ++k) e = cudaGraphLaunch(slot->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        m->cont_u = nullptr;
        return cuda_fail(e, "graph launch");
    }
    m->cont_u = u;
    m->cont_cfg = *c;
    return HS3D_OK;
}

hs3d_status hs3d_dt(const hs3d_mesh *m, const hs3d_solver_cfg *c, const double *u, double *dt_out, void *stream)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK) st = check_mesh_cfg(m, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK && !dt_out) st = fail(HS3D_ERR_INVALID, "dt_out is NULL");
    if (st != HS3D_OK) return st;
    Item it = make_item(m, c, u, nullptr, dt_out);
    Batch b = single_batch(it);
    cont_forget(m, u);   // (the pass rewrites the FP32 shadow for u)
    cudaError_t e = launch_lambda(m->N, c->precision, c->physics, b, 0, (cudaStream_t)stream);
    if (e == cudaSuccess) e = launch_dt_finalize(m->N, b, 2, 0, (cudaStream_t)stream);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "dt launch");
}

hs3d_status hs3d_clock(const hs3d_mesh *m, double *t, int64_t *steps, int reset, void *stream)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    Clock h{};
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&h, m->clk, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && reset) {
        cont_forget(m, nullptr);
        e = cudaMemsetAsync(m->clk, 0, sizeof(Clock), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "clock read");
    if (t) *t = h.t;
    if (steps) *steps = h.step;
    if (h.bad == 2) return fail(HS3D_ERR_TIMEOUT, "a device-side wait for a bulk copy ran out of polls");
    if (h.bad) return fail(HS3D_ERR_NONPHYSICAL, "non-physical state detected (rho <= 0, p <= 0 or NaN)");
    return HS3D_OK;
}

hs3d_status hs3d_diagnostics(const hs3d_mesh *m, const hs3d_solver_cfg *c, const double *u, const double *dudt,
                             double *out, void *stream)
{
    if (!m) return fail(HS3D_ERR_INVALID, "mesh is NULL");
    hs3d_status st = check_ptr(u, "u");
    if (st == HS3D_OK && !out) st = fail(HS3D_ERR_INVALID, "out is NULL");
    if (st != HS3D_OK) return st;
    Item it = make_item(m, c, u, nullptr, nullptr);
    int nb = diagnostics_blocks(m->N, m->E);
    cudaError_t e = launch_diagnostics(m->N, it, dudt, m->diag_partials, nb, out, (cudaStream_t)stream);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "diagnostics launch");
}

}  // extern "C"
