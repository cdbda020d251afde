// Meshes whose elements carry their own polynomial degree (Sec. 3.6: the
// degree of every element may differ; neighbours of different degree are
// coupled by mortars).
//
// The elements are grouped by degree into buckets.  Each bucket is a
// conforming-path mesh object of its own degree (geometry, FP32 shadow,
// gradient scratch, clock) whose element kernels run with Item::face6: they
// take their six face fluxes (and BR1 interface values) from per-element
// blocks that the mortar face kernel (mortar.cu) writes for every face of
// the whole mesh.  A stage is
//   [k_mortar interface values -> k_grad per bucket]  (Navier-Stokes)
//   k_mortar face fluxes -> k_volume per bucket (volume + lift + 1/J + RK stage)
// and a step starts with the dt rule over all buckets (k_pdt_finalize).
//
// Geometry (the free-stream rules for p-non-conforming faces that Sec. 3.6
// follows): every element's map is the polynomial of degree
// Ngeo = max(1, floor(Nmin/2)) that interpolates the box map at the
// element's Gauss-Lobatto points of degree Ngeo, evaluated at its own nodes;
// the metric terms are the curl form at the element's own degree.  The
// products X_l dX_m then have degree 2 Ngeo <= Nmin per direction, every
// element represents them exactly, and the face metric terms are one
// polynomial seen from both sides.  Nmin = 1 allows only an affine map
// (perturb_amp = 0).
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "aniso.cuh"
#include "api_internal.h"
#include "mortar.cuh"

using namespace hs3d;

struct hs3d_pmesh {
    int ex = 0, ey = 0, ez = 0, E = 0, Nmin = 0, Nmax = 0, Ngeo = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0}, amp = 0.0;
    std::vector<int> deg;
    std::vector<int64_t> off;   // [E+1] state offsets (doubles)
    AnisoMesh *an = nullptr;    // degrees that differ between directions: the anisotropic path (aniso.cu),
                                // which then holds everything below instead of the buckets
    struct Bucket {
        int N = 0, E = 0;
        int64_t base = 0;
        hs3d_mesh *m = nullptr;
        void *fstar6 = nullptr, *qhat6 = nullptr;
    };
    std::vector<Bucket> b;
    double *diag_tmp = nullptr;    // device [nb][7]: per-bucket diagnostics before their fixed-order sum
    MortarFace *faces = nullptr;   // device [3E], sorted into groups (see launch_mortar)
    int group_begin[2 * kMaxn + 1] = {0};   // group g: faces [group_begin[g], group_begin[g + 1])
    MortarSide *sides = nullptr;   // device [nb]
    Clock **clks = nullptr;        // device [nb]
    int *nb_n = nullptr;           // device [nb]
    cudaStream_t stream = nullptr;
    // the degree buckets (and the mortar-degree groups) of one phase are independent: they run on
    // these streams, forked from and joined back to the caller's stream (parallel graph branches
    // when captured)
    static constexpr int kAux = 2 * kMaxn;   // at most 14 face groups, 7 buckets
    cudaStream_t aux[kAux] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kAux] = {};
    std::mutex mu;
    // continuation record: the state and configuration the last hs3d_pmesh_run advanced (its last
    // stage left the dt maxima in clock slot 1 and the FP32 shadow of that state)
    const double *cont_u = nullptr;
    hs3d_solver_cfg cont_cfg{};
    cudaGraphExec_t gexec = nullptr;   // one step of hs3d_pmesh_run for (gcfg, gu, gg, gdt)
    hs3d_solver_cfg gcfg{};
    const double *gu = nullptr, *gg = nullptr;
    double gdt = 0.0;
};

namespace {

void pmesh_free(hs3d_pmesh *pm)
{
    if (!pm) return;
    if (pm->an) aniso_free(pm->an);
    if (pm->gexec) cudaGraphExecDestroy(pm->gexec);
    for (auto &bk : pm->b) {
        if (bk.m) mesh_free(bk.m);
        if (bk.fstar6) cudaFree(bk.fstar6);
        if (bk.qhat6) cudaFree(bk.qhat6);
    }
    void *ptrs[] = {pm->faces, pm->sides, pm->clks, pm->nb_n, pm->diag_tmp};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (int k = 0; k < hs3d_pmesh::kAux; ++k) {
        if (pm->aux[k]) cudaStreamDestroy(pm->aux[k]);
        if (pm->ev_join[k]) cudaEventDestroy(pm->ev_join[k]);
    }
    if (pm->ev_fork) cudaEventDestroy(pm->ev_fork);
    if (pm->stream) cudaStreamDestroy(pm->stream);
    delete pm;
}

// The box map (with its perturbation) at reference point r of element e.
void box_point(const hs3d_pmesh *pm, int e, const double r[3], double x[3])
{
    const int Ed[3] = {pm->ex, pm->ey, pm->ez};
    const int ab[3] = {e % pm->ex, (e / pm->ex) % pm->ey, e / (pm->ex * pm->ey)};
    double th[3];
    for (int c = 0; c < 3; ++c) {
        const double L = pm->hi[c] - pm->lo[c];
        x[c] = pm->lo[c] + (L / Ed[c]) * (ab[c] + 0.5 * (r[c] + 1.0));
        th[c] = -M_PI + 2.0 * M_PI * (x[c] - pm->lo[c]) / L;
    }
    const double s = sin(th[0]) * sin(th[1]) * sin(th[2]);
    for (int c = 0; c < 3; ++c) x[c] += pm->amp * ((pm->hi[c] - pm->lo[c]) / (2.0 * M_PI)) * s;
}

void lagrange_row(int n, const double *x, double y, double *l)
{
    for (int j = 0; j < n; ++j) {
        double v = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) v *= (y - x[k]) / (x[j] - x[k]);
        l[j] = v;
    }
}

// Node coordinates [3][n3] of element e at degree N: the degree-Ngeo
// interpolant of the box map evaluated at the degree-N Gauss-Lobatto nodes.
void element_nodes(const hs3d_pmesh *pm, int e, int N, double *X)
{
    const int G = pm->Ngeo, ng = G + 1, n = N + 1, n3 = n * n * n;
    const Ops &og = host_ops(G), &on = host_ops(N);
    std::vector<double> Xg(3 * ng * ng * ng);
    for (int k = 0; k < ng; ++k)
        for (int j = 0; j < ng; ++j)
            for (int i = 0; i < ng; ++i) {
                const double r[3] = {og.xi[i], og.xi[j], og.xi[k]};
                double x[3];
                box_point(pm, e, r, x);
                for (int c = 0; c < 3; ++c) Xg[(size_t)c * ng * ng * ng + i + ng * (j + ng * k)] = x[c];
            }
    double L[kMaxn][kMaxn];
    for (int t = 0; t < n; ++t) lagrange_row(ng, og.xi, on.xi[t], L[t]);
    for (int c = 0; c < 3; ++c)
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double acc = 0.0;
                    for (int kk = 0; kk < ng; ++kk)
                        for (int jj = 0; jj < ng; ++jj)
                            for (int ii = 0; ii < ng; ++ii)
                                acc += L[k][kk] * L[j][jj] * L[i][ii] *
                                       Xg[(size_t)c * ng * ng * ng + ii + ng * (jj + ng * kk)];
                    X[(size_t)c * n3 + i + n * (j + n * k)] = acc;
                }
}

hs3d_status pmesh_build(const hs3d_mesh_desc *desc, const int *degree, hs3d_pmesh **out)
{
    if (!desc || !degree) return fail(HS3D_ERR_INVALID, "desc or degree is NULL");
    if (desc->node_xyz) return fail(HS3D_ERR_UNSUPPORTED, "per-element degrees take no node_xyz");
    if (desc->nodes != HS3D_NODES_LOBATTO)
        return fail(HS3D_ERR_UNSUPPORTED, "per-element degrees need Gauss-Lobatto nodes");
    if (desc->ex < 1 || desc->ey < 1 || desc->ez < 1) return fail(HS3D_ERR_INVALID, "element counts must be >= 1");
    const long long E = (long long)desc->ex * desc->ey * desc->ez;
    if (E > (1 << 26)) return fail(HS3D_ERR_UNSUPPORTED, "too many elements");
    int Nmin = 99, Nmax = 0;
    for (long long e = 0; e < E; ++e) {
        if (degree[e] < 1 || degree[e] > kMaxN)
            return fail(HS3D_ERR_UNSUPPORTED, "degree %d of element %lld outside 1..%d", degree[e], e, kMaxN);
        Nmin = degree[e] < Nmin ? degree[e] : Nmin;
        Nmax = degree[e] > Nmax ? degree[e] : Nmax;
    }
    hs3d_mesh_desc chk = *desc;
    chk.N = Nmax;
    hs3d_status st = validate_desc(&chk);
    if (st != HS3D_OK) return st;
    if (Nmin == 1 && desc->perturb_amp != 0.0)
        return fail(HS3D_ERR_INVALID, "a degree-1 element allows only an affine map (perturb_amp = 0)");
    hs3d_pmesh *pm = new (std::nothrow) hs3d_pmesh();
    if (!pm) return fail(HS3D_ERR_NOMEM, "host allocation failed");
    pm->ex = desc->ex;
    pm->ey = desc->ey;
    pm->ez = desc->ez;
    pm->E = (int)E;
    pm->Nmin = Nmin;
    pm->Nmax = Nmax;
    pm->Ngeo = Nmin / 2 >= 1 ? Nmin / 2 : 1;
    for (int c = 0; c < 3; ++c) {
        pm->lo[c] = desc->lo[c];
        pm->hi[c] = desc->hi[c];
    }
    pm->amp = desc->perturb_amp;
    pm->deg.assign(degree, degree + E);
    pm->off.assign(E + 1, 0);
    cudaError_t e = cudaStreamCreateWithFlags(&pm->stream, cudaStreamNonBlocking);
    for (int k = 0; k < hs3d_pmesh::kAux && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&pm->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pm->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pm->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        pmesh_free(pm);
        return cuda_fail(e, "cudaStreamCreate");
    }
    // buckets in increasing degree
    std::vector<int> bucket_of(E), local_of(E);
    int64_t base = 0;
    for (int N = 1; N <= kMaxN; ++N) {
        std::vector<int> els;
        for (int i = 0; i < pm->E; ++i)
            if (pm->deg[i] == N) els.push_back(i);
        if (els.empty()) continue;
        const int n = N + 1, n2 = n * n, n3 = n2 * n;
        hs3d_pmesh::Bucket bk;
        bk.N = N;
        bk.E = (int)els.size();
        bk.base = base;
        std::vector<double> X((size_t)bk.E * 3 * n3);
        for (int l = 0; l < bk.E; ++l) {
            element_nodes(pm, els[l], N, X.data() + (size_t)l * 3 * n3);
            bucket_of[els[l]] = (int)pm->b.size();
            local_of[els[l]] = l;
            pm->off[els[l]] = base + (int64_t)l * 5 * n3;
        }
        hs3d_mesh_desc bd = *desc;
        bd.ex = bk.E;
        bd.ey = bd.ez = 1;
        bd.N = N;
        bd.node_xyz = X.data();
        st = mesh_build(&bd, &bk.m);
        if (st == HS3D_OK) {
            // the mortar kernels read the bucket's FP32 shadow of the state
            e = cudaMalloc(&bk.m->uf, sizeof(float) * (size_t)bk.E * 5 * n3);
            if (e == cudaSuccess) bk.m->bytes += sizeof(float) * (size_t)bk.E * 5 * n3;
            if (e == cudaSuccess) e = cudaMalloc(&bk.fstar6, sizeof(double) * 6 * (size_t)bk.E * 5 * n2);
            if (e == cudaSuccess) e = cudaMalloc(&bk.qhat6, sizeof(double) * 6 * (size_t)bk.E * 4 * n2);
            if (e != cudaSuccess) {
                cudaGetLastError();
                st = cuda_fail(e, "cudaMalloc of face blocks");
            }
        }
        pm->b.push_back(bk);
        if (st != HS3D_OK) {
            pmesh_free(pm);
            return st;
        }
        // the next bucket starts at a multiple of 160 doubles: 16-byte aligned
        // for the bulk copies, and a multiple of 5 so that node offsets
        // (state offset / 5) are whole
        base += (int64_t)bk.E * 5 * n3;
        base = (base + 159) / 160 * 160;
    }
    pm->off[E] = base;
    // face and bucket tables
    const int nb = (int)pm->b.size();
    // faces grouped by mortar degree NM (group NM), element-major within a
    // group; on a mesh of a single degree N every face is conforming and goes
    // to group kMaxn + N (the barrier-free face kernel: -11% per step at 32^3,
    // N = 3).  On mixed meshes the faces between equal degrees stay in their
    // degree's mortar group: splitting them off measured 2-5% slower (more,
    // smaller launches).
    std::vector<MortarFace> by_deg[2 * kMaxn];
    for (int i = 0; i < pm->E; ++i) {
        const int ab[3] = {i % pm->ex, (i / pm->ex) % pm->ey, i / (pm->ex * pm->ey)};
        const int Ed[3] = {pm->ex, pm->ey, pm->ez};
        for (int d = 0; d < 3; ++d) {
            int c[3] = {ab[0], ab[1], ab[2]};
            c[d] = (c[d] + 1) % Ed[d];
            const int r = c[0] + pm->ex * (c[1] + pm->ey * c[2]);
            const int NM = pm->deg[i] > pm->deg[r] ? pm->deg[i] : pm->deg[r];
            const int grp = pm->Nmin == pm->Nmax ? kMaxn + NM : NM;
            by_deg[grp].push_back(MortarFace{bucket_of[i], local_of[i], bucket_of[r], local_of[r], d});
        }
    }
    std::vector<MortarFace> faces;
    for (int g = 0; g < 2 * kMaxn; ++g) {
        pm->group_begin[g] = (int)faces.size();
        faces.insert(faces.end(), by_deg[g].begin(), by_deg[g].end());
    }
    pm->group_begin[2 * kMaxn] = (int)faces.size();
    std::vector<MortarSide> sides(nb);
    std::vector<Clock *> clks(nb);
    std::vector<int> nbn(nb);
    for (int k = 0; k < nb; ++k) {
        const auto &bk = pm->b[k];
        sides[k] = MortarSide{bk.N, bk.E, (long long)bk.base, bk.m->uf, bk.m->grad, bk.m->Ja, bk.m->Jaf,
                              bk.fstar6, bk.qhat6};
        clks[k] = bk.m->clk;
        nbn[k] = bk.N + 1;
    }
    e = cudaMalloc(&pm->faces, sizeof(MortarFace) * faces.size());
    if (e == cudaSuccess) e = cudaMalloc(&pm->sides, sizeof(MortarSide) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&pm->clks, sizeof(Clock *) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&pm->nb_n, sizeof(int) * nb);
    if (e == cudaSuccess) e = cudaMalloc(&pm->diag_tmp, sizeof(double) * 7 * nb);
    if (e == cudaSuccess)
        e = cudaMemcpy(pm->faces, faces.data(), sizeof(MortarFace) * faces.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pm->sides, sides.data(), sizeof(MortarSide) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pm->clks, clks.data(), sizeof(Clock *) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pm->nb_n, nbn.data(), sizeof(int) * nb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !device_mortar_ops()) e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        cudaGetLastError();
        pmesh_free(pm);
        return cuda_fail(e, "mortar tables");
    }
    *out = pm;
    return HS3D_OK;
}

// Items of every bucket for state u (and g / dudt), on the face6 path.
std::vector<Batch> bucket_batches(const hs3d_pmesh *pm, const hs3d_solver_cfg *c, const double *u, double *g,
                                  double *out, bool with_clock)
{
    std::vector<Batch> v;
    for (const auto &bk : pm->b) {
        Item it = make_item(bk.m, c, u + bk.base, g ? g + bk.base : nullptr, out ? out + bk.base : nullptr);
        it.face6 = 1;
        it.fstar = bk.fstar6;
        it.qhat6 = bk.qhat6;
        if (!with_clock) it.clk = nullptr;
        v.push_back(single_batch(it));
    }
    return v;
}

MortarPhys<double> mortar_phys(const hs3d_pmesh *pm, const hs3d_solver_cfg *c)
{
    const Item it = make_item(pm->b[0].m, c, nullptr, nullptr, nullptr);
    return MortarPhys<double>{it.gamma, it.gm1, it.hg, it.mu, it.kappa};
}

// fn(k, stream) for every k of ks, each on its own auxiliary stream ordered
// after the work already on s; s then waits for all of them.
template <class F>
cudaError_t fork_join(const hs3d_pmesh *pm, cudaStream_t s, const std::vector<int> &ks, F fn)
{
    if (ks.size() <= 1) return ks.empty() ? cudaSuccess : fn(ks[0], s);
    if (ks.size() > (size_t)hs3d_pmesh::kAux) return cudaErrorInvalidValue;
    cudaError_t e = cudaEventRecord(pm->ev_fork, s);
    for (size_t i = 0; i < ks.size() && e == cudaSuccess; ++i) {
        e = cudaStreamWaitEvent(pm->aux[i], pm->ev_fork, 0);
        if (e == cudaSuccess) e = fn(ks[i], pm->aux[i]);
        if (e == cudaSuccess) e = cudaEventRecord(pm->ev_join[i], pm->aux[i]);
    }
    for (size_t i = 0; i < ks.size() && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(s, pm->ev_join[i], 0);
    return e;
}

// One residual evaluation or RK stage over all buckets.
cudaError_t p_stage(const hs3d_pmesh *pm, const hs3d_solver_cfg *c, const std::vector<Batch> &bb, const double *u,
                    int stage, int lam_slot, cudaStream_t s)
{
    const MortarPhys<double> P = mortar_phys(pm, c);
    const int *gb = pm->group_begin;
    std::vector<int> groups, buckets;
    for (int g = 0; g < 2 * kMaxn; ++g)
        if (gb[g + 1] > gb[g]) groups.push_back(g);
    for (size_t k = 0; k < bb.size(); ++k) buckets.push_back((int)k);
    auto mortar = [&](int mode) {
        return [&, mode](int NM, cudaStream_t st) {
            return launch_mortar(c->precision, c->physics, mode, c->surface_flux, pm->faces, gb, NM, pm->sides, u, P,
                                 st);
        };
    };
    cudaError_t e = cudaSuccess;
    if (c->physics == HS3D_NS) {
        e = fork_join(pm, s, groups, mortar(0));
        if (e == cudaSuccess)
            e = fork_join(pm, s, buckets,
                          [&](int k, cudaStream_t st) { return launch_grad(pm->b[k].N, c->precision, bb[k], st); });
    }
    if (e == cudaSuccess) e = fork_join(pm, s, groups, mortar(1));
    if (e == cudaSuccess)
        e = fork_join(pm, s, buckets, [&](int k, cudaStream_t st) {
            return launch_volume(pm->b[k].N, c->precision, c->physics, c->volume_form, c->time_scheme, bb[k], stage,
                                 lam_slot, st);
        });
    return e;
}

// One step: dt from clock slot `slot` (filled by a fresh pass over u when
// fresh != 0), then the stages; the last stage refills slot 1.
cudaError_t p_step(const hs3d_pmesh *pm, const hs3d_solver_cfg *c, double *u, double *g, double dt, bool fresh,
                   cudaStream_t s)
{
    if (pm->an) return aniso_step(pm->an, c, u, g, dt, fresh, s);
    std::vector<Batch> bb = bucket_batches(pm, c, u, g, nullptr, true);
    cudaError_t e = cudaSuccess;
    if (fresh) {
        for (size_t k = 0; k < bb.size() && e == cudaSuccess; ++k) {
            if (!(dt > 0.0)) e = launch_lambda(pm->b[k].N, c->precision, c->physics, bb[k], 0, s);
            else if (c->precision != HS3D_FP64) e = launch_shadow(pm->b[k].N, bb[k], s);
        }
    }
    if (e == cudaSuccess)
        e = launch_pdt_finalize(pm->clks, pm->nb_n, (int)pm->b.size(), c->cfl, 8.0, 12.0, fresh ? 0 : 1,
                                dt > 0.0 ? dt : 0.0, s);
    const int ns = rk_stages(c->time_scheme);
    for (int k = 0; k < ns && e == cudaSuccess; ++k) e = p_stage(pm, c, bb, u, k, k == ns - 1 ? 1 : -1, s);
    return e;
}

hs3d_status p_check(const hs3d_pmesh *pm, const hs3d_solver_cfg *c)
{
    if (!pm) return fail(HS3D_ERR_INVALID, "pmesh is NULL");
    hs3d_status st = validate_cfg(c);
    if (st == HS3D_OK && pm->an && c->precision != HS3D_FP64)
        return fail(HS3D_ERR_UNSUPPORTED, "meshes with per-direction degrees run in FP64");
    return st;
}

}  // namespace

extern "C" {

hs3d_status hs3d_pmesh_create(const hs3d_mesh_desc *desc, const int *degree, hs3d_pmesh **out)
{
    if (!out) return fail(HS3D_ERR_INVALID, "out is NULL");
    *out = nullptr;
    return pmesh_build(desc, degree, out);
}

hs3d_status hs3d_pmesh_create3(const hs3d_mesh_desc *desc, const int *degree3, hs3d_pmesh **out)
{
    if (!out) return fail(HS3D_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!desc || !degree3) return fail(HS3D_ERR_INVALID, "desc or degree3 is NULL");
    if (desc->ex < 1 || desc->ey < 1 || desc->ez < 1) return fail(HS3D_ERR_INVALID, "element counts must be >= 1");
    const long long E = (long long)desc->ex * desc->ey * desc->ez;
    if (E > (1 << 24)) return fail(HS3D_ERR_UNSUPPORTED, "too many elements");
    bool iso = true;
    int Pmin = 99, Pmax = 0;
    for (long long t = 0; t < 3 * E; ++t) {
        if (degree3[t] < 1 || degree3[t] > kMaxN)
            return fail(HS3D_ERR_UNSUPPORTED, "degree %d (element %lld) outside 1..%d", degree3[t], t / 3, kMaxN);
        Pmin = degree3[t] < Pmin ? degree3[t] : Pmin;
        Pmax = degree3[t] > Pmax ? degree3[t] : Pmax;
        iso = iso && degree3[t] == degree3[3 * (t / 3)];
    }
    if (iso) {   // one degree per element: the bucketed path
        std::vector<int> deg(E);
        for (long long e = 0; e < E; ++e) deg[e] = degree3[3 * e];
        return pmesh_build(desc, deg.data(), out);
    }
    if (desc->node_xyz) return fail(HS3D_ERR_UNSUPPORTED, "per-element degrees take no node_xyz");
    if (desc->nodes != HS3D_NODES_LOBATTO)
        return fail(HS3D_ERR_UNSUPPORTED, "per-element degrees need Gauss-Lobatto nodes");
    hs3d_mesh_desc chk = *desc;
    chk.N = Pmax;
    hs3d_status st = validate_desc(&chk);
    if (st != HS3D_OK) return st;
    if (Pmin == 1 && desc->perturb_amp != 0.0)
        return fail(HS3D_ERR_INVALID, "a degree-1 direction allows only an affine map (perturb_amp = 0)");
    hs3d_pmesh *pm = new (std::nothrow) hs3d_pmesh();
    if (!pm) return fail(HS3D_ERR_NOMEM, "host allocation failed");
    pm->ex = desc->ex;
    pm->ey = desc->ey;
    pm->ez = desc->ez;
    pm->E = (int)E;
    pm->Nmin = Pmin;
    pm->Nmax = Pmax;
    for (int c = 0; c < 3; ++c) {
        pm->lo[c] = desc->lo[c];
        pm->hi[c] = desc->hi[c];
    }
    pm->amp = desc->perturb_amp;
    cudaError_t e = cudaStreamCreateWithFlags(&pm->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        pmesh_free(pm);
        return cuda_fail(e, "cudaStreamCreate");
    }
    st = aniso_build(desc, degree3, &pm->an);
    if (st != HS3D_OK) {
        pmesh_free(pm);
        return st;
    }
    pm->Ngeo = pm->an->Ngeo;
    pm->off = pm->an->off;
    *out = pm;
    return HS3D_OK;
}

void hs3d_pmesh_destroy(hs3d_pmesh *pm) { pmesh_free(pm); }

hs3d_status hs3d_pmesh_layout(const hs3d_pmesh *pm, int64_t *offset, int *Ngeo)
{
    if (!pm) return fail(HS3D_ERR_INVALID, "pmesh is NULL");
    if (offset) memcpy(offset, pm->off.data(), sizeof(int64_t) * (pm->E + 1));
    if (Ngeo) *Ngeo = pm->Ngeo;
    return HS3D_OK;
}

hs3d_status hs3d_pmesh_geometry(const hs3d_pmesh *pm, double *X, double *J, void *stream)
{
    if (!pm) return fail(HS3D_ERR_INVALID, "pmesh is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (pm->an) {
        const size_t nodes = (size_t)pm->an->noff[pm->E];
        if (X) e = cudaMemcpyAsync(X, pm->an->X, sizeof(double) * 3 * nodes, cudaMemcpyDeviceToDevice, s);
        if (J && e == cudaSuccess) e = cudaMemcpyAsync(J, pm->an->J, sizeof(double) * nodes, cudaMemcpyDeviceToDevice, s);
    }
    for (const auto &bk : pm->b) {
        const size_t en = (size_t)bk.E * bk.m->n3;
        const size_t nb = (size_t)bk.base / 5;   // node offset of the bucket (bases are multiples of 5)
        if (X && e == cudaSuccess)
            e = cudaMemcpyAsync(X + 3 * nb, bk.m->X, sizeof(double) * 3 * en, cudaMemcpyDeviceToDevice, s);
        if (J && e == cudaSuccess) e = cudaMemcpyAsync(J + nb, bk.m->J, sizeof(double) * en, cudaMemcpyDeviceToDevice, s);
    }
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "geometry copy");
}

hs3d_status hs3d_pmesh_init_state(const hs3d_pmesh *pm, const hs3d_ic *ic, double *u, void *stream)
{
    if (!pm || !ic) return fail(HS3D_ERR_INVALID, "pmesh or ic is NULL");
    hs3d_status st = check_ptr(u, "u");
    if (st != HS3D_OK) return st;
    {
        hs3d_pmesh *m = const_cast<hs3d_pmesh *>(pm);
        std::lock_guard<std::mutex> lock(m->mu);
        if (m->cont_u == u) m->cont_u = nullptr;   // the state itself is rewritten
    }
    if (pm->an) {
        cudaError_t e = aniso_init_state(pm->an, *ic, u, (cudaStream_t)stream);
        return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "init launch");
    }
    for (size_t k = 0; k < pm->b.size() && st == HS3D_OK; ++k)
        st = hs3d_init_state(pm->b[k].m, ic, u + pm->b[k].base, stream);
    return st;
}

// out[k] = sum over the buckets b, in bucket order, of tmp[b][k] (one thread:
// a fixed order, so the result is reproducible bit for bit).
__global__ void k_pdiag_sum(const double *tmp, int nb, double *out)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int k = 0; k < 7; ++k) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += tmp[b * 7 + k];
        out[k] = acc;
    }
}

hs3d_status hs3d_pmesh_diagnostics(const hs3d_pmesh *pm, const hs3d_solver_cfg *c, const double *u, const double *dudt,
                                   double *out, void *stream)
{
    hs3d_status st = p_check(pm, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK && dudt) st = check_ptr(dudt, "dudt");
    if (st == HS3D_OK && !out) st = fail(HS3D_ERR_INVALID, "out is NULL");
    if (st != HS3D_OK) return st;
    hs3d_pmesh *m = const_cast<hs3d_pmesh *>(pm);
    std::lock_guard<std::mutex> lock(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (pm->an) {
        e = aniso_diagnostics(pm->an, c, u, dudt, out, s);
        return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "diagnostics launch");
    }
    for (size_t k = 0; k < pm->b.size() && e == cudaSuccess; ++k) {
        const auto &bk = pm->b[k];
        const Item it = make_item(bk.m, c, u + bk.base, nullptr, nullptr);
        e = launch_diagnostics(bk.N, it, dudt ? dudt + bk.base : nullptr, bk.m->diag_partials,
                               diagnostics_blocks(bk.N, bk.E), pm->diag_tmp + 7 * k, s);
    }
    if (e == cudaSuccess) {
        k_pdiag_sum<<<1, 1, 0, s>>>(pm->diag_tmp, (int)pm->b.size(), out);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "diagnostics launch");
}

hs3d_status hs3d_pmesh_residual(const hs3d_pmesh *pm, const hs3d_solver_cfg *c, const double *u, double *dudt,
                                void *stream)
{
    hs3d_status st = p_check(pm, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK) st = check_ptr(dudt, "dudt");
    if (st != HS3D_OK) return st;
    if ((const void *)u == (const void *)dudt) return fail(HS3D_ERR_INVALID, "u and dudt must differ");
    hs3d_pmesh *m = const_cast<hs3d_pmesh *>(pm);
    std::lock_guard<std::mutex> lock(m->mu);
    cudaStream_t s = (cudaStream_t)stream;
    if (pm->an) {
        cudaError_t e = aniso_stage(pm->an, c, const_cast<double *>(u), nullptr, dudt, -1, -1, s);
        return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "residual launch");
    }
    std::vector<Batch> bb = bucket_batches(pm, c, u, nullptr, dudt, false);
    cudaError_t e = cudaSuccess;
    if (c->precision != HS3D_FP64) {
        if (m->cont_u != u) m->cont_u = nullptr;   // the FP32 shadow now holds another state
        for (size_t k = 0; k < bb.size() && e == cudaSuccess; ++k) e = launch_shadow(pm->b[k].N, bb[k], s);
    }
    if (e == cudaSuccess) e = p_stage(pm, c, bb, u, -1, -1, s);
    return e == cudaSuccess ? HS3D_OK : cuda_fail(e, "residual launch");
}

hs3d_status hs3d_pmesh_run(const hs3d_pmesh *pmc, const hs3d_solver_cfg *c, double *u, double *g, double dt,
                           int nsteps, void *stream)
{
    hs3d_status st = p_check(pmc, c);
    if (st == HS3D_OK) st = check_ptr(u, "u");
    if (st == HS3D_OK) st = check_ptr(g, "g");
    if (st != HS3D_OK) return st;
    if (u == g) return fail(HS3D_ERR_INVALID, "u and g must differ");
    if (nsteps < 0) return fail(HS3D_ERR_INVALID, "nsteps < 0");
    if (nsteps == 0) return HS3D_OK;
    hs3d_pmesh *pm = const_cast<hs3d_pmesh *>(pmc);
    std::lock_guard<std::mutex> lock(pm->mu);
    cudaStream_t s = (cudaStream_t)stream;
    // dt < 0: continue the state the previous run on this mesh advanced with this cfg
    const bool cont = dt < 0.0 && pm->cont_u == u && same_cfg(pm->cont_cfg, *c);
    if (dt < 0.0) dt = 0.0;
    pm->cont_u = nullptr;
    cudaError_t e = cudaSuccess;
    int replays = nsteps;
    if (!cont) {
        // the first step reads a fresh dt pass (or writes the FP32 shadow for a fixed dt)
        e = p_step(pm, c, u, g, dt, true, s);
        replays = nsteps - 1;
        if (e != cudaSuccess) return cuda_fail(e, "step launch");
    }
    if (replays == 0) {
        pm->cont_u = u;
        pm->cont_cfg = *c;
        return HS3D_OK;
    }
    // the remaining steps replay one captured step that continues from clock slot 1
    if (!(pm->gexec && pm->gu == u && pm->gg == g && pm->gdt == dt && same_cfg(pm->gcfg, *c))) {
        if (pm->gexec) cudaGraphExecDestroy(pm->gexec);
        pm->gexec = nullptr;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(pm->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = p_step(pm, c, u, g, dt, false, pm->stream);
            e = cudaStreamEndCapture(pm->stream, &graph);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&pm->gexec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            pm->gexec = nullptr;
            cudaGetLastError();
            return cuda_fail(e, "graph capture");
        }
        pm->gu = u;
        pm->gg = g;
        pm->gdt = dt;
        pm->gcfg = *c;
    }
    for (int k = 0; k < replays && e == cudaSuccess; ++k) e = cudaGraphLaunch(pm->gexec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    pm->cont_u = u;
    pm->cont_cfg = *c;
    return HS3D_OK;
}

hs3d_status hs3d_pmesh_clock(const hs3d_pmesh *pm, double *t, int64_t *steps, int reset, void *stream)
{
    if (!pm) return fail(HS3D_ERR_INVALID, "pmesh is NULL");
    if (reset) {   // the reset clears the dt maxima a continuing run would read
        hs3d_pmesh *m = const_cast<hs3d_pmesh *>(pm);
        std::lock_guard<std::mutex> lock(m->mu);
        m->cont_u = nullptr;
    }
    if (pm->an) {
        Clock h{};
        cudaStream_t s = (cudaStream_t)stream;
        cudaError_t e = cudaMemcpyAsync(&h, pm->an->clk, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && reset) {
            e = cudaMemsetAsync(pm->an->clk, 0, sizeof(Clock), s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) return cuda_fail(e, "clock read");
        if (t) *t = h.t;
        if (steps) *steps = h.step;
        if (h.bad) return fail(HS3D_ERR_NONPHYSICAL, "non-physical state detected (rho <= 0, p <= 0 or NaN)");
        return HS3D_OK;
    }
    hs3d_status worst = HS3D_OK;
    for (size_t k = 0; k < pm->b.size(); ++k) {
        double tk = 0.0;
        int64_t sk = 0;
        hs3d_status st = hs3d_clock(pm->b[k].m, &tk, &sk, reset, stream);
        if (st == HS3D_ERR_CUDA) return st;
        if (st != HS3D_OK && worst == HS3D_OK) worst = st;
        if (k == 0) {
            if (t) *t = tk;
            if (steps) *steps = sk;
        }
    }
    return worst;   // (its message set by hs3d_clock)
}

}  // extern "C"
