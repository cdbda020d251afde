// Gauss-Lobatto operators, mesh geometry and initial conditions.
//
// Geometry (Sec. 3.3): node coordinates of a periodic box with an optional
// smooth perturbation, the Jacobian J = det(dX/dxi) and the metric terms in
// the conservative curl form (Kopriva 2006), which satisfy the discrete
// metric identity sum_d D_d Ja^d = 0 and so preserve a free stream on curved
// elements:
//   Ja^i_c = D_{i+2}(X_l D_{i+1} X_m) - D_{i+1}(X_l D_{i+2} X_m),  (c,m,l) cyclic.
// All in FP64, one CTA per element, one thread per node.
#include <math.h>

#include <map>
#include <mutex>
#include <vector>

#include "ic.cuh"
#include "internal.cuh"

namespace hs3d {

// ---------------------------------------------------------------- 1-D operators

// L_{N-1}(x), L_N(x), L_{N+1}(x) by the three-term recurrence.
static void legendre3(int N, double x, double &Lm, double &L, double &Lp)
{
    double lkm1 = 1.0, lk = x, lkm2 = 0.0;   // L_{k-1}, L_k, L_{k-2} for k = 1
    for (int k = 1; k <= N; ++k) {
        double lkp1 = ((2.0 * k + 1.0) * x * lk - k * lkm1) / (k + 1.0);
        lkm2 = lkm1;
        lkm1 = lk;
        lk = lkp1;
    }
    Lm = lkm2;   // L_{N-1}
    L = lkm1;    // L_N
    Lp = lk;     // L_{N+1}
}

static Ops make_ops(int N)
{
    Ops o{};
    int n = N + 1;
    // Nodes: roots of q = L_{N+1} - L_{N-1}, q' = (2N+1) L_N (Newton from
    // Chebyshev-Gauss-Lobatto points), symmetrised.
    for (int j = 0; j < n; ++j) {
        double x = -cos(M_PI * j / N);
        if (j == 0) x = -1.0;
        if (j == N) x = 1.0;
        if (j != 0 && j != N) {
            for (int it = 0; it < 200; ++it) {
                double Lm, L, Lp;
                legendre3(N, x, Lm, L, Lp);
                double dx = (Lp - Lm) / ((2.0 * N + 1.0) * L);
                x -= dx;
                if (fabs(dx) <= 1e-17) break;
            }
        }
        o.xi[j] = x;
    }
    for (int j = 0; j < n / 2; ++j) {
        double s = 0.5 * (o.xi[N - j] - o.xi[j]);
        o.xi[j] = -s;
        o.xi[N - j] = s;
    }
    if (n % 2) o.xi[N / 2] = 0.0;
    double LN[kMaxn];
    for (int j = 0; j < n; ++j) {
        double Lm, L, Lp;
        legendre3(N, o.xi[j], Lm, L, Lp);
        LN[j] = L;
        o.w[j] = 2.0 / (N * (N + 1.0) * L * L);
    }
    // Derivative matrix in the closed form for Gauss-Lobatto nodes:
    //   D_ij = L_N(x_i) / (L_N(x_j) (x_i - x_j)), i != j;
    //   D_00 = -N(N+1)/4, D_NN = N(N+1)/4, other diagonal entries 0.
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double v;
            if (i != j) v = LN[i] / (LN[j] * (o.xi[i] - o.xi[j]));
            else if (i == 0) v = -0.25 * N * (N + 1.0);
            else if (i == N) v = 0.25 * N * (N + 1.0);
            else v = 0.0;
            o.D[i * n + j] = v;
            o.Df[i * n + j] = (float)v;
            o.Dlo[i * n + j] = (float)(v - (double)o.Df[i * n + j]);
        }
    o.iw0 = 1.0 / o.w[0];
    o.iw0f = (float)o.iw0;
    // boundary interpolation: the end nodes themselves
    o.gauss = 0;
    for (int j = 0; j < n; ++j) {
        o.lb[j] = (j == 0) ? 1.0 : 0.0;
        o.rb[j] = (j == N) ? 1.0 : 0.0;
        for (int s = 0; s < n; ++s) o.IL[j * n + s] = (j == s) ? 1.0 : 0.0;
    }
    return o;
}

// Gauss-Legendre operators for degree N (n = N+1 points):
//   nodes  roots of L_n by Newton (L_n' from L_n' (x^2 - 1) = n (x L_n - L_{n-1})),
//   weights 2 / ((1 - x^2) L_n'(x)^2),
//   D_ij = L_n'(x_i) / (L_n'(x_j) (x_i - x_j)) (i != j), D_ii = x_i / (1 - x_i^2)
//          (Legendre's equation at a root of L_n),
//   l_j(+1) = 1 / (L_n'(x_j) (1 - x_j)),  l_j(-1) = (-1)^n / (L_n'(x_j) (-1 - x_j)),
// and the Gauss-Lobatto basis of degree N at the Gauss points,
//   l^L_s(x) = (x^2 - 1) L_N'(x) / (N (N+1) L_N(x_s) (x - x_s)).
static Ops make_ops_gauss(int N)
{
    const Ops lob = make_ops(N);
    Ops o{};
    const int n = N + 1;
    double dL[kMaxn];
    for (int j = 0; j < n; ++j) {
        double x = -cos(M_PI * (j + 0.75) / (n + 0.5));
        double Lm, L, Lp, d = 1.0;
        for (int it = 0; it < 200; ++it) {
            legendre3(n, x, Lm, L, Lp);   // L = L_n, Lm = L_{n-1}
            d = n * (x * L - Lm) / (x * x - 1.0);
            const double dx = L / d;
            x -= dx;
            if (fabs(dx) <= 1e-17) break;
        }
        legendre3(n, x, Lm, L, Lp);
        d = n * (x * L - Lm) / (x * x - 1.0);
        o.xi[j] = x;
        dL[j] = d;
    }
    for (int j = 0; j < n / 2; ++j) {   // symmetrise
        const double s = 0.5 * (o.xi[N - j] - o.xi[j]);
        o.xi[j] = -s;
        o.xi[N - j] = s;
    }
    if (n % 2) o.xi[N / 2] = 0.0;
    for (int j = 0; j < n; ++j) {
        double Lm, L, Lp;
        legendre3(n, o.xi[j], Lm, L, Lp);
        dL[j] = n * (o.xi[j] * L - Lm) / (o.xi[j] * o.xi[j] - 1.0);
        o.w[j] = 2.0 / ((1.0 - o.xi[j] * o.xi[j]) * dL[j] * dL[j]);
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            const double v = (i != j) ? dL[i] / (dL[j] * (o.xi[i] - o.xi[j])) : o.xi[i] / (1.0 - o.xi[i] * o.xi[i]);
            o.D[i * n + j] = v;
            o.Df[i * n + j] = (float)v;
            o.Dlo[i * n + j] = (float)(v - (double)o.Df[i * n + j]);
        }
    o.iw0 = 0.0;
    o.iw0f = 0.0f;
    o.gauss = 1;
    const double sgn = (n % 2) ? -1.0 : 1.0;
    for (int j = 0; j < n; ++j) {
        o.rb[j] = 1.0 / (dL[j] * (1.0 - o.xi[j]));
        o.lb[j] = sgn / (dL[j] * (-1.0 - o.xi[j]));
    }
    for (int t = 0; t < n; ++t) {
        const double x = o.xi[t];
        double Lm, L, Lp;
        legendre3(N, x, Lm, L, Lp);   // L = L_N, Lm = L_{N-1}
        const double dLN = N * (x * L - Lm) / (x * x - 1.0);
        for (int s = 0; s < n; ++s) {
            const double xs = lob.xi[s];
            double v;
            if (fabs(x - xs) < 1e-15) {
                v = 1.0;   // a Gauss point on a Gauss-Lobatto node (x = 0 for even N)
            } else {
                double Lms, Ls, Lps;
                legendre3(N, xs, Lms, Ls, Lps);
                v = (x * x - 1.0) * dLN / (N * (N + 1.0) * Ls * (x - xs));
            }
            o.IL[t * n + s] = v;
        }
    }
    for (int j = 0; j < n; ++j) {
        if (fabs(o.xi[j]) < 1e-15)   // zero row except the coincident node
            for (int s = 0; s < n; ++s)
                if (fabs(lob.xi[s]) >= 1e-15) o.IL[j * n + s] = 0.0;
    }
    return o;
}

static void finish_ops(Ops &o, int n)
{
    for (int j = 0; j < n; ++j) {
        o.lbw[j] = o.lb[j] / o.w[j];
        o.rbw[j] = o.rb[j] / o.w[j];
        o.lbf[j] = (float)o.lb[j];
        o.rbf[j] = (float)o.rb[j];
        o.lbwf[j] = (float)o.lbw[j];
        o.rbwf[j] = (float)o.rbw[j];
    }
}

const Ops &host_ops(int N, int nodes)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, Ops> cache;
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(N, nodes);
    auto it = cache.find(key);
    if (it == cache.end()) {
        Ops o = (nodes == HS3D_NODES_GAUSS) ? make_ops_gauss(N) : make_ops(N);
        finish_ops(o, N + 1);
        it = cache.emplace(key, o).first;
    }
    return it->second;
}

const Ops *device_ops(int N, int nodes)
{
    static std::mutex mu;
    static std::map<std::pair<int, int>, Ops *> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    const Ops &h = host_ops(N, nodes);
    std::lock_guard<std::mutex> g(mu);
    auto key = std::make_pair(dev, N + 16 * nodes);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    Ops *d = nullptr;
    if (cudaMalloc(&d, sizeof(Ops)) != cudaSuccess) return nullptr;
    if (cudaMemcpy(d, &h, sizeof(Ops), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return nullptr;
    }
    cache[key] = d;
    return d;
}

// ---------------------------------------------------------------- geometry kernel

template <int N>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1))
k_geometry(const double *__restrict__ xyz, int ex, int ey, int ez, double lo0, double lo1, double lo2, double hi0,
           double hi1, double hi2, double amp, const Ops *__restrict__ ops, double *__restrict__ X,
           double *__restrict__ Ja, float *__restrict__ Jaf, double *__restrict__ J, double *__restrict__ invJ,
           float *__restrict__ invJf, double *__restrict__ fn, float *__restrict__ fnf, double *__restrict__ dXout)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    __shared__ double sD[n * n];
    __shared__ double sX[3][n3];
    __shared__ double sT[2][n3];
    const int e = blockIdx.x;
    const int E = ex * ey * ez;
    const int p = threadIdx.x;
    const int ijk[3] = {p % n, (p / n) % n, p / n2};
    for (int t = p; t < n * n; t += n3) sD[t] = ops->D[t];
    const double lo[3] = {lo0, lo1, lo2}, hi[3] = {hi0, hi1, hi2};
    const int ab[3] = {e % ex, (e / ex) % ey, e / (ex * ey)};
    const int Ed[3] = {ex, ey, ez};
    double x[3];
    if (xyz) {
        for (int c = 0; c < 3; ++c) x[c] = xyz[((size_t)e * 3 + c) * n3 + p];
    } else {
        double th[3];
        for (int c = 0; c < 3; ++c) {
            double L = hi[c] - lo[c];
            double h = L / Ed[c];
            x[c] = lo[c] + h * (ab[c] + 0.5 * (ops->xi[ijk[c]] + 1.0));
            th[c] = -M_PI + 2.0 * M_PI * (x[c] - lo[c]) / L;
        }
        double s = sin(th[0]) * sin(th[1]) * sin(th[2]);
        for (int c = 0; c < 3; ++c) x[c] += amp * ((hi[c] - lo[c]) / (2.0 * M_PI)) * s;
    }
    for (int c = 0; c < 3; ++c) sX[c][p] = x[c];
    __syncthreads();

    // a[d][c] = dX_c/dxi_d at this node
    auto deriv = [&](const double *f, int d) {
        double acc = 0.0;
        const int stride = (d == 0) ? 1 : (d == 1) ? n : n2;
        const int base = p - ijk[d] * stride;
        const double *Drow = sD + ijk[d] * n;
#pragma unroll
        for (int m = 0; m < n; ++m) acc += Drow[m] * f[base + m * stride];
        return acc;
    };
    double a[3][3];
    for (int d = 0; d < 3; ++d)
        for (int c = 0; c < 3; ++c) a[d][c] = deriv(sX[c], d);
    double Jp = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) + a[0][1] * (a[1][2] * a[2][0] - a[1][0] * a[2][2]) +
                a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
    J[(size_t)e * n3 + p] = Jp;
    invJ[(size_t)e * n3 + p] = 1.0 / Jp;
    invJf[(size_t)e * n3 + p] = (float)(1.0 / Jp);
    for (int c = 0; c < 3; ++c) X[((size_t)e * 3 + c) * n3 + p] = x[c];
    if (dXout)   // dX_c/dxi_d, [E][c*3 + d][n3] (Gauss-Legendre meshes evaluate it at their nodes)
        for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) dXout[((size_t)e * 9 + c * 3 + d) * n3 + p] = a[d][c];

    for (int i = 0; i < 3; ++i) {
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        for (int c = 0; c < 3; ++c) {
            const int m = (c + 1) % 3, l = (c + 2) % 3;
            __syncthreads();
            sT[0][p] = x[l] * a[i1][m];
            sT[1][p] = x[l] * a[i2][m];
            __syncthreads();
            double v = deriv(sT[0], i2) - deriv(sT[1], i1);
            Ja[(((size_t)e * 3 + i) * 3 + c) * n3 + p] = v;
            Jaf[(((size_t)e * 3 + i) * 3 + c) * n3 + p] = (float)v;
            if (ijk[i] == N) {
                // tangential (a,b) index of this node on the +i face
                int ta = (i == 0) ? ijk[1] : ijk[0];
                int tb = (i == 2) ? ijk[1] : ijk[2];
                fn[(((size_t)i * E + e) * 3 + c) * n2 + ta + n * tb] = v;
                fnf[(((size_t)i * E + e) * 3 + c) * n2 + ta + n * tb] = (float)v;
            }
        }
    }
}

// Gauss-Legendre meshes: the element map, the curl-form metric polynomials
// and dX/dxi come from the Gauss-Lobatto construction above; here they are
// evaluated at the Gauss points by tensor-product interpolation (three 1-D
// passes with the Gauss-Lobatto basis, exact for these degree-N
// polynomials), and J = det(dX/dxi) is formed there.
template <int N>
__global__ void __launch_bounds__((N + 1) * (N + 1) * (N + 1))
k_geometry_gauss(const double *__restrict__ XL, const double *__restrict__ JaL, const double *__restrict__ dXL,
                 const Ops *__restrict__ ops, double *__restrict__ X, double *__restrict__ Ja, float *__restrict__ Jaf,
                 double *__restrict__ J, double *__restrict__ invJ, float *__restrict__ invJf)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    __shared__ double sI[n * n];
    __shared__ double sA[n3], sB[n3];
    const int e = blockIdx.x;
    const int p = threadIdx.x;
    const int i = p % n, j = (p / n) % n, k = p / n2;
    for (int t = p; t < n * n; t += n3) sI[t] = ops->IL[t];
    double dx[9];
    for (int f = 0; f < 21; ++f) {
        const double *src = (f < 3) ? XL + ((size_t)e * 3 + f) * n3
                          : (f < 12) ? JaL + ((size_t)e * 9 + (f - 3)) * n3
                                     : dXL + ((size_t)e * 9 + (f - 12)) * n3;
        __syncthreads();
        sA[p] = src[p];
        __syncthreads();
        double acc = 0.0;
        for (int s = 0; s < n; ++s) acc += sI[i * n + s] * sA[s + n * (j + n * k)];
        sB[p] = acc;
        __syncthreads();
        acc = 0.0;
        for (int s = 0; s < n; ++s) acc += sI[j * n + s] * sB[i + n * (s + n * k)];
        sA[p] = acc;
        __syncthreads();
        acc = 0.0;
        for (int s = 0; s < n; ++s) acc += sI[k * n + s] * sA[i + n * (j + n * s)];
        if (f < 3) {
            X[((size_t)e * 3 + f) * n3 + p] = acc;
        } else if (f < 12) {
            Ja[((size_t)e * 9 + (f - 3)) * n3 + p] = acc;
            Jaf[((size_t)e * 9 + (f - 3)) * n3 + p] = (float)acc;
        } else {
            dx[f - 12] = acc;
        }
    }
    // a[d][c] = dx[c*3 + d]
    const double Jp = dx[0] * (dx[4] * dx[8] - dx[7] * dx[5]) + dx[3] * (dx[7] * dx[2] - dx[1] * dx[8]) +
                      dx[6] * (dx[1] * dx[5] - dx[4] * dx[2]);
    J[(size_t)e * n3 + p] = Jp;
    invJ[(size_t)e * n3 + p] = 1.0 / Jp;
    invJf[(size_t)e * n3 + p] = (float)(1.0 / Jp);
}

// Face metrics at the face Gauss points: the Gauss-Lobatto face values of
// Ja^d (which both neighbours share) interpolated in the two tangential
// directions.  One thread per (d, e, c, face point).
__global__ void k_facemetric_gauss(int n, long long total, const double *__restrict__ fnL, const Ops *__restrict__ ops,
                                   double *__restrict__ fn, float *__restrict__ fnf)
{
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    const int n2 = n * n;
    const int ab = (int)(t % n2);
    const long long row = t / n2;   // (d*E + e)*3 + c
    const int ta = ab % n, tb = ab / n;
    const double *F = fnL + row * n2;
    double acc = 0.0;
    for (int b = 0; b < n; ++b) {
        double r = 0.0;
        for (int a = 0; a < n; ++a) r += ops->IL[ta * n + a] * F[a + n * b];
        acc += ops->IL[tb * n + b] * r;
    }
    fn[t] = acc;
    fnf[t] = (float)acc;
}

cudaError_t launch_geometry(int N, int nodes, const double *node_xyz_dev, int ex, int ey, int ez, const double *lo,
                            const double *hi, double amp, double *X, double *Ja, float *Jaf, double *J, double *invJ,
                            float *invJf, double *fn, float *fnf, cudaStream_t s)
{
    const Ops *ops = device_ops(N, HS3D_NODES_LOBATTO);
    if (!ops) return cudaErrorMemoryAllocation;
    const int E = ex * ey * ez;
    const int n = N + 1, n2 = n * n, n3 = n2 * n;
    const bool gauss = nodes == HS3D_NODES_GAUSS;
    double *XL = X, *JaL = Ja, *fnL = fn, *dXL = nullptr;
    if (gauss) {
        const Ops *opsg = device_ops(N, HS3D_NODES_GAUSS);
        if (!opsg) return cudaErrorMemoryAllocation;
        XL = JaL = fnL = dXL = nullptr;
        cudaError_t e = cudaMalloc(&XL, sizeof(double) * (size_t)E * 3 * n3);
        if (e == cudaSuccess) e = cudaMalloc(&JaL, sizeof(double) * (size_t)E * 9 * n3);
        if (e == cudaSuccess) e = cudaMalloc(&dXL, sizeof(double) * (size_t)E * 9 * n3);
        if (e == cudaSuccess) e = cudaMalloc(&fnL, sizeof(double) * (size_t)3 * E * 3 * n2);
        if (e != cudaSuccess) {
            cudaFree(XL);
            cudaFree(JaL);
            cudaFree(dXL);
            cudaFree(fnL);
            return e;
        }
    }
#define HS3D_GEO(NN)                                                                                            \
    case NN:                                                                                                    \
        k_geometry<NN><<<E, n3, 0, s>>>(node_xyz_dev, ex, ey, ez, lo[0], lo[1], lo[2], hi[0], hi[1], hi[2], amp, \
                                        ops, XL, JaL, Jaf, J, invJ, invJf, fnL, fnf, dXL);                      \
        if (gauss)                                                                                              \
            k_geometry_gauss<NN><<<E, n3, 0, s>>>(XL, JaL, dXL, device_ops(N, HS3D_NODES_GAUSS), X, Ja, Jaf, J,  \
                                                  invJ, invJf);                                                 \
        break;
    cudaError_t e = cudaSuccess;
    switch (N) {
        HS3D_GEO(1) HS3D_GEO(2) HS3D_GEO(3) HS3D_GEO(4) HS3D_GEO(5) HS3D_GEO(6) HS3D_GEO(7)
        default: e = cudaErrorInvalidValue;
    }
#undef HS3D_GEO
    if (e == cudaSuccess) e = cudaGetLastError();
    if (gauss) {
        const long long total = 3LL * E * 3 * n2;
        if (e == cudaSuccess)
            k_facemetric_gauss<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(
                n, total, fnL, device_ops(N, HS3D_NODES_GAUSS), fn, fnf);
        if (e == cudaSuccess) e = cudaGetLastError();
        cudaError_t e2 = cudaStreamSynchronize(s);   // the temporaries are freed below
        if (e == cudaSuccess) e = e2;
        cudaFree(XL);
        cudaFree(JaL);
        cudaFree(dXL);
        cudaFree(fnL);
    }
    return e;
}

// ---------------------------------------------------------------- initial conditions

// Isentropic vortex (Shu) and Taylor-Green vortex at the mesh nodes.
__global__ void k_init_state(int n3, long long total, const double *__restrict__ X, hs3d_ic ic, double Lx, double Ly,
                             double *__restrict__ u)
{
    long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= total) return;
    long long e = t / n3;
    int p = (int)(t % n3);
    const double x = X[(e * 3 + 0) * n3 + p], y = X[(e * 3 + 1) * n3 + p], z = X[(e * 3 + 2) * n3 + p];
    double w[5];
    ic_point(ic, Lx, Ly, x, y, z, w);
    double *ue = u + e * 5 * n3 + p;
#pragma unroll
    for (int v = 0; v < 5; ++v) ue[(size_t)v * n3] = w[v];
}

cudaError_t launch_init_state(int N, int E, const double *X, const hs3d_ic &ic, const double *lo, const double *hi,
                              double *u, cudaStream_t s)
{
    int n3 = (N + 1) * (N + 1) * (N + 1);
    long long total = (long long)E * n3;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    k_init_state<<<(unsigned)blocks, threads, 0, s>>>(n3, total, X, ic, hi[0] - lo[0], hi[1] - lo[1], u);
    return cudaGetLastError();
}

// Low part of the FP32 metric terms: Jalo = Ja - Jaf rounded to FP32.
__global__ void k_metric_lo(const double *__restrict__ Ja, const float *__restrict__ Jaf, float *__restrict__ Jalo,
                            long long count)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < count) Jalo[i] = (float)(Ja[i] - (double)Jaf[i]);
}

cudaError_t launch_metric_lo(const double *Ja, const float *Jaf, float *Jalo, long long count, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    k_metric_lo<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(Ja, Jaf, Jalo, count);
    return cudaGetLastError();
}

}  // namespace hs3d
