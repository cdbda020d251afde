/*
 * hs3d oracle -- a plain, slow FP64 CPU implementation of the DGSEM residual
 * and the Williamson low-storage RK3 step for the compressible Euler and
 * Navier-Stokes equations on periodic curvilinear hexahedral boxes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call this file:
 * only the tests, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Everything is computed in the order the method states it, with one loop per
 * formula.  Sources (HORSES3D paper, arXiv 2206.09733):
 *   - conservative variables, Euler flux F_e, viscous flux F_v  (Sec. 3.2,
 *     Eq. compressibleNScompact and Eq. viscousfluxes)
 *   - mapped equations J u_t + div_xi F~ = 0 with contravariant fluxes
 *     (Sec. 3.3, Eq. compressibleNScompact_transformed)
 *   - weak form with a numerical flux at element faces, Gauss-Lobatto
 *     quadrature (Sec. 3.3, Eqs. NS2-NS5)
 *   - Lax-Friedrichs, Rusanov, Roe, low-dissipation Roe, matrix-dissipation
 *     and central surface fluxes, BR1 viscous scheme (Sec. 3.3, list of
 *     convective and viscous fluxes)
 *   - split forms: Chandrashekar, Kennedy-Gruber, Pirozzoli, Ducros,
 *     Morinishi, entropy conserving (Ismail-Roe) (Sec. 3.5)
 *   - entropy S = -rho s, s = ln p - gamma ln rho, w = dS/du (Sec. 4.4,
 *     Eq. shock:entropy)
 *   - Williamson low-storage RK3 (Sec. 3.7)
 * The paper prints no formula for the fluxes, the split form, the RK
 * coefficients, the metric terms, the time-step rule or BR1; those are the
 * published methods it cites, restated here (each function says which).
 *
 * Layout (shared with callers, not with the CUDA code): polynomial degree N
 * (the paper's P), n = N+1 Gauss-Lobatto nodes per direction, node
 * (i,j,k) -> i + n*(j + n*k).  State u[e][v][node] with v = rho, rho v1,
 * rho v2, rho v3, rho e.  Node coordinates X[e][c][node].  Metric terms
 * Ja[e][d][c][node] = J * d xi_d / d x_c, Jacobian J[e][node].
 * Elements of an ex*ey*ez box: e = a + ex*(b + ey*c), all faces periodic.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NVAR 5
#define NGRAD 4 /* gradient variables q = (v1, v2, v3, T) */

void orc_flux_roe_signed(const double *uL, const double *uR, const double *nh, double g, double *f, int sign_mode);
void orc_flux_ec(const double *uL, const double *uR, const double *a, double g, double *f);
double orc_logmean(double a, double b);

/* ------------------------------------------------------------------------ */
/* 1-D Gauss-Lobatto operators (Sec. 3.3: GL quadrature)                    */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial L_N(x) and its derivative by the three-term recurrence. */
static void legendre_and_derivative(int N, double x, double *L, double *dL)
{
    double Lm1 = 1.0, L0 = x;          /* L_0, L_1 */
    double dLm1 = 0.0, dL0 = 1.0;
    if (N == 0) { *L = 1.0; *dL = 0.0; return; }
    for (int k = 2; k <= N; ++k) {
        double Lk = ((2.0 * k - 1.0) * x * L0 - (k - 1.0) * Lm1) / k;
        double dLk = dLm1 + (2.0 * k - 1.0) * L0;   /* L_k' = L_{k-2}' + (2k-1) L_{k-1} */
        Lm1 = L0; L0 = Lk;
        dLm1 = dL0; dL0 = dLk;
    }
    *L = L0; *dL = dL0;
}

/* Gauss-Lobatto nodes: -1, +1 and the roots of L_N'.  Newton on L_N' with the
 * second derivative taken from Legendre's equation
 *   (1-x^2) L'' - 2x L' + N(N+1) L = 0.
 * Weights w_i = 2 / (N(N+1) L_N(x_i)^2).  Nodes in ascending order. */
int orc_lgl(int N, double *x, double *w)
{
    if (N < 1) return -1;
    int n = N + 1;
    for (int j = 0; j < n; ++j) {
        double xj;
        if (j == 0) xj = -1.0;
        else if (j == N) xj = 1.0;
        else {
            xj = -cos(M_PI * j / N);     /* Chebyshev-Gauss-Lobatto start */
            for (int it = 0; it < 100; ++it) {
                double L, dL;
                legendre_and_derivative(N, xj, &L, &dL);
                double d2L = (2.0 * xj * dL - N * (N + 1.0) * L) / (1.0 - xj * xj);
                double dx = dL / d2L;
                xj -= dx;
                if (fabs(dx) < 1e-16) break;
            }
        }
        double L, dL;
        legendre_and_derivative(N, xj, &L, &dL);
        x[j] = xj;
        w[j] = 2.0 / (N * (N + 1.0) * L * L);
    }
    return 0;
}

/* Nodal derivative matrix D_ij = l_j'(x_i) from barycentric weights
 * lambda_j = 1 / prod_{k != j} (x_j - x_k):
 *   D_ij = (lambda_j / lambda_i) / (x_i - x_j),   i != j
 *   D_ii = - sum_{j != i} D_ij.
 * D is stored row-major: D[i*n + j]. */
int orc_dmatrix(int N, const double *x, double *D)
{
    int n = N + 1;
    double lam[16];
    if (n > 16) return -1;
    for (int j = 0; j < n; ++j) {
        double p = 1.0;
        for (int k = 0; k < n; ++k) if (k != j) p *= (x[j] - x[k]);
        lam[j] = 1.0 / p;
    }
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            D[i * n + j] = (lam[j] / lam[i]) / (x[i] - x[j]);
            s += D[i * n + j];
        }
        D[i * n + i] = -s;
    }
    return 0;
}

/* Gauss-Legendre nodes (Sec. 3.3: the solver allows Gauss or Gauss-Lobatto
 * quadrature points): the n = N+1 roots of L_n, by Newton from the estimate
 * cos(pi (4j + 3) / (4n + 2)), weights w_j = 2 / ((1 - x_j^2) L_n'(x_j)^2).
 * Ascending order. */
int orc_gauss(int N, double *x, double *w)
{
    if (N < 0) return -1;
    int n = N + 1;
    for (int j = 0; j < n; ++j) {
        double xj = cos(M_PI * (4.0 * j + 3.0) / (4.0 * n + 2.0));
        for (int it = 0; it < 100; ++it) {
            double L, dL;
            legendre_and_derivative(n, xj, &L, &dL);
            double dx = L / dL;
            xj -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        double L, dL;
        legendre_and_derivative(n, xj, &L, &dL);
        x[n - 1 - j] = xj;
        w[n - 1 - j] = 2.0 / ((1.0 - xj * xj) * dL * dL);
    }
    return 0;
}

/* Lagrange basis of the nodes x[0..n-1] at the point y:
 *   l_j(y) = prod_{k != j} (y - x_k) / (x_j - x_k). */
void orc_lagrange_at(int n, const double *x, double y, double *l)
{
    for (int j = 0; j < n; ++j) {
        double p = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) p *= (y - x[k]) / (x[j] - x[k]);
        l[j] = p;
    }
}

/* ------------------------------------------------------------------------ */
/* Mesh: periodic box of ex*ey*ez hexahedra, optional smooth perturbation    */
/* ------------------------------------------------------------------------ */

typedef struct {
    int ex, ey, ez, N;
    double lo[3], hi[3];
    double amp;   /* x_c += amp*(L_c/2pi)*sin(t_x)sin(t_y)sin(t_z), t = box mapped to [-pi,pi] */
    int nodes;    /* solution nodes: 0 Gauss-Lobatto, 1 Gauss-Legendre */
} orc_box;

typedef struct {
    orc_box box;
    int n, n3, E;
    double xi[16], w[16], D[256];   /* solution nodes, weights, derivative matrix */
    double lb[16], rb[16];          /* l_j(-1), l_j(+1) of the solution nodes */
    double *X;    /* [E][3][n3] at the solution nodes */
    double *Ja;   /* [E][3][3][n3] */
    double *J;    /* [E][n3] */
    double *Sf;   /* [E][3 d][2 side][3 c][n2]: the element's own Ja^d on its faces xi_d = -1, +1 */
} orc_mesh;

static int node_index(int n, int i, int j, int k) { return i + n * (j + n * k); }

/* Element neighbour across face (d, side), side = +1 or -1, periodic wrap. */
static int neighbour(const orc_box *b, int e, int d, int side)
{
    int ab[3];
    int E3[3] = {b->ex, b->ey, b->ez};
    ab[0] = e % b->ex;
    ab[1] = (e / b->ex) % b->ey;
    ab[2] = e / (b->ex * b->ey);
    ab[d] = (ab[d] + side + E3[d]) % E3[d];
    return ab[0] + b->ex * (ab[1] + b->ey * ab[2]);
}

int orc_neighbour(const orc_mesh *m, int e, int d, int side)
{
    return neighbour(&m->box, e, d, side);
}

/* Gauss-Lobatto node coordinates of every element:
 *   x_c = lo_c + h_c*(index_c + (xi+1)/2)
 * then the smooth displacement (same scalar for every coordinate, scaled by the
 * box length so that [-pi,pi]^3 gets exactly amp*sin(x)sin(y)sin(z)), evaluated
 * at the unperturbed position. */
static void box_nodes(const orc_box *b, const double *xi, double *X)
{
    int n = b->N + 1, n3 = n * n * n;
    int E3[3] = {b->ex, b->ey, b->ez};
    int E = b->ex * b->ey * b->ez;
    for (int e = 0; e < E; ++e) {
        int ab[3] = {e % b->ex, (e / b->ex) % b->ey, e / (b->ex * b->ey)};
        for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            int ijk[3] = {i, j, k};
            double x0[3], th[3];
            for (int c = 0; c < 3; ++c) {
                double L = b->hi[c] - b->lo[c];
                double h = L / E3[c];
                x0[c] = b->lo[c] + h * (ab[c] + 0.5 * (xi[ijk[c]] + 1.0));
                th[c] = -M_PI + 2.0 * M_PI * (x0[c] - b->lo[c]) / L;
            }
            double s = sin(th[0]) * sin(th[1]) * sin(th[2]);
            for (int c = 0; c < 3; ++c) {
                double L = b->hi[c] - b->lo[c];
                X[(e * 3 + c) * n3 + node_index(n, i, j, k)] = x0[c] + b->amp * (L / (2.0 * M_PI)) * s;
            }
        }
    }
}

/* Derivative along reference direction d of a nodal field f (one element):
 * (D_d f)_ijk = sum_m D[ind_d][m] f(node with ind_d -> m). */
static double dir_derivative(int n, const double *D, const double *f, int d, int i, int j, int k)
{
    double s = 0.0;
    for (int m = 0; m < n; ++m) {
        int idx;
        if (d == 0) idx = node_index(n, m, j, k);
        else if (d == 1) idx = node_index(n, i, m, k);
        else idx = node_index(n, i, j, m);
        int row = (d == 0) ? i : (d == 1) ? j : k;
        s += D[row * n + m] * f[idx];
    }
    return s;
}

/* Metric terms in the conservative curl form (Kopriva 2006, the
 * free-stream-preserving form for curved DGSEM; Sec. 3.3 "contravariant
 * fluxes"): for reference direction i and physical component c with
 * (c, m, l) cyclic,
 *   Ja^i_c = d/dxi_{i+2} ( X_l dX_m/dxi_{i+1} ) - d/dxi_{i+1} ( X_l dX_m/dxi_{i+2} ),
 * indices mod 3, the products taken pointwise at the nodes (interpolation onto
 * degree N).  J = det(dX/dxi) with the derivatives from D. */
int orc_metrics(int E, int N, const double *D, const double *X, double *Ja, double *J)
{
    int n = N + 1, n3 = n * n * n;
    double *tmp = (double *)malloc(sizeof(double) * n3 * 2);
    double *dX = (double *)malloc(sizeof(double) * n3 * 9);   /* dX[c][d][node] */
    if (!tmp || !dX) { free(tmp); free(dX); return -1; }
    for (int e = 0; e < E; ++e) {
        const double *Xe = X + (size_t)e * 3 * n3;
        /* dX_c / dxi_d at every node */
        for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d)
        for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i)
            dX[(c * 3 + d) * n3 + node_index(n, i, j, k)] =
                dir_derivative(n, D, Xe + c * n3, d, i, j, k);
        /* J = a1 . (a2 x a3), a_d = dX/dxi_d */
        for (int p = 0; p < n3; ++p) {
            double a[3][3];
            for (int d = 0; d < 3; ++d) for (int c = 0; c < 3; ++c) a[d][c] = dX[(c * 3 + d) * n3 + p];
            double cx = a[1][1] * a[2][2] - a[1][2] * a[2][1];
            double cy = a[1][2] * a[2][0] - a[1][0] * a[2][2];
            double cz = a[1][0] * a[2][1] - a[1][1] * a[2][0];
            J[(size_t)e * n3 + p] = a[0][0] * cx + a[0][1] * cy + a[0][2] * cz;
        }
        for (int i = 0; i < 3; ++i) {
            int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
            for (int c = 0; c < 3; ++c) {
                int m = (c + 1) % 3, l = (c + 2) % 3;
                /* tmp0 = X_l dX_m/dxi_{i1},  tmp1 = X_l dX_m/dxi_{i2} */
                for (int p = 0; p < n3; ++p) {
                    tmp[p] = Xe[l * n3 + p] * dX[(m * 3 + i1) * n3 + p];
                    tmp[n3 + p] = Xe[l * n3 + p] * dX[(m * 3 + i2) * n3 + p];
                }
                for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int ii = 0; ii < n; ++ii) {
                    int p = node_index(n, ii, j, k);
                    double v = dir_derivative(n, D, tmp, i2, ii, j, k)
                             - dir_derivative(n, D, tmp + n3, i1, ii, j, k);
                    Ja[(((size_t)e * 3 + i) * 3 + c) * n3 + p] = v;
                }
            }
        }
    }
    free(tmp); free(dX);
    return 0;
}

/* Tangential directions of face direction d (in increasing order) and the
 * face node index ab = t0 + n*t1. */
static void face_dirs(int d, int *d0, int *d1)
{
    *d0 = (d == 0) ? 1 : 0;
    *d1 = (d == 2) ? 1 : 2;
}

/* Interpolate a nodal field of one element along direction d with the
 * matrix I[t*n + s] (target node t from source node s). */
static void interp_dir(int n, const double *I, const double *fs, double *ft, int d)
{
    for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
        int ijk[3] = {i, j, k};
        double acc = 0.0;
        for (int s = 0; s < n; ++s) {
            int src[3] = {i, j, k};
            src[d] = s;
            acc += I[ijk[d] * n + s] * fs[node_index(n, src[0], src[1], src[2])];
        }
        ft[node_index(n, i, j, k)] = acc;
    }
}

/* Tensor-product interpolation of an n^3 nodal field (three 1-D passes). */
static void interp3(int n, const double *I, const double *fs, double *ft, double *tmp)
{
    interp_dir(n, I, fs, ft, 0);
    interp_dir(n, I, ft, tmp, 1);
    interp_dir(n, I, tmp, ft, 2);
}

/* Build a mesh.  If X_in is given ([E][3][n3], at the Gauss-Lobatto nodes) it
 * replaces the box generator.
 *
 * Gauss-Lobatto solution nodes: the geometry, metric terms and J live on the
 * same nodes; the face metrics Sf are the metric terms at the boundary nodes.
 *
 * Gauss-Legendre solution nodes: the geometry is the degree-N interpolant of
 * the map through the Gauss-Lobatto nodes (neighbours share their face
 * nodes, so the mesh is watertight).  The curl-form metric terms are formed
 * on that grid; each Ja^d is then a polynomial of degree N per direction
 * whose divergence vanishes identically, so its values at the Gauss nodes
 * (exact Lobatto-to-Gauss interpolation) satisfy the discrete metric
 * identity there, and its values on a face depend only on the face's
 * Lobatto nodes, which both neighbours share.  X and J = det(dX/dxi) are the
 * geometry polynomial and its derivatives evaluated at the Gauss nodes; the
 * face metrics Sf are the face values interpolated to the face's Gauss
 * points. */
orc_mesh *orc_mesh_create(const orc_box *b, const double *X_in)
{
    if (b->N < 1 || b->N > 15 || b->ex < 1 || b->ey < 1 || b->ez < 1) return NULL;
    if (b->nodes != 0 && b->nodes != 1) return NULL;
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    if (!m) return NULL;
    m->box = *b;
    int N = b->N, n = N + 1, n2 = n * n, n3 = n2 * n;
    m->n = n;
    m->n3 = n3;
    m->E = b->ex * b->ey * b->ez;
    double xL[16], wL[16], DL[256];
    orc_lgl(N, xL, wL);
    orc_dmatrix(N, xL, DL);
    if (b->nodes == 1) orc_gauss(N, m->xi, m->w);
    else { memcpy(m->xi, xL, sizeof(double) * n); memcpy(m->w, wL, sizeof(double) * n); }
    orc_dmatrix(N, m->xi, m->D);
    orc_lagrange_at(n, m->xi, -1.0, m->lb);
    orc_lagrange_at(n, m->xi, 1.0, m->rb);
    size_t en = (size_t)m->E * n3;
    m->X = (double *)malloc(sizeof(double) * en * 3);
    m->Ja = (double *)malloc(sizeof(double) * en * 9);
    m->J = (double *)malloc(sizeof(double) * en);
    m->Sf = (double *)malloc(sizeof(double) * (size_t)m->E * 18 * n2);
    double *XL = (double *)malloc(sizeof(double) * en * 3);
    double *JaL = (double *)malloc(sizeof(double) * en * 9);
    double *JL = (double *)malloc(sizeof(double) * en);
    if (!m->X || !m->Ja || !m->J || !m->Sf || !XL || !JaL || !JL) {
        free(m->X); free(m->Ja); free(m->J); free(m->Sf); free(XL); free(JaL); free(JL); free(m);
        return NULL;
    }
    if (X_in) memcpy(XL, X_in, sizeof(double) * en * 3);
    else box_nodes(b, xL, XL);
    orc_metrics(m->E, N, DL, XL, JaL, JL);
    if (b->nodes == 0) {
        memcpy(m->X, XL, sizeof(double) * en * 3);
        memcpy(m->Ja, JaL, sizeof(double) * en * 9);
        memcpy(m->J, JL, sizeof(double) * en);
    } else {
        double I[256], tmp[4096], dX[4096];
        for (int t = 0; t < n; ++t) orc_lagrange_at(n, xL, m->xi[t], I + t * n);
        for (int e = 0; e < m->E; ++e) {
            for (int c = 0; c < 3; ++c)
                interp3(n, I, XL + ((size_t)e * 3 + c) * n3, m->X + ((size_t)e * 3 + c) * n3, tmp);
            for (int k9 = 0; k9 < 9; ++k9)
                interp3(n, I, JaL + ((size_t)e * 9 + k9) * n3, m->Ja + ((size_t)e * 9 + k9) * n3, tmp);
            /* a_d = dX/dxi_d of the geometry polynomial at the Gauss nodes */
            double *dXG = (double *)malloc(sizeof(double) * 9 * n3);
            for (int c = 0; c < 3; ++c)
            for (int d = 0; d < 3; ++d) {
                for (int kk = 0; kk < n; ++kk) for (int jj = 0; jj < n; ++jj) for (int ii = 0; ii < n; ++ii)
                    dX[node_index(n, ii, jj, kk)] = dir_derivative(n, DL, XL + ((size_t)e * 3 + c) * n3, d, ii, jj, kk);
                interp3(n, I, dX, dXG + (c * 3 + d) * n3, tmp);
            }
            for (int p = 0; p < n3; ++p) {
                double A[3][3];
                for (int d = 0; d < 3; ++d) for (int c = 0; c < 3; ++c) A[d][c] = dXG[(c * 3 + d) * n3 + p];
                double cx = A[1][1] * A[2][2] - A[1][2] * A[2][1];
                double cy = A[1][2] * A[2][0] - A[1][0] * A[2][2];
                double cz = A[1][0] * A[2][1] - A[1][1] * A[2][0];
                m->J[(size_t)e * n3 + p] = A[0][0] * cx + A[0][1] * cy + A[0][2] * cz;
            }
            free(dXG);
        }
    }
    /* own face metrics: Ja^d at the Lobatto boundary nodes xi_d = -1 (side 0)
     * and +1 (side 1), interpolated to the face points of the solution nodes */
    double I2[256];
    for (int t = 0; t < n; ++t) orc_lagrange_at(n, xL, m->xi[t], I2 + t * n);
    for (int e = 0; e < m->E; ++e)
    for (int d = 0; d < 3; ++d)
    for (int side = 0; side < 2; ++side)
    for (int c = 0; c < 3; ++c) {
        int d0, d1;
        face_dirs(d, &d0, &d1);
        double fL[256];
        for (int tb = 0; tb < n; ++tb) for (int ta = 0; ta < n; ++ta) {
            int idx[3];
            idx[d] = side ? N : 0;
            idx[d0] = ta;
            idx[d1] = tb;
            fL[ta + n * tb] = JaL[(((size_t)e * 3 + d) * 3 + c) * n3 + node_index(n, idx[0], idx[1], idx[2])];
        }
        double *out = m->Sf + ((((size_t)e * 3 + d) * 2 + side) * 3 + c) * n2;
        if (b->nodes == 0) { memcpy(out, fL, sizeof(double) * n2); continue; }
        double t1[256];
        for (int tb = 0; tb < n; ++tb) for (int ta = 0; ta < n; ++ta) {
            double acc = 0.0;
            for (int s = 0; s < n; ++s) acc += I2[ta * n + s] * fL[s + n * tb];
            t1[ta + n * tb] = acc;
        }
        for (int tb = 0; tb < n; ++tb) for (int ta = 0; ta < n; ++ta) {
            double acc = 0.0;
            for (int s = 0; s < n; ++s) acc += I2[tb * n + s] * t1[ta + n * s];
            out[ta + n * tb] = acc;
        }
    }
    free(XL); free(JaL); free(JL);
    return m;
}

void orc_mesh_destroy(orc_mesh *m)
{
    if (!m) return;
    free(m->X); free(m->Ja); free(m->J); free(m->Sf); free(m);
}

int orc_mesh_E(const orc_mesh *m) { return m->E; }
void orc_mesh_arrays(const orc_mesh *m, double *xi, double *w, double *D, double *X, double *Ja, double *J)
{
    size_t en = (size_t)m->E * m->n3;
    if (xi) memcpy(xi, m->xi, sizeof(double) * m->n);
    if (w) memcpy(w, m->w, sizeof(double) * m->n);
    if (D) memcpy(D, m->D, sizeof(double) * m->n * m->n);
    if (X) memcpy(X, m->X, sizeof(double) * en * 3);
    if (Ja) memcpy(Ja, m->Ja, sizeof(double) * en * 9);
    if (J) memcpy(J, m->J, sizeof(double) * en);
}

/* ------------------------------------------------------------------------ */
/* Physics (Sec. 3.2)                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int physics;       /* 0 Euler, 1 Navier-Stokes */
    int surface_flux;  /* 0 Lax-Friedrichs, 1 Roe, 2 entropy-conservative (central), 3 Rusanov,
                          4 low-dissipation Roe, 5 entropy-stable matrix dissipation */
    int volume_form;   /* 0 standard; split forms: 1 Chandrashekar, 2 Kennedy-Gruber, 3 Pirozzoli, 4 Ducros,
                          5 Morinishi, 6 Ismail-Roe */
    double gamma, Re, Pr, cfl;
    int time_scheme;   /* 0 Williamson RK3, 1 Carpenter-Kennedy RK4(5) */
} orc_cfg;

/* rho, v, p from u; p = (gamma-1)(rho e - rho |v|^2 / 2). */
static void primitives(const double *u, double g, double *rho, double v[3], double *p)
{
    *rho = u[0];
    v[0] = u[1] / u[0];
    v[1] = u[2] / u[0];
    v[2] = u[3] / u[0];
    *p = (g - 1.0) * (u[4] - 0.5 * u[0] * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]));
}

/* F_e . a for any vector a (the columns of the paper's F_e matrix, combined):
 * [rho v.a, rho v1 v.a + p a1, rho v2 v.a + p a2, rho v3 v.a + p a3, rho H v.a],
 * H = (rho e + p)/rho. */
void orc_flux_euler(const double *u, const double *a, double g, double *f)
{
    double rho, v[3], p;
    primitives(u, g, &rho, v, &p);
    double va = v[0] * a[0] + v[1] * a[1] + v[2] * a[2];
    f[0] = rho * va;
    f[1] = u[1] * va + p * a[0];
    f[2] = u[2] * va + p * a[1];
    f[3] = u[3] * va + p * a[2];
    f[4] = (u[4] + p) * va;
}

/* Lax-Friedrichs flux with unit normal nh:
 *   F* = (F_L + F_R).nh / 2 - lambda (u_R - u_L) / 2,
 *   lambda = max(|v_L.nh| + c_L, |v_R.nh| + c_R),  c = sqrt(gamma p / rho). */
void orc_flux_lf(const double *uL, const double *uR, const double *nh, double g, double *f)
{
    double FL[NVAR], FR[NVAR], rL, vL[3], pL, rR, vR[3], pR;
    orc_flux_euler(uL, nh, g, FL);
    orc_flux_euler(uR, nh, g, FR);
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double sL = fabs(vL[0] * nh[0] + vL[1] * nh[1] + vL[2] * nh[2]) + sqrt(g * pL / rL);
    double sR = fabs(vR[0] * nh[0] + vR[1] * nh[1] + vR[2] * nh[2]) + sqrt(g * pR / rR);
    double lam = sL > sR ? sL : sR;
    for (int v = 0; v < NVAR; ++v) f[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* Rusanov flux: as Lax-Friedrichs with the wave-speed bound
 *   lambda = max(|v_L.nh|, |v_R.nh|) + max(c_L, c_R)
 * (each side's largest convective and acoustic speeds combined). */
void orc_flux_rusanov(const double *uL, const double *uR, const double *nh, double g, double *f)
{
    double FL[NVAR], FR[NVAR], rL, vL[3], pL, rR, vR[3], pR;
    orc_flux_euler(uL, nh, g, FL);
    orc_flux_euler(uR, nh, g, FR);
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double vnL = fabs(vL[0] * nh[0] + vL[1] * nh[1] + vL[2] * nh[2]);
    double vnR = fabs(vR[0] * nh[0] + vR[1] * nh[1] + vR[2] * nh[2]);
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    double lam = (vnL > vnR ? vnL : vnR) + (cL > cR ? cL : cR);
    for (int v = 0; v < NVAR; ++v) f[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (uR[v] - uL[v]);
}

/* Entropy variables in the usual normalisation, w = dS'/du for
 * S' = -rho s / (gamma-1), s = ln p - gamma ln rho:
 *   w = [(gamma - s)/(gamma-1) - rho|v|^2/(2p), rho v / p, -rho / p]
 * (the paper's S = -rho s gives (gamma-1) times these). */
static void entropy_vars_std(const double *u, double g, double *w)
{
    double rho, v[3], p;
    primitives(u, g, &rho, v, &p);
    double s = log(p) - g * log(rho);
    w[0] = (g - s) / (g - 1.0) - rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / (2.0 * p);
    for (int c = 0; c < 3; ++c) w[1 + c] = rho * v[c] / p;
    w[4] = -rho / p;
}

/* Entropy-stable flux with matrix dissipation (Winters, Derigs, Gassner and
 * Walch 2017): the Chandrashekar flux minus a dissipation built from the
 * scaled eigenvectors of the flux Jacobian in direction nh, applied to the
 * jump of the entropy variables,
 *   F* = F_EC(u_L, u_R).nh - (1/2) sum_k |lambda_k| T_k r_k (r_k . [[w]]),
 * evaluated at the averages
 *   rho^ = ln-mean(rho), beta^ = ln-mean(beta), beta = rho/(2p),
 *   p^ = {rho}/(2{beta}), v^ = {v}, v2^ = 2|{v}|^2 - {|v|^2},
 *   a^ = sqrt(gamma p^/rho^), h^ = gamma/(2(gamma-1) beta^) + v2^/2:
 *   k = 1, 5: lambda = v^.n -+ a^, r = [1, v^ -+ a^ n, h^ -+ a^ v^.n], T = rho^/(2 gamma)
 *   k = 2:    lambda = v^.n,       r = [1, v^, v2^/2],                T = rho^ (gamma-1)/gamma
 *   shear:    lambda = v^.n,       sum over two unit tangents t of r = [0, t, v^.t], T = p^
 * (the shear pair is summed with the projector I - n n^T, so no tangent
 * basis is chosen).  For equal states sum_k T_k r_k r_k^T = du/dw, so the
 * dissipation is |A| du/dw [[w]] ~ |A| [[u]] for small jumps; it is positive
 * semi-definite in [[w]] for any states, so the flux is entropy stable. */
void orc_flux_matrix(const double *uL, const double *uR, const double *nh, double g, double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double bL = rL / (2.0 * pL), bR = rR / (2.0 * pR);
    double rho_h = orc_logmean(rL, rR), beta_ln = orc_logmean(bL, bR);
    double p_h = 0.5 * (rL + rR) / (bL + bR);
    double v[3], v2av = 0.5 * ((vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2]) +
                               (vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2]));
    for (int c = 0; c < 3; ++c) v[c] = 0.5 * (vL[c] + vR[c]);
    double v2h = 2.0 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) - v2av;
    double a_h = sqrt(g * p_h / rho_h);
    double h_h = g / (2.0 * (g - 1.0) * beta_ln) + 0.5 * v2h;
    double vn = v[0] * nh[0] + v[1] * nh[1] + v[2] * nh[2];
    double wL[NVAR], wR[NVAR], dw[NVAR];
    entropy_vars_std(uL, g, wL);
    entropy_vars_std(uR, g, wR);
    for (int k = 0; k < NVAR; ++k) dw[k] = wR[k] - wL[k];
    double r1[NVAR] = {1.0, v[0] - a_h * nh[0], v[1] - a_h * nh[1], v[2] - a_h * nh[2], h_h - a_h * vn};
    double r2[NVAR] = {1.0, v[0], v[1], v[2], 0.5 * v2h};
    double r5[NVAR] = {1.0, v[0] + a_h * nh[0], v[1] + a_h * nh[1], v[2] + a_h * nh[2], h_h + a_h * vn};
    double T15 = rho_h / (2.0 * g), T2 = rho_h * (g - 1.0) / g;
    double l1 = fabs(vn - a_h), l2 = fabs(vn), l5 = fabs(vn + a_h);
    double c1 = 0.0, c2 = 0.0, c5 = 0.0;
    for (int k = 0; k < NVAR; ++k) { c1 += r1[k] * dw[k]; c2 += r2[k] * dw[k]; c5 += r5[k] * dw[k]; }
    /* shear: q = [[w_m]] + v^ [[w_E]], projected on the face plane */
    double q[3], qn = 0.0;
    for (int c = 0; c < 3; ++c) q[c] = dw[1 + c] + v[c] * dw[4];
    for (int c = 0; c < 3; ++c) qn += q[c] * nh[c];
    double Pq[3];
    for (int c = 0; c < 3; ++c) Pq[c] = q[c] - qn * nh[c];
    double Dsh[NVAR] = {0.0, Pq[0], Pq[1], Pq[2], v[0] * Pq[0] + v[1] * Pq[1] + v[2] * Pq[2]};
    double fec[NVAR];
    orc_flux_ec(uL, uR, nh, g, fec);
    for (int k = 0; k < NVAR; ++k) {
        double D = l1 * T15 * c1 * r1[k] + l2 * T2 * c2 * r2[k] + l5 * T15 * c5 * r5[k] + l2 * p_h * Dsh[k];
        f[k] = fec[k] - 0.5 * D;
    }
}

/* Roe flux with unit normal nh (Roe 1981; no entropy fix):
 *   F* = (F_L + F_R).nh / 2 - (1/2) sum_k |lambda_k| alpha_k r_k
 * with sqrt(rho)-weighted averages v~, H~, c~^2 = (gamma-1)(H~ - |v~|^2/2),
 * rho~ = sqrt(rho_L rho_R), eigenvalues v~.n - c~, v~.n (x3), v~.n + c~, and
 * wave strengths from the jumps of rho, v, p:
 *   alpha_1 = (dp - rho~ c~ dvn)/(2 c~^2)       r_1 = [1, v~ - c~ n, H~ - c~ v~n]
 *   alpha_2 = drho - dp/c~^2                    r_2 = [1, v~, |v~|^2/2]
 *   shear   = rho~ (dv - dvn n)                 r_s = [0, shear, v~.shear]
 *   alpha_5 = (dp + rho~ c~ dvn)/(2 c~^2)       r_5 = [1, v~ + c~ n, H~ + c~ v~n]. */
static void roe_flux(const double *uL, const double *uR, const double *nh, double g, double zvel, int sign_mode,
                     double *f);

void orc_flux_roe(const double *uL, const double *uR, const double *nh, double g, double *f)
{
    roe_flux(uL, uR, nh, g, 1.0, 0, f);
}

/* sign_mode = 0: the Roe flux above.  sign_mode = 1: f receives the wave sum
 * sum_k lambda_k alpha_k r_k with SIGNED eigenvalues (used by the tests to
 * check Roe's property that it equals F_R.n - F_L.n). */
void orc_flux_roe_signed(const double *uL, const double *uR, const double *nh, double g, double *f, int sign_mode)
{
    roe_flux(uL, uR, nh, g, 1.0, sign_mode, f);
}

/* Low-dissipation Roe flux (the L2Roe of Osswald et al. 2016): the Roe flux
 * with the velocity jump in the dissipation (dvn and the shear jump) scaled by
 *   z = min(1, max(M_L, M_R)),  M = |v| / c,
 * so that at low Mach numbers the velocity dissipation falls like M while the
 * density and pressure waves keep Roe's upwinding; identical to Roe for
 * M >= 1. */
void orc_flux_ldroe(const double *uL, const double *uR, const double *nh, double g, double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double ML = sqrt(vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2]) / sqrt(g * pL / rL);
    double MR = sqrt(vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2]) / sqrt(g * pR / rR);
    double z = ML > MR ? ML : MR;
    if (z > 1.0) z = 1.0;
    roe_flux(uL, uR, nh, g, z, 0, f);
}

/* Roe flux whose dissipation sees the velocity jump times zvel (1: Roe). */
static void roe_flux(const double *uL, const double *uR, const double *nh, double g, double zvel, int sign_mode,
                     double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double HL = (uL[4] + pL) / rL, HR = (uR[4] + pR) / rR;
    double sL = sqrt(rL), sR = sqrt(rR);
    double vt[3];
    for (int c = 0; c < 3; ++c) vt[c] = (sL * vL[c] + sR * vR[c]) / (sL + sR);
    double Ht = (sL * HL + sR * HR) / (sL + sR);
    double q2 = vt[0] * vt[0] + vt[1] * vt[1] + vt[2] * vt[2];
    double ct = sqrt((g - 1.0) * (Ht - 0.5 * q2));
    double rt = sL * sR;
    double vnt = vt[0] * nh[0] + vt[1] * nh[1] + vt[2] * nh[2];
    double drho = rR - rL, dp = pR - pL;
    double dv[3] = {zvel * (vR[0] - vL[0]), zvel * (vR[1] - vL[1]), zvel * (vR[2] - vL[2])};
    double dvn = dv[0] * nh[0] + dv[1] * nh[1] + dv[2] * nh[2];
    double a1 = (dp - rt * ct * dvn) / (2.0 * ct * ct);
    double a5 = (dp + rt * ct * dvn) / (2.0 * ct * ct);
    double a2 = drho - dp / (ct * ct);
    double sh[3];
    for (int c = 0; c < 3; ++c) sh[c] = rt * (dv[c] - dvn * nh[c]);
    double l1 = vnt - ct, l2 = vnt, l5 = vnt + ct;
    if (!sign_mode) { l1 = fabs(l1); l2 = fabs(l2); l5 = fabs(l5); }
    double W[NVAR];
    W[0] = l1 * a1 + l2 * a2 + l5 * a5;
    for (int c = 0; c < 3; ++c)
        W[1 + c] = l1 * a1 * (vt[c] - ct * nh[c]) + l2 * (a2 * vt[c] + sh[c]) + l5 * a5 * (vt[c] + ct * nh[c]);
    W[4] = l1 * a1 * (Ht - ct * vnt) + l2 * (a2 * 0.5 * q2 + vt[0] * sh[0] + vt[1] * sh[1] + vt[2] * sh[2])
         + l5 * a5 * (Ht + ct * vnt);
    if (sign_mode) { for (int v = 0; v < NVAR; ++v) f[v] = W[v]; return; }
    double FL[NVAR], FR[NVAR];
    orc_flux_euler(uL, nh, g, FL);
    orc_flux_euler(uR, nh, g, FR);
    for (int v = 0; v < NVAR; ++v) f[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * W[v];
}

/* Logarithmic mean (a-b)/(ln a - ln b) in the Ismail-Roe form:
 * zeta = a/b, f = (zeta-1)/(zeta+1), u = f^2,
 * F = 1 + u/3 + u^2/5 + u^3/7 for u < 1e-4, else ln(zeta)/(2f);
 * result (a+b)/(2F). */
double orc_logmean(double a, double b)
{
    double zeta = a / b;
    double f = (zeta - 1.0) / (zeta + 1.0);
    double u = f * f;
    double F;
    if (u < 1e-4) F = 1.0 + u / 3.0 + u * u / 5.0 + u * u * u / 7.0;
    else F = log(zeta) / (2.0 * f);
    return (a + b) / (2.0 * F);
}

/* Chandrashekar's entropy-conservative, kinetic-energy-preserving two-point
 * flux (Sec. 3.5 lists it; formula from Chandrashekar 2013), dotted with an
 * arbitrary vector a:
 *   beta = rho/(2p); rho^ = ln-mean(rho), beta^ = ln-mean(beta);
 *   {.} arithmetic mean; p~ = {rho}/(2{beta});
 *   f_rho = rho^ {v}.a;  f_m = f_rho {v} + p~ a;
 *   f_E = f_rho [ 1/(2(gamma-1) beta^) - {|v|^2}/2 ] + {v}.f_m. */
void orc_flux_ec(const double *uL, const double *uR, const double *a, double g, double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double bL = rL / (2.0 * pL), bR = rR / (2.0 * pR);
    double rho_ln = orc_logmean(rL, rR);
    double beta_ln = orc_logmean(bL, bR);
    double rho_av = 0.5 * (rL + rR), beta_av = 0.5 * (bL + bR);
    double vav[3] = {0.5 * (vL[0] + vR[0]), 0.5 * (vL[1] + vR[1]), 0.5 * (vL[2] + vR[2])};
    double v2av = 0.5 * ((vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2]) + (vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2]));
    double pt = rho_av / (2.0 * beta_av);
    double van = vav[0] * a[0] + vav[1] * a[1] + vav[2] * a[2];
    f[0] = rho_ln * van;
    for (int c = 0; c < 3; ++c) f[1 + c] = f[0] * vav[c] + pt * a[c];
    f[4] = f[0] * (1.0 / (2.0 * (g - 1.0) * beta_ln) - 0.5 * v2av)
         + vav[0] * f[1] + vav[1] * f[2] + vav[2] * f[3];
}

/* Further split forms of Sec. 3.5, each a symmetric two-point flux dotted
 * with a ({.} arithmetic mean of the two states, v_a = v.a, e = rho e / rho,
 * h = (rho e + p)/rho):
 *   Kennedy-Gruber (2008):  f_rho = {rho}{v_a},  f_m = {rho}{v_a}{v} + {p} a,
 *                           f_E = {rho}{v_a}{e} + {p}{v_a}
 *   Pirozzoli (2010):       f_rho = {rho}{v_a},  f_m = {rho}{v_a}{v} + {p} a,
 *                           f_E = {rho}{v_a}{h}
 *   Ducros et al. (2000):   f_rho = {rho}{v_a},  f_m = {rho v}{v_a} + {p} a,
 *                           f_E = {rho e + p}{v_a}
 * kind: 2 Kennedy-Gruber, 3 Pirozzoli, 4 Ducros. */
void orc_flux_split(int kind, const double *uL, const double *uR, const double *a, double g, double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double rho_av = 0.5 * (rL + rR), p_av = 0.5 * (pL + pR);
    double vaL = vL[0] * a[0] + vL[1] * a[1] + vL[2] * a[2];
    double vaR = vR[0] * a[0] + vR[1] * a[1] + vR[2] * a[2];
    double va_av = 0.5 * (vaL + vaR);
    if (kind == 4) {
        f[0] = rho_av * va_av;
        for (int c = 0; c < 3; ++c) f[1 + c] = 0.5 * (uL[1 + c] + uR[1 + c]) * va_av + p_av * a[c];
        f[4] = 0.5 * ((uL[4] + pL) + (uR[4] + pR)) * va_av;
        return;
    }
    double m = rho_av * va_av;
    f[0] = m;
    for (int c = 0; c < 3; ++c) f[1 + c] = m * 0.5 * (vL[c] + vR[c]) + p_av * a[c];
    if (kind == 2) {
        double e_av = 0.5 * (uL[4] / rL + uR[4] / rR);
        f[4] = m * e_av + p_av * va_av;
    } else {
        double h_av = 0.5 * ((uL[4] + pL) / rL + (uR[4] + pR) / rR);
        f[4] = m * h_av;
    }
}

/* Morinishi's split form (Morinishi 2010, skew-symmetric convective terms
 * with the mass flux rho v kept whole), as a two-point flux dotted with a:
 *   f_rho = {rho v_a},  f_m = {rho v_a}{v} + {p} a,
 *   f_E   = {rho v_a}{|v|^2/2} + gamma/(gamma-1) {p v_a}
 * (kinetic energy carried in the same skew-symmetric way as momentum,
 * enthalpy of the internal energy in divergence form). */
void orc_flux_morinishi(const double *uL, const double *uR, const double *a, double g, double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double vaL = vL[0] * a[0] + vL[1] * a[1] + vL[2] * a[2];
    double vaR = vR[0] * a[0] + vR[1] * a[1] + vR[2] * a[2];
    double m = 0.5 * (rL * vaL + rR * vaR);
    double p_av = 0.5 * (pL + pR);
    double kL = 0.5 * (vL[0] * vL[0] + vL[1] * vL[1] + vL[2] * vL[2]);
    double kR = 0.5 * (vR[0] * vR[0] + vR[1] * vR[1] + vR[2] * vR[2]);
    f[0] = m;
    for (int c = 0; c < 3; ++c) f[1 + c] = m * 0.5 * (vL[c] + vR[c]) + p_av * a[c];
    f[4] = m * 0.5 * (kL + kR) + g / (g - 1.0) * 0.5 * (pL * vaL + pR * vaR);
}

/* Ismail and Roe's entropy-conservative flux (Ismail & Roe 2009), dotted
 * with a: parameter vector z = sqrt(rho/p) (1, v, p), so z1 = sqrt(rho/p),
 * z_v = z1 v, z5 = sqrt(rho p); with {.} arithmetic and (.)^ln logarithmic
 * means:
 *   rho^ = {z1} z5^ln,  v^ = {z_v}/{z1},  p1^ = {z5}/{z1},
 *   p2^ = (gamma+1)/(2 gamma) z5^ln/z1^ln + (gamma-1)/(2 gamma) {z5}/{z1},
 *   h^ = gamma p2^ / ((gamma-1) rho^) + |v^|^2/2,
 *   f = (rho^ v^.a, rho^ v^.a v^ + p1^ a, rho^ v^.a h^). */
void orc_flux_ir(const double *uL, const double *uR, const double *a, double g, double *f)
{
    double rL, vL[3], pL, rR, vR[3], pR;
    primitives(uL, g, &rL, vL, &pL);
    primitives(uR, g, &rR, vR, &pR);
    double z1L = sqrt(rL / pL), z1R = sqrt(rR / pR);
    double z5L = sqrt(rL * pL), z5R = sqrt(rR * pR);
    double z1a = 0.5 * (z1L + z1R), z5a = 0.5 * (z5L + z5R);
    double z1ln = orc_logmean(z1L, z1R), z5ln = orc_logmean(z5L, z5R);
    double rho = z1a * z5ln;
    double v[3];
    for (int c = 0; c < 3; ++c) v[c] = 0.5 * (z1L * vL[c] + z1R * vR[c]) / z1a;
    double p1 = z5a / z1a;
    double p2 = (g + 1.0) / (2.0 * g) * z5ln / z1ln + (g - 1.0) / (2.0 * g) * z5a / z1a;
    double h = g * p2 / ((g - 1.0) * rho) + 0.5 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double va = v[0] * a[0] + v[1] * a[1] + v[2] * a[2];
    f[0] = rho * va;
    for (int c = 0; c < 3; ++c) f[1 + c] = rho * va * v[c] + p1 * a[c];
    f[4] = rho * va * h;
}

/* Two-point volume flux of split form `form` (1..6) dotted with a. */
static void split_flux(int form, const double *ui, const double *um, const double *a, double g, double *f)
{
    if (form == 1) orc_flux_ec(ui, um, a, g, f);
    else if (form == 5) orc_flux_morinishi(ui, um, a, g, f);
    else if (form == 6) orc_flux_ir(ui, um, a, g, f);
    else orc_flux_split(form, ui, um, a, g, f);
}

/* Entropy variables w = dS/du for S = -rho s, s = ln p - gamma ln rho
 * (Sec. 4.4, Eq. shock:entropy):
 *   w = [gamma - s - (gamma-1) rho |v|^2/(2p), (gamma-1) rho v/p, -(gamma-1) rho/p]. */
void orc_entropy_vars(const double *u, double g, double *w)
{
    double rho, v[3], p;
    primitives(u, g, &rho, v, &p);
    double s = log(p) - g * log(rho);
    double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    w[0] = g - s - (g - 1.0) * rho * v2 / (2.0 * p);
    w[1] = (g - 1.0) * rho * v[0] / p;
    w[2] = (g - 1.0) * rho * v[1] / p;
    w[3] = (g - 1.0) * rho * v[2] / p;
    w[4] = -(g - 1.0) * rho / p;
}

/* Gradient variables q = (v1, v2, v3, T), T = p/rho (gas constant 1). */
static void grad_vars(const double *u, double g, double *q)
{
    double rho, v[3], p;
    primitives(u, g, &rho, v, &p);
    q[0] = v[0]; q[1] = v[1]; q[2] = v[2]; q[3] = p / rho;
}

/* Viscous flux F_v . a (Sec. 3.2, Eq. viscousfluxes) from q = (v, T) and
 * G[v][c] = d q_v / d x_c:
 *   tau = mu (grad v + grad v^T) - (2/3) mu I div v,
 *   row 5 = sum_j v_j tau_{cj} + kappa dT/dx_c. */
void orc_flux_visc(const double *q, const double *G, double mu, double kappa, const double *a, double *f)
{
    double div = G[0 * 3 + 0] + G[1 * 3 + 1] + G[2 * 3 + 2];
    double tau[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            tau[i][j] = mu * (G[i * 3 + j] + G[j * 3 + i]) - (i == j ? (2.0 / 3.0) * mu * div : 0.0);
    f[0] = 0.0;
    for (int i = 0; i < 3; ++i) f[1 + i] = tau[i][0] * a[0] + tau[i][1] * a[1] + tau[i][2] * a[2];
    double fe = 0.0;
    for (int c = 0; c < 3; ++c) {
        double col = q[0] * tau[0][c] + q[1] * tau[1][c] + q[2] * tau[2][c] + kappa * G[3 * 3 + c];
        fe += col * a[c];
    }
    f[4] = fe;
}

/* ------------------------------------------------------------------------ */
/* Residual (Sec. 3.3, Eq. NS4/NS5 in strong form on GL nodes)              */
/* ------------------------------------------------------------------------ */

static double visc_mu(const orc_cfg *cfg) { return 1.0 / cfg->Re; }
static double visc_kappa(const orc_cfg *cfg)
{
    /* kappa = mu c_p / Pr with c_p = gamma/(gamma-1) for gas constant 1 */
    return visc_mu(cfg) * cfg->gamma / ((cfg->gamma - 1.0) * cfg->Pr);
}

/* Index of the node of an element with index m along direction d and the
 * other two indices taken from (i,j,k). */
static int node_along(int n, int d, int m, int i, int j, int k)
{
    if (d == 0) return node_index(n, m, j, k);
    if (d == 1) return node_index(n, i, m, k);
    return node_index(n, i, j, m);
}

/* The node of the neighbour that coincides with face node p of element e on
 * face (d, side): same tangential indices, index along d at the opposite end. */
static int matching_node(int n, int d, int side, int i, int j, int k)
{
    int m = (side > 0) ? 0 : n - 1;
    return node_along(n, d, m, i, j, k);
}

/* BR1 gradients of q = (v, T) (Bassi & Rebay 1997; Sec. 3.3 lists BR1):
 *   J grad q_c = sum_d D_d (Ja^d_c q) + sum_faces (1/w_end) (q* - q_in) (s n)_c,
 *   q* = (q_in + q_out)/2, (s n) = outward scaled normal = +-Ja^d at the node.
 * grad[e][v][c][node]. */
static void br1_gradients(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *grad)
{
    int n = m->n, n3 = m->n3, E = m->E, N = n - 1;
    double g = cfg->gamma;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        double *q = (double *)malloc(sizeof(double) * NGRAD * n3);
        double *f = (double *)malloc(sizeof(double) * 3 * n3);   /* Ja^d_c q_v for d = 0..2 */
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], qp[NGRAD];
            for (int v = 0; v < NVAR; ++v) up[v] = u[((size_t)e * NVAR + v) * n3 + p];
            grad_vars(up, g, qp);
            for (int v = 0; v < NGRAD; ++v) q[v * n3 + p] = qp[v];
        }
        for (int v = 0; v < NGRAD; ++v)
        for (int c = 0; c < 3; ++c) {
            for (int d = 0; d < 3; ++d)
                for (int p = 0; p < n3; ++p)
                    f[d * n3 + p] = m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + p] * q[v * n3 + p];
            for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
                int p = node_index(n, i, j, k);
                double acc = 0.0;
                for (int d = 0; d < 3; ++d) acc += dir_derivative(n, m->D, f + d * n3, d, i, j, k);
                grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p] = acc;
            }
        }
        /* surface lifting */
        int ijk[3];
        for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
            ijk[0] = i; ijk[1] = j; ijk[2] = k;
            int p = node_index(n, i, j, k);
            for (int d = 0; d < 3; ++d)
            for (int side = -1; side <= 1; side += 2) {
                int at = (side > 0) ? N : 0;
                if (ijk[d] != at) continue;
                int nb = neighbour(&m->box, e, d, side);
                int pn = matching_node(n, d, side, i, j, k);
                double un[NVAR], qn[NGRAD];
                for (int v = 0; v < NVAR; ++v) un[v] = u[((size_t)nb * NVAR + v) * n3 + pn];
                grad_vars(un, g, qn);
                for (int v = 0; v < NGRAD; ++v) {
                    double jump = 0.5 * (qn[v] + q[v * n3 + p]) - q[v * n3 + p];
                    for (int c = 0; c < 3; ++c) {
                        double sn = side * m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + p];
                        grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p] += jump * sn / m->w[at];
                    }
                }
            }
        }
        for (int v = 0; v < NGRAD; ++v)
            for (int c = 0; c < 3; ++c)
                for (int p = 0; p < n3; ++p)
                    grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p] /= m->J[(size_t)e * n3 + p];
        free(q); free(f);
    }
}

/* Inviscid numerical flux times the face scale: s F*(u_in, u_out; n^) with
 * Sn = s n^ the outward scaled normal. */
static void surface_flux(int kind, const double *uin, const double *uout, const double *Sn, double g, double *f)
{
    if (kind == 2) { orc_flux_ec(uin, uout, Sn, g, f); return; }
    double s = sqrt(Sn[0] * Sn[0] + Sn[1] * Sn[1] + Sn[2] * Sn[2]);
    double nh[3] = {Sn[0] / s, Sn[1] / s, Sn[2] / s};
    if (kind == 0) orc_flux_lf(uin, uout, nh, g, f);
    else if (kind == 1) orc_flux_roe(uin, uout, nh, g, f);
    else if (kind == 3) orc_flux_rusanov(uin, uout, nh, g, f);
    else if (kind == 4) orc_flux_ldroe(uin, uout, nh, g, f);
    else orc_flux_matrix(uin, uout, nh, g, f);
    for (int v = 0; v < NVAR; ++v) f[v] *= s;
}

/* du/dt = -(V + S)/J per element, with
 *   standard form  V = sum_d D_d F~^d,  F~^d = sum_c Ja^d_c (F_e - F_v)_c
 *   split form     V = sum_d [ 2 sum_m D_im F#(u_i, u_m).(Ja^d_i + Ja^d_m)/2 ] - sum_d D_d F~_v^d
 *                  (F# the Chandrashekar, Kennedy-Gruber, Pirozzoli or Ducros two-point flux)
 *   surface        S = (1/w_end) [ +-(F^*(L,R; Sn_L) - F_v^*.Sn_L) - (F_e - F_v)(in).(+-Ja^d_in) ]
 * on each face node (+ on the element's +d face, - on its -d face),
 * F_v^* = (F_v(L) + F_v(R))/2 (BR1), Sn_L = Ja^d of the face's minus-side element. */
static int residual_general(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *dudt);

int orc_residual(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *dudt)
{
    if (m->box.nodes == 1) return residual_general(m, cfg, u, dudt);
    int n = m->n, n3 = m->n3, E = m->E, N = n - 1;
    double g = cfg->gamma;
    int ns = (cfg->physics == 1);
    double mu = ns ? visc_mu(cfg) : 0.0, kappa = ns ? visc_kappa(cfg) : 0.0;
    double *grad = NULL;
    if (ns) {
        grad = (double *)malloc(sizeof(double) * (size_t)E * NGRAD * 3 * n3);
        if (!grad) return -1;
        br1_gradients(m, cfg, u, grad);
    }
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        double *Ft = (double *)malloc(sizeof(double) * 3 * NVAR * n3);   /* total contravariant flux */
        double *Fv = (double *)malloc(sizeof(double) * 3 * NVAR * n3);   /* viscous contravariant flux */
        double *R = (double *)calloc(NVAR * n3, sizeof(double));
        /* contravariant fluxes at every node */
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], qp[NGRAD], G[12];
            for (int v = 0; v < NVAR; ++v) up[v] = u[((size_t)e * NVAR + v) * n3 + p];
            if (ns) {
                grad_vars(up, g, qp);
                for (int v = 0; v < NGRAD; ++v)
                    for (int c = 0; c < 3; ++c) G[v * 3 + c] = grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p];
            }
            for (int d = 0; d < 3; ++d) {
                double a[3], fe[NVAR], fv[NVAR] = {0, 0, 0, 0, 0};
                for (int c = 0; c < 3; ++c) a[c] = m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + p];
                orc_flux_euler(up, a, g, fe);
                if (ns) orc_flux_visc(qp, G, mu, kappa, a, fv);
                for (int v = 0; v < NVAR; ++v) {
                    Ft[(d * NVAR + v) * n3 + p] = fe[v] - fv[v];
                    Fv[(d * NVAR + v) * n3 + p] = fv[v];
                }
            }
        }
        /* volume term */
        for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
            int p = node_index(n, i, j, k);
            int ijk[3] = {i, j, k};
            for (int d = 0; d < 3; ++d) {
                if (cfg->volume_form == 0) {
                    for (int v = 0; v < NVAR; ++v)
                        R[v * n3 + p] += dir_derivative(n, m->D, Ft + (d * NVAR + v) * n3, d, i, j, k);
                } else {
                    double ui[NVAR];
                    for (int v = 0; v < NVAR; ++v) ui[v] = u[((size_t)e * NVAR + v) * n3 + p];
                    for (int mm = 0; mm < n; ++mm) {
                        int pm = node_along(n, d, mm, i, j, k);
                        double um[NVAR], a[3], fs[NVAR];
                        for (int v = 0; v < NVAR; ++v) um[v] = u[((size_t)e * NVAR + v) * n3 + pm];
                        for (int c = 0; c < 3; ++c)
                            a[c] = 0.5 * (m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + p]
                                        + m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + pm]);
                        split_flux(cfg->volume_form, ui, um, a, g, fs);
                        double Dim = m->D[ijk[d] * n + mm];
                        for (int v = 0; v < NVAR; ++v) R[v * n3 + p] += 2.0 * Dim * fs[v];
                    }
                    if (ns)
                        for (int v = 0; v < NVAR; ++v)
                            R[v * n3 + p] -= dir_derivative(n, m->D, Fv + (d * NVAR + v) * n3, d, i, j, k);
                }
            }
        }
        /* surface term.  The numerical flux is single-valued on each face
         * (Eq. NS4: F* couples the two elements): it is evaluated once per
         * face node with the face's scaled normal, taken from the element on
         * the face's minus side ("left", L) and pointing into the plus side
         * (R); the element on the plus side receives it with the opposite
         * sign.  The element's own boundary flux uses its own Ja^d, as the
         * volume term does. */
        for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
            int p = node_index(n, i, j, k);
            int ijk[3] = {i, j, k};
            for (int d = 0; d < 3; ++d)
            for (int side = -1; side <= 1; side += 2) {
                int at = (side > 0) ? N : 0;
                if (ijk[d] != at) continue;
                int nb = neighbour(&m->box, e, d, side);
                int pn = matching_node(n, d, side, i, j, k);
                int eL = (side > 0) ? e : nb, pL = (side > 0) ? p : pn;
                int eR = (side > 0) ? nb : e, pR = (side > 0) ? pn : p;
                double uL[NVAR], uR[NVAR], Sn[3], fstar[NVAR];
                for (int v = 0; v < NVAR; ++v) {
                    uL[v] = u[((size_t)eL * NVAR + v) * n3 + pL];
                    uR[v] = u[((size_t)eR * NVAR + v) * n3 + pR];
                }
                for (int c = 0; c < 3; ++c) Sn[c] = m->Ja[(((size_t)eL * 3 + d) * 3 + c) * n3 + pL];
                surface_flux(cfg->surface_flux, uL, uR, Sn, g, fstar);
                if (ns) {
                    double qL[NGRAD], qR[NGRAD], GL[12], GR[12], fvL[NVAR], fvR[NVAR];
                    grad_vars(uL, g, qL);
                    grad_vars(uR, g, qR);
                    for (int v = 0; v < NGRAD; ++v)
                        for (int c = 0; c < 3; ++c) {
                            GL[v * 3 + c] = grad[(((size_t)eL * NGRAD + v) * 3 + c) * n3 + pL];
                            GR[v * 3 + c] = grad[(((size_t)eR * NGRAD + v) * 3 + c) * n3 + pR];
                        }
                    orc_flux_visc(qL, GL, mu, kappa, Sn, fvL);
                    orc_flux_visc(qR, GR, mu, kappa, Sn, fvR);
                    for (int v = 0; v < NVAR; ++v) fstar[v] -= 0.5 * (fvL[v] + fvR[v]);
                }
                for (int v = 0; v < NVAR; ++v) {
                    /* outward flux side*F*, own flux (F_e - F_v)(in).(side Ja^d) = side * F~^d(in) */
                    double own = side * Ft[(d * NVAR + v) * n3 + p];
                    R[v * n3 + p] += (side * fstar[v] - own) / m->w[at];
                }
            }
        }
        for (int v = 0; v < NVAR; ++v)
            for (int p = 0; p < n3; ++p)
                dudt[((size_t)e * NVAR + v) * n3 + p] = -R[v * n3 + p] / m->J[(size_t)e * n3 + p];
        free(Ft); free(Fv); free(R);
    }
    free(grad);
    return 0;
}

/* BR1 gradients exposed for tests: grad[e][v][c][node]. */
/* ------------------------------------------------------------------------ */
/* Residual with the face interpolation written out (any nodal set; the only  */
/* form for Gauss-Legendre nodes)                                             */
/* ------------------------------------------------------------------------ */

/* Node (i, j, k) of the line along d through face point (ta, tb), index m. */
static int line_index(int n, int d, int m, int ta, int tb)
{
    int d0, d1, idx[3];
    face_dirs(d, &d0, &d1);
    idx[d] = m;
    idx[d0] = ta;
    idx[d1] = tb;
    return node_index(n, idx[0], idx[1], idx[2]);
}

/* Value at the face xi_d = side (side -1 or +1) of the nodal field f of one
 * element (stride n3 between variables), on the line through (ta, tb):
 *   f(side) = sum_j l_j(side) f_j. */
static double face_value(const orc_mesh *m, const double *f, int d, int side, int ta, int tb)
{
    const double *l = (side > 0) ? m->rb : m->lb;
    double acc = 0.0;
    for (int j = 0; j < m->n; ++j) acc += l[j] * f[line_index(m->n, d, j, ta, tb)];
    return acc;
}

static const double *own_face_metric(const orc_mesh *m, int e, int d, int side, int c)
{
    return m->Sf + ((((size_t)e * 3 + d) * 2 + (side > 0 ? 1 : 0)) * 3 + c) * m->n * m->n;
}

/* BR1 gradients with interpolated traces (strong form, any nodes):
 *   J grad q_c = sum_d D_d (Ja^d_c q)
 *              + sum_faces (l_i(side)/w_i) side [ q* Sf_c - (Ja^d_c q)(side) ],
 * q* = (q(u_in(side)) + q(u_out(side)))/2 from the interpolated conserved
 * traces of the two elements, Sf the element's own face metric, and
 * (Ja^d_c q)(side) the interpolated product.  On Gauss-Lobatto nodes
 * l(side) is a unit vector and this is br1_gradients. */
static void br1_gradients_general(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *grad)
{
    int n = m->n, n3 = m->n3, E = m->E;
    double g = cfg->gamma;
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        double *q = (double *)malloc(sizeof(double) * NGRAD * n3);
        double *f = (double *)malloc(sizeof(double) * 3 * n3);
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], qp[NGRAD];
            for (int v = 0; v < NVAR; ++v) up[v] = u[((size_t)e * NVAR + v) * n3 + p];
            grad_vars(up, g, qp);
            for (int v = 0; v < NGRAD; ++v) q[v * n3 + p] = qp[v];
        }
        for (int v = 0; v < NGRAD; ++v)
        for (int c = 0; c < 3; ++c) {
            for (int d = 0; d < 3; ++d)
                for (int p = 0; p < n3; ++p)
                    f[d * n3 + p] = m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + p] * q[v * n3 + p];
            for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
                int p = node_index(n, i, j, k);
                double acc = 0.0;
                for (int d = 0; d < 3; ++d) acc += dir_derivative(n, m->D, f + d * n3, d, i, j, k);
                grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p] = acc;
            }
        }
        for (int d = 0; d < 3; ++d)
        for (int side = -1; side <= 1; side += 2) {
            int nb = neighbour(&m->box, e, d, side);
            const double *l = (side > 0) ? m->rb : m->lb;
            for (int tb = 0; tb < n; ++tb) for (int ta = 0; ta < n; ++ta) {
                double uin[NVAR], uout[NVAR], qin[NGRAD], qout[NGRAD];
                for (int v = 0; v < NVAR; ++v) {
                    uin[v] = face_value(m, u + ((size_t)e * NVAR + v) * n3, d, side, ta, tb);
                    uout[v] = face_value(m, u + ((size_t)nb * NVAR + v) * n3, d, -side, ta, tb);
                }
                grad_vars(uin, g, qin);
                grad_vars(uout, g, qout);
                for (int v = 0; v < NGRAD; ++v)
                for (int c = 0; c < 3; ++c) {
                    for (int jj = 0; jj < n; ++jj) {
                        int pj = line_index(n, d, jj, ta, tb);
                        f[pj] = m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + pj] * q[v * n3 + pj];
                    }
                    double jaq = face_value(m, f, d, side, ta, tb);
                    double sf = own_face_metric(m, e, d, side, c)[ta + n * tb];
                    double flux = side * (0.5 * (qin[v] + qout[v]) * sf - jaq);
                    for (int i = 0; i < n; ++i) {
                        int pi = line_index(n, d, i, ta, tb);
                        grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + pi] += l[i] / m->w[i] * flux;
                    }
                }
            }
        }
        for (int v = 0; v < NGRAD; ++v)
            for (int c = 0; c < 3; ++c)
                for (int p = 0; p < n3; ++p)
                    grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p] /= m->J[(size_t)e * n3 + p];
        free(q); free(f);
    }
}

/* Residual with interpolated traces (strong form, standard volume term):
 *   du/dt = -(1/J) [ sum_d D_d F~^d
 *                    + sum_faces (l_i(side)/w_i) side (F* - F~^d(side)) ],
 * F~^d(side) = sum_j l_j(side) F~^d_j the element's own contravariant flux
 * (Euler minus viscous) interpolated to the face, F* the single-valued
 * numerical flux of the face (Eq. NS4) from the interpolated conserved
 * traces of its two elements with the scaled normal Sf of its minus-side
 * element (BR1 viscous part (F_v(L) + F_v(R))/2 . Sf with interpolated
 * gradient traces).  On Gauss-Lobatto nodes this is the standard-form
 * orc_residual. */
static int residual_general(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *dudt)
{
    if (cfg->volume_form != 0) return -2;   /* split forms need the Gauss-Lobatto SBP property */
    int n = m->n, n3 = m->n3, E = m->E;
    double g = cfg->gamma;
    int ns = (cfg->physics == 1);
    double mu = ns ? visc_mu(cfg) : 0.0, kappa = ns ? visc_kappa(cfg) : 0.0;
    double *grad = NULL;
    if (ns) {
        grad = (double *)malloc(sizeof(double) * (size_t)E * NGRAD * 3 * n3);
        if (!grad) return -1;
        br1_gradients_general(m, cfg, u, grad);
    }
#pragma omp parallel for schedule(static)
    for (int e = 0; e < E; ++e) {
        double *Ft = (double *)malloc(sizeof(double) * 3 * NVAR * n3);
        double *R = (double *)calloc(NVAR * n3, sizeof(double));
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], qp[NGRAD], G[12];
            for (int v = 0; v < NVAR; ++v) up[v] = u[((size_t)e * NVAR + v) * n3 + p];
            if (ns) {
                grad_vars(up, g, qp);
                for (int v = 0; v < NGRAD; ++v)
                    for (int c = 0; c < 3; ++c) G[v * 3 + c] = grad[(((size_t)e * NGRAD + v) * 3 + c) * n3 + p];
            }
            for (int d = 0; d < 3; ++d) {
                double a[3], fe[NVAR], fv[NVAR] = {0, 0, 0, 0, 0};
                for (int c = 0; c < 3; ++c) a[c] = m->Ja[(((size_t)e * 3 + d) * 3 + c) * n3 + p];
                orc_flux_euler(up, a, g, fe);
                if (ns) orc_flux_visc(qp, G, mu, kappa, a, fv);
                for (int v = 0; v < NVAR; ++v) Ft[(d * NVAR + v) * n3 + p] = fe[v] - fv[v];
            }
        }
        for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
            int p = node_index(n, i, j, k);
            for (int d = 0; d < 3; ++d)
                for (int v = 0; v < NVAR; ++v)
                    R[v * n3 + p] += dir_derivative(n, m->D, Ft + (d * NVAR + v) * n3, d, i, j, k);
        }
        for (int d = 0; d < 3; ++d)
        for (int side = -1; side <= 1; side += 2) {
            int nb = neighbour(&m->box, e, d, side);
            int eL = (side > 0) ? e : nb, eR = (side > 0) ? nb : e;
            const double *l = (side > 0) ? m->rb : m->lb;
            for (int tb = 0; tb < n; ++tb) for (int ta = 0; ta < n; ++ta) {
                double uL[NVAR], uR[NVAR], Sn[3], fstar[NVAR];
                for (int v = 0; v < NVAR; ++v) {
                    uL[v] = face_value(m, u + ((size_t)eL * NVAR + v) * n3, d, +1, ta, tb);
                    uR[v] = face_value(m, u + ((size_t)eR * NVAR + v) * n3, d, -1, ta, tb);
                }
                for (int c = 0; c < 3; ++c) Sn[c] = own_face_metric(m, eL, d, +1, c)[ta + n * tb];
                surface_flux(cfg->surface_flux, uL, uR, Sn, g, fstar);
                if (ns) {
                    double qL[NGRAD], qR[NGRAD], GL[12], GR[12], fvL[NVAR], fvR[NVAR];
                    grad_vars(uL, g, qL);
                    grad_vars(uR, g, qR);
                    for (int v = 0; v < NGRAD; ++v)
                        for (int c = 0; c < 3; ++c) {
                            GL[v * 3 + c] = face_value(m, grad + (((size_t)eL * NGRAD + v) * 3 + c) * n3, d, +1, ta, tb);
                            GR[v * 3 + c] = face_value(m, grad + (((size_t)eR * NGRAD + v) * 3 + c) * n3, d, -1, ta, tb);
                        }
                    orc_flux_visc(qL, GL, mu, kappa, Sn, fvL);
                    orc_flux_visc(qR, GR, mu, kappa, Sn, fvR);
                    for (int v = 0; v < NVAR; ++v) fstar[v] -= 0.5 * (fvL[v] + fvR[v]);
                }
                for (int v = 0; v < NVAR; ++v) {
                    double own = face_value(m, Ft + (d * NVAR + v) * n3, d, side, ta, tb);
                    double flux = side * (fstar[v] - own);
                    for (int i = 0; i < n; ++i)
                        R[v * n3 + line_index(n, d, i, ta, tb)] += l[i] / m->w[i] * flux;
                }
            }
        }
        for (int v = 0; v < NVAR; ++v)
            for (int p = 0; p < n3; ++p)
                dudt[((size_t)e * NVAR + v) * n3 + p] = -R[v * n3 + p] / m->J[(size_t)e * n3 + p];
        free(Ft); free(R);
    }
    free(grad);
    return 0;
}

/* The residual through the interpolated-trace path on any mesh (tests run it
 * on Gauss-Lobatto meshes against orc_residual). */
int orc_residual_nodal(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *dudt)
{
    return residual_general(m, cfg, u, dudt);
}

int orc_gradients(const orc_mesh *m, const orc_cfg *cfg, const double *u, double *grad)
{
    if (m->box.nodes == 1) br1_gradients_general(m, cfg, u, grad);
    else br1_gradients(m, cfg, u, grad);
    return 0;
}

void orc_mesh_faces(const orc_mesh *m, double *Sf, double *lb, double *rb)
{
    if (Sf) memcpy(Sf, m->Sf, sizeof(double) * (size_t)m->E * 18 * m->n * m->n);
    if (lb) memcpy(lb, m->lb, sizeof(double) * m->n);
    if (rb) memcpy(rb, m->rb, sizeof(double) * m->n);
}

/* ------------------------------------------------------------------------ */
/* Time step and low-storage RK3 (Sec. 3.7)                                 */
/* ------------------------------------------------------------------------ */

/* Williamson (1980) 3-stage low-storage RK coefficients. */
static const double RK3_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK3_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
static const double RK3_C[3] = {0.0, 1.0 / 3.0, 3.0 / 4.0};

/* Carpenter & Kennedy (1994) 5-stage, fourth-order 2N-storage RK
 * coefficients (their fourth-order five-stage solution; the paper's
 * "explicit Runge-Kutta 4th order" option, Sec. 3.7). */
static const double RK4_A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
static const double RK4_B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                2277821191437.0 / 14882151754819.0};
static const double RK4_C[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                                2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};

static int lsrk_stages(int scheme) { return scheme == 1 ? 5 : 3; }
static const double *lsrk_A(int scheme) { return scheme == 1 ? RK4_A : RK3_A; }
static const double *lsrk_B(int scheme) { return scheme == 1 ? RK4_B : RK3_B; }

void orc_rk3_coefficients(double *A, double *B, double *C)
{
    for (int k = 0; k < 3; ++k) { A[k] = RK3_A[k]; B[k] = RK3_B[k]; C[k] = RK3_C[k]; }
}

void orc_rk4_coefficients(double *A, double *B, double *C)
{
    for (int k = 0; k < 5; ++k) { A[k] = RK4_A[k]; B[k] = RK4_B[k]; C[k] = RK4_C[k]; }
}

/* One low-storage stage on a flat array: g <- A_k g + dt R; u <- u + B_k g.
 * Stage 0 (A_0 = 0) does not read g. */
void orc_lsrk_stage(int scheme, long long count, int k, double dt, double *u, double *g, const double *R)
{
    const double *A = lsrk_A(scheme), *B = lsrk_B(scheme);
    for (long long i = 0; i < count; ++i) {
        double gi = (k == 0) ? dt * R[i] : A[k] * g[i] + dt * R[i];
        g[i] = gi;
        u[i] = u[i] + B[k] * gi;
    }
}

void orc_lsrk3_stage(long long count, int k, double dt, double *u, double *g, const double *R)
{
    orc_lsrk_stage(0, count, k, dt, u, g, R);
}

/* Time step (no formula in the paper; the reading used by this library):
 *   convective  dt_c = cfl * 8 / (n^2 * max_nodes sum_d (|Ja^d.v| + c |Ja^d|)/J)
 *               (the RK3 stability limit of the DGSEM operator shrinks like 1/n^2;
 *               at n = 4 this equals cfl * 2 / (n * ...))
 *   viscous     dt_v = 12 / (n^4 * max_nodes (mu/rho) sum_d (|Ja^d|/J)^2)
 *               (= h^2/(nu n^4) on a straight box; Navier-Stokes only)
 *   dt = min(dt_c, dt_v).
 * On Gauss-Legendre nodes the spectral radius of the operator is about twice
 * that on Gauss-Lobatto nodes (the boundary terms act on interpolated
 * traces), so the constants 8 and 12 become 3 and 4. */
double orc_dt(const orc_mesh *m, const orc_cfg *cfg, const double *u)
{
    int n = m->n, n3 = m->n3, E = m->E;
    double g = cfg->gamma;
    double lam_c = 0.0, lam_v = 0.0;
    double mu = (cfg->physics == 1) ? visc_mu(cfg) : 0.0;
    for (int e = 0; e < E; ++e)
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], rho, v[3], pr;
            for (int vv = 0; vv < NVAR; ++vv) up[vv] = u[((size_t)e * NVAR + vv) * n3 + p];
            primitives(up, g, &rho, v, &pr);
            double c = sqrt(g * pr / rho);
            double Jp = m->J[(size_t)e * n3 + p];
            double sc = 0.0, sv = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double *a0 = m->Ja + (((size_t)e * 3 + d) * 3) * n3 + p;
                double a[3] = {a0[0], a0[n3], a0[2 * n3]};
                double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                sc += (fabs(a[0] * v[0] + a[1] * v[1] + a[2] * v[2]) + c * an) / Jp;
                sv += (an / Jp) * (an / Jp);
            }
            if (sc > lam_c) lam_c = sc;
            if (mu * sv / rho > lam_v) lam_v = mu * sv / rho;
        }
    double kc = (m->box.nodes == 1) ? 3.0 : 8.0, kv = (m->box.nodes == 1) ? 4.0 : 12.0;
    double dt = cfg->cfl * kc / ((double)n * n * lam_c);
    if (lam_v > 0.0) {
        double dtv = kv / ((double)n * n * n * n * lam_v);
        if (dtv < dt) dt = dtv;
    }
    return dt;
}

/* One low-storage RK step of the configured scheme (Williamson RK3 or
 * Carpenter-Kennedy RK4).  dt_in > 0 is used as given; dt_in <= 0 computes dt
 * from the state at the start of the step.  Returns the dt used through *dt_used. */
int orc_rk3_step(const orc_mesh *m, const orc_cfg *cfg, double *u, double *g, double dt_in, double *dt_used)
{
    long long count = (long long)m->E * NVAR * m->n3;
    double dt = dt_in > 0.0 ? dt_in : orc_dt(m, cfg, u);
    double *R = (double *)malloc(sizeof(double) * count);
    if (!R) return -1;
    for (int k = 0; k < lsrk_stages(cfg->time_scheme); ++k) {
        orc_residual(m, cfg, u, R);
        orc_lsrk_stage(cfg->time_scheme, count, k, dt, u, g, R);
    }
    free(R);
    if (dt_used) *dt_used = dt;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Initial conditions                                                        */
/* ------------------------------------------------------------------------ */

static void conservative(double rho, const double v[3], double p, double g, double *u)
{
    u[0] = rho;
    u[1] = rho * v[0];
    u[2] = rho * v[1];
    u[3] = rho * v[2];
    u[4] = p / (g - 1.0) + 0.5 * rho * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
}

/* Isentropic vortex (Shu's form) in the x-y plane, advected at u_inf = Ma sqrt(gamma)
 * along x, free stream rho = p = 1:
 *   r^2 = dx^2 + dy^2 (nearest periodic image of the centre moved to xc + u_inf t),
 *   du = -beta/(2pi) e^{(1-r^2)/2} dy,  dv = beta/(2pi) e^{(1-r^2)/2} dx,
 *   T = 1 - (gamma-1) beta^2/(8 gamma pi^2) e^{1-r^2},  rho = T^{1/(gamma-1)},  p = rho^gamma.
 * An exact solution of the Euler equations; at time t it is the state at t=0
 * translated by u_inf t. */
void orc_ic_vortex(const orc_mesh *m, double g, double Ma, double beta, double xc, double yc, double t, double *u)
{
    int n3 = m->n3, E = m->E;
    double uinf = Ma * sqrt(g);
    double Lx = m->box.hi[0] - m->box.lo[0], Ly = m->box.hi[1] - m->box.lo[1];
    double cx = xc + uinf * t;
    for (int e = 0; e < E; ++e)
        for (int p = 0; p < n3; ++p) {
            double x = m->X[((size_t)e * 3 + 0) * n3 + p];
            double y = m->X[((size_t)e * 3 + 1) * n3 + p];
            double dx = x - cx, dy = y - yc;
            dx -= Lx * floor(dx / Lx + 0.5);
            dy -= Ly * floor(dy / Ly + 0.5);
            double r2 = dx * dx + dy * dy;
            double ex = exp(0.5 * (1.0 - r2));
            double v[3] = {uinf - beta / (2.0 * M_PI) * ex * dy, beta / (2.0 * M_PI) * ex * dx, 0.0};
            double T = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * M_PI * M_PI) * ex * ex;
            double rho = pow(T, 1.0 / (g - 1.0));
            double pr = pow(rho, g);
            double up[NVAR];
            conservative(rho, v, pr, g, up);
            for (int vv = 0; vv < NVAR; ++vv) u[((size_t)e * NVAR + vv) * n3 + p] = up[vv];
        }
}

/* Taylor-Green vortex, rho0 = V0 = L = 1, p0 = 1/(gamma Ma^2):
 *   v1 = sin x cos y cos z,  v2 = -cos x sin y cos z,  v3 = 0,
 *   p = p0 + (cos 2x + cos 2y)(cos 2z + 2)/16,  rho = p/p0. */
void orc_ic_tgv(const orc_mesh *m, double g, double Ma, double *u)
{
    int n3 = m->n3, E = m->E;
    double p0 = 1.0 / (g * Ma * Ma);
    for (int e = 0; e < E; ++e)
        for (int p = 0; p < n3; ++p) {
            double x = m->X[((size_t)e * 3 + 0) * n3 + p];
            double y = m->X[((size_t)e * 3 + 1) * n3 + p];
            double z = m->X[((size_t)e * 3 + 2) * n3 + p];
            double v[3] = {sin(x) * cos(y) * cos(z), -cos(x) * sin(y) * cos(z), 0.0};
            double pr = p0 + (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0) / 16.0;
            double rho = pr / p0;
            double up[NVAR];
            conservative(rho, v, pr, g, up);
            for (int vv = 0; vv < NVAR; ++vv) u[((size_t)e * NVAR + vv) * n3 + p] = up[vv];
        }
}

/* ------------------------------------------------------------------------ */
/* Diagnostics                                                               */
/* ------------------------------------------------------------------------ */

/* Quadrature integrals sum_e sum_ijk J w_i w_j w_k f_v, f = u or du/dt (5 values),
 * plus the entropy rate sum J w w w (w(u) . dudt) in out[5] when dudt is given,
 * and sum |J w w w w_v dudt_v| in out[6] (the scale for relative checks).
 * Sequential, fixed order. */
void orc_integrals(const orc_mesh *m, double g, const double *u, const double *dudt, double *out)
{
    int n = m->n, n3 = m->n3, E = m->E;
    for (int v = 0; v < 7; ++v) out[v] = 0.0;
    for (int e = 0; e < E; ++e)
        for (int k = 0; k < n; ++k) for (int j = 0; j < n; ++j) for (int i = 0; i < n; ++i) {
            int p = node_index(n, i, j, k);
            double wq = m->J[(size_t)e * n3 + p] * m->w[i] * m->w[j] * m->w[k];
            const double *f = dudt ? dudt : u;
            for (int v = 0; v < NVAR; ++v) out[v] += wq * f[((size_t)e * NVAR + v) * n3 + p];
            if (dudt) {
                double up[NVAR], wv[NVAR];
                for (int v = 0; v < NVAR; ++v) up[v] = u[((size_t)e * NVAR + v) * n3 + p];
                orc_entropy_vars(up, g, wv);
                for (int v = 0; v < NVAR; ++v) {
                    double t = wq * wv[v] * dudt[((size_t)e * NVAR + v) * n3 + p];
                    out[5] += t;
                    out[6] += fabs(t);
                }
            }
        }
}

/* ------------------------------------------------------------------------ */
/* Per-element, per-direction polynomial degree with mortar coupling         */
/* (Sec. 3.6)                                                                */
/* ------------------------------------------------------------------------ */
/*
 * Element e of the ex*ey*ez periodic box carries its own degrees
 * (P_x, P_y, P_z) in 1..7, one per reference direction (Sec. 3.6: the order
 * may differ per element and per direction, anisotropic p-adaptation);
 * Gauss-Lobatto nodes n_d = P_d + 1 per direction, n_x n_y n_z per element,
 * node (i, j, k) at i + n_x (j + n_y k).  An isotropic element has
 * P_x = P_y = P_z.  Sec. 3.6 names the two ingredients:
 *
 * Geometry (the rules of Kopriva et al. 2019 for p-non-conforming faces).
 *   Every element's map is the polynomial of degree Ngeo = max(1, floor(Pmin/2))
 *   per direction (Pmin = smallest degree of the mesh, over elements and
 *   directions) that interpolates the box map (with its perturbation) at the
 *   element's Gauss-Lobatto points of degree Ngeo; X is that polynomial at the
 *   element's own nodes and the metric terms are the curl form with the
 *   element's own derivative matrix in each direction.  The products
 *   X_l dX_m of a degree-Ngeo map have degree 2 Ngeo <= Pmin per direction,
 *   so every element interpolates them exactly: the face metric terms are the
 *   same polynomial seen from both sides of a face, whatever the degrees.
 *   With Pmin = 1 that holds only for an affine map, so amp must be 0.
 *
 * Coupling (the mortar method of Kopriva et al. 2002, which Sec. 3.6 notes
 * does not keep entropy stability).  The face normal to direction d between
 * L (its +d face) and R (its -d face) has the tangential directions d0 < d1
 * with degrees (P_L[d0], P_L[d1]) and (P_R[d0], P_R[d1]); it carries a
 * mortar of degree M_k = max(P_L[dk], P_R[dk]) in tangential direction k, on
 * the Gauss-Lobatto points of those degrees:
 *   - the conservative traces of both sides (and, for Navier-Stokes, their
 *     gradients) are interpolated to the mortar points (tensor-product
 *     Lagrange interpolation, each tangential direction with its own pair of
 *     degrees);
 *   - the numerical flux s F*(u_L, u_R; n) - (F_v(L) + F_v(R)).Sn/2 is
 *     evaluated at the mortar points, with Sn the face metric Ja^d of a side
 *     whose tangential degrees are the mortar's (L when both are; R when only
 *     R is); when neither side's are (e.g. (3,5) against (5,3)) it is L's face
 *     metric interpolated to the mortar points, which is exact: the face
 *     metric has degree <= Pmin in each direction;
 *   - the BR1 interface value q* = (q(u_L) + q(u_R))/2 likewise;
 *   - each side receives the L2 projection of the mortar function onto its
 *     own tangential degrees, P = M_s^{-1} S with M_s[i][k] = int l_i l_k and
 *     S[i][j] = int l_i^s l_j^M integrated exactly (Gauss quadrature with
 *     M + 1 points), applied in both face directions; a direction in which
 *     the side's degree is the mortar's takes the identity.
 * With equal degrees on every face this is the conforming method (the
 * mortar is the face itself).
 *
 * State layout: element blocks [5][n_x n_y n_z] in element order, block e at
 * off[e] doubles.
 */
#define PM_MAXN 7

typedef struct {
    orc_box box;       /* ex, ey, ez, lo, hi, amp (N and nodes unused) */
    int E, Nmin, Nmax, Ngeo;
    int *P;            /* [3E] degree of element e in direction d at P[3e + d] */
    long long *off;    /* [E+1] state offsets: element e at off[e], 5 n_x n_y n_z values */
    long long *noff;   /* [E+1] node offsets: element e's nodes at noff[e] */
    double *X;         /* [3][nodes_e] per element at 3 noff[e] */
    double *Ja;        /* [3 d][3 c][nodes_e] per element at 9 noff[e] */
    double *J;         /* [nodes_e] per element at noff[e] */
    double xi[PM_MAXN + 1][16], w[PM_MAXN + 1][16], D[PM_MAXN + 1][256];
    double Pi[PM_MAXN + 1][PM_MAXN + 1][64];  /* Pi[s][m][a*ns + i] = l_i^{(s)}(xi_a^{(m)}), s <= m */
    double Pr[PM_MAXN + 1][PM_MAXN + 1][64];  /* Pr[s][m][i*nm + j]: L2 projection, degree m -> s, s <= m */
} orc_pmesh;

/* Nodes per direction of element e, and their product. */
static void pm_shape(const orc_pmesh *m, int e, int n[3])
{
    for (int d = 0; d < 3; ++d) n[d] = m->P[3 * e + d] + 1;
}
static int pm_nodes(const int n[3]) { return n[0] * n[1] * n[2]; }
static int aidx(const int n[3], int i, int j, int k) { return i + n[0] * (j + n[1] * k); }

/* Index of the node with index mm along direction d, the other two indices
 * taken from (i, j, k). */
static int anode_along(const int n[3], int d, int mm, int i, int j, int k)
{
    if (d == 0) return aidx(n, mm, j, k);
    if (d == 1) return aidx(n, i, mm, k);
    return aidx(n, i, j, mm);
}

/* Derivative along reference direction d of a nodal field f of one element
 * with n[d] nodes in that direction, D the derivative matrix of degree n[d]-1:
 * (D_d f)_ijk = sum_m D[ind_d][m] f(node with ind_d -> m). */
static double adir_derivative(const int n[3], const double *D, const double *f, int d, int i, int j, int k)
{
    int row = (d == 0) ? i : (d == 1) ? j : k;
    double s = 0.0;
    for (int mm = 0; mm < n[d]; ++mm) s += D[row * n[d] + mm] * f[anode_along(n, d, mm, i, j, k)];
    return s;
}

/* The curl-form metric terms and J of one element with n[d] nodes per
 * direction (the formulas of orc_metrics, each derivative along d with the
 * derivative matrix Dd[d] of that direction's degree). */
static int ametrics(const int n[3], const double *const Dd[3], const double *X, double *Ja, double *J)
{
    int n3 = pm_nodes(n);
    double *tmp = (double *)malloc(sizeof(double) * n3 * 2);
    double *dX = (double *)malloc(sizeof(double) * n3 * 9);   /* dX[c][d][node] */
    if (!tmp || !dX) { free(tmp); free(dX); return -1; }
    for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d)
    for (int k = 0; k < n[2]; ++k) for (int j = 0; j < n[1]; ++j) for (int i = 0; i < n[0]; ++i)
        dX[(c * 3 + d) * n3 + aidx(n, i, j, k)] = adir_derivative(n, Dd[d], X + c * n3, d, i, j, k);
    for (int p = 0; p < n3; ++p) {
        double a[3][3];
        for (int d = 0; d < 3; ++d) for (int c = 0; c < 3; ++c) a[d][c] = dX[(c * 3 + d) * n3 + p];
        double cx = a[1][1] * a[2][2] - a[1][2] * a[2][1];
        double cy = a[1][2] * a[2][0] - a[1][0] * a[2][2];
        double cz = a[1][0] * a[2][1] - a[1][1] * a[2][0];
        J[p] = a[0][0] * cx + a[0][1] * cy + a[0][2] * cz;
    }
    for (int i = 0; i < 3; ++i) {
        int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        for (int c = 0; c < 3; ++c) {
            int mc = (c + 1) % 3, l = (c + 2) % 3;
            for (int p = 0; p < n3; ++p) {
                tmp[p] = X[l * n3 + p] * dX[(mc * 3 + i1) * n3 + p];
                tmp[n3 + p] = X[l * n3 + p] * dX[(mc * 3 + i2) * n3 + p];
            }
            for (int k = 0; k < n[2]; ++k) for (int j = 0; j < n[1]; ++j) for (int ii = 0; ii < n[0]; ++ii) {
                int p = aidx(n, ii, j, k);
                Ja[(i * 3 + c) * n3 + p] = adir_derivative(n, Dd[i2], tmp, i2, ii, j, k)
                                         - adir_derivative(n, Dd[i1], tmp + n3, i1, ii, j, k);
            }
        }
    }
    free(tmp); free(dX);
    return 0;
}

/* Interpolation from degree Ns to degree Nm >= Ns (Gauss-Lobatto points) and
 * the L2 projection back, as nm x ns and ns x nm row-major matrices.  Equal
 * degrees give identities. */
int orc_mortar_matrices(int Ns, int Nm, double *Pi, double *P)
{
    if (Ns < 1 || Nm < Ns || Nm > 15) return -1;
    int ns = Ns + 1, nm = Nm + 1;
    double xs[16], ws[16], xm[16], wm[16];
    orc_lgl(Ns, xs, ws);
    orc_lgl(Nm, xm, wm);
    if (Ns == Nm) {
        for (int a = 0; a < nm; ++a)
            for (int i = 0; i < ns; ++i) Pi[a * ns + i] = P[a * ns + i] = (a == i) ? 1.0 : 0.0;
        return 0;
    }
    for (int a = 0; a < nm; ++a) orc_lagrange_at(ns, xs, xm[a], Pi + a * ns);
    /* exact integrals of products of degree <= 2 Nm with Nm + 1 Gauss points */
    double xg[16], wg[16];
    orc_gauss(Nm, xg, wg);
    double M[16 * 16], S[16 * 16];
    for (int i = 0; i < ns; ++i) {
        for (int k = 0; k < ns; ++k) M[i * ns + k] = 0.0;
        for (int j = 0; j < nm; ++j) S[i * nm + j] = 0.0;
    }
    for (int q = 0; q < Nm + 1; ++q) {
        double ls[16], lm[16];
        orc_lagrange_at(ns, xs, xg[q], ls);
        orc_lagrange_at(nm, xm, xg[q], lm);
        for (int i = 0; i < ns; ++i) {
            for (int k = 0; k < ns; ++k) M[i * ns + k] += wg[q] * ls[i] * ls[k];
            for (int j = 0; j < nm; ++j) S[i * nm + j] += wg[q] * ls[i] * lm[j];
        }
    }
    /* solve M P = S by Gaussian elimination with partial pivoting */
    for (int c = 0; c < ns; ++c) {
        int piv = c;
        for (int r = c + 1; r < ns; ++r)
            if (fabs(M[r * ns + c]) > fabs(M[piv * ns + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < ns; ++k) { double t = M[c * ns + k]; M[c * ns + k] = M[piv * ns + k]; M[piv * ns + k] = t; }
            for (int j = 0; j < nm; ++j) { double t = S[c * nm + j]; S[c * nm + j] = S[piv * nm + j]; S[piv * nm + j] = t; }
        }
        for (int r = c + 1; r < ns; ++r) {
            double f = M[r * ns + c] / M[c * ns + c];
            for (int k = c; k < ns; ++k) M[r * ns + k] -= f * M[c * ns + k];
            for (int j = 0; j < nm; ++j) S[r * nm + j] -= f * S[c * nm + j];
        }
    }
    for (int c = ns - 1; c >= 0; --c)
        for (int j = 0; j < nm; ++j) {
            double acc = S[c * nm + j];
            for (int k = c + 1; k < ns; ++k) acc -= M[c * ns + k] * P[k * nm + j];
            P[c * nm + j] = acc / M[c * ns + c];
        }
    return 0;
}

/* The box map at reference point r (in [-1,1]^3) of element e: the affine
 * box position plus the perturbation amp (L_c/2pi) sin(t_x) sin(t_y) sin(t_z)
 * of the unperturbed position, t the position mapped to [-pi, pi]. */
static void box_map_point(const orc_box *b, int e, const double r[3], double X[3])
{
    int E3[3] = {b->ex, b->ey, b->ez};
    int ab[3] = {e % b->ex, (e / b->ex) % b->ey, e / (b->ex * b->ey)};
    double x0[3], th[3];
    for (int c = 0; c < 3; ++c) {
        double L = b->hi[c] - b->lo[c];
        x0[c] = b->lo[c] + (L / E3[c]) * (ab[c] + 0.5 * (r[c] + 1.0));
        th[c] = -M_PI + 2.0 * M_PI * (x0[c] - b->lo[c]) / L;
    }
    double s = sin(th[0]) * sin(th[1]) * sin(th[2]);
    for (int c = 0; c < 3; ++c) X[c] = x0[c] + b->amp * ((b->hi[c] - b->lo[c]) / (2.0 * M_PI)) * s;
}

void orc_pmesh_destroy(orc_pmesh *m)
{
    if (!m) return;
    free(m->P); free(m->off); free(m->noff); free(m->X); free(m->Ja); free(m->J); free(m);
}

/* Degrees deg3[3e + d] (element e, direction d), each in 1..PM_MAXN. */
orc_pmesh *orc_pmesh_create3(const orc_box *b, const int *deg3)
{
    if (b->ex < 1 || b->ey < 1 || b->ez < 1 || !deg3) return NULL;
    int E = b->ex * b->ey * b->ez;
    int Nmin = 99, Nmax = 0;
    for (int t = 0; t < 3 * E; ++t) {
        if (deg3[t] < 1 || deg3[t] > PM_MAXN) return NULL;
        if (deg3[t] < Nmin) Nmin = deg3[t];
        if (deg3[t] > Nmax) Nmax = deg3[t];
    }
    if (Nmin == 1 && b->amp != 0.0) return NULL;
    orc_pmesh *m = (orc_pmesh *)calloc(1, sizeof(orc_pmesh));
    if (!m) return NULL;
    m->box = *b;
    m->E = E;
    m->Nmin = Nmin;
    m->Nmax = Nmax;
    m->Ngeo = Nmin / 2 >= 1 ? Nmin / 2 : 1;
    m->P = (int *)malloc(sizeof(int) * 3 * E);
    m->off = (long long *)malloc(sizeof(long long) * (E + 1));
    m->noff = (long long *)malloc(sizeof(long long) * (E + 1));
    if (!m->P || !m->off || !m->noff) { orc_pmesh_destroy(m); return NULL; }
    memcpy(m->P, deg3, sizeof(int) * 3 * E);
    m->off[0] = m->noff[0] = 0;
    for (int e = 0; e < E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        m->noff[e + 1] = m->noff[e] + pm_nodes(n);
        m->off[e + 1] = m->off[e] + 5LL * pm_nodes(n);
    }
    for (int N = 1; N <= PM_MAXN; ++N) {
        orc_lgl(N, m->xi[N], m->w[N]);
        orc_dmatrix(N, m->xi[N], m->D[N]);
    }
    for (int s = 1; s <= PM_MAXN; ++s)
        for (int t = s; t <= PM_MAXN; ++t) orc_mortar_matrices(s, t, m->Pi[s][t], m->Pr[s][t]);
    long long nodes = m->noff[E];
    m->X = (double *)malloc(sizeof(double) * 3 * nodes);
    m->Ja = (double *)malloc(sizeof(double) * 9 * nodes);
    m->J = (double *)malloc(sizeof(double) * nodes);
    if (!m->X || !m->Ja || !m->J) { orc_pmesh_destroy(m); return NULL; }
    int G = m->Ngeo, ng = G + 1;
    for (int e = 0; e < E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        int n3 = pm_nodes(n);
        /* the map at the degree-Ngeo points, then its interpolant at the own nodes */
        double Xg[3][512];
        for (int k = 0; k < ng; ++k) for (int j = 0; j < ng; ++j) for (int i = 0; i < ng; ++i) {
            double r[3] = {m->xi[G][i], m->xi[G][j], m->xi[G][k]}, x[3];
            box_map_point(b, e, r, x);
            for (int c = 0; c < 3; ++c) Xg[c][node_index(ng, i, j, k)] = x[c];
        }
        double L[3][16][16];   /* L[d][t][s] = l_s^{(Ngeo)}(xi_t^{(P_d)}) */
        for (int d = 0; d < 3; ++d)
            for (int t = 0; t < n[d]; ++t) orc_lagrange_at(ng, m->xi[G], m->xi[n[d] - 1][t], L[d][t]);
        double *Xe = m->X + 3 * m->noff[e];
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < n[2]; ++k) for (int j = 0; j < n[1]; ++j) for (int i = 0; i < n[0]; ++i) {
                double acc = 0.0;
                for (int kk = 0; kk < ng; ++kk) for (int jj = 0; jj < ng; ++jj) for (int ii = 0; ii < ng; ++ii)
                    acc += L[0][i][ii] * L[1][j][jj] * L[2][k][kk] * Xg[c][node_index(ng, ii, jj, kk)];
                Xe[c * n3 + aidx(n, i, j, k)] = acc;
            }
        const double *Dd[3] = {m->D[n[0] - 1], m->D[n[1] - 1], m->D[n[2] - 1]};
        if (ametrics(n, Dd, Xe, m->Ja + 9 * m->noff[e], m->J + m->noff[e]) != 0) {
            orc_pmesh_destroy(m);
            return NULL;
        }
    }
    return m;
}

/* Isotropic degrees: deg[e] in every direction. */
orc_pmesh *orc_pmesh_create(const orc_box *b, const int *deg)
{
    if (b->ex < 1 || b->ey < 1 || b->ez < 1 || !deg) return NULL;
    int E = b->ex * b->ey * b->ez;
    int *deg3 = (int *)malloc(sizeof(int) * 3 * E);
    if (!deg3) return NULL;
    for (int e = 0; e < E; ++e) deg3[3 * e] = deg3[3 * e + 1] = deg3[3 * e + 2] = deg[e];
    orc_pmesh *m = orc_pmesh_create3(b, deg3);
    free(deg3);
    return m;
}

int orc_pmesh_E(const orc_pmesh *m) { return m->E; }
int orc_pmesh_Ngeo(const orc_pmesh *m) { return m->Ngeo; }

/* Copies of the mesh arrays: off [E+1], noff [E+1], X [3 nodes], Ja [9 nodes], J [nodes]
 * (each element's blocks at 3 noff[e], 9 noff[e], noff[e]). */
void orc_pmesh_arrays(const orc_pmesh *m, long long *off, long long *noff, double *X, double *Ja, double *J)
{
    long long nodes = m->noff[m->E];
    if (off) memcpy(off, m->off, sizeof(long long) * (m->E + 1));
    if (noff) memcpy(noff, m->noff, sizeof(long long) * (m->E + 1));
    if (X) memcpy(X, m->X, sizeof(double) * 3 * nodes);
    if (Ja) memcpy(Ja, m->Ja, sizeof(double) * 9 * nodes);
    if (J) memcpy(J, m->J, sizeof(double) * nodes);
}

/* nf fields of one element ([nf][nodes] from base, n[d] nodes per direction)
 * on its face xi_d = end: out[v][ta + n[d0] tb], (ta, tb) the face's
 * tangential indices in increasing direction order. */
static void pm_face_values(const double *base, int nf, const int n[3], int d, int end, double *out)
{
    int n3 = pm_nodes(n), d0, d1;
    face_dirs(d, &d0, &d1);
    int f2 = n[d0] * n[d1];
    for (int v = 0; v < nf; ++v)
        for (int tb = 0; tb < n[d1]; ++tb) for (int ta = 0; ta < n[d0]; ++ta) {
            int idx[3];
            idx[d] = end;
            idx[d0] = ta;
            idx[d1] = tb;
            out[v * f2 + ta + n[d0] * tb] = base[(size_t)v * n3 + aidx(n, idx[0], idx[1], idx[2])];
        }
}

/* Face field of degrees (S0, S1) -> mortar of degrees (M0, M1), Sk <= Mk
 * (tensor-product interpolation, fm[a + (M0+1) b]). */
static void pm_to_mortar(const orc_pmesh *m, int S0, int S1, int M0, int M1, const double *fs, double *fm)
{
    int ns0 = S0 + 1, ns1 = S1 + 1, nm0 = M0 + 1, nm1 = M1 + 1;
    const double *I0 = m->Pi[S0][M0], *I1 = m->Pi[S1][M1];
    for (int b = 0; b < nm1; ++b) for (int a = 0; a < nm0; ++a) {
        double acc = 0.0;
        for (int j = 0; j < ns1; ++j)
            for (int i = 0; i < ns0; ++i) acc += I0[a * ns0 + i] * I1[b * ns1 + j] * fs[i + ns0 * j];
        fm[a + nm0 * b] = acc;
    }
}

/* Mortar field of degrees (M0, M1) -> face of degrees (S0, S1) (tensor-product
 * L2 projection). */
static void pm_from_mortar(const orc_pmesh *m, int M0, int M1, int S0, int S1, const double *fm, double *fs)
{
    int ns0 = S0 + 1, ns1 = S1 + 1, nm0 = M0 + 1, nm1 = M1 + 1;
    const double *P0 = m->Pr[S0][M0], *P1 = m->Pr[S1][M1];
    for (int b = 0; b < ns1; ++b) for (int a = 0; a < ns0; ++a) {
        double acc = 0.0;
        for (int j = 0; j < nm1; ++j)
            for (int i = 0; i < nm0; ++i) acc += P0[a * nm0 + i] * P1[b * nm1 + j] * fm[i + nm0 * j];
        fs[a + ns0 * b] = acc;
    }
}

/* The mortar computation for face (d, side) of element e, returned on e's own
 * face nodes (out[v][ta + n_e[d0] tb]):
 *   mode 0: the BR1 interface value q* (4 values);
 *   mode 1: the face flux s F*(u_L, u_R; n) - (F_v(L) + F_v(R)).Sn/2 oriented along +d (5 values).
 * L is the element on the face's minus side, R on its plus side. */
static void pm_mortar(const orc_pmesh *m, const orc_cfg *cfg, const double *u, const double *grad, int e, int d,
                      int side, int mode, double *out)
{
    int nb = neighbour(&m->box, e, d, side);
    int eL = side > 0 ? e : nb, eR = side > 0 ? nb : e;
    int d0, d1;
    face_dirs(d, &d0, &d1);
    int nLs[3], nRs[3];
    pm_shape(m, eL, nLs);
    pm_shape(m, eR, nRs);
    int L0 = nLs[d0] - 1, L1 = nLs[d1] - 1, R0 = nRs[d0] - 1, R1 = nRs[d1] - 1;
    int M0 = L0 > R0 ? L0 : R0, M1 = L1 > R1 ? L1 : R1;
    int fL = (L0 + 1) * (L1 + 1), fR = (R0 + 1) * (R1 + 1), nM2 = (M0 + 1) * (M1 + 1);
    double g = cfg->gamma;
    double tL[NVAR * 64], tR[NVAR * 64], mL[NVAR * 64], mR[NVAR * 64];
    pm_face_values(u + m->off[eL], NVAR, nLs, d, nLs[d] - 1, tL);
    pm_face_values(u + m->off[eR], NVAR, nRs, d, 0, tR);
    for (int v = 0; v < NVAR; ++v) {
        pm_to_mortar(m, L0, L1, M0, M1, tL + v * fL, mL + v * nM2);
        pm_to_mortar(m, R0, R1, M0, M1, tR + v * fR, mR + v * nM2);
    }
    int nv = mode == 0 ? NGRAD : NVAR;
    double fM[NVAR * 64];
    if (mode == 0) {
        for (int p = 0; p < nM2; ++p) {
            double uL[NVAR], uR[NVAR], qL[NGRAD], qR[NGRAD];
            for (int v = 0; v < NVAR; ++v) { uL[v] = mL[v * nM2 + p]; uR[v] = mR[v * nM2 + p]; }
            grad_vars(uL, g, qL);
            grad_vars(uR, g, qR);
            for (int v = 0; v < NGRAD; ++v) fM[v * nM2 + p] = 0.5 * (qL[v] + qR[v]);
        }
    } else {
        /* the face metric at the mortar points */
        double Sn[3 * 64];
        int nL3 = pm_nodes(nLs), nR3 = pm_nodes(nRs);
        if (L0 == M0 && L1 == M1) {
            pm_face_values(m->Ja + 9 * m->noff[eL] + (size_t)d * 3 * nL3, 3, nLs, d, nLs[d] - 1, Sn);
        } else if (R0 == M0 && R1 == M1) {
            pm_face_values(m->Ja + 9 * m->noff[eR] + (size_t)d * 3 * nR3, 3, nRs, d, 0, Sn);
        } else {
            double SL[3 * 64];
            pm_face_values(m->Ja + 9 * m->noff[eL] + (size_t)d * 3 * nL3, 3, nLs, d, nLs[d] - 1, SL);
            for (int c = 0; c < 3; ++c) pm_to_mortar(m, L0, L1, M0, M1, SL + c * fL, Sn + c * nM2);
        }
        double gL[12 * 64], gR[12 * 64], gmL[12 * 64], gmR[12 * 64];
        int ns = cfg->physics == 1;
        if (ns) {
            pm_face_values(grad + 12 * m->noff[eL], 12, nLs, d, nLs[d] - 1, gL);
            pm_face_values(grad + 12 * m->noff[eR], 12, nRs, d, 0, gR);
            for (int k = 0; k < 12; ++k) {
                pm_to_mortar(m, L0, L1, M0, M1, gL + k * fL, gmL + k * nM2);
                pm_to_mortar(m, R0, R1, M0, M1, gR + k * fR, gmR + k * nM2);
            }
        }
        double mu = ns ? visc_mu(cfg) : 0.0, kappa = ns ? visc_kappa(cfg) : 0.0;
        for (int p = 0; p < nM2; ++p) {
            double uL[NVAR], uR[NVAR], s[3] = {Sn[p], Sn[nM2 + p], Sn[2 * nM2 + p]}, f[NVAR];
            for (int v = 0; v < NVAR; ++v) { uL[v] = mL[v * nM2 + p]; uR[v] = mR[v * nM2 + p]; }
            surface_flux(cfg->surface_flux, uL, uR, s, g, f);
            if (ns) {
                double qL[NGRAD], qR[NGRAD], GL[12], GR[12], fvL[NVAR], fvR[NVAR];
                grad_vars(uL, g, qL);
                grad_vars(uR, g, qR);
                for (int k = 0; k < 12; ++k) { GL[k] = gmL[k * nM2 + p]; GR[k] = gmR[k * nM2 + p]; }
                orc_flux_visc(qL, GL, mu, kappa, s, fvL);
                orc_flux_visc(qR, GR, mu, kappa, s, fvR);
                for (int v = 0; v < NVAR; ++v) f[v] -= 0.5 * (fvL[v] + fvR[v]);
            }
            for (int v = 0; v < NVAR; ++v) fM[v * nM2 + p] = f[v];
        }
    }
    int ne[3];
    pm_shape(m, e, ne);
    int E0 = ne[d0] - 1, E1 = ne[d1] - 1;
    for (int v = 0; v < nv; ++v) pm_from_mortar(m, M0, M1, E0, E1, fM + v * nM2, out + v * (E0 + 1) * (E1 + 1));
}

/* BR1 gradients on the p-non-conforming mesh, grad per element [4][3][nodes_e]
 * at 12 noff[e]:
 *   J grad q_c = sum_d D_d (Ja^d_c q) + sum_faces (1/w_end) (q*_e - q_in) (+-Ja^d_c),
 * D_d and w of the element's degree in direction d, q*_e the mortar interface
 * value projected onto the element's face. */
static void pm_br1(const orc_pmesh *m, const orc_cfg *cfg, const double *u, double *grad)
{
    double g = cfg->gamma;
#pragma omp parallel for schedule(dynamic)
    for (int e = 0; e < m->E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        int n3 = pm_nodes(n);
        const double *Dd[3] = {m->D[n[0] - 1], m->D[n[1] - 1], m->D[n[2] - 1]};
        const double *Ja = m->Ja + 9 * m->noff[e], *J = m->J + m->noff[e];
        const double *ue = u + m->off[e];
        double *G = grad + 12 * m->noff[e];
        double q[NGRAD * 512], f[3 * 512];
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], qp[NGRAD];
            for (int v = 0; v < NVAR; ++v) up[v] = ue[v * n3 + p];
            grad_vars(up, g, qp);
            for (int v = 0; v < NGRAD; ++v) q[v * n3 + p] = qp[v];
        }
        for (int v = 0; v < NGRAD; ++v)
        for (int c = 0; c < 3; ++c) {
            for (int d = 0; d < 3; ++d)
                for (int p = 0; p < n3; ++p) f[d * n3 + p] = Ja[(d * 3 + c) * n3 + p] * q[v * n3 + p];
            for (int k = 0; k < n[2]; ++k) for (int j = 0; j < n[1]; ++j) for (int i = 0; i < n[0]; ++i) {
                double acc = 0.0;
                for (int d = 0; d < 3; ++d) acc += adir_derivative(n, Dd[d], f + d * n3, d, i, j, k);
                G[(v * 3 + c) * n3 + aidx(n, i, j, k)] = acc;
            }
        }
        for (int d = 0; d < 3; ++d)
        for (int side = -1; side <= 1; side += 2) {
            double qs[NGRAD * 64];
            pm_mortar(m, cfg, u, NULL, e, d, side, 0, qs);
            int at = side > 0 ? n[d] - 1 : 0, d0, d1;
            face_dirs(d, &d0, &d1);
            int f2 = n[d0] * n[d1];
            const double *w = m->w[n[d] - 1];
            for (int tb = 0; tb < n[d1]; ++tb) for (int ta = 0; ta < n[d0]; ++ta) {
                int idx[3];
                idx[d] = at;
                idx[d0] = ta;
                idx[d1] = tb;
                int p = aidx(n, idx[0], idx[1], idx[2]);
                for (int v = 0; v < NGRAD; ++v) {
                    double jump = qs[v * f2 + ta + n[d0] * tb] - q[v * n3 + p];
                    for (int c = 0; c < 3; ++c)
                        G[(v * 3 + c) * n3 + p] += jump * side * Ja[(d * 3 + c) * n3 + p] / w[at];
                }
            }
        }
        for (int k = 0; k < 12; ++k)
            for (int p = 0; p < n3; ++p) G[k * n3 + p] /= J[p];
    }
}

int orc_pgradients(const orc_pmesh *m, const orc_cfg *cfg, const double *u, double *grad)
{
    pm_br1(m, cfg, u, grad);
    return 0;
}

/* du/dt = -(V + S)/J per element of the p-non-conforming mesh: the volume
 * term exactly as on a conforming mesh (standard or split form), each
 * direction d with the derivative matrix of the element's degree in d, and
 * the surface term
 *   S = (1/w_end) [ +-F*_e - (F_e - F_v)(in).(+-Ja^d_in) ]
 * with F*_e the mortar flux projected onto the element's face and w_end the
 * end weight of the element's degree in d. */
int orc_presidual(const orc_pmesh *m, const orc_cfg *cfg, const double *u, double *dudt)
{
    double g = cfg->gamma;
    int ns = cfg->physics == 1;
    double mu = ns ? visc_mu(cfg) : 0.0, kappa = ns ? visc_kappa(cfg) : 0.0;
    double *grad = NULL;
    if (ns) {
        grad = (double *)malloc(sizeof(double) * 12 * m->noff[m->E]);
        if (!grad) return -1;
        pm_br1(m, cfg, u, grad);
    }
#pragma omp parallel for schedule(dynamic)
    for (int e = 0; e < m->E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        int n3 = pm_nodes(n);
        const double *Dd[3] = {m->D[n[0] - 1], m->D[n[1] - 1], m->D[n[2] - 1]};
        const double *Ja = m->Ja + 9 * m->noff[e], *J = m->J + m->noff[e];
        const double *ue = u + m->off[e];
        double *Ft = (double *)malloc(sizeof(double) * 3 * NVAR * n3);
        double *Fv = (double *)malloc(sizeof(double) * 3 * NVAR * n3);
        double *R = (double *)calloc(NVAR * n3, sizeof(double));
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], qp[NGRAD], G[12];
            for (int v = 0; v < NVAR; ++v) up[v] = ue[v * n3 + p];
            if (ns) {
                grad_vars(up, g, qp);
                for (int k = 0; k < 12; ++k) G[k] = grad[12 * m->noff[e] + (size_t)k * n3 + p];
            }
            for (int d = 0; d < 3; ++d) {
                double a[3] = {Ja[(d * 3) * n3 + p], Ja[(d * 3 + 1) * n3 + p], Ja[(d * 3 + 2) * n3 + p]};
                double fe[NVAR], fv[NVAR] = {0, 0, 0, 0, 0};
                orc_flux_euler(up, a, g, fe);
                if (ns) orc_flux_visc(qp, G, mu, kappa, a, fv);
                for (int v = 0; v < NVAR; ++v) {
                    Ft[(d * NVAR + v) * n3 + p] = fe[v] - fv[v];
                    Fv[(d * NVAR + v) * n3 + p] = fv[v];
                }
            }
        }
        for (int k = 0; k < n[2]; ++k) for (int j = 0; j < n[1]; ++j) for (int i = 0; i < n[0]; ++i) {
            int p = aidx(n, i, j, k), ijk[3] = {i, j, k};
            for (int d = 0; d < 3; ++d) {
                if (cfg->volume_form == 0) {
                    for (int v = 0; v < NVAR; ++v)
                        R[v * n3 + p] += adir_derivative(n, Dd[d], Ft + (d * NVAR + v) * n3, d, i, j, k);
                    continue;
                }
                double ui[NVAR];
                for (int v = 0; v < NVAR; ++v) ui[v] = ue[v * n3 + p];
                for (int mm = 0; mm < n[d]; ++mm) {
                    int pm = anode_along(n, d, mm, i, j, k);
                    double um[NVAR], a[3], fs[NVAR];
                    for (int v = 0; v < NVAR; ++v) um[v] = ue[v * n3 + pm];
                    for (int c = 0; c < 3; ++c) a[c] = 0.5 * (Ja[(d * 3 + c) * n3 + p] + Ja[(d * 3 + c) * n3 + pm]);
                    split_flux(cfg->volume_form, ui, um, a, g, fs);
                    for (int v = 0; v < NVAR; ++v) R[v * n3 + p] += 2.0 * Dd[d][ijk[d] * n[d] + mm] * fs[v];
                }
                if (ns)
                    for (int v = 0; v < NVAR; ++v)
                        R[v * n3 + p] -= adir_derivative(n, Dd[d], Fv + (d * NVAR + v) * n3, d, i, j, k);
            }
        }
        for (int d = 0; d < 3; ++d)
        for (int side = -1; side <= 1; side += 2) {
            double fs[NVAR * 64];
            pm_mortar(m, cfg, u, grad, e, d, side, 1, fs);
            int at = side > 0 ? n[d] - 1 : 0, d0, d1;
            face_dirs(d, &d0, &d1);
            int f2 = n[d0] * n[d1];
            const double *w = m->w[n[d] - 1];
            for (int tb = 0; tb < n[d1]; ++tb) for (int ta = 0; ta < n[d0]; ++ta) {
                int idx[3];
                idx[d] = at;
                idx[d0] = ta;
                idx[d1] = tb;
                int p = aidx(n, idx[0], idx[1], idx[2]);
                for (int v = 0; v < NVAR; ++v)
                    R[v * n3 + p] += (side * fs[v * f2 + ta + n[d0] * tb] - side * Ft[(d * NVAR + v) * n3 + p]) / w[at];
            }
        }
        for (int v = 0; v < NVAR; ++v)
            for (int p = 0; p < n3; ++p) dudt[m->off[e] + (size_t)v * n3 + p] = -R[v * n3 + p] / J[p];
        free(Ft); free(Fv); free(R);
    }
    free(grad);
    return 0;
}

/* Time step on the p-non-conforming mesh: the conforming rule per element
 * with each direction's resolution n_d^2 inside the sum (the reference grid
 * spacing of degree P_d scales like 1/n_d^2; an isotropic element gives the
 * conforming rule with n^2 taken outside, the same value up to rounding),
 * minimised over the elements:
 *   dt = min_e min( cfl 8 / max_nodes sum_d n_d^2 (|Ja^d.v| + c|Ja^d|)/J,
 *                   12 / max_nodes (mu/rho) sum_d n_d^4 (|Ja^d|/J)^2 ). */
double orc_pdt(const orc_pmesh *m, const orc_cfg *cfg, const double *u)
{
    double g = cfg->gamma, mu = cfg->physics == 1 ? visc_mu(cfg) : 0.0, dt = INFINITY;
    for (int e = 0; e < m->E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        int n3 = pm_nodes(n);
        const double *Ja = m->Ja + 9 * m->noff[e], *J = m->J + m->noff[e];
        double lam_c = 0.0, lam_v = 0.0;
        for (int p = 0; p < n3; ++p) {
            double up[NVAR], rho, v[3], pr;
            for (int vv = 0; vv < NVAR; ++vv) up[vv] = u[m->off[e] + (size_t)vv * n3 + p];
            primitives(up, g, &rho, v, &pr);
            double c = sqrt(g * pr / rho), sc = 0.0, sv = 0.0;
            for (int d = 0; d < 3; ++d) {
                double a[3] = {Ja[(d * 3) * n3 + p], Ja[(d * 3 + 1) * n3 + p], Ja[(d * 3 + 2) * n3 + p]};
                double an = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
                double n2 = (double)n[d] * n[d];
                sc += n2 * (fabs(a[0] * v[0] + a[1] * v[1] + a[2] * v[2]) + c * an) / J[p];
                sv += n2 * n2 * (an / J[p]) * (an / J[p]);
            }
            if (sc > lam_c) lam_c = sc;
            if (mu * sv / rho > lam_v) lam_v = mu * sv / rho;
        }
        double dte = cfg->cfl * 8.0 / lam_c;
        if (lam_v > 0.0) {
            double dtv = 12.0 / lam_v;
            if (dtv < dte) dte = dtv;
        }
        if (dte < dt) dt = dte;
    }
    return dt;
}

int orc_prk_step(const orc_pmesh *m, const orc_cfg *cfg, double *u, double *g, double dt_in, double *dt_used)
{
    long long count = m->off[m->E];
    double dt = dt_in > 0.0 ? dt_in : orc_pdt(m, cfg, u);
    double *R = (double *)malloc(sizeof(double) * count);
    if (!R) return -1;
    for (int k = 0; k < lsrk_stages(cfg->time_scheme); ++k) {
        orc_presidual(m, cfg, u, R);
        orc_lsrk_stage(cfg->time_scheme, count, k, dt, u, g, R);
    }
    free(R);
    if (dt_used) *dt_used = dt;
    return 0;
}

/* Taylor-Green vortex (kind 0: gamma, Ma) or isentropic vortex (kind 1:
 * gamma, Ma, beta, xc, yc) at the nodes of the p-non-conforming mesh, the
 * same point formulas as orc_ic_tgv / orc_ic_vortex (t = 0). */
void orc_pic(const orc_pmesh *m, int kind, const double *par, double *u)
{
    double g = par[0], Ma = par[1];
    double p0 = 1.0 / (g * Ma * Ma);
    double Lx = m->box.hi[0] - m->box.lo[0], Ly = m->box.hi[1] - m->box.lo[1];
    for (int e = 0; e < m->E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        int n3 = pm_nodes(n);
        const double *X = m->X + 3 * m->noff[e];
        for (int p = 0; p < n3; ++p) {
            double x = X[p], y = X[n3 + p], z = X[2 * n3 + p], v[3], pr, rho, up[NVAR];
            if (kind == 0) {
                v[0] = sin(x) * cos(y) * cos(z);
                v[1] = -cos(x) * sin(y) * cos(z);
                v[2] = 0.0;
                pr = p0 + (cos(2.0 * x) + cos(2.0 * y)) * (cos(2.0 * z) + 2.0) / 16.0;
                rho = pr / p0;
            } else {
                double beta = par[2], dx = x - par[3], dy = y - par[4], uinf = Ma * sqrt(g);
                dx -= Lx * floor(dx / Lx + 0.5);
                dy -= Ly * floor(dy / Ly + 0.5);
                double ex = exp(0.5 * (1.0 - dx * dx - dy * dy));
                v[0] = uinf - beta / (2.0 * M_PI) * ex * dy;
                v[1] = beta / (2.0 * M_PI) * ex * dx;
                v[2] = 0.0;
                double T = 1.0 - (g - 1.0) * beta * beta / (8.0 * g * M_PI * M_PI) * ex * ex;
                rho = pow(T, 1.0 / (g - 1.0));
                pr = pow(rho, g);
            }
            conservative(rho, v, pr, g, up);
            for (int vv = 0; vv < NVAR; ++vv) u[m->off[e] + (size_t)vv * n3 + p] = up[vv];
        }
    }
}

/* Quadrature integrals on the p-non-conforming mesh (each element with its
 * own weights per direction), as orc_integrals. */
void orc_pintegrals(const orc_pmesh *m, double g, const double *u, const double *dudt, double *out)
{
    for (int v = 0; v < 7; ++v) out[v] = 0.0;
    for (int e = 0; e < m->E; ++e) {
        int n[3];
        pm_shape(m, e, n);
        int n3 = pm_nodes(n);
        const double *wx = m->w[n[0] - 1], *wy = m->w[n[1] - 1], *wz = m->w[n[2] - 1], *J = m->J + m->noff[e];
        const double *f = (dudt ? dudt : u) + m->off[e];
        for (int k = 0; k < n[2]; ++k) for (int j = 0; j < n[1]; ++j) for (int i = 0; i < n[0]; ++i) {
            int p = aidx(n, i, j, k);
            double wq = J[p] * wx[i] * wy[j] * wz[k];
            for (int v = 0; v < NVAR; ++v) out[v] += wq * f[(size_t)v * n3 + p];
            if (dudt) {
                double up[NVAR], wv[NVAR];
                for (int v = 0; v < NVAR; ++v) up[v] = u[m->off[e] + (size_t)v * n3 + p];
                orc_entropy_vars(up, g, wv);
                for (int v = 0; v < NVAR; ++v) {
                    double t = wq * wv[v] * f[(size_t)v * n3 + p];
                    out[5] += t;
                    out[6] += fabs(t);
                }
            }
        }
    }
}
