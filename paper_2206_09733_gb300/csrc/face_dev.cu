// Face Riemann solve of the mixed path: FP32 flux arithmetic on deviations.
//
// One thread per face node (element-major walk, as the FP64 face kernel).
// The two traces are read in FP64; the face's reference state is the minus
// side's trace rounded to FP32 and both traces become FP64-formed deviations
// from it (lowmach.cuh), so every jump the flux needs (u_R - u_L, p_R - p_L,
// ...) is accurate relative to the jump, not to the state.  The kernel writes
// for each side the quantity that side lifts:
//   G_L = F* - F(u_L).Sn,   G_R = F* - F(u_R).Sn      (viscous parts included)
// in the layout fstar[d][e][side][5][n2] (side 0: the minus element e, side 1:
// its +d neighbour), so the element kernels add iw G_L on the +d face and
// -iw G_R on the -d face without forming a large own flux.  Fluxes that are
// "central + dissipation" (LF, Rusanov, Roe, low-dissipation Roe) are
//   G_L = (F_R - F_L).Sn/2 - D/2,   G_R = -(F_R - F_L).Sn/2 - D/2,
// with F_R - F_L from the one-point flux deviations and D from accurate
// jumps; the entropy-conservative flux (and matrix dissipation) is the
// deviation form of the Chandrashekar flux minus F(u_L) - F(ubar).
// Viscous part: F*_v - F_v(side) = +-(F_v(R) - F_v(L)).Sn/2.
#include "internal.cuh"
#include "lowmach.cuh"
#include "physics.cuh"

namespace hs3d {

template <int n>
__device__ __forceinline__ int face_node_dev(int d, int end, int ta, int tb)
{
    if (d == 0) return end + n * (ta + n * tb);
    if (d == 1) return ta + n * (end + n * tb);
    return ta + n * (tb + n * end);
}

// Roe dissipation times the face scale, s |A_roe| (u_R - u_L) / 2, from the
// primitive jumps (dr, dp, dv) (Roe averages of the FP32 primitive
// variables; zvel scales the velocity jump as in the low-dissipation Roe
// flux).
__device__ __forceinline__ void roe_diss(const Prim<float> &L, const Prim<float> &Rr, float gamma, float s1, float s2,
                                         float s3, float dr, float dp, float d1, float d2, float d3, float zvel,
                                         float D[5])
{
    const float s = sqrtf(s1 * s1 + s2 * s2 + s3 * s3);
    const float is = __fdividef(1.0f, s);
    const float n1 = s1 * is, n2 = s2 * is, n3 = s3 * is;
    const float sl = sqrtf(L.rho), sr = sqrtf(Rr.rho);
    const float iw = __fdividef(1.0f, sl + sr);
    const float HL = (L.E + L.p) / L.rho, HR = (Rr.E + Rr.p) / Rr.rho;
    const float vt1 = (sl * L.v1 + sr * Rr.v1) * iw;
    const float vt2 = (sl * L.v2 + sr * Rr.v2) * iw;
    const float vt3 = (sl * L.v3 + sr * Rr.v3) * iw;
    const float Ht = (sl * HL + sr * HR) * iw;
    const float q2 = vt1 * vt1 + vt2 * vt2 + vt3 * vt3;
    const float c2 = (gamma - 1.0f) * (Ht - 0.5f * q2);
    const float ct = sqrtf(c2);
    const float ic2 = __fdividef(1.0f, c2);
    const float rt = sl * sr;
    const float vnt = vt1 * n1 + vt2 * n2 + vt3 * n3;
    d1 *= zvel;
    d2 *= zvel;
    d3 *= zvel;
    const float dvn = d1 * n1 + d2 * n2 + d3 * n3;
    const float a1 = (dp - rt * ct * dvn) * 0.5f * ic2;
    const float a5 = (dp + rt * ct * dvn) * 0.5f * ic2;
    const float a2 = dr - dp * ic2;
    const float sh1 = rt * (d1 - dvn * n1), sh2 = rt * (d2 - dvn * n2), sh3 = rt * (d3 - dvn * n3);
    const float l1 = fabsf(vnt - ct) * a1, l2 = fabsf(vnt), l5 = fabsf(vnt + ct) * a5;
    const float hs = 0.5f * s;
    D[0] = hs * (l1 + l2 * a2 + l5);
    D[1] = hs * (l1 * (vt1 - ct * n1) + l2 * (a2 * vt1 + sh1) + l5 * (vt1 + ct * n1));
    D[2] = hs * (l1 * (vt2 - ct * n2) + l2 * (a2 * vt2 + sh2) + l5 * (vt2 + ct * n2));
    D[3] = hs * (l1 * (vt3 - ct * n3) + l2 * (a2 * vt3 + sh3) + l5 * (vt3 + ct * n3));
    D[4] = hs * (l1 * (Ht - ct * vnt) + l2 * (a2 * 0.5f * q2 + vt1 * sh1 + vt2 * sh2 + vt3 * sh3) +
                 l5 * (Ht + ct * vnt));
}

// Matrix dissipation of the entropy-stable flux (as flux_matrix in
// physics.cuh) from accurate jumps: [[ln rho]] = log1p(drho/rho_L),
// [[ln beta]] = log1p(dbeta/beta_L), [[beta |v|^2]] = dbeta |v_R|^2 + beta_L dv.(v_R + v_L),
// [[beta v]] = dbeta v_R + beta_L dv.
__device__ __forceinline__ void matrix_diss(const Prim<float> &L, const Prim<float> &Rr, float bL, float bR, float lrL,
                                            float lrR, float lbL, float lbR, float dr, float db, float d1, float d2,
                                            float d3, float gamma, float hg, float s1, float s2, float s3, float D[5])
{
    const float s = sqrtf(s1 * s1 + s2 * s2 + s3 * s3);
    const float is = __fdividef(1.0f, s);
    const float n1 = s1 * is, n2 = s2 * is, n3 = s3 * is;
    const float rho_h = ln_mean(L.rho, Rr.rho, lrL, lrR);
    const float ib_ln = inv_ln_mean(bL, bR, lbL, lbR);
    const float p_h = 0.5f * (L.rho + Rr.rho) * __fdividef(1.0f, bL + bR);
    const float v1 = 0.5f * (L.v1 + Rr.v1), v2 = 0.5f * (L.v2 + Rr.v2), v3 = 0.5f * (L.v3 + Rr.v3);
    const float qL = L.v1 * L.v1 + L.v2 * L.v2 + L.v3 * L.v3, qR = Rr.v1 * Rr.v1 + Rr.v2 * Rr.v2 + Rr.v3 * Rr.v3;
    const float v2h = 2.0f * (v1 * v1 + v2 * v2 + v3 * v3) - 0.5f * (qL + qR);
    const float a_h = sqrtf(gamma * p_h / rho_h);
    const float h_h = gamma * hg * ib_ln + 0.5f * v2h;
    const float vn = v1 * n1 + v2 * n2 + v3 * n3;
    const float dlr = log1pf(dr / L.rho), dlb = log1pf(db / bL);
    const float dq = d1 * (Rr.v1 + L.v1) + d2 * (Rr.v2 + L.v2) + d3 * (Rr.v3 + L.v3);
    float dw[5];
    dw[0] = dlr + 2.0f * hg * dlb - (db * qR + bL * dq);
    dw[1] = 2.0f * (db * Rr.v1 + bL * d1);
    dw[2] = 2.0f * (db * Rr.v2 + bL * d2);
    dw[3] = 2.0f * (db * Rr.v3 + bL * d3);
    dw[4] = -2.0f * db;
    const float r1[5] = {1.0f, v1 - a_h * n1, v2 - a_h * n2, v3 - a_h * n3, h_h - a_h * vn};
    const float r5[5] = {1.0f, v1 + a_h * n1, v2 + a_h * n2, v3 + a_h * n3, h_h + a_h * vn};
    const float c1 = dw[0] + r1[1] * dw[1] + r1[2] * dw[2] + r1[3] * dw[3] + r1[4] * dw[4];
    const float c5 = dw[0] + r5[1] * dw[1] + r5[2] * dw[2] + r5[3] * dw[3] + r5[4] * dw[4];
    const float c2 = dw[0] + v1 * dw[1] + v2 * dw[2] + v3 * dw[3] + 0.5f * v2h * dw[4];
    const float T15 = rho_h / (2.0f * gamma), T2 = rho_h * (gamma - 1.0f) / gamma;
    const float k1 = fabsf(vn - a_h) * T15 * c1, k5 = fabsf(vn + a_h) * T15 * c5;
    const float l2 = fabsf(vn);
    const float k2 = l2 * T2 * c2;
    const float q1 = dw[1] + v1 * dw[4], q2 = dw[2] + v2 * dw[4], q3 = dw[3] + v3 * dw[4];
    const float qn = q1 * n1 + q2 * n2 + q3 * n3;
    const float ks = l2 * p_h;
    const float P1 = ks * (q1 - qn * n1), P2 = ks * (q2 - qn * n2), P3 = ks * (q3 - qn * n3);
    const float hs = 0.5f * s;
    D[0] = hs * (k1 + k2 + k5);
    D[1] = hs * (k1 * r1[1] + k2 * v1 + k5 * r5[1] + P1);
    D[2] = hs * (k1 * r1[2] + k2 * v2 + k5 * r5[2] + P2);
    D[3] = hs * (k1 * r1[3] + k2 * v3 + k5 * r5[3] + P3);
    D[4] = hs * (k1 * r1[4] + k2 * 0.5f * v2h + k5 * r5[4] + v1 * P1 + v2 * P2 + v3 * P3);
}

// Face point t (face gf = t / n^2, point ab = t mod n^2) of the batch.  TWO:
// the flux is one of the two-point family (EC, matrix dissipation), else of
// the central + dissipation family (LF, Rusanov, Roe, low-dissipation Roe);
// a kernel per family keeps the other family's registers out of it.
template <int N, bool NS, bool TWO>
__device__ __forceinline__ void face_dev_point(const Batch &b, int flux, long long t)
{
    constexpr int n = N + 1, n2 = n * n, n3 = n2 * n;
    const long long gf = t / n2;
    const int ab = (int)(t - gf * n2);
    const Item &it = find_item_face(b, gf);
    if (it.clk && it.clk->done) return;
    const int E = it.E;
    const int lf = (int)(gf - it.face_begin);
    const int eL = lf / 3;
    const int d = lf - 3 * eL;
    const int f = d * E + eL;
    const int eR = nbr_plus(eL, d, it.ex, it.ey, it.ez);
    const int ta = ab % n, tb = ab / n;
    const int pL = face_node_dev<n>(d, N, ta, tb), pR = face_node_dev<n>(d, 0, ta, tb);
    const size_t iL = (size_t)eL * 5 * n3 + pL, iR = (size_t)eR * 5 * n3 + pR;
    double uL[5], uR[5];
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        uL[v] = it.u[iL + (size_t)v * n3];
        uR[v] = it.u[iR + (size_t)v * n3];
    }
    const float gm1 = it.gm1f, hg = it.hgf, gamma = it.gammaf;
    // the entropy-conservative fluxes mix one- and two-point deviations and need
    // the reference state whose identities hold exactly; the others only differences
    double ad[5];
    Anchor A;
    Dev DL, DR;
    if constexpr (TWO) {
        // the minus element's reference state, left by the pass before
        const AnchorRec &R = ((const AnchorRec *)it.anc)[eL];
        A = R.a;
#pragma unroll
        for (int v = 0; v < 5; ++v) ad[v] = R.ad[v];
        DL = make_dev(uL, ad, A, gm1);
        DR = make_dev(uR, ad, A, gm1);
    } else {
        // the reference is u_L itself (its FP32 values serve as the coefficients):
        // u_L's deviation is zero and u_R's is the jump, one FP64 subtraction each
        A = make_anchor_face(uL, gm1, ad);
        DL = make_dev_f(0.0f, 0.0f, 0.0f, 0.0f, 0.0f, A, gm1);
        DR = make_dev_f(dev_round(uR[0] - uL[0]), dev_round(uR[1] - uL[1]), dev_round(uR[2] - uL[2]),
                        dev_round(uR[3] - uL[3]), dev_round(uR[4] - uL[4]), A, gm1);
    }
    const float *Fn = it.fnf + (size_t)f * 3 * n2 + ab;
    const float s1 = Fn[0], s2 = Fn[n2], s3 = Fn[2 * n2];
    const Prim<float> qL = dev_prim(DL, A), qR = dev_prim(DR, A);
    float fL[5], fR[5], GL[5], GR[5];
    dflux_euler(DL, A, s1, s2, s3, fL);
    if constexpr (TWO) {
        const ECDev zL = ec_dev(DL, A), zR = ec_dev(DR, A);
        float frho, rmass, fm[3], rest;
        dflux_ec(zL, zR, A, hg, s1, s2, s3, frho, rmass, fm, rest);
        // F* - F(u_L) = (f# - F(ubar)) - (F(u_L) - F(ubar))
        GL[0] = frho - fL[0];
        GL[1] = fm[0] - fL[1];
        GL[2] = fm[1] - fL[2];
        GL[3] = fm[2] - fL[3];
        GL[4] = (A.H * frho + rest) - fL[4];
        if (flux == HS3D_FLUX_MATRIX) {
            float Dm[5];
            const float bL = A.beta + zL.db, bR = A.beta + zR.db;
            matrix_diss(qL, qR, bL, bR, logf(qL.rho), logf(qR.rho), logf(bL), logf(bR), DR.dr - DL.dr,
                        zR.db - zL.db, DR.dv1 - DL.dv1, DR.dv2 - DL.dv2, DR.dv3 - DL.dv3, gamma, hg, s1, s2, s3, Dm);
#pragma unroll
            for (int v = 0; v < 5; ++v) GL[v] -= Dm[v];
        }
        dflux_euler(DR, A, s1, s2, s3, fR);
#pragma unroll
        for (int v = 0; v < 5; ++v) GR[v] = GL[v] - (fR[v] - fL[v]);
    } else {
        dflux_euler(DR, A, s1, s2, s3, fR);
        float Dv[5];
        if (flux == HS3D_FLUX_LF || flux == HS3D_FLUX_RUSANOV) {
            const float s = sqrtf(s1 * s1 + s2 * s2 + s3 * s3);
            const float vnL = fabsf(qL.v1 * s1 + qL.v2 * s2 + qL.v3 * s3),
                        vnR = fabsf(qR.v1 * s1 + qR.v2 * s2 + qR.v3 * s3);
            const float cL = sqrtf(gamma * qL.p / qL.rho), cR = sqrtf(gamma * qR.p / qR.rho);
            const float lam = (flux == HS3D_FLUX_LF) ? fmaxf(vnL + s * cL, vnR + s * cR) : fmaxf(vnL, vnR) + s * fmaxf(cL, cR);
            const float ju[5] = {DR.dr - DL.dr, DR.dm1 - DL.dm1, DR.dm2 - DL.dm2, DR.dm3 - DL.dm3, DR.dE - DL.dE};
#pragma unroll
            for (int v = 0; v < 5; ++v) Dv[v] = 0.5f * lam * ju[v];
        } else {
            float z = 1.0f;
            if (flux == HS3D_FLUX_LDROE) {
                const float mL = (qL.v1 * qL.v1 + qL.v2 * qL.v2 + qL.v3 * qL.v3) * qL.rho / (gamma * qL.p);
                const float mR = (qR.v1 * qR.v1 + qR.v2 * qR.v2 + qR.v3 * qR.v3) * qR.rho / (gamma * qR.p);
                z = fminf(1.0f, sqrtf(fmaxf(mL, mR)));
            }
            roe_diss(qL, qR, gamma, s1, s2, s3, DR.dr - DL.dr, DR.dp - DL.dp, DR.dv1 - DL.dv1, DR.dv2 - DL.dv2,
                     DR.dv3 - DL.dv3, z, Dv);
        }
#pragma unroll
        for (int v = 0; v < 5; ++v) {
            const float h = 0.5f * (fR[v] - fL[v]);
            GL[v] = h - Dv[v];
            GR[v] = -h - Dv[v];
        }
    }
    if (NS) {
        const float *GLp = (const float *)it.grad + (size_t)eL * 12 * n3 + pL;
        const float *GRp = (const float *)it.grad + (size_t)eR * 12 * n3 + pR;
        float gl[12], gr[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            gl[k] = GLp[k * n3];
            gr[k] = GRp[k * n3];
        }
        float vl[5], vr[5];
        visc_flux(qL, gl, it.muf, it.kappaf, s1, s2, s3, vl);
        visc_flux(qR, gr, it.muf, it.kappaf, s1, s2, s3, vr);
#pragma unroll
        for (int v = 1; v < 5; ++v) {
            const float h = 0.5f * (vr[v] - vl[v]);
            GL[v] -= h;
            GR[v] += h;
        }
    }
    float *out = (float *)it.fstar + (size_t)f * 10 * n2 + ab;
#pragma unroll
    for (int v = 0; v < 5; ++v) {
        out[v * n2] = GL[v];
        out[(5 + v) * n2] = GR[v];
    }
}

// The face kernel: one thread per face point, or (Batch::persistent) a
// persistent grid striding over the face points.
template <int N, bool NS, bool TWO>
__global__ void __launch_bounds__(256, 4) k_face_dev(const __grid_constant__ Batch b, int flux)
{
    pdl_wait();
    constexpr int n2 = (N + 1) * (N + 1);
    const long long total = b.total_faces * n2;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x)
        face_dev_point<N, NS, TWO>(b, flux, t);
}

template <int N, bool NS, bool TWO>
static cudaError_t face_dev_launch3(int flux, const Batch &b, unsigned blocks, cudaStream_t s)
{
    const unsigned grid = b.persistent ? persistent_grid(k_face_dev<N, NS, TWO>, 256, 0, blocks) : blocks;
    return launch_pdl(k_face_dev<N, NS, TWO>, grid, 256, 0, s, b, flux);
}

template <int N>
static cudaError_t face_dev_launch(int physics, int flux, const Batch &b, cudaStream_t s)
{
    constexpr int n2 = (N + 1) * (N + 1);
    const long long total = b.total_faces * n2;
    if (total == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    const bool two = (flux == HS3D_FLUX_EC || flux == HS3D_FLUX_MATRIX);
    if (physics == HS3D_NS)
        return two ? face_dev_launch3<N, true, true>(flux, b, blocks, s) : face_dev_launch3<N, true, false>(flux, b, blocks, s);
    return two ? face_dev_launch3<N, false, true>(flux, b, blocks, s) : face_dev_launch3<N, false, false>(flux, b, blocks, s);
}

cudaError_t launch_face_dev(int N, int physics, int flux, const Batch &b, cudaStream_t s)
{
    switch (N) {
        case 1: return face_dev_launch<1>(physics, flux, b, s);
        case 2: return face_dev_launch<2>(physics, flux, b, s);
        case 3: return face_dev_launch<3>(physics, flux, b, s);
        case 4: return face_dev_launch<4>(physics, flux, b, s);
        case 5: return face_dev_launch<5>(physics, flux, b, s);
        case 6: return face_dev_launch<6>(physics, flux, b, s);
        case 7: return face_dev_launch<7>(physics, flux, b, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace hs3d
