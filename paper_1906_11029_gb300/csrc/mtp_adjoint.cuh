// Reverse-in-time discrete adjoint of the tent maps (not in the paper).
//
// One CTA per tent and right-hand side, layers in reverse order.  The CTA replays the
// tent's forward SAT stages from its bottom state (recorded into a per-CTA tape in global
// memory: Y_{i,0} and U_{i,n}), then runs the transposed recursion.  With M_i = M(i/m),
// lam = dJ/dY_out and mu_n = dJ/dU_n, per sub-interval i (reverse order):
//   for n = q..1:  nu_n = M_i^-T mu_n (n < q),   lamY_n = c_n lam + nu_n,
//                  mu_{n-1} = A^T lamY_n - n M'^T nu_n
//   nu_0 = M_i^-T mu_0,   dJ/dY_in = lam + nu_0.
// M_i^-1 is the closed-form G_i^-1 (symmetric, like M' = G'), so M^-T = M^-1 and M'^T = M'.
// A^T: lift transpose (-L^T), transpose of the upwind / PEC flux (written out below), trace
// transpose (Tr^T) and the volume transpose Ubar_H[b] += sum_a w_ab x lamY_E[a],
// Ubar_E[b] -= sum_a w_ab x lamY_H[a] with w_ab = sum_l S[j][l][a][b] dt grad(lambda_{l+1}).
// Material gradients: each solve contributes -nu^T (dM/dp) U (dM/deps = E block, dM/dmu = H
// block); A depends on eps, mu through Z = sqrt(mu/eps) in the fluxes: dJ/dZ from forward-mode
// dual numbers through the same flux routine, then dZ/deps = -Z/(2 eps), dZ/dmu = Z/(2 mu).
#pragma once

#include "mtp_kernels.cuh"

namespace mtp {

struct AdjArgs {
    KArgs k;               // tau = the reverse-sweep front (front after the current layer)
    const void* ybot;      // state before the current layer [rhs][ne][nf][nb]
    void* lam;             // adjoint state, in: dJ/dY after the layer, out: before it
    double* geps;          // dJ/deps [ne], accumulated
    double* gmu;           // dJ/dmu  [ne], accumulated
    void* tape;            // per-CTA tape, tape_stride entries each
    int64_t tape_stride;
};

template <typename T>
struct Dual {
    T v, d;
    __device__ Dual() : v(0), d(0) {}
    __device__ Dual(T x) : v(x), d(0) {}
    __device__ Dual(T x, T dx) : v(x), d(dx) {}
};
template <typename T> __device__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __device__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __device__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T> __device__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T> __device__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
    return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)};
}
template <typename T> __device__ Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a = a + b; return a; }
template <typename T> __device__ Dual<T>& operator-=(Dual<T>& a, Dual<T> b) { a = a - b; return a; }

// Transpose of the linear map (u-, u+) -> F*(u-, u+) of upwind6: given Fb = dJ/dF*, returns
// dJ/du- and dJ/du+.  With X v = v x n and P_t = I - n n^T:
//   F_E = (Zm X H- + Zp X H+ + P_t E- - P_t E+) / (Zm + Zp),  F_H = -X e,
//   e   = (Zp P_t E- + Zm P_t E+ + Zp Zm X (H- - H+)) / (Zm + Zp),  X^T w = n x w.
template <typename Real>
__device__ __forceinline__ void upwind6_adjoint(const Real Fb[6], const Real n[3], Real Zm, Real Zp, Real um_b[6],
                                                Real up_b[6]) {
    const Real inv = Real(1) / (Zm + Zp);
    Real eb[3] = {-(n[1] * Fb[5] - n[2] * Fb[4]), -(n[2] * Fb[3] - n[0] * Fb[5]), -(n[0] * Fb[4] - n[1] * Fb[3])};
    const Real fn = Fb[0] * n[0] + Fb[1] * n[1] + Fb[2] * n[2];
    const Real en = eb[0] * n[0] + eb[1] * n[1] + eb[2] * n[2];
    Real Ptf[3], Pte[3];
    for (int q = 0; q < 3; ++q) {
        Ptf[q] = Fb[q] - fn * n[q];
        Pte[q] = eb[q] - en * n[q];
    }
    const Real nf[3] = {n[1] * Fb[2] - n[2] * Fb[1], n[2] * Fb[0] - n[0] * Fb[2], n[0] * Fb[1] - n[1] * Fb[0]};
    const Real ne[3] = {n[1] * eb[2] - n[2] * eb[1], n[2] * eb[0] - n[0] * eb[2], n[0] * eb[1] - n[1] * eb[0]};
    const Real zz = Zm * Zp;
    for (int q = 0; q < 3; ++q) {
        um_b[q] = (Ptf[q] + Zp * Pte[q]) * inv;
        up_b[q] = (-Ptf[q] + Zm * Pte[q]) * inv;
        um_b[3 + q] = (Zm * nf[q] + zz * ne[q]) * inv;
        up_b[3 + q] = (Zp * nf[q] - zz * ne[q]) * inv;
    }
}

template <typename Real, int DIM, int P>
struct AdjLayout {
    SmemLayout<Real, DIM, P> base;
    size_t off_lam, off_nu, off_ly, off_up, off_trU, off_g, bytes;
    __host__ __device__ explicit AdjLayout(int mp) : base(mp, 0, true) {
        size_t o = base.bytes;
        off_lam = o; o = base.align16(o + base.state_bytes);
        off_nu = o; o = base.align16(o + base.state_bytes);
        off_ly = o; o = base.align16(o + base.state_bytes);
        off_up = o; o = base.align16(o + base.state_bytes);
        off_trU = o; o = base.align16(o + base.tr_bytes);
        off_g = o; o = base.align16(o + (size_t)mp * 3 * sizeof(double));
        bytes = o;
    }
};

template <typename Real, int DIM, int P>
__global__ void __launch_bounds__(Shape<DIM, P>::NT) tent_adjoint_kernel(const AdjArgs A, int64_t t0) {
    using Sh = Shape<DIM, P>;
    constexpr int NF = Sh::NF, NB = Sh::NB, NFB = Sh::NFB, NV = Sh::NV, NT = Sh::NT;
    constexpr int NBP = Sh::NBP, NFBP = Sh::NFBP, ESZ = NF * NBP, TSZ = Strides<Real, DIM, P>::TSZ;
    constexpr int FSZ = Strides<Real, DIM, P>::FSZ;
    const KArgs& a = A.k;
    extern __shared__ __align__(16) unsigned char smem[];
    const AdjLayout<Real, DIM, P> lay(a.max_patch);
    TentCtx<Real, DIM, P> c;
    c.carve(smem, lay.base);
    Real* sLam = (Real*)(smem + lay.off_lam);
    Real* sNu = (Real*)(smem + lay.off_nu);
    Real* sLY = (Real*)(smem + lay.off_ly);
    Real* sUp = (Real*)(smem + lay.off_up);
    Real* sTrU = (Real*)(smem + lay.off_trU);
    double* sG = (double*)(smem + lay.off_g);     // [k][3]: eps part, mu part, dJ/dZ
    const int tid = threadIdx.x;
    const int64_t tent = t0 + blockIdx.x;
    const int64_t rhs_off = (int64_t)blockIdx.y * a.rhs_stride;
    Real* tape = (Real*)A.tape + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * A.tape_stride;
    const size_t slot = (size_t)a.max_patch * ESZ;

    // forward replay from the tent's bottom state, recording the tape
    tent_setup(c, a, tent, (const Real*)A.ybot + rhs_off);
    tent_sat(c, a, tape);
    const int ns = c.ns;
    const Real* S = (const Real*)a.S;
    const Real* Tr = (const Real*)a.Tr;
    const Real* Lf = (const Real*)a.L;
    const Real* lam_g = (const Real*)A.lam + rhs_off;
    for (int idx = tid; idx < ns * ESZ; idx += NT) {
        const int k = idx / ESZ, r = idx - k * ESZ, s = r / NBP, b = r - s * NBP;
        sLam[idx] = b < NB ? lam_g[((int64_t)a.patch_elem[c.pb + k] * NF + s) * NB + b] : Real(0);
        sNu[idx] = sLY[idx] = sUp[idx] = Real(0);
    }
    for (int idx = tid; idx < ns * TSZ; idx += NT) sTrU[idx] = c.sTr[idx] = Real(0);
    for (int idx = tid; idx < ns * 3; idx += NT) sG[idx] = 0.0;
    __syncthreads();

    Real* sLamIn = c.sY;
    Real* sMu = c.sUa;
    Real* sMuPrev = c.sUb;
    Real* sGh = c.sTr;
    for (int i = a.m - 1; i >= 0; --i) {
        tent_ginv(c, a, i);
        for (int idx = tid; idx < ns * ESZ; idx += NT) {
            sLamIn[idx] = sLam[idx];
            sMu[idx] = Real(0);
        }
        __syncthreads();
        for (int n = a.q; n >= 1; --n) {
            const Real cn = (Real)a.taylor[n];
            const Real* Un = tape + (size_t)(a.m + i * a.q + n) * slot;        // U_{i,n} (n < q)
            const Real* Uprev = tape + (size_t)(a.m + i * a.q + n - 1) * slot;  // U_{i,n-1}
            // nu = G_i^-1 mu; lamY = c_n lam + nu; U_{i,n-1} from the tape
            if (n < a.q) tent_apply_ginv(c, sMu, sNu);
            __syncthreads();
            for (int idx = tid; idx < ns * ESZ; idx += NT) {
                sLY[idx] = cn * sLam[idx] + (n < a.q ? sNu[idx] : Real(0));
                sUp[idx] = Uprev[idx];
            }
            if (n < a.q) {
                for (int k = tid; k < ns; k += NT) {   // -nu^T dM/dp U_{i,n}
                    double ge = 0, gm = 0;
                    for (int s = 0; s < NF; ++s) {
                        const bool isE = DIM == 3 ? s < 3 : s < 2;
                        double acc = 0;
                        for (int b = 0; b < NB; ++b)
                            acc += (double)sNu[k * ESZ + s * NBP + b] * (double)Un[k * ESZ + s * NBP + b];
                        if (isE) ge -= acc; else gm -= acc;
                    }
                    sG[3 * k] += ge;
                    sG[3 * k + 1] += gm;
                }
            }
            __syncthreads();
            // forward traces of U_{i,n-1} (for dJ/dZ) and ghat = -L^T lamY per facet mode
            tent_traces(c, a, sUp, sTrU);
            for (int idx = tid; idx < ns * DIM * NFB; idx += NT) {
                const int k = idx / (DIM * NFB), rem = idx - k * DIM * NFB, fi = rem / NFB, cc = rem - fi * NFB;
                const int j = c.sJ[k];
                const int f = fi + (fi >= j ? 1 : 0);
                const Real* Lr = Lf + (((size_t)j * NV + f) * NB) * NFBP + cc;
                Real acc[NF];
                for (int s = 0; s < NF; ++s) acc[s] = 0;
                for (int av = 0; av < NB; ++av) {
                    const Real l = __ldg(Lr + (size_t)av * NFBP);
                    for (int s = 0; s < NF; ++s) acc[s] += l * sLY[k * ESZ + s * NBP + av];
                }
                for (int s = 0; s < NF; ++s) sGh[k * TSZ + fi * FSZ + s * NFBP + cc] = -acc[s];
            }
            __syncthreads();
            // flux transpose (owner of each facet) and dJ/dZ
            for (int idx = tid; idx < ns * DIM * NFB; idx += NT) {
                const int k = idx / (DIM * NFB), rem = idx - k * DIM * NFB, fi = rem / NFB, cc = rem - fi * NFB;
                const int s2 = c.sNslot[k * DIM + fi];
                if (s2 >= 0 && s2 < k) continue;
                const int fi2 = s2 >= 0 ? c.sNfi[k * DIM + fi] : 0;
                Real* gmine = sGh + k * TSZ + fi * FSZ + cc;
                Real* gother = s2 >= 0 ? sGh + s2 * TSZ + fi2 * FSZ + cc : nullptr;
                const Real lc = c.sLiftc[k * DIM + fi];
                Real Fb[6] = {0, 0, 0, 0, 0, 0};
                for (int s = 0; s < NF; ++s) {
                    Real v = lc * gmine[s * NFBP];
                    if (gother) v -= c.sLiftc[s2 * DIM + fi2] * gother[s * NFBP];
                    Fb[field6<DIM>(s)] = v;
                }
                Real nrm[3];
                for (int q = 0; q < 3; ++q) nrm[q] = c.sNrm[(k * DIM + fi) * 3 + q];
                const Real Zm = c.sZ[k * (1 + DIM)], Zp = c.sZ[k * (1 + DIM) + 1 + fi];
                Real ubm[6], ubp[6];
                upwind6_adjoint<Real>(Fb, nrm, Zm, Zp, ubm, ubp);
                // forward traces for the impedance derivatives
                const Real* tm = sTrU + k * TSZ + fi * FSZ + cc;
                Dual<Real> um[6], up[6], dn[3], F[6];
                for (int s = 0; s < 6; ++s) um[s] = up[s] = Dual<Real>(Real(0));
                for (int s = 0; s < NF; ++s) um[field6<DIM>(s)] = Dual<Real>(tm[s * NFBP]);
                if (gother) {
                    const Real* tp = sTrU + s2 * TSZ + fi2 * FSZ + cc;
                    for (int s = 0; s < NF; ++s) up[field6<DIM>(s)] = Dual<Real>(tp[s * NFBP]);
                } else {
                    for (int s = 0; s < 6; ++s) up[s] = s < 3 ? -um[s] : um[s];
                }
                for (int q = 0; q < 3; ++q) dn[q] = Dual<Real>(nrm[q]);
                if (gother) {
                    upwind6<Dual<Real>>(um, up, dn, Dual<Real>(Zm, Real(1)), Dual<Real>(Zp), F);
                    Real dzm = 0;
                    for (int s = 0; s < 6; ++s) dzm += Fb[s] * F[s].d;
                    upwind6<Dual<Real>>(um, up, dn, Dual<Real>(Zm), Dual<Real>(Zp, Real(1)), F);
                    Real dzp = 0;
                    for (int s = 0; s < 6; ++s) dzp += Fb[s] * F[s].d;
                    atomicAdd(&sG[3 * k + 2], (double)dzm);
                    atomicAdd(&sG[3 * s2 + 2], (double)dzp);
                    for (int s = 0; s < NF; ++s) {
                        gmine[s * NFBP] = ubm[field6<DIM>(s)];
                        gother[s * NFBP] = ubp[field6<DIM>(s)];
                    }
                } else {
                    upwind6<Dual<Real>>(um, up, dn, Dual<Real>(Zm, Real(1)), Dual<Real>(Zm, Real(1)), F);
                    Real dz = 0;
                    for (int s = 0; s < 6; ++s) dz += Fb[s] * F[s].d;
                    atomicAdd(&sG[3 * k + 2], (double)dz);
                    // u+ = D u- (D = diag(-1,-1,-1,1,1,1)): ubar- = ubm + D ubp
                    for (int s = 0; s < NF; ++s) {
                        const int q = field6<DIM>(s);
                        gmine[s * NFBP] = ubm[q] + (q < 3 ? -ubp[q] : ubp[q]);
                    }
                }
            }
            __syncthreads();
            // mu_{n-1} = Tr^T (trace adjoint) + volume transpose - n M' nu
            for (int idx = tid; idx < ns * NB; idx += NT) {
                const int k = idx / NB, b = idx - k * NB;
                const int j = c.sJ[k];
                Real u[NF];
                for (int s = 0; s < NF; ++s) u[s] = 0;
                const Real sc = c.sTrs[k];
                for (int fi = 0; fi < DIM; ++fi) {
                    const int f = fi + (fi >= j ? 1 : 0);
                    const Real* gh = sGh + k * TSZ + fi * FSZ;
                    for (int cc = 0; cc < NFB; ++cc) {
                        const Real t = __ldg(Tr + ((size_t)f * NFB + cc) * NBP + b) * sc;
                        for (int s = 0; s < NF; ++s) u[s] += t * gh[s * NFBP + cc];
                    }
                }
                const Real* ac = c.sAc + k * DIM * 3;
                const Real* LY = sLY + k * ESZ;
                for (int av = 0; av < NB; ++av) {
                    Real w[3] = {0, 0, 0};
                    for (int l = 0; l < DIM; ++l) {
                        const Real sv = __ldg(S + (((size_t)j * DIM + l) * NB + av) * NBP + b);
                        for (int q = 0; q < 3; ++q) w[q] += sv * ac[3 * l + q];
                    }
                    if constexpr (DIM == 3) {
                        const Real lE[3] = {LY[0 * NBP + av], LY[1 * NBP + av], LY[2 * NBP + av]};
                        const Real lH[3] = {LY[3 * NBP + av], LY[4 * NBP + av], LY[5 * NBP + av]};
                        // Ubar_H += w x lamY_E ; Ubar_E -= w x lamY_H
                        u[3] += w[1] * lE[2] - w[2] * lE[1];
                        u[4] += w[2] * lE[0] - w[0] * lE[2];
                        u[5] += w[0] * lE[1] - w[1] * lE[0];
                        u[0] -= w[1] * lH[2] - w[2] * lH[1];
                        u[1] -= w[2] * lH[0] - w[0] * lH[2];
                        u[2] -= w[0] * lH[1] - w[1] * lH[0];
                    } else {
                        const Real lEx = LY[0 * NBP + av], lEy = LY[1 * NBP + av], lHz = LY[2 * NBP + av];
                        u[2] += -w[1] * lEx + w[0] * lEy;
                        u[0] += -w[1] * lHz;
                        u[1] += w[0] * lHz;
                    }
                }
                if (n < a.q) {
                    const Real* gd = c.sGd + 3 * k;
                    const Real* nu = sNu + k * ESZ;
                    const Real nn = (Real)n;
                    if constexpr (DIM == 3) {
                        const Real E0 = nu[0 * NBP + b], E1 = nu[1 * NBP + b], E2 = nu[2 * NBP + b];
                        const Real H0 = nu[3 * NBP + b], H1 = nu[4 * NBP + b], H2 = nu[5 * NBP + b];
                        u[0] += nn * (H1 * gd[2] - H2 * gd[1]);   // -n [-H x gd]
                        u[1] += nn * (H2 * gd[0] - H0 * gd[2]);
                        u[2] += nn * (H0 * gd[1] - H1 * gd[0]);
                        u[3] -= nn * (E1 * gd[2] - E2 * gd[1]);   // -n [E x gd]
                        u[4] -= nn * (E2 * gd[0] - E0 * gd[2]);
                        u[5] -= nn * (E0 * gd[1] - E1 * gd[0]);
                    } else {
                        const Real Ex = nu[0 * NBP + b], Ey = nu[1 * NBP + b], Hz = nu[2 * NBP + b];
                        u[0] -= nn * (Hz * gd[1]);
                        u[1] += nn * (Hz * gd[0]);
                        u[2] -= nn * (Ex * gd[1] - Ey * gd[0]);
                    }
                }
                for (int s = 0; s < NF; ++s) sMuPrev[k * ESZ + s * NBP + b] = u[s];
            }
            __syncthreads();
            Real* tmp = sMu; sMu = sMuPrev; sMuPrev = tmp;
        }
        // nu_0 = G_i^-1 mu_0; lam_in = lam + nu_0; gradient of the solve for U_{i,0}
        tent_apply_ginv(c, sMu, sNu);
        __syncthreads();
        const Real* U0 = tape + (size_t)(a.m + i * a.q) * slot;
        for (int k = tid; k < ns; k += NT) {
            double ge = 0, gm = 0;
            for (int s = 0; s < NF; ++s) {
                const bool isE = DIM == 3 ? s < 3 : s < 2;
                double acc = 0;
                for (int b = 0; b < NB; ++b)
                    acc += (double)sNu[k * ESZ + s * NBP + b] * (double)U0[k * ESZ + s * NBP + b];
                if (isE) ge -= acc; else gm -= acc;
            }
            sG[3 * k] += ge;
            sG[3 * k + 1] += gm;
        }
        for (int idx = tid; idx < ns * ESZ; idx += NT) sLam[idx] = sLamIn[idx] + sNu[idx];
        __syncthreads();
    }
    // write dJ/dY at the tent bottom and the material gradients; move the reverse front
    Real* lam_o = (Real*)A.lam + rhs_off;
    for (int idx = tid; idx < ns * NF * NB; idx += NT) {
        const int k = idx / (NF * NB), r = idx - k * NF * NB, s = r / NB, b = r - s * NB;
        lam_o[(int64_t)a.patch_elem[c.pb + k] * NF * NB + r] = sLam[k * ESZ + s * NBP + b];
    }
    for (int k = tid; k < ns; k += NT) {
        const int e = a.patch_elem[c.pb + k];
        const double eps = c.sMat[2 * k], mu = c.sMat[2 * k + 1];
        const double z = sqrt(mu / eps);
        atomicAdd(&A.geps[e], sG[3 * k] + sG[3 * k + 2] * (-z / (2.0 * eps)));
        atomicAdd(&A.gmu[e], sG[3 * k + 1] + sG[3 * k + 2] * (z / (2.0 * mu)));
    }
    if (tid == 0 && blockIdx.y == 0) a.tau[c.V] = c.tb;
}

}  // namespace mtp
