// CUDA kernels of the MTP-SAT hot path (sm_103a).
//
// One CTA evolves one tent (for one right-hand side) from bottom to top:
//   (a) gather  the patch's state Y (all elements of omega_V) and FP64 geometry
//   (b) operator A U: facet traces -> upwind / PEC flux -> lambda_V-weighted volume
//       term + lift (Sec. 3, mapped DG semi-discretisation)
//   (c) SAT recursion (Sec. 4, eqs. coeff_rec / recursion-init) with the closed-form
//       pointwise mass inverse of Sec. 4, all m*q stages on shared-memory data
//   (d) scatter the tent-top Y (patches of one layer are element-disjoint: no atomics)
//
// Discretisation on each element T of the patch (orthonormal basis psi_a, mass = I):
//   volume:  Y_E[a] += -sum_l a_l x P_{l,H}[a],   Y_H[a] += sum_l a_l x P_{l,E}[a]
//            with a_l = dt grad(lambda_{l+1}) and P_{l,s}[a] = sum_b S[j][l][a][b] U_s[b],
//            S[j][l][a][b] = int lambda_j psi_b d_l psi_a on the reference simplex
//            (delta = dt lambda_V with V the local vertex j of T).
//   facets containing V: trace coefficients tr = Tr_f U / sqrt|det J| in the facet's
//            orthonormal basis (facet parametrised on the ascending vertex ids, so the two
//            sides agree), flux F*(tr-, tr+) pointwise on coefficients (the flux is linear
//            with constant coefficients on a flat facet), lift
//            Y[a] -= dt (d-1)!|F| / sqrt|det J| sum_c L[j][f][a][c] F*[c].
//   mass:    U = G(t_i)^-1 Y per coefficient (6x6, closed form of Sec. 4, built in FP64)
//            M' U = [-H x dt grad(lambda_j) ; E x dt grad(lambda_j)].
//
// Memory layout for the SIMT contractions: every table row and every shared-memory
// coefficient row is padded to a multiple of 4 entries (zeros in the pad) and read as
// 16-byte vectors; a thread owns two basis functions (or two facet modes), so each
// vector of U read from shared memory feeds 2 x 3 x 6 FMAs per entry.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

namespace mtp {

constexpr int kMaxTaylor = 9;
constexpr int kMaxSub = 64;   // largest number m of SAT sub-intervals the options accept

struct KArgs {
    const int32_t* tent_v;
    const double* tent_tb;
    const double* tent_tt;
    const int64_t* patch_ptr;
    const int32_t* patch_elem;
    const int8_t* patch_info;   // [entry][12]: j, slot[4], nbr_face[4] (see mtp_internal.h)
    const int32_t* elems;       // [ne][dim+1] sorted vertex ids
    const double* geo;          // [ne][32]
    double* tau;                // vertex times of the current front
    const void* S;              // [j][l][a][NBP]  reference tables in the state precision,
    const void* Tr;             // [f][c][NBP]     rows padded with zeros (see pad4)
    const void* L;              // [j][f][a][NFBP]
    // thread-major tables of the SIMT kernels: with G = ceil(rows / AP) row groups (NWG,
    // NAG or NCG, see Shape), entry (r, c) of one matrix at [c / W][r / G][r % G][c % W],
    // W = elements per 16-byte vector; a thread owns rows g and g + G.  The volume term uses
    // the factorisation S[j][l] = D[l]^T M[j] (d_l psi_a lies in P_{p-1}):
    const void* Mc;             // matrices j, NBM x NB:  M[j][c][b] = int psi_c lambda_j psi_b
    const void* Dc;             // matrices l, NB x NBM:  D[l]^T[a][c] = int psi_c d_l psi_a
    const void* Trc;            // matrices f, NFB x NB
    const void* Lc;             // matrices (j, f), NB x NFB
    // tensor-core modes: A-operand tables in m16n8k8 fragment order (32 lanes x 4 TF32 values
    // per fragment), hi part and (split mode) lo part
    const float4* Sf;           // [j][l][mt][kt]
    const float4* Lfr;          // [j][f][mt][ktl]
    const float4* Trf;          // [f][kt]
    const float4* Sf_lo;
    const float4* Lfr_lo;
    const float4* Trf_lo;
    // tcgen05 volume operator (shapes v = 3, 4): A operand D^T[a][(l, c)] (rows a padded to 64)
    // in the K-major core-matrix layout, TF32 hi part then lo part, each 64 x TK floats
    const float* Dtc;
    void* state;                // [rhs][ne][nf][nb]
    int64_t rhs_stride;         // ne * nf * nb
    int* err;                   // error word (0 = ok, 1 = causality, 2 = non-finite)
    int q, m;
    int max_patch;
    double taylor[kMaxTaylor];  // (1/m)^n / n!
    double tsub[kMaxSub + 1];   // sub-interval starts i / m, i = 0..m
};

__host__ __device__ constexpr int pad4(int n) { return (n + 3) & ~3; }
// dim P_k on a simplex of dimension `dim` (0 for k < 0), and the degree of the r-th basis
// function when the basis is ordered by total degree (as the reference tables are)
__host__ __device__ constexpr int dim_pk(int dim, int k) {
    return k < 0 ? 0 : dim == 1 ? k + 1 : dim == 2 ? (k + 1) * (k + 2) / 2 : (k + 1) * (k + 2) * (k + 3) / 6;
}
__host__ __device__ constexpr int degree_of(int dim, int r) {
    int k = 0;
    while (r >= dim_pk(dim, k)) ++k;
    return k;
}

// Kernel shape variants travel in the degree template argument as PV = p + 16 v.
// v = 0 (default): an FP32 stage item covers a pair of patch elements with the same local index
// of V (they share every table read); v = 1: one element per item, twice the items at half
// the work each, which shortens a tent when the layers have fewer tents than the GPU has CTA
// slots (3D, 512 threads per CTA from p = 4 so that a 24-element patch still fits one round);
// v = 2: one element and one basis function (or facet mode) per item, 512 threads per CTA in
// 3D: every phase of a 24-element p <= 3 patch in one round at a quarter of the default's
// per-thread work, for the shortest tents on latency-bound layers.  v = 3, 4: the item shapes
// of v = 1, 2 (512 threads) with the volume term on the tcgen05 tensor cores (3D FP32, see
// the tcgen05 section at the end of this file).
template <int DIM, int PV>
struct Shape {
    static constexpr int P = PV & 15, V = PV >> 4;
    static constexpr bool TC5 = V >= 3;                   // volume term on tcgen05
    static constexpr int VB = V == 3 ? 1 : V == 4 ? 2 : V;   // item shape
    static constexpr bool PAIRS = VB == 0;                // FP32 items pair elements (FP64 never)
    static constexpr int NF = DIM == 2 ? 3 : 6;
    static constexpr int NB = DIM == 2 ? (P + 1) * (P + 2) / 2 : (P + 1) * (P + 2) * (P + 3) / 6;
    static constexpr int NFB = DIM == 2 ? P + 1 : (P + 1) * (P + 2) / 2;
    static constexpr int NBP = pad4(NB);
    static constexpr int NFBP = pad4(NFB);
    static constexpr int GIS = pad4(NF);                  // row stride of G^-1 in shared memory
    static constexpr int NV = DIM + 1;
    static constexpr int NT = DIM == 2 ? 128 : ((VB == 1 && (P >= 4 || TC5)) || VB == 2 ? 512 : 256);   // threads per CTA
    static constexpr int AP = VB == 2 ? 1 : 2;         // basis functions (facet modes) per thread
    static constexpr int NAG = (NB + AP - 1) / AP;     // basis groups per element
    static constexpr int NCG = (NFB + AP - 1) / AP;    // facet-mode groups per facet
    // Degree structure of the tables (basis ordered by degree): S[a][b] = 0 for deg b > deg a
    // and Tr[c][b] = 0 for deg b < deg c.  A thread's first row a = g < NAG has degree
    // < P when NAG <= dim P_{P-1}, so the volume term needs it only for b < NBLO; its second
    // facet row c = g + NCG has degree >= TDEG, so the traces need it only for
    // b >= dim P_{TDEG-1}.
    static constexpr int NBLO = dim_pk(DIM, P - 1);
    static constexpr bool VSPLIT = NAG <= NBLO;
    static constexpr int TDEG = degree_of(DIM - 1, NCG);
    static constexpr int TLO = dim_pk(DIM, TDEG - 1);
    // Factored volume term: W = M_j U (rows c < NBM = dim P_{P-1}), then P_l = D_l^T W.
    // D_l^T[a][c] = 0 unless deg c < deg a: a thread's first row (a < NAG, degree <= DA1) needs
    // only c < CV1.  M_j[c][b] = 0 unless |deg b - deg c| <= 1: first W rows (c < NWG, degree
    // <= DC1) need only b < BW1, second W rows (degree >= DC2) only b >= BW2.
    static constexpr int NBM = dim_pk(DIM, P - 1);
    static constexpr int NBMP = pad4(NBM);
    static constexpr int NWG = (NBM + AP - 1) / AP;
    static constexpr int DA1 = degree_of(DIM, NAG - 1);
    static constexpr int CV1 = dim_pk(DIM, DA1 - 1);
    static constexpr int DC1 = degree_of(DIM, NWG - 1);
    static constexpr int BW1 = dim_pk(DIM, DC1 + 1);
    static constexpr int DC2 = degree_of(DIM, NWG);
    static constexpr int BW2 = dim_pk(DIM, DC2 - 2);
    // tcgen05 volume operator: M = 64 rows a (basis functions, NB used), N = the patch's
    // (element, field) rows padded to 16 (at most TCOLS = 256 TMEM columns), K = (direction l,
    // row c < NBM) padded to the MMA's k = 8; the volume result goes to shared memory with the
    // odd row stride VS (conflict-free banks)
    static constexpr int TK = (DIM * NBM + 7) / 8 * 8;
    static constexpr int TCOLS = 256;
    static constexpr int VS = NB % 2 ? NB : NB + 1;
    static_assert(!TC5 || (DIM == 3 && NB <= 64 && VS <= 2 * TK), "tcgen05 volume layout");
};

// CTAs per SM the register budget is shaped for (two 256-thread CTAs fit the FP32 3D
// shared-memory footprint up to p = 4; FP64 p >= 3 fits one)
template <typename Real, int DIM, int PV>
struct MinBlocks {
    static constexpr int P = Shape<DIM, PV>::P;
    static constexpr int value = Shape<DIM, PV>::NT > 256 ? 1 : (((sizeof(Real) == 4 && P <= 4) || P <= 2) ? 2 : 1);
};

template <typename Real>
struct Vec;
template <>
struct Vec<float> {
    using T = float4;
    static constexpr int W = 4;
    static __device__ __forceinline__ void get(const T& v, float o[4]) { o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w; }
};
template <>
struct Vec<double> {
    using T = double2;
    static constexpr int W = 2;
    static __device__ __forceinline__ void get(const T& v, double o[2]) { o[0] = v.x; o[1] = v.y; }
};

// Shared-memory strides of the per-element blocks that threads of one warp access for
// different elements: facet traces / fluxes (FSZ per facet, TSZ per element) and G^-1 (GSZ per
// element) are padded so that the facets of one element and elements one or two slots apart
// start in different shared-memory banks (BANKW = banks per bank row in units of Real).
template <typename Real, int DIM, int P>
struct Strides {
    using Sh = Shape<DIM, P>;
    static constexpr int BANKW = 32 * 4 / (int)sizeof(Real);
    static constexpr int up_to(int x, int r) { return x + ((r - x % BANKW) % BANKW + BANKW) % BANKW; }
    static constexpr int FSZ = up_to(Sh::NF * Sh::NFBP, BANKW / 2);
    static constexpr int TSZ = up_to(DIM * FSZ, 3 * BANKW / 4);
    static constexpr int GSZ = (Sh::NF * Sh::GIS) % (BANKW / 2) == 0 ? Sh::NF * Sh::GIS + 4 : Sh::NF * Sh::GIS;
};

// MODE 0: SIMT contractions in the state precision; 1: TF32 tensor-core MMAs (FP32 state,
// FP32 accumulate); 2: the same with a 3-term hi + lo split of both operands; 3: SIMT FP32
// contractions with the Taylor sum carried as an FP32 pair hi + lo (two-sum) and an FP64
// state between tents; 4: SIMT contractions, but the tent ODE advanced by the classical
// Runge-Kutta method on the substituted equation d/dt Y = A M^-1 Y instead of SAT (the
// approach Sec. 3 contrasts with SAT; a negative control for convergence studies).
template <int MODE>
struct ModeTraits {
    static constexpr bool simt = MODE == 0 || MODE == 3 || MODE == 4;
    static constexpr bool split = MODE == 3;
    static constexpr bool rk4 = MODE == 4;
};
template <typename Real, int MODE>
using StateOf = typename std::conditional<ModeTraits<MODE>::split, double, Real>::type;

// shared-memory carve-up, sizes from the mesh's largest patch
template <typename Real, int DIM, int P>
struct SmemLayout {
    using Sh = Shape<DIM, P>;
    static __host__ __device__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
    size_t off_Y, off_Ylo, off_Ua, off_Ub, off_W, off_tr, off_Gi, off_gphi, off_gdel, off_mat, off_ac, off_gd, off_gpr,
        off_nrm, off_liftc, off_trs, off_Z, off_j, off_nslot, off_nfi, off_pair, off_own, bytes, state_bytes, tr_bytes;
    size_t off_tW, off_tD, off_tbar;   // tcgen05 operands (hi, lo parts), mbarriers + TMEM address
    int tc_rows;                       // rows of the W operand: (element, field) rows padded to 16
    bool split, factored, twobuf, rk4;   // rk4: Y at the sub-step start (Ylo slot), stage input (Ub)
    // mode (see ModeTraits): split carries the Taylor accumulator Y as an unevaluated pair
    // hi + lo (one more patch-state buffer); the SIMT modes use the factored volume term (a W
    // buffer) and update U in place, the tensor-core modes keep two U buffers (twobuf also
    // asks for the second one, for the adjoint's reverse recursion)
    __host__ __device__ explicit SmemLayout(int mp, int mode = 0, bool two = false)
        : split(mode == 3), factored((mode == 0 || mode == 3 || mode == 4) && !Sh::TC5),
          twobuf(two || mode == 1 || mode == 2 || mode == 4), rk4(mode == 4) {
        size_t o = 0;
        state_bytes = (size_t)mp * Sh::NF * Sh::NBP * sizeof(Real);
        tr_bytes = (size_t)mp * Strides<Real, DIM, P>::TSZ * sizeof(Real);
        off_Y = o; o = align16(o + state_bytes);
        off_Ylo = o; if (split || rk4) o = align16(o + state_bytes);
        off_Ua = o; o = align16(o + state_bytes);
        off_Ub = o; if (twobuf) o = align16(o + state_bytes);
        off_W = o; if (factored) o = align16(o + (size_t)mp * Sh::NF * Sh::NBMP * sizeof(Real));
        off_tr = o; o = align16(o + tr_bytes);
        off_Gi = o; o = align16(o + (size_t)mp * Strides<Real, DIM, P>::GSZ * sizeof(Real));
        off_gphi = o; o = align16(o + (size_t)mp * 3 * sizeof(double));
        off_gdel = o; o = align16(o + (size_t)mp * 3 * sizeof(double));
        off_mat = o; o = align16(o + (size_t)mp * 2 * sizeof(double));
        off_ac = o; o = align16(o + (size_t)mp * DIM * 3 * sizeof(Real));
        off_gd = o; o = align16(o + (size_t)mp * 3 * sizeof(Real));
        off_gpr = o; o = align16(o + (size_t)mp * 5 * sizeof(Real));
        off_nrm = o; o = align16(o + (size_t)mp * DIM * 3 * sizeof(Real));
        off_liftc = o; o = align16(o + (size_t)mp * DIM * sizeof(Real));
        off_trs = o; o = align16(o + (size_t)mp * sizeof(Real));
        off_Z = o; o = align16(o + (size_t)mp * (1 + DIM) * sizeof(Real));
        off_j = o; o = align16(o + (size_t)mp);
        off_nslot = o; o = align16(o + (size_t)mp * DIM);
        off_nfi = o; o = align16(o + (size_t)mp * DIM);
        off_pair = o; o = align16(o + (size_t)mp * 2 + 4);
        off_own = o; o = align16(o + (size_t)mp * DIM * 2 + 4);
        tc_rows = 0;
        off_tW = off_tD = off_tbar = o;
        if (Sh::TC5) {
            tc_rows = (mp * Sh::NF + 15) / 16 * 16;
            off_tW = o = (o + 127) & ~size_t(127); o += (size_t)2 * tc_rows * Sh::TK * sizeof(float);
            off_tD = o; o += (size_t)2 * 64 * Sh::TK * sizeof(float);
            off_tbar = o; o += 32;
        }
        bytes = o;
    }
};

// Upwind flux on coefficient vectors (Sec. 3 upwind flux, impedance form; PEC = mirror
// state E+ = -E-, H+ = H-).  um/up/out in the 6-component (E, H) ordering.
template <typename Real>
__device__ __forceinline__ void upwind6(const Real um[6], const Real up[6], const Real n[3], Real Zm, Real Zp,
                                        Real out[6]) {
    Real Emn = um[0] * n[0] + um[1] * n[1] + um[2] * n[2];
    Real Epn = up[0] * n[0] + up[1] * n[1] + up[2] * n[2];
    Real Emt[3], Ept[3], dH[3];
    for (int c = 0; c < 3; ++c) {
        Emt[c] = um[c] - Emn * n[c];
        Ept[c] = up[c] - Epn * n[c];
        dH[c] = um[3 + c] - up[3 + c];
    }
    const Real inv = Real(1) / (Zm + Zp);
    // H* x n = (Zm Hm x n + Zp Hp x n + Emt - Ept) / (Zm + Zp)
    Real hx[3] = {Zm * um[3] + Zp * up[3], Zm * um[4] + Zp * up[4], Zm * um[5] + Zp * up[5]};
    out[0] = (hx[1] * n[2] - hx[2] * n[1] + Emt[0] - Ept[0]) * inv;
    out[1] = (hx[2] * n[0] - hx[0] * n[2] + Emt[1] - Ept[1]) * inv;
    out[2] = (hx[0] * n[1] - hx[1] * n[0] + Emt[2] - Ept[2]) * inv;
    // E*_t = (Zp Emt + Zm Ept + Zp Zm (Hm - Hp) x n) / (Zm + Zp); F_H = -E*_t x n
    const Real zz = Zp * Zm;
    Real et[3] = {(Zp * Emt[0] + Zm * Ept[0] + zz * (dH[1] * n[2] - dH[2] * n[1])) * inv,
                  (Zp * Emt[1] + Zm * Ept[1] + zz * (dH[2] * n[0] - dH[0] * n[2])) * inv,
                  (Zp * Emt[2] + Zm * Ept[2] + zz * (dH[0] * n[1] - dH[1] * n[0])) * inv};
    out[3] = -(et[1] * n[2] - et[2] * n[1]);
    out[4] = -(et[2] * n[0] - et[0] * n[2]);
    out[5] = -(et[0] * n[1] - et[1] * n[0]);
}

template <int DIM>
__device__ __forceinline__ int field6(int r) {   // index of field r inside (Ex,Ey,Ez,Hx,Hy,Hz)
    if (DIM == 3) return r;
    return r == 2 ? 5 : r;
}

// Per-CTA view of one tent: shared-memory buffers and tent scalars.
template <typename Real, int DIM, int P>
struct TentCtx {
    using Sh = Shape<DIM, P>;
    Real *sY, *sYlo, *sUa, *sUb, *sW, *sTr, *sGi;   // sYlo / sUb / sW null when the layout has none
    Real* sY0;                                     // RK4 mode: Y at the start of the sub-step
    double *sGphi, *sGdel, *sMat;
    Real *sAc, *sGd, *sNrm, *sLiftc, *sTrs, *sZ;
    Real* sGpr;   // [k][5]: grad phi at the tent bottom, eps, mu in the state precision
    int8_t *sJ, *sNslot, *sNfi, *sPair;   // sPair: [pair][2] element slots (second -1: single)
    int8_t* sOwn;                         // [facet][2]: (slot, facet position) owning each facet
    int* sNpair;
    int* sNown;
    // tcgen05 volume operator: W operand (the MMA's B) hi / lo, D table (the MMA's A) hi / lo,
    // volume result (over the W operand once the MMAs have read it), mbarriers [MMA done, table
    // loaded] and [TMEM address, MMA phase, failure flag]
    float *sWh, *sWl, *sDh, *sDl, *sVol;
    uint64_t* sBar;
    uint32_t* sTc;
    int tc_rows;
    int V, ns;
    int64_t pb;
    double tb, dt;

    __device__ void carve(unsigned char* smem, const SmemLayout<Real, DIM, P>& lay) {
        sY = (Real*)(smem + lay.off_Y);
        sYlo = lay.split ? (Real*)(smem + lay.off_Ylo) : nullptr;
        sY0 = lay.rk4 ? (Real*)(smem + lay.off_Ylo) : nullptr;
        sUa = (Real*)(smem + lay.off_Ua);
        sUb = lay.twobuf ? (Real*)(smem + lay.off_Ub) : nullptr;
        sW = lay.factored ? (Real*)(smem + lay.off_W) : nullptr;
        sTr = (Real*)(smem + lay.off_tr);
        sGi = (Real*)(smem + lay.off_Gi);
        sGphi = (double*)(smem + lay.off_gphi);
        sGdel = (double*)(smem + lay.off_gdel);
        sMat = (double*)(smem + lay.off_mat);
        sAc = (Real*)(smem + lay.off_ac);
        sGd = (Real*)(smem + lay.off_gd);
        sGpr = (Real*)(smem + lay.off_gpr);
        sNrm = (Real*)(smem + lay.off_nrm);
        sLiftc = (Real*)(smem + lay.off_liftc);
        sTrs = (Real*)(smem + lay.off_trs);
        sZ = (Real*)(smem + lay.off_Z);
        sJ = (int8_t*)(smem + lay.off_j);
        sNslot = (int8_t*)(smem + lay.off_nslot);
        sNfi = (int8_t*)(smem + lay.off_nfi);
        sPair = (int8_t*)(smem + lay.off_pair + 4);
        sNpair = (int*)(smem + lay.off_pair);
        sOwn = (int8_t*)(smem + lay.off_own + 4);
        sNown = (int*)(smem + lay.off_own);
        tc_rows = lay.tc_rows;
        if (Sh::TC5) {
            sWh = (float*)(smem + lay.off_tW);
            sWl = sWh + (size_t)lay.tc_rows * Sh::TK;
            sDh = (float*)(smem + lay.off_tD);
            sDl = sDh + 64 * Sh::TK;
            sVol = sWh;
            sBar = (uint64_t*)(smem + lay.off_tbar);
            sTc = (uint32_t*)(smem + lay.off_tbar + 16);
        } else {
            sWh = sWl = sDh = sDl = sVol = nullptr;
            sBar = nullptr;
            sTc = nullptr;
        }
    }
};

// ---------------------------------------------------------------------------------------
// tcgen05 primitives (inline PTX, sm_103a) for the volume operator of kernel shapes v = 3, 4.
// Operands live in shared memory in the no-swizzle K-major layout: 8-row x 16-byte core
// matrices, the 4-element k groups of one 8-row group 128 B apart, 8-row groups TK x 32 B
// apart; the FP32 accumulator of a 64-row MMA keeps row r in TMEM lane 32 (r / 16) + r % 16.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t tf32_bits(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ long long tc_clock() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// float index of entry (row r, k) of a K-major operand with TK columns
template <int TK>
__device__ __forceinline__ int tc_off(int r, int k) {
    return (r >> 3) * TK * 8 + (k >> 2) * 32 + (r & 7) * 4 + (k & 3);
}
// shared-memory matrix descriptor: start address, k-group stride (LBO), 8-row-group stride
// (SBO), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// bounded wait for the phase of `parity` of a shared-memory mbarrier (false after one second)
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    long long deadline = 0;
    for (int it = 0;; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(addr), "r"(parity)
            : "memory");
        if (ok) return true;
        const long long now = tc_clock();
        if (it == 0) deadline = now + 1000000000LL;
        else if (now > deadline) return false;
    }
}
// 16 consecutive TMEM columns of this warp's 32 lanes, one column per register
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t v[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Once per CTA before its first tent: zero the W operand (its K padding and spare rows must be
// finite), initialise the two mbarriers, bring both parts of the D table into shared memory with
// one bulk asynchronous copy (the TMA engine's non-tensor form) and allocate the TMEM columns.
template <typename Real, int DIM, int P>
__device__ void tc5_begin(TentCtx<Real, DIM, P>& c, const KArgs& a) {
    using Sh = Shape<DIM, P>;
    float4* A4 = (float4*)c.sWh;
    const int n4 = 2 * c.tc_rows * Sh::TK / 4;
    for (int i = threadIdx.x; i < n4; i += Sh::NT) A4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) {
        c.sTc[1] = 0;
        c.sTc[2] = a.Dtc ? 0u : 1u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&c.sBar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&c.sBar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool have_tables = a.Dtc != nullptr;
    if (threadIdx.x == 0 && have_tables) {
        const uint32_t bytes = 2u * 64u * Sh::TK * 4u, bar = smem_u32(&c.sBar[1]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(c.sDh)),
                     "l"(a.Dtc), "r"(bytes), "r"(bar)
                     : "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&c.sTc[0])),
                     "r"(Sh::TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (!have_tables) {
        if (threadIdx.x == 0) atomicCAS(a.err, 0, 3);
    } else if (!tc_wait(&c.sBar[1], 0)) {
        atomicCAS(a.err, 0, 3);
        c.sTc[2] = 1;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// After the CTA's last tent: release the TMEM columns
template <typename Real, int DIM, int P>
__device__ void tc5_end(TentCtx<Real, DIM, P>& c) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.sTc[0]), "r"(Shape<DIM, P>::TCOLS)
                     : "memory");
}

// One thread issues the stage's volume MMAs: vol[a][(k, f)] = sum over K of D[a][K] W[(k, f)][K]
// as D_lo W_hi + D_hi W_lo + D_hi W_hi (TF32 operands, FP32 accumulation in TMEM; M = 64 rows a,
// N = the tent's (element, field) rows padded to 16), then a commit to the MMA mbarrier.
template <typename Real, int DIM, int P>
__device__ void tc5_issue(TentCtx<Real, DIM, P>& c) {
    using Sh = Shape<DIM, P>;
    constexpr uint32_t SBO = Sh::TK * 32;
    const uint32_t n = (uint32_t)((c.ns * Sh::NF + 15) / 16 * 16);
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((uint32_t)(64 >> 4) << 24);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t d = c.sTc[0];
    const uint32_t dop[2] = {smem_u32(c.sDh), smem_u32(c.sDl)}, wop[2] = {smem_u32(c.sWh), smem_u32(c.sWl)};
    uint32_t acc = 0;
    for (int t = 0; t < 3; ++t) {
        const uint32_t A = dop[t == 0 ? 1 : 0], B = wop[t == 1 ? 1 : 0];
        for (int s = 0; s < Sh::TK / 8; ++s) {
            const uint64_t ad = tc_desc(A + s * 256, 128, SBO), bd = tc_desc(B + s * 256, 128, SBO);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                : "memory");
            acc = 1;
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&c.sBar[0]))
                 : "memory");
}

// All threads: wait (bounded) for the stage's MMAs, then the warps of the lane quarters that
// hold basis functions copy the accumulators to sVol[(k, f)][a] (row stride VS) over the W
// operand, which the finished MMAs no longer read.  A 64-row accumulator keeps row a in TMEM
// lane 32 (a / 16) + a % 16, column (k, f): lanes 0..15 of each quarter.
template <typename Real, int DIM, int P>
__device__ void tc5_collect(TentCtx<Real, DIM, P>& c, const KArgs& a, uint32_t parity) {
    using Sh = Shape<DIM, P>;
    constexpr int VS = Sh::VS, NB = Sh::NB, NQ = (NB + 15) / 16;
    if (c.sTc[2] == 0 && !tc_wait(&c.sBar[0], parity)) {
        atomicCAS(a.err, 0, 3);
        c.sTc[2] = 1;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, q = warp & 3;
    const int rows = c.ns * Sh::NF;
    const int ncb = (rows + 15) / 16;
    const uint32_t tbase = c.sTc[0];
    if (q < NQ) {
        const int av = lane < 16 ? 16 * q + lane : NB;
        for (int cb = warp >> 2; cb < ncb; cb += Sh::NT / 128) {
            uint32_t v[16];
            tc_ld16(tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(cb * 16), v);
            if (av < NB) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int r = cb * 16 + j;
                    if (r < rows) c.sVol[r * VS + av] = __uint_as_float(v[j]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// (a) gather: per-element setup from FP64 geometry and the current front; patch state of
// `src` into sY (pads zero); U and facet buffers zeroed so their pads stay zero.
template <typename T>
__device__ __forceinline__ T load_cg(const T* p) { return __ldcg(p); }

template <typename Real, int DIM, int P, bool CG = false, typename SrcT = Real>
__device__ void tent_setup(TentCtx<Real, DIM, P>& c, const KArgs& a, int64_t tent, const SrcT* src) {
    using Sh = Shape<DIM, P>;
    constexpr int NF = Sh::NF, NB = Sh::NB, NV = Sh::NV, NT = Sh::NT, NBP = Sh::NBP;
    constexpr int ESZ = NF * NBP, TSZ = Strides<Real, DIM, P>::TSZ;
    const int tid = threadIdx.x;
    c.V = a.tent_v[tent];
    c.tb = a.tent_tb[tent];
    c.dt = a.tent_tt[tent] - c.tb;
    c.pb = a.patch_ptr[c.V];
    c.ns = (int)(a.patch_ptr[c.V + 1] - c.pb);
    const int ns = c.ns;
    const double dt = c.dt;
    for (int k = tid; k < ns; k += NT) {
        const int e = a.patch_elem[c.pb + k];
        const int8_t* info = a.patch_info + (c.pb + k) * 12;
        const int j = info[0];
        const double* g = a.geo + (int64_t)e * 32;
        double gp[3] = {0, 0, 0};
        for (int i = 0; i < NV; ++i) {
            const double* tp = a.tau + a.elems[(int64_t)e * NV + i];
            const double tv = (i == j) ? c.tb : (CG ? load_cg(tp) : *tp);
            for (int q = 0; q < 3; ++q) gp[q] += tv * g[3 * i + q];
        }
        for (int q = 0; q < 3; ++q) {
            c.sGphi[3 * k + q] = gp[q];
            c.sGdel[3 * k + q] = dt * g[3 * j + q];
            c.sGd[3 * k + q] = (Real)(dt * g[3 * j + q]);
        }
        for (int l = 0; l < DIM; ++l)
            for (int q = 0; q < 3; ++q) c.sAc[(k * DIM + l) * 3 + q] = (Real)(dt * g[3 * (l + 1) + q]);
        c.sMat[2 * k] = g[29];
        c.sMat[2 * k + 1] = g[30];
        for (int q = 0; q < 3; ++q) c.sGpr[5 * k + q] = (Real)gp[q];
        c.sGpr[5 * k + 3] = (Real)g[29];
        c.sGpr[5 * k + 4] = (Real)g[30];
        c.sZ[k * (1 + DIM)] = (Real)g[31];
        c.sTrs[k] = (Real)g[28];
        c.sJ[k] = (int8_t)j;
        for (int f = 0, fi = 0; f < NV; ++f) {
            if (f == j) continue;
            for (int q = 0; q < 3; ++q) c.sNrm[(k * DIM + fi) * 3 + q] = (Real)g[12 + 3 * f + q];
            c.sLiftc[k * DIM + fi] = (Real)(dt * g[24 + f] * g[28]);
            c.sNslot[k * DIM + fi] = info[4 + f];
            ++fi;
        }
    }
    for (int idx = tid; idx < ns * ESZ; idx += NT) {
        const int k = idx / ESZ, r = idx - k * ESZ, s = r / NBP, b = r - s * NBP;
        const SrcT* sp = src + ((int64_t)a.patch_elem[c.pb + k] * NF + s) * NB + b;
        const SrcT v = b < NB ? (CG ? load_cg(sp) : *sp) : SrcT(0);
        if constexpr (std::is_same<SrcT, Real>::value) {
            c.sY[idx] = v;
        } else {   // FP64 state -> FP32 pair hi + lo (exact: |lo| <= ulp(hi) / 2)
            const Real hi = (Real)v;
            c.sY[idx] = hi;
            c.sYlo[idx] = (Real)(v - (SrcT)hi);
        }
        c.sUa[idx] = Real(0);
        if (c.sUb) c.sUb[idx] = Real(0);
    }
    if (c.sW)
        for (int idx = tid; idx < ns * NF * Sh::NBMP; idx += NT) c.sW[idx] = Real(0);
    for (int idx = tid; idx < ns * TSZ; idx += NT) c.sTr[idx] = Real(0);
    __syncthreads();
    // neighbour's facet position (needs the neighbour's j) and impedance
    for (int k = tid; k < ns; k += NT) {
        const int8_t* info = a.patch_info + (c.pb + k) * 12;
        const int j = c.sJ[k];
        for (int f = 0, fi = 0; f < NV; ++f) {
            if (f == j) continue;
            const int s2 = info[4 + f];
            int8_t nfi = -1;
            Real z2 = c.sZ[k * (1 + DIM)];
            if (s2 >= 0) {
                const int f2 = info[8 + f];
                nfi = (int8_t)(f2 - (f2 > c.sJ[s2] ? 1 : 0));
                z2 = c.sZ[s2 * (1 + DIM)];
            }
            c.sNfi[k * DIM + fi] = nfi;
            c.sZ[k * (1 + DIM) + 1 + fi] = z2;
            ++fi;
        }
    }
    if (tid == 0) {   // pairs of consecutive elements with the same local index of V
        int np = 0;
        for (int k = 0; k < ns;) {
            const bool pair = k + 1 < ns && c.sJ[k + 1] == c.sJ[k];
            c.sPair[2 * np] = (int8_t)k;
            c.sPair[2 * np + 1] = pair ? (int8_t)(k + 1) : (int8_t)-1;
            ++np;
            k += pair ? 2 : 1;
        }
        *c.sNpair = np;
        int no = 0;   // facets containing V, each once: boundary facets and the lower slot of interior ones
        for (int k = 0; k < ns; ++k)
            for (int fi = 0; fi < DIM; ++fi) {
                const int s2 = c.sNslot[k * DIM + fi];
                if (s2 < 0 || s2 > k) {
                    c.sOwn[2 * no] = (int8_t)k;
                    c.sOwn[2 * no + 1] = (int8_t)fi;
                    ++no;
                }
            }
        *c.sNown = no;
    }
    __syncthreads();
}

// G(t_i)^-1 per element from the closed form (Sec. 4): with P = I - g g^T / (eps mu) and
// s = 1 / (eps mu - |g|^2),  G^-1 = s [[mu P, -[g]x], [[g]x, eps P]]  ([g]x w = g x w),
// one row per thread, in the state precision.  The causality test |g| < sqrt(eps mu) at
// t_i (and at the tent top when i = 0) decides an error and is taken in FP64.
template <typename Real, int DIM, int P>
__device__ void tent_ginv_into(TentCtx<Real, DIM, P>& c, const KArgs& a, double ti, Real tr, bool check, Real* dst,
                               int t0, int nthr) {
    using Sh = Shape<DIM, P>;
    constexpr int NF = Sh::NF;
    const int me = (int)threadIdx.x - t0;
    if (me < 0) return;
    if (check)   // grad phi is affine in t^, so |grad phi|^2 is convex: bottom and top bound the tent
        for (int k = me; k < c.ns; k += nthr) {
            const double eps = c.sMat[2 * k], mu = c.sMat[2 * k + 1];
            double gg = 0, gt = 0;
            for (int q = 0; q < 3; ++q) {
                const double g = c.sGphi[3 * k + q] + ti * c.sGdel[3 * k + q];
                const double h = c.sGphi[3 * k + q] + c.sGdel[3 * k + q];
                gg += g * g;
                gt += h * h;
            }
            if (!(gg < eps * mu) || !(gt < eps * mu)) atomicCAS(a.err, 0, 1);
        }
    for (int idx = me; idx < c.ns * NF; idx += nthr) {
        const int k = idx / NF, R = field6<DIM>(idx - k * NF);
        const Real* gp = c.sGpr + 5 * k;
        Real g[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) g[q] = gp[q] + tr * c.sGd[3 * k + q];
        const Real eps = gp[3], mu = gp[4], em = eps * mu;
        const Real s = Real(1) / (em - (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]));
        const int rq = R < 3 ? R : R - 3;                  // component of the row's field
        const Real d = s * (R < 3 ? mu : eps);             // diagonal block: s mu P or s eps P
        const Real pr = d * g[rq] / em;
        const Real sx = R < 3 ? -s : s;                    // off-diagonal block: -s [g]x or s [g]x
        Real row[6];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const Real cr = q == rq ? Real(0) : ((q == (rq + 1) % 3) ? -g[(rq + 2) % 3] : g[(rq + 1) % 3]);
            const Real diag = (q == rq ? d : Real(0)) - pr * g[q];
            row[R < 3 ? q : 3 + q] = diag;
            row[R < 3 ? 3 + q : q] = sx * cr;
        }
        Real* out = dst + k * Strides<Real, DIM, P>::GSZ + (idx - k * NF) * Sh::GIS;
#pragma unroll
        for (int q = 0; q < NF; ++q) out[q] = row[field6<DIM>(q)];
    }
}

template <typename Real, int DIM, int P>
__device__ __forceinline__ void tent_ginv_at(TentCtx<Real, DIM, P>& c, const KArgs& a, double ti, bool check_top) {
    tent_ginv_into(c, a, ti, (Real)ti, check_top, c.sGi, 0, (int)blockDim.x);
}

// G(t_i)^-1 at the start of sub-interval i (the tent bottom and top are checked at i = 0)
template <typename Real, int DIM, int P>
__device__ __forceinline__ void tent_ginv(TentCtx<Real, DIM, P>& c, const KArgs& a, int i) {
    tent_ginv_into(c, a, 0.0, (Real)a.tsub[i], i == 0, c.sGi, 0, (int)blockDim.x);
}

// Error-free sum of two floats (Knuth's two-sum): hi + lo == a + b exactly, hi = fl(a + b).
// The explicit round-to-nearest intrinsics keep the compiler from contracting or reordering.
__device__ __forceinline__ void two_sum(float a, float b, float& hi, float& lo) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float aa = __fsub_rn(s, bb);
    lo = __fadd_rn(__fsub_rn(a, aa), __fsub_rn(b, bb));
    hi = s;
}
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ void two_sum(double a, double b, double& hi, double& lo) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double aa = __dsub_rn(s, bb);
    lo = __dadd_rn(__dsub_rn(a, aa), __dsub_rn(b, bb));
    hi = s;
}

// dst = G^-1 src per coefficient column (b < NB).  With a split accumulator the pair
// (src, sYlo) is first renormalised so that src holds the correctly rounded sum.
template <typename Real, int DIM, int P>
__device__ void tent_apply_ginv(TentCtx<Real, DIM, P>& c, Real* src, Real* dst) {
    using Sh = Shape<DIM, P>;
    constexpr int NF = Sh::NF, NB = Sh::NB, ESZ = NF * Sh::NBP, NBP = Sh::NBP, GIS = Sh::GIS;
    for (int idx = threadIdx.x; idx < c.ns * NB; idx += blockDim.x) {
        const int k = idx / NB, b = idx - k * NB;
        const Real* Gi = c.sGi + k * Strides<Real, DIM, P>::GSZ;
        Real y[NF];
#pragma unroll
        for (int s = 0; s < NF; ++s) {
            const int i = k * ESZ + s * NBP + b;
            if (c.sYlo) {
                Real hi, lo;
                two_sum(src[i], c.sYlo[i], hi, lo);
                src[i] = hi;
                c.sYlo[i] = lo;
            }
            y[s] = src[i];
        }
#pragma unroll
        for (int r = 0; r < NF; ++r) {
            Real acc = 0;
#pragma unroll
            for (int s = 0; s < NF; ++s) acc += Gi[r * GIS + s] * y[s];
            dst[k * ESZ + r * NBP + b] = acc;
        }
    }
}

// W = M_j U for the factored volume term (rows c < NBM): one thread per (pair of elements
// with the same local index j, or single element in FP64, two rows c and c + NWG); the rows'
// zero blocks (|deg b - deg c| > 1) are skipped
template <typename Real, int DIM, int P>
__device__ __forceinline__ void tent_w_item(TentCtx<Real, DIM, P>& c, const KArgs& a, const Real* Ucur, int w) {
    using Sh = Shape<DIM, P>;
    using VT = typename Vec<Real>::T;
    constexpr int NF = Sh::NF, NBP = Sh::NBP, NBM = Sh::NBM, NBMP = Sh::NBMP, NWG = Sh::NWG;
    constexpr int AP = Sh::AP, W = Vec<Real>::W, ESZ = NF * NBP, WSZ = NF * NBMP;
    constexpr int EP = (sizeof(Real) == 4 && Sh::PAIRS) ? 2 : 1;
    constexpr int WMAT = NBP * AP * NWG;
    const int pi = w / NWG, g = w - pi * NWG;
    const int k0 = EP == 2 ? c.sPair[2 * pi] : pi;
    const int kk1 = EP == 2 ? c.sPair[2 * pi + 1] : -1;
    const int kk[2] = {k0, kk1 >= 0 ? kk1 : k0};
    const Real* Mg = (const Real*)a.Mc + (size_t)c.sJ[k0] * WMAT + g * W;
    Real acc[EP][AP][NF];
#pragma unroll
    for (int e = 0; e < EP; ++e)
#pragma unroll
        for (int ci = 0; ci < AP; ++ci)
#pragma unroll
            for (int s = 0; s < NF; ++s) acc[e][ci][s] = 0;
    // column block [b, b + W): rows R0 <= ci < R1
    auto block = [&](int b, auto r0, auto r1) {
        constexpr int R0 = decltype(r0)::value, R1 = decltype(r1)::value < AP ? decltype(r1)::value : AP;
        Real mv[AP][W];
#pragma unroll
        for (int ci = R0; ci < R1; ++ci) Vec<Real>::get(__ldg((const VT*)(Mg + b * AP * NWG + ci * NWG * W)), mv[ci]);
#pragma unroll
        for (int e = 0; e < EP; ++e) {
            const Real* U = Ucur + kk[e] * ESZ;
#pragma unroll
            for (int s = 0; s < NF; ++s) {
                Real u[W];
                Vec<Real>::get(*(const VT*)(U + s * NBP + b), u);
#pragma unroll
                for (int v = 0; v < W; ++v)
#pragma unroll
                    for (int ci = R0; ci < R1; ++ci) acc[e][ci][s] += mv[ci][v] * u[v];
            }
        }
    };
    using I0 = std::integral_constant<int, 0>;
    using I1 = std::integral_constant<int, 1>;
    using I2 = std::integral_constant<int, 2>;
    constexpr int B2 = Sh::BW2 / W * W;                       // second rows vanish below
    constexpr int B1 = (Sh::BW1 + W - 1) / W * W;             // first rows vanish from here
    constexpr int B1c = B1 < NBP ? B1 : NBP;
#pragma unroll 1
    for (int b = 0; b < B2; b += W) block(b, I0{}, I1{});
#pragma unroll 1
    for (int b = B2; b < B1c; b += W) block(b, I0{}, I2{});
#pragma unroll 1
    for (int b = B1c; b < NBP; b += W) block(b, I1{}, I2{});
    if constexpr (Sh::TC5 && DIM == 3) {
        // W operand of the tcgen05 volume term: the curl combination folded into W,
        // Wt[(k, f)][(l, c)] = (E rows: -a_l x W_H, H rows: a_l x W_E)_f, so that the MMA with
        // D[a][(l, c)] = D_l^T[a][c] gives the element's volume term directly; TF32 hi + lo
        const Real* ac = c.sAc + k0 * DIM * 3;
#pragma unroll
        for (int ci = 0; ci < AP; ++ci) {
            const int row = g + ci * NWG;
            if (row < NBM) {
                const Real* w = acc[0][ci];
#pragma unroll
                for (int l = 0; l < DIM; ++l) {
                    const Real ax = ac[3 * l], ay = ac[3 * l + 1], az = ac[3 * l + 2];
                    const Real v[6] = {az * w[4] - ay * w[5], ax * w[5] - az * w[3], ay * w[3] - ax * w[4],
                                       ay * w[2] - az * w[1], az * w[0] - ax * w[2], ax * w[1] - ay * w[0]};
#pragma unroll
                    for (int f = 0; f < 6; ++f) {
                        const int o = tc_off<Sh::TK>(k0 * 6 + f, l * NBM + row);
                        const float h = __uint_as_float(tf32_bits(v[f]));
                        c.sWh[o] = h;
                        c.sWl[o] = v[f] - h;   // exact; the MMA reads its top 19 bits
                    }
                }
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < EP; ++e) {
            if (e == 1 && kk1 < 0) break;
            Real* out = c.sW + kk[e] * WSZ;
#pragma unroll
            for (int ci = 0; ci < AP; ++ci) {
                const int row = g + ci * NWG;
                if (row < NBM) {
#pragma unroll
                    for (int s = 0; s < NF; ++s) out[s * NBMP + row] = acc[e][ci][s];
                }
            }
        }
    }
}

// (b1) facet traces of U on the facets containing V: one thread per (element, two facet
// modes), all DIM facets, so every 16-byte read of U feeds DIM x 2 x W FMAs; with the
// factored volume term (sW set) the same phase computes W = M_j U on the threads that the
// last round of trace items leaves idle
template <typename Real, int DIM, int P>
__device__ void tent_traces(TentCtx<Real, DIM, P>& c, const KArgs& a, const Real* Ucur, Real* tr) {
    // W = M_j U (or the tcgen05 W operand built from it) on the threads the trace items leave idle
    if (c.sW || Shape<DIM, P>::TC5) {
        constexpr int NT = Shape<DIM, P>::NT;
        const int nitems = ((sizeof(Real) == 4 && Shape<DIM, P>::PAIRS) ? *c.sNpair : c.ns) * Shape<DIM, P>::NWG;
        const int busy = (c.ns * Shape<DIM, P>::NCG) % NT, idle = NT - busy;
        if ((int)threadIdx.x >= busy)
            for (int w = threadIdx.x - busy; w < nitems; w += idle) tent_w_item(c, a, Ucur, w);
    }
    using Sh = Shape<DIM, P>;
    using VT = typename Vec<Real>::T;
    constexpr int NF = Sh::NF, NFB = Sh::NFB, NT = Sh::NT, NBP = Sh::NBP, NFBP = Sh::NFBP;
    constexpr int AP = Sh::AP, NCG = Sh::NCG, W = Vec<Real>::W, ESZ = NF * NBP, TSZ = Strides<Real, DIM, P>::TSZ, FSZ = Strides<Real, DIM, P>::FSZ;
    constexpr int TMAT = NBP * AP * NCG;   // one thread-major facet table
    const Real* Tr = (const Real*)a.Trc;
    for (int idx = threadIdx.x; idx < c.ns * NCG; idx += NT) {
        const int k = idx / NCG;
        const int cg = idx - k * NCG;     // facet modes cg and cg + NCG
        const bool two = cg + NCG < NFB;
        const int j = c.sJ[k];
        const Real* U = Ucur + k * ESZ;
        const Real* T[DIM];
#pragma unroll
        for (int fi = 0; fi < DIM; ++fi) {
            const int f = fi + (fi >= j ? 1 : 0);
            T[fi] = Tr + (size_t)f * TMAT + cg * W;
        }
        Real acc[DIM][AP][NF];
#pragma unroll
        for (int fi = 0; fi < DIM; ++fi)
#pragma unroll
            for (int ci = 0; ci < AP; ++ci)
#pragma unroll
                for (int s = 0; s < NF; ++s) acc[fi][ci][s] = 0;
        // column block [b, b + W) for the first row only (NR = 1) or both rows (NR = 2)
        auto block = [&](int b, auto nr) {
            constexpr int NR = decltype(nr)::value;
            Real tv[DIM][AP][W];
#pragma unroll
            for (int fi = 0; fi < DIM; ++fi)
#pragma unroll
                for (int ci = 0; ci < NR; ++ci)
                    Vec<Real>::get(__ldg((const VT*)(T[fi] + b * AP * NCG + ci * NCG * W)), tv[fi][ci]);
#pragma unroll
            for (int s = 0; s < NF; ++s) {
                Real u[W];
                Vec<Real>::get(*(const VT*)(U + s * NBP + b), u);
#pragma unroll
                for (int v = 0; v < W; ++v)
#pragma unroll
                    for (int fi = 0; fi < DIM; ++fi)
#pragma unroll
                        for (int ci = 0; ci < NR; ++ci) acc[fi][ci][s] += tv[fi][ci][v] * u[v];
            }
        };
        if constexpr (AP == 1) {
#pragma unroll 1
            for (int b = 0; b < NBP; b += W) block(b, std::integral_constant<int, 1>{});
        } else {
            constexpr int BT = Sh::TLO / W * W;   // second rows vanish on the blocks below
#pragma unroll 1
            for (int b = 0; b < BT; b += W) block(b, std::integral_constant<int, 1>{});
#pragma unroll 1
            for (int b = BT; b < NBP; b += W) block(b, std::integral_constant<int, 2>{});
        }
        const Real sc = c.sTrs[k];
#pragma unroll
        for (int fi = 0; fi < DIM; ++fi) {
            Real* out = tr + k * TSZ + fi * FSZ + cg;
#pragma unroll
            for (int s = 0; s < NF; ++s) {
                out[s * NFBP] = acc[fi][0][s] * sc;
                if constexpr (AP == 2)
                    if (two) out[s * NFBP + NCG] = acc[fi][AP - 1][s] * sc;
            }
        }
    }
}

// (b2) numerical flux, once per facet (lower slot owns an interior facet), in place in tr,
// pre-scaled by each side's lift factor dt (d-1)!|F| / sqrt|det J|; one thread per (facet,
// facet mode)
template <typename Real, int DIM, int P>
__device__ void tent_fluxes(TentCtx<Real, DIM, P>& c, Real* tr) {
    using Sh = Shape<DIM, P>;
    constexpr int NF = Sh::NF, NFB = Sh::NFB, NFBP = Sh::NFBP, TSZ = Strides<Real, DIM, P>::TSZ, FSZ = Strides<Real, DIM, P>::FSZ;
    const int nown = *c.sNown;
    const int nitems = nown * NFB;
    for (int idx = threadIdx.x; idx < nitems; idx += blockDim.x) {
        const int oi = idx / NFB, cc = idx - oi * NFB;
        const int k = c.sOwn[2 * oi], fi = c.sOwn[2 * oi + 1];
        const int s2 = c.sNslot[k * DIM + fi];
        Real* mine = tr + k * TSZ + fi * FSZ + cc;
        Real um[6] = {0, 0, 0, 0, 0, 0}, up[6] = {0, 0, 0, 0, 0, 0}, F[6], nrm[3];
#pragma unroll
        for (int s = 0; s < NF; ++s) um[field6<DIM>(s)] = mine[s * NFBP];
        Real* other = nullptr;
        if (s2 >= 0) {
            other = tr + s2 * TSZ + c.sNfi[k * DIM + fi] * FSZ + cc;
#pragma unroll
            for (int s = 0; s < NF; ++s) up[field6<DIM>(s)] = other[s * NFBP];
        } else {
#pragma unroll
            for (int s = 0; s < 6; ++s) up[s] = s < 3 ? -um[s] : um[s];
        }
        for (int q = 0; q < 3; ++q) nrm[q] = c.sNrm[(k * DIM + fi) * 3 + q];
        upwind6<Real>(um, up, nrm, c.sZ[k * (1 + DIM)], c.sZ[k * (1 + DIM) + 1 + fi], F);
        const Real lc = c.sLiftc[k * DIM + fi];
#pragma unroll
        for (int s = 0; s < NF; ++s) mine[s * NFBP] = lc * F[field6<DIM>(s)];
        if (other) {
            const Real lc2 = c.sLiftc[s2 * DIM + c.sNfi[k * DIM + fi]];
#pragma unroll
            for (int s = 0; s < NF; ++s) other[s * NFBP] = -lc2 * F[field6<DIM>(s)];
        }
    }
}

// (b3)+(c) Y_{i,n} = A U_{i,n-1} (volume + lift of the scaled fluxes in tr), Taylor
// accumulation into sY, and U_{i,n} = G_i^-1 (Y_{i,n} - n M' U_{i,n-1}) into Unext (n < q).
// One thread per (pair of elements with the same local index j, two basis functions): every
// 16-byte read of the j-dependent tables S and L feeds both elements.
// EPI 0: SAT (Taylor accumulation and the next U); 1: SAT with the split accumulator;
// 2: RK4 stage on d/dt Y = A M^-1 Y: K = A U, Y += rk_w K, and (rk_c > 0) the next stage input
// Unext = Y_start + rk_c K (a Y-space value; the caller solves for U)
template <typename Real, int DIM, int P, int EPI = 0>
__device__ void tent_stage(TentCtx<Real, DIM, P>& c, const KArgs& a, int n, const Real* Ucur, Real* Unext,
                           const Real* tr, Real rk_w = 0, Real rk_c = 0) {
    constexpr bool SPLIT = EPI == 1;
    using Sh = Shape<DIM, P>;
    using VT = typename Vec<Real>::T;
    constexpr int NF = Sh::NF, NB = Sh::NB, NV = Sh::NV, NT = Sh::NT, NBP = Sh::NBP, NFBP = Sh::NFBP;
    constexpr int AP = Sh::AP, NAG = Sh::NAG, W = Vec<Real>::W, ESZ = NF * NBP, TSZ = Strides<Real, DIM, P>::TSZ, FSZ = Strides<Real, DIM, P>::FSZ;
    constexpr int EP = (sizeof(Real) == 4 && Sh::PAIRS) ? 2 : 1;   // elements per item (FP64: register budget)
    constexpr int NBMP = Sh::NBMP, WSZ = NF * NBMP;
    constexpr int DMAT = NBMP * AP * NAG, LMAT = NFBP * AP * NAG;   // thread-major D^T and L matrices
    const Real* Lf = (const Real*)a.Lc;
    const Real cn = (Real)a.taylor[n];
    const Real nn = (Real)n;
    const int nitems = EP == 2 ? *c.sNpair : c.ns;   // pairs, or single elements
    for (int idx = threadIdx.x; idx < nitems * NAG; idx += NT) {
        const int pi = idx / NAG, ag = idx - pi * NAG;   // basis functions ag and ag + NAG
        const bool two = ag + NAG < NB;
        const int k0 = EP == 2 ? c.sPair[2 * pi] : pi;
        const int kk1 = EP == 2 ? c.sPair[2 * pi + 1] : -1;
        const bool has1 = kk1 >= 0;
        int kk[2] = {k0, has1 ? kk1 : k0};
        const int j = c.sJ[k0];
        Real Yn[EP][AP][NF];
        if constexpr (Sh::TC5) {   // volume term from the tcgen05 accumulators
#pragma unroll
            for (int ai = 0; ai < AP; ++ai)
#pragma unroll
                for (int s = 0; s < NF; ++s)
                    Yn[0][ai][s] = (ai == 0 || two) ? c.sVol[(k0 * NF + s) * Sh::VS + ag + ai * NAG] : Real(0);
        } else {
            const Real* Dg = (const Real*)a.Dc + ag * W;
            Real Pm[EP][AP][DIM][NF];
#pragma unroll
            for (int e = 0; e < EP; ++e)
#pragma unroll
                for (int ai = 0; ai < AP; ++ai)
#pragma unroll
                    for (int l = 0; l < DIM; ++l)
#pragma unroll
                        for (int s = 0; s < NF; ++s) Pm[e][ai][l][s] = 0;
            // P_l = D_l^T W (factored volume, W = M_j U from phase b1); the D tables do not
            // depend on j.  Column block [c, c + W) for both rows (A0 = 0) or the second only.
            auto block = [&](int cb, auto a0) {
                constexpr int A0 = decltype(a0)::value;
                Real dv[AP][DIM][W];
                const Real* Db = Dg + cb * AP * NAG;
#pragma unroll
                for (int l = 0; l < DIM; ++l)
#pragma unroll
                    for (int ai = A0; ai < AP; ++ai)
                        Vec<Real>::get(__ldg((const VT*)(Db + l * DMAT + ai * NAG * W)), dv[ai][l]);
#pragma unroll
                for (int e = 0; e < EP; ++e) {
                    const Real* Wv = c.sW + kk[e] * WSZ;
#pragma unroll
                    for (int s = 0; s < NF; ++s) {
                        Real u[W];
                        Vec<Real>::get(*(const VT*)(Wv + s * NBMP + cb), u);
#pragma unroll
                        for (int v = 0; v < W; ++v)
#pragma unroll
                            for (int ai = A0; ai < AP; ++ai)
#pragma unroll
                                for (int l = 0; l < DIM; ++l) Pm[e][ai][l][s] += dv[ai][l][v] * u[v];
                    }
                }
            };
            // first rows (degree <= DA1) need only columns c < CV1
            constexpr int BV0 = (Sh::CV1 + W - 1) / W * W;
            constexpr int BV = BV0 < NBMP ? BV0 : NBMP;
#pragma unroll 1
            for (int cb = 0; cb < BV; cb += W) block(cb, std::integral_constant<int, 0>{});
#pragma unroll 1
            for (int cb = BV; cb < NBMP; cb += W) block(cb, std::integral_constant<int, 1>{});
#pragma unroll
            for (int e = 0; e < EP; ++e) {
                const Real* ac = c.sAc + kk[e] * DIM * 3;
#pragma unroll
                for (int ai = 0; ai < AP; ++ai) {
                    if constexpr (DIM == 3) {
                        Real vE[3] = {0, 0, 0}, vH[3] = {0, 0, 0};
#pragma unroll
                        for (int l = 0; l < DIM; ++l) {
                            const Real ax = ac[3 * l], ay = ac[3 * l + 1], az = ac[3 * l + 2];
                            const Real* Pl = Pm[e][ai][l];
                            vE[0] -= ay * Pl[5] - az * Pl[4];   // -a x P_H
                            vE[1] -= az * Pl[3] - ax * Pl[5];
                            vE[2] -= ax * Pl[4] - ay * Pl[3];
                            vH[0] += ay * Pl[2] - az * Pl[1];   //  a x P_E
                            vH[1] += az * Pl[0] - ax * Pl[2];
                            vH[2] += ax * Pl[1] - ay * Pl[0];
                        }
#pragma unroll
                        for (int q = 0; q < 3; ++q) { Yn[e][ai][q] = vE[q]; Yn[e][ai][3 + q] = vH[q]; }
                    } else {
                        Real ex = 0, ey = 0, hz = 0;
#pragma unroll
                        for (int l = 0; l < DIM; ++l) {
                            const Real ax = ac[3 * l], ay = ac[3 * l + 1];
                            const Real* Pl = Pm[e][ai][l];
                            ex -= ay * Pl[2];
                            ey += ax * Pl[2];
                            hz += ax * Pl[1] - ay * Pl[0];
                        }
                        Yn[e][ai][0] = ex; Yn[e][ai][1] = ey; Yn[e][ai][2] = hz;
                    }
                }
            }
        }
        // lift of the (already scaled) facet fluxes; the facet of local index f is the same for
        // both elements (same j)
#pragma unroll
        for (int fi = 0; fi < DIM; ++fi) {
            const int f = fi + (fi >= j ? 1 : 0);
            const Real* Lg = Lf + ((size_t)j * NV + f) * LMAT + ag * W;
            Real acc[EP][AP][NF];
#pragma unroll
            for (int e = 0; e < EP; ++e)
#pragma unroll
                for (int ai = 0; ai < AP; ++ai)
#pragma unroll
                    for (int s = 0; s < NF; ++s) acc[e][ai][s] = 0;
#pragma unroll
            for (int cc = 0; cc < NFBP; cc += W) {
                Real lv[AP][W];
#pragma unroll
                for (int ai = 0; ai < AP; ++ai)
                    Vec<Real>::get(__ldg((const VT*)(Lg + cc * AP * NAG + ai * NAG * W)), lv[ai]);
#pragma unroll
                for (int e = 0; e < EP; ++e) {
                    const Real* Fx = tr + kk[e] * TSZ + fi * FSZ;
#pragma unroll
                    for (int s = 0; s < NF; ++s) {
                        Real fv[W];
                        Vec<Real>::get(*(const VT*)(Fx + s * NFBP + cc), fv);
#pragma unroll
                        for (int v = 0; v < W; ++v)
#pragma unroll
                            for (int ai = 0; ai < AP; ++ai) acc[e][ai][s] += lv[ai][v] * fv[v];
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < EP; ++e)
#pragma unroll
                for (int ai = 0; ai < AP; ++ai)
#pragma unroll
                    for (int s = 0; s < NF; ++s) Yn[e][ai][s] -= acc[e][ai][s];
        }
#pragma unroll
        for (int e = 0; e < EP; ++e) {
            if (e == 1 && !has1) break;
            const int k = kk[e];
            const Real* U = Ucur + k * ESZ;
            const Real* gd = c.sGd + 3 * k;
            const Real* Gi = c.sGi + k * Strides<Real, DIM, P>::GSZ;
#pragma unroll
            for (int ai = 0; ai < AP; ++ai) {
                if (ai == 1 && !two) break;
                const int av = ag + ai * NAG;
                if constexpr (EPI == 2) {
#pragma unroll
                    for (int s = 0; s < NF; ++s) {
                        const int i = k * ESZ + s * NBP + av;
                        c.sY[i] += rk_w * Yn[e][ai][s];
                        if (rk_c != Real(0)) Unext[i] = c.sY0[i] + rk_c * Yn[e][ai][s];
                    }
                    continue;
                }
                if constexpr (SPLIT) {
#pragma unroll
                    for (int s = 0; s < NF; ++s) {   // (hi, lo) += cn Yn: two-sum, error into lo
                        const int i = k * ESZ + s * NBP + av;
                        Real hi, err;
                        two_sum(c.sY[i], mul_rn(cn, Yn[e][ai][s]), hi, err);
                        c.sY[i] = hi;
                        c.sYlo[i] += err;
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < NF; ++s) c.sY[k * ESZ + s * NBP + av] += cn * Yn[e][ai][s];
                }
                if (n < a.q) {
                    Real r6[NF];
                    if constexpr (DIM == 3) {
                        const Real E0 = U[0 * NBP + av], E1 = U[1 * NBP + av], E2 = U[2 * NBP + av];
                        const Real H0 = U[3 * NBP + av], H1 = U[4 * NBP + av], H2 = U[5 * NBP + av];
                        // M'U = [-H x gd ; E x gd]
                        r6[0] = Yn[e][ai][0] + nn * (H1 * gd[2] - H2 * gd[1]);
                        r6[1] = Yn[e][ai][1] + nn * (H2 * gd[0] - H0 * gd[2]);
                        r6[2] = Yn[e][ai][2] + nn * (H0 * gd[1] - H1 * gd[0]);
                        r6[3] = Yn[e][ai][3] - nn * (E1 * gd[2] - E2 * gd[1]);
                        r6[4] = Yn[e][ai][4] - nn * (E2 * gd[0] - E0 * gd[2]);
                        r6[5] = Yn[e][ai][5] - nn * (E0 * gd[1] - E1 * gd[0]);
                    } else {
                        const Real Ex = U[0 * NBP + av], Ey = U[1 * NBP + av], Hz = U[2 * NBP + av];
                        // M'U (TE) = (Hz gy, -Hz gx, Ex gy - Ey gx)
                        r6[0] = Yn[e][ai][0] - nn * (Hz * gd[1]);
                        r6[1] = Yn[e][ai][1] + nn * (Hz * gd[0]);
                        r6[2] = Yn[e][ai][2] - nn * (Ex * gd[1] - Ey * gd[0]);
                    }
#pragma unroll
                    for (int r = 0; r < NF; ++r) {
                        Real gr[Sh::GIS];
#pragma unroll
                        for (int q = 0; q < Sh::GIS; q += W) Vec<Real>::get(*(const VT*)(Gi + r * Sh::GIS + q), gr + q);
                        Real acc = 0;
#pragma unroll
                        for (int s = 0; s < NF; ++s) acc += gr[s] * r6[s];
                        Unext[k * ESZ + r * NBP + av] = acc;
                    }
                }
            }
        }
    }
}

// copy ns x ESZ coefficients between shared memory and a tape slot in global memory
template <typename Real, int DIM, int P>
__device__ void tent_copy(int ns, const Real* src, Real* dst) {
    constexpr int ESZ = Shape<DIM, P>::NF * Shape<DIM, P>::NBP;
    for (int idx = threadIdx.x; idx < ns * ESZ; idx += Shape<DIM, P>::NT) dst[idx] = src[idx];
}

// All m x q SAT stages of one tent on the shared-memory state sY.  With a tape, Y_{i,0}
// goes to slot i and U_{i,n} to slot m + i q + n (each slot max_patch x ESZ entries).
template <typename Real, int DIM, int P, int MODE>
__device__ void tent_traces_tc(TentCtx<Real, DIM, P>& c, const KArgs& a, const Real* Ucur, Real* tr);
template <typename Real, int DIM, int P, int MODE>
__device__ void tent_stage_tc(TentCtx<Real, DIM, P>& c, const KArgs& a, int n, const Real* Ucur, Real* Unext,
                              const Real* tr);

// Classical RK4 with m steps on the substituted tent ODE d/dt Y = A M(t)^-1 Y (Sec. 3, after
// eq. equ_ode): per step with start t0 and size h = 1/m, stages at t0, t0 + h/2, t0 + h/2, t0 + h
// with weights 1/6, 1/3, 1/3, 1/6; each stage solves U = M(t_s)^-1 Y_s and applies A.
template <typename Real, int DIM, int P>
__device__ void tent_rk4(TentCtx<Real, DIM, P>& c, const KArgs& a) {
    constexpr int ESZ = Shape<DIM, P>::NF * Shape<DIM, P>::NBP;
    const double h = 1.0 / (double)a.m;
    const double toff[4] = {0.0, 0.5, 0.5, 1.0}, wts[4] = {1.0 / 6, 1.0 / 3, 1.0 / 3, 1.0 / 6};
    const double cns[4] = {0.5, 0.5, 1.0, 0.0};
    Real* Ys = c.sUb;                                  // stage input (Y space)
    for (int i = 0; i < a.m; ++i) {
        for (int idx = threadIdx.x; idx < c.ns * ESZ; idx += blockDim.x) c.sY0[idx] = c.sY[idx];
        for (int st = 0; st < 4; ++st) {
            tent_ginv_at(c, a, ((double)i + toff[st]) * h, i == 0 && st == 0);
            __syncthreads();
            tent_apply_ginv(c, st == 0 ? c.sY0 : Ys, c.sUa);
            __syncthreads();
            tent_traces(c, a, c.sUa, c.sTr);
            __syncthreads();
            tent_fluxes(c, c.sTr);
            __syncthreads();
            tent_stage<Real, DIM, P, 2>(c, a, 1, c.sUa, Ys, c.sTr, (Real)(wts[st] * h), (Real)(cns[st] * h));
            __syncthreads();
        }
    }
}

template <typename Real, int DIM, int P, int MODE = 0>
__device__ void tent_sat(TentCtx<Real, DIM, P>& c, const KArgs& a, Real* tape) {
    if constexpr (ModeTraits<MODE>::rk4) {
        tent_rk4(c, a);
        return;
    }
    constexpr int ESZ = Shape<DIM, P>::NF * Shape<DIM, P>::NBP;
    const size_t slot = (size_t)a.max_patch * ESZ;
    if constexpr (Shape<DIM, P>::TC5) {
        // SIMT traces (+ W operand), fluxes and epilogue; the volume MMAs run on the tensor
        // cores while the fluxes are computed.  U is updated in place.
        Real* U = c.sUa;
        uint32_t ph = c.sTc[1];
        for (int i = 0; i < a.m; ++i) {
            tent_ginv(c, a, i);
            __syncthreads();
            tent_apply_ginv(c, c.sY, U);
            __syncthreads();
            for (int n = 1; n <= a.q; ++n) {
                tent_traces(c, a, U, c.sTr);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // W operand visible to the MMAs
                __syncthreads();
                if (threadIdx.x == 0) tc5_issue(c);
                tent_fluxes(c, c.sTr);
                tc5_collect(c, a, ph);
                ph ^= 1u;
                __syncthreads();
                tent_stage<Real, DIM, P, 0>(c, a, n, U, U, c.sTr);
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) c.sTc[1] = ph;
        return;
    } else if constexpr (ModeTraits<MODE>::simt) {
        // U is updated in place: the factored stage reads only its own rows of U
        Real* U = c.sUa;
        for (int i = 0; i < a.m; ++i) {
            tent_ginv(c, a, i);
            if (tape) tent_copy<Real, DIM, P>(c.ns, c.sY, tape + (size_t)i * slot);
            __syncthreads();
            tent_apply_ginv(c, c.sY, U);
            __syncthreads();
            for (int n = 1; n <= a.q; ++n) {
                if (tape) tent_copy<Real, DIM, P>(c.ns, U, tape + (size_t)(a.m + i * a.q + n - 1) * slot);
                tent_traces(c, a, U, c.sTr);
                __syncthreads();
                tent_fluxes(c, c.sTr);
                __syncthreads();
                tent_stage<Real, DIM, P, ModeTraits<MODE>::split ? 1 : 0>(c, a, n, U, U, c.sTr);
                __syncthreads();
            }
        }
    } else {
        for (int i = 0; i < a.m; ++i) {
            tent_ginv(c, a, i);
            if (tape) tent_copy<Real, DIM, P>(c.ns, c.sY, tape + (size_t)i * slot);
            __syncthreads();
            Real* Ucur = c.sUa;
            Real* Unext = c.sUb;
            tent_apply_ginv(c, c.sY, Ucur);
            __syncthreads();
            for (int n = 1; n <= a.q; ++n) {
                if (tape) tent_copy<Real, DIM, P>(c.ns, Ucur, tape + (size_t)(a.m + i * a.q + n - 1) * slot);
                tent_traces_tc<Real, DIM, P, MODE>(c, a, Ucur, c.sTr);
                __syncthreads();
                tent_fluxes(c, c.sTr);
                __syncthreads();
                tent_stage_tc<Real, DIM, P, MODE>(c, a, n, Ucur, Unext, c.sTr);
                __syncthreads();
                Real* tmp = Ucur; Ucur = Unext; Unext = tmp;
            }
        }
    }
}

template <typename Real, int DIM, int P, int MODE = 0>
__global__ void __launch_bounds__(Shape<DIM, P>::NT, MinBlocks<Real, DIM, P>::value) tent_layer_kernel(const KArgs a, int64_t t0) {
    using Sh = Shape<DIM, P>;
    constexpr int NF = Sh::NF, NB = Sh::NB, NT = Sh::NT, NBP = Sh::NBP, ESZ = NF * NBP;
    using StateT = StateOf<Real, MODE>;
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemLayout<Real, DIM, P> lay(a.max_patch, MODE);
    TentCtx<Real, DIM, P> c;
    c.carve(smem, lay);
    const int64_t tent = t0 + blockIdx.x;
    StateT* state = (StateT*)a.state + (int64_t)blockIdx.y * a.rhs_stride;
    if constexpr (Sh::TC5) tc5_begin(c, a);
    tent_setup(c, a, tent, state);
    tent_sat<Real, DIM, P, MODE>(c, a, (Real*)nullptr);
    if constexpr (Sh::TC5) tc5_end(c);
    // ---- (d) scatter the tent-top Y; advance the front at V ----
    bool bad = false;
    for (int idx = threadIdx.x; idx < c.ns * NF * NB; idx += NT) {
        const int k = idx / (NF * NB), r = idx - k * NF * NB, s = r / NB, b = r - s * NB;
        StateT v = c.sY[k * ESZ + s * NBP + b];
        if constexpr (ModeTraits<MODE>::split) v += (StateT)c.sYlo[k * ESZ + s * NBP + b];
        if (!isfinite((double)v)) bad = true;
        state[(int64_t)a.patch_elem[c.pb + k] * NF * NB + r] = v;
    }
    if (bad) atomicCAS(a.err, 0, 2);
    if (threadIdx.x == 0 && blockIdx.y == 0) a.tau[c.V] = a.tent_tt[tent];
}

// Persistent evolve over the whole tent DAG: CTAs pull tents in (layer, vertex) order from a
// ticket counter; tent s at V waits until every vertex U of {V} u N(V) has completed all its
// tents of earlier layers (cnt[U] >= number of U's tents with layer < layer(s), found by binary
// search in U's sorted tent layers), runs all right-hand sides, then publishes cnt[V] += 1.
// Tickets are only taken by running CTAs and dependencies have smaller tickets, so progress
// never depends on CTA residency.  Every wait is bounded (globaltimer deadline); on expiry, or
// when another CTA has already failed, the CTA sets the error word and stops.
struct PArgs {
    int64_t n_tents;               // tickets: tents ticket0 .. ticket0 + n_tents - 1
    int64_t ticket0;
    unsigned long long* next;      // ticket counter
    int* cnt;                      // completed tents per vertex
    const int64_t* vt_ptr;         // tents of vertex U: layers vt_layer[vt_ptr[U] .. vt_ptr[U+1])
    const int32_t* vt_layer;
    const int64_t* adj_ptr;        // neighbours of U: adj[adj_ptr[U] .. adj_ptr[U+1])
    const int32_t* adj;
    const int32_t* tent_layer;
    long long timeout_ns;
    int n_rhs;
    int withhold_first;            // failure injection: never publish ticket 0's completion
};

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long globaltimer() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One DAG-walk step for ticket `tent` of an instance: bounded wait on the closed neighbourhood,
// all right-hand sides, publish.  Returns false when the CTA must stop (error / timeout).
template <typename Real, int DIM, int P, int MODE = 0>
__device__ bool tent_dag_step(unsigned char* smem, const KArgs& a, const PArgs& pa, int64_t tent, int* s_abort) {
    using Sh = Shape<DIM, P>;
    using StateT = StateOf<Real, MODE>;
    constexpr int NF = Sh::NF, NB = Sh::NB, NT = Sh::NT, NBP = Sh::NBP, ESZ = NF * NBP;
    const SmemLayout<Real, DIM, P> lay(a.max_patch, MODE);
    TentCtx<Real, DIM, P> c;
    c.carve(smem, lay);
    const int V = a.tent_v[tent];
    const int L = pa.tent_layer[tent];
    const int64_t a0 = pa.adj_ptr[V], deg = pa.adj_ptr[V + 1] - a0;
    for (int u = threadIdx.x; u <= deg; u += NT) {
        const int U = u == 0 ? V : pa.adj[a0 + u - 1];
        int64_t lo = pa.vt_ptr[U], hi = pa.vt_ptr[U + 1];
        const int64_t base = lo;
        while (lo < hi) {                      // first tent of U with layer >= L
            const int64_t mid = (lo + hi) / 2;
            if (pa.vt_layer[mid] < L) lo = mid + 1; else hi = mid;
        }
        const int need = (int)(lo - base);
        if (load_acquire(pa.cnt + U) < need) {
            const long long deadline = globaltimer() + pa.timeout_ns;
            while (load_acquire(pa.cnt + U) < need) {
                if (*(volatile int*)a.err != 0 || globaltimer() > deadline) {
                    atomicCAS(a.err, 0, 3);
                    *s_abort = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
    }
    __syncthreads();
    if (*s_abort) return false;
    for (int r = 0; r < pa.n_rhs; ++r) {
        StateT* state = (StateT*)a.state + (int64_t)r * a.rhs_stride;
        tent_setup<Real, DIM, P, true>(c, a, tent, state);
        tent_sat<Real, DIM, P, MODE>(c, a, (Real*)nullptr);
        bool bad = false;
        for (int idx = threadIdx.x; idx < c.ns * NF * NB; idx += NT) {
            const int k = idx / (NF * NB), rr = idx - k * NF * NB, s = rr / NB, b = rr - s * NB;
            StateT v = c.sY[k * ESZ + s * NBP + b];
            if constexpr (ModeTraits<MODE>::split) v += (StateT)c.sYlo[k * ESZ + s * NBP + b];
            if (!isfinite((double)v)) bad = true;
            state[(int64_t)a.patch_elem[c.pb + k] * NF * NB + rr] = v;
        }
        if (bad) atomicCAS(a.err, 0, 2);
        __threadfence();                       // publish this thread's state writes (gpu scope)
        __syncthreads();
    }
    if (threadIdx.x == 0 && !(pa.withhold_first && tent == pa.ticket0)) {
        a.tau[V] = a.tent_tt[tent];
        __threadfence();
        atomicAdd(pa.cnt + V, 1);
    }
    __syncthreads();
    return true;
}

template <typename Real, int DIM, int P, int MODE = 0>
__global__ void __launch_bounds__(Shape<DIM, P>::NT, MinBlocks<Real, DIM, P>::value)
    tent_persistent_kernel(const KArgs a, const PArgs pa) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_ticket;
    __shared__ int s_abort;
    TentCtx<Real, DIM, P> tc;
    if constexpr (Shape<DIM, P>::TC5) {
        tc.carve(smem, SmemLayout<Real, DIM, P>(a.max_patch, MODE));
        tc5_begin(tc, a);
    }
    while (true) {
        if (threadIdx.x == 0) {
            s_ticket = (long long)atomicAdd(pa.next, 1ull);
            s_abort = 0;
        }
        __syncthreads();
        const long long ticket = s_ticket;
        if (ticket >= pa.n_tents) break;
        if (!tent_dag_step<Real, DIM, P, MODE>(smem, a, pa, pa.ticket0 + ticket, &s_abort)) break;
    }
    if constexpr (Shape<DIM, P>::TC5) tc5_end(tc);
}

// Many independent problems (meshes of any degree 1..5, same dimension and precision) in one
// persistent launch: tickets run over the merged tent lists ordered by (layer, instance,
// vertex); each ticket names its instance, whose KArgs / PArgs (own counters) live in global
// memory.  Instances never wait on each other.
struct BatchArgs {
    int64_t n_tickets;
    unsigned long long* next;
    const int32_t* ticket_inst;
    const int64_t* ticket_tent;
    const KArgs* kargs;
    const PArgs* pargs;
    const int32_t* inst_p;
};

template <typename Real, int DIM>
__global__ void __launch_bounds__(Shape<DIM, 4>::NT, sizeof(Real) == 4 ? 2 : 1) tent_batch_kernel(const BatchArgs b) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_ticket;
    __shared__ int s_abort;
    while (true) {
        if (threadIdx.x == 0) {
            s_ticket = (long long)atomicAdd(b.next, 1ull);
            s_abort = 0;
        }
        __syncthreads();
        const long long t = s_ticket;
        if (t >= b.n_tickets) break;
        const int inst = b.ticket_inst[t];
        const int64_t tent = b.ticket_tent[t];
        const KArgs& a = b.kargs[inst];      // per-instance arguments stay in global memory
        const PArgs& pa = b.pargs[inst];
        bool ok = true;
        switch (b.inst_p[inst]) {
            case 1: ok = tent_dag_step<Real, DIM, 1>(smem, a, pa, tent, &s_abort); break;
            case 2: ok = tent_dag_step<Real, DIM, 2>(smem, a, pa, tent, &s_abort); break;
            case 3: ok = tent_dag_step<Real, DIM, 3>(smem, a, pa, tent, &s_abort); break;
            case 4: ok = tent_dag_step<Real, DIM, 4>(smem, a, pa, tent, &s_abort); break;
            default: ok = tent_dag_step<Real, DIM, 5>(smem, a, pa, tent, &s_abort); break;
        }
        if (!ok) break;
    }
}

// ---------------------------------------------------------------------------------------
// Tensor-core contractions (warp-level m16n8k8 TF32 MMA, FP32 accumulate), 3D.  One warp
// owns a pair of elements with the same local index j (both share the A operands):
// N = 2 tiles of 8 columns (the 6 fields of each element), M over basis functions / facet
// modes, K over basis functions / facet modes.  Operands: A from the fragment-ordered tables
// (one 16-byte load per lane), B from the shared-memory state (converted to TF32).  The curl
// combination and the mass solve need all 6 fields of one coefficient, spread over the 3
// lanes of a quad: they are gathered with quad shuffles.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void mma_tf32(float d[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// B fragment (k8 x n8) from a row-major [n][k] source: rows n = g (< nrow), k = k0 + t, k0 + t + 4 (< kmax)
template <int MODE>
__device__ __forceinline__ void load_b(const float* row, bool valid, int k, int kmax, uint32_t hi[2], uint32_t lo[2]) {
    const float x0 = (valid && k < kmax) ? row[k] : 0.f;
    const float x1 = (valid && k + 4 < kmax) ? row[k + 4] : 0.f;
    hi[0] = to_tf32(x0);
    hi[1] = to_tf32(x1);
    if constexpr (MODE == 2) {
        lo[0] = to_tf32(x0 - __uint_as_float(hi[0]));
        lo[1] = to_tf32(x1 - __uint_as_float(hi[1]));
    }
}
template <int MODE>
__device__ __forceinline__ void mma_mode(float d[4], const float4& ah, const float4& al, const uint32_t bh[2],
                                         const uint32_t bl[2]) {
    const uint32_t a[4] = {__float_as_uint(ah.x), __float_as_uint(ah.y), __float_as_uint(ah.z), __float_as_uint(ah.w)};
    mma_tf32(d, a, bh);
    if constexpr (MODE == 2) {
        const uint32_t l[4] = {__float_as_uint(al.x), __float_as_uint(al.y), __float_as_uint(al.z),
                               __float_as_uint(al.w)};
        mma_tf32(d, a, bl);
        mma_tf32(d, l, bh);
    }
}

template <int P>
struct TcShape {
    static_assert(P <= 4, "tensor-core traces keep all facet modes in one m16 tile");
    static constexpr int NB = (P + 1) * (P + 2) * (P + 3) / 6;
    static constexpr int NFB = (P + 1) * (P + 2) / 2;
    static constexpr int MT = (NB + 15) / 16;      // m16 tiles over basis functions
    static constexpr int KT = (NB + 7) / 8;        // k8 steps over basis functions
    static constexpr int KTL = (NFB + 7) / 8;      // k8 steps over facet modes
};

template <typename Real, int DIM, int P, int MODE>
__device__ void tent_traces_tc(TentCtx<Real, DIM, P>& c, const KArgs& a, const Real* Ucur, Real* tr) {
    static_assert(DIM == 3 && sizeof(Real) == 4, "tensor-core path: 3D FP32 state");
    using Sh = Shape<DIM, P>;
    using Tc = TcShape<P>;
    constexpr int NF = Sh::NF, NB = Sh::NB, NFB = Sh::NFB, NBP = Sh::NBP, NFBP = Sh::NFBP;
    constexpr int ESZ = NF * NBP, TSZ = Strides<Real, DIM, P>::TSZ, FSZ = Strides<Real, DIM, P>::FSZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int npair = *c.sNpair;
    for (int item = warp; item < npair * DIM; item += nwarps) {
        const int pi = item / DIM, fi = item - pi * DIM;
        const int k0 = c.sPair[2 * pi], kk1 = c.sPair[2 * pi + 1];
        const int ke[2] = {k0, kk1 >= 0 ? kk1 : k0};
        const int j = c.sJ[k0];
        const int f = fi + (fi >= j ? 1 : 0);
        float acc[2][4] = {};
#pragma unroll
        for (int kt = 0; kt < Tc::KT; ++kt) {
            const float4 ah = __ldg(a.Trf + ((size_t)f * Tc::KT + kt) * 32 + lane);
            float4 al = ah;
            if constexpr (MODE == 2) al = __ldg(a.Trf_lo + ((size_t)f * Tc::KT + kt) * 32 + lane);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t bh[2], bl[2];
                load_b<MODE>(Ucur + ke[nt] * ESZ + g * NBP, g < NF, 8 * kt + t, NB, bh, bl);
                mma_mode<MODE>(acc[nt], ah, al, bh, bl);
            }
        }
        // acc[nt]: rows c = g (cols s = 2t, 2t+1), c = g + 8
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            if (nt == 1 && kk1 < 0) break;
            const int k = ke[nt];
            const Real sc = c.sTrs[k];
            Real* out = tr + k * TSZ + fi * FSZ;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = g + 8 * h;
                if (cc < NFB && t < 3) {
                    out[(2 * t) * NFBP + cc] = acc[nt][2 * h] * sc;
                    out[(2 * t + 1) * NFBP + cc] = acc[nt][2 * h + 1] * sc;
                }
            }
        }
    }
}

template <typename Real, int DIM, int P, int MODE>
__device__ void tent_stage_tc(TentCtx<Real, DIM, P>& c, const KArgs& a, int n, const Real* Ucur, Real* Unext,
                              const Real* tr) {
    static_assert(DIM == 3 && sizeof(Real) == 4, "tensor-core path: 3D FP32 state");
    using Sh = Shape<DIM, P>;
    using Tc = TcShape<P>;
    constexpr int NF = Sh::NF, NB = Sh::NB, NFB = Sh::NFB, NBP = Sh::NBP, NFBP = Sh::NFBP, NV = Sh::NV;
    constexpr int ESZ = NF * NBP, TSZ = Strides<Real, DIM, P>::TSZ, FSZ = Strides<Real, DIM, P>::FSZ;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const unsigned full = 0xffffffffu;
    const float cn = (float)a.taylor[n];
    const float nn = (float)n;
    const int npair = *c.sNpair;
    for (int item = warp; item < npair * Tc::MT; item += nwarps) {
        const int pi = item / Tc::MT, mt = item - pi * Tc::MT;
        const int k0 = c.sPair[2 * pi], kk1 = c.sPair[2 * pi + 1];
        const int ke[2] = {k0, kk1 >= 0 ? kk1 : k0};
        const int j = c.sJ[k0];
        // volume: P_l[a][(s, e)] = sum_b S_{j,l}[a][b] U_e[s][b]
        float Pv[3][2][4] = {};
#pragma unroll
        for (int kt = 0; kt < Tc::KT; ++kt) {
            uint32_t bh[2][2], bl[2][2];
#pragma unroll
            for (int nt = 0; nt < 2; ++nt)
                load_b<MODE>(Ucur + ke[nt] * ESZ + g * NBP, g < NF, 8 * kt + t, NB, bh[nt], bl[nt]);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                const size_t fr = (((size_t)j * 3 + l) * Tc::MT + mt) * Tc::KT + kt;
                const float4 ah = __ldg(a.Sf + fr * 32 + lane);
                float4 al = ah;
                if constexpr (MODE == 2) al = __ldg(a.Sf_lo + fr * 32 + lane);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) mma_mode<MODE>(Pv[l][nt], ah, al, bh[nt], bl[nt]);
            }
        }
        // lift: Lc[a][(r, e)] = sum_{fi, c} L_{j,f}[a][c] F_e[fi][r][c]
        float Lc[2][4] = {};
#pragma unroll
        for (int fi = 0; fi < DIM; ++fi) {
            const int f = fi + (fi >= j ? 1 : 0);
#pragma unroll
            for (int kt = 0; kt < Tc::KTL; ++kt) {
                const size_t fr = (((size_t)j * NV + f) * Tc::MT + mt) * Tc::KTL + kt;
                const float4 ah = __ldg(a.Lfr + fr * 32 + lane);
                float4 al = ah;
                if constexpr (MODE == 2) al = __ldg(a.Lfr_lo + fr * 32 + lane);
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t bh[2], bl[2];
                    load_b<MODE>(tr + ke[nt] * TSZ + fi * FSZ + g * NFBP, g < NF, 8 * kt + t, NFB, bh, bl);
                    mma_mode<MODE>(Lc[nt], ah, al, bh, bl);
                }
            }
        }
        // per element and row half: curl combination, Taylor accumulation, mass solve
        const int src0 = lane & ~3;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int k = ke[nt];
            const float* ac = c.sAc + k * DIM * 3;
            const float* U = Ucur + k * ESZ;
            const float* gd = c.sGd + 3 * k;
            const float* Gi = c.sGi + k * Strides<Real, DIM, P>::GSZ;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int av = 16 * mt + g + 8 * h;
                float Pf[3][6];
#pragma unroll
                for (int l = 0; l < 3; ++l)
#pragma unroll
                    for (int u = 0; u < 3; ++u) {
                        Pf[l][2 * u] = __shfl_sync(full, Pv[l][nt][2 * h], src0 + u);
                        Pf[l][2 * u + 1] = __shfl_sync(full, Pv[l][nt][2 * h + 1], src0 + u);
                    }
                float Yf[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    const float ax = ac[3 * l], ay = ac[3 * l + 1], az = ac[3 * l + 2];
                    const float* Pl = Pf[l];
                    Yf[0] -= ay * Pl[5] - az * Pl[4];   // -a x P_H
                    Yf[1] -= az * Pl[3] - ax * Pl[5];
                    Yf[2] -= ax * Pl[4] - ay * Pl[3];
                    Yf[3] += ay * Pl[2] - az * Pl[1];   //  a x P_E
                    Yf[4] += az * Pl[0] - ax * Pl[2];
                    Yf[5] += ax * Pl[1] - ay * Pl[0];
                }
                // subtract the lift: this lane holds columns r = 2t, 2t+1
                float y0 = (t < 3 ? Yf[2 * t] : 0.f) - Lc[nt][2 * h];
                float y1 = (t < 3 ? Yf[2 * t + 1] : 0.f) - Lc[nt][2 * h + 1];
                float Yn[6];
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    Yn[2 * u] = __shfl_sync(full, y0, src0 + u);
                    Yn[2 * u + 1] = __shfl_sync(full, y1, src0 + u);
                }
                const bool own = (nt == 0 || kk1 >= 0) && av < NB && t < 3;
                if (own) {
                    float* Y = c.sY + k * ESZ + av;
                    Y[(2 * t) * NBP] += cn * y0;
                    Y[(2 * t + 1) * NBP] += cn * y1;
                    if (n < a.q) {
                        const float E0 = U[0 * NBP + av], E1 = U[1 * NBP + av], E2 = U[2 * NBP + av];
                        const float H0 = U[3 * NBP + av], H1 = U[4 * NBP + av], H2 = U[5 * NBP + av];
                        float r6[6];
                        r6[0] = Yn[0] + nn * (H1 * gd[2] - H2 * gd[1]);
                        r6[1] = Yn[1] + nn * (H2 * gd[0] - H0 * gd[2]);
                        r6[2] = Yn[2] + nn * (H0 * gd[1] - H1 * gd[0]);
                        r6[3] = Yn[3] - nn * (E1 * gd[2] - E2 * gd[1]);
                        r6[4] = Yn[4] - nn * (E2 * gd[0] - E0 * gd[2]);
                        r6[5] = Yn[5] - nn * (E0 * gd[1] - E1 * gd[0]);
#pragma unroll
                        for (int q = 0; q < 2; ++q) {
                            const int r = 2 * t + q;
                            float acc = 0;
#pragma unroll
                            for (int s = 0; s < 6; ++s) acc += Gi[r * Sh::GIS + s] * r6[s];
                            Unext[k * ESZ + r * NBP + av] = acc;
                        }
                    }
                }
            }
        }
    }
}

}  // namespace mtp
