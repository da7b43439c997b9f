// Device-side management of the MTP library: uploads, lattice exchange, energy,
// and the layer-by-layer evolution driver (layers replayed from a CUDA graph).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mtp_adjoint.cuh"
#include "mtp_internal.h"
#include "mtp_launch.cuh"

namespace mtp {

#define CUDA_TRY(call)                                                                       \
    do {                                                                                     \
        cudaError_t _e = (call);                                                             \
        if (_e != cudaSuccess)                                                               \
            return set_error(_e == cudaErrorMemoryAllocation ? MTP_ENOMEM : MTP_ECUDA,       \
                             std::string(#call) + ": " + cudaGetErrorString(_e));            \
    } while (0)

struct DeviceMesh {
    int device = -1;
    double* geo = nullptr;
    int32_t* elems = nullptr;
    int64_t* patch_ptr = nullptr;
    int32_t* patch_elem = nullptr;
    int8_t* patch_info = nullptr;
    void* S = nullptr;
    void* Tr = nullptr;
    void* L = nullptr;
    void* Mc = nullptr;           // thread-major copies of M, D^T, Tr, L for the SIMT tent kernels
    void* Dc = nullptr;
    void* Trc = nullptr;
    void* Lc = nullptr;
    void* Mc1 = nullptr;          // the same four tables with one row per thread (shape variant 2)
    void* Dc1 = nullptr;
    void* Trc1 = nullptr;
    void* Lc1 = nullptr;
    double* V = nullptr;
    double* Vinv = nullptr;
    float* Sf = nullptr;          // tensor-core fragment tables (TF32 modes)
    float* Lfr = nullptr;
    float* Trf = nullptr;
    float* Sf_lo = nullptr;
    float* Lfr_lo = nullptr;
    float* Trf_lo = nullptr;
    float* Dtc = nullptr;         // tcgen05 A operand (variants 3, 4): D^T in core-matrix layout, hi then lo
    double* partial = nullptr;    // energy reduction scratch: [n_rhs][kEnergyBlocks] partials, then [n_rhs] sums
};

struct DeviceTents {
    int32_t* v = nullptr;
    double* tb = nullptr;
    double* tt = nullptr;
    double* tau = nullptr;
    int* err = nullptr;
    int* err_host = nullptr;      // pinned
    void* host_state = nullptr;   // device buffer for mtp_evolve_host
    cudaStream_t capture = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* graph_state = nullptr;  // state pointer baked into the graph
    // persistent DAG walk
    int32_t* tent_layer = nullptr;
    int64_t* vt_ptr = nullptr;
    int32_t* vt_layer = nullptr;
    int64_t* adj_ptr = nullptr;
    int32_t* adj = nullptr;
    int* cnt = nullptr;
    unsigned long long* next = nullptr;
    // adjoint work buffers (grown on demand)
    void* adj_buf = nullptr;
    size_t adj_bytes = 0;
    double* tau_rev = nullptr;
    int64_t* tent_off = nullptr;   // [n_tents + 1]: patch entries of the tents before each tent
};

constexpr int kEnergyBlocks = 304;
constexpr int kEnergyThreads = 256;

// the state between tents is FP64 for MTP_FP64 and MTP_FP32_SPLIT, FP32 otherwise; the reference
// tables and the tent kernels' arithmetic are FP64 only for MTP_FP64
static bool state_f64(const Mesh& m) { return m.precision == MTP_FP64 || m.precision == MTP_FP32_SPLIT; }
static size_t real_size(const Mesh& m) { return state_f64(m) ? sizeof(double) : sizeof(float); }

template <typename T>
static int upload(T** dst, const T* src, size_t n) {
    CUDA_TRY(cudaMalloc((void**)dst, n * sizeof(T) + 16));
    CUDA_TRY(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return MTP_OK;
}

// rows of `cols` entries -> rows of pad4(cols) entries, zeros in the pad (16-byte vector reads)
static std::vector<double> pad_rows(const std::vector<double>& src, int cols) {
    const int pc = pad4(cols);
    const size_t rows = src.size() / cols;
    std::vector<double> out(rows * pc, 0.0);
    for (size_t r = 0; r < rows; ++r)
        for (int c = 0; c < cols; ++c) out[r * pc + c] = src[r * cols + c];
    return out;
}

// Thread-major layout of `nmat` row-major rows x cols matrices for the SIMT tent kernels.
// With nrg = ceil(rows / ap) row groups, a thread owns rows g, g + nrg, ..., and reads, per
// step, `w` consecutive columns of each of them as one 16-byte vector; consecutive threads
// own consecutive groups.  Entry (r, c) of matrix mt goes to
//   [mt][c / w][r / nrg][r % nrg][c % w]   (columns padded to pad4(cols), rows to ap * nrg)
// so that the vectors that the lanes of a warp read for one (matrix, column block, row of
// the group) are contiguous in memory, and the rows the lanes write are consecutive.
static std::vector<double> thread_major(const std::vector<double>& src, int nmat, int rows, int cols, int w,
                                        int ap) {
    const int nch = pad4(cols) / w, nrg = (rows + ap - 1) / ap;
    const size_t msz = (size_t)nch * ap * nrg * w;
    std::vector<double> out(nmat * msz, 0.0);
    for (int mt = 0; mt < nmat; ++mt)
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c)
                out[mt * msz + (((size_t)(c / w) * ap + r / nrg) * nrg + r % nrg) * w + c % w] =
                    src[((size_t)mt * rows + r) * cols + c];
    return out;
}

static int upload_real(const Mesh& m, void** dst, const std::vector<double>& src) {
    if (m.precision == MTP_FP64) return upload((double**)dst, src.data(), src.size());   // FP32 arithmetic otherwise
    std::vector<float> f(src.begin(), src.end());
    return upload((float**)dst, f.data(), f.size());
}

#define MTP_TRY(call)                  \
    do {                               \
        int _rc = (call);              \
        if (_rc != MTP_OK) return _rc; \
    } while (0)

// A-operand tables in m16n8k8 fragment order: fragment (mt, kt) of a row-major M x K matrix
// A (zero outside rows < rows, cols < cols) is 32 lanes x 4 values: lane (g = lane/4,
// t = lane%4) holds A[16mt+g][8kt+t], A[16mt+g+8][8kt+t], A[16mt+g][8kt+t+4], A[16mt+g+8][8kt+t+4].
// Values are TF32-rounded (round to nearest even at 10 mantissa bits); `lo` receives the
// TF32-rounded remainder for the split mode.
static float tf32_round(float x) {
    uint32_t u;
    std::memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) != 0x7f800000u) u += 0xfffu + ((u >> 13) & 1u);
    u &= 0xffffe000u;
    std::memcpy(&x, &u, 4);
    return x;
}
template <typename Get>
static void append_fragments(std::vector<float>& hi, std::vector<float>& lo, int MT, int KT, Get A) {
    for (int mt = 0; mt < MT; ++mt)
        for (int kt = 0; kt < KT; ++kt)
            for (int lane = 0; lane < 32; ++lane) {
                const int g = lane >> 2, t = lane & 3;
                const double v[4] = {A(16 * mt + g, 8 * kt + t), A(16 * mt + g + 8, 8 * kt + t),
                                     A(16 * mt + g, 8 * kt + t + 4), A(16 * mt + g + 8, 8 * kt + t + 4)};
                for (int q = 0; q < 4; ++q) {
                    const float h = tf32_round((float)v[q]);
                    hi.push_back(h);
                    lo.push_back(tf32_round((float)(v[q] - (double)h)));
                }
            }
}

int device_mesh_upload(Mesh& m) {
    int dev;
    CUDA_TRY(cudaGetDevice(&dev));
    if (m.dev) {
        if (m.dev->device == dev) return MTP_OK;
        return set_error(MTP_EINVAL, "mesh was uploaded to another device");
    }
    m.dev = new DeviceMesh();
    DeviceMesh& d = *m.dev;
    d.device = dev;
    MTP_TRY(upload(&d.geo, m.geo.data(), m.geo.size()));
    MTP_TRY(upload(&d.elems, m.elems.data(), m.elems.size()));
    MTP_TRY(upload(&d.patch_ptr, m.patch_ptr.data(), m.patch_ptr.size()));
    MTP_TRY(upload(&d.patch_elem, m.patch_elem.data(), m.patch_elem.size()));
    MTP_TRY(upload(&d.patch_info, m.patch_info.data(), m.patch_info.size()));
    MTP_TRY(upload_real(m, &d.S, pad_rows(m.ref.S, m.nb)));     // [j][l][a][NBP]
    MTP_TRY(upload_real(m, &d.Tr, pad_rows(m.ref.Tr, m.nb)));   // [f][c][NBP]
    MTP_TRY(upload_real(m, &d.L, pad_rows(m.ref.L, m.nfb)));    // [j][f][a][NFBP]
    {
        const int w = m.precision == MTP_FP64 ? 2 : 4, ap = 2, nv = m.dim + 1;
        // factored volume: M[j] (rows c < nbm, columns b) and D[l]^T (rows a, columns c < nbm)
        const int nbm = m.ref.nbm;
        std::vector<double> Dt((size_t)m.dim * m.nb * nbm);
        for (int l = 0; l < m.dim; ++l)
            for (int c = 0; c < nbm; ++c)
                for (int a = 0; a < m.nb; ++a)
                    Dt[((size_t)l * m.nb + a) * nbm + c] = m.ref.D[((size_t)l * nbm + c) * m.nb + a];
        MTP_TRY(upload_real(m, &d.Mc, thread_major(m.ref.M, nv, nbm, m.nb, w, ap)));
        MTP_TRY(upload_real(m, &d.Dc, thread_major(Dt, m.dim, m.nb, nbm, w, ap)));
        MTP_TRY(upload_real(m, &d.Trc, thread_major(m.ref.Tr, nv, m.nfb, m.nb, w, ap)));
        MTP_TRY(upload_real(m, &d.Lc, thread_major(m.ref.L, nv * nv, m.nb, m.nfb, w, ap)));
        if (m.precision == MTP_FP32 && m.dim == 3 && m.p >= 2 && m.p <= 4) {
            // A operand of the tcgen05 volume term: D[a][k], k = l nbm + c, = D_l^T[a][c], rows a
            // padded to tn = 64 (the MMA's M), k to tk = 8, K-major core matrices (8 rows x 4
            // values), 8-row groups tk x 8 floats apart; TF32 hi part, then the TF32 remainder
            const int tk = (3 * nbm + 7) / 8 * 8, tn = 64;
            std::vector<float> bt((size_t)2 * tn * tk, 0.0f);
            for (int a = 0; a < m.nb; ++a)
                for (int l = 0; l < 3; ++l)
                    for (int c = 0; c < nbm; ++c) {
                        const int k = l * nbm + c;
                        const size_t o = (size_t)(a >> 3) * tk * 8 + (k >> 2) * 32 + (a & 7) * 4 + (k & 3);
                        const double v = Dt[((size_t)l * m.nb + a) * nbm + c];
                        const float h = tf32_round((float)v);
                        bt[o] = h;
                        bt[(size_t)tn * tk + o] = tf32_round((float)(v - (double)h));
                    }
            MTP_TRY(upload(&d.Dtc, bt.data(), bt.size()));
        }
        if (m.precision == MTP_FP32) {
            MTP_TRY(upload_real(m, &d.Mc1, thread_major(m.ref.M, nv, nbm, m.nb, w, 1)));
            MTP_TRY(upload_real(m, &d.Dc1, thread_major(Dt, m.dim, m.nb, nbm, w, 1)));
            MTP_TRY(upload_real(m, &d.Trc1, thread_major(m.ref.Tr, nv, m.nfb, m.nb, w, 1)));
            MTP_TRY(upload_real(m, &d.Lc1, thread_major(m.ref.L, nv * nv, m.nb, m.nfb, w, 1)));
        }
    }
    if (m.precision == MTP_TF32 || m.precision == MTP_TF32X3) {
        const RefTables& r = m.ref;
        const int nb = m.nb, nfb = m.nfb, d3 = m.dim, nvx = m.dim + 1;
        const int MT = (nb + 15) / 16, KT = (nb + 7) / 8, KTL = (nfb + 7) / 8;
        std::vector<float> sh, sl, lh, ll, th, tl;
        for (int j = 0; j <= d3; ++j)
            for (int l = 0; l < d3; ++l)
                append_fragments(sh, sl, MT, KT, [&](int a, int b) {
                    return (a < nb && b < nb) ? r.S[(((size_t)j * d3 + l) * nb + a) * nb + b] : 0.0;
                });
        for (int j = 0; j <= d3; ++j)
            for (int f = 0; f < nvx; ++f)
                append_fragments(lh, ll, MT, KTL, [&](int a, int cc) {
                    return (a < nb && cc < nfb) ? r.L[(((size_t)j * nvx + f) * nb + a) * nfb + cc] : 0.0;
                });
        for (int f = 0; f < nvx; ++f)
            append_fragments(th, tl, 1, KT, [&](int cc, int b) {
                return (cc < nfb && b < nb) ? r.Tr[((size_t)f * nfb + cc) * nb + b] : 0.0;
            });
        MTP_TRY(upload(&d.Sf, sh.data(), sh.size()));
        MTP_TRY(upload(&d.Lfr, lh.data(), lh.size()));
        MTP_TRY(upload(&d.Trf, th.data(), th.size()));
        MTP_TRY(upload(&d.Sf_lo, sl.data(), sl.size()));
        MTP_TRY(upload(&d.Lfr_lo, ll.data(), ll.size()));
        MTP_TRY(upload(&d.Trf_lo, tl.data(), tl.size()));
    }
    MTP_TRY(upload(&d.V, m.ref.V.data(), m.ref.V.size()));
    MTP_TRY(upload(&d.Vinv, m.ref.Vinv.data(), m.ref.Vinv.size()));
    CUDA_TRY(cudaMalloc((void**)&d.partial, sizeof(double) * (kEnergyBlocks + 1) * m.n_rhs));
    return MTP_OK;
}

void device_mesh_free(Mesh& m) {
    if (!m.dev) return;
    DeviceMesh& d = *m.dev;
    void* ptrs[] = {d.geo, d.elems, d.patch_ptr, d.patch_elem, d.patch_info, d.S, d.Tr, d.L, d.Mc, d.Dc, d.Trc, d.Lc, d.Mc1, d.Dc1, d.Trc1, d.Lc1,
                    d.V, d.Vinv, d.partial,
                    d.Sf, d.Lfr, d.Trf, d.Sf_lo, d.Lfr_lo, d.Trf_lo, d.Dtc};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete m.dev;
    m.dev = nullptr;
}

void device_tents_free(Tents& t) {
    if (!t.dev) return;
    DeviceTents& d = *t.dev;
    if (d.exec) cudaGraphExecDestroy(d.exec);
    if (d.capture) cudaStreamDestroy(d.capture);
    void* ptrs[] = {d.v, d.tb, d.tt, d.tau, d.err, d.host_state, d.adj_buf, d.tau_rev, d.tent_off, d.tent_layer, d.vt_ptr,
                    d.vt_layer, d.adj_ptr, d.adj, d.cnt, d.next};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (d.err_host) cudaFreeHost(d.err_host);
    delete t.dev;
    t.dev = nullptr;
}

static int device_tents_upload(Tents& t) {
    MTP_TRY(device_mesh_upload(*t.mesh));
    if (t.dev) return MTP_OK;
    t.dev = new DeviceTents();
    DeviceTents& d = *t.dev;
    MTP_TRY(upload(&d.v, t.vertex.data(), t.vertex.size()));
    MTP_TRY(upload(&d.tb, t.t_bot.data(), t.t_bot.size()));
    MTP_TRY(upload(&d.tt, t.t_top.data(), t.t_top.size()));
    CUDA_TRY(cudaMalloc((void**)&d.tau, sizeof(double) * t.mesh->nv));
    CUDA_TRY(cudaMalloc((void**)&d.err, sizeof(int)));
    CUDA_TRY(cudaMallocHost((void**)&d.err_host, sizeof(int)));
    CUDA_TRY(cudaStreamCreateWithFlags(&d.capture, cudaStreamNonBlocking));
    // per-vertex tent layers (tents are sorted by layer, so each list is ascending)
    const Mesh& m = *t.mesh;
    std::vector<int64_t> vt_ptr(m.nv + 1, 0);
    for (int32_t v : t.vertex) vt_ptr[v + 1]++;
    for (int64_t v = 0; v < m.nv; ++v) vt_ptr[v + 1] += vt_ptr[v];
    std::vector<int32_t> vt_layer(t.vertex.size());
    {
        std::vector<int64_t> fill(vt_ptr.begin(), vt_ptr.end() - 1);
        for (size_t i = 0; i < t.vertex.size(); ++i) vt_layer[fill[t.vertex[i]]++] = t.layer[i];
    }
    MTP_TRY(upload(&d.tent_layer, t.layer.data(), t.layer.size()));
    MTP_TRY(upload(&d.vt_ptr, vt_ptr.data(), vt_ptr.size()));
    MTP_TRY(upload(&d.vt_layer, vt_layer.data(), vt_layer.size()));
    MTP_TRY(upload(&d.adj_ptr, m.adj_ptr.data(), m.adj_ptr.size()));
    MTP_TRY(upload(&d.adj, m.adj.data(), m.adj.size()));
    CUDA_TRY(cudaMalloc((void**)&d.cnt, sizeof(int) * m.nv));
    CUDA_TRY(cudaMalloc((void**)&d.next, sizeof(unsigned long long)));
    return MTP_OK;
}

static const KernelEntry& kernel_entry(const Mesh& m, int variant = 0) {
    static KernelEntry f64[2][5], f32[2][5], tc[2][5], split[2][5], rk4[2][5], f32v1[2][5], f32v2[2][5], tc5[2][5];
    static bool init = false;
    if (!init) {
        kernel_table_f32_tc5(tc5);
        kernel_table_f64(f64);
        kernel_table_f32(f32);
        kernel_table_tc(tc);
        kernel_table_split(split);
        kernel_table_rk4(rk4);
        kernel_table_f32_v1(f32v1);
        kernel_table_f32_v2(f32v2);
        init = true;
    }
    if ((variant == 3 || variant == 4) && m.precision == MTP_FP32 && m.dim == 3 && !(m.flags & MTP_FLAG_SUBSTITUTED_RK4))
        return tc5[variant - 3][m.p - 1];   // null entries outside p = 2..4 (refused when the variant is set)
    if (variant == 2 && m.precision == MTP_FP32 && !(m.flags & MTP_FLAG_SUBSTITUTED_RK4))
        return f32v2[m.dim - 2][m.p - 1];
    if (variant == 1 && m.precision == MTP_FP32 && !(m.flags & MTP_FLAG_SUBSTITUTED_RK4))
        return f32v1[m.dim - 2][m.p - 1];
    if (m.flags & MTP_FLAG_SUBSTITUTED_RK4) return rk4[m.dim - 2][m.p - 1];   // FP64 only (checked at creation)
    if (m.precision == MTP_FP32_SPLIT) return split[m.dim - 2][m.p - 1];
    if (m.precision == MTP_TF32 || m.precision == MTP_TF32X3)
        return tc[m.precision == MTP_TF32 ? 0 : 1][m.p - 1];
    return (m.precision == MTP_FP64 ? f64 : f32)[m.dim - 2][m.p - 1];
}


// ---------------------------------------------------------------------------------
// lattice exchange: y(x_k) = (1/sqrt|det J|) sum_a V[k][a] Y_a and its inverse
// ---------------------------------------------------------------------------------
template <typename Real>
__global__ void from_lattice_kernel(const double* vals, Real* state, const double* geo, const double* Vinv,
                                    int64_t ne, int nf, int nb, int nrhs) {
    const int64_t n = (int64_t)nrhs * ne * nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t re = i / nb;
        const int a = (int)(i - re * nb);
        const int64_t e = re % ne;
        const double sq = 1.0 / geo[e * kGeoStride + 28];
        const double* v = vals + re * nb * nf;
        for (int f = 0; f < nf; ++f) {
            double acc = 0;
            for (int k = 0; k < nb; ++k) acc += Vinv[a * nb + k] * v[k * nf + f];
            state[(re * nf + f) * nb + a] = (Real)(sq * acc);
        }
    }
}

template <typename Real>
__global__ void to_lattice_kernel(const Real* state, double* vals, const double* geo, const double* V,
                                  int64_t ne, int nf, int nb, int nrhs) {
    const int64_t n = (int64_t)nrhs * ne * nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t re = i / nb;
        const int k = (int)(i - re * nb);
        const int64_t e = re % ne;
        const double is = geo[e * kGeoStride + 28];
        for (int f = 0; f < nf; ++f) {
            double acc = 0;
            for (int a = 0; a < nb; ++a) acc += V[k * nb + a] * (double)state[(re * nf + f) * nb + a];
            vals[(re * nb + k) * nf + f] = is * acc;
        }
    }
}

static int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

int device_from_lattice(Mesh& m, const double* vals, void* state, void* stream) {
    MTP_TRY(device_mesh_upload(m));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)m.n_rhs * m.ne * m.nb;
    if (state_f64(m))
        from_lattice_kernel<double><<<grid_for(n, 256), 256, 0, st>>>(vals, (double*)state, m.dev->geo, m.dev->Vinv,
                                                                       m.ne, m.nf, m.nb, m.n_rhs);
    else
        from_lattice_kernel<float><<<grid_for(n, 256), 256, 0, st>>>(vals, (float*)state, m.dev->geo, m.dev->Vinv,
                                                                      m.ne, m.nf, m.nb, m.n_rhs);
    CUDA_TRY(cudaGetLastError());
    return MTP_OK;
}

int device_to_lattice(Mesh& m, const void* state, double* vals, void* stream) {
    MTP_TRY(device_mesh_upload(m));
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)m.n_rhs * m.ne * m.nb;
    if (state_f64(m))
        to_lattice_kernel<double><<<grid_for(n, 256), 256, 0, st>>>((const double*)state, vals, m.dev->geo, m.dev->V,
                                                                     m.ne, m.nf, m.nb, m.n_rhs);
    else
        to_lattice_kernel<float><<<grid_for(n, 256), 256, 0, st>>>((const float*)state, vals, m.dev->geo, m.dev->V,
                                                                    m.ne, m.nf, m.nb, m.n_rhs);
    CUDA_TRY(cudaGetLastError());
    return MTP_OK;
}

// ---------------------------------------------------------------------------------
// energy on a flat front: 1/2 sum (|Y_E|^2/eps + |Y_H|^2/mu); two-pass deterministic
// reduction through the per-block partials buffer
// ---------------------------------------------------------------------------------
template <typename Real>
__global__ void energy_partial_kernel(const Real* state, const double* geo, int64_t ne, int nf, int nb,
                                      double* partial) {
    __shared__ double red[kEnergyThreads];
    const int rhs = blockIdx.y;
    const Real* s = state + (int64_t)rhs * ne * nf * nb;
    const int64_t n = ne * nf * nb;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = i / (nf * nb);
        const int f = (int)((i / nb) % nf);
        const double y = (double)s[i];
        const double* g = geo + e * kGeoStride;
        const bool isE = nf == 6 ? f < 3 : f < 2;   // E fields first, then H (2D: Ex, Ey | Hz)
        acc += y * y / (isE ? g[29] : g[30]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[rhs * gridDim.x + blockIdx.x] = red[0];
}

__global__ void energy_final_kernel(const double* partial, int nblocks, double* out) {
    __shared__ double red[kEnergyThreads];
    const int rhs = blockIdx.x;
    double acc = 0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) acc += partial[rhs * nblocks + i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[rhs] = 0.5 * red[0];
}

int device_energy(Mesh& m, const void* state, double* out_host, void* stream) {
    MTP_TRY(device_mesh_upload(m));
    cudaStream_t st = (cudaStream_t)stream;
    dim3 grid(kEnergyBlocks, m.n_rhs);
    if (state_f64(m))
        energy_partial_kernel<double><<<grid, kEnergyThreads, 0, st>>>((const double*)state, m.dev->geo, m.ne, m.nf,
                                                                        m.nb, m.dev->partial);
    else
        energy_partial_kernel<float><<<grid, kEnergyThreads, 0, st>>>((const float*)state, m.dev->geo, m.ne, m.nf,
                                                                       m.nb, m.dev->partial);
    CUDA_TRY(cudaGetLastError());
    double* out_dev = m.dev->partial + (size_t)kEnergyBlocks * m.n_rhs;
    energy_final_kernel<<<m.n_rhs, kEnergyThreads, 0, st>>>(m.dev->partial, kEnergyBlocks, out_dev);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(out_host, out_dev, sizeof(double) * m.n_rhs, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return MTP_OK;
}

// ---------------------------------------------------------------------------------
// evolution
// ---------------------------------------------------------------------------------
static void fill_args(Tents& t, void* state, KArgs& a) {
    Mesh& m = *t.mesh;
    DeviceMesh& dm = *m.dev;
    DeviceTents& dt = *t.dev;
    std::memset(&a, 0, sizeof(a));
    a.tent_v = dt.v;
    a.tent_tb = dt.tb;
    a.tent_tt = dt.tt;
    a.patch_ptr = dm.patch_ptr;
    a.patch_elem = dm.patch_elem;
    a.patch_info = dm.patch_info;
    a.elems = dm.elems;
    a.geo = dm.geo;
    a.tau = dt.tau;
    a.S = dm.S;
    a.Tr = dm.Tr;
    a.L = dm.L;
    a.Mc = dm.Mc;
    a.Dc = dm.Dc;
    a.Trc = dm.Trc;
    a.Lc = dm.Lc;
    if (t.variant == 2 || t.variant == 4) {   // one row per thread: one row group per matrix row
        a.Mc = dm.Mc1;
        a.Dc = dm.Dc1;
        a.Trc = dm.Trc1;
        a.Lc = dm.Lc1;
    }
    a.Sf = (const float4*)dm.Sf;
    a.Lfr = (const float4*)dm.Lfr;
    a.Trf = (const float4*)dm.Trf;
    a.Sf_lo = (const float4*)dm.Sf_lo;
    a.Lfr_lo = (const float4*)dm.Lfr_lo;
    a.Trf_lo = (const float4*)dm.Trf_lo;
    a.Dtc = dm.Dtc;
    a.state = state;
    a.rhs_stride = m.ne * m.nf * m.nb;
    a.err = dt.err;
    a.q = m.q;
    a.m = m.m;
    a.max_patch = m.max_patch;
    double f = 1.0;
    for (int i = 0; i <= kMaxSub; ++i) a.tsub[i] = i <= m.m ? (double)i / (double)m.m : 1.0;
    for (int n = 0; n < kMaxTaylor; ++n) {
        if (n > 0) f = f / (double)m.m / (double)n;
        a.taylor[n] = f;
    }
}

static int enqueue_layers(Tents& t, const KArgs& a, int64_t lb, int64_t le, cudaStream_t st) {
    const KernelEntry& ke = kernel_entry(*t.mesh, t.variant);
    for (int64_t l = lb; l < le; ++l) {
        const int64_t t0 = t.layer_ptr[l];
        const int64_t n = t.layer_ptr[l + 1] - t0;
        if (n == 0) continue;
        CUDA_TRY(ke.launch(a, t0, (int)n, t.mesh->n_rhs, st));
    }
    return MTP_OK;
}

static int check_error_word(Tents& t, cudaStream_t st) {
    DeviceTents& d = *t.dev;
    CUDA_TRY(cudaMemcpyAsync(d.err_host, d.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (*d.err_host == 1) return set_error(MTP_ECAUSAL, "a tent violated |grad phi| < sqrt(eps mu)");
    if (*d.err_host == 2) return set_error(MTP_ENUMERIC, "non-finite value in the evolved state");
    if (*d.err_host == 3) return set_error(MTP_ETIMEOUT, "a tent's wait for its predecessors exceeded the limit");
    if (*d.err_host != 0) return set_error(MTP_ECUDA, "unknown device error word");
    return MTP_OK;
}

// front before layer lb (each vertex at the top of its last earlier tent) -> dst (device)
static int set_front(Tents& t, int64_t lb, double* dst, cudaStream_t st) {
    std::vector<double> tau(t.mesh->nv, 0.0);
    for (int64_t i = 0; i < t.layer_ptr[lb]; ++i) tau[t.vertex[i]] = std::fmax(tau[t.vertex[i]], t.t_top[i]);
    CUDA_TRY(cudaMemcpyAsync(dst, tau.data(), sizeof(double) * t.mesh->nv, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));   // the host vector goes out of scope
    return MTP_OK;
}

int device_evolve(Tents& t, void* state, int64_t lb, int64_t le, bool use_graph, void* stream) {
    MTP_TRY(device_tents_upload(t));
    Mesh& m = *t.mesh;
    DeviceTents& d = *t.dev;
    cudaStream_t st = (cudaStream_t)stream;
    const KernelEntry& ke = kernel_entry(m, t.variant);
    size_t smem = 0;
    const cudaError_t pe = ke.prepare(m.max_patch, &smem);
    int dev, smem_max;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if ((int64_t)smem > smem_max)
        return set_error(MTP_EUNSUPPORTED, "tent kernel needs " + std::to_string(smem) +
                                               " bytes of shared memory per block; the device allows " +
                                               std::to_string(smem_max));
    CUDA_TRY(pe);
    MTP_TRY(set_front(t, lb, d.tau, st));
    CUDA_TRY(cudaMemsetAsync(d.err, 0, sizeof(int), st));
    KArgs a;
    fill_args(t, state, a);
    const bool full = lb == 0 && le == (int64_t)t.layer_ptr.size() - 1;
    const int launch = (m.flags & MTP_FLAG_LAYER_LAUNCHES) ? 2 : t.launch;
    if (launch != 2 && le > lb) {
        int bpsm = 0, nsm = 0;
        CUDA_TRY(ke.persistent_prepare(m.max_patch, &bpsm));
        CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int64_t t0 = t.layer_ptr[lb], nt = t.layer_ptr[le] - t0;
        const int cps = launch == 1 ? 1 : std::max(1, bpsm);
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(nt, (int64_t)cps * nsm));
        if (lb == 0) {
            CUDA_TRY(cudaMemsetAsync(d.cnt, 0, sizeof(int) * m.nv, st));
        } else {   // tents completed before the window, per vertex
            std::vector<int> done(m.nv, 0);
            for (int64_t i = 0; i < t0; ++i) done[t.vertex[i]]++;
            CUDA_TRY(cudaMemcpyAsync(d.cnt, done.data(), sizeof(int) * m.nv, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaStreamSynchronize(st));
        }
        CUDA_TRY(cudaMemsetAsync(d.next, 0, sizeof(unsigned long long), st));
        PArgs pa;
        pa.n_tents = nt;
        pa.ticket0 = t0;
        pa.next = d.next;
        pa.cnt = d.cnt;
        pa.vt_ptr = d.vt_ptr;
        pa.vt_layer = d.vt_layer;
        pa.adj_ptr = d.adj_ptr;
        pa.adj = d.adj;
        pa.tent_layer = d.tent_layer;
        pa.timeout_ns = (m.flags & MTP_FLAG_TEST_STALL) ? 200000000LL : 10000000000LL;   // 0.2 s / 10 s per wait
        pa.n_rhs = m.n_rhs;
        pa.withhold_first = (m.flags & MTP_FLAG_TEST_STALL) ? 1 : 0;
        CUDA_TRY(ke.persistent(a, pa, grid, st));
    } else if (use_graph && full) {
        if (!d.exec || d.graph_state != state) {
            if (d.exec) { cudaGraphExecDestroy(d.exec); d.exec = nullptr; }
            cudaGraph_t g;
            CUDA_TRY(cudaStreamBeginCapture(d.capture, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_layers(t, a, lb, le, d.capture);
            cudaError_t ce = cudaStreamEndCapture(d.capture, &g);
            if (rc != MTP_OK) return rc;
            CUDA_TRY(ce);
            CUDA_TRY(cudaGraphInstantiate(&d.exec, g, 0));
            cudaGraphDestroy(g);
            d.graph_state = state;
        }
        CUDA_TRY(cudaGraphLaunch(d.exec, st));
    } else {
        MTP_TRY(enqueue_layers(t, a, lb, le, st));
    }
    return check_error_word(t, st);
}

int device_evolve_host(Tents& t, const void* in, void* out, void* stream) {
    MTP_TRY(device_tents_upload(t));
    Mesh& m = *t.mesh;
    DeviceTents& d = *t.dev;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)m.n_rhs * m.ne * m.nf * m.nb * real_size(m);
    if (!d.host_state) CUDA_TRY(cudaMalloc(&d.host_state, bytes));
    CUDA_TRY(cudaMemcpyAsync(d.host_state, in, bytes, cudaMemcpyHostToDevice, st));
    MTP_TRY(device_evolve(t, d.host_state, 0, (int64_t)t.layer_ptr.size() - 1, true, stream));
    CUDA_TRY(cudaMemcpyAsync(out, d.host_state, bytes, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return MTP_OK;
}

}  // namespace mtp

namespace mtp {

// Patch tape of one layer: the coefficients of the elements of every tent's patch, tents in
// layer order, each patch's elements in patch order; entry e of the tape holds nc = n_fields
// x n_basis values per right-hand side, tape[rhs][e][nc].  One block per (tent, rhs).
template <typename Real, bool GATHER>
__global__ void patch_tape_kernel(Real* state, Real* tape, const int32_t* tent_v, const int64_t* tent_off,
                                  const int64_t* patch_ptr, const int32_t* patch_elem, int64_t t0, int64_t e0,
                                  int nc, int64_t state_rhs_stride, int64_t tape_rhs_stride) {
    const int64_t t = t0 + blockIdx.x;
    const int V = tent_v[t];
    const int64_t pb = patch_ptr[V], ns = patch_ptr[V + 1] - pb;
    Real* st = state + (int64_t)blockIdx.y * state_rhs_stride;
    Real* tp = tape + (int64_t)blockIdx.y * tape_rhs_stride + (tent_off[t] - e0) * nc;
    for (int64_t i = threadIdx.x; i < ns * nc; i += blockDim.x) {
        const int64_t k = i / nc, r = i - k * nc;
        Real* g = st + (int64_t)patch_elem[pb + k] * nc + r;
        if (GATHER) tp[i] = *g; else *g = tp[i];
    }
}

static int patch_tape(Tents& t, void* state, void* tape, int64_t layer, int64_t e0, int64_t tape_entries,
                      bool gather, cudaStream_t st) {
    Mesh& m = *t.mesh;
    const int64_t t0 = t.layer_ptr[layer], n = t.layer_ptr[layer + 1] - t0;
    if (n == 0) return MTP_OK;
    const int nc = m.nf * m.nb;
    dim3 grid((unsigned)n, m.n_rhs);
    const int64_t srs = m.ne * nc, trs = tape_entries * nc;
    DeviceMesh& dm = *m.dev;
    DeviceTents& d = *t.dev;
    if (m.precision == MTP_FP64) {
        if (gather)
            patch_tape_kernel<double, true><<<grid, 128, 0, st>>>((double*)state, (double*)tape, d.v, d.tent_off,
                                                                  dm.patch_ptr, dm.patch_elem, t0, e0, nc, srs, trs);
        else
            patch_tape_kernel<double, false><<<grid, 128, 0, st>>>((double*)state, (double*)tape, d.v, d.tent_off,
                                                                   dm.patch_ptr, dm.patch_elem, t0, e0, nc, srs, trs);
    } else {
        if (gather)
            patch_tape_kernel<float, true><<<grid, 128, 0, st>>>((float*)state, (float*)tape, d.v, d.tent_off,
                                                                 dm.patch_ptr, dm.patch_elem, t0, e0, nc, srs, trs);
        else
            patch_tape_kernel<float, false><<<grid, 128, 0, st>>>((float*)state, (float*)tape, d.v, d.tent_off,
                                                                  dm.patch_ptr, dm.patch_elem, t0, e0, nc, srs, trs);
    }
    CUDA_TRY(cudaGetLastError());
    return MTP_OK;
}

// Reverse sweep with layer checkpointing: the forward pass keeps the state before every
// K-th layer; each segment is recomputed from its checkpoint, saving before each of its
// layers only the patch elements that layer touches (a compact patch tape), and is then
// reversed layer by layer: the layer's patch tape is scattered into a work state and the
// adjoint tent kernel reads its bottom values there.
int device_adjoint(Tents& t, const void* state0, const void* lamT, void* lam0, double* geps, double* gmu,
                   int64_t K, void* stream) {
    MTP_TRY(device_tents_upload(t));
    Mesh& m = *t.mesh;
    DeviceTents& d = *t.dev;
    cudaStream_t st = (cudaStream_t)stream;
    static AdjEntry table[2][2][5];
    static bool init = false;
    if (!init) { adjoint_table(table); init = true; }
    if (m.precision == MTP_FP32_SPLIT || (m.flags & MTP_FLAG_SUBSTITUTED_RK4))
        return set_error(MTP_EUNSUPPORTED, "the adjoint runs SAT meshes in FP64, FP32 or a tensor-core mode");
    const AdjEntry& ae = table[m.precision == MTP_FP64 ? 0 : 1][m.dim - 2][m.p - 1];
    const KernelEntry& ke = kernel_entry(m, t.variant);
    size_t smem = 0, smem_f = 0;
    const cudaError_t pa_ = ae.prepare(m.max_patch, &smem);
    const cudaError_t pf_ = ke.prepare(m.max_patch, &smem_f);
    int dev, smem_max;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if ((int64_t)std::max(smem, smem_f) > smem_max)
        return set_error(MTP_EUNSUPPORTED, "adjoint tent kernel needs " + std::to_string(smem) +
                                               " bytes of shared memory per block; the device allows " +
                                               std::to_string(smem_max));
    CUDA_TRY(pa_);
    CUDA_TRY(pf_);
    const int64_t nl = (int64_t)t.layer_ptr.size() - 1;
    if (K <= 0) K = std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)nl)));
    K = std::min(K, nl);
    const int64_t nck = (nl + K - 1) / K;
    const size_t sbytes = (size_t)m.n_rhs * m.ne * m.nf * m.nb * real_size(m);
    int64_t max_tents = 0;
    for (int64_t l = 0; l < nl; ++l) max_tents = std::max(max_tents, t.layer_ptr[l + 1] - t.layer_ptr[l]);
    // patch entries before each tent; the largest segment's patch tape
    std::vector<int64_t> off(t.vertex.size() + 1, 0);
    for (size_t i = 0; i < t.vertex.size(); ++i)
        off[i + 1] = off[i] + (m.patch_ptr[t.vertex[i] + 1] - m.patch_ptr[t.vertex[i]]);
    if (!d.tent_off) MTP_TRY(upload(&d.tent_off, off.data(), off.size()));
    int64_t seg_entries = 0;
    for (int64_t c = 0; c < nck; ++c) {
        const int64_t l0 = c * K, l1 = std::min((c + 1) * K, nl);
        seg_entries = std::max(seg_entries, off[t.layer_ptr[l1]] - off[t.layer_ptr[l0]]);
    }
    const size_t ptape_bytes = (size_t)seg_entries * m.n_rhs * m.nf * m.nb * real_size(m);
    const int64_t tstride = ae.tape_stride(m.max_patch, m.m, m.q);
    const size_t tape_bytes = (size_t)max_tents * m.n_rhs * tstride * real_size(m);
    auto align = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t need = align((size_t)(nck + 2) * sbytes) + align(ptape_bytes) + tape_bytes + 256;
    if (d.adj_bytes < need) {
        if (d.adj_buf) cudaFree(d.adj_buf);
        d.adj_buf = nullptr;
        d.adj_bytes = 0;
        CUDA_TRY(cudaMalloc(&d.adj_buf, need));
        d.adj_bytes = need;
    }
    if (!d.tau_rev) CUDA_TRY(cudaMalloc((void**)&d.tau_rev, sizeof(double) * m.nv));
    char* base = (char*)d.adj_buf;
    auto ckpt = [&](int64_t c) { return (void*)(base + c * sbytes); };
    void* work = (void*)(base + nck * sbytes);          // the recomputed state
    void* ybot = (void*)(base + (nck + 1) * sbytes);    // bottom values of the layer being reversed
    void* ptape = (void*)(base + align((size_t)(nck + 2) * sbytes));
    void* tape = (void*)(base + align((size_t)(nck + 2) * sbytes) + align(ptape_bytes));

    CUDA_TRY(cudaMemsetAsync(d.err, 0, sizeof(int), st));
    // forward pass with checkpoints
    MTP_TRY(set_front(t, 0, d.tau, st));
    CUDA_TRY(cudaMemcpyAsync(work, state0, sbytes, cudaMemcpyDeviceToDevice, st));
    KArgs fa;
    for (int64_t c = 0; c < nck; ++c) {
        CUDA_TRY(cudaMemcpyAsync(ckpt(c), work, sbytes, cudaMemcpyDeviceToDevice, st));
        fill_args(t, work, fa);
        MTP_TRY(enqueue_layers(t, fa, c * K, std::min((c + 1) * K, nl), st));
    }
    // reverse sweep
    CUDA_TRY(cudaMemcpyAsync(lam0, lamT, sbytes, cudaMemcpyDeviceToDevice, st));
    CUDA_TRY(cudaMemsetAsync(geps, 0, sizeof(double) * m.ne, st));
    CUDA_TRY(cudaMemsetAsync(gmu, 0, sizeof(double) * m.ne, st));
    {
        std::vector<double> top(m.nv, t.T);
        CUDA_TRY(cudaMemcpyAsync(d.tau_rev, top.data(), sizeof(double) * m.nv, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    AdjArgs aa;
    for (int64_t c = nck - 1; c >= 0; --c) {
        const int64_t l0 = c * K, l1 = std::min((c + 1) * K, nl);
        const int64_t e0 = off[t.layer_ptr[l0]];
        MTP_TRY(set_front(t, l0, d.tau, st));
        CUDA_TRY(cudaMemcpyAsync(work, ckpt(c), sbytes, cudaMemcpyDeviceToDevice, st));
        fill_args(t, work, fa);
        for (int64_t l = l0; l < l1; ++l) {
            MTP_TRY(patch_tape(t, work, ptape, l, e0, seg_entries, true, st));
            if (l + 1 < l1) MTP_TRY(enqueue_layers(t, fa, l, l + 1, st));
        }
        for (int64_t l = l1 - 1; l >= l0; --l) {
            const int64_t t0 = t.layer_ptr[l], n = t.layer_ptr[l + 1] - t0;
            if (n == 0) continue;
            MTP_TRY(patch_tape(t, ybot, ptape, l, e0, seg_entries, false, st));
            fill_args(t, nullptr, aa.k);
            aa.k.tau = d.tau_rev;
            aa.ybot = ybot;
            aa.lam = lam0;
            aa.geps = geps;
            aa.gmu = gmu;
            aa.tape = tape;
            aa.tape_stride = tstride;
            CUDA_TRY(ae.launch(aa, t0, (int)n, m.n_rhs, st));
        }
    }
    return check_error_word(t, st);
}

}  // namespace mtp

namespace mtp {

struct DeviceBatch {
    int32_t* ticket_inst = nullptr;
    int64_t* ticket_tent = nullptr;
    KArgs* kargs = nullptr;
    PArgs* pargs = nullptr;
    int32_t* inst_p = nullptr;
    unsigned long long* next = nullptr;
    int* err = nullptr;
    int* err_host = nullptr;
};

void device_batch_free(Batch& b) {
    if (!b.dev) return;
    DeviceBatch& d = *b.dev;
    void* ptrs[] = {d.ticket_inst, d.ticket_tent, d.kargs, d.pargs, d.inst_p, d.next, d.err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (d.err_host) cudaFreeHost(d.err_host);
    delete b.dev;
    b.dev = nullptr;
}

int device_batch_evolve(Batch& b, void* const* states, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t ni = (int64_t)b.inst.size();
    for (Tents* t : b.inst) MTP_TRY(device_tents_upload(*t));
    const Mesh& m0 = *b.inst[0]->mesh;
    static BatchEntry table[2][2];
    static bool init = false;
    if (!init) { batch_table(table); init = true; }
    for (Tents* t : b.inst)
        if (t->mesh->flags & MTP_FLAG_SUBSTITUTED_RK4)
            return set_error(MTP_EUNSUPPORTED, "batches run SAT meshes; MTP_FLAG_SUBSTITUTED_RK4 is per mesh");
    if (m0.precision == MTP_TF32 || m0.precision == MTP_TF32X3 || m0.precision == MTP_FP32_SPLIT)
        return set_error(MTP_EUNSUPPORTED, "batches run FP64 or FP32 SIMT meshes; tensor-core and split modes are per mesh");
    const BatchEntry& be = table[m0.precision == MTP_FP64 ? 0 : 1][m0.dim - 2];
    if (!b.dev) {
        b.dev = new DeviceBatch();
        DeviceBatch& d = *b.dev;
        MTP_TRY(upload(&d.ticket_inst, b.ticket_inst.data(), b.ticket_inst.size()));
        MTP_TRY(upload(&d.ticket_tent, b.ticket_tent.data(), b.ticket_tent.size()));
        std::vector<int32_t> ps(ni);
        for (int64_t i = 0; i < ni; ++i) ps[i] = b.inst[i]->mesh->p;
        MTP_TRY(upload(&d.inst_p, ps.data(), ps.size()));
        CUDA_TRY(cudaMalloc((void**)&d.kargs, sizeof(KArgs) * ni));
        CUDA_TRY(cudaMalloc((void**)&d.pargs, sizeof(PArgs) * ni));
        CUDA_TRY(cudaMalloc((void**)&d.next, sizeof(unsigned long long)));
        CUDA_TRY(cudaMalloc((void**)&d.err, sizeof(int)));
        CUDA_TRY(cudaMallocHost((void**)&d.err_host, sizeof(int)));
    }
    DeviceBatch& d = *b.dev;
    size_t smem = 0;
    std::vector<KArgs> ka(ni);
    std::vector<PArgs> pa(ni);
    for (int64_t i = 0; i < ni; ++i) {
        Tents& t = *b.inst[i];
        Mesh& m = *t.mesh;
        smem = std::max(smem, be.smem_bytes(m.p, m.max_patch));
        fill_args(t, states[i], ka[i]);
        ka[i].err = d.err;
        DeviceTents& dt = *t.dev;
        pa[i].n_tents = (int64_t)t.vertex.size();
        pa[i].ticket0 = 0;
        pa[i].next = nullptr;
        pa[i].cnt = dt.cnt;
        pa[i].vt_ptr = dt.vt_ptr;
        pa[i].vt_layer = dt.vt_layer;
        pa[i].adj_ptr = dt.adj_ptr;
        pa[i].adj = dt.adj;
        pa[i].tent_layer = dt.tent_layer;
        pa[i].timeout_ns = 10000000000LL;
        pa[i].n_rhs = m.n_rhs;
        pa[i].withhold_first = 0;
        CUDA_TRY(cudaMemsetAsync(dt.tau, 0, sizeof(double) * m.nv, st));   // flat front t = 0
        CUDA_TRY(cudaMemsetAsync(dt.cnt, 0, sizeof(int) * m.nv, st));
    }
    int dev, smem_max, bpsm = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if ((int64_t)smem > smem_max)
        return set_error(MTP_EUNSUPPORTED, "batch kernel needs " + std::to_string(smem) +
                                               " bytes of shared memory per block; the device allows " +
                                               std::to_string(smem_max));
    CUDA_TRY(be.prepare(smem, &bpsm));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaMemcpyAsync(d.kargs, ka.data(), sizeof(KArgs) * ni, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(d.pargs, pa.data(), sizeof(PArgs) * ni, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemsetAsync(d.next, 0, sizeof(unsigned long long), st));
    CUDA_TRY(cudaMemsetAsync(d.err, 0, sizeof(int), st));
    BatchArgs ba;
    ba.n_tickets = (int64_t)b.ticket_inst.size();
    ba.next = d.next;
    ba.ticket_inst = d.ticket_inst;
    ba.ticket_tent = d.ticket_tent;
    ba.kargs = d.kargs;
    ba.pargs = d.pargs;
    ba.inst_p = d.inst_p;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ba.n_tickets, (int64_t)std::max(1, bpsm) * nsm));
    CUDA_TRY(be.launch(ba, grid, smem, st));
    CUDA_TRY(cudaMemcpyAsync(d.err_host, d.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));     // also keeps ka / pa alive until copied
    if (*d.err_host == 1) return set_error(MTP_ECAUSAL, "a tent violated |grad phi| < sqrt(eps mu)");
    if (*d.err_host == 2) return set_error(MTP_ENUMERIC, "non-finite value in the evolved state");
    if (*d.err_host == 3) return set_error(MTP_ETIMEOUT, "a tent's wait for its predecessors exceeded the limit");
    if (*d.err_host != 0) return set_error(MTP_ECUDA, "unknown device error word");
    return MTP_OK;
}

}  // namespace mtp

namespace mtp {

// Times the three evolve launch configurations on layers [lb, le) of `state` (overwritten) and
// keeps the fastest in the tents handle.
int device_autotune(Tents& t, void* state, int64_t lb, int64_t le, int* best, double* ms_out, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    double best_ms = 1e300;
    int best_c = 0;
    for (int c = 0; c < 3; ++c) {
        t.launch = c;
        MTP_TRY(device_evolve(t, state, lb, le, false, stream));          // warm-up
        CUDA_TRY(cudaEventRecord(e0, st));
        MTP_TRY(device_evolve(t, state, lb, le, false, stream));
        CUDA_TRY(cudaEventRecord(e1, st));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms_out) ms_out[c] = ms;
        if (ms < best_ms) { best_ms = ms; best_c = c; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    t.launch = best_c;
    if (best) *best = best_c;
    return MTP_OK;
}

}  // namespace mtp
