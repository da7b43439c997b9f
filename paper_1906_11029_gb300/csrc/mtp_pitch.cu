// Tent pitching on the GPU (mtp_pitch_tents_device, see include/mtp.h): the same rounds and
// the same FP64 arithmetic as the host pitcher, so the tent list is bit-identical.
//
// One round (Sec. 2: vertices that are not neighbours may be advanced independently):
//   select: every vertex V with tau_V < T that is a strict local minimum of (tau, id) over
//           its neighbours gets tau'_V = min(T, min_W tau_W + b_VW) and
//           layer_V = 1 + max(last_V, last_W), all from the values at the start of the round;
//   scan:   one block prefix-sums the per-block counts of selected vertices and commits the
//           round (or stops: nothing selected, or the output arrays are full);
//   emit:   the selected vertices write their tents in ascending vertex order and apply
//           tau'_V, layer_V.
// Selected vertices are never neighbours of each other, so select reads only values that
// no thread of the same round changes before emit runs.
//
// Layer = round: if V is selected in round r and no vertex of {V} u N(V) moved in round
// r - 1, V's test gave the same answer in round r - 1 and V would have moved then; so some
// vertex of the closed neighbourhood has last = r - 1 and layer_V = r (by induction, no
// last exceeds r - 1). Emitting each round in vertex order therefore produces the list
// sorted by (layer, vertex) without a sort; emit checks layer == round and reports an
// internal error otherwise.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "mtp_internal.h"

namespace mtp {

constexpr int kPitchThreads = 1024;   // vertices per block (select / emit) and scan width
constexpr int kPitchRoundsPerSync = 32;
constexpr int kPitchMaxRounds = 50000000;

struct PitchCtl {
    long long count;      // tents committed
    long long capacity;   // tent capacity of the output arrays
    long long base;       // first tent of the round being emitted
    int round;            // next round to run
    int cur;              // round being emitted
    int layer_cap;        // capacity of layer_ptr (entries after the first)
    int stop;             // 0 running, 1 finished (a round selected nothing), 2 out of capacity
    int err;              // 1: a tent's layer differs from its round
};

__global__ void __launch_bounds__(kPitchThreads) pitch_select_kernel(
    const PitchCtl* ctl, int64_t nv, double T, const int64_t* ptr, const int32_t* dst, const double* bnd,
    const double* tau, const int32_t* last, uint8_t* flag, double* newt, int32_t* newl, int* blockcnt) {
    if (ctl->stop) return;
    const int64_t v = (int64_t)blockIdx.x * kPitchThreads + threadIdx.x;
    int sel = 0;
    if (v < nv) {
        const double tv = tau[v];
        if (tv < T) {
            sel = 1;
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q) {
                const int32_t w = dst[q];
                const double tw = tau[w];
                if (!((tv < tw) || (tv == tw && v < w))) { sel = 0; break; }
            }
        }
        if (sel) {
            double cm = INFINITY;
            int32_t lm = last[v];
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q) {
                const double x = __dadd_rn(tau[dst[q]], bnd[q]);
                if (x < cm) cm = x;
                const int32_t lw = last[dst[q]];
                if (lw > lm) lm = lw;
            }
            newt[v] = fmin(T, cm);
            newl[v] = lm + 1;
        }
        flag[v] = (uint8_t)sel;
    }
    const int n = __syncthreads_count(sel);
    if (threadIdx.x == 0) blockcnt[blockIdx.x] = n;
}

// exclusive prefix sum of one value per thread over the block; returns the block total
__device__ __forceinline__ int block_exclusive_scan(int x, int* excl, int* warp_tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = lane < kPitchThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;   // inclusive over warps
    }
    __syncthreads();
    *excl = incl - x + (wid > 0 ? warp_tot[wid - 1] : 0);
    const int total = warp_tot[kPitchThreads / 32 - 1];
    __syncthreads();   // warp_tot may be reused by the caller
    return total;
}

__global__ void __launch_bounds__(kPitchThreads) pitch_scan_kernel(PitchCtl* ctl, int nblocks, const int* blockcnt,
                                                                   int* blockoff, int64_t* layer_ptr) {
    __shared__ int warp_tot[32];
    if (ctl->stop) return;
    long long carry = 0;
    for (int b0 = 0; b0 < nblocks; b0 += kPitchThreads) {
        const int b = b0 + (int)threadIdx.x;
        const int x = b < nblocks ? blockcnt[b] : 0;
        int excl;
        const int tot = block_exclusive_scan(x, &excl, warp_tot);
        if (b < nblocks) blockoff[b] = (int)(carry + excl);
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (carry == 0) {
            ctl->stop = 1;
        } else if (ctl->count + carry > ctl->capacity || ctl->round >= ctl->layer_cap) {
            ctl->stop = 2;
        } else {
            ctl->base = ctl->count;
            ctl->count += carry;
            ctl->cur = ctl->round;
            layer_ptr[ctl->round + 1] = ctl->count;
            ctl->round += 1;
        }
    }
}

__global__ void __launch_bounds__(kPitchThreads) pitch_emit_kernel(
    PitchCtl* ctl, int64_t nv, const uint8_t* flag, const double* newt, const int32_t* newl, const int* blockoff,
    double* tau, int32_t* last, int32_t* out_v, double* out_tb, double* out_tt, int32_t* out_l) {
    __shared__ int warp_tot[32];
    if (ctl->stop) return;
    const int64_t v = (int64_t)blockIdx.x * kPitchThreads + threadIdx.x;
    const int sel = v < nv ? (int)flag[v] : 0;
    int rank;
    block_exclusive_scan(sel, &rank, warp_tot);
    if (sel) {
        const long long pos = ctl->base + blockoff[blockIdx.x] + rank;
        const int32_t l = newl[v];
        out_v[pos] = (int32_t)v;
        out_tb[pos] = tau[v];
        out_tt[pos] = newt[v];
        out_l[pos] = l;
        if (l != ctl->cur) atomicExch(&ctl->err, 1);
        tau[v] = newt[v];
        last[v] = l;
    }
}

__global__ void pitch_init_kernel(int64_t nv, double* tau, int32_t* last) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
        tau[v] = 0.0;
        last[v] = -1;
    }
}

#define PITCH_TRY(call)                                                                          \
    do {                                                                                         \
        cudaError_t _e = (call);                                                                 \
        if (_e != cudaSuccess)                                                                   \
            return set_error(_e == cudaErrorMemoryAllocation ? MTP_ENOMEM : MTP_ECUDA,           \
                             std::string(#call) + ": " + cudaGetErrorString(_e));                \
    } while (0)

namespace {

// device buffers of one pitching call, freed on every exit path
struct PitchBuffers {
    std::vector<void*> owned;
    ~PitchBuffers() {
        for (void* p : owned)
            if (p) cudaFree(p);
    }
    template <typename T>
    cudaError_t alloc(T** p, size_t n) {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
        if (e == cudaSuccess) owned.push_back(*p);
        return e;
    }
    // replace *p (n_old valid entries) by a buffer of n_new entries
    template <typename T>
    cudaError_t grow(T** p, size_t n_old, size_t n_new, cudaStream_t st) {
        T* q = nullptr;
        cudaError_t e = alloc(&q, n_new);
        if (e != cudaSuccess) return e;
        if (n_old) e = cudaMemcpyAsync(q, *p, n_old * sizeof(T), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        for (void*& o : owned)
            if (o == (void*)*p) {
                cudaFree(o);
                o = nullptr;
            }
        *p = q;
        return cudaSuccess;
    }
};

}  // namespace

int device_pitch(const Mesh& m, const PitchGraph& g, double T, Tents& out, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t nv = m.nv;
    const int nblocks = (int)((nv + kPitchThreads - 1) / kPitchThreads);
    PitchBuffers B;
    int64_t* d_ptr;
    int32_t* d_dst;
    double* d_bnd;
    double *d_tau, *d_newt;
    int32_t *d_last, *d_newl;
    uint8_t* d_flag;
    int *d_bcnt, *d_boff;
    PitchCtl* d_ctl;
    PITCH_TRY(B.alloc(&d_ptr, g.ptr.size()));
    PITCH_TRY(B.alloc(&d_dst, g.dst.size()));
    PITCH_TRY(B.alloc(&d_bnd, g.bnd.size()));
    PITCH_TRY(B.alloc(&d_tau, nv));
    PITCH_TRY(B.alloc(&d_newt, nv));
    PITCH_TRY(B.alloc(&d_last, nv));
    PITCH_TRY(B.alloc(&d_newl, nv));
    PITCH_TRY(B.alloc(&d_flag, nv));
    PITCH_TRY(B.alloc(&d_bcnt, nblocks));
    PITCH_TRY(B.alloc(&d_boff, nblocks));
    PITCH_TRY(B.alloc(&d_ctl, 1));
    PITCH_TRY(cudaMemcpyAsync(d_ptr, g.ptr.data(), g.ptr.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (!g.dst.empty()) {
        PITCH_TRY(cudaMemcpyAsync(d_dst, g.dst.data(), g.dst.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        PITCH_TRY(cudaMemcpyAsync(d_bnd, g.bnd.data(), g.bnd.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    pitch_init_kernel<<<(int)std::min<int64_t>(nblocks, 1024), kPitchThreads, 0, st>>>(nv, d_tau, d_last);
    PITCH_TRY(cudaGetLastError());

    // output arrays, grown when a round does not fit (the round is then run again)
    size_t cap = (size_t)std::max<int64_t>(nv * 16, 1 << 16);
    int layer_cap = 4096;
    int32_t *o_v, *o_l;
    double *o_tb, *o_tt;
    int64_t* d_lptr;
    PITCH_TRY(B.alloc(&o_v, cap));
    PITCH_TRY(B.alloc(&o_l, cap));
    PITCH_TRY(B.alloc(&o_tb, cap));
    PITCH_TRY(B.alloc(&o_tt, cap));
    PITCH_TRY(B.alloc(&d_lptr, (size_t)layer_cap + 1));
    PITCH_TRY(cudaMemsetAsync(d_lptr, 0, sizeof(int64_t), st));
    PitchCtl h{};
    h.capacity = (long long)cap;
    h.layer_cap = layer_cap;
    PITCH_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    while (true) {
        for (int r = 0; r < kPitchRoundsPerSync; ++r) {
            pitch_select_kernel<<<nblocks, kPitchThreads, 0, st>>>(d_ctl, nv, T, d_ptr, d_dst, d_bnd, d_tau, d_last,
                                                                   d_flag, d_newt, d_newl, d_bcnt);
            pitch_scan_kernel<<<1, kPitchThreads, 0, st>>>(d_ctl, nblocks, d_bcnt, d_boff, d_lptr);
            pitch_emit_kernel<<<nblocks, kPitchThreads, 0, st>>>(d_ctl, nv, d_flag, d_newt, d_newl, d_boff, d_tau,
                                                                 d_last, o_v, o_tb, o_tt, o_l);
        }
        PITCH_TRY(cudaGetLastError());
        PITCH_TRY(cudaMemcpyAsync(&h, d_ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
        PITCH_TRY(cudaStreamSynchronize(st));
        if (h.err) return set_error(MTP_ECUDA, "device pitcher: a tent's layer differs from its round (internal error)");
        if (h.stop == 1) break;
        if (h.round > kPitchMaxRounds)
            return set_error(MTP_ECAUSAL, "device pitcher: no end after " + std::to_string(kPitchMaxRounds) +
                                              " rounds (edge bounds below the resolution of tau?)");
        if (h.stop == 2) {   // the pending round did not fit: grow and run it again
            if (h.round >= h.layer_cap) {
                const int nc = h.layer_cap * 2;
                PITCH_TRY(B.grow(&d_lptr, (size_t)h.layer_cap + 1, (size_t)nc + 1, st));
                h.layer_cap = nc;
            } else {
                const size_t nc = std::max<size_t>(cap * 2, (size_t)h.count + (size_t)nv);
                PITCH_TRY(B.grow(&o_v, (size_t)h.count, nc, st));
                PITCH_TRY(B.grow(&o_l, (size_t)h.count, nc, st));
                PITCH_TRY(B.grow(&o_tb, (size_t)h.count, nc, st));
                PITCH_TRY(B.grow(&o_tt, (size_t)h.count, nc, st));
                cap = nc;
                h.capacity = (long long)cap;
            }
            h.stop = 0;
            PITCH_TRY(cudaMemcpyAsync(d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice, st));
        }
    }
    const size_t n = (size_t)h.count;
    const int64_t nl = h.round;
    out.vertex.resize(n);
    out.layer.resize(n);
    out.t_bot.resize(n);
    out.t_top.resize(n);
    out.layer_ptr.resize(nl + 1);
    std::vector<double> tau(nv);
    if (n) {
        PITCH_TRY(cudaMemcpyAsync(out.vertex.data(), o_v, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PITCH_TRY(cudaMemcpyAsync(out.layer.data(), o_l, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        PITCH_TRY(cudaMemcpyAsync(out.t_bot.data(), o_tb, n * sizeof(double), cudaMemcpyDeviceToHost, st));
        PITCH_TRY(cudaMemcpyAsync(out.t_top.data(), o_tt, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    PITCH_TRY(cudaMemcpyAsync(out.layer_ptr.data(), d_lptr, (nl + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    PITCH_TRY(cudaMemcpyAsync(tau.data(), d_tau, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
    PITCH_TRY(cudaStreamSynchronize(st));
    for (int64_t v = 0; v < nv; ++v)
        if (tau[v] != T) return set_error(MTP_ECAUSAL, "pitching stalled before reaching T");
    return MTP_OK;
}

}  // namespace mtp
