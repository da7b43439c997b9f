/*
 * mtp.h — C ABI of the GB300 explicit Mapped Tent Pitching (MTP) library for the
 * time-domain Maxwell equations with structure-aware Taylor (SAT) time stepping
 * (Gopalakrishnan, Hochsteger, Schoeberl, Wintersteiger, arXiv:1906.11029).
 *
 * Problem (Sec. 3, eq. maxwell):  d_t(eps E) = curl H,  d_t(mu H) = -curl E  on a
 * conforming simplicial mesh of a bounded domain (2D: TE fields Ex, Ey, Hz; 3D: E, H),
 * eps and mu constant per element, perfectly conducting (PEC) boundary everywhere.
 *
 * Conventions for every call:
 *   - Return value: MTP_OK (0) or a negative MTP_E* code; mtp_last_error() then gives
 *     a thread-local message.  No C++ exception crosses this boundary.
 *   - Host input arrays are read during the call and copied; the caller keeps ownership.
 *   - Handles (mtp_mesh_t, mtp_tents_t) are owned by the library until *_destroy.
 *     A tents handle refers to its mesh: destroy tents before the mesh.
 *   - "dev" pointers are CUDA device pointers owned by the caller (e.g. PyTorch
 *     tensors); "stream" is a cudaStream_t passed as void* (NULL = legacy default).
 *     Device work is enqueued on that stream; calls return when it is enqueued
 *     unless stated otherwise.
 *   - State layout ("library layout"): state[r][e][f][a], r < n_rhs, e < n_elems,
 *     f < n_fields, a < n_basis, in the mesh's state precision (double for MTP_FP64 and
 *     MTP_FP32_SPLIT, float for the others).  The coefficients are those of the conserved variable
 *     y = g(u) - f(u) grad(phi) (Sec. 3, transformed equation; y = (eps E, mu H) on
 *     a flat front) in an L2-orthonormal basis of P_p on each element.
 *   - Lattice layout: vals[r][e][k][f] in double, the value of y at lattice point k
 *     of element e.  Lattice points: with s_0 < ... < s_d the element's vertex ids
 *     sorted ascending, point k is v_{s0} + sum_l (i_l/p)(v_{sl} - v_{s0}) for the
 *     k-th integer tuple (i_1..i_d), sum <= p, enumerated with i_d outermost and i_1
 *     innermost.  P_p is unisolvent on this lattice, so it exchanges states with any
 *     other discretisation of the same space without sharing a basis.
 */
#ifndef MTP_H
#define MTP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MTP_OK            0
#define MTP_EINVAL       -1   /* bad argument (null pointer, size, option, T mismatch) */
#define MTP_EMESH        -2   /* degenerate or non-conforming mesh */
#define MTP_ECAUSAL      -3   /* a tent violates |grad phi| < sqrt(eps mu) or t_top <= t_bot */
#define MTP_ENOMEM       -4   /* host or device allocation failed */
#define MTP_ECUDA        -5   /* a CUDA runtime call failed (message has the CUDA error) */
#define MTP_ETIMEOUT     -6   /* a bounded device-side wait expired */
#define MTP_ENUMERIC     -7   /* NaN / Inf detected */
#define MTP_EUNSUPPORTED -8   /* combination not built (e.g. degree > 5, patch too large) */

/* mtp_options.flags bits */
#define MTP_FLAG_LAYER_LAUNCHES 1   /* mtp_evolve: one launch per layer (CUDA graph) instead of the
                                       persistent DAG-walking kernel */
#define MTP_FLAG_TEST_STALL     2   /* failure injection for tests: the persistent evolve never
                                       publishes the completion of its first tent and waits at most
                                       0.2 s, so it must return MTP_ETIMEOUT */
#define MTP_FLAG_SUBSTITUTED_RK4 4  /* negative control for convergence studies (Sec. 3, after eq.
                                       equ_ode; Sec. 5.1, Fig. 3 right): advance each tent with m
                                       classical RK4 steps on d/dt Y = A M(t)^-1 Y instead of SAT;
                                       MTP_FP64 only; not for batches or the adjoint */

/* precision of the state and of the operator arithmetic */
#define MTP_FP64   0   /* FP64 state and arithmetic */
#define MTP_FP32   1   /* FP32 state and arithmetic (element geometry and causality test in FP64) */
#define MTP_TF32   2   /* 3D: FP32 state; traces, volume and lift contractions on tensor cores
                          with TF32 operands and FP32 accumulation */
#define MTP_TF32X3 3   /* 3D: as MTP_TF32 with each operand split into TF32 hi + lo parts and
                          three products (hi*hi + hi*lo + lo*hi), about FP32 accuracy */
#define MTP_FP32_SPLIT 4 /* FP32 operator arithmetic (as MTP_FP32); the Taylor sum of each tent
                          (Sec. 4, eq. recursion-init) is carried as an unevaluated FP32 pair
                          hi + lo updated by error-free two-sum, and the state between tents is
                          stored in FP64 (library layout in double).  Removes the rounding of the
                          accumulation and of the stored state, the dominant FP32 error terms.
                          Not available for batches or the adjoint. */

typedef struct mtp_mesh*  mtp_mesh_t;
typedef struct mtp_tents* mtp_tents_t;
typedef struct mtp_batch* mtp_batch_t;

typedef struct {
    int p;          /* polynomial degree of V_h, 1..5 (Sec. 3, DG space)                   */
    int q;          /* SAT stages; 0 selects p+1 (Sec. 5.1)                                */
    int m;          /* SAT sub-intervals per tent; 0 selects 2p (Sec. 5.1)                 */
    int precision;  /* MTP_FP64, MTP_FP32, MTP_TF32, MTP_TF32X3 or MTP_FP32_SPLIT            */
    int n_rhs;      /* independent states evolved with the same tents (>= 1; 0 means 1)   */
    int flags;      /* MTP_FLAG_* bits; 0 by default                                       */
} mtp_options;

/* Spatial mesh and materials (Sec. 2: conforming mesh of elements T and vertices V;
 * Sec. 3: eps, mu per element).  vertices[n_verts][dim], elements[n_elems][dim+1]
 * (0-based vertex ids, any orientation), eps/mu[n_elems] > 0.  Host only: validates
 * (MTP_EMESH on zero-volume elements, repeated vertices or a facet shared by more
 * than two elements), builds facets, neighbours, vertex patches, FP64 element
 * geometry and the reference tables of degree p.  No device memory is touched here. */
int mtp_mesh_create(int dim, int64_t n_verts, const double* vertices,
                    int64_t n_elems, const int32_t* elements,
                    const double* eps, const double* mu,
                    const mtp_options* opts, mtp_mesh_t* out);
void mtp_mesh_destroy(mtp_mesh_t mesh);

/* Sizes: n_fields = 3 (2D TE) or 6 (3D); n_basis = dim P_p; max_patch = largest
 * vertex patch |omega_V|.  Any output pointer may be NULL. */
int mtp_mesh_info(mtp_mesh_t mesh, int* dim, int* n_fields, int* n_basis,
                  int64_t* n_elems, int64_t* n_verts, int* max_patch);

/* Tent pitching to time T (Sec. 2).  Host only, deterministic FP64 (timed separately
 * from evolution).  wavespeed[n_elems] (NULL: 1/sqrt(eps mu)); causality_factor in
 * (0, 1): every front satisfies |grad tau| <= causality_factor / c on every element
 * (0.5 reproduces the slope bound 1/(2c) of Sec. 5.1).  Rule: per vertex
 * k_V = min element height at V; edge bound b_VW = cf min(k_V, k_W) / (d c_VW) with
 * c_VW the largest wave speed on the edge; rounds move every strict local minimum of
 * (tau, vertex id) to min(T, min_W tau_W + b_VW); tent layer = 1 + max(layer of the
 * previous tents at V and its neighbours).  Tents of one layer have disjoint patches
 * (Sec. 2: vertices at graph distance >= 2 are independent).  Output sorted by
 * (layer, vertex). */
int mtp_pitch_tents(mtp_mesh_t mesh, const double* wavespeed, double causality_factor,
                    double T, mtp_tents_t* out);

/* The same pitcher with its rounds on the current CUDA device (Sec. 2: tents at vertices
 * that are not neighbours are pitched independently, so each round is one parallel step).
 * Same rule, arguments and errors as mtp_pitch_tents, and the same tent list bit for bit
 * (identical FP64 operations; each round's tents are emitted in vertex order, and a
 * tent's layer equals its round, so the list comes out sorted by (layer, vertex)).
 * The per-edge bounds are computed on the host as in mtp_pitch_tents; the rounds run on
 * `stream`, and the call returns when the tent list is on the host.  Device memory: about
 * 70 bytes per vertex plus 24 bytes per tent of output, allocated and freed inside the
 * call.  MTP_ECUDA / MTP_ENOMEM on CUDA failures. */
int mtp_pitch_tents_device(mtp_mesh_t mesh, const double* wavespeed, double causality_factor,
                           double T, mtp_tents_t* out, void* stream);
void mtp_tents_destroy(mtp_tents_t tents);

/* n_tents, n_layers, and the spacetime DOF count of one evolve (Sec. 5.2):
 * sum_i N_dof,i * m * q * n_rhs with N_dof,i = n_fields * n_basis * |omega_V|.
 * Any output pointer may be NULL. */
int mtp_tents_info(mtp_tents_t tents, int64_t* n_tents, int64_t* n_layers,
                   double* spacetime_dofs);

/* Copy the tent list to host arrays vertex/t_bot/t_top/layer[n_tents] and
 * layer_ptr[n_layers+1] (tents of layer l are [layer_ptr[l], layer_ptr[l+1])).
 * Any pointer may be NULL. */
int mtp_tents_get(mtp_tents_t tents, int32_t* vertex, double* t_bot, double* t_top,
                  int32_t* layer, int64_t* layer_ptr);

/* Lattice values of y (FP64, lattice layout, dev) -> state (library layout, dev).
 * Exact up to rounding for y in P_p on each element. */
int mtp_state_from_lattice(mtp_mesh_t mesh, const double* vals_dev, void* state_dev,
                           void* stream);
/* State (dev) -> lattice values of y (FP64, dev). */
int mtp_state_to_lattice(mtp_mesh_t mesh, const void* state_dev, double* vals_dev,
                         void* stream);

/* Evolve the state in place from the flat front t = 0 to the flat front t = T through
 * every tent, layer by layer (Sec. 2 and 3), each tent advanced bottom to top with
 * q-stage SAT over m sub-intervals (Sec. 4, eqs. coeff_rec and recursion-init), with
 * the mass solve in the closed form of Sec. 4.  Default: one persistent kernel walks the
 * tent DAG (tents taken in layer order; a tent starts once the earlier-layer tents of its
 * vertex and of its neighbours are done, tracked by per-vertex counters; every wait is
 * bounded and reports MTP_ETIMEOUT); with MTP_FLAG_LAYER_LAUNCHES all tents of a layer
 * (times n_rhs) run in one launch and the layers are replayed from a CUDA graph.  T must equal
 * the pitched T (MTP_EINVAL otherwise).  Returns after the work has completed on the
 * stream: the device-side error word is read back (MTP_ECAUSAL if a tent violated
 * causality, MTP_ENUMERIC on a non-finite result). */
int mtp_evolve(mtp_tents_t tents, void* state_dev, double T, void* stream);

/* Evolve launch configuration of this tents handle: 0 (default) the persistent DAG walk with as
 * many CTAs per SM as fit, 1 the DAG walk with one CTA per SM, 2 one launch per layer (CUDA
 * graph).  MTP_FLAG_LAYER_LAUNCHES on the mesh forces 2. */
int mtp_tents_set_launch(mtp_tents_t tents, int launch);

/* Kernel shape variant of this tents handle (MTP_FP32 SAT meshes): 0 (default) each stage item
 * of the tent kernel covers a pair of patch elements with the same local index of the tent
 * vertex, which share every reference-table read; 1 each item covers one element: twice the
 * items at half the work each, so a tent finishes sooner when the layers hold fewer tents than
 * the GPU has CTA slots (e.g. small meshes), at a lower throughput when they hold more;
 * 2 each item covers one element and one basis function (or facet mode), with 512 threads per
 * CTA in 3D: the shortest tents for such latency-bound layers.  3 and 4 (3D, p = 2..4, patches
 * of at most 42 tetrahedra): the item shapes of 1 and 2 on 512 threads, with the volume term of
 * the operator (Sec. 3, the element integrals of the DG semi-discretisation) computed on the
 * tcgen05 tensor cores as TF32 MMAs with a three-term hi + lo operand split and FP32
 * accumulation in tensor memory (FP32-level accuracy).  Results are identical up to rounding
 * order (variants 3 and 4: up to the split's rounding).  MTP_EINVAL for a number outside 0..4,
 * MTP_EUNSUPPORTED for variants 1..4 on meshes they are not built for. */
int mtp_tents_set_variant(mtp_tents_t tents, int variant);

/* Autotuner: times the three launch configurations on layers [layer_begin, layer_end) of
 * scratch_state_dev (overwritten with evolved values) and keeps the fastest for this handle;
 * *best receives it and ms_out[3] (may be NULL) the measured milliseconds. */
int mtp_tents_autotune(mtp_tents_t tents, void* scratch_state_dev, int64_t layer_begin,
                       int64_t layer_end, int* best, double* ms_out, void* stream);

/* Apply only layers [layer_begin, layer_end) to a state that sits on the front just
 * before layer_begin (each vertex at the top of its last earlier tent).  Completion and
 * errors as for mtp_evolve. */
int mtp_evolve_layers(mtp_tents_t tents, void* state_dev, int64_t layer_begin,
                      int64_t layer_end, void* stream);

/* mtp_evolve on host buffers: copies state_in_host (library layout) to a device buffer
 * owned by the tents handle, evolves, copies the result to state_out_host, and
 * synchronises the stream before returning.  state_in_host may equal state_out_host. */
int mtp_evolve_host(mtp_tents_t tents, const void* state_in_host, void* state_out_host,
                    double T, void* stream);

/* Many independent problems evolved in one persistent launch (Sec. 2: tents of different
 * meshes are trivially independent).  tents[n]: pitched tent lists of meshes with the same
 * dimension and precision, any degrees 1..5 (default q = p + 1, m = 2p), any n_rhs each.
 * Tents of all instances are taken in (layer, instance, vertex) order; each instance keeps its
 * own dependency counters.  The batch refers to the tents handles: destroy it first. */
int mtp_batch_create(int64_t n, const mtp_tents_t* tents, mtp_batch_t* out);
void mtp_batch_destroy(mtp_batch_t batch);
/* number of instances, total tents, total spacetime DOF count of one batch evolve */
int mtp_batch_info(mtp_batch_t batch, int64_t* n_instances, int64_t* n_tents,
                   double* spacetime_dofs);
/* Evolve every instance i in place, states_dev[i] in its mesh's library layout, from t = 0 to
 * the T its tents were pitched to.  Completion and errors as for mtp_evolve. */
int mtp_batch_evolve(mtp_batch_t batch, void* const* states_dev, void* stream);

/* Discrete adjoint of mtp_evolve (not in the paper): the reverse-in-time sweep through the
 * tent maps.  Given state0_dev (the state at t = 0) and lambda_T_dev = dJ/dY(T) for a
 * functional J of the final state (both library layout, dev), writes lambda_0_dev =
 * dJ/dY(0) and dJ_deps_dev, dJ_dmu_dev [n_elems] (double, dev, overwritten, summed over the
 * right-hand sides) = the derivatives of J through the tent maps' dependence on eps and mu
 * (the mass operator g(u) - f(u) grad(phi) and the facet impedances).  Dependence of the
 * initial state or of J on eps, mu is the caller's to add.  The forward pass keeps the state
 * before every checkpoint_every-th layer (0: about sqrt(n_layers)); each segment is
 * recomputed from its checkpoint and reversed layer by layer, one CTA per tent, replaying
 * the tent's SAT stages into a device tape.  Device work buffers are owned by the tents
 * handle.  Completion and errors as for mtp_evolve; MTP_EUNSUPPORTED if the adjoint kernel's
 * shared memory for this degree and patch size exceeds the device limit. */
int mtp_adjoint(mtp_tents_t tents, const void* state0_dev, const void* lambda_T_dev,
                void* lambda_0_dev, double* dJ_deps_dev, double* dJ_dmu_dev,
                int64_t checkpoint_every, void* stream);

/* Electromagnetic energy of a state on a flat front, per right-hand side:
 * out_host[r] = 1/2 sum_T int_T (|y_E|^2 / eps + |y_H|^2 / mu)  (= 1/2 int eps|E|^2 + mu|H|^2).
 * Synchronises the stream. */
int mtp_energy(mtp_mesh_t mesh, const void* state_dev, double* out_host, void* stream);

/* Energy of flat-front states, like mtp_energy, for callers that cannot allocate device
 * memory when they need it (for example a host framework that owns all device memory
 * through its own allocator and budget, or a loop that must not allocate after start-up).
 * The paper has no counterpart to this call.
 * Inputs and outputs are all the caller's: state_dev (library layout, n_rhs states of
 * n_elems elements of degree p in the given precision: double for MTP_FP64 and
 * MTP_FP32_SPLIT, float for MTP_FP32, MTP_TF32 and MTP_TF32X3), eps_dev and mu_dev [n_elems] (double, device),
 * out_dev[n_rhs] (double, device) receives the energies.  Nothing is allocated: the
 * reduction scratch is a fixed static device array of 304 x 64 doubles (152 KiB) that every
 * GPU loading this library holds until the process exits; n_rhs above 64 is rejected with
 * MTP_EINVAL.  Every call writes all the scratch it reads, so no clearing is needed, but all
 * calls share that one array: calls that overlap on the GPU (e.g. on two streams at once)
 * race and give wrong results.  Every call looks the array's device address up again
 * (cudaGetSymbolAddress, with the calling thread's current device), so nothing stale survives a
 * device reset; the first call on a device may load the library's device code for it, so make
 * that first call before any stream capture.  Asynchronous on the stream. */
int mtp_energy_noalloc(const void* state_dev, const double* eps_dev, const double* mu_dev,
                       int dim, int64_t n_elems, int p, int precision, int n_rhs,
                       double* out_dev, void* stream);

/* Measured arithmetic rates of the current device, in TFLOP/s (roofline denominators that the
 * host cannot look up): out_tflops[0] FP32 FMA, [1] FP64 FMA, [2] warp-level tensor-core MMA
 * TF32 (m16n8k8, FP32 accumulate), [3] warp-level MMA BF16 (m16n8k16, FP32 accumulate).
 * Synchronises the stream; allocates a small scratch buffer. */
int mtp_probe_rates(double* out_tflops, void* stream);

/* Thread-local description of the last error returned on this thread. */
const char* mtp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MTP_H */
