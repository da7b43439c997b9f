// Internal data structures shared by the host library and the CUDA launch code.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mtp.h"

namespace mtp {

constexpr int kMaxDegree = 5;
constexpr int kMaxPatch3D = 32;   // Kuhn/Freudenthal meshes have 24 tets per interior vertex
constexpr int kMaxPatch2D = 16;

inline int n_basis(int dim, int p) {
    return dim == 2 ? (p + 1) * (p + 2) / 2 : (p + 1) * (p + 2) * (p + 3) / 6;
}
inline int n_face_basis(int dim, int p) { return dim == 2 ? p + 1 : (p + 1) * (p + 2) / 2; }
inline int n_fields(int dim) { return dim == 2 ? 3 : 6; }

// Reference-element tables of the orthonormal (Dubiner) basis on the unit simplex,
// all integrals exact (polynomial arithmetic + monomial integration formula).
struct RefTables {
    int dim = 0, p = 0, nb = 0, nfb = 0;
    // S[j][l][a][b] = int_{T^} lambda_j psi_b d_l psi_a            (j <= dim, l < dim)
    std::vector<double> S;
    // Factored volume tables, nbm = dim P_{p-1}: d_l psi_a lies in P_{p-1}, so with
    // D[l][c][a] = int psi_c d_l psi_a and M[j][c][b] = int psi_c lambda_j psi_b (c < nbm),
    // S[j][l][a][b] = sum_c D[l][c][a] M[j][c][b] exactly.
    int nbm = 0;
    std::vector<double> D;   // [l][c][a]
    std::vector<double> M;   // [j][c][b]
    // Tr[f][c][a] = int_{F^} chi_c(s) psi_a(x_f(s)) ds              (facet f opposite vertex f)
    std::vector<double> Tr;
    // L[j][f][a][c] = int_{F^} lambda_j(x_f(s)) psi_a(x_f(s)) chi_c(s) ds
    std::vector<double> L;
    // V[k][a] = psi_a(lattice point k), Vinv its inverse
    std::vector<double> V, Vinv;
    double max_orth_err = 0;   // max |int psi_a psi_b - delta_ab| (diagnostic)
};
RefTables build_ref_tables(int dim, int p);

// Per-element FP64 geometry, packed for the device (one record per element).
// layout (3D; 2D uses the same slots with z entries 0):
//   [0..11]  grad lambda_i (i = 0..3), xyz
//   [12..23] outward unit normal of facet f (opposite local vertex f), xyz
//   [24..27] facet measure |F_f| * (dim-1)!
//   [28] 1/sqrt|det J|  [29] eps  [30] mu  [31] Z = sqrt(mu/eps)
constexpr int kGeoStride = 32;

struct Mesh {
    int dim = 0, p = 0, q = 0, m = 0, precision = 0, n_rhs = 1, flags = 0;
    int nf = 0, nb = 0, nfb = 0, max_patch = 0;
    int64_t nv = 0, ne = 0;
    std::vector<double> verts;         // [nv][dim]
    std::vector<int32_t> elems;        // [ne][dim+1] vertex ids sorted ascending
    std::vector<double> eps, mu;
    std::vector<double> geo;           // [ne][kGeoStride]
    std::vector<int32_t> nbr;          // [ne][dim+1] neighbour element or -1 (PEC)
    std::vector<int8_t> nbr_face;      // [ne][dim+1] neighbour's local facet
    std::vector<int64_t> patch_ptr;    // [nv+1]
    std::vector<int32_t> patch_elem;   // elements of omega_V, ordered by (local index of V, id)
    // per patch entry: local index j of V, then for each local facet f the patch slot of
    // the neighbour across f (-1: PEC boundary facet; -2: f == j), then the neighbour's
    // local facet index.  Packed as 4 bytes + 4 bytes + 4 bytes (3D; 2D pads).
    std::vector<int8_t> patch_info;    // [n_entries][12]
    std::vector<int64_t> adj_ptr;      // vertex adjacency (CSR, ascending)
    std::vector<int32_t> adj;
    RefTables ref;
    struct DeviceMesh* dev = nullptr;  // lazily created device copies
};

struct Tents {
    Mesh* mesh = nullptr;
    double T = 0, cf = 0;
    std::vector<int32_t> vertex, layer;
    std::vector<double> t_bot, t_top;
    std::vector<int64_t> layer_ptr;
    double spacetime_dofs = 0;
    // evolve launch configuration (see mtp_tents_set_launch): 0 DAG walk at the occupancy
    // limit of CTAs per SM, 1 DAG walk with one CTA per SM, 2 one launch per layer
    int launch = 0;
    // kernel shape variant (see mtp_tents_set_variant): 0 paired elements, 1 one element per item
    int variant = 0;
    struct DeviceTents* dev = nullptr;
};

struct Batch {
    std::vector<Tents*> inst;
    std::vector<int32_t> ticket_inst;
    std::vector<int64_t> ticket_tent;
    double spacetime_dofs = 0;
    struct DeviceBatch* dev = nullptr;
};

// error reporting
int set_error(int code, const std::string& msg);

// pitcher: vertex graph with per-edge bounds b_VW (rows sorted by neighbour id), host
// rounds, device rounds (mtp_pitch.cu), and the common tail (spacetime DOF count, T, cf)
struct PitchGraph {
    std::vector<int64_t> ptr;   // [nv + 1]
    std::vector<int32_t> dst;   // neighbours W of V: dst[ptr[V] .. ptr[V+1])
    std::vector<double> bnd;    // b_VW beside each neighbour
};
int pitch_graph(const Mesh& mesh, const double* wavespeed, double cf, PitchGraph& g);
int pitch(const Mesh& mesh, const double* wavespeed, double cf, double T, Tents& out);
int device_pitch(const Mesh& mesh, const PitchGraph& g, double T, Tents& out, void* stream);
void pitch_finish(const Mesh& mesh, double T, double cf, Tents& out);

// device side (mtp_cuda.cu)
int device_mesh_upload(Mesh& m);
void device_mesh_free(Mesh& m);
void device_tents_free(Tents& t);
int device_from_lattice(Mesh& m, const double* vals, void* state, void* stream);
int device_to_lattice(Mesh& m, const void* state, double* vals, void* stream);
int device_evolve(Tents& t, void* state, int64_t layer_begin, int64_t layer_end, bool use_graph,
                  void* stream);
int device_evolve_host(Tents& t, const void* in, void* out, void* stream);
int device_energy(Mesh& m, const void* state, double* out_host, void* stream);
int device_batch_evolve(Batch& b, void* const* states, void* stream);
int device_autotune(Tents& t, void* state, int64_t lb, int64_t le, int* best, double* ms_out, void* stream);
void device_batch_free(Batch& b);
int device_adjoint(Tents& t, const void* state0, const void* lamT, void* lam0, double* geps, double* gmu,
                   int64_t checkpoint_every, void* stream);

}  // namespace mtp
