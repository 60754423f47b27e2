// Host-side finite-element assembly of the diffusion sub-problem (Eq. 2b/2c):
// stiffness k_ij = sum_e int grad N_i . D_e grad N_j and row-sum lumped mass
// m_i = sum_e int N_i (the diagonal m_ii that Eq. 3 and the explicit update
// use), for 4-node bilinear quads, 8-node trilinear hexes and 4-node tets.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace daeti {

// D = d_t I + (d_l - d_t) f f^T (fibre normalised; zero fibre -> d_t I).
void conductivity_tensor(double d_long, double d_trans, const double* fibre, int dim, double D[9]);

// Stiffness of an axis-aligned box element of side h (2^dim local nodes,
// local node a at offsets (a&1, a>>1&1, a>>2&1)), tensor-product 2-point Gauss.
void box_stiffness(int dim, double h, const double D[9], double* Ke /* (2^dim)^2 */);

// Stiffness of a P1 tetrahedron; returns its volume (0 if degenerate).
double tet_stiffness(const double X[12], const double D[9], double Ke[16]);

// Structured grid whose D depends at most on the element layer ez: the
// stencil table per node class (z layer, y class, x class).
struct GridTable {
    int dim = 3, nx = 0, ny = 0, nz = 0;
    std::vector<double> K;   // [nz*9][27] k_ij (diagonal at the centre entry)
    std::vector<double> m;   // [nz*9] lumped mass
};

// Returns false (and leaves `out` empty) if D is not constant on each layer.
bool build_grid_table(int dim, const int64_t n[3], double h, const double* d_long, const double* d_trans,
                      const double* fibre, GridTable& out);

// The two halves of build_grid_table, writing into caller arrays (no
// allocation).  grid_layer_stiffness: the element stiffness of each element
// layer into layerK (ez_n blocks of (2^dim)^2, ez_n = nz - 1 in 3D, 1 in 2D;
// d_trans may be null for d_long); false if D varies within a layer.
// grid_class_table: the stencil row (27 entries) and lumped mass of each node
// class (z layer, y class, x class) from those blocks, K[nz*9*27], m[nz*9].
bool grid_layer_stiffness(int dim, const int64_t n[3], double h, const double* d_long, const double* d_trans,
                          const double* fibre, double* layerK);
void grid_class_table(int dim, const int64_t n[3], double h, const double* layerK, double* K, double* m);

// General sparse operator: CSR of K (with diagonal) and lumped mass.
struct CsrK {
    int64_t n = 0;
    std::vector<int64_t> rowptr;
    std::vector<int> col;
    std::vector<double> val;
    std::vector<double> m;
};

bool assemble_grid_csr(int dim, const int64_t n[3], double h, const double* d_long, const double* d_trans,
                       const double* fibre, CsrK& out, std::string& err);
bool assemble_tet_csr(int64_t n_nodes, const double* xyz, int64_t n_tets, const int64_t* tets,
                      const double* d_long, const double* d_trans, const double* fibre, CsrK& out,
                      std::string& err);

// SELL-32 of the off-diagonal part of K (rows in chunks of 32, column-major
// within a chunk, padded with zero entries pointing at the row itself),
// with each entry scaled by `scale[row]` (pass null for no scaling).
struct Sell32 {
    int64_t n_chunks = 0;
    std::vector<int64_t> chunk_ptr;
    std::vector<int> chunk_w;
    std::vector<int> col;
    std::vector<double> val;
    std::vector<double> diag;
};
void csr_to_sell32(const CsrK& K, const double* scale, Sell32& out);

}  // namespace daeti
