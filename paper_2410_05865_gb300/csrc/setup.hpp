// Host-side setup of the cut-cell multigrid hierarchy (C++17, OpenMP).
//
// Geometry, cut-cell quadrature, cell merging, the phi1/phi2 split, the
// regular/ghost rows, FV-PLG lattices with their weighted least-squares rows,
// and the sparse LU factors used by the LU-correction (SMO-2) and the bottom
// solver.  Everything here runs once per geometry; the V-cycle itself runs in
// the CUDA kernels of kernels.cu.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace ccmg {

constexpr int kQ = 8;            // Gauss-Legendre points per piece and axis
constexpr int kDMax = 3;         // subdivision depth for boxes met by >= 2 surfaces
constexpr double kEmptyVol = 1e-14;
constexpr double kTheta = 0.02;   // merging threshold (units of h^3)
constexpr double kAreaTie = 1e-12;  // common-face areas this close (units h^2) are ties
constexpr double kRankTol = 1e-10;
constexpr int kNMono = 35;       // monomials of degree <= 4 in 3 variables
constexpr int kNMono3 = 20;      // degree <= 3

enum Bc { BC_DIRICHLET = 0, BC_NEUMANN = 1 };

struct Ellipsoid {
  double c[3];
  double a[3];
};

// Quadrature nodes of one cut cell (absolute coordinates).
struct CutNodes {
  std::vector<double> vp;  // 3 per node
  std::vector<double> vw;
  std::vector<double> sp;  // 3 per node
  std::vector<double> sw;
  std::vector<double> sn;  // outward normal of the fluid, 3 per node
};

// Per cut cell: moments about the cell centre in units of h.
struct CutMoments {
  double vol[kNMono];         // int xi^a dV / h^3
  double srf[kNMono];         // int_S xi^a dS / h^2
  double srfn[3][kNMono3];    // int_S n_d xi^b dS / h^2
};

// The monomial table (exponent triples by total degree, then a desc, b desc).
struct Mono {
  int e[kNMono][3];
  int idx[5][5][5];  // -1 where a+b+c > 4
  Mono();
};
const Mono& mono();

// ----------------------------------------------------------------- geometry
struct Geometry {
  int n = 0;
  double h = 0;
  std::vector<Ellipsoid> shapes;
  std::vector<int8_t> kind;     // 0 exterior, 1 full, 2 cut
  std::vector<double> vol;      // units of h^3
  std::vector<int> cut_id;      // grid -> index into cut arrays, -1 otherwise
  std::vector<int> cut_cells;   // cut index -> grid
  std::vector<CutMoments> mom;
  std::vector<CutNodes> nodes;  // kept only when requested (finest level)
};

void build_geometry(Geometry& g, int n, const std::vector<Ellipsoid>& shapes, bool keep_nodes);
double face_area(const Geometry& g, int i1, int i2);  // units of h^2, i1 < i2 face neighbours

// ----------------------------------------------------------------- a level
struct Level {
  int n = 0;
  double h = 0;
  bool coarse = false;
  int shape_bc = BC_DIRICHLET;
  int box_bc[6] = {0, 0, 0, 0, 0, 0};
  Geometry geo;
  std::vector<int> owner;       // -1 for empty cells
  std::vector<uint8_t> merged;  // takes part in a merge
  std::vector<uint8_t> typ;     // 0 none, 1 phi1, 2 phi2
  // merged owners that are not plain full cells: moments about the owner centre
  std::vector<int> mom_id;      // grid -> index into mvol/msrf/msrfn, -1 = plain full cell
  std::vector<std::vector<double>> mvol, msrf, msrfn;  // 35, 35, 60
  std::vector<std::vector<int>> groups;                // per mom_id: member cells (owner first)
  // phi2 rows, in increasing grid order
  std::vector<int> p2_cell;
  std::vector<int> p2_ptr, p2_col;      // CSR, columns are grid indices
  std::vector<double> p2_val;
  std::vector<int> p2_bptr, p2_bpatch;  // boundary terms: patch owner grid index
  std::vector<double> p2_bcoef;         // coefficient on <<g>> (h already folded for Neumann)
  std::vector<int> p2_degree;
  int n_unknowns = 0;
  int n_phi1 = 0;
};

struct HierarchyParams {
  int min_n = 16;
  int max_levels = 16;
  int nthreads = 0;
};

// Builds level 0 (PLG degree 4 required) and coarser levels h^(m) = 2^m h until
// n < min_n or a PLG search fails (that level is dropped).  Returns 0 or an error
// code: 1 = PLG failed on the finest level, 2 = merging failed, 3 = bad input.
int build_hierarchy(std::vector<Level>& levels, int n, const std::vector<Ellipsoid>& shapes,
                    int shape_bc, const int box_bc[6], const HierarchyParams& prm, std::string* err);

// Regular (ghost-eliminated) 1-D coefficient rows.  For position class
// c in {0: p=0, 1: p=1, 2: interior, 3: p=n-2, 4: p=n-1}: 7 coefficients at
// offsets -3..3 (times 1/(12 h^2) in the 3-D row) and the coefficient of the
// face average g of the nearer wall.
struct Rows1D {
  double c[5][7];
  double g[5];
};
Rows1D regular_rows_1d(int bc_low, int bc_high, double h);

// --------------------------------------------------------------- sparse LU
// Supernodal LU (partial pivoting inside supernodes) in a nested-dissection
// order, stored for the GPU triangular solves in block-elimination form.  With
// P_s the pivoting of supernode s, L_ss U_ss its diagonal block and L_{struct,s},
// U_{s,struct} its off-diagonal blocks, each supernode keeps
//   G = U_ss^{-1} L_ss^{-1}        (k x k, dense)
//   W = L_{struct,s} L_ss^{-1}     (m x k)
//   V = U_ss^{-1} U_{s,struct}     (k x m)
// so that the forward sweep is b_struct -= W P_s b_s (children first) and the
// backward sweep is x_s = G P_s b_s - V x_struct (parents first): one dense
// matrix-vector product per supernode and sweep.  P_s is folded into the
// columns of G and W, which therefore multiply b_s in ND order directly.  The
// blocks are stored column-major (entry (r, c) of an R x C block at c R + r).
struct SuperLU {
  int n = 0;                        // matrix dimension
  std::vector<int> perm;            // perm[p] = original row/col of ND position p
  int nsuper = 0;
  std::vector<int> sn_first;        // first ND position of each supernode (size nsuper+1)
  std::vector<int> sn_height;       // height in the supernode tree (leaves 0)
  std::vector<int> sn_parent;       // parent in the supernode tree (-1 for roots); subtrees are contiguous
  std::vector<long long> sn_struct; // offset into structs (size nsuper+1)
  std::vector<int> structs;         // ND positions of struct(s), ascending
  // value offsets (doubles) into vals for each supernode's blocks (column-major)
  std::vector<long long> off_g, off_w, off_v;
  std::vector<double> vals;
  std::vector<int> pivrow;          // ND position of the t-th pivot row of each supernode (P_s; folded into G, W)
  int height = 0;
  double min_pivot = 0, max_pivot = 0;
  long long nnz_factor = 0;         // entries stored (G, W and V of every supernode)
};

// Host solve with the stored factors, in the same order the GPU uses
// (x = P^T U^{-1} L^{-1} P b); b and x in the original numbering.
void super_solve_host(const SuperLU& F, const std::vector<double>& b, std::vector<double>& x);

// A is square CSR (n x n) with coordinates per row for the geometric ND.
// Returns 0, or 1 if a pivot was zero / tiny (relative 1e-14).
int factor_nd(const std::vector<int>& ptr, const std::vector<int>& col, const std::vector<double>& val,
              const std::vector<int>& coords /* 3 per row */, SuperLU& out, int leaf_size, std::string* err);

}  // namespace ccmg
