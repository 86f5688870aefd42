// Host-side construction of the multigrid hierarchy (setup phase, FP64).
// Everything the device kernels read is produced here once and uploaded.
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <array>
#include <type_traits>
#include <utility>
#include <vector>

#include "geometry.hpp"

namespace cutmg {

// Allocator for the large host arrays whose every element the setup writes
// itself, block by block in parallel: resize leaves the new elements
// uninitialised instead of zero-filling them on one thread.
template <class T>
struct DefaultInitAllocator : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = DefaultInitAllocator<U>;
  };
  DefaultInitAllocator() noexcept = default;
  template <class U>
  DefaultInitAllocator(const DefaultInitAllocator<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
using HostBlocks = std::vector<double, DefaultInitAllocator<double>>;

constexpr uint8_t kFlagActive = 1;
constexpr uint8_t kFlagCut = 2;

struct SetupParams {
  int dim = 3, degree = 2, n_cells = 16, n_levels = 2;
  double lo = -1.0, hi = 1.0;
  double gamma_D = 80.0;
  double gamma_ghost[4] = {0.1, 0.1, 0.1, 0.1};
  int n_c = 2;
  int quad_q = 4;
  int smoother = 0;     // 0 vertex-patch smoother, 1 Chebyshev
  int cheb_degree = 5;
  // sizes only: classification, DoFs, faces and patch lists, but no cut-cell
  // quadrature, no element matrices, no inverses and no right-hand side
  // (what a device-footprint estimate needs before a full setup)
  bool dry = false;
  // the cut-patch inverses of the block kernel ((2p+1)^d > 64) are formed on
  // the device (FP64) from the assembled A_j; the host then keeps A_j (packed
  // in the records, full in inv) instead of the inverse
  bool device_inverse = false;
  LevelSet ls;
};

// One level of the hierarchy in lattice ("box") layout: every vector lives on
// the full (pN+1)^d node lattice; inactive nodes stay zero.
struct HostLevel {
  int d = 3, p = 2, N = 0, n = 0;  // cells and nodes per direction
  double h = 0.0, lo = -1.0;
  // cells
  std::vector<uint8_t> cflag;   // N^d: kFlagActive | kFlagCut
  std::vector<int> cut_id;      // N^d: row block in cutmat or -1
  HostBlocks cutmat;            // [n_cut][NB][NB] volume + Nitsche terms
  int64_t n_cut = 0, n_active = 0, n_ghost = 0;
  bool inv_on_device = false;   // inv / rec hold A_j, inverted by the engine (SetupParams::device_inverse)
  int64_t n_inv = 0;            // entries of the cut-patch inverse storage (inv.size() unless dry)
  // nodes
  std::vector<uint8_t> nact;    // n^d: node belongs to an active cell
  std::vector<int64_t> dofs;    // lattice index of each DoF (ascending)
  int bb_lo[3] = {0, 0, 0}, bb_hi[3] = {0, 0, 0};  // inclusive node bbox of the DoFs
  // matrix-free apply: positions a own the nodes p a + alpha, alpha in
  // [0, p)^d; bulk positions have 2^d plain interior cells around them
  std::vector<int> bulk_pos;    // packed a_0 + (N+1)(a_1 + (N+1) a_2)
  std::vector<int> bnd_node;    // active nodes not owned by a bulk position
  // ghost faces (c, c + e_k): packed c * d + k, and the id of each face per cell
  std::vector<int> ghost_faces;
  std::vector<int> face_id;     // N^d * d, -1 where (c, c + e_k) is not a ghost face
  // patches (sorted by colour; start offsets per colour, 2^d + 1 entries)
  std::vector<int> cart_vert;   // packed vertex v_0 + (N+1)(v_1 + (N+1) v_2)
  std::vector<int> cart_start;
  std::vector<int> cut_vert, cut_n, cut_moff;
  std::vector<int64_t> cut_ioff;  // inverse offsets, multiples of 4 elements
  std::vector<int> cut_maxm2;     // per colour: largest m^2 of its cut patches
  std::vector<int> cut_maxit;     // per colour: most row items of one of its cut patches
  std::vector<int> cut_start;
  std::vector<uint16_t> members;  // closure-local node index per cut-patch DoF
  std::vector<int> member_node;   // lattice index per cut-patch DoF
  // ghost-face terms of each cut-patch DoF's row: entries fent[fofs[i] ..
  // fofs[i+1]) = (face id * (p+1)^(d-1) + t) * 16 + i_k, and per colour the
  // ghost faces those rows need (colour c: cfaces[cf_start[c] .. cf_start[c+1]))
  std::vector<int> fofs, fent;
  std::vector<int> cfaces, cf_start;
  // per cut patch j: its ghost-face entries are fent[cut_fo[j] .. cut_fo[j+1]);
  // cut_cell[j * 2^d + s] = cut-cell matrix of patch cell s (-1 uncut, -2
  // inactive); cut_items[cut_item_off[j] ..] = s * NB + i for the rows
  // (patch cell s, local node i) that belong to a patch DoF
  std::vector<int> cut_fo, cut_cell, cut_item_off;
  std::vector<uint8_t> cut_items;
  HostBlocks inv;                 // explicit FP64 inverses A_j^{-1}, row-major
  // Per cut patch record of the record kernel ((2p+1)^d > 64, i.e. 3D Q2):
  // rec[cut_roff[j] ..] = the inverse by rows with row stride MP = 4 ceil(m /
  // 4) (entry (i, c) at i MP + c; zeros in the padding), then the rows of the
  // cut-cell matrices its items use, in item order, each NB entries padded
  // with zeros to NBP = 4 ceil(NB / 4) (16-byte rows in FP32 and FP64);
  // cut_roff[j + 1] - cut_roff[j] = its length = m MP + rows NBP.
  // cut_pk[j * 2^d + s] = -2 inactive cell, -1 uncut, else (r0 << 8) | q0:
  // the first pack row r0 and first item q0 of cut patch cell s.
  // cut_gmask[j] bit (k * 3 + L) * 2^(d-1) + u: the face normal to k on
  // cell-layer plane L of the patch block (0 lower boundary, 1 middle, 2
  // upper boundary) at tangential cell u is a ghost face.
  std::vector<int64_t> cut_roff;
  std::vector<int> cut_pk;
  std::vector<uint64_t> cut_gmask;
  std::vector<int> cut_maxrec;    // per colour: longest record
  HostBlocks rec;
  int64_t n_rec = 0;              // rec.size() unless dry
  // Moments of the ghost faces on the block's boundary planes (computed by a
  // separate launch from the x before the colour step: the cell across such a
  // face can hold DoFs of a same-colour patch): patch j reads them from
  // slots cut_gboff[j] .. cut_gboff[j + 1] (one per set boundary bit of
  // cut_gmask[j], in bit order; P (p+1)^(d-1) values each).  Per colour c the
  // faces to compute are bf_face[bf_start[c] .. bf_start[c + 1]) (ghost-face
  // ids) with their slots bf_dst[2 i], bf_dst[2 i + 1] (-1: none).
  std::vector<int> cut_gboff, bf_start, bf_face, bf_dst;
  // Ghost-entry lists of the cut patches: patch j's run cut_gent[cut_geoff[j]
  // .. cut_geoff[j + 1]) (a multiple of 8 entries) holds m + 1 row offsets,
  // then per DoF row (member order) the ghost faces whose stencil contains
  // the DoF: slot | (i << 6) | (t << 10), with i the node along the face's
  // normal, t the tangential node and slot the face's moment slot in the
  // patch: the set block-boundary bits of cut_gmask[j] first (bit order, the
  // order of its cut_gboff slots), then the set middle-plane bits (bit
  // order).
  std::vector<int> cut_geoff;
  std::vector<uint16_t> cut_gent;
  // algorithmic work per launch, used to report achieved FLOP/s and bytes:
  // per colour of the cut-patch solve and of the interior-patch step
  // {flops, scalars moved, index bytes moved}
  std::vector<std::array<double, 3>> work_cut, work_cart, work_face;
  // reference tables
  std::vector<double> Kref;       // NB x NB stiffness of an uncut cell
  std::vector<double> Kunit;      // the same for h = 1: Kref = kscale Kunit, kscale = h^(d-2)
  double kscale = 1.0;
  std::vector<double> Mr, Kr;     // M x C rows of the two-cell 1D mass / stiffness
  std::vector<double> S, lam;     // fast-diagonalisation eigenvectors / values (M)
  std::vector<double> Wcart;      // (2p-1)^d x (2p+1)^d dense interior-patch update
  std::vector<double> diag;       // diagonal of A_l per DoF (levels >= 1)
  double dvec[4][9] = {};         // ghost normal-derivative jump weights (m = 1..p, 2p + 1 nodes)
  double coef[4] = {};            // gamma_m h^(2m-1)/(m!)^2 * h^(d-1)
  double Mhat[5][5] = {};         // reference 1D mass on [0, 1]
  // transfer from the next coarser level (l >= 1)
  std::vector<int> pro_col;       // n x (p+1): coarse 1D column per fine 1D index
  std::vector<double> pro_w;
  std::vector<int> res_col;       // n_coarse x (4p+1): fine columns per coarse index
  std::vector<double> res_w;
  // coarsest level
  std::vector<double> coarse_inv; // ndof x ndof explicit inverse (row-major)
};

struct Hierarchy {
  SetupParams prm;
  std::vector<HostLevel> levels;
  std::vector<double> rhs;  // finest-level manufactured right-hand side (per DoF)
};

// Builds the hierarchy.  Throws std::runtime_error with a message on error.
void build_hierarchy(const SetupParams& prm, Hierarchy& H);

// finest-level right-hand side b_i = (f, phi_i)_Omega + (g, gamma_D/h phi_i
// - d_n phi_i)_Gamma for user data (f, g called sequentially on the calling
// thread with a 3-component point; a null function is zero)
void build_rhs_user(const Hierarchy& H, double (*f)(const double*, void*), double (*g)(const double*, void*),
                    void* user, std::vector<double>& b);

}  // namespace cutmg
