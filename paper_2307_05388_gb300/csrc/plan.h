// Symbolic phase (paper Sec. II, "symbolic factorization"; Fig. 1): the
// sparsity pattern of A depends only on the grid, never on eps or omega, so
// the elimination order, the elimination tree, the front structure and every
// index map are computed once on the host and reused for all wavelengths and
// all design iterations.
//
// Ordering: geometric nested dissection of the nx x ny grid.  A rectangle is
// split by a full grid line (the separator) into two rectangles.  Rectangles
// that straddle the edge of the design box are split on the line just outside
// the box, so that every leaf subtree lies wholly inside or wholly outside the
// design box; this is what lets a design update refactor only the fronts on the
// paths from design pixels to the root.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace fdfd {

// Direction codes of one stencil entry A[row][col]: col = row + offset.
enum StencilDir { DIR_DIAG = 0, DIR_XM = 1, DIR_XP = 2, DIR_YM = 3, DIR_YP = 4 };

struct FrontDesc {           // plain-old-data, uploaded to the device as is
  int k;                     // pivots (fully summed variables) of this front
  int m;                     // boundary variables (eliminated in ancestors)
  int n;                     // k + m
  int ld;                    // row stride of the dense front (elements)
  long long st_off;          // element offset of the dense front in front storage
  long long v_off;           // element offset of the front vector (n entries) per RHS
  int idx_off;               // offset into idx: n grid cells (k pivots, then m boundary)
  int inv_off;               // offset into inv: n_parent entries (parent local -> my boundary t, or -1)
  int orig_off;              // offset into orig_ptr: n + 1 row pointers into orig entries
  int piv_off;               // offset into perm: k entries
  int parent;                // -1 for a root
  int child0;                // offset into children
  int nchild;
  int level;                 // 0 for leaves; parent level > child level
  int design;                // 1 if the subtree holds a design pixel (refactored on design change)
  int ldk;                   // row stride of the k x k inverse block (k rounded up to 4)
  long long iv_off;          // element offset of the inverse block (L11^-1 strictly lower, U11^-1 upper)
};

struct Plan {
  int nx = 0, ny = 0;
  int bx0 = 0, by0 = 0, bw = 0, bh = 0;
  int leaf_area = 0;
  std::vector<FrontDesc> fronts;      // postorder: children precede parents
  std::vector<int> children;
  std::vector<int> idx;               // grid cells of each front
  std::vector<int> inv;               // extend-add inverse maps
  std::vector<int> orig_ptr;          // per front: n+1 offsets (absolute) into orig_entries
  std::vector<int> orig_col;          // local column of each original entry
  std::vector<int> orig_code;         // cell * 5 + direction of each original entry
  std::vector<int> pos;               // elimination position of each grid cell
  int n_levels = 0;
  std::vector<std::vector<int>> level_fronts;  // front ids per level
  long long store_total = 0;          // elements of front storage per omega
  long long inv_total = 0;            // elements of the triangular-inverse storage per omega
  long long vec_total = 0;            // elements of front vectors per RHS per omega
  int perm_total = 0;
  double flops_factor = 0;            // complex LU flops (8 real flops per complex FMA)
  double flops_design = 0;            // same, restricted to design-affected fronts
  long long factor_entries = 0;       // stored L and U entries (k*k + 2*k*m per front)
  int max_front = 0;
};

// Builds the plan.  Returns an empty string on success, otherwise an error message.
std::string build_plan(int nx, int ny, int bx0, int by0, int bw, int bh, int leaf_area, Plan* out);

// Checks the plan's invariants (every original entry assembled once, injective
// extend-add maps, boundary eliminated after pivots).  Empty string when valid.
std::string validate_plan(const Plan& p);

}  // namespace fdfd
