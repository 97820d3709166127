// Host-side plan of the multilevel fast multipole product (FP64 tables).
// Section III-C: oct-tree with level 0 the enclosing cube; far work from
// level 2 to the leaf level; uniform phi / Gauss-Legendre theta sampling;
// local Lagrange interpolation between levels.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace mlfma {

using cd = std::complex<double>;

struct RwgList {
    std::vector<int32_t> edge_v;  // [N][2]  smaller, larger vertex index
    std::vector<int32_t> tri;     // [N][2]  T+, T-
    std::vector<int32_t> vfree;   // [N][2]  free vertex of T+, of T-
    std::vector<double> len;      // [N]
};

// Row-wise sparse stencil: row r uses entries ptr[r] .. ptr[r+1]-1.
struct Stencil {
    std::vector<int32_t> ptr;
    std::vector<int32_t> idx;
    std::vector<int32_t> refl;    // theta stencils: 1 = sample taken at phi + pi
    std::vector<double> coef;     // pole reflection sign folded in
};

// A stencil's rows in groups of kWinRows, each group's taps placed on one
// window of consecutive source positions (tw wide, tap f at position
// start + f), with one coefficient per row of the group (zero where a row
// has no tap at that position).  Periodic (phi) stencils over n source
// samples: position e is sample e mod n, start in [0, n).  Theta stencils:
// position e in [0, n) is sample e; e < 0 is sample -e-1 and e >= n is
// sample 2n-e-1, both taken at phi + pi (the pole reflection, whose sign
// is already in the coefficient); start >= -n and start + tw <= 2n.
constexpr int kWinRows = 4;
struct WinStencil {
    int groups = 0;                 // ceil(rows / kWinRows); 0: not built (a window wider than allowed)
    int tw = 0;                     // window width
    std::vector<int32_t> start;     // [groups]
    std::vector<double> coef;       // [groups][tw][kWinRows]
};

// Builds W from S (n source samples).  False, with W.groups = 0, when a
// group's window would be wider than tw_max (or than n for phi).
bool win_stencil(const Stencil &S, int n, bool theta, int tw_max, WinStencil &W);

struct Level {
    int l = 0;
    double a = 0.0;                 // box side
    // sampling grid (levels with far work)
    int L = 0, nth = 0, nph = 0, K = 0;
    std::vector<double> ct, th, wt, ph;   // cos theta, theta, GL weight, phi
    // boxes
    std::vector<uint64_t> code;     // occupied boxes, Morton order
    std::vector<double> center;     // [nbox][3]
    std::vector<int32_t> parent;    // index into level l-1
    std::vector<int32_t> octant;    // position within the parent (x<<2 | y<<1 | z)
    std::vector<int32_t> child_ptr; // [nbox+1] range in level l+1
    // translation (l >= 2)
    std::vector<int32_t> il_ptr, il_src, il_type;
    // the same lists grouped by parent (level l-1): for parent P, entries
    // grp_ptr[P] .. grp_ptr[P+1]-1 name a source box and, for each of P's
    // children (slot 0..7 in child order), the translation type or -1
    std::vector<int32_t> grp_ptr, grp_src;
    std::vector<int16_t> grp_ty;    // [entries][8]
    int max_grp = 0;
    // per parent, the distinct translation types its entries use
    // (lty[lty_ptr[P] ..]) and each entry slot's index into that list or -1
    std::vector<int32_t> lty_ptr, lty;
    std::vector<int16_t> grp_lty;   // [entries][8]
    int max_lty = 0;
    std::vector<int32_t> type_off;  // [ntype][3]
    int ntype = 0;
    std::vector<cd> alpha;          // [ntype][K]
    std::vector<cd> alpha_dk;       // [ntype][K]: d alpha / dk
    // alpha = alpha_j + i alpha_y: the j_l and y_l halves of Eq. (8),
    // sum i^l (2l+1) j_l P_l and sum i^l (2l+1) y_l P_l (translation of the
    // sin(kR)/R and cos(kR)/R kernels, Eqs. (SinKer), (CosKer), up to -i, i)
    std::vector<cd> alpha_j, alpha_y;
    // to/from children (2 <= l < leaf)
    std::vector<cd> shift;          // [8][K]: exp(i k khat.(r_parent - r_child))
    std::vector<cd> shift_dk;       // [8][K]: d shift / dk = i khat.(r_parent - r_child) shift
    // the shift split as shift = shift_xy(theta, phi) * gam(theta): the factor of
    // the z offset depends on theta alone, so two children that differ only in
    // z can share the phi interpolation (after theta, before phi)
    std::vector<cd> shift_xy;       // [8][K]: exp(i k (khat_x d_x + khat_y d_y))
    std::vector<cd> gam;            // [8][nth]: exp(i k cos(theta) d_z)
    Stencil th_up, ph_up;           // child grid -> this grid (rows: nth / nph of this level)
    Stencil ph_dn, th_dn;           // weighted transposes (rows: child nph / child nth)
    WinStencil wu_th, wu_ph, wd_ph, wd_th;   // the four stencils above on windows (kernels that take taps at fixed offsets)
    int nbox() const { return (int)code.size(); }
};

// Translations between sibling boxes at one level (the sin-kernel product
// of Eq. (RI): every pair of distinct leaf boxes is translated once, at the
// level where their ancestors are siblings; coarsest level 1).
struct SibLevel {
    int ntype = 0;
    std::vector<int32_t> type_off;           // [ntype][3] r_m - r_m' in boxes
    std::vector<int32_t> grp_ptr, grp_src;   // per parent (level l-1): its children as sources
    std::vector<int16_t> grp_ty;             // [entries][8] type per child slot or -1 (itself)
    int max_grp = 0;
    std::vector<cd> alpha;                   // [ntype][K] sum i^l (2l+1) j_l(k r) P_l
};

struct PlanHost {
    // inputs
    std::vector<double> V;          // [nv][3]
    std::vector<int32_t> T;         // [nt][3]
    double k = 0, digits = 3, eta = 376.730313668;
    int levels = 0, leaf = 0, order = 6;
    // derived
    RwgList rwg;
    int64_t N = 0;
    double root_side = 0, root_center[3] = {0, 0, 0}, origin[3] = {0, 0, 0};
    std::vector<int64_t> perm;      // leaf-order position -> canonical index
    std::vector<int32_t> leaf_box;  // canonical index -> leaf box
    std::vector<int32_t> box_ptr;   // [nleaf+1] positions in leaf order
    std::vector<Level> lv;          // [levels]; level 1 carries a grid and stencils for the sibling scheme
    std::vector<SibLevel> sib;      // [levels], used for 1 <= l <= leaf
    // near field: per leaf box, a dense strip [rows of the box] x
    // [columns of all neighbour boxes], column-major
    std::vector<int32_t> nb_ptr, nb_box;
    std::vector<int64_t> strip_off; // [nleaf+1] element offsets
    std::vector<int32_t> col_ptr;   // [nleaf+1] into strip_col
    std::vector<int32_t> strip_col; // leaf-order unknown of each strip column
    // self strips (the leaf box's own columns): the near part of Eq. (RI)
    std::vector<int64_t> self_off;  // [nleaf+1]
    std::vector<int32_t> self_col_ptr, self_col;
    int64_t self_nnz = 0;
    int64_t nnz = 0;
    int max_leaf = 0;
};

// Builds everything above from (verts, tris).  Returns "" or an error text.
std::string build_plan_host(PlanHost &P, const double *verts, int64_t nv, const int32_t *tris,
                            int64_t nt, double k, int levels, double digits, int order, double eta);

// Truncation number of Section V, Eq. (9), d = sqrt(3) a.
int truncation_number(double k, double a, double digits);

// Special functions (FP64), exported for the plan's own use.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w);
void sph_bessel_j(int nmax, double x, std::vector<double> &j);
void sph_bessel_y(int nmax, double x, std::vector<double> &y);

}  // namespace mlfma
