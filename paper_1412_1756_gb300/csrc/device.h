// Device-side data of a plan and the launchers of its kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace mlfma {

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
inline bool byte_ranges_overlap(const void *a, int64_t na, const void *b, int64_t nb)
{
    const uintptr_t pa = reinterpret_cast<uintptr_t>(a), pb = reinterpret_cast<uintptr_t>(b);
    return na > 0 && nb > 0 && pa < pb + (uintptr_t)nb && pb < pa + (uintptr_t)na;
}

// Mesh and RWG data used by the FP64 setup kernels (leaf order for RWGs).
struct DevMesh {
    int nt = 0;
    const double *tq = nullptr;     // [nt][7][3] quadrature points
    const double *tv = nullptr;     // [nt][9]    vertices of each triangle
    const int32_t *tvi = nullptr;   // [nt][3]    vertex indices
    const double *area = nullptr;   // [nt]
    const double *cen = nullptr;    // [nt][3]
    const double *hmax = nullptr;   // [nt]
    int64_t n = 0;
    const int32_t *rtri = nullptr;  // [N][2] leaf order
    const double *rvf = nullptr;    // [N][2][3] free vertex coordinates
    const double *rlen = nullptr;   // [N]
};

struct DevNear {
    int nleaf = 0;
    const int32_t *box_ptr = nullptr;    // [nleaf+1]
    const int64_t *strip_off = nullptr;  // [nleaf+1]
    const int32_t *col_ptr = nullptr;    // [nleaf+1]
    const int32_t *strip_col = nullptr;  // columns (leaf-order unknowns)
    int max_cols = 0;                    // largest strip width
    int max_rows = 0;                    // largest leaf box
};

// One dense step of the tensor-core interpolation: the image of the step's
// matrix as the B operand of tcgen05.mma kind::tf32 (N rows of K values,
// K-major, 128-byte swizzle; TF32 hi part, then the lo part).
struct UmmaStep {
    int K = 0;            // contraction length (multiple of 8)
    int N = 0;            // output columns (multiple of 16)
    int kr0 = 0;          // theta steps: first K column of the block taken at phi + pi
    uint32_t kmask = 0;   // bit s set: K-step s (columns 8s .. 8s+7) holds a nonzero coefficient
    int off = 0;          // byte offset of the hi image in the level's image buffer (lo follows)
    int bytes = 0;        // bytes of one image: ceil(K / 32) * N * 128
};

// One tap shared by a pair of stencil rows: source index (as in Tap) and the
// coefficient of each row (zero where the tap is not one of that row's).
template <class R>
struct Tap2 {
    int32_t i;
    R c[2];
};

// One stencil tap: source index (theta stencils: bit 30 set = take the
// sample at phi + pi) and its coefficient.
template <class R>
struct Tap {
    int32_t i;
    R c;
};
constexpr int32_t kTapRefl = 1 << 30;

// A stencil's rows in groups of four on windows of consecutive source
// positions, for the FP32 windowed kernels: tap f of group g is position
// start[g] + f with coefficients coef[g * tw + f] (one per row of the
// group).  Periodic (phi) stencils: position e is sample e mod n.  Theta
// stencils: e in [0, n) is row e; e < 0 is row -e-1 and e >= n is row
// 2n-e-1, both at phi + pi (pole reflection; its sign is in the
// coefficients).
struct WinDev {
    int groups = 0, tw = 0;   // groups = 0: not available at this level
    const int32_t *start = nullptr;
    const float4 *coef = nullptr;
};

// One far level's tables in arithmetic type R (complex values as R pairs).
template <class R>
struct DevLevel {
    int nbox = 0, L = 0, nth = 0, nph = 0, K = 0, ntype = 0;
    const int32_t *il_ptr = nullptr, *il_src = nullptr, *il_type = nullptr;
    int nparent = 0, max_grp = 0;        // translation grouped by parent (level l-1)
    const int32_t *grp_ptr = nullptr, *grp_src = nullptr;
    const int16_t *grp_ty = nullptr;     // [entries][8]
    const int32_t *lty_ptr = nullptr, *lty = nullptr;   // per parent: distinct types used
    const int16_t *grp_lty = nullptr;    // [entries][8] index into the parent's type list, or -1
    int max_lty = 0;
    const int32_t *pchild_ptr = nullptr; // parent level's child ranges into this level
    const R *alpha = nullptr;            // [ntype][K][2]
    const R *alpha_dk = nullptr;         // [ntype][K][2] d alpha / dk (derivative tables, when set up)
    const int32_t *parent = nullptr;     // [nbox] into level l-1
    const int32_t *octant = nullptr;     // [nbox]
    const int32_t *child_ptr = nullptr;  // [nbox+1] into level l+1
    const R *shift = nullptr;            // [8][K][2] (parents only)
    const R *shift_dk = nullptr;         // [8][K][2] d shift / dk (parents only, when set up)
    const R *shift_xy = nullptr;         // [8][K][2] shift without its z factor (parents only)
    const R *gam = nullptr;              // [8][nth][2] the z factor, a function of theta (parents only)
    // the children in down-pass groups (parents only): a pair of siblings that
    // differ only in z (first, second), or one child (first, -1)
    const int2 *dgrp = nullptr;
    int ndgrp = 0;
    // to children (parents only): up stencils rows = this level's nth / nph;
    // down stencils rows = child nth / nph
    const int32_t *thu_ptr = nullptr, *thu_idx = nullptr, *thu_refl = nullptr;
    const R *thu_c = nullptr;
    const int32_t *phu_ptr = nullptr, *phu_idx = nullptr;
    const R *phu_c = nullptr;
    const int32_t *thd_ptr = nullptr, *thd_idx = nullptr, *thd_refl = nullptr;
    const R *thd_c = nullptr;
    const int32_t *phd_ptr = nullptr, *phd_idx = nullptr;
    const R *phd_c = nullptr;
    const Tap<R> *thu = nullptr, *phu = nullptr, *thd = nullptr, *phd = nullptr;   // packed taps
    // the interpolation stencils with the rows in pairs: per pair the union of
    // both rows' taps, one coefficient per row, zero-padded to up2_taps entries
    // (0: not built)
    const Tap2<R> *thu2 = nullptr, *phu2 = nullptr;
    int up2_taps = 0;
    // anterpolation stencils zero-padded to dn_taps taps per row (16, 20, 24 or 32)
    const Tap<R> *thd_pad = nullptr, *phd_pad = nullptr;
    int dn_taps = 0;
    // the same with the rows in pairs: per pair the union of both rows' taps
    // with one coefficient per row, zero-padded to dn2_taps entries (0: not built)
    const Tap2<R> *thd2 = nullptr, *phd2 = nullptr;
    int dn2_taps = 0;
    // the four stencils on windows (up theta, up phi, down phi, down theta)
    WinDev wu_th, wu_ph, wd_ph, wd_th;
    // FP32 parents: the interpolation (up: phi then theta) and anterpolation
    // (down: theta then phi) steps as dense matrices for the tcgen05 tensor
    // cores (null where a level's dimensions do not fit the kernels)
    const unsigned char *um_up = nullptr, *um_dn = nullptr;   // step 1 hi, lo, step 2 hi, lo
    int um_up_bytes = 0, um_dn_bytes = 0;
    UmmaStep um_up1, um_up2, um_dn1, um_dn2;
    int *um_err = nullptr;   // set to 1 by a tensor-core kernel whose bounded wait ran out
    int um_test = 0;         // test hook: the first CTA of a launch withholds its first arrival
    int up_order = 0;           // taps per forward stencil row (the interpolation order)
    const R *wq = nullptr;               // [K] quadrature weight (leaf: times -k^2 eta / 4 pi)
    R *S = nullptr;                      // outgoing field [nbox][2][K][B]
    R *G = nullptr;                      // incoming field [nbox][2][K][B]
};

// ------------------------------------------------------------ setup ---
cudaError_t launch_mesh_geometry(const double *V, const int32_t *T, int nt, double *tq, double *tv, double *area,
                                 double *cen, double *hmax, cudaStream_t s);
cudaError_t launch_near_fill(const DevMesh &m, const DevNear &nr, double k, double eta, double2 *val,
                             cudaStream_t s);
// near blocks of dZ/dk in the strip layout of launch_near_fill
cudaError_t launch_near_fill_dk(const DevMesh &m, const DevNear &nr, double k, double eta, double2 *val,
                                cudaStream_t s);
// mode 0: patterns V; 1: dV/dk; 2: dV/dk + (2/k) V
cudaError_t launch_leaf_patterns(const DevMesh &m, const int32_t *ubox, const double *box_center, int K,
                                 const double *grid /* [K][9]: khat, theta-hat, phi-hat */, double k, double2 *V, cudaStream_t s,
                                 int mode = 0);
cudaError_t launch_cast_c64_to_c32(const double2 *src, float2 *dst, int64_t n, cudaStream_t s);
// dst[i] = (Re src[i], 0) (part 0) or (Im src[i], 0) (part 1)
cudaError_t launch_part_c64(const double2 *src, double2 *dst, int64_t n, int part, cudaStream_t s);
cudaError_t launch_part_c32(const double2 *src, float2 *dst, int64_t n, int part, cudaStream_t s);

// ------------------------------------------------------------ product ---
// Launch choices of one product, 0 = the built-in heuristic; mlfma_tune
// picks them per (precision, columns) by timing the candidates.
struct Tuning {
    int near = 0;          // 1 / 2: one CTA per strip, 8 / 16 columns per thread; 3: 16-column chunks
    int radiate = 0;       // 1: one CTA per box; 2, 3, 4: 32, 16, 8 columns per CTA
    int receive = 0;       // 1, 2, 3: 32, 16, 8 columns per CTA
    int up_nb[22] = {};    // columns per CTA of the up pass into level l: 1, 2, 4, 8, 16
    int down_nb[22] = {};  // columns per CTA of the down pass from level l
    int tr[22] = {};       // translation at level l: 1 two columns per thread; 2..6 1, 2, 4, 8, 16 lanes per output
};

template <class R>
struct ProductArgs {
    int64_t n = 0;
    int B = 0;                 // internal real columns
    int leaf = 0, levels = 0;  // levels with far work: coarsest..leaf
    int coarsest = 2;          // 2 for the standard tree, 1 for the sibling scheme
    Tuning tune;
    DevNear nr;
    const R *near_val = nullptr;    // complex, strip layout
    const R *V = nullptr;           // leaf patterns [N][K][2] complex
    // derivative tables (set up on the first dZ/dk product in this precision)
    const R *near_dk = nullptr;     // near blocks of dZ/dk, strip layout
    const R *Vd = nullptr;          // dV/dk [N][K][2]
    const R *Wd = nullptr;          // dV/dk + (2/k) V [N][K][2]
    const int32_t *ubox = nullptr;  // [N] leaf box of each leaf-order unknown
    const int64_t *perm = nullptr;  // [N]
    R *xp = nullptr;                // [N][B] real
    R *yp = nullptr;                // [N][B] complex
    int *um_err = nullptr;          // set by a tensor-core kernel whose bounded wait ran out
    int umma = 0;                   // FP32 fields: 0 CUDA-core interpolation; 1 TF32, 3 3xTF32 tensor cores
    DevLevel<R> lv[22];
};

// Stage numbering of the per-stage timer (level-indexed stages add l).
enum {
    STAGE_PREPARE = 0, STAGE_NEAR = 1, STAGE_RADIATE = 2, STAGE_UP = 3, STAGE_TRANSLATE = 25,
    STAGE_DOWN = 47, STAGE_RECEIVE = 69, STAGE_FINALIZE = 70, STAGE_COUNT = 71
};

// Serial per-stage timing: an event recorded after every stage.
struct StageClock {
    cudaEvent_t start = nullptr;
    cudaEvent_t ev[96] = {};
    int stage[96] = {};
    int n = 0;
};

// Streams and events of the concurrent core pass (near || far chain, and
// each level's translation as soon as its outgoing field exists).
struct CoreStreams {
    cudaStream_t main = nullptr, far = nullptr, tr = nullptr;
    cudaEvent_t ev[64] = {};
};

// Kernel attributes (dynamic shared memory); call before launching or capturing.
template <class R>
cudaError_t prime_kernels();

// x (caller layout [N][Bu], real or complex) -> leaf-order real columns.
template <class R>
cudaError_t launch_prepare(const ProductArgs<R> &a, const void *x_user, int x_complex, int Bu, int adjoint,
                           cudaStream_t s);
// leaf-order complex columns -> y (caller layout [N][Bu]).
template <class R>
cudaError_t launch_finalize(const ProductArgs<R> &a, void *y_user, int x_complex, int Bu, int adjoint,
                            cudaStream_t s);
// near field and the whole far pass into a.yp.  With clk: everything on
// cs.main in order, an event after each stage.  Without: concurrent
// branches on the three streams, joined back into cs.main.
template <class R>
cudaError_t launch_core(const ProductArgs<R> &a, const CoreStreams &cs, StageClock *clk);
// (dZ/dk) x into a.yp: the near blocks of dZ/dk, and the far pass carried as
// value and k-tangent side by side (fields hold 2 a.B columns: value in
// [0, a.B), tangent in [a.B, 2 a.B)); on one stream, an event per stage
// with clk.
template <class R>
cudaError_t launch_core_dk(const ProductArgs<R> &a, cudaStream_t s, StageClock *clk);

// One stage of the core pass with a given choice (mlfma_tune): stage is
// STAGE_NEAR, STAGE_RADIATE, STAGE_RECEIVE, STAGE_UP + l, STAGE_TRANSLATE + l
// or STAGE_DOWN + l; `choice` as the matching Tuning field.  Returns an
// error for a choice that does not apply (the tuner skips it).
template <class R>
cudaError_t launch_stage(const ProductArgs<R> &a, int stage, int choice, cudaStream_t s);

// Tensor-core (tcgen05) interpolation and anterpolation of FP32 fields
// (umma_interp.cu).  cudaErrorInvalidConfiguration, with nothing launched,
// when the level has no tensor-core tables or does not fit the kernels.
cudaError_t launch_up_umma(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int acc, bool split,
                           cudaStream_t s);
cudaError_t launch_down_umma(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, bool split,
                             cudaStream_t s);

// Windowed CUDA-core interpolation and anterpolation of FP32 fields
// (window_interp.cu), NB = 4, 8 or 16 columns per CTA.
// cudaErrorInvalidConfiguration, with nothing launched, when the level has
// no windowed tables or does not fit the kernels.
cudaError_t launch_up_win(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int acc, int nb,
                          cudaStream_t s);
cudaError_t launch_down_win(const DevLevel<float> &P, const DevLevel<float> &Ch, int B, int Bs, int nb,
                            cudaStream_t s);
cudaError_t prime_win_kernels();

// Translation of FP32 fields grouped by parent, four columns per thread and
// the children four at a time (translate_quad.cu), NB = 16, 32 or 64
// columns per CTA.  cudaErrorInvalidConfiguration, with nothing launched,
// when the level's tables or shared memory do not fit the kernel.
cudaError_t launch_translate_quad(const DevLevel<float> &lv, int B, int Bs, int acc, int nb, cudaStream_t s);
cudaError_t prime_translate_quad();

// Reception of FP32 fields, two columns per thread with the field tile
// scaled by the weights as it is staged (leaf_pairs.cu), NB = 16, 32 or
// 64 columns per CTA.
cudaError_t launch_receive_pairs(const ProductArgs<float> &a, int Bs, int nb, cudaStream_t s);
// Radiation of FP32 fields, four columns and two samples per thread, 64
// columns per CTA (leaf_pairs.cu).
cudaError_t launch_radiate_quads(const ProductArgs<float> &a, int Bs, cudaStream_t s);
cudaError_t prime_receive_pairs();

}  // namespace mlfma
