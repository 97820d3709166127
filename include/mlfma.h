/*
 * mlfma.h - C ABI of the GB300 (sm_103a) multilevel fast multipole matrix-
 * vector product for the Galerkin EFIE with RWG basis functions on a
 * triangulated PEC surface.
 *
 * The product is y = Z x with Z_ij = i k eta < f_i, G, f_j > (Section II,
 * Eq. (5)), G = [I - grad grad'/k^2] exp(ikR)/R (Eqs. (2)-(3)): no 1/(4 pi),
 * time convention exp(-i w t).  Characteristic-mode analysis uses
 * R = -Re Z (positive semidefinite) and X = Im Z; for a real x these are
 * -Re(Z x) and Im(Z x).
 *
 * Z x is split as in the two-level formula (Section III-B, Eq. (ZI)): an
 * explicitly stored near-field part over each leaf group's neighbours B_m,
 * and a far part evaluated by aggregation, translation (Section III-A,
 * Eqs. (7)-(8)) and disaggregation, extended over an oct-tree with
 * interpolation and anterpolation between levels (Section III-C).
 *
 * Conventions for every entry point
 * - Every function returns an mlfma_status; none aborts, traps or exits.  On
 *   failure a message is kept per thread and returned by mlfma_last_error().
 * - Mesh arrays are host memory, read during mlfma_plan() only.
 * - Vector arguments of mlfma_matvec*() are DEVICE pointers on the plan's
 *   device, row-major [N][B] with the batch index innermost, in canonical
 *   RWG order (below).  mlfma_matvec_host() takes HOST pointers instead.
 * - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *   void*, NULL = legacy default stream); device-side failures surface at the
 *   next call on the plan or at mlfma_sync().
 * - A plan is not thread-safe: serialise calls on one plan; calls on
 *   different plans may run concurrently.
 *
 * Canonical RWG order: one basis function per edge shared by exactly two
 * triangles, edges sorted by (smaller vertex index, larger vertex index).
 * T+ is the triangle whose vertex cycle runs along the edge from the smaller
 * to the larger index; f = +l/(2A+) (r - v+) on T+ and -l/(2A-) (r - v-) on
 * T-.  Boundary edges carry no function; an edge on three or more triangles,
 * or with both triangles running the same way along it, is MLFMA_EINVAL.
 */
#ifndef MLFMA_H
#define MLFMA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlfma_plan_s *mlfma_plan_t;   /* opaque; owns all memory it allocates */

typedef enum {
    MLFMA_OK = 0,
    MLFMA_EINVAL = 1,    /* bad argument, mesh or size */
    MLFMA_ENOMEM = 2,    /* host or device allocation failed */
    MLFMA_ECUDA = 3,     /* a CUDA runtime call failed; message has the CUDA error */
    MLFMA_ENOTCONV = 4,  /* reserved for iterative solvers */
    MLFMA_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
    MLFMA_ENOTSUP = 6    /* valid request the library does not support */
} mlfma_status;

/* Arithmetic of a product.  MLFMA_FP64: complex FP64 everywhere (near field,
 * radiation patterns, translations, interpolation, accumulation).
 * MLFMA_FP32: complex FP32 near field, patterns, translation tables and
 * fields, FP32 interpolation coefficients, FP32 accumulation; the tables are
 * built in FP64 and rounded once.
 * MLFMA_MIXED_TF32 / MLFMA_MIXED_3XTF32: MLFMA_FP32, except that the local
 * interpolation and anterpolation between levels (Section III-C) run as dense
 * products on the tensor cores (tcgen05.mma kind::tf32, FP32 accumulation in
 * tensor memory): one TF32 product (operands truncated to 10 mantissa bits),
 * or three (hi/lo split of both operands, accurate to FP32 rounding).  They
 * use the FP32 tables of the plan and apply to Z products (mlfma_matvec,
 * mlfma_matvec_adjoint, mlfma_matvec_host, mlfma_profile_stages); other
 * entry points return MLFMA_ENOTSUP.  Levels whose grids exceed the
 * tensor-core kernels' limits use the FP32 CUDA-core kernels.  A tensor-core
 * kernel whose bounded wait ran out is reported as MLFMA_ETIMEOUT by the
 * next mlfma_sync (or by mlfma_matvec_host, which waits). */
typedef enum { MLFMA_FP64 = 0, MLFMA_FP32 = 1, MLFMA_MIXED_TF32 = 2, MLFMA_MIXED_3XTF32 = 3 } mlfma_prec;

typedef struct {
    int interp_order;   /* points per dimension of the local Lagrange
                           interpolation between levels (Section III-C);
                           even, 4..12; default 10 */
    int max_batch;      /* largest B (real columns; a complex column counts
                           two) a product may use; fields are sized for it;
                           1..4096, default 64 */
    int precisions;     /* bit mask (1 << mlfma_prec) of arithmetic to set up;
                           default both */
    int host_only;      /* 1: build the host tables only and never touch a
                           GPU (for inspection with mlfma_export); products
                           are refused with MLFMA_EINVAL */
    int device;         /* CUDA device ordinal; -1 = the current device */
    double eta;         /* wave impedance eta in Eq. (1); default 376.730313668 */
} mlfma_opts;

/* Fill *opts with the defaults above.  Always MLFMA_OK unless opts is NULL. */
mlfma_status mlfma_default_opts(mlfma_opts *opts);

/*
 * Build a plan: RWG list, oct-tree (Section III-C: level 0 is the cube
 * enclosing the mesh, each level halves the box side; `levels` counts level
 * 0, like Table II's nlv), near lists, sampling grids, interpolation
 * stencils, translation tables (Eq. (8)), and on the GPU the FP64 near-field
 * blocks (with singularity extraction) and leaf radiation patterns.
 *
 *  verts  [nv][3] float64, metres            tris  [nt][3] int32, 0-based
 *  k      wavenumber (rad/m), > 0            levels  2..21
 *  digits d0 of the truncation number L = ceil(k d + 1.8 d0^(2/3) (k d)^(1/3)),
 *         d = sqrt(3) a for box side a (Section V, Eq. (9)); 1..15
 *  opts   NULL for defaults
 *  out    receives the plan; untouched on failure
 * Far interactions start at level 2 (Section III-C).  The root cube's side is
 * the mesh's largest bounding-box extent; an RWG belongs to the leaf box
 * holding its edge midpoint (faces belong to the upper box).
 * Errors: EINVAL (arguments, mesh), ENOMEM, ECUDA.
 */
mlfma_status mlfma_plan(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                        double k, int levels, double digits, const mlfma_opts *opts,
                        mlfma_plan_t *out);

/* Number of unknowns N (RWG functions). */
mlfma_status mlfma_num_unknowns(mlfma_plan_t plan, int64_t *n);

/* Canonical RWG list: edge_v [N][2] (smaller, larger vertex index) and
 * tri_pm [N][2] (T+, T-), both host int32 arrays of the caller. Either may be
 * NULL. */
mlfma_status mlfma_rwg_edges(mlfma_plan_t plan, int32_t *edge_v, int32_t *tri_pm);

/*
 * y = Z x on the GPU (Eq. (ZI), multilevel).
 *  x      device, [N][B]: float (FP32) or double (FP64) real values; or, when
 *         x_is_complex, interleaved complex [N][B] of that real type
 *  y      device, [N][B] interleaved complex of the same real type; must not
 *         overlap x
 *  B      columns, 1..max_batch (complex x: 1..max_batch/2)
 *  prec   an mlfma_prec set up in the plan
 *  stream cudaStream_t or NULL
 * Asynchronous.  The near field and the far pass are captured into a CUDA
 * graph on the plan's own streams the first time a (precision, column
 * count) pair is used and replayed afterwards; the graph's branches (near
 * field, aggregation, per-level translations) run concurrently and join
 * back into `stream`.  Errors: EINVAL (sizes, precision not set up,
 * host-only plan), ECUDA.
 */
mlfma_status mlfma_matvec(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                          int64_t B, int prec, void *stream);

/*
 * y = Z^H x.  Z is symmetric (Z = Z^T, Section II; the near blocks are
 * symmetrised explicitly), so Z^H x = conj(Z conj(x)): the same pass with
 * the input and output conjugated.  Arguments as mlfma_matvec.
 */
mlfma_status mlfma_matvec_adjoint(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                                  int64_t B, int prec, void *stream);

/*
 * y = (dZ/dk) x: the wavenumber derivative of the EFIE matrix of Section II,
 * Eq. (5), applied through the multilevel product of Eq. (ZI), with the
 * plan's quadrature, tree, sample grids, stencils and truncation numbers
 * held fixed.  Near blocks: i eta (A + Phi/k^2) + i k eta (A' - Phi'/k^2),
 * A and Phi the vector- and scalar-potential integrals of Z and A', Phi'
 * those of dg/dk = i exp(ikR).  Far part: every stage of Eq. (ZI) carried as
 * value and k-tangent (dual numbers): derivative patterns, shifts
 * (i khat.d exp(i k khat.d)), translations (Eq. (8) with r h_l'(kr)) and
 * the far constant (-2 k eta / 4 pi).
 * Arguments, layouts and stream behaviour as mlfma_matvec, except that the
 * fields carry 2 x the internal columns: B must satisfy 2 B <= max_batch
 * (complex x: 4 B <= max_batch).  The first call in a precision builds the
 * derivative tables (one FP64 near-field fill and two pattern tables; it
 * allocates device memory and synchronises the device), so make it outside
 * any stream capture; later calls replay a captured graph per column count.
 * Errors: EINVAL (sizes, precision not set up, host-only plan), ENOMEM,
 * ECUDA.
 */
mlfma_status mlfma_matvec_dk(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                             int64_t B, int prec, void *stream);

/*
 * y = (dZ/dk)^H x = conj((dZ/dk) conj(x)) (dZ/dk is symmetric like Z).
 * Arguments as mlfma_matvec_dk.
 */
mlfma_status mlfma_matvec_dk_adjoint(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                                     int64_t B, int prec, void *stream);

/*
 * y = X x with X = Im Z (Section IV, the reactance matrix), by the
 * cos(kR)/R kernel of Eq. (CosKer) in the multilevel product of Eq. (XI):
 * the same tree, lists and grids as mlfma_matvec, near blocks Im Z, and the
 * translation table of Eq. (CosKer) (spherical Neumann functions y_l).  As
 * Section V's point test shows, the expansion is accurate only where the
 * addition theorem holds and the leaf boxes are not small: below about half
 * a wavelength the y_l terms grow and the product loses accuracy (the
 * low-frequency breakdown the paper assigns to LF-FMA).  For real x the
 * result is real up to quadrature rounding; y is returned complex.
 * Arguments as mlfma_matvec.  The first call in a precision builds the
 * tables (an FP64 near-field fill; allocates and synchronises the device).
 * Errors as mlfma_matvec.
 */
mlfma_status mlfma_matvec_x(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                            int64_t B, int prec, void *stream);

/*
 * y = R x with R = Re Z (Section IV, the resistance matrix as the paper
 * defines it; the characteristic-mode pencil uses -R, see cm_ira_solve), by
 * the sin(kR)/R kernel of Eq. (SinKer) in the multilevel form of Eq. (RI):
 * the near part is each leaf box with itself only; every other pair of
 * leaf boxes is translated once, at the level where their ancestors are
 * siblings (boxes with the same parent), level 1 being the coarsest, with
 * the spherical-Bessel table of Eq. (SinKer).  The regular kernel has no
 * addition-theorem restriction, so nearby boxes translate too.  Needs a plan
 * with at least 3 levels (MLFMA_ENOTSUP otherwise).  Arguments, result type
 * and first-call behaviour as mlfma_matvec_x.
 */
mlfma_status mlfma_matvec_r(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                            int64_t B, int prec, void *stream);

/*
 * y = Z x with HOST x and y (same layouts and types as mlfma_matvec): copies
 * x to the device, runs the product on `stream`, copies y back and waits for
 * the stream.  Uses the plan's own device staging buffers.
 */
mlfma_status mlfma_matvec_host(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                               int64_t B, int prec, void *stream);

/*
 * Autotuning of the launch choices (no counterpart in the paper): for the
 * product y = Z x with B columns (complex x: 2B internal columns) in `prec`,
 * every stage's candidate launch shapes - near field (one CTA per strip with
 * 8 or 16 columns per thread, or 16-column chunks), radiation and reception
 * tile widths, per level the column chunk of the up and down passes and the
 * translation's columns or lanes per output - are timed serially with CUDA
 * events on `stream` (one warm-up launch, then three) after one full pass,
 * and the fastest kept for later mlfma_matvec / adjoint / profile calls
 * with the same (prec, columns); a captured graph for them is re-captured.
 * ms_default / ms_tuned (may be NULL) receive the sums of the stage times
 * with the built-in and with the chosen shapes.  A candidate that does not
 * apply to the plan (its launcher refuses it or the launch is rejected) is
 * skipped; the call fails only when the built-in pass fails or a timed
 * launch faults.  A built-in shape is kept unless a candidate is at least
 * 2 % faster.  Synchronous; overwrites the plan's internal buffers.
 * Errors: EINVAL (host-only plan, B outside 1..max_batch, precision not set
 * up), ECUDA.
 */
mlfma_status mlfma_tune(mlfma_plan_t plan, int64_t B, int x_is_complex, int prec, void *stream,
                        double *ms_default, double *ms_tuned);

/*
 * Read or pin the launch shapes used for (B, x_is_complex, prec) as
 * MLFMA_TUNE_FIELDS int32 values (0 = the built-in choice):
 *   [0] near field: 1 / 2 one CTA per strip with 8 / 16 columns per thread,
 *       3 chunks of 16 columns
 *   [1] radiation: 1 one CTA per box, 2 / 3 / 4 tiles of 32 / 16 / 8 columns,
 *       5 four columns and two samples per thread, 64 columns per CTA (FP32
 *       only)
 *   [2] reception: 1 / 2 / 3 tiles of 32 / 16 / 8 columns; 4 / 5 / 6 two
 *       columns per thread with the field tile scaled by the weights as it
 *       is staged, 64 / 32 / 16 columns per CTA (FP32 only)
 *   [3 + l]       up pass into level l: columns per CTA 1..16, or 202 / 204 /
 *                 208 / 216 with 2 / 4 / 8 / 16 columns and the interpolation
 *                 rows taken in pairs (FP32 only), or 304 / 308 / 316 the
 *                 windowed kernel (rows in groups of four on windows of
 *                 consecutive source samples, MLFMA_X_WIN_SHAPE) with
 *                 4 / 8 / 16 columns, 404 / 408 the same with 4 / 8 columns
 *                 and a register budget for one more CTA per SM, 704 / 708 /
 *                 716 the windowed kernel with the children that differ only
 *                 in z sharing one phi step (the shift split into a theta-only
 *                 z factor and the rest), 4 / 8 / 16 columns (FP32 only)
 *   [3 + 22 + l]  down pass from level l: columns per CTA 1..16 (one CTA per
 *                 child), 104 / 108 one CTA per parent with 4 / 8 columns,
 *                 204 / 208 / 216 one CTA per child with 4 / 8 / 16 columns and
 *                 the anterpolation rows taken in pairs (FP32 only), or
 *                 304 / 308 / 316 the windowed kernel with 4 / 8 / 16 columns,
 *                 404 / 408 with 4 / 8 columns and a register budget for one
 *                 more CTA per SM, 504 / 508 the windowed kernel with one CTA
 *                 per parent (its field loaded once for all its children),
 *                 4 / 8 columns, 804 / 808 one CTA per pair of children that
 *                 differ only in z, sharing one phi step (4 / 8 columns; FP32
 *                 only)
 *   [3 + 44 + l]  translation at level l: 1 two columns per thread; 2..6 one
 *                 column with 1, 2, 4, 8, 16 lanes per output; 7 / 8 one warp
 *                 per (child, sample) with 2 / 1 columns per lane; 9 / 10 / 11
 *                 four columns per thread and the children four at a time,
 *                 64 / 32 / 16 columns per CTA (FP32 only)
 * Columns per CTA are powers of two (1, 2, 4, 8, 16).  mlfma_tune_set
 * returns MLFMA_EINVAL, and pins nothing, for B outside 1..max_batch, an
 * unknown prec or a value outside the sets above; a listed shape that does
 * not apply to the plan makes the product fail with MLFMA_ECUDA (invalid
 * configuration).  mlfma_tune_set drops a graph captured for the key (and
 * waits for the device to do so).
 */
#define MLFMA_TUNE_FIELDS (3 + 3 * 22)
mlfma_status mlfma_tune_get(mlfma_plan_t plan, int64_t B, int x_is_complex, int prec, int32_t *choices);
mlfma_status mlfma_tune_set(mlfma_plan_t plan, int64_t B, int x_is_complex, int prec,
                            const int32_t *choices);

/*
 * Measurement aid: the same product as mlfma_matvec, run serially on
 * `stream` (no graph, no overlap) with a CUDA event after every stage, then
 * waits for the stream.  stage_ms[MLFMA_STAGE_COUNT] receives the device
 * time of each stage in ms: 0 prepare, 1 near field, 2 leaf radiation,
 * 3 + l interpolation into level l, 25 + l translation at level l, 47 + l
 * anterpolation from level l, 69 leaf reception, 70 finalize; stages that do
 * not exist are 0.
 */
#define MLFMA_STAGE_COUNT 71
mlfma_status mlfma_profile_stages(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                                  int64_t B, int prec, void *stream, double *stage_ms);

/*
 * y = Z x without allocating anything.  The paper has no counterpart: this
 * is a service for callers that cannot call cudaMalloc at the moment they
 * need a product - code whose device memory is entirely reserved by another
 * allocator (a framework's caching pool holding the whole GPU), and
 * real-time loops that must not allocate or wait on the allocator.  It runs
 * the same kernels as mlfma_matvec, with the launch shapes mlfma_matvec uses
 * for the same columns (built-in, tuned or pinned), in order on `stream`,
 * but takes every per-call buffer (leaf-order columns, each level's outgoing
 * and incoming fields) from one static device array of
 * MLFMA_NOALLOC_SCRATCH_BYTES inside this library instead of the plan's own
 * buffers.  The caller still passes x and y, with the layouts and types of
 * mlfma_matvec (x and y must not share a byte: MLFMA_EINVAL); the plan's
 * tables must already exist (mlfma_plan allocates them once, earlier).
 *
 * - A product needing more scratch than the array holds (columns x fields
 *   of all levels) is refused with MLFMA_EINVAL and a message giving the
 *   bytes needed; so is B > max_batch.
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current and keeps it for the
 *   life of the process; do not call this entry point across a
 *   cudaDeviceReset of the device (the kept address belongs to the old
 *   context).
 * - Every call, on every plan, shares the one array and leaves its contents
 *   behind.  Nothing in it needs to start at zero: each pass writes every
 *   scratch value before reading it.  Calls whose work overlaps on the GPU
 *   (other streams, other threads, other plans) race on the array: order
 *   them.
 * - Every GPU that loads the library holds the array until the process exits.
 * Errors: EINVAL, ECUDA.
 */
#define MLFMA_NOALLOC_SCRATCH_BYTES (32 * 1024 * 1024)
mlfma_status mlfma_matvec_noalloc(mlfma_plan_t plan, const void *x, int x_is_complex, void *y,
                                  int64_t B, int prec, void *stream);

/* Wait for the plan's work on `stream` and report any pending device-side
 * error. */
mlfma_status mlfma_sync(mlfma_plan_t plan, void *stream);

/*
 * Characteristic modes (Section IV): the nev characteristic values nearest
 * zero of X J = lambda R J (Eq. (GEP)) with R = -Re Z, X = Im Z, by the
 * implicitly restarted Arnoldi method (exact shifts) on
 *   MLFMA_CM_ZINV_R: Z_H^-1 R, Z_H = R + iX, eigenvalues 1/(1 + i lambda)
 *                    (Eq. (SEP1), the paper's preferred form), or
 *   MLFMA_CM_XINV_R: X^-1 R, eigenvalues 1/lambda (Eq. (SEP)),
 * selecting the largest magnitudes.  Every operator application is one
 * product with R and one inner solve (with Z or X) by restarted GMRES,
 * right-preconditioned with a sparse approximate inverse P of the stored
 * near-field matrix (minimising ||I - A_near P||_F, Section IV) on the
 * near-field pattern (column j lives on the unknowns of j's leaf box and its
 * neighbours; the thresholds of the paper's cited SAI variant are not given,
 * so the whole near pattern is kept); all products run
 * through the GPU MLFMA in `prec`, an inner solve done with FP32 products is
 * checked with an FP64 product when the plan has FP64 and refined if needed.
 * The Arnoldi basis (ncv + 1 complex FP64 vectors) lives on the device:
 * classical Gram-Schmidt twice, normalisation, the restart's recombination
 * and the Ritz vectors are FP64 kernels; the Hessenberg matrix and its Ritz
 * pairs are FP64 on the host.  The options are checked before any device
 * work: EINVAL for nev < 1, ncv outside nev + 2..N, an unknown op or prec,
 * tol or gmres_tol not positive, gmres_restart < 2, max_inner or
 * max_restarts < 1, and for a host-only plan.
 *  lambda  host [nev], sorted by |lambda|
 *  J       host [N][nev] real characteristic currents (unit 2-norm), canonical
 *          RWG order; may be NULL
 *  stats   may be NULL
 * Synchronous.  Errors: EINVAL, ENOTCONV (Arnoldi did not converge within
 * max_restarts, or a near-field block of the preconditioner is singular;
 * lambda then holds the current Ritz values), ECUDA.
 */
typedef enum { MLFMA_CM_ZINV_R = 0, MLFMA_CM_XINV_R = 1 } mlfma_cm_op;
typedef struct {
    int nev;            /* characteristic values wanted (default 10) */
    int ncv;            /* Arnoldi basis size, nev + 2 <= ncv <= N (default 30) */
    int op;             /* mlfma_cm_op (default MLFMA_CM_ZINV_R) */
    int prec;           /* mlfma_prec of the products (default MLFMA_FP32) */
    double tol;         /* Ritz residual tolerance, relative (default 1e-8) */
    double gmres_tol;   /* inner relative residual (default 1e-6) */
    int gmres_restart;  /* GMRES restart length (default 50) */
    int max_inner;      /* GMRES iterations per solve (default 2000) */
    int max_restarts;   /* implicit restarts (default 200) */
    int use_sai;        /* 1: sparse-approximate-inverse preconditioner (default 1) */
    uint64_t seed;      /* start vector: N(0,1) from a 64-bit Mersenne twister */
} mlfma_cm_opts;
typedef struct {
    int restarts;
    int64_t inner_iterations;
    int64_t products;   /* MLFMA products issued */
    int converged;
    int inner_converged;
    double seconds;
} mlfma_cm_stats;
mlfma_status mlfma_cm_default_opts(mlfma_cm_opts *opts);
mlfma_status cm_ira_solve(mlfma_plan_t plan, const mlfma_cm_opts *opts, double *lambda, double *J,
                          mlfma_cm_stats *stats);

/*
 * Characteristic modes with a block of vectors (Section IV, Eq. (SEP), with
 * the single Arnoldi vector replaced by a block): the nev characteristic
 * values nearest zero of X J = lambda R J by shift-invert subspace iteration
 * (simultaneous iteration, Rutishauser 1970) on T = X^-1 R.  opts->ncv is
 * the block size p (nev <= p <= min(N, max_batch)); opts->op must be
 * MLFMA_CM_XINV_R.  Each iteration
 *   1. solves X W = R Y for all p columns together by restarted GMRES on the
 *      device (opts->gmres_restart, opts->max_inner steps, relative residual
 *      opts->gmres_tol per column), right-preconditioned by the sparse
 *      approximate inverse of the near part of X (as cm_ira_solve); every
 *      GMRES step is one MLFMA product of p real columns in FP32 with FP64
 *      inner products; a column holding a Ritz pair (lambda, y) with
 *      residual below 0.1 starts from y / lambda, the others from 0.  The
 *      wanted modes are near-null vectors of X, which restarted GMRES
 *      loses at each restart: a long restart (hundreds of steps; device
 *      memory (restart + 1) N p 4 bytes) is the remedy;
 *   2. takes the Ritz pairs of T on span Y in the R inner product
 *      (cm_rayleigh_ritz, FP64 on the host; no further solve);
 *   3. moves to the improved Ritz vectors Y' = W coef and applies Z to them
 *      once in opts->prec (X Y' = Im Z Y', R Y' = -Re Z Y').
 * The values are the Rayleigh quotients y^T X y / y^T R y of the vectors;
 * converged when the nev pairs nearest zero have
 *   ||X y - lambda R y|| / (||X y|| + |lambda| ||R y||) <= opts->tol.
 * The residual cannot fall much below the inner tolerance (FP32 inner solves
 * reach ~1e-6).  A degenerate cluster of values converges as a whole when
 * it fits in the block; the rate for value i is |lambda_i| /
 * |lambda_(p+1)| per iteration.  opts->max_restarts bounds the iterations.
 * Needs a device plan with FP32 (and FP64 for prec = MLFMA_FP64).  With the
 * environment variable MLFMA_CM_TRACE set, one line per iteration goes to
 * stderr (MLFMA_CM_TRACE=2: also one per wanted column).
 *  lambda  host [nev], sorted by |lambda|
 *  J       host [N][nev] real currents, unit 2-norm, largest entry positive;
 *          may be NULL
 *  stats   restarts = iterations, inner_iterations = GMRES steps (each one
 *          product of p columns), products = all block products,
 *          inner_converged = every inner solve met gmres_tol; may be NULL
 * Synchronous.  Errors: EINVAL, ENOTCONV (not converged within
 * max_restarts: lambda holds the current values; or a singular near-field
 * block of the preconditioner), ECUDA.
 */
mlfma_status cm_block_solve(mlfma_plan_t plan, const mlfma_cm_opts *opts, double *lambda, double *J,
                            mlfma_cm_stats *stats);

/*
 * The Rayleigh-Ritz step of cm_block_solve, on host memory only (no device
 * work): for a real basis Y, its product RY = R Y and W = X^-1 R Y (all
 * [n][p] row-major FP64; X, R symmetric, R positive semidefinite), the
 * Ritz pairs of T = X^-1 R on span Y in the R inner product, where T is
 * self-adjoint: A c = mu B c with A = (R Y)^T W and B = Y^T R Y
 * (symmetrised).  B = Ub D Ub^T; directions with D < 1e-9 max D carry no R
 * energy (mu = 0) and are dropped; mu are the eigenvalues of
 * D^-1/2 Ub^T A Ub D^-1/2 (cyclic Jacobi).  On the kept directions B is
 * definite, so the Ritz values interlace the eigenvalues mu = 1 / lambda of
 * T and none exceeds the largest |mu|, whatever the inertia of X.
 *  mu      [p] out: the *rank Ritz values sorted by |mu| (largest first,
 *          i.e. lambda = 1 / mu nearest zero first), 0 after
 *  coef    [p][p] out: Ritz vectors Y coef (improved: W coef = T Y coef);
 *          columns beyond *rank zero
 *  rank    out: number of Ritz pairs
 * Errors: EINVAL for NULL pointers or an empty block.
 */
mlfma_status cm_rayleigh_ritz(int64_t n, int p, const double *Y, const double *RY, const double *W, double *mu,
                              double *coef, int *rank);

/*
 * Wavenumber slopes of characteristic values, for tracking modes over
 * frequency: for each pair (lambda_m, J_m) of X J = lambda R J (R = -Re Z,
 * X = Im Z, J real, e.g. from cm_ira_solve), by first-order perturbation of
 * the pencil,  dlambda_m/dk = J^T (X' - lambda R') J / (J^T R J)  with
 * X' = Im dZ/dk, R' = -Re dZ/dk.  Each column costs one mlfma_matvec and
 * one mlfma_matvec_dk in `prec` (the first dZ/dk call builds its tables);
 * the dot products are FP64 on the host.  Within a degenerate cluster the
 * individual slopes depend on the basis the eigensolver returned; their sum
 * over the cluster does not.
 *  lambda  host [nev]       J  host [N][nev] (the layout cm_ira_solve writes)
 *  dlambda host [nev] out
 * Synchronous.  Allocates device buffers for min(nev, max_batch/2) columns.
 * Errors: EINVAL, ENOMEM, ECUDA.
 */
mlfma_status cm_eig_derivatives(mlfma_plan_t plan, int nev, const double *lambda, const double *J,
                                int prec, double *dlambda);

/*
 * Following characteristic modes over frequency (Section V tracks the values
 * over a frequency sweep; the paper does not say how modes are paired):
 * pairs the nb modes (lambda_b, Jb) found at one wavenumber with the na modes
 * (lambda_a, Ja) of the previous one by their currents.  Clusters of values
 * (sorted values whose neighbours differ by at most cluster_tol times their
 * magnitude) are paired first, by the share of the smaller cluster's span
 * that lies in the other's (||Ja_A^T Jb_B||_F^2 / min(|A|, |B|) with unit
 * columns; pairs of score >= 0.5, greedily by score, each cluster once); the
 * modes of paired clusters are then matched greedily by |Ja_i . Jb_j|.  Inside
 * a degenerate cluster the single pairings are as arbitrary as the basis the
 * eigensolver returned; compare cluster sums or means there.  Host only.
 *  Ja [n][na], Jb [n][nb] host, real (the layout cm_ira_solve writes)
 *  match   [nb] out: index into set a of each mode of set b, -1 if none
 *  overlap [nb] out: score of the cluster pair the mode belongs to (0 if none)
 * Errors: EINVAL for NULL pointers, empty sets or cluster_tol < 0.
 */
mlfma_status cm_track_modes(int64_t n, int na, const double *lambda_a, const double *Ja, int nb,
                            const double *lambda_b, const double *Jb, double cluster_tol, int *match,
                            double *overlap);

/* Summary of a plan (host copy; all fields filled). */
#define MLFMA_MAX_LEVELS 22
typedef struct {
    int64_t n;                         /* unknowns */
    int levels;                        /* incl. level 0 */
    int leaf_level;                    /* levels - 1 */
    double root_side;                  /* m */
    double root_center[3];
    int64_t near_nnz;                  /* stored near-field entries */
    int64_t leaf_boxes;
    int max_leaf_unknowns;
    int box_count[MLFMA_MAX_LEVELS];   /* occupied boxes per level */
    int trunc_L[MLFMA_MAX_LEVELS];     /* L per level (0 where no far work) */
    int samples_K[MLFMA_MAX_LEVELS];   /* (L+1) * 2(L+1) */
    int64_t translations[MLFMA_MAX_LEVELS];  /* interaction-list entries */
    int64_t device_bytes;              /* device memory held by the plan */
    double setup_seconds;              /* wall time of mlfma_plan */
} mlfma_info;

mlfma_status mlfma_plan_info(mlfma_plan_t plan, mlfma_info *info);

/*
 * Copy a host-side table of the plan into `dst` (host memory of `cap`
 * bytes); *needed receives the size in bytes (call with dst = NULL to ask).
 * Tables (level = the far level they belong to):
 *   MLFMA_X_PERM       int64 [N]       leaf-order position -> canonical index
 *   MLFMA_X_LEAF_BOX   int32 [N]       leaf box of each unknown, canonical order
 *   MLFMA_X_GRID       float64 [K][4]  (cos theta, phi, weight, theta) per sample,
 *                                      theta-major (q = it * 2(L+1) + ip)
 *   MLFMA_X_ALPHA      float64 [T][K][2] translation table per offset type
 *   MLFMA_X_ALPHA_OFFS int32 [T][3]    offset (in boxes) of each type
 *   MLFMA_X_INTERP     float64 [K_parent][K_child]  dense form of the level+1 ->
 *                                      level interpolation (applied to each tangential
 *                                      component alike; pole reflection sign folded in)
 *   MLFMA_X_BOX_CENTERS float64 [boxes][3]
 *   MLFMA_X_NEAR_COUNT int64 [1]       near entries
 *   MLFMA_X_ANTERP     float64 [K_child][K_parent]  dense form of the level ->
 *                                      level+1 anterpolation, built from its own
 *                                      (transposed, weighted) stencils
 *   MLFMA_X_ALPHA_J    float64 [T][K][2] the j_l half of MLFMA_X_ALPHA,
 *                                      sum i^l (2l+1) j_l(kr) P_l (= i x Eq. (SinKer)'s
 *                                      alpha), same types as MLFMA_X_ALPHA_OFFS
 *   MLFMA_X_ALPHA_Y    float64 [T][K][2] the y_l half, sum i^l (2l+1) y_l(kr) P_l
 *                                      (= -i x Eq. (CosKer)'s alpha); ALPHA = J + i Y
 *   MLFMA_X_SIB_ALPHA  float64 [T][K][2] sin-kernel table of the sibling
 *                                      translations of Eq. (RI) at `level` (1..leaf)
 *   MLFMA_X_SIB_OFFS   int32 [T][3]    their offsets (in boxes)
 *   MLFMA_X_WIN_INTERP float64 [K_parent][K_child]  MLFMA_X_INTERP as the FP32
 *                                      windowed kernels apply it: rebuilt from the
 *                                      stencil rows in groups of four, each group's
 *                                      taps on one window of consecutive positions
 *                                      (theta: pole reflections at -i-1 / 2n-i-1;
 *                                      phi: modulo the grid); EINVAL where a window
 *                                      would exceed 32 taps (those levels keep the
 *                                      other kernels)
 *   MLFMA_X_WIN_ANTERP float64 [K_child][K_parent]  the same for MLFMA_X_ANTERP
 *   MLFMA_X_WIN_SHAPE  int32 [8]       (groups, window width) of the four windowed
 *                                      stencils: up theta, up phi, down phi, down theta
 *   MLFMA_X_SHIFT      float64 [8][K][2] phase shift exp(i k khat . (r_parent -
 *                                      r_child)) of the aggregation (Section III-C) into `level`
 *                                      (1..leaf-1) per child octant o (bit 2: the
 *                                      child lies at +x, bit 1: +y, bit 0: +z)
 *   MLFMA_X_SHIFT_XY   float64 [8][K][2] its x and y part (the z pair kernels'
 *                                      table: octants o and o ^ 1 share it)
 *   MLFMA_X_SHIFT_Z    float64 [8][nth][2] its z part, one value per theta row
 *                                      (MLFMA_X_SHIFT = SHIFT_XY x SHIFT_Z of the
 *                                      sample's row)
 * The grid of level 1 exists for plans with at least 3 levels (it serves the
 * sibling scheme only).
 */
enum {
    MLFMA_X_PERM = 1, MLFMA_X_LEAF_BOX = 2, MLFMA_X_GRID = 3, MLFMA_X_ALPHA = 4,
    MLFMA_X_ALPHA_OFFS = 5, MLFMA_X_INTERP = 6, MLFMA_X_BOX_CENTERS = 7, MLFMA_X_NEAR_COUNT = 8,
    MLFMA_X_ANTERP = 9, MLFMA_X_ALPHA_J = 10, MLFMA_X_ALPHA_Y = 11, MLFMA_X_SIB_ALPHA = 12,
    MLFMA_X_SIB_OFFS = 13, MLFMA_X_WIN_INTERP = 14, MLFMA_X_WIN_ANTERP = 15, MLFMA_X_WIN_SHAPE = 16,
    MLFMA_X_SHIFT = 17, MLFMA_X_SHIFT_XY = 18, MLFMA_X_SHIFT_Z = 19
};
mlfma_status mlfma_export(mlfma_plan_t plan, int what, int level, void *dst, int64_t cap,
                          int64_t *needed);

/*
 * Copy a far level's field as the last Z product (mlfma_matvec, adjoint,
 * host or profile variant) in `prec` left it, for per-stage error reports:
 * which = 0 the outgoing field S (after aggregation, Eq. (11) and the upward
 * pass), 1 the incoming field G (after translation, Eq. (8), and the
 * downward pass), level 2..leaf, B = the internal real columns of that
 * product (2 per complex column).  dst: host [boxes][2][K][B] interleaved
 * complex of the precision's real type, in leaf (Morton) box order; *needed
 * receives the byte count (dst may be NULL to ask).  Waits for the device.
 * Errors: EINVAL, ECUDA.
 */
mlfma_status mlfma_export_field(mlfma_plan_t plan, int prec, int which, int level, int64_t B, void *dst,
                                int64_t cap, int64_t *needed);

/* Release everything the plan owns (waits for its work).  NULL is a no-op. */
void mlfma_destroy(mlfma_plan_t plan);

/*
 * Frequency sweeps (Section V sweeps frequencies one after another; here
 * the plans of a sweep share the GPU).  A set holds one plan per wavenumber
 * ks[0..nk-1] on one mesh (levels, digits and opts as mlfma_plan; each plan
 * has its own grids and tables).  Memory admission: the host tables of every
 * plan are built first and give an estimate of its peak device bytes; the
 * plans are grouped, in wavenumber order, into waves whose estimates fit
 * `budget_bytes` (<= 0: 90 % of the device's free memory), and the first
 * wave is put on the device.  A plan larger than the budget is MLFMA_ENOMEM.
 */
typedef struct mlfma_set_s *mlfma_set_t;
mlfma_status mlfma_set_create(const double *verts, int64_t nv, const int32_t *tris, int64_t nt,
                              const double *ks, int nk, int levels, double digits,
                              const mlfma_opts *opts, int64_t budget_bytes, mlfma_set_t *out);

/*
 * y_f = Z(k_f) x_f for every wavenumber of the set.
 *  x  device: [nk][N][B] (x_shared = 0) or one [N][B] block for all
 *     (x_shared = 1); real or, with x_is_complex, interleaved complex
 *  y  device: [nk][N][B] interleaved complex
 * Types, B and prec as mlfma_matvec (prec must be in opts.precisions).  The
 * far and near passes of all plans of a wave run as parallel branches of one
 * CUDA graph, captured on first use per (wave, precision, columns) and
 * replayed; with one wave nothing is rebuilt between calls.  With several
 * waves each call waits for a wave's work, releases its plans' device memory
 * and builds the next wave's (near fields and patterns are recomputed):
 * that is the price of a budget smaller than the sweep.
 */
mlfma_status mlfma_set_matvec(mlfma_set_t set, const void *x, int x_shared, int x_is_complex,
                              void *y, int64_t B, int prec, void *stream);

/* Per wavenumber (arrays of nk, each may be NULL): admission wave, estimated
 * peak device bytes, device bytes now held (0 when not admitted). */
mlfma_status mlfma_set_info(mlfma_set_t set, int *nk, int *waves, int *wave_of,
                            int64_t *est_bytes, int64_t *device_bytes);

/* The set's plan for ks[f] (owned by the set; a device plan while its wave is
 * admitted, host-only otherwise). */
mlfma_status mlfma_set_plan(mlfma_set_t set, int f, mlfma_plan_t *plan);

/* Release the set and its plans (waits for their work).  NULL is a no-op. */
void mlfma_set_destroy(mlfma_set_t set);

/* Message of the last failure on this thread ("" if none). */
const char *mlfma_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MLFMA_H */
