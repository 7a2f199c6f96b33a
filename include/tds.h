/*
 * tds.h -- C ABI of the GB300 compact finite-difference derivative library (libtds.so).
 *
 * The library computes batched sixth-order compact finite-difference derivatives (and the
 * tridiagonal solve alone, compact filters and interpolations, and the transport-equation
 * right-hand side built on them) along one direction of a 3D field with the DistD2 algorithm (Sec. 4.2 of Akkurt et al., "A
 * Distributed-memory Tridiagonal Solver Based on a Specialised Data Structure Optimised for
 * CPU and GPU Architectures"): the stencil right-hand side (Eq. cfds) is fused into a
 * modified-Thomas decoupling sweep over P chunks per line (Algorithm 5), a reduced system
 * couples the chunk ends, and a substitution finishes each line (Algorithm 6).  The P chunks
 * stand in for the paper's ranks; all of them live on one GPU.
 *
 * Conventions shared by every call:
 *  - Data pointers are DEVICE pointers unless a name says "host".  The caller owns them.
 *  - Fields use the interleaved group data structure of Sec. 4.1: for derivative direction
 *    d with n points per line and N lines, element (s, j, g) of the direction-d layout is at
 *    flat offset s + SZ*(j + n*g), for line l = g*SZ + s.  Lines are numbered
 *        x lines: l = y + ny*z   (n = nx)
 *        y lines: l = x + nx*z   (n = ny)
 *        z lines: l = x + nx*y   (n = nz)
 *    The Cartesian layout is x + nx*(y + ny*z).  Only SZ = 32 is supported.
 *  - Element type: TDS_F64 = IEEE double, TDS_F32 = IEEE float.
 *  - "stream" is a cudaStream_t passed as void* (NULL = the legacy default stream).  All
 *    work is asynchronous on that stream.  Argument and shape errors are returned before any
 *    launch; launch failures come back as TDS_ERR_CUDA.  No C++ exception crosses the ABI.
 *  - The hot calls (tds_deriv, tds_deriv_adjoint, tds_reorder) allocate nothing.  Device
 *    memory is allocated only by tds_plan_create and freed by tds_plan_destroy.
 *  - A plan is immutable after creation and may be used from several streams at once,
 *    each with its own workspace.
 */
#ifndef TDS_H
#define TDS_H

#include <stddef.h>

#if defined(__GNUC__)
#define TDS_API __attribute__((visibility("default")))
#else
#define TDS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDS_OK = 0,
    TDS_ERR_ARG = 1,        /* invalid argument (null pointer, unknown enum, bad h or SZ)  */
    TDS_ERR_SHAPE = 2,      /* shape rule violated (see tds_plan_create)                    */
    TDS_ERR_ALIAS = 3,      /* input and output buffers overlap                             */
    TDS_ERR_WORKSPACE = 4,  /* workspace missing or smaller than tds_workspace_bytes        */
    TDS_ERR_CUDA = 5,       /* a CUDA runtime call or kernel launch failed                  */
    TDS_ERR_TIMEOUT = 6,    /* a device-side bounded wait gave up (see tds_device_status)   */
    TDS_ERR_NOMEM = 7       /* device or host allocation failed in tds_plan_create          */
} tds_status;

typedef enum { TDS_DIR_X = 0, TDS_DIR_Y = 1, TDS_DIR_Z = 2 } tds_dir;
typedef enum { TDS_LAYOUT_CART = 0, TDS_LAYOUT_X = 1, TDS_LAYOUT_Y = 2, TDS_LAYOUT_Z = 3 } tds_layout;
typedef enum { TDS_BC_PERIODIC = 0, TDS_BC_CLOSED = 1 } tds_bc;
typedef enum { TDS_F64 = 0, TDS_F32 = 1 } tds_dtype;
typedef enum { TDS_REDUCED_EXACT = 0, TDS_REDUCED_PAPER_DROP = 1 } tds_reduced;

/* Kernel pipeline a plan uses; TDS_VARIANT_AUTO lets the plan choose. */
typedef enum {
    TDS_VARIANT_AUTO = 0,
    TDS_VARIANT_RESIDENT = 1,   /* one CTA holds a whole group of SZ lines on chip          */
    TDS_VARIANT_STREAMING = 2,  /* decouple / reduced / substitute as three kernels         */
    TDS_VARIANT_PIPELINED = 3,  /* persistent CTAs, each sweeping many groups through
                                   several on-chip tile buffers filled ahead by TMA         */
    TDS_VARIANT_SEGMENTED = 4   /* segments of 64..256 rows that subdivide the chunks, one
                                   warp each, in two kernels: lines too long for one CTA,
                                   and plans whose resident CTAs would be too thin          */
} tds_variant;

/* Arithmetic of an FP64 plan's sweeps (tds_plan_set_arith). */
typedef enum { TDS_ARITH_NATIVE = 0, TDS_ARITH_SPLIT = 1 } tds_arith;

typedef struct tds_plan tds_plan;

/*
 * tds_plan_create -- operator preprocessing (Algorithm 4, Sec. 4.2), in FP64 on the host; it
 * depends only on the operator, so a plan is built once and reused for every field.
 *   out   : receives the new plan (set to NULL on error).
 *   nx, ny, nz : Cartesian grid; the line length n is the extent along dir, the number of
 *           lines N is the product of the two others.
 *   dir   : derivative direction.
 *   order : 1 (first derivative, Eq. cfds: alpha=1/3, a=14/9, b=1/9) or 2 (second
 *           derivative: alpha=2/11, a=12/11, b=3/11).
 *   bc    : TDS_BC_PERIODIC (cyclic lines) or TDS_BC_CLOSED (one-sided closures:
 *           first derivative f'0 + 2f'1 = (-5f0 + 4f1 + f2)/2h, f'0/4 + f'1 + f'2/4 =
 *           (3/2)(f2 - f0)/2h; second derivative f''0 + 11f''1 = (13f0 - 27f1 + 15f2 - f3)/h^2,
 *           f''0/10 + f''1 + f''2/10 = (6/5)(f0 - 2f1 + f2)/h^2; mirrored at the far end).
 *   P     : chunks per line (the emulated ranks); n % P == 0, m = n/P >= 4.
 *   h     : grid spacing (> 0).
 *   dtype : storage and sweep precision.  TDS_F32 keeps the reduced chunk-end system and the
 *           Sherman-Morrison correction in FP64; on closed lines whose closure magnifies end-row
 *           rounding (the second derivative's), its four rows at each end run in float pairs.
 *   sz    : group size SZ; must be 32.
 *   mode  : TDS_REDUCED_EXACT solves the full 2P-unknown chunk-end system;
 *           TDS_REDUCED_PAPER_DROP drops the two sub-machine-epsilon couplings per chunk
 *           (Fig. alg), leaving independent 2x2 systems across chunk boundaries.
 * Shape rules (TDS_ERR_SHAPE): n >= 8, n % P == 0, n / P >= 4, N % 32 == 0.
 */
TDS_API tds_status tds_plan_create(tds_plan **out, int nx, int ny, int nz, tds_dir dir, int order,
                           tds_bc bc, int P, double h, tds_dtype dtype, int sz,
                           tds_reduced mode);

/*
 * tds_plan_create_filter -- a plan whose operator is the compact filter g = A^{-1} B f (the paper
 * notes, citing Lele 1992, that compact schemes also give filters; it prints none, so this is
 * the fourth-order tridiagonal member of Lele's family):
 *     alpha_f g[i-1] + g[i] + alpha_f g[i+1]
 *       = a0 f[i] + (a1/2)(f[i+1] + f[i-1]) + (a2/2)(f[i+2] + f[i-2]),
 *     a0 = 5/8 + 3 alpha_f/4, a1 = 1/2 + alpha_f, a2 = -1/8 + alpha_f/4,
 * which keeps polynomials through degree 3 and removes the grid's odd-even mode; on closed lines
 * the end values are kept and rows 1 and n-2 use the second-order member (a0 = a1 = 1/2 + alpha_f,
 * a2 = 0).  alpha_f must lie in (-1/2, 1/2) (TDS_ERR_ARG); values near 1/2 filter least.  Every
 * other argument, rule and error is that of tds_plan_create; tds_deriv applies the filter,
 * tds_deriv_adjoint its transpose (on periodic lines the filter itself).
 */
TDS_API tds_status tds_plan_create_filter(tds_plan **out, int nx, int ny, int nz, tds_dir dir, double alpha_f,
                                          tds_bc bc, int P, tds_dtype dtype, int sz, tds_reduced mode);

/*
 * tds_plan_create_interp -- a plan whose operator is the sixth-order compact interpolation from
 * the nodes to the mid-points (Lele 1992's family, as for the filter):
 *     3/10 g[i-1] + g[i] + 3/10 g[i+1] = 3/4 (f[i] + f[i+1]) + 1/20 (f[i-1] + f[i+2]),
 * g[i] approximating f at x_i + h/2.  Periodic lines have n mid-points.  A closed line has n-1
 * (g[0..n-2]): the first and the last use the compact closure exact through degree 4 (the paper
 * prints none), g[0] + 5/3 g[1] = 5/24 f[0] + 15/8 f[1] + 5/8 f[2] - 1/24 f[3] and its mirror
 * image, and the result's last slot g[n-1] is set to zero so that the layout maps n points to
 * n.  tds_deriv interpolates to the mid-points; tds_deriv_adjoint applies the transpose, which is
 * the interpolation from mid-points (g[i] at x_i + h/2) back to the nodes (on closed lines the
 * input's last slot is not read).  Arguments, rules and errors as tds_plan_create.
 */
TDS_API tds_status tds_plan_create_interp(tds_plan **out, int nx, int ny, int nz, tds_dir dir, tds_bc bc,
                                          int P, tds_dtype dtype, int sz, tds_reduced mode);

/*
 * tds_plan_create_band -- a plan for the batched tridiagonal solve A x = d with a caller-given
 * band (Algorithms 4-6 solve any such system; not restricted to the compact schemes), e.g. the
 * implicit systems of ADI schemes.  Row j of every line is
 *     a[j] x_{j-1} + b[j] x_j + c[j] x_{j+1} = d_j,   j = 0 .. n-1,
 * with a[0] coupling to x_{n-1} and c[n-1] to x_0 on periodic lines (ignored on closed lines).
 *   a, b, c : host arrays of n doubles each (n = the extent along dir), copied by the call.
 *   other arguments as in tds_plan_create.
 * The method sweeps without pivoting: the band should be diagonally dominant.  Any band is
 * accepted, variable coefficients along the line included (non-uniform grids, variable
 * diffusivity): the preprocessing of Algorithm 4 runs per chunk, once for every chunk when
 * the chunks' bands differ, else once per class of equal chunks (first / interior / last).
 * Errors: TDS_ERR_ARG for a NULL array, a non-finite entry or a zero pivot; the shape rules
 * of tds_plan_create.  Only tds_solve (and the plan
 * queries and tuning calls) accept a band plan; the derivative calls return TDS_ERR_ARG.
 */
TDS_API tds_status tds_plan_create_band(tds_plan **out, int nx, int ny, int nz, tds_dir dir,
                                const double *a, const double *b, const double *c, tds_bc bc,
                                int P, tds_dtype dtype, int sz, tds_reduced mode);

/* Choose the kernel pipeline of a plan (tuning and test hook; call before first use, not
 * concurrently with a call that uses the plan).  TDS_ERR_ARG if the plan cannot run the
 * requested variant (a resident group larger than one CTA's shared memory).  AUTO picks
 * RESIDENT when the lines fit in a CTA (one thread per line and chunk, at most 512 per CTA)
 * unless, in FP64, its CTAs would leave fewer than 6 warps per SM (few chunks, large tiles)
 * or, in FP32, the lines need 8-line CTAs, while the chunk splits into at least two segments;
 * then SEGMENTED (segments of 64 up to the cap, 128 rows FP64 / 256 FP32, dividing the chunk
 * length); else STREAMING.  An FP32 RESIDENT
 * choice may run on finer chunks (tds_plan_run_chunks).  The adjoint of a SEGMENTED plan runs
 * on the segment partition on periodic lines, else resident when the lines fit in a CTA, else
 * through the streaming pipeline. */
TDS_API tds_status tds_plan_set_variant(tds_plan *plan, tds_variant variant);

/* Lines of a group held by one CTA of the RESIDENT variant: 32 (the whole group, one bulk
 * copy per chunk), 16 or 8 (the group is split over 32/lines CTAs whose rows move as 2-D TMA
 * tensor boxes, so that several CTAs share an SM and one CTA's copies overlap another's sweep).
 * A layout choice only: every width gives the same result.  tds_plan_create picks, among the
 * widths that let two CTAs share an SM, the largest for FP32 and the smallest for FP64.
 * TDS_ERR_ARG when the width is not 32, 16 or 8, the tile does not fit in one CTA's shared
 * memory, fewer than two warps would remain per CTA (widths below 32), or the CTA would need
 * more than 512 threads (P x lines > 512).  A width set here also drops the finer chunks of
 * tds_plan_run_chunks.  Not part of the method (Sec. 4.1 fixes the 32-line group; its split
 * over CTAs is a GPU layout decision). */
TDS_API tds_status tds_plan_set_width(tds_plan *plan, int lines);

/* How an FP64 plan's resident sweeps do their arithmetic (a GB300 choice; the paper's sweeps
 * are plain FP64).  TDS_ARITH_NATIVE (the default): FP64 throughout.  TDS_ARITH_SPLIT: the
 * field stays FP64 in memory and the reduced chunk-end system stays FP64, but the stencil's
 * differences are taken in FP64 and split into pairs of floats (hi + lo, about 48 significant
 * bits), and the forward elimination, the accumulation of the chunk ends and the
 * back-substitution run in float-pair arithmetic on the FP32 pipes, which on GB300 issue 64
 * times the FP64 rate.  Results agree with FP64 to about 1e-14 of max|result| on the tested
 * fields.  Values (inputs and results, and the differences of neighbouring inputs) must lie in
 * float's exponent range with room for the low word, |x| in [2^-74, 2^126]: smaller
 * differences lose low-word bits, larger ones overflow.  Applies to tds_deriv, the host entry
 * points, tds_deriv_multi (one launch per operator: these sweeps are bound by their own issue
 * rate, not by HBM reads, so the fused pass gains nothing) and tds_transport when they run the
 * RESIDENT variant on a forward-form operator (the stencil right-hand side: first and second
 * derivatives and their adjoints on periodic lines, the filter, the mid-point interpolation and
 * its transpose on periodic lines); the closed-line adjoints, tds_solve and every other variant
 * run native FP64.  The plan's CTA width follows the arithmetic its forward operator runs
 * (split sweeps, bound by the FP32 issue rate, take the widest CTA that lets two share an SM, as
 * FP32 plans do) and the variant is chosen again (AUTO): call this before tds_plan_set_width
 * and tds_plan_set_variant.
 * TDS_ERR_ARG for an FP32 plan, a band plan or an unknown value. */
TDS_API tds_status tds_plan_set_arith(tds_plan *plan, tds_arith arith);

/* Describe a plan: line length n, lines N, chunks P, the variant it will run, and the
 * dynamic shared memory per CTA of its resident kernel (0 if streaming).  Any output
 * pointer may be NULL.  tds_plan_width gives the resident CTA width (0 if the plan cannot run
 * resident). */
TDS_API tds_status tds_plan_info(const tds_plan *plan, int *n, int *nlines, int *P, int *variant,
                         int *smem_bytes);
TDS_API tds_status tds_plan_width(const tds_plan *plan, int *lines);

/* tds_plan_run_chunks -- the chunks per line the plan's kernels run with: P, or P x 2^k when the
 * AUTO variant of an FP32 plan (EXACT mode, no band) found that one-warp-per-chunk resident CTAs
 * would leave fewer than 8 warps per SM and runs the same operator on finer chunks of at least 64
 * rows instead (results equal to rounding: the reduced system over all chunk ends is solved
 * exactly; the partition is not part of the method's result).  A variant or width set by the
 * caller runs on the plan's own P chunks.  tds_plan_info and tds_plan_width describe the kernels
 * that run. */
TDS_API tds_status tds_plan_run_chunks(const tds_plan *plan, int *chunks);

/* Bytes of device workspace tds_deriv / tds_deriv_adjoint need with this plan (0 is
 * possible).  The workspace must be 256-byte aligned; its contents need no initialisation
 * and are garbage afterwards. */
TDS_API tds_status tds_workspace_bytes(const tds_plan *plan, size_t *bytes);

/*
 * tds_deriv -- out = A^{-1} B in along the plan's direction (Algorithms 5 and 6 with the
 * reduced chunk-end system in between).
 *   in, out : device arrays of N*n elements of the plan's dtype, both in the direction
 *             layout of the plan; they must not overlap (TDS_ERR_ALIAS).  16-byte aligned.
 *   ws, ws_bytes : device workspace of at least tds_workspace_bytes (may be NULL if that
 *             is 0), TDS_ERR_WORKSPACE otherwise.
 */
TDS_API tds_status tds_deriv(const tds_plan *plan, const void *in, void *out, void *ws,
                     size_t ws_bytes, void *stream);

/*
 * tds_deriv_adjoint -- out = B^T A^{-T} g, the transpose of tds_deriv's operator (not in
 * the paper: used to back-propagate through a derivative).  Same arguments and rules as
 * tds_deriv; the transposed tridiagonal solve runs through the same DistD2 pipeline on
 * A^T, followed by the transposed stencil.
 */
TDS_API tds_status tds_deriv_adjoint(const tds_plan *plan, const void *g, void *out, void *ws,
                             size_t ws_bytes, void *stream);

/*
 * tds_solve -- x = A^{-1} d: the DistD2 tridiagonal solve of the plan's compact scheme alone
 * (Algorithms 4-6 with the reduced chunk-end system between them, the right-hand side given
 * instead of computed from a stencil), e.g. for a caller that forms its own right-hand side.
 * A is the plan's left-hand side: alpha on the off-diagonals and 1 on the diagonal (cyclic on
 * periodic lines), with the closure rows on closed lines.  Same arguments, layout and errors
 * as tds_deriv.  Runs resident when the plan's lines fit a CTA (any variant but STREAMING),
 * else through the streaming pipeline.
 */
TDS_API tds_status tds_solve(const tds_plan *plan, const void *d, void *x, void *ws, size_t ws_bytes,
                     void *stream);

/*
 * tds_deriv_thomas -- the plan's operator (derivative, filter or interpolation; not its
 * adjoint) by the plain Thomas algorithm (Algorithm 1) on each whole line, the single-rank
 * baseline DistD2 is measured against (Table BW): one thread per line, the stencil right-hand
 * side fused into the forward pass, the forward values kept in `out` and read back by the
 * backward pass; cyclic lines by Sherman-Morrison (Sec. 2.1): Thomas on the modified matrix A'
 * then a third pass x = y - (v.y / (1 + v.z)) z with z = A'^{-1} u from the planner.  The
 * plan's chunking and variant are ignored.  FP32 plans run every step in FP32 (no FP64 chunk-end
 * system: there is none).
 *   plan   : a derivative, filter or interpolation plan; a band plan, or one whose whole-line
 *            elimination meets a zero pivot, gives TDS_ERR_ARG.
 *   in, out: device arrays in the plan's direction layout, 16-byte aligned, not overlapping
 *            (TDS_ERR_ALIAS).  No workspace.
 * HBM traffic: `in` read once, `out` written twice and read once (cyclic lines: once more
 * each), against one read and one write for the resident DistD2 kernels.
 */
TDS_API tds_status tds_deriv_thomas(const tds_plan *plan, const void *in, void *out, void *stream);

/*
 * tds_deriv_multi -- several operators of one input: outs[i] = plans[i]'s derivative
 * (adjoint[i] = 0) or its adjoint (adjoint[i] = 1) of `in`, 1 <= count <= 4.  When every plan
 * runs RESIDENT with the same chunks and CTA width and every operator has the forward form
 * (derivatives, and adjoints on periodic lines) and no plan has split-precision FP64 sweeps
 * (tds_plan_set_arith), one kernel computes them all from a single
 * read of `in` (the field is read from HBM once and each result written once; Sec. 5 fuses the
 * transport equation's derivative operators the same way): one CTA per (group of lines,
 * operator), the operators' CTAs of a group adjacent so that they share the input through L2
 * (the environment variable TDS_MULTI_FORM=seq selects one CTA per group sweeping the operators
 * in turn, for tuning); otherwise the operators run one after another on `stream`.  Results are
 * bitwise those of the single calls.
 *   plans   : count plans over the same field shape, direction and dtype (TDS_ERR_ARG otherwise).
 *   adjoint : count flags, 0 or 1.
 *   in, outs: device arrays as in tds_deriv; no output may overlap `in` or another output
 *             (TDS_ERR_ALIAS).
 *   ws, ws_bytes : one workspace of at least the largest tds_workspace_bytes of the plans
 *             (used only when the operators run one after another).
 */
TDS_API tds_status tds_deriv_multi(int count, const tds_plan *const *plans, const int *adjoint,
                           const void *in, void *const *outs, void *ws, size_t ws_bytes, void *stream);

/*
 * tds_transport -- one term group of the skew-symmetric momentum transport equation (Sec. 5,
 * Eq. mom-comps) along the plans' direction j, with the three operators sharing one read of
 * the fields (the fused "abstract kernel" of Sec. 5):
 *     out = -1/2 (u_j * D1 u_i + D1 (u_j u_i)) + nu * D2 u_i
 * (products pointwise; D1, D2 the first and second compact derivatives of d1, d2).
 *   d1, d2 : order-1 and order-2 plans (no band) over the same field shape, direction, dtype,
 *            chunk count P and CTA width, each able to hold its lines in a CTA (a nonzero
 *            tds_plan_width, whatever the plan's variant); TDS_ERR_ARG otherwise.  Their
 *            boundary conditions may differ.
 *   ui, uj : device arrays in the plans' direction layout, 16-byte aligned; the same array
 *            when i = j.
 *   nu     : the kinematic viscosity.
 *   out    : device array in that layout, overwritten; must not overlap ui or uj
 *            (TDS_ERR_ALIAS).
 * One kernel, no workspace: HBM sees ui and uj read once and out written once (the result of
 * each operator is combined in L2).  The three sweeps round like tds_deriv's (FP32 plans:
 * FP32 storage and sweeps, FP64 chunk-end system); the products and the combination are taken
 * in the plan's arithmetic type.
 */
TDS_API tds_status tds_transport(const tds_plan *d1, const tds_plan *d2, const void *ui, const void *uj,
                                 double nu, void *out, void *stream);

/*
 * tds_deriv_host -- tds_deriv with the input and the result in HOST memory (not in the paper:
 * the end-to-end form of the call).
 *   host_in  : N*n elements in the plan's direction layout, copied to d_in; NULL when the
 *              input is already in d_in (no host-to-device copy).
 *   host_out : N*n elements receiving the result (copied from d_out).
 *   d_in, d_out, ws, ws_bytes : caller-owned device buffers, the same rules as tds_deriv.
 * The lines are cut into up to 8 slabs of whole groups; each slab is copied in, computed and
 * copied out as soon as it can, so the copies of one slab overlap the compute of the next
 * (two copy streams owned by the plan, created by tds_plan_create).  The call is ordered on
 * `stream`: it starts after the work already queued there, and work queued on `stream` after
 * it (including a synchronisation) sees host_out complete.  Pinned host memory makes the
 * copies asynchronous.  Host calls with one plan must not run concurrently (they share the
 * plan's copy streams and events).  Errors: those of tds_deriv (checked before any copy),
 * TDS_ERR_ARG for a NULL host_out, d_in or d_out, TDS_ERR_CUDA when a copy fails to queue.
 */
TDS_API tds_status tds_deriv_host(const tds_plan *plan, const void *host_in, void *host_out,
                          void *d_in, void *d_out, void *ws, size_t ws_bytes, void *stream);

/* tds_deriv_adjoint_host -- tds_deriv_adjoint with host buffers: host_g (or NULL when the
 * input is already in d_in) and host_out; the same rules and pipeline as tds_deriv_host. */
TDS_API tds_status tds_deriv_adjoint_host(const tds_plan *plan, const void *host_g, void *host_out,
                                  void *d_in, void *d_out, void *ws, size_t ws_bytes, void *stream);

/*
 * tds_reorder -- permute a field between the Cartesian layout and the x, y, z direction
 * layouts (Sec. 4.1: each derivative direction has its own interleaved layout, so a change of
 * direction moves the data); a pure permutation, bit-exact.
 *   in, out : device arrays of nx*ny*nz elements, non-overlapping (TDS_ERR_ALIAS), 16-byte
 *             aligned.
 * Shape rules (TDS_ERR_SHAPE): nx % 32 == 0 and ny % 32 == 0 (so that every layout's SZ-row
 * is a run of 32 consecutive x or y), ny <= 65535, nz <= 65535; from == to is a plain copy.
 */
TDS_API tds_status tds_reorder(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                       tds_layout to, tds_dtype dtype, int sz, void *stream);

/*
 * tds_reorder_add -- out += the reorder of in (the accumulation of Table transport, fused with
 * the reorder: the transport right-hand side adds each y and z result into the x-layout field
 * in one pass).  Same arguments and rules as tds_reorder; from == to adds in place of a copy.
 * Each element of out receives exactly one addition, so the result is bit-exact against
 * reorder-then-add.
 */
TDS_API tds_status tds_reorder_add(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                                   tds_layout to, tds_dtype dtype, int sz, void *stream);

/*
 * tds_fanout_copy -- copy `bytes` of `in` to each of `count` outputs (1 <= count <= 4), reading
 * the input once: a copy with the memory traffic of tds_deriv_multi's fused pass (one read of
 * the field, one write per result), the ceiling that pass is measured against.  Not part of the
 * method (a measurement aid).  Device pointers, 16-byte aligned, bytes a multiple of 16, no
 * two buffers overlapping (TDS_ERR_ALIAS); TDS_ERR_ARG otherwise.  Asynchronous on `stream`.
 */
TDS_API tds_status tds_fanout_copy(const void *in, void *const *outs, int count, size_t bytes, void *stream);

/* Free a plan and its device arrays (NULL is a no-op).  Not stream-ordered: the caller makes
 * sure no work that uses the plan is still running. */
TDS_API void tds_plan_destroy(tds_plan *plan);

/* Static, human-readable name of a status code. */
TDS_API const char *tds_status_string(tds_status status);

/*
 * tds_device_status -- read and clear the device-side status word of the current device.
 * Kernels that wait on an asynchronous copy bound their waits; a wait that gives up sets this
 * word (TDS_ERR_TIMEOUT), skips its writes and returns.  Synchronises the device.
 */
TDS_API tds_status tds_device_status(void);

/*
 * tds_selftest_timeout -- exercise the device-side failure path: launch one warp that waits on
 * a barrier nothing completes; the wait gives up after `seconds` (0 < seconds <= 2), records
 * TDS_ERR_TIMEOUT in the device status word and the kernel returns normally, leaving the
 * context usable.  Read the result with tds_device_status().
 */
TDS_API tds_status tds_selftest_timeout(double seconds, void *stream);

/*
 * tds_plan_reduced_coeffs -- copy the plan's reduced chunk-end system to host memory for
 * inspection: for chunk k, row 2k (first unknown F_k) is sub[2k]*L_{k-1} + F_k + sup[2k]*L_k
 * and row 2k+1 (last unknown L_k) is sub[2k+1]*F_k + L_k + sup[2k+1]*F_{k+1}; on periodic
 * lines sub[0] couples to L_{P-1} and sup[2P-1] to F_0.  sub and sup hold 2P doubles each.
 */
TDS_API tds_status tds_plan_reduced_coeffs(const tds_plan *plan, double *host_sub, double *host_sup);

/*
 * tds_reduced_solve -- solve the plan's reduced system for many lines (a test entry point
 * for the communication phase alone): rhs and x are device arrays of N*2P doubles, line
 * after line, unknowns ordered F_0, L_0, F_1, L_1, ...
 */
TDS_API tds_status tds_reduced_solve(const tds_plan *plan, const double *rhs, double *x, void *stream);

/* Size of the scratch array built into the library for tds_deriv_noalloc (16 MiB). */
#define TDS_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)

/*
 * tds_deriv_noalloc -- tds_deriv for callers that cannot allocate device memory (no
 * counterpart in the paper).  Some callers cannot call cudaMalloc or an allocator at all: a
 * host application that owns every device buffer, a real-time loop that must never allocate,
 * or a plugin that may only touch the buffers it is given.  They cannot supply tds_deriv's
 * workspace, so this call takes its scratch from an array of TDS_NOALLOC_SCRATCH_BYTES
 * compiled into the library (held on every GPU that loads the library until the process
 * exits) and allocates nothing.
 *   plan    : an existing plan (created beforehand; plan creation itself allocates).
 *   in, out : as in tds_deriv (device, 16-byte aligned, non-overlapping: TDS_ERR_ALIAS).
 * Always runs the three-kernel streaming pipeline on the plan's own P chunks (an AUTO FP32
 * plan that tds_deriv runs on finer chunks gives the same result to rounding).  Its chunk ends
 * need 16*N*P bytes; a plan needing more than TDS_NOALLOC_SCRATCH_BYTES (N*P > 1,048,576
 * lines x chunks) is rejected with TDS_ERR_WORKSPACE before any launch.
 * The first call on each device looks up the array's device address with that device
 * current (cudaGetSymbolAddress) and caches it with the driver's identity of the context; a
 * new context on the device (after cudaDeviceReset) gets a fresh lookup.  Make the first
 * call on a device, and the first after a reset, before any stream capture.  All calls share
 * the one array, which keeps the last call's contents (nothing in it needs to start at zero):
 * calls that overlap on the GPU -- concurrent streams, or several host threads -- race on it
 * and must be serialised by the caller.
 */
TDS_API tds_status tds_deriv_noalloc(const tds_plan *plan, const void *in, void *out,
                                     void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TDS_H */
