// tds_internal.h -- types shared by the host planner, the kernels and the C ABI of libtds.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "tds.h"

namespace tds {

constexpr int kSZ = 32;           // lines per group: one warp lane per line (Sec. 4.1, SZ=32)
constexpr int kTaps = 7;          // stencil offsets -3..3 (closure rows reach 3 points in)
constexpr int kEdgeRows = 4;      // closed lines: rows 0..3 and n-4..n-1 carry their own taps
constexpr int kMaxResidentP = 16; // resident kernels: at most 16 x 32 = 512 threads per CTA (one per
                                   // line and chunk: P x lines <= 512)
constexpr int kHostSlabs = 8;     // host entry points: copies and compute pipelined over 8 slabs
constexpr int kMaxMulti = 4;      // operators one fused pass (tds_deriv_multi) may compute

// Number of per-row coefficient arrays of one operator (Algorithm 4 output, per chunk class):
//   f  : forward factor, 1/b_j for j <= 1, 1/(b_j - a_j s^c_{j-1}) for j >= 2
//   r  : sub-diagonal a_j (eliminated in the forward pass, j >= 2)
//   w  : backward multiplier (j = 1..m-3) and c_0/b_0 for the final row-0 step (j = 0)
//   sa : coupling of row j to the chunk's first unknown after both passes (s^a)
//   sc : coupling of row j to the chunk's last unknown after both passes (s^c)
enum { kF = 0, kR = 1, kW = 2, kSA = 3, kSC = 4, kNumRowArrays = 5 };

// Reduced-system arrays (2P entries each): sub-diagonal, forward factor, backward multiplier
// of the (Sherman-Morrison-modified if cyclic) tridiagonal factorisation, q = T'^{-1} u; and,
// for the decoupled form, per chunk boundary k (between chunk k-1 and k, cyclically) the
// coupling a_k of F_k to L_{k-1}, c_k of L_{k-1} to F_k, and 1/(1 - a_k c_k).
enum { kRedSub = 0, kRedWf = 1, kRedCp = 2, kRedQ = 3, kRedBa = 4, kRedBc = 5, kRedBinv = 6,
       kNumRedArrays = 7 };

// The decoupled form is used when every coupling it ignores is below this magnitude
// (relative to the unit diagonal): the solution then agrees with the full solve to rounding.
constexpr double kDecoupleTol = 5.421010862427522e-20;   // 2^-64

// Operator descriptor passed by value to every kernel.
struct DevOp {
    int n, m, P, nlines, ngroups;
    int periodic;   // cyclic lines
    int adjoint;    // how the sweep runs: 0 stencil right-hand side (A^{-1} B, and B^T A^{-T} on
                    // periodic lines); 1 identity right-hand side on A^T, then the B^T taps
                    // (the adjoint on closed lines); 2 identity right-hand side, no taps (A^{-1})
    int symmetric;  // interior taps: -1 antisymmetric (first derivative), +1 symmetric (filter),
                    // +2 pairs about +1/2 (nodes -> mid-points), +3 pairs about -1/2 (mid-points
                    // -> nodes), +4 symmetric with vanishing sum (second derivative); FP32
                    // sweeps apply symmetric taps to second differences (see tapsum)
    int e64;        // FP32 and split-precision FP64 sweeps of closed lines: the closure rows' steps
                    // in FP64 (the solve magnifies an end row's rounding by more than 16); native
                    // FP64 sweeps ignore it
    int ncls;       // chunk classes (first / interior / last differ on closed lines)
    int cls_first, cls_mid, cls_last;
    int bt_fold;    // closed-line adjoint (adjoint 1) with m >= 16: x = B^T y formed inside the
                    // back-substitution (FP32 plans; TDS_ADJOINT_FOLD = 0 / 1 forces either form)
    int cls_each;   // 1: every chunk is its own class (ncls = P; a band whose chunks differ), and
                    // the per-class scalars below hold one entry (index 0) valid for all chunks
    const double *row64;  // [kNumRowArrays][ncls*m]
    const float *row32;   // the same arrays rounded to float (FP32 sweeps)
    // Row records of the resident sweep, [ncls][m] each, FP64 and FP32 copies:
    //   fwd = {f_j, r_j, pi_j, 0}: forward factor, sub-diagonal, and the weight of the forward
    //         value d_j in the back-swept row 1 (pi_1 = 1, pi_j = -pi_{j-1} s^c_{j-1}, 0 at
    //         rows 0 and m-1), so that row 1 after the backward pass is sum_j pi_j d_j;
    //   bwd = {s^a_j, s^c_j} after the forward pass only (coupling to the chunk's first unknown
    //         and to the next row), for the back-substitution u_j = d_j - s^a_j F - s^c_j u_{j+1}.
    const double *fwd64;
    const float *fwd32;
    const double *bwd64;
    const float *bwd32;
    // interior rows of the forward pass with f_j folded in: {f t_0, f t_1, f t_2, f r} so that
    // d_j = c1 (v[j+1] -+ v[j-1]) + c2 (v[j+2] -+ v[j-2]) (+ c0 v[j]) - g d_{j-1}; for the
    // adjoint (identity right-hand side) {f, 0, 0, f r}.  [ncls][m] records.  The FP32 copy of
    // symmetric taps holds f tapsum in place of f t_0 (the second-difference form).
    const double *ifw64;
    const float *ifw32;
    // per chunk class: rows j >= jpi carry |pi_j| below the cut-off and rows j >= jsa carry
    // |s^a_j| below it (2^-60 for FP64 sweeps, 2^-30 for FP32): those terms are not issued
    int jpi64[3], jsa64[3], jpi32[3], jsa32[3];
    int jpid[3], jsad[3];   // the same at 2^-56 for the split-precision FP64 sweeps (float pairs
                            // carry about 47 bits; the margin covers closed lines' end gain of ~100)
    // per chunk class: rows [kfl, kfh) carry the same folded forward record (bitwise, in the
    // sweep's precision) kf = {c0, c1, c2, g}, and rows [kbl, kbh) the same back-substitution
    // coupling kb = s^c_j: the forward factor converges geometrically away from the chunk's
    // first rows, so the sweeps take these rows' coefficients from registers
    int kfl64[3], kfh64[3], kbl64[3], kbh64[3], kfl32[3], kfh32[3], kbl32[3], kbh32[3];
    double kf64[3][4], kb64[3];
    float kf32[3][4], kb32[3];
    // The same records as float pairs (hi, lo) for the split-precision FP64 sweeps, [ncls][m]
    // each: fwdd {f, r, pi, 0} (8 floats), bwdd {s^a, s^c} (4), ifwd {c0, c1, c2, g} (8) with the
    // interior taps in the form those sweeps apply them (antisymmetric: c0 = 0, c1 = f t1,
    // c2 = f t2 on v[j+1] - v[j-1] and v[j+2] - v[j-2]; symmetric: c0 = f tapsum on v[j],
    // c1 = f (t1 + 2 t2) on e_j = v[j+1] - 2 v[j] + v[j-1], c2 = f t2 on e_{j+1} + e_{j-1});
    // kfd / kbd: the constant-run records (rows [kfl64, kfh64), [kbl64, kbh64)) as pairs
    const float *fwdd;
    const float *bwdd;
    const float *ifwd;
    float kfd[3][8], kbd[3][2];
    const double *n1;     // [ncls] row-0 normaliser 1/(1 - s^c_1 s^a_2) (Algorithm 4, last lines)
    const double *red;    // [kNumRedArrays][2P]
    int red_cyclic;
    int red_decoupled;    // 1: the 2P system splits into P independent 2x2 boundary systems
    double red_vlast;     // last entry of the Sherman-Morrison v vector
    double red_den_inv;   // 1/(1 + v.q)
    double tap[kTaps];                 // interior stencil taps, offsets -3..3
    double tapsum;                     // symmetric taps: t0 + 2 t1 + 2 t2 (0 for a second derivative)
    // the same taps, tap sum and second-difference weights rounded to float once on the host (FP32
    // sweeps read them without a conversion, which would issue on the FP64 pipe)
    float tap32[kTaps], tapsum32, edge_dd32[2 * kEdgeRows][5];
    double edge[2 * kEdgeRows][kTaps]; // closed lines: rows 0..3 then n-4..n-1
    float edge_pf[2 * kEdgeRows][kTaps][2]; // the same taps as float pairs (hi, lo): FP32 sweeps
                                            // evaluate closure rows with e64 in pair arithmetic
    // How each edge row is evaluated: 0 as the taps; 1 from first differences v[J+o] - v[J] (taps
    // summing to 0: rows of a first derivative); 2 from second differences with the weights
    // edge_dd (taps with vanishing sum and first moment: rows of a second derivative).  On
    // smooth data the differences of nearby values are exact, so a closure's large taps no
    // longer cancel most of an FP32 mantissa.
    int edge_form[2 * kEdgeRows];
    double edge_dd[2 * kEdgeRows][5];  // form 2: weight of v[J+k-4] - 2 v[J+k-3] + v[J+k-2], k = 1..5
};

} // namespace tds

struct tds_plan {
    int nx, ny, nz;
    tds_dir dir;
    int order;
    tds_bc bc;
    int P;
    double h;
    tds_dtype dtype;
    tds_reduced mode;
    int n, m, nlines;
    tds_variant variant;   // resolved: RESIDENT, PIPELINED, SEGMENTED or STREAMING
    int resident_smem;     // dynamic shared memory of the resident kernel (0 = cannot run)
    int width;             // lines per resident CTA: 32 (a whole group), 16 or 8
    int box_rows;          // rows per TMA tensor box when width < 32
    int smem_optin;        // device limits at plan creation: shared memory per block (opt-in)
    int smem_sm;           //   and per SM
    int nsm;               //   and the SM count
    int pipe_nbuf;         // > 0: run the persistent multi-buffered resident kernel
    int pipe_grid;         // its grid (resident CTAs the device holds at once)
    int lanes;             // lines per thread in the resident kernels (FP32: 1, 2, 4; FP64: 1, 2)
    int split;             // FP64 plans: 1 = the resident sweeps of forward-form operators carry
                           // their recurrences as float pairs (tds_plan_set_arith)
    tds::DevOp op[3];      // [0] = A^{-1} B, [1] = B^T A^{-T}, [2] = A^{-1} (the solve alone)
    tds::DevOp seg;        // A^{-1} B on the segment partition of the SEGMENTED variant (P = 0: none)
    tds::DevOp seg_adj;    // periodic lines: the adjoint (forward form) on that partition (P = 0: none)
    double *red_sub_host[2], *red_sup_host[2];
    // host entry points: two copy streams (in, out) and their events (start, done, per slab:
    // input landed, slab computed), created with the plan
    cudaStream_t copy_in, copy_out;
    cudaEvent_t ev[2 + 2 * tds::kHostSlabs];
    double *band;          // band plan: the caller's band of A (a, b, c; 3 x n), else NULL
    tds_plan *sub;         // AUTO, FP32: the same operator on finer chunks (P x 2^k), run in this
                           // plan's place when this plan's resident CTAs would be too thin; NULL
    bool is_sub;           // this plan is another plan's `sub` (it gets none of its own)
    // tds_deriv_thomas: the whole-line Thomas records (device, one allocation): [n] folded
    // forward records {f t0, f t1, f t2, f a} (FP64, then FP32 with f tapsum for t0 on
    // symmetric taps), [n] {f, c'} (FP64, FP32), and on cyclic lines z = A'^{-1} u (FP64, FP32);
    // thomas_ratio = A[0][n-1] / gamma, thomas_inv_den = 1 / (1 + v.z) (Sherman-Morrison)
    void *thomas_mem;
    double thomas_ratio, thomas_inv_den;
    // the four rows at each end of a closed line for FP32 sweeps with e64 (rows 0..3, n-4..n-1):
    // {f, c', f a} of each row as float pairs (hi, lo)
    float thomas_end_pf[2 * tds::kEdgeRows][3][2];
    void *dmem;            // one device allocation holding every array of both operators
    void *hmem;            // host copies (reduced coefficients)
};

namespace tds {

// Planner (host, FP64): fills both operator descriptors; returns TDS_ERR_ARG on a zero pivot.
tds_status build_plan(tds_plan *p);

// Kernel launchers (tds_kernels.cu).  Each returns TDS_ERR_CUDA on a launch failure.
size_t resident_smem_bytes(int n, int P, tds_dtype dtype, int w);
// Rows per TMA box for a resident CTA of w < 32 lines (m itself for w = 32); 0 when the
// chunk or box starts in the tile would not be 128-byte aligned.
int resident_box_rows(int n, int m, tds_dtype dtype, int w);
size_t pipe_smem_bytes(int n, int P, tds_dtype dtype, int nbuf, int w);
tds_status launch_resident(const tds_plan *p, int which, const void *in, void *out,
                           cudaStream_t st);
// Fused pass: operators plans[i]->op[which[i]] (forward form, one shared geometry, resident
// width and shared memory of plans[0]) of one input into outs[i].
tds_status launch_resident_multi(const tds_plan *const *plans, const int *which, int count, const void *in,
                                 void *const *outs, cudaStream_t st);
// One transport term (resident, the width and shared memory of d1): out = -1/2 (uj * D1 ui +
// D1 (uj ui)) + nu * D2 ui with d1 / d2 the first / second derivative plans of one geometry.
tds_status launch_resident_transport(const tds_plan *d1, const tds_plan *d2, const void *ui, const void *uj,
                                     double nu, void *out, cudaStream_t st);
tds_status launch_pipelined(const tds_plan *p, int which, const void *in, void *out,
                            cudaStream_t st);
size_t segmented_ws_bytes(const tds_plan *p);
tds_status launch_segmented(const tds_plan *p, int which, const void *in, void *out, void *ws,
                            cudaStream_t st);
size_t streaming_ws_bytes(const tds_plan *p);
tds_status launch_streaming(const tds_plan *p, int which, const void *in, void *out,
                            void *ws, cudaStream_t st);
tds_status launch_reduced_only(const tds_plan *p, const double *rhs, double *x,
                               cudaStream_t st);
// The plain Thomas algorithm on whole lines (tds_thomas.cu), stencil fused, cyclic lines by
// Sherman-Morrison; the plan's Thomas records must exist (p->thomas_mem).
tds_status launch_thomas(const tds_plan *p, const void *in, void *out, cudaStream_t st);
tds_status launch_reorder(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                          tds_layout to, size_t elem, cudaStream_t st);
// out += the reorder of in (the accumulation of a direction's result into another layout).
tds_status launch_reorder_add(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                              tds_layout to, size_t elem, cudaStream_t st);
// out[o] = in for o < count (<= kMaxMulti), bytes a multiple of 16 (tds_fanout_copy).
tds_status launch_fanout(const void *in, void *const *outs, int count, size_t bytes, int nsm, cudaStream_t st);
tds_status read_device_status();
// Whether operator `which` of an FP64 plan runs the split-precision sweep (the plan asks for it
// and the operator has a split form).
bool runs_split(const tds_plan *p, int which);
tds_status launch_selftest_wait(double seconds, cudaStream_t st);

} // namespace tds
