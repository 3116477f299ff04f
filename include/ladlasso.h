/*
 * ladlasso.h -- C ABI of the batched LAD-LASSO coordinate-descent library
 * (CUDA, sm_103a, one GPU).
 *
 * Problem (paper, Sections 1-2): for each problem q with rows i < n_q and
 * leading columns j < p_q,
 *
 *     minimise  F_q(b) = sum_i |y_i - x_i . b|  +  lambda * sum_j |b_j|
 *
 * solved by the paper's method: cyclical coordinate descent whose axis
 * step is the exact 1-D minimiser (a weighted median, Sections 3.3-3.4),
 * a ternary chop along the locus of axis-wise minima with restricted
 * sub-searches and range extension (Sections 3.4-3.5), and an exact
 * vertex polish that certifies the LP optimum the paper's Section 3.2
 * shows lies at a vertex.  The paper's LP (Section 3.1) places its
 * constant C on the residual term; lambda here equals 1/C.
 *
 * Conventions shared by every entry point:
 *  - Every array argument is DEVICE memory owned by the caller, except
 *    `opts` (host).  The library keeps no pointer after a call returns and
 *    allocates nothing inside a call; scratch comes from the caller's
 *    workspace.
 *  - Calls are asynchronous on `stream` and never synchronise.  Outputs
 *    and per-fit status are valid once the caller synchronises the stream.
 *  - Host-checkable argument errors return a negative ladlasso_status and
 *    launch nothing.  Data-dependent errors (non-monotone offsets, a row
 *    index out of range, more rows than `n_max`, a NaN or negative lambda)
 *    never trap: they set LADLASSO_FIT_BAD_INPUT in that fit's status and
 *    zero its outputs.
 *  - A CUDA launch or runtime error returns LADLASSO_ERR_CUDA.
 *
 * Batch layout ("problem set"):
 *  - X        float [rows_X x ldX] row-major; a problem uses its leading
 *             p_q columns (p_q <= P_cols <= ldX).
 *  - y        float [total_rows]; slot t is one (problem, row) pair.
 *  - row_idx  int32 [total_rows]: row of X used by slot t; NULL means slot
 *             t uses row t of X (problems stored contiguously).
 *  - offsets  int64 [B+1]: problem q owns slots offsets[q] ..
 *             offsets[q+1]-1, so n_q = offsets[q+1] - offsets[q].
 *  - p        int32 [B] or NULL (every problem uses P_cols columns).
 * Results for problem q and path position l are stored at q*L + l;
 * coefficients at (q*L + l)*P_cols + j, zero-padded for j >= p_q.
 */
#ifndef LADLASSO_H
#define LADLASSO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ladlasso_stream_t; /* same handle as cudaStream_t */

typedef enum {
  LADLASSO_OK = 0,
  LADLASSO_ERR_INVALID = -1,   /* bad host-visible argument; nothing launched */
  LADLASSO_ERR_CUDA = -2,      /* CUDA launch/runtime error */
  LADLASSO_ERR_NOMEM = -3,     /* a size exceeds what the kernel supports */
  LADLASSO_ERR_WORKSPACE = -4  /* workspace missing or smaller than required */
} ladlasso_status;

/* Per-fit status bits (fit_status[q*L + l]). */
enum {
  LADLASSO_FIT_OK = 0,
  LADLASSO_FIT_MAX_ITERS = 1,  /* a sweep/pivot cap was hit; best point returned */
  LADLASSO_FIT_BAD_INPUT = 2,  /* data-dependent input error; outputs zeroed */
  LADLASSO_FIT_NONUNIQUE = 4   /* optimum certified but not a strict vertex */
};

/* Method options: the paper's speed/accuracy hyper-parameters (Section 5)
 * plus the exact polish controls.  Tolerances are relative to
 * max(1, |b|_inf) (moves) or max(1, lambda) (multipliers). */
typedef struct ladlasso_opts {
  float tol_move;         /* CCD stops after a sweep with max|db| below this  (1e-6) */
  int32_t max_sweeps;     /* CCD sweep cap                                    (1000) */
  int32_t chop;           /* 1: ternary chop when a CCD stall is not optimal  (1) */
  float chop_bracket;     /* initial half-range, times max(1,|b_k|)           (0.05) */
  float chop_tol;         /* chop stops at this range, times max(1,|b_k|)     (1e-3) */
  int32_t chop_max_probes;  /* ternary probes after bracketing                (12) */
  int32_t chop_max_extend;  /* range extensions (Section 3.5)                 (20) */
  int32_t probe_max_sweeps; /* restricted-CCD sweeps per probe                (4) */
  int32_t polish;         /* 1: exact vertex polish                           (1) */
  int32_t max_pivots;     /* polish step cap; 0 = 4*p + 64                    (0) */
  float tol_opt;          /* multiplier tolerance                             (2e-5) */
  float lambda_min_floor; /* lambda := max(lambda, floor), Section 3.5        (0) */
  int32_t chop_sections;  /* 3: ternary chop (Section 3.4); 4: the "quadrature"
                             search read as four sections probed at the three
                             inner points, keeping the two around the lowest
                             (Sections 1 and 5 name it, undefined)        (3) */
} ladlasso_opts;

/* Fills `o` with the defaults above.  Never fails. */
void ladlasso_default_opts(ladlasso_opts* o);

/* Problem-set dimensions and optional side arrays.
 * B        problems (>= 0)                    P_cols  columns used for b (1..256;
 *                                              the batched fit holds about 220 at most)
 * L        path length (>= 1)                 ldX     row stride of X (>= P_cols)
 * rows_X   rows of X (row_idx range check)    total_rows  offsets[B] (slots)
 * n_max    host-known bound on n_q; problems with more rows get BAD_INPUT
 * p        [B] device or NULL
 * n_rows   [B] device or NULL: problem q uses only the first n_rows[q]
 *          slots of its range offsets[q] .. offsets[q+1]-1 (a count above
 *          the range is BAD_INPUT); lets fixed-capacity slots hold problems
 *          of any size (serving)
 * b_init   [B*P_cols] device or NULL: warm start for path position 0 (may
 *          alias b_out when L == 1: each problem reads its own start before
 *          writing its result)
 * fit_status [B*L] device or NULL
 * basis_out  [B*L*P_cols] device or NULL: the final vertex's hyperplanes
 *            (row slot index i >= 0, or -(j+1) for b_j = 0); consumed by
 *            ladlasso_fit_backward
 * counters   [B*L*8] device or NULL: sweeps, chop probes, polish steps,
 *            flags (1: CCD point optimal, 2: chop ran, 4: chop point optimal;
 *            bits 3-5, batched kernel: how the pivoting polish ended, 0
 *            optimal, 1 basis cycle accepted as a degenerate optimum, 2 basis
 *            cycle with violations left, 3 pivot cap, 4 singular basis,
 *            5 flat edge),
 *            selection passes over the rows, 1-D selections, kilocycles in
 *            descent + chop, kilocycles in basis/polish work (the last four
 *            are counted by the batched kernel only, else 0)
 * workspace  device scratch of at least ladlasso_workspace_size(...) bytes,
 *            256-byte aligned; contents need not be initialised.  It serves
 *            one call at a time (it holds the call's work counter and
 *            gathered designs): calls that may run at the same time, on
 *            different streams, need workspaces of their own
 * opts     host pointer or NULL for defaults
 * group_threads   launch shape of ladlasso_fit_batched (and _noalloc):
 *            threads per fit.  0 = automatic (one warp per fit up to 8192
 *            rows, else one 512-thread block per fit); 32 = one warp per
 *            fit; 64 or 128 = two or four warps per fit (each keeps the
 *            current column in shared memory; the warps split the row
 *            passes); 512 = one block per fit (columns read from global
 *            memory); any other value is LADLASSO_ERR_INVALID.  The
 *            automatic choice also takes one block per fit when one warp's
 *            share of shared memory cannot hold n_max rows of P_cols columns
 *            but a block's can (from P_cols = 159 a warp holds fewer than
 *            8192 rows); ladlasso_launch_shape reports the limits.  The
 *            shapes sum in different orders: results agree within the
 *            float32 tolerance, not bit for bit
 * fits_per_block  shapes of up to 128 threads per fit: at most this many
 *            fits per thread block (0 = as many as shared memory holds, at
 *            most 512 threads a block, and no more than B / (SM count)
 *            rounded up, so that a small problem set still spreads over
 *            every SM); results do not depend on it.
 * work_order order in which the fits take problems: 0 = longest first
 *            (estimated cost p * (n + 1024): each 1-D step has a fixed
 *            part worth about a thousand rows), 1 = longest and shortest
 *            alternately (a smaller L2
 *            working set of resident designs); any other value is
 *            LADLASSO_ERR_INVALID.  Results do not depend on it.
 *            The three are chosen by the autotuner of the Python binding;
 *            zero-initialise them otherwise */
typedef struct ladlasso_dims {
  int32_t B, P_cols, L;
  int32_t n_max;
  int64_t ldX, rows_X, total_rows;
  const int32_t* p;
  const int32_t* n_rows;
  const float* b_init;
  int32_t* fit_status;
  int32_t* basis_out;
  int32_t* counters;
  void* workspace;
  size_t workspace_bytes;
  const ladlasso_opts* opts;
  int32_t group_threads;
  int32_t fits_per_block;
  int32_t work_order;
} ladlasso_dims;

/* Bytes of device workspace any entry point below needs for a problem set
 * of B problems, P_cols columns and total_rows slots (path length L does
 * not change it).  Returns 0 for invalid sizes. */
size_t ladlasso_workspace_size(int32_t B, int32_t P_cols, int64_t total_rows, int32_t L);

/* lambda_max per problem (Sections 2-3: the smallest lambda for which
 * b = 0 is optimal): lmax_out[q] = max_{j<p_q} |sum_i x_ij sign(y_i)|.
 * lmax_out [B] device.  Uses the same validation as ladlasso_fit_batched;
 * a problem with bad input gets lmax_out[q] = NaN. */
int ladlasso_lambda_max(const float* X, const float* y, const int32_t* row_idx,
                        const int64_t* offsets, const ladlasso_dims* dims,
                        float* lmax_out, ladlasso_stream_t stream);

/* Geometric lambda path: lambdas[q*L + l] = lmax[q] * ratio^(l/(L-1))
 * (lmax[q] alone when L == 1).  lmax [B], lambdas [B*L] device; 0 < ratio <= 1. */
int ladlasso_lambda_path(const float* lmax, int32_t B, int32_t L, float ratio,
                         float* lambdas, ladlasso_stream_t stream);

/* Fit every problem along its lambda path (descending order expected;
 * each path position warm-starts from the previous solution).
 * One warp holds one fit (several independent fits per thread block) while
 * n_max <= 8192: residual, the current and next column, selection buffer
 * and the p x p algebra in shared memory.  Beyond 8192 rows one 512-thread
 * block holds one fit: residual, selection buffers and the p x p algebra in
 * shared memory, the columns streamed from the gathered design in the
 * workspace.  Warps (blocks) take problems from a device work queue, longest
 * first.  LADLASSO_ERR_NOMEM when n_max exceeds what one block's shared
 * memory holds (23,385 rows at P_cols = 128; no row count beyond about 220
 * columns); ladlasso_launch_shape reports the exact limit.
 *   lambdas [B*L], b_out [B*L*P_cols], obj_out [B*L] device.
 * obj_out holds F at the returned b. */
int ladlasso_fit_batched(const float* X, const float* y, const int32_t* row_idx,
                         const int64_t* offsets, const float* lambdas,
                         float* b_out, float* obj_out, const ladlasso_dims* dims,
                         ladlasso_stream_t stream);

/* LAD loss of every path position on a set of held-out rows:
 *   loss_out[q*L + l] = sum over rows v of problem q of |y_v - x_v . b_{q,l}|
 * with b_{q,l} = b_out[(q*L + l)*P_cols ..] (the first p_q entries), the
 * validation loss by which a lambda is chosen (Sections 2 and 6 fit the
 * regularisation on held-out data; the paper gives no formula).  X, y,
 * row_idx, offsets and dims describe the held-out rows like a problem set
 * (dims: B, P_cols, L, ldX, rows_X, total_rows, p; other fields unused; no
 * workspace).  A problem with out-of-range rows, bad offsets or a
 * non-finite residual gets NaN.  loss_out [B*L] device.
 * LADLASSO_ERR_INVALID, before any launch, for a NULL dims, offsets, b_out
 * or loss_out, B < 0, L < 1, P_cols outside 1..256, ldX < P_cols, missing
 * X or y for a nonempty set, or more slots than X rows without row_idx. */
int ladlasso_path_loss(const float* X, const float* y, const int32_t* row_idx,
                       const int64_t* offsets, const ladlasso_dims* dims, const float* b_out,
                       float* loss_out, ladlasso_stream_t stream);

/* The launch shape ladlasso_fit_batched would use for `dims` (only
 * B-independent fields are read: P_cols, n_max, group_threads,
 * fits_per_block): threads per fit (32, 64, 128 or 512), fits per thread block, and
 * the largest n_max that shape supports at this P_cols.  No launch, no
 * device access.  Returns LADLASSO_ERR_NOMEM when n_max exceeds max_rows,
 * LADLASSO_ERR_INVALID for invalid fields.  The paper has no counterpart:
 * it serves the autotuner. */
int ladlasso_launch_shape(const ladlasso_dims* dims, int32_t* group_threads,
                          int32_t* fits_per_block, int32_t* max_rows);

/* The same method and options with one GPU thread per fit -- the layout the
 * paper proposes for a browser GPU (Sections 1 and 5) -- kept as the plain
 * comparison.  Same arguments and outputs as ladlasso_fit_batched. */
int ladlasso_fit_batched_thread(const float* X, const float* y, const int32_t* row_idx,
                                const int64_t* offsets, const float* lambdas,
                                float* b_out, float* obj_out, const ladlasso_dims* dims,
                                ladlasso_stream_t stream);

/* Gradient of a validation LAD loss sum_v |y_v - x_v . b_q| per problem at
 * the solution of one path position (implicit differentiation on the final
 * vertex; the paper has no counterpart -- it extends the method).  At a
 * strict vertex with hyperplane rows R and support S, b_S = X_{R,S}^-1 y_R
 * and b is locally independent of lambda, so with
 * g_S = -sum_v sign(r_v) x_{v,S} and X_{R,S}^T w = g_S:
 *   dL/dy_R = w, dL/dX_{R,S} = -w b_S^T, other training entries 0,
 *   dL/dy_v = sign(r_v), dL/dX_v = -sign(r_v) b^T, dL/dlambda = 0.
 * Inputs: the forward problem set (X, y, row_idx, offsets, dims; dims->L is
 * the forward path length), `pos` the path position, b_out and the
 * basis_out produced by the forward call (dims->basis_out must be set),
 * the validation set (Xv [.. x ldXv], yv, vrow_idx or NULL, voffsets [B+1]),
 * grad_up [B] the upstream derivative per problem.
 * Outputs (device, fully overwritten):
 *   grad_lambda [B]; grad_y [total_rows]; grad_X [total_rows x P_cols]
 *   (per slot, so no atomics); grad_yv [total validation rows];
 *   grad_Xv [total validation rows x P_cols].
 * A problem whose vertex is not strict gets NaN gradients and status bit
 * LADLASSO_FIT_NONUNIQUE in grad_status [B] (may be NULL).  val_loss [B]
 * (may be NULL) receives the validation loss itself.
 * Host-checkable errors, before any launch: the problem-set checks of
 * ladlasso_fit_batched; LADLASSO_ERR_INVALID for pos outside 0..L-1, a NULL
 * b_out, basis_out, voffsets, grad_up or gradient output, ldXv < P_cols,
 * total_vrows < 0, or validation rows without Xv or yv. */
int ladlasso_fit_backward(const float* X, const float* y, const int32_t* row_idx,
                          const int64_t* offsets, const ladlasso_dims* dims, int32_t pos,
                          const float* b_out, const int32_t* basis_out,
                          const float* Xv, int64_t ldXv, const float* yv,
                          const int32_t* vrow_idx, const int64_t* voffsets,
                          int64_t total_vrows, const float* grad_up,
                          float* grad_lambda, float* grad_y, float* grad_X,
                          float* grad_yv, float* grad_Xv, int32_t* grad_status,
                          float* val_loss, ladlasso_stream_t stream);

/* ladlasso_fit_batched without a caller workspace.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory when they fit -- a plugin inside a framework that owns all
 * device allocations, or a serving loop that must not call cudaMalloc (which
 * may synchronise the device) once it runs.  Same arguments, outputs, method
 * and per-fit status as ladlasso_fit_batched; dims->workspace and
 * dims->workspace_bytes are ignored.  The library allocates nothing: its
 * scratch is one fixed 32 MiB device array inside the library, which every
 * GPU that loads the library holds until the process exits.  A problem set
 * whose scratch, 256 + round_up(4*B, 256) + (total_rows + 4*B) *
 * (round_up(P_cols, 4) + 4) * 4 bytes, exceeds 32 MiB is rejected with
 * LADLASSO_ERR_NOMEM before any launch.
 * The first call on a device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * First calls from several host threads at once are safe: each looks the
 * address up and records the same value.
 * All calls on a device share the array and it keeps the last call's
 * contents: each call clears its control words itself, and calls whose
 * kernels overlap on the GPU (e.g. on two streams) race on the array --
 * serialise them. */
int ladlasso_fit_batched_noalloc(const float* X, const float* y, const int32_t* row_idx,
                                 const int64_t* offsets, const float* lambdas,
                                 float* b_out, float* obj_out, const ladlasso_dims* dims,
                                 ladlasso_stream_t stream);

/* Human-readable name of a ladlasso_status value. */
const char* ladlasso_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* LADLASSO_H */
