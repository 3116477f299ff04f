// Host side of the C ABI declared in include/ladlasso.h: argument checks,
// workspace carving and kernel launches.  No allocation, no synchronisation.
#include <string.h>

#include "common.cuh"

namespace ll {
cudaError_t launch_fit_block(const FitArgs& a, cudaStream_t st, int num_sms, int G,
                             int fits_per_block);
int launch_group(const ladlasso_dims* d);
int fit_block_fits_per_block(int G, int P, int n_max, int fits_per_block);
int fit_block_group(int n_max);
int fit_block_max_rows(int G, int P);
cudaError_t launch_fit_thread(const FitArgs& a, cudaStream_t st, int num_sms);
cudaError_t launch_validate_offsets(const int64_t* offsets, int B, int64_t total_rows, int* ctrl,
                                    cudaStream_t st);
cudaError_t launch_lambda_max(const FitArgs& a, float* lmax, cudaStream_t st, int num_sms);
cudaError_t launch_order(const int64_t* offsets, const int32_t* nr, const int32_t* p, int P, int B,
                         int policy, int* order, cudaStream_t st);
cudaError_t launch_lambda_path(const float* lmax, int B, int L, float ratio, float* lam,
                               cudaStream_t st);
cudaError_t launch_path_loss(const float* X, int64_t ldX, int64_t rows_X, const float* y,
                             const int32_t* row_idx, const int64_t* offsets, int64_t total_rows,
                             const int32_t* p, int P, const float* b, int B, int L, float* loss,
                             cudaStream_t st, int num_sms);
cudaError_t launch_backward(const FitArgs& a, int pos, const float* b_out, const int32_t* basis,
                            const float* Xv, int64_t ldXv, const float* yv, const int32_t* vrow,
                            const int64_t* voff, int64_t total_vrows, const float* gup,
                            float* glam, float* gy, float* gX, float* gyv, float* gXv,
                            int32_t* gstat, float* vloss, cudaStream_t st, int num_sms);
}  // namespace ll

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cache[dev] = v;
  }
  return cache[dev];
}

struct WsLayout {
  size_t ctrl, xg, scratch, total;
};

bool ws_layout(int32_t B, int32_t P, int64_t total_rows, WsLayout* w) {
  if (B < 0 || P < 1 || P > ll::kMaxP || total_rows < 0) return false;
  size_t P4 = ((size_t)P + 3) & ~(size_t)3;
  size_t rows = (size_t)total_rows + 4 * (size_t)B;
  w->ctrl = 0;
  w->xg = ll::ws_xg_offset(B);
  size_t xg_bytes = align256(rows * (size_t)ll::xg_slots((int)P4) * sizeof(float));
  w->scratch = w->xg + xg_bytes;
  // thread-per-fit scratch: per slot (key, weight, id, residual) for
  // total_rows + B*(P+1) slots, plus per problem a P x P matrix and 16 P-vectors
  size_t slots = (size_t)total_rows + (size_t)B * (P + 1);
  size_t per_q = ((size_t)P * P + 16 * (size_t)P) * 4;
  w->total = w->scratch + align256(slots * 16) + align256((size_t)B * per_q);
  return true;
}

ll::Opts to_opts(const ladlasso_opts* o) {
  ladlasso_opts d;
  ladlasso_default_opts(&d);
  if (!o) o = &d;
  ll::Opts r;
  r.tol_move = o->tol_move;
  r.max_sweeps = o->max_sweeps;
  r.chop = o->chop;
  r.chop_bracket = o->chop_bracket;
  r.chop_tol = o->chop_tol;
  r.chop_max_probes = o->chop_max_probes;
  r.chop_max_extend = o->chop_max_extend;
  r.probe_max_sweeps = o->probe_max_sweeps;
  r.polish = o->polish;
  r.max_pivots = o->max_pivots;
  r.tol_opt = o->tol_opt;
  r.lambda_min_floor = o->lambda_min_floor;
  r.chop_sections = o->chop_sections;
  return r;
}

bool opts_ok(const ll::Opts& o) {
  return o.tol_move >= 0.f && o.max_sweeps >= 1 && o.chop_bracket > 0.f && o.chop_tol >= 0.f &&
         o.chop_max_probes >= 0 && o.chop_max_extend >= 0 && o.probe_max_sweeps >= 1 &&
         o.max_pivots >= 0 && o.tol_opt >= 0.f && o.lambda_min_floor >= 0.f &&
         (o.chop_sections == 3 || o.chop_sections == 4);
}

// Common checks and FitArgs set-up.  Returns LADLASSO_OK or an error.
int prepare(const float* X, const float* y, const int32_t* row_idx, const int64_t* offsets,
            const ladlasso_dims* d, ll::FitArgs* a) {
  if (!d) return LADLASSO_ERR_INVALID;
  if (d->B < 0 || d->L < 1 || d->P_cols < 1 || d->P_cols > ll::kMaxP || d->ldX < d->P_cols ||
      d->rows_X < 0 || d->total_rows < 0 || d->n_max < 0)
    return LADLASSO_ERR_INVALID;
  if (!offsets) return LADLASSO_ERR_INVALID;
  if (d->total_rows > 0 && (!y || (!X && d->rows_X > 0))) return LADLASSO_ERR_INVALID;
  if (!row_idx && d->total_rows > d->rows_X) return LADLASSO_ERR_INVALID;
  WsLayout w;
  if (!ws_layout(d->B, d->P_cols, d->total_rows, &w)) return LADLASSO_ERR_INVALID;
  if (!d->workspace || d->workspace_bytes < w.total) return LADLASSO_ERR_WORKSPACE;
  if (((uintptr_t)d->workspace & 255u) != 0) return LADLASSO_ERR_WORKSPACE;
  memset(a, 0, sizeof(*a));
  a->X = X;
  a->y = y;
  a->row_idx = row_idx;
  a->offsets = offsets;
  a->p = d->p;
  a->n_rows = d->n_rows;
  a->b_init = d->b_init;
  a->status = d->fit_status;
  a->basis_out = d->basis_out;
  a->counters = d->counters;
  unsigned char* ws = (unsigned char*)d->workspace;
  a->queue = (int*)(ws + w.ctrl);
  a->order = (int*)(ws + ll::ws_order_offset());
  a->Xg = (float*)(ws + w.xg);
  a->scratch = ws + w.scratch;
  a->B = d->B;
  a->P = d->P_cols;
  a->L = d->L;
  a->n_max = d->n_max;
  a->ldX = d->ldX;
  a->rows_X = d->rows_X;
  a->total_rows = d->total_rows;
  a->P4 = (d->P_cols + 3) & ~3;
  a->o = to_opts(d->opts);
  if (!opts_ok(a->o)) return LADLASSO_ERR_INVALID;
  return LADLASSO_OK;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LADLASSO_OK : LADLASSO_ERR_CUDA; }

int start(const ll::FitArgs& a, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(a.queue, 0, 256, st);
  if (e != cudaSuccess) return LADLASSO_ERR_CUDA;
  e = ll::launch_validate_offsets(a.offsets, a.B, a.total_rows, a.queue, st);
  return cuda_status(e);
}

}  // namespace

extern "C" {

void ladlasso_default_opts(ladlasso_opts* o) {
  if (!o) return;
  o->tol_move = 1e-6f;
  o->max_sweeps = 1000;
  o->chop = 1;
  o->chop_bracket = 0.05f;
  o->chop_tol = 1e-3f;
  o->chop_max_probes = 12;
  o->chop_max_extend = 20;
  o->probe_max_sweeps = 4;
  o->polish = 1;
  o->max_pivots = 0;
  o->tol_opt = 2e-5f;
  o->lambda_min_floor = 0.f;
  o->chop_sections = 3;
}

size_t ladlasso_workspace_size(int32_t B, int32_t P_cols, int64_t total_rows, int32_t L) {
  WsLayout w;
  if (L < 1 || !ws_layout(B, P_cols, total_rows, &w)) return 0;
  return w.total;
}

int ladlasso_lambda_max(const float* X, const float* y, const int32_t* row_idx,
                        const int64_t* offsets, const ladlasso_dims* dims, float* lmax_out,
                        ladlasso_stream_t stream) {
  ll::FitArgs a;
  int rc = prepare(X, y, row_idx, offsets, dims, &a);
  if (rc != LADLASSO_OK) return rc;
  if (!lmax_out) return LADLASSO_ERR_INVALID;
  if (a.B == 0) return LADLASSO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  rc = start(a, st);
  if (rc != LADLASSO_OK) return rc;
  return cuda_status(ll::launch_lambda_max(a, lmax_out, st, num_sms()));
}

int ladlasso_lambda_path(const float* lmax, int32_t B, int32_t L, float ratio, float* lambdas,
                         ladlasso_stream_t stream) {
  if (B < 0 || L < 1 || !(ratio > 0.f && ratio <= 1.f)) return LADLASSO_ERR_INVALID;
  if (B == 0) return LADLASSO_OK;
  if (!lmax || !lambdas) return LADLASSO_ERR_INVALID;
  return cuda_status(ll::launch_lambda_path(lmax, B, L, ratio, lambdas, (cudaStream_t)stream));
}

static int fit_common(const float* X, const float* y, const int32_t* row_idx,
                      const int64_t* offsets, const float* lambdas, float* b_out, float* obj_out,
                      const ladlasso_dims* dims, ladlasso_stream_t stream, bool per_thread) {
  ll::FitArgs a;
  int rc = prepare(X, y, row_idx, offsets, dims, &a);
  if (rc != LADLASSO_OK) return rc;
  if (!lambdas || !b_out || !obj_out) return LADLASSO_ERR_INVALID;
  const int G = ll::launch_group(dims);
  if (G == 0 || dims->fits_per_block < 0 || dims->work_order < 0 || dims->work_order > 1)
    return LADLASSO_ERR_INVALID;
  if (!per_thread && dims->n_max > ll::fit_block_max_rows(G, dims->P_cols)) return LADLASSO_ERR_NOMEM;
  a.lambdas = lambdas;
  a.b_out = b_out;
  a.obj_out = obj_out;
  if (a.B == 0) return LADLASSO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  rc = start(a, st);
  if (rc != LADLASSO_OK) return rc;
  int sms = num_sms();
  if (sms <= 0) return LADLASSO_ERR_CUDA;
  if (!per_thread && ll::launch_order(a.offsets, a.n_rows, a.p, a.P, a.B, dims->work_order,
                                      a.order, st) != cudaSuccess)
    return LADLASSO_ERR_CUDA;
  cudaError_t e = per_thread ? ll::launch_fit_thread(a, st, sms)
                             : ll::launch_fit_block(a, st, sms, G, dims->fits_per_block);
  return cuda_status(e);
}

int ladlasso_fit_batched(const float* X, const float* y, const int32_t* row_idx,
                         const int64_t* offsets, const float* lambdas, float* b_out,
                         float* obj_out, const ladlasso_dims* dims, ladlasso_stream_t stream) {
  return fit_common(X, y, row_idx, offsets, lambdas, b_out, obj_out, dims, stream, false);
}

int ladlasso_path_loss(const float* X, const float* y, const int32_t* row_idx,
                       const int64_t* offsets, const ladlasso_dims* d, const float* b_out,
                       float* loss_out, ladlasso_stream_t stream) {
  if (!d || !offsets || !b_out || !loss_out) return LADLASSO_ERR_INVALID;
  if (d->B < 0 || d->L < 1 || d->P_cols < 1 || d->P_cols > ll::kMaxP || d->ldX < d->P_cols ||
      d->rows_X < 0 || d->total_rows < 0)
    return LADLASSO_ERR_INVALID;
  if (d->total_rows > 0 && (!y || (!X && d->rows_X > 0))) return LADLASSO_ERR_INVALID;
  if (!row_idx && d->total_rows > d->rows_X) return LADLASSO_ERR_INVALID;
  if (d->B == 0) return LADLASSO_OK;
  const int sms = num_sms();
  if (sms <= 0) return LADLASSO_ERR_CUDA;
  return cuda_status(ll::launch_path_loss(X, d->ldX, d->rows_X, y, row_idx, offsets,
                                          d->total_rows, d->p, d->P_cols, b_out, d->B, d->L,
                                          loss_out, (cudaStream_t)stream, sms));
}

int ladlasso_launch_shape(const ladlasso_dims* dims, int32_t* group_threads,
                          int32_t* fits_per_block, int32_t* max_rows) {
  if (!dims || !group_threads || !fits_per_block || !max_rows) return LADLASSO_ERR_INVALID;
  if (dims->P_cols < 1 || dims->P_cols > ll::kMaxP || dims->n_max < 0 || dims->fits_per_block < 0)
    return LADLASSO_ERR_INVALID;
  const int G = ll::launch_group(dims);
  if (G == 0) return LADLASSO_ERR_INVALID;
  *group_threads = G;
  *fits_per_block = ll::fit_block_fits_per_block(G, dims->P_cols, dims->n_max, dims->fits_per_block);
  *max_rows = ll::fit_block_max_rows(G, dims->P_cols);
  return dims->n_max > *max_rows ? LADLASSO_ERR_NOMEM : LADLASSO_OK;
}

int ladlasso_fit_batched_thread(const float* X, const float* y, const int32_t* row_idx,
                                const int64_t* offsets, const float* lambdas, float* b_out,
                                float* obj_out, const ladlasso_dims* dims,
                                ladlasso_stream_t stream) {
  return fit_common(X, y, row_idx, offsets, lambdas, b_out, obj_out, dims, stream, true);
}

int ladlasso_fit_backward(const float* X, const float* y, const int32_t* row_idx,
                          const int64_t* offsets, const ladlasso_dims* dims, int32_t pos,
                          const float* b_out, const int32_t* basis_out, const float* Xv,
                          int64_t ldXv, const float* yv, const int32_t* vrow_idx,
                          const int64_t* voffsets, int64_t total_vrows, const float* grad_up,
                          float* grad_lambda, float* grad_y, float* grad_X, float* grad_yv,
                          float* grad_Xv, int32_t* grad_status, float* val_loss,
                          ladlasso_stream_t stream) {
  ll::FitArgs a;
  int rc = prepare(X, y, row_idx, offsets, dims, &a);
  if (rc != LADLASSO_OK) return rc;
  if (pos < 0 || pos >= dims->L || !b_out || !basis_out || !voffsets || !grad_up ||
      !grad_lambda || !grad_y || !grad_X || !grad_yv || !grad_Xv || total_vrows < 0 ||
      ldXv < dims->P_cols)
    return LADLASSO_ERR_INVALID;
  if (total_vrows > 0 && (!yv || !Xv)) return LADLASSO_ERR_INVALID;
  if (a.B == 0) return LADLASSO_OK;
  cudaStream_t st = (cudaStream_t)stream;
  rc = start(a, st);
  if (rc != LADLASSO_OK) return rc;
  return cuda_status(ll::launch_backward(a, pos, b_out, basis_out, Xv, ldXv, yv, vrow_idx,
                                         voffsets, total_vrows, grad_up, grad_lambda, grad_y,
                                         grad_X, grad_yv, grad_Xv, grad_status, val_loss, st,
                                         num_sms()));
}

const char* ladlasso_status_string(int status) {
  switch (status) {
    case LADLASSO_OK: return "ok";
    case LADLASSO_ERR_INVALID: return "invalid argument";
    case LADLASSO_ERR_CUDA: return "CUDA error";
    case LADLASSO_ERR_NOMEM: return "size exceeds kernel limits";
    case LADLASSO_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    default: return "unknown status";
  }
}

}  // extern "C"
