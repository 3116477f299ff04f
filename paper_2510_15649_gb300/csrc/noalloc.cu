// ladlasso_fit_batched_noalloc: the block-per-fit fit with its scratch in a
// fixed device array owned by this library instead of a caller workspace.
//
// Some callers cannot allocate device memory at the point where they fit:
// a plugin running inside a host framework that owns every device
// allocation, a serving loop that must not call cudaMalloc once it is
// running (cudaMalloc can synchronise the device and stall other streams),
// or code whose memory budget is fixed at start-up.  They still own their
// inputs and outputs; only the library's scratch (control words and the
// gathered designs) comes from the array below.
#include <atomic>

#include "common.cuh"

namespace ll {
cudaError_t launch_fit_block(const FitArgs& a, cudaStream_t st, int num_sms, int G,
                             int fits_per_block);
int launch_group(const ladlasso_dims* d);
cudaError_t launch_validate_offsets(const int64_t* offsets, int B, int64_t total_rows, int* ctrl,
                                    cudaStream_t st);
cudaError_t launch_order(const int64_t* offsets, const int32_t* nr, const int32_t* p, int P, int B,
                         int policy,
                         int* order, cudaStream_t st);
int fit_block_group(int n_max);
int fit_block_max_rows(int G, int P);
}  // namespace ll

using namespace ll;

namespace {

// Scratch shared by every call on a device; held by each GPU that loads the
// library until the process exits.  Layout as in the caller workspace:
// 256 bytes of control words, the work order, then the gathered designs.
constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Per-device address of g_noalloc_scratch, found once with that device
// current.  Atomic: host threads that make their first calls on one device
// at the same time each look the address up and store the same value.
constexpr int kMaxDevices = 64;
std::atomic<unsigned char*> g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LADLASSO_ERR_CUDA;
  unsigned char* ptr = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!ptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return LADLASSO_ERR_CUDA;
    ptr = (unsigned char*)p;
    g_scratch_ptr[dev].store(ptr, std::memory_order_release);
  }
  *out = ptr;
  return LADLASSO_OK;
}

}  // namespace

extern "C" int ladlasso_fit_batched_noalloc(const float* X, const float* y, const int32_t* row_idx,
                                            const int64_t* offsets, const float* lambdas,
                                            float* b_out, float* obj_out,
                                            const ladlasso_dims* d, ladlasso_stream_t stream) {
  if (!d || !offsets || !lambdas || !b_out || !obj_out) return LADLASSO_ERR_INVALID;
  if (d->B < 0 || d->L < 1 || d->P_cols < 1 || d->P_cols > kMaxP || d->ldX < d->P_cols ||
      d->rows_X < 0 || d->total_rows < 0 || d->n_max < 0)
    return LADLASSO_ERR_INVALID;
  if (d->total_rows > 0 && (!y || (!X && d->rows_X > 0))) return LADLASSO_ERR_INVALID;
  if (!row_idx && d->total_rows > d->rows_X) return LADLASSO_ERR_INVALID;
  // scratch needed: control words, work order, gathered designs (see common.cuh)
  const size_t P4 = ((size_t)d->P_cols + 3) & ~(size_t)3;
  const size_t need = ws_xg_offset(d->B) + ((size_t)d->total_rows + 4 * (size_t)d->B) *
                                                (size_t)xg_slots((int)P4) * sizeof(float);
  if (need > kScratchBytes) return LADLASSO_ERR_NOMEM;  // problem set too large for the fixed array
  const int G = launch_group(d);
  if (G == 0 || d->fits_per_block < 0 || d->work_order < 0 || d->work_order > 1)
    return LADLASSO_ERR_INVALID;
  if (d->n_max > fit_block_max_rows(G, d->P_cols)) return LADLASSO_ERR_NOMEM;
  ladlasso_opts dflt;
  ladlasso_default_opts(&dflt);
  const ladlasso_opts* o = d->opts ? d->opts : &dflt;
  if (!(o->tol_move >= 0.f && o->max_sweeps >= 1 && o->chop_bracket > 0.f &&
        o->chop_tol >= 0.f && o->chop_max_probes >= 0 && o->chop_max_extend >= 0 &&
        o->probe_max_sweeps >= 1 && o->max_pivots >= 0 && o->tol_opt >= 0.f &&
        o->lambda_min_floor >= 0.f && (o->chop_sections == 3 || o->chop_sections == 4)))
    return LADLASSO_ERR_INVALID;
  if (d->B == 0) return LADLASSO_OK;
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc != LADLASSO_OK) return rc;

  FitArgs a = {};
  a.X = X; a.y = y; a.row_idx = row_idx; a.offsets = offsets; a.p = d->p; a.n_rows = d->n_rows;
  a.lambdas = lambdas; a.b_init = d->b_init;
  a.b_out = b_out; a.obj_out = obj_out;
  a.status = d->fit_status; a.basis_out = d->basis_out; a.counters = d->counters;
  a.queue = (int*)base;
  a.order = (int*)(base + ws_order_offset());
  a.Xg = (float*)(base + ws_xg_offset(d->B));
  a.scratch = nullptr;
  a.B = d->B; a.P = d->P_cols; a.L = d->L; a.n_max = d->n_max;
  a.ldX = d->ldX; a.rows_X = d->rows_X; a.total_rows = d->total_rows;
  a.P4 = (int)P4;
  a.o = {o->tol_move, o->max_sweeps, o->chop, o->chop_bracket, o->chop_tol, o->chop_max_probes,
         o->chop_max_extend, o->probe_max_sweeps, o->polish, o->max_pivots, o->tol_opt,
         o->lambda_min_floor, o->chop_sections};
  cudaStream_t st = (cudaStream_t)stream;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return LADLASSO_ERR_CUDA;
  // the work counter and the offsets flag must start at zero on every call
  if (cudaMemsetAsync(a.queue, 0, 256, st) != cudaSuccess) return LADLASSO_ERR_CUDA;
  if (launch_validate_offsets(offsets, a.B, a.total_rows, a.queue, st) != cudaSuccess)
    return LADLASSO_ERR_CUDA;
  if (launch_order(offsets, a.n_rows, a.p, a.P, a.B, d->work_order, a.order, st) != cudaSuccess)
    return LADLASSO_ERR_CUDA;
  return launch_fit_block(a, st, sms, G, d->fits_per_block) == cudaSuccess ? LADLASSO_OK
                                                                          : LADLASSO_ERR_CUDA;
}
