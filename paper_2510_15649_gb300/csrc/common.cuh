// Shared device-side definitions for the batched LAD-LASSO library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ladlasso.h"

namespace ll {

constexpr int kFitOk = LADLASSO_FIT_OK;
constexpr int kFitMaxIters = LADLASSO_FIT_MAX_ITERS;
constexpr int kFitBadInput = LADLASSO_FIT_BAD_INPUT;
constexpr int kFitNonunique = LADLASSO_FIT_NONUNIQUE;

// Breakpoint owner codes: rows are >= 0; coordinate j is -(j+1);
// kNone marks a result strictly inside a flat segment.
constexpr int kNone = -0x40000000;
__host__ __device__ inline int coord_code(int j) { return -j - 1; }

constexpr int kMaxP = 256;  // largest supported P_cols
constexpr int kCounters = 8;  // per-fit counters (see ladlasso_dims.counters)

struct Opts {
  float tol_move;
  int max_sweeps;
  int chop;
  float chop_bracket;
  float chop_tol;
  int chop_max_probes;
  int chop_max_extend;
  int probe_max_sweeps;
  int polish;
  int max_pivots;
  float tol_opt;
  float lambda_min_floor;
  int chop_sections;  // 3 ternary, 4 four-section ("quadrature")
};

// Everything a fit kernel needs; passed by value.
struct FitArgs {
  const float* X;
  const float* y;
  const int32_t* row_idx;
  const int64_t* offsets;
  const int32_t* p;
  const int32_t* n_rows;  // optional: problem q uses the first n_rows[q] slots of its range
  const float* lambdas;
  const float* b_init;
  float* b_out;
  float* obj_out;
  int32_t* status;
  int32_t* basis_out;
  int32_t* counters;
  float* Xg;        // workspace: gathered column-major designs
  int* queue;       // workspace: work counter (queue[0]) and offsets flag (queue[1])
  int* order;       // workspace: problems in decreasing estimated cost
  unsigned char* scratch;  // workspace: per-fit scratch (thread-per-fit kernel)
  int B, P, L, n_max;
  int64_t ldX, rows_X, total_rows;
  int P4;           // P rounded up to a multiple of 4
  Opts o;
};

// Workspace layout (bytes, 256-aligned sections):
//   [0, 256)            control words (work counters)
//   order               B ints: problems in decreasing estimated cost
//   Xg                  (total_rows + 4 B) * (P4 + 4) floats: problem q's
//                       column j starts at xg_base(q) + j * ld(n_q),
//                       ld = round_up(n, 4); column slot P4 holds the edge
//                       products x_i . d of the block-per-fit polish
//   thread scratch      per-slot and per-problem scratch for the
//                       thread-per-fit kernel
__host__ __device__ inline int64_t xg_slots(int P4) { return (int64_t)P4 + 4; }
__host__ __device__ inline int64_t xg_base(int64_t off_q, int q, int P4) {
  return (off_q + 4 * (int64_t)q) * xg_slots(P4);
}
__host__ __device__ inline int64_t xg_ld(int n) { return ((int64_t)n + 3) & ~(int64_t)3; }
__host__ __device__ inline size_t ws_order_offset() { return 256; }
__host__ __device__ inline size_t ws_xg_offset(int B) {
  return 256 + ((4 * (size_t)B + 255) & ~(size_t)255);
}

// Shared-window accessors: keep hot loops on the shared-memory pipe when the
// pointer has travelled through generic code.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ float lds_f(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts_f(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void sts_i(uint32_t a, int v) {
  asm volatile("st.shared.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
// Global-window load (data written earlier in the same launch: a plain
// coherent load, kept in program order with the barriers around it).
__device__ __forceinline__ float ldg_f(const float* p) {
  float v;
  asm volatile("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(__cvta_generic_to_global(p)));
  return v;
}
// Hint: bring the 128-byte line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p)));
}
// 16-byte global -> shared copy that bypasses registers (completes
// asynchronously; wait with cp_async_wait_all).  Measured against one
// 1-D bulk copy (cp.async.bulk with an mbarrier) per column, issued by one
// thread: the bulk copy was 5 % slower on the batched workload, whose
// columns are 0.2-8 KB.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float fsign(float v) { return (float)((v > 0.f) - (v < 0.f)); }

// Rows of problem q: slots offsets[q] .. offsets[q] + n - 1 with
// n = offsets[q+1] - offsets[q], or n_rows[q] (<= that range) when given.
// Returns false on inconsistent offsets / counts.
__device__ inline bool problem_rows(const FitArgs& a, int q, int64_t& off0, int64_t& n) {
  off0 = a.offsets[q];
  const int64_t off1 = a.offsets[q + 1];
  if (off0 < 0 || off1 < off0 || off1 > a.total_rows) return false;
  n = off1 - off0;
  if (a.n_rows) {
    const int64_t m = a.n_rows[q];
    if (m < 0 || m > n) return false;
    n = m;
  }
  return true;
}

// Validate problem q; on success fill off0, n, p.  Returns false on bad input.
__device__ inline bool problem_ok(const FitArgs& a, int q, int64_t& off0, int& n, int& p,
                                  int n_cap) {
  if (a.queue[1] != 0) return false;  // offsets failed the monotonicity check
  int64_t nn = 0;
  if (!problem_rows(a, q, off0, nn)) return false;
  if (nn > (int64_t)a.n_max || nn > (int64_t)n_cap) return false;
  n = (int)nn;
  p = a.p ? a.p[q] : a.P;
  if (p < 1 || p > a.P) return false;
  return true;
}

}  // namespace ll
