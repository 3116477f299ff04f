// Small kernels around the fit: offset validation, lambda_max, lambda path.
#include "common.cuh"

namespace ll {
namespace {

// ctrl[1] = 1 if offsets are not non-decreasing from 0 to total_rows.
__global__ void validate_offsets_kernel(const int64_t* offsets, int B, int64_t total_rows,
                                        int* ctrl) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= B; q += gridDim.x * blockDim.x) {
    int64_t o = offsets[q];
    bool bad = o < 0 || o > total_rows || (q > 0 && offsets[q - 1] > o) ||
               (q == B && o != total_rows);
    if (bad) atomicOr(ctrl + 1, 1);
  }
}

// lambda_max per problem: max_j |sum_i x_ij sign(y_i)|.  One block per
// problem (grid-stride over problems); threads stride over rows, one
// column at a time, fixed-order reductions.
__global__ void lambda_max_kernel(FitArgs a, float* lmax) {
  __shared__ float red[32];
  __shared__ int bad_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x / 32;
  const int* ctrl = a.queue;
  for (int q = blockIdx.x; q < a.B; q += gridDim.x) {
    int64_t o0 = 0, nn = 0;
    int p = a.p ? a.p[q] : a.P;
    bool ok = ctrl[1] == 0 && problem_rows(a, q, o0, nn) && nn <= (int64_t)a.n_max && p >= 1 &&
              p <= a.P;
    if (tid == 0) bad_s = ok ? 0 : 1;
    __syncthreads();
    int n = ok ? (int)nn : 0;
    float best = 0.f;
    for (int c = 0; c < p && ok; ++c) {
      float s = 0.f;
      int bad = 0;
      for (int i = tid; i < n; i += blockDim.x) {
        int64_t row = a.row_idx ? (int64_t)a.row_idx[o0 + i] : o0 + i;
        if (row < 0 || row >= a.rows_X) { bad = 1; continue; }
        float yv = a.y[o0 + i];
        float x = a.X[row * a.ldX + c];
        if (!isfinite(x) || !isfinite(yv)) bad = 1;
        s += x * fsign(yv);
      }
      if (bad) atomicOr(&bad_s, 1);
      s = warp_sum(s);
      __syncthreads();
      if (lane == 0) red[warp] = s;
      __syncthreads();
      float t = 0.f;
      for (int w = 0; w < nw; ++w) t += red[w];
      best = fmaxf(best, fabsf(t));
    }
    __syncthreads();
    if (tid == 0) lmax[q] = bad_s ? NAN : best;
    __syncthreads();
  }
}

// Work order for the persistent fit kernels: problems sorted by decreasing
// estimated cost p * (n + kStepRows) (longest first keeps the tail short).
// A fit's 1-D steps number about p per sweep, and each costs a pass over
// its n rows plus a fixed part (window sums, the buffered selection,
// barriers) that takes about as long as a pass over a thousand rows: on
// 4096 problems (n 50-2000, p 4-32) the per-problem cycle counters follow
// p * (n + 1250) closely (correlation 0.98, against 0.85 for n * p), and
// the launch on that workload takes 4 % less time than in n * p order.
// One block; counting sort over logarithmic cost buckets (order within a bucket is
// arbitrary and does not affect any result).  policy 1 interleaves the two
// ends of that order (longest, shortest, second longest, ...): the fits
// resident at one time then hold designs of mixed size, a smaller L2
// working set than the largest-first wave.  No result depends on it.
constexpr int kBuckets = 128;
constexpr int kStepRows = 1024;  // a 1-D step's fixed work, in rows
__device__ __forceinline__ int cost_bucket(const int64_t* offsets, const int32_t* nr,
                                           const int32_t* p, int P, int q) {
  int64_t n = nr ? (int64_t)nr[q] : offsets[q + 1] - offsets[q];
  int pq = p ? p[q] : P;
  if (n < 0) n = 0;
  if (pq < 0) pq = 0;
  float cost = (float)(n + kStepRows) * (float)pq;
  int b = (int)(3.f * log2f(1.f + cost));
  return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

__global__ void order_kernel(const int64_t* offsets, const int32_t* nr, const int32_t* p, int P,
                             int B, int policy, int* order) {
  __shared__ int hist[kBuckets];
  for (int b = threadIdx.x; b < kBuckets; b += blockDim.x) hist[b] = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < B; q += blockDim.x) atomicAdd(&hist[cost_bucket(offsets, nr, p, P, q)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;  // largest bucket first
    for (int b = kBuckets - 1; b >= 0; --b) { int c = hist[b]; hist[b] = run; run += c; }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < B; q += blockDim.x) {
    int pos = atomicAdd(&hist[cost_bucket(offsets, nr, p, P, q)], 1);
    if (policy == 1) pos = pos < (B + 1) / 2 ? 2 * pos : 2 * (B - 1 - pos) + 1;
    order[pos] = q;
  }
}

__global__ void lambda_path_kernel(const float* lmax, int B, int L, float ratio, float* lam) {
  int64_t total = (int64_t)B * L;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int q = (int)(e / L), l = (int)(e % L);
    float t = L > 1 ? (float)l / (float)(L - 1) : 0.f;
    lam[e] = lmax[q] * powf(ratio, t);
  }
}

// LAD loss of every path position on a row set: one block per problem
// (grid-stride), threads stride over the rows, fixed-order reductions.
// A problem with bad rows, offsets or p gets NaN.
__global__ void path_loss_kernel(const float* X, int64_t ldX, int64_t rows_X, const float* y,
                                 const int32_t* row_idx, const int64_t* offsets,
                                 int64_t total_rows, const int32_t* pv, int P, const float* b,
                                 int B, int L, float* loss) {
  __shared__ float bs[kMaxP];
  __shared__ float red[32];
  __shared__ int bad_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x / 32;
  for (int q = blockIdx.x; q < B; q += gridDim.x) {
    const int64_t o0 = offsets[q], o1 = offsets[q + 1];
    const int p = pv ? pv[q] : P;
    const bool ok = o0 >= 0 && o1 >= o0 && o1 <= total_rows && p >= 1 && p <= P;
    if (tid == 0) bad_s = ok ? 0 : 1;
    __syncthreads();
    for (int l = 0; l < L; ++l) {
      const float* bq = b + ((int64_t)q * L + l) * P;
      for (int c = tid; c < P; c += blockDim.x) bs[c] = bq[c];
      __syncthreads();
      float acc = 0.f;
      int bad = 0;
      if (ok) {
        for (int64_t i = o0 + tid; i < o1; i += blockDim.x) {
          const int64_t row = row_idx ? (int64_t)row_idx[i] : i;
          if (row < 0 || row >= rows_X) { bad = 1; continue; }
          const float* x = X + row * ldX;
          float r = y[i];
          for (int c = 0; c < p; ++c) r -= x[c] * bs[c];
          if (!isfinite(r)) bad = 1;
          acc += fabsf(r);
        }
      }
      if (bad) atomicOr(&bad_s, 1);
      acc = warp_sum(acc);
      if (lane == 0) red[warp] = acc;
      __syncthreads();
      if (tid == 0) {
        float t = 0.f;
        for (int w = 0; w < nw; ++w) t += red[w];
        loss[(int64_t)q * L + l] = bad_s ? NAN : t;
      }
      __syncthreads();
    }
  }
}

}  // namespace

cudaError_t launch_path_loss(const float* X, int64_t ldX, int64_t rows_X, const float* y,
                             const int32_t* row_idx, const int64_t* offsets, int64_t total_rows,
                             const int32_t* p, int P, const float* b, int B, int L, float* loss,
                             cudaStream_t st, int num_sms) {
  if (B <= 0) return cudaSuccess;
  int grid = B < num_sms * 8 ? B : num_sms * 8;
  path_loss_kernel<<<grid, 256, 0, st>>>(X, ldX, rows_X, y, row_idx, offsets, total_rows, p, P,
                                         b, B, L, loss);
  return cudaGetLastError();
}

cudaError_t launch_validate_offsets(const int64_t* offsets, int B, int64_t total_rows, int* ctrl,
                                    cudaStream_t st) {
  int threads = 256;
  int blocks = (B + 1 + threads - 1) / threads;
  if (blocks > 4096) blocks = 4096;
  validate_offsets_kernel<<<blocks, threads, 0, st>>>(offsets, B, total_rows, ctrl);
  return cudaGetLastError();
}

cudaError_t launch_order(const int64_t* offsets, const int32_t* nr, const int32_t* p, int P, int B,
                         int policy, int* order, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  order_kernel<<<1, 1024, 0, st>>>(offsets, nr, p, P, B, policy, order);
  return cudaGetLastError();
}

cudaError_t launch_lambda_max(const FitArgs& a, float* lmax, cudaStream_t st, int num_sms) {
  int grid = a.B < num_sms * 8 ? a.B : num_sms * 8;
  if (grid < 1) return cudaSuccess;
  lambda_max_kernel<<<grid, 256, 0, st>>>(a, lmax);
  return cudaGetLastError();
}

cudaError_t launch_lambda_path(const float* lmax, int B, int L, float ratio, float* lam,
                               cudaStream_t st) {
  int64_t total = (int64_t)B * L;
  if (total == 0) return cudaSuccess;
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 65535) blocks = 65535;
  lambda_path_kernel<<<(int)blocks, threads, 0, st>>>(lmax, B, L, ratio, lam);
  return cudaGetLastError();
}

}  // namespace ll
