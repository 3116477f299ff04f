// Adjoint of the fit: gradient of a validation LAD loss with respect to
// (lambda, y, X) by implicit differentiation at the final vertex.  The paper
// has no counterpart; this extends its method to a differentiable layer.
//
// At a strict optimal vertex the basis holds rows R and zero coordinates Z
// with |R| = |S|, S = the support.  There b_S = X_{R,S}^-1 y_R and b_Z = 0,
// independent of lambda, so for L = sum_v |y_v - x_v . b|:
//   g_S = -sum_v sign(r_v) x_{v,S};   X_{R,S}^T w = g_S
//   dL/dy_R = w,  dL/dX_{R,S} = -w b_S^T,  other training entries 0,
//   dL/dy_v = sign(r_v),  dL/dX_v = -sign(r_v) b^T,  dL/dlambda = 0.
// One block (one warp) per problem; the |S| x |S| system is solved by
// Gaussian elimination with partial pivoting in the problem's workspace slice.
#include "common.cuh"

namespace ll {
namespace {

struct BwdArgs {
  FitArgs a;
  int pos;
  const float* b_out;
  const int32_t* basis;
  const float* Xv;
  int64_t ldXv;
  const float* yv;
  const int32_t* vrow;
  const int64_t* voff;
  int64_t total_vrows;
  const float* gup;
  float* glam;
  float* gy;
  float* gX;
  float* gyv;
  float* gXv;
  int32_t* gstat;
  float* vloss;
};

__global__ void __launch_bounds__(32) backward_kernel(BwdArgs g) {
  const FitArgs& a = g.a;
  const int lane = threadIdx.x;
  const int P = a.P;
  size_t slots = (size_t)a.total_rows + (size_t)a.B * (P + 1);
  size_t slot_bytes = (slots * 16 + 255) & ~(size_t)255;
  for (int q = blockIdx.x; q < a.B; q += gridDim.x) {
    int64_t o0 = 0, nn = 0;
    int64_t v0 = g.voff[q], v1 = g.voff[q + 1];
    int p = a.p ? a.p[q] : P;
    bool ok = a.queue[1] == 0 && problem_rows(a, q, o0, nn) && p >= 1 && p <= P && v0 >= 0 &&
              v1 >= v0 && v1 <= g.total_vrows;
    int n = ok ? (int)nn : 0;
    int nv = ok ? (int)(v1 - v0) : 0;
    int64_t f = (int64_t)q * a.L + g.pos;
    const float* b = g.b_out + f * P;
    const int32_t* code = g.basis + f * P;
    float up = ok ? g.gup[q] : 0.f;
    // per-problem scratch: M [P*P], rhs/w [P], S list [P], R list [P]
    float* M = reinterpret_cast<float*>(a.scratch + slot_bytes) + (int64_t)q * ((int64_t)P * P + 16 * P);
    float* wv = M + (int64_t)P * P;
    int* S = reinterpret_cast<int*>(wv + P);
    int* R = S + P;
    // zero the training gradients of this problem
    if (ok) {
      for (int64_t e = lane; e < (int64_t)n; e += 32) g.gy[o0 + e] = 0.f;
      for (int64_t e = lane; e < (int64_t)n * P; e += 32) g.gX[o0 * P + e] = 0.f;
    }
    // supports and validity of the vertex
    int ns = 0, nr = 0;
    bool strict = ok;
    if (ok && lane == 0) {
      for (int k = 0; k < p; ++k) {
        int cd = code[k];
        if (cd >= 0) {
          if (cd >= n) strict = false;
          else R[nr++] = cd;
        }
      }
      for (int c = 0; c < p; ++c) {
        bool z = false;
        for (int k = 0; k < p; ++k) z |= code[k] == coord_code(c);
        if (!z) S[ns++] = c;
      }
      if (nr != ns) strict = false;
    }
    ns = __shfl_sync(0xffffffffu, ns, 0);
    nr = __shfl_sync(0xffffffffu, nr, 0);
    strict = __shfl_sync(0xffffffffu, (int)strict, 0) != 0;
    __syncwarp();
    // validation residual signs, direct terms and g_S
    for (int a2 = lane; a2 < ns; a2 += 32) wv[a2] = 0.f;
    __syncwarp();
    float loss = 0.f;
    for (int v = 0; v < nv; ++v) {
      int64_t row = g.vrow ? (int64_t)g.vrow[v0 + v] : v0 + v;
      const float* xr = g.Xv + row * g.ldXv;
      float s = 0.f;
      for (int c = lane; c < p; c += 32) s += xr[c] * b[c];
      s = warp_sum(s);
      const float rv = g.yv[v0 + v] - s;
      float sg = fsign(rv);
      loss += fabsf(rv);
      if (lane == 0) g.gyv[v0 + v] = up * sg;
      for (int c = lane; c < P; c += 32) g.gXv[(v0 + v) * P + c] = c < p ? -up * sg * b[c] : 0.f;
      for (int a2 = lane; a2 < ns; a2 += 32) wv[a2] -= sg * xr[S[a2]];
      __syncwarp();
    }
    // solve X_{R,S}^T w = g_S  (M[a][c] = x_{R_c, S_a})
    if (strict && ns > 0) {
      for (int e = lane; e < ns * ns; e += 32) {
        int ia = e / ns, ic = e % ns;
        int64_t row = a.row_idx ? (int64_t)a.row_idx[o0 + R[ic]] : o0 + R[ic];
        M[ia * ns + ic] = a.X[row * a.ldX + S[ia]];
      }
      __syncwarp();
      float amax = 0.f;
      for (int e = lane; e < ns * ns; e += 32) amax = fmaxf(amax, fabsf(M[e]));
      amax = warp_max(amax);
      for (int k = 0; k < ns && strict; ++k) {
        float bvv = -1.f;
        int bi = k;
        for (int i = k + lane; i < ns; i += 32)
          if (fabsf(M[i * ns + k]) > bvv) { bvv = fabsf(M[i * ns + k]); bi = i; }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          float ov = __shfl_xor_sync(0xffffffffu, bvv, o);
          int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ov > bvv || (ov == bvv && oi < bi)) { bvv = ov; bi = oi; }
        }
        if (!(bvv > 1e-7f * amax)) { strict = false; break; }
        if (bi != k) {
          for (int c = lane; c < ns; c += 32) {
            float t = M[k * ns + c]; M[k * ns + c] = M[bi * ns + c]; M[bi * ns + c] = t;
          }
          if (lane == 0) { float t = wv[k]; wv[k] = wv[bi]; wv[bi] = t; }
        }
        __syncwarp();
        float pv = M[k * ns + k];
        float rk = wv[k];
        for (int i = k + 1 + lane; i < ns; i += 32) {
          float l = M[i * ns + k] / pv;
          for (int c = k; c < ns; ++c) M[i * ns + c] -= l * M[k * ns + c];
          wv[i] -= l * rk;
        }
        __syncwarp();
      }
      if (strict) {
        for (int k = ns - 1; k >= 0; --k) {
          if (lane == 0) {
            float s = wv[k];
            for (int c = k + 1; c < ns; ++c) s -= M[k * ns + c] * wv[c];
            wv[k] = s / M[k * ns + k];
          }
          __syncwarp();
        }
        for (int c = lane; c < ns; c += 32) g.gy[o0 + R[c]] = up * wv[c];
        for (int e = lane; e < ns * ns; e += 32) {
          int ic = e / ns, ia = e % ns;
          g.gX[(o0 + R[ic]) * P + S[ia]] = -up * wv[ic] * b[S[ia]];
        }
      }
    }
    __syncwarp();
    if (lane == 0) {
      if (g.vloss) g.vloss[q] = ok ? loss : NAN;
      g.glam[q] = (ok && strict) ? 0.f : NAN;
      if (g.gstat) g.gstat[q] = !ok ? kFitBadInput : (strict ? kFitOk : kFitNonunique);
    }
    if (ok && !strict) {
      for (int64_t e = lane; e < (int64_t)n; e += 32) g.gy[o0 + e] = NAN;
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_backward(const FitArgs& a, int pos, const float* b_out, const int32_t* basis,
                            const float* Xv, int64_t ldXv, const float* yv, const int32_t* vrow,
                            const int64_t* voff, int64_t total_vrows, const float* gup,
                            float* glam, float* gy, float* gX, float* gyv, float* gXv,
                            int32_t* gstat, float* vloss, cudaStream_t st, int num_sms) {
  BwdArgs g;
  g.a = a; g.pos = pos; g.b_out = b_out; g.basis = basis; g.Xv = Xv; g.ldXv = ldXv; g.yv = yv;
  g.vrow = vrow; g.voff = voff; g.total_vrows = total_vrows; g.gup = gup; g.glam = glam;
  g.gy = gy; g.gX = gX; g.gyv = gyv; g.gXv = gXv; g.gstat = gstat; g.vloss = vloss;
  int grid = a.B < num_sms * 16 ? a.B : num_sms * 16;
  if (grid < 1) grid = 1;
  backward_kernel<<<grid, 32, 0, st>>>(g);
  return cudaGetLastError();
}

}  // namespace ll
