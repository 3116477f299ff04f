// Batched fit kernel: a "group" of G threads owns one LAD-LASSO fit at a
// time and takes problems from a device work queue (persistent grid).
//   G = 32   one warp per fit, NW independent warps per block, no block
//            barriers; each 1-D step is one fused pass over the rows (below)
//            reading the column from a shared-memory double buffer
//   G > 32   one block per fit (long problems, or wide ones whose rows a
//            warp's share of shared memory cannot hold): the same windowed passes,
//            the warps classifying interleaved row chunks into per-warp
//            sub-buffers, the columns streamed from the gathered design
//
// Per fit:
//   shared   residual r (n floats), selection buffers of breakpoints, the
//            coefficient vector and the p x p basis algebra of the polish
//   global   the problem's design gathered column-major (workspace), so a
//            column read is one coalesced sweep
//
// Method, per lambda of the path (paper, Sections 3.3-3.5):
//   1. cyclical coordinate descent, each axis step the exact 1-D minimiser:
//      the weighted median of z_i = b_j + r_i / x_ij (weights |x_ij|) and 0
//      (weight lambda);
//   2. if the CCD fixed point is not optimal: ternary chop along the axis
//      of largest |b_k|, each probe a CCD restricted to the other axes,
//      with range extension; then CCD again;
//   3. exact polish: edge line searches between vertices (each again a
//      weighted median) until the optimality multipliers certify the vertex.
//
// Weighted median on one warp (G = 32): the target is the smallest key z*
// with W(key <= z*) >= W/2.  A pass computes every row's key on the fly,
// classifies it against a window [lo, hi] (weight below, weight inside,
// count inside) and compacts only the keys inside into a small shared
// buffer.  The window for an axis step is centred on the current b_j with
// a half-width of four times that axis' last move, so near convergence one pass holding a
// handful of keys decides the step.  A miss shrinks the open interval known
// to hold z* and draws the next window from 32 sampled keys in it; every
// pass either finishes or strictly shrinks that interval.  Sums are per-lane
// in row order then warp butterflies: deterministic for a given problem.
#include "common.cuh"

namespace ll {
namespace {

constexpr float kInf = INFINITY;
#ifndef LL_SAMPM
#define LL_SAMPM 3
#endif
#ifndef LL_WINM
#define LL_WINM 2
#endif
#ifndef LL_DLF
#define LL_DLF 4.f
#endif
constexpr int kSampM = LL_SAMPM;  // bracket half-width (samples) on buffer levels
constexpr int kWinM = LL_WINM;    // bracket half-width (samples) for pass windows
constexpr float kDlf = LL_DLF;    // axis window half-width, times the axis' last move
                                  // (4, with 2-sample pass brackets, measured best on the bench mix)
#ifndef LL_KU
#define LL_KU 1
#endif
#ifndef LL_PASSU
#define LL_PASSU 2
#endif
#ifndef LL_ROWU
#define LL_ROWU 8
#endif
#ifndef LL_FINU
#define LL_FINU 4
#endif
constexpr int kU = LL_KU;      // elements per thread per compaction chunk
constexpr int kFinU = LL_FINU; // buffered keys per lane in the selection's finish
constexpr int kFinCap = 32 * kFinU;  // the finish takes at most this many keys
constexpr int kBufCap = 256;   // selection buffer of the one-warp path
constexpr int kMaxPasses = 64; // cap on fused passes per 1-D step
constexpr int kSubCap = 128;   // block path: selection sub-buffer per warp
constexpr int kBlockG = 512;   // block path: threads per fit
constexpr int kHist = 32;               // polish: bases remembered for cycle detection
constexpr int kReanchor = 8;            // polish: pivots between residuals from the design
constexpr int kChgW = 256;              // block polish: changed rows per warp before a full recompute
constexpr float kStallTolFactor = 50.f; // cycling vertex accepted when violations are below this x tol

// Uniform per-group state, resident in shared memory.
struct St {
  float* rr;                           // residual [ncap]
  float* ck; float* cw; int* cid;      // selection buffer [cap]
  float* bv; float* bbest; float* dv; float* mu; float* tv; float* hv; float* dl;  // [P]
  float* rv;                           // [P] refinement residual
  float* Bm;                           // [P*P]
  float* red2;                         // [W*P]
  int* code; int* phan; int* piv; int* perm; int* pcol;  // [P]
  int* code_prev; int* phan_prev;  // [P] last path position's final basis
  int* code_alt; int* phan_alt;    // [P] the other polish start
  unsigned* bhist;                 // [kHist] hashes of the polish's recent bases
  // block path, incremental column sums of the polish:
  signed char* sgn;                // [ncap] sign of row i in the last sums (0 in basis)
  double* gd;                      // [P] g_c = -sum_i sgn_i x_ic
  int* chg;                        // [W * kChgW] changed rows, packed (i << 3) | (delta + 2)
  float* sk; float* sw; int* sid;      // special breakpoints [P+1]
  unsigned* mask;                      // basis-row bitmap [maskw]
  float* redf; int* redi;              // reductions [W*16]
  float* sampk; float* sampw;          // [32]
  int cap, maskw;
  int* wcnt;         // block path: keys inside the window per warp [W]
  float* vdg;        // block path: edge products x_i . d (global scratch)
  const FitArgs* a;
  const float* Xq;   // gathered design (column j at Xq + j*ld)
  float* cb[2];      // small groups: double-buffered copy of the current column
  int cur;           // buffer holding the column of the current axis step
  const float* yq;   // targets
  const float* colp; // per-row factor of the current 1-D problem: the column
                     // (axis step) or the edge products x_i . d (polish)
  float pbase;       // key offset: b_j (axis step) or 0 (edge line search)
  int pq;            // row whose key is pinned at 0 (the released basis row), or -1
  int n, p, ld, nspec, qcode;
  float lam, bj;
  // broadcast slots
  float lo, hi, acc, wpart, half, zstar, above;
  int part, m, owner, q, flag, iter, first, has_prev, bland;
  int above_ok;   // s.above is the smallest key above the buffer (not a bound)
  int need_next;  // an exact half needs the next key, which a pass must find
  int pexit;    // how the last polish ended (see polish)
  float worst;  // largest multiplier violation at the last test
  // fused-pass results
  float p_wl, p_wi, p_wt;
  int p_cnt, p_ovf;
  // per-fit counters
  int passes, selects, sel_fail;
};

// dynamic shared memory one block may take: 227 KB less the static state of
// the one-warp kernel (16 group states and the argument copy)
constexpr size_t kDynSmemLimit =
    227 * 1024 - ((16 * sizeof(St) + sizeof(FitArgs) + 256 + 1023) / 1024) * 1024;

template <int G> __device__ __forceinline__ int gtid() { return threadIdx.x & (G - 1); }
template <int G> __device__ __forceinline__ int gwarp() { return G == 32 ? 0 : (gtid<G>() >> 5); }
__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Groups of up to 128 threads keep the current column in a shared-memory
// double buffer; the block-per-fit group streams columns from global memory.
template <int G> constexpr bool kSmemCols = G <= 128;

// Barrier of one group: the warp itself, or the group's named barrier
// (id 1 + group index; barrier 0 is the block's), which also orders the
// group's shared- and global-memory accesses like __syncthreads.
template <int G>
__device__ __forceinline__ void gsync() {
  if (G == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / G)), "n"(G) : "memory");
  }
}

__device__ __forceinline__ float next_up(float v) { return v == -kInf ? v : nextafterf(v, kInf); }
__device__ __forceinline__ float next_down(float v) { return v == kInf ? v : nextafterf(v, -kInf); }

// Deterministic group reductions: warp butterflies, then warps combined in a
// fixed order.  NS float sums, NM float mins, NI int sums, NJ int mins.
template <int G, int NS, int NM, int NI, int NJ>
__device__ __forceinline__ void reduce(St& s, float (&fs)[NS], float (&mn)[NM], int (&si)[NI],
                                       int (&mi)[NJ]) {
  constexpr int W = G / 32;
#pragma unroll
  for (int e = 0; e < NS; ++e) fs[e] = warp_sum(fs[e]);
#pragma unroll
  for (int e = 0; e < NM; ++e) mn[e] = warp_min(mn[e]);
#pragma unroll
  for (int e = 0; e < NI; ++e) si[e] = warp_sum_i(si[e]);
#pragma unroll
  for (int e = 0; e < NJ; ++e) {
    int v = mi[e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    mi[e] = v;
  }
  if (W == 1) return;
  const int lane = lane_id(), warp = gwarp<G>();
  gsync<G>();
  if (lane == 0) {
#pragma unroll
    for (int e = 0; e < NS; ++e) s.redf[warp * 16 + e] = fs[e];
#pragma unroll
    for (int e = 0; e < NM; ++e) s.redf[warp * 16 + NS + e] = mn[e];
#pragma unroll
    for (int e = 0; e < NI; ++e) s.redi[warp * 16 + e] = si[e];
#pragma unroll
    for (int e = 0; e < NJ; ++e) s.redi[warp * 16 + NI + e] = mi[e];
  }
  gsync<G>();
#pragma unroll
  for (int e = 0; e < NS; ++e) {
    float t = 0.f;
    for (int w = 0; w < W; ++w) t += s.redf[w * 16 + e];
    fs[e] = t;
  }
#pragma unroll
  for (int e = 0; e < NM; ++e) {
    float t = kInf;
    for (int w = 0; w < W; ++w) t = fminf(t, s.redf[w * 16 + NS + e]);
    mn[e] = t;
  }
#pragma unroll
  for (int e = 0; e < NI; ++e) {
    int t = 0;
    for (int w = 0; w < W; ++w) t += s.redi[w * 16 + e];
    si[e] = t;
  }
#pragma unroll
  for (int e = 0; e < NJ; ++e) {
    int t = INT32_MAX;
    for (int w = 0; w < W; ++w) t = min(t, s.redi[w * 16 + NI + e]);
    mi[e] = t;
  }
}

template <int G>
__device__ __forceinline__ float gsum2(St& s, float a, float b, float& bsum) {
  float f[2] = {a, b}, m[1] = {kInf};
  int si[1] = {0}, mi[1] = {0};
  reduce<G, 2, 1, 1, 1>(s, f, m, si, mi);
  bsum = f[1];
  return f[0];
}

// Exclusive scan of per-thread counts in thread order.
template <int G>
__device__ __forceinline__ int gscan(St& s, int cnt, int& total) {
  constexpr int W = G / 32;
  const int lane = lane_id(), warp = gwarp<G>();
  int inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  int wtot = __shfl_sync(0xffffffffu, inc, 31);
  if (W == 1) { total = wtot; return inc - cnt; }
  gsync<G>();
  if (lane == 0) s.redi[warp * 16 + 15] = wtot;
  gsync<G>();
  int base = 0, tot = 0;
  for (int w = 0; w < W; ++w) {
    int c = s.redi[w * 16 + 15];
    if (w < warp) base += c;
    tot += c;
  }
  total = tot;
  return base + inc - cnt;
}

// (one warp) sort (k, w, id) ascending by (k, id) across the 32 lanes.
__device__ __forceinline__ void warp_sort(float& k, float& w, int& id) {
  const int lane = lane_id();
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      float ok = __shfl_xor_sync(0xffffffffu, k, stride);
      float ow = __shfl_xor_sync(0xffffffffu, w, stride);
      int oi = __shfl_xor_sync(0xffffffffu, id, stride);
      bool up = (lane & size) == 0;
      bool lower = (lane & stride) == 0;
      bool other_less = ok < k || (ok == k && oi < id);
      bool take = (lower == up) ? other_less : !other_less;
      if (take) { k = ok; w = ow; id = oi; }
    }
  }
}

__device__ __forceinline__ float warp_incl_scan(float v) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    float t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// ------------------------------------------------------------------ buffer selection

// (one warp) sort 32 (key, weight) samples and bracket the sample position
// where the cumulative weight reaches `frac` of the sample total.
__device__ __noinline__ void bracket_from_samples(St& s, int ns, float frac) {
  const int lane = lane_id();
  float k = lane < ns ? s.sampk[lane] : kInf;
  float w = lane < ns ? s.sampw[lane] : 0.f;
  int id = lane;
  warp_sort(k, w, id);
  float cum = warp_incl_scan(w);
  float tot = __shfl_sync(0xffffffffu, cum, 31);
  unsigned hit = __ballot_sync(0xffffffffu, cum >= frac * tot);
  int a = hit ? __ffs(hit) - 1 : 31;
  int ilo = a - kSampM, ihi = a + kSampM;
  float lo = __shfl_sync(0xffffffffu, k, max(ilo, 0));
  float hi = __shfl_sync(0xffffffffu, k, min(ihi, 31));
  if (lane == 0) {
    s.lo = ilo < 0 ? -kInf : lo;
    s.hi = ihi > 31 ? kInf : hi;
  }
  __syncwarp();
}

// Crossing at the group of keys equal to z with cumulative weight `cum`
// after it.  Exactly half: every t in [z, next] minimises; keep `cur`
// inside, else take the nearer end (the far end gets no owner: the basis
// builder then completes with coordinate hyperplanes).
__device__ __forceinline__ void flat_rule(St& s, float z, float next, float cur) {
  if (next < kInf) {
    if (cur > z && cur < next) { s.zstar = cur; s.owner = kNone; }
    else if (cur >= next) { s.zstar = next; s.owner = kNone; }
  }
}

// `next` is the smallest buffered key above z (or the kept part's upper
// bracket key); all keys outside the buffer above it are larger, so a
// finite `next` is exact.  +inf is exact only when s.above is (no key
// lies above the buffer); otherwise the caller's pass finds the key.
__device__ __forceinline__ void finalize(St& s, float z, int owner, float cum, float next,
                                         float cur) {
  s.flag = 1;
  s.zstar = z;
  s.owner = owner;
  if (cum == s.half) {
    if (next < kInf || s.above_ok) flat_rule(s, z, next, cur);
    else s.need_next = 1;
  }
}

// Thread 0: where does the cumulative weight reach half?
__device__ __forceinline__ void decide(St& s, const float (&w5)[5], const float (&mn)[2],
                                       const int (&si)[3], const int (&mi)[2], float cur) {
  float c[5];
  c[0] = s.acc + w5[0];
  c[1] = c[0] + w5[1];
  c[2] = c[1] + w5[2];
  c[3] = c[2] + w5[3];
  c[4] = c[3] + w5[4];
  // first group reaching half; rounding can leave every cumulative just
  // below it, then the last group with positive weight takes the crossing
  int g = 0;
  while (g < 4 && !(s.half <= c[g])) ++g;
  while (g > 0 && !(w5[g] > 0.f)) --g;
  s.flag = 0;
  // s.above: the smallest key above the part kept.  A bracket end is a key
  // when finite; an open end (+inf) leaves the smallest key above the
  // buffer, which the flat-segment rule needs for the next breakpoint
  if (g == 0) {
    s.part = 0; s.m = si[0]; s.wpart = w5[0];
    if (s.lo < kInf) { s.above = s.lo; s.above_ok = 1; }
  } else if (g == 1) {
    finalize(s, s.lo, mi[0], c[1], fminf(mn[0], s.above), cur);
  } else if (g == 2) {
    s.part = 2; s.m = si[1]; s.wpart = w5[2]; s.acc = c[1];
    if (s.hi < kInf) { s.above = s.hi; s.above_ok = 1; }
  } else if (g == 3) {
    finalize(s, s.hi, mi[1], c[3], fminf(mn[1], s.above), cur);
  } else {
    s.part = 4; s.m = si[2]; s.wpart = w5[4]; s.acc = c[3];
  }
}

__device__ __forceinline__ bool in_part(float kk, float lo, float hi, int part) {
  return part == 0 ? kk < lo : (part == 2 ? (kk > lo && kk < hi) : kk > hi);
}

// The key of one row: the correctly rounded quotient.  (Kept inline:
// calling it out of line, to keep one copy of the division's code, measured
// 4 % slower on the batched workload.)
__device__ __forceinline__ float key_div(float r, float x) { return __fdiv_rn(r, x); }

// (all G threads) the smallest key above z of the current 1-D problem:
// rows (the quotient r_i / x_i, IEEE; only rows whose exact quotient lies
// above z are divided), the pinned row and the special breakpoints.
// Needed only when the cumulative weight reaches exactly half at z.
template <int G>
__device__ __noinline__ float min_key_above(St& s, float z) {
  const int tid = gtid<G>();
  float m = kInf;
  for (int i = tid; i < s.n; i += G) {
    const float x = s.colp[i], r = s.rr[i];
    float k = kInf;
    if (i == s.pq) {
      k = -s.pbase;
    } else if (x != 0.f) {
      const float c = fmaf(-z, x, r);  // sign of r - z x, exact
      if (c != 0.f && signbit(c) == signbit(x)) k = key_div(r, x);
    }
    if (k > z) m = fminf(m, k);
  }
  for (int e = tid; e < s.nspec; e += G)
    if (s.sk[e] > z) m = fminf(m, s.sk[e]);
  float f[1] = {0.f}, mn[1] = {m};
  int si[1] = {0}, mi[1] = {0};
  reduce<G, 1, 1, 1, 1>(s, f, mn, si, mi);
  return mn[0];
}

// Weighted-median finish over the m0 elements of the selection buffer (ck,
// cw, ids implicit = position below s.n when `first`, else cid).  acc0 is
// the weight of all keys below the buffer's, half0 the target, above0 the
// smallest key above the buffer's (for exact halves).  Each level brackets
// the target with 32 samples, classifies the elements into (<lo, ==lo,
// (lo,hi), ==hi, >hi) with fixed-order sums and compacts the part holding
// the target in place.  At most kFinCap elements are finished by one warp,
// kFinU per lane: each element's cumulative weight is summed over the
// buffer in buffer order (a level costs more than this quadratic finish
// at these sizes).
template <int G>
__device__ __noinline__ void select_buf(St& s, int m0, float cur, int first0, float acc0,
                                        float half0, int above_ok0, float wbuf) {
  const int tid = gtid<G>(), lane = lane_id(), warp = gwarp<G>();
  gsync<G>();
  if (tid == 0) {
    s.half = half0; s.acc = acc0; s.above = kInf; s.above_ok = above_ok0; s.m = m0;
    s.first = first0; s.flag = 0; s.need_next = 0;
    s.wpart = wbuf;  // only steers the sample brackets
  }
  gsync<G>();
  const int n = s.n;
  for (;;) {
    const int m = s.m;
    const int first = s.first;
    if (m <= kFinCap) break;
    if (warp == 0) {
      int e = (int)(((int64_t)lane * m) / 32);
      s.sampk[lane] = s.ck[e];
      s.sampw[lane] = s.cw[e];
      __syncwarp();
      float wp = s.wpart;
      float frac = wp > 0.f ? (s.half - s.acc) / wp : 0.5f;
      bracket_from_samples(s, 32, fminf(fmaxf(frac, 0.f), 1.f));
    }
    gsync<G>();
    const float lo = s.lo, hi = s.hi;
    float w5[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, mn[2] = {kInf, kInf};
    int si[3] = {0, 0, 0}, mi[2] = {INT32_MAX, INT32_MAX};
    for (int e = tid; e < m; e += G) {
      float kk = s.ck[e], ww = s.cw[e];
      int id = (first && e < n) ? e : s.cid[e];
      if (kk < lo) { w5[0] += ww; si[0] += 1; }
      else if (kk == lo) { w5[1] += ww; if (ww > 0.f) mi[0] = min(mi[0], id); }
      else if (kk < hi) { w5[2] += ww; si[1] += 1; }
      else if (kk == hi) { w5[3] += ww; if (ww > 0.f) mi[1] = min(mi[1], id); }
      else { w5[4] += ww; si[2] += 1; }
      if (kk > lo) mn[0] = fminf(mn[0], kk);
      if (kk > hi) mn[1] = fminf(mn[1], kk);
    }
    reduce<G, 5, 2, 3, 2>(s, w5, mn, si, mi);
    gsync<G>();
    if (tid == 0) decide(s, w5, mn, si, mi, cur);
    gsync<G>();
    if (s.flag) break;
    const int part = s.part;
    // in-place compaction in chunks of G*kU: all reads of a chunk happen
    // before its scan barrier; writes land at positions already read
    int base = 0;
    for (int c0 = 0; c0 < m; c0 += G * kU) {
      float bk[kU], bw[kU];
      int bi[kU];
      int cnt = 0;
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        int e = c0 + u * G + tid;
        bool in = false;
        if (e < m) {
          bk[u] = s.ck[e]; bw[u] = s.cw[e];
          bi[u] = (first && e < n) ? e : s.cid[e];
          in = in_part(bk[u], lo, hi, part);
        }
        if (!in) bk[u] = NAN;  // marks "not kept"
        cnt += in;
      }
      int total, pos;
      if constexpr (G == 32 && kU == 1) {  // one warp, one element a lane
        const unsigned msk = __ballot_sync(0xffffffffu, cnt != 0);
        total = __popc(msk);
        pos = base + __popc(msk & ((1u << lane) - 1u));
      } else {
        pos = base + gscan<G>(s, cnt, total);
      }
      __syncwarp();
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (bk[u] == bk[u]) { s.ck[pos] = bk[u]; s.cw[pos] = bw[u]; s.cid[pos] = bi[u]; ++pos; }
      }
      base += total;
      gsync<G>();
    }
    if (tid == 0) s.first = 0;
    gsync<G>();
  }
  if (!s.flag && warp == 0) {
    // at most kFinCap candidates, kFinU per lane.  For each, the weight of
    // all candidates with key <= its key (one pass over the candidates in
    // buffer order, read as shared-memory broadcasts); the target key is
    // the smallest key whose cumulative weight (plus acc) reaches half.
    const int m = s.m;
    const int first = s.first;
    const float* __restrict__ ck = s.ck;
    const float* __restrict__ cw = s.cw;
    float k[kFinU], w[kFinU], cle[kFinU];
    int id[kFinU];
#pragma unroll
    for (int u = 0; u < kFinU; ++u) {
      const int e = u * 32 + lane;
      const bool have = e < m;
      k[u] = have ? ck[e] : kInf;
      w[u] = have ? cw[e] : 0.f;
      id[u] = have ? ((first && e < n) ? e : s.cid[e]) : INT32_MAX;
      cle[u] = 0.f;
    }
    for (int j = 0; j < m; ++j) {
      const float kj = ck[j], wj = cw[j];
#pragma unroll
      for (int u = 0; u < kFinU; ++u)
        if (kj <= k[u]) cle[u] += wj;
    }
    const float acc = s.acc, half = s.half;
    float zc = kInf;
#pragma unroll
    for (int u = 0; u < kFinU; ++u)
      if (u * 32 + lane < m && acc + cle[u] >= half) zc = fminf(zc, k[u]);
    float z = warp_min(zc);
    if (!(z < kInf)) {
      // rounding left every cumulative below half: the largest positive-weight key
      float zmax = -kInf;
#pragma unroll
      for (int u = 0; u < kFinU; ++u)
        if (u * 32 + lane < m && w[u] > 0.f) zmax = fmaxf(zmax, k[u]);
      z = warp_max(zmax);
    }
    int own = INT32_MAX;
    float cz = -1.f, nx = kInf;
#pragma unroll
    for (int u = 0; u < kFinU; ++u) {
      if (u * 32 + lane >= m) continue;
      if (k[u] == z) {
        if (w[u] > 0.f) own = min(own, id[u]);
        cz = cle[u];  // the same for every key equal to z
      } else if (k[u] > z) {
        nx = fminf(nx, k[u]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) own = min(own, __shfl_xor_sync(0xffffffffu, own, o));
    const float cum_g = acc + warp_max(cz);
    const float next_in = warp_min(nx);
    if (lane == 0) {
      const float next = fminf(next_in, s.above);
      if (m > 0 && z < kInf && z > -kInf) finalize(s, z, own == INT32_MAX ? kNone : own, cum_g, next, cur);
      else { s.flag = 1; s.zstar = cur; s.owner = kNone; }  // nothing selectable: no move
    }
    __syncwarp();
  }
  gsync<G>();
  if (s.need_next) {  // an exact half whose next key lies outside the buffer
    const float nx = min_key_above<G>(s, s.zstar);
    if (tid == 0) { s.need_next = 0; flat_rule(s, s.zstar, nx, cur); }
    gsync<G>();
  }
}

__device__ __forceinline__ float xval(const St& s, int c, int i) {
  return s.Xq[(int64_t)c * s.ld + i];
}
__device__ __forceinline__ const float* colptr(const St& s, int c) {
  return s.Xq + (int64_t)c * s.ld;
}

// ------------------------------------------------------------------ one-warp fused selection

// Keys are kept relative to the current value: the breakpoint of row i is
// u_i = r_i / x_i, the point t = pbase + u_i where row i's term vanishes.
//   axis step:   x_i = x_ij,    pbase = b_j, pq = -1
//   polish edge: x_i = x_i . d, pbase = 0, the released basis row pinned at
//                t = 0 (u = -pbase); other basis rows have x_i = 0
// weight |x_i|; x_i = 0 gives key +inf and no weight.  The special
// breakpoints (sk) are stored on the same relative scale.  Rows are placed
// against a window by the exact sign of r_i - t x_i (one fused multiply-
// add, see smem_rows), so the selection orders rows by their exact
// quotients; a key itself is the correctly rounded quotient (IEEE division),
// formed only for rows inside the window and for samples.
__device__ __forceinline__ void row_key(const St& s, int i, float& k, float& w) {
  const float x = s.colp[i];
  k = x != 0.f ? key_div(s.rr[i], x) : kInf;
  if (i == s.pq) k = -s.pbase;
  w = fabsf(x);
}

// Where the exact quotient r / x (x != 0) lies against the window [lo, hi]:
// r / x < lo  iff  r - lo x is nonzero with the sign opposite to x's, and
// r / x > hi  iff  r - hi x is nonzero with x's sign.  fmaf rounds once, so
// the sign of the exact difference survives.  Open ends (+-inf) place
// nothing beyond them.
__device__ __forceinline__ void place(float r, float x, float lo, float hi, bool& below,
                                      bool& above) {
  const float a = fmaf(-lo, x, r), c = fmaf(-hi, x, r);
  below = a != 0.f && signbit(a) != signbit(x);
  above = c != 0.f && signbit(c) == signbit(x);
}

// (one warp) one pass over rows and specials against the window [lo, hi]:
// weight below lo, weight at or below hi (accumulated on its own, so that
// the same set of keys always sums to the same value whichever window
// selects it), total, count inside, smallest key above hi; the first
// kBufCap keys inside go to the buffer (row order, then specials).  Rows
// are taken kPassU per lane at a time so their loads overlap.
constexpr int kPassU = LL_PASSU;
// rows per thread per batch in the whole-design loops (residual, edge
// products, column sums), which read the gathered design straight from L2
// or HBM.  The block path keeps 16 loads in flight per thread, the small
// groups 8 (measured 2 % faster than 4 on the batched workload; the fused
// pass, by contrast, is fastest with 2 rows per lane: more unrolled code
// there costs more in instruction fetch than it hides).  The rows a thread
// visits, and their order, do not depend on it.
template <int G>
constexpr int kRowU = kSmemCols<G> ? LL_ROWU : 16;

// The buffer pointers are passed in registers (restrict-qualified): going
// through the shared state struct would reload them after every store.
__device__ __forceinline__ void classify_one(float* __restrict__ bk, float* __restrict__ bw,
                                             int* __restrict__ bi, float k, float w, int id,
                                             bool valid, float lo, float hi, float& al, float& ale,
                                             float& at, int& base, int cap) {
  const int lane = lane_id();
  at += w;
  if (k < lo) al += w;
  if (k <= hi) ale += w;
  const bool in = valid && k >= lo && k <= hi;
  const unsigned msk = __ballot_sync(0xffffffffu, in);
  const int pos = base + __popc(msk & ((1u << lane) - 1u));
  if (in && pos < cap) { bk[pos] = k; bw[pos] = w; bi[pos] = id; }
  base += __popc(msk);
}

// Rows from shared memory (a per-row factor x_i and the residual r_i):
//   axis step:   x_i = x_ij,    key u_i = r_i / x_i on the scale relative
//                to b_j (pb = b_j, qc = -1), weight |x_i|
//   polish edge: x_i = x_i . d, key u_i = r_i / x_i (pb = 0), the released
//                row qc pinned at -pb
// Each row is placed against the window [lo, hi] without a division
// (place); the correctly rounded key is formed only for rows inside it.
// Batches of 32 * kPassU rows; the compaction code runs only when some lane
// of the warp holds a key inside the window.
__device__ __forceinline__ void smem_rows(uint32_t col_s, uint32_t rr_s, float pb, int qc, int n,
                                          float lo, float hi, uint32_t bk_s, uint32_t bw_s,
                                          uint32_t bi_s, float& al, float& ale, float& at,
                                          int& base) {
  const int lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const float qk = -pb;  // key of the pinned row
  for (int i0 = 0; i0 < n; i0 += 32 * kPassU) {
    float xv[kPassU], rv[kPassU];
#pragma unroll
    for (int u = 0; u < kPassU; ++u) {
      const int e = i0 + u * 32 + lane;
      xv[u] = e < n ? lds_f(col_s + 4u * e) : 0.f;
      rv[u] = e < n ? lds_f(rr_s + 4u * e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPassU; ++u) {
      if (i0 + u * 32 >= n) break;  // uniform
      const int e = i0 + u * 32 + lane;
      const float x = xv[u], r = rv[u];  // x zero beyond n: no weight, no key
      const float w = fabsf(x);
      bool below, above;
      place(r, x, lo, hi, below, above);
      const bool pin = e == qc;
      if (pin) { below = qk < lo; above = qk > hi; }
      at += w;
      al += below ? w : 0.f;
      ale += above ? 0.f : w;
      const bool in = e < n && (pin || x != 0.f) && !below && !above;
      const unsigned msk = __ballot_sync(0xffffffffu, in);
      if (msk) {
        const int pos = base + __popc(msk & lt);
        if (in && pos < kBufCap) {
          sts_f(bk_s + 4u * pos, pin ? qk : key_div(r, x));
          sts_f(bw_s + 4u * pos, w);
          sts_i(bi_s + 4u * pos, e);
        }
        base += __popc(msk);
      }
    }
  }
}

// (one warp) one pass over the rows and the special breakpoints against
// the window [lo, hi]; every lane gets the weight below lo (wl), at or
// below hi (wle), the total (wt) and the count of keys inside (cnt), the
// first kBufCap of which are in the buffer.
__device__ __noinline__ void fused_pass(St& s, float lo, float hi, float& wl_o, float& wle_o,
                                        float& wt_o, int& cnt_o) {
  const int lane = lane_id();
  const int n = s.n, nspec = s.nspec;
  float* __restrict__ bk = s.ck;
  float* __restrict__ bw = s.cw;
  int* __restrict__ bi = s.cid;
  float al = 0.f, ale = 0.f, at = 0.f;
  int base = 0;
  // one warp: the per-row factors are in shared memory (a column buffer)
  smem_rows(smem_u32(s.colp), smem_u32(s.rr), s.pbase, s.pq, n, lo, hi, smem_u32(bk),
            smem_u32(bw), smem_u32(bi), al, ale, at, base);
  const float* __restrict__ sk = s.sk;
  const float* __restrict__ sw = s.sw;
  const int* __restrict__ sid = s.sid;
  for (int j0 = 0; j0 < nspec; j0 += 32) {
    const int e = j0 + lane;
    const bool v = e < nspec;
    classify_one(bk, bw, bi, v ? sk[e] : kInf, v ? sw[e] : 0.f, v ? sid[e] : 0, v, lo, hi, al,
                 ale, at, base, kBufCap);
  }
  wl_o = warp_sum(al);
  wle_o = warp_sum(ale);
  wt_o = warp_sum(at);
  cnt_o = base;  // uniform: every lane counted every ballot
  __syncwarp();
}

// (one warp) window inside the open interval (rl, ru) around the fraction
// `frac` of its weight, from 32 sampled keys: strided rows, or strided
// buffer entries when `nbuf` > 0.  Fewer than 8 samples inside: the whole
// interval.
// (one warp) the window from one sampled key per lane (k, w).
__device__ __noinline__ void window_from_samples(St& s, float k, float w, float rl, float ru,
                                                 float frac) {
  const int lane = lane_id();
  const bool ok = k > rl && k < ru && w > 0.f;
  if (!ok) { k = kInf; w = 0.f; }
  const int cnt = __popc(__ballot_sync(0xffffffffu, ok));
  // too few samples: the closed window [rl, ru].  Rows are placed by their
  // exact quotients, and the target may lie strictly between rl and the
  // next float (or ru and the float before it), where no key value exists
  float lo = rl, hi = ru;
  if (cnt >= 8) {
    int id = lane;
    warp_sort(k, w, id);  // inside samples first, in key order
    const float cum = warp_incl_scan(w);
    const float tot = __shfl_sync(0xffffffffu, cum, 31);
    const unsigned hit = __ballot_sync(0xffffffffu, lane < cnt && cum >= frac * tot);
    const int a = hit ? __ffs(hit) - 1 : cnt - 1;
    const int ilo = a - kWinM, ihi = a + kWinM;
    const float klo = __shfl_sync(0xffffffffu, k, max(ilo, 0));
    const float khi = __shfl_sync(0xffffffffu, k, min(ihi, cnt - 1));
    if (ilo >= 0) lo = klo;
    if (ihi < cnt) hi = khi;
  }
  __syncwarp();
  if (lane == 0) { s.lo = lo; s.hi = hi; }
  __syncwarp();
}

__device__ __noinline__ void region_window(St& s, float rl, float ru, float frac, int nbuf) {
  const int lane = lane_id();
  const int n = s.n;
  float k = kInf, w = 0.f;
  if (nbuf > 0) {
    const int e = (int)(((int64_t)lane * nbuf) / 32);
    k = s.ck[e];
    w = s.cw[e];
  } else if (n > 0) {
    const int i = n >= 32 ? (int)(((int64_t)lane * n) / 32) : lane;
    if (i < n) row_key(s, i, k, w);
  }
  window_from_samples(s, k, w, rl, ru, frac);
}

// (one warp) weighted median of the current 1-D problem (rows via row_key,
// specials in sk/sw/sid).  With `prior`, the first window is [lo0, hi0].
// Result in s.zstar / s.owner.
__device__ __noinline__ void select_fused(St& s, float cur, bool prior, float lo0, float hi0) {
  const int lane = lane_id();
  float rl = -kInf, ru = kInf;  // open interval known to hold the target
  float wrl = 0.f, wru = -1.f;  // weight of keys <= rl, < ru
  float lo = lo0, hi = hi0;
  if (!prior) {
    region_window(s, rl, ru, 0.5f, 0);
    lo = s.lo; hi = s.hi;
  }
  float half = -1.f;
  if (lane == 0) s.selects++;
  for (int it = 0; it < kMaxPasses; ++it) {
    float wl, wle, wt;
    int cnt;
    fused_pass(s, lo, hi, wl, wle, wt, cnt);
    if (lane == 0) s.passes++;
    if (half < 0.f) {
      if (!(wt > 0.f)) {
        __syncwarp();
        if (lane == 0) { s.zstar = cur; s.owner = kNone; }
        __syncwarp();
        return;
      }
      half = 0.5f * wt;
      wru = wt;
    }
    if (half <= wl) {                       // target below the window
      ru = lo; wru = wl;
      region_window(s, rl, ru, (half - wrl) / fmaxf(wru - wrl, 1e-30f), 0);
    } else if (half > wle) {                // target above the window
      rl = hi; wrl = wle;
      region_window(s, rl, ru, (half - wrl) / fmaxf(wru - wrl, 1e-30f), 0);
    } else if (cnt <= kBufCap) {            // target inside, all keys buffered
      select_buf<32>(s, cnt, cur, 0, wl, half, hi == kInf, wle - wl);
      return;
    } else {                                // inside but too many keys: narrow
      rl = next_down(lo); ru = next_up(hi); wrl = wl; wru = wle;
      region_window(s, rl, ru, (half - wl) / fmaxf(wle - wl, 1e-30f), kBufCap);
      if (s.lo == lo && s.hi == hi) {
        // no narrower window from the samples (keys tie at the ends): finish
        // on the buffered keys, which begin the window in row order
        select_buf<32>(s, kBufCap, cur, 0, wl, half, hi == kInf, wle - wl);
        return;
      }
    }
    lo = s.lo; hi = s.hi;
    if (!(lo <= hi)) break;  // empty interval: only reachable through inconsistent input
  }
  __syncwarp();
  if (lane == 0) { s.zstar = cur; s.owner = kNone; s.sel_fail = 1; }
  __syncwarp();
}

// ------------------------------------------------------------------ block-per-fit fused selection
//
// The same windowed weighted median with W = G / 32 warps sharing one fit
// (long problems): warp w takes the row batches w, w + W, w + 2W, ... of
// 32 * kPU rows (kPU rows per lane) and compacts its keys inside the window into its own
// sub-buffer of kSubCap entries; per-warp sums are combined in warp order.
// The per-row factor (the column for axis steps, the edge products for the
// polish) is read from global memory, the residual from shared memory.

template <int G>
__device__ __noinline__ void fused_pass_blk(St& s, float lo, float hi) {
  constexpr int W = G / 32;
  const int lane = lane_id(), warp = gwarp<G>(), tid = gtid<G>();
  const int n = s.n, nspec = s.nspec;
  const float* __restrict__ xs = s.colp;
  uint32_t col_s = 0u;
  if constexpr (kSmemCols<G>) col_s = smem_u32(xs);
  const float bj = s.pbase;
  const int qc = s.pq;
  const uint32_t rr_s = smem_u32(s.rr);
  float* __restrict__ bk = s.ck + warp * kSubCap;
  float* __restrict__ bw = s.cw + warp * kSubCap;
  int* __restrict__ bi = s.cid + warp * kSubCap;
  const uint32_t bk_s = smem_u32(bk), bw_s = smem_u32(bw), bi_s = smem_u32(bi);
  const unsigned lt = (1u << lane) - 1u;
  float al = 0.f, ale = 0.f, at = 0.f;
  int base = 0;
  const float qk = -bj;  // key of the pinned row
  // rows per lane per batch: columns read from global memory (the block
  // shape) keep four loads in flight, shared-memory columns two
  constexpr int kPU = kSmemCols<G> ? kPassU : 4;
  for (int i0 = warp * 32 * kPU; i0 < n; i0 += G * kPU) {
    float xv[kPU], rv[kPU];
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      const int e = i0 + u * 32 + lane;
      if constexpr (kSmemCols<G>) xv[u] = e < n ? lds_f(col_s + 4u * e) : 0.f;
      else xv[u] = e < n ? ldg_f(xs + e) : 0.f;
      rv[u] = e < n ? lds_f(rr_s + 4u * e) : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPU; ++u) {
      if (i0 + u * 32 >= n) break;  // uniform
      const int e = i0 + u * 32 + lane;
      const float x = xv[u], r = rv[u];  // x zero beyond n: no weight, no key
      const float w = fabsf(x);
      bool below, above;
      place(r, x, lo, hi, below, above);
      const bool pin = e == qc;
      if (pin) { below = qk < lo; above = qk > hi; }
      at += w;
      al += below ? w : 0.f;
      ale += above ? 0.f : w;
      const bool in = e < n && (pin || x != 0.f) && !below && !above;
      const unsigned msk = __ballot_sync(0xffffffffu, in);
      if (msk) {
        const int pos = base + __popc(msk & lt);
        if (in && pos < kSubCap) {
          sts_f(bk_s + 4u * pos, pin ? qk : key_div(r, x));
          sts_f(bw_s + 4u * pos, w);
          sts_i(bi_s + 4u * pos, e);
        }
        base += __popc(msk);
      }
    }
  }
  if (warp == 0) {
    for (int j0 = 0; j0 < nspec; j0 += 32) {
      const int e = j0 + lane;
      const bool v = e < nspec;
      classify_one(bk, bw, bi, v ? s.sk[e] : kInf, v ? s.sw[e] : 0.f, v ? s.sid[e] : 0, v, lo, hi,
                   al, ale, at, base, kSubCap);
    }
  }
  al = warp_sum(al);
  ale = warp_sum(ale);
  at = warp_sum(at);
  if (lane == 0) {
    s.redf[warp * 16 + 0] = al;
    s.redf[warp * 16 + 1] = ale;
    s.redf[warp * 16 + 2] = at;
    s.wcnt[warp] = base;
  }
  gsync<G>();
  if (tid == 0) {
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    int c = 0, ov = 0;
    for (int w = 0; w < W; ++w) {
      a0 += s.redf[w * 16 + 0];
      a1 += s.redf[w * 16 + 1];
      a2 += s.redf[w * 16 + 2];
      c += s.wcnt[w];
      ov |= s.wcnt[w] > kSubCap;
    }
    s.p_wl = a0; s.p_wi = a1; s.p_wt = a2; s.p_cnt = c; s.p_ovf = ov;
  }
  gsync<G>();
}

// Move the buffered keys of every warp (up to kSubCap each) to the front of
// the selection buffer, in warp order.  Returns their number.
template <int G>
__device__ __forceinline__ int compact_sub(St& s) {
  constexpr int W = G / 32, kPer = kSubCap / 32;
  const int lane = lane_id(), warp = gwarp<G>();
  int pre = 0, tot = 0;
  for (int w = 0; w < W; ++w) {
    const int c = min(s.wcnt[w], kSubCap);
    if (w < warp) pre += c;
    tot += c;
  }
  const int c = min(s.wcnt[warp], kSubCap);
  float k[kPer], wv[kPer];
  int id[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = u * 32 + lane;
    if (e < c) {
      k[u] = s.ck[warp * kSubCap + e];
      wv[u] = s.cw[warp * kSubCap + e];
      id[u] = s.cid[warp * kSubCap + e];
    }
  }
  gsync<G>();
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int e = u * 32 + lane;
    if (e < c) { s.ck[pre + e] = k[u]; s.cw[pre + e] = wv[u]; s.cid[pre + e] = id[u]; }
  }
  gsync<G>();
  return tot;
}

// (warp 0) window from keys spread over the warps' sub-buffers.
template <int G>
__device__ __noinline__ void sub_window(St& s, float rl, float ru, float frac) {
  constexpr int W = G / 32, kPerW = 32 / W;
  const int lane = lane_id();
  const int w = lane % W, r = lane / W;
  const int c = min(s.wcnt[w], kSubCap);
  float k = kInf, wt = 0.f;
  if (c > 0) {
    const int e = (r * c) / kPerW;
    k = s.ck[w * kSubCap + e];
    wt = s.cw[w * kSubCap + e];
  }
  window_from_samples(s, k, wt, rl, ru, frac);
}

// Block version of select_fused (same contract).
template <int G>
__device__ __noinline__ void select_fused_blk(St& s, float cur, bool prior, float lo0, float hi0) {
  const int tid = gtid<G>(), warp = gwarp<G>();
  float rl = -kInf, ru = kInf;  // open interval known to hold the target
  float wrl = 0.f, wru = -1.f;  // weight of keys <= rl, < ru
  float lo = lo0, hi = hi0;
  gsync<G>();
  if (!prior) {
    if (warp == 0) region_window(s, rl, ru, 0.5f, 0);
    gsync<G>();
    lo = s.lo; hi = s.hi;
  }
  float half = -1.f;
  if (tid == 0) s.selects++;
  for (int it = 0; it < kMaxPasses; ++it) {
    fused_pass_blk<G>(s, lo, hi);
    if (tid == 0) s.passes++;
    const float wl = s.p_wl, wle = s.p_wi, wt = s.p_wt;
    const int cnt = s.p_cnt, ovf = s.p_ovf;
    if (half < 0.f) {
      if (!(wt > 0.f)) {
        gsync<G>();
        if (tid == 0) { s.zstar = cur; s.owner = kNone; }
        gsync<G>();
        return;
      }
      half = 0.5f * wt;
      wru = wt;
    }
    if (half <= wl) {                       // target below the window
      ru = lo; wru = wl;
      if (warp == 0) region_window(s, rl, ru, (half - wrl) / fmaxf(wru - wrl, 1e-30f), 0);
    } else if (half > wle) {                // target above the window
      rl = hi; wrl = wle;
      if (warp == 0) region_window(s, rl, ru, (half - wrl) / fmaxf(wru - wrl, 1e-30f), 0);
    } else if (!ovf) {                      // target inside, all keys buffered
      compact_sub<G>(s);
      select_buf<G>(s, cnt, cur, 0, wl, half, hi == kInf, wle - wl);
      return;
    } else {                                // inside but too many keys: narrow
      rl = next_down(lo); ru = next_up(hi); wrl = wl; wru = wle;
      if (warp == 0) sub_window<G>(s, rl, ru, (half - wl) / fmaxf(wle - wl, 1e-30f));
      gsync<G>();
      if (s.lo == lo && s.hi == hi) {
        // no narrower window from the samples (keys tie at the ends): finish
        // on the buffered keys
        const int m = compact_sub<G>(s);
        select_buf<G>(s, m, cur, 0, wl, half, hi == kInf, wle - wl);
        return;
      }
    }
    gsync<G>();
    lo = s.lo; hi = s.hi;
    if (!(lo <= hi)) break;  // empty interval: only reachable through inconsistent input
  }
  gsync<G>();
  if (tid == 0) { s.zstar = cur; s.owner = kNone; s.sel_fail = 1; }
  gsync<G>();
}

// ------------------------------------------------------------------ warp-0 algebra

// (one warp) normal of constraint `cd` into v[0..p)
__device__ __forceinline__ void normal_to(St& s, int cd, float* v) {
  const int lane = lane_id();
  for (int c = lane; c < s.p; c += 32)
    v[c] = cd >= 0 ? xval(s, c, cd) : (c == -cd - 1 ? 1.f : 0.f);
}

// (one warp) try to add constraint cd to the echelon rows Bm[0..m)
__device__ __noinline__ bool try_add(St& s, int cd, int m) {
  const int lane = lane_id(), p = s.p;
  float* v = s.tv;
  normal_to(s, cd, v);
  __syncwarp();
  float vmax0 = 0.f;
  for (int c = lane; c < p; c += 32) vmax0 = fmaxf(vmax0, fabsf(v[c]));
  vmax0 = warp_max(vmax0);
  if (!(vmax0 > 0.f)) return false;
  for (int q = 0; q < m; ++q) {
    const float* e = s.Bm + q * p;
    float f = v[s.pcol[q]] / e[s.pcol[q]];
    __syncwarp();
    if (f != 0.f)
      for (int c = lane; c < p; c += 32) v[c] -= f * e[c];
    __syncwarp();
  }
  float bvv = 0.f;
  int bj = p;
  for (int c = lane; c < p; c += 32)
    if (fabsf(v[c]) > bvv) { bvv = fabsf(v[c]); bj = c; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, bvv, o);
    int oj = __shfl_xor_sync(0xffffffffu, bj, o);
    if (ov > bvv || (ov == bvv && oj < bj)) { bvv = ov; bj = oj; }
  }
  if (!(bvv > 1e-4f * vmax0)) return false;
  for (int c = lane; c < p; c += 32) s.Bm[m * p + c] = v[c];
  if (lane == 0) s.pcol[m] = bj;
  __syncwarp();
  return true;
}

// (one warp) basis at a CCD fixed point: the hyperplanes the axis steps
// landed on (kept when independent), completed with coordinate hyperplanes.
__device__ __noinline__ void build_basis(St& s) {
  const int lane = lane_id(), p = s.p;
  int m = 0;
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = 0; j < p && m < p; ++j) {
      int cd;
      if (pass == 0) {
        int pv = s.piv[j];
        if (pv == -2) continue;
        cd = pv >= 0 ? pv : coord_code(j);
      } else {
        cd = coord_code(j);
      }
      bool dup = false;
      for (int q = 0; q < m; ++q) dup |= s.code[q] == cd;
      if (dup) continue;
      if (try_add(s, cd, m)) {
        if (lane == 0) { s.code[m] = cd; s.phan[m] = pass == 1 && s.bv[j] != 0.f; }
        __syncwarp();
        ++m;
      }
    }
  }
  for (int j = 0; m < p && j < p; ++j) {  // unreachable: coordinates span
    if (lane == 0) { s.code[m] = coord_code(j); s.phan[m] = s.bv[j] != 0.f; }
    __syncwarp();
    ++m;
  }
}

// (one warp) LU with partial pivoting of Bm in place; perm[k] = original row.
__device__ __noinline__ bool lu(St& s) {
  const int lane = lane_id(), p = s.p;
  float* B = s.Bm;
  for (int c = lane; c < p; c += 32) s.perm[c] = c;
  float amax = 0.f;
  for (int e = lane; e < p * p; e += 32) amax = fmaxf(amax, fabsf(B[e]));
  amax = warp_max(amax);
  __syncwarp();
  for (int k = 0; k < p; ++k) {
    float bvv = -1.f;
    int bi = k;
    for (int i = k + lane; i < p; i += 32)
      if (fabsf(B[i * p + k]) > bvv) { bvv = fabsf(B[i * p + k]); bi = i; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      float ov = __shfl_xor_sync(0xffffffffu, bvv, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bvv || (ov == bvv && oi < bi)) { bvv = ov; bi = oi; }
    }
    if (!(bvv > 1e-7f * amax)) return false;
    if (bi != k) {
      for (int c = lane; c < p; c += 32) {
        float t = B[k * p + c]; B[k * p + c] = B[bi * p + c]; B[bi * p + c] = t;
      }
      if (lane == 0) { int t = s.perm[k]; s.perm[k] = s.perm[bi]; s.perm[bi] = t; }
    }
    __syncwarp();
    float pv = B[k * p + k];
    for (int i = k + 1 + lane; i < p; i += 32) B[i * p + k] /= pv;
    __syncwarp();
    // trailing update, rows in turn, lanes over columns (no index division)
    for (int i = k + 1; i < p; ++i) {
      const float l = B[i * p + k];
      if (l != 0.f)
        for (int c = k + 1 + lane; c < p; c += 32) B[i * p + c] -= l * B[k * p + c];
    }
    __syncwarp();
  }
  return true;
}

// (one warp) solve B x = rhs, rhs in x (overwritten), with the LU in Bm.
__device__ __noinline__ void lu_solve(St& s, float* x) {
  const int lane = lane_id(), p = s.p;
  const float* B = s.Bm;
  float* t = s.tv;
  for (int c = lane; c < p; c += 32) t[c] = x[s.perm[c]];
  __syncwarp();
  for (int k = 0; k < p; ++k) {
    float v = t[k];
    for (int i = k + 1 + lane; i < p; i += 32) t[i] -= B[i * p + k] * v;
    __syncwarp();
  }
  for (int k = p - 1; k >= 0; --k) {
    if (lane == 0) t[k] /= B[k * p + k];
    __syncwarp();
    float v = t[k];
    for (int i = lane; i < k; i += 32) t[i] -= B[i * p + k] * v;
    __syncwarp();
  }
  for (int c = lane; c < p; c += 32) x[c] = t[c];
  __syncwarp();
}

// (one warp) solve B^T x = rhs with the LU (B = P^T L U).
__device__ __noinline__ void lu_solve_t(St& s, float* x) {
  const int lane = lane_id(), p = s.p;
  const float* B = s.Bm;
  float* t = s.tv;
  for (int c = lane; c < p; c += 32) t[c] = x[c];
  __syncwarp();
  for (int k = 0; k < p; ++k) {
    if (lane == 0) t[k] /= B[k * p + k];
    __syncwarp();
    float v = t[k];
    for (int i = k + 1 + lane; i < p; i += 32) t[i] -= B[k * p + i] * v;
    __syncwarp();
  }
  for (int k = p - 1; k >= 0; --k) {
    float v = t[k];
    for (int i = lane; i < k; i += 32) t[i] -= B[k * p + i] * v;
    __syncwarp();
  }
  for (int c = lane; c < p; c += 32) x[s.perm[c]] = t[c];
  __syncwarp();
}

// (one warp) one step of iterative refinement of x solving B x = h
// (trans = false) or B^T x = h (trans = true) with the FP32 factors in Bm:
// the residual is formed in FP64 from the basis normals (rows of X and unit
// vectors, exact in FP32), the correction solved with the factors.  At
// p = 128 the FP32 solve alone leaves multiplier errors of the order of the
// optimality tolerance.
__device__ __noinline__ void refine(St& s, float* x, const float* h, bool trans) {
  const int lane = lane_id(), p = s.p;
  for (int e = lane; e < p; e += 32) {
    double acc = 0.0;
    if (!trans) {  // e: basis position
      const int cd = s.code[e];
      if (cd >= 0)
        for (int c = 0; c < p; ++c) acc += (double)xval(s, c, cd) * (double)x[c];
      else
        acc = (double)x[-cd - 1];
    } else {       // e: column
      for (int k = 0; k < p; ++k) {
        const int cd = s.code[k];
        const float nv = cd >= 0 ? xval(s, e, cd) : (e == -cd - 1 ? 1.f : 0.f);
        acc += (double)nv * (double)x[k];
      }
    }
    s.rv[e] = (float)((double)h[e] - acc);
  }
  __syncwarp();
  if (trans) lu_solve_t(s, s.rv);
  else lu_solve(s, s.rv);
  for (int e = lane; e < p; e += 32) x[e] += s.rv[e];
  __syncwarp();
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (all G threads) LU with partial pivoting of Bm in place, the row
// operations of each elimination step spread over the block; the pivot
// choice is the one-warp routine's (largest |entry|, lowest row on ties).
template <int G>
__device__ __noinline__ bool lu_blk(St& s) {
  const int tid = gtid<G>(), lane = lane_id(), warp = gwarp<G>(), p = s.p;
  float* B = s.Bm;
  for (int c = tid; c < p; c += G) s.perm[c] = c;
  float am = 0.f;
  for (int e = tid; e < p * p; e += G) am = fmaxf(am, fabsf(B[e]));
  {
    float f[1] = {0.f}, m[1] = {-am};
    int si[1] = {0}, mi[1] = {0};
    reduce<G, 1, 1, 1, 1>(s, f, m, si, mi);
    am = -m[0];
  }
  for (int k = 0; k < p; ++k) {
    if (warp == 0) {
      float bvv = -1.f;
      int bi = k;
      for (int i = k + lane; i < p; i += 32)
        if (fabsf(B[i * p + k]) > bvv) { bvv = fabsf(B[i * p + k]); bi = i; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, bvv, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bvv || (ov == bvv && oi < bi)) { bvv = ov; bi = oi; }
      }
      if (lane == 0) { s.m = bi; s.flag = bvv > 1e-7f * am; }
    }
    gsync<G>();
    if (!s.flag) return false;  // uniform
    const int bi = s.m;
    if (bi != k) {
      for (int c = tid; c < p; c += G) {
        float t = B[k * p + c]; B[k * p + c] = B[bi * p + c]; B[bi * p + c] = t;
      }
      if (tid == 0) { int t = s.perm[k]; s.perm[k] = s.perm[bi]; s.perm[bi] = t; }
    }
    gsync<G>();
    const float pv = B[k * p + k];
    for (int i = k + 1 + tid; i < p; i += G) B[i * p + k] /= pv;
    gsync<G>();
    // trailing update: warps over rows, lanes over columns (no index division)
    for (int i = k + 1 + warp; i < p; i += G / 32) {
      const float l = B[i * p + k];
      if (l != 0.f)
        for (int c = k + 1 + lane; c < p; c += 32) B[i * p + c] -= l * B[k * p + c];
    }
    gsync<G>();
  }
  return true;
}

// (all G threads) the refinement of `refine` with the FP64 residual
// spread over the warps (one basis position or column per warp, lanes over
// the inner index); warp 0 solves for the correction.
template <int G>
__device__ __noinline__ void refine_blk(St& s, float* x, const float* h, bool trans) {
  constexpr int W = G / 32;
  const int lane = lane_id(), warp = gwarp<G>(), p = s.p;
  gsync<G>();
  for (int e = warp; e < p; e += W) {
    double acc = 0.0;
    if (!trans) {
      const int cd = s.code[e];
      if (cd >= 0) {
        for (int c = lane; c < p; c += 32) acc += (double)xval(s, c, cd) * (double)x[c];
      } else if (lane == 0) {
        acc = (double)x[-cd - 1];
      }
    } else {
      for (int k = lane; k < p; k += 32) {
        const int cd = s.code[k];
        const float nv = cd >= 0 ? xval(s, e, cd) : (e == -cd - 1 ? 1.f : 0.f);
        acc += (double)nv * (double)x[k];
      }
    }
    acc = warp_sum_d(acc);
    if (lane == 0) s.rv[e] = (float)((double)h[e] - acc);
  }
  gsync<G>();
  if (warp == 0) {
    if (trans) lu_solve_t(s, s.rv);
    else lu_solve(s, s.rv);
    for (int e = lane; e < p; e += 32) x[e] += s.rv[e];
  }
  gsync<G>();
}

// (one warp) form the basis matrix, factor it and snap b onto the basis
// hyperplanes (phantom coordinates keep their value).  Sets s.flag.
__device__ __noinline__ void snap(St& s) {
  const int lane = lane_id(), p = s.p;
  // basis matrix rows = constraint normals; element (k, c) of a row
  // constraint is x_{code_k, c}: strided loads, eight rows at a time so
  // that eight loads per lane are in flight
  for (int k0 = 0; k0 < p; k0 += 8) {
    for (int c = lane; c < p; c += 32) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int k = k0 + u;
        v[u] = 0.f;
        if (k < p) {
          const int cd = s.code[k];
          v[u] = cd >= 0 ? xval(s, c, cd) : (c == -cd - 1 ? 1.f : 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (k0 + u < p) s.Bm[(k0 + u) * p + c] = v[u];
    }
  }
  for (int k = lane; k < p; k += 32) {
    int cd = s.code[k];
    s.hv[k] = cd >= 0 ? s.yq[cd] : (s.phan[k] ? s.bv[-cd - 1] : 0.f);
  }
  __syncwarp();
  for (int k = lane; k < p; k += 32) s.mu[k] = s.hv[k];  // right-hand side (mu is free here)
  __syncwarp();
  bool ok = lu(s);
  if (lane == 0) s.flag = ok;
  if (ok) {
    lu_solve(s, s.hv);
    refine(s, s.hv, s.mu, false);
    for (int c = lane; c < p; c += 32) s.bv[c] = s.hv[c];
    __syncwarp();
    for (int k = lane; k < p; k += 32)
      if (s.code[k] < 0 && !s.phan[k]) s.bv[-s.code[k] - 1] = 0.f;
  }
  __syncwarp();
}

// (all G threads) snap: the one-warp routine for a warp; for a block the
// basis matrix is formed, factored and refined by all warps.
template <int G>
__device__ __noinline__ void snap_g(St& s) {
  if (G == 32) {
    snap(s);
    return;
  }
  if (kSmemCols<G>) {  // small groups: p <= 256 algebra on warp 0
    if (gwarp<G>() == 0) snap(s);
    gsync<G>();
    return;
  }
  const int tid = gtid<G>(), warp = gwarp<G>(), lane = lane_id(), p = s.p;
  for (int k = warp; k < p; k += G / 32) {  // warps over rows, lanes over columns
    const int cd = s.code[k];
#pragma unroll 4
    for (int c = lane; c < p; c += 32)
      s.Bm[k * p + c] = cd >= 0 ? xval(s, c, cd) : (c == -cd - 1 ? 1.f : 0.f);
  }
  for (int k = tid; k < p; k += G) {
    const int cd = s.code[k];
    const float h = cd >= 0 ? s.yq[cd] : (s.phan[k] ? s.bv[-cd - 1] : 0.f);
    s.hv[k] = h;
    s.mu[k] = h;  // right-hand side (mu is free here)
  }
  gsync<G>();
  const bool ok = lu_blk<G>(s);  // group-uniform
  if (ok) {
    if (warp == 0) lu_solve(s, s.hv);
    refine_blk<G>(s, s.hv, s.mu, false);
    for (int c = tid; c < p; c += G) s.bv[c] = s.hv[c];
    gsync<G>();
    for (int k = tid; k < p; k += G)
      if (s.code[k] < 0 && !s.phan[k]) s.bv[-s.code[k] - 1] = 0.f;
  }
  gsync<G>();
  if (tid == 0) s.flag = ok;
  gsync<G>();
}

// (one warp) multipliers from the column sums in red2: right-hand side
// into mu and hv, mu := B^-T mu (refined by the caller).
template <int G>
__device__ __noinline__ void mult_solve(St& s) {
  constexpr int W = G / 32;
  const int lane = lane_id(), p = s.p;
  const float lam = s.lam;
  for (int c = lane; c < p; c += 32) {
    float g = 0.f;
    for (int w = 0; w < W; ++w) g += s.red2[w * p + c];
    bool real = false;
    for (int k = 0; k < p; ++k) real |= (s.code[k] == coord_code(c) && !s.phan[k]);
    if (!real) g += lam * fsign(s.bv[c]);
    s.mu[c] = -g;
    s.hv[c] = -g;  // right-hand side (hv is free after the snap)
  }
  __syncwarp();
  lu_solve_t(s, s.mu);
}

// (one warp) pick the most violated basis hyperplane (Bland's rule: the
// lowest id) and, if stepping, the edge direction dv.
__device__ __noinline__ void mult_pick(St& s, bool step) {
  const int lane = lane_id(), p = s.p;
  const float lam = s.lam;
  const float tol = s.a->o.tol_opt * fmaxf(1.f, lam);
  float worst = tol, vmax = 0.f;
  int q = -1, phantoms = 0, atcap = 0, lowest = INT32_MAX, qb = -1;
  for (int k = lane; k < p; k += 32) {
    float cap = s.code[k] >= 0 ? 1.f : (s.phan[k] ? 0.f : lam);
    float viol = fabsf(s.mu[k]) - cap;
    if (s.phan[k]) phantoms++;
    else if (viol > -1e-4f * fmaxf(1.f, cap)) atcap++;
    if (viol > worst) { worst = viol; q = k; }
    if (viol > tol && s.code[k] < lowest) { lowest = s.code[k]; qb = k; }
    vmax = fmaxf(vmax, viol);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float ov = __shfl_xor_sync(0xffffffffu, worst, o);
    int oq = __shfl_xor_sync(0xffffffffu, q, o);
    if (ov > worst || (ov == worst && oq >= 0 && (q < 0 || oq < q))) { worst = ov; q = oq; }
    int ol = __shfl_xor_sync(0xffffffffu, lowest, o);
    int oqb = __shfl_xor_sync(0xffffffffu, qb, o);
    if (ol < lowest) { lowest = ol; qb = oqb; }
  }
  vmax = warp_max(vmax);
  phantoms = warp_sum_i(phantoms);
  atcap = warp_sum_i(atcap);
  // Bland's rule (release the violating hyperplane of lowest id) while the
  // polish is not decreasing F: no basis repeats, so no cycling
  if (s.bland) q = qb;
  if (lane == 0) { s.q = q; s.iter = (phantoms > 0 || atcap > 0); s.worst = vmax; }
  __syncwarp();
  if (q >= 0 && step) {
    float sg = s.mu[q] > 0.f ? 1.f : -1.f;
    for (int c = lane; c < p; c += 32) s.dv[c] = c == q ? sg : 0.f;
    __syncwarp();
    lu_solve(s, s.dv);
  }
}

// (thread 0) coordinate breakpoints of the edge line search into sk/sw/sid.
__device__ __noinline__ int edge_specials(St& s, int q) {
  const int p = s.p;
  // coordinate -> basis position (perm is free until the next factorisation)
  int* pos = s.perm;
  for (int c = 0; c < p; ++c) pos[c] = -1;
  for (int k = 0; k < p; ++k)
    if (s.code[k] < 0) pos[-s.code[k] - 1] = k;
  int ns = 0;
  for (int c = 0; c < p; ++c) {
    const int kk = pos[c];
    if (kk >= 0 && kk != q) continue;  // other basis coordinates stay at 0
    float dc = s.dv[c];
    if (kk == q && !s.phan[q]) {
      s.sk[ns] = 0.f; s.sw[ns] = s.lam * fabsf(dc); s.sid[ns] = coord_code(c); ++ns;
    } else if (dc != 0.f) {
      s.sk[ns] = -s.bv[c] / dc; s.sw[ns] = s.lam * fabsf(dc); s.sid[ns] = coord_code(c); ++ns;
    }
  }
  return ns;
}

// ------------------------------------------------------------------ row passes

// r = y - X b, one column at a time, skipping zero coefficients (b is
// sparse along most of the path); loads batched kRowU<G> per thread.
template <int G>
__device__ __noinline__ void recompute_r(St& s) {
  const int n = s.n, p = s.p;
  const int t = gtid<G>();
  const float* __restrict__ yq = s.yq;
  const float* __restrict__ bv = s.bv;
  float* __restrict__ rr = s.rr;
  for (int i0 = 0; i0 < n; i0 += G * kRowU<G>) {
    float v[kRowU<G>];
#pragma unroll
    for (int u = 0; u < kRowU<G>; ++u) {
      const int i = i0 + u * G + t;
      v[u] = i < n ? yq[i] : 0.f;
    }
    for (int c = 0; c < p; ++c) {
      const float b = bv[c];
      if (b == 0.f) continue;  // uniform
      const float* __restrict__ col = colptr(s, c);
#pragma unroll
      for (int u = 0; u < kRowU<G>; ++u) {
        const int i = i0 + u * G + t;
        if (i < n) v[u] -= col[i] * b;
      }
    }
#pragma unroll
    for (int u = 0; u < kRowU<G>; ++u) {
      const int i = i0 + u * G + t;
      if (i < n) rr[i] = v[u];
    }
  }
}

// (all G threads) r = y - X b at the vertex of the current basis, with
// every sign exact.  A float32 residual can put a row whose residual lies
// within float32 rounding of zero on the wrong side, and that row's sign
// then enters the column sums, so the multiplier test can pass at a vertex
// that is not optimal.  Each r_i is formed in float32 together with the
// magnitude S_i = |y_i| + sum_c |x_ic b_c| of its terms; the rounding error
// of that sum, and the error of the float vertex itself, stay below
// 2^-14 S_i for p <= 256.  Only rows inside that band (a few per thousand)
// are formed again in FP64, at the vertex b + e, where e is one correction
// solved with the basis factors from the basis equations' residual formed
// in FP64; a residual within FP64 resolution of zero (2^-40 of the
// magnitude of its terms) is set to 0 (the row lies on its hyperplane).
// FP64 is kept to these few rows: its throughput on this part is a small
// fraction of float32's.  Needs the current basis factored (snap) and s.bv
// its float vertex.
template <int G>
__device__ __noinline__ void exact_residual(St& s) {
  constexpr int W = G / 32;
  const int lane = lane_id(), warp = gwarp<G>(), tid = gtid<G>(), p = s.p, n = s.n;
  gsync<G>();
  for (int e = warp; e < p; e += W) {  // basis equation e: x_cd . b = y_cd, or b_j = const
    const int cd = s.code[e];
    double acc = 0.0;
    if (cd >= 0) {
      for (int c = lane; c < p; c += 32) acc += (double)xval(s, c, cd) * (double)s.bv[c];
      acc = warp_sum_d(acc);
      acc = (double)s.yq[cd] - acc;
    }
    if (lane == 0) s.rv[e] = (float)acc;  // coordinate equations hold exactly (snap)
  }
  gsync<G>();
  if (warp == 0) lu_solve(s, s.rv);
  gsync<G>();
  const float* __restrict__ bv = s.bv;
  const float* __restrict__ ev = s.rv;
  for (int i = tid; i < n; i += G) {
    const float yi = s.yq[i];
    float acc = yi, mag = fabsf(yi);
    for (int c = 0; c < p; ++c) {
      const float t = xval(s, c, i) * bv[c];
      acc -= t;
      mag += fabsf(t);
    }
    if (fabsf(acc) <= 0x1p-14f * mag) {  // sign within float32 rounding
      double a = (double)yi, m = fabs(a);
      for (int c = 0; c < p; ++c) {
        const double t = (double)xval(s, c, i) * ((double)bv[c] + (double)ev[c]);
        a -= t;
        m += fabs(t);
      }
      acc = fabs(a) <= 0x1p-40 * m ? 0.f : (float)a;
    }
    s.rr[i] = acc;
  }
  gsync<G>();
}

// r -= d * column (global or shared), loads batched kRowU<G> per thread.
template <int G>
__device__ __noinline__ void axpy_r(St& s, const float* __restrict__ col, float d) {
  const int n = s.n, t = gtid<G>();
  const uint32_t rr_s = smem_u32(s.rr);
  for (int i0 = 0; i0 < n; i0 += G * kRowU<G>) {
    float xv[kRowU<G>];
#pragma unroll
    for (int u = 0; u < kRowU<G>; ++u) {
      const int i = i0 + u * G + t;
      xv[u] = i < n ? col[i] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kRowU<G>; ++u) {
      const int i = i0 + u * G + t;
      if (i < n) sts_f(rr_s + 4u * i, lds_f(rr_s + 4u * i) - xv[u] * d);
    }
  }
}

// v_i = x_i . d for the edge direction d into `vd` (shared for one warp,
// global scratch for a block), zero on basis rows other than the released
// one (they stay on their hyperplanes along the edge).  Column loads
// batched kRowU<G> per thread.
template <int G>
__device__ __forceinline__ void edge_products(St& s, float* __restrict__ vd) {
  const int n = s.n, p = s.p, lane = gtid<G>(), qc = s.qcode;
  const float* __restrict__ dv = s.dv;
  const unsigned* __restrict__ mask = s.mask;
  for (int i0 = 0; i0 < n; i0 += G * kRowU<G>) {
    float v[kRowU<G>];
#pragma unroll
    for (int u = 0; u < kRowU<G>; ++u) v[u] = 0.f;
    for (int c = 0; c < p; ++c) {
      const float dc = dv[c];
      if (dc == 0.f) continue;  // uniform; d is zero on basis coordinates
      const float* __restrict__ col = colptr(s, c);
#pragma unroll
      for (int u = 0; u < kRowU<G>; ++u) {
        const int i = i0 + u * G + lane;
        if (i < n) v[u] += col[i] * dc;
      }
    }
#pragma unroll
    for (int u = 0; u < kRowU<G>; ++u) {
      const int i = i0 + u * G + lane;
      if (i < n) {
        const bool inb = (mask[i >> 5] >> (i & 31)) & 1u;
        vd[i] = inb && i != qc ? 0.f : v[u];
      }
    }
  }
}

// (all G threads) start copying column j into column buffer `buf` with
// 16-byte asynchronous copies (the gathered column is 16-byte aligned and
// padded to a multiple of 4 floats); wait with cp_async_wait_all.
template <int G>
__device__ __forceinline__ void prefetch_all(St& s, int j, int buf) {
  const float* src = s.Xq + (int64_t)j * s.ld;
  const uint32_t dst = smem_u32(s.cb[buf]);
  for (int q = gtid<G>(); q < (s.ld >> 2); q += G) cp_async16(dst + 16u * q, src + 4 * q);
  cp_async_commit();
}

template <int G>
__device__ __noinline__ float objective(St& s) {
  float a = 0.f;
  for (int i = gtid<G>(); i < s.n; i += G) a += fabsf(s.rr[i]);
  float b = 0.f;
  if (gwarp<G>() == 0)
    for (int c = lane_id(); c < s.p; c += 32) b += fabsf(s.bv[c]);
  float bs;
  float as = gsum2<G>(s, a, b, bs);
  return as + s.lam * bs;
}

// Exact minimisation along axis j (Section 3.3): the weighted median of
// z_i = b_j + r_i / x_ij (weights |x_ij|) and 0 (weight lambda).  Returns
// the move; records the breakpoint landed on in piv[j].
template <int G>
__device__ __noinline__ float axis_update(St& s, int j, int jnext) {
  const float bj = s.bv[j];
  const float* col = colptr(s, j);
  if (kSmemCols<G>) {
    // the column of this step was copied into cb[cur] (each thread's share;
    // the barrier makes all of it visible); start the next column's copy
    // into the other buffer (read by no one since the last step's barrier)
    cp_async_wait_all();
    gsync<G>();
    if (jnext >= 0) prefetch_all<G>(s, jnext, s.cur ^ 1);
    col = s.cb[s.cur];
  } else if (jnext >= 0) {
    // block path: the columns stream from global memory; pull the next
    // one into L2 while this step runs
    const float* nx = colptr(s, jnext);
    for (int o = gtid<G>() * 32; o < s.ld; o += G * 32) prefetch_l2(nx + o);
  }
  gsync<G>();
  if (gtid<G>() == 0) {
    s.colp = col;
    s.bj = bj;
    s.pbase = bj;
    s.pq = -1;
    s.nspec = s.lam > 0.f ? 1 : 0;
    s.sk[0] = -bj; s.sw[0] = s.lam; s.sid[0] = coord_code(j);  // the penalty's breakpoint 0
  }
  gsync<G>();
  {
    // keys relative to b_j: the current value is 0, the window [-dl, dl]
    const float dl = s.dl[j];
    if (G == 32) select_fused(s, 0.f, true, -dl, dl);
    else select_fused_blk<G>(s, 0.f, true, -dl, dl);
  }
  const float z = bj + s.zstar;
  const int own = s.owner;
  const float d = z - bj;
  if (d != 0.f) axpy_r<G>(s, col, d);
  gsync<G>();
  if (gtid<G>() == 0) {
    s.bv[j] = z;
    s.piv[j] = own == kNone ? -2 : (own < 0 ? -1 : own);
    s.dl[j] = fmaxf(kDlf * fabsf(d), 1e-5f * fmaxf(1.f, fabsf(z)));
    if (kSmemCols<G>) s.cur ^= 1;
  }
  gsync<G>();
  return d;
}

// Cyclical coordinate descent (Section 3.3) skipping axis `skip`.
template <int G>
__device__ __noinline__ int ccd(St& s, int skip, int max_sweeps) {
  const float tol = s.a->o.tol_move;
  const int p = s.p;
  const int j0 = skip == 0 ? 1 : 0;  // first axis of a sweep
  if (j0 >= p) return 1;              // nothing to move
  if (kSmemCols<G>) {
    cp_async_wait_all();
    gsync<G>();
    if (gtid<G>() == 0) s.cur = 0;
    gsync<G>();
    prefetch_all<G>(s, j0, 0);
  }
  for (int sw = 1; sw <= max_sweeps; ++sw) {
    float mx = 0.f;
    for (int j = j0; j < p; ++j) {
      if (j == skip) continue;
      int jn = j + 1;
      if (jn == skip) ++jn;
      if (jn >= p) jn = j0;  // first axis of the next sweep
      mx = fmaxf(mx, fabsf(axis_update<G>(s, j, jn)));
    }
    float bmax = 0.f;
    for (int c = lane_id(); c < s.p; c += 32) bmax = fmaxf(bmax, fabsf(s.bv[c]));
    bmax = warp_max(bmax);
    if (mx <= tol * fmaxf(1.f, bmax)) return sw;
  }
  return -max_sweeps;
}

// One chop probe: b_k := t, restricted CCD from the previous probe's point.
template <int G>
__device__ __noinline__ float probe(St& s, int k, float t, float& best_f, int& sweeps,
                                       int& probes) {
  const float d = t - s.bv[k];
  if (d != 0.f) axpy_r<G>(s, colptr(s, k), d);
  gsync<G>();
  if (gtid<G>() == 0) s.bv[k] = t;
  gsync<G>();
  int sw = ccd<G>(s, k, s.a->o.probe_max_sweeps);
  sweeps += sw < 0 ? -sw : sw;
  probes += 1;
  float f = objective<G>(s);
  if (f < best_f) {
    best_f = f;
    for (int c = gtid<G>(); c < s.p; c += G) s.bbest[c] = s.bv[c];
  }
  gsync<G>();
  return f;
}

// Ternary chop on axis k (Sections 3.4-3.5): bracket around b_k, move the
// bracket while an end is lower than the centre (range extension), then
// ternary steps; b ends at the best probe (or the start if none improved).
template <int G>
__device__ __noinline__ void chop(St& s, int k, int& sweeps, int& probes) {
  const Opts& o = s.a->o;
  const float f0 = objective<G>(s);
  float best_f = f0;
  for (int c = gtid<G>(); c < s.p; c += G) s.bbest[c] = s.bv[c];
  gsync<G>();
  const float c0 = s.bv[k];
  const float scale = fmaxf(1.f, fabsf(c0));
  float delta = o.chop_bracket * scale;
  float pa = c0 - delta, pm = c0, pe = c0 + delta, gm = f0;
  float ga = probe<G>(s, k, pa, best_f, sweeps, probes);
  float ge = probe<G>(s, k, pe, best_f, sweeps, probes);
  for (int ext = 0; ext < o.chop_max_extend; ++ext) {
    if (ga < gm) {
      pe = pm; ge = gm; pm = pa; gm = ga; delta *= 2.f; pa = pm - delta;
      ga = probe<G>(s, k, pa, best_f, sweeps, probes);
    } else if (ge < gm) {
      pa = pm; ga = gm; pm = pe; gm = ge; delta *= 2.f; pe = pm + delta;
      ge = probe<G>(s, k, pe, best_f, sweeps, probes);
    } else {
      break;
    }
  }
  float lo = pa, hi = pe;
  int np = 0;
  if (o.chop_sections == 4) {
    // four sections, probes at the inner points; keep the two sections
    // around the lowest probe (leftmost on ties)
    while (hi - lo > o.chop_tol * scale && np + 3 <= o.chop_max_probes) {
      const float h = (hi - lo) / 4.f;
      const float t1 = lo + h, t2 = lo + 2.f * h, t3 = hi - h;
      const float g1 = probe<G>(s, k, t1, best_f, sweeps, probes);
      const float g2 = probe<G>(s, k, t2, best_f, sweeps, probes);
      const float g3 = probe<G>(s, k, t3, best_f, sweeps, probes);
      np += 3;
      if (g1 <= g2 && g1 <= g3) hi = t2;
      else if (g2 <= g3) { lo = t1; hi = t3; }
      else lo = t2;
    }
  } else {
    while (hi - lo > o.chop_tol * scale && np + 2 <= o.chop_max_probes) {
      float m1 = lo + (hi - lo) / 3.f, m2 = hi - (hi - lo) / 3.f;
      float g1 = probe<G>(s, k, m1, best_f, sweeps, probes);
      float g2 = probe<G>(s, k, m2, best_f, sweeps, probes);
      np += 2;
      if (g1 < g2) hi = m2;
      else if (g1 > g2) lo = m1;
      else { lo = m1; hi = m2; }
    }
  }
  for (int c = gtid<G>(); c < s.p; c += G) s.bv[c] = s.bbest[c];
  gsync<G>();
  recompute_r<G>(s);
  gsync<G>();
}

// (all G threads) the polish's column sums
//   g_c = -sum_{rows not in basis} sign(r_i) x_ic
// into red2 (warp 0's slot; the others 0).  `full`: every column over every
// row (compensated float sums per thread, FP64 across warps), remembering
// each row's sign.  Otherwise only rows whose sign or basis membership
// changed since the last sums contribute, g kept in FP64: at p = 128,
// n = 2e4 the full sums are 2.6 M loads per pivot, the changes typically a
// few hundred.  More than kChgW changed rows in some warp falls back to full.
template <int G>
__device__ __noinline__ void colsums(St& s, bool full) {
  constexpr int W = G / 32;
  const int tid = gtid<G>(), lane = lane_id(), warp = gwarp<G>();
  const int n = s.n, p = s.p;
  if (!full) {
    // changed rows, per warp in row order (warp w: row chunks w, w + W, ...)
    int cnt = 0;
    for (int i0 = warp * 32; i0 < n; i0 += G) {
      const int i = i0 + lane;
      int d = 0;
      if (i < n) {
        const bool inb = (s.mask[i >> 5] >> (i & 31)) & 1u;
        const int st = inb ? 0 : (int)fsign(s.rr[i]);
        d = st - (int)s.sgn[i];
        if (d != 0) s.sgn[i] = (signed char)st;
      }
      const unsigned m = __ballot_sync(0xffffffffu, d != 0);
      const int pos = cnt + __popc(m & ((1u << lane) - 1u));
      // delta in [-2, 2] (a sign flip is 2): three bits
      if (d != 0 && pos < kChgW) s.chg[warp * kChgW + pos] = (i << 3) | (d + 2);
      cnt += __popc(m);
    }
    if (lane == 0) s.wcnt[warp] = cnt;
    gsync<G>();
    int over = 0;
    for (int w = 0; w < W; ++w) over |= s.wcnt[w] > kChgW;
    if (!over) {
      // per-warp partial updates, lanes over columns
      constexpr int kPc = kMaxP / 32;
      float part[kPc];
#pragma unroll
      for (int u = 0; u < kPc; ++u) part[u] = 0.f;
      const int m = min(s.wcnt[warp], kChgW);
#pragma unroll 4
      for (int e = 0; e < m; ++e) {
        const int code = s.chg[warp * kChgW + e];
        const int i = code >> 3;
        const float dl = (float)((code & 7) - 2);
#pragma unroll
        for (int u = 0; u < kPc; ++u) {
          const int c = lane + 32 * u;
          if (c < p) part[u] += dl * xval(s, c, i);
        }
      }
#pragma unroll
      for (int u = 0; u < kPc; ++u) {
        const int c = lane + 32 * u;
        if (c < p) s.red2[warp * p + c] = part[u];
      }
      gsync<G>();
      for (int c = tid; c < p; c += G) {
        double g = s.gd[c];
        for (int w = 0; w < W; ++w) g -= (double)s.red2[w * p + c];
        s.gd[c] = g;
      }
      gsync<G>();
      for (int e = tid; e < W * p; e += G) s.red2[e] = e < p ? (float)s.gd[e] : 0.f;
      gsync<G>();
      return;
    }
    // too many changes: the full sums below (signs re-recorded there)
  }
  for (int c = 0; c < p; ++c) {
    const float* __restrict__ col = colptr(s, c);
    float a = 0.f, comp = 0.f;
    for (int i0 = 0; i0 < n; i0 += G * kRowU<G>) {
      float xv[kRowU<G>];
#pragma unroll
      for (int u = 0; u < kRowU<G>; ++u) {
        const int i = i0 + u * G + tid;
        xv[u] = i < n ? col[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < kRowU<G>; ++u) {
        const int i = i0 + u * G + tid;
        if (i < n && !((s.mask[i >> 5] >> (i & 31)) & 1u)) {
          const float t = -fsign(s.rr[i]) * xv[u] - comp;
          const float nb = a + t;
          comp = (nb - a) - t;
          a = nb;
        }
      }
    }
    a = warp_sum(a) - warp_sum(comp);
    if (lane == 0) s.red2[warp * p + c] = a;
  }
  for (int i = tid; i < n; i += G) {
    const bool inb = (s.mask[i >> 5] >> (i & 31)) & 1u;
    s.sgn[i] = (signed char)(inb ? 0 : (int)fsign(s.rr[i]));
  }
  gsync<G>();
  for (int c = tid; c < p; c += G) {
    double g = 0.0;
    for (int w = 0; w < W; ++w) g += (double)s.red2[w * p + c];
    s.gd[c] = g;
  }
  gsync<G>();
  for (int e = tid; e < W * p; e += G) s.red2[e] = e < p ? (float)s.gd[e] : 0.f;
  gsync<G>();
}

__device__ __forceinline__ unsigned mix32(unsigned x) {
  x *= 0x9E3779B1u;
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

// (warp 0) order-independent hash of the basis set; s.flag = 1 when it is
// among the last kHist bases of this polish (then appended).
__device__ __noinline__ void basis_seen(St& s, int nh) {
  const int lane = lane_id();
  unsigned h = 0u;
  for (int k = lane; k < s.p; k += 32) h += mix32((unsigned)s.code[k] * 2u + (unsigned)s.phan[k]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
  bool seen = false;
  for (int e = lane; e < min(nh, kHist); e += 32) seen |= s.bhist[e] == h;
  seen = __any_sync(0xffffffffu, seen);
  __syncwarp();
  if (lane == 0) {
    s.bhist[nh % kHist] = h;
    s.flag = seen;
  }
  __syncwarp();
}

// Exact polish from the current basis (code/phan); max_piv = 0 only tests.
template <int G>
__device__ __noinline__ int polish(St& s, int max_piv, int* is_opt, int* nonunique) {
  const int tid = gtid<G>(), lane = lane_id(), warp = gwarp<G>();
  const int p = s.p;
  int it = 0, nh = 0, cycled = 0;  // nh: bases hashed so far
  // exit: 0 optimal, 1 cycle accepted, 2 cycle rejected, 3 pivot cap,
  // 4 singular basis, 5 flat edge
  int exit_code = 0;
  *is_opt = 0;
  *nonunique = 0;
  if (tid == 0) s.bland = 0;
  if (kSmemCols<G>) { cp_async_wait_all(); gsync<G>(); }
  if (warp == 0) basis_seen(s, 0);  // the starting basis
  gsync<G>();
  nh = 1;
  int fresh = 1;  // r was recomputed from the design at this vertex
  int exact = 0;  // r is the exact-sign residual of this vertex (exact_residual)
  for (;;) {
    if (!exact) {  // the retest (exact) stays at the vertex: factors, b and mask hold
      snap_g<G>(s);
      gsync<G>();
      if (!s.flag) { exit_code = 4; break; }  // singular basis: give up (status MAX_ITERS)
      // r: moved along the edge by the last step (below), recomputed from
      // the design at the first vertex and every kReanchor pivots
      if (it % kReanchor == 0) { recompute_r<G>(s); fresh = 1; }
      for (int w = tid; w < s.maskw; w += G) s.mask[w] = 0u;
      gsync<G>();
      if (tid == 0)
        for (int k = 0; k < p; ++k)
          if (s.code[k] >= 0) s.mask[s.code[k] >> 5] |= 1u << (s.code[k] & 31);
      gsync<G>();
    }
    // column sums g_c = -sum_{rows not in basis} sign(r_i) x_ic: in full at
    // the first pivot, then from the rows that changed (colsums; in the
    // retest, the rows whose exact sign differs from the float32 one)
    colsums<G>(s, it == 0 && !exact);
    gsync<G>();
    if (warp == 0) mult_solve<G>(s);
    if (G == 32) refine(s, s.mu, s.hv, true);
    else refine_blk<G>(s, s.mu, s.hv, true);
    if (warp == 0) mult_pick(s, it < max_piv);
    gsync<G>();
    const int q = s.q;
    if (q < 0 && !exact) {
      // the test passed on float32 residuals: repeat it at this vertex
      // with every residual's sign exact before accepting
      exact_residual<G>(s);
      exact = 1;
      fresh = 1;
      continue;
    }
    if (q < 0) { *is_opt = 1; *nonunique = s.iter; exit_code = 0; break; }
    if (cycled) {
      // a basis repeated under Bland's rule: each iteration is a function
      // of the basis alone, so the polish would loop (float32 noise in the
      // multipliers of a degenerate vertex).  Remaining violations within
      // float32 resolution accept the vertex as a (non-unique) optimum
      if (s.worst <= kStallTolFactor * s.a->o.tol_opt * fmaxf(1.f, s.lam)) {
        *is_opt = 1;
        *nonunique = 1;
        exit_code = 1;
      } else {
        exit_code = 2;
      }
      break;
    }
    if (it >= max_piv) { exit_code = max_piv > 0 ? 3 : 0; break; }
    // edge line search: breakpoints of t -> F(b + t d)
    if (tid == 0) {
      s.qcode = s.code[q];
      s.nspec = edge_specials(s, q);
    }
    gsync<G>();
    {
      float* vd = kSmemCols<G> ? s.cb[0] : s.vdg;
      edge_products<G>(s, vd);
      gsync<G>();
      if (tid == 0) { s.colp = vd; s.pbase = 0.f; s.pq = s.qcode; }
      gsync<G>();
      if (G == 32) select_fused(s, 0.f, false, 0.f, 0.f);
      else select_fused_blk<G>(s, 0.f, false, 0.f, 0.f);
      gsync<G>();
    }
    const float ts = s.zstar;
    const int own = s.owner;
    if (own == kNone) { exit_code = 5; break; }  // flat along the edge (cannot happen when F decreases)
    // residual along the edge: r_i -= t x_i . d (the edge products are in
    // the line search's factor; zero on the basis rows that stay)
    axpy_r<G>(s, s.colp, ts);
    fresh = 0;
    exact = 0;
    if (warp == 0) {
      for (int c = lane; c < p; c += 32) s.bv[c] += ts * s.dv[c];
      __syncwarp();
      if (lane == 0) {
        s.code[q] = own;
        s.phan[q] = 0;
      }
      __syncwarp();
      basis_seen(s, nh);
    }
    gsync<G>();
    // group-uniform: every thread reads the same flag.  A repeated basis
    // switches the release rule to Bland's (lowest id), which does not
    // cycle in exact arithmetic; a repeat under Bland's rule ends the polish
    const int rep_seen = s.flag;
    ++nh;
    if (rep_seen) {
      if (s.bland) cycled = 1;
      nh = 0;  // fresh history for the new rule
    }
    gsync<G>();
    if (tid == 0 && rep_seen) s.bland = 1;
    ++it;
  }
  gsync<G>();
  if (!fresh) recompute_r<G>(s);  // r exact at the vertex the polish ends on
  gsync<G>();
  if (tid == 0) s.pexit = exit_code;
  gsync<G>();
  return it;
}

// Stall test (no pivots): is the descent point's vertex already optimal?
// The test snaps b onto the vertex of the basis built from the hyperplanes
// the axis steps landed on; an optimal vertex is kept, otherwise b and r
// return to the descent point, where the method continues.
template <int G>
__device__ __noinline__ int stall_test(St& s, int* nonu) {
  for (int c = gtid<G>(); c < s.p; c += G) s.bbest[c] = s.bv[c];
  if (kSmemCols<G>) {
    // the residual is kept in the second column buffer (idle until the
    // descent resumes) instead of being recomputed from the design
    cp_async_wait_all();
    gsync<G>();
    for (int i = gtid<G>(); i < s.n; i += G) s.cb[1][i] = s.rr[i];
  }
  if (gwarp<G>() == 0) build_basis(s);
  gsync<G>();
  int is_opt = 0;
  polish<G>(s, 0, &is_opt, nonu);
  if (!is_opt) {
    for (int c = gtid<G>(); c < s.p; c += G) s.bv[c] = s.bbest[c];
    if (kSmemCols<G>) {
      for (int i = gtid<G>(); i < s.n; i += G) s.rr[i] = s.cb[1][i];
    } else {
      gsync<G>();
      recompute_r<G>(s);
    }
    gsync<G>();
  }
  return is_opt;
}

// F at the vertex of the current basis (snap; +inf when singular).
template <int G>
__device__ __noinline__ float vertex_objective(St& s) {
  snap_g<G>(s);
  gsync<G>();
  if (!s.flag) return kInf;
  recompute_r<G>(s);
  gsync<G>();
  return objective<G>(s);
}

template <int G>
__device__ __forceinline__ void copy_basis(St& s, int* cd, int* ph, const int* cs, const int* ps) {
  gsync<G>();
  for (int k = gtid<G>(); k < s.p; k += G) { cd[k] = cs[k]; ph[k] = ps[k]; }
  gsync<G>();
}

// Polish start: the basis built at the descent point, or the previous path
// position's final basis when its vertex has the lower objective at this
// lambda (along a path the optimal basis changes by a few hyperplanes, the
// descent point's basis can be many pivots away).  The descent point
// itself is kept in bbest for the fallback.
template <int G>
__device__ __noinline__ void choose_polish_start(St& s) {
  if (gwarp<G>() == 0) build_basis(s);
  gsync<G>();
  if (!s.has_prev) return;
  for (int c = gtid<G>(); c < s.p; c += G) s.bbest[c] = s.bv[c];
  const float fa = vertex_objective<G>(s);
  copy_basis<G>(s, s.code_alt, s.phan_alt, s.code, s.phan);
  for (int c = gtid<G>(); c < s.p; c += G) s.bv[c] = s.bbest[c];  // phantoms keep descent values
  copy_basis<G>(s, s.code, s.phan, s.code_prev, s.phan_prev);
  const float fb = vertex_objective<G>(s);
  if (!(fb < fa)) copy_basis<G>(s, s.code, s.phan, s.code_alt, s.phan_alt);
  for (int c = gtid<G>(); c < s.p; c += G) s.bv[c] = s.bbest[c];
  gsync<G>();
}

// ------------------------------------------------------------------ one problem

__device__ __forceinline__ void write_fit(const FitArgs& A, int64_t f, int status, float F,
                                          const int (&cnt)[kCounters]) {
  A.obj_out[f] = F;
  if (A.status) A.status[f] = status;
  if (A.counters)
    for (int e = 0; e < kCounters; ++e) A.counters[f * kCounters + e] = cnt[e];
}

template <int G>
__device__ __forceinline__ void write_bad_path(St& s, int q) {
  const FitArgs& A = *s.a;
  const int zero[kCounters] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int l = 0; l < A.L; ++l) {
    int64_t f = (int64_t)q * A.L + l;
    for (int c = gtid<G>(); c < A.P; c += G) {
      A.b_out[f * A.P + c] = 0.f;
      if (A.basis_out) A.basis_out[f * A.P + c] = coord_code(c);
    }
    if (gtid<G>() == 0) write_fit(A, f, kFitBadInput, 0.f, zero);
  }
}

template <int G>
__device__ __forceinline__ void run_problem(St& s, int q, int ncap) {
  const int tid = gtid<G>();
  const FitArgs& A = *s.a;
  int64_t o0 = 0;
  int n = 0, p = 0;
  bool ok = problem_ok(A, q, o0, n, p, ncap);
  int bad = 0;
  float* Xw = nullptr;
  int ld = 0;
  if (ok) {
    ld = (int)xg_ld(n);
    Xw = A.Xg + xg_base(o0, q, A.P4);
    if (G == 32) {
      // short problems: rows of the shared design sit in L2
      for (int64_t e = tid; e < (int64_t)n * p; e += G) {
        int c = (int)(e / n), i = (int)(e % n);
        int64_t row = A.row_idx ? (int64_t)A.row_idx[o0 + i] : o0 + i;
        if (row < 0 || row >= A.rows_X) { bad = 1; continue; }
        float v = A.X[row * A.ldX + c];
        if (!isfinite(v)) bad = 1;
        Xw[(int64_t)c * ld + i] = v;
      }
    } else {
      // long problems: transpose 32 rows at a time through shared memory
      // (the basis-matrix area), reading rows and writing columns coalesced
      float* tile = s.Bm;  // >= 33 * P floats
      for (int i0 = 0; i0 < n; i0 += 32) {
        const int rows = min(32, n - i0);
        for (int e = tid; e < rows * p; e += G) {
          const int i = e / p, c = e - i * p;
          const int64_t row = A.row_idx ? (int64_t)A.row_idx[o0 + i0 + i] : o0 + i0 + i;
          float v = 0.f;
          if (row < 0 || row >= A.rows_X) bad = 1;
          else v = A.X[row * A.ldX + c];
          if (!isfinite(v)) bad = 1;
          tile[c * 33 + i] = v;
        }
        gsync<G>();
        for (int e = tid; e < p * 32; e += G) {
          const int c = e >> 5, i = e & 31;
          if (i < rows) Xw[(int64_t)c * ld + i0 + i] = tile[c * 33 + i];
        }
        gsync<G>();
      }
    }
    for (int i = tid; i < n; i += G) if (!isfinite(A.y[o0 + i])) bad = 1;
  }
  {
    float f[1] = {0.f}, m[1] = {kInf};
    int si[1] = {bad}, mi[1] = {0};
    reduce<G, 1, 1, 1, 1>(s, f, m, si, mi);
    ok = ok && si[0] == 0;
  }
  gsync<G>();
  if (!ok) { write_bad_path<G>(s, q); return; }
  if (tid == 0) {
    s.n = n; s.p = p; s.ld = ld;
    s.Xq = Xw; s.yq = A.y + o0;
    s.vdg = Xw + (int64_t)A.P4 * ld;  // the spare column slot
  }
  gsync<G>();
  for (int c = tid; c < p; c += G) s.bv[c] = A.b_init ? A.b_init[(int64_t)q * A.P + c] : 0.f;
  if (tid == 0) s.has_prev = 0;
  gsync<G>();
  recompute_r<G>(s);
  gsync<G>();
  for (int l = 0; l < A.L; ++l) {
    const int64_t f = (int64_t)q * A.L + l;
    const float lraw = A.lambdas[f];
    if (!(lraw >= 0.f) || !isfinite(lraw)) {
      const int zero[kCounters] = {0, 0, 0, 0, 0, 0, 0, 0};
      for (int c = tid; c < A.P; c += G) {
        A.b_out[f * A.P + c] = 0.f;
        if (A.basis_out) A.basis_out[f * A.P + c] = coord_code(c);
      }
      if (tid == 0) write_fit(A, f, kFitBadInput, 0.f, zero);
      continue;
    }
    if (tid == 0) {
      s.lam = fmaxf(lraw, A.o.lambda_min_floor);
      s.passes = 0; s.selects = 0; s.sel_fail = 0;
    }
    for (int c = tid; c < p; c += G) {
      s.piv[c] = -2;
      // axis windows for the new lambda: moves are a fraction of |b_j|
      s.dl[c] = fmaxf(0.25f * fabsf(s.bv[c]), 1e-5f);
    }
    gsync<G>();
    int status = kFitOk, sweeps = 0, probes = 0, pivots = 0, flags = 0;
    long long t_cd = 0, t_vx = 0, t0 = clock64();  // cycles: descent+chop, vertex work
    int sw = ccd<G>(s, -1, A.o.max_sweeps);
    sweeps += sw < 0 ? -sw : sw;
    if (sw < 0) status |= kFitMaxIters;
    int is_opt = 0, nonu = 0;
    long long t1 = clock64(); t_cd += t1 - t0; t0 = t1;
    is_opt = stall_test<G>(s, &nonu);
    if (is_opt) flags |= 1;
    t1 = clock64(); t_vx += t1 - t0; t0 = t1;
    if (!is_opt && A.o.chop && p >= 2) {
      // Section 3.4: any axis will do; take the largest |b_k|
      int kax = 0;
      for (int c = 1; c < p; ++c) if (fabsf(s.bv[c]) > fabsf(s.bv[kax])) kax = c;
      gsync<G>();
      flags |= 2;
      chop<G>(s, kax, sweeps, probes);
      for (int c = tid; c < p; c += G) s.piv[c] = -2;
      gsync<G>();
      sw = ccd<G>(s, -1, A.o.max_sweeps);
      sweeps += sw < 0 ? -sw : sw;
      t1 = clock64(); t_cd += t1 - t0; t0 = t1;
      is_opt = stall_test<G>(s, &nonu);
      if (is_opt) flags |= 4;
    }
    if (!is_opt && A.o.polish) {
      choose_polish_start<G>(s);
      const int mp = A.o.max_pivots > 0 ? A.o.max_pivots : 4 * p + 64;
      pivots = polish<G>(s, mp, &is_opt, &nonu);
      flags |= s.pexit << 3;
      if (!is_opt) status |= kFitMaxIters;
    }
    if (is_opt) {  // warm start for the next path position's polish
      copy_basis<G>(s, s.code_prev, s.phan_prev, s.code, s.phan);
      if (tid == 0) s.has_prev = 1;
    }
    t1 = clock64(); t_vx += t1 - t0;
    if (is_opt && nonu) status |= kFitNonunique;
    if (s.sel_fail) status |= kFitMaxIters;
    const float F = objective<G>(s);
    for (int c = tid; c < A.P; c += G) {
      A.b_out[f * A.P + c] = c < p ? s.bv[c] : 0.f;
      if (A.basis_out) A.basis_out[f * A.P + c] = c < p ? s.code[c] : coord_code(c);
    }
    if (tid == 0) {
      const int cnt[kCounters] = {sweeps, probes, pivots, flags, s.passes, s.selects,
                                  (int)(t_cd >> 10), (int)(t_vx >> 10)};
      write_fit(A, f, status, F, cnt);
    }
    gsync<G>();
  }
}

// Shared-memory bytes of one group: G threads, row capacity ncap, P columns.
template <int G>
__host__ __device__ size_t group_smem_bytes(int ncap, int P) {
  constexpr int W = G / 32;
  size_t cap = G == 32 ? (size_t)kBufCap : (size_t)W * kSubCap;
  // the basis matrix overlays the selection buffer (never live together:
  // the polish rebuilds it after every edge line search); the block path's
  // gather also stages 32 x P tiles there
  size_t sel_bm = 3 * cap > (size_t)P * P ? 3 * cap : (size_t)P * P;
  if (G > 32 && sel_bm < 33 * (size_t)P) sel_bm = 33 * (size_t)P;
  size_t colbuf = kSmemCols<G> ? 2 * (size_t)ncap : 0;
  size_t words = (size_t)ncap + colbuf + sel_bm + 7 * (size_t)P + (size_t)W * P +
                 9 * (size_t)P + 3 * ((size_t)P + 1) + (size_t)ncap / 32 + 1 +
                 2 * (size_t)W * 16 + 64 + W + kHist;
  words += ((size_t)ncap + 3) / 4 + 2 * (size_t)P + 2 + (size_t)W * kChgW;
  return ((words * 4 + 15) / 16) * 16;
}

template <int G>
__device__ void carve(St& s, unsigned char* raw, int ncap, int P) {
  constexpr int W = G / 32;
  s.cap = G == 32 ? kBufCap : W * kSubCap;
  s.maskw = ncap / 32 + 1;
  s.vdg = nullptr;
  s.pq = -1;
  s.pbase = 0.f;
  float* f = reinterpret_cast<float*>(raw);
  s.rr = f; f += ncap;
  if (kSmemCols<G>) { s.cb[0] = f; f += ncap; s.cb[1] = f; f += ncap; }
  else { s.cb[0] = s.cb[1] = nullptr; }
  float* sel = f;
  s.ck = f; f += s.cap;
  s.cw = f; f += s.cap;
  s.cid = reinterpret_cast<int*>(f); f += s.cap;
  s.Bm = sel;  // overlay (see group_smem_bytes)
  {
    int sel_bm = 3 * s.cap > P * P ? 3 * s.cap : P * P;
    if (G > 32 && sel_bm < 33 * P) sel_bm = 33 * P;
    f = sel + sel_bm;
  }
  s.bv = f; f += P; s.bbest = f; f += P; s.dv = f; f += P;
  s.mu = f; f += P; s.tv = f; f += P; s.hv = f; f += P; s.dl = f; f += P;
  s.rv = s.dv;  // refinement scratch: dv is free whenever a solve is refined
  s.red2 = f; f += W * P;
  int* ip = reinterpret_cast<int*>(f);
  s.code = ip; ip += P; s.phan = ip; ip += P; s.piv = ip; ip += P; s.perm = ip; ip += P;
  s.pcol = ip; ip += P;
  s.code_prev = ip; ip += P; s.phan_prev = ip; ip += P;
  s.code_alt = ip; ip += P; s.phan_alt = ip; ip += P;
  f = reinterpret_cast<float*>(ip);
  s.sk = f; f += P + 1; s.sw = f; f += P + 1;
  s.sid = reinterpret_cast<int*>(f); f += P + 1;
  s.mask = reinterpret_cast<unsigned*>(f); f += s.maskw;
  s.redf = f; f += W * 16;
  s.redi = reinterpret_cast<int*>(f); f += W * 16;
  s.sampk = f; f += 32;
  s.sampw = f; f += 32;
  s.wcnt = reinterpret_cast<int*>(f); f += W;
  s.bhist = reinterpret_cast<unsigned*>(f); f += kHist;
  s.sgn = nullptr; s.gd = nullptr; s.chg = nullptr;
  {
    s.chg = reinterpret_cast<int*>(f); f += W * kChgW;
    if ((reinterpret_cast<uintptr_t>(f) & 7u) != 0) f += 1;  // 8-byte alignment
    s.gd = reinterpret_cast<double*>(f); f += 2 * P;
    s.sgn = reinterpret_cast<signed char*>(f); f += (ncap + 3) / 4;
  }
}

template <int G, int NW>
__global__ void __launch_bounds__(G * NW) fit_block_kernel(FitArgs args, int ncap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ St sarr[NW];  // blockDim.x / G of them are used
  __shared__ FitArgs A;
  const int grp = threadIdx.x / G;
  if (threadIdx.x == 0) A = args;
  __syncthreads();
  if (gtid<G>() == 0) {
    carve<G>(sarr[grp], smem_raw + (size_t)grp * group_smem_bytes<G>(ncap, args.P), ncap, args.P);
    sarr[grp].a = &A;
  }
  __syncthreads();
  St& s = sarr[grp];
  for (;;) {
    if (gtid<G>() == 0) {
      const int t = atomicAdd(A.queue, 1);
      s.q = t < A.B ? A.order[t] : A.B;  // longest problems first
    }
    gsync<G>();
    const int q = s.q;
    gsync<G>();
    if (q >= A.B) break;
    run_problem<G>(s, q, ncap);
    // no copy may outlive the problem (or the block)
    if (kSmemCols<G>) cp_async_wait_all();
    gsync<G>();
  }
}

// nw groups per block (nw <= NW).
template <int G, int NW>
cudaError_t launch_variant(const FitArgs& a, cudaStream_t st, int num_sms, int ncap, int nw) {
  size_t smem = group_smem_bytes<G>(ncap, a.P) * nw;
  auto kern = fit_block_kernel<G, NW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G * nw, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int64_t grid = (int64_t)per_sm * num_sms;
  int64_t need = ((int64_t)a.B + nw - 1) / nw;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(int)grid, G * nw, smem, st>>>(a, ncap);
  return cudaGetLastError();
}

}  // namespace

// Largest row capacity one group of G threads can hold with P columns in
// the shared memory one block may use (227 KB).
int fit_block_max_rows(int G, int P) {
  const size_t limit = kDynSmemLimit;
  int lo = 0, hi = 1 << 16;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    size_t b = G == 32    ? group_smem_bytes<32>(mid, P)
               : G == 64  ? group_smem_bytes<64>(mid, P)
               : G == 128 ? group_smem_bytes<128>(mid, P)
                          : group_smem_bytes<kBlockG>(mid, P);
    if (b <= limit) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Default group size for a problem set: one warp per fit while its rows fit
// a warp's share of shared memory, else a block per fit.
int fit_block_group(int n_max) { return n_max <= 8192 ? 32 : kBlockG; }

// Group size a call asks for (dims->group_threads), 0 when invalid.  The
// automatic choice (0) also takes the block shape when a warp's share of
// shared memory cannot hold n_max rows of these columns but a block's can
// (wide problems: from about 160 columns a warp holds fewer than 8192 rows).
int launch_group(const ladlasso_dims* d) {
  if (d->group_threads == 0) {
    int G = fit_block_group(d->n_max);
    if (G == 32 && d->P_cols >= 1 && d->P_cols <= kMaxP &&
        d->n_max > fit_block_max_rows(32, d->P_cols) &&
        d->n_max <= fit_block_max_rows(kBlockG, d->P_cols))
      G = kBlockG;
    return G;
  }
  const int g = d->group_threads;
  return g == 32 || g == 64 || g == 128 || g == kBlockG ? g : 0;
}

static int row_cap(int n_max) {
  int ncap = (n_max + 31) & ~31;
  return ncap < 32 ? 32 : ncap;
}

// Fits per thread block for group size G: one-warp groups, as many as
// shared memory allows (at most 16, at most `fits_per_block` when > 0);
// one block per fit otherwise.
int fit_block_fits_per_block(int G, int P, int n_max, int fits_per_block) {
  if (G == kBlockG) return 1;
  const int ncap = row_cap(n_max);
  const size_t per = G == 32 ? group_smem_bytes<32>(ncap, P)
                     : G == 64 ? group_smem_bytes<64>(ncap, P)
                               : group_smem_bytes<128>(ncap, P);
  int nw = (int)(kDynSmemLimit / (per ? per : 1));
  if (nw > 512 / G) nw = 512 / G;  // at most 512 threads a block
  if (fits_per_block > 0 && nw > fits_per_block) nw = fits_per_block;
  return nw < 1 ? 1 : nw;
}

cudaError_t launch_fit_block(const FitArgs& a, cudaStream_t st, int num_sms, int G,
                             int fits_per_block) {
  const int ncap = row_cap(a.n_max);
  int nw = G == kBlockG ? 1 : fit_block_fits_per_block(G, a.P, a.n_max, fits_per_block);
  if (fits_per_block == 0 && G != kBlockG) {
    // automatic: a problem set with fewer problems than the SMs can hold
    // spreads over every SM instead of filling a few blocks
    const int spread = (int)(((int64_t)a.B + num_sms - 1) / num_sms);
    if (spread < nw) nw = spread < 1 ? 1 : spread;
  }
  switch (G) {
    case 32:
      return launch_variant<32, 16>(a, st, num_sms, ncap, nw);
    case 64:
      return launch_variant<64, 8>(a, st, num_sms, ncap, nw);
    case 128:
      return launch_variant<128, 4>(a, st, num_sms, ncap, nw);
    case kBlockG: return launch_variant<kBlockG, 1>(a, st, num_sms, ncap, 1);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace ll
