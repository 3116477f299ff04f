// Thread-per-fit kernel: the layout the paper proposes for a browser GPU
// (one fit per GPU thread, Sections 1 and 5), written in CUDA as the plain
// comparison for the block-per-fit kernel.  Same method and options:
// CCD with exact weighted-median axis steps (Section 3.3), ternary chop with
// restricted sub-searches and range extension (Sections 3.4-3.5), exact
// vertex polish.  Each thread keeps its residual, selection buffer and basis
// matrix in its own slice of the global workspace, and first copies its
// design rows into its own column-major slice of the workspace.
#include "common.cuh"

namespace ll {
namespace {

constexpr float kInf = INFINITY;
constexpr int kHist = 32;               // polish: bases remembered for cycle detection
constexpr float kStallTolFactor = 50.f; // cycling vertex accepted when violations are below this x tol

__device__ __forceinline__ unsigned mix32(unsigned x) {
  x *= 0x9E3779B1u;
  x ^= x >> 16;
  x *= 0x85EBCA6Bu;
  x ^= x >> 13;
  x *= 0xC2B2AE35u;
  x ^= x >> 16;
  return x;
}

struct TFit {
  // problem
  const FitArgs* a;
  int q, n, p, ld;
  int64_t off0;
  float lam;
  const float* Xq;   // gathered design, column c at Xq + c*ld
  // scratch (global)
  float* zk;   // [n + P + 1] keys
  float* zw;   // weights
  int* zi;     // owner ids
  float* r;    // [n] residual
  float* Bm;   // [P * P]
  float* bv; float* bbest; float* dv; float* mu; float* hv; float* tv;  // [P]
  int* code; int* phan; int* piv; int* perm; int* pcol;  // [P]
  int* code_prev; int* phan_prev; int* code_alt; int* phan_alt;  // [P]
  int has_prev;

  __device__ __forceinline__ float x(int i, int c) const { return Xq[(int64_t)c * ld + i]; }
  __device__ float yv(int i) const { return a->y[off0 + i]; }

  // Weighted median of zk/zw/zi[0..m): smallest key whose cumulative weight
  // reaches half the total; exact halves keep `cur` inside the flat segment.
  // In-place three-way quickselect.
  __device__ float wmedian(int m, float cur, int* owner) {
    *owner = kNone;
    float W = 0.f;
    for (int e = 0; e < m; ++e) W += zw[e];
    if (!(W > 0.f) || m == 0) return cur;
    float half = 0.5f * W, acc = 0.f, above = kInf;
    int lo = 0, hi = m - 1;
    for (;;) {
      // pivot: median of three keys
      int mid = lo + (hi - lo) / 2;
      float a0 = zk[lo], a1 = zk[mid], a2 = zk[hi];
      float pv = fmaxf(fminf(a0, a1), fminf(fmaxf(a0, a1), a2));
      // three-way partition [lo, lt) < pv, [lt, gt] == pv, (gt, hi] > pv
      int lt = lo, i = lo, gt = hi;
      float wl = 0.f, we = 0.f;
      while (i <= gt) {
        float k = zk[i];
        if (k < pv) {
          float tk = zk[lt], tw = zw[lt]; int ti = zi[lt];
          zk[lt] = k; zw[lt] = zw[i]; zi[lt] = zi[i];
          zk[i] = tk; zw[i] = tw; zi[i] = ti;
          wl += zw[lt];
          ++lt; ++i;
        } else if (k > pv) {
          float tk = zk[gt], tw = zw[gt]; int ti = zi[gt];
          zk[gt] = k; zw[gt] = zw[i]; zi[gt] = zi[i];
          zk[i] = tk; zw[i] = tw; zi[i] = ti;
          --gt;
        } else {
          we += zw[i];
          ++i;
        }
      }
      if (half <= acc + wl && lt > lo) {
        hi = lt - 1;
        above = pv;
        continue;
      }
      if (half <= acc + wl + we || gt >= hi) {
        // crossing at the pivot group (or rounding left nothing above)
        float cum = acc + wl + we;
        float next = above;
        for (int e = gt + 1; e <= hi; ++e) next = fminf(next, zk[e]);
        int own = INT32_MAX;
        for (int e = lt; e <= gt; ++e) if (zw[e] > 0.f) own = min(own, zi[e]);
        float z = pv;
        if (cum == half && next < kInf) {
          if (cur > z && cur < next) return cur;
          if (cur >= next) {
            own = INT32_MAX;
            for (int e = gt + 1; e <= hi; ++e) if (zk[e] == next && zw[e] > 0.f) own = min(own, zi[e]);
            *owner = own == INT32_MAX ? kNone : own;
            return next;
          }
        }
        *owner = own == INT32_MAX ? kNone : own;
        return z;
      }
      acc += wl + we;
      lo = gt + 1;
    }
  }

  __device__ float objective() {
    float s = 0.f;
    for (int i = 0; i < n; ++i) s += fabsf(r[i]);
    float t = 0.f;
    for (int c = 0; c < p; ++c) t += fabsf(bv[c]);
    return s + lam * t;
  }

  __device__ void recompute_r() {
    for (int i = 0; i < n; ++i) {
      float s = yv(i);
      for (int c = 0; c < p; ++c) s -= x(i, c) * bv[c];
      r[i] = s;
    }
  }

  __device__ float axis_update(int j) {
    float bj = bv[j];
    int m = 0;
    const float* __restrict__ col = Xq + (int64_t)j * ld;
    const float* __restrict__ rr = r;
    float* __restrict__ k_ = zk;
    float* __restrict__ w_ = zw;
    int* __restrict__ i_ = zi;
    for (int i = 0; i < n; ++i) {
      float xv = col[i];
      if (xv != 0.f) { k_[m] = bj + __fdiv_rn(rr[i], xv); w_[m] = fabsf(xv); i_[m] = i; ++m; }
    }
    if (lam > 0.f) { zk[m] = 0.f; zw[m] = lam; zi[m] = coord_code(j); ++m; }
    int own;
    float z = wmedian(m, bj, &own);
    float d = z - bj;
    if (d != 0.f) {
      float* __restrict__ rw = r;
      for (int i = 0; i < n; ++i) rw[i] -= col[i] * d;
      bv[j] = z;
    }
    piv[j] = own == kNone ? -2 : (own < 0 ? -1 : own);
    return d;
  }

  __device__ int ccd(int skip, int max_sweeps) {
    for (int s = 1; s <= max_sweeps; ++s) {
      float mx = 0.f, bmax = 0.f;
      for (int j = 0; j < p; ++j) {
        if (j == skip) continue;
        mx = fmaxf(mx, fabsf(axis_update(j)));
      }
      for (int c = 0; c < p; ++c) bmax = fmaxf(bmax, fabsf(bv[c]));
      if (mx <= a->o.tol_move * fmaxf(1.f, bmax)) return s;
    }
    return -max_sweeps;
  }

  __device__ float probe(int k, float t, float& best_f, int& sweeps, int& probes) {
    float d = t - bv[k];
    if (d != 0.f) {
      for (int i = 0; i < n; ++i) r[i] -= x(i, k) * d;
      bv[k] = t;
    }
    int s = ccd(k, a->o.probe_max_sweeps);
    sweeps += s < 0 ? -s : s;
    probes += 1;
    float f = objective();
    if (f < best_f) {
      best_f = f;
      for (int c = 0; c < p; ++c) bbest[c] = bv[c];
    }
    return f;
  }

  __device__ void chop(int k, int& sweeps, int& probes) {
    const Opts& o = a->o;
    float f0 = objective(), best_f = f0;
    for (int c = 0; c < p; ++c) bbest[c] = bv[c];
    float c0 = bv[k], scale = fmaxf(1.f, fabsf(c0)), delta = o.chop_bracket * scale;
    float pa = c0 - delta, pm = c0, pe = c0 + delta, gm = f0;
    float ga = probe(k, pa, best_f, sweeps, probes);
    float ge = probe(k, pe, best_f, sweeps, probes);
    for (int ext = 0; ext < o.chop_max_extend; ++ext) {
      if (ga < gm) {
        pe = pm; ge = gm; pm = pa; gm = ga; delta *= 2.f; pa = pm - delta;
        ga = probe(k, pa, best_f, sweeps, probes);
      } else if (ge < gm) {
        pa = pm; ga = gm; pm = pe; gm = ge; delta *= 2.f; pe = pm + delta;
        ge = probe(k, pe, best_f, sweeps, probes);
      } else {
        break;
      }
    }
    float lo = pa, hi = pe;
    int np = 0;
    if (o.chop_sections == 4) {
      while (hi - lo > o.chop_tol * scale && np + 3 <= o.chop_max_probes) {
        const float h = (hi - lo) / 4.f;
        const float t1 = lo + h, t2 = lo + 2.f * h, t3 = hi - h;
        const float g1 = probe(k, t1, best_f, sweeps, probes);
        const float g2 = probe(k, t2, best_f, sweeps, probes);
        const float g3 = probe(k, t3, best_f, sweeps, probes);
        np += 3;
        if (g1 <= g2 && g1 <= g3) hi = t2;
        else if (g2 <= g3) { lo = t1; hi = t3; }
        else lo = t2;
      }
    } else {
      while (hi - lo > o.chop_tol * scale && np + 2 <= o.chop_max_probes) {
        float m1 = lo + (hi - lo) / 3.f, m2 = hi - (hi - lo) / 3.f;
        float g1 = probe(k, m1, best_f, sweeps, probes);
        float g2 = probe(k, m2, best_f, sweeps, probes);
        np += 2;
        if (g1 < g2) hi = m2;
        else if (g1 > g2) lo = m1;
        else { lo = m1; hi = m2; }
      }
    }
    for (int c = 0; c < p; ++c) bv[c] = bbest[c];
    recompute_r();
  }

  __device__ void normal_to(int cd, float* v) {
    for (int c = 0; c < p; ++c) v[c] = cd >= 0 ? x(cd, c) : (c == -cd - 1 ? 1.f : 0.f);
  }

  __device__ bool try_add(int cd, int& m) {
    float* v = tv;
    normal_to(cd, v);
    float vmax0 = 0.f;
    for (int c = 0; c < p; ++c) vmax0 = fmaxf(vmax0, fabsf(v[c]));
    if (!(vmax0 > 0.f)) return false;
    for (int qq = 0; qq < m; ++qq) {
      const float* e = Bm + qq * p;
      float f = v[pcol[qq]] / e[pcol[qq]];
      if (f != 0.f) for (int c = 0; c < p; ++c) v[c] -= f * e[c];
    }
    float bvv = 0.f;
    int bj = p;
    for (int c = 0; c < p; ++c) if (fabsf(v[c]) > bvv) { bvv = fabsf(v[c]); bj = c; }
    if (!(bvv > 1e-4f * vmax0)) return false;
    for (int c = 0; c < p; ++c) Bm[m * p + c] = v[c];
    pcol[m] = bj;
    ++m;
    return true;
  }

  __device__ void build_basis() {
    int m = 0;
    for (int j = 0; j < p && m < p; ++j) {
      int pvv = piv[j];
      if (pvv == -2) continue;
      int cd = pvv >= 0 ? pvv : coord_code(j);
      bool dup = false;
      for (int qq = 0; qq < m; ++qq) dup |= code[qq] == cd;
      if (dup) continue;
      if (try_add(cd, m)) { code[m - 1] = cd; phan[m - 1] = 0; }
    }
    for (int j = 0; j < p && m < p; ++j) {
      int cd = coord_code(j);
      bool dup = false;
      for (int qq = 0; qq < m; ++qq) dup |= code[qq] == cd;
      if (dup) continue;
      if (try_add(cd, m)) { code[m - 1] = cd; phan[m - 1] = bv[j] != 0.f; }
    }
    for (int j = 0; m < p && j < p; ++j) { code[m] = coord_code(j); phan[m] = bv[j] != 0.f; ++m; }
  }

  __device__ bool lu() {
    for (int c = 0; c < p; ++c) perm[c] = c;
    float amax = 0.f;
    for (int e = 0; e < p * p; ++e) amax = fmaxf(amax, fabsf(Bm[e]));
    for (int k = 0; k < p; ++k) {
      int bi = k;
      float bvv = fabsf(Bm[k * p + k]);
      for (int i = k + 1; i < p; ++i) if (fabsf(Bm[i * p + k]) > bvv) { bvv = fabsf(Bm[i * p + k]); bi = i; }
      if (!(bvv > 1e-7f * amax)) return false;
      if (bi != k) {
        for (int c = 0; c < p; ++c) { float t = Bm[k * p + c]; Bm[k * p + c] = Bm[bi * p + c]; Bm[bi * p + c] = t; }
        int t = perm[k]; perm[k] = perm[bi]; perm[bi] = t;
      }
      float pv = Bm[k * p + k];
      for (int i = k + 1; i < p; ++i) {
        float l = Bm[i * p + k] / pv;
        Bm[i * p + k] = l;
        for (int c = k + 1; c < p; ++c) Bm[i * p + c] -= l * Bm[k * p + c];
      }
    }
    return true;
  }

  __device__ void lu_solve(float* xv) {
    for (int c = 0; c < p; ++c) tv[c] = xv[perm[c]];
    for (int k = 0; k < p; ++k) for (int i = k + 1; i < p; ++i) tv[i] -= Bm[i * p + k] * tv[k];
    for (int k = p - 1; k >= 0; --k) {
      tv[k] /= Bm[k * p + k];
      for (int i = 0; i < k; ++i) tv[i] -= Bm[i * p + k] * tv[k];
    }
    for (int c = 0; c < p; ++c) xv[c] = tv[c];
  }

  __device__ void lu_solve_t(float* xv) {
    for (int c = 0; c < p; ++c) tv[c] = xv[c];
    for (int k = 0; k < p; ++k) {
      tv[k] /= Bm[k * p + k];
      for (int i = k + 1; i < p; ++i) tv[i] -= Bm[k * p + i] * tv[k];
    }
    for (int k = p - 1; k >= 0; --k) for (int i = 0; i < k; ++i) tv[i] -= Bm[k * p + i] * tv[k];
    for (int c = 0; c < p; ++c) xv[perm[c]] = tv[c];
  }

  // One step of iterative refinement of x solving B x = h (trans false) or
  // B^T x = h (trans true): residual in FP64 from the basis normals (exact
  // in FP32), correction from the FP32 factors; `rs` is scratch [p].
  __device__ void refine(float* xv, const float* h, float* rs, bool trans) {
    for (int e = 0; e < p; ++e) {
      double acc = 0.0;
      if (!trans) {
        const int cd = code[e];
        if (cd >= 0) for (int c = 0; c < p; ++c) acc += (double)x(cd, c) * (double)xv[c];
        else acc = (double)xv[-cd - 1];
      } else {
        for (int k = 0; k < p; ++k) {
          const int cd = code[k];
          const float nv = cd >= 0 ? x(cd, e) : (e == -cd - 1 ? 1.f : 0.f);
          acc += (double)nv * (double)xv[k];
        }
      }
      rs[e] = (float)((double)h[e] - acc);
    }
    if (trans) lu_solve_t(rs); else lu_solve(rs);
    for (int e = 0; e < p; ++e) xv[e] += rs[e];
  }

  __device__ bool in_basis_row(int i) const {
    for (int k = 0; k < p; ++k) if (code[k] == i) return true;
    return false;
  }

  // r = y - X b at the vertex of the current basis with every sign exact
  // (a float32 residual within rounding of zero can take the wrong side,
  // and its sign enters the multipliers): each r_i in float32 with the
  // magnitude S_i = |y_i| + sum_c |x_ic b_c| of its terms, whose rounding
  // error stays below 2^-14 S_i for p <= 256; rows inside that band again
  // in FP64 at b + e (e: one correction solved from the basis equations'
  // FP64 residual), 0 within FP64 resolution (2^-40 of the magnitude of
  // its terms).  Needs the current basis factored; dv is scratch.
  __device__ void exact_residual() {
    for (int e = 0; e < p; ++e) {
      const int cd = code[e];
      double acc = 0.0;
      if (cd >= 0) {  // coordinate equations hold exactly (snap)
        for (int c = 0; c < p; ++c) acc += (double)x(cd, c) * (double)bv[c];
        acc = (double)yv(cd) - acc;
      }
      dv[e] = (float)acc;
    }
    lu_solve(dv);
    for (int i = 0; i < n; ++i) {
      float acc = yv(i), mag = fabsf(acc);
      for (int c = 0; c < p; ++c) {
        const float t = x(i, c) * bv[c];
        acc -= t;
        mag += fabsf(t);
      }
      if (fabsf(acc) <= 0x1p-14f * mag) {
        double a = (double)yv(i), m = fabs(a);
        for (int c = 0; c < p; ++c) {
          const double t = (double)x(i, c) * ((double)bv[c] + (double)dv[c]);
          a -= t;
          m += fabs(t);
        }
        acc = fabs(a) <= 0x1p-40 * m ? 0.f : (float)a;
      }
      r[i] = acc;
    }
  }

  // b := the vertex of the current basis (phantom coordinates keep their
  // value), r recomputed.  False when the basis matrix is singular.
  __device__ bool snap() {
    for (int k = 0; k < p; ++k) {
      normal_to(code[k], Bm + k * p);
      int cd = code[k];
      hv[k] = cd >= 0 ? yv(cd) : (phan[k] ? bv[-cd - 1] : 0.f);
    }
    for (int k = 0; k < p; ++k) mu[k] = hv[k];  // right-hand side (mu is free here)
    if (!lu()) return false;
    lu_solve(hv);
    refine(hv, mu, dv, false);
    for (int c = 0; c < p; ++c) bv[c] = hv[c];
    for (int k = 0; k < p; ++k) if (code[k] < 0 && !phan[k]) bv[-code[k] - 1] = 0.f;
    recompute_r();
    return true;
  }

  // Polish start: the descent point's basis, or the previous path
  // position's final basis when its vertex has the lower objective here.
  __device__ void choose_polish_start() {
    build_basis();
    if (!has_prev) return;
    for (int c = 0; c < p; ++c) bbest[c] = bv[c];
    const float fa = snap() ? objective() : kInf;
    for (int k = 0; k < p; ++k) { code_alt[k] = code[k]; phan_alt[k] = phan[k]; }
    for (int c = 0; c < p; ++c) bv[c] = bbest[c];
    for (int k = 0; k < p; ++k) { code[k] = code_prev[k]; phan[k] = phan_prev[k]; }
    const float fb = snap() ? objective() : kInf;
    if (!(fb < fa))
      for (int k = 0; k < p; ++k) { code[k] = code_alt[k]; phan[k] = phan_alt[k]; }
    for (int c = 0; c < p; ++c) bv[c] = bbest[c];
    recompute_r();
  }

  // Stall test (no pivots): the vertex of the descent point's basis is kept
  // when optimal; otherwise b and r return to the descent point.
  __device__ int stall_test(int& nonu) {
    for (int c = 0; c < p; ++c) bbest[c] = bv[c];
    build_basis();
    int is_opt = 0;
    polish(0, is_opt, nonu);
    if (!is_opt) {
      for (int c = 0; c < p; ++c) bv[c] = bbest[c];
      recompute_r();
    }
    return is_opt;
  }

  // order-independent hash of the basis set
  __device__ unsigned basis_hash() const {
    unsigned h = 0u;
    for (int k = 0; k < p; ++k) h += mix32((unsigned)code[k] * 2u + (unsigned)phan[k]);
    return h;
  }

  __device__ int polish(int max_piv, int& is_opt, int& nonunique) {
    const float tol = a->o.tol_opt * fmaxf(1.f, lam);
    // recent bases: a repeat switches to Bland's rule, a repeat under it
    // ends the polish (each iteration is a function of the basis alone)
    unsigned hist[kHist];
    int it = 0, nh = 1, bland = 0, cycled = 0;
    hist[0] = basis_hash();
    is_opt = 0;
    nonunique = 0;
    for (;;) {
      if (!snap()) break;
      int qq, qb, phantoms, atcap;
      float vmax;
      for (int exact = 0;; exact = 1) {
        // mu = -g, row part with compensated sums
        for (int c = 0; c < p; ++c) { mu[c] = 0.f; tv[c] = 0.f; }
        for (int i = 0; i < n; ++i) {
          if (in_basis_row(i)) continue;
          float sg = fsign(r[i]);
          if (sg != 0.f)
            for (int c = 0; c < p; ++c) {
              const float t = sg * x(i, c) - tv[c];
              const float nb = mu[c] + t;
              tv[c] = (nb - mu[c]) - t;
              mu[c] = nb;
            }
        }
        for (int c = 0; c < p; ++c) {
          bool real = false;
          for (int k = 0; k < p; ++k) real |= (code[k] == coord_code(c) && !phan[k]);
          if (!real) mu[c] -= lam * fsign(bv[c]);
          hv[c] = mu[c];  // right-hand side (hv is free after the snap)
        }
        lu_solve_t(mu);
        refine(mu, hv, dv, true);
        qq = -1; qb = -1; phantoms = 0; atcap = 0;
        int lowest = INT32_MAX;
        float worst = tol;
        vmax = 0.f;
        for (int k = 0; k < p; ++k) {
          float cap = code[k] >= 0 ? 1.f : (phan[k] ? 0.f : lam);
          float viol = fabsf(mu[k]) - cap;
          if (phan[k]) phantoms++;
          else if (viol > -1e-4f * fmaxf(1.f, cap)) atcap++;
          if (viol > worst) { worst = viol; qq = k; }
          if (viol > tol && code[k] < lowest) { lowest = code[k]; qb = k; }
          vmax = fmaxf(vmax, viol);
        }
        if (bland) qq = qb;  // Bland's rule: lowest id
        if (qq >= 0 || exact) break;
        // the test passed on float32 residuals: repeat it at this vertex
        // with every residual's sign exact before accepting
        exact_residual();
      }
      if (qq < 0) { is_opt = 1; nonunique = phantoms > 0 || atcap > 0; break; }
      if (cycled) {
        if (vmax <= kStallTolFactor * tol) { is_opt = 1; nonunique = 1; }
        break;
      }
      if (it >= max_piv) break;
      float sg = mu[qq] > 0.f ? 1.f : -1.f;
      for (int c = 0; c < p; ++c) dv[c] = c == qq ? sg : 0.f;
      lu_solve(dv);
      int qcode = code[qq];
      int m = 0;
      for (int i = 0; i < n; ++i) {
        bool inb = in_basis_row(i);
        if (inb && i != qcode) continue;
        float v = 0.f;
        for (int c = 0; c < p; ++c) v += x(i, c) * dv[c];
        if (i == qcode) { zk[m] = 0.f; zw[m] = fabsf(v); zi[m] = i; ++m; }
        else if (v != 0.f) { zk[m] = __fdiv_rn(r[i], v); zw[m] = fabsf(v); zi[m] = i; ++m; }
      }
      for (int c = 0; c < p; ++c) {
        int kk = -1;
        for (int k = 0; k < p; ++k) if (code[k] == coord_code(c)) kk = k;
        if (kk >= 0 && kk != qq) continue;
        float dc = dv[c];
        if (kk == qq && !phan[qq]) { zk[m] = 0.f; zw[m] = lam * fabsf(dc); zi[m] = coord_code(c); ++m; }
        else if (dc != 0.f) { zk[m] = -bv[c] / dc; zw[m] = lam * fabsf(dc); zi[m] = coord_code(c); ++m; }
      }
      int own;
      float ts = wmedian(m, 0.f, &own);
      if (own == kNone) break;
      for (int c = 0; c < p; ++c) bv[c] += ts * dv[c];
      code[qq] = own;
      phan[qq] = 0;
      const unsigned h = basis_hash();
      bool seen = false;
      for (int e = 0; e < min(nh, kHist); ++e) seen |= hist[e] == h;
      hist[nh % kHist] = h;
      ++nh;
      if (seen) {
        if (bland) cycled = 1;
        bland = 1;
        nh = 0;
      }
      ++it;
    }
    return it;
  }

  __device__ void write_bad() {
    const FitArgs& A = *a;
    for (int l = 0; l < A.L; ++l) {
      int64_t f = (int64_t)q * A.L + l;
      for (int c = 0; c < A.P; ++c) {
        A.b_out[f * A.P + c] = 0.f;
        if (A.basis_out) A.basis_out[f * A.P + c] = coord_code(c);
      }
      A.obj_out[f] = 0.f;
      if (A.status) A.status[f] = kFitBadInput;
      if (A.counters) for (int e = 0; e < kCounters; ++e) A.counters[f * kCounters + e] = 0;
    }
  }

  __device__ void run() {
    const FitArgs& A = *a;
    for (int c = 0; c < p; ++c) bv[c] = A.b_init ? A.b_init[(int64_t)q * A.P + c] : 0.f;
    has_prev = 0;
    recompute_r();
    for (int l = 0; l < A.L; ++l) {
      int64_t f = (int64_t)q * A.L + l;
      float lraw = A.lambdas[f];
      if (!(lraw >= 0.f) || !isfinite(lraw)) {
        for (int c = 0; c < A.P; ++c) {
          A.b_out[f * A.P + c] = 0.f;
          if (A.basis_out) A.basis_out[f * A.P + c] = coord_code(c);
        }
        A.obj_out[f] = 0.f;
        if (A.status) A.status[f] = kFitBadInput;
        if (A.counters) for (int e = 0; e < kCounters; ++e) A.counters[f * kCounters + e] = 0;
        continue;
      }
      lam = fmaxf(lraw, A.o.lambda_min_floor);
      int status = kFitOk, sweeps = 0, probes = 0, pivots = 0, flags = 0;
      for (int c = 0; c < p; ++c) piv[c] = -2;
      int s = ccd(-1, A.o.max_sweeps);
      sweeps += s < 0 ? -s : s;
      if (s < 0) status |= kFitMaxIters;
      int is_opt = 0, nonu = 0;
      is_opt = stall_test(nonu);
      if (is_opt) flags |= 1;
      if (!is_opt && A.o.chop && p >= 2) {
        int kk = 0;
        for (int c = 1; c < p; ++c) if (fabsf(bv[c]) > fabsf(bv[kk])) kk = c;
        flags |= 2;
        chop(kk, sweeps, probes);
        for (int c = 0; c < p; ++c) piv[c] = -2;
        s = ccd(-1, A.o.max_sweeps);
        sweeps += s < 0 ? -s : s;
        is_opt = stall_test(nonu);
        if (is_opt) flags |= 4;
      }
      if (!is_opt && A.o.polish) {
        choose_polish_start();
        int mp = A.o.max_pivots > 0 ? A.o.max_pivots : 4 * p + 64;
        pivots = polish(mp, is_opt, nonu);
        if (!is_opt) status |= kFitMaxIters;
      }
      if (is_opt) {
        for (int k = 0; k < p; ++k) { code_prev[k] = code[k]; phan_prev[k] = phan[k]; }
        has_prev = 1;
      }
      if (is_opt && nonu) status |= kFitNonunique;
      float F = objective();
      for (int c = 0; c < A.P; ++c) {
        A.b_out[f * A.P + c] = c < p ? bv[c] : 0.f;
        if (A.basis_out) A.basis_out[f * A.P + c] = c < p ? code[c] : coord_code(c);
      }
      A.obj_out[f] = F;
      if (A.status) A.status[f] = status;
      if (A.counters) {
        A.counters[f * kCounters + 0] = sweeps;
        A.counters[f * kCounters + 1] = probes;
        A.counters[f * kCounters + 2] = pivots;
        A.counters[f * kCounters + 3] = flags;
        for (int e = 4; e < kCounters; ++e) A.counters[f * kCounters + e] = 0;
      }
    }
  }
};

__global__ void __launch_bounds__(128) fit_thread_kernel(FitArgs args) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= args.B) return;
  TFit t;
  t.a = &args;
  t.q = q;
  int64_t o0 = 0, nn = 0;
  int P = args.P;
  bool ok = args.queue[1] == 0 && problem_rows(args, q, o0, nn) && nn <= (int64_t)args.n_max;
  int p = args.p ? args.p[q] : P;
  ok = ok && p >= 1 && p <= P;
  t.off0 = o0;
  t.n = ok ? (int)nn : 0;
  t.p = p;
  if (ok) {
    // validate and gather this problem's rows column-major into its own
    // slice of the workspace
    t.ld = (int)xg_ld(t.n);
    float* Xw = args.Xg + xg_base(o0, q, args.P4);
    for (int i = 0; i < t.n && ok; ++i) {
      int64_t row = args.row_idx ? (int64_t)args.row_idx[o0 + i] : o0 + i;
      if (row < 0 || row >= args.rows_X || !isfinite(args.y[o0 + i])) { ok = false; break; }
      for (int c = 0; c < p; ++c) {
        float v = args.X[row * args.ldX + c];
        if (!isfinite(v)) ok = false;
        Xw[(int64_t)c * t.ld + i] = v;
      }
    }
    t.Xq = Xw;
  }
  if (!ok) { t.write_bad(); return; }
  // scratch slices
  int64_t slots = args.total_rows + (int64_t)args.B * (P + 1);
  int64_t s0 = o0 + (int64_t)q * (P + 1);
  float* zk = reinterpret_cast<float*>(args.scratch);
  t.zk = zk + s0;
  t.zw = zk + slots + s0;
  t.zi = reinterpret_cast<int*>(zk + 2 * slots) + s0;
  t.r = zk + 3 * slots + s0;
  size_t slot_bytes = ((size_t)slots * 16 + 255) & ~(size_t)255;
  float* perq = reinterpret_cast<float*>(args.scratch + slot_bytes) + (int64_t)q * ((int64_t)P * P + 16 * P);
  t.Bm = perq;
  float* v = perq + (int64_t)P * P;
  t.bv = v; t.bbest = v + P; t.dv = v + 2 * P; t.mu = v + 3 * P; t.hv = v + 4 * P; t.tv = v + 5 * P;
  int* iv = reinterpret_cast<int*>(v + 6 * P);
  t.code = iv; t.phan = iv + P; t.piv = iv + 2 * P; t.perm = iv + 3 * P; t.pcol = iv + 4 * P;
  t.code_prev = iv + 5 * P; t.phan_prev = iv + 6 * P; t.code_alt = iv + 7 * P;
  t.phan_alt = iv + 8 * P;  // 6 P floats + 9 P ints <= the 16 P per-problem slots
  t.run();
}

}  // namespace

cudaError_t launch_fit_thread(const FitArgs& a, cudaStream_t st, int) {
  int threads = 128;
  int blocks = (a.B + threads - 1) / threads;
  fit_thread_kernel<<<blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace ll
