"""The oracle's pins catch plausible mistakes in the oracle.

Each mutant below is the oracle's C source with one planted mistake of the
kinds a restatement of the method can contain: a dropped or halved term, a
flipped sign, a wrong index or a transposed operand, a wrong tie rule, a
wrong branch of the chop.  Every mutant is compiled on the CPU, and the
pins of tests/test_oracle.py run against it in a child process (cheapest
first, stopping at the first failure); the test requires that some pin
fails for every mutant, and that the unmodified source passes them all
when built and run the same way.  No GPU is involved.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ladlasso_oracle.c")
WORK = os.path.join(ROOT, "oracle", "_build", "mutants")

# name -> (exact text in the oracle source, its replacement); each text
# occurs exactly once in the source
MUTANTS = {
    # objective and residual
    "objective: halved penalty": (
        "for (int j = 0; j < p; ++j) f += lam * fabs(b[j]);\n  return f;\n}\n\nstatic void residual",
        "for (int j = 0; j < p; ++j) f += 0.5 * lam * fabs(b[j]);\n  return f;\n}\n\nstatic void residual"),
    "residual: wrong sign": (
        "ri -= X[(size_t)i * p + j] * b[j];\n    r[i] = ri;",
        "ri += X[(size_t)i * p + j] * b[j];\n    r[i] = ri;"),
    "gauss_solve: back substitution sign": (
        "s -= A[k * m + c] * rhs[c];",
        "s += A[k * m + c] * rhs[c];"),
    # weighted median (Sections 3.3-3.5)
    "weighted median: wrong half weight": (
        "double half = 0.5 * W", "double half = 0.4 * W"),
    "weighted median: flat segment moves to its left end": (
        "if (cur > lo && cur < hi) return cur;", "if (cur > lo && cur < hi) return lo;"),
    "weighted median: strict half": (
        "if (cum >= half) {", "if (cum > half) {"),
    # axis update (Section 3.3)
    "axis update: key sign": (
        "work[m].z = b[j] + r[i] / x;", "work[m].z = b[j] - r[i] / x;"),
    "axis update: squared weights": (
        "work[m].w = fabs(x);", "work[m].w = x * x;"),
    "axis update: doubled penalty weight": (
        "work[m].w = lam; work[m].id = COORD_ID(j);", "work[m].w = 2.0 * lam; work[m].id = COORD_ID(j);"),
    "axis update: b_j not updated with the residual": (
        "    for (int i = 0; i < n; ++i) r[i] -= X[(size_t)i * p + j] * d;\n    b[j] = t;",
        "    for (int i = 0; i < n; ++i) r[i] -= X[(size_t)i * p + j] * d;"),
    "ccd: convergence measured on the last move only": (
        "mx = fmax(mx, fabs(d));", "mx = fabs(d);"),
    "chop: probe objective without the absolute value": (
        "for (int i = 0; i < n; ++i) f += fabs(r[i]);\n  for (int j = 0; j < p; ++j) f += lam * fabs(b[j]);\n  return f;\n}\n\n/* ---",
        "for (int i = 0; i < n; ++i) f += r[i];\n  for (int j = 0; j < p; ++j) f += lam * fabs(b[j]);\n  return f;\n}\n\n/* ---"),
    "polish: gradient includes the basis rows": (
        "      if (inb[i]) continue;\n      double s = sgn(r[i]);", "      double s = sgn(r[i]);"),
    "axis update: residual update sign": (
        "for (int i = 0; i < n; ++i) r[i] -= X[(size_t)i * p + j] * d;\n    b[j] = t;",
        "for (int i = 0; i < n; ++i) r[i] += X[(size_t)i * p + j] * d;\n    b[j] = t;"),
    # chop (Sections 3.4-3.5)
    "chop: sub-search also moves the chop axis": (
        "if (j == skip) continue;", "if (j == skip && 0) continue;"),
    "chop: ternary drops the wrong third": (
        "if (g1 < g2) hi = m2;", "if (g1 < g2) lo = m1;"),
    "chop: range extension never triggers left": (
        "if (ga < gm) {", "if (ga < gm && 0) {"),
    "chop: four sections drop the lowest probe's section": (
        "if (g1 <= g2 && g1 <= g3) hi = t2;", "if (g1 <= g2 && g1 <= g3) lo = t1;"),
    # vertex polish (Section 3.2 optimum at a vertex; multipliers, edge search)
    "polish: gradient sign of the row terms": (
        "if (s != 0.0) for (int j = 0; j < p; ++j) g[j] -= s * X[(size_t)i * p + j];",
        "if (s != 0.0) for (int j = 0; j < p; ++j) g[j] += s * X[(size_t)i * p + j];"),
    "polish: penalty gradient sign": (
        "if (!real) g[j] += lam * sgn(b[j]);", "if (!real) g[j] -= lam * sgn(b[j]);"),
    "polish: row and coordinate caps swapped": (
        "double cap = basis[k].code >= 0 ? 1.0 : (basis[k].phantom ? 0.0 : lam);",
        "double cap = basis[k].code >= 0 ? lam : (basis[k].phantom ? 0.0 : 1.0);"),
    "polish: multipliers solved with B instead of its transpose": (
        "Bt[(size_t)c * p + k] = B[(size_t)k * p + c];",
        "Bt[(size_t)k * p + c] = B[(size_t)k * p + c];"),
    "polish: edge breakpoint sign": (
        "bp[m].z = r[i] / vi;", "bp[m].z = -r[i] / vi;"),
    "polish: coordinate breakpoint sign": (
        "bp[m].z = -b[j] / d[j];", "bp[m].z = b[j] / d[j];"),
    "polish: the released hyperplane stays in the basis": (
        "basis[q].code = own;", "basis[q].code = basis[q].code;"),
    "polish: zero coordinates snapped to 1": (
        "if (basis[k].code < 0 && !basis[k].phantom) b[-basis[k].code - 1] = 0.0;",
        "if (basis[k].code < 0 && !basis[k].phantom) b[-basis[k].code - 1] = 1.0;"),
    "polish: non-unique optima never flagged": (
        "*nonunique = phantoms > 0 || at_cap > 0;", "*nonunique = 0;"),
    # lambda_max
    "lambda_max: y instead of sign(y)": (
        "c += X[(size_t)i * p + j] * sgn(y[i]);", "c += X[(size_t)i * p + j] * y[i];"),
    # brute-force vertex enumeration (Section 3.2)
    "brute force: row hyperplane right-hand side sign": (
        "rhs[k] = y[hk];", "rhs[k] = -y[hk];"),
    "brute force: row hyperplanes only (no b_j = 0)": (
        "int H = n + p;", "int H = n;"),
    # dense simplex of the LP (Section 3.1)
    "simplex: coefficient cost 1 instead of lambda": (
        "for (int j = 0; j < 2 * p; ++j) cost[j] = lam;", "for (int j = 0; j < 2 * p; ++j) cost[j] = 1.0;"),
    "simplex: negative part added": (
        "else if (bas[i] < 2 * p) b_out[bas[i] - p] -= xv;",
        "else if (bas[i] < 2 * p) b_out[bas[i] - p] += xv;"),
    "simplex: ratio test on negative entries": (
        "if (a > eps) {\n        double ratio", "if (a < -eps) {\n        double ratio"),
    "simplex: enters a positive reduced cost": (
        "for (int j = 0; j < m; ++j) if (z[j] < -eps) { e = j; break; }",
        "for (int j = 0; j < m; ++j) if (z[j] > eps) { e = j; break; }"),
    "simplex: pivot row not normalised": (
        "for (int j = 0; j <= m; ++j) pr[j] /= pv;", ""),
    "gauss_solve: right-hand side not eliminated": (
        "      rhs[i] -= l * rhs[k];\n", ""),
    "brute force: keeps the last minimiser, not the first": (
        "      if (f < fbest - tolf) {", "      if (f <= fbest + tolf) {"),
    # duality-gap certificate
    "certificate: dual signs flipped": (
        "if (fabs(r[i]) > eps_r * fmax(1.0, ymax)) u[i] = sgn(r[i]);",
        "if (fabs(r[i]) > eps_r * fmax(1.0, ymax)) u[i] = -sgn(r[i]);"),
    "certificate: uniqueness without |E| = |S|": (
        "int solved = 1, unique_ok = (ne == ns);", "int solved = 1, unique_ok = 1;"),
    "certificate: no scaling into the lambda box": (
        "if (lam > 0) theta = fmax(theta, cmax / lam);", "if (lam > 0 && 0) theta = fmax(theta, cmax / lam);"),
    # active-set gradient
    "gradient: validation term sign": (
        "for (int a = 0; a < ns; ++a) gS[a] -= s * Xv[(size_t)v * p + S[a]];",
        "for (int a = 0; a < ns; ++a) gS[a] += s * Xv[(size_t)v * p + S[a]];"),
    "gradient: X_RS instead of its transpose": (
        "M[(size_t)a * ns + c] = X[(size_t)R[c] * p + S[a]];",
        "M[(size_t)a * ns + c] = X[(size_t)R[a] * p + S[c]];"),
    "gradient: validation target term sign": (
        "gyv[v] = up * s;", "gyv[v] = -up * s;"),
    "gradient: training design rows term sign": (
        "gX[(size_t)R[c] * p + S[a]] = -up * gS[c] * b[S[a]];",
        "gX[(size_t)R[c] * p + S[a]] = up * gS[c] * b[S[a]];"),
    "gradient: nonzero lambda derivative": (
        "  *glam = 0.0;\n  double* gS", "  *glam = 1.0;\n  double* gS"),
    "lambda_max: no absolute value": (
        "best = fmax(best, fabs(c));", "best = fmax(best, c);"),
    "weighted median: flat segment's upper end returns the lower": (
        "if (cur >= hi) { *owner = bp[g].id; return hi; }",
        "if (cur >= hi) { *owner = bp[g].id; return lo; }"),
    "chop: never run at p = 2": (
        "if (!is_opt && o->chop && p >= 2) {", "if (!is_opt && o->chop && p >= 3) {"),
    "chop: probe does not fix b_k": (
        "    c->b[k] = t;\n  }", "  }"),
    "chop: stale residual after an improving chop": (
        "    memcpy(b, bb, sizeof(double) * p);\n    residual(n, p, X, y, b, r);",
        "    memcpy(b, bb, sizeof(double) * p);"),
    "gradient: validation design term sign": (
        "gXv[(size_t)v * p + j] = -up * s * b[j];", "gXv[(size_t)v * p + j] = up * s * b[j];"),
}

# the pins of tests/test_oracle.py, cheapest first: (function, arguments)
PINS = [
    ("test_axis_update_is_exact_1d_minimum", ()),
    ("test_p1_closed_form_weighted_median", ()),
    ("test_flat_segment_tie_rule_keeps_current_value", ()),
    ("test_lambda_max_gives_zero_and_below_does_not", ()),
    ("test_square_system_tiny_lambda_interpolates", ()),
    ("test_intercept_only_gives_sample_median", ()),
    ("test_invariances", ()),
    ("test_sign_symmetries_and_a_zero_column", ()),
    ("test_optimum_along_lambda_is_nondecreasing_and_concave", ()),
    ("test_bad_lambda_status", ()),
    ("test_non_unique_optima_are_flagged", ()),
    ("test_tiny_golden_brute_simplex_method_agree", ()),
] + [("test_random_tiny_brute_equals_simplex_equals_method", (s,)) for s in range(6)] + [
    ("test_chop_is_exact_on_two_coordinates", (3,)),
    ("test_chop_is_exact_on_two_coordinates", (4,)),
    ("test_certificate_detects_suboptimal_points", ()),
    ("test_plain_ccd_stalls_but_method_does_not", ()),
    ("test_chop_only_variant_is_not_always_optimal_but_never_worse", ()),
    ("test_lambda_path_warm_start_matches_cold_fits", ()),
    ("test_exact_finish_makes_the_result_independent_of_chop_settings", ()),
    ("test_fit_batch_matches_single_fits", ()),
    ("test_active_set_gradient_matches_finite_differences", ()),
    ("test_simplex_matches_scipy_highs", ()),
    ("test_dual_lp_value_equals_the_method_optimum", ()),
    ("test_medium_method_equals_simplex_and_certificate", ()),
]


def run_pins(lib_path: str) -> int:
    """Child process: run the pins against the oracle built at lib_path.
    Prints the first failing pin and returns 1, or returns 0 if all pass."""
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    import importlib.util
    import oracle
    oracle.use_library(lib_path)
    spec = importlib.util.spec_from_file_location(
        "oracle_pins", os.path.join(ROOT, "tests", "test_oracle.py"))
    pins = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(pins)
    for name, args in PINS:
        try:
            getattr(pins, name)(*args)
        except Exception as ex:  # an assertion, or a NaN/shape error downstream of one
            print(f"caught by {name}{args}: {type(ex).__name__}")
            return 1
    return 0


def _build_and_run(tag: str, source: str) -> tuple:
    """Compile `source` as the oracle, run the pins in a child process;
    returns (exit code, last output line)."""
    c = os.path.join(WORK, f"{tag}.c")
    so = os.path.join(WORK, f"{tag}.so")
    with open(c, "w") as f:
        f.write(source)
    try:
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", so, c, "-lm"])
        env = dict(os.environ, OMP_NUM_THREADS="1")
        try:
            pr = subprocess.run([sys.executable, os.path.abspath(__file__), so], env=env,
                                capture_output=True, text=True, timeout=300)
        except subprocess.TimeoutExpired:
            return ("timeout", "no pin finished within 300 s")
        out = (pr.stdout + pr.stderr).strip().split("\n")
        return (pr.returncode, out[-1] if out else "")
    finally:
        for path in (c, so):
            if os.path.exists(path):
                os.remove(path)


def _mutate(src: str, name: str) -> str:
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"{name}: the text to mutate occurs {src.count(old)} times"
    return src.replace(old, new)


@pytest.fixture(scope="module")
def outcomes():
    os.makedirs(WORK, exist_ok=True)
    src = open(SRC).read()
    jobs = {"unmodified": src}
    for i, name in enumerate(MUTANTS):
        jobs[f"m{i:02d}"] = _mutate(src, name)
    tags = list(jobs)
    workers = max(1, min(8, os.cpu_count() or 1))
    with ThreadPoolExecutor(workers) as ex:
        res = list(ex.map(lambda t: _build_and_run(t, jobs[t]), tags))
    return dict(zip(tags, res))


def test_unmodified_oracle_passes_every_pin(outcomes):
    rc, last = outcomes["unmodified"]
    assert rc == 0, last


@pytest.mark.parametrize("i,name", list(enumerate(MUTANTS)), ids=list(MUTANTS))
def test_planted_mistake_is_caught(outcomes, i, name):
    rc, last = outcomes[f"m{i:02d}"]
    # 1: a pin failed; a crash or a timeout would also expose the mistake,
    # but every mutant here is expected to fail a pin cleanly
    assert rc == 1, (name, rc, last)


if __name__ == "__main__":
    sys.exit(run_pins(sys.argv[1]))
