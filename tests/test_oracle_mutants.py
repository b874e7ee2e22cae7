"""The oracle's pins catch plausible mistakes.  Each mutant is a copy of oracle/ozaki_oracle.c
with one mistake planted (a dropped term, a wrong sign or index, a transposed operand, a wrong
rounding rule), compiled on the CPU into its own library, or a copy of the oracle package whose
Python half (oracle/__init__.py) carries the mistake; the pin suites (tests/test_oracle.py,
tests/test_oracle_selector.py) then run against it in a subprocess and must fail.  The
unmodified sources, compiled and copied the same way, must pass (the controls), so a failure
comes from the planted mistake and not from the harness.  No GPU is involved."""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ozaki_oracle.c")
PY_SRC = os.path.join(ROOT, "oracle", "__init__.py")

# (name, text in the source, replacement): each text occurs exactly once
MUTANTS = [
    ("digits rounded instead of truncated", "    double q = trunc(y);", "    double q = round(y);"),
    ("row exponent off by one", "    e[i] = ex;\n    for (int64_t l = 0; l < k; ++l) {\n      double a = ldexp(",
     "    e[i] = ex + 1;\n    for (int64_t l = 0; l < k; ++l) {\n      double a = ldexp("),
    ("last group dropped", "  for (int gi = 0; gi < ng; ++gi) {\n    int g = gi + 2;",
     "  for (int gi = 0; gi < ng - 1; ++gi) {\n    int g = gi + 2;"),
    ("triangle bound p + q <= s", "if (!square && p + q > s + 1) continue;", "if (!square && p + q > s) continue;"),
    ("column exponent with the wrong sign", "int64_t E = (int64_t)ei + fj - 7 * top;",
     "int64_t E = (int64_t)ei - fj - 7 * top;"),
    ("op(X) indexes transposed", "return (t == 'N' || t == 'n') ? X[r + c * ld] : X[c + r * ld];",
     "return (t == 'N' || t == 'n') ? X[c + r * ld] : X[r + c * ld];"),
    ("final rounding: ties away from zero", "if (rbit && (sticky || (Q & 1ull))) Q += 1;", "if (rbit) Q += 1;"),
    ("final rounding: sticky bits ignored", "if (rbit && (sticky || (Q & 1ull))) Q += 1;",
     "if (rbit && (Q & 1ull)) Q += 1;"),
    ("two_sum without the error of b", "dd_t r = {s, (a - (s - bb)) + (b - bb)};", "dd_t r = {s, (a - (s - bb))};"),
    ("double-double reference drops beta C", "if (beta != 0.0) r = dd_add(r, two_prod(beta, C[i + j * ldc]));",
     "if (0) r = dd_add(r, two_prod(beta, C[i + j * ldc]));"),
    ("complex combine Re = rr + ii", "Gc[((int64_t)gi * m + i) * n + j] = rr - ii;",
     "Gc[((int64_t)gi * m + i) * n + j] = rr + ii;"),
    ("conjugation not applied", "*im = (t == 'C' || t == 'c') ? -p[1] : p[1];", "*im = p[1];"),
    ("complex exponent from the real parts only",
     "      if (fabs(re) > amax) amax = fabs(re);\n      if (fabs(im) > amax) amax = fabs(im);\n",
     "      if (fabs(re) > amax) amax = fabs(re);\n"),
    ("3M imaginary part RN(P3 - P1) + P2", "double ti = d - p2;", "double ti = d + p2;"),
    ("alpha and beta in two roundings instead of one fma",
     "*c = (beta == 0.0) ? alpha * t : fma(alpha, t, beta * (*c));",
     "*c = (beta == 0.0) ? alpha * t : alpha * t + beta * (*c);"),
    ("a priori bound 2^7 too small", "ldexp(acc * (1.0 + 4.0 * k * ldexp(1.0, -53)), e[i] + f[j] - 7 * s)",
     "ldexp(acc * (1.0 + 4.0 * k * ldexp(1.0, -53)), e[i] + f[j] - 7 * s - 7)"),
    ("feature bins five wide", "bin = gap < 36 ? (gap < 0 ? 0 : gap / 4) : 9;",
     "bin = gap < 36 ? (gap < 0 ? 0 : gap / 5) : 9;"),
    ("BF16 rounding ties away", "u += 0x7FFFu + ((u >> 16) & 1u);", "u += 0x8000u;"),
    ("ReLU derivative dropped in layer 1", "dh1[j] = h1[j] > 0 ? a : 0;", "dh1[j] = a;"),
    ("selector decision one class high", "int s = chosen < 0 ? fallback : s_lo + chosen;",
     "int s = chosen < 0 ? fallback : s_lo + chosen + 1;"),
    ("complex alpha in two roundings", "double re = fma(alpha[0], tr, -(alpha[1] * ti));\n      double im = fma(alpha[0], ti, alpha[1] * tr);\n      if (do_beta) {\n        double br = fma(beta[0], c[0], -(beta[1] * c[1]));\n        double bi = fma(beta[0], c[1], beta[1] * c[0]);\n        re += br; im += bi;\n      }\n      c[0] = re; c[1] = im;\n    }\n  free(e);",
     "double re = alpha[0] * tr - alpha[1] * ti;\n      double im = fma(alpha[0], ti, alpha[1] * tr);\n      if (do_beta) {\n        double br = fma(beta[0], c[0], -(beta[1] * c[1]));\n        double bi = fma(beta[0], c[1], beta[1] * c[0]);\n        re += br; im += bi;\n      }\n      c[0] = re; c[1] = im;\n    }\n  free(e);"),
    ("double-double times a double drops the low part", "  p.lo += a.lo * b;\n", ""),
    ("naive GEMM ignores alpha when beta != 0", "alpha * acc + beta * (*c);", "acc + beta * (*c);"),
    ("slice products pair digits of different k", "for (int64_t l = 0; l < k; ++l) acc += (int64_t)a[l] * (int64_t)b[l];",
     "for (int64_t l = 0; l < k; ++l) acc += (int64_t)a[l] * (int64_t)b[k - 1 - l];"),
    ("op(B) = B^H without the conjugation", "digits_of(ldexp(-p[1], -ex), s, &DB[(2 * j + 1) * k + l], R2 * k);",
     "digits_of(ldexp(p[1], -ex), s, &DB[(2 * j + 1) * k + l], R2 * k);"),
    ("subnormal results not clamped to 2^-1074", "  if (q < -1074) q = -1074;\n", ""),
    ("overflow saturates at the largest finite value", "if (top > 1023) return neg ? -INFINITY : INFINITY;",
     "if (top > 1023) return neg ? -1.7976931348623157e308 : 1.7976931348623157e308;"),
    ("a dropped dd error term in the complex reference", "        sr = dd_add(sr, two_prod(-ai, bi));\n", ""),
    ("softmax denominator off", "for (int o = 0; o < SEL_OUT; ++o) p[o] = exp(z[o] - zm) / se;",
     "for (int o = 0; o < SEL_OUT; ++o) p[o] = exp(z[o] - zm) / (se + 1e-3);"),
    ("loss without the max shift", "loss += (log(se) + zm - z[y[b]]) / B;", "loss += (log(se) - z[y[b]]) / B;"),
    ("layer-2 weight gradient with the wrong activation", "grad[O_W2 + o * SEL_H + j] += dh2[o] * h1[j];",
     "grad[O_W2 + o * SEL_H + j] += dh2[o] * h2[j];"),
    ("inference drops the layer-1 bias", "    float a = b1[o];\n", "    float a = 0.f;\n"),
    ("inference without the layer-1 ReLU", "h1[o] = a > 0.f ? a : 0.f;", "h1[o] = a;"),
    ("feature log2 k off by one", "out[2] = log2f((float)k);", "out[2] = log2f((float)(k + 1));"),
    ("B histogram normalised by m k", "out[13 + b] = (float)(hist[1][b] / ((double)n * (double)k));",
     "out[13 + b] = (float)(hist[1][b] / ((double)m * (double)k));"),
    ("naive complex alpha sign", "ti = alpha[0] * si + alpha[1] * sr;", "ti = alpha[0] * si - alpha[1] * sr;"),
    ("complex split writes Im digits into the Re row",
     "digits_of(ldexp(im, -ex), s, &D[(2 * i + 1) * k + l], R2 * k);",
     "digits_of(ldexp(im, -ex), s, &D[(2 * i) * k + l], R2 * k);"),
    ("row maximum from the first entry only", "      double a = fabs(op_r(trans, X, ld, i, l));\n      if (a > amax) amax = a;",
     "      double a = fabs(op_r(trans, X, ld, i, l));\n      if (l == 0) amax = a;"),
    ("dd addition drops the high error", "  s.lo += t.hi;\n  s = quick_two_sum(s.hi, s.lo);", "  s = quick_two_sum(s.hi, s.lo);"),
    ("3M real part P1 + P2", "double tr = p1 - p2;", "double tr = p1 + p2;"),
    ("rounding gives up on long tails", "if (r > 255) { /* everything", "if (r > 60) { /* everything"),
    ("negative group products not sign-extended", "uint64_t fill = v < 0 ? ~0ull : 0ull;", "uint64_t fill = 0ull;"),
    ("256-bit addition drops carries", "    c >>= 64;\n", "    c = 0;\n"),
    ("negation without the +1", "one.w[0] = 1;", "one.w[0] = 0;"),
    ("group weights one bit too high", "i256_from_i64_shl(&t, G[((int64_t)gi * m + i) * n + j], 7 * (top - g));",
     "i256_from_i64_shl(&t, G[((int64_t)gi * m + i) * n + j], 7 * (top - g) + 1);"),
    ("complex beta in two roundings",
     "        double br = fma(beta[0], c[0], -(beta[1] * c[1]));\n        double bi = fma(beta[0], c[1], beta[1] * c[0]);\n        re += br; im += bi;\n      }\n      c[0] = re; c[1] = im;\n    }\n  free(e);",
     "        double br = beta[0] * c[0] - beta[1] * c[1];\n        double bi = fma(beta[0], c[1], beta[1] * c[0]);\n        re += br; im += bi;\n      }\n      c[0] = re; c[1] = im;\n    }\n  free(e);"),
    ("output gradient not averaged over the batch", "dz[o] = (p[o] - (o == y[b] ? 1.0 : 0.0)) / B;",
     "dz[o] = (p[o] - (o == y[b] ? 1.0 : 0.0));"),
    ("BF16 bits widened one place short", "uint32_t u = (uint32_t)h << 16;", "uint32_t u = (uint32_t)h << 15;"),
    ("zero entries counted in the first feature bin", "        int bin = 9;\n        if (v != 0) {",
     "        int bin = 0;\n        if (v != 0) {"),
]

# mistakes planted in the Python half of the oracle (oracle/__init__.py)
PY_MUTANTS = [
    ("3M operand Sa = Ar - Ai", "return (Ar, Ai, np.asfortranarray(Ar + Ai)), (Br, Bi, np.asfortranarray(Br + Bi))",
     "return (Ar, Ai, np.asfortranarray(Ar - Ai)), (Br, Bi, np.asfortranarray(Br + Bi))"),
    ("op(X) = X^T for 'C' (no conjugation)", "return np.asfortranarray(X if t in \"Nn\" else (X.T if t in \"Tt\" else X.conj().T))",
     "return np.asfortranarray(X if t in \"Nn\" else X.T)"),
    ("3M product P3 one slice short", "P3 = dgemm_emu(Ar, Br, s), dgemm_emu(Ai, Bi, s), dgemm_emu(Sa, Sb, s)",
     "P3 = dgemm_emu(Ar, Br, s), dgemm_emu(Ai, Bi, s), dgemm_emu(Sa, Sb, s - 1)"),
    ("|A||B| without the absolute values", "return dgemm_naive(np.abs(np.asarray(A)), np.abs(np.asarray(B)), transa, transb)",
     "return dgemm_naive(np.asarray(A), np.asarray(B), transa, transb)"),
    ("error metric ignores alpha", "scale = abs(alpha) * abs_product(A, B, transa, transb)",
     "scale = abs_product(A, B, transa, transb)"),
    ("3M bound without the third product's error", "im = e3 + e1 + e2 + u * (P3 + P1 + P2)",
     "im = e1 + e2 + u * (P3 + P1 + P2)"),
    ("error metric without the beta C0 term", "        scale = scale + abs(beta) * np.abs(np.asarray(C0))\n", ""),
    ("features with the operands' transposes swapped",
     "_load().orc_features(_b(transa), _b(transb), m, n, k,", "_load().orc_features(_b(transb), _b(transa), m, n, k,"),
    ("inference with the threshold of a different model", "float(model[\"thr\"]), int(model[\"s_lo\"]),",
     "float(model[\"thr\"]) * 0.5, int(model[\"s_lo\"]),"),
    ("columns of op(B) split without the flip", "return split(X, s, \"T\" if trans in \"Nn\" else \"N\")",
     "return split(X, s, trans)"),
    ("3M operands of B taken with op(A)'s transpose",
     "oA, oB = _op(np.asarray(A, dtype=np.complex128), transa), _op(np.asarray(B, dtype=np.complex128), transb)",
     "oA, oB = _op(np.asarray(A, dtype=np.complex128), transa), _op(np.asarray(B, dtype=np.complex128), transa)"),
    ("a priori bound for one slice more", "max(B.shape[0], 1), int(s), _ptr(out))", "max(B.shape[0], 1), int(s) + 1, _ptr(out))"),
]

PIN_SUITES = ["tests/test_oracle.py", "tests/test_oracle_selector.py"]
# a workload-generator test with no oracle arithmetic, and the slowest of the suites
DESELECT = "not kkr_kappa"


def _compile(text, out):
    c_path = out + ".c"
    with open(c_path, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", *oracle._CFLAGS, c_path, "-o", out, "-lm"])
    return out


def _run_pins(job):
    """job = (library, tree): the pin suites of `tree` (the repository, or a copy holding a mutated
    oracle package) against the compiled oracle `library`."""
    lib, tree = job
    env = dict(os.environ, OZG_ORACLE_LIB=lib, OMP_NUM_THREADS="2",
               PYTHONPATH=os.pathsep.join([ROOT, os.environ.get("PYTHONPATH", "")]))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "-k", DESELECT, *PIN_SUITES], cwd=tree, env=env, capture_output=True, text=True,
                       timeout=900)
    return r.returncode, (r.stdout + r.stderr)[-2000:]


def _py_tree(d, text):
    """A copy of the oracle package (with __init__.py replaced by `text`) and of the pin suites."""
    os.makedirs(os.path.join(d, "oracle"))
    os.makedirs(os.path.join(d, "tests"))
    with open(os.path.join(d, "oracle", "__init__.py"), "w") as f:
        f.write(text)
    shutil.copy(SRC, os.path.join(d, "oracle"))
    for name in ("conftest.py", "test_oracle.py", "test_oracle_selector.py"):
        shutil.copy(os.path.join(ROOT, "tests", name), os.path.join(d, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(d, "tests", "golden"))
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    return d


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    src = open(SRC).read()
    py = open(PY_SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    control = _compile(src, str(d / "control.so"))
    jobs = {"control": (control, ROOT), "control (copied tree)": (control, _py_tree(str(d / "pyc"), py))}
    for idx, (name, old, new) in enumerate(MUTANTS):
        assert src.count(old) == 1, f"mutant '{name}': its text must occur exactly once"
        jobs[name] = (_compile(src.replace(old, new), str(d / f"m{idx}.so")), ROOT)
    for idx, (name, old, new) in enumerate(PY_MUTANTS):
        assert py.count(old) == 1, f"mutant '{name}': its text must occur exactly once"
        jobs[name] = (control, _py_tree(str(d / f"py{idx}"), py.replace(old, new)))
    with ThreadPoolExecutor(max_workers=max(1, min(8, (os.cpu_count() or 2) // 2))) as ex:
        res = dict(zip(jobs, ex.map(_run_pins, jobs.values())))
    return res


@pytest.mark.parametrize("name", ["control", "control (copied tree)"])
def test_control_copy_passes_the_pins(outcomes, name):
    rc, log = outcomes[name]
    assert rc == 0, log


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS + PY_MUTANTS])
def test_planted_mistake_fails_a_pin(outcomes, name):
    rc, log = outcomes[name]
    assert rc == 1, f"mutant '{name}' survived the pins (pytest rc {rc}):\n{log}"
