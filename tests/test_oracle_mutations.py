"""Plant plausible mistakes in copies of the oracle's C source and check that
the pins catch every one: a dropped term, a wrong sign, a wrong index, a
transposed operand, a reversed loop.  Runs on the CPU only; the oracle itself
is never modified."""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
import oracle_pins as pins
from oracle import build as ob

# (name, text in mp_oracle.c, replacement)
MUTANTS = [
    ("two_sum error sign", "*e = ea + eb;", "*e = ea - eb;"),
    ("two_sum without the a correction", "double av = sum - bv;", "double av = a;"),
    ("quick_two_sum error sign", "*e = b - bv;", "*e = bv - b;"),
    ("two_prod fma sign", "*e = fma(a, b, -prod);", "*e = fma(a, b, prod);"),
    ("three_sum dropped low term", "or_two_sum(t2, t3, &nb, &nc);", "or_two_sum(t2, 0.0, &nb, &nc);"),
    ("three_sum2 dropped t3", "*b = t2 + t3;", "*b = t2;"),
    ("renorm drops folded terms", "s = s + t[i];", "s = s;"),
    ("renorm emits the error first", "r[k] = hi;\n                k = k + 1;\n                s = lo;",
     "r[k] = lo;\n                k = k + 1;\n                s = hi;"),
    ("renorm bottom-up pass skips c4", "double s = c[4];", "double s = 0.0;"),
    ("vec_sum with QuickTwoSum", "or_two_sum(x[i], s, &hi, &lo);", "or_quick_two_sum(x[i], s, &hi, &lo);"),
    ("vec_sum error slot", "e[i + 1] = lo;\n        s = hi;\n    }\n    e[0] = s;", "e[i + 1] = hi;\n        s = lo;\n    }\n    e[0] = s;"),
    ("vseb keeps the error in the else branch", "eps = hi;\n        }", "eps = lo;\n        }"),
    ("vseb off by one in the tail", "if (eps != 0.0 && j <= k - 1)", "if (eps != 0.0 && j < k - 1)"),
    ("dd_add dropped trailing sum", "e = e + w;", "e = e;"),
    ("dd_mul dropped cross product", "w3 = w1 + w2;", "w3 = w1;"),
    ("dd_mul wrong index", "w2 = x[1] * y[0];", "w2 = x[1] * y[1];"),
    ("dd_mul cross term fused (contracted)", "w1 = x[0] * y[1];\n    w2 = x[1] * y[0];\n    w3 = w1 + w2;",
     "w1 = 0.0;\n    w2 = x[1] * y[0];\n    w3 = fma(x[0], y[1], w2);"),
    ("td_mul wrong fma index", "double c = fma(x[1], y[1], b[2]);", "double c = fma(x[1], y[0], b[2]);"),
    ("td_mul dropped z32", "double z3 = z31 + z32;", "double z3 = z31;"),
    ("td_mul vseb off by one", "or_vseb(3, &e[1], 2, &r[1]);", "or_vseb(3, &e[0], 2, &r[1]);"),
    ("td_add merge order", "fabs(x[i]) >= fabs(y[j])", "fabs(x[i]) <= fabs(y[j])"),
    ("qd_add dropped t3", "t0 = (t0 + t1) + t3;", "t0 = (t0 + t1);"),
    ("qd_add wrong index", "t2 = w2 + u2;", "t2 = w2 + u1;"),
    ("qd_add wrong sign", "v3 = s3 - x[3];", "v3 = s3 + x[3];"),
    ("qd_mul dropped x3*y0", "s1 = s1 + x[3] * y[0];", ""),
    ("qd_mul dropped q5", "s1 = s1 + q5;", ""),
    ("qd_mul wrong three_sum operand", "or_three_sum(&p2, &q1, &q2);", "or_three_sum(&p2, &q1, &q1);"),
    ("qd_mul transposed operand", "or_two_prod(x[1], y[0], &p2, &q2);", "or_two_prod(x[0], y[1], &p2, &q2);"),
    ("td_addq drops a component", "or_qd_add(x4, y4, r4);\n    r[0] = r4[0];\n    r[1] = r4[1];\n    r[2] = r4[2];",
     "or_qd_add(x4, y4, r4);\n    r[0] = r4[0];\n    r[1] = r4[1];\n    r[2] = 0.0;"),
    ("td_mulq drops a component", "or_qd_mul(x4, y4, r4);\n    r[0] = r4[0];\n    r[1] = r4[1];\n    r[2] = r4[2];",
     "or_qd_mul(x4, y4, r4);\n    r[0] = r4[0];\n    r[1] = r4[1];\n    r[2] = 0.0;"),
    ("td_mulq pads with a nonzero", "double x4[4] = {x[0], x[1], x[2], 0.0};\n    double y4[4] = {y[0], y[1], y[2], 0.0};\n    double r4[4];\n    or_qd_mul",
     "double x4[4] = {x[0], x[1], x[2], x[2]};\n    double y4[4] = {y[0], y[1], y[2], 0.0};\n    double r4[4];\n    or_qd_mul"),
    ("accurate sort ascending", "while (j > 0 && fabs(v) > fabs(z[j - 1])) {", "while (j > 0 && fabs(v) < fabs(z[j - 1])) {"),
    ("accurate sort by value", "while (j > 0 && fabs(v) > fabs(z[j - 1])) {", "while (j > 0 && v > z[j - 1]) {"),
    ("accumulate emits the error", "c[k] = s;\n            k = k + 1;\n            u = e2;", "c[k] = e2;\n            k = k + 1;\n            u = s;"),
    ("accumulate emits on one error", "if (e2 != 0.0 && e1 != 0.0) {", "if (e2 != 0.0 || e1 != 0.0) {"),
    ("accumulate keeps the wrong error", "u = s;\n            v = e1;", "u = s;\n            v = e2;"),
    ("accumulate drops the accumulator", "c[k] = u;\n        c[k + 1] = v;", "c[k] = u;"),
    ("accumulate drops the tail", "double t = u + v;", "double t = 0.0;"),
    ("accurate td mul dropped p11", "p02, p11, p20, t3}", "p02, 0.0, p20, t3}"),
    ("accurate td mul wrong index", "or_two_prod(x[1], y[1], &p11, &q11);", "or_two_prod(x[1], y[0], &p11, &q11);"),
    ("accurate td mul dropped q01", "q01, q10, p02", "0.0, q10, p02"),
    ("accurate td mul dropped x1 y2", "t3 = fma(x[1], y[2], t3);", ""),
    ("accurate qd add drops a y component", "z[4 + c] = y[c];", "z[4 + c] = c < 3 ? y[c] : 0.0;"),
    ("gemm transposed B", "b[c] = B[c][p * ldb + j];", "b[c] = B[c][j * ldb + p];"),
    ("gemm swapped mul operands", "mp_mul(P, a, b, prod);", "mp_mul(P, b, a, prod);"),
    ("gemm skips the first term", "for (int64_t p = 0; p < k; ++p) {", "for (int64_t p = 1; p < k; ++p) {"),
    ("dgemm multiply and add rounded separately", "acc = fma(A[i * lda + p], B[p * ldb + j], acc);",
     "acc = acc + A[i * lda + p] * B[p * ldb + j];"),
    ("dgemm decreasing k", "for (int64_t p = 0; p < k; ++p)\n                acc = fma(",
     "for (int64_t p = k - 1; p >= 0; --p)\n                acc = fma("),
    ("dgemm skips the last term", "for (int64_t p = 0; p < k; ++p)\n                acc = fma(",
     "for (int64_t p = 0; p + 1 < k; ++p)\n                acc = fma("),
]

# a lighter pass of every pin (fewer random cases) for each mutant
QUICK = [(p, {"n": 150}) if p.__code__.co_varnames[:p.__code__.co_argcount].count("n") else (p, {})
         for p in pins.ALL_PINS]


@pytest.fixture(scope="module")
def src():
    with open(ob.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(src, name, old, new):
    assert src.count(old) == 1, "mutation site must be unique: %r" % old
    d = tempfile.mkdtemp(prefix="mutant_")
    try:
        path = os.path.join(d, "mp_oracle.c")
        shutil.copy(os.path.join(os.path.dirname(ob.SRC), "mp_oracle.h"), d)
        with open(path, "w") as f:
            f.write(src.replace(old, new))
        lib = ob.build(force=True, src=path, out=os.path.join(d, "libmutant.so"))
        L = oracle.lib(lib)
        caught = []
        for pin, kw in QUICK:
            try:
                pin(L, **kw)
            except AssertionError:
                caught.append(pin.__name__)
                break
        assert caught, "mutant '%s' passed every pin" % name
    finally:
        shutil.rmtree(d, ignore_errors=True)
