"""Plant plausible mistakes in a copy of the oracle and check that the pins
catch every one (CPU only).  The planted copies are built in a temporary
directory; the oracle itself is never modified."""
import os
import subprocess
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import oracle  # noqa: E402
from oracle import build as obuild  # noqa: E402
from oracle_pins import ALL_PINS  # noqa: E402

# (name, text in oracle.c, replacement)
MUTANTS = [
    ("add_sign", "case ORC_ADD: acc = (acc + v) & mask;", "case ORC_ADD: acc = (acc - v) & mask;"),
    ("dropped_first_term", "    for (i = 0; i < n; ++i) {\n        uint64_t v",
     "    for (i = 1; i < n; ++i) {\n        uint64_t v"),
    ("max_identity", "case ORC_MAX: v = INT32_MIN; break;", "case ORC_MAX: v = INT32_MIN + 1; break;"),
    ("zero_extension", "return (int64_t)((const int32_t *)x)[i];",
     "return (int64_t)((const uint32_t *)x)[i];"),
    ("land_not_normalised", "case ORC_LAND: acc = (acc != 0) && (v != 0); break;",
     "case ORC_LAND: acc = acc & v; break;"),
    ("min_uses_unsigned", "case ORC_MIN: if (sv < sa) acc = v; break;",
     "case ORC_MIN: if (v < acc) acc = v; break;"),
    ("signed_zero_order", "if (v == a && v == 0.0 && signbit(a) && !signbit(v)) return 1;",
     "if (v == a && v == 0.0 && !signbit(a) && signbit(v)) return 1;"),
    ("f32_accumulates_in_double",
     "static float fold_f32(const float *x, int64_t n, int64_t stride, int op, float acc)",
     "static float fold_f32(const float *x, int64_t n, int64_t stride, int op, double acc)"),
    ("truth_exponent", "off = e - 53 + 1074;", "off = e - 52 + 1074;"),
    ("truth_ties_away", "if (rnd && (sticky || (M & 1))) M += 1;", "if (rnd) M += 1;"),
    ("truth_no_sticky", "for (i = p - 54; i >= 0 && !sticky; --i) sticky = la_bit(A, i);", ""),
    ("matmul_transposed_b", "sum += a[i * len + l] * b[l * len + j];", "sum += a[i * len + l] * b[j * len + l];"),
    ("matmul_sum_init", "    float sum = 0;\n    for (l = 0;", "    float sum = 0.5f;\n    for (l = 0;"),
    ("row_stride", "(size_t)(r * ld) * (size_t)ib", "(size_t)(r * cols) * (size_t)ib"),
    ("segment_bound", "int64_t lo = offsets[s], hi = offsets[s + 1];",
     "int64_t lo = offsets[s], hi = offsets[s + 1] - (offsets[s + 1] > offsets[s]);"),
    ("nearest_tie_order", "return da < db || (da == db && ia < ib);", "return da < db || (da == db && ia > ib);"),
    ("nearest_fma_like", "float d = dx * dx + dy * dy;", "float d = (float)((double)dx * dx + (double)dy * dy);"),
    ("variance_sign", "var = n > 0 ? s2 / (double)n - mean * mean : 0.0;", "var = n > 0 ? s2 / (double)n + mean * mean : 0.0;"),
    ("bfs_no_left_move", "if (q > 0) nb[cnt++] = u - 1;", ""),
    ("bfs_ignores_walls", "if (open[v] && dist[v] < 0) {", "if (dist[v] < 0) {"),
    ("rows_bt_reads_b_layout", "for (l = 0; l < len; ++l) sum += ar[l] * bc[l];",
     "for (l = 0; l < len; ++l) sum += ar[l] * bt[l * len + j];"),
    ("rows_bt_truth_transposed", "double p = (double)ar[l] * (double)bc[l];",
     "double p = (double)ar[l] * (double)bt[l * len + j];"),
    ("rows_bt_abs_is_signed", "absab[i * len + j] = t;", "absab[i * len + j] = s;"),
    ("truth_abs_drops_sign", "la_add(&A, fabs(load_fp(x, in_type, i * stride)));",
     "la_add(&A, load_fp(x, in_type, i * stride));"),
]


def test_mutant_texts_present():
    src = open(obuild.SRC).read()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, name, old, new):
    src = open(obuild.SRC).read()
    assert src.count(old) == 1
    d = tmp_path
    with open(os.path.join(d, "oracle.c"), "w") as f:
        f.write(src.replace(old, new))
    with open(os.path.join(obuild.HERE, "oracle.h")) as f:
        hdr = f.read()
    with open(os.path.join(d, "oracle.h"), "w") as f:
        f.write(hdr)
    lib = os.path.join(d, "libmutant.so")
    subprocess.run(["gcc"] + obuild.CFLAGS + ["-o", lib, os.path.join(d, "oracle.c"), "-lm"],
                   check=True)
    orc = oracle.OracleLib(lib)
    caught = []
    for pin in ALL_PINS:
        try:
            pin(orc)
        except (AssertionError, ValueError):
            caught.append(pin.__name__)
    assert caught, "no pin caught mutant %s" % name
