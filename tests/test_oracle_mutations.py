"""Plant plausible mistakes in copies of the oracle and check that the pins catch every one.

Each mutation is a textual edit of ``oracle/rct_oracle.c`` compiled into a
temporary library on the CPU; the original source is never modified.
"""
import pytest

import oracle
import oracle_checks as oc
from oracle.oracle import compile_oracle

MUTATIONS = {
    # the printed kernel's (int) truncation instead of floor for the default rule
    "truncate": [("? trunc(c) : floor(c);", "? trunc(c) : trunc(c);")],
    # the printed bounds test with width and height swapped
    "swapped_bounds": [("if (!(a >= 0.0 && a < (double)W && b >= 0.0 && b < (double)H)) return 0.0;",
                        "if (!(a >= 0.0 && a < (double)H && b >= 0.0 && b < (double)W)) return 0.0;")],
    # the weights along s and t transposed
    "transposed_weights": [("const double ws[2] = {1.0 - alpha, alpha};", "const double ws[2] = {1.0 - beta, beta};"),
                           ("const double wt[2] = {1.0 - beta, beta};", "const double wt[2] = {1.0 - alpha, alpha};")],
    # a sign slip in one weight
    "lerp_sign": [("const double wt[2] = {1.0 - beta, beta};", "const double wt[2] = {1.0 - beta, -beta};")],
    # distance weight 1/w instead of 1/w^2
    "weight_power": [("/ (q[2] * q[2]);", "/ q[2];")],
    # matrix read column-major as printed, while the API passes row-major
    "column_major": [("q[r] = A[4 * r] * p[0] + A[4 * r + 1] * p[1] + A[4 * r + 2] * p[2] + A[4 * r + 3];",
                      "q[r] = A[r] * p[0] + A[r + 3] * p[1] + A[r + 6] * p[2] + A[r + 9];")],
    # dropped translation column
    "dropped_translation": [("A[4 * r + 2] * p[2] + A[4 * r + 3];", "A[4 * r + 2] * p[2];")],
    # wrong tap: the grid offsets along s and t exchanged
    "wrong_tap": [("extended_pixel(img, W, H, a0 + da, b0 + db)", "extended_pixel(img, W, H, a0 + db, b0 + da)")],
    # image addressed column-major
    "transposed_image": [("return img[(long)b * W + (long)a];", "return img[(long)a * H + (long)b];")],
    # voxel corner instead of voxel centre
    "half_voxel": [("p[0] = origin[0] + x * spacing[0];", "p[0] = origin[0] + (x + 0.5) * spacing[0];")],
    # the truncating index rule falls back to floor
    "trunc_as_floor": [("? trunc(c) : floor(c);", "? floor(c) : floor(c);")],
    # the truncating index rule rounds to nearest instead of toward zero
    "trunc_as_round": [("? trunc(c) : floor(c);", "? round(c) : floor(c);")],
    # last view dropped
    "dropped_view": [("for (int i = 0; i < n_views; ++i) {\n        const double *Ai",
                      "for (int i = 0; i + 1 < n_views; ++i) {\n        const double *Ai")],
    # the two weights of one axis swapped
    "swapped_lerp": [("const double ws[2] = {1.0 - alpha, alpha};", "const double ws[2] = {alpha, 1.0 - alpha};")],
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    src = oracle.ORACLE_SRC.read_text()
    for old, new in MUTATIONS[name]:
        assert old in src, f"mutation {name}: target text not found in the oracle source"
        src = src.replace(old, new)
    mutated = tmp_path / f"mut_{name}.c"
    mutated.write_text(src)
    lib = oracle.load(compile_oracle(mutated, tmp_path / f"libmut_{name}.so"))
    caught = []
    for check in oc.ALL_CHECKS:
        try:
            check(lib)
        except (AssertionError, RuntimeError) as e:
            caught.append((check.__name__, str(e)[:80]))
    assert caught, f"planted mistake {name!r} passed every pin"
