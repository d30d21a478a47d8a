"""Plant plausible mistakes in copies of the oracle and check that the pins catch every one.

Each mutation is a textual edit of ``oracle/rct_oracle.c`` compiled into a
temporary library on the CPU; the original source is never modified.
"""
import pytest

import oracle
import oracle_checks as oc
from oracle.oracle import compile_oracle

MUTATIONS = {
    # the listing's (int) truncation instead of floor
    "truncate": [("double fi0 = floor(ix);", "double fi0 = trunc(ix);"),
                 ("double fj0 = floor(iy);", "double fj0 = trunc(iy);")],
    # the listing's bound tests with width and height swapped
    "swapped_bounds": [("int in_i0 = (i0 >= 0 && i0 < W);", "int in_i0 = (i0 >= 0 && i0 < H);"),
                       ("int in_i1 = (i0 + 1 >= 0 && i0 + 1 < W);", "int in_i1 = (i0 + 1 >= 0 && i0 + 1 < H);"),
                       ("int in_j0 = (j0 >= 0 && j0 < H);", "int in_j0 = (j0 >= 0 && j0 < W);"),
                       ("int in_j1 = (j0 + 1 >= 0 && j0 + 1 < H);", "int in_j1 = (j0 + 1 >= 0 && j0 + 1 < W);"),
                       ("fi0 < (double)W && fj0 >= -1.0 && fj0 < (double)H", "fi0 < (double)H && fj0 >= -1.0 && fj0 < (double)W")],
    # x and y interpolation weights transposed
    "transposed_weights": [("double valb = (1.0 - fx) * bl + fx * br;", "double valb = (1.0 - fy) * bl + fy * br;"),
                           ("double valt = (1.0 - fx) * tl + fx * tr;", "double valt = (1.0 - fy) * tl + fy * tr;"),
                           ("double val = (1.0 - fy) * valb + fy * valt;", "double val = (1.0 - fx) * valb + fx * valt;")],
    # a sign slip inside one lerp
    "lerp_sign": [("double valt = (1.0 - fx) * tl + fx * tr;", "double valt = (1.0 - fx) * tl - fx * tr;")],
    # weight 1/w instead of 1/w^2
    "weight_power": [("*out = val / (w * w);", "*out = val / w;")],
    # matrix read column-major as printed in the listing, while the API passes row-major
    "column_major": [("double u = A[0] * wx + A[1] * wy + A[2] * wz + A[3];", "double u = A[0] * wx + A[3] * wy + A[6] * wz + A[9];"),
                     ("double v = A[4] * wx + A[5] * wy + A[6] * wz + A[7];", "double v = A[1] * wx + A[4] * wy + A[7] * wz + A[10];"),
                     ("double w = A[8] * wx + A[9] * wy + A[10] * wz + A[11];", "double w = A[2] * wx + A[5] * wy + A[8] * wz + A[11];")],
    # dropped translation column
    "dropped_translation": [("double u = A[0] * wx + A[1] * wy + A[2] * wz + A[3];", "double u = A[0] * wx + A[1] * wy + A[2] * wz;")],
    # wrong tap: top-left fetches the top-right pixel
    "wrong_tap": [("if (in_j1 && in_i0) tl = img[(j0 + 1) * (long)W + i0];", "if (in_j1 && in_i0) tl = img[(j0 + 1) * (long)W + i0 + 1];")],
    # image addressed column-major
    "transposed_image": [("bl = img[j0 * (long)W + i0];", "bl = img[i0 * (long)H + j0];"),
                         ("br = img[j0 * (long)W + i0 + 1];", "br = img[(i0 + 1) * (long)H + j0];"),
                         ("tl = img[(j0 + 1) * (long)W + i0];", "tl = img[i0 * (long)H + j0 + 1];"),
                         ("tr = img[(j0 + 1) * (long)W + i0 + 1];", "tr = img[(i0 + 1) * (long)H + j0 + 1];")],
    # voxel corner instead of voxel centre
    "half_voxel": [("double wx = origin[0] + x * spacing[0];\n                    double upd;",
                    "double wx = origin[0] + (x + 0.5) * spacing[0];\n                    double upd;")],
    # the truncating index rule falls back to floor
    "trunc_as_floor": [("        fi0 = trunc(ix);\n        fj0 = trunc(iy);", "        fi0 = floor(ix);\n        fj0 = floor(iy);")],
    # the truncating index rule rounds to nearest instead of toward zero
    "trunc_as_round": [("        fi0 = trunc(ix);\n        fj0 = trunc(iy);", "        fi0 = round(ix);\n        fj0 = round(iy);")],
    # last view dropped
    "dropped_view": [("for (int i = 0; i < n_views; ++i) {\n        const double *Ai", "for (int i = 0; i + 1 < n_views; ++i) {\n        const double *Ai")],
    # weights swapped within a lerp: (fx) on the left tap
    "swapped_lerp": [("double valb = (1.0 - fx) * bl + fx * br;", "double valb = fx * bl + (1.0 - fx) * br;")],
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
