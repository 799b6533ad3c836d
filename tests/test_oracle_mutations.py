"""Each plausible mistake planted in a copy of the oracle's C source must fail
at least one pin. The mutants are built into a temporary directory on the CPU;
the real oracle is untouched."""
import os

import pytest

import oracle
from tests import pins

MUTANTS = {
    "y_sign": ("double s = -g[i];", "double s = g[i];"),
    "cholesky_index": ("s -= L[a * p + c] * L[b * p + c];", "s -= L[a * p + c] * L[a * p + c];"),
    "forward_sign": ("s -= L[a * p + c] * z[c];", "s += L[a * p + c] * z[c];"),
    "backward_transposed": ("s -= L[c * p + a] * z[c];", "s -= L[a * p + c] * z[c];"),
    "gram_operand": ("s += X[i * k + a] * X[i * k + b];", "s += X[i * k + a] * X[i * k + a];"),
    "objective_dropped_term": ("wh += W[i * k + r] * Ht[j * k + r];",
                               "wh += W[i * k + r] * Ht[j * k + r] * (r > 0);"),
    "mm_wrong_operand": ("s += (double)A[i * lda + j] * F[i * k + r];",
                         "s += (double)A[i * lda + j] * F[i * k + 0];"),
    "csr_objective_dropped_term": ("si += d * d - wh * wh;", "si += d * d;"),
    "infeasible_sign": ("int inf = usable[i] && ((F[i] && x[i] < 0.0) || (!F[i] && y[i] < 0.0));",
                        "int inf = usable[i] && ((F[i] && x[i] < 0.0) || (!F[i] && y[i] > 0.0));"),
    "h_update_wrong_gram": ("oracle_gram(W, m, k, G);", "oracle_gram(Ht, n, k, G);"),
    "mu_dropped_factor": ("x[j] = x[j] * R[r * k + j] / den[j];", "x[j] = R[r * k + j] / den[j];"),
    "mu_wrong_gram_index": ("d += x[l] * G[l * k + j];", "d += x[l] * G[l * k + l];"),
    "hals_dropped_new_values": ("num -= G[l * k + i] * x[l];", "num -= G[l * k + i] * (l < i ? 0.0 : x[l]);"),
    "pgrad_projection_sign": ("const double pj = x[j] > 0.0 ? gj : (gj < 0.0 ? gj : 0.0);",
                              "const double pj = x[j] > 0.0 ? gj : (gj > 0.0 ? gj : 0.0);"),
    "hals_no_projection": ("x[i] = (num > 0.0 ? num : 0.0) / gii;", "x[i] = num / gii;"),
    # BPP's backup rule: alpha must be refilled whenever the infeasible count
    # reaches a new low, and the single exchange takes the largest index.
    "bpp_alpha_not_reset": ("beta = nv;\n            alpha = 3;", "beta = nv;"),
    "bpp_backup_smallest_index": ("vmax = i;", "if (vmax < 0)\n                    vmax = i;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(oracle.SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    path = os.path.join(tmp_path, "mutant.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    lib = oracle.compile_source(path, os.path.join(tmp_path, f"lib_{name}.so"))
    orc = oracle.Oracle(lib)
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(orc)
        except Exception as exc:  # noqa: BLE001 - any failure counts as caught
            caught.append((pin.__name__, type(exc).__name__))
    assert caught, f"mutant {name} passed every pin"
