"""Plant plausible mistakes in copies of the oracle (on the CPU) and check that
the pins catch every one: a dropped term, a wrong index, a wrong sign, a divide
instead of the rounded 1/6 product, a reordered sum, a
truncating bf16 conversion, a lost boundary gradient, a wrong residual, a
correction sweep that drops rho, a truncating or unconverted bf16 residual path.
"""
import os

import pytest

import oracle
from oracle import build as obuild
from tests import oracle_pins

SRC = obuild.SRC

MUTATIONS = {
    "drop_k_plus_1": ("                s = s + A[LIN(i, j, k + 1)];\n"
                      "                B[LIN(i, j, k)] = s * ORACLE_SIXTH;",
                      "                B[LIN(i, j, k)] = s * ORACLE_SIXTH;"),
    "j_for_k_index": ("                s = s + A[LIN(i, j, k - 1)];\n"
                      "                s = s + A[LIN(i, j, k + 1)];\n"
                      "                B[LIN(i, j, k)] = s * ORACLE_SIXTH;",
                      "                s = s + A[LIN(i, j - 1, k)];\n"
                      "                s = s + A[LIN(i, j, k + 1)];\n"
                      "                B[LIN(i, j, k)] = s * ORACLE_SIXTH;"),
    "wrong_sign": ("                double s = A[LIN(i - 1, j, k)];\n"
                   "                s = s + A[LIN(i + 1, j, k)];",
                   "                double s = A[LIN(i - 1, j, k)];\n"
                   "                s = s - A[LIN(i + 1, j, k)];"),
    "divide_by_6": ("                B[LIN(i, j, k)] = s * ORACLE_SIXTH;",
                    "                B[LIN(i, j, k)] = s / 6.0;"),
    "k_terms_first": ("                double s = A[LIN(i - 1, j, k)];\n"
                      "                s = s + A[LIN(i + 1, j, k)];\n"
                      "                s = s + A[LIN(i, j - 1, k)];\n"
                      "                s = s + A[LIN(i, j + 1, k)];\n"
                      "                s = s + A[LIN(i, j, k - 1)];\n"
                      "                s = s + A[LIN(i, j, k + 1)];",
                      "                double s = A[LIN(i, j, k - 1)];\n"
                      "                s = s + A[LIN(i, j, k + 1)];\n"
                      "                s = s + A[LIN(i - 1, j, k)];\n"
                      "                s = s + A[LIN(i + 1, j, k)];\n"
                      "                s = s + A[LIN(i, j - 1, k)];\n"
                      "                s = s + A[LIN(i, j + 1, k)];"),
    "pairwise_sum": ("                double s = A[LIN(i - 1, j, k)];\n"
                     "                s = s + A[LIN(i + 1, j, k)];\n"
                     "                s = s + A[LIN(i, j - 1, k)];\n"
                     "                s = s + A[LIN(i, j + 1, k)];\n"
                     "                s = s + A[LIN(i, j, k - 1)];\n"
                     "                s = s + A[LIN(i, j, k + 1)];",
                     "                double s = (A[LIN(i - 1, j, k)] + A[LIN(i + 1, j, k)])\n"
                     "                    + ((A[LIN(i, j - 1, k)] + A[LIN(i, j + 1, k)])\n"
                     "                    + (A[LIN(i, j, k - 1)] + A[LIN(i, j, k + 1)]));"),
    "off_by_one_row_bound": ("        for (int j = 1; j <= ny; ++j)\n            for (int i = 1; i <= nx; ++i) {\n                double s",
                             "        for (int j = 1; j <= ny - 1; ++j)\n            for (int i = 1; i <= nx; ++i) {\n                double s"),
    "rows_for_planes_stride": ("                s = s + A[LIN(i, j - 1, k)];\n                s = s + A[LIN(i, j + 1, k)];\n                s = s + A[LIN(i, j, k - 1)];\n                s = s + A[LIN(i, j, k + 1)];\n                B[LIN(i, j, k)] = s * ORACLE_SIXTH;",
                               "                s = s + A[LIN(i, j, k - 1)];\n                s = s + A[LIN(i, j, k + 1)];\n                s = s + A[LIN(i, j - 1, k)];\n                s = s + A[LIN(i, j + 1, k)];\n                B[LIN(i, j, k)] = s * ORACLE_SIXTH;"),
    "bf16_truncate": ("    if (rest > 0x8000u || (rest == 0x8000u && (keep & 1u)))\n        keep += 1u;",
                      "    (void)rest;"),
    "grad_no_boundary_copy": ("                    if (bnd) grad[LIN(i, j, k)] += lam[LIN(i, j, k)];\n                }\n        /* interior",
                              "                    (void)bnd;\n                }\n        /* interior"),
    "grad_missing_sixth": ("                    double lam_sum = ORACLE_SIXTH * lam[LIN(i, j, k)];",
                           "                    double lam_sum = lam[LIN(i, j, k)];"),
    "residual_sign": ("                double r = s - six_u;", "                double r = six_u - s;"),
    "residual_no_accumulate": ("                u[x] = u[x] + ev;", "                (void)ev;"),
    "rhs_drops_rho_bf16": ("                    v = v + bf16_to_f32(rho[LIN(i, j, k)]);\n",
                           ""),
    "residual_bf16_truncate": ("                else                ((uint16_t *)rho)[x] = f32_to_bf16((float)r);",
                               "                else { float fr = (float)r; uint32_t ub; memcpy(&ub, &fr, 4);\n"
                               "                       ((uint16_t *)rho)[x] = (uint16_t)(ub >> 16); }"),
    "residual_bf16_widen_wrong": ("                else                ev = (double)bf16_to_f32(((const uint16_t *)e)[x]);",
                                  "                else                ev = (double)((const uint16_t *)e)[x];"),
    "rhs_drops_rho_f32": ("                    v = v + rho[LIN(i, j, k)];\n                    b[LIN(i, j, k)] = v * c;",
                          "                    b[LIN(i, j, k)] = v * c;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    # every planted mistake keeps all accesses in bounds, so it runs in-process
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {name}"
    mutant = src.replace(old, new, 1)
    path = os.path.join(tmp_path, "mutant.c")
    with open(path, "w") as f:
        f.write(mutant)
    lib = oracle.load(obuild.build(path, os.path.join(tmp_path, "libmutant.so")))
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught the planted mistake {name}"
