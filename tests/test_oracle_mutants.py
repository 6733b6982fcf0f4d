"""The oracle's pins are strong enough: each plausible mistake planted in a copy of
oracle.c (a dropped term, a wrong sign, an off-by-one index, a swapped operand) makes at
least one pin fail.  Mutants are built from text substitutions into a temporary copy of the
source, compiled with the oracle's own gcc command, and never touch the real oracle."""
import importlib
import os
import subprocess

import numpy as np
import pytest

import oracle as O

from test_oracle_pins import (GOLDEN_FILES, U, _mp_cholesky_r, _planted_q0, _rand_upper,
                              _read_golden)

MUTANTS = {
    "tau_sign": ("*tau = (beta - a) / beta;", "*tau = (a - beta) / beta;"),
    "v_scale_multiplies": ("x[i * incx] = x[i * incx] / d;", "x[i * incx] = x[i * incx] * d;"),
    "norm_drops_scale": ("return s * sqrt(q);", "return sqrt(q);"),
    "beta_unstable_sign": ("double beta = (a >= 0.0) ? -r : r;",
                           "double beta = (a >= 0.0) ? r : -r;"),
    "update_pivot_sign": ("y[j] = y[j] - tw;", "y[j] = y[j] + tw;"),
    "update_skips_first_row": ("for (int64_t i = j + 1; i < m; ++i) y[i] = fma(-tw",
                               "for (int64_t i = j + 2; i < m; ++i) y[i] = fma(-tw"),
    "dot_skips_first_row": ("for (int64_t i = j + 1; i < m; ++i) w = fma(v[i], y[i], w);",
                            "for (int64_t i = j + 2; i < m; ++i) w = fma(v[i], y[i], w);"),
    "trailing_skips_next_column": ("for (int64_t k = j + 1; k < a->n; ++k)",
                                   "for (int64_t k = j + 2; k < a->n; ++k)"),
    "signfix_inverted": ("if (AT(R, ldr, k, k) < 0.0)", "if (AT(R, ldr, k, k) > 0.0)"),
    "op_drops_R1_term": ("double w = AT(R1, ld1, j, k);", "double w = 0.0;"),
    "op_dot_short_range": ("for (int64_t i = 0; i <= j; ++i) w = fma(AT(R2, ld2, i, j)",
                           "for (int64_t i = 0; i < j; ++i) w = fma(AT(R2, ld2, i, j)"),
    "op_update_short_range": ("for (int64_t i = 0; i <= j; ++i)\n                    AT(R2, ld2, i, k)",
                              "for (int64_t i = 0; i < j; ++i)\n                    AT(R2, ld2, i, k)"),
    "op_transposed_R2": ("fma(AT(R2, ld2, i, j), AT(R2, ld2, i, k), w)",
                         "fma(AT(R2, ld2, j, i), AT(R2, ld2, i, k), w)"),
    "op_reflector_too_short": ("oracle_reflector(j + 2, &AT(R1, ld1, j, j)",
                               "oracle_reflector(j + 1, &AT(R1, ld1, j, j)"),
    "tile_padding_dropped": ("int64_t h = rows < n ? n : rows;", "int64_t h = rows;"),
    "dot2_drops_product_error": ("c += pe + se;", "c += se;"),
    "cholesky_drops_square": ("for (int64_t i = 0; i < k; ++i) d -= G[i + k * n] * G[i + k * n];",
                              "for (int64_t i = 0; i < k; ++i) d -= G[i + k * n];"),
    "residual_drops_last_row": ("int64_t len = (k < l ? k : l) + 1;",
                                "int64_t len = (k < l ? k : l);"),
    "q_reflectors_in_forward_order": ("for (int64_t j = k; j >= 0; --j) {",
                                      "for (int64_t j = 0; j <= k; ++j) {"),
    "q_skips_first_reflector": ("for (int64_t j = k; j >= 0; --j) {",
                                "for (int64_t j = k; j > 0; --j) {"),
    "q_column_not_flipped": ("AT(Q, ldq, i, k) = -AT(Q, ldq, i, k);",
                             "AT(Q, ldq, i, k) = AT(Q, ldq, i, k);"),
    "q_wrong_identity_column": ("q[i] = (i == k) ? 1.0 : 0.0;", "q[i] = (i == 0) ? 1.0 : 0.0;"),
    "q_dot_drops_pivot_entry": ("double s = q[j];", "double s = 0.0;"),
}


def _pins_pass(lib) -> bool:
    """A compact copy of the pin suite run against a (possibly mutated) library."""
    try:
        for path in GOLDEN_FILES:
            A, Rg = _read_golden(path)
            tol = 16 * U * max(1.0, np.abs(A).max()) * A.shape[0]
            for R in (O.householder_r(A, lib=lib), O.tsqr_r(A, b=1, tree="binary", lib=lib),
                      O.tsqr_r(A, b=2, tree="flat", lib=lib)):
                if not np.allclose(R, Rg, rtol=0, atol=tol):
                    return False
        rng = np.random.default_rng(5)
        R0 = _rand_upper(rng, 8, 100.0)
        Q0 = _planted_q0(rng, 120, 8)
        A = Q0 @ R0
        kap = np.linalg.cond(R0)
        for R in (O.householder_r(A, lib=lib), O.tsqr_r(A, b=16, tree="binary", lib=lib)):
            if not O.rel_err(R, R0) <= 50 * kap * U:
                return False
        # the thin Q factor: planted, and A = Q R with orthonormal columns
        Q, Rq = O.householder_qr(A, lib=lib)
        if not (O.rel_err(Rq, R0) <= 50 * kap * U and O.rel_err(Q, Q0) <= 50 * kap * U):
            return False
        G = rng.standard_normal((60, 5))
        Qg, Rg = O.householder_qr(G, lib=lib)
        if not (np.abs(Qg.T @ Qg - np.eye(5)).max() <= 300 * U
                and np.linalg.norm(G - Qg @ Rg) <= 300 * U * np.linalg.norm(G)):
            return False
        A = np.array([[1.0, 2.0], [1e-9, 3.0], [0.0, 4.0], [1e-12, -1.0]])
        if not O.rel_err(O.householder_r(A, lib=lib), _mp_cholesky_r(A)) <= 50 * np.linalg.cond(A) * U:
            return False
        # the operator against a dense QR of the stack
        R1, R2 = _rand_upper(rng, 6), _rand_upper(rng, 6)
        Rop = O.sign_fix(O.qr_uppers(R1, R2, lib=lib)[0], lib=lib)
        Rl = np.linalg.qr(np.vstack([R1, R2]), mode="r")
        Rl = Rl * np.sign(np.diag(Rl))[:, None]
        if not O.rel_err(Rop, Rl) <= 1e-13:
            return False
        # long-double Cholesky and the compensated checker
        B = rng.standard_normal((30, 4))
        if not O.rel_err(O.cholesky_r_ld(B, lib=lib), _mp_cholesky_r(B)) <= 1e-12:
            return False
        C = np.array([[1e16, 1.0], [1.0, 1.0], [-1e16, 1.0]])
        if O.gram_dot2(C, lib=lib)[0, 1] != 1.0:
            return False
        t = 2.0 ** -30
        D = np.array([[1 + t, 1 + t], [1.0, -(1 + 2 * t)]])  # exact x.y = 2^-60
        if O.gram_dot2(D, lib=lib)[0, 1] != 2.0 ** -60:
            return False
        Rb = O.householder_r(B, lib=lib)
        if not O.gram_residual(B, Rb, lib=lib) <= 1e-15:
            return False
        Rbad = Rb.copy()
        Rbad[3, 3] *= 1.0 + 1e-10
        if not O.gram_residual(B, Rbad, lib=lib) > 1e-12:
            return False
        return True
    except (np.linalg.LinAlgError, RuntimeError, FloatingPointError, ValueError):
        return False


def test_unmutated_oracle_passes_the_compact_pins(oracle):
    assert _pins_pass(None)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    src = open(O._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    path = tmp_path / "oracle_mutant.c"
    path.write_text(src.replace(old, new))
    out = str(tmp_path / f"lib_{name}.so")
    subprocess.run(O.compile_command(str(path), out), check=True)
    lib = O.load_variant(out)
    with np.errstate(all="ignore"):
        assert not _pins_pass(lib), f"mutant {name} survived the pins"
