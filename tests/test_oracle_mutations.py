"""Plants plausible mistakes in a copy of the oracle (on the CPU) and checks
that the pins in test_oracle_pins catch every one of them.  Each mutation is a
dropped term, a wrong sign, a wrong index, a transposed operand or a wrong
constant in one oracle function."""
import os
import subprocess

import pytest

import oracle
import tests.test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "perm_oracle.c")

MUTATIONS = {
    "nw_half_constant": ("x[i] = (ld)a[i * n + (n - 1)] - rowsum / 2;", "x[i] = (ld)a[i * n + (n - 1)] - rowsum / 3;"),
    "nw_last_column_index": ("x[i] = (ld)a[i * n + (n - 1)] - rowsum / 2;", "x[i] = (ld)a[i * n + (n - 2 + (n < 2))] - rowsum / 2;"),
    "nw_step_sign": ("ld s = ((Gg >> j) & 1ull) ? 1.0L : -1.0L;", "ld s = ((Gg >> j) & 1ull) ? -1.0L : 1.0L;"),
    "nw_term_sign": ("if (g & 1ull) p -= prod; else p += prod;\n        pabs", "if (g & 1ull) p += prod; else p -= prod;\n        pabs"),
    "nw_update_transposed": ("if (a[i * n + j] != 0.0) x[i] += s * (ld)a[i * n + j];", "if (a[j * n + i] != 0.0) x[i] += s * (ld)a[j * n + i];"),
    "nw_no_start_vector": ("for (int i = 0; i < n; ++i) x[i] += (ld)a[i * n + j];", "for (int i = 0; i < n; ++i) x[i] += 0 * (ld)a[i * n + j];"),
    "nw_gray_is_binary": ("uint64_t G = g_lo ^ (g_lo >> 1);\n    for (int j = 0; j < n - 1; ++j)\n        if ((G >> j) & 1ull)\n            for (int i = 0; i < n; ++i) x[i] += (ld)a",
                          "uint64_t G = g_lo;\n    for (int j = 0; j < n - 1; ++j)\n        if ((G >> j) & 1ull)\n            for (int i = 0; i < n; ++i) x[i] += (ld)a"),
    "nw_final_factor": ("ld f = (ld)(4 * (n % 2) - 2);", "ld f = (ld)(4 * (n % 2) - 1);"),
    "ryser_subset_sign": ("if (__builtin_popcountll(S) & 1) total -= prod; else total += prod;", "if (__builtin_popcountll(S) & 1) total += prod; else total -= prod;"),
    "ryser_missing_outer_sign": ("if (n & 1) total = (u128)0 - total;\n    u128_store(total, lo, hi);\n    return 0;\n}\n\n/* ---", "u128_store(total, lo, hi);\n    return 0;\n}\n\n/* ---"),
    "ryser_drops_last_column": ("            for (int j = 0; j < n; ++j)\n                if ((S >> j) & 1ull) rowsum", "            for (int j = 0; j < n - 1; ++j)\n                if ((S >> j) & 1ull) rowsum"),
    "ryser_gray_direction": ("int added = (int)((Gk >> j) & 1ull);", "int added = (int)((Gp >> j) & 1ull);"),
    "brute_reuses_columns": ("        brute_u128_rec(n, a, i + 1, used, prod * u128_from_i64(a[i * n + c]), acc);\n        used[c] = 0;",
                             "        brute_u128_rec(n, a, i + 1, used, prod * u128_from_i64(a[i * n + c]), acc);"),
    "brute_ld_wrong_index": ("brute_ld_rec(n, a, i + 1, used, prod * (ld)a[i * n + c], acc);", "brute_ld_rec(n, a, i + 1, used, prod * (ld)a[c * n + c], acc);"),
    "nw2_shift_sign": ("x2[i] = 2 * u128_from_i64(a[i * n + (n - 1)]) - rowsum;", "x2[i] = 2 * u128_from_i64(a[i * n + (n - 1)]) + rowsum;"),
    "band_no_preset_past_end": ("                if (!col_exists(n, i + 1 + w)) u |= 1 << (W - 1);\n                nxt[u] += cur[s] * v;", "                nxt[u] += cur[s] * v;"),
    "band_wrong_window": ("                int c = i - w + k;\n                if (!col_exists(n, c)) continue;\n                ld v", "                int c = i - w + k + 1;\n                if (!col_exists(n, c)) continue;\n                ld v"),
    "rowdp_reuses_columns": ("if (!ROWDP_NZ(r, j) || ((taken >> j) & 1ull)) continue;", "if (!ROWDP_NZ(r, j)) continue;"),
    "rowdp_forgets_taken": ("const uint64_t t = (taken | (1ull << j)) & reach[k + 1];", "const uint64_t t = (1ull << j) & reach[k + 1];"),
    "rowdp_weight_transposed": ("if (is_int) nxt.iv[g] += cur.iv[h] * u128_from_i64(ai[r * n + j]);", "if (is_int) nxt.iv[g] += cur.iv[h] * u128_from_i64(ai[j * n + r]);"),
    "rowdp_ld_drops_weight": ("else nxt.fv[g] += cur.fv[h] * (ld)af[r * n + j];", "else nxt.fv[g] += cur.fv[h];"),
    "mt_chunk_short": ("uint64_t lo = jb->g_lo + c * jb->chunk, hi = lo + jb->chunk;", "uint64_t lo = jb->g_lo + c * jb->chunk, hi = lo + jb->chunk - (c == 3);"),
}

PIN_TESTS = [
    lambda: [pins.test_brute_closed_forms(n) for n in range(1, 8)],
    pins.test_brute_triangular_and_scaled_permutation,
    pins.test_brute_small_by_hand,
    lambda: [pins.test_ryser_matches_brute_force(n) for n in range(1, 8)],
    lambda: pins.test_ryser_closed_forms(10),
    lambda: [pins.test_ryser_gray_matches_ryser(n) for n in range(1, 10)],
    lambda: [pins.test_nw_matches_brute_force(n) for n in range(1, 8)],
    lambda: pins.test_nw_closed_forms(12),
    pins.test_nw_depends_on_the_last_column_entry,
    pins.test_nw_range_additivity_and_start_vector,
    lambda: pins.test_nw_range_threads_do_not_change_result(5),
    lambda: [pins.test_nw2_full_range_is_scaled_permanent(n) for n in range(1, 10)],
    pins.test_nw2_additivity_and_threads,
    lambda: [pins.test_band_dp_matches_brute_force(n, w) for n in (3, 5, 8) for w in (1, 2, 3)],
    pins.test_band_dp_fibonacci_and_rejects_offband,
    pins.test_band_dp_matches_nw_on_band_sibling,
    lambda: [pins.test_rowdp_matches_brute_force_in_any_row_order(n) for n in (3, 5, 8)],
    pins.test_rowdp_closed_forms,
]


def _caught() -> bool:
    for t in PIN_TESTS:
        try:
            t()
        except (AssertionError, ValueError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation target not found: " + name
    mutated = src.replace(old, new, 1)
    assert mutated != src
    c = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-w", str(c), "-o", str(so)])
    with oracle.using_library(str(so)):
        assert _caught(), "planted mistake %r went unnoticed by the pins" % name


def test_unmutated_oracle_passes_the_same_pins():
    assert not _caught()
