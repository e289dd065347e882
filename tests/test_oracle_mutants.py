"""The oracle's pins have teeth: plant plausible mistakes in a copy of the oracle (on the CPU)
and check that the pin suite rejects every mutant."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fciqmc_oracle.c")

# (name, original text, planted mistake)
MUTANTS = [
    ("philox_multiplier", "0xD2511F53u * (uint64_t)c0", "0xD2511F55u * (uint64_t)c0"),
    ("single_drops_exchange", "if (spin_of(j) == spin_of(i)) v = v - eri4(q, I, J, J, A);", ""),
    ("diag_drops_exchange", "if (spin_of(occ[x]) == spin_of(occ[y])) t = t - eri4(q, p, r, r, p);", ""),
    ("double_wrong_index", "v = v - eri4(q, spat_of(i), spat_of(b), spat_of(j), spat_of(a));",
     "v = v - eri4(q, spat_of(i), spat_of(j), spat_of(b), spat_of(a));"),
    ("parity_inclusive", "for (int m = lo + 1; m < hi; ++m)", "for (int m = lo; m < hi; ++m)"),
    ("pgen_drops_reverse_order", "info[4] = m_ba + m_ab;", "info[4] = m_ba + m_ba;"),
    ("singles_not_renormalised", "info[5] = (int64_t)mallow * (int64_t)nok;", "info[5] = (int64_t)mallow * (int64_t)n;"),
    ("spawn_sign", "return -(int64_t)sgn_c * sgn_h * nsp;", "return (int64_t)sgn_c * sgn_h * nsp;"),
    ("death_sign", "if (r >= 0.0) { nc = (int64_t)c - sc * nd;", "if (r >= 0.0) { nc = (int64_t)c + sc * nd;"),
    ("initiator_flag_and", "m.flag |= sp[y].flag;", "m.flag &= sp[y].flag;"),
    ("spin_rule_double", "if (si == sj && sa != si) continue;", "if (sa != si) continue;"),
    ("accept_single_offset_dropped", "uint64_t off = kind == 2 ? 0 : q->d53;", "uint64_t off = 0;"),
    ("accept_range_swapped", "uint64_t range = kind == 2 ? q->d53 : ((uint64_t)1 << 53) - q->d53;",
     "uint64_t range = kind == 1 ? q->d53 : ((uint64_t)1 << 53) - q->d53;"),
    ("rdm_half_dropped", "0.5 * cc * (double)(s1 * s2 * s3 * s4);", "cc * (double)(s1 * s2 * s3 * s4);"),
    ("rdm_spin_rule", "if ((p & 1) != (qq & 1) || (r & 1) != (s & 1)) continue;",
     "if ((p & 1) != (s & 1) || (r & 1) != (qq & 1)) continue;"),
    ("space_excitation_off_by_one", "if (exc > q->max_exc) return 0;", "if (exc >= q->max_exc) return 0;"),
    ("space_seniority_pairing", "if (det_bit(q, d, 2 * p) != det_bit(q, d, 2 * p + 1)) sen++;",
     "if (det_bit(q, d, p) != det_bit(q, d, p + q->n_orb)) sen++;"),
    ("space_frozen_inverted", "if (det_bit(q, q->froz_occ, k) && !det_bit(q, d, k)) return 0;",
     "if (det_bit(q, q->froz_occ, k) && det_bit(q, d, k)) return 0;"),
    ("space_check_skipped", "if (!in_space(q, child)) { *is_null = 1; return 0; }", ""),
    ("hphf_second_primitive_dropped", "if (!det_eq(q, xb, child)) g = g + oq_gen_prob(q, d, xb);", ""),
    ("hphf_pair_sign", "return (n_open(q, d) / 2) % 2 ? -1.0 : 1.0;", "return (n_open(q, d) / 2) % 2 ? 1.0 : -1.0;"),
    ("hphf_sqrt2_dropped", "if (a_open || b_open) return hab * SQRT2;", "if (a_open || b_open) return hab;"),
    ("hphf_diag_coupling_dropped", "if (!det_eq(q, a, ab)) v = v + pair_sign(q, a) * oq_hij(q, a, ab);", ""),
    ("hphf_projected_sqrt2", "if (q->hphf && n_open(q, d) > 0) h0 = h0 * SQRT2;", ""),
    ("choice_word_not_advanced", "*R = x & ((((unsigned __int128)1) << 75) - 1);", ""),
    ("choice_word_low_bits_dropped", " | (unsigned __int128)(r0 & 0x7FFu);", ";"),
    ("shift_update_sign", "q->shift = q->shift - q->c_shift * oq_log(ratio);",
     "q->shift = q->shift + q->c_shift * oq_log(ratio);"),
    ("gen_prob_double_orders", "return (q->p_double * (double)(m_ba + m_ab)) /", "return (q->p_double * (double)(m_ba + m_ba)) /"),
    ("clone_sign", "else { nc = (int64_t)c + sc * nd; clone_w += nd; }", "else { nc = (int64_t)c - sc * nd; clone_w += nd; }"),
    ("fingerprint_prime", "hsh = 1099511628211ull * hsh", "hsh = 1099511628213ull * hsh"),
    ("fingerprint_zero_based", "q->map1[occ[i - 1]] * (uint64_t)i;", "q->map1[occ[i - 1]] * (uint64_t)(i - 1);"),
    ("fingerprint_descending", "q->map1[occ[i - 1]] * (uint64_t)i;", "q->map1[occ[n - i]] * (uint64_t)i;"),
    ("fingerprint_map_key", "key[2] = {0x46434951u, 0x4D415031u}", "key[2] = {0x46434951u, 0x4D415032u}"),
    ("hybrid_attempts_floored", "        if (unit53(u) < (double)frac * ldexp(1.0, -q->frac_bits)) n++;\n", ""),
    ("hybrid_threshold_inverted", "int keep = unit53(u) < (double)ac / (double)q->occ_units;",
     "int keep = unit53(u) >= (double)ac / (double)q->occ_units;"),
    ("hybrid_spawn_unscaled", "    q->tau_s = q->tau * R;", "    q->tau_s = q->tau;"),
    ("hybrid_death_scaled", "double r = (q->tau * (q->hd[x] - q->shift)) * (double)ac;",
     "double r = (q->tau_s * (q->hd[x] - q->shift)) * (double)ac;"),
]

FAST_PINS = ("philox or fingerprint_is_algorithm1 or hybrid_one_step or hybrid_attempts or choice_digits or keeps_the_invariants or holds_the_population or own_log or second_quantisation or symmetry_and_spin or two_words and hamiltonian "
             "or pdouble or normalised or eq1 or initiator_rule or on_a_subset or functional_two_words "
             "or membership or outside_the_space or expectation_in_the_space "
             "or spin_flip or projection or probability_of_any_target or spin_coupled or numerator or stored_form")


@pytest.mark.slow
def test_every_planted_mistake_is_caught():
    src = open(SRC).read()
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")
    procs = {}
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        path_c = os.path.join(tmp, f"{name}.c")
        path_so = os.path.join(tmp, f"{name}.so")
        with open(path_c, "w") as f:
            f.write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", path_so, path_c, "-lm"])
        env = dict(os.environ, FCIQMC_ORACLE_LIB=path_so, OMP_NUM_THREADS="1")
        procs[name] = subprocess.Popen(
            [sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
             os.path.join(ROOT, "tests", "test_oracle_rdm.py"), os.path.join(ROOT, "tests", "test_oracle_space.py"),
             os.path.join(ROOT, "tests", "test_oracle_hphf.py"),
             os.path.join(ROOT, "tests", "test_oracle_invariants.py"),
             os.path.join(ROOT, "tests", "test_oracle_real.py"),
             "-x", "-q",
             "-p", "no:cacheprovider", "-k", FAST_PINS],
            env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, cwd=ROOT)
    survivors = []
    for name, p in procs.items():
        out, _ = p.communicate(timeout=600)
        if p.returncode == 0:
            survivors.append((name, out.decode()[-400:]))
    assert not survivors, survivors
