"""Planted mistakes in the oracle, on the CPU: each mutant of oracle.c below is
a plausible slip in one step of the method, and each must fail at least one of
the pins in test_oracle_pins.py.  A mutant runs in a child process (a broken
list update may crash it); a crash or a hang counts as caught, and the
unmodified source must pass the same battery, so a failure is the mutation's.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# name -> (text in oracle.c, replacement, what the slip breaks)
MUTANTS = {
    "tie_break_to_last": ("int32_t x = s.cfirst[c0];", "int32_t x = s.clast[c0];",
                          "the pick takes the highest id of the top class (Section 4.2 pick)"),
    "new_class_after_parent": (
        "s->cprev[d] = p; s->cnext[d] = c; s->cprev[c] = d;\n    if (p >= 0) s->cnext[p] = d; else s->chead = d;",
        "(void)p; s->cnext[d] = s->cnext[c]; s->cprev[d] = c; if (s->cnext[c] >= 0) s->cprev[s->cnext[c]] = d; "
        "s->cnext[c] = d;",
        "C ∩ N_x placed after C \\ N_x instead of before it (Observation 6.2)"),
    "neighbour_inserted_before_tail": ("vl_insert_after(&s, s.clast[d], y);", "vl_insert_before(&s, s.clast[d], y);",
                                       "the new class loses its id order"),
    "parent_is_leftmost": ("(p < 0 || pos[u] > pos[p])", "(p < 0 || pos[u] < pos[p])",
                           "p(v) = the earliest instead of the latest earlier neighbour (Section 5.2)"),
    "parent_not_excluded": ("u != p && !adjacent_sorted", "!adjacent_sorted",
                            "p itself counted as a violation"),
    "later_neighbours_tested": ("if (pos[u] < pos[v] && u != p", "if (u != p",
                                "LN_v replaced by all of N_v"),
    "adjacency_of_wrong_vertex": ("!adjacent_sorted(rp, col, p, u)", "!adjacent_sorted(rp, col, v, u)",
                                  "u tested against N(v) instead of N(p)"),
    "mcs_tie_to_highest_id": ("(a.label == b.label && a.v < b.v)", "(a.label == b.label && a.v > b.v)",
                              "MCS ties to the highest id (Section 5.1 with the lowest-id rule)"),
    "mcs_fewest_numbered": ("return a.label > b.label ||", "return a.label < b.label ||",
                            "MCS numbers a vertex with the fewest numbered neighbours"),
    "rank_sorted_descending": ("return (ka > kb) - (ka < kb);", "return (ka < kb) - (ka > kb);",
                               "multi-sweep neighbours taken in decreasing rank"),
}

BATTERY = r"""
import sys
sys.path[:0] = [{root!r}, {here!r}]
import oracle
oracle.use_library({lib!r})
import test_oracle_pins as P
checks = [
    (P.test_hand_c4, ()), (P.test_hand_c5, ()), (P.test_hand_path_and_diamond, ()),
    (P.test_order_min_id_tie_break, ()),
    (P.test_order_equals_explicit_labels, (50, 0.1)), (P.test_order_equals_explicit_labels, (120, 0.05)),
    (P.test_witness_is_canonical, (80, 0.1)), (P.test_parent_array_by_definition, ()),
    (P.test_peo_check_of_arbitrary_order, ()), (P.test_verdict_exhaustive_small, (5,)),
    (P.test_cycles_not_chordal, (6,)), (P.test_planted_cycle_and_closing_edges_not_chordal, ()),
    (P.test_mcs_order_equals_definition, (60, 0.1)), (P.test_mcs_hand_c4_and_clique, ()),
    (P.test_tiebreak_order_equals_explicit_labels, (60, 0.1)), (P.test_tiebreak_identity_and_relabelling, ()),
]
for fn, args in checks:
    try:
        fn(*args)
    except Exception as e:
        print("FAILED", fn.__name__, args, type(e).__name__)
        sys.exit(1)
print("ALL PASSED")
"""


def _build(tmp, name, text):
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(text)
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", c, "-o", so])
    return so


def _battery(so):
    code = BATTERY.format(root=ROOT, here=HERE, lib=so)
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    except subprocess.TimeoutExpired:
        return "hang"
    if r.returncode == 0:
        return "passed"
    return "failed: " + (r.stdout.strip().splitlines() or [f"exit {r.returncode}"])[-1]


@pytest.fixture(scope="module")
def source():
    with open(SRC) as f:
        return f.read()


def test_unmodified_source_passes_the_battery(source, tmp_path):
    assert _battery(_build(str(tmp_path), "unmodified", source)) == "passed"


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source, tmp_path):
    old, new, _ = MUTANTS[name]
    assert source.count(old) == 1, f"mutation site of {name} not found once in oracle.c"
    verdict = _battery(_build(str(tmp_path), name, source.replace(old, new)))
    assert verdict != "passed", f"mutant {name} ({MUTANTS[name][2]}) passed every pin"
