"""Hand-derived plans of the Section III naive strategy that fix the cost of a rewritten row.

Section III counts an original row as 2*nnz - 1 flops and a level as 2*sum(nnz) - rows.  For
a rewritten (rearranged) row the planner charges 2*|D'|, where D' is the row's dependency
set after substitution: its division is folded into the coefficients while rewriting, which
takes one flop off 2*nnz - 1 (Section IV, Table I discussion), and a row whose dependencies
all disappear costs nothing (same passage: no computation is left for rows rewritten to the
first level).

Every plan below was worked out by hand from those rules, the greedy prefix stop rule
(a row moves while cur + c <= avgLevelCost; the first row that does not fit makes its own
level the next target, holding its remaining rows at their original costs) and the fixed
average.  Case EQUALITY accepts a row at cur + c == avg; charging 2|D'| + 1 rejects it and
changes the plan.  Case OVER rejects a row at cur + c == avg + 1; charging 2|D'| - 1 accepts
it and changes the plan.  Case ZERO moves a chain onto level 0 with 2|D'| = 0 per row;
charging 2|D'| + 1 stops the chain before its last level.

Structure of EQUALITY and OVER: w "fat" rows f_0..f_{w-1} without dependencies (level 0,
cost 1 each), then a chain a_1..a_5 in rows w..w+4: a_1 reads f_0; a_k reads f_{k-1} and
a_{k-1}.  Levels 1..5 hold one chain row each: costs 3, 5, 5, 5, 5.
"""


def chain_deps(w: int) -> dict[int, list[int]]:
    deps = {i: [] for i in range(w)}
    deps[w] = [0]
    for k in range(2, 6):
        deps[w + k - 1] = [k - 1, w + k - 2]
    return deps


CASES = {
    # w = 103: level costs [103, 3, 5, 5, 5, 5], total 126 over 6 levels, avg 21.
    # Level 0 is not thin (103 >= 21); levels 1..5 are.  Target level 1, cur = 3.
    #   a_2: D' = {f0, f1}            |D'| = 2, c = 4,  cur = 7  <= 21 -> level 1
    #   a_3: D' = {f0, f1, f2}        |D'| = 3, c = 6,  cur = 13 <= 21 -> level 1
    #   a_4: D' = {f0, ..., f3}       |D'| = 4, c = 8,  cur = 21 <= 21 -> level 1 (equality)
    #   a_5: D' = {f0, ..., f4}       |D'| = 5, c = 10, cur = 31 >  21 -> stays, level 5 is the next target
    # (With 2|D'| + 1: a_4 gives 24 > 21, level 4 becomes the target and a_5, D' = {f3, f4, a_3},
    #  joins it at 5 + 7 = 12: a_4 and a_5 end on level 4.)
    "equality": {
        "w": 103,
        "deps": chain_deps(103),
        "avg": 21.0,
        "level_cost": [103, 3, 5, 5, 5, 5],
        "deps_after": {104: 2, 105: 3, 106: 4},
        "chain_target": [1, 1, 1, 1, 5],
        "chain_row_cost": [3, 4, 6, 8, 5],
        "levels_after": 3,
        "target_level_cost": {1: 21, 5: 5},
    },
    # w = 49: level costs [49, 3, 5, 5, 5, 5], total 72 over 6 levels, avg 12.  Target level 1, cur = 3.
    #   a_2: D' = {f0, f1}            c = 4, cur = 7  <= 12 -> level 1
    #   a_3: D' = {f0, f1, f2}        c = 6, cur = 13 >  12 -> stays; level 3 is the target, cur = 5
    #   a_4: D' = {f2, f3, a_2}       c = 6, cur = 11 <= 12 -> level 3 (a_2 sits on level 1, above the target)
    #   a_5: D' = {f2, f3, f4, a_2}   c = 8, cur = 19 >  12 -> stays; level 5 is the target
    # (With 2|D'| - 1: a_3 gives 11 <= 12 and joins level 1, a_4 gives 18 > 12 and becomes the target,
    #  a_5, D' = {f3, f4, a_3}, joins it at 5 + 5 = 10: the chain ends as 1, 1, 1, 4, 4.)
    "over": {
        "w": 49,
        "deps": chain_deps(49),
        "avg": 12.0,
        "level_cost": [49, 3, 5, 5, 5, 5],
        "deps_after": {50: 2, 52: 3},
        "chain_target": [1, 1, 3, 3, 5],
        "chain_row_cost": [3, 4, 5, 6, 5],
        "levels_after": 4,
        "target_level_cost": {1: 7, 3: 11, 5: 5},
    },
    # A chain c_0..c_3 (c_0 without dependencies, c_k reads c_{k-1}) and a level of three rows
    # that read c_3.  Level costs [1, 3, 3, 3, 9], total 19 over 5 levels, avg 3.8; levels 0..3
    # are thin.  Target level 0, cur = 1: every chain row loses all its dependencies (D' = {}),
    # costs 0 and moves to level 0.  (With 2|D'| + 1 the costs 1, 1, 1 bring cur to 2, 3, 4:
    # c_3 does not fit 3.8 and stays on level 3.)
    "zero": {
        "w": 0,
        "deps": {0: [], 1: [0], 2: [1], 3: [2], 4: [3], 5: [3], 6: [3]},
        "avg": 3.8,
        "level_cost": [1, 3, 3, 3, 9],
        "deps_after": {1: 0, 2: 0, 3: 0},
        "target": [0, 0, 0, 0, 4, 4, 4],
        "row_cost": [1, 0, 0, 0, 3, 3, 3],
        "levels_after": 2,
        "target_level_cost": {0: 1, 4: 9},
    },
}


def expected_target(case: dict) -> list[int]:
    if "target" in case:
        return list(case["target"])
    w = case["w"]
    return [0] * w + list(case["chain_target"])


def expected_row_cost(case: dict) -> list[int]:
    if "row_cost" in case:
        return list(case["row_cost"])
    w = case["w"]
    return [1] * w + list(case["chain_row_cost"])


def csr_arrays(case: dict):
    """(n, counts, flattened sorted columns) of a case's dependency structure."""
    deps = case["deps"]
    n = len(deps)
    counts = [len(deps[i]) for i in range(n)]
    cols = [c for i in range(n) for c in sorted(deps[i])]
    return n, counts, cols
