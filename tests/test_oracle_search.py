"""Pins for the oracle's MWP-CWP evaluation and exhaustive argmin.

The paper names the MWP-CWP model (Sec. 2, Example 2) without printing its
formulas, so these pins are hand-worked examples, occupancy facts, model
invariants and brute force -- not values printed by the paper.
"""
import json
import os

import numpy as np

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
HW = W.HW_FIXED_DEFAULT


def const_program(metric_rows, grid_dims):
    """Program whose metrics do not depend on N or the configuration."""
    K = len(metric_rows)
    tab = np.zeros((K, 66, 8, 2, 2), np.float32)
    for k, mv in enumerate(metric_rows):
        tab[k, :, :, 0, 0] = np.asarray(mv, np.float32)[None, :]
        tab[k, :, :, 1, 0] = 1.0
    return dict(aN=np.zeros((K, 8), np.float32), bN=np.zeros((K, 8), np.float32),
                table=tab, grid_dims=np.asarray(grid_dims, np.int32), d=1)


def query(N, nsm, f, memld, bw, ddc, ddu, kid):
    q = np.array([[N, nsm, f, memld, bw, ddc, ddu, 0]], np.float32)
    q[0, 7] = np.array([kid], np.int32).view(np.float32)[0]
    return q


def test_hand_worked_examples():
    g = json.load(open(os.path.join(GOLD, "mwpcwp_worked.json")))
    for case in g["cases"]:
        prog = const_program([case["metrics"]], [case["grid_dims"]])
        qq = case["query"]
        q = query(qq["N"], qq["n_sm"], qq["f_ghz"], qq["mem_ld"], qq["bw_gbs"], qq["dd_coal"],
                  qq["dd_uncoal"], 0)
        ev = oracle.evaluate(prog, g["hw"], q)
        c = case["config_index"]
        assert tuple(W.CONFIGS[c]) == tuple(case["config"])
        assert ev["case"][0, c] == case["case"], case["name"]
        # the f32 query stores f_ghz=1.5 etc exactly; exec is exact arithmetic
        if "exec" in case:
            assert abs(ev["exec"][0, c] - case["exec"]) <= 1e-9 * case["exec"], (
                case["name"], ev["exec"][0, c])
        else:
            ref = eval(case["exec_formula"])
            assert abs(ev["exec"][0, c] - ref) <= case["exec_rel_tol"] * ref


def test_occupancy_limits():
    """Register and shared-memory limits decide residency (Example 1)."""
    q = query(4096, 100, 1.5, 400, 4000, 10, 10, 0)
    c1024 = [i for i, (a, b) in enumerate(W.CONFIGS) if a * b == 1024]
    # 64 regs x 1024 threads = 65536 registers: exactly one block fits
    ev = oracle.evaluate(const_program([[100, 10, 0, 1, 0, 128, 64, 0]], [2]), HW, q)
    assert np.isfinite(ev["exec"][0, c1024]).all()
    # 65 regs x 1024 threads exceeds the register file: not resident
    ev = oracle.evaluate(const_program([[100, 10, 0, 1, 0, 128, 65, 0]], [2]), HW, q)
    assert (ev["case"][0, c1024] == oracle.EV_INVALID).all()
    assert np.isinf(ev["exec"][0, c1024]).all()
    # shared memory above the SM's capacity: nothing resident anywhere
    ev = oracle.evaluate(const_program([[100, 10, 0, 1, 0, 128, 16, 60000]], [2]), HW, q)
    assert (ev["case"][0] == oracle.EV_INVALID).all()
    s = oracle.search(const_program([[100, 10, 0, 1, 0, 128, 16, 60000]], [2]), HW, q)
    assert s["argmin"][0] == -1 and s["status"][0] & oracle.QS_NO_VALID


def test_no_memory_instructions():
    q = query(2048, 100, 1.5, 400, 4000, 10, 10, 0)
    ev = oracle.evaluate(const_program([[50, 0, 0, 1, 3, 128, 32, 0]], [2]), HW, q)
    c = 42  # 16x16: B_active 8, blocks 128*128 -> rep = ceil(16384/800) = 21
    assert ev["case"][0, c] == 0
    assert ev["exec"][0, c] == 50.0 * 21


def test_pole_marks_configuration_invalid():
    prog = const_program([[100, 10, 0, 1, 0, 128, 32, 0]], [2])
    prog["table"][0, 5, 2, 1, 0] = -1.0      # denominator of metric 2 negative at config 5
    q = query(2048, 100, 1.5, 400, 4000, 10, 10, 0)
    ev = oracle.evaluate(prog, HW, q)
    assert ev["case"][0, 5] == oracle.EV_POLE
    s = oracle.search(prog, HW, q)
    assert s["status"][0] & oracle.QS_POLE and s["argmin"][0] >= 0


def test_bad_query():
    prog = const_program([[100, 10, 0, 1, 0, 128, 32, 0]], [2])
    for q in [query(2048, 100, 1.5, 400, 4000, 10, 10, 3),      # kernel id out of range
              query(np.nan, 100, 1.5, 400, 4000, 10, 10, 0),
              query(0.0, 100, 1.5, 400, 4000, 10, 10, 0)]:
        s = oracle.search(prog, HW, q)
        assert s["argmin"][0] == -1 and s["status"][0] & oracle.QS_BAD


def _synthetic(K=6, Q=300, seed=1):
    prog = W.synthetic_program(K, 3, seed)
    q = W.queries(Q, K, seed + 1)
    return prog, q


def test_brute_force_argmin_and_second():
    prog, q = _synthetic()
    ev = oracle.evaluate(prog, HW, q)
    s = oracle.search(prog, HW, q)
    for i in range(len(q)):
        e = ev["exec"][i]
        fin = np.isfinite(e)
        if not fin.any():
            assert s["argmin"][i] == -1
            continue
        order = sorted(range(66), key=lambda c: (e[c], c))
        assert s["argmin"][i] == order[0]
        assert s["best"][i] == e[order[0]]
        assert s["second"][i] == e[order[1]]


def test_tie_break_lowest_index():
    """(B0, B1) and (B1, B0) give identical 2-D grids; with constant metrics
    their exec cycles tie exactly and the lower canonical index wins."""
    prog = const_program([[100, 10, 0, 1, 0, 128, 32, 0]], [2])
    q = query(1 << 20, 100, 1.5, 400, 4000, 10, 10, 0)
    ev = oracle.evaluate(prog, HW, q)
    s = oracle.search(prog, HW, q)
    e = ev["exec"][0]
    best = s["argmin"][0]
    ties = [c for c in range(66) if e[c] == e[best]]
    assert best == min(ties)
    b0, b1 = W.CONFIGS[best]
    if b0 != b1:
        mirror = [c for c in range(66) if tuple(W.CONFIGS[c]) == (b1, b0)][0]
        assert mirror in ties


def test_case_selection_invariants():
    """MWP <= Nw and CWP <= Nw; case 1 exactly when both are capped at Nw;
    case 3 exactly when MWP > CWP and compute does not exceed memory
    cycles (the latter is checked through case 2's complement)."""
    prog, q = _synthetic(K=6, Q=1000, seed=3)
    ev = oracle.evaluate(prog, HW, q)
    ok = np.isin(ev["case"], [1, 2, 3])
    mwp, cwp, nw, cs = ev["mwp"][ok], ev["cwp"][ok], ev["nw"][ok], ev["case"][ok]
    assert ok.sum() > 10000
    assert (mwp <= nw).all() and (cwp <= nw).all()
    both = (mwp == nw) & (cwp == nw)
    assert (cs[both] == 1).all()
    assert (mwp[cs == 3] > cwp[cs == 3]).all()
    assert (cwp[(cs == 2) & ~both] >= 0).all()
    # where neither cap binds and CWP >= MWP the case is 2
    sel = (~both) & (cwp >= mwp)
    assert (cs[sel] == 2).all()


def test_synthetic_workload_exercises_all_cases():
    prog, q = _synthetic(K=8, Q=2000, seed=5)
    ev = oracle.evaluate(prog, HW, q)
    cases = set(np.unique(ev["case"]).tolist())
    assert {1, 2, 3}.issubset(cases), cases


def test_hand_worked_occupancy():
    """B_active and W_active (Sec. 2 Example 1) of the hand-worked cases, as
    written out in their steps."""
    g = json.load(open(os.path.join(GOLD, "mwpcwp_worked.json")))
    for case in g["cases"]:
        prog = const_program([case["metrics"]], [case["grid_dims"]])
        qq = case["query"]
        q = query(qq["N"], qq["n_sm"], qq["f_ghz"], qq["mem_ld"], qq["bw_gbs"], qq["dd_coal"],
                  qq["dd_uncoal"], 0)
        ev = oracle.evaluate(prog, g["hw"], q)
        c = case["config_index"]
        assert ev["bact"][0, c] == case["b_active"], case["name"]
        assert ev["nw"][0, c] == case["w_active"], case["name"]


def test_occupancy_invariants():
    """W_active = min(B_active wpb, W_max) wherever resident; B_active within
    B_max and W_max / wpb; 0 (not resident) exactly where exec is +inf for a
    non-pole configuration."""
    prog, q = _synthetic(K=4, Q=300, seed=11)
    ev = oracle.evaluate(prog, HW, q)
    T = W.CONFIGS[:, 0] * W.CONFIGS[:, 1]
    wpb = (T + 31) // 32
    ok = np.isin(ev["case"], [0, 1, 2, 3])
    b = ev["bact"]
    assert (b[ok] >= 1).all()
    res = ok
    assert (ev["nw"][res] == np.minimum(b * wpb[None, :], HW["w_max"])[res]).all()
    assert (b[res] <= HW["b_max"]).all() and (b * wpb[None, :] <= np.maximum(HW["w_max"], wpb))[res].all()
    inval = ev["case"] == oracle.EV_INVALID
    assert (b[inval] == 0).all() and np.isinf(ev["exec"][inval]).all()


def test_tiebreak_second_metric():
    """Step 5 with occupancy as the second metric: tie_rel = 0 chooses the
    lowest-index optimum among configurations of equal W_active (the plain
    search's choice for the mirrored ties of a constant program); every
    choice lies within (1 + tie_rel) of the best; a wider window never
    lowers the chosen W_active; with a window wide enough to hold every
    valid configuration the choice has the largest W_active of them all."""
    prog = const_program([[100, 10, 0, 1, 0, 128, 32, 0], [400, 4, 2, 3, 1, 256, 24, 64]], [2, 2])
    q = W.queries(300, 2, seed=12, n_log2=(6, 20))
    s = oracle.search(prog, HW, q)
    a0, ev = oracle.search_tiebreak(prog, HW, q, 0.0)
    assert (a0 == s["argmin"]).all()
    prev = ev["nw"][np.arange(len(q)), a0]
    rows = np.arange(len(q))
    for rel in (0.01, 0.1, 0.5):
        a, _ = oracle.search_tiebreak(prog, HW, q, rel)
        assert (ev["exec"][rows, a] <= s["best"] * (1 + rel)).all()
        nw = ev["nw"][rows, a]
        assert (nw >= prev).all()
        prev = nw
    a, _ = oracle.search_tiebreak(prog, HW, q, np.inf)
    valid = np.isfinite(ev["exec"])
    assert (ev["nw"][rows, a] == np.where(valid, ev["nw"], -1).max(axis=1)).all()


def test_error_pct_table_definition():
    """Error % of a chosen configuration (Sec. 5), row by row: the Table 3
    formula on the row's finite runtimes; degenerate rows."""
    inf = np.inf
    rt = np.full((5, 66), inf)
    rt[0, :3] = [3.0, 1.0, 2.0]          # choice 2: (2 - 1) / (3 - 1) = 50 %
    rt[1, :2] = [5.0, 5.0]               # W == B: 0
    rt[3, :2] = [1.0, 4.0]               # choice not run
    rt[4, 10] = 7.0                      # one runtime, chosen
    e = oracle.error_pct_table(rt, [2, 1, 0, 5, 10])
    assert e[0] == 50.0 and e[1] == 0.0 and np.isnan(e[2]) and np.isnan(e[3]) and e[4] == 0.0
    assert np.isnan(oracle.error_pct_table(rt[:1], [-1])[0])
