"""Stored values from outside this code: the paper's Table II and the published
SplitMix64 reference outputs (tests/golden/, each file cites its source)."""
import os

import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), 'golden')


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith('#')]


def table2():
    return {r[0]: dict(M5=float(r[1]), L5=int(r[2]), b5=float(r[3]), c5=float(r[4]), tgf=float(r[5]),
                       ml=float(r[6]), ms=float(r[7])) for r in _rows('table2_tuned_mdwf.txt')}


def test_splitmix64_matches_published_outputs():
    for r in _rows('splitmix64_reference.txt'):
        state, outs = int(r[0]), [int(v, 16) for v in r[1:]]
        assert [int(v) for v in synth.splitmix64(state, len(outs))] == outs


def test_table2_tuning_constraint_and_flow_time():
    """Every tuned action has b5 - c5 = 1 (the constraint of the tuning, under which
    the Moebius kernel is a rescaled Shamir kernel) and t_gf = 1."""
    t = table2()
    assert len(t) == 10
    for name, r in t.items():
        assert abs(r['b5'] - r['c5'] - 1.0) < 1e-12, name
        assert r['tgf'] == 1.0


def test_workloads_take_table2_actions():
    import bench
    t = table2()
    # 16^3 x 48: a15m310 as printed; 24^3 x 64: a12m310 with its light mass and 0.0102 (the
    # sea light-quark mass in the ensemble's name); 48^3 x 64: the a12m310 (M5, b5, c5) at
    # L5 = 8 with m_f = 0.0022, the a12m130 lattice shape (the paper's a12m130 row has L5 = 20)
    w, a = bench.WORKLOADS['16x48'], t['a15m310']
    assert (w['M5'], w['L5'], w['b5'], w['c5']) == (a['M5'], a['L5'], a['b5'], a['c5'])
    assert set(w['masses']) == {a['ml']}
    w, a = bench.WORKLOADS['24x64'], t['a12m310']
    assert (w['M5'], w['L5'], w['b5'], w['c5']) == (a['M5'], a['L5'], a['b5'], a['c5'])
    assert set(w['masses']) == {a['ml'], 0.0102}
    w = bench.WORKLOADS['48x64']
    assert (w['M5'], w['L5'], w['b5'], w['c5']) == (a['M5'], a['L5'], a['b5'], a['c5'])
    assert bench.WORKLOAD is bench.WORKLOADS['16x48']
    # serving mix: L5 = 12 and L5 = 8 take the a15m310 and a12m310 actions; the 32^3 x 96, L5 = 6
    # configuration keeps a15m310's (M5, b5, c5) rather than a09m310's (1.1, 1.25, 0.25)
    for l5, ens in ((12, 'a15m310'), (8, 'a12m310')):
        assert bench.SERVE_ACTIONS[l5] == (t[ens]['M5'], t[ens]['b5'], t[ens]['c5'])
    assert bench.SERVE_ACTIONS[6] == (t['a15m310']['M5'], t['a15m310']['b5'], t['a15m310']['c5'])
