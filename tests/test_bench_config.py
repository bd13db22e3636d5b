"""Host logic of bench.py (no GPU): both arms name a workload with the same
config, the batches of a step cover every right-hand side once, and the L2
statement matches the bytes a batch holds."""
import argparse
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _workload(name, **kw):
    a = argparse.Namespace(workload=name, precision=kw.get('precision'), lattice=kw.get('lattice'),
                           rhs=kw.get('rhs', 0), batch=kw.get('batch', 0))
    return bench.workload(a)


@pytest.mark.parametrize('name', sorted(bench.WORKLOADS))
def test_both_arms_name_the_workload_alike(name):
    W = _workload(name)
    ours = bench.config_of(W, W['nsrc'], 'single process')
    ref = bench.config_of(_workload(name), W['nsrc'], 'single process')
    assert ours == ref
    assert set(ours) >= {'workload', 'lattice', 'L5', 'rhs_per_step', 'action', 'gauge', 'precision', 'l2'}


@pytest.mark.parametrize('name,batch,nbatches', [('16x48', 12, 1), ('24x64', 24, 1), ('48x64', 3, 4), ('4x8', 1, 1)])
def test_batches_cover_every_source_once(name, batch, nbatches):
    W = _workload(name)
    n = W['nsrc']
    chunks = [list(range(i, min(i + W['batch'], n))) for i in range(0, n, W['batch'])]
    assert W['batch'] == batch and len(chunks) == nbatches
    assert sorted(k for c in chunks for k in c) == list(range(n))
    assert len(W['masses']) == n


def test_l2_statement_follows_the_batch_bytes():
    big = bench.config_of(_workload('16x48'), 12, 'single process')['l2']
    small = bench.config_of(_workload('4x8'), 1, 'single process')['l2']
    assert big.startswith('inputs larger than L2') and '4.42 GB' in big
    assert small.startswith('inputs fit in L2')


def test_batch_option_overrides_the_workload_default():
    W = _workload('48x64', batch=2)
    assert W['batch'] == 2 and W['nsrc'] == 12
    W = _workload('16x48', rhs=5)
    assert W['batch'] == 5 and W['masses'] == [0.0158] * 5


def test_solver_flop_count():
    # 4 hops x 1320 + 2 A^-1 x 48 L5 + 6 x 72 (B, A) + 240 (vector updates)
    assert bench.cgnr_flops_per_unit_iteration(12) == 5280 + 1152 + 432 + 240
    # one iteration of one RHS on 16^3 x 48 (98,304 half-lattice sites), L5 = 12, in one second
    t = bench.solver_tflops(98304, 12, [1], 1.0)
    assert abs(t - 7104 * 98304 * 12 / 1e12) < 1e-15
