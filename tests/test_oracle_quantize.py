"""Pins for oracle.quantize: error within half a step, exact endpoints, monotonicity, and the
bit budget."""
import numpy as np

from oracle import quantize as oq


def test_quantize_error_and_endpoints():
    rng = np.random.default_rng(0)
    s = np.concatenate([[-1.0, 1.0, 0.0], rng.uniform(-1, 1, 1000)])
    o = np.concatenate([[-40.0, 300.0], rng.uniform(-40, 300, 1001)])
    for bs, bo in ((5, 7), (3, 4), (12, 12)):
        qs, qo, sh, oh, lo, hi = oq.quantize(s, o, bs, bo)
        assert lo == -40.0 and hi == 300.0
        assert np.all(np.abs(sh - s) <= 1.0 / ((1 << bs) - 1) + 1e-12)
        assert np.all(np.abs(oh - o) <= 0.5 * (hi - lo) / ((1 << bo) - 1) + 1e-9)
        assert qs[0] == 0 and qs[1] == (1 << bs) - 1 and sh[0] == -1.0 and sh[1] == 1.0
        assert qo[0] == 0 and qo[1] == (1 << bo) - 1 and oh[0] == lo and oh[1] == hi
        order = np.argsort(s, kind="stable")
        assert np.all(np.diff(qs[order]) >= 0)
        order = np.argsort(o, kind="stable")
        assert np.all(np.diff(qo[order]) >= 0)


def test_quantize_constant_brightness_and_budget():
    qs, qo, sh, oh, lo, hi = oq.quantize(np.zeros(5), np.full(5, 77.0))
    assert np.all(qo == 0) and np.all(oh == 77.0) and lo == hi == 77.0
    # 5 bits at s = 0: (0 + 1) / 2 * 31 = 15.5 rounds half to even -> 16
    assert np.all(qs == 16)
    assert oq.bits_per_range(64009) == 16 + 3 + 5 + 7
