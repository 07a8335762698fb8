"""Host logic of the studies' steady-state rule (reading R20): the batch is stepped in chunks of
at least one time unit of its smallest dt until every instance's monitored quantity changed by
less than rel x scale over the last chunk, a failed instance counting as done; a fake solver
stands in for the library (no GPU)."""
import numpy as np

from paper_2308_15407_gb300 import quadrature_study as qs


class FakeF:
    ACTIVE, FAILED_NONFINITE = 0, 2


class FakeSolver:
    """Instance i relaxes as G_i(t) = 1 - exp(-rate_i t); instance `fail` fails at t_fail."""

    def __init__(self, dts, rates, fail=None, t_fail=1e9):
        self.dt = list(dts)
        self.rates = np.asarray(rates, float)
        self.steps = 0
        self.calls = []
        self.fail, self.t_fail = fail, t_fail

    def step(self, n):
        self.calls.append(n)
        self.steps += n

    def value(self, i):
        return 1.0 - np.exp(-self.rates[i] * self.steps * self.dt[i])

    def status(self):
        st = np.zeros(len(self.dt), dtype=int)
        if self.fail is not None and self.steps * self.dt[self.fail] >= self.t_fail:
            st[self.fail] = FakeF.FAILED_NONFINITE
        return None, st, None


def test_chunks_cover_a_time_unit_of_the_smallest_dt_and_stop_when_steady():
    s = FakeSolver([1e-3, 2.5e-4], [1.0, 0.5])
    mon = lambda i: (np.array([s.value(i)]), 1.0)
    vals, change, steps, sec, dt, chunk = qs._step_until_steady(FakeF, s, 2, mon, cap_s=60.0, window=1.0, rel=1e-4)
    assert chunk == 4000 and all(c == 4000 for c in s.calls)
    assert np.all(change < 1e-4)
    # the slower instance decides: its change over one chunk (1 time unit) falls below 1e-4
    t = steps * 2.5e-4
    assert np.exp(-0.5 * t) * (np.exp(0.5) - 1) < 1e-4 <= np.exp(-0.5 * (t - 1)) * (np.exp(0.5) - 1)
    assert abs(vals[1][0] - (1 - np.exp(-0.5 * t))) < 1e-15


def test_failed_instance_counts_as_done():
    s = FakeSolver([1e-3, 1e-3], [1.0, 1e-9], fail=1, t_fail=3.0)
    mon = lambda i: (np.array([s.value(i)]), max(abs(s.value(i)), 1e-30))
    _, change, steps, _, _, _ = qs._step_until_steady(FakeF, s, 2, mon, cap_s=60.0, window=1.0, rel=1e-4)
    assert change[0] < 1e-4 and not change[1] < 1e-4      # stopped by the failure, not by its change
    assert steps * 1e-3 >= 3.0


def test_wall_clock_cap_ends_an_unsteady_batch():
    s = FakeSolver([1e-3], [1e-6])
    mon = lambda i: (np.array([s.value(i) + 1e-3 * (s.steps // 1000 % 2)]), 1.0)   # never settles
    _, change, steps, sec, _, _ = qs._step_until_steady(FakeF, s, 1, mon, cap_s=0.05, window=1.0, rel=1e-6)
    assert not change[0] < 1e-6 and steps > 0 and sec >= 0.05
