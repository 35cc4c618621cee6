"""Host logic of the warm-start study on the CPU: the converged-mean criterion
(relative L2 change of the running mean of hub-plane u_x over one window) and
the window-error helpers, on synthetic window means."""
import numpy as np
import pytest

from paper_2402_13171_gb300 import surrogate as S


class _Windows:
    """Stands in for WindowMeans: a list of window means and their end steps."""

    def __init__(self, means, window=1000):
        self.means = [np.asarray(m, dtype=float) for m in means]
        self.ends = [window * (k + 1) for k in range(len(self.means))]


def test_running_mean_change_closed_forms():
    a, b = np.array([1.0, 2.0, 2.0]), np.array([1.5, 2.0, 3.0])
    w = _Windows([a, b, b, b])
    ch = S.running_mean_changes(w)
    assert [e for e, _ in ch] == [2000, 3000, 4000]
    # R_1 = a, R_2 = (a + b)/2: change |b - a| / |a + b|
    assert ch[0][1] == pytest.approx(np.linalg.norm(b - a) / np.linalg.norm(a + b), rel=1e-14)
    # R_k = (a + (k-1) b)/k: R_k - R_(k-1) = (b - a)/(k (k-1))
    for k, (_, c) in zip((3, 4), ch[1:]):
        r = (a + (k - 1) * b) / k
        assert c == pytest.approx(np.linalg.norm(b - a) / (k * (k - 1)) / np.linalg.norm(r), rel=1e-13)


def test_running_mean_settles_on_constant_and_decaying_transients():
    ref = np.linspace(0.5, 1.0, 50)
    assert S.running_mean_settle_step(_Windows([ref] * 5)) == 2000     # no change from the second window on
    # a transient decaying by half per window settles later than a faster one
    slow = _Windows([ref * (1 + 0.3 * 0.5 ** k) for k in range(40)])
    fast = _Windows([ref * (1 + 0.3 * 0.1 ** k) for k in range(40)])
    ts, tf = S.running_mean_settle_step(slow), S.running_mean_settle_step(fast)
    assert tf is not None and ts is not None and tf < ts
    assert S.running_mean_settle_step(_Windows([ref, 2 * ref])) is None   # never within 1e-3
    # the reference-based helpers agree on a run that sits at the reference
    assert S.settle_step(_Windows([ref * 1.5, ref]), ref, 1e-12) == 2000
    np.testing.assert_allclose(S.window_errors(_Windows([ref * 1.5, ref]), ref), [0.5, 0.0], atol=1e-15)
