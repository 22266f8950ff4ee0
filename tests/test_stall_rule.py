"""The stall test behind the mixed form's precision escalation (hbsd_res_stalled, host only).

The mixed form switches its double-float products (and then its Gram and update) to FP64 when the
best Res_max has not halved over the last 10 outer iterations once it has been below 1e4 tol, or
over the last 30 at any level.  Pinned here on the oracle's own FP64 trajectories, which converge
and must never trip it, and on the shapes of the two situations it separates: a floor of the
residual (what ~48-bit products produce on strongly cancelling problems) and the plateaus of a
cluster cut by the block edge.
"""
import json
import os

import numpy as np
import pytest

from paper_1308_2445_gb300 import hbsd

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = 1e-8


def fires(hist, mark=0):
    return hbsd.res_stalled(hist, mark, 10, 1e4 * TOL) or hbsd.res_stalled(hist, mark, 30, 1e300)


@pytest.mark.parametrize("name", ["medium_seed1", "medium_m0_21_seed1", "medium_nonlocal_seed1", "large_seed1"])
def test_quiet_on_the_oracle_trajectories(name):
    with open(os.path.join(HERE, "golden", name + ".json")) as f:
        h = json.load(f)["res_history"]
    assert not any(fires(h[:k]) for k in range(1, len(h) + 1))


def test_a_ten_iteration_window_at_every_level_would_trip_on_a_cluster_plateau():
    # why the 10-iteration window carries a level condition: the 32^3 trajectory at m0 = 7
    # (the 64th eigenvalue inside a 24-fold shell) idles near 1e-2 for a while
    with open(os.path.join(HERE, "golden", "medium_seed1.json")) as f:
        h = json.load(f)["res_history"]
    first = next(k for k in range(1, len(h) + 1) if hbsd.res_stalled(h[:k], 0, 10, 1e300))
    assert 20 < first < 40 and h[first - 1] > 1e-3


def test_fires_within_ten_iterations_of_a_residual_floor():
    rng = np.random.default_rng(3)
    descent = [0.7 * 0.6 ** i for i in range(25)]                 # down to ~2e-6
    floor = list(10 ** rng.uniform(-6.0, -5.1, size=20))          # stuck between 1e-6 and 8e-6
    h = descent + floor
    first = next(k for k in range(1, len(h) + 1) if fires(h[:k]))
    assert len(descent) < first <= len(descent) + 11
    assert not any(fires(h[:k]) for k in range(1, len(descent) + 1))


def test_fires_on_a_thirty_iteration_plateau_at_any_level():
    h = [1.0, 0.5, 0.2, 0.1, 0.05] + [0.04 + 0.01 * ((i * 7) % 3) for i in range(31)]
    first = next(k for k in range(1, len(h) + 1) if fires(h[:k]))
    assert first == 5 + 30   # as soon as the last 30 entries all lie on the plateau


def test_counts_the_window_from_the_last_switch():
    h = [1.0, 0.5, 0.2] + [1e-5] * 12                              # a floor below 1e4 tol
    assert fires(h)
    assert not fires(h, mark=len(h) - 1)                           # just switched: wait a window
    assert not fires(h + [1e-5] * 9, mark=len(h) - 1)
    assert fires(h + [1e-5] * 10, mark=len(h) - 1)


def test_argument_errors():
    with pytest.raises(hbsd.HbsdError):
        hbsd.res_stalled([1.0, 0.5], 3, 10, 1.0)                   # mark past the end
    with pytest.raises(hbsd.HbsdError):
        hbsd.res_stalled([1.0, 0.5], 0, 0, 1.0)                    # empty window
    assert hbsd.res_stalled([], 0, 10, 1.0) is False
