"""Pins of the oracle's g1 table (Sec. IV, Eq. 3: the middle bead's
mean-square displacement, averaged over chains and time origins) over
log-spaced lags j P^k: a ballistic trajectory with integer steps gives
g1 = |v|^2 dt^2 exactly; the number of origins of each lag has the closed
form floor(T / P^k) - j + 1; a random walk's table equals a vectorised
numpy average over the same origins.  No GPU."""
import numpy as np

import oracle


def test_ballistic_trajectory_exact():
    T, nch, P, K = 70, 5, 4, 3
    v = np.array([1.0, 2.0, 2.0])  # |v|^2 = 9
    traj = np.array([[np.array([ch, -ch, 3.0 * ch]) + t * v for ch in range(nch)]
                     for t in range(T + 1)])
    lags, g1, cnt, _ = oracle.g1_table(traj, P, K)
    assert list(lags) == [1, 2, 3, 4, 8, 12, 16, 32, 48]
    assert (g1 == 9.0 * lags.astype(float) ** 2).all()
    for q, lag in enumerate(lags):
        k = 0 if lag < P else (1 if lag < P * P else 2)
        pk, j = P ** k, lag // P ** k
        assert cnt[q] == max(T // pk - j + 1, 0)


def test_random_walk_matches_vectorised_average():
    rng = np.random.default_rng(5)
    T, nch, P, K = 90, 7, 3, 4
    traj = np.cumsum(rng.normal(size=(T + 1, nch, 3)), axis=0)
    lags, g1, cnt, sums = oracle.g1_table(traj, P, K)
    for q, lag in enumerate(lags):
        k = int(round(np.log(lag / (q % (P - 1) + 1)) / np.log(P)))
        pk = P ** k
        origins = np.arange(0, T - lag + 1, pk)
        assert cnt[q] == len(origins)
        d = traj[origins + lag] - traj[origins]
        ref = (d * d).sum(axis=2).mean() if len(origins) else 0.0
        assert abs(g1[q] - ref) <= 1e-12 * max(ref, 1.0)
    # an empty lag (longer than the run) reports zero with no origin
    lags2, g12, cnt2, _ = oracle.g1_table(traj[:5], 4, 3)
    assert (cnt2[lags2 > 4] == 0).all() and (g12[lags2 > 4] == 0).all()
