"""Symbolic check of the cycle schedule, without arithmetic (after the
paper's symbolic prototype of the task flow, Sec. 4): the phase list of
schedule.phases (the library's host schedule, compared with the oracle's in
test_host_logic) is replayed on per-level clocks only.

For every phase, every level whose state the phase reads must be defined at
the phase time T: at its step start, or inside a step whose predicted state
exists (linear interpolation); the paper's order may also take a finer
level one step past its predicted state (the extrapolation of its coarse
corrector).  Then: each level is updated 2^(theta - k) times per cycle (the
C(tau) of Sec. 2.2), the faces of each level are evaluated twice per step
(predictor and corrector), and every level ends the cycle at 2^theta with no
pending predicted state.
"""
import pytest

from paper_1704_01144_gb300 import schedule as S


def replay(theta, order):
    L = theta + 1
    tn, pred = [0] * L, [False] * L
    face_evals, updates = [0] * L, [0] * L

    def readable(j, T, extrapolate):
        if j < 0 or j >= L:
            return True  # no neighbours on that level
        d, span = T - tn[j], 1 << j
        if d == 0:
            return True
        return pred[j] and 0 < d <= (2 * span if extrapolate else span)

    for kind, lev, T in S.phases(theta, order):
        if kind == "B":
            # faces of level <= tau join cells of levels <= tau + 1, whose
            # gradients read neighbours up to level tau + 2
            for j in range(lev + 3):
                assert readable(j, T, False), (theta, order, kind, lev, T, j)
            for k in range(lev + 1):
                face_evals[k] += 1
                pred[k] = True
        elif kind in "EC":
            # faces of level k join cells of levels k, k + 1; gradients read
            # levels k - 1 .. k + 2
            for j in range(lev - 1, lev + 3):
                assert readable(j, T, kind == "C"), (theta, order, kind, lev, T, j)
            assert T == tn[lev] + (1 << lev) and pred[lev]
            face_evals[lev] += 1
            updates[lev] += 1
            if kind == "E":
                tn[lev], pred[lev] = T, False
        else:  # "I": the levels 0..lev end their steps at T
            for j in range(lev + 1):
                assert T == tn[j] + (1 << j) and pred[j], (theta, kind, lev, T, j)
                tn[j], pred[j] = T, False
    return tn, pred, face_evals, updates


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("theta", range(7))
def test_schedule_reads_only_defined_states(theta, order):
    tn, pred, face_evals, updates = replay(theta, order)
    for k in range(theta + 1):
        assert updates[k] == 2 ** (theta - k)          # C(tau) / |Omega(tau)|
        assert face_evals[k] == 2 * 2 ** (theta - k)   # predictor + corrector per step
    assert tn == [2 ** theta] * (theta + 1) and not any(pred)


def test_cost_of_a_cycle_matches_the_update_counts():
    """sum_k updates_k |Omega_k| is the cycle cost of Sec. 2.2."""
    counts = [5, 5, 10, 80]
    _, _, _, updates = replay(3, 0)
    assert sum(u * c for u, c in zip(updates, counts)) == S.cycle_cost(counts)


def test_replay_catches_a_wrong_order():
    """The checker is not vacuous: ending a coarse level before a finer one
    that it reads at that time breaks it."""
    bad = [("B", 1, 0), ("E", 1, 2), ("E", 0, 1)]

    def replay_list(phs, L=2):
        tn, pred = [0] * L, [False] * L
        for kind, lev, T in phs:
            if kind == "B":
                for k in range(lev + 1):
                    pred[k] = True
            else:
                for j in (lev - 1, lev + 1):
                    if 0 <= j < L:
                        d = T - tn[j]
                        if not (d == 0 or (pred[j] and 0 < d <= 1 << j)):
                            return False
                tn[lev], pred[lev] = T, False
        return True

    assert not replay_list(bad)
    assert replay_list([("B", 1, 0), ("E", 0, 1), ("B", 0, 1), ("E", 0, 2), ("E", 1, 2)])
