"""Host-side schedule and cost model of the temporally adaptive cycle.

Algorithm 2 (Sec. 2.2): one iteration ("cycle") has 2^theta subiterations;
subiteration s starts the levels 0..tau(s), where tau(s) is the largest
tmp <= theta with (s - 1) mod 2^tmp == 0 (for theta = 3 the paper lists
tau = 3, 0, 1, 0, 2, 0, 1, 0).  Level k advances with dt_k = 2^k dt_min and is
therefore updated 2^(theta - k) times per cycle.

Sec. 2.2 cost model: C(tau) = 2^(theta - tau) |Omega(tau)|; one cycle costs
sum_tau C(tau) cell-updates, against 2^theta |Omega| for global stepping to
the same time.  The benchmark's throughput metric counts exactly these
C(tau)-weighted cell-updates per second.
"""
from __future__ import annotations

from typing import Sequence


def tau_sequence(theta: int) -> list[int]:
    """tau(s) for s = 1..2^theta (Alg. 2, the loop that computes tau)."""
    out = []
    for s in range(1, (1 << theta) + 1):
        tau = 0
        for tmp in range(1, theta + 1):
            if (s - 1) % (1 << tmp) == 0:
                tau = tmp
        out.append(tau)
    return out


def ending_levels(theta: int, s: int) -> list[int]:
    """Levels whose step ends after subiteration s (finest first)."""
    out = []
    k = 0
    while k <= theta and s % (1 << k) == 0:
        out.append(k)
        k += 1
    return out


def phases(theta: int, order: int = 0) -> list[tuple[str, int, int]]:
    """The phase list of one cycle as (kind, level, T), the host schedule of
    the library (fv_internal.h, make_phases).  Order 0: 'B' starts the levels
    0..level at time T (units of dt_min from the cycle start), 'E' ends the
    step of `level` at T; 3 * 2^theta - 1 phases.  Order 1 (the paper's):
    'I' commits the levels 0..level at T, 'B' as before, 'C' corrects `level`
    at the end T of its step, coarsest first; 4 * 2^theta - 1 phases."""
    out = []
    taus = tau_sequence(theta)
    for s in range(1, (1 << theta) + 1):
        tau = taus[s - 1]
        if order == 1:
            if s > 1:
                out.append(("I", tau, s - 1))
            out.append(("B", tau, s - 1))
            for k in range(tau, -1, -1):
                out.append(("C", k, s - 1 + (1 << k)))
        else:
            out.append(("B", tau, s - 1))
            for k in ending_levels(theta, s):
                out.append(("E", k, s))
    if order == 1:
        out.append(("I", theta, 1 << theta))
    return out


def cycle_cost(counts: Sequence[int], theta: int | None = None) -> int:
    """sum_tau 2^(theta - tau) |Omega(tau)|: cell-updates per cycle."""
    if theta is None:
        theta = len(counts) - 1
    return sum((1 << (theta - k)) * int(c) for k, c in enumerate(counts))


def level_cost_shares(fractions: Sequence[float]) -> list[float]:
    """Share of the cycle cost per level, from the cell fraction per level."""
    theta = len(fractions) - 1
    w = [(2.0 ** (theta - k)) * f for k, f in enumerate(fractions)]
    tot = sum(w)
    return [x / tot for x in w]


def global_cost_ratio(counts: Sequence[int], theta: int | None = None) -> float:
    """2^theta |Omega| / sum_tau C(tau): the saving over global stepping."""
    if theta is None:
        theta = len(counts) - 1
    n = sum(int(c) for c in counts)
    return (1 << theta) * n / cycle_cost(counts, theta)
