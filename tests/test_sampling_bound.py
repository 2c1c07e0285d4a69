"""The bound behind q-gram sampling (the GPU index's stride): an alignment of a read of length m
with at most k edits leaves at least
    t_s = ceil(nq / s) - min(ceil(nq / s), k * ceil(q / s)),   nq = m - q + 1,
of the q-grams at read offsets 0, s, 2s, ... untouched (the q-gram lemma of Section "The q-group
index" for s = 1, where it reads m + 1 - q(k + 1)).

Checked here by brute force over every placement of up to k edits on small reads: a substitution
or insertion at read position x touches the q-grams starting at x - q + 1 .. x, a deletion between
positions x - 1 and x touches those spanning both, x - q + 1 .. x - 1.  The minimum over all
placements must reach the closed form (it is a lower bound) and, for these sizes, equal it (it is
not loose).
"""
import itertools

import pytest


def closed_form(m, q, k, s):
    nq = m - q + 1
    na = -(-nq // s)
    return na - min(na, k * -(-q // s))


def touched(m, q, kind, x):
    lo = x - q + 1
    hi = x if kind in ("sub", "ins") else x - 1
    return set(range(max(0, lo), min(m - q, hi) + 1))


def brute_min(m, q, k, s):
    sampled = set(range(0, m - q + 1, s))
    edits = [(kind, x) for kind in ("sub", "ins") for x in range(m)] + [("del", x) for x in range(1, m)]
    best = len(sampled)
    for e in range(k + 1):
        for combo in itertools.combinations(edits, e):
            hit = set()
            for kind, x in combo:
                hit |= touched(m, q, kind, x)
            best = min(best, len(sampled - hit))
    return best


@pytest.mark.parametrize("m,q,k,s", [(12, 3, 2, 1), (12, 3, 2, 2), (12, 3, 2, 3), (13, 4, 2, 2), (14, 4, 2, 4),
                                     (15, 5, 1, 5), (16, 4, 3, 3), (11, 2, 3, 2), (18, 6, 2, 6), (17, 4, 2, 8)])
def test_sampled_bound_is_tight(m, q, k, s):
    assert brute_min(m, q, k, s) == max(0, closed_form(m, q, k, s))


def test_stride_one_is_the_qgram_lemma():
    for m in range(20, 260, 7):
        for q in range(4, 17):
            for k in range(0, 14):
                if m + 1 - q * (k + 1) >= 1:
                    assert closed_form(m, q, k, 1) == m + 1 - q * (k + 1)


def test_bench_workload_settings_admit_their_strides():
    """The settings the autotuner picks on the benchmark workloads keep a threshold of at least 1."""
    def k_of(m):
        return (m * 50 + 999) // 1000
    assert closed_form(100, 16, k_of(100), 16) == 1
    assert closed_form(50, 12, k_of(50), 12) == 1
    assert closed_form(75, 15, k_of(75), 3) >= 1
    assert closed_form(250, 16, k_of(250), 16) >= 1 and closed_form(150, 16, k_of(150), 16) >= 1
