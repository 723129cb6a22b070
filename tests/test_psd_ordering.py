"""The pair orderings of the PSD eigensolver's sweeps, checked on the CPU:
each sweep must rotate every index pair (i < j) of the padded order exactly
once, and the pairs of one round must be disjoint.  The orderings are
restated here from their definitions in csrc/psd.cuh: the round-robin
tournament (player ne - 1 stays, the others turn), and, for the blocked
sweep, 8-index blocks paired by the same tournament, with the 15-round
tournament on each pair's 16 indices in a sweep's first block round and the
cross rounds (a, 8 + (a + m) mod 8), m = 0..7, in the others."""
import itertools

import pytest


def tournament(r, k, ne):
    """Pair k of round r of the round-robin tournament on ne players."""
    m = ne - 1
    if k == 0:
        return r, m
    return (r + k) % m, (r - k + m) % m


def scalar_sweep(ne):
    for r in range(ne - 1):
        yield [tournament(r, k, ne) for k in range(ne // 2)]


def blocked_sweep(ne, b=8):
    nb = ne // b
    for br in range(nb - 1):
        blocks = [tournament(br, k, nb) for k in range(nb // 2)]
        idx = [[bi * b + a for a in range(b)] + [bj * b + a for a in range(b)] for bi, bj in blocks]
        rounds = []
        if br == 0:
            for ir in range(2 * b - 1):
                rounds.append([tournament(ir, lane, 2 * b) for lane in range(b)])
        else:
            for m in range(b):
                rounds.append([(lane, b + (lane + m) % b) for lane in range(b)])
        for rnd in rounds:                    # one round of every block pair at once
            yield [(R[p], R[q]) for R in idx for p, q in rnd]


def check_sweep(rounds, ne):
    seen = {}
    for rnd in rounds:
        flat = [i for pq in rnd for i in pq]
        assert len(flat) == len(set(flat)), "pairs of a round overlap"
        for p, q in rnd:
            key = (min(p, q), max(p, q))
            assert key[0] != key[1]
            seen[key] = seen.get(key, 0) + 1
    want = set(itertools.combinations(range(ne), 2))
    assert set(seen) == want
    assert all(v == 1 for v in seen.values())


@pytest.mark.parametrize("ne", [4, 8, 12, 48])
def test_scalar_sweep_rotates_every_pair_once(ne):
    check_sweep(scalar_sweep(ne), ne)


@pytest.mark.parametrize("ne", [64, 80, 128, 208])
def test_blocked_sweep_rotates_every_pair_once(ne):
    check_sweep(blocked_sweep(ne), ne)


def test_blocked_sweep_round_count():
    # 15 rounds in the first block round, 8 in each of the other nb - 2
    ne = 128
    assert sum(1 for _ in blocked_sweep(ne)) == 15 + 8 * (ne // 8 - 2)
