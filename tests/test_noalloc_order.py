"""Index arithmetic of the allocation-free fit's window order, checked on the host.

mdhp_fit_batch_noalloc (csrc/mdhp_noalloc.cu) orders windows longest first
without a sort workspace: each window falls in bucket floor(log2(N + 1))
(capped at 31), a count per bucket, an exclusive scan over the buckets from
the longest, and an atomic scatter of every window into its bucket's range
of the fixed scratch array (head of 128 words, then B window slots).  This
replays those formulas, with the scatter's atomics taken in an arbitrary
order, and checks that every write lands inside the array, that the order
is a permutation of the batch, and that it is longest-bucket first."""
import numpy as np
import pytest

HEAD = 128
MAX_WINDOWS = 65536  # MDHP_NOALLOC_MAX_WINDOWS in include/mdhp.h


def bucket(n):
    v = max(int(n), 0) + 1
    return min(v.bit_length() - 1, 31)


def replay(counts, rng):
    B = len(counts)
    s = np.zeros(HEAD + MAX_WINDOWS, dtype=np.int64)
    for b in range(B):  # k_na_count
        s[bucket(counts[b])] += 1
    run = 0
    for k in range(31, -1, -1):  # k_na_scan: longest bucket first
        s[32 + k] = run
        run += s[k]
    s[64], s[65], s[66] = 0, 0, B
    for b in rng.permutation(B):  # k_na_scatter, atomics in any order
        pos = s[32 + bucket(counts[b])]
        s[32 + bucket(counts[b])] += 1
        assert 0 <= pos < B
        assert HEAD + pos < len(s)
        s[HEAD + pos] = b
    return s[HEAD:HEAD + B], s


@pytest.mark.parametrize("B", [1, 2, 33, 1000, MAX_WINDOWS])
def test_order_is_a_longest_first_permutation(B):
    rng = np.random.default_rng(B)
    counts = np.concatenate([[0, 1, 2, 3, (1 << 31) - 1][: min(B, 5)],
                             rng.integers(0, 200000, max(B - 5, 0))])[:B]
    order, s = replay(counts, rng)
    assert sorted(order.tolist()) == list(range(B))
    bk = np.array([bucket(counts[b]) for b in order])
    assert np.all(np.diff(bk) <= 0)  # buckets never grow along the order
    assert s[66] == B and s[64] == 0 and s[65] == 0  # work range [0, B), queue at 0
