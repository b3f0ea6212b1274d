"""The seeded minibatch shuffle (synth.shuffle): a keyed permutation of the
rollout rows per epoch, minibatch m = positions [mN/M, (m+1)N/M).

Pins: it is a permutation of [0, N) for bit counts odd and even, powers of two
and their neighbours, N = 1 and 2; an epoch's minibatches partition the rows;
with an even bit count it is the balanced Feistel network (written out here
with left and right halves); the key and the epoch counter change it; the
image of a fixed position is spread over [0, N) across counters."""
import numpy as np
import pytest

from synth import shuffle
from synth.philox import philox4x32_10, seed_key


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 9, 63, 64, 65, 100, 1000, 4095, 4096, 4097, 65535, 300000])
def test_permutation_of_the_rows(N):
    p = shuffle.permute(np.arange(N, dtype=np.uint32), N, 5, 9)
    assert np.array_equal(np.sort(p), np.arange(N))


@pytest.mark.parametrize("N,M", [(1000, 8), (4097, 8), (26, 4), (7, 8)])
def test_minibatches_partition_an_epoch(N, M):
    rows = np.concatenate([shuffle.minibatch_rows(m, M, N, 11, 3) for m in range(M)])
    assert len(rows) == N and np.array_equal(np.sort(rows), np.arange(N))
    sizes = [len(shuffle.minibatch_rows(m, M, N, 11, 3)) for m in range(M)]
    assert max(sizes) - min(sizes) <= 1


def _balanced(x, half, seed, ctr):
    """Four-round balanced Feistel network on 2 * half bits, halves L and R."""
    k0, k1 = seed_key(seed)
    mask = (1 << half) - 1
    out = []
    for v in np.asarray(x, np.uint64):
        L, R = (int(v) >> half) & mask, int(v) & mask
        for rnd in range(4):
            F = int(philox4x32_10(np.uint32(R), np.uint32(rnd), np.uint32(ctr), np.uint32(shuffle.STREAM_SHUFFLE),
                                  k0, k1)[0]) & mask
            L, R = R, L ^ F
        out.append((L << half) | R)
    return np.array(out, np.uint64)


@pytest.mark.parametrize("bits", [4, 10, 18])
def test_even_bit_count_is_the_balanced_network(bits):
    x = np.arange(min(1 << bits, 3000), dtype=np.uint32)
    got = shuffle.feistel(x, bits, 21, 6).astype(np.uint64)
    assert np.array_equal(got, _balanced(x, bits // 2, 21, 6))


def test_odd_bit_count_uses_the_smallest_power_of_two():
    # N = 3000: 12 bits (even); N = 5000: 13 bits (odd)
    assert shuffle.domain_bits(3000) == 12 and shuffle.domain_bits(5000) == 13
    assert shuffle.domain_bits(1) == 2 and shuffle.domain_bits(4) == 2 and shuffle.domain_bits(5) == 3
    x = np.arange(1 << 13, dtype=np.uint32)
    y = shuffle.feistel(x, 13, 2, 1)
    assert np.array_equal(np.sort(y), x.astype(y.dtype))       # a permutation of [0, 2^13) itself


def test_key_and_counter_change_the_permutation():
    N = 1000
    base = shuffle.permute(np.arange(N, dtype=np.uint32), N, 5, 9)
    assert not np.array_equal(base, shuffle.permute(np.arange(N, dtype=np.uint32), N, 5, 10))
    assert not np.array_equal(base, shuffle.permute(np.arange(N, dtype=np.uint32), N, 6, 9))


def test_image_of_a_position_spreads_over_the_rows():
    N, n = 1000, 400
    img = np.array([shuffle.permute(np.array([0], np.uint32), N, 3, c)[0] for c in range(n)])
    # uniform on [0, N): mean N/2 with standard error N / sqrt(12 n); every decile hit
    assert abs(img.mean() - (N - 1) / 2) < 5 * N / np.sqrt(12 * n)
    assert len(np.unique(img // (N // 10))) == 10
