"""Pins of the lossless stage (canonical Huffman coding of the edit stream): a worked
example, optimality against an independent cost computation, the Kraft equality and the
length limit, and exact round trips of real and random edit streams."""
import heapq

import numpy as np
import pytest

import oracle
from oracle import huffman
from paper_2604_18801_gb300 import synth


def test_worked_example():
    freq = [5, 2, 1, 1] + [0] * 252
    lengths = huffman.code_lengths(freq)
    assert lengths[:4] == [1, 2, 3, 3] and sum(lengths[4:]) == 0
    codes = huffman.canonical_codes(lengths)
    assert codes[:4] == [0b0, 0b10, 0b110, 0b111]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lengths_are_optimal_and_complete(seed):
    rng = np.random.default_rng(seed)
    freq = rng.integers(1, 1000, 256) * (rng.random(256) < 0.7)
    lengths = huffman.code_lengths(freq)
    used = [s for s in range(256) if freq[s] > 0]
    assert all(lengths[s] > 0 for s in used) and all(lengths[s] == 0 for s in range(256) if freq[s] == 0)
    assert sum(2.0 ** -lengths[s] for s in used) == 1.0                 # Kraft equality
    # the optimal total cost equals the sum of the merged weights (independent computation)
    h = [int(freq[s]) for s in used]
    heapq.heapify(h)
    cost = 0
    while len(h) > 1:
        a, b = heapq.heappop(h), heapq.heappop(h)
        cost += a + b
        heapq.heappush(h, a + b)
    assert sum(int(freq[s]) * lengths[s] for s in used) == cost


def test_length_limit_keeps_a_complete_prefix_code():
    fib = [1, 1]
    while len(fib) < 40:
        fib.append(fib[-1] + fib[-2])
    freq = fib + [0] * (256 - len(fib))
    lengths = huffman.code_lengths(freq)
    used = [s for s in range(256) if freq[s] > 0]
    assert max(lengths) == huffman.MAX_LEN
    assert sum(2.0 ** -lengths[s] for s in used) == 1.0
    order = sorted(used, key=lambda s: freq[s])
    assert all(lengths[a] >= lengths[b] for a, b in zip(order, order[1:]))   # rarer: never shorter


def test_round_trip_of_real_and_random_streams():
    w = synth.tiny_cosmo(seed=5, n=3000)
    kw = w.params(mode=2)
    corr, st = oracle.correct(w.orig, w.recon, **kw)
    stream = oracle.encode(w.recon, corr, **kw)
    blob = huffman.encode(stream)
    assert huffman.decode(blob) == stream
    # an optimal prefix code is never longer than 8 bits per byte
    for lane in huffman.lanes_of(stream):
        lengths = huffman.code_lengths(np.bincount(lane, minlength=256))
        assert sum(lengths[b] for b in lane.tolist()) <= 8 * len(lane)
    # a stream with random body bytes and another with a single repeated byte
    rng = np.random.default_rng(4)
    for body in (rng.integers(0, 256, 5000, dtype=np.uint8), np.full(5000, 7, np.uint8)):
        raw = bytearray(stream[:64])
        n = 8 * 1000
        raw[8:16] = n.to_bytes(8, "little")
        raw[16:20] = (16).to_bytes(4, "little")
        raw[48:56] = (1000).to_bytes(8, "little")
        raw[56:64] = (4000).to_bytes(8, "little")
        s2 = bytes(raw) + body.tobytes()
        assert huffman.decode(huffman.encode(s2)) == s2
