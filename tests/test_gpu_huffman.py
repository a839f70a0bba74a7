"""Lossless stage (Sec. 3.3, "Compaction, quantization, and lossless compression"): the
CUDA library's canonical Huffman container equals the oracle's byte for byte, the GPU
decoder returns the edit stream byte for byte (also from the oracle's container), and a
malformed container is rejected.

Inputs: edit streams the library writes for the parity workloads, and synthetic streams
that reach what those may not (many chunks with a ragged last one, an empty code lane, a
lane with a single symbol, frequencies that force the 15-bit length limit).
"""
import numpy as np
import pytest

import oracle
from oracle import huffman as oh
from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu


def dev(a, d):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(d)


def synthetic_stream(n, m, density, seed, skew="fib"):
    """A well-formed edit stream v1 of n particles: flag bits set with the given density,
    the codes' bytes drawn from a skewed distribution over few symbols ("fib": weights
    of the Fibonacci numbers, deep enough to exceed 15 bits) or uniform over 0..255."""
    rng = np.random.default_rng(seed)
    flags = rng.random(n) < density
    fb = (n + 7) // 8
    flag_bytes = np.packbits(flags, bitorder="little")[:fb]
    cb = (m + 7) // 8
    nc = int(flags.sum()) * 3 * cb
    if skew == "fib":
        f = [1, 1]
        while len(f) < 26:
            f.append(f[-1] + f[-2])
        p = np.array(f[::-1], np.float64)
        codes = rng.choice(26, size=nc, p=p / p.sum()).astype(np.uint8) * 7
    else:
        codes = rng.integers(0, 256, nc).astype(np.uint8)
    head = bytearray(64)
    head[0:4] = b"PCE1"
    head[4:8] = (1).to_bytes(4, "little")
    head[8:16] = int(n).to_bytes(8, "little")
    head[16:20] = int(m).to_bytes(4, "little")
    head[32:40] = np.float64(0.01).tobytes()
    head[40:48] = int(flags.sum()).to_bytes(8, "little")
    head[48:56] = int(fb).to_bytes(8, "little")
    head[56:64] = int(nc).to_bytes(8, "little")
    return bytes(head) + flag_bytes.tobytes() + codes.tobytes()


def _roundtrip(pc, cuda, stream: bytes, oracle_decode=True):
    import torch
    s = dev(np.frombuffer(stream, np.uint8), cuda)
    blob = pc.huff_encode(s)
    ref = oh.encode(stream)
    got = bytes(blob.cpu().numpy())
    assert len(got) == len(ref)
    assert got == ref
    back = pc.huff_decode(blob)
    assert torch.equal(back, s)
    # the oracle's container decodes on the GPU, and the GPU's on the oracle
    assert torch.equal(pc.huff_decode(dev(np.frombuffer(ref, np.uint8), cuda)), s)
    if oracle_decode:
        assert oh.decode(got) == stream
    return got


@pytest.mark.parametrize("m_bits", [8, 12, 16, 32])
def test_container_of_a_corrected_stream_is_bit_exact(cuda, m_bits):
    import paper_2604_18801_gb300 as pc
    w = synth.md_box(n_clusters=300, eps_over_b=0.3, seed=5)
    prm = w.params(mode=2, m_bits=m_bits)
    o, r = dev(w.orig, cuda), dev(w.recon, cuda)
    corr, _, _ = pc.correct(o, r, prm)
    s = pc.encode_edits(r, corr, prm)
    _roundtrip(pc, cuda, bytes(s.cpu().numpy()))
    dec = pc.apply_edits(r, pc.huff_decode(pc.huff_encode(s)))
    assert np.array_equal(dec.cpu().numpy(), pc.apply_edits(r, s).cpu().numpy())


def test_container_of_a_hacc_box(cuda):
    import paper_2604_18801_gb300 as pc
    w = synth.hacc_box(eps_over_b=0.5, n=64 ** 3, seed=4)
    prm = w.params(mode=0)
    o, r = dev(w.orig, cuda), dev(w.recon, cuda)
    corr, st, code = pc.correct(o, r, prm)
    assert code == 0
    s = pc.encode_edits(r, corr, prm)
    blob = _roundtrip(pc, cuda, bytes(s.cpu().numpy()), oracle_decode=False)
    assert len(blob) < s.numel()


@pytest.mark.parametrize("n,m,density,skew", [
    (8, 16, 1.0, "fib"),                    # one chunk per lane, a handful of symbols
    (1024 * 8, 16, 0.3, "fib"),             # the flag lane is exactly one chunk
    (1024 * 8 + 8, 8, 0.3, "uniform"),      # one symbol past a chunk
    (4096 * 8 + 8, 8, 0.3, "uniform"),      # several chunks, one symbol past the last full one
    (1_000_003, 24, 0.05, "fib"),           # many chunks, ragged tails, 3 code lanes
    (50_000, 16, 0.0, "fib"),               # no edits: flag lane of one symbol, empty code lanes
    (50_001, 32, 1.0, "uniform"),           # every particle edited
])
def test_synthetic_streams_bit_exact(cuda, n, m, density, skew):
    import paper_2604_18801_gb300 as pc
    stream = synthetic_stream(n, m, density, seed=n % 97, skew=skew)
    _roundtrip(pc, cuda, stream, oracle_decode=n <= 100_000)


def test_length_limit_is_reached(cuda):
    import paper_2604_18801_gb300 as pc
    stream = synthetic_stream(400_000, 8, 1.0, seed=3, skew="fib")
    blob = _roundtrip(pc, cuda, stream, oracle_decode=False)
    lane1 = 96 + 24 + 256 + 8 * int.from_bytes(blob[96 + 16:96 + 24], "little")
    lane1 += 4 * ((int.from_bytes(blob[96 + 8:96 + 16], "little") + 31) // 32)
    lengths = np.frombuffer(blob[lane1 + 24:lane1 + 24 + 256], np.uint8)
    assert lengths.max() == 15


def test_malformed_container_rejected(cuda):
    import paper_2604_18801_gb300 as pc
    stream = synthetic_stream(50_000, 16, 0.0, seed=1)
    blob = pc.huff_encode(dev(np.frombuffer(stream, np.uint8), cuda))
    h = blob.cpu().numpy()

    def rejected(b):
        with pytest.raises(pc.PcError) as e:
            pc.huff_decode(dev(b, cuda))
        assert e.value.code == -5

    bad = h.copy()
    bad[0] = ord("X")
    rejected(bad)                                           # magic
    rejected(h[:200].copy())                                # truncated
    bad = h.copy()
    bad[96 + 24:96 + 24 + 256] = 1                          # lengths that are no prefix code
    rejected(bad)
    # the flag lane has one symbol (code 0, one bit): a set bit is no code
    words_at = 96 + 24 + 256 + 8 * int.from_bytes(bytes(h[96 + 16:96 + 24]), "little")
    bad = h.copy()
    bad[words_at + 3] |= 0x80
    rejected(bad)
    # a chunk offset that does not match where the previous chunk ends
    bad = h.copy()
    bad[96 + 24 + 256 + 8] ^= 1
    rejected(bad)
    bad = h.copy()
    bad[32] = ord("X")                                      # the wrapped stream header
    rejected(bad)
    # a container that does not start on a 4-byte boundary is refused before any kernel
    import torch
    shifted = torch.zeros(blob.numel() + 1, dtype=torch.uint8, device=cuda)
    shifted[1:].copy_(blob)
    with pytest.raises(pc.PcError) as e:
        pc.huff_decode(shifted[1:])
    assert e.value.code == -1
