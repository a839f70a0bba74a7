"""Lossless stage of the edit stream (Algorithm 1, last line; Sec. 3.3 "Compaction,
quantization, and lossless compression"): canonical Huffman coding of the stream's bytes.

Test infrastructure only, written out from the definitions; the CUDA library's
pc_huff_encode / pc_huff_decode are checked against it bit for bit.  The paper follows
Huffman with ZSTD; the ZSTD stage is not part of this container.

Container "PCH1" (little endian), wrapping an edit stream v1:
  0   "PCH1" | 4 u32 version = 1 | 8 u64 raw_bytes | 16 u32 n_lanes | 20 u32 chunk
  24  u32 max_len = 15 | 28 u32 0 | 32..95 the stream's 64-byte header, verbatim
  96  per lane: u64 n_syms | u64 bit_len | u64 n_chunks | 256 x u8 code length |
      n_chunks x u64 chunk bit offset | ceil(bit_len / 32) x u32 words
The body after the stream's header is split into lanes: lane 0 the flag bytes, lane
1 + k byte k (0 = least significant) of every code.  Each lane is coded on its own.

Code lengths: Huffman's algorithm with ties broken by node id (symbols 0..255, then
merged nodes in order of creation); when a length exceeds 15, the longest codes are
folded back to 15 and the Kraft inequality restored by deepening the deepest codes
shorter than 15 (the rebalancing that deflate encoders use), and lengths are dealt out
again from longest to shortest in ascending order of (frequency, -symbol).
Codes are canonical: ordered by (length, symbol) and assigned consecutively.  Bits
are written most significant first into 32-bit words, from bit 31 down.
"""
from __future__ import annotations

import heapq

import numpy as np

MAX_LEN = 15
CHUNK = 1024
HEADER = 64


def code_lengths(freq) -> list:
    freq = [int(f) for f in freq]
    syms = [s for s in range(256) if freq[s] > 0]
    lengths = [0] * 256
    if not syms:
        return lengths
    if len(syms) == 1:
        lengths[syms[0]] = 1
        return lengths
    heap = [(freq[s], s) for s in syms]
    heapq.heapify(heap)
    parent = {}
    nxt = 256
    while len(heap) > 1:
        w1, a = heapq.heappop(heap)
        w2, b = heapq.heappop(heap)
        parent[a] = nxt
        parent[b] = nxt
        heapq.heappush(heap, (w1 + w2, nxt))
        nxt += 1
    for s in syms:
        d, x = 0, s
        while x in parent:
            x = parent[x]
            d += 1
        lengths[s] = d
    if max(lengths) <= MAX_LEN:
        return lengths
    # fold into MAX_LEN and restore the Kraft inequality
    bl = [0] * (max(lengths) + 1)
    for s in syms:
        bl[lengths[s]] += 1
    overflow = 0
    for b in range(MAX_LEN + 1, len(bl)):
        overflow += bl[b]
        bl[MAX_LEN] += bl[b]
        bl[b] = 0
    bl = bl[:MAX_LEN + 1]
    # Kraft excess in units of 2^-MAX_LEN; each step moves the deepest code shorter than
    # MAX_LEN one level down and gives it a folded code as its sibling (net -1 unit)
    excess = sum(bl[l] << (MAX_LEN - l) for l in range(1, MAX_LEN + 1)) - (1 << MAX_LEN)
    while excess > 0:
        b = MAX_LEN - 1
        while bl[b] == 0:
            b -= 1
        bl[b] -= 1
        bl[b + 1] += 2
        bl[MAX_LEN] -= 1
        excess -= 1
    order = sorted(syms, key=lambda s: (freq[s], -s))      # rarest first
    out = [0] * 256
    i = 0
    for length in range(MAX_LEN, 0, -1):
        for _ in range(bl[length]):
            out[order[i]] = length
            i += 1
    return out


def canonical_codes(lengths) -> list:
    codes = [0] * 256
    code = 0
    prev = 0
    for s in sorted((s for s in range(256) if lengths[s] > 0), key=lambda s: (lengths[s], s)):
        code <<= lengths[s] - prev
        prev = lengths[s]
        codes[s] = code
        code += 1
    return codes


def lanes_of(stream: bytes):
    b = np.frombuffer(stream, np.uint8)
    n = int.from_bytes(stream[8:16], "little")
    m = int.from_bytes(stream[16:20], "little")
    fb = int.from_bytes(stream[48:56], "little")
    cb = (m + 7) // 8
    flags = b[HEADER:HEADER + fb]
    codes = b[HEADER + fb:]
    assert fb == (n + 7) // 8 and len(codes) % cb == 0
    return [flags] + [codes[k::cb] for k in range(cb)]


def encode_lane(sym: np.ndarray) -> bytes:
    freq = np.bincount(sym, minlength=256)
    lengths = code_lengths(freq)
    codes = canonical_codes(lengths)
    n = len(sym)
    nchunks = (n + CHUNK - 1) // CHUNK
    lens = np.array(lengths, np.int64)[sym]
    offsets = [0] * nchunks
    total = 0
    for c in range(nchunks):
        offsets[c] = total
        total += int(lens[c * CHUNK:(c + 1) * CHUNK].sum())
    # bit j of the lane is bit (len - 1 - k) of the code of the symbol whose code starts
    # at position j - k; the bit string is then cut into big-endian 32-bit words
    nwords = (total + 31) // 32
    bits = np.zeros(32 * nwords, np.uint8)
    start = np.concatenate([[0], np.cumsum(lens)[:-1]]).astype(np.int64) if n else np.zeros(0, np.int64)
    cd = np.array(codes, np.int64)[sym]
    for k in range(MAX_LEN):
        has = lens > k
        bits[start[has] + k] = (cd[has] >> (lens[has] - 1 - k)) & 1
    words = np.packbits(bits).view(">u4").astype(np.uint32) if nwords else np.zeros(0, np.uint32)
    out = bytearray()
    out += int(n).to_bytes(8, "little") + int(total).to_bytes(8, "little") + int(nchunks).to_bytes(8, "little")
    out += bytes(lengths)
    for o in offsets:
        out += int(o).to_bytes(8, "little")
    out += words.astype("<u4").tobytes()
    return bytes(out)


def encode(stream: bytes) -> bytes:
    lanes = lanes_of(stream)
    body = b"".join(encode_lane(l) for l in lanes)
    head = b"PCH1" + (1).to_bytes(4, "little") + len(stream).to_bytes(8, "little")
    head += len(lanes).to_bytes(4, "little") + CHUNK.to_bytes(4, "little") + MAX_LEN.to_bytes(4, "little")
    head += (0).to_bytes(4, "little") + stream[:HEADER]
    return head + body


def decode(blob: bytes) -> bytes:
    assert blob[:4] == b"PCH1"
    raw = int.from_bytes(blob[8:16], "little")
    nl = int.from_bytes(blob[16:20], "little")
    header = blob[32:32 + HEADER]
    at = 32 + HEADER
    lanes = []
    for _ in range(nl):
        n = int.from_bytes(blob[at:at + 8], "little")
        total = int.from_bytes(blob[at + 8:at + 16], "little")
        nch = int.from_bytes(blob[at + 16:at + 24], "little")
        lengths = list(blob[at + 24:at + 24 + 256])
        at += 24 + 256 + 8 * nch
        nwords = (total + 31) // 32
        words = np.frombuffer(blob[at:at + 4 * nwords], "<u4")
        at += 4 * nwords
        codes = canonical_codes(lengths)
        table = {(lengths[s], codes[s]): s for s in range(256) if lengths[s] > 0}
        out = np.empty(n, np.uint8)
        pos = 0
        for i in range(n):
            cd, ln = 0, 0
            while True:
                bit = (int(words[pos >> 5]) >> (31 - (pos & 31))) & 1
                pos += 1
                cd = (cd << 1) | bit
                ln += 1
                if (ln, cd) in table:
                    out[i] = table[(ln, cd)]
                    break
                assert ln < MAX_LEN
        lanes.append(out)
    flags = lanes[0]
    cb = nl - 1
    codes = np.empty(sum(len(l) for l in lanes[1:]), np.uint8)
    for k in range(cb):
        codes[k::cb] = lanes[1 + k]
    res = bytes(header) + flags.tobytes() + codes.tobytes()
    assert len(res) == raw
    return res
