"""Full-size checks on the HACC-shaped 256^3 box (16.8M particles, eps = 0.1 b) in the
launch configuration the benchmark times.

The oracle cannot run the whole pipeline at this size in test time, so it checks what it
can compute one by one or as a property that holds at any size:

* for sampled particles, the oracle classifies the pair with every other particle of the
  box; the vulnerable partners (potentially broken or created) must be exactly the
  partners the GPU put in the vulnerable-pair set, with the same link flag;
* after correction, encoding and decoding, the oracle counts the active pairs of the mode
  whose link state changed (must be none; for VP, A = V holds every pair that could flip,
  so the link set itself is unchanged) and decodes the edit stream itself (must equal the
  GPU decoder bit for bit); every decoded coordinate stays within xi of the original, and
  the friends-of-friends labels of the decoded data equal the oracle's labels of the
  original (its own grid pair search and sequential union-find over the links, about
  3e7 of them, computed once);
* the lossless container of each stream equals the oracle's byte for byte;
* the box reconstructed by the Morton-order baseline instead of the quantizer converges
  in HF mode with the same guarantees.
"""
import numpy as np
import pytest

import oracle
from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def box():
    return synth.hacc_box(eps_over_b=0.1, mode="VP", seed=1)


@pytest.fixture(scope="module")
def oracle_labels(box):
    # labels depend on b alone: with xi = 0 the oracle enumerates only the links
    lab, _, n_comp = oracle.fof_labels(box.orig, **box.params(xi=0.0))
    return lab, n_comp


def test_vulnerable_pairs_of_sampled_particles(cuda, box):
    import torch
    import paper_2604_18801_gb300 as pc
    w = box
    kw = w.params(mode=0)
    o = torch.from_numpy(w.orig).to(cuda)
    cons = pc.select_constraints(o, kw)
    gi, gj, gl = [x.cpu().numpy() for x in cons.pairs()]
    cons.close()
    assert len(gi) == cons.stats["n_vulnerable"] > 10 ** 7
    rng = np.random.default_rng(5)
    # half the sample from particles that have vulnerable pairs, half uniformly
    with_pairs = np.unique(np.concatenate([gi[:: max(1, len(gi) // 5000)], gj[:: max(1, len(gj) // 5000)]]))
    sample = np.concatenate([rng.choice(with_pairs, 24, replace=False), rng.choice(w.n, 24, replace=False)])
    everyone = np.arange(w.n, dtype=np.uint32)
    for i in sample:
        others = everyone[everyone != i]
        cls = oracle.classify(w.orig, np.full(len(others), i, np.uint32), others, **kw)
        vul = cls >= oracle.CLS_PB
        want = np.sort(others[vul])
        want_link = cls[vul][np.argsort(others[vul])] == oracle.CLS_PB
        m1, m2 = gi == i, gj == i
        got = np.concatenate([gj[m1], gi[m2]])
        got_link = np.concatenate([gl[m1], gl[m2]]).astype(bool)
        order = np.argsort(got)
        assert np.array_equal(got[order], want), f"particle {i}"
        assert np.array_equal(got_link[order], want_link), f"particle {i}"


@pytest.mark.parametrize("mode", ["VP", "SC", "HF"])
def test_full_size_correction_keeps_every_active_link_state(cuda, box, oracle_labels, mode):
    import torch
    import paper_2604_18801_gb300 as pc
    w = box
    kw = w.params(mode=synth.MODES[mode])
    o = torch.from_numpy(w.orig).to(cuda)
    r = torch.from_numpy(w.recon).to(cuda)
    cons = pc.select_constraints(o, kw)
    ai, aj, al = [x.cpu().numpy() for x in cons.pairs()]
    corr, st, code = pc.correct(o, r, kw, constraints=cons)
    cons.close()
    assert code == 0 and st["converged"] == 1 and len(ai) == st["n_active"]
    stream = pc.encode_edits(r, corr, kw)
    dec = pc.apply_edits(r, stream)
    dec_h = dec.cpu().numpy()
    assert np.abs(dec_h.astype(np.float64) - w.orig).max() <= w.xi
    # the oracle's own decoder gives the same coordinates
    assert np.array_equal(oracle.decode(w.recon, stream.cpu().numpy().tobytes()), dec_h)
    # the lossless container equals the oracle's and decodes to the stream
    from oracle import huffman
    blob = pc.huff_encode(stream)
    assert bytes(blob.cpu().numpy()) == huffman.encode(stream.cpu().numpy().tobytes())
    assert torch.equal(pc.huff_decode(blob), stream)
    # every active pair keeps its original link state after decoding
    assert oracle.count_flips(dec_h, ai, aj, al, **kw) == 0
    # the decoded data's labels are the oracle's labels of the original
    lab0, n0 = oracle_labels
    l1, n1 = pc.fof_labels(dec, kw)
    assert n1 == n0 and np.array_equal(l1.cpu().numpy(), lab0)
    assert st["resets"] == 0   # Algorithm 1 as printed


def test_full_size_oracle_labels_of_decoded_data(cuda, box, oracle_labels):
    """The whole membership check on the oracle's side for one mode: its labels of the
    GPU-decoded VP output equal its labels of the original."""
    import torch
    import paper_2604_18801_gb300 as pc
    w = box
    kw = w.params(mode=0)
    o = torch.from_numpy(w.orig).to(cuda)
    r = torch.from_numpy(w.recon).to(cuda)
    corr, st, code = pc.correct(o, r, kw)
    assert code == 0
    dec_h = pc.apply_edits(r, pc.encode_edits(r, corr, kw)).cpu().numpy()
    lab1, _, n1 = oracle.fof_labels(dec_h, **dict(kw, xi=0.0))
    lab0, n0 = oracle_labels
    assert n1 == n0 and np.array_equal(lab1, lab0)


def test_full_size_morton_baseline_halo_forest(cuda, box, oracle_labels):
    """The same box reconstructed by the Morton-order baseline (Sec. 4.1): HF correction
    converges, keeps every active link state and gives the original labels."""
    import torch
    import paper_2604_18801_gb300 as pc
    w = synth.with_base(box, "morton")
    kw = w.params(mode=2)
    o = torch.from_numpy(w.orig).to(cuda)
    r = torch.from_numpy(w.recon).to(cuda)
    cons = pc.select_constraints(o, kw)
    ai, aj, al = [x.cpu().numpy() for x in cons.pairs()]
    corr, st, code = pc.correct(o, r, kw, constraints=cons)
    cons.close()
    assert code == 0 and st["converged"] == 1
    dec = pc.apply_edits(r, pc.huff_decode(pc.huff_encode(pc.encode_edits(r, corr, kw))))
    dec_h = dec.cpu().numpy()
    assert np.abs(dec_h.astype(np.float64) - w.orig).max() <= w.xi
    assert oracle.count_flips(dec_h, ai, aj, al, **kw) == 0
    lab0, n0 = oracle_labels
    l1, n1 = pc.fof_labels(dec, kw)
    assert n1 == n0 and np.array_equal(l1.cpu().numpy(), lab0)
