"""Several linking lengths at once (Sec. 1 and Sec. 5: a range of thresholds is supported
by enforcing the union of the pairs each threshold selects).  The oracle's PGD takes a
linking length per active pair; it is pinned here to its single-threshold form, to torch
autograd + torch.optim.Adam with per-pair thresholds, and to the guarantee the union
gives: after convergence and decoding, the friends-of-friends labels at every threshold
equal the original's."""
import numpy as np
import pytest

import oracle
from paper_2604_18801_gb300 import synth
from test_oracle_pins import _torch_pgd


def test_one_threshold_per_pair_reduces_to_the_plain_solver():
    w = synth.tiny_cosmo(seed=9, n=600)
    kw = w.params(mode=0, replay_iters=8)
    ai, aj, al, _ = oracle.select(w.orig, **kw)
    _, d0, e0, s0 = oracle.pgd(w.orig, w.recon, ai, aj, al, **kw)
    _, d1, e1, s1 = oracle.pgd_multi(w.orig, w.recon, ai, aj, al, np.full(len(ai), w.b), **kw)
    assert np.array_equal(d0, d1) and np.array_equal(e0, e1) and s0 == s1


@pytest.mark.parametrize("mode", [0, 2])
def test_union_pgd_matches_torch_autograd_and_adam(mode):
    w = synth.tiny_cosmo(seed=9, n=600)
    kw = w.params(mode=mode)
    bl = [0.8 * w.b, w.b, 1.25 * w.b]
    ai, aj, al, ab = oracle.select_multi(w.orig, bl, **kw)
    assert len(set(ab.tolist())) == 3 and len(ai) > 50
    # per pair, the thresholds of Eq. 3 at its own linking length
    cs = {b: oracle.constants(w.orig, w.recon, **dict(kw, b=b)) for b in bl}
    c = dict(cs[w.b], thr_link=np.array([cs[b]["thr_link"] for b in ab]),
             thr_non=np.array([cs[b]["thr_non"] for b in ab]))
    steps = 6
    _, delta, ed, st = oracle.pgd_multi(w.orig, w.recon, ai, aj, al, ab, **dict(kw, replay_iters=steps))
    d = oracle.DEFAULTS
    E, dref, _ = _torch_pgd(w.orig, w.recon, ai, aj, al, c, w.xi, d["alpha_rel"], d["eps_rel"], steps, True)
    assert np.array_equal(np.flatnonzero(ed), E)
    assert np.abs(delta[E] - dref).max() <= 1e-9 * w.xi
    # a plausible slip -- every pair held to the middle threshold -- is far from it
    _, wrong, _, _ = oracle.pgd_multi(w.orig, w.recon, ai, aj, al, np.full(len(ai), w.b),
                                      **dict(kw, replay_iters=steps))
    assert np.abs(wrong[E] - dref).max() > 1e-3 * w.xi


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_union_preserves_membership_at_every_threshold(mode):
    w = synth.tiny_cosmo(seed=7, n=1500)
    kw = w.params(mode=mode)
    bl = [0.8 * w.b, w.b, 1.25 * w.b]
    ai, aj, al, ab = oracle.select_multi(w.orig, bl, **kw)
    corr, _, _, st = oracle.pgd_multi(w.orig, w.recon, ai, aj, al, ab, **kw)
    assert st["converged"] == 1 and st["viol_final"] == 0
    dec = oracle.decode(w.recon, oracle.encode(w.recon, corr, **kw))
    assert np.abs(dec.astype(np.float64) - w.orig).max() <= w.xi
    for b in bl:
        kb = dict(kw, b=b)
        assert np.array_equal(oracle.fof_labels(dec, **kb)[0], oracle.fof_labels(w.orig, **kb)[0])
        m = ab == b
        assert oracle.count_flips(dec, ai[m], aj[m], al[m], **kb) == 0
    # one threshold alone does not protect the others
    ai1, aj1, al1, _ = oracle.select(w.orig, **kw)
    c1, _, _, s1 = oracle.pgd(w.orig, w.recon, ai1, aj1, al1, **kw)
    broken = 0
    for b in bl:
        kb = dict(kw, b=b)
        broken += not np.array_equal(oracle.fof_labels(c1, **kb)[0], oracle.fof_labels(w.orig, **kb)[0])
    assert broken >= 1


def test_overlapping_windows_keep_both_constraints():
    # thresholds closer than the vulnerable window: a pair can be active for both, once
    # as a link of the larger and once as a non-link of the smaller; both hold after PGD
    w = synth.tiny_cosmo(seed=5, n=1500)
    kw = w.params(mode=0)
    bl = [w.b, w.b * 1.02]
    ai, aj, al, ab = oracle.select_multi(w.orig, bl, **kw)
    keys = ai.astype(np.int64) * w.n + aj
    u, cnt = np.unique(keys, return_counts=True)
    twice = np.isin(keys, u[cnt == 2])
    assert twice.sum() >= 2 and not np.all(al[twice] == al[twice][0])
    corr, _, _, st = oracle.pgd_multi(w.orig, w.recon, ai, aj, al, ab, **kw)
    assert st["converged"] == 1
    for b in bl:
        kb = dict(kw, b=b)
        assert np.array_equal(oracle.fof_labels(corr, **kb)[0], oracle.fof_labels(w.orig, **kb)[0])
