"""Batched form: independent blocks corrected together equal each block corrected alone.

Blocks never interact and every row's gradient is summed in a fixed order of its own
edges, so the batched result must be bit-identical to pc_correct on each block.
"""
import numpy as np
import pytest

import oracle
from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu


def _blocks():
    return [synth.hacc_box(eps_over_b=0.5, mode="HF", seed=31, n=3000),
            synth.md_box(n_clusters=20, eps_over_b=0.3, mode="SC", seed=32),
            synth.tiny_cosmo(seed=33, n=2048, mode="VP"),
            synth.fluid_box(n=5000, eps_over_b=0.5, seed=34, mode="HF"),
            synth.hacc_box(eps_over_b=0.1, mode="VP", seed=35, n=1500),
            synth.md_box(n_clusters=7, eps_over_b=0.3, mode="HF", seed=36)]


def test_batch_equals_blocks_alone(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    ws = _blocks()
    orig = torch.from_numpy(np.concatenate([w.orig for w in ws])).to(cuda)
    recon = torch.from_numpy(np.concatenate([w.recon for w in ws])).to(cuda)
    sizes = [w.n for w in ws]
    prms = [w.params() for w in ws]
    out, stats, code = pc.correct_batch(orig, recon, sizes, prms)
    assert code == 0
    at = 0
    for w, st in zip(ws, stats):
        o = orig[at:at + w.n].contiguous()
        r = recon[at:at + w.n].contiguous()
        alone, sa, ca = pc.correct(o, r, w.params())
        assert ca == 0 and st["converged"] == 1
        assert st["iters"] == sa["iters"] and st["n_active"] == sa["n_active"] and st["n_editable"] == sa["n_editable"]
        assert st["n_vulnerable"] == sa["n_vulnerable"] and st["viol0"] == sa["viol0"]
        assert torch.equal(out[at:at + w.n], alone)
        at += w.n


def test_batch_membership_is_exact(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    ws = _blocks()
    orig = torch.from_numpy(np.concatenate([w.orig for w in ws])).to(cuda)
    recon = torch.from_numpy(np.concatenate([w.recon for w in ws])).to(cuda)
    out, stats, code = pc.correct_batch(orig, recon, [w.n for w in ws], [w.params() for w in ws])
    at = 0
    for w in ws:
        c = out[at:at + w.n].contiguous()
        r = recon[at:at + w.n].contiguous()
        dec = pc.apply_edits(r, pc.encode_edits(r, c, w.params())).cpu().numpy()
        assert np.abs(dec.astype(np.float64) - w.orig).max() <= w.xi
        lab0, _, _ = oracle.fof_labels(w.orig, **w.params())
        lab1, _, _ = oracle.fof_labels(dec, **w.params())
        assert np.array_equal(lab0, lab1)
        at += w.n


def test_batch_rejects_bad_tiling_and_names_the_block(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    ws = _blocks()[:2]
    orig = torch.from_numpy(np.concatenate([w.orig for w in ws])).to(cuda)
    recon = torch.from_numpy(np.concatenate([w.recon for w in ws])).to(cuda)
    bad = recon.clone()
    bad[ws[0].n + 3, 1] += 3 * ws[1].xi
    with pytest.raises(pc.PcError) as e:
        pc.correct_batch(orig, bad, [w.n for w in ws], [w.params() for w in ws])
    assert e.value.code == -2 and "block 1" in str(e.value)


def test_cell_factor_changes_speed_only(cuda):
    # the autotuner's knob: the selected pairs are the same for every cell factor
    import torch
    import paper_2604_18801_gb300 as pc
    w = synth.hacc_box(eps_over_b=0.5, mode="SC", seed=61, n=60000)
    o = torch.from_numpy(w.orig).to(cuda)
    best, ms = pc.autotune_cells(o, w.params())
    assert best in (2, 4, 8, 16, 32) and all(v > 0 for v in ms.values())
    ref = None
    for f in (2, 8, 32):
        cons = pc.select_constraints(o, w.params(cell_factor=f))
        got = [x.cpu().numpy() for x in cons.pairs()]
        cons.close()
        if ref is None:
            ref = got
        else:
            assert all(np.array_equal(a, b) for a, b in zip(ref, got))


@pytest.mark.parametrize("mode", [0, 2])
def test_tuning_knobs_change_speed_only(cuda, mode):
    # The pair search's knobs (cell factor, dense-cell threshold) change the binning, but the
    # correction numbers its editable particles in a canonical order, so the corrected
    # coordinates are the same bits for every setting; pc_autotune returns a valid setting.
    # The PGD screen's chunk length changes only how its walk is split among warps (its
    # outputs are set unions), so it too leaves every bit and counter unchanged.
    import torch
    import paper_2604_18801_gb300 as pc
    w = synth.hacc_box(eps_over_b=0.1, mode="VP", seed=62, n=120000)
    o, r = torch.from_numpy(w.orig).to(cuda), torch.from_numpy(w.recon).to(cuda)
    cf, dc, times = pc.autotune(o, w.params(mode=mode))
    assert cf in (2, 4, 8, 16, 32) and dc in (0, 32, 128, 512)
    assert all(v > 0 for t in times.values() for v in t.values())
    ref = None
    for f, d, k in ((2, 0, 0), (8, 32, 0), (32, 12, 0), (cf, dc, 0), (8, 0, 100), (8, 0, 1 << 30)):
        c, st, code = pc.correct(o, r, w.params(mode=mode, cell_factor=f, dense_cell=d, screen_chunk=k))
        assert code == 0
        if ref is None:
            ref = (c, st["iters"], st["pair_evals"], st["row_updates"])
        else:
            assert (st["iters"], st["pair_evals"], st["row_updates"]) == ref[1:], (f, d, k)
            assert torch.equal(c, ref[0]), (f, d, k)
