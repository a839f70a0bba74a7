"""Iteration-capped correction and the cluster-query metrics (Sec. 4.1, Sec. 4.2 with a
100-iteration cap): the GPU metrics equal the oracle's on the same labelings, a capped
correction improves ARI and MWM-IoU over the bare reconstruction, and a converged one
scores exactly 1."""
import numpy as np
import pytest

from oracle import metrics
from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu


def _check(pc, torch, l0, l1, mm, nb):
    g = pc.cluster_metrics(l0, l1, min_members=mm, n_bins=nb, volume=1.0)
    o = metrics.cluster_metrics(l0.cpu().numpy(), l1.cpu().numpy(), min_members=mm, n_bins=nb, volume=1.0)
    for k in ("tp", "fp", "fn", "tn", "halos0", "halos1", "members0"):
        assert g[k] == o[k], k
    assert g["ari"] == pytest.approx(o["ari"], abs=1e-12)
    assert g["mwm_iou"] == pytest.approx(o["mwm_iou"], abs=1e-8)
    if nb:
        assert np.allclose(g["hmf0"], o["hmf0"], rtol=1e-12) and np.allclose(g["hmf1"], o["hmf1"], rtol=1e-12)
        assert np.allclose(g["bin_edges"], o["bin_edges"], rtol=1e-12)
    return g


def test_capped_correction_metrics_match_the_oracle(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    w = synth.hacc_box(eps_over_b=0.5, mode="VP", seed=71, n=200000)
    o = torch.from_numpy(w.orig).to(cuda)
    r = torch.from_numpy(w.recon).to(cuda)
    prm = w.params(t_max=20)
    l0, _ = pc.fof_labels(o, prm)
    lr, _ = pc.fof_labels(r, prm)
    corr, st, code = pc.correct(o, r, prm)
    assert code == 1 and st["iters"] == 20            # capped: valid output, not converged
    dec = pc.apply_edits(r, pc.encode_edits(r, corr, prm))
    lc, _ = pc.fof_labels(dec, prm)
    native = _check(pc, torch, l0, lr, 20, 50)
    capped = _check(pc, torch, l0, lc, 20, 50)
    _check(pc, torch, l0, lc, 1, 0)
    assert capped["ari"] > native["ari"] and capped["mwm_iou"] > native["mwm_iou"]
    assert native["ari"] < 1.0
    full, st2, code2 = pc.correct(o, r, w.params())
    assert code2 == 0
    lf, _ = pc.fof_labels(pc.apply_edits(r, pc.encode_edits(r, full, prm)), prm)
    exact = pc.cluster_metrics(l0, lf, min_members=20, n_bins=50)
    assert exact["ari"] == 1.0 and exact["mwm_iou"] == 1.0 and exact["hmf0"] == exact["hmf1"]
