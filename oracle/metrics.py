"""Cluster-query metrics of Sec. 4.1 ("Metrics") written out from their definitions.

Test infrastructure only (like the rest of this package): the CUDA library's
pc_cluster_metrics is checked against these functions.

Reading: a halo is a friends-of-friends component with at least ``min_members``
particles; a particle outside every halo shares a halo with no other particle.
Labels are "smallest id of the component".

* ARI: particle pairs are counted by halo co-membership in the original (lab0) and
  the decoded data (lab1): TP same halo in both, FN same only in the original (split),
  FP same only in the decoded data (merged), TN different in both; then
  ARI = 2 (TP TN - FP FN) / ((TP + FN)(FN + TN) + (TP + FP)(FP + TN)).
* IoU of original halo H_i: max over decoded halos H'_j of |H_i & H'_j| / |H_i | H'_j|
  (0 without overlap); MWM-IoU weights it by |H_i|.
* HMF: halos counted per equal-width bin of log10(members) from log10(min_members) to
  log10 of the largest original halo, per volume and per unit of log10 mass.
"""
from __future__ import annotations

import math

import numpy as np


def _pairs(k: int) -> int:
    return k * (k - 1) // 2


def halo_sizes(lab: np.ndarray) -> np.ndarray:
    """Members per component, indexed by the component's label."""
    return np.bincount(np.asarray(lab, np.int64), minlength=len(lab))


def cluster_metrics(lab0, lab1, min_members: int = 20, n_bins: int = 50, volume: float = 1.0) -> dict:
    lab0 = np.asarray(lab0, np.int64)
    lab1 = np.asarray(lab1, np.int64)
    n = len(lab0)
    s0, s1 = halo_sizes(lab0), halo_sizes(lab1)
    halos0 = [int(i) for i in np.flatnonzero(s0 >= min_members)]
    halos1 = [int(j) for j in np.flatnonzero(s1 >= min_members)]
    p0 = sum(_pairs(int(s0[i])) for i in halos0)
    p1 = sum(_pairs(int(s1[j])) for j in halos1)
    # contingency of (original halo, decoded halo) over particles in a halo on both sides
    both = (s0[lab0] >= min_members) & (s1[lab1] >= min_members)
    if both.any():
        ij, nij = np.unique(np.stack([lab0[both], lab1[both]], axis=1), axis=0, return_counts=True)
    else:
        ij, nij = np.zeros((0, 2), np.int64), np.zeros(0, np.int64)
    tp = sum(_pairs(int(c)) for c in nij)
    fn = p0 - tp
    fp = p1 - tp
    tn = _pairs(n) - tp - fn - fp
    den = (tp + fn) * (fn + tn) + (tp + fp) * (fp + tn)
    ari = 2 * (tp * tn - fp * fn) / den if den > 0 else 1.0
    best = {}
    for (i, j), c in zip(ij.tolist(), nij.tolist()):
        v = c / (float(s0[i]) + float(s1[j]) - c)
        best[i] = max(best.get(i, 0.0), v)
    members0 = sum(int(s0[i]) for i in halos0)
    mwm = sum(int(s0[i]) * best.get(i, 0.0) for i in halos0) / members0 if members0 else 1.0
    out = dict(tp=tp, fp=fp, fn=fn, tn=tn, ari=ari, mwm_iou=mwm, halos0=len(halos0), halos1=len(halos1),
               members0=members0)
    if n_bins > 0:
        mx = max([int(s0[i]) for i in halos0] + [min_members])
        lo = math.log10(min_members)
        hi = math.log10(mx) + 1e-9
        width = (hi - lo) / n_bins
        edges = [10.0 ** (lo + k * width) for k in range(n_bins + 1)]

        def hmf(sizes, halos):
            counts = [0] * n_bins
            for h in halos:
                b = int(math.floor((math.log10(float(sizes[h])) - lo) / width))
                counts[min(max(b, 0), n_bins - 1)] += 1
            return [c / (volume * width) for c in counts]

        out["hmf0"] = hmf(s0, halos0)
        out["hmf1"] = hmf(s1, halos1)
        out["bin_edges"] = edges
    return out
