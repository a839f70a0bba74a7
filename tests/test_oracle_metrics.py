"""Pins of the cluster-query metrics (Sec. 4.1): the pair-counting ARI equals
scikit-learn's adjusted Rand index on the same partition, the IoU equals a brute-force
set computation, the HMF counts equal a plain histogram, and identical labelings score 1."""
import itertools

import numpy as np
import pytest

from oracle import metrics


def _labels_from_groups(groups, n):
    """min-id labels of a partition given as lists of particle ids (the rest singletons)."""
    lab = np.arange(n)
    for g in groups:
        lab[list(g)] = min(g)
    return lab


def _random_partition(rng, n, k):
    assign = rng.integers(0, k, n)
    groups = [np.flatnonzero(assign == c).tolist() for c in range(k)]
    return _labels_from_groups([g for g in groups if g], n)


def _as_halo_partition(lab, min_members):
    # particles outside halos become singletons, each with its own id
    size = np.bincount(lab, minlength=len(lab))
    return np.where(size[lab] >= min_members, lab, len(lab) + np.arange(len(lab)))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ari_equals_library_adjusted_rand_index(seed):
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(seed)
    n = 3000
    lab0 = _random_partition(rng, n, 60)
    # the decoded labels: the original with some halos merged and some particles moved
    lab1 = lab0.copy()
    move = rng.choice(n, 300, replace=False)
    lab1[move] = lab0[rng.choice(n, 300)]
    lab1 = _labels_from_groups([np.flatnonzero(lab1 == v).tolist() for v in np.unique(lab1)], n)
    for mm in (1, 20, 60):
        m = metrics.cluster_metrics(lab0, lab1, min_members=mm, n_bins=0)
        ref = skm.adjusted_rand_score(_as_halo_partition(lab0, mm), _as_halo_partition(lab1, mm))
        assert m["ari"] == pytest.approx(ref, abs=1e-12)
        assert m["tp"] + m["fp"] + m["fn"] + m["tn"] == n * (n - 1) // 2


def test_pair_counts_and_iou_by_brute_force():
    rng = np.random.default_rng(7)
    n = 60
    lab0 = _random_partition(rng, n, 5)
    lab1 = _random_partition(rng, n, 4)
    mm = 8
    m = metrics.cluster_metrics(lab0, lab1, min_members=mm, n_bins=0)
    h0 = _as_halo_partition(lab0, mm)
    h1 = _as_halo_partition(lab1, mm)
    tp = fp = fn = tn = 0
    for a, b in itertools.combinations(range(n), 2):
        s0, s1 = h0[a] == h0[b], h1[a] == h1[b]
        tp += s0 and s1
        fn += s0 and not s1
        fp += s1 and not s0
        tn += not s0 and not s1
    assert (m["tp"], m["fp"], m["fn"], m["tn"]) == (tp, fp, fn, tn)
    size0 = np.bincount(lab0, minlength=n)
    size1 = np.bincount(lab1, minlength=n)
    halos0 = [set(np.flatnonzero(lab0 == i)) for i in range(n) if size0[i] >= mm]
    halos1 = [set(np.flatnonzero(lab1 == j)) for j in range(n) if size1[j] >= mm]
    num = sum(len(H) * max([len(H & G) / len(H | G) for G in halos1] + [0.0]) for H in halos0)
    assert m["mwm_iou"] == pytest.approx(num / sum(len(H) for H in halos0), abs=1e-12)


def test_identical_labelings_score_one_and_hmf_is_a_histogram():
    rng = np.random.default_rng(3)
    n = 20000
    lab = _random_partition(rng, n, 400)
    m = metrics.cluster_metrics(lab, lab, min_members=20, n_bins=12, volume=2.0)
    assert m["ari"] == 1.0 and m["mwm_iou"] == 1.0 and m["fp"] == 0 and m["fn"] == 0
    assert m["hmf0"] == m["hmf1"]
    sizes = np.bincount(lab, minlength=n)
    halo_sizes = sizes[sizes >= 20]
    counts, _ = np.histogram(np.log10(halo_sizes), bins=np.log10(np.array(m["bin_edges"])))
    width = np.log10(m["bin_edges"][1]) - np.log10(m["bin_edges"][0])
    assert np.allclose(np.array(m["hmf0"]) * 2.0 * width, counts)
    assert sum(counts) == len(halo_sizes) == m["halos0"]
