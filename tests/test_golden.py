"""Values the paper prints (tests/golden/paper_parameters.txt, each line cited) against
the defaults of the oracle, the workload generators and the metrics."""
import inspect
import os

import pytest

import oracle
from oracle import metrics
from paper_2604_18801_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_parameters.txt")


def _golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            name, value = line.split()[:2]
            out[name] = float(value)
    return out


def test_adam_defaults_follow_the_paper():
    g, d = _golden(), oracle.DEFAULTS
    assert d["beta1"] == g["adam_beta1"] and d["beta2"] == g["adam_beta2"]
    # step and epsilon scaled to xi with the paper's ratio
    assert d["alpha_rel"] / d["eps_rel"] == pytest.approx(g["adam_alpha"] / g["adam_eps"], rel=1e-12)


def test_linking_length_follows_eta():
    eta = _golden()["eta"]
    for n in (32 ** 3, 64 ** 3):
        assert synth.hacc_box(eps_over_b=0.1, n=n, seed=1).b == pytest.approx(eta / round(n ** (1 / 3)), rel=1e-12)
    assert synth.tiny_cosmo(seed=0, n=32768).b == pytest.approx(eta / 32, rel=1e-12)


def test_metric_defaults_follow_the_paper():
    g = _golden()
    sig = inspect.signature(metrics.cluster_metrics)
    assert sig.parameters["n_bins"].default == g["hmf_bins"]
    assert sig.parameters["min_members"].default == g["halo_min"]


def test_capped_benchmark_uses_the_papers_cap(monkeypatch):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    monkeypatch.syspath_prepend(root)
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", "--workload", "capped"])
    assert bench.parse().t_max == _golden()["iteration_cap"]
