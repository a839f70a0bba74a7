"""Serving form: jobs that arrive at different times are batched into cohorts that run side
by side; each job's corrected coordinates and edit stream must be bit-identical to
pc_correct and pc_encode_edits on that job alone, its decoded output must have the oracle's
friends-of-friends labels of the original, and memory and input errors end only the job
concerned."""
import time

import numpy as np
import pytest

import oracle
from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu


def _requests():
    return [synth.hacc_box(eps_over_b=0.5, mode="HF", seed=41, n=3000),
            synth.md_box(n_clusters=30, eps_over_b=0.3, mode="SC", seed=42),
            synth.tiny_cosmo(seed=43, n=4096, mode="VP"),
            synth.fluid_box(n=6000, eps_over_b=0.5, seed=44, mode="HF"),
            synth.hacc_box(eps_over_b=0.1, mode="VP", seed=45, n=20000),
            synth.md_box(n_clusters=9, eps_over_b=0.5, mode="VP", seed=46),
            synth.fluid_box(n=40000, eps_over_b=0.1, seed=47, mode="SC"),
            synth.hacc_box(eps_over_b=0.5, mode="SC", seed=48, n=8000)]


def test_each_result_is_the_same_alone_and_in_the_mix(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    ws = _requests()
    dev = [(torch.from_numpy(w.orig).to(cuda), torch.from_numpy(w.recon).to(cuda)) for w in ws]
    tickets = []
    with pc.Server(mem_budget=8 << 30, max_slots=64) as srv:
        # the first half together, the rest while those are running
        for k, (w, (o, r)) in enumerate(zip(ws, dev)):
            tickets.append(srv.submit(o, r, w.params(), stream_cap=64 + w.n + 12 * w.n))
            if k >= len(ws) // 2:
                time.sleep(0.003)
        results = [srv.result(t) for t in tickets]
        counters = srv.counters()
    assert counters["submitted"] == len(ws) and counters["finished"] == len(ws)
    assert max(d["cohort_jobs"] for _, _, d in results) > 1        # jobs really were batched
    for w, (o, r), (out, stream, d) in zip(ws, dev, results):
        assert d["state"] == "DONE" and d["status"] == 0, d
        assert d["done_ns"] >= d["start_ns"] >= d["submit_ns"] > 0
        alone, st, code = pc.correct(o, r, w.params())
        assert code == 0
        assert torch.equal(out, alone), w.name
        assert d["stats"]["iters"] == st["iters"] and d["stats"]["n_active"] == st["n_active"]
        assert torch.equal(stream, pc.encode_edits(r, alone, w.params())), w.name
        dec = pc.apply_edits(r, stream)
        assert float((dec.double() - o.double()).abs().max()) <= w.xi
        # membership of the served result against the oracle's labels
        lab0, _, _ = oracle.fof_labels(w.orig, **w.params(xi=0.0))
        lab1, _, _ = oracle.fof_labels(dec.cpu().numpy(), **w.params(xi=0.0))
        assert np.array_equal(lab0, lab1), w.name


def test_errors_end_only_the_job_concerned(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    good = synth.hacc_box(eps_over_b=0.1, mode="HF", seed=51, n=5000)
    bad = synth.hacc_box(eps_over_b=0.1, mode="HF", seed=52, n=5000)
    big = synth.hacc_box(eps_over_b=0.1, mode="HF", seed=53, n=200000)
    og, rg = torch.from_numpy(good.orig).to(cuda), torch.from_numpy(good.recon).to(cuda)
    ob = torch.from_numpy(bad.orig).to(cuda)
    rb = ob + 2.0 * bad.xi                                  # violates |recon - orig| <= xi
    obig, rbig = torch.from_numpy(big.orig).to(cuda), torch.from_numpy(big.recon).to(cuda)
    with pc.Server(mem_budget=16 << 20) as srv:             # 16 MiB: the large job can never fit
        t_bad = srv.submit(ob, rb, bad.params())
        t_big = srv.submit(obig, rbig, big.params())
        t_good = srv.submit(og, rg, good.params())
        r_bad, r_big = srv.wait(t_bad, 120000), srv.wait(t_big, 120000)
        out, _, r_good = srv.result(t_good)
        with pytest.raises(pc.PcError):
            srv.poll(987654321)
    assert r_bad["state"] == "ERROR" and r_bad["status"] == -2            # PC_EBOUND
    assert r_big["state"] == "ERROR" and r_big["status"] == -3            # PC_ENOMEM
    assert r_good["state"] == "DONE" and r_good["status"] == 0
    alone, _, _ = pc.correct(og, rg, good.params())
    assert torch.equal(out, alone)


def test_jobs_that_fit_only_one_at_a_time_both_finish(cuda):
    # Two jobs whose joint memory estimate exceeds the budget while each fits alone: the
    # cohort they were admitted in cannot proceed, so its jobs go back to the queue and run
    # in cohorts of their own (instead of both failing with PC_ENOMEM).
    import torch
    import paper_2604_18801_gb300 as pc
    ws = [synth.hacc_box(eps_over_b=0.1, mode="VP", seed=70 + k, n=100000) for k in range(2)]
    dev = [(torch.from_numpy(w.orig).to(cuda), torch.from_numpy(w.recon).to(cuda)) for w in ws]
    with pc.Server(mem_budget=8 << 30) as probe:
        probe.result(probe.submit(dev[0][0], dev[0][1], ws[0].params()))
        one = probe.counters()["peak_bytes"]
    with pc.Server(mem_budget=int(1.3 * one)) as srv:
        tickets = [srv.submit(o, r, w.params()) for w, (o, r) in zip(ws, dev)]
        results = [srv.result(t) for t in tickets]
    for w, (o, r), (out, _, d) in zip(ws, dev, results):
        assert d["state"] == "DONE" and d["status"] == 0, d
        assert d["cohort_jobs"] == 1
        alone, _, _ = pc.correct(o, r, w.params())
        assert torch.equal(out, alone)
