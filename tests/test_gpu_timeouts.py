"""PC_ETIMEOUT paths, exercised on the host without faulting or hanging the GPU.

* The PGD host loop gives up after a bounded number of iteration launches.  Every block
  stops by its last check, so the bound is never reached in a correct run;
  PC_PGD_LAUNCH_LIMIT (a host-side test hook) lowers it so that the loop runs out: the call
  fails with PC_ETIMEOUT, the launches already queued finish on the stream, and the context
  stays usable (the same call without the hook succeeds).
* pc_serve_wait with a 1 ms limit on a job that takes longer returns PC_ETIMEOUT with the
  job's current state; waiting again without a limit gives the finished job.
"""
import ctypes as C

import pytest

from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu


def test_pgd_launch_limit_gives_etimeout(cuda, monkeypatch):
    import torch
    import paper_2604_18801_gb300 as pc
    w = synth.tiny_cosmo(seed=1, n=4096)
    o, r = torch.from_numpy(w.orig).to(cuda), torch.from_numpy(w.recon).to(cuda)
    prm = w.params(mode=0)
    monkeypatch.setenv("PC_PGD_LAUNCH_LIMIT", "2")
    with pytest.raises(pc.PcError) as e:
        pc.correct(o, r, prm)
    assert e.value.code == -6
    monkeypatch.delenv("PC_PGD_LAUNCH_LIMIT")
    corr, st, code = pc.correct(o, r, prm)
    assert code == 0 and st["converged"] == 1 and st["iters"] > 8


def test_serve_wait_times_out_then_finishes(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    from paper_2604_18801_gb300 import _native
    w = synth.hacc_box(eps_over_b=0.1, mode="VP", seed=61, n=300000)
    o, r = torch.from_numpy(w.orig).to(cuda), torch.from_numpy(w.recon).to(cuda)
    with pc.Server(mem_budget=4 << 30) as srv:
        t = srv.submit(o, r, w.params())
        res = _native.JobResult()
        code = _native.lib().pc_serve_wait(srv.h, t, 1, C.byref(res))
        assert code == -6 and res.state in (0, 1)          # PC_ETIMEOUT; PENDING or RUNNING
        out, _, d = srv.result(t)
    assert d["state"] == "DONE" and d["status"] == 0
    alone, _, _ = pc.correct(o, r, w.params())
    assert torch.equal(out, alone)
