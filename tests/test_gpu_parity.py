"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer results (labels, vulnerable/active pairs, link flags, edit-stream
bytes) must be bit-exact.  Corrected coordinates must equal a float32
rounding of a value within 1e-6 * xi of the oracle's float64 result:
|gpu - (orig + delta_oracle)| <= ulp(gpu)/2 + 1e-6 xi.

The projected Adam iteration can be ill-conditioned: Adam's normalised step
turns a last-bit difference in a gradient near its epsilon into a visible
move, and long runs amplify it further.  Every compared case first shows that
it is well conditioned at the GPU's precision: the oracle agrees with itself
to 1e-7 xi under reversed pair order and under a 1e-13 relative change of the
step size (the double-float path rounds at about 2^-44 per operation).  The
converged MD runs (about 100 Adam steps) fail that test -- a 1e-13 change of
the step moves the oracle by 2e-5 xi (quantizer) and 4e-4 xi (Morton
baseline) -- and so does the 32^3 HACC-shaped box at eps = 0.5 b (HF) at
convergence.  Converged coordinates are therefore compared where the answer
is well conditioned, and after a fixed number of replayed iterations
elsewhere; every converged run, in every mode, is also checked through the
invariants the method guarantees (membership, box, zero untightened loss
after decoding).
"""
import numpy as np
import pytest

import oracle
from paper_2604_18801_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-6


def dev(a, d):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(d)


def ragged_points(n, seed, periodic=True):
    rng = np.random.default_rng(seed)
    c = rng.random((5, 3))
    P = c[rng.integers(0, 5, n)] + 0.02 * rng.standard_normal((n, 3))
    if periodic:
        P = np.mod(P, 1.0)
    P = np.minimum(P.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))
    return np.ascontiguousarray(P)


def workloads():
    out = {
        "cosmo4096": synth.tiny_cosmo(seed=1, n=4096),
        "md300": synth.md_box(n_clusters=300, eps_over_b=0.3, seed=5),
        "fluid20k": synth.fluid_box(n=20000, eps_over_b=0.5, seed=3),
        "hacc32k": synth.hacc_box(eps_over_b=0.5, n=32 ** 3, seed=4),
    }
    # the same problems reconstructed by the Morton-order baseline (Sec. 4.1)
    for k in ("cosmo4096", "md300", "hacc32k", "fluid20k"):
        out[k + "_morton"] = synth.with_base(out[k], "morton")
    return out


W = None


def W_(name):
    global W
    if W is None:
        W = workloads()
    return W[name]


# ----------------------------------------------------------------- labels
@pytest.mark.parametrize("name", ["cosmo4096", "md300", "fluid20k", "hacc32k"])
def test_fof_labels_bit_exact(cuda, name):
    import paper_2604_18801_gb300 as pc
    w = W_(name)
    lab, nc = pc.fof_labels(dev(w.orig, cuda), w.params())
    ref, _, nh = oracle.fof_labels(w.orig, **w.params())
    assert nc == nh
    assert np.array_equal(lab.cpu().numpy(), ref)


@pytest.mark.parametrize("n", [2, 3, 255, 257, 777, 5000])
def test_fof_labels_ragged_sizes(cuda, n):
    import paper_2604_18801_gb300 as pc
    P = ragged_points(n, seed=n)
    prm = dict(b=0.01, xi=0.002, periodic=1)
    lab, nc = pc.fof_labels(dev(P, cuda), prm)
    ref, _, nh = oracle.fof_labels(P, **prm)
    assert nc == nh and np.array_equal(lab.cpu().numpy(), ref)


def test_fof_labels_degenerate_coincident_points(cuda):
    import paper_2604_18801_gb300 as pc
    P = np.full((1000, 3), 0.25, np.float32)
    lab, nc = pc.fof_labels(dev(P, cuda), dict(b=0.01, periodic=1))
    assert nc == 1 and np.all(lab.cpu().numpy() == 0)
    lab, nc = pc.fof_labels(dev(P, cuda), dict(b=0.01, periodic=0))
    assert nc == 1 and np.all(lab.cpu().numpy() == 0)


# ----------------------------------------------------------------- selection
@pytest.mark.parametrize("name", ["cosmo4096", "md300", "fluid20k", "hacc32k"])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_active_pairs_bit_exact(cuda, name, mode):
    import paper_2604_18801_gb300 as pc
    w = W_(name)
    prm = w.params(mode=mode)
    cons = pc.select_constraints(dev(w.orig, cuda), prm)
    i, j, lk = (t.cpu().numpy() for t in cons.pairs())
    ai, aj, al, nv = oracle.select(w.orig, **prm)
    assert cons.stats["n_vulnerable"] == nv
    assert cons.stats["n_active"] == len(ai)
    assert np.array_equal(i.astype(np.uint32), ai)
    assert np.array_equal(j.astype(np.uint32), aj)
    assert np.array_equal(lk, al)


# ----------------------------------------------------------------- correction
def _check_coords(gpu, w, delta, editable, iters):
    g = gpu.astype(np.float64)
    if iters == 0:
        assert np.array_equal(gpu, w.recon)
        return
    assert np.array_equal(gpu[~editable], w.recon[~editable])
    exact = w.orig[editable].astype(np.float64) + delta[editable]
    half_ulp = 0.5 * np.spacing(np.abs(gpu[editable])).astype(np.float64)
    err = np.abs(g[editable] - exact) - half_ulp
    assert err.max() <= TOL * w.xi, f"max excess {err.max() / w.xi:.3e} xi"


def _well_conditioned(w, prm, ai, aj, al, delta):
    """The case is well conditioned at the GPU's precision: the oracle agrees with itself to
    1e-7 xi when its pair order is reversed, and when its step size is scaled by 1 + 1e-13
    (a relative perturbation of each step of the size of the double-float path's
    rounding, about 2^-44 per operation)."""
    _, d_rev, _, _ = oracle.pgd(w.orig, w.recon, ai[::-1], aj[::-1], al[::-1], **prm)
    _, d_eps, _, _ = oracle.pgd(w.orig, w.recon, ai, aj, al, **dict(prm, alpha_rel=0.2 * (1 + 1e-13)))
    return max(np.abs(delta - d_rev).max(), np.abs(delta - d_eps).max()) <= 1e-7 * w.xi


@pytest.mark.parametrize("name", ["cosmo4096", "cosmo4096_morton"])
def test_correct_halo_forest_converged_parity(cuda, name):
    import paper_2604_18801_gb300 as pc
    w = W_(name)
    prm = w.params(mode=2)
    corr, st, code = pc.correct(dev(w.orig, cuda), dev(w.recon, cuda), prm)
    assert code == 0 and st["converged"] == 1
    ai, aj, al, _ = oracle.select(w.orig, **prm)
    ocorr, delta, ed, ost = oracle.pgd(w.orig, w.recon, ai, aj, al, **prm)
    assert _well_conditioned(w, prm, ai, aj, al, delta)
    assert st["iters"] == ost["iters"] and st["viol0"] == ost["viol0"] and st["n_editable"] == ost["n_editable"]
    _check_coords(corr.cpu().numpy(), w, delta, ed, st["iters"])


@pytest.mark.parametrize("name,mode,R", [("cosmo4096", 0, 10), ("cosmo4096", 1, 10), ("cosmo4096", 0, 30),
                                         ("cosmo4096", 2, 5), ("md300", 2, 20), ("hacc32k", 2, 3),
                                         ("hacc32k", 0, 3), ("hacc32k", 1, 5), ("fluid20k", 1, 10),
                                         ("fluid20k", 0, 10), ("fluid20k", 2, 20),
                                         ("cosmo4096_morton", 0, 10), ("md300_morton", 2, 20),
                                         ("hacc32k_morton", 0, 3), ("hacc32k_morton", 1, 5),
                                         ("hacc32k_morton", 2, 3), ("fluid20k_morton", 1, 10)])
def test_correct_replayed_iterations_parity(cuda, name, mode, R):
    import paper_2604_18801_gb300 as pc
    w = W_(name)
    prm = w.params(mode=mode, replay_iters=R)
    corr, st, code = pc.correct(dev(w.orig, cuda), dev(w.recon, cuda), prm)
    assert st["iters"] == R
    ai, aj, al, _ = oracle.select(w.orig, **prm)
    _, delta, ed, ost = oracle.pgd(w.orig, w.recon, ai, aj, al, **prm)
    assert _well_conditioned(w, prm, ai, aj, al, delta)
    assert ost["iters"] == R and st["viol0"] == ost["viol0"]
    _check_coords(corr.cpu().numpy(), w, delta, ed, R)


@pytest.mark.parametrize("name,mode,R", [("cosmo4096", 0, 16), ("hacc32k", 2, 16), ("fluid20k", 1, 16),
                                         ("hacc32k_morton", 2, 16)])
def test_stall_resets_parity(cuda, name, mode, R):
    # stall_patience = 1 makes the stall rule fire early (patience 1, 2, 4, ...): the GPU's
    # reset path (light and heavy rows) against the oracle's, on cases where the resets
    # move the offsets by a sizeable fraction of xi
    import paper_2604_18801_gb300 as pc
    w = W_(name)
    prm = w.params(mode=mode, replay_iters=R, stall_patience=1)
    corr, st, code = pc.correct(dev(w.orig, cuda), dev(w.recon, cuda), prm)
    assert st["iters"] == R
    ai, aj, al, _ = oracle.select(w.orig, **prm)
    _, delta, ed, ost = oracle.pgd(w.orig, w.recon, ai, aj, al, **prm)
    _, plain, _, _ = oracle.pgd(w.orig, w.recon, ai, aj, al, **dict(prm, stall_patience=0))
    assert np.abs(delta - plain).max() > 0.1 * w.xi
    assert _well_conditioned(w, prm, ai, aj, al, delta)
    _check_coords(corr.cpu().numpy(), w, delta, ed, R)


@pytest.mark.parametrize("name", ["md300", "md300_morton"])
def test_ill_conditioned_converged_cases_are_detected(name):
    # converged HF on the MD clusters (about 100 Adam steps): a 1e-13 relative change of
    # the step size moves the oracle's own offsets by more than 1e-7 xi, so these runs are
    # checked by their invariants (test_correct_converged_invariants), not compared
    w = W_(name)
    prm = w.params(mode=2)
    ai, aj, al, _ = oracle.select(w.orig, **prm)
    _, delta, _, _ = oracle.pgd(w.orig, w.recon, ai, aj, al, **prm)
    assert not _well_conditioned(w, prm, ai, aj, al, delta)


def test_ill_conditioned_case_is_detected():
    # md300 in VP mode: reversing the float64 pair order alone moves the oracle by > 1e-7 xi
    # within 3 iterations, so no pair of implementations can be held to 1e-6 xi there.
    w = W_("md300")
    prm = w.params(mode=0, replay_iters=3)
    ai, aj, al, _ = oracle.select(w.orig, **prm)
    _, d1, _, _ = oracle.pgd(w.orig, w.recon, ai, aj, al, **prm)
    _, d2, _, _ = oracle.pgd(w.orig, w.recon, ai[::-1], aj[::-1], al[::-1], **prm)
    assert np.abs(d1 - d2).max() > 1e-7 * w.xi


@pytest.mark.parametrize("name,mode", [("cosmo4096", 0), ("cosmo4096", 1), ("fluid20k", 0), ("md300", 1),
                                       ("hacc32k", 0), ("hacc32k", 2), ("fluid20k", 2),
                                       ("hacc32k_morton", 0), ("hacc32k_morton", 1), ("hacc32k_morton", 2),
                                       ("md300_morton", 0), ("fluid20k_morton", 2), ("md300", 2),
                                       ("md300_morton", 2)])
def test_correct_converged_invariants(cuda, name, mode):
    import paper_2604_18801_gb300 as pc
    w = W_(name)
    prm = w.params(mode=mode)
    o, r = dev(w.orig, cuda), dev(w.recon, cuda)
    corr, st, code = pc.correct(o, r, prm)
    assert code == 0 and st["converged"] == 1 and st["viol_final"] == 0
    stream = pc.encode_edits(r, corr, prm)
    dec = pc.apply_edits(r, stream).cpu().numpy()
    assert np.abs(dec.astype(np.float64) - w.orig).max() <= w.xi
    lab0, _, _ = oracle.fof_labels(w.orig, **prm)
    lab1, _, _ = oracle.fof_labels(dec, **prm)
    assert np.array_equal(lab0, lab1)
    ai, aj, al, _ = oracle.select(w.orig, **prm)
    assert oracle.count_flips(dec, ai, aj, al, **prm) == 0


# ----------------------------------------------------------------- edit stream
@pytest.mark.parametrize("m_bits", [8, 16, 32, 12])
def test_encode_decode_bit_exact(cuda, m_bits):
    import torch
    import paper_2604_18801_gb300 as pc
    w = W_("md300")
    prm = w.params(mode=2, m_bits=m_bits)
    o, r = dev(w.orig, cuda), dev(w.recon, cuda)
    corr, st, _ = pc.correct(o, r, prm)
    c = corr.cpu().numpy()
    s = pc.encode_edits(r, corr, prm)
    ref = oracle.encode(w.recon, c, **prm)
    assert bytes(s.cpu().numpy()) == ref
    dec = pc.apply_edits(r, s).cpu().numpy()
    assert np.array_equal(dec, oracle.decode(w.recon, ref))
    # a stream written by the oracle decodes identically on the GPU
    s2 = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).to(cuda)
    assert np.array_equal(pc.apply_edits(r, s2).cpu().numpy(), dec)


def test_malformed_stream_rejected(cuda):
    import torch
    import paper_2604_18801_gb300 as pc
    w = W_("md300")
    r = dev(w.recon, cuda)
    s = pc.encode_edits(r, r, w.params())
    bad = s.clone()
    bad[0] = ord("X")
    with pytest.raises(pc.PcError) as e:
        pc.apply_edits(r, bad)
    assert e.value.code == -5
    with pytest.raises(pc.PcError):
        pc.apply_edits(r, s[:40].contiguous())


def test_input_errors(cuda):
    import paper_2604_18801_gb300 as pc
    w = W_("md300")
    bad = w.recon.copy()
    bad[7, 1] = w.orig[7, 1] + np.float32(2 * w.xi)
    with pytest.raises(pc.PcError) as e:
        pc.correct(dev(w.orig, cuda), dev(bad, cuda), w.params())
    assert e.value.code == -2
    nan = w.orig.copy()
    nan[3, 0] = np.nan
    with pytest.raises(pc.PcError) as e:
        pc.fof_labels(dev(nan, cuda), w.params())
    assert e.value.code == -1


def test_zero_violations_zero_iterations(cuda):
    import paper_2604_18801_gb300 as pc
    g = np.arange(6) * 0.45
    orig = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3).astype(np.float32)
    rng = np.random.default_rng(0)
    recon = (orig + rng.uniform(-0.001, 0.001, orig.shape)).astype(np.float32)
    prm = dict(b=1.0, xi=0.003, periodic=0)
    o, r = dev(orig, cuda), dev(recon, cuda)
    corr, st, code = pc.correct(o, r, prm)
    assert code == 0 and st["iters"] == 0 and st["n_vulnerable"] > 0
    assert np.array_equal(corr.cpu().numpy(), recon)
    s = pc.encode_edits(r, corr, prm).cpu().numpy()
    assert len(s) == 64 + (len(orig) + 7) // 8 and not s[64:].any()


def test_results_are_deterministic(cuda):
    import paper_2604_18801_gb300 as pc
    w = W_("hacc32k")
    prm = w.params(mode=0)
    o, r = dev(w.orig, cuda), dev(w.recon, cuda)
    a, sa, _ = pc.correct(o, r, prm)
    b, sb, _ = pc.correct(o, r, prm)
    assert sa["iters"] == sb["iters"] and np.array_equal(a.cpu().numpy(), b.cpu().numpy())
