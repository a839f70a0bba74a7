"""The Morton-order baseline of Sec. 4.1, used as a second base-compressor stand-in
(an input generator, not part of the method): its visiting order, its closed-loop
first-order prediction and its bound, checked against a per-particle loop written out
here on a small box."""
import numpy as np
import pytest

from paper_2604_18801_gb300 import synth


def _morton_key(x, cell, lo, ncell):
    # per particle: cell row-major, then the 10-bit-per-axis interleaved code (x highest)
    keys = []
    for i, p in enumerate(x.astype(np.float64)):
        c = [min(max(int(np.floor((p[a] - lo[a]) / cell)), 0), ncell[a] - 1) for a in range(3)]
        f = [min(max(int(((p[a] - lo[a]) / cell - c[a]) * 1024.0), 0), 1023) for a in range(3)]
        code = 0
        for bit in range(9, -1, -1):
            for a in range(3):
                code = (code << 1) | ((f[a] >> bit) & 1)
        keys.append(((c[0] * ncell[1] + c[1]) * ncell[2] + c[2], code, i))
    return keys


def test_morton_baseline_matches_a_per_particle_loop():
    rng = np.random.default_rng(11)
    x = (rng.random((3000, 3)) * [1.0, 0.5, 0.5]).astype(np.float32)
    eps, cell, lo, hi = 1e-3, 0.125, (0.0, 0.0, 0.0), (1.0, 0.5, 0.5)
    got = synth.morton_recon(x, eps, cell, lo, hi)
    ncell = [8, 4, 4]
    order = [k[2] for k in sorted(_morton_key(x, cell, lo, ncell))]
    cells = {k[2]: k[0] for k in _morton_key(x, cell, lo, ncell)}
    want = np.empty_like(x)
    prev_cell, prev = None, None
    for i in order:
        if cells[i] != prev_cell:
            want[i] = x[i]                        # first particle of a cell: exact
        else:
            for a in range(3):
                p = float(prev[a])
                v = np.float32(p + 2 * eps * round((float(x[i, a]) - p) / (2 * eps)))
                if abs(float(v) - float(x[i, a])) > eps:
                    v = np.nextafter(v, x[i, a])
                want[i, a] = v
        prev_cell, prev = cells[i], want[i]
    assert np.array_equal(got, want)


@pytest.mark.parametrize("gen", ["hacc", "md", "fluid"])
def test_morton_baseline_bound_and_error_structure(gen):
    w = {"hacc": lambda: synth.hacc_box(eps_over_b=0.5, n=32 ** 3, seed=4),
         "md": lambda: synth.md_box(n_clusters=300, eps_over_b=0.3, seed=5),
         "fluid": lambda: synth.fluid_box(n=20000, eps_over_b=0.5, seed=3)}[gen]()
    m = synth.with_base(w, "morton")
    e = (m.recon.astype(np.float64) - w.orig) / w.xi
    assert np.abs(e).max() <= 1.0
    # unlike the global quantizer, the reconstruction is not on the 2 xi lattice ...
    step = 2 * w.xi
    on_lattice = np.abs(m.recon / step - np.round(m.recon / step)) < 1e-3
    assert on_lattice.mean() < 0.05
    # ... and its errors spread over [-xi, xi] (a few percent exact: the cells' anchors)
    assert (e == 0).mean() < 0.05
    hist = np.histogram(e, bins=4, range=(-1, 1))[0] / len(e.ravel())
    assert hist.min() > 0.15
