"""Seeded synthetic particle workloads.

This module only draws inputs: original float32 coordinates, the parameters of
each workload, and the base-compressor stand-in that produces the lossy
reconstruction. It contains none of the correction method's arithmetic, so both
the CUDA path and the CPU oracle can be fed from it.

The datasets of the paper (HACC cosmology, EXAALT molecular dynamics, FPM
fluid; Table 1, Sec. 4.1) are not available; these generators stand in for
them with the shapes, densities and structure described there:

* ``cosmo_box``  -- periodic unit box, Gaussian halos with power-law member
  counts plus a uniform background (HACC-like).  The linking length follows
  Sec. 2.4: b = eta * mean spacing with eta = 0.2.
* ``md_clusters`` -- compact random-walk clusters of atoms with step 0.8 b and a
  minimum gap of 1.2 b between clusters, non-periodic cube (EXAALT-like).
* ``fluid_box`` -- 2:1:1 non-periodic box, rejection-sampled density
  1 + 0.8 sin(2 pi x) cos(2 pi y) (FPM-like).
* ``quantize_recon`` -- the absolute-error quantizer x' = 2e*round(x/2e) used
  as the base compressor (|x' - x| <= e per coordinate).
* ``morton_recon`` -- the Morton-order baseline of Sec. 4.1: particles visited cell
  by cell in Morton order inside each cell, each coordinate predicted by the
  previous particle's reconstruction (first order) and the residual quantized in
  bins of 2e; the first particle of a cell is kept exact.  Its errors lie on a
  lattice whose offset changes from cell to cell.  ``with_base`` swaps it in,
  with cells holding 64 particles on average.

Every function takes an explicit seed and returns float32 arrays of shape
(N, 3), C-contiguous (x, y, z per particle).  Particle order is shuffled so
that ids carry no spatial locality.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Workload",
    "quantize_recon",
    "morton_recon",
    "with_base",
    "cosmo_box",
    "md_clusters",
    "fluid_box",
    "tiny_cosmo",
    "hacc_box",
    "md_box",
    "mixed_blocks",
    "serve_requests",
    "MODES",
]

MODES = {"VP": 0, "SC": 1, "HF": 2}

_ONE_BELOW = np.nextafter(np.float32(1.0), np.float32(0.0))


@dataclasses.dataclass
class Workload:
    """One correction problem: originals, reconstruction and parameters."""

    name: str
    orig: np.ndarray            # (N, 3) float32
    recon: np.ndarray           # (N, 3) float32, |recon - orig| <= xi per coordinate
    b: float                    # linking length
    xi: float                   # pointwise absolute error bound
    periodic: bool
    box_lo: tuple
    box_hi: tuple
    mode: str = "VP"
    aux: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.orig.shape[0])

    def params(self, **over) -> dict:
        p = dict(b=self.b, xi=self.xi, periodic=int(self.periodic),
                 box_lo=tuple(self.box_lo), box_hi=tuple(self.box_hi),
                 mode=MODES[self.mode])
        p.update(self.aux.get("params", {}))   # solver settings this input is run with
        p.update(over)
        return p


def quantize_recon(x: np.ndarray, eps: float) -> np.ndarray:
    """Base-compressor stand-in x' = 2 eps * round(x / 2 eps), per coordinate.

    Computed in float64 and rounded to float32.  Should float32 rounding push
    |x' - x| above eps, x' is moved one ulp toward x, so the bound holds exactly.
    """
    x64 = x.astype(np.float64)
    step = 2.0 * float(eps)
    q = step * np.round(x64 / step)
    r = q.astype(np.float32)
    bad = np.abs(r.astype(np.float64) - x64) > eps
    if np.any(bad):
        r[bad] = np.nextafter(r[bad], x[bad])
    assert np.all(np.abs(r.astype(np.float64) - x64) <= eps)
    return np.ascontiguousarray(r)


def _fix_bound(r: np.ndarray, x: np.ndarray, eps: float) -> np.ndarray:
    """Moves float32 values one ulp toward x where rounding broke |r - x| <= eps."""
    bad = np.abs(r.astype(np.float64) - x.astype(np.float64)) > eps
    if np.any(bad):
        r[bad] = np.nextafter(r[bad], x[bad])
    return r


def morton_order(x: np.ndarray, cell: float, lo, hi) -> np.ndarray:
    """Particle order of the Morton baseline: by cell (row-major over the grid of cubes
    of side ``cell`` from ``lo``), then by the 10-bit-per-axis Morton code of the
    position inside the cell, then by id."""
    x64 = x.astype(np.float64)
    lo = np.asarray(lo, np.float64)
    ncell = np.maximum(1, np.ceil((np.asarray(hi, np.float64) - lo) / cell)).astype(np.int64)
    c = np.clip(np.floor((x64 - lo) / cell).astype(np.int64), 0, ncell - 1)
    lin = (c[:, 0] * ncell[1] + c[:, 1]) * ncell[2] + c[:, 2]
    f = np.clip(((x64 - lo) / cell - c) * 1024.0, 0, 1023).astype(np.int64)
    code = np.zeros(len(x), np.int64)
    for bit in range(10):
        for ax in range(3):
            code |= ((f[:, ax] >> bit) & 1) << (3 * bit + (2 - ax))
    return np.lexsort((np.arange(len(x)), code, lin)), lin


def morton_recon(x: np.ndarray, eps: float, cell: float, lo, hi) -> np.ndarray:
    """Morton-order baseline (Sec. 4.1) as a base-compressor stand-in.

    In the order of ``morton_order``, the first particle of each cell is kept exact;
    every later coordinate is predicted by the previous particle's reconstruction p
    and reconstructed as p + 2 eps * round((x - p) / (2 eps)) (float64, rounded to
    float32; a value that rounding moved beyond eps is moved one ulp back).  The loop
    runs over the rank inside a cell, vectorised across cells."""
    order, lin = morton_order(x, cell, lo, hi)
    xs = x[order]
    ls = lin[order]
    n = len(x)
    rs = np.empty_like(xs)
    first = np.ones(n, bool)
    first[1:] = ls[1:] != ls[:-1]
    start = np.maximum.accumulate(np.where(first, np.arange(n), 0))
    rank = np.arange(n) - start
    rs[first] = xs[first]
    step = 2.0 * float(eps)
    by_rank = np.argsort(rank, kind="stable")
    bounds = np.searchsorted(rank[by_rank], np.arange(int(rank.max()) + 2 if n else 1))
    for k in range(1, len(bounds) - 1):
        sel = by_rank[bounds[k]:bounds[k + 1]]
        p = rs[sel - 1].astype(np.float64)
        v = (p + step * np.round((xs[sel].astype(np.float64) - p) / step)).astype(np.float32)
        rs[sel] = _fix_bound(v, xs[sel], eps)
    out = np.empty_like(x)
    out[order] = rs
    assert np.all(np.abs(out.astype(np.float64) - x.astype(np.float64)) <= eps)
    return np.ascontiguousarray(out)


def with_base(w: "Workload", base: str, cell_particles: int = 64) -> "Workload":
    """The same workload with the reconstruction of another base-compressor stand-in:
    "quant" (the global quantizer) or "morton" (cubic cells holding ``cell_particles``
    particles on average)."""
    if base == "quant":
        return w
    if base != "morton":
        raise ValueError(f"unknown base compressor {base!r}")
    vol = float(np.prod(np.asarray(w.box_hi, np.float64) - np.asarray(w.box_lo, np.float64)))
    cell = (vol * cell_particles / max(1, w.n)) ** (1.0 / 3.0)
    recon = morton_recon(w.orig, w.xi, cell, w.box_lo, w.box_hi)
    # On this reconstruction plain Adam-PGD can settle in a local minimum of the
    # non-convex loss (at eps = 0.5 b it does on the 32^3 HACC-shaped box and the fluid
    # box); such inputs are run with the stall rule on (100 checks of patience).
    aux = dict(w.aux, params=dict(w.aux.get("params", {}), stall_patience=100))
    return dataclasses.replace(w, recon=recon, name=w.name + "_morton", aux=aux)


def _wrap_unit(x: np.ndarray) -> np.ndarray:
    """Wrap float64 coordinates into [0, 1) and round to float32 inside it."""
    y = np.mod(x, 1.0).astype(np.float32)
    return np.minimum(y, _ONE_BELOW)


def _rescale_counts(raw: np.ndarray, total: int) -> np.ndarray:
    """Scale integer-ish counts so they sum exactly to ``total`` (largest remainders)."""
    raw = raw.astype(np.float64)
    share = raw * (total / raw.sum())
    c = np.floor(share).astype(np.int64)
    rem = total - int(c.sum())
    if rem > 0:
        order = np.argsort(-(share - c), kind="stable")
        c[order[:rem]] += 1
    return c


def cosmo_box(n: int, n_halos: int, halo_frac: float, sigma_lo: float, sigma_hi: float,
              alpha: float, nmin: int, nmax: Optional[float], eps_over_b: float,
              seed: int, eta: float = 0.2, mode: str = "VP", name: str = "cosmo") -> Workload:
    """HACC-like periodic unit box.

    ``halo_frac`` of the particles sit in ``n_halos`` isotropic Gaussian halos
    whose widths are log-uniform in [sigma_lo, sigma_hi] and whose member
    counts follow a power law pdf ~ n^alpha from ``nmin`` (truncated at
    ``nmax`` when given), rescaled to the halo total; the rest are uniform.
    b = eta * (1/N)^(1/3) (Sec. 2.4), eps = eps_over_b * b.
    """
    rng = np.random.default_rng(seed)
    n_halo_tot = int(round(halo_frac * n))
    g = 1.0 + alpha  # exponent of the CDF integrand (alpha < -1)
    u = rng.random(n_halos)
    if nmax is None:
        raw = nmin * u ** (1.0 / g)
    else:
        a0, a1 = nmin ** g, float(nmax) ** g
        raw = (a0 + u * (a1 - a0)) ** (1.0 / g)
    counts = _rescale_counts(raw, n_halo_tot)
    centres = rng.random((n_halos, 3))
    if sigma_lo == sigma_hi:
        sig = np.full(n_halos, sigma_lo)
    else:
        sig = np.exp(rng.uniform(math.log(sigma_lo), math.log(sigma_hi), n_halos))
    reps = np.repeat(np.arange(n_halos), counts)
    pos_h = centres[reps] + sig[reps, None] * rng.standard_normal((n_halo_tot, 3))
    pos_b = rng.random((n - n_halo_tot, 3))
    pos = np.concatenate([pos_h, pos_b], axis=0)
    perm = rng.permutation(n)
    orig = np.ascontiguousarray(_wrap_unit(pos[perm]))
    b = eta * (1.0 / n) ** (1.0 / 3.0)
    xi = eps_over_b * b
    recon = quantize_recon(orig, xi)
    halo_of = np.concatenate([reps, np.full(n - n_halo_tot, -1)])[perm]
    return Workload(name=name, orig=orig, recon=recon, b=b, xi=xi, periodic=True,
                    box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 1.0), mode=mode,
                    aux={"halo_of": halo_of, "counts": counts})


def md_clusters(n_clusters: int, atoms: int, eps_over_b: float, seed: int, b: float = 1.0,
                step: float = 0.8, gap: float = 1.2, side: Optional[float] = None,
                mode: str = "HF", name: str = "md") -> Workload:
    """EXAALT-like non-periodic cube of compact clusters.

    Each cluster is a random walk of ``atoms`` atoms with fixed step
    ``step * b`` in uniformly random directions, placed at a uniform random
    centre; a cluster is rejected when any of its atoms lies within
    ``gap * b`` of an atom of an already placed cluster.  Because step < b
    and gap > b, the friends-of-friends components are exactly the clusters.
    The cube side defaults to 555 b for 40,000 clusters and scales with the
    cube root of the cluster count (about 35% of the volume covered).
    """
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    if side is None:
        side = 555.0 * b * (n_clusters / 40000.0) ** (1.0 / 3.0)
    acc = []                      # accepted clusters, each (atoms, 3) float64
    tree = None
    tree_n = 0
    pending = []                  # accepted since the last tree rebuild
    batch = max(64, min(4096, n_clusters // 8 or 1))
    while len(acc) < n_clusters:
        m = batch
        d = rng.standard_normal((m, atoms - 1, 3))
        d *= (step * b) / np.linalg.norm(d, axis=2, keepdims=True)
        walk = np.concatenate([np.zeros((m, 1, 3)), np.cumsum(d, axis=1)], axis=1)
        walk -= walk.mean(axis=1, keepdims=True)
        cand = walk + rng.random((m, 1, 3)) * side
        ok = np.ones(m, dtype=bool)
        if tree is not None:
            dist, _ = tree.query(cand.reshape(-1, 3), k=1, distance_upper_bound=gap * b)
            ok &= ~np.isfinite(dist.reshape(m, atoms)).any(axis=1)
        # conflicts within this batch and with clusters accepted since the rebuild
        flat = cand.reshape(-1, 3)
        bt = cKDTree(flat)
        conflict = [set() for _ in range(m)]
        for i, j in bt.query_pairs(gap * b, output_type="ndarray"):
            ci, cj = i // atoms, j // atoms
            if ci != cj:
                conflict[ci].add(cj)
                conflict[cj].add(ci)
        chosen = []
        for k in range(m):
            if not ok[k] or len(acc) + len(chosen) >= n_clusters:
                continue
            if any(c in conflict[k] for c in chosen):
                continue
            chosen.append(k)
        if pending and chosen:
            pt = cKDTree(np.concatenate(pending, axis=0))
            keep = []
            for k in chosen:
                dk, _ = pt.query(cand[k], k=1, distance_upper_bound=gap * b)
                if not np.isfinite(dk).any():
                    keep.append(k)
            chosen = keep
        for k in chosen:
            acc.append(cand[k])
            pending.append(cand[k])
        if sum(len(p) for p in pending) > max(200000, tree_n):
            allpts = np.concatenate(acc, axis=0)
            tree = cKDTree(allpts)
            tree_n = len(allpts)
            pending = []
    pos = np.concatenate(acc[:n_clusters], axis=0)
    n = pos.shape[0]
    cluster = np.repeat(np.arange(n_clusters), atoms)
    perm = rng.permutation(n)
    orig = np.ascontiguousarray(pos[perm].astype(np.float32))
    xi = eps_over_b * b
    recon = quantize_recon(orig, xi)
    lo = tuple(float(v) for v in orig.min(axis=0))
    hi = tuple(float(v) for v in orig.max(axis=0))
    return Workload(name=name, orig=orig, recon=recon, b=b, xi=xi, periodic=False,
                    box_lo=lo, box_hi=hi, mode=mode, aux={"cluster_of": cluster[perm]})


def fluid_box(n: int, eps_over_b: float = 0.1, seed: int = 5, mode: str = "SC", name: str = "fluid") -> Workload:
    """FPM-like 2:1:1 non-periodic box with density 1 + 0.8 sin(2 pi x) cos(2 pi y).

    Points are drawn by rejection sampling; b = 0.2 (V/N)^(1/3) with V = 2.
    """
    rng = np.random.default_rng(seed)
    out = []
    have = 0
    while have < n:
        m = int((n - have) * 1.9) + 1024
        p = rng.random((m, 3)) * np.array([2.0, 1.0, 1.0])
        rho = 1.0 + 0.8 * np.sin(2 * np.pi * p[:, 0]) * np.cos(2 * np.pi * p[:, 1])
        keep = p[rng.random(m) * 1.8 < rho]
        out.append(keep)
        have += len(keep)
    pos = np.concatenate(out, axis=0)[:n]
    orig = np.ascontiguousarray(pos.astype(np.float32))
    b = 0.2 * (2.0 / n) ** (1.0 / 3.0)
    xi = eps_over_b * b
    recon = quantize_recon(orig, xi)
    lo = tuple(float(v) for v in orig.min(axis=0))
    hi = tuple(float(v) for v in orig.max(axis=0))
    return Workload(name=name, orig=orig, recon=recon, b=b, xi=xi, periodic=False,
                    box_lo=lo, box_hi=hi, mode=mode)


# --- the named workloads -----------------------------------------------------

def tiny_cosmo(seed: int = 0, n: int = 32768, mode: str = "VP") -> Workload:
    """32^3 periodic unit box, 60% in 64 halos (sigma 0.01, counts ~ n^-2, min 20),
    b = 0.2/32, eps = 0.25 b, vulnerable-pair mode."""
    return cosmo_box(n=n, n_halos=max(1, round(64 * n / 32768)), halo_frac=0.6,
                     sigma_lo=0.01, sigma_hi=0.01, alpha=-2.0, nmin=20, nmax=None,
                     eps_over_b=0.25, seed=seed, mode=mode, name=f"cosmo{n}_eps0.25b_{mode}")


def hacc_box(eps_over_b: float = 0.1, mode: str = "HF", seed: int = 1, n: int = 256 ** 3,
             ref_n: int = 256 ** 3) -> Workload:
    """HACC-shaped periodic unit box: 20,000 halos per 256^3 particles holding 55%,
    sigma log-uniform [0.002, 0.02], counts ~ n^-1.9 truncated to [20, 0.001 * 256^3],
    b = 0.2 / N^(1/3).

    For n < ref_n the box stands for a sub-volume of the ref_n-particle box scaled to
    unit side: the halo count scales with n / ref_n and the halo widths scale with
    the mean spacing, (ref_n / n)^(1/3), so halo widths in units of b, the member-count
    law and the halo fraction are those of the full box."""
    nh = max(1, round(20000 * n / ref_n))
    zoom = (ref_n / n) ** (1.0 / 3.0)
    return cosmo_box(n=n, n_halos=nh, halo_frac=0.55, sigma_lo=0.002 * zoom, sigma_hi=0.02 * zoom,
                     alpha=-1.9, nmin=20, nmax=0.001 * ref_n, eps_over_b=eps_over_b,
                     seed=seed, mode=mode, name=f"hacc{n}_eps{eps_over_b:g}b_{mode}")


def md_box(n_clusters: int = 40000, eps_over_b: float = 0.3, mode: str = "HF", seed: int = 2) -> Workload:
    """MD-like cube: clusters of 100 atoms, random-walk step 0.8 b, gap 1.2 b, b = 1."""
    return md_clusters(n_clusters=n_clusters, atoms=100, eps_over_b=eps_over_b, seed=seed,
                       mode=mode, name=f"md{n_clusters * 100}_eps{eps_over_b:g}b_{mode}")


def mixed_blocks(n_blocks: int = 512, seed: int = 3, lo: float = 1e3, hi: float = 1e6,
                 kinds=("hacc", "md")) -> list:
    """Independent blocks of log-uniform size drawn from the given generators, each
    with eps in {0.1 b, 0.5 b} and a mode drawn from VP/SC/HF.  Block k uses seed
    ``1000 * seed + k``."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_blocks)).astype(np.int64)
    eps = rng.choice([0.1, 0.5], n_blocks)
    modes = rng.choice(["VP", "SC", "HF"], n_blocks)
    out = []
    for k in range(n_blocks):
        kind = kinds[k % len(kinds)]
        s = 1000 * seed + k
        nk = int(sizes[k])
        if kind == "hacc":
            w = hacc_box(eps_over_b=float(eps[k]), mode=str(modes[k]), seed=s, n=nk)
        elif kind == "md":
            w = md_box(n_clusters=max(1, nk // 100), eps_over_b=float(eps[k]), mode=str(modes[k]), seed=s)
        else:
            w = fluid_box(n=nk, eps_over_b=float(eps[k]), seed=s, mode=str(modes[k]))
        out.append(w)
    return out


def serve_requests(n_req: int = 2000, seed: int = 4, lo: float = 1e3, hi: float = 2e6):
    """Request sizes (log-uniform), generator kinds (hacc / md / fluid, a third each),
    eps and mode per request.  Returns a list of dicts; the particles of request k
    are drawn lazily with seed ``1000 * seed + k`` through :func:`make_request`."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_req)).astype(np.int64)
    kinds = np.array(["hacc", "md", "fluid"])[rng.integers(0, 3, n_req)]
    eps = rng.choice([0.1, 0.5], n_req)
    modes = rng.choice(["VP", "SC", "HF"], n_req)
    return [dict(k=k, n=int(sizes[k]), kind=str(kinds[k]), eps=float(eps[k]), mode=str(modes[k]),
                 seed=1000 * seed + k) for k in range(n_req)]


def make_request(spec: dict) -> Workload:
    kind, n, e, m, s = spec["kind"], spec["n"], spec["eps"], spec["mode"], spec["seed"]
    if kind == "hacc":
        return hacc_box(eps_over_b=e, mode=m, seed=s, n=n)
    if kind == "md":
        return md_box(n_clusters=max(1, n // 100), eps_over_b=e, mode=m, seed=s)
    return fluid_box(n=n, eps_over_b=e, seed=s, mode=m)
