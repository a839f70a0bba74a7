"""GB300-native cluster-preserving correction of lossy particle data.

Python face of the CUDA library ``libpc.so`` (C ABI in ``include/pc.h``).
Tensors live on the GPU (torch supplies device memory and streams); every
step of the method runs in the library's CUDA kernels:

* :func:`fof_labels`            -- friends-of-friends labels (Sec. 2.4)
* :func:`select_constraints`    -- vulnerable pairs and the active set A (Sec. 3.1-3.2)
* :func:`correct`               -- projected Adam descent on the tight loss (Alg. 1, Eq. 3)
* :func:`encode_edits` / :func:`apply_edits` -- edit stream and decoder (Sec. 3.3)
* :func:`correct_batch`         -- many independent blocks in one pass (batching layer)
* :class:`Server`               -- request loop with continuous batching (serving layer)
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _native
from ._native import PcError, make_params, struct_dict

__all__ = ["Context", "fof_labels", "select_constraints", "Constraints", "correct", "correct_detail", "correct_batch",
           "correct_multi",
           "encode_edits", "apply_edits", "huff_encode", "huff_decode", "Server", "autotune_cells", "cluster_metrics", "PcError", "make_params",
           "default_context"]

MODES = {"VP": 0, "SC": 1, "HF": 2}


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _xyz(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2
            and t.shape[1] == 3 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor of shape (N, 3)")
    return t


class Context:
    """A library context on one CUDA device (keeps pinned scratch and the device pool)."""

    def __init__(self, device: int = 0, arena_bytes: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        _native.check(_native.lib().pc_ctx_create(self.device, arena_bytes, C.byref(h)), "pc_ctx_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _native.lib().pc_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_ctx = {}


def default_context(device: int = 0) -> Context:
    if device not in _ctx:
        _ctx[device] = Context(device)
    return _ctx[device]


def _params(params) -> _native.Params:
    if isinstance(params, _native.Params):
        return params
    d = dict(params)
    if isinstance(d.get("mode"), str):
        d["mode"] = MODES[d["mode"]]
    return make_params(**d)


def fof_labels(xyz: torch.Tensor, params, ctx: Context = None):
    """Labels (int32, smallest id of the component) and the component count."""
    _xyz(xyz, "xyz")
    ctx = ctx or default_context(xyz.device.index)
    p = _params(params)
    lab = torch.empty(xyz.shape[0], dtype=torch.int32, device=xyz.device)
    nc = C.c_int64(0)
    _native.check(_native.lib().pc_fof_labels(ctx.h, xyz.data_ptr(), xyz.shape[0], C.byref(p), lab.data_ptr(),
                                              C.byref(nc), _stream(xyz.device)), "pc_fof_labels")
    return lab, int(nc.value)


class Constraints:
    """Active pairs selected on the device (owned by the library)."""

    def __init__(self, ctx: Context, h: C.c_void_p, stats: dict, n: int, device):
        self.ctx, self.h, self.stats, self.n, self.device = ctx, h, stats, n, device

    def pairs(self):
        """(i, j, link) as CUDA tensors in canonical order (i < j, sorted by (i, j))."""
        m = self.stats["n_active"]
        i = torch.empty(m, dtype=torch.int32, device=self.device)
        j = torch.empty(m, dtype=torch.int32, device=self.device)
        lk = torch.empty(m, dtype=torch.uint8, device=self.device)
        if m:
            _native.check(_native.lib().pc_constraints_copy(self.ctx.h, self.h, i.data_ptr(), j.data_ptr(),
                                                            lk.data_ptr(), _stream(self.device)),
                          "pc_constraints_copy")
        return i, j, lk

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _native.lib().pc_constraints_free(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def select_constraints(orig: torch.Tensor, params, ctx: Context = None) -> Constraints:
    _xyz(orig, "orig")
    ctx = ctx or default_context(orig.device.index)
    p = _params(params)
    h = C.c_void_p()
    st = _native.SelectStats()
    _native.check(_native.lib().pc_select_constraints(ctx.h, orig.data_ptr(), orig.shape[0], C.byref(p), C.byref(h),
                                                      C.byref(st), _stream(orig.device)), "pc_select_constraints")
    return Constraints(ctx, h, struct_dict(st), orig.shape[0], orig.device)


def correct(orig: torch.Tensor, recon: torch.Tensor, params, constraints: Constraints = None,
            out: torch.Tensor = None, ctx: Context = None):
    """Correction pass: returns (corrected (N,3) float32 CUDA tensor, stats dict, status code)."""
    _xyz(orig, "orig")
    _xyz(recon, "recon")
    if recon.shape != orig.shape:
        raise ValueError("orig and recon differ in shape")
    ctx = ctx or default_context(orig.device.index)
    p = _params(params)
    out = torch.empty_like(orig) if out is None else _xyz(out, "out")
    st = _native.CorrectStats()
    code = _native.lib().pc_correct(ctx.h, orig.data_ptr(), recon.data_ptr(), orig.shape[0], C.byref(p),
                                    constraints.h if constraints is not None else None, out.data_ptr(),
                                    C.byref(st), _stream(orig.device))
    _native.check(code, "pc_correct", allow_warn=True)
    return out, struct_dict(st), code


def correct_multi(orig: torch.Tensor, recon: torch.Tensor, params, b_list, out: torch.Tensor = None,
                  ctx: Context = None):
    """Correction for several linking lengths at once (the union of their active sets):
    returns (corrected (N,3) float32 CUDA tensor, stats dict, status code).  params' b is
    ignored; b_list holds 1 to 4 ascending lengths."""
    _xyz(orig, "orig")
    _xyz(recon, "recon")
    if recon.shape != orig.shape:
        raise ValueError("orig and recon differ in shape")
    ctx = ctx or default_context(orig.device.index)
    p = _params(params)
    bl = (C.c_double * len(b_list))(*[float(b) for b in b_list])
    out = torch.empty_like(orig) if out is None else _xyz(out, "out")
    st = _native.CorrectStats()
    code = _native.lib().pc_correct_multi(ctx.h, orig.data_ptr(), recon.data_ptr(), orig.shape[0], C.byref(p), bl,
                                          len(b_list), out.data_ptr(), C.byref(st), _stream(orig.device))
    _native.check(code, "pc_correct_multi", allow_warn=True)
    return out, struct_dict(st), code


def correct_detail(orig: torch.Tensor, recon: torch.Tensor, params, constraints: Constraints = None,
                   ctx: Context = None):
    """Correction pass with the float64 offsets and the loss history.

    Returns (corrected, delta (N,3) float64, hist_loss float64, hist_viol int64, stats, status); the
    histories are cut to the iterations run (iters + 1 entries)."""
    _xyz(orig, "orig")
    _xyz(recon, "recon")
    ctx = ctx or default_context(orig.device.index)
    p = _params(params)
    cap = (p.replay_iters if p.replay_iters >= 0 else p.t_max) + 1
    out = torch.empty_like(orig)
    delta = torch.empty((orig.shape[0], 3), dtype=torch.float64, device=orig.device)
    hl = torch.zeros(cap, dtype=torch.float64, device=orig.device)
    hv = torch.zeros(cap, dtype=torch.int64, device=orig.device)
    st = _native.CorrectStats()
    code = _native.lib().pc_correct_detail(ctx.h, orig.data_ptr(), recon.data_ptr(), orig.shape[0], C.byref(p),
                                           constraints.h if constraints is not None else None, out.data_ptr(),
                                           delta.data_ptr(), hl.data_ptr(), hv.data_ptr(), C.byref(st),
                                           _stream(orig.device))
    _native.check(code, "pc_correct_detail", allow_warn=True)
    d = struct_dict(st)
    k = d["iters"] + 1
    return out, delta, hl[:k], hv[:k], d, code


def correct_batch(orig: torch.Tensor, recon: torch.Tensor, sizes, params_list, out: torch.Tensor = None,
                  ctx: Context = None):
    """Batched correction of independent blocks concatenated along the rows of orig/recon.

    sizes[k] rows belong to block k (in order); params_list[k] are its parameters.
    Returns (corrected, [stats per block], status)."""
    _xyz(orig, "orig")
    _xyz(recon, "recon")
    if len(sizes) != len(params_list) or sum(int(n) for n in sizes) != orig.shape[0]:
        raise ValueError("sizes must match params_list and sum to the number of rows")
    ctx = ctx or default_context(orig.device.index)
    nb = len(sizes)
    blocks = (_native.Block * nb)()
    at = 0
    for k, (n, prm) in enumerate(zip(sizes, params_list)):
        blocks[k].offset = at
        blocks[k].n = int(n)
        blocks[k].params = _params(prm)
        at += int(n)
    out = torch.empty_like(orig) if out is None else _xyz(out, "out")
    stats = (_native.CorrectStats * nb)()
    code = _native.lib().pc_correct_batch(ctx.h, orig.data_ptr(), recon.data_ptr(), blocks, nb, out.data_ptr(), stats,
                                          _stream(orig.device))
    _native.check(code, "pc_correct_batch", allow_warn=True)
    return out, [struct_dict(st) for st in stats], code


def autotune_cells(xyz: torch.Tensor, params, ctx: Context = None):
    """Cell factor (cells per particle) with the fastest selection on this point set, and
    the time of each candidate {2, 4, 8, 16, 32} in ms.  Results never depend on it."""
    _xyz(xyz, "xyz")
    ctx = ctx or default_context(xyz.device.index)
    p = _params(params)
    best = C.c_int32(0)
    ms = (C.c_double * 5)()
    _native.check(_native.lib().pc_autotune_cells(ctx.h, xyz.data_ptr(), xyz.shape[0], C.byref(p), C.byref(best), ms,
                                                  _stream(xyz.device)), "pc_autotune_cells")
    return int(best.value), dict(zip((2, 4, 8, 16, 32), list(ms)))


def autotune(xyz: torch.Tensor, params, ctx: Context = None):
    """Pair-search knobs with the fastest selection on this point set: (cell_factor,
    dense_cell, times in ms of the 5 cell factors and the 4 dense-cell thresholds).
    Results never depend on either knob."""
    _xyz(xyz, "xyz")
    ctx = ctx or default_context(xyz.device.index)
    p = _params(params)
    q = _native.Params()
    ms = (C.c_double * 9)()
    _native.check(_native.lib().pc_autotune(ctx.h, xyz.data_ptr(), xyz.shape[0], C.byref(p), C.byref(q), ms,
                                            _stream(xyz.device)), "pc_autotune")
    times = {"cell_factor": dict(zip((2, 4, 8, 16, 32), list(ms)[:5])),
             "dense_cell": dict(zip((0, 32, 128, 512), list(ms)[5:]))}
    return int(q.cell_factor), int(q.dense_cell), times


def cluster_metrics(lab0: torch.Tensor, lab1: torch.Tensor, min_members: int = 20, n_bins: int = 50,
                    volume: float = 1.0, ctx: Context = None) -> dict:
    """ARI, MWM-IoU and halo mass functions (Sec. 4.1) between two labelings of the same
    particles (int32 CUDA tensors, "smallest id of the component" as fof_labels gives)."""
    for t, nm in ((lab0, "lab0"), (lab1, "lab1")):
        if not (t.is_cuda and t.dtype == torch.int32 and t.dim() == 1 and t.is_contiguous()):
            raise ValueError(f"{nm} must be a contiguous int32 CUDA vector")
    if lab0.shape != lab1.shape:
        raise ValueError("labelings differ in length")
    ctx = ctx or default_context(lab0.device.index)
    m = _native.ClusterMetrics()
    nb = max(0, int(n_bins))
    h0, h1, ed = (C.c_double * max(1, nb))(), (C.c_double * max(1, nb))(), (C.c_double * (nb + 1))()
    _native.check(_native.lib().pc_cluster_metrics(ctx.h, lab0.data_ptr(), lab1.data_ptr(), lab0.shape[0],
                                                   int(min_members), nb, float(volume), C.byref(m),
                                                   h0 if nb else None, h1 if nb else None, ed if nb else None,
                                                   _stream(lab0.device)), "pc_cluster_metrics")
    d = struct_dict(m)
    if nb:
        d["hmf0"], d["hmf1"], d["bin_edges"] = list(h0)[:nb], list(h1)[:nb], list(ed)
    return d


def encode_edits(recon: torch.Tensor, corrected: torch.Tensor, params, ctx: Context = None) -> torch.Tensor:
    """Edit stream (uint8 CUDA tensor, format v1 of include/pc.h)."""
    _xyz(recon, "recon")
    _xyz(corrected, "corrected")
    ctx = ctx or default_context(recon.device.index)
    p = _params(params)
    nb = C.c_size_t(0)
    s = _stream(recon.device)
    L = _native.lib()
    _native.check(L.pc_encode_edits(ctx.h, recon.data_ptr(), corrected.data_ptr(), recon.shape[0], C.byref(p), None,
                                    0, C.byref(nb), s), "pc_encode_edits")
    buf = torch.empty(nb.value, dtype=torch.uint8, device=recon.device)
    _native.check(L.pc_encode_edits(ctx.h, recon.data_ptr(), corrected.data_ptr(), recon.shape[0], C.byref(p),
                                    buf.data_ptr(), nb.value, C.byref(nb), s), "pc_encode_edits")
    return buf


def apply_edits(recon: torch.Tensor, stream: torch.Tensor, out: torch.Tensor = None, ctx: Context = None):
    """Decoder: reconstruction + dequantized edits (float32 CUDA tensor)."""
    _xyz(recon, "recon")
    if not (stream.is_cuda and stream.dtype == torch.uint8 and stream.is_contiguous()):
        raise ValueError("stream must be a contiguous uint8 CUDA tensor")
    ctx = ctx or default_context(recon.device.index)
    out = torch.empty_like(recon) if out is None else _xyz(out, "out")
    _native.check(_native.lib().pc_apply_edits(ctx.h, recon.data_ptr(), recon.shape[0], stream.data_ptr(),
                                               stream.numel(), out.data_ptr(), _stream(recon.device)),
                  "pc_apply_edits")
    return out


def _huff(fn: str, data: torch.Tensor, ctx: Context) -> torch.Tensor:
    if not (data.is_cuda and data.dtype == torch.uint8 and data.is_contiguous() and data.dim() == 1):
        raise ValueError("input must be a contiguous 1-D uint8 CUDA tensor")
    ctx = ctx or default_context(data.device.index)
    f = getattr(_native.lib(), fn)
    nb = C.c_size_t(0)
    s = _stream(data.device)
    _native.check(f(ctx.h, data.data_ptr(), data.numel(), None, 0, C.byref(nb), s), fn)
    out = torch.empty(nb.value, dtype=torch.uint8, device=data.device)
    _native.check(f(ctx.h, data.data_ptr(), data.numel(), out.data_ptr(), nb.value, C.byref(nb), s), fn)
    return out


def huff_encode(stream: torch.Tensor, ctx: Context = None) -> torch.Tensor:
    """Lossless stage: an edit stream (uint8 CUDA tensor) to a "PCH1" container of
    per-lane canonical Huffman codes (uint8 CUDA tensor)."""
    return _huff("pc_huff_encode", stream, ctx)


def huff_decode(blob: torch.Tensor, ctx: Context = None) -> torch.Tensor:
    """Inverse of :func:`huff_encode`: the edit stream, byte for byte."""
    return _huff("pc_huff_decode", blob, ctx)


class Server:
    """Request loop of the library (pc_server_*): jobs are admitted under a device-memory
    budget, set up together as they arrive and iterate side by side; each job's result is
    bit-identical to :func:`correct` (and :func:`encode_edits`) on that job alone.

    The tensors of a submitted job are kept referenced here until the job is finished."""

    def __init__(self, mem_budget: int = 0, max_slots: int = 0, max_cohort_particles: int = 0,
                 ctx: Context = None, device: int = 0):
        self.ctx = ctx or default_context(device)
        self.device = torch.device("cuda", self.ctx.device)
        h = C.c_void_p()
        _native.check(_native.lib().pc_server_create(self.ctx.h, int(mem_budget), int(max_slots),
                                                     int(max_cohort_particles), C.byref(h)), "pc_server_create")
        self.h = h
        self._keep = {}

    def submit(self, orig: torch.Tensor, recon: torch.Tensor, params, out: torch.Tensor = None,
               stream_cap: int = 0) -> int:
        """Queues one job; returns its ticket.  stream_cap > 0 also asks for the edit stream
        (a uint8 buffer of that many bytes, see :meth:`result`).  The inputs must be ready
        (the current stream is synchronised here)."""
        _xyz(orig, "orig")
        _xyz(recon, "recon")
        out = torch.empty_like(orig) if out is None else _xyz(out, "out")
        buf = torch.empty(int(stream_cap), dtype=torch.uint8, device=orig.device) if stream_cap > 0 else None
        torch.cuda.current_stream(orig.device).synchronize()
        j = _native.Job()
        j.orig_dev, j.recon_dev, j.n = orig.data_ptr(), recon.data_ptr(), orig.shape[0]
        j.params = _params(params)
        j.corrected_dev = out.data_ptr()
        j.stream_dev = buf.data_ptr() if buf is not None else None
        j.stream_cap = int(stream_cap)
        t = C.c_uint64(0)
        _native.check(_native.lib().pc_serve_submit(self.h, C.byref(j), C.byref(t)), "pc_serve_submit")
        self._keep[t.value] = (orig, recon, out, buf)
        return t.value

    def _res(self, r) -> dict:
        d = {k: getattr(r, k) for k in ("status", "submit_ns", "start_ns", "done_ns", "stream_bytes", "cohort_jobs")}
        d["state"] = _native.JOB_STATES[r.state]
        d["stats"] = struct_dict(r.stats)
        d["error"] = r.error.decode(errors="replace")
        return d

    def poll(self, ticket: int) -> dict:
        r = _native.JobResult()
        _native.check(_native.lib().pc_serve_poll(self.h, ticket, C.byref(r)), "pc_serve_poll")
        return self._res(r)

    def wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        r = _native.JobResult()
        code = _native.lib().pc_serve_wait(self.h, ticket, int(timeout_ms), C.byref(r))
        if code == -6:
            return self._res(r)
        _native.check(code, "pc_serve_wait")
        return self._res(r)

    def result(self, ticket: int, release: bool = True, timeout_ms: int = 600000):
        """(corrected, edit stream or None, result dict) of a finished job; TimeoutError if
        the job has not finished within timeout_ms."""
        d = self.wait(ticket, timeout_ms)
        if d["state"] not in ("DONE", "ERROR"):
            raise TimeoutError(f"job {ticket} still {d['state']} after {timeout_ms} ms")
        orig, recon, out, buf = self._keep[ticket] if not release else self._keep.pop(ticket)
        if buf is not None:
            buf = buf[: d["stream_bytes"]]
        return out, buf, d

    def counters(self) -> dict:
        a = (C.c_int64 * 4)()
        _native.check(_native.lib().pc_serve_counters(self.h, a), "pc_serve_counters")
        return dict(submitted=a[0], finished=a[1], cohorts=a[2], peak_bytes=a[3])

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            _native.lib().pc_server_destroy(self.h)
            self.h = C.c_void_p()
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
