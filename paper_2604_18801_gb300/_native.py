"""ctypes binding of libpc.so (include/pc.h).  Argument marshalling only.

Every computation runs in the CUDA library; there is no CPU fallback.  When
``libpc.so`` is missing this module raises at first use.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpc.so")

PC_OK, PC_WARN_NOT_CONVERGED = 0, 1
STATUS = {0: "PC_OK", 1: "PC_WARN_NOT_CONVERGED", -1: "PC_EINVAL", -2: "PC_EBOUND", -3: "PC_ENOMEM",
          -4: "PC_ECUDA", -5: "PC_EFORMAT", -6: "PC_ETIMEOUT", -7: "PC_EBUSY"}


class PcError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("b", C.c_double), ("xi", C.c_double), ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
                ("periodic", C.c_int32), ("mode", C.c_int32), ("m_bits", C.c_int32), ("t_max", C.c_int32),
                ("alpha_rel", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double), ("eps_rel", C.c_double),
                ("loss_tol", C.c_double), ("replay_iters", C.c_int32), ("cell_cap_log2", C.c_int32),
                ("stall_patience", C.c_int32), ("cell_factor", C.c_int32), ("dense_cell", C.c_int32),
                ("screen_chunk", C.c_int32)]


class SelectStats(C.Structure):
    _fields_ = [("n_links", C.c_int64), ("n_safe", C.c_int64), ("n_pb", C.c_int64), ("n_pc", C.c_int64),
                ("n_vulnerable", C.c_int64), ("n_active", C.c_int64), ("n_active_links", C.c_int64),
                ("n_halos", C.c_int64), ("n_safe_comps", C.c_int64), ("n_forest", C.c_int64), ("ms", C.c_double)]


class CorrectStats(C.Structure):
    _fields_ = [("iters", C.c_int64), ("loss_evals", C.c_int64), ("viol0", C.c_int64), ("viol_final", C.c_int64),
                ("loss0", C.c_double), ("loss_final", C.c_double), ("n_vulnerable", C.c_int64),
                ("n_active", C.c_int64), ("n_editable", C.c_int64), ("converged", C.c_int32), ("pad_", C.c_int32),
                ("ms_setup", C.c_double), ("ms_pgd", C.c_double), ("ms_pgd_iter", C.c_double),
                ("pgd_launches", C.c_int64), ("resets", C.c_int64), ("row_updates", C.c_int64),
                ("pair_evals", C.c_int64)]


class Block(C.Structure):
    _fields_ = [("offset", C.c_int64), ("n", C.c_int64), ("params", Params)]


class Job(C.Structure):
    _fields_ = [("orig_dev", C.c_void_p), ("recon_dev", C.c_void_p), ("n", C.c_int64), ("params", Params),
                ("corrected_dev", C.c_void_p), ("stream_dev", C.c_void_p), ("stream_cap", C.c_size_t)]


class JobResult(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("submit_ns", C.c_int64), ("start_ns", C.c_int64),
                ("done_ns", C.c_int64), ("stream_bytes", C.c_uint64), ("cohort_jobs", C.c_int32),
                ("pad_", C.c_int32), ("stats", CorrectStats), ("error", C.c_char * 160)]


JOB_STATES = {0: "PENDING", 1: "RUNNING", 2: "DONE", 3: "ERROR"}


class ClusterMetrics(C.Structure):
    _fields_ = [("tp", C.c_uint64), ("fp", C.c_uint64), ("fn", C.c_uint64), ("tn", C.c_uint64),
                ("ari", C.c_double), ("mwm_iou", C.c_double), ("halos0", C.c_int64), ("halos1", C.c_int64),
                ("members0", C.c_int64), ("pad_", C.c_int64)]


def struct_dict(s) -> dict:
    return {k: getattr(s, k) for k, _ in s._fields_ if not k.endswith("_")}


_lock = threading.Lock()
_lib = None


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built: run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        vp, i64, sz = C.c_void_p, C.c_int64, C.c_size_t
        P = C.POINTER(Params)
        L.pc_params_default.argtypes = [P]
        L.pc_params_default.restype = None
        L.pc_last_error.restype = C.c_char_p
        L.pc_kernel_launches.restype = C.c_uint64
        L.pc_ctx_create.argtypes = [C.c_int, sz, C.POINTER(vp)]
        L.pc_ctx_destroy.argtypes = [vp]
        L.pc_ctx_destroy.restype = None
        L.pc_fof_labels.argtypes = [vp, vp, i64, P, vp, C.POINTER(i64), vp]
        L.pc_select_constraints.argtypes = [vp, vp, i64, P, C.POINTER(vp), C.POINTER(SelectStats), vp]
        L.pc_constraints_copy.argtypes = [vp, vp, vp, vp, vp, vp]
        L.pc_constraints_free.argtypes = [vp]
        L.pc_constraints_free.restype = None
        L.pc_correct.argtypes = [vp, vp, vp, i64, P, vp, vp, C.POINTER(CorrectStats), vp]
        L.pc_correct_detail.argtypes = [vp, vp, vp, i64, P, vp, vp, vp, vp, vp, C.POINTER(CorrectStats), vp]
        L.pc_correct_multi.argtypes = [vp, vp, vp, i64, P, C.POINTER(C.c_double), C.c_int32, vp,
                                       C.POINTER(CorrectStats), vp]
        L.pc_correct_batch.argtypes = [vp, vp, vp, C.POINTER(Block), C.c_int32, vp, C.POINTER(CorrectStats), vp]
        L.pc_encode_edits.argtypes = [vp, vp, vp, i64, P, vp, sz, C.POINTER(sz), vp]
        L.pc_apply_edits.argtypes = [vp, vp, i64, vp, sz, vp, vp]
        L.pc_huff_encode.argtypes = [vp, vp, sz, vp, sz, C.POINTER(sz), vp]
        L.pc_huff_decode.argtypes = [vp, vp, sz, vp, sz, C.POINTER(sz), vp]
        L.pc_autotune_cells.argtypes = [vp, vp, i64, P, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]
        L.pc_autotune.argtypes = [vp, vp, i64, P, P, C.POINTER(C.c_double), vp]
        L.pc_cluster_metrics.argtypes = [vp, vp, vp, i64, C.c_int32, C.c_int32, C.c_double,
                                         C.POINTER(ClusterMetrics), vp, vp, vp, vp]
        L.pc_server_create.argtypes = [vp, sz, C.c_int32, i64, C.POINTER(vp)]
        L.pc_server_destroy.argtypes = [vp]
        L.pc_server_destroy.restype = None
        L.pc_serve_submit.argtypes = [vp, C.POINTER(Job), C.POINTER(C.c_uint64)]
        L.pc_serve_poll.argtypes = [vp, C.c_uint64, C.POINTER(JobResult)]
        L.pc_serve_wait.argtypes = [vp, C.c_uint64, i64, C.POINTER(JobResult)]
        L.pc_serve_counters.argtypes = [vp, C.POINTER(i64)]
        for f in ("pc_ctx_create", "pc_fof_labels", "pc_select_constraints", "pc_constraints_copy", "pc_correct",
                  "pc_correct_detail", "pc_correct_batch", "pc_correct_multi", "pc_autotune_cells", "pc_autotune",
                  "pc_cluster_metrics",
                  "pc_server_create", "pc_serve_submit",
                  "pc_serve_poll",
                  "pc_serve_wait", "pc_serve_counters",
                  "pc_encode_edits", "pc_apply_edits", "pc_huff_encode", "pc_huff_decode"):
            getattr(L, f).restype = C.c_int
        _lib = L
        return L


def check(code: int, where: str, allow_warn: bool = False) -> int:
    if code == PC_OK or (allow_warn and code > 0):
        return code
    msg = lib().pc_last_error().decode(errors="replace")
    raise PcError(code, where, msg)


def make_params(**kw) -> Params:
    p = Params()
    lib().pc_params_default(C.byref(p))
    for k, v in kw.items():
        if k in ("box_lo", "box_hi"):
            getattr(p, k)[:] = [float(x) for x in v]
        elif k in ("b", "xi", "alpha_rel", "beta1", "beta2", "eps_rel", "loss_tol"):
            setattr(p, k, float(v))
        else:
            setattr(p, k, int(v))
    return p
