"""The C ABI library builds, loads and exports every entry point include/pc.h declares (no GPU needed)."""
import ctypes as C
import os
import re

from paper_2604_18801_gb300 import _native
from paper_2604_18801_gb300 import build as _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            names |= set(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = C.CDLL(path)
    syms = declared_symbols()
    assert {"pc_correct", "pc_fof_labels", "pc_select_constraints", "pc_encode_edits", "pc_apply_edits",
            "pc_correct_batch", "pc_server_create", "pc_serve_submit", "pc_serve_poll", "pc_serve_wait"} <= syms
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_param_defaults():
    p = _native.make_params()
    assert p.m_bits == 16 and p.t_max == 10000 and p.replay_iters == -1
    assert abs(p.beta1 - 0.9) < 1e-15 and abs(p.beta2 - 0.999) < 1e-15 and p.loss_tol == 0.0
    import oracle
    for k in ("m_bits", "t_max", "alpha_rel", "beta1", "beta2", "eps_rel", "loss_tol", "replay_iters",
              "stall_patience"):
        assert getattr(p, k) == oracle.DEFAULTS[k], k
    q = _native.make_params(b=0.5, xi=0.1, mode=2, box_hi=(2, 3, 4))
    assert q.b == 0.5 and q.mode == 2 and list(q.box_hi) == [2.0, 3.0, 4.0]


def test_struct_sizes_match_the_header():
    # pc_params: 2+3+3 doubles, 4 ints, 5 doubles, 6 ints
    assert C.sizeof(_native.Params) == 8 * 8 + 4 * 4 + 5 * 8 + 6 * 4
    assert C.sizeof(_native.SelectStats) == 10 * 8 + 8
    assert C.sizeof(_native.CorrectStats) == 4 * 8 + 2 * 8 + 3 * 8 + 8 + 3 * 8 + 8 + 3 * 8


def test_struct_layouts_match_a_c_compiler(tmp_path):
    # sizes and field offsets as a C compiler lays out include/pc.h
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    checks = [("pc_params", _native.Params, ["b", "xi", "periodic", "t_max", "alpha_rel", "loss_tol", "replay_iters",
                                              "stall_patience", "cell_factor", "dense_cell"]),
              ("pc_select_stats", _native.SelectStats, ["n_links", "ms"]),
              ("pc_correct_stats", _native.CorrectStats, ["converged", "ms_setup", "pgd_launches", "resets", "pair_evals"]),
              ("pc_block", _native.Block, ["n", "params"]),
              ("pc_job", _native.Job, ["n", "params", "corrected_dev", "stream_cap"]),
              ("pc_job_result", _native.JobResult, ["done_ns", "stream_bytes", "cohort_jobs", "stats", "error"]),
              ("pc_cluster_metrics_t", _native.ClusterMetrics, ["tn", "ari", "mwm_iou", "members0"])]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pc.h"', "int main(void) {"]
    for cname, _, fields in checks:
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("%zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = []
    for _, cls, fields in checks:
        want.append(C.sizeof(cls))
        want += [getattr(cls, f).offset for f in fields]
    assert got == want


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2604_18801_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f
