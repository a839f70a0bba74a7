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
    assert {"pc_correct", "pc_fof_labels", "pc_select_constraints", "pc_encode_edits", "pc_apply_edits"} <= syms
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
    # pc_params: 2+3+3 doubles, 4 ints, 5 doubles, 2 ints
    assert C.sizeof(_native.Params) == 8 * 8 + 4 * 4 + 5 * 8 + 4 * 4
    assert C.sizeof(_native.SelectStats) == 10 * 8 + 8
    assert C.sizeof(_native.CorrectStats) == 4 * 8 + 2 * 8 + 3 * 8 + 8 + 3 * 8 + 8


def test_product_path_has_no_oracle_import():
    pkg = os.path.join(ROOT, "paper_2604_18801_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "liboracle" not in txt, f
