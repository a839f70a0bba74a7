"""The allocation-free decoder pc_apply_edits_static, called through the C ABI.

It serves callers that cannot allocate device memory while decoding (codes that
hold nearly all of the GPU's memory in their own arena, or callers in a region
where allocation is not allowed).  Its output must equal pc_apply_edits bit for
bit, on consecutive calls that share its static scratch array.  This file is
collected last, so a run that stops at the first failure has already run
everything else; it also passes when run alone in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_decode(lib, recon, stream, out, torch_stream):
    f = lib.pc_apply_edits_static
    f.argtypes = [C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f(recon.data_ptr(), recon.shape[0], stream.data_ptr(), stream.numel(), out.data_ptr(),
             torch_stream.cuda_stream)


def test_static_decoder_matches_pool_decoder_on_consecutive_calls(cuda):
    import torch

    import paper_2604_18801_gb300 as pc
    from paper_2604_18801_gb300 import _native, synth

    lib = _native.lib()
    ts = torch.cuda.current_stream(cuda)
    results = []
    for seed, n, m_bits in ((11, 20000, 16), (12, 7777, 8)):
        w = synth.tiny_cosmo(seed=seed, n=n, mode="HF")
        prm = w.params(m_bits=m_bits)
        o = torch.from_numpy(w.orig).to(cuda)
        r = torch.from_numpy(w.recon).to(cuda)
        corr, st, code = pc.correct(o, r, prm)
        assert code == 0
        s = pc.encode_edits(r, corr, prm)
        ref = pc.apply_edits(r, s)
        out = torch.full_like(r, float("nan"))
        rc = _static_decode(lib, r, s, out, ts)
        assert rc == 0, lib.pc_last_error()
        torch.cuda.synchronize(cuda)
        assert torch.equal(out, ref)            # same decoder arithmetic: bit-exact
        assert int((corr != r).any(dim=1).sum()) > 0
        results.append(out.cpu().numpy())
    assert results[0].shape != results[1].shape


def test_static_decoder_rejects_sizes_beyond_its_scratch(cuda):
    import torch

    from paper_2604_18801_gb300 import _native

    lib = _native.lib()
    n = (1 << 24) + 1
    recon = torch.zeros((n, 3), dtype=torch.float32, device=cuda)
    stream = torch.zeros(64 + (n + 7) // 8, dtype=torch.uint8, device=cuda)
    out = torch.empty_like(recon)
    rc = _static_decode(lib, recon, stream, out, torch.cuda.current_stream(cuda))
    assert rc == -1
    assert b"16777216" in lib.pc_last_error()
