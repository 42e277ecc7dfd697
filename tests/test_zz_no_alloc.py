"""bridge_delta0_noalloc: the linear density delta0 (App. A) without a context and
without allocating device memory (scratch in a 4 MiB static device array).

It must agree with BRIDGE_FIELD_DELTA0 of a context: relative L2 <= 1e-6 in FP32
and <= 1e-13 in FP64 (the same kernels; only the radial table is computed on the
device instead of the host, which can move a few FP32 roundings), on two calls in
a row with different noise.  Problems beyond the scratch are rejected before
anything is launched.  The file name sorts last, so the GPU test also runs after
the rest of the suite.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_2506_03969_gb300")

TOL = {pkg.BRIDGE_FP32: 1e-6, pkg.BRIDGE_FP64: 1e-13}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_03969_gb300 import build
    build.build()


def _cfg(n, batch, precision):
    c = synth.config(0)
    c.n = n
    return pkg.config_from(c, precision=precision, batch=batch)


def rel_l2(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_rejects_beyond_static_scratch():
    """Host-side checks, before any device work (runs without a GPU)."""
    L = pkg.lib()
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    for n, batch, prec in ((128, 1, pkg.BRIDGE_FP32), (64, 2, pkg.BRIDGE_FP64), (64, 4, pkg.BRIDGE_FP32)):
        st = L.bridge_delta0_noalloc(ctypes.byref(_cfg(n, batch, prec)), dummy, dummy, None)
        assert st == pkg.BRIDGE_EINVAL
        msg = L.bridge_last_error(None).decode()
        assert "static scratch" in msg and str(4 << 20) in msg
    st = L.bridge_delta0_noalloc(ctypes.byref(_cfg(32, 1, pkg.BRIDGE_FP32)), None, dummy, None)
    assert st == pkg.BRIDGE_EINVAL and "required" in L.bridge_last_error(None).decode()
    bad = _cfg(32, 1, pkg.BRIDGE_FP32)
    bad.n = 48
    assert L.bridge_delta0_noalloc(ctypes.byref(bad), dummy, dummy, None) == pkg.BRIDGE_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("n,batch,precision", [(32, 2, pkg.BRIDGE_FP32), (64, 1, pkg.BRIDGE_FP32),
                                               (64, 1, pkg.BRIDGE_FP64), (16, 3, pkg.BRIDGE_FP64)])
def test_matches_context_delta0_two_calls(n, batch, precision):
    cfg = _cfg(n, batch, precision)
    dt = torch.float64 if precision == pkg.BRIDGE_FP64 else torch.float32
    bias = synth.default_bias(synth.config(0))
    nus = [torch.tensor(synth.white_noise(n, seed, batch), dtype=dt, device="cuda").reshape(batch, -1).contiguous()
           for seed in (4101, 4202)]
    counts = torch.tensor(synth.timing_counts(n, 4303, 0.5, batch=batch), dtype=torch.int32,
                          device="cuda").reshape(batch, -1).contiguous()
    outs = [torch.empty_like(nus[0]) for _ in nus]
    # the first call on this device does the one-time setup; the next two are the ones compared
    pkg.bridge_delta0_noalloc(cfg, nus[0], outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for nu, out in zip(nus, outs):
        pkg.bridge_delta0_noalloc(cfg, nu, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "device free memory changed across the calls"

    ctx = pkg.Context(cfg)
    for nu, out in zip(nus, outs):
        ref = ctx.bridge_debug_field(nu, counts, [bias] * batch, pkg.FIELD_DELTA0).reshape(batch, -1)
        for b in range(batch):
            err = rel_l2(out[b], ref[b])
            assert err <= TOL[precision], f"chain {b}: rel L2 {err:.3e}"
    assert rel_l2(outs[0], outs[1]) > 0.5   # the two calls saw different noise


@pytest.mark.gpu
def test_first_call_in_a_fresh_process_before_any_context():
    """The one-time set-up of the first call (scratch address, twiddle tables) is what the call
    itself does, not something an earlier context left behind: a new process calls
    bridge_delta0_noalloc before any context exists, twice, and only then creates a context
    whose delta0 it is compared with."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = textwrap.dedent("""
        import sys, numpy as np, torch
        sys.path.insert(0, %r)
        import synth, paper_2506_03969_gb300 as pkg
        c = synth.config(0)
        cfg = pkg.config_from(c, batch=2)
        nu = torch.tensor(synth.white_noise(32, 4404, 2), dtype=torch.float32, device="cuda").reshape(2, -1).contiguous()
        out = torch.empty_like(nu)
        pkg.bridge_delta0_noalloc(cfg, nu, out)
        first = out.clone()
        pkg.bridge_delta0_noalloc(cfg, nu, out)
        torch.cuda.synchronize()
        counts = torch.ones_like(nu, dtype=torch.int32)
        ctx = pkg.Context(cfg)
        ref = ctx.bridge_debug_field(nu, counts, [synth.default_bias(c)] * 2, pkg.FIELD_DELTA0).reshape(2, -1)
        for o in (first, out):
            e = float(torch.linalg.vector_norm(o.double() - ref.double()) / torch.linalg.vector_norm(ref.double()))
            print("rel", e)
            assert e <= 1e-6, e
    """) % root
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    print(r.stdout, r.stderr[-2000:])
    assert r.returncode == 0
