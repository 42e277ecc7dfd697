"""The C ABI library on the CPU host: it builds, loads, exports every function
declared in include/bridge.h, and its host-only calls behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import cosmo

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    from paper_2506_03969_gb300 import build
    build.build()
    import paper_2506_03969_gb300 as p
    p.lib()
    return p


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bridge.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(bridge_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("bridge_create", "bridge_destroy", "bridge_forward", "bridge_logpost_grad", "bridge_leapfrog",
              "bridge_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(pkg):
    lib = ctypes.CDLL(pkg.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_validate_config(pkg):
    good = pkg.make_config(32, 300.0, pk_amp=1.0)
    assert pkg.lib().bridge_validate_config(ctypes.byref(good)) == pkg.BRIDGE_OK
    assert pkg.lib().bridge_workspace_bytes(ctypes.byref(good)) > 0
    for field, value in (("n", 48), ("n", 8), ("n", 1024), ("batch", 0), ("box", -1.0), ("n_regions", 5),
                         ("sharpness", 0.0), ("rho_floor", 0.0), ("precision", 7), ("r_s", float("nan")),
                         ("recompute_alpt", 2), ("rsd_los", 2), ("rsd_los", -1), ("rsd_f", float("inf")),
                         ("deterministic", 2)):
        bad = pkg.make_config(32, 300.0, pk_amp=1.0)
        setattr(bad, field, value)
        assert pkg.lib().bridge_validate_config(ctypes.byref(bad)) == pkg.BRIDGE_EINVAL, field
        assert pkg.lib().bridge_workspace_bytes(ctypes.byref(bad)) == 0
    big64 = pkg.make_config(512, 2000.0, pk_amp=1.0, precision=pkg.BRIDGE_FP64)
    assert pkg.lib().bridge_validate_config(ctypes.byref(big64)) == pkg.BRIDGE_OK
    assert pkg.lib().bridge_validate_config(None) == pkg.BRIDGE_EINVAL


def test_workspace_scales_with_mesh_and_batch(pkg):
    def ws(n, batch=1):
        return pkg.lib().bridge_workspace_bytes(ctypes.byref(pkg.make_config(n, 300.0, pk_amp=1.0, batch=batch)))
    # field storage grows as N^3 and with the batch; a fixed part (node slabs) does not
    d1, d2 = ws(128) - ws(64), ws(256) - ws(128)
    assert 7.5 < d2 / d1 < 8.5
    b1, b2 = ws(128, 2) - ws(128, 1), ws(128, 3) - ws(128, 2)
    assert abs(b2 / b1 - 1) < 0.01
    # 512^3 FP32 fits comfortably in a GB300's HBM
    d = pkg.lib().bridge_workspace_bytes(ctypes.byref(pkg.make_config(512, 2000.0, pk_amp=1.0, n_regions=16)))
    assert d < 60e9
    # recomputing the ALPT spectra in the adjoint drops ten half spectra from the workspace
    r = pkg.lib().bridge_workspace_bytes(ctypes.byref(pkg.make_config(512, 2000.0, pk_amp=1.0, n_regions=16,
                                                                        recompute_alpt=True)))
    spec = 8 * (512 // 2 + 1) * 512 * 512
    assert abs((d - r) - 10 * spec) < 4096
    # the radial line of sight keeps Psi_1 and its adjoint: six more half spectra (plane-parallel: none)
    pp = pkg.lib().bridge_workspace_bytes(ctypes.byref(pkg.make_config(512, 2000.0, pk_amp=1.0, n_regions=16,
                                                                         rsd_f=0.8)))
    rad = pkg.lib().bridge_workspace_bytes(ctypes.byref(pkg.make_config(512, 2000.0, pk_amp=1.0, n_regions=16,
                                                                          rsd_f=0.8, rsd_los=1)))
    assert pp == d and abs((rad - d) - 6 * spec) < 4096
    # the deterministic mass assignment adds one 64-bit field
    det = pkg.lib().bridge_workspace_bytes(ctypes.byref(pkg.make_config(512, 2000.0, pk_amp=1.0, n_regions=16,
                                                                          deterministic=True)))
    assert abs((det - d) - 8 * 512 ** 3) < 4096


def test_pk_amplitude_matches_oracle_quadrature(pkg):
    """The library's composite Simpson rule and the oracle's adaptive quadrature agree."""
    for ns, kc, pw in ((0.96, 0.02, 1.5), (1.0, 0.05, 1.0), (-1.0, 1.0, 0.0)):
        a_lib = pkg.bridge_pk_amplitude(0.8, 8.0, ns, kc, pw)
        a_or = cosmo.amplitude_for_sigma(0.8, 8.0, ns, kc, pw)
        assert abs(a_lib / a_or - 1) < 1e-6, (ns, a_lib, a_or)
    assert pkg.bridge_pk_amplitude(-1.0, 8.0, 0.96, 0.02, 1.5) < 0


def test_status_strings(pkg):
    for s in range(7):
        assert pkg.lib().bridge_status_string(s)
    assert pkg.lib().bridge_last_error(None)


def test_bias_marshalling(pkg):
    b = synth.bias_hierarchical()
    arr = pkg.bias_array([b, b])
    assert arr[1].alpha[15] == b.alpha[15] and arr[0].rho[3] == b.rho[3]
    assert arr[0].prior_mask == 0xFFFF
    # Table 2 reading: alpha_j, beta_j of the four Phi classes, tied over their delta sub-classes
    assert arr[0].free_mask == 0xFF and arr[0].tie_classes == 1 and pkg.n_free([b]) == 8
    u = synth.bias_phi_web()
    u.free_mask = None
    assert pkg.bias_array([u])[0].free_mask == 0xFF and pkg.bias_array([u])[0].tie_classes == 0
    u.free_mask = 0b1010
    assert pkg.n_free([u]) == 2


def test_create_without_device_fails_cleanly(pkg):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = pkg.make_config(32, 300.0, pk_amp=1.0)
    h = ctypes.c_void_p()
    st = pkg.lib().bridge_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == pkg.BRIDGE_ENODEVICE and not h.value
    assert b"device" in pkg.lib().bridge_last_error(None)
