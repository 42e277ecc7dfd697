"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP32 fields relative L2 <= 1e-5, FP32 gradients <= 1e-4, log
posterior |d|/|lp| <= 1e-6; the FP64 path <= 1e-10 (fields, gradients) and
1e-12 (log posterior).  Nothing is bit-exact: CIC atomics reorder sums.
"""
import math

import numpy as np
import pytest

import synth
from oracle import hmc, mock, model

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_2506_03969_gb300")

pytestmark = pytest.mark.gpu

FP32_FIELD, FP32_GRAD, FP32_LP = 1e-5, 1e-4, 1e-6
FP64_FIELD, FP64_GRAD, FP64_LP = 1e-10, 1e-10, 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_03969_gb300 import build
    build.build()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(n, box, n_regions, seed, beta=None, mean=0.5):
    cfg = synth.Config(f"{n}^3", n, box, n_regions=n_regions, nb_beta=beta, mean_tracers=mean,
                       seed_truth=seed, seed_counts=seed + 1, seed_eval=seed + 2)
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    nu = synth.eval_point(n, cfg.seed_truth, cfg.seed_eval)
    return cfg, bias, nu, counts


def run_gpu(cfg, bias, nu, counts, precision):
    ctx = pkg.Context(pkg.config_from(cfg, precision=precision, batch=1))
    dt = torch.float64 if precision == pkg.BRIDGE_FP64 else torch.float32
    nu_d = torch.tensor(nu, dtype=dt, device="cuda").contiguous()
    c_d = torch.tensor(counts, dtype=torch.int32, device="cuda").contiguous()
    return ctx, nu_d, c_d


ORACLE = {}


def oracle_ref(key, cfg, bias, nu, counts):
    if key not in ORACLE:
        f = model.forward_fields(nu, counts, cfg, bias)
        lp, g, ga, gb = model.logpost_and_grad(nu, counts, cfg, bias)
        ORACLE[key] = (f, lp, g, np.concatenate([ga, gb]))
    return ORACLE[key]


CASES = {
    "16_phi": (16, 160.0, 4, 1101),
    "32_phi": (32, 300.0, 4, 1001),        # workload 0 geometry
    "64_hier": (64, 500.0, 16, 1201),
    "128_hier": (128, 1000.0, 16, 1002),   # workload 1 geometry
}


def _fields_check(ctx, nu_d, c_d, bias, f, tol):
    checks = [(pkg.FIELD_DELTA0, f["delta0"]), (pkg.FIELD_PSI, f["psi"]), (pkg.FIELD_DELTA, f["delta"]),
              (pkg.FIELD_TIDAL, f["T"]), (pkg.FIELD_LAMBDA, f["lam_phi"]), (pkg.FIELD_LNNBAR, f["ln_nbar"])]
    if f.get("H") is not None:
        checks.append((pkg.FIELD_HESSIAN, f["H"]))
    errs = {}
    for which, ref in checks:
        got = ctx.bridge_debug_field(nu_d, c_d, [bias], which).double().cpu().numpy().reshape(ref.shape)
        errs[which] = rel_l2(got, ref)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"field rel L2 above {tol}: {errs}"


@pytest.mark.parametrize("name", ["16_phi", "32_phi", "64_hier", "128_hier"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_forward_fields_and_gradient(name, precision):
    n, box, nr, seed = CASES[name]
    if precision == "fp64" and n > 64:
        pytest.skip("FP64 parity covered at n <= 64")
    cfg, bias, nu, counts = case(n, box, nr, seed)
    f, lp_o, g_o, gbias_o = oracle_ref(name, cfg, bias, nu, counts)
    prec = pkg.BRIDGE_FP64 if precision == "fp64" else pkg.BRIDGE_FP32
    ftol, gtol, ltol = (FP64_FIELD, FP64_GRAD, FP64_LP) if precision == "fp64" else (FP32_FIELD, FP32_GRAD, FP32_LP)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec)
    _fields_check(ctx, nu_d, c_d, bias, f, ftol)
    lp, g, gb = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
    assert abs(lp[0] - lp_o) / abs(lp_o) <= ltol, (lp[0], lp_o)
    assert rel_l2(g.double().cpu().numpy().reshape(g_o.shape), g_o) <= gtol
    # bias-table gradients, relative to the largest entry
    assert np.max(np.abs(gb[0] - gbias_o)) <= gtol * np.max(np.abs(gbias_o)) * 10
    lp2, _ = ctx.bridge_forward(nu_d, c_d, [bias])
    # a second evaluation differs only by the CIC atomic summation order
    assert abs(lp2[0] - lp[0]) <= (1e-7 if precision == "fp32" else 1e-13) * abs(lp[0])
    ctx.close()


def test_batched_chains_match_single_and_oracle():
    cfgs = [case(32, 300.0, 4, 1001 + 10 * b) for b in range(3)]
    biases = synth.perturbed_biases(cfgs[0][1], 3, 6001)
    cfg = cfgs[0][0]
    ctx = pkg.Context(pkg.config_from(cfg, batch=3))
    nu = torch.tensor(np.stack([c[2] for c in cfgs]), dtype=torch.float32, device="cuda").contiguous()
    counts = torch.tensor(np.stack([c[3] for c in cfgs]), dtype=torch.int32, device="cuda").contiguous()
    lp, g, gb = ctx.bridge_logpost_grad(nu, counts, biases)
    single = pkg.Context(pkg.config_from(cfg, batch=1))
    for b in range(3):
        lp1, g1, gb1 = single.bridge_logpost_grad(nu[b].contiguous(), counts[b].contiguous(), [biases[b]])
        assert abs(lp1[0] - lp[b]) <= 1e-7 * abs(lp[b])
        assert rel_l2(g1.cpu().numpy(), g[b].cpu().numpy()) <= 1e-5
        lp_o, g_o, _, _ = model.logpost_and_grad(cfgs[b][2], cfgs[b][3], cfg, biases[b])
        assert abs(lp[b] - lp_o) / abs(lp_o) <= FP32_LP
        assert rel_l2(g[b].double().cpu().numpy(), g_o) <= FP32_GRAD


def test_autograd_function_and_host_api():
    cfg, bias, nu, counts = case(32, 300.0, 4, 1001)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    x = nu_d.clone().requires_grad_(True)
    lp = pkg.log_posterior(ctx, x, c_d, [bias])
    (gx,) = torch.autograd.grad(lp.sum(), x)
    _, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
    assert torch.equal(gx, g)
    nu_h = torch.tensor(nu, dtype=torch.float32).pin_memory()
    c_h = torch.tensor(counts, dtype=torch.int32).pin_memory()
    g_h = torch.empty_like(nu_h).pin_memory()
    lp_h = ctx.bridge_logpost_grad_host(nu_h, c_h, [bias], g_h)
    assert abs(lp_h[0] - float(lp)) <= 1e-7 * abs(float(lp))
    assert rel_l2(g_h.numpy(), g.cpu().numpy()) <= 1e-6


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_leapfrog_matches_oracle(precision):
    cfg, bias, nu, counts = case(16, 160.0, 4, 1301)
    p0 = synth.momentum(16, 1304)
    nu_o, p_o, h0_o, h1_o = hmc.leapfrog(nu, p0, counts, cfg, bias, 4, 0.05)
    prec = pkg.BRIDGE_FP64 if precision == "fp64" else pkg.BRIDGE_FP32
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec)
    p_d = torch.tensor(p0, dtype=nu_d.dtype, device="cuda").contiguous()
    h0, h1 = ctx.bridge_leapfrog(nu_d, p_d, c_d, [bias], 4, 0.05)
    tol = 1e-10 if precision == "fp64" else 1e-5
    assert rel_l2(nu_d.double().cpu().numpy(), nu_o) <= tol
    assert rel_l2(p_d.double().cpu().numpy(), p_o) <= tol * 10
    assert abs(h0[0] - h0_o) <= tol * abs(h0_o)
    if precision == "fp64":
        assert abs((h1[0] - h0[0]) - (h1_o - h0_o)) <= 1e-8 * max(1.0, abs(h1_o - h0_o))
    else:
        assert abs((h1[0] - h0[0]) - (h1_o - h0_o)) <= 1e-2 * max(1.0, abs(h1_o - h0_o))


def test_invalid_inputs_return_errors():
    cfg, bias, nu, counts = case(16, 160.0, 4, 1401)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    bad = c_d.clone()
    bad[0, 0, 0] = 70000
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_logpost_grad(nu_d, bad, [bias])
    assert e.value.status == pkg.BRIDGE_EINVAL
    bad[0, 0, 0] = -1
    with pytest.raises(pkg.BridgeError):
        ctx.bridge_forward(nu_d, bad, [bias])
    b2 = bias.copy()
    b2.rho[0] = -1.0
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_logpost_grad(nu_d, c_d, [b2])
    assert e.value.status == pkg.BRIDGE_EINVAL
    # the context stays usable after errors
    lp, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
    assert np.isfinite(lp[0])
    nan_nu = nu_d.clone()
    nan_nu[0, 0, 0] = float("nan")
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_logpost_grad(nan_nu, c_d, [bias])
    assert e.value.status == pkg.BRIDGE_ENONFINITE


def test_full_size_256_properties_and_linear_field():
    """256^3 (the timed workload): linear field and displacement equal the oracle on the
    full mesh; mass conservation; gradient directional derivative vs FP64 finite differences."""
    cfg = synth.config(2)
    bias = synth.default_bias(cfg)
    nu = synth.white_noise(cfg.n, cfg.seed_eval)
    counts = synth.timing_counts(cfg.n, cfg.seed_counts, cfg.mean_tracers)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    d0 = ctx.bridge_debug_field(nu_d, c_d, [bias], pkg.FIELD_DELTA0).double().cpu().numpy()[0, 0]
    with torch.no_grad():
        d0_o = model.delta0_from_nu(torch.tensor(nu, dtype=torch.float64), cfg).numpy()
    assert rel_l2(d0, d0_o) <= FP32_FIELD
    delta = ctx.bridge_debug_field(nu_d, c_d, [bias], pkg.FIELD_DELTA).double().cpu().numpy()
    assert abs(delta.sum()) <= 1e-6 * delta.size      # CIC conserves mass
    lp, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
    assert np.isfinite(lp[0]) and torch.isfinite(g).all()
    # directional derivative against central differences of the FP64 GPU path
    ctx64, nu64, _ = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP64)
    d = torch.tensor(synth.directions(cfg.n, 77, 1)[0], dtype=torch.float64, device="cuda")
    lp64, g64, _ = ctx64.bridge_logpost_grad(nu64, c_d, [bias])
    h = 1e-3
    lpp, _ = ctx64.bridge_forward((nu64 + h * d).contiguous(), c_d, [bias])
    lpm, _ = ctx64.bridge_forward((nu64 - h * d).contiguous(), c_d, [bias])
    fd = (lpp[0] - lpm[0]) / (2 * h)
    dd64 = float((g64 * d).sum())
    dd32 = float((g.double() * d).sum())
    assert abs(fd - dd64) <= 1e-4 * abs(fd)
    assert abs(dd32 - dd64) <= 1e-3 * abs(dd64)
    assert rel_l2(g.double().cpu().numpy(), g64.cpu().numpy()) <= FP32_GRAD
