"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides always see the same input: nu is rounded to FP32 before the oracle
gets it, so the FP32 path's input rounding is never part of a measured error.

Bounds (the target tolerances): FP32 fields relative L2 <= 1e-5, gradients <= 1e-4, log
posterior |d|/|lp| <= 1e-6; FP64 path fields and gradients <= 1e-10, log
posterior <= 1e-12.  They are held at well-conditioned points (see
``parity_points``): every cell at least 1e-3 in D delta0 away from the
spherical-collapse threshold, and, away from the data-generating field, the
counts of near-empty cells (CIC mass < 1e-2) cleared.  There the exact FP64
gradient moves by S <~ 1e-5 under an FP32 rounding of the input (measured by the
oracle and printed), so an error above the bound is the GPU path's own.

At the unmodified off-truth points a few cells dominate the gradient and S
reaches 1e-3 (128^3) to 4e-2 (256^3): no FP32 evaluation can hold 1e-4 there.
Those points check the fields and the log posterior; a field tolerance scaled
by its own conditioning is capped at 1e-3, and the gradient error is printed
next to S, asserted only where 10 S <= 1e-3.  Nothing matches the oracle bit for bit;
with float CIC atomics two GPU evaluations also differ by rounding, with the
deterministic mass assignment they are bit-identical.
"""
import math

import numpy as np
import pytest

import parity_points as pp
import synth
from oracle import hmc, mock, model

torch = pytest.importorskip("torch")
pkg = pytest.importorskip("paper_2506_03969_gb300")

pytestmark = pytest.mark.gpu

FP32_FIELD, FP32_GRAD, FP32_LP = 1e-5, 1e-4, 1e-6
FP64_FIELD, FP64_GRAD, FP64_LP = 1e-10, 1e-10, 1e-12
CAP = 1e-3   # largest tolerance ever derived from a point's conditioning


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2506_03969_gb300 import build
    build.build()


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_case(n, box, n_regions, seed, beta=None, mean=0.5, point="eval", gap=1e-3, **cfg_kw):
    """Workload geometry at mesh n; counts are the oracle's gamma-Poisson mock of nu_true (Sect. 3).
    point: "truth" (nu_true) or "eval" (nu_true + 0.3 noise), each treated -- kept off the
    collapse threshold, near-empty counts cleared -- or "raw" (nu_true + 0.3 noise as it is;
    only rounded to FP32)."""
    cfg = synth.Config(f"{n}^3", n, box, n_regions=n_regions, nb_beta=beta, mean_tracers=mean,
                       seed_truth=seed, seed_counts=seed + 1, seed_eval=seed + 2, **cfg_kw)
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    if point == "truth":
        nu, counts, moved, cleared = pp.condition(nu_t, counts, cfg, bias, gap=gap, clear_empty=True)
    elif point == "eval":
        nu0 = synth.eval_point(n, cfg.seed_truth, cfg.seed_eval, scale=0.3 if n < 256 else 0.1)
        nu, counts, moved, cleared = pp.condition(nu0, counts, cfg, bias, gap=gap, clear_empty=True)
    else:
        nu = pp.f32(synth.eval_point(n, cfg.seed_truth, cfg.seed_eval, scale=0.3 if n < 256 else 0.1))
        moved = cleared = 0
    return cfg, bias, nu, counts, (moved, cleared)


def run_gpu(cfg, bias, nu, counts, precision, **kw):
    ctx = pkg.Context(pkg.config_from(cfg, precision=precision, batch=1, **kw))
    dt = torch.float64 if precision == pkg.BRIDGE_FP64 else torch.float32
    nu_d = torch.tensor(nu, dtype=dt, device="cuda").contiguous()
    c_d = torch.tensor(counts, dtype=torch.int32, device="cuda").contiguous()
    return ctx, nu_d, c_d


def free_grad(ga, gb, bias):
    """The free-parameter gradient the library returns, formed from the oracle's per-entry
    gradients: parameters in bit order of free_mask; tied classes sum their four entries."""
    nr = len(bias.alpha)
    tie = getattr(bias, "tie_classes", 0)
    P = 4 if tie else nr
    mask = pkg.bias_array([bias])[0].free_mask
    full_a = np.asarray(ga).reshape(4, 4).sum(1) if tie else np.asarray(ga)
    full_b = np.asarray(gb).reshape(4, 4).sum(1) if tie else np.asarray(gb)
    vals = np.concatenate([full_a, full_b])
    return np.array([vals[q] for q in range(2 * P) if (mask >> q) & 1])


ORACLE = {}


def oracle_ref(key, cfg, bias, nu, counts, conditioning=True, psi=False):
    """Oracle fields, log posterior, gradient, free bias gradient and conditioning: the relative
    change of the gradient (cond), of the free bias gradient (f["cond_bias"]) and of each field
    (f["cond"]) under a 2^-23 relative perturbation of nu, and the free bias gradient's
    cancellation factor |sum_i |t_i|| / |sum_i t_i| over its per-cell terms (f["kappa_bias"]).
    conditioning: True (all), "fields"
    (fields only) or False.  psi: also the relative change of the gradient and of the free bias
    gradient (f["cond_psi"], f["cond_psi_bias"]) when white noise of 3e-7 times the rms
    displacement -- the FP32 displacement error of the GPU path -- is added to Psi."""
    if key not in ORACLE:
        f = model.forward_fields(nu, counts, cfg, bias)
        lp, g, ga, gb = model.logpost_and_grad(nu, counts, cfg, bias)
        fb = free_grad(ga, gb, bias)
        cond, f["cond"], f["cond_bias"], f["kappa_bias"] = 0.0, {}, None, None
        f["cond_psi"] = f["cond_psi_bias"] = None
        if psi:
            rms = float(np.sqrt((f["psi"] ** 2).mean()))
            shift = np.random.default_rng(54321).standard_normal(f["psi"].shape) * 3e-7 * rms
            _, g3, ga3, gb3 = model.logpost_and_grad(nu, counts, cfg, bias, psi_shift=shift)
            f["cond_psi"] = float(np.linalg.norm(g3 - g) / np.linalg.norm(g))
            f["cond_psi_bias"] = float(np.linalg.norm(free_grad(ga3, gb3, bias) - fb) / np.linalg.norm(fb))
        if conditioning:
            pert = np.random.default_rng(12345).standard_normal(nu.shape) * (2.0 ** -23) * float(np.std(nu))
            if conditioning is True:
                _, g2, ga2, gb2 = model.logpost_and_grad(nu + pert, counts, cfg, bias)
                cond = float(np.linalg.norm(g2 - g) / np.linalg.norm(g))
                f["cond_bias"] = float(np.linalg.norm(free_grad(ga2, gb2, bias) - fb) / np.linalg.norm(fb))
            if conditioning is True:
                abs_a, abs_b, _, _ = pp.bias_abs_terms(nu, counts, cfg, bias)
                f["kappa_bias"] = float(np.linalg.norm(free_grad(abs_a, abs_b, bias)) / np.linalg.norm(fb))
            f2 = model.forward_fields(nu + pert, counts, cfg, bias)
            f["cond"] = {k: float(np.linalg.norm(f2[k] - f[k]) / np.linalg.norm(f[k]))
                         for k in f if isinstance(f[k], np.ndarray) and f[k] is not None}
        ORACLE[key] = (f, lp, g, fb, cond)
    return ORACLE[key]


FIELD_NAMES = {pkg.FIELD_DELTA0: "delta0", pkg.FIELD_PSI: "psi", pkg.FIELD_DELTA: "delta", pkg.FIELD_TIDAL: "T",
               pkg.FIELD_LAMBDA: "lam_phi", pkg.FIELD_LNNBAR: "ln_nbar", pkg.FIELD_HESSIAN: "H"}


def check_fields(ctx, nu_d, c_d, bias, f, base, scaled=False):
    """Every intermediate field against the oracle at the fixed bound `base`.

    ln nbar is local and, in cells with almost no CIC mass, follows alpha ln rho, i.e. the
    relative change of that mass -- the last bits of the displacement -- so it is held at `base`
    on the cells with mass >= 1e-2; over all cells its tolerance is its measured conditioning S
    (10 S FP32, 1e-7 S FP64, never above 1e-3) or, where S was not measured, 1e-3.
    scaled: every field gets max(base, that conditioning-scaled tolerance)."""
    checks = [pkg.FIELD_DELTA0, pkg.FIELD_PSI, pkg.FIELD_DELTA, pkg.FIELD_TIDAL, pkg.FIELD_LAMBDA, pkg.FIELD_LNNBAR]
    if f.get("H") is not None:
        checks.append(pkg.FIELD_HESSIAN)
    fp32 = base >= FP32_FIELD

    def cond_tol(k):
        if k not in f["cond"]:
            return CAP if fp32 else 1e-7
        c = f["cond"][k]
        return max(base, min(10.0 * c, CAP)) if fp32 else max(base, 1e-7 * c)

    errs, bad = {}, {}
    for which in checks:
        k = FIELD_NAMES[which]
        ref = f[k]
        got = ctx.bridge_debug_field(nu_d, c_d, [bias], which).double().cpu().numpy().reshape(ref.shape)
        errs[k] = rel_l2(got, ref)
        tol = cond_tol(k) if (scaled or k == "ln_nbar") else base
        if not errs[k] <= tol:
            bad[k] = (errs[k], tol)
        if k == "ln_nbar":
            keep = (1.0 + f["delta"]).reshape(ref.shape) >= 1e-2
            errs["ln_nbar_mass>=1e-2"] = rel_l2(got[keep], ref[keep])
            if not errs["ln_nbar_mass>=1e-2"] <= base:
                bad["ln_nbar_mass>=1e-2"] = (errs["ln_nbar_mass>=1e-2"], base)
    print("field rel L2:", {k: f"{v:.2e}" for k, v in errs.items()})
    assert not bad, f"field rel L2 above tolerance (err, tol): {bad}"
    return errs


def bounds(precision):
    return (FP64_FIELD, FP64_GRAD, FP64_LP) if precision == "fp64" else (FP32_FIELD, FP32_GRAD, FP32_LP)


def prec_code(precision):
    return pkg.BRIDGE_FP64 if precision == "fp64" else pkg.BRIDGE_FP32


CASES = {
    "16_phi": (16, 160.0, 4, 1101),
    "32_phi": (32, 300.0, 4, 1001),        # workload geometry: 32^3, L = 300, Phi-web
    "64_hier": (64, 500.0, 16, 1201),
    "128_hier": (128, 1000.0, 16, 1002),   # workload geometry: 128^3, L = 1000, Phi x delta web
}


def _full_check(name, cfg, bias, nu, counts, precision, conditioning=True, psi=False, **ctx_kw):
    ftol, gtol, ltol = bounds(precision)
    f, lp_o, g_o, gb_o, cond = oracle_ref(name, cfg, bias, nu, counts, conditioning, psi)
    gtol = grad_tol(precision, f)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec_code(precision), **ctx_kw)
    check_fields(ctx, nu_d, c_d, bias, f, ftol)
    lp, g, gb = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
    e_lp = abs(lp[0] - lp_o) / abs(lp_o)
    e_g = rel_l2(g.double().cpu().numpy().reshape(g_o.shape), g_o)
    e_b = rel_l2(gb[0], gb_o)
    btol = bias_tol(precision, f)
    sp = f.get("cond_psi")
    print(f"{name} {precision}: logpost rel {e_lp:.2e}  grad rel L2 {e_g:.2e} (tol {gtol:.1e}, S {cond:.1e}"
          + (f", S_psi {sp:.1e}" if sp is not None else "") + f")  "
          f"free bias grad rel L2 {e_b:.2e} (tol {btol:.1e}, {gb.shape[1]} parameters"
          + (f", kappa {f['kappa_bias']:.0f}" if f.get("kappa_bias") is not None else "") + ")")
    assert e_lp <= ltol, (lp[0], lp_o)
    assert e_g <= gtol
    assert e_b <= btol
    return ctx, nu_d, c_d, lp, g


CAP_PSI = 5e-3   # largest tolerance ever derived from the displacement conditioning S_psi


def grad_tol(precision, f):
    """The fixed bound, unless the gradient's displacement conditioning S_psi (measured by the
    oracle at the test point) puts it out of FP32 reach: the CIC weights are piecewise linear, so
    the exact gradient jumps where a particle crosses a cell face, and particles that sit within
    the FP32 position error of a face (a few at 128^3, tens at 256^3) take the other one-sided
    derivative.  FP32: max(1e-4, 3 S_psi), never above 5e-3."""
    _, gtol, _ = bounds(precision)
    sp = f.get("cond_psi")
    if precision != "fp32" or sp is None:
        return gtol
    return max(gtol, min(3.0 * sp, CAP_PSI))


def bias_tol(precision, f):
    """The free bias gradient is a sum over all cells, which nearly cancels at the data-
    generating field (its expectation is zero there): its tolerance is scaled by its own
    measured conditioning, never above 1e-3 (FP32), by its displacement conditioning as the
    gradient is (grad_tol), and by its cancellation factor kappa: per-cell terms each rounded
    to a few FP32 ulps leave an error of about 2^-23 kappa in their sum, so FP32 allows
    2 * 2^-23 * kappa, never above 1e-3."""
    _, gtol, _ = bounds(precision)
    sb = f.get("cond_bias")
    t = gtol
    if sb is not None:
        t = max(gtol, min(10.0 * sb, CAP)) if precision == "fp32" else max(gtol, 1e-7 * sb)
    kb = f.get("kappa_bias")
    if precision == "fp32" and kb is not None:
        t = max(t, min(2.0 * 2.0 ** -23 * kb, CAP))
    spb = f.get("cond_psi_bias")
    if precision == "fp32" and spb is not None:
        t = max(t, min(3.0 * spb, CAP_PSI))
    return t


@pytest.mark.parametrize("name", ["16_phi", "32_phi", "64_hier", "128_hier"])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_forward_fields_and_gradient(name, precision):
    """Off the data-generating field (nu_true + 0.3 noise), treated as described above."""
    n, box, nr, seed = CASES[name]
    cfg, bias, nu, counts, (moved, cleared) = make_case(n, box, nr, seed, point="eval")
    print(f"{name}: {moved} cells moved off the collapse threshold, {cleared} near-empty cells cleared")
    ctx, nu_d, c_d, lp, _ = _full_check(name, cfg, bias, nu, counts, precision)
    lp2, _ = ctx.bridge_forward(nu_d, c_d, [bias])
    # a second evaluation differs only by the CIC atomic summation order
    assert abs(lp2[0] - lp[0]) <= (1e-7 if precision == "fp32" else 1e-13) * abs(lp[0])
    ctx.close()


@pytest.mark.parametrize("name", ["64_hier", "128_hier"])
def test_data_consistent_point(name):
    """At the field the counts were drawn from (nu_true, treated): fixed bounds, both precisions."""
    n, box, nr, seed = CASES[name]
    cfg, bias, nu, counts, (moved, _) = make_case(n, box, nr, seed, point="truth")
    print(f"{name} truth: {moved} cells moved off the collapse threshold")
    for precision in ("fp32", "fp64"):
        ctx = _full_check(name + "_truth", cfg, bias, nu, counts, precision, psi=True)[0]
        ctx.close()


def test_unmodified_points_fields_and_report():
    """nu_true + 0.3 noise at 128^3 as it is: fields and log posterior against the oracle (a
    field's conditioning-scaled tolerance capped at 1e-3); the gradient error is printed beside
    its conditioning S and asserted only where 10 S <= 1e-3."""
    n, box, nr, seed = CASES["128_hier"]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, seed, point="raw")
    f, lp_o, g_o, _, cond = oracle_ref("128_raw", cfg, bias, nu, counts)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    check_fields(ctx, nu_d, c_d, bias, f, FP32_FIELD, scaled=True)
    lp, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias], want_bias_grad=False)
    e_g = rel_l2(g.double().cpu().numpy().reshape(g_o.shape), g_o)
    print(f"128 raw fp32: logpost rel {abs(lp[0] - lp_o) / abs(lp_o):.2e} grad rel L2 {e_g:.2e} S {cond:.2e}")
    assert abs(lp[0] - lp_o) <= FP32_LP * abs(lp_o)
    if 10 * cond <= CAP:
        assert e_g <= max(FP32_GRAD, 10 * cond)
    ctx.close()


def test_full_size_256_against_oracle():
    """256^3, L = 1000, 16 regions: the timed workload's mesh and launch configuration.  At the
    data-consistent point (treated) every field, the log posterior and the gradient hold the
    fixed bounds in both precisions; at nu_true + 0.1 noise as it is, the fields and the log
    posterior are checked (conditioning-scaled field tolerances capped at 1e-3), the gradient
    error is printed beside S, and the CIC mass is conserved."""
    cfg = synth.config(2)
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(cfg.n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    nu, c_t, moved, cleared = pp.condition(nu_t, counts, cfg, bias, gap=1e-3, clear_empty=True)
    print(f"256 truth: {moved} cells moved off the collapse threshold, {cleared} near-empty cells cleared")
    for precision in ("fp64", "fp32"):
        ctx = _full_check("256_truth", cfg, bias, nu, c_t, precision, conditioning="fields", psi=True)[0]
        ctx.close()
        del ctx
    nu_r = pp.f32(synth.eval_point(cfg.n, cfg.seed_truth, cfg.seed_eval, scale=0.1))
    f, lp_o, g_o, _, cond = oracle_ref("256_raw", cfg, bias, nu_r, counts)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu_r, counts, pkg.BRIDGE_FP32)
    check_fields(ctx, nu_d, c_d, bias, f, FP32_FIELD, scaled=True)
    lp, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias], want_bias_grad=False)
    e_g = rel_l2(g.double().cpu().numpy().reshape(g_o.shape), g_o)
    print(f"256 raw fp32: logpost rel {abs(lp[0] - lp_o) / abs(lp_o):.2e} grad rel L2 {e_g:.2e} S {cond:.2e}")
    assert abs(lp[0] - lp_o) <= FP32_LP * abs(lp_o)
    if 10 * cond <= CAP:
        assert e_g <= max(FP32_GRAD, 10 * cond)
    delta = ctx.bridge_debug_field(nu_d, c_d, [bias], pkg.FIELD_DELTA).double().cpu().numpy()
    assert abs(delta.sum()) <= 1e-6 * delta.size      # CIC conserves mass
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_second_cutoff_against_oracle(precision):
    """Eq. local_bias with the second cut-off switched on (rho' > 0 in every region; Table 3 has
    rho' = 0, so the default workloads never exercise it), at the data-consistent point."""
    cfg = synth.Config("32^3 cut2", 32, 300.0, n_regions=16, mean_tracers=0.5, seed_truth=1501,
                       seed_counts=1502, seed_eval=1503)
    bias = synth.default_bias(cfg).copy()
    bias.rhop = [0.2] * 16
    bias.epsp = [1.2] * 16
    nu_t = synth.white_noise(cfg.n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    nu, counts, _, _ = pp.condition(nu_t, counts, cfg, bias, clear_empty=True)
    ctx = _full_check("32_cut2", cfg, bias, nu, counts, precision)[0]
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_collapse_branch_and_density_floor(precision):
    """Edge cases of Sect. 2.3 and reading G8: growth D = 2.5 puts a third of the cells on the
    collapsed spherical-collapse branch (theta_SC = -3, zero derivative) and empties cells, and
    rho_floor = 1e-3 floors them.  Counts of cells between the floor and a mass of 1e-2 are
    cleared (ill-conditioned); cells deep on the floor (mass < 1e-4) get tracers, so the floored
    likelihood term -- constant in nu -- is exercised."""
    cfg = synth.Config("32^3 collapse", 32, 300.0, n_regions=4, nb_beta=5.0, growth_d=2.5, rho_floor=1e-3,
                       seed_truth=1601, seed_counts=1602, seed_eval=1603)
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(cfg.n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    nu, _ = pp.off_collapse(nu_t, cfg, 1e-3)
    counts = pp.clear_near_empty(nu, counts, cfg, bias, mass=1e-2, keep_below=1e-4)
    f = model.forward_fields(nu, counts, cfg, bias)
    rho = 1.0 + f["delta"]
    deep = np.flatnonzero(rho.ravel() < 1e-4)
    collapsed = float(np.mean(cfg.growth_d * f["delta0"] >= 1.5))
    print(f"collapsed fraction {collapsed:.2f}, cells on the floor {int((rho < 1e-3).sum())}, deep {deep.size}")
    assert collapsed > 0.2 and deep.size >= 8
    counts = counts.copy()
    counts.ravel()[deep[:: max(1, deep.size // 8)][:8]] = 2
    ctx = _full_check("32_collapse", cfg, bias, nu, counts, precision)[0]
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_plane_wave_eigenvalue_tie(precision):
    """A white noise that varies along x only gives x-only delta0, displacement and density, so
    T = diag(t(x), 0, 0) and H = diag(h(x), 0, 0): two eigenvalues tie at 0 in every cell, and
    the web adjoint takes its tie branch (reading G9).  At a tie the gradient is a subgradient,
    defined up to the split between the tied pair; the split changes only the y-z components
    of the tensor adjoint, which an x-only spectrum multiplies by ky^2/k^2 = kz^2/k^2 = 0.  So
    the x-only part of the gradient (its mean over y, z) is unique and is compared with the
    oracle's; the rest must be finite.  Fields and the log posterior are compared as usual.
    The amplitude keeps |t| and |h| away from 0 (no triple tie) and D delta0 < 3/2."""
    n, box = 32, 300.0
    cfg = synth.Config("32^3 plane wave", n, box, n_regions=16, seed_truth=1701, seed_counts=1702)
    bias = synth.default_bias(cfg)
    x = np.arange(n)
    prof = 0.18 * np.cos(2 * np.pi * 2 * (x + 0.37) / n) + 0.05 * np.sin(2 * np.pi * 3 * x / n)
    nu = pp.f32(np.broadcast_to(prof[:, None, None], (n, n, n)).copy())
    counts = mock.mock_counts(nu, cfg, bias, cfg.seed_counts)
    f = model.forward_fields(nu, counts, cfg, bias)
    t_xx, h_xx = f["T"][0][:, 0, 0], f["H"][0][:, 0, 0]
    print(f"min |t| {np.abs(t_xx).min():.2e} min |h| {np.abs(h_xx).min():.2e} "
          f"max D delta0 {cfg.growth_d * f['delta0'].max():.2f}")
    assert np.abs(t_xx).min() > 1e-3 and np.abs(h_xx).min() > 1e-4 and cfg.growth_d * f["delta0"].max() < 1.4
    ftol, gtol, ltol = bounds(precision)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec_code(precision))
    f["cond"] = {}
    check_fields(ctx, nu_d, c_d, bias, f, ftol)
    lp_o, g_o, _, _ = model.logpost_and_grad(nu, counts, cfg, bias)
    lp, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias], want_bias_grad=False)
    g = g.double().cpu().numpy().reshape(n, n, n)
    assert np.all(np.isfinite(g))
    e_x = rel_l2(g.mean(axis=(1, 2)), g_o.mean(axis=(1, 2)))
    print(f"plane wave {precision}: logpost rel {abs(lp[0] - lp_o) / abs(lp_o):.2e} x-only gradient rel L2 {e_x:.2e}")
    assert abs(lp[0] - lp_o) <= ltol * abs(lp_o)
    assert e_x <= gtol
    ctx.close()


@pytest.mark.parametrize("name,precision", [("64_hier", "fp32"), ("16_phi", "fp64")])
def test_autotune_keeps_results_and_later_calls_work(name, precision):
    """bridge_autotune only changes launch shapes: the gradient after tuning matches the oracle
    and the one before tuning, on two calls, and a leapfrog trajectory (its own captured graph)
    still runs.  Before and after are not bit-identical (float atomics of the CIC deposit)."""
    n, box, nr, seed = CASES[name]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, seed, point="eval")
    f, lp_o, g_o, _, cond = oracle_ref(name, cfg, bias, nu, counts)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec_code(precision))
    _, g0, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias], want_bias_grad=False)
    g0 = g0.double().cpu().numpy()
    choices = ctx.bridge_autotune(nu_d, c_d, [bias])
    print(f"autotune {name} {precision}: {choices}")
    assert len(choices) == 4 and all(c in (0, 1, 2, 3, 4, 5, 6, 8) for c in choices[:3]) and choices[3] >= 0
    _, gtol, ltol = bounds(precision)
    for _ in range(2):
        lp, g, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias], want_bias_grad=False)
        g = g.double().cpu().numpy()
        assert abs(lp[0] - lp_o) <= ltol * abs(lp_o)
        assert rel_l2(g.reshape(g_o.shape), g_o) <= gtol
        assert rel_l2(g, g0) <= 0.1 * gtol
    p_d = torch.tensor(synth.momentum(n, seed + 7), dtype=nu_d.dtype, device="cuda").contiguous()
    h0, h1 = ctx.bridge_leapfrog(nu_d.clone(), p_d, c_d, [bias], 3, 1e-4)
    assert np.all(np.isfinite(h0)) and np.all(np.isfinite(h1))
    ctx.close()


@pytest.mark.parametrize("rsd_f,rsd_los", [(0.0, 0), (0.8, 0), (0.8, 1)])
def test_recompute_alpt_matches_stored(rsd_f, rsd_los):
    """recompute_alpt (the adjoint recomputes the ALPT spectra from nu) gives the same fields and
    gradient as the default path that keeps them, and both match the oracle, in real space and
    in redshift space (plane-parallel and radial line of sight)."""
    n, box, nr, seed = CASES["64_hier"]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, seed, point="eval", rsd_f=rsd_f, rsd_los=rsd_los)
    f, lp_o, g_o, gb_o, _ = oracle_ref(f"64_hier_rsd{rsd_f}_{rsd_los}", cfg, bias, nu, counts, conditioning=False)
    out = {}
    for rec in (False, True):
        ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32, recompute_alpt=rec)
        check_fields(ctx, nu_d, c_d, bias, f, FP32_FIELD)
        lp, g, gb = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
        out[rec] = (lp[0], g.double().cpu().numpy(), gb[0])
        assert rel_l2(out[rec][1].reshape(g_o.shape), g_o) <= FP32_GRAD
        assert abs(lp[0] - lp_o) <= FP32_LP * abs(lp_o)
        ctx.close()
    assert rel_l2(out[True][1], out[False][1]) <= 1e-5
    assert np.max(np.abs(out[True][2] - out[False][2])) <= 1e-5 * np.max(np.abs(out[False][2]))


@pytest.mark.parametrize("n,precision", [(32, "fp32"), (32, "fp64"), (64, "fp32"), (64, "fp64")])
def test_redshift_space_against_oracle(n, precision):
    """Sect. 2.9, plane-parallel along z with the linear velocity (f = 0.8, the large-field
    workload's value): counts drawn from the redshift-space model; every field (the displacement
    includes f Psi_1,z), the log posterior and the gradient (through the transposed RSD term)
    against the oracle at the fixed bounds."""
    box, nr = {32: (300.0, 4), 64: (500.0, 16)}[n]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, 1900 + n, point="eval", rsd_f=0.8)
    ctx, nu_d, c_d, _, _ = _full_check(f"rsd_{n}", cfg, bias, nu, counts, precision)
    real = synth.Config("real", n, box, n_regions=nr)
    psi_real = model.alpt_displacement(model.delta0_from_nu(torch.tensor(nu), real), real).numpy()
    psi = ctx.bridge_debug_field(nu_d, c_d, [bias], pkg.FIELD_PSI).double().cpu().numpy().reshape(psi_real.shape)
    moved = rel_l2(psi[2], psi_real[2])
    print(f"RSD moves Psi_z by {moved:.2e} (relative); Psi_x unchanged to {rel_l2(psi[0], psi_real[0]):.1e}")
    assert moved > 0.1 and rel_l2(psi[0], psi_real[0]) <= bounds(precision)[0]
    ctx.close()


def test_redshift_space_256():
    """The 256^3 workload in redshift space (f = 0.8), FP32, at the data-consistent point:
    fields, log posterior and gradient at the fixed bounds."""
    cfg = synth.config(2)
    cfg.rsd_f = 0.8
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(cfg.n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    nu, counts, _, cleared = pp.condition(nu_t, counts, cfg, bias, clear_empty=True)
    print(f"256 RSD truth: {cleared} near-empty cells cleared")
    ctx = _full_check("256_rsd", cfg, bias, nu, counts, "fp32", conditioning="fields", psi=True)[0]
    ctx.close()


@pytest.mark.parametrize("n,precision", [(32, "fp32"), (32, "fp64"), (64, "fp32"), (64, "fp64")])
def test_radial_redshift_space_against_oracle(n, precision):
    """Sect. 2.9 with the observer at the centre of the volume (radial line of sight, f = 0.8):
    counts drawn from the radial redshift-space model; every field (the displacement is the
    redshift-space one), the log posterior and the gradient (through the transposed per-particle
    projection and the linear displacement's k-space adjoint) against the oracle at the fixed
    bounds.  The displacement differs from the plane-parallel one in every component."""
    box, nr = {32: (300.0, 4), 64: (500.0, 16)}[n]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, 1950 + n, point="eval", rsd_f=0.8, rsd_los=1)
    ctx, nu_d, c_d, _, _ = _full_check(f"rsd_radial_{n}", cfg, bias, nu, counts, precision)
    plane = synth.Config("plane", n, box, n_regions=nr, rsd_f=0.8)
    psi_pp = model.alpt_displacement(model.delta0_from_nu(torch.tensor(nu), plane), plane).numpy()
    psi = ctx.bridge_debug_field(nu_d, c_d, [bias], pkg.FIELD_PSI).double().cpu().numpy().reshape(psi_pp.shape)
    diff = [rel_l2(psi[j], psi_pp[j]) for j in range(3)]
    print("radial vs plane-parallel displacement, per component: " + ", ".join(f"{d:.2e}" for d in diff))
    assert min(diff) > 0.05
    ctx.close()


def test_radial_redshift_space_256():
    """The 256^3 workload with the radial line of sight (f = 0.8), FP32, at the data-consistent
    point: fields, log posterior and gradient (tolerances as for the real-space workload)."""
    cfg = synth.config(2)
    cfg.rsd_f, cfg.rsd_los = 0.8, 1
    bias = synth.default_bias(cfg)
    nu_t = synth.white_noise(cfg.n, cfg.seed_truth)
    counts = mock.mock_counts(nu_t, cfg, bias, cfg.seed_counts)
    nu, counts, _, cleared = pp.condition(nu_t, counts, cfg, bias, clear_empty=True)
    print(f"256 radial RSD truth: {cleared} near-empty cells cleared")
    ctx = _full_check("256_rsd_radial", cfg, bias, nu, counts, "fp32", conditioning="fields", psi=True)[0]
    ctx.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_deterministic_mass_assignment(precision):
    """deterministic = 1: the CIC sums are 64-bit fixed point, so two evaluations of one input
    give bit-identical log posteriors and gradients (float atomics differ by rounding from run
    to run), and the results still match the oracle at the fixed bounds; the batched path gives
    each chain the same bits as its single-chain call."""
    n, box, nr, seed = CASES["64_hier"]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, seed, point="eval")
    f, lp_o, g_o, gb_o, _ = oracle_ref(f"64_hier_det_{precision}", cfg, bias, nu, counts, conditioning=False)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec_code(precision), deterministic=True)
    ftol, gtol, ltol = bounds(precision)
    check_fields(ctx, nu_d, c_d, bias, f, ftol)
    runs = [ctx.bridge_logpost_grad(nu_d, c_d, [bias]) for _ in range(3)]
    for lp, g, gb in runs[1:]:
        assert lp[0] == runs[0][0][0]
        assert torch.equal(g, runs[0][1]) and np.array_equal(gb, runs[0][2])
    lp, g, gb = runs[0]
    e_g = rel_l2(g.double().cpu().numpy().reshape(g_o.shape), g_o)
    print(f"deterministic {precision}: logpost rel {abs(lp[0] - lp_o) / abs(lp_o):.2e}, grad rel L2 {e_g:.2e}, "
          f"3 evaluations bit-identical")
    assert abs(lp[0] - lp_o) <= ltol * abs(lp_o) and e_g <= gtol
    # batched: each chain bit-identical to its single-chain evaluation
    cb = pkg.Context(pkg.config_from(cfg, precision=prec_code(precision), batch=2, deterministic=True))
    nu2 = torch.stack([nu_d, nu_d.flip(0)]).contiguous()
    c2 = torch.stack([c_d, c_d]).contiguous()
    lpb, gbt, _ = cb.bridge_logpost_grad(nu2, c2, [bias, bias])
    lp1, g1, _ = ctx.bridge_logpost_grad(nu2[1].contiguous(), c_d, [bias])
    assert lpb[0] == lp[0] and torch.equal(gbt[0], g)
    assert lpb[1] == lp1[0] and torch.equal(gbt[1], g1)
    cb.close()
    ctx.close()


def test_free_mask_and_tied_classes():
    """The library returns the gradient of the free bias parameters only: every entry untied,
    a subset in bit order, and the tied Phi-class parameters (sum over the delta sub-classes)."""
    n, box, nr, seed = CASES["64_hier"]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, seed, point="eval")
    _, _, ga, gbeta = model.logpost_and_grad(nu, counts, cfg, bias)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    for mask, tie in ((None, 0), (0b1000_0000_0000_0000_0000_0000_0000_0101, 0), (0xFF, 1), (0b0110_0001, 1)):
        b = bias.copy()
        b.free_mask, b.tie_classes = mask, tie
        _, _, gb = ctx.bridge_logpost_grad(nu_d, c_d, [b])
        ref = free_grad(ga, gbeta, b)
        assert gb.shape == (1, ref.size)
        err = np.max(np.abs(gb[0] - ref)) / np.max(np.abs(ref))
        print(f"free_mask {pkg.bias_array([b])[0].free_mask:#x} tie {tie}: {ref.size} parameters, rel {err:.2e}")
        assert err <= FP32_GRAD
    b = bias.copy()
    b.free_mask, b.tie_classes = 0, 0
    lp, _, gb = ctx.bridge_logpost_grad(nu_d, c_d, [b])
    assert gb is None and np.isfinite(lp[0])
    b.free_mask, b.tie_classes = 0x1FF, 1          # bit 8 is beyond 2 x 4 tied parameters
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_logpost_grad(nu_d, c_d, [b])
    assert e.value.status == pkg.BRIDGE_EINVAL
    ctx.close()


def test_batched_chains_match_single_and_oracle():
    """Three 32^3 chains with their own seeds and bias tables in one launch per pass: each
    matches a single-chain call and the oracle."""
    cases = [make_case(32, 300.0, 4, 1001 + 10 * b, point="eval") for b in range(3)]
    biases = synth.perturbed_biases(cases[0][1], 3, 6001)
    cfg = cases[0][0]
    ctx = pkg.Context(pkg.config_from(cfg, batch=3))
    nu = torch.tensor(np.stack([c[2] for c in cases]), dtype=torch.float32, device="cuda").contiguous()
    counts = torch.tensor(np.stack([c[3] for c in cases]), dtype=torch.int32, device="cuda").contiguous()
    lp, g, gb = ctx.bridge_logpost_grad(nu, counts, biases)
    single = pkg.Context(pkg.config_from(cfg, batch=1))
    for b in range(3):
        lp1, g1, gb1 = single.bridge_logpost_grad(nu[b].contiguous(), counts[b].contiguous(), [biases[b]])
        _, lp_o, g_o, _, cond = oracle_ref(f"batched{b}", cfg, biases[b], cases[b][2], cases[b][3])
        e = (abs(lp1[0] - lp[b]) / abs(lp[b]), rel_l2(g1.cpu().numpy(), g[b].cpu().numpy()),
             abs(lp[b] - lp_o) / abs(lp_o), rel_l2(g[b].double().cpu().numpy(), g_o))
        print(f"chain {b}: single-vs-batched lp {e[0]:.2e} grad {e[1]:.2e}; oracle lp {e[2]:.2e} grad {e[3]:.2e} "
              f"(S {cond:.1e})")
        assert e[0] <= 1e-7 and e[1] <= 1e-5
        assert e[2] <= FP32_LP and e[3] <= FP32_GRAD
        assert np.max(np.abs(gb1[0] - gb[b])) <= 1e-5 * np.max(np.abs(gb[b]))


def test_batched_16x128_workload():
    """The batched workload: 16 chains at 128^3 (L = 1000, 16 regions), each with its own seeds
    and perturbed alpha/beta tables, advanced in one launch per pass.  Every chain matches a
    single-chain call on the same input; chains 0 and 15 (treated data-consistent points) match
    the oracle at the fixed bounds."""
    cb = synth.config(3)
    base = synth.default_bias(cb)
    biases = synth.perturbed_biases(base, cb.batch, cb.seed_perturb)
    nus, cnts, ref = [], [], {}
    for b in range(cb.batch):
        if b in (0, cb.batch - 1):
            c = synth.Config(cb.name, cb.n, cb.box, n_regions=16, seed_truth=cb.seed_truth + 100 * b,
                             seed_counts=cb.seed_counts + 100 * b)
            nu_t = synth.white_noise(cb.n, c.seed_truth)
            counts = mock.mock_counts(nu_t, c, biases[b], c.seed_counts)
            nu, counts, _, _ = pp.condition(nu_t, counts, c, biases[b], clear_empty=True)
            ref[b] = oracle_ref(f"b16_{b}", c, biases[b], nu, counts, psi=True)
        else:
            nu = pp.f32(synth.white_noise(cb.n, cb.seed_truth + 100 * b))
            counts = synth.timing_counts(cb.n, cb.seed_counts + 100 * b, cb.mean_tracers)
        nus.append(nu)
        cnts.append(counts)
    ctx = pkg.Context(pkg.config_from(cb))
    nu_d = torch.tensor(np.stack(nus), dtype=torch.float32, device="cuda").contiguous()
    c_d = torch.tensor(np.stack(cnts), dtype=torch.int32, device="cuda").contiguous()
    lp, g, gb = ctx.bridge_logpost_grad(nu_d, c_d, biases)
    del ctx
    single = pkg.Context(pkg.config_from(cb, batch=1))
    # Two evaluations of one input differ by the order of the CIC atomic adds; at the untreated
    # chains that difference is amplified by their conditioning.  The batched gradient must agree
    # with the single-chain one to 1e-5 or, where larger, to three times the largest difference
    # between two single-chain evaluations of the same input.
    e_bat, e_rr, lps = [], [], []
    for b in range(cb.batch):
        lp1, g1, _ = single.bridge_logpost_grad(nu_d[b].contiguous(), c_d[b].contiguous(), [biases[b]])
        g1 = g1.cpu().numpy()
        _, g1b, _ = single.bridge_logpost_grad(nu_d[b].contiguous(), c_d[b].contiguous(), [biases[b]])
        e_bat.append(rel_l2(g1, g[b].cpu().numpy()))
        e_rr.append(rel_l2(g1b.cpu().numpy(), g1))
        lps.append(lp1[0])
    tol_b = max(1e-5, 3.0 * max(e_rr))
    print(f"16 x 128^3: batched vs single gradient rel L2 max {max(e_bat):.2e}, run-to-run max {max(e_rr):.2e} "
          f"(tolerance {tol_b:.1e})")
    for b in range(cb.batch):
        assert abs(lps[b] - lp[b]) <= 1e-7 * abs(lp[b]) and e_bat[b] <= tol_b, (b, e_bat[b], tol_b)
        if b in ref:
            f_o, lp_o, g_o, gb_o, cond = ref[b]
            e_o = rel_l2(g[b].double().cpu().numpy(), g_o)
            e_b = rel_l2(gb[b], gb_o)
            print(f"chain {b} vs oracle: lp {abs(lp[b] - lp_o) / abs(lp_o):.2e} grad {e_o:.2e} (S {cond:.1e}, "
                  f"S_psi {f_o['cond_psi']:.1e}) bias {e_b:.2e} (tol {bias_tol('fp32', f_o):.1e}, S {f_o['cond_bias']:.1e}, "
                  f"S_psi {f_o['cond_psi_bias']:.1e}, kappa {f_o['kappa_bias']:.0f})")
            assert abs(lp[b] - lp_o) <= FP32_LP * abs(lp_o) and e_o <= grad_tol("fp32", f_o)
            assert e_b <= bias_tol("fp32", f_o)


def central_differences(ctx, nu_d, c_d, bias, dirs, h):
    """(lp(nu + h d) - lp(nu - h d)) / 2h for each direction, log posteriors from bridge_forward."""
    out = []
    for d in dirs:
        dd = torch.tensor(d, dtype=torch.float64, device="cuda").reshape(nu_d.shape)
        lp_p, _ = ctx.bridge_forward((nu_d.double() + h * dd).to(nu_d.dtype).contiguous(), c_d, [bias])
        lp_m, _ = ctx.bridge_forward((nu_d.double() - h * dd).to(nu_d.dtype).contiguous(), c_d, [bias])
        out.append((lp_p[0] - lp_m[0]) / (2 * h))
        del dd
    return np.array(out)


def test_gradient_against_central_differences_128():
    """128^3 hierarchical workload: the hand-written gradient against central finite differences
    of the log posterior along 64 random unit directions.  The CIC weights are piecewise linear,
    so a difference quotient is exact only while no particle crosses a cell face within the
    step; the oracle itself reaches 1e-7 at 64^3 only below h = 1e-4.  Such steps need the FP64
    log posterior (the FP32 one carries ~1e-4 of field noise), so the differences come from the
    FP64 instantiation of the same kernels (h = 1e-5), and both the FP64 and the FP32 gradient
    are compared with them.  Point: data-consistent, 1e-2 off the collapse threshold."""
    n, box, nr, seed = CASES["128_hier"]
    cfg, bias, nu, counts, _ = make_case(n, box, nr, seed, point="truth", gap=1e-2)
    dirs = synth.directions(n, 4002, 64)
    c64, nu64, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP64)
    fd = central_differences(c64, nu64, c_d, bias, dirs, 1e-5)
    _, g64, _ = c64.bridge_logpost_grad(nu64, c_d, [bias], want_bias_grad=False)
    c32, nu32, _ = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    _, g32, _ = c32.bridge_logpost_grad(nu32, c_d, [bias], want_bias_grad=False)
    an64 = np.array([float(g64.double().cpu().numpy().ravel() @ d.ravel()) for d in dirs])
    an32 = np.array([float(g32.double().cpu().numpy().ravel() @ d.ravel()) for d in dirs])
    e64, e32 = rel_l2(an64, fd), rel_l2(an32, fd)
    med = np.median(np.abs(an64 - fd) / np.abs(fd))
    print(f"FD 128^3 (FP64, h = 1e-5, 64 directions): FP64 gradient rel L2 {e64:.2e} (median per direction "
          f"{med:.1e}), FP32 gradient {e32:.2e}; |<g,d>| median {np.median(np.abs(fd)):.2e}")
    assert e64 <= 1e-3 and e32 <= 1e-3
    c64.close()
    c32.close()


def test_large_single_field_512():
    """512^3, L = 2000, beta = 2, 0.05 tracers per cell, the large-field workload.  Checks that
    hold at any size or that the oracle can do cell by cell: delta0 at 16 cells against the
    inverse DFT written out at each cell; CIC mass conservation; sum of nbar = N_tr; the FP32
    gradient against the FP64 path's gradient on the same input (the FP64 path matches the
    oracle at <= 256^3 with the same kernel templates); the FP64 gradient against central
    differences along 4 random directions (h = 1e-5).  Counts: a gamma-Poisson draw (beta = 2)
    from the FP64 path's own nbar at nu (a data-consistent point), tracers removed from cells
    with a CIC mass below 1e-2, nu kept 1e-3 off the collapse threshold."""
    c5 = synth.config(4)
    b5 = synth.default_bias(c5)
    nu, moved = pp.off_collapse(synth.white_noise(c5.n, c5.seed_eval), c5, 1e-3)
    seed_counts = np.zeros(c5.n ** 3, dtype=np.int32) + 1
    c64, nu64, ones = run_gpu(c5, b5, nu, seed_counts, pkg.BRIDGE_FP64)
    _, lnnbar = c64.bridge_forward(nu64, ones, [b5], want_ln_nbar=True)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(c5.seed_counts)
    # nbar of the model normalised to N_tr = N^3 (unit counts), rescaled to 0.05 tracers per cell
    lam = c5.mean_tracers * torch.exp(lnnbar) * torch._standard_gamma(torch.full_like(lnnbar, 2.0), generator=gen) / 2.0
    lnnbar = None
    counts = torch.poisson(lam, generator=gen).clamp_(max=65535).to(torch.int32).reshape(ones.shape).contiguous()
    del lam, ones
    # as at the smaller meshes, no tracers in cells with a CIC mass below 1e-2 (here the FP64
    # path's mass: this check compares two precisions of the library, no oracle output involved)
    rho = c64.bridge_debug_field(nu64, counts, [b5], pkg.FIELD_DELTA).reshape(counts.shape) + 1.0
    cleared = int(((rho < 1e-2) & (counts > 0)).sum())
    counts[rho < 1e-2] = 0
    del rho
    ntr = float(counts.sum())
    d0 = c64.bridge_debug_field(nu64, counts, [b5], pkg.FIELD_DELTA0).cpu().numpy().reshape(-1)
    cells = np.random.default_rng(5).integers(0, c5.n ** 3, 16)
    e0_64 = rel_l2(d0[cells], model.delta0_at_cells(nu, c5, cells))
    _, g64, _ = c64.bridge_logpost_grad(nu64, counts, [b5], want_bias_grad=False)
    dirs = synth.directions(c5.n, 4005, 4)
    fd = central_differences(c64, nu64, counts, b5, dirs, 1e-5)
    an = np.array([float((g64.reshape(-1) * torch.tensor(d, device="cuda").reshape(-1)).sum()) for d in dirs])
    e_fd = rel_l2(an, fd)
    g64 = g64.cpu()
    c64.close()
    del c64, nu64
    c32 = pkg.Context(pkg.config_from(c5, batch=1))
    nu32 = torch.tensor(nu, dtype=torch.float32, device="cuda").contiguous()
    d0 = c32.bridge_debug_field(nu32, counts, [b5], pkg.FIELD_DELTA0).double().cpu().numpy().reshape(-1)
    e0 = rel_l2(d0[cells], model.delta0_at_cells(nu, c5, cells))
    delta = c32.bridge_debug_field(nu32, counts, [b5], pkg.FIELD_DELTA).double().cpu().numpy()
    lnn = c32.bridge_debug_field(nu32, counts, [b5], pkg.FIELD_LNNBAR).double().cpu().numpy()
    e_n = abs(np.exp(lnn).sum() / ntr - 1)
    _, g32, _ = c32.bridge_logpost_grad(nu32, counts, [b5], want_bias_grad=False)
    e_g = rel_l2(g32.double().cpu().numpy(), g64.numpy())
    print(f"512: moved {moved}, cleared {cleared}; delta0 samples rel FP32 {e0:.2e} FP64 {e0_64:.2e}; mass "
          f"{abs(delta.sum()) / delta.size:.2e}; sum nbar / N_tr - 1 = {e_n:.2e}; FP32 vs FP64 gradient {e_g:.2e}; "
          f"FP64 gradient vs FD (4 directions) {e_fd:.2e}")
    assert e0 <= FP32_FIELD and e0_64 <= FP64_FIELD
    assert abs(delta.sum()) <= 1e-6 * delta.size
    assert e_n <= 1e-6
    # FP32 vs FP64: bounded by the particles within the FP32 position error of a CIC cell face
    # (grad_tol; 2.3e-3 measured against the oracle at 256^3), never above 5e-3
    assert e_g <= CAP_PSI
    assert e_fd <= 1e-3
    c32.close()


def test_autograd_function_against_oracle_and_fd():
    """torch.autograd through log_posterior: forward runs bridge_forward only; backward runs
    bridge_logpost_vjp (forward again from nu, then the adjoint).  FP32 and FP64 contexts: the
    gradient matches the oracle at 32^3 (fixed bounds); the FP64 one matches central
    differences along 4 directions (h = 1e-6: no particle crosses a cell face within the step);
    the incoming gradient scales the result."""
    cfg, bias, nu, counts, _ = make_case(32, 300.0, 4, 1001, point="eval")
    _, lp_o, g_o, _, _ = oracle_ref("32_phi_ag", cfg, bias, nu, counts, conditioning=False)
    for precision in ("fp32", "fp64"):
        _, gtol, ltol = bounds(precision)
        ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec_code(precision))
        x = nu_d.clone().requires_grad_(True)
        lp = pkg.log_posterior(ctx, x, c_d, [bias])
        fwd_launches = ctx.launches()
        (gx,) = torch.autograd.grad(3.0 * lp.sum(), x)
        gx = gx.double().cpu().numpy() / 3.0
        assert abs(float(lp.detach()[0]) - lp_o) <= ltol * abs(lp_o)
        e = rel_l2(gx, g_o.reshape(gx.shape))
        _, g_full, _ = ctx.bridge_logpost_grad(nu_d, c_d, [bias], want_bias_grad=False)
        print(f"autograd {precision}: grad rel L2 vs oracle {e:.2e}; launches forward-only {fwd_launches}, "
              f"full evaluation {ctx.launches()}")
        assert e <= gtol
        assert fwd_launches < ctx.launches()
        if precision == "fp64":
            dirs = synth.directions(32, 4001, 4)
            fd = central_differences(ctx, nu_d, c_d, bias, dirs, 1e-6)
            an = np.array([float(gx.ravel() @ d.ravel()) for d in dirs])
            print(f"autograd fp64 vs FD: rel L2 {rel_l2(an, fd):.2e}")
            assert rel_l2(an, fd) <= 1e-6
        # vjp with per-chain cotangents
        g2, gb2 = ctx.bridge_logpost_vjp(nu_d, c_d, [bias], cotangent=[-0.5], want_bias_grad=True)
        _, g1, gb1 = ctx.bridge_logpost_grad(nu_d, c_d, [bias])
        assert rel_l2(g2.cpu().numpy(), -0.5 * g1.cpu().numpy()) <= 1e-6
        assert np.max(np.abs(gb2 + 0.5 * gb1)) <= 1e-6 * np.max(np.abs(gb1))
        # host-buffer entry point (counts copied and prepared while the forward fields run):
        # the same results as the device path, on repeated calls with new inputs, with the bias
        # gradient, and an out-of-range count still reported
        hdt = torch.float64 if precision == "fp64" else torch.float32
        htol = 1e-12 if precision == "fp64" else 1e-6
        c_h = torch.tensor(counts, dtype=torch.int32).pin_memory()
        for k, shift in enumerate((0.0, 0.01)):
            nu_k = nu + shift * pp.f32(synth.white_noise(32, 4100 + k))
            nu_h = torch.tensor(nu_k, dtype=hdt).pin_memory()
            g_h = torch.empty_like(nu_h).pin_memory()
            lp_h, gb_h = ctx.bridge_logpost_grad_host(nu_h, c_h, [bias], g_h, want_bias_grad=True)
            lp_d, g_dev, gb_d = ctx.bridge_logpost_grad(nu_h.to("cuda"), c_d, [bias])
            assert abs(lp_h[0] - lp_d[0]) <= htol * abs(lp_d[0])
            assert rel_l2(g_h.numpy(), g_dev.cpu().numpy()) <= htol
            assert np.max(np.abs(gb_h - gb_d)) <= htol * np.max(np.abs(gb_d))
        bad = c_h.clone()
        bad[0, 0, 0] = 70000
        with pytest.raises(pkg.BridgeError) as e:
            ctx.bridge_logpost_grad_host(nu_h, bad, [bias], g_h)
        assert e.value.status == pkg.BRIDGE_EINVAL
        ctx.bridge_logpost_grad_host(nu_h, c_h, [bias], g_h)
        ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_leapfrog_matches_oracle(precision):
    cfg, bias, nu, counts, _ = make_case(16, 160.0, 4, 1301, point="eval")
    p0 = pp.f32(synth.momentum(16, 1304))
    nu_o, p_o, h0_o, h1_o = hmc.leapfrog(nu, p0, counts, cfg, bias, 4, 0.05)
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, prec_code(precision))
    p_d = torch.tensor(p0, dtype=nu_d.dtype, device="cuda").contiguous()
    h0, h1 = ctx.bridge_leapfrog(nu_d, p_d, c_d, [bias], 4, 0.05)
    tol = 1e-10 if precision == "fp64" else 1e-5
    e_nu = rel_l2(nu_d.double().cpu().numpy(), nu_o)
    e_p = rel_l2(p_d.double().cpu().numpy(), p_o)
    print(f"leapfrog {precision}: nu {e_nu:.2e} p {e_p:.2e} dH gpu {h1[0] - h0[0]:.6e} oracle {h1_o - h0_o:.6e}")
    assert e_nu <= tol and e_p <= tol * 10
    assert abs(h0[0] - h0_o) <= tol * abs(h0_o)
    if precision == "fp64":
        assert abs((h1[0] - h0[0]) - (h1_o - h0_o)) <= 1e-8 * max(1.0, abs(h1_o - h0_o))
    else:
        assert abs((h1[0] - h0[0]) - (h1_o - h0_o)) <= 1e-2 * max(1.0, abs(h1_o - h0_o))


def test_leapfrog_restores_a_diverged_chain():
    """Two chains in one call; chain 1 starts from a non-finite white noise (made on the host).
    Its Hamiltonian is not finite: the call reports ENONFINITE, writes H for both chains, puts
    chain 1's nu and p back as they were, and leaves chain 0 at the end point that a
    single-chain call reaches."""
    cfg, bias, nu, counts, _ = make_case(16, 160.0, 4, 1801, point="eval")
    p0 = pp.f32(synth.momentum(16, 1802))
    ctx = pkg.Context(pkg.config_from(cfg, batch=2))
    nu2 = np.stack([nu, nu]).astype(np.float32)
    nu2[1, 3, 4, 5] = np.nan
    nu_d = torch.tensor(nu2, device="cuda").contiguous()
    p_d = torch.tensor(np.stack([p0, p0]), dtype=torch.float32, device="cuda").contiguous()
    c_d = torch.tensor(np.stack([counts, counts]), dtype=torch.int32, device="cuda").contiguous()
    nu_start, p_start = nu_d.clone(), p_d.clone()
    st = pkg.lib().bridge_leapfrog(ctx.handle, nu_d.data_ptr(), p_d.data_ptr(), c_d.data_ptr(),
                                   pkg.bias_array([bias, bias]), 3, 0.02, None, None)
    assert st == pkg.BRIDGE_ENONFINITE
    assert b"1 of 2" in pkg.lib().bridge_last_error(ctx.handle)
    nu_d.copy_(nu_start)
    p_d.copy_(p_start)
    h0, h1 = ctx.bridge_leapfrog(nu_d, p_d, c_d, [bias, bias], 3, 0.02)
    assert np.isfinite(h0[0]) and np.isfinite(h1[0]) and not (np.isfinite(h0[1]) and np.isfinite(h1[1]))
    # bit-for-bit (the start state holds a NaN, which compares unequal to itself)
    assert torch.equal(nu_d[1].view(torch.int32), nu_start[1].view(torch.int32))
    assert torch.equal(p_d[1].view(torch.int32), p_start[1].view(torch.int32))
    one = pkg.Context(pkg.config_from(cfg, batch=1))
    nu1, p1 = nu_start[0].clone(), p_start[0].clone()
    g0, g1 = one.bridge_leapfrog(nu1, p1, c_d[0].contiguous(), [bias], 3, 0.02)
    assert rel_l2(nu_d[0].cpu().numpy(), nu1.cpu().numpy()) <= 1e-6
    assert abs(h1[0] - g1[0]) <= 1e-6 * abs(g1[0])


def test_invalid_inputs_return_errors():
    cfg, bias, nu, counts, _ = make_case(16, 160.0, 4, 1401, point="raw")
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
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_logpost_vjp(nu_d, c_d, [bias], cotangent=[float("inf")])
    assert e.value.status == pkg.BRIDGE_EINVAL
    # a buffer that does not start on a 16-byte boundary is refused before any launch
    raw = torch.empty(nu_d.numel() + 1, dtype=nu_d.dtype, device="cuda")
    shifted = raw[1:]
    shifted.copy_(nu_d.reshape(-1))
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_logpost_grad(shifted, c_d, [bias])
    assert e.value.status == pkg.BRIDGE_EINVAL and "16-byte" in str(e.value)


@pytest.mark.parametrize("n,precision", [(32, "fp32"), (256, "fp32"), (64, "fp64"), (256, "fp64")])
def test_fft_roundtrip(n, precision):
    """The pass kernels' 3D real DFT followed by its inverse returns the input (App. A
    conventions: the inverse carries 1/N^3), for two chains at once."""
    cfg = synth.Config("fft", n, 1000.0 * n / 256, n_regions=4)
    ctx = pkg.Context(pkg.config_from(cfg, precision=prec_code(precision), batch=2))
    dt = torch.float64 if precision == "fp64" else torch.float32
    x = torch.tensor(synth.white_noise(n, 77, 2), dtype=dt, device="cuda").reshape(2, -1).contiguous()
    y = ctx.bridge_fft_roundtrip(x)
    e = rel_l2(y.cpu().numpy(), x.cpu().numpy())
    print(f"fft roundtrip {n}^3 {precision}: rel L2 {e:.2e}")
    assert e <= (1e-6 if precision == "fp32" else 1e-14)
    ctx.close()


@pytest.mark.parametrize("n,precision", [(32, "fp32"), (32, "fp64"), (128, "fp32"), (128, "fp64")])
def test_wiener_init_against_oracle(n, precision):
    """Sect. 2.2 chain initialisation: two chains (own mock counts) in one call against the
    oracle's Wiener filter (itself pinned to the dense real-space S (S + N)^-1 d); a chain with
    no tracers is refused."""
    box, nr = {32: (300.0, 4), 128: (1000.0, 16)}[n]
    counts, refs = [], []
    for b in range(2):
        cfg = synth.Config(f"{n}^3", n, box, n_regions=nr, seed_truth=2100 + 10 * b, seed_counts=2101 + 10 * b)
        bias = synth.default_bias(cfg)
        c = mock.mock_counts(synth.white_noise(n, cfg.seed_truth), cfg, bias, cfg.seed_counts)
        counts.append(c)
        refs.append(model.wiener_init(c, cfg))
    ctx = pkg.Context(pkg.config_from(cfg, precision=prec_code(precision), batch=2))
    c_d = torch.tensor(np.stack(counts), dtype=torch.int32, device="cuda").contiguous()
    nu0 = ctx.bridge_wiener_init(c_d).double().cpu().numpy()
    errs = [rel_l2(nu0[b], refs[b]) for b in range(2)]
    print(f"Wiener init {n}^3 {precision}: rel L2 {errs[0]:.2e} {errs[1]:.2e}; mean {np.abs(nu0.mean(axis=(1, 2, 3))).max():.1e}")
    tol = FP32_FIELD if precision == "fp32" else FP64_FIELD
    assert max(errs) <= tol
    empty = c_d.clone()
    empty[1].zero_()
    with pytest.raises(pkg.BridgeError) as e:
        ctx.bridge_wiener_init(empty)
    assert e.value.status == pkg.BRIDGE_EINVAL and "no tracers" in str(e.value)
    ctx.close()


@pytest.mark.parametrize("scheme", ["bcss2", "yoshida4"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_higher_order_integrators_match_oracle(scheme, precision):
    """Two-stage (Blanes et al. 2014) and fourth-order (Yoshida) splittings against the oracle's
    integrator: end state and Hamiltonians after 3 steps, 16^3, two chains in one call."""
    cfg, bias, nu, counts, _ = make_case(16, 160.0, 4, 1311, point="eval")
    p0 = pp.f32(synth.momentum(16, 1314))
    nu_o, p_o, h0_o, h1_o = hmc.integrate(nu, p0, counts, cfg, bias, 3, 0.04, scheme)
    code = {"bcss2": pkg.BRIDGE_TWO_STAGE, "yoshida4": pkg.BRIDGE_FOURTH_ORDER}[scheme]
    ctx = pkg.Context(pkg.config_from(cfg, precision=prec_code(precision), batch=2))
    dt = torch.float64 if precision == "fp64" else torch.float32
    nu_d = torch.tensor(np.stack([nu, nu]), dtype=dt, device="cuda").contiguous()
    p_d = torch.tensor(np.stack([p0, p0]), dtype=dt, device="cuda").contiguous()
    c_d = torch.tensor(np.stack([counts, counts]), dtype=torch.int32, device="cuda").contiguous()
    h0, h1 = ctx.bridge_integrate(nu_d, p_d, c_d, [bias, bias], code, 3, 0.04)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for b in range(2):
        e_nu = rel_l2(nu_d[b].double().cpu().numpy(), nu_o)
        e_p = rel_l2(p_d[b].double().cpu().numpy(), p_o)
        print(f"{scheme} {precision} chain {b}: nu {e_nu:.2e} p {e_p:.2e} dH {h1[b] - h0[b]:.6e} oracle {h1_o - h0_o:.6e}")
        assert e_nu <= tol and e_p <= 10 * tol
        assert abs(h0[b] - h0_o) <= tol * abs(h0_o)
        dtol = 1e-8 if precision == "fp64" else 1e-2
        assert abs((h1[b] - h0[b]) - (h1_o - h0_o)) <= dtol * max(1.0, abs(h1_o - h0_o))
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_joint_bias_integration_matches_oracle(precision):
    """Joint (nu, ln b) trajectory, 3 leapfrog steps, two chains with their own theta and momenta,
    against the oracle's joint integrator: end states of nu, p, theta, p_theta and the
    Hamiltonians (with the Jacobian term)."""
    cfg, bias, nu, counts, _ = make_case(16, 160.0, 4, 1331, point="eval")
    bias = bias.copy()
    bias.free_mask, bias.tie_classes = 0xFF, 0
    rng = np.random.default_rng(1332)
    p0 = pp.f32(synth.momentum(16, 1333))
    th0 = [np.log(np.concatenate([bias.alpha, bias.beta])) + 0.02 * rng.standard_normal(8) for _ in range(2)]
    pt0 = [rng.standard_normal(8) for _ in range(2)]
    ref = [hmc.integrate_joint(nu, p0, th0[b], pt0[b], counts, cfg, bias, 3, 0.01) for b in range(2)]
    ctx = pkg.Context(pkg.config_from(cfg, precision=prec_code(precision), batch=2))
    dt = torch.float64 if precision == "fp64" else torch.float32
    nu_d = torch.tensor(np.stack([nu, nu]), dtype=dt, device="cuda").contiguous()
    p_d = torch.tensor(np.stack([p0, p0]), dtype=dt, device="cuda").contiguous()
    c_d = torch.tensor(np.stack([counts, counts]), dtype=torch.int32, device="cuda").contiguous()
    th = np.ascontiguousarray(np.stack(th0))
    pt = np.ascontiguousarray(np.stack(pt0))
    h0, h1 = ctx.bridge_integrate_joint(nu_d, p_d, th, pt, c_d, [bias, bias], pkg.BRIDGE_LEAPFROG, 3, 0.01)
    tol = 1e-10 if precision == "fp64" else 1e-5
    for b in range(2):
        nu_o, p_o, th_o, pt_o, h0_o, h1_o = ref[b]
        e = (rel_l2(nu_d[b].double().cpu().numpy(), nu_o), rel_l2(p_d[b].double().cpu().numpy(), p_o),
             rel_l2(th[b], th_o), rel_l2(pt[b], pt_o))
        print(f"joint {precision} chain {b}: nu {e[0]:.2e} p {e[1]:.2e} theta {e[2]:.2e} p_theta {e[3]:.2e} "
              f"dH {h1[b] - h0[b]:.6e} oracle {h1_o - h0_o:.6e}")
        assert e[0] <= tol and e[1] <= 10 * tol and e[2] <= tol and e[3] <= 10 * tol
        assert abs(h0[b] - h0_o) <= tol * abs(h0_o)
        assert abs((h1[b] - h0[b]) - (h1_o - h0_o)) <= (1e-8 if precision == "fp64" else 1e-2) * max(1.0, abs(h1_o - h0_o))
    tied = bias.copy()
    tied.free_mask, tied.tie_classes = 0xF, 0
    with pytest.raises(ValueError):
        ctx.bridge_integrate_joint(nu_d, p_d, th, pt, c_d, [tied, tied], pkg.BRIDGE_LEAPFROG, 1, 0.01)
    ctx.close()


def test_nuts_host_driver_matches_oracle():
    """The host-driven NUTS (paper_2506_03969_gb300.nuts) on the FP64 path against the oracle's
    NUTS with the same seeded draws, 16^3: three transitions, each started from the oracle's
    previous sample, take the same tree depth and number of leapfrog steps and reach the same
    sample.  (The FP64 path is not bit-reproducible -- CIC float atomics -- and differences of
    1e-16 grow to ~1e-9 along a 63-step trajectory, enough to flip a U-turn test that sits near
    zero; trees are therefore kept to depth 5 and not chained.)  An FP32 context runs the same
    transition to a finite sample."""
    from paper_2506_03969_gb300 import nuts
    cfg, bias, nu, counts, _ = make_case(16, 160.0, 4, 1341, point="eval")
    x_o = nu.copy()
    rng_p = np.random.default_rng(8)
    moms = [pp.f32(rng_p.standard_normal(nu.shape)) for _ in range(3)]
    ctx, nu_d, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP64)
    sampler = nuts.NUTS(ctx, c_d, [bias], eps=0.05, max_depth=5)
    for t in range(3):
        rng_o, rng_g = np.random.default_rng(7 + t), np.random.default_rng(7 + t)
        x_g = torch.tensor(x_o, dtype=torch.float64, device="cuda").contiguous()
        lp, g, _ = ctx.bridge_logpost_grad(x_g, c_d, [bias], want_bias_grad=False)
        x_new, depth_o, steps_o, acc_o = hmc.nuts_step(x_o, moms[t], counts, cfg, bias, 0.05, rng_o, max_depth=5,
                                                       with_accept=True)
        p_d = torch.tensor(moms[t], dtype=torch.float64, device="cuda").contiguous()
        res = sampler.step(x_g, p_d, g, float(lp[0]), rng_g)
        e = rel_l2(res.nu.cpu().numpy(), x_new)
        print(f"NUTS transition {t}: depth {res.depth} / {depth_o}, leapfrog steps {res.n_leapfrog} / {steps_o}, "
              f"sample rel L2 {e:.2e}, acceptance statistic {res.accept_stat:.6f} / {acc_o:.6f}")
        assert res.depth == depth_o and res.n_leapfrog == steps_o and e <= 1e-8
        assert abs(res.accept_stat - acc_o) <= 1e-5
        x_o = x_new
    ctx.close()
    c32, nu32, c_d = run_gpu(cfg, bias, nu, counts, pkg.BRIDGE_FP32)
    s32 = nuts.NUTS(c32, c_d, [bias], eps=0.05, max_depth=6)
    lp, g, _ = c32.bridge_logpost_grad(nu32, c_d, [bias], want_bias_grad=False)
    res = s32.step(nu32, torch.tensor(moms[0], dtype=torch.float32, device="cuda").contiguous(), g, float(lp[0]),
                   np.random.default_rng(7))
    assert torch.isfinite(res.nu).all() and 2 ** (res.depth - 1) <= res.n_leapfrog <= 2 ** res.depth - 1
    c32.close()
