"""GPU parity for periodic systems (Sec. 2.3, Navon's reduction) through the C ABI:
general cyclic bands and the periodic hyperdiffusion matrix, implicit and
Crank-Nicolson steps, the paper's convergence study (Sec. 2.5, Fig. 2) run on
the GPU, and the singular-Schur-complement report.  Error metric and tolerance
as in test_gpu_solve.py: per-system max|x - x_ref| / max|x_ref| <= 1e-12."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1807_07382_gb300 as pb  # noqa: E402
from paper_1807_07382_gb300 import build  # noqa: E402

TOL = 1e-12
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def sys_err(x, ref, n):
    x = x.reshape(-1, n)
    ref = ref.reshape(-1, n)
    return float(np.max(np.max(np.abs(x - ref), axis=1) / np.max(np.abs(ref), axis=1)))


@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("n", [5, 6, 7, 8, 33, 256, 1024])
def test_periodic_general_band(n, shared):
    batch = 70
    nb = 1 if shared else batch
    band = synth.random_bands(nb, n, seed=700 + n, kind="diagdom")
    f = synth.uniform(710 + n, 0, batch * n, -1, 1)
    full = band if not shared else tuple(np.tile(v, batch) for v in band)
    ref = oracle.periodic_solve_batch(n, full, f)
    plan = pb.Plan(n, batch=batch, shared=shared, periodic=True)
    plan.factor(*[dev(v) for v in band])
    x = plan.solve(dev(f))
    assert plan.info()[0] == pb.PENT_OK
    assert sys_err(x.cpu().numpy(), ref, n) <= TOL
    # in place
    y = dev(f)
    plan.solve(y, y)
    assert sys_err(y.cpu().numpy(), ref, n) <= TOL


@pytest.mark.parametrize("sig_hi", [10.0, 1e3])
@pytest.mark.parametrize("cn", [False, True])
def test_periodic_hyperdiff_steps(cn, sig_hi):
    """sigma up to 10 (the workloads' range, kappa(A) <= 1 + 16 sigma = 161): 1e-12.  Up to 1e3 the two
    sides' rounding differences scale with kappa: 4 kappa u (u = 2^-53) is the bar there."""
    n, batch, steps = 200, 97, 12
    tol = max(TOL, 4 * (1 + 16 * sig_hi) * 2.0 ** -53)
    sig = synth.log_uniform(720, 0, batch, 1e-3, sig_hi)
    C0 = synth.uniform(720, batch, batch * n, -1, 1)
    ref = oracle.periodic_steps(n, sig, C0, steps, cn=cn)
    plan = pb.Plan(n, batch=batch, periodic=True)
    s = dev(sig)
    plan.factor_hyperdiff(s)
    C = dev(C0)
    if cn:
        plan.step(C, nu=s, nsteps=steps)
    else:
        plan.solve_steps(C, steps)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_err(C.cpu().numpy(), ref, n) <= tol


def test_periodic_cahn_hilliard_shared():
    n, batch, steps = 128, 40, 9
    sigma, mu = 4.0, 0.3
    C0 = synth.uniform(730, 0, batch * n, -0.5, 0.5)
    ref = oracle.explicit_steps(np.full(batch, n), [sigma], [mu], None, C0, steps, periodic=True, shared=True)
    plan = pb.Plan(n, batch=batch, shared=True, periodic=True)
    plan.factor_hyperdiff(dev([sigma]))
    C = dev(C0)
    for _ in range(steps):
        plan.step(C, mu=dev([mu]))
    assert sys_err(C.cpu().numpy(), ref, n) <= TOL
    mass0 = C0.reshape(batch, n).sum(1)
    assert np.max(np.abs(C.cpu().numpy().reshape(batch, n).sum(1) - mass0)) <= 1e-12 * np.abs(C0).reshape(batch, n).sum(1).max()


def test_periodic_convergence_exponent_on_gpu():
    """The paper's validation case (Sec. 2.5) run by the library: periodic Crank-Nicolson, 10^4 steps of
    dt = 1e-8 in one CUDA graph per N; Eq. (myerr) against the exact decaying harmonic, fitted exponent
    compared with the caption of Fig. 2.  Every field is also compared with the oracle; over 10^4 steps
    the high modes are barely damped (G -> -1), so the two sides' rounding differences add up: per step
    at most about 4 (1 + 32 sigma) u max|C| (right-hand-side terms up to 16 sigma |C|, and the solve),
    at most `steps` times, relative to the final amplitude."""
    g = json.load(open(os.path.join(GOLDEN, "paper_convergence.json")))
    k = 2 * math.pi * g["n"] / g["L"]
    T, dt = g["T"], g["dt"]
    steps = int(round(T / dt))
    Ns = [16, 32, 64, 128, 256]
    errs = []
    for N in Ns:
        dx = g["L"] / N
        x = np.arange(N) * dx
        sigma = g["gamma"] * g["D"] * dt / (2 * dx ** 4)
        c0 = g["amplitude"] * np.cos(k * x + g["phase"])
        plan = pb.Plan(N, batch=1, periodic=True)
        s = dev([sigma])
        plan.factor_hyperdiff(s)
        C = dev(c0)
        plan.step(C, nu=s, nsteps=steps)
        num = C.cpu().numpy()
        ref = oracle.periodic_steps(N, [sigma], c0, steps, cn=True)
        bound = steps * 4 * (1 + 32 * sigma) * 2.0 ** -53 / np.max(np.abs(ref))
        assert sys_err(num, ref, N) <= bound
        exact = g["amplitude"] * math.exp(-g["gamma"] * g["D"] * k ** 4 * T) * np.cos(k * x + g["phase"])
        errs.append(math.sqrt(np.mean((num - exact) ** 2)))
    slope = np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert abs(slope - g["fitted_exponent"]) < 0.03


def test_periodic_singular_schur_complement_reported():
    n, batch = 6, 3
    a, b, c, d, e = (np.zeros(batch * n) for _ in range(5))
    c[:] = 1.0
    c[1 * n + n - 2: 1 * n + n] = 0.0  # system 1: zero trailing 2 x 2 block, so S = 0
    plan = pb.Plan(n, batch=batch, periodic=True)
    plan.factor(*[dev(v) for v in (a, b, c, d, e)])
    st, bs, br, _ = plan.info()
    assert (st, bs, br) == (pb.PENT_ESINGULAR, 1, n - 2)


def test_periodic_rejects_unsupported_calls():
    plan = pb.Plan(16, batch=4, periodic=True)
    plan.factor_hyperdiff(dev(np.full(4, 0.5)))
    with pytest.raises(pb.PentError):
        plan.adjoint_solve(dev(np.zeros(64)))


# ----------------------------------------------------------------------------- FP32 + refinement

@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("n", [5, 6, 7, 9, 33, 256, 512, 1024, 3000, 6000])
def test_periodic_f32_refine_solve(n, shared):
    """The periodic hyperdiffusion matrix in FP32 + refinement: the FP32 solve of E, Navon's 2 x 2 tail, the
    float-float residual with wrapped neighbours; one CTA per system (a cluster beyond 4,096 rows)."""
    batch = 37
    nsig = 1 if shared else batch
    sig = synth.log_uniform(900 + n, 0, nsig, 1e-3, 10.0)
    f = synth.uniform(900 + n, nsig, batch * n, -1, 1)
    full_sig = np.broadcast_to(sig, (batch,))
    ref = np.concatenate([oracle.periodic_solve(oracle.band_periodic_hyperdiff(n, full_sig[s]), f[s * n:(s + 1) * n])
                          for s in range(batch)])
    plan = pb.Plan(n, batch=batch, shared=shared, periodic=True, precision=pb.PENT_F32_REFINE)
    plan.factor_hyperdiff(dev(sig))
    x = plan.solve(dev(f), max_refine=4)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_err(x.cpu().numpy(), ref, n) <= TOL


@pytest.mark.parametrize("cn", [False, True])
def test_periodic_f32_refine_steps(cn):
    n, batch, steps = 512, 70, 6
    sig = synth.log_uniform(910, 0, batch, 1e-3, 10.0)
    C0 = synth.uniform(910, batch, batch * n, -1, 1)
    ref = oracle.periodic_steps(n, sig, C0, steps, cn=cn)
    plan = pb.Plan(n, batch=batch, periodic=True, precision=pb.PENT_F32_REFINE)
    s = dev(sig)
    plan.factor_hyperdiff(s)
    C = dev(C0)
    if cn:
        plan.step(C, nu=s, nsteps=steps, max_refine=3)
    else:
        plan.solve_steps(C, steps, max_refine=3)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_err(C.cpu().numpy(), ref, n) <= TOL


def test_periodic_f32_refine_cahn_hilliard():
    n, batch, steps = 256, 50, 8
    sig = synth.log_uniform(920, 0, batch, 1e-2, 5.0)
    mu = synth.log_uniform(920, batch, batch, 1e-3, 0.3)
    C0 = synth.uniform(920, 2 * batch, batch * n, -0.8, 0.8)
    ref = oracle.explicit_steps(np.full(batch, n), sig, mu, None, C0, steps, periodic=True)
    plan = pb.Plan(n, batch=batch, periodic=True, precision=pb.PENT_F32_REFINE)
    plan.factor_hyperdiff(dev(sig))
    C = dev(C0)
    plan.step(C, mu=dev(mu), nsteps=steps, max_refine=3)
    assert sys_err(C.cpu().numpy(), ref, n) <= TOL


def test_periodic_f32_refine_convergence_exponent():
    """The paper's validation case (Sec. 2.5) in FP32 + refinement: 10^4 Crank-Nicolson steps per N."""
    g = json.load(open(os.path.join(GOLDEN, "paper_convergence.json")))
    k = 2 * math.pi * g["n"] / g["L"]
    T, dt = g["T"], g["dt"]
    steps = int(round(T / dt))
    Ns = [16, 32, 64, 128, 256]
    errs = []
    for N in Ns:
        dx = g["L"] / N
        x = np.arange(N) * dx
        sigma = g["gamma"] * g["D"] * dt / (2 * dx ** 4)
        c0 = g["amplitude"] * np.cos(k * x + g["phase"])
        plan = pb.Plan(N, batch=1, periodic=True, precision=pb.PENT_F32_REFINE)
        s = dev([sigma])
        plan.factor_hyperdiff(s)
        C = dev(c0)
        plan.step(C, nu=s, nsteps=steps, max_refine=3)
        num = C.cpu().numpy()
        ref = oracle.periodic_steps(N, [sigma], c0, steps, cn=True)
        # the FP32 path carries the field between steps as float pairs (48 bits): the per-step bound of
        # the FP64 test with 2^-48 in place of u
        bound = steps * 4 * (1 + 32 * sigma) * 2.0 ** -48 / np.max(np.abs(ref))
        assert sys_err(num, ref, N) <= bound
        exact = g["amplitude"] * math.exp(-g["gamma"] * g["D"] * k ** 4 * T) * np.cos(k * x + g["phase"])
        errs.append(math.sqrt(np.mean((num - exact) ** 2)))
    slope = np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert abs(slope - g["fitted_exponent"]) < 0.03


@pytest.mark.parametrize("prec", [pb.PENT_F64, pb.PENT_F32_REFINE])
def test_periodic_crank_nicolson_at_the_workloads_sigma(prec):
    """sigma_x = dt / (2 dx^4) = 343.6 (dt = 1e-8, N = 512: the periodic workload): the Crank-Nicolson
    right-hand side (I - sigma D4) C sums terms up to (1 + 16 sigma) |C| ~ 5500 |C|, so the FP32 path
    solves A y = 2 C and takes C' = y - C instead (the same scheme, without the cancellation).  The
    oracle evaluates that right-hand side in FP64: five rounded products summed, so its forward error is
    bounded by about 6 u (1 + 16 sigma) max|C| per step (u = 2^-53; the standard bound gamma_6 times the
    sum of the terms' magnitudes), which sets the bar above 1e-12 here."""
    w = synth.periodic_cn(batch=64, steps=3)
    n = int(w.n[0])
    ref = oracle.periodic_steps(n, w.sigma, w.field0, w.steps, cn=True, shared=True)
    plan = pb.Plan(n, batch=w.batch, shared=True, periodic=True, precision=prec)
    s = dev(w.sigma)
    plan.factor_hyperdiff(s)
    C = dev(w.field0)
    plan.step(C, nu=s, nsteps=w.steps, max_refine=3)
    assert plan.info()[0] == pb.PENT_OK
    tol = max(TOL, w.steps * 6 * (1 + 16 * w.sigma[0]) * 2.0 ** -53 * np.max(np.abs(w.field0)) / np.max(np.abs(ref)))
    assert sys_err(C.cpu().numpy(), ref, n) <= tol


@pytest.mark.parametrize("prec", [pb.PENT_F64, pb.PENT_F32_REFINE])
def test_full_size_periodic_crank_nicolson_sampled(prec):
    """The periodic workload at full size (65,536 systems x 512, shared sigma_x = 343.6) as bench.py times
    it: one Crank-Nicolson step, 128 sampled systems against the oracle, with the bar of the oracle's own
    right-hand-side rounding at this sigma (see test_periodic_crank_nicolson_at_the_workloads_sigma)."""
    w = synth.periodic_cn(steps=1)
    n = int(w.n[0])
    plan = pb.Plan(n, batch=w.batch, shared=True, periodic=True, precision=prec)
    s = dev(w.sigma)
    plan.factor_hyperdiff(s)
    C = dev(w.field0)
    plan.step(C, nu=s, max_refine=3)
    assert plan.info()[0] == pb.PENT_OK
    pick = np.arange(0, w.batch, 512)
    f0 = w.field0.reshape(w.batch, n)[pick].reshape(-1)
    ref = oracle.periodic_steps(n, w.sigma, f0, 1, cn=True, shared=True)
    got = C.cpu().numpy().reshape(w.batch, n)[pick].reshape(-1)
    tol = max(TOL, 6 * (1 + 16 * w.sigma[0]) * 2.0 ** -53 * np.max(np.abs(f0)) / np.max(np.abs(ref)))
    assert sys_err(got, ref, n) <= tol


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("prec", [pb.PENT_F64, pb.PENT_F32_REFINE])
def test_periodic_crank_nicolson_against_the_exact_step(prec, n):
    """One periodic Crank-Nicolson step at the workload's sigma_x = 343.6, both GPU paths against
    the step computed in exact rational arithmetic (oracle/exact.py: the scheme's right-hand side
    and Navon's reduction in Fractions, the inputs taken as the rationals the doubles are).  The
    exact step has no rounding: both paths are within 1e-12 of it, element by element, although the
    FP64 oracle's own rounding bound at this sigma (the right-hand side's cancellation) is ~4e-12."""
    from oracle import exact as ex
    sigma = 1e-8 / (2 * (1.0 / 512) ** 4)
    batch = 6
    f0 = synth.uniform(4400 + n, 0, batch * n, -1, 1)
    ref = np.concatenate([np.array([float(v) for v in ex.periodic_cn_step(sigma, f0[s * n:(s + 1) * n])])
                          for s in range(batch)])
    plan = pb.Plan(n, batch=batch, shared=True, periodic=True, precision=prec)
    s = dev(np.array([sigma]))
    plan.factor_hyperdiff(s)
    C = dev(f0)
    plan.step(C, nu=s, max_refine=3)
    assert plan.info()[0] == pb.PENT_OK
    err = sys_err(C.cpu().numpy(), ref, n)
    print(f"periodic CN n={n} precision={prec}: GPU vs exact step {err:.2e}")
    assert err <= TOL
