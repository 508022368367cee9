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
