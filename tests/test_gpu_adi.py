"""GPU parity of the 2D alternating-direction Cahn-Hilliard step (adi_step_2d)
against the CPU oracle.

Tolerances.  Where sigma is moderate the step is well conditioned and the bar is
1e-12 relative to max|C|.  At the workload's sigma = gamma dt / dx^4 ~ 1.76e5
the implicit factors have condition ~2.8e6 and two independent FP64
implementations already differ by ~1e-8 relative after one step; there the bar
is 4x the difference between the oracle and an independent FP64 reference
(LAPACK's banded solver, scipy.linalg.solve_banded), computed in the test.
Mass is conserved to 1e-12 of sum|C0| in every case (the step removes the mean of
dC, so this holds by construction); the sweeps themselves are pinned on small
grids to an exact rational step, in which dC sums to zero with no removal."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1807_07382_gb300 as pb  # noqa: E402
from paper_1807_07382_gb300 import build  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def run_gpu(C0, gamma, dt, dx, steps, graph=False):
    ny, nx = C0.shape
    adi = pb.ADI2D(nx, ny, gamma, dt, dx)
    C = torch.from_numpy(np.ascontiguousarray(C0)).cuda()
    if graph:
        adi.step(C, steps)
    else:
        for _ in range(steps):
            adi.step(C)
    torch.cuda.synchronize()
    return C.cpu().numpy()


def lapack_step(C, gamma, dt, dx):
    """Independent FP64 reference: the oracle's right-hand side, LAPACK banded solves."""
    sl = pytest.importorskip("scipy.linalg")
    ny, nx = C.shape
    mu, sigma = dt / dx ** 2, gamma * dt / dx ** 4

    def ab(n):
        a, b, c, d, e = oracle.band_hyperdiff(n, sigma)
        m = np.zeros((5, n))
        m[0, 2:] = e[:-2]
        m[1, 1:] = d[:-1]
        m[2, :] = c
        m[3, :-1] = b[1:]
        m[4, :-2] = a[2:]
        return m
    rhs = oracle.ch_rhs(C, mu, sigma)
    W = sl.solve_banded((2, 2), ab(nx), rhs.T).T
    dC = sl.solve_banded((2, 2), ab(ny), W)
    return C + (dC - dC.mean())


@pytest.mark.parametrize("nx,ny", [(40, 48), (33, 7), (64, 64)])
def test_adi_moderate_sigma_matches_oracle(nx, ny):
    w = synth.ch_adi(nx=nx, ny=ny, steps=5)
    dt, dx = 1e-4, 1.0 / 64      # sigma ~ 16.8, mu ~ 0.41
    ref = w.field0.copy()
    for _ in range(w.steps):
        ref = oracle.adi_step(ref, w.gamma, dt, dx)
    got = run_gpu(w.field0, w.gamma, dt, dx, w.steps)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert abs(got.sum() - w.field0.sum()) <= 1e-12 * np.abs(w.field0).sum()


def test_adi_workload_sigma_matches_oracle_within_conditioning():
    w = synth.ch_adi(nx=96, ny=80, steps=1)
    dx = 1.0 / 2048               # sigma ~ 1.76e5 as in the 2048^2 workload
    ref = oracle.adi_step(w.field0, w.gamma, w.dt, dx)
    indep = lapack_step(w.field0, w.gamma, w.dt, dx)
    got = run_gpu(w.field0, w.gamma, w.dt, dx, 1)
    bar = max(1e-12 * np.max(np.abs(ref)), 4.0 * np.max(np.abs(ref - indep)))
    print("oracle vs LAPACK", np.max(np.abs(ref - indep)), "gpu vs oracle", np.max(np.abs(got - ref)))
    assert np.max(np.abs(got - ref)) <= bar


def test_adi_graph_equals_steps_and_conserves_mass():
    w = synth.ch_adi(nx=128, ny=96, steps=10)
    dx = 1.0 / 2048
    a = run_gpu(w.field0, w.gamma, w.dt, dx, w.steps, graph=False)
    b = run_gpu(w.field0, w.gamma, w.dt, dx, w.steps, graph=True)
    assert np.array_equal(a, b)
    assert abs(b.sum() - w.field0.sum()) <= 1e-12 * np.abs(w.field0).sum()


def test_adi_full_grid_one_step_and_mass():
    """2048 x 2048, gamma = 0.01, dt = 1e-6, dx = 1/2048: one step against the
    oracle (whole field), then 20 graph steps for mass conservation."""
    w = synth.ch_adi(steps=20)
    ref = oracle.adi_step(w.field0, w.gamma, w.dt, w.dx)
    indep = lapack_step(w.field0, w.gamma, w.dt, w.dx)
    adi = pb.ADI2D(w.nx, w.ny, w.gamma, w.dt, w.dx)
    C = torch.from_numpy(w.field0).cuda()
    adi.step(C)
    got = C.cpu().numpy()
    bar = max(1e-12 * np.max(np.abs(ref)), 4.0 * np.max(np.abs(ref - indep)))
    print("full grid: oracle vs LAPACK", np.max(np.abs(ref - indep)), "gpu vs oracle", np.max(np.abs(got - ref)))
    assert np.max(np.abs(got - ref)) <= bar
    adi.step(C, w.steps)
    C1 = C.cpu().numpy()
    assert abs(C1.sum() - w.field0.sum()) <= 1e-12 * np.abs(w.field0).sum()


def test_adi_rejects_bad_plans():
    px = pb.Plan(16, batch=8, shared=True)
    py = pb.Plan(8, batch=16, shared=True)
    C = torch.zeros(8, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(pb.PentError):
        pb.adi_step_2d(px, py, C, 0.01, 1e-6, 1 / 16)       # not factored
    pb.adi_plans_factor(px, py, 0.01, 1e-6, 1 / 16)
    with pytest.raises(pb.PentError):
        pb.adi_step_2d(py, px, C, 0.01, 1e-6, 1 / 16)       # swapped plans
    with pytest.raises(pb.PentError):
        pb.adi_step_2d(px, py, C, 0.01, 1e-6, 1 / 16, max_refine=1)


def test_adi_refuses_parameters_the_plans_were_not_factored_for():
    """adi_step_2d runs only on plans factored by adi_plans_factor for its exact (gamma, dt, dx):
    another dt (a different sigma than the sweeps were factored with), plans factored by
    pent_factor_hyperdiff, or plans refactored since, return PENT_EINVAL and leave C untouched."""
    nx, ny, gamma, dt, dx = 16, 8, 0.01, 1e-6, 1.0 / 16
    L = pb._lib.load()
    px = pb.Plan(nx, batch=ny, shared=True)
    py = pb.Plan(ny, batch=nx, shared=True)
    C = torch.from_numpy(synth.uniform(9, 0, nx * ny, -0.1, 0.1).reshape(ny, nx)).cuda()
    C0 = C.clone()

    def step(g, t, h):
        return L.adi_step_2d(px._h, py._h, C.data_ptr(), nx, ny, g, t, h, 0)

    sig = torch.full((1,), gamma * dt / dx ** 4, dtype=torch.float64, device="cuda")
    px.factor_hyperdiff(sig)
    py.factor_hyperdiff(sig)
    assert step(gamma, dt, dx) == pb._lib.PENT_EINVAL     # factored, but not for an ADI step
    pb.adi_plans_factor(px, py, gamma, dt, dx)
    assert step(gamma, 2 * dt, dx) == pb._lib.PENT_EINVAL
    assert step(gamma, dt, dx * (1 + 1e-15)) == pb._lib.PENT_EINVAL
    assert step(2 * gamma, dt, dx) == pb._lib.PENT_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(C, C0)
    assert step(gamma, dt, dx) == pb._lib.PENT_OK
    torch.cuda.synchronize()
    assert not torch.equal(C, C0)
    px.factor_hyperdiff(sig)                               # refactored otherwise: the record is gone
    assert step(gamma, dt, dx) == pb._lib.PENT_EINVAL


@pytest.mark.parametrize("ny,nx,dt,dx,bar", [(20, 24, 1e-4, 1 / 64, 1e-13), (20, 24, 1e-6, 1 / 2048, 2e-9),
                                             (32, 40, 1e-6, 1 / 2048, 2e-9)])
def test_adi_step_against_the_exact_step(ny, nx, dt, dx, bar):
    """The sweeps (and the right-hand side) against one exact rational ADI step (oracle/exact.py: the
    same doubles taken as rationals, every operation in Fractions), relative to max|dC|: to within
    rounding at sigma = 16.8, and at the workload's sigma = 1.76e5 (condition ~3e6) within that
    condition times FP64 rounding, as close as the FP64 oracle comes (printed beside it).  The mean
    removal changes nothing here: the exact dC sums to zero."""
    from oracle import exact as ex
    C0 = synth.uniform(4242, 0, nx * ny, -0.1, 0.1).reshape(ny, nx)
    gamma = 0.01
    mu, sigma = dt / (dx * dx), gamma * dt / (dx * dx * dx * dx)
    E = np.array([[float(v) for v in row] for row in ex.adi_step(C0.tolist(), mu, sigma)])
    scale = np.max(np.abs(E - C0))
    got = run_gpu(C0, gamma, dt, dx, 1)
    orc = oracle.adi_step(C0, gamma, dt, dx)
    e_gpu, e_orc = np.max(np.abs(got - E)) / scale, np.max(np.abs(orc - E)) / scale
    print(f"sigma {sigma:.3g}: gpu vs exact {e_gpu:.2e}, oracle vs exact {e_orc:.2e}")
    assert e_gpu <= bar
