"""GPU parity for pent_step_batch on no-flux grids: semi-implicit Cahn-Hilliard
steps with per-system parameters (Sec. 2.1, Eq. temporal) and Crank-Nicolson
hyperdiffusion steps (Sec. 2.2), the right-hand side assembled inside the FP64
solve kernel, against the oracle.  Uneven lengths cover one-row systems, odd and
even lengths and the row pairs at the walls; a forced partition covers the
chunked path of long systems.  Tolerance 1e-12 (per-system max error over max
|x|), as for the plain solves."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1807_07382_gb300 as pb  # noqa: E402
from paper_1807_07382_gb300 import build  # noqa: E402

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def sys_err(x, ref, ns):
    off = oracle.offsets(ns)
    worst = 0.0
    for s in range(len(ns)):
        r = ref[off[s]:off[s + 1]]
        worst = max(worst, np.max(np.abs(x[off[s]:off[s + 1]] - r)) / max(np.max(np.abs(r)), 1e-300))
    return worst


UNEVEN = np.array([1, 2, 3, 4, 5, 6, 7, 8, 9, 31, 32, 33, 64, 100, 255, 256, 257, 1000, 1023, 1024] * 4)


@pytest.mark.parametrize("graph", [False, True])
def test_cahn_hilliard_uneven_per_system(graph):
    ns = UNEVEN
    batch = len(ns)
    sig = synth.log_uniform(800, 0, batch, 1e-3, 10.0)
    mu = synth.log_uniform(800, batch, batch, 1e-4, 0.5)
    C0 = synth.uniform(800, 2 * batch, int(ns.sum()), -0.9, 0.9)
    steps = 6
    ref = oracle.explicit_steps(ns, sig, mu, None, C0, steps)
    plan = pb.Plan(list(ns))
    plan.factor_hyperdiff(dev(sig))
    C, m = dev(C0), dev(mu)
    if graph:
        plan.step(C, mu=m, nsteps=steps)
    else:
        for _ in range(steps):
            plan.step(C, mu=m)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_err(C.cpu().numpy(), ref, ns) <= TOL


def test_crank_nicolson_noflux():
    ns = UNEVEN[:23]
    batch = len(ns)
    sig = synth.log_uniform(810, 0, batch, 1e-2, 50.0)
    C0 = synth.uniform(810, batch, int(ns.sum()), -1, 1)
    ref = oracle.explicit_steps(ns, sig, None, sig, C0, 5)
    plan = pb.Plan(list(ns))
    s = dev(sig)
    plan.factor_hyperdiff(s)
    C = dev(C0)
    plan.step(C, nu=s, nsteps=5)
    assert sys_err(C.cpu().numpy(), ref, ns) <= TOL


def test_both_terms_and_long_systems_partitioned():
    """Long systems whose groups are solved in chunks: the right-hand side is written out, then solved."""
    ns = np.array([3000, 2500, 40, 2049, 7, 4096] * 6)
    batch = len(ns)
    sig = synth.log_uniform(820, 0, batch, 1e-2, 5.0)
    mu = synth.log_uniform(820, batch, batch, 1e-3, 0.2)
    nu = 0.5 * sig
    C0 = synth.uniform(820, 2 * batch, int(ns.sum()), -0.8, 0.8)
    ref = oracle.explicit_steps(ns, sig, mu, nu, C0, 4)
    plan = pb.Plan(list(ns), options={pb.PENT_OPT_PARTITION_ROWS: 1024})
    plan.factor_hyperdiff(dev(sig))
    assert any(plan.system_config(s)[0] == 0 for s in range(batch)), "no group was partitioned"
    C = dev(C0)
    plan.step(C, mu=dev(mu), nu=dev(nu), nsteps=4)
    assert sys_err(C.cpu().numpy(), ref, ns) <= TOL


def test_cahn_hilliard_batch_mass_and_sampled_parity():
    """4,096 systems of N = 1024, 20 steps: exact mass conservation per system, oracle parity on a sample."""
    batch, n, steps = 4096, 1024, 20
    sig = synth.log_uniform(830, 0, batch, 1e-3, 10.0)
    mu = synth.log_uniform(830, batch, batch, 1e-4, 0.1)
    C0 = synth.uniform(830, 2 * batch, batch * n, -1, 1)
    plan = pb.Plan(n, batch=batch)
    plan.factor_hyperdiff(dev(sig))
    C = dev(C0)
    plan.step(C, mu=dev(mu), nsteps=steps)
    out = C.cpu().numpy().reshape(batch, n)
    m0 = C0.reshape(batch, n).sum(1)
    scale = np.abs(C0).reshape(batch, n).sum(1)
    assert np.max(np.abs(out.sum(1) - m0) / scale) <= 1e-12
    idx = np.arange(0, batch, 97)
    ref = oracle.explicit_steps(np.full(len(idx), n), sig[idx], mu[idx], None, C0.reshape(batch, n)[idx].reshape(-1),
                                steps)
    assert sys_err(out[idx].reshape(-1), ref, np.full(len(idx), n)) <= TOL


def test_step_rejects_shared_and_general_band_plans():
    plan = pb.Plan(32, batch=4, shared=True)
    plan.factor_hyperdiff(dev([1.0]))
    with pytest.raises(pb.PentError):
        plan.step(dev(np.zeros(128)), mu=dev([0.1]))
    plan2 = pb.Plan(32, batch=4)
    plan2.factor(*[dev(v) for v in synth.random_bands(4, 32, seed=1, kind="diagdom")])
    with pytest.raises(pb.PentError):
        plan2.step(dev(np.zeros(128)), mu=dev(np.zeros(4)))


# ----------------------------------------------------------------------------- refactor + solve every call

def _oracle_refactor_solve(ns, sig, f):
    band = oracle.band_hyperdiff_batch(ns, sig)
    fac, bad, _ = oracle.factor_batch(ns, band)
    assert bad == -1
    return oracle.solve_batch(ns, fac, f)


@pytest.mark.parametrize("case", ["uneven", "shared", "partitioned"])
def test_refactor_solve_each_step(case):
    """A new sigma every step (the paper's Rewrite use): factor and solve in one call, three steps in a
    row, then a plain solve that must reuse the last factorisation."""
    if case == "shared":
        ns = np.full(50, 300)
        plan = pb.Plan(300, batch=50, shared=True)
    elif case == "partitioned":
        ns = np.array([2100, 64, 3000, 5, 2049] * 7)
        plan = pb.Plan(list(ns), options={pb.PENT_OPT_PARTITION_ROWS: 1024})
    else:
        ns = UNEVEN
        plan = pb.Plan(list(ns))
    batch = len(ns)
    nsig = 1 if case == "shared" else batch
    sig0 = synth.log_uniform(840, 0, nsig, 1e-3, 10.0)
    x = synth.uniform(840, nsig, int(ns.sum()), -1, 1)
    X = dev(x)
    for k in range(3):
        sig = sig0 * (1.0 + 0.25 * k)
        ref = _oracle_refactor_solve(ns, np.broadcast_to(sig, (batch,)) if case == "shared" else sig, x)
        plan.refactor_solve(dev(sig), X, X)
        assert plan.info()[0] == pb.PENT_OK
        got = X.cpu().numpy()
        assert sys_err(got, ref, ns) <= TOL, f"step {k}"
        x = ref
    f = synth.uniform(841, 0, int(ns.sum()), -1, 1)
    ref = _oracle_refactor_solve(ns, np.broadcast_to(sig, (batch,)) if case == "shared" else sig, f)
    assert sys_err(plan.solve(dev(f)).cpu().numpy(), ref, ns) <= TOL


# ----------------------------------------------------------------------------- FP32 + refinement

LONG = np.array([5000, 9000, 4097, 300, 1, 2, 3, 64, 129, 1024, 2048, 4096])


@pytest.mark.parametrize("cn", [False, True])
def test_steps_f32_refine_match_oracle(cn):
    """FP32+refine steps: the right-hand side in float-float, FP32 solves refined against the float-float
    residual; uneven lengths from one row to clusters of CTAs (up to 9,000 rows)."""
    ns = np.concatenate([UNEVEN, LONG])
    batch = len(ns)
    sig = synth.log_uniform(850, 0, batch, 1e-3, 10.0)
    mu = None if cn else synth.log_uniform(850, batch, batch, 1e-4, 0.5)
    nu = sig if cn else None
    C0 = synth.uniform(850, 2 * batch, int(ns.sum()), -0.9, 0.9)
    steps = 5
    ref = oracle.explicit_steps(ns, sig, mu, nu, C0, steps)
    plan = pb.Plan(list(ns), precision=pb.PENT_F32_REFINE)
    plan.factor_hyperdiff(dev(sig))
    C = dev(C0)
    plan.step(C, mu=dev(mu) if mu is not None else None, nu=dev(nu) if nu is not None else None, nsteps=steps,
              max_refine=3)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_err(C.cpu().numpy(), ref, ns) <= TOL


def test_cahn_hilliard_f32_refine_shared_and_mass():
    n, batch, steps = 1024, 256, 10
    sigma, mu = 2.5, 0.05
    C0 = synth.uniform(860, 0, batch * n, -1, 1)
    ref = oracle.explicit_steps(np.full(batch, n), [sigma], [mu], None, C0, steps, shared=True)
    plan = pb.Plan(n, batch=batch, shared=True, precision=pb.PENT_F32_REFINE)
    plan.factor_hyperdiff(dev([sigma]))
    C = dev(C0)
    plan.step(C, mu=dev([mu]), nsteps=steps, max_refine=2)
    out = C.cpu().numpy()
    assert sys_err(out, ref, np.full(batch, n)) <= TOL
    m0 = C0.reshape(batch, n).sum(1)
    assert np.max(np.abs(out.reshape(batch, n).sum(1) - m0)) <= 1e-12 * np.abs(C0).reshape(batch, n).sum(1).max()


@pytest.mark.parametrize("prec", [pb.PENT_F64, pb.PENT_F32_REFINE])
def test_full_size_cahn_hilliard_batch_sampled(prec):
    """The 1D Cahn-Hilliard workload at full size (65,536 systems x 1024, per-system sigma and mu) in the
    launch configuration bench.py times: one step, 128 sampled systems against the oracle."""
    w = synth.ch_batch(steps=1)
    n = int(w.n[0])
    plan = pb.Plan(n, batch=w.batch, precision=prec)
    plan.factor_hyperdiff(dev(w.sigma))
    C = dev(w.field0)
    plan.step(C, mu=dev(w.extra["mu"]), max_refine=1)
    assert plan.info()[0] == pb.PENT_OK
    pick = np.arange(0, w.batch, 512)
    ref = oracle.explicit_steps(np.full(len(pick), n), w.sigma[pick], w.extra["mu"][pick], None,
                                w.field0.reshape(w.batch, n)[pick].reshape(-1), 1)
    got = C.cpu().numpy().reshape(w.batch, n)[pick].reshape(-1)
    assert sys_err(got, ref, np.full(len(pick), n)) <= TOL
