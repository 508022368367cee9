"""GPU parity of the windowed FP32 solve of long systems (csrc/f32u.cu, k_solve32u with
windows) against the CPU oracle.

A system longer than one CTA of W warps x 8 rows (R = 256 W rows) is solved as windows of R
rows, one CTA each, that overlap by O rows: a window enters and leaves its cuts with zero
states and keeps only the rows at least O from a cut.  O is the fewest multiple of 8 rows
over which both interior chunk maps shrink to 2^-56, so the rows kept agree with the whole
system's direct solve far below FP64 rounding; the results are held to the same bar as every
FP32+refine solve: 1e-12 relative (per system, max |x - x_ref| / max |x_ref|) after one
refinement step for sigma in [1e-3, 10], and 1e-4 for the plain FP32 solve.  Systems whose
decay is too slow for the window (the overlap above R / 8) keep the cluster path.

FP64 per-system hyperdiffusion plans walk the groups of 32 length-sorted systems longer than
one window (1024 rows) in windows too: as system windows (PENT_OPT_WINDOW_FORM 1, the default),
one thread per window of one system with the system's own overlap, or as group windows (0), one
warp per window of a group with the group's largest overlap; both against the oracle at 1e-12
and within 1e-14 of the whole-group walk."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1807_07382_gb300 as pb  # noqa: E402
from paper_1807_07382_gb300 import build  # noqa: E402

TOL = 1e-12
TOL_FP32 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def sys_rel_err(x, ref, n_per_system):
    off = oracle.offsets(n_per_system)
    worst = 0.0
    for s in range(len(off) - 1):
        r = ref[off[s]:off[s + 1]]
        d = np.max(np.abs(x[off[s]:off[s + 1]] - r))
        worst = max(worst, d / max(np.max(np.abs(r)), 1e-300))
    return worst


def plan_for(ns, sigma, window_warps=None, kernel=0, shared=False):
    opts = {pb.PENT_OPT_FP32_KERNEL: kernel}
    if window_warps is not None:
        opts[pb.PENT_OPT_WINDOW_WARPS] = window_warps
    if shared:
        plan = pb.Plan(int(ns[0]), batch=len(ns), shared=True, precision=pb.PENT_F32_REFINE, options=opts)
    else:
        plan = pb.Plan(list(ns), precision=pb.PENT_F32_REFINE, options=opts)
    plan.factor_hyperdiff(dev(sigma))
    return plan


def workload(n, batch, seed_index, sigma_range=(1e-3, 10.0)):
    return synth.hyperdiff_parametric(batch=batch, n=n, steps=1, seed_index=seed_index, sigma_range=sigma_range)


@pytest.mark.parametrize("n", [1025, 1100, 2047, 2048, 2049, 3000, 4097, 8192, 12345, 16384])
def test_windows_meet_the_bar(n):
    """Lengths from just above one window (two windows, the last a sliver) to 16 windows,
    out of place and in place (the overlap rows copied out first)."""
    w = workload(n, 12, 40 + n % 7)
    ref = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, 1)
    plan = plan_for(w.n, w.sigma)
    assert plan.get_option(pb.PENT_OPT_WINDOWS) >= 2 * len(w.n)
    x = plan.solve(dev(w.field0), max_refine=1)
    st, _, _, used = plan.info()
    assert st == pb.PENT_OK and used == 1
    assert sys_rel_err(host(x), ref, w.n) <= TOL
    x0 = plan.solve(dev(w.field0), max_refine=0)
    assert sys_rel_err(host(x0), ref, w.n) <= TOL_FP32
    xi = dev(w.field0)
    plan.solve(xi, xi, max_refine=1)
    assert sys_rel_err(host(xi), ref, w.n) <= TOL


@pytest.mark.parametrize("window_warps", [4, 8, 16])
def test_window_widths(window_warps):
    """Every window width on the longest FP32 systems (30,000 rows) and ragged lengths."""
    ns = np.array([30000, 9999, 4100, 20001])
    sig = np.array([10.0, 1e-3, 0.5, 3.0])
    f = synth.uniform(777, 0, int(ns.sum()), -1, 1)
    ref = oracle.hyperdiff_steps(ns, sig, f, 1)
    plan = plan_for(ns, sig, window_warps=window_warps)
    R = 256 * window_warps
    assert plan.get_option(pb.PENT_OPT_WINDOWS) >= sum(len(pb.window_layout(int(n), R, 8)) for n in ns)
    x = dev(f)
    plan.solve(x, x, max_refine=1)
    assert sys_rel_err(host(x), ref, ns) <= TOL


@pytest.mark.parametrize("steps", [1, 3, 8])
def test_windowed_graph_steps_in_place(steps):
    """pent_solve_steps runs in place: every step copies the overlap rows out before its
    windows overwrite them.  Bar: steps x 1e-12 (each solve within 1e-12, carried forward),
    and no worse than the same plan with windows off (clusters)."""
    ns = np.array([16384, 5000, 700, 12000, 1024, 9000])
    sig = synth.log_uniform(91, 0, len(ns), 1e-3, 10.0)
    f = synth.uniform(92, 0, int(ns.sum()), -1, 1)
    ref = oracle.hyperdiff_steps(ns, sig, f, steps)
    errs = []
    for ww in (4, 0):
        plan = plan_for(ns, sig, window_warps=ww)
        assert (plan.get_option(pb.PENT_OPT_WINDOWS) > 0) == (ww > 0)
        x = dev(f)
        plan.solve_steps(x, steps, max_refine=1)
        assert plan.info()[0] == pb.PENT_OK
        errs.append(sys_rel_err(host(x), ref, ns))
    print("errors (windows, clusters):", errs)
    assert errs[0] <= steps * TOL
    assert errs[0] <= 1.5 * errs[1] + 1e-13


def test_slow_decay_systems_keep_their_clusters():
    """sigma = 300 needs an overlap above R / 8 = 128 rows for 4-warp windows: that system keeps
    its cluster and is solved exactly as with windows off (bitwise), while its neighbours run in
    windows and meet the bar."""
    ns = np.array([8192, 8192, 6000])
    sig = np.array([300.0, 0.01, 5.0])
    f = synth.uniform(55, 0, int(ns.sum()), -1, 1)
    plan = plan_for(ns, sig)
    off = plan_for(ns, sig, window_warps=0)
    nwin = plan.get_option(pb.PENT_OPT_WINDOWS)
    assert 0 < nwin <= len(pb.window_layout(8192, 1024, 128)) + len(pb.window_layout(6000, 1024, 128))
    assert off.get_option(pb.PENT_OPT_WINDOWS) == 0
    a = host(plan.solve(dev(f), max_refine=1))
    b = host(off.solve(dev(f), max_refine=1))
    assert np.array_equal(a[:8192], b[:8192])
    ref = oracle.hyperdiff_steps(ns[1:], sig[1:], f[8192:], 1)
    assert sys_rel_err(a[8192:], ref, ns[1:]) <= TOL


def test_shared_matrix_in_windows():
    n, batch = 9000, 6
    f = synth.uniform(4102, 0, n * batch, -1, 1)
    ns = np.full(batch, n)
    ref = oracle.hyperdiff_steps(ns, np.full(batch, 2.5), f, 2)
    plan = plan_for(ns, np.array([2.5]), shared=True)
    assert plan.get_option(pb.PENT_OPT_WINDOWS) >= 10 * batch
    x = dev(f)
    plan.solve_steps(x, 2, max_refine=1)
    assert sys_rel_err(host(x), ref, ns) <= 2 * TOL


def test_more_refinement_steps_and_the_general_kernel_bypass_windows():
    """max_refine = 2 and PENT_OPT_FP32_KERNEL = 1 take the bucket path (clusters for the long
    systems): the same results within the bar."""
    w = workload(7000, 6, 47)
    ref = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, 1)
    plan = plan_for(w.n, w.sigma)
    assert plan.get_option(pb.PENT_OPT_WINDOWS) > 0
    x = plan.solve(dev(w.field0), max_refine=2)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_rel_err(host(x), ref, w.n) <= TOL
    gen = plan_for(w.n, w.sigma, kernel=1)
    assert sys_rel_err(host(gen.solve(dev(w.field0), max_refine=1)), ref, w.n) <= TOL


def test_refactor_rebuilds_the_windows():
    """A second factorisation with other sigmas lays the windows out anew (the overlap grows
    with sigma) and the step graphs captured for the first one are not reused."""
    ns = np.full(4, 12000)
    f = synth.uniform(61, 0, int(ns.sum()), -1, 1)
    plan = plan_for(ns, np.full(4, 1e-3))
    n_small = plan.get_option(pb.PENT_OPT_WINDOWS)
    x = dev(f)
    plan.solve_steps(x, 2, max_refine=1)
    assert sys_rel_err(host(x), oracle.hyperdiff_steps(ns, np.full(4, 1e-3), f, 2), ns) <= 2 * TOL
    plan.factor_hyperdiff(dev(np.full(4, 10.0)))
    assert plan.get_option(pb.PENT_OPT_WINDOWS) > n_small
    x = dev(f)
    plan.solve_steps(x, 2, max_refine=1)
    assert sys_rel_err(host(x), oracle.hyperdiff_steps(ns, np.full(4, 10.0), f, 2), ns) <= 2 * TOL


# ----------------------------------------------------------------------------- FP64 windows

def plan64(ns, sigma, window_rows=None):
    opts = {} if window_rows is None else {pb.PENT_OPT_WINDOW_ROWS: window_rows}
    plan = pb.Plan(list(ns), precision=pb.PENT_F64, options=opts)
    plan.factor_hyperdiff(dev(sigma))
    return plan


@pytest.mark.parametrize("n", [1025, 2049, 4097, 8192, 16384, 40000])
def test_f64_windows_meet_the_bar(n):
    """Groups of 32 systems longer than one window (1024 rows) walked in windows: against the
    oracle at 1e-12 and within 1e-14 of the same plan walking whole groups (windows off), out of
    place and in place."""
    batch = 40 if n <= 8192 else 33
    w = workload(n, batch, 60 + n % 5)
    ref = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, 1)
    plan = plan64(w.n, w.sigma)
    assert plan.get_option(pb.PENT_OPT_WINDOWS) >= 2 * ((batch + 31) // 32)
    x = host(plan.solve(dev(w.field0)))
    assert sys_rel_err(x, ref, w.n) <= TOL
    whole = host(plan64(w.n, w.sigma, window_rows=0).solve(dev(w.field0)))
    assert sys_rel_err(x, whole, w.n) <= 1e-14
    xi = dev(w.field0)
    plan.solve(xi, xi)
    assert np.array_equal(host(xi), x)


def test_f64_windows_of_uneven_groups_and_steps_in_place():
    """Systems of one group end at different rows (lengths 3,000 .. 9,000, sorted into groups),
    so windows cut some lanes inside their systems and run others through padding; several steps
    in place in one graph, against the oracle (bar: steps x 1e-12) and the whole-group walks."""
    ns = np.floor(synth.log_uniform(71, 0, 80, 3000.0, 9000.0)).astype(np.int64)
    sig = synth.log_uniform(72, 0, len(ns), 1e-2, 10.0)
    f = synth.uniform(73, 0, int(ns.sum()), -1, 1)
    steps = 3
    ref = oracle.hyperdiff_steps(ns, sig, f, steps)
    got = []
    for wr in (1024, 0):
        plan = plan64(ns, sig, window_rows=wr)
        assert (plan.get_option(pb.PENT_OPT_WINDOWS) > 0) == (wr > 0)
        x = dev(f)
        plan.solve_steps(x, steps)
        got.append(host(x))
    assert sys_rel_err(got[0], ref, ns) <= steps * TOL
    assert sys_rel_err(got[0], got[1], ns) <= 1e-14


@pytest.mark.parametrize("window_rows,sigma_hi", [(256, 0.05), (512, 1.0), (2048, 10.0)])
def test_f64_window_sizes(window_rows, sigma_hi):
    """Other window lengths (the overlap room is 1/8 of the window: smaller windows take the
    faster-decaying systems)."""
    ns = np.array([20000] * 20 + [3000] * 20 + [700] * 20)
    sig = synth.log_uniform(74, 0, len(ns), 1e-3, sigma_hi)
    f = synth.uniform(75, 0, int(ns.sum()), -1, 1)
    ref = oracle.hyperdiff_steps(ns, sig, f, 1)
    plan = plan64(ns, sig, window_rows=window_rows)
    assert plan.get_option(pb.PENT_OPT_WINDOWS) > 0
    x = dev(f)
    plan.solve(x, x)
    assert sys_rel_err(host(x), ref, ns) <= TOL


def test_f64_slow_decay_and_general_bands_keep_their_walks():
    """A run of groups one of which decays too slowly for the window (sigma = 1e4: an overlap
    above 128 rows) keeps its solves, bitwise as with windows off, while the run of another
    launch setting takes windows (here the 6,000-row groups are partitioned, PENT_OPT_PARTITION_ROWS
    = 5,000, and the 1,500-row group is walked); a general band (pent_factor_batch) lays out no
    windows at all."""
    ns = np.array([6000] * 32 + [6000] * 32 + [1500] * 32)
    sig = np.concatenate([np.full(32, 1e4), np.full(32, 0.5), np.full(32, 2.0)])
    f = synth.uniform(76, 0, int(ns.sum()), -1, 1)
    runs = []
    for wr, form in ((1024, 0), (1024, 1), (0, 1)):
        plan = pb.Plan(list(ns), precision=pb.PENT_F64,
                       options={pb.PENT_OPT_PARTITION_ROWS: 5000, pb.PENT_OPT_WINDOW_ROWS: wr,
                                pb.PENT_OPT_WINDOW_FORM: form})
        plan.factor_hyperdiff(dev(sig))
        runs.append((plan.get_option(pb.PENT_OPT_WINDOWS), host(plan.solve(dev(f)))))
    (nwg, ag), (nw, a), (nw0, b) = runs
    assert nw0 == 0 and 2 <= nwg <= len(pb.window_layout(1500, 1024, 128))
    assert nw == 32 * 2  # system windows: two of 512 row pairs for each 1,500-row system
    assert np.array_equal(ag[:64 * 6000], b[:64 * 6000])
    assert np.array_equal(a[:64 * 6000], b[:64 * 6000])
    ref = oracle.hyperdiff_steps(ns[32:], sig[32:], f[32 * 6000:], 1)
    assert sys_rel_err(a[32 * 6000:], ref, ns[32:]) <= TOL
    band = oracle.band_hyperdiff_batch(ns, sig)
    gen = pb.Plan(list(ns), precision=pb.PENT_F64)
    gen.factor(*[dev(v) for v in band])
    assert gen.get_option(pb.PENT_OPT_WINDOWS) == 0
    g = host(gen.solve(dev(f)))
    assert sys_rel_err(g[32 * 6000:], ref, ns[32:]) <= TOL  # (sigma = 1e4 is left out: kappa ~ 1.6e5)


@pytest.mark.parametrize("prec", [pb.PENT_F32_REFINE, pb.PENT_F64])
def test_persistent_windows_give_the_same_bits(prec):
    """PENT_OPT_PERSISTENT = 1 launches the windows as a resident grid whose CTAs (FP32) or warps
    (FP64) take the windows in turn: each window's arithmetic is unchanged, so the results are
    bitwise those of one CTA or warp per window, out of place, in place and in step graphs."""
    ns = np.array([16384] * 40 + [3000] * 40 + [500] * 40)
    sig = synth.log_uniform(81, 0, len(ns), 1e-2, 10.0)
    f = synth.uniform(82, 0, int(ns.sum()), -1, 1)
    out = []
    for pers in (0, 1):
        plan = pb.Plan(list(ns), precision=prec, options={pb.PENT_OPT_PERSISTENT: pers})
        plan.factor_hyperdiff(dev(sig))
        assert plan.get_option(pb.PENT_OPT_WINDOWS) > 0 and plan.get_option(pb.PENT_OPT_PERSISTENT) == pers
        a = host(plan.solve(dev(f), max_refine=1))
        x = dev(f)
        plan.solve(x, x, max_refine=1)
        y = dev(f)
        plan.solve_steps(y, 3, max_refine=1)
        out.append((a, host(x), host(y)))
    for u, v in zip(*out):
        assert np.array_equal(u, v)
    ref = oracle.hyperdiff_steps(ns, sig, f, 1)
    assert sys_rel_err(out[1][0], ref, ns) <= TOL


@pytest.mark.parametrize("case", ["uniform", "uneven", "steps"])
def test_f64_interior_records_from_registers_give_the_same_bits(case):
    """PENT_OPT_FP64_INTERIOR: the hyperdiffusion walks (whole groups and windows) take the interior
    rows' records from registers once the factorisation has settled on them; the arithmetic is the
    same, so the results are bitwise those of reading every record, and they meet the oracle."""
    if case == "uniform":
        ns = np.full(96, 1024)
    else:
        ns = np.floor(synth.log_uniform(84, 0, 300, 8.0, 16384.0)).astype(np.int64)
    sig = synth.log_uniform(85, 0, len(ns), 1e-3, 10.0)
    f = synth.uniform(86, 0, int(ns.sum()), -1, 1)
    steps = 3 if case == "steps" else 1
    out = []
    for ic in (1, 0):
        plan = pb.Plan(list(ns), precision=pb.PENT_F64, options={pb.PENT_OPT_FP64_INTERIOR: ic})
        plan.factor_hyperdiff(dev(sig))
        x = dev(f)
        if steps > 1:
            plan.solve_steps(x, steps)
        else:
            plan.solve(x, x)
        out.append(host(x))
    assert np.array_equal(out[0], out[1])
    ref = oracle.hyperdiff_steps(ns, sig, f, steps)
    assert sys_rel_err(out[0], ref, ns) <= steps * TOL


@pytest.mark.parametrize("prec", [pb.PENT_F32_REFINE, pb.PENT_F64])
def test_windows_with_odd_offsets_and_unaligned_vectors(prec):
    """Systems of odd lengths (so half of them start at odd rows: their pairs are read and written
    as the aligned pairs one row over) and f / x views one double off a 16-byte boundary (every
    access scalar): bitwise the results of aligned vectors, and the oracle's."""
    ns = np.array([3001, 4097, 2049, 5001, 1025, 7777] * 6)
    sig = synth.log_uniform(87, 0, len(ns), 1e-2, 10.0)
    f = synth.uniform(88, 0, int(ns.sum()), -1, 1)
    plan = pb.Plan(list(ns), precision=prec)
    plan.factor_hyperdiff(dev(sig))
    assert plan.get_option(pb.PENT_OPT_WINDOWS) > 0
    a = host(plan.solve(dev(f), max_refine=1))
    rows = int(ns.sum())
    fb = torch.zeros(rows + 1, dtype=torch.float64, device="cuda")
    xb = torch.zeros(rows + 1, dtype=torch.float64, device="cuda")
    fb[1:] = dev(f)
    plan.solve(fb[1:], xb[1:], max_refine=1)
    assert np.array_equal(host(xb[1:]), a)
    y = dev(f)
    plan.solve(y, y, max_refine=1)
    assert np.array_equal(host(y), a)
    ref = oracle.hyperdiff_steps(ns, sig, f, 1)
    assert sys_rel_err(a, ref, ns) <= TOL


def test_f64_refactorisations_drop_stale_windows_and_interior_records():
    """A plan with windows (hyperdiffusion factorisation) then factored from a general band, or
    refactored from a new sigma inside a solve, must not keep walking windows or interior records
    of the old factors: each later solve meets the oracle for the factors it has."""
    ns = np.array([6000] * 40 + [900] * 24)
    sig1 = synth.log_uniform(91, 0, len(ns), 1e-2, 10.0)
    sig2 = synth.log_uniform(92, 0, len(ns), 1e-2, 10.0)
    f = synth.uniform(93, 0, int(ns.sum()), -1, 1)
    plan = pb.Plan(list(ns), precision=pb.PENT_F64)
    plan.factor_hyperdiff(dev(sig1))
    assert plan.get_option(pb.PENT_OPT_WINDOWS) > 0
    assert sys_rel_err(host(plan.solve(dev(f))), oracle.hyperdiff_steps(ns, sig1, f, 1), ns) <= TOL
    # a general band with sigma2's entries: no windows, every record read
    plan.factor(*[dev(v) for v in oracle.band_hyperdiff_batch(ns, sig2)])
    assert plan.get_option(pb.PENT_OPT_WINDOWS) == 0
    ref2 = oracle.hyperdiff_steps(ns, sig2, f, 1)
    assert sys_rel_err(host(plan.solve(dev(f))), ref2, ns) <= TOL
    # back to windows, then a refactorisation inside a solve (the new sigma's records and interior)
    plan.factor_hyperdiff(dev(sig1))
    assert plan.get_option(pb.PENT_OPT_WINDOWS) > 0
    x = dev(f)
    y = torch.empty_like(x)
    plan.refactor_solve(dev(sig2), x, y)
    assert sys_rel_err(host(y), ref2, ns) <= TOL
    assert plan.get_option(pb.PENT_OPT_WINDOWS) == 0
    assert sys_rel_err(host(plan.solve(dev(f))), ref2, ns) <= TOL
    xs = dev(f)
    plan.solve_steps(xs, 2)
    assert sys_rel_err(host(xs), oracle.hyperdiff_steps(ns, sig2, f, 2), ns) <= 2 * TOL


@pytest.mark.parametrize("case", ["uniform", "uneven", "odd", "steps", "short_lanes", "tiny_lanes"])
def test_f64_system_windows_against_group_windows_and_the_oracle(case):
    """System windows (PENT_OPT_WINDOW_FORM 1): each system of a windowed group cut at its own
    rows with its own overlap, the windows in the caller's row order.  Against the oracle at
    1e-12 (steps x 1e-12 for graph steps), within 1e-14 of group windows and of the whole-group
    walk; in place bitwise the out-of-place result.  Cases: equal lengths; log-uniform lengths
    8 .. 16,384 (groups of both kinds); odd lengths (half the systems start at odd rows);
    in-place steps in one graph; groups whose shortest systems fit one window (a window of
    fewer rows than the others in the same warp); a group whose last lanes hold systems of 1, 2,
    3 and 5 rows (one row pair or a few, no interior rows)."""
    if case == "uniform":
        ns = np.full(40, 8192)
    elif case == "uneven":
        ns = np.floor(synth.log_uniform(94, 0, 300, 8.0, 16384.0)).astype(np.int64)
    elif case == "odd":
        ns = np.array([3001, 4097, 2049, 5001, 1025, 7777, 1023, 999] * 5)
    elif case == "steps":
        ns = np.floor(synth.log_uniform(95, 0, 120, 1000.0, 9000.0)).astype(np.int64)
    elif case == "short_lanes":
        ns = np.array([1100] * 20 + [1000] * 12 + [700] * 10)
    else:
        ns = np.array([3000] * 28 + [1, 2, 3, 5])
    sig = synth.log_uniform(96, 0, len(ns), 1e-2, 10.0)
    f = synth.uniform(97, 0, int(ns.sum()), -1, 1)
    steps = 3 if case == "steps" else 1
    ref = oracle.hyperdiff_steps(ns, sig, f, steps)
    got = {}
    for name, opts in (("system", {pb.PENT_OPT_WINDOW_FORM: 1}), ("group", {pb.PENT_OPT_WINDOW_FORM: 0}),
                       ("whole", {pb.PENT_OPT_WINDOW_ROWS: 0})):
        plan = pb.Plan(list(ns), precision=pb.PENT_F64, options=opts)
        plan.factor_hyperdiff(dev(sig))
        assert (plan.get_option(pb.PENT_OPT_WINDOWS) > 0) == (name != "whole")
        x = dev(f)
        if steps > 1:
            plan.solve_steps(x, steps)
        else:
            plan.solve(x, x)
        got[name] = host(x)
        if name == "system" and steps == 1:
            assert np.array_equal(host(plan.solve(dev(f))), got[name])
    assert sys_rel_err(got["system"], ref, ns) <= steps * TOL
    assert sys_rel_err(got["system"], got["group"], ns) <= 1e-14
    assert sys_rel_err(got["system"], got["whole"], ns) <= 1e-14
