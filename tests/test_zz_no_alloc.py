"""The allocation-free entry point, pent_gbsv_batch_noalloc, called through the C ABI.

It exists for callers that may not allocate device memory (a framework whose
allocator owns the GPU, plug-ins handed buffers but no allocator, work about to
be captured into a CUDA graph); its scratch is a fixed array owned by the
library, shared by every call.  Its results are checked element by element
against the CPU oracle's factorisation and substitutions (and against the
plan-based path), on two calls in a row with different inputs so that nothing
stale from the first call leaks into the second; also in place (x aliases f),
for the smallest systems, with a zero pivot reported through d_info, at the
scratch array's exact capacity, and replayed from a CUDA graph.  This file is
collected last so that a run that stops at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1807_07382_gb300 as pb  # noqa: E402
from paper_1807_07382_gb300 import _lib, build  # noqa: E402

TOL = 1e-12  # the tolerance of the other GPU parity tests
NONE = 0x7f7f7f7f7f7f7f7f  # d_info when no pivot failed


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    assert torch.cuda.is_available()


def _noalloc(batch, n, band, f, x, info=None, stream=None):
    L = _lib.load()
    st = (stream or torch.cuda.current_stream()).cuda_stream
    return L.pent_gbsv_batch_noalloc(batch, n, *[t.data_ptr() for t in band], f.data_ptr(), x.data_ptr(),
                                     info.data_ptr() if info is not None else None, ctypes.c_void_p(st))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def _oracle(batch, n, band, f):
    ns = np.full(batch, n)
    fac, bad, _ = oracle.factor_batch(ns, band)
    assert bad == -1
    return oracle.solve_batch(ns, fac, f)


def _rel(x, ref, batch, n):
    x = np.asarray(x).reshape(batch, n)
    ref = np.asarray(ref).reshape(batch, n)
    return float(np.max(np.max(np.abs(x - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def test_noalloc_matches_the_oracle_twice():
    batch, n = 300, 1024          # 10 warps (the last ragged) x 1024 rows: 7.5 MiB of scratch
    for call, seed in enumerate((11, 12)):
        band = synth.random_bands(batch, n, seed=seed, kind="diagdom")
        f = synth.uniform(seed + 100, 0, batch * n, -1, 1)
        ref = _oracle(batch, n, band, f)
        bd = [_dev(v) for v in band]
        fd = _dev(f)
        x = torch.full_like(fd, float("nan"))
        info = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert _noalloc(batch, n, bd, fd, x, info) == pb._lib.PENT_OK
        torch.cuda.synchronize()
        assert int(info.item()) == NONE, f"call {call}: a pivot was reported"
        assert _rel(x.cpu().numpy(), ref, batch, n) <= TOL, f"call {call}"
        # and the plan-based path on the same inputs
        plan = pb.Plan(n, batch=batch)
        plan.factor(*bd)
        assert _rel(x.cpu().numpy(), plan.solve(fd).cpu().numpy(), batch, n) <= TOL


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_noalloc_smallest_systems_in_place(n):
    """n < 4 exercises every band-edge guard; x aliases f."""
    batch = 37
    band = synth.random_bands(batch, n, seed=300 + n, kind="spd")
    f = synth.uniform(400 + n, 0, batch * n, -1, 1)
    ref = _oracle(batch, n, band, f)
    fx = _dev(f)
    assert _noalloc(batch, n, [_dev(v) for v in band], fx, fx) == pb._lib.PENT_OK
    torch.cuda.synchronize()
    assert _rel(fx.cpu().numpy(), ref, batch, n) <= TOL


def test_noalloc_reports_the_lowest_zero_pivot():
    """Systems 2 and 4 of 5 have alpha_4 = 0 exactly (row 3): d_info holds (2 << 32 | 3), the
    same encoding as the plan's info word; the healthy systems still solve."""
    n = 6
    good = synth.random_bands(1, n, seed=5, kind="diagdom")
    a, b, c, d, e = (np.full(n, v) for v in (0.1, 0.2, 3.0, 0.2, 0.1))
    d[:3] = 0.0
    e[:3] = 0.0
    c[3] = 0.0  # rows before it do not couple forward
    bad = (a, b, c, d, e)
    band = tuple(np.concatenate(parts) for parts in zip(good, good, bad, good, bad))
    f = synth.uniform(3, 0, 5 * n, -1, 1)
    x = torch.zeros(5 * n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert _noalloc(5, n, [_dev(v) for v in band], _dev(f), x, info) == pb._lib.PENT_OK
    torch.cuda.synchronize()
    assert int(info.item()) == (2 << 32) | 3
    fac, _ = oracle.factor(good)
    got = x.cpu().numpy()
    for s in (0, 1, 3):
        ref = oracle.solve(fac, f[s * n:(s + 1) * n])
        assert np.max(np.abs(got[s * n:(s + 1) * n] - ref)) <= TOL * np.max(np.abs(ref))


def test_noalloc_capacity_boundary():
    """1,344 systems of 1,024 rows (42 warps: 31.5 MiB) fit the 32 MiB array; 1,345 do not."""
    n = 1024
    batch = 1344
    band = synth.random_bands(batch, n, seed=77, kind="diagdom")
    f = synth.uniform(78, 0, batch * n, -1, 1)
    bd = [_dev(v) for v in band]
    fd = _dev(f)
    x = torch.empty_like(fd)
    assert _noalloc(batch, n, bd, fd, x) == pb._lib.PENT_OK
    torch.cuda.synchronize()
    pick = np.arange(0, batch, 83)
    sub = tuple(np.concatenate([v[s * n:(s + 1) * n] for s in pick]) for v in band)
    ref = _oracle(len(pick), n, sub, np.concatenate([f[s * n:(s + 1) * n] for s in pick]))
    got = x.view(batch, n)[torch.as_tensor(pick, device="cuda")].cpu().numpy()
    assert _rel(got, ref, len(pick), n) <= TOL
    assert _noalloc(batch + 1, n, bd, fd, x) == pb._lib.PENT_EINVAL
    big = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(5)]
    assert _noalloc(2048, n, big, big[0], big[0]) == pb._lib.PENT_EINVAL  # 48 MiB of records


def test_noalloc_replays_from_a_cuda_graph():
    """One call outside any capture (it finds the scratch address), then one captured into
    a CUDA graph and replayed with new inputs copied into the captured buffers."""
    batch, n = 200, 512
    band = [_dev(v) for v in synth.random_bands(batch, n, seed=21, kind="diagdom")]
    f = _dev(synth.uniform(22, 0, batch * n, -1, 1))
    x = torch.empty_like(f)
    assert _noalloc(batch, n, band, f, x) == pb._lib.PENT_OK
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            st = _noalloc(batch, n, band, f, x, stream=side)
    assert st == pb._lib.PENT_OK
    for seed in (23, 24):
        fh = synth.uniform(seed, 0, batch * n, -1, 1)
        f.copy_(torch.from_numpy(fh))
        x.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        ref = _oracle(batch, n, tuple(v.cpu().numpy() for v in band), fh)
        assert _rel(x.cpu().numpy(), ref, batch, n) <= TOL
