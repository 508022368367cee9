"""The allocation-free entry point, pent_gbsv_batch_noalloc, against the regular
plan-based path (pent_factor_batch + pent_solve_batch), called through the C ABI.

It exists for callers that cannot allocate device memory; its scratch is a fixed
array owned by the library, shared by every call.  Two calls in a row with
different inputs check that nothing stale from the first call leaks into the
second.  This file is collected last so that a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1807_07382_gb300 as pb  # noqa: E402
from paper_1807_07382_gb300 import _lib, build  # noqa: E402

TOL = 1e-12  # the tolerance of the other GPU parity tests


def _noalloc(batch, n, band, f, x, info=None):
    L = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    return L.pent_gbsv_batch_noalloc(batch, n, *[t.data_ptr() for t in band], f.data_ptr(), x.data_ptr(),
                                     info.data_ptr() if info is not None else None, ctypes.c_void_p(stream))


def _rel(x, ref, batch, n):
    x = x.view(batch, n).cpu().numpy()
    ref = ref.view(batch, n).cpu().numpy()
    return float(np.max(np.max(np.abs(x - ref), axis=1) / np.max(np.abs(ref), axis=1)))


def test_noalloc_matches_plan_path_twice():
    build.build()
    batch, n = 300, 1024          # 10 warps (the last ragged) x 1024 rows: 7.4 MiB of scratch
    for call, seed in enumerate((11, 12)):
        band = [torch.from_numpy(v).cuda() for v in synth.random_bands(batch, n, seed=seed, kind="diagdom")]
        f = torch.from_numpy(synth.uniform(seed + 100, 0, batch * n, -1, 1)).cuda()
        plan = pb.Plan(n, batch=batch)
        plan.factor(*band)
        ref = plan.solve(f)
        x = torch.full_like(f, float("nan"))
        info = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert _noalloc(batch, n, band, f, x, info) == pb._lib.PENT_OK
        torch.cuda.synchronize()
        assert int(info.item()) == 0x7f7f7f7f7f7f7f7f, f"call {call}: a pivot was reported"
        assert _rel(x, ref, batch, n) <= TOL, f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_scratch():
    build.build()
    batch, n = 2048, 1024         # 48 MiB of records: more than the 32 MiB array
    band = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in range(5)]
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert _noalloc(batch, n, band, f, f) == pb._lib.PENT_EINVAL
