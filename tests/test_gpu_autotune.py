"""The autotuner on the GPU: it times its candidates, writes a cache, and plans
built from that cache solve uneven batches to the oracle's parity bar."""
import numpy as np
import pytest
import torch

import oracle
import paper_1807_07382_gb300 as pb
import synth
from paper_1807_07382_gb300 import autotune

pytestmark = pytest.mark.gpu
TOL = 1e-12


def sys_rel_err(x, ref, ns):
    off = np.concatenate([[0], np.cumsum(ns)])
    return max(np.max(np.abs(x[a:b] - ref[a:b])) / max(np.max(np.abs(ref[a:b])), 1e-300)
               for a, b in zip(off[:-1], off[1:]))


@pytest.fixture(scope="module")
def cache(tmp_path_factory):
    rules = autotune.tune(buckets=(128, 2048), rows=1 << 20, steps=3, log=None)
    assert {r[0] for r in rules} == {"f64", "f32"} and len(rules) == 4
    path = tmp_path_factory.mktemp("tune") / "tune.txt"
    path.write_text(autotune.format_cache(rules, header="test"))
    return path, rules


@pytest.mark.parametrize("prec", [pb.PENT_F64, pb.PENT_F32_REFINE])
def test_tuned_plan_solves_an_uneven_batch(cache, prec):
    path, rules = cache
    w = synth.uneven(batch=96, steps=1, n_range=(64, 4096))
    ref = oracle.hyperdiff_steps(w.n, w.sigma, w.field0, 1)
    plan = pb.Plan(list(w.n), precision=prec, tune_cache=str(path))
    plan.factor_hyperdiff(torch.from_numpy(w.sigma).cuda())
    x = plan.solve(torch.from_numpy(w.field0).cuda(), max_refine=2)
    assert plan.info()[0] == pb.PENT_OK
    assert sys_rel_err(x.cpu().numpy(), ref, w.n) <= TOL
    # every system runs with the settings of the rule that covers it
    kind = "f64" if prec == pb.PENT_F64 else "f32"
    mine = [r for r in rules if r[0] == kind]
    order = np.argsort(-np.asarray(w.n), kind="stable")  # the plan's length-sorted groups of 32
    pos = np.empty_like(order)
    pos[order] = np.arange(len(order))
    for s in range(0, w.batch, 7):
        # FP32 shapes follow each system's length; FP64 settings its group's longest system
        n = int(w.n[s]) if kind == "f32" else int(w.n[order[(pos[s] // 32) * 32]])
        r = next((r for r in mine if r[1] <= n <= r[2]), mine[-1])
        a, b = plan.system_config(s)
        if kind == "f64" and a == 0:  # a group of long systems, solved by the partitioned kernels
            assert b == 256 and n >= 64
            continue
        assert a == r[3]
        if kind == "f32" and r[4]:
            assert b == r[4]
