"""Batched solves (segmented launches over many instances of uneven n and k):
each instance's result in the batch is bit-identical to the same instance
solved alone, and close to the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import maxabs, to_scipy

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2506_04045_b300")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.load()


def _instances(specs, ks=None):
    out = []
    for i, sp in enumerate(specs):
        k = sp.k if ks is None else ks[i]
        rp, c, v = synth.make_graph(sp)
        U0 = synth.dirichlet_u0(sp.n, k, sp.seed)
        out.append(tuple(t.cuda().contiguous() for t in (rp, c, v, U0)))
    return out


MIXED_SPECS = [
    synth.GraphSpec("dcsbm", 500, 4, 301, mean_deg=12.0),
    synth.GraphSpec("dcsbm", 3001, 3, 302, mean_deg=20.0, blocks=3),
    synth.GraphSpec("dcsbm", 7000, 8, 303, mean_deg=30.0),
    synth.GraphSpec("dcsbm", 20000, 32, 304, mean_deg=25.0),
    synth.GraphSpec("dcsbm", 1200, 32, 305, mean_deg=35.0),
    synth.GraphSpec("dcsbm", 9000, 20, 306, mean_deg=18.0),
    synth.GraphSpec("dcsbm", 4000, 64, 307, mean_deg=22.0),
    synth.GraphSpec("dcsbm", 2500, 2, 308, mean_deg=15.0, blocks=2),
    synth.GraphSpec("dcsbm", 15000, 16, 309, mean_deg=40.0),
    synth.GraphSpec("dcsbm", 800, 8, 310, mean_deg=10.0),
]


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_solo_bitwise(precision):
    inst = _instances(MIXED_SPECS)
    opts = dict(stop_rule=pkg.STOP_NONE, max_iter=40, precision=precision)
    b = pkg.Batch(inst, **opts)
    reps = b.step(40)
    for i, (rp, c, v, U0) in enumerate(inst):
        s = pkg.Solver(rp, c, v, U0, **opts)
        rs = s.step(40)
        assert reps[i]["iters"] == rs["iters"] == 40
        assert torch.equal(b.get_U(i), s.get_U()), i
        assert reps[i]["f"] == rs["f"] and reps[i]["pg_norm"] == rs["pg_norm"]
        s.close()
    b.close()


def test_autotuned_batch_still_equals_solo():
    # every tuning trial is a real iteration with a candidate gather tile shape
    # (nonzeros per batch, rows per work unit) and launch shape: a shape that
    # changed any value would show in the bitwise comparison with solo runs
    inst = _instances(MIXED_SPECS[:7])
    opts = dict(stop_rule=pkg.STOP_NONE, max_iter=120)
    b = pkg.Batch(inst, **opts)
    desc = b.autotune(trials=1)
    assert all(c["tuned"] == 1 for c in desc["classes"])
    assert all(c["gather_nonzeros_per_batch"] >= 1 and c["gather_rows_per_unit"] >= 1 for c in desc["classes"])
    done = b.step(0)[0]["iters"]
    assert 0 < done < 100
    b.step(100 - done)
    for i, (rp, c, v, U0) in enumerate(inst):
        s = pkg.Solver(rp, c, v, U0, **opts)
        s.step(100)
        assert torch.equal(b.get_U(i), s.get_U()), i
        s.close()
    b.close()


def test_batch_against_oracle():
    specs = [MIXED_SPECS[2], MIXED_SPECS[5]]
    inst = _instances(specs)
    b = pkg.Batch(inst, stop_rule=pkg.STOP_NONE, max_iter=50)
    b.step(50)
    for i, (sp, (rp, c, v, U0)) in enumerate(zip(specs, inst)):
        S = to_scipy(rp, c, v, sp.n)
        o = oracle.fista(S, U0.cpu().numpy().astype(np.float64), 1.0 / oracle.lipschitz(S), max_iter=50,
                         stop="none")
        assert maxabs(b.get_U(i).cpu().numpy(), o.U) <= 1e-5


def test_batch_instances_stop_on_their_own_rule():
    specs = MIXED_SPECS[:6]
    inst = _instances(specs)
    opts = dict(stop_rule=pkg.STOP_PG_REL, tol=0.3, max_iter=300)
    b = pkg.Batch(inst, **opts)
    reps = b.step(300)
    outs = set()
    for i, (rp, c, v, U0) in enumerate(inst):
        s = pkg.Solver(rp, c, v, U0, **opts)
        rs = s.step(300)
        assert reps[i]["done"] == 1 and rs["done"] == 1
        assert reps[i]["out_iter"] == rs["out_iter"]
        outs.add(rs["out_iter"])
        assert torch.equal(b.get_U(i), s.get_U())
        s.close()
    assert len(outs) > 1        # the instances really stopped at different iterations
    # further steps leave finished instances untouched
    before = [b.get_U(i).clone() for i in range(len(inst))]
    reps2 = b.step(5)
    for i in range(len(inst)):
        assert reps2[i]["iters"] == reps[i]["iters"]
        assert torch.equal(b.get_U(i), before[i])
    b.close()


def test_batch_workload_generator_shapes():
    specs = synth.batch_specs(64, seed=3)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 500 and ns.max() <= 200_000
    assert {s.k for s in specs} <= {4, 8, 16, 32, 64}
    assert all(10.0 <= s.mean_deg <= 40.0 for s in specs)
