"""The bench's host-side pieces on a small workload: the oracle reference arm prints the
contract's keys, and the per-kernel byte model matches its definition."""
import argparse
import json

import bench


def test_reference_arm_contract(monkeypatch):
    monkeypatch.setattr(bench, "SAMPLE_GRID", (8, 4, 4))
    args = argparse.Namespace(steps=2, warmup=1, gpus=1, smoother="chebyshev", cheb_degree=2)
    out = bench.run_reference(args, rank=0, world=1)
    json.dumps(out)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
              "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] > 0
    assert out["e2e"]["h2d_bytes_per_step"] == 0
    # one step is one complete oracle solve, timed: steps x ms_per_step is the arm's run time
    assert out["ms_per_step"] > 0 and out["steps"] == 2
    assert bench.run_reference(args, rank=1, world=2) is None


def test_kernel_bytes_model():
    import workloads as W
    p = W.cantilever_2d(8, 4, seed=0)
    nn = p.n // 2
    assert bench.kernel_bytes("outer", "fp64", p) == 2 * 8 * p.n + 8 * p.nel + nn
    assert bench.kernel_bytes("residual", "fp32", p) == 3 * 4 * p.n + 4 * p.nel + nn
    assert bench.kernel_bytes("jacobi", "fp32", p) == 3 * 4 * p.n + 4 * p.nel + nn + 2 * 4 * nn


def test_throughput_helpers():
    assert bench.throughput(10, 1, 1000.0) == 10.0
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_golden_fixtures_parse():
    import os
    import sys
    sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
    import refs
    for name, nrhs in (("cantilever3d_192x96x96", 1), ("batched3d_128x64x64", 16),
                       ("cantilever2d_768x384", 1), ("mbb_96x32", 1)):
        r = refs.load(name)
        assert len(r) == nrhs
        for e in r:
            assert e["true_rel_residual"] < 1e-8 and len(e["uniform"]) == 200
            assert e["proj"].shape == (refs.N_PROJ,) and e["compliance"] > 0
