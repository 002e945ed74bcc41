"""Host logic of bench.py on CPU: kernel families and source hashes of the
ncu traffic table, the committed traffic figures against the algorithmic
bytes, and the workload description of the bench line."""
import argparse
import json
import os

import pytest

import bench


def test_kernel_families():
    assert bench.family_of("cg_p") == bench.family_of("cg_r") == "cg"
    assert bench.family_of("mg_post1.L0") == bench.family_of("mg_tail") == "mg"
    assert bench.family_of("cg_finish") == bench.family_of("extrap") == "flat"
    assert bench.family_of("rhs") == bench.family_of("tdgl") == "step"
    assert bench.family_of("tdgl_adj") == "adj"
    assert bench.family_of("diag") == "diag"


def test_source_hash_ignores_comments_only():
    code = "int f(int a) {\n  return a + 1;  // one more\n}\n"
    assert bench._code_only(code) == bench._code_only("/* doc */ int f(int a) {\n  return a + 1;\n}\n")
    assert bench._code_only(code) != bench._code_only(code.replace("+ 1", "+ 2"))
    h = bench.kernel_source_hash("cg_p")
    assert len(h) == 16 and h == bench.kernel_source_hash("cg_r")      # one family, one hash


def test_committed_traffic_is_at_most_the_algorithmic_bytes():
    """The ncu summary's claim: no kernel moves more DRAM bytes than the
    arrays it must read and write once (L2 can only lower the figure)."""
    path = os.path.join(bench.ROOT, "profiles", "traffic.json")
    d = json.load(open(path))
    assert d["kernels"]
    for name, e in d["kernels"].items():
        assert e["workload"] == "tip"
        assert 0 < e["dram_bytes_per_cell"] <= 1.02 * e["algorithmic_bytes_per_cell"], name
    assert bench.ncu_traffic(next(iter(d["kernels"])), "strips", 1000) is None       # other workload


@pytest.mark.parametrize("noise,rtol,order", [(0.0, 1e-7, 3), (0.0, 1e-6, 2), (0.05, 1e-7, 1)])
def test_workload_line_names_the_extrapolation_order(noise, rtol, order):
    w = bench.make_workload("tip", size=(16, 16, 8)).with_(rtol=rtol)
    args = argparse.Namespace(integrator="euler", poisson_every=1, warm_last=False, noise=noise, extrap_order=0)
    c = bench.workload_config(w, "tip", "flushed", args)
    assert ("order %d" % order) in c["warm_start"]
    assert c["cells"] == 16 * 16 * 8 and c["solver"] == "mg"
    args.warm_last = True
    assert bench.workload_config(w, "tip", "flushed", args)["warm_start"] == "last potential"
