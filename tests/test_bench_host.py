"""Host-side logic of bench.py that needs no GPU: the config record, the
roofline helpers (measured peak, DRAM-traffic lookup keyed on the kernel
source), the job value, and one oracle step of the reference arm."""

import json
import os
import re

import bench


def test_config_names_workload_and_method():
    c = bench.config(48, "mixed")
    assert c["workload"].startswith("kuhn48^3") and c["n_cubes"] == 48
    assert c["dofs_per_solve"] == 3 * 97 ** 3 + 49 ** 3
    assert c["solves_per_step"] == len(bench.MUS) and c["tol"] == 1e-8
    assert c["method"] == "schur-cg" and c["schur_prec"] == "C^Lambda"
    json.dumps(c)                                    # one JSON line


def test_job_value_is_aggregate_dofs_per_second():
    assert bench.job_value(1, 3, 1000, 1000.0) == 3000.0
    assert bench.job_value(4, 3, 1000, 1000.0) == 12000.0


def test_traffic_lookup_matches_committed_profile():
    sha = bench.kernel_source_sha()
    assert re.fullmatch(r"[0-9a-f]{16}", sha)
    lines = []
    for fn in os.listdir(os.path.join(bench.ROOT, "profiles")):
        for line in open(os.path.join(bench.ROOT, "profiles", fn)):
            m = re.search(r"bench-traffic: kernel=(\w+) bytes_per_launch=(\S+) sparse_cu_sha=(\w+)", line)
            if m:
                lines.append(m.groups())
    assert lines, "no traffic record in profiles/"
    got = bench.ncu_traffic("SPMM_A3")
    current = [float(b) for k, b, s in lines if k == "SPMM_A3" and s == sha]
    assert got == (current[0] if current else None)
    assert bench.ncu_traffic("NO_SUCH_KERNEL") is None


def test_measured_peak_is_positive():
    peak, kind = bench.measured_peak_gbs()
    assert peak > 0 and kind in ("measured", "fallback")


def test_oracle_step_of_the_reference_arm():
    t, worst = bench.oracle_step(n=2)
    assert t > 0 and worst < 1e-12
