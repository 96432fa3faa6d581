"""bench.py's host side on CPU: the algorithmic byte counts behind the
roofline (pinned to the closed forms of the two Poisson workloads) and the
reference arm's JSON line (the CPU oracle; no GPU involved)."""
import contextlib
import io
import json
import os
import sys

import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("s", [2, 3, 5, 8])
def test_poisson_nnz_closed_forms(s):
    # 7-point: s^3 diagonal entries plus two per interior face in each of 3 directions
    assert synth.poisson7(s).nnz == s ** 3 + 6 * s * s * (s - 1)
    # 27-point: (3s - 2)^3 (each axis contributes 3s - 2 neighbour pairs, counting the centre)
    assert synth.poisson27(s).nnz == (3 * s - 2) ** 3


def test_algorithmic_bytes():
    import bench
    # the 7-point 16^3 system: n = 4096, nnz = 27,136 -> 702,468 B per iteration
    A = synth.poisson7(16)
    assert (A.n, A.nnz) == (4096, 27136)
    assert bench.iter_bytes(A.n, A.nnz) == 702_468
    # the 27-point 256^3 system from its closed form (too large to build here)
    n, nnz = 256 ** 3, (3 * 256 - 2) ** 3
    assert nnz == 449_455_096
    assert bench.iter_bytes(n, nnz) == 6_936_965_028
    assert bench.pass_a_bytes(n, nnz) == 5_729_005_476
    # the passes' own bytes (A, B 56 n, C 32 n) exceed the iteration's minimum by the two
    # re-reads of d in passes B and C (16 n): the iteration counts d once
    assert bench.pass_a_bytes(n, nnz) + 56 * n + 32 * n == bench.iter_bytes(n, nnz) + 16 * n


def test_reference_arm_json_line():
    import bench

    class A:
        side, stencil, steps, warmup, tol, band, band_n = 6, 7, 1, 1, 1e-8, 0, 0
        variant, max_iter, gpus = "exblas", 5000, 1

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.reference_arm(A, 0, 1)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "iters/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"] == "poisson7_6 exblas"
    # the same workload record as the GPU arm's line (the driver compares the two arms)
    assert line["config"] == bench.workload_config(A, line["config"]["n"], line["config"]["nnz"])


def test_pass_a_traffic_record():
    """The roofline record's DRAM traffic: the full-size capture at 27-point
    256^3 (within 0.1% of the algorithmic bytes: every entry and vector
    element crosses HBM once), the 128^3 ratio at other 27-point sizes, and
    no figure where no capture applies."""
    import bench

    class A:
        band, stencil, side = 0, 27, 256

    n, nnz = 256 ** 3, (3 * 256 - 2) ** 3
    t, src = bench.pass_a_traffic(A, n, nnz)
    assert t == 5_726_131_968 and "256^3" in src and "full size" in src
    assert abs(t / bench.pass_a_bytes(n, nnz) - 1.0) < 1e-3
    A.side = 128
    n, nnz = 128 ** 3, (3 * 128 - 2) ** 3
    t, src = bench.pass_a_traffic(A, n, nnz)
    assert "128^3" in src and abs(t / bench.pass_a_bytes(n, nnz) - 702.0 / 710.9) < 1e-12
    A.stencil = 7
    assert bench.pass_a_traffic(A, n, nnz) == (None, None)
    A.stencil, A.band = 27, 100
    assert bench.pass_a_traffic(A, n, nnz) == (None, None)
