"""Host-side arithmetic of bench.py: algorithmic bytes, percentiles, the
whole-job throughput and the block-diagonal replication used for the
bandwidth workload.  CPU only."""
import numpy as np
import pytest

import bench
from paper_1604_07491_gb300 import gen


def test_algorithmic_bytes_counts_each_unit():
    m, n, nnz = 10, 30, 100
    one = dict(sweep_passes=0, row_passes=0, csc_passes=0, krylov_iters=0, basis_passes=0)
    assert bench.algorithmic_bytes(one, m, n, nnz, "mixed") == 0
    assert bench.algorithmic_bytes(dict(one, sweep_passes=1), m, n, nnz, "mixed") == nnz * 24 + m * 28
    assert bench.algorithmic_bytes(dict(one, sweep_passes=1), m, n, nnz, "fp64") == nnz * 28 + m * 28
    assert bench.algorithmic_bytes(dict(one, row_passes=2), m, n, nnz, "fp64") == 2 * (nnz * 20 + m * 12)
    assert bench.algorithmic_bytes(dict(one, csc_passes=1), m, n, nnz, "fp64") == nnz * 20 + n * 12
    assert bench.algorithmic_bytes(dict(one, krylov_iters=1), m, n, nnz, "fp64") == 8 * (12 * n + 12 * m)
    assert bench.algorithmic_bytes(dict(one, basis_passes=3), m, n, nnz, "fp64") == 3 * 8 * m


def test_percentile_nearest_rank():
    v = list(range(1, 101))
    assert bench.percentile(v, 0.5) == 50 and bench.percentile(v, 0.99) == 99
    assert bench.percentile([7.0], 0.99) == 7.0


def test_weak_throughput_and_offsets():
    assert bench.weak_throughput(2, 16, 5, 10000.0) == pytest.approx(16.0)
    assert bench.replica_offsets(1, 4) == [4, 5, 6, 7]
    assert bench.max_over_ranks(3.5, None) == 3.5


def test_replicated_csr_is_block_diagonal():
    lp = gen.tiny_lp()
    m, n, rp, ci, val = bench.replicated_csr(lp, 3)
    A = lp.scipy().toarray()
    import scipy.sparse as sp
    B = sp.csr_matrix((val, ci, rp), shape=(m, n)).toarray()
    for k in range(3):
        assert np.array_equal(B[k * lp.m:(k + 1) * lp.m, k * lp.n:(k + 1) * lp.n], A)
    assert np.count_nonzero(B) == 3 * np.count_nonzero(A)


def test_reference_arm_prints_the_contract_line():
    # bench.py --impl reference: the oracle on the host cores, one JSON line
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--workload", "tiny", "--batch", "2", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=root)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "LPs/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_large_byte_formulas():
    # one NE-SOR pass over FP32 values (half of the FP32 NE-SSOR sweep formula)
    # and the FP64 product y = A x
    assert bench.sweep_pass_bytes(1000, 10) == 1000 * 16 + 10 * 20
    assert bench.sweep_pass_bytes_moved(1000, 10) == 1000 * 24 + 10 * 20
    assert bench.spmv_bytes(1000, 10, 30) == 1000 * 12 + 10 * 16 + 30 * 8
    # the large LP: about 44 MB per NE-SOR pass, about 34 MB per product
    lp = gen.large_lp(1.0)
    assert 40e6 < bench.sweep_pass_bytes(lp.nnz, lp.m) < 48e6
    assert 30e6 < bench.spmv_bytes(lp.nnz, lp.m, lp.n) < 38e6


def test_traffic_record_requires_unchanged_sources(tmp_path, monkeypatch):
    import json
    import os
    rec_dir = tmp_path / "profiles"
    rec_dir.mkdir()
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    digest = bench.source_digest(["k.cu"])
    (rec_dir / "ncu_traffic.json").write_text(json.dumps(
        {"sweep": {"sources": ["k.cu"], "sources_sha256": digest, "dram_bytes_per_launch": 1.5e7,
                   "command": "ncu ..."}}))
    assert bench.measured_traffic("sweep")[0] == 1.5e7
    assert bench.measured_traffic("other")[0] is None
    src.write_text("kernel v2")          # the kernel changed since the capture
    assert bench.measured_traffic("sweep")[0] is None
    assert os.path.exists(rec_dir / "ncu_traffic.json")


def test_reference_arm_large_prints_the_contract_line():
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GB/s" and line["value"] > 0
    assert line["config"]["workload"].startswith("large") and line["config"]["m"] == 150000
    assert line["cpu_baseline"]["cores"] == 1
