"""Host-side bookkeeping of bench.py (CPU): the kernel-source hash that keys
the recorded ncu DRAM figures ignores comments and blank lines but not code,
and the recorded figures are looked up per kernel kind and workload."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_lines_drop_comments_and_blank_lines():
    a = "int x = 1;  // first\n\n// a whole comment line\nfloat y;   \n"
    b = "int x = 1;\nfloat y;"
    assert bench._code_lines(a) == b
    assert bench._code_lines("int x = 2;\nfloat y;") != b


def test_source_hash_is_stable_and_short():
    h = bench._source_hash()
    assert h == bench._source_hash()
    assert len(h) == 12 and all(c in "0123456789abcdef" for c in h)


def test_traffic_lookup_follows_the_recorded_hash(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    h = bench._source_hash()
    (prof / "dram_traffic.txt").write_text(
        "# kind workload hash bytes\n"
        f"xy_inv_score {bench.WORKLOAD} {h} 1234\n"
        f"z_inv_score {bench.WORKLOAD} 000000000000 99\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "_source_hash", lambda: h)
    assert bench._ncu_traffic("xy_inv_score") == 1234.0
    assert bench._ncu_traffic("z_inv_score") is None     # recorded on other sources
    assert bench._ncu_traffic("xy_fwd_score") is None    # not recorded


def test_oracle_on_host_cores_equals_the_oracle():
    """The bench's multi-process run of the oracle (orientations dealt over
    spawned single-threaded workers, the orientation sums of M and of the
    inverse added up from the parts) gives the oracle's own inverse(forward(f))
    up to the summation order."""
    import numpy as np
    from oracle import os3d_oracle as O
    dims = (8, 10, 12)
    f = np.random.default_rng(41).standard_normal(dims)
    V = O.icosa_orientations(1)
    bank = O.Bank(dims, V, O.Params(L=8))
    ref = O.inverse(O.forward(f, bank), bank)
    oc = bench.OracleOnCores(dims, V, 8, f, cores=3)
    try:
        assert oc.cores == 3 and sorted(sum(oc.parts, [])) == list(range(len(V)))
        assert np.abs(oc.bank.M() - bank.M()).max() < 1e-13 * bank.M().max()
        out, dt = oc.step()
    finally:
        oc.close()
    assert dt > 0
    assert np.abs(out - ref).max() < 1e-12 * np.abs(ref).max()


def test_oracle_sample_on_cores_runs_one_orientation_per_process():
    """The bounded oracle sample of the large workload, here on the small one:
    one orientation per process, the throughput over the slowest process."""
    v, desc, n = bench.oracle_sample_on_cores("tubes32_no42", cores=3)
    assert n == 3 and v > 0
    assert desc.startswith("3 of the 42 orientations")
