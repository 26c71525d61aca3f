"""The benchmark's roofline arithmetic (no GPU): algorithmic bytes of the operator, useful
flops of a Schwarz domain visit, operator equivalents of a solve, and the source-hash
gate on the committed ncu traffic."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_operator_bytes_per_site(bench):
    # 4 forward links x 18 reals + 72 clover reals + 24 in + 24 out = 192 reals (Sec. II-B)
    assert bench.dslash_bytes_per_site("fp32") == 768
    assert bench.dslash_bytes_per_site("fp64") == 1536
    assert bench.dslash_bytes_per_site("fp16") == 392   # plus two 4-byte spinor norms


def test_paper_flop_counts(bench):
    # 8 hops x 168 = 1344 for the hopping term, 504 for the clover term, 1848 in all
    assert 8 * bench.FLOP_HOP + bench.FLOP_CLOVER == bench.FLOP_A == 1848


def test_schwarz_visit_flops_for_8x4x4x4(bench):
    # worked by hand: 6.25 inside and 1.75 crossing hops per site; MR step 168 * 6.25 + 504
    # + 192 = 1746; preparation = reconstruction = 525 + 252 + 24 = 801; faces
    # 1.75 * 90 + 1.75 * 78 + 72 = 366; 4 * 1746 + 2 * 801 + 366 = 8952
    useful, nominal = bench.sap_visit_flops((8, 4, 4, 4), 4)
    assert useful == pytest.approx(8952.0)
    assert nominal == pytest.approx(4 * (1848 + 192) + 1848)


def test_schwarz_visit_flops_tend_to_the_full_operator(bench):
    # a domain as large as the lattice has no crossing hops: every MR step then costs a full
    # operator application plus the 192 flops of inner products and updates
    big = (1 << 20,) * 4
    u1, n1 = bench.sap_visit_flops(big, 1)
    u5, n5 = bench.sap_visit_flops(big, 5)
    assert (u5 - u1) / 4 == pytest.approx(bench.FLOP_A + 192.0, rel=1e-5)
    assert (n5 - n1) / 4 == pytest.approx(bench.FLOP_A + 192.0)
    # and smaller domains lose hops to the faces
    assert bench.sap_visit_flops((4, 4, 4, 4), 4)[0] < bench.sap_visit_flops((8, 8, 8, 8), 4)[0]


def test_operator_equivalents_of_a_solve(bench):
    import synth
    w = synth.WORKLOADS["32^3x64"]
    # per iteration one A plus I_S x 2 half-sweeps of (I_d + 1) / 2 A-equivalents, plus the
    # FP64 residuals
    n = bench.a_equivalents(w, 10, 3)
    assert n == pytest.approx(10 * (1 + w.i_schwarz * (w.i_domain + 1)) + 3)


def test_profile_traffic_needs_the_current_source(bench, tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k.txt").write_text("# summary\nsource_sha: abc123\ndram_bytes_per_launch: 1234\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_profile("k.txt", "abc123") == 1234.0
    assert bench.read_profile("k.txt", "ffffff") is None
    assert bench.read_profile("missing.txt", "abc123") is None


def test_oracle_all_cores_sample_runs_and_fails_cleanly():
    """The all-cores oracle baseline: one spawned process per core times the same small
    samples concurrently and returns the slowest times; a process that fails (a lattice the
    domain shape does not divide) releases the others and raises instead of hanging."""
    import sys
    sys.path.insert(0, ROOT)
    import bench as B
    import synth
    w = synth.WORKLOADS["32^3x64"]
    fa = B.oracle_fields(w, (8, 8, 8, 8))
    n, t_a, t_s = B.oracle_all_cores(w, fa, B.oracle_fields(w, (16, 8, 8, 8)))
    assert n == (os.cpu_count() or 1) and t_a > 0 and t_s > 0
    with pytest.raises(RuntimeError):
        B.oracle_all_cores(w, fa, B.oracle_fields(w, (12, 8, 8, 8)))
