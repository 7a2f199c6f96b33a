"""Host-side helpers of bench.py (CPU): the code fingerprint that keys the stored DRAM traffic, the
traffic lookup, and the whole-job throughput formula."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_fingerprint_ignores_comments_and_whitespace(tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    c = tmp_path / "c.cu"
    a.write_text("// header\nint f(int x) { return x + 1; }  /* note */\n")
    b.write_text("int  f(int x)\n{\n    return x + 1;   // another note\n}\n")
    c.write_text("int f(int x) { return x + 2; }\n")
    assert bench.code_fingerprint([str(a)]) == bench.code_fingerprint([str(b)])
    assert bench.code_fingerprint([str(a)]) != bench.code_fingerprint([str(c)])
    assert bench.code_fingerprint([str(a), str(c)]) != bench.code_fingerprint([str(c), str(a)])


def test_traffic_lookup_is_keyed_by_the_current_code():
    """A stored value is returned only while its fingerprint matches the kernel source (else the
    bench reports traffic null rather than counters of other code)."""
    cur = bench.code_fingerprint(bench.KERNEL_SRC)
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    keys = []
    with open(path) as fh:
        for line in fh:
            parts = line.split()
            if len(parts) == 3 and not line.startswith("#"):
                keys.append(parts[0])
                want = float(parts[1]) if parts[2] == cur else None
                assert bench.traffic_from_profiles(parts[0]) == want
                assert float(parts[1]) > 0
    assert "f64_multi_resident_512" in keys
    assert bench.traffic_from_profiles("no_such_kernel") is None


def test_whole_job_throughput():
    # 2 ranks x 18 operators x 2^27 points x 10 steps in 100 ms
    v = bench.job_throughput(2, 18, 2 ** 27, 10, 100.0)
    assert abs(v - 2 * 18 * 2 ** 27 * 10 / 0.1 / 1e9) < 1e-9
