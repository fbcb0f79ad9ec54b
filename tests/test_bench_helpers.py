"""Host-side helpers of bench.py (no GPU): the whole-path roofline counts and
the oracle's sample shapes."""
import math

import bench
import synth


def test_path_roofline_counts_match_the_definitions():
    # Permutations N ceil(c/8) + (N - 2^h); NTT products
    # c [(n/2) log n + n + 2^r ((n/2) log n + n)] (the tabulated C1-C3 counts).
    cases = [(synth.PLAIN_8x2_10, 16_383, 4.4e5), (synth.TRACE_135x2_16, 9_437_168, 7.17e8),
             (synth.LARGE_135x2_20, 150_994_928, 1.40e10)]
    for s, perms, ntt in cases:
        assert s.perms() == perms
        n = 1 << s.log_n
        muls = s.c * ((n // 2) * s.log_n + n + (1 << s.rate_bits) * ((n // 2) * s.log_n + n))
        assert math.isclose(muls, ntt, rel_tol=0.02)
        r = bench.path_roofline(s, 1.0, 6789.0)
        assert r["W_alg"] == 6792 * perms + 4 * muls
        N = 1 << s.log_N
        assert r["bytes_alg"] == 8 * (s.c * n + 2 * s.c * N + 4 * N)


def test_path_roofline_large_commit():
    r = bench.path_roofline(synth.LARGE_135x2_20, 180.0, 6789.0)
    assert r["bound"] == "alu"
    # 1.08e12 wide multiplies at 152 x 32 x 2.07 GHz = 10.07e12 per second
    assert math.isclose(r["T_roof_ms"], r["W_alg"] / (152 * 32 * 2.07e9) * 1e3)
    assert 100.0 < r["T_roof_ms"] < 115.0
    assert math.isclose(r["fraction"], r["T_roof_ms"] / 180.0)


def test_cpu_sample_rules():
    s, whole = bench.cpu_sample(synth.PLAIN_8x2_10)
    assert whole and s == synth.PLAIN_8x2_10
    s, whole = bench.cpu_sample(synth.LARGE_135x2_20)
    assert not whole and (s.c, s.log_n, s.rate_bits, s.cap_height, s.mix) == (135, 14, 3, 4, "trace")
    s, whole = bench.cpu_sample(synth.PROFILE_8x2_20)
    assert not whole and s.c == 8 and s.c << s.log_n <= bench.CPU_SAMPLE.c << bench.CPU_SAMPLE.log_n


def test_reference_arm_line_contract():
    """--impl reference runs the oracle on the host and prints one JSON line
    with the keys of the bench contract."""
    import json
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload",
                        "plain_8x2_10", "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["workload"] == "plain_8x2_10"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
