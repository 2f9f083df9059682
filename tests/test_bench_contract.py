"""The bench's reference arm (the FP64 oracle on the host cores) runs
without a GPU: its JSON line carries the contract's keys, and the oracle
sampler's pair count and rate are consistent; the per-face work the
roofline uses equals a fresh count by the oracle's counting build, and its
DRAM traffic per face the committed flux-kernel captures.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0", "--cpu-n", "4096"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["e2e"]["value"] == line["value"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["config"]["workload"] == "lognormal3d_134217728_mfv_exact"


def test_oracle_sampler_counts_pairs_like_the_metric():
    sys.path.insert(0, ROOT)
    import bench
    r1, t1 = bench.oracle_sample_rate("wave", 10, 1)
    r2, t2 = bench.oracle_sample_rate("wave", 10, 1, threads=1)
    assert r1["cores"] >= 1 and r2["cores"] == 1
    assert r1["value"] > 0 and r2["value"] > 0
    # the same sample: the same pair count in the description
    count = lambda r: int(r["sample"].split(" pair-interactions")[0].split()[-1])
    assert count(r1) == count(r2) > 0


def test_face_work_constants_match_a_fresh_count():
    sys.path.insert(0, ROOT)
    import bench
    from oracle import face_work
    t = face_work.table()
    assert set(t) == set(bench.FACE_OPS)
    for kind, v in t.items():
        for k, c in bench.FACE_OPS[kind].items():
            assert abs(v[k] - c) <= 1e-3 * max(1.0, abs(c)), (kind, k, v[k], c)
    # the counts measure real work: a Newton iteration evaluates both sides'
    # pressure functions (two powers at least when a side rarefies)
    assert 30 < t["sod"]["flop_per_iter"] < 80 and t["wave"]["flop_per_iter"] == 0.0


def test_traffic_constants_match_the_committed_captures():
    """The roofline's DRAM traffic per face is the one the committed ncu
    summaries of the flux kernel state (read + write over the faces of the
    captured launch), workload by workload."""
    import re
    sys.path.insert(0, ROOT)
    import bench
    files = {"sod": "k_fluxes_sod3d_n60.md", "lognormal": "k_fluxes_lognormal_2097152.md"}
    assert set(files) == set(bench.FLUX_TRAFFIC_BYTES_PER_FACE)
    for kind, name in files.items():
        text = open(os.path.join(ROOT, "profiles", name)).read()
        rd = float(re.search(r"dram__bytes_read\.sum`\) \| ([0-9.]+) Mbyte", text).group(1))
        wr = float(re.search(r"dram__bytes_write\.sum`\) \| ([0-9.]+) Mbyte", text).group(1))
        faces = int(re.search(r"MB / ([0-9,]+) = ", text).group(1).replace(",", ""))
        per_face = (rd + wr) * 1e6 / faces
        assert abs(per_face - bench.FLUX_TRAFFIC_BYTES_PER_FACE[kind]) < 0.006, (kind, per_face)
