"""The benchmark's reference arm (the oracle timed on the host cores) runs
without a GPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    env = dict(os.environ, PFFT_REF_STEP_S="0.2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["value"] > 0 and j["steps"] == 2
    assert j["config"]["workload"]
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["cores"] >= 1
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["value"] == j["value"]


def test_smith_fftn_context_baseline_matches_oracle():
    """The bench's library CPU transform (numpy fftn after the Smith gather)
    agrees with the oracle's direct sum."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import oracle
    import seeded_inputs as SI
    from oracle import lattice as L

    for M in (SI.M_SMALL_2D, [[8, 2], [2, -4]], [[3, 1, 2], [0, 2, 1], [1, 0, 4]], [[4, 1, 0], [0, 4, 1], [0, 0, 4]],
              [[1, 0], [0, 1]]):
        m = abs(L.det(M))
        c = SI.complex_normal(1, m, 3, dtype=np.complex128)
        assert np.allclose(bench.smith_fftn(M, c[0]), oracle.pattern_fft(M, c)[0], atol=1e-12)
