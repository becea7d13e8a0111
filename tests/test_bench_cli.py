"""bench.py's contract on the CPU: every workload has its GPU body, and the
reference arm (the oracle, timed on the host) prints one JSON line with the
keys the contract asks for."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_every_workload_has_a_gpu_body():
    sys.path.insert(0, str(ROOT))
    import bench
    names = {"poisson3d": "gpu_poisson", "poisson2d": "gpu_poisson", "wave": "gpu_wave", "batched": "gpu_batched",
             "learned": "gpu_learned", "conv": "gpu_conv"}
    names.update({w: "gpu_paper" for w in bench.PAPER_WORKLOADS})
    assert set(bench.WORKLOADS) == set(names)
    for w, fn in names.items():
        assert callable(getattr(bench, fn)), w


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "conv", "--steps", "1",
                          "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0



def test_paper_workload_oracle_samples_run():
    """Every paper workload's CPU oracle sample runs and reports its units."""
    sys.path.insert(0, str(ROOT))
    import bench
    for w in ("rs_w", "qoi"):
        v, sample, rec = bench.cpu_oracle_sample(w)
        assert v > 0 and rec["units"] > 0 and sample
