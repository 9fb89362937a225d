"""The JSON line of `bench.py --impl reference` (the FP64 oracle timed on the host cores),
on a small sample of the 120-day workload: the keys and units the contract fixes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--cpu-days", "2"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["unit"] == "template*bins/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]


def test_roofline_flop_count_at_the_120_day_band():
    """The numerator of the bench's roofline: the spectrum kernel's algorithmic flops per
    template on the 120-day band (N_FFT = 32768, M = 2880 segments of 3600 samples, 12356
    bins, R = 1, two detectors), written out here term by term: 2 weights x 2 detectors x
    2880 segments of 5 N log2 N, and 8 flops per (weight, detector, segment, bin) and
    partner with 2R + 2 = 4 partners."""
    sys.path.insert(0, ROOT)
    import bench
    info = {"N_FFT": 32768, "M": 2880, "N_f": 12356, "N_tau": 2880 * 3600, "R": 1}
    c = bench.algorithmic_costs(info, 2, 1)
    fft = 2 * 2 * 2880 * (5 * 32768 * 15)
    pairs = 2 * 2 * 2880 * 12356 * 8 * 4
    assert c["fft_flops"] == fft == 28_311_552_000
    assert c["pair_flops"] == pairs == 4_554_915_840
    assert abs(c["fft_flops"] + c["pair_flops"] - 3.2866e10) < 1e6
    # resampling: 17 taps x 8 flops + 30 per sample and detector
    assert c["interp_flops"] == 2 * 2880 * 3600 * (8 * 17 + 30)


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm and prints; the others exit 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0", "--cpu-days", "2"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [l for l in out.stdout.splitlines() if l.startswith("{")]


def test_gpus_flag_launches_ranks_itself():
    """`--gpus 2` outside a launcher re-runs the bench under torch.distributed.run with two
    ranks on this node: rank 0 alone prints one JSON line and it saw a world of 2."""
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR",
                                                            "MASTER_PORT")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                          "--steps", "1", "--warmup", "0", "--cpu-days", "1"], capture_output=True, text=True,
                         timeout=900, cwd=ROOT, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2 and d["ranks_seen"] == 2
