"""bench.py's reference arm (the FP64 oracle on the host) prints one JSON line with the
contract's keys; run on the small 64^2 T-only workload so it takes seconds."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "t64_1det_2^15", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["metric"] == "messenger iters/s" and d["unit"] == "iter/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "t64_1det_2^15"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_bytes_of_the_headline_workload():
    """The byte model behind `roofline` and `iteration_hbm` on the 512^2 IQU, 8 x 2^22 FP32
    workload: A n(4+w) + 4n + 16 n_pix, B 14n, C 4n + n(4+w) + 24 n_pix, D 112 B per pixel,
    the fused launch A + B + C; B_pass and B_strict per iteration (46 B/sample + 152 B/px
    and 28 B/sample + 104 B/px)."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    n, npix = 8 << 22, 512 * 512
    s = {"offsets": np.arange(9, dtype=np.int64) << 22, "ncomp": 3, "npix": npix,
         "cos": np.zeros(1, dtype=np.float32)}
    stages, strict, bpass = bench.bytes_model(s)
    assert stages["gather_fft"] == n * 12 + 4 * n + 16 * npix          # 541 MB
    assert stages["filter"] == 14 * n                                 # 470 MB
    assert stages["ifft_bin"] == 4 * n + 12 * n + 24 * npix           # 543 MB
    assert stages["map"] == 112 * npix                                # 29 MB
    assert stages["fused_passes"] == stages["gather_fft"] + stages["filter"] + stages["ifft_bin"]
    assert bpass == 46 * n + 152 * npix                               # 1.58 GB
    assert strict == 28 * n + 104 * npix                              # 0.97 GB
