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
    assert d["metric"] == "messenger TOD Gsamples/s" and d["unit"] == "Gsamples/s"
    assert d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "t64_1det_2^15"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"]
    # value = samples of the sample per second: one chunk of 32768 samples per step
    assert abs(d["value"] - 32768 / (d["ms_per_step"] * 1e-3) / 1e9) <= 1e-9 * d["value"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0


def test_algorithmic_bytes_model():
    """The bytes model behind `roofline` and `iteration_hbm`.  For the 2048^2 IQU, 32 x 2^24
    FP16 workload: per iteration B_strict = 20 B/sample + 104 B/pixel and B_pass = 36 B/sample
    + 104 B/pixel; per kernel A n(4+4) + 4n + 16 n_pix, B 12n, C 4n + 8n + 24 n_pix, D 64 B
    per pixel, summing to B_pass.  For the 512^2 IQU, 8 x 2^22 FP32 workload: 28 and 44
    B/sample.  The FP32 Nbar table the filter also reads is 2 B/sample, reported apart."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    for nchunk, logn, width, wdt, ws, wp in ((32, 24, 2048, np.float16, 20, 36),
                                             (8, 22, 512, np.float32, 28, 44)):
        n, npix = nchunk << logn, width * width
        w = 4 if wdt == np.float16 else 8
        s = {"offsets": np.arange(nchunk + 1, dtype=np.int64) << logn, "ncomp": 3, "npix": npix,
             "cos": np.zeros(1, dtype=wdt)}
        stages, strict, bpass, tables = bench.bytes_model(s)
        assert stages["gather_fft"] == n * (4 + w) + 4 * n + 16 * npix
        assert stages["filter"] == 12 * n
        assert stages["ifft_bin"] == 4 * n + n * (4 + w) + 24 * npix
        assert stages["map"] == 64 * npix
        assert stages["fused_passes"] == stages["gather_fft"] + stages["filter"] + stages["ifft_bin"]
        assert strict == ws * n + 104 * npix
        assert bpass == wp * n + 104 * npix
        assert bpass == sum(v for k, v in stages.items() if k != "fused_passes")
        assert tables == 2 * n
    # T-only, one chunk of 2^15 samples (above the on-chip size): 12 B/sample + 24 B/pixel
    # strict, plus 16 B/sample of exchange
    s = {"offsets": np.array([0, 1 << 15], dtype=np.int64), "ncomp": 1, "npix": 4096, "cos": None}
    _, strict, bpass, _ = bench.bytes_model(s)
    assert strict == 12 * (1 << 15) + 24 * 4096 and bpass == strict + 16 * (1 << 15)
