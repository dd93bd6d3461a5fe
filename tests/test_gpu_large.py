"""The 2048^2 IQU workload (32 detectors x 2^24 samples, FP16 weights, rasters at four
angles) at full size, in the launch configuration the benchmark times.  The oracle cannot
iterate on 537 M samples in reasonable time; it is applied to samples of the output (pixels
drawn at random, with every sample that hits them) and to properties that hold at any
size.  Marked slow (its inputs take about half a minute to generate)."""
import math

import numpy as np
import pytest

import oracle.messenger as O
from paper_1705_01893_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1705_01893_gb300 import build
    build.build()
    binding.load()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_crosslinked_2048_full_size():
    s = synth.config_crosslinked()
    plan = binding.plan_from_synth(s, DEV)
    npix = s["npix"]
    pix = s["pix"]
    # hit counts: bit-exact
    hits = torch.empty(npix, dtype=torch.int32, device=DEV)
    valid = torch.empty(npix, dtype=torch.uint8, device=DEV)
    plan.maps(hits, valid)
    torch.cuda.synchronize()
    ref_hits = np.bincount(pix[pix >= 0], minlength=npix)
    assert np.array_equal(hits.cpu().numpy(), ref_hits)
    # one 2^24-point chunk's rfft
    n0 = int(s["offsets"][1])
    spec = torch.empty((len(s["offsets"]) - 1) * (n0 // 2 + 1), 2, dtype=torch.float32, device=DEV)
    plan.rfft(plan.tod, spec)
    g = spec[:n0 // 2 + 1].double().cpu().numpy()
    assert rel(g[:, 0] + 1j * g[:, 1], np.fft.rfft(s["tod"][:n0].astype(np.float64))) <= 1e-6
    del spec
    # the binned map (lambda = inf step) at 256 random hit pixels, against the oracle run on
    # exactly the samples that hit them (the binned map of a pixel depends on no others)
    m = torch.zeros(npix, 3, dtype=torch.float64, device=DEV)
    plan.messenger(m, [math.inf])
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    pick = rng.choice(np.flatnonzero(ref_hits > 0), 256, replace=False)
    sel = np.isin(pix, pick)
    lut = np.full(npix, -1, np.int64)
    lut[pick] = np.arange(len(pick))
    off = s["offsets"]
    sub_off = np.concatenate([[0], np.cumsum([int(sel[off[c]:off[c + 1]].sum())
                                              for c in range(len(off) - 1)])])
    psd = [np.ones(int(sub_off[c + 1] - sub_off[c]) // 2 + 1) for c in range(len(off) - 1)]
    prob = O.Problem(lut[pix[sel]], s["cos"][sel], s["sin"][sel], s["tod"][sel], sub_off,
                     len(pick), 3, psd, np.ones(len(off) - 1), 1e-3)
    m_ref, _ = O.messenger_step(prob, np.zeros((len(pick), 3)), math.inf)
    got = m.cpu().numpy()[pick]
    keep = prob.valid
    near = np.abs(prob.rcond - 1e-3) <= 1e-9
    assert np.array_equal(valid.cpu().numpy()[pick].astype(bool)[~near], keep[~near])
    assert rel(got[keep], m_ref[keep]) <= 1e-5
    # fixed lambda: chi^2(m_i, lambda) never increases (App. A), here over 3 iterations
    chi = torch.zeros(4, dtype=torch.float64, device=DEV)
    plan.messenger(m, [10.0] * 4, chi)
    c = chi.cpu().numpy()
    assert np.all(np.diff(c) <= 1e-9 * c[0]), c
