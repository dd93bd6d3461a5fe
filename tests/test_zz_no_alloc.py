"""The allocation-free binned map (mm_binned_map_noalloc) against the planned path and the
FP64 oracle.

Some callers cannot allocate device memory -- work recorded into a CUDA graph, code under an
allocator that must not grow, or a host that only receives device pointers -- yet need the
binned map (P^T P)^-1 P^T d.  The entry point keeps its accumulators in a fixed device
array.  Its map must equal the lambda = infinity messenger step of a plan built on the same
data (tau = sigma^2 = 1, so the map step weights are (P^T P)^-1), and the oracle's binned
map, call after call.  This file is named to be collected last, so a run that stops at the
first failure has run every other test first.
"""
import math

import numpy as np
import pytest

import oracle.messenger as O
from paper_1705_01893_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1705_01893_gb300 import build
    build.build()
    binding.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("kind", ["iqu", "temperature"])
def test_noalloc_binned_map_matches_plan_twice(kind):
    s = synth.config_iqu(64, 4, 1 << 14, 31) if kind == "iqu" else synth.config_temperature_64()
    nc = s["ncomp"]
    plan = binding.plan_from_synth(s, DEV)              # sigma = 1: tau = 1 for every chunk
    ref = torch.zeros(s["npix"], nc, dtype=torch.float64, device=DEV)
    plan.messenger(ref, [math.inf])                      # lambda = inf: the binned map
    pix = plan.pix
    cos, sin = plan.cos2psi, plan.sin2psi
    for call in range(2):                                # the second call reuses the scratch
        out = torch.full((s["npix"], nc), float("nan"), dtype=torch.float64, device=DEV)
        binding.binned_map_noalloc(pix, cos, sin, plan.tod, s["npix"], nc, out)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert rel(got, want) <= 1e-5, (call, rel(got, want))


@pytest.mark.parametrize("wdtype", [np.float32, np.float16])
def test_noalloc_matches_oracle_with_ignored_samples(wdtype):
    """FP32 and FP16 weights, with samples at -1 and at indices past the map (both ignored):
    two calls in a row against the oracle's FP64 binned map of the same data with those
    samples excluded.  Everything the entry point computes is FP64 from exactly widened
    inputs, so the maps agree to FP64 rounding amplified by the blocks' condition (<= 1e3 on
    kept pixels): 1e-9.  The pixel cut agrees away from the rcond threshold."""
    s = synth.config_iqu(64, 4, 1 << 14, 33, weight_dtype=wdtype)
    npix, n = s["npix"], len(s["pix"])
    rng = np.random.default_rng(7)
    pix = s["pix"].copy()
    pick = rng.choice(n, 3000, replace=False)
    pix[pick[:1000]] = -1
    pix[pick[1000:2000]] = npix + rng.integers(0, 5000, 1000)
    pix[pick[2000:]] = np.iinfo(np.int32).max
    ignored = (pix < 0) | (pix >= npix)
    psd = [np.ones(int(s["offsets"][c + 1] - s["offsets"][c]) // 2 + 1)
           for c in range(len(s["offsets"]) - 1)]
    prob = O.Problem(np.where(ignored, -1, pix), s["cos"], s["sin"], s["tod"], s["offsets"],
                     npix, 3, psd, np.ones(len(psd)), 1e-3)
    ref, _ = O.messenger_step(prob, np.zeros((npix, 3)), math.inf)
    near = np.abs(prob.rcond - 1e-3) <= 1e-9
    keep = prob.valid & ~near
    cut = ~prob.valid & ~near
    tpix = torch.from_numpy(pix).to(DEV)
    tc = torch.from_numpy(s["cos"]).to(DEV)
    ts = torch.from_numpy(s["sin"]).to(DEV)
    ttod = torch.from_numpy(s["tod"]).to(DEV)
    for call in range(2):
        out = torch.full((npix, 3), float("nan"), dtype=torch.float64, device=DEV)
        binding.binned_map_noalloc(tpix, tc, ts, ttod, npix, 3, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call
        assert rel(got[keep], ref[keep]) <= 1e-9, (call, rel(got[keep], ref[keep]))
        assert np.all(got[cut] == 0.0), call


def test_noalloc_rejects_too_many_pixels():
    pix = torch.zeros(1024, dtype=torch.int32, device=DEV)
    tod = torch.zeros(1024, dtype=torch.float32, device=DEV)
    out = torch.zeros((1 << 18) + 1, dtype=torch.float64, device=DEV)
    with pytest.raises(binding.MMError) as e:
        binding.binned_map_noalloc(pix, None, None, tod, (1 << 18) + 1, 1, out)
    assert e.value.code == binding.MM_ERR_ARG
    assert "262144" in str(e.value)
