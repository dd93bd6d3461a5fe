"""The allocation-free binned map (mm_binned_map_noalloc) against the planned path.

Some callers cannot allocate device memory -- work recorded into a CUDA graph, code under an
allocator that must not grow, or a host that only receives device pointers -- yet need the
binned map (P^T P)^-1 P^T d.  The entry point keeps its accumulators in a fixed device
array.  Its map must equal the lambda = infinity messenger step of a plan built on the same
data (tau = sigma^2 = 1, so the map step weights are (P^T P)^-1), call after call.  This file
is named to be collected last, so a run that stops at the first failure has run every other
test first.
"""
import math

import numpy as np
import pytest

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


def test_noalloc_rejects_too_many_pixels():
    pix = torch.zeros(1024, dtype=torch.int32, device=DEV)
    tod = torch.zeros(1024, dtype=torch.float32, device=DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    with pytest.raises(binding.MMError) as e:
        binding.binned_map_noalloc(pix, None, None, tod, (1 << 18) + 1, 1, out)
    assert e.value.code == binding.MM_ERR_ARG
    assert "262144" in str(e.value)
