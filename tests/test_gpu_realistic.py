"""GPU parity at the sizes of the differentiation workload (256^2 IQU, 4 detectors x 2^20
samples) and of the large single-GPU run's chunks (2^24-sample FP16-weight chunks on the
2048^2 IQU map), element by element against the FP64 oracle.  The oracle takes minutes at
these sizes, so the tests are marked slow; they are not gated.

Tolerances are those of the smaller parity tests: final map relative rms <= 1e-4 after 101
cooled iterations and chi^2 of every iteration <= 1e-5 relative; one messenger step <= 1e-5
relative L2; the FP32 adjoint within 1e-3 of the FP64 adjoint (L2 over dL/dd, per chunk
relative to its largest component for dL/dtheta); integer work bit-exact.
"""
import math

import numpy as np
import pytest

import oracle.adjoint as A
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


def test_differentiation_workload_101_cooled_iterations():
    """256^2 IQU, 4 x 2^20 samples: one lambda = inf step and 10 levels x 10 iterations."""
    s = synth.config_iqu_256()
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 10, 10)
    m_ref, chi_ref = O.run_messenger(prob, lam)
    plan = binding.plan_from_synth(s, DEV)
    m = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    chi = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
    plan.messenger(m, lam, chi)
    torch.cuda.synchronize()
    got, c = m.cpu().numpy(), chi.cpu().numpy()
    rms = np.sqrt(np.mean((got - m_ref) ** 2)) / np.sqrt(np.mean(m_ref ** 2))
    assert rms <= 1e-4, rms
    assert np.max(np.abs(c - chi_ref) / chi_ref) <= 1e-5, np.max(np.abs(c - chi_ref) / chi_ref)


def test_differentiation_workload_pcg_and_map_sized_form():
    """256^2 IQU, 4 x 2^20 samples: the comparison solver (PCG with the 3x3 block-Jacobi
    preconditioner, 30 iterations from m = 0) against the FP64 PCG oracle, and 20 cooled
    iterations of the map-sized form m' = m_d(lambda) + F(lambda) m (Sec. 2.1) against the
    oracle's messenger iterates.  PCG: iterate <= 1e-4 relative L2 and chi^2 of every
    iterate <= 1e-5 (the tolerances of the small-size PCG test; measured 2.8e-5 and 1.1e-7);
    map-sized form: final map <= 1e-4 relative rms, chi^2 per iteration <= 1e-5 (measured
    3.6e-7 and 7.0e-7)."""
    s = synth.config_iqu_256()
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    x_ref, chi_ref = O.pcg(prob, 30)
    x = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    chi = torch.zeros(30, dtype=torch.float64, device=DEV)
    plan.pcg(x, 30, restart=True, chi2_out=chi)
    torch.cuda.synchronize()
    e_x = rel(x.cpu().numpy(), x_ref)
    e_c = float(np.max(np.abs(chi.cpu().numpy() - chi_ref) / chi_ref))
    assert e_x <= 1e-4, e_x
    assert e_c <= 1e-5, e_c
    lam = O.cooling_schedule(O.lambda_max(prob), 5, 4)
    m_ref, c_ref = O.run_messenger(prob, lam)
    m = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    cm = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
    plan.messenger_md(m, lam, cm)
    torch.cuda.synchronize()
    got = m.cpu().numpy()
    rms = np.sqrt(np.mean((got - m_ref) ** 2)) / np.sqrt(np.mean(m_ref ** 2))
    assert rms <= 1e-4, rms
    e_m = float(np.max(np.abs(cm.cpu().numpy() - c_ref) / c_ref))
    assert e_m <= 1e-5, e_m


def test_differentiation_workload_adjoint_k50():
    """The gradient of L = 1/2 |m_K - m_true|^2 through K = 50 cooled iterations (5 levels x
    10), checkpoints every 10, against the FP64 adjoint oracle on the same data: dL/dd and
    dL/dtheta for every chunk."""
    s = synth.config_iqu_256()
    theta = np.array([[p[0], p[1], p[2]] for p in s["params"]])
    prob = A.build_problem(s, theta)
    lam = O.cooling_schedule(O.lambda_max(prob), 5, 10)[:50]
    m_true = s["m_true"] * prob.valid[:, None]
    dd_ref, dth_ref, _ = A.adjoint(s, theta, lam, m_true)
    plan = binding.plan_from_synth(s, DEV)
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    m = m0.clone()
    plan.messenger(m, lam)
    g = m - torch.as_tensor(m_true, device=DEV)
    gt = torch.empty(len(s["pix"]), dtype=torch.float32, device=DEV)
    gth = torch.empty(len(s["offsets"]) - 1, 3, dtype=torch.float64, device=DEV)
    plan.adjoint(lam, m0, g, gt, gth, ckpt_every=10)
    torch.cuda.synchronize()
    dd = gt.cpu().numpy().astype(np.float64)
    dth = gth.cpu().numpy()
    assert rel(dd, dd_ref) <= 1e-3, rel(dd, dd_ref)
    for c in range(dth_ref.shape[0]):
        scale = np.max(np.abs(dth_ref[c]))
        assert np.max(np.abs(dth[c] - dth_ref[c])) <= 1e-3 * scale, (c, dth[c], dth_ref[c])


def test_large_run_chunks_four_detectors():
    """The large run's chunk shape at a size the oracle finishes: 4 detectors x 2^24 samples
    (one per raster angle, 0/45/90/135 degrees) on the 2048^2 IQU map with FP16 weights.
    Hit counts bit-exact, the pixel cut identical away from the threshold, and three
    messenger steps (lambda = inf, lambda_max, 3) from the binned map element by element."""
    s = synth.config_crosslinked(n_det=4)
    npix = s["npix"]
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    hits = torch.empty(npix, dtype=torch.int32, device=DEV)
    valid = torch.empty(npix, dtype=torch.uint8, device=DEV)
    plan.maps(hits, valid)
    torch.cuda.synchronize()
    assert np.array_equal(hits.cpu().numpy(), prob.hits)
    near = np.abs(prob.rcond - 1e-3) <= 1e-9
    assert np.array_equal(valid.cpu().numpy().astype(bool)[~near], prob.valid[~near])
    lm = O.lambda_max(prob)
    assert abs(plan.lambda_max() - lm) <= 1e-12 * lm
    m_ref = np.zeros((npix, 3))
    m = torch.zeros(npix, 3, dtype=torch.float64, device=DEV)
    chi = torch.zeros(1, dtype=torch.float64, device=DEV)
    for lam in (math.inf, lm, 3.0):
        m_ref, chi_ref = O.messenger_step(prob, m_ref, lam)
        plan.messenger(m, [lam], chi)
        torch.cuda.synchronize()
        got = m.cpu().numpy()
        assert rel(got, m_ref) <= 1e-5, (lam, rel(got, m_ref))
        assert abs(float(chi[0]) - chi_ref) <= 1e-5 * chi_ref, (lam, float(chi[0]), chi_ref)
        m = torch.as_tensor(m_ref, device=DEV).clone()   # each step from the oracle's map
