"""GPU adjoint (mm_messenger_adjoint) against the FP64 adjoint oracle.

Tolerance: the FP32 adjoint may differ from the FP64 adjoint by <= 1e-3 relative (L2 over
dL/dd, and per parameter for dL/dtheta relative to the largest component of its chunk).
At the 256^2 IQU, 4 x 2^20 differentiation workload, where the oracle is slow, the data
gradient is checked by the adjoint identity <c, M e> = <M^T c, e> of the linear map
m_K = M d.
"""

import numpy as np
import pytest

import oracle.adjoint as A
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


def gpu_grads(s, lam, m_true, ckpt_every=3):
    plan = binding.plan_from_synth(s, DEV)
    nc = s["ncomp"]
    m0 = torch.zeros(s["npix"], nc, dtype=torch.float64, device=DEV)
    m = m0.clone()
    plan.messenger(m, lam)
    g = m - torch.as_tensor(m_true, device=DEV)
    gt = torch.empty(len(s["pix"]), dtype=torch.float32, device=DEV)
    gth = torch.empty(len(s["offsets"]) - 1, 3, dtype=torch.float64, device=DEV)
    plan.adjoint(lam, m0, g, gt, gth, ckpt_every=ckpt_every)
    torch.cuda.synchronize()
    return gt.cpu().numpy().astype(np.float64), gth.cpu().numpy(), plan


def check_theta(got, ref, tol=1e-3):
    for c in range(ref.shape[0]):
        scale = np.max(np.abs(ref[c]))
        assert np.max(np.abs(got[c] - ref[c])) <= tol * scale, (c, got[c], ref[c])


@pytest.mark.parametrize("cfg", ["iqu16", "t64"])
def test_adjoint_matches_fp64_oracle(cfg):
    if cfg == "iqu16":
        s = synth.config_iqu(16, 3, 1 << 12, 21)
    else:
        s = synth.config_temperature_64(seed=17050005)
    theta = np.array([[p[0], p[1], p[2]] for p in s["params"]])
    prob = A.build_problem(s, theta)
    lam = O.cooling_schedule(O.lambda_max(prob), 3, 2)
    m_true = s["m_true"] * prob.valid[:, None]
    dd_ref, dth_ref, _ = A.adjoint(s, theta, lam, m_true)
    dd, dth, _ = gpu_grads(s, lam, m_true)
    assert np.linalg.norm(dd - dd_ref) <= 1e-3 * np.linalg.norm(dd_ref)
    check_theta(dth, dth_ref)


def test_adjoint_checkpoint_spacing_invariant():
    s = synth.config_iqu(16, 2, 1 << 12, 22)
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 4, 3)
    m_true = s["m_true"] * prob.valid[:, None]
    a, ta, _ = gpu_grads(s, lam, m_true, ckpt_every=1)
    b, tb, _ = gpu_grads(s, lam, m_true, ckpt_every=10)
    assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
    assert np.max(np.abs(ta - tb)) <= 1e-6 * np.max(np.abs(ta))


def test_autograd_function_backward():
    s = synth.config_iqu(16, 2, 1 << 12, 23)
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 2, 2)
    m_true = torch.as_tensor(s["m_true"] * prob.valid[:, None], device=DEV)
    plan = binding.plan_from_synth(s, DEV)
    tod = plan.tod.clone().requires_grad_(True)
    theta = torch.as_tensor(s["params"][:, :3].copy(), device=DEV).requires_grad_(True)
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    mK = binding.messenger_fn().apply(plan, lam, m0, tod, theta)
    loss = 0.5 * ((mK - m_true) ** 2).sum()
    loss.backward()
    dd, dth, _ = gpu_grads(s, lam, m_true.cpu().numpy())
    assert np.linalg.norm(tod.grad.cpu().numpy() - dd) <= 1e-6 * np.linalg.norm(dd)
    assert np.max(np.abs(theta.grad.cpu().numpy() - dth)) <= 1e-6 * np.max(np.abs(dth))


def test_data_gradient_without_theta_matches():
    """With grad_theta = NULL the backward runs no forward iterate (the transposed step does
    not depend on them): dL/dd must equal the one computed beside the theta terms."""
    s = synth.config_iqu(16, 2, 1 << 12, 24)
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 3, 3)
    m_true = s["m_true"] * prob.valid[:, None]
    dd, _, plan = gpu_grads(s, lam, m_true, ckpt_every=4)
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    m = m0.clone()
    plan.messenger(m, lam)
    g = m - torch.as_tensor(m_true, device=DEV)
    gt = torch.empty(len(s["pix"]), dtype=torch.float32, device=DEV)
    plan.adjoint(lam, m0, g, gt, None, ckpt_every=4)
    torch.cuda.synchronize()
    d2 = gt.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(d2 - dd) <= 1e-6 * np.linalg.norm(dd)


def test_forward_ckpt_then_backward_matches_all_in_one():
    """mm_messenger_forward_ckpt + mm_messenger_adjoint_ckpt against mm_messenger_adjoint:
    the same final map and the same gradients (checkpoint spacing 4 over 11 iterations, so
    the last segment is short)."""
    s = synth.config_iqu(16, 2, 1 << 12, 25)
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 2, 5)
    assert len(lam) == 11
    m_true = s["m_true"] * prob.valid[:, None]
    dd, dth, plan = gpu_grads(s, lam, m_true, ckpt_every=4)
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    m_ref = m0.clone()
    plan.messenger(m_ref, lam)
    m = m0.clone()
    ckpt = plan.forward_ckpt(m, lam, 4)
    assert ckpt.shape == (3, s["npix"], 3)
    torch.cuda.synchronize()
    assert torch.equal(m, m_ref)
    assert torch.equal(ckpt[0], m0)
    g = m - torch.as_tensor(m_true, device=DEV)
    gt = torch.empty(len(s["pix"]), dtype=torch.float32, device=DEV)
    gth = torch.empty(len(s["offsets"]) - 1, 3, dtype=torch.float64, device=DEV)
    plan.adjoint_ckpt(lam, ckpt, g, gt, gth, ckpt_every=4)
    torch.cuda.synchronize()
    assert np.linalg.norm(gt.cpu().numpy() - dd) <= 1e-7 * np.linalg.norm(dd)
    assert np.max(np.abs(gth.cpu().numpy() - dth)) <= 1e-7 * np.max(np.abs(dth))


def test_autograd_function_data_gradient_only():
    """theta without requires_grad: the autograd backward takes the path without forward
    iterates and gives the same dL/dd."""
    s = synth.config_iqu(16, 2, 1 << 12, 23)
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 2, 2)
    m_true = torch.as_tensor(s["m_true"] * prob.valid[:, None], device=DEV)
    plan = binding.plan_from_synth(s, DEV)
    tod = plan.tod.clone().requires_grad_(True)
    theta = torch.as_tensor(s["params"][:, :3].copy(), device=DEV)
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    mK = binding.messenger_fn().apply(plan, lam, m0, tod, theta)
    loss = 0.5 * ((mK - m_true) ** 2).sum()
    loss.backward()
    assert theta.grad is None
    dd, _, _ = gpu_grads(s, lam, m_true.cpu().numpy())
    assert np.linalg.norm(tod.grad.cpu().numpy() - dd) <= 1e-6 * np.linalg.norm(dd)


@pytest.mark.slow
def test_adjoint_full_size_dot_product():
    """256^2 IQU, 4 detectors x 2^20 samples, 20 cooled iterations, checkpoint every 10:
    the forward is linear in the data (m_K = M d from m_0 = 0), so for any map c and data
    e the adjoint must satisfy <c, M e> = <M^T c, e>.  Run the forward on random data e
    and the adjoint from gbar = c."""
    s = synth.config_iqu_256()
    rng = np.random.default_rng(9)
    s = dict(s)
    s["tod"] = rng.standard_normal(len(s["pix"])).astype(np.float32)   # e
    plan = binding.plan_from_synth(s, DEV)
    lam = binding.cooling_schedule(plan.lambda_max(), 4, 5)[:20]
    valid = torch.empty(s["npix"], dtype=torch.uint8, device=DEV)
    plan.maps(valid=valid)
    c = torch.as_tensor(rng.standard_normal((s["npix"], 3)), device=DEV) * valid[:, None].double()
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    m = m0.clone()
    plan.messenger(m, lam)
    gt = torch.empty(len(s["pix"]), dtype=torch.float32, device=DEV)
    plan.adjoint(lam, m0, c, gt, None, ckpt_every=10)
    torch.cuda.synchronize()
    lhs = float((c * m).sum())
    rhs = float(gt.double().cpu().numpy() @ s["tod"].astype(np.float64))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs), (lhs, rhs)
