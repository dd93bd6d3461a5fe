"""The fused iteration kernel (one launch for the column, row and inverse column passes of a
batch of 2^22-sample chunks, its work items ordered by chunk and waiting on per-chunk
counters) against the three separate kernels of the stage API and against the FP64 oracle.

Tolerances: the fused and the separate kernels do the same FP32 arithmetic per tile and row
job; only the order of the FP64 pixel additions differs, so their maps agree to 1e-9
(a rare FP32 rounding of the gather copy may differ after that).  Against the oracle the
FP32 path keeps the 1e-5 map tolerance of the other one-step tests."""
import math

import numpy as np
import pytest

import oracle.messenger as O
from paper_1705_01893_gb300 import binding, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N22 = 1 << 22


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1705_01893_gb300 import build
    build.build()
    binding.load()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def stage_iterate(plan, m, lams):
    plan.stage(binding.MM_STAGE_LOAD, map_inout=m)
    for i, lam in enumerate(lams):
        for b in range(plan.n_batches()):
            plan.stage(binding.MM_STAGE_GATHER_FFT, b)
            plan.stage(binding.MM_STAGE_FILTER, b, lam)
            plan.stage(binding.MM_STAGE_IFFT_BIN, b)
        plan.stage(binding.MM_STAGE_MAP, map_inout=m if i == len(lams) - 1 else None)


@pytest.mark.parametrize("n_det", [1, 3, 5])
def test_fused_matches_separate_kernels(n_det):
    """1, 3 and 5 chunks: fewer chunks than the lag between the passes, and more."""
    s = synth.config_iqu(64, n_det, N22, 40 + n_det)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_batches() == 1 and plan.n_fused_batches() == 1
    lams = [math.inf, 300.0, 30.0, 3.0, 1.0]
    m_f = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    chi_f = torch.zeros(len(lams), dtype=torch.float64, device=DEV)
    plan.messenger(m_f, lams, chi2_out=chi_f)
    m_s = torch.zeros_like(m_f)
    stage_iterate(plan, m_s, lams)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    assert rel(m_f.cpu().numpy(), m_s.cpu().numpy()) <= 1e-9
    # chi^2 of each iteration's input map from the fused row jobs, against mm_chi2 of the
    # separate path's iterates
    m_c = torch.zeros_like(m_f)
    for i, lam in enumerate(lams):
        if i > 0:
            ref = plan.chi2(m_c).item()
            assert abs(chi_f[i].item() - ref) <= 1e-7 * ref, (i, chi_f[i].item(), ref)
        stage_iterate(plan, m_c, [lam])


@pytest.mark.parametrize("log_n,n_det", [(23, 2), (24, 1), (24, 3)])
def test_fused_long_chunks_match_separate_kernels(log_n, n_det):
    """Chunks of 2^23 and 2^24 samples (columns of 1024 and 2048 points in tiles of 8 and 4
    columns, rows of 4096) with FP16 weights: the fused launch against the three separate
    kernels, maps to 1e-9 and no fault flag, then the PCG operator's fused launch against
    the oracle's PCG.  PCG's step lengths amplify the FP32 operator error (about 3e-7 rms
    for a 2^23-point transform): its second iterate is compared at the 1e-4 tolerance of
    the long runs (measured 2.0e-5 for the 2^24-sample chunk)."""
    s = synth.config_iqu(64, n_det, 1 << log_n, 70 + log_n + n_det, weight_dtype=np.float16)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_batches() == 1 and plan.n_fused_batches() == 1
    lams = [math.inf, 1e4, 30.0, 1.0]
    m_f = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan.messenger(m_f, lams)
    m_s = torch.zeros_like(m_f)
    stage_iterate(plan, m_s, lams)
    m_g = torch.zeros_like(m_f)
    plan.messenger_graph(m_g, lams)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    assert rel(m_f.cpu().numpy(), m_s.cpu().numpy()) <= 1e-9
    assert rel(m_g.cpu().numpy(), m_s.cpu().numpy()) <= 1e-9
    if n_det == 1:
        prob = O.problem_from_synth(s)
        x = torch.zeros_like(m_f)
        plan.pcg(x, 2)
        torch.cuda.synchronize()
        x_ref, _ = O.pcg(prob, 2)
        assert rel(x.cpu().numpy(), x_ref) <= 1e-4


def test_fused_graph_and_repeated_launches():
    """The graph-replayed iteration (counters reset by each launch's last CTA) gives the
    iterate of the host-launched one, twice in a row."""
    s = synth.config_iqu(64, 2, N22, 46)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_fused_batches() == 1
    lams = np.array([math.inf] + [100.0] * 4 + [10.0] * 4 + [1.0] * 4)
    m1 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan.messenger(m1, lams)
    for _ in range(2):
        m2 = torch.zeros_like(m1)
        plan.messenger_graph(m2, lams)
        torch.cuda.synchronize()
        assert rel(m2.cpu().numpy(), m1.cpu().numpy()) <= 1e-9
    assert plan.fault_flags() == 0


def test_fused_one_step_against_oracle():
    """Two chunks of 2^22 samples, 32x32 IQU: the binned start and one cooled step."""
    s = synth.config_iqu(32, 2, N22, 47)
    prob = O.problem_from_synth(s)
    lams = [math.inf, O.lambda_max(prob)]
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_fused_batches() == 1
    m = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan.messenger(m, lams)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    m_ref, _ = O.run_messenger(prob, lams)
    assert rel(m.cpu().numpy(), m_ref) <= 1e-5


def test_fused_not_used_for_other_shapes():
    """Chunks of other lengths keep the three separate kernels."""
    s = synth.config_iqu(32, 2, 1 << 18, 48)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_fused_batches() == 0


def test_fused_pcg_operator_against_oracle():
    """PCG on a chunk of 2^22 samples runs its operator A p = P^T N^-1 P p as one fused
    launch per iteration (row jobs in the 1/N mode): 2 iterations against the FP64 PCG."""
    s = synth.config_iqu(16, 1, N22, 49)
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_fused_batches() == 1
    x_ref, chi_ref = O.pcg(prob, 2)
    x = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    chi = torch.zeros(2, dtype=torch.float64, device=DEV)
    plan.pcg(x, 2, restart=True, chi2_out=chi)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    assert rel(x.cpu().numpy(), x_ref) <= 1e-5
    c = chi.cpu().numpy()
    assert np.max(np.abs(c - chi_ref) / chi_ref) <= 1e-5


def test_fused_map_sized_form_matches_step():
    """The map-sized form m' = m_d(lambda) + F(lambda) m (Sec. 2.1) with its F part as the
    fused launch (row jobs in the F mode) against the fused messenger step on the same plan
    (two chunks of 2^22 samples; same tolerances as the small-size map-sized test)."""
    s = synth.config_iqu(32, 2, N22, 50)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_fused_batches() == 1
    lam = binding.cooling_schedule(plan.lambda_max(), 3, 2)
    m0 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    a = m0.clone()
    ca = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
    plan.messenger_md(a, lam, ca)
    b = m0.clone()
    cb = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
    plan.messenger(b, lam, cb)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-5
    c_a, c_b = ca.cpu().numpy()[1:], cb.cpu().numpy()[1:]
    assert np.max(np.abs(c_a - c_b) / c_b) <= 1e-5


def test_fused_stage_matches_iterate_and_refuses_other_batches():
    """MM_STAGE_FUSED through the stage API gives mm_messenger_iterate's iterate; on a batch
    that is not fused it returns MM_ERR_UNSUPPORTED and launches nothing."""
    s = synth.config_iqu(32, 2, N22, 51)
    plan = binding.plan_from_synth(s, DEV)
    lams = [math.inf, 200.0, 20.0]
    m1 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan.messenger(m1, lams)
    m2 = torch.zeros_like(m1)
    plan.stage(binding.MM_STAGE_LOAD, map_inout=m2)
    for i, lam in enumerate(lams):
        for b in range(plan.n_batches()):
            plan.stage(binding.MM_STAGE_FUSED, b, lam)
        plan.stage(binding.MM_STAGE_MAP, map_inout=m2 if i == len(lams) - 1 else None)
    torch.cuda.synchronize()
    assert rel(m2.cpu().numpy(), m1.cpu().numpy()) <= 1e-9
    assert plan.fault_flags() == 0
    small = binding.plan_from_synth(synth.config_iqu(16, 2, 1 << 14, 52), DEV)
    with pytest.raises(binding.MMError) as e:
        small.stage(binding.MM_STAGE_FUSED, 0, 10.0)
    assert e.value.code == binding.MM_ERR_UNSUPPORTED


def test_fused_several_batches(monkeypatch):
    """A 16 MB intermediate budget puts each 2^22-sample chunk in its own batch: three fused
    launches per iteration, one after the other, against the single-batch plan."""
    s = synth.config_iqu(32, 3, N22, 53)
    lams = [math.inf, 100.0, 10.0, 1.0]
    plan1 = binding.plan_from_synth(s, DEV)
    assert plan1.n_batches() == 1
    m1 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan1.messenger(m1, lams)
    monkeypatch.setenv("MM_YBUF_MB", "16")
    plan3 = binding.plan_from_synth(s, DEV)
    assert plan3.n_batches() == 3 and plan3.n_fused_batches() == 3
    m3 = torch.zeros_like(m1)
    plan3.messenger(m3, lams)
    m4 = torch.zeros_like(m1)
    plan3.messenger_graph(m4, lams)
    torch.cuda.synchronize()
    assert plan3.fault_flags() == 0
    assert rel(m3.cpu().numpy(), m1.cpu().numpy()) <= 1e-9
    assert rel(m4.cpu().numpy(), m1.cpu().numpy()) <= 1e-9


def test_bounded_wait_runs_out_and_reports():
    """The fused kernel's bounded wait on a flag that nothing sets: it ends after its poll
    limit and reports expiry, the context stays usable; with the flag set it returns at
    once without a report."""
    assert binding.check_bounded_wait(2000, flag_set=False) is True
    assert binding.check_bounded_wait(2000, flag_set=True) is False
    x = torch.ones(1024, device=DEV)
    assert float((x * 2).sum()) == 2048.0


def test_solver_calls_report_an_expired_wait():
    """With a one-poll limit and check-on-return, the fused launch's first row jobs (taken
    at the start of the launch, beside the chunk's 256 column tiles, each of which takes
    microseconds) poll their chunk's counter once, give up and set the fault flag; the
    solver calls then synchronise and return MM_ERR_TIMEOUT.  A wait that gives up is a
    loop that ends, not a fault: with the default policy back, the same plan gives the
    correct iteration again."""
    s = synth.config_iqu(64, 1, N22, 61)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_fused_batches() == 1
    lams = [math.inf, 30.0]
    ref = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan.messenger(ref, lams)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    plan.set_wait_policy(1, True)
    m = torch.zeros_like(ref)
    calls = [lambda: plan.messenger(m, lams), lambda: plan.messenger_graph(m, lams),
             lambda: plan.pcg(m, 2)]
    for call in calls:
        with pytest.raises(binding.MMError) as e:
            call()
        assert e.value.code == binding.MM_ERR_TIMEOUT
        assert "bounded wait" in str(e.value)
    plan.set_wait_policy()
    m2 = torch.zeros_like(ref)
    plan.messenger(m2, lams)
    plan.messenger_graph(m, lams)
    torch.cuda.synchronize()
    assert plan.fault_flags() == 0
    assert rel(m2.cpu().numpy(), ref.cpu().numpy()) <= 1e-9
    assert rel(m.cpu().numpy(), ref.cpu().numpy()) <= 1e-9
