"""GPU parity of the general path: chunk lengths whose prime factors are 2, 3 and 5 (not
powers of two, odd lengths included), transformed by the runtime mixed-radix kernels, many
lengths in one persistent launch per stage.  Same tolerances as the power-of-two path:
rfft <= 1e-6 relative L2, one messenger step <= 1e-5, 100 cooled iterations <= 1e-4 map
relative rms and <= 1e-5 chi^2, PCG <= 1e-4."""
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
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x)).to(DEV, dtype)


def t_only(lens, seed=3, first=0):
    """T-only problem with chunks of the given lengths (pixel 0 everywhere); `first` leading
    samples that belong to no chunk shift every chunk's offset."""
    pix = [np.zeros(n, dtype=np.int32) for n in lens]
    k = len(lens)
    s = synth.make_problem(4, 1, pix, 100.0, [1.0] * k, [1.0] * k, [2.0] * k, [0.0] * k, 0.0, seed)
    if first:
        s = dict(s)
        s["offsets"] = s["offsets"] + first
        s["pix"] = np.concatenate([np.zeros(first, np.int32), s["pix"]])
        s["tod"] = np.concatenate([np.zeros(first, np.float32), s["tod"]])
    return s


def rfft_check(s):
    plan = binding.plan_from_synth(s, DEV)
    off = s["offsets"]
    lens = np.diff(off)
    tot = int(sum(n // 2 + 1 for n in lens))
    spec = torch.empty(tot, 2, dtype=torch.float32, device=DEV)
    plan.rfft(to_dev(s["tod"], torch.float32), spec)
    got = spec.cpu().numpy().astype(np.float64)
    got = got[:, 0] + 1j * got[:, 1]
    o = 0
    for c, n in enumerate(lens):
        ref = np.fft.rfft(s["tod"][off[c]:off[c + 1]].astype(np.float64))
        e = rel(got[o:o + n // 2 + 1], ref)
        assert e <= 1e-6, (int(n), e)
        o += n // 2 + 1


@pytest.mark.parametrize("n", [4, 6, 18, 45, 243, 250, 256, 1000, 3125, 4374, 6000, 21600,
                               3 ** 9, 2 * 3 ** 10, 5 ** 7, 983040, 3 ** 12, 2 * 5 ** 8])
def test_rfft_general_lengths(n):
    """Even and odd lengths, radices 2..8, columns up to 512 and rows up to 4096."""
    rfft_check(t_only([n, n]))


def test_rfft_mixed_plan_and_unaligned_offsets():
    """Power-of-two and general chunks in one plan (the 2^21-sample chunk keeps the
    compile-time kernels); power-of-two chunks that do not start on a 16-byte boundary take
    the general path; a plan that starts at an odd offset."""
    rfft_check(t_only([1 << 21, 3375, 4096, 1024, 6250]))
    rfft_check(t_only([4096, 1536, 2048], first=3))


def test_small_power_of_two_chunks_join_the_general_batch():
    """In a plan with general chunks, a power-of-two length whose chunks hold at most 2^20
    samples in all runs in the general batch (one batch in all); a longer one keeps a
    compile-time batch of its own.  Without general chunks nothing changes.  One messenger
    step of the joined plan against the oracle."""
    # power-of-two chunks first, so that they start on 16-byte boundaries
    assert binding.plan_from_synth(t_only([1 << 14, 1 << 14, 1 << 16, 3375]), DEV).n_batches() == 1
    assert binding.plan_from_synth(t_only([1 << 16] * 17 + [3375]), DEV).n_batches() == 2
    assert binding.plan_from_synth(t_only([1 << 21, 3375]), DEV).n_batches() == 2
    assert binding.plan_from_synth(t_only([1 << 14, 1 << 16]), DEV).n_batches() == 2
    lens = [1 << 14, 1 << 16, 3375, 6250]
    chunks = [synth.raster_alternating(16, 2, n, k) for k, n in enumerate(lens)]
    s = synth.make_problem(16, 3, chunks, 100.0, [1.0, 1.2, 0.9, 1.1], [1.0, 0.5, 2.0, 0.3],
                           [2.0, 1.5, 1.0, 2.5], [0.0, 45.0, 90.0, 135.0], 0.5, 23)
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_batches() == 1
    m0 = np.random.default_rng(5).standard_normal((s["npix"], 3)) * prob.valid[:, None]
    m_ref, _ = O.messenger_step(prob, m0, 10.0)
    m = to_dev(m0)
    plan.messenger(m, [10.0])
    torch.cuda.synchronize()
    assert rel(m.cpu().numpy(), m_ref) <= 1e-5


def test_power_of_two_chunk_after_odd_spectrum_block():
    """A power-of-two chunk (compile-time kernels: its offset 4500 is a multiple of 4, and
    its 2^21 samples are too many to join the general batch) after two chunks of 2250
    samples, whose complex lengths 1125 sum to 2250 slots, then odd-length and power-of-two
    chunks on the general path: every chunk's block in the spectrum-sized buffers starts on
    a multiple of 4 slots, so the row jobs' bulk prefetches of d~ / Nbar rows stay 16-byte
    aligned.  rfft and one messenger step at lambda = 10 against the oracle."""
    lens = [2250, 2250, 1 << 21, 3375, 1 << 14]
    chunks = [synth.raster_alternating(16, 2, n, k) for k, n in enumerate(lens)]
    k = len(lens)
    s = synth.make_problem(16, 3, chunks, 100.0, [1.0, 1.2, 0.9, 1.1, 1.0][:k],
                           [1.0, 0.5, 2.0, 0.3, 0.7][:k], [2.0, 1.5, 1.0, 2.5, 2.0][:k],
                           [0.0, 30.0, 60.0, 90.0, 120.0][:k], 0.5, 21)
    rfft_check(s)
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    assert plan.n_batches() == 2          # the 2^21-sample chunk has a batch of its own
    m0 = np.random.default_rng(2).standard_normal((s["npix"], 3)) * prob.valid[:, None]
    m_ref, _ = O.messenger_step(prob, m0, 10.0)
    m = to_dev(m0)
    plan.messenger(m, [10.0])
    torch.cuda.synchronize()
    assert rel(m.cpu().numpy(), m_ref) <= 1e-5


@pytest.fixture(scope="module")
def uneven():
    s = synth.config_uneven(32, 5, 2000, 12000, seed=17050112)
    assert any(n % 2 for n in np.diff(s["offsets"]))        # at least one odd chunk
    return s


def test_uneven_single_steps(uneven):
    s = uneven
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    lm = O.lambda_max(prob)
    assert abs(plan.lambda_max() - lm) <= 1e-12 * lm
    m0 = np.random.default_rng(4).standard_normal((s["npix"], 3)) * prob.valid[:, None]
    for lam in (math.inf, lm, 3.0, 1.0):
        m_ref, chi_ref = O.run_messenger(prob, [lam], m0)
        m = to_dev(m0)
        chi = torch.zeros(1, dtype=torch.float64, device=DEV)
        plan.messenger(m, [lam], chi)
        torch.cuda.synchronize()
        assert rel(m.cpu().numpy(), m_ref) <= 1e-5, lam
        assert abs(chi.item() - chi_ref[0]) <= 1e-5 * chi_ref[0]


def test_uneven_100_iterations_and_graph(uneven):
    s = uneven
    prob = O.problem_from_synth(s)
    lam = O.cooling_schedule(O.lambda_max(prob), 10, 10)
    m_ref, chi_ref = O.run_messenger(prob, lam)
    plan = binding.plan_from_synth(s, DEV)
    m = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    chi = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
    plan.messenger(m, lam, chi)
    g = torch.zeros_like(m)
    cg = torch.zeros_like(chi)
    plan.messenger_graph(g, lam, cg)
    torch.cuda.synchronize()
    m = m.cpu().numpy()
    rms = np.sqrt(np.mean((m - m_ref) ** 2)) / np.sqrt(np.mean(m_ref ** 2))
    assert rms <= 1e-4, rms
    assert np.max(np.abs(chi.cpu().numpy() - chi_ref) / chi_ref) <= 1e-5
    assert rel(g.cpu().numpy(), m) <= 1e-12
    assert np.max(np.abs(cg.cpu().numpy() - chi.cpu().numpy()) / chi_ref) <= 1e-12


def test_uneven_pcg_and_chi2(uneven):
    s = uneven
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    x_ref, chi_ref = O.pcg(prob, 30)
    x = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    chi = torch.zeros(30, dtype=torch.float64, device=DEV)
    plan.pcg(x, 30, restart=True, chi2_out=chi)
    torch.cuda.synchronize()
    assert rel(x.cpu().numpy(), x_ref) <= 1e-4
    assert np.max(np.abs(chi.cpu().numpy() - chi_ref) / chi_ref) <= 1e-5
    m = np.random.default_rng(5).standard_normal((s["npix"], 3)) * prob.valid[:, None]
    for lam in (1.0, 25.0):
        tot, modes = plan.chi2_modes(to_dev(m), lam)
        ref = np.concatenate(O.chi2_modes(prob, m, lam))
        assert rel(modes.cpu().numpy(), ref) <= 1e-5
        c_ref = O.chi2(prob, m, lam)
        assert abs(tot.item() - c_ref) <= 1e-5 * c_ref
        assert abs(plan.chi2(to_dev(m), lam).item() - c_ref) <= 1e-5 * c_ref


def test_uneven_batches_match(monkeypatch):
    """A small intermediate budget splits the general chunks over several batches (one
    launch per stage each); the stage entry point gives the iterate of one batch."""
    s = synth.config_uneven(32, 5, 100000, 300000, seed=17050112)
    prob = O.problem_from_synth(s)
    lam = [math.inf, O.lambda_max(prob), 2.0]
    plan1 = binding.plan_from_synth(s, DEV)
    assert plan1.n_batches() == 1
    m1 = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan1.messenger(m1, lam)
    monkeypatch.setenv("MM_YBUF_MB", "1")
    plan2 = binding.plan_from_synth(s, DEV)
    assert plan2.n_batches() >= 2
    m2 = torch.zeros_like(m1)
    plan2.stage(binding.MM_STAGE_LOAD, map_inout=m2)
    for i, l in enumerate(lam):
        for b in range(plan2.n_batches()):
            plan2.stage(binding.MM_STAGE_GATHER_FFT, b)
            plan2.stage(binding.MM_STAGE_FILTER, b, l)
            plan2.stage(binding.MM_STAGE_IFFT_BIN, b)
        plan2.stage(binding.MM_STAGE_MAP, map_inout=m2 if i == len(lam) - 1 else None)
    torch.cuda.synchronize()
    assert rel(m2.cpu().numpy(), m1.cpu().numpy()) <= 1e-12


def test_uneven_fp16_weights():
    s = synth.config_uneven(24, 4, 1500, 6000, seed=17050105)
    s = dict(s)
    s["cos"] = s["cos"].astype(np.float16)
    s["sin"] = s["sin"].astype(np.float16)
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    lam = [math.inf, 5.0, 1.0]
    m_ref, _ = O.run_messenger(prob, lam)
    m = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
    plan.messenger(m, lam)
    torch.cuda.synchronize()
    assert rel(m.cpu().numpy(), m_ref) <= 1e-5


def test_general_plans_refuse_adjoint_and_plain(uneven):
    plan = binding.plan_from_synth(uneven, DEV)
    m = torch.zeros(uneven["npix"], 3, dtype=torch.float64, device=DEV)
    with pytest.raises(binding.MMError) as e:
        plan.adjoint([2.0], m, m, torch.empty(len(uneven["pix"]), device=DEV))
    assert e.value.code == binding.MM_ERR_UNSUPPORTED
    with pytest.raises(binding.MMError) as e:
        plan.messenger_plain_fp64(m, [2.0])
    assert e.value.code == binding.MM_ERR_UNSUPPORTED


def test_unsupported_length_rejected():
    s = t_only([7 * 64])
    with pytest.raises(binding.MMError) as e:
        binding.plan_from_synth(s, DEV)
    assert e.value.code == binding.MM_ERR_UNSUPPORTED


@pytest.mark.slow
def test_uneven_full_size_one_step():
    """64 chunks of 2-3-5-smooth lengths in [2^16, 2^20] on a 1024^2 IQU map.

    From the binned map (the solver's own start, Sec. 3.1) at lambda = sqrt(lambda_max) and
    lambda = 3: <= 1e-5 like every other single step.  From the true sky at lambda = 3 the
    step's output is small next to the data, and the FP32 spectrum of the data sets the
    error: the data are dominated by 1/f noise (f_knee up to 3 Hz, alpha up to 3), so the
    FP32 FFT's absolute rounding error, ~u ||d~||, is large relative to the white-noise bins
    of the upper half of the spectrum (measured up to 8e-5 there), and those bins pass into
    t unfiltered where Nbar << lambda tau.  Bound used: 5e-5 (measured 2.5e-5; the same step
    with the GPU's own data spectrum given to the oracle agrees to 8e-7)."""
    s = synth.config_uneven()
    prob = O.problem_from_synth(s)
    plan = binding.plan_from_synth(s, DEV)
    hits = torch.empty(s["npix"], dtype=torch.int32, device=DEV)
    plan.maps(hits)
    torch.cuda.synchronize()
    assert np.array_equal(hits.cpu().numpy(), prob.hits)
    lm = O.lambda_max(prob)
    mb, _ = O.messenger_step(prob, np.zeros((s["npix"], 3)), math.inf)
    cases = [(mb, lm ** 0.5, 1e-5), (mb, 3.0, 1e-5), (s["m_true"] * prob.valid[:, None], 3.0, 5e-5)]
    for m0, lam, tol in cases:
        m_ref, chi_ref = O.messenger_step(prob, m0, lam)
        m = to_dev(m0)
        chi = torch.zeros(1, dtype=torch.float64, device=DEV)
        plan.messenger(m, [lam], chi)
        torch.cuda.synchronize()
        assert rel(m.cpu().numpy(), m_ref) <= tol, (lam, tol)
        assert abs(chi.item() - chi_ref) <= 1e-5 * chi_ref


def test_every_schedule_gives_the_same_iterate(uneven):
    """Each tile width, thread count and radix order of the general kernels (and the one the
    autotuner picks) reproduces the oracle's step; schedules differ only by FP32 rounding."""
    s = uneven
    prob = O.problem_from_synth(s)
    lam = [math.inf, O.lambda_max(prob) ** 0.5, 1.0]
    m_ref, chi_ref = O.run_messenger(prob, lam)
    plan = binding.plan_from_synth(s, DEV)
    outs = []
    for tune in [(8, 256, 256, 0), (16, 512, 1024, 1), (8, 512, 512, 2), (16, 256, 256, 2), None]:
        if tune is None:
            plan.autotune()
            assert plan.tune[0] in (8, 16) and plan.tune[3] in (0, 1, 2)
        else:
            plan.set_tune(*tune)
            assert plan.tune == tune
        m = torch.zeros(s["npix"], 3, dtype=torch.float64, device=DEV)
        chi = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
        plan.messenger(m, lam, chi)
        g = torch.zeros_like(m)
        plan.messenger_graph(g, lam)
        torch.cuda.synchronize()
        assert rel(m.cpu().numpy(), m_ref) <= 1e-5, tune
        assert np.max(np.abs(chi.cpu().numpy() - chi_ref) / chi_ref) <= 1e-5
        assert rel(g.cpu().numpy(), m.cpu().numpy()) <= 1e-12
        outs.append(m.cpu().numpy())
    for o in outs[1:]:
        assert rel(o, outs[0]) <= 1e-5
    with pytest.raises(binding.MMError):
        plan.set_tune(12, 256, 256, 0)
