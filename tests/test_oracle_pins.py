"""Pins of the FP64 oracle to facts the paper and the mathematics fix (CPU only).

None of these expected values comes from the CUDA path.  Each pin is chosen so that a
plausible slip in the oracle (a dropped term, a wrong sign, a swapped weight, a missing
normalisation) breaks at least one of them; ``test_planted_mistakes`` proves that for a
list of such slips.
"""
import numpy as np
import pytest

import oracle.messenger as O
from paper_1705_01893_gb300 import synth


def tiny(seed=11, noiseless=False, width=8, ndet=2, n=512):
    return synth.config_iqu(width, ndet, n, seed, noiseless=noiseless)


def exact_signal(s, m=None):
    """d = P m written out in float64 straight from Eq. 1 (independent of the oracle)."""
    m = s["m_true"] if m is None else m
    pix = s["pix"].astype(np.int64)
    d = m[pix, 0].copy()
    if s["ncomp"] == 3:
        d += m[pix, 1] * s["cos"].astype(np.float64) + m[pix, 2] * s["sin"].astype(np.float64)
    return d


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# --------------------------------------------------------------------------- pins
def pin_fourier_chi2(prob, rng):
    """chi^2 summed over Fourier modes (Sec. 3.1) equals the explicit quadratic form
    (d - Pm)^T N'^-1 (d - Pm) with a dense circulant N' (Eq. 3), at lambda = 1 and 7."""
    m = rng.standard_normal((prob.npix, prob.ncomp))
    for lam in (1.0, 7.0):
        a = O.chi2(prob, m, lam)
        b = O.dense_chi2(prob, m, lam)
        assert abs(a - b) <= 1e-10 * abs(b), (lam, a, b)


def pin_white_noise(s):
    """White noise (Nbar = 0): t = d, so one iteration from any start is the binned map,
    which is then the exact GLS solution (Sec. 2.1 with T = N)."""
    off = s["offsets"]
    psd = [np.full(int(off[c + 1] - off[c]) // 2 + 1, 2.0) for c in range(len(off) - 1)]
    prob = O.problem_from_synth(s, psd=psd, tau=np.full(len(off) - 1, 2.0))
    m_any = np.random.default_rng(3).standard_normal((prob.npix, prob.ncomp))
    m1, _ = O.messenger_step(prob, m_any, 1.0)
    ref = O.dense_solve(prob)
    assert rel(m1, ref) < 1e-12


def pin_noiseless(s):
    """Noiseless d = P m_true: the binned map recovers m_true on valid pixels and m_true is
    a fixed point of the iteration at any lambda (unbiasedness, Sec. 2.1)."""
    prob = O.problem_from_synth(s)
    v = prob.valid
    mt = s["m_true"] * v[:, None]          # cut pixels carry no signal in this pin
    prob.tod = exact_signal(s, mt)
    prob.dtilde = [np.fft.rfft(prob.tod[a:b]) for a, b in prob.chunks()]
    mb, _ = O.messenger_step(prob, np.zeros_like(mt), np.inf)
    assert np.max(np.abs(mb - mt)) < 1e-12
    for lam in (1.0, 30.0):
        m1, x2 = O.messenger_step(prob, mt, lam)
        assert np.max(np.abs(m1 - mt)) < 1e-12
        assert x2 < 1e-20


def pin_gls_convergence(prob):
    """lambda = 1 iterations converge to the brute-force dense GLS solution (Eq. 2)."""
    ref = O.dense_solve(prob)
    m, ch = O.run_messenger(prob, np.r_[np.inf, np.ones(300)])
    assert rel(m, ref) < 1e-8
    assert abs(ch[-1] - O.chi2(prob, ref)) < 1e-9 * ch[-1]


def pin_fixed_lambda(prob, lam=5.0):
    """Fixed-lambda iterations converge to m(lambda) with N' = N + (lambda - 1) T
    (Sec. 2.1), and chi^2(m_i, lambda) never increases (App. A: each half-step minimises
    the augmented chi^2_1, whose minimum over t is chi^2(m, lambda))."""
    ref = O.dense_solve(prob, lam)
    m = np.zeros((prob.npix, prob.ncomp))
    m, _ = O.messenger_step(prob, m, np.inf)
    vals = []
    for _ in range(200):
        vals.append(O.chi2(prob, m, lam))
        m, _ = O.messenger_step(prob, m, lam)
    assert rel(m, ref) < 1e-8
    d = np.diff(vals)
    assert np.all(d <= 1e-10 * abs(vals[0])), d.max()


def pin_pcg(prob):
    """PCG converges to the same dense solution; messenger and PCG end points agree."""
    ref = O.dense_solve(prob)
    x, ch = O.pcg(prob, 80)
    assert rel(x, ref) < 1e-10
    assert np.all(np.diff(ch[:20]) <= 1e-9 * ch[0])


def explicit_pointing(prob, a, b):
    """Pointing rows of samples a..b as a dense [n, npix * ncomp] matrix, written straight
    from Eq. 1 (weights 1, cos 2psi, sin 2psi; excluded and cut pixels give zero rows)."""
    nc = prob.ncomp
    Pm = np.zeros((b - a, prob.npix * nc))
    for s in range(a, b):
        p = int(prob.pix[s])
        if p < 0 or not prob.valid[p]:
            continue
        Pm[s - a, p * nc] = 1.0
        if nc == 3:
            Pm[s - a, p * nc + 1] = prob.cos[s]
            Pm[s - a, p * nc + 2] = prob.sin[s]
    return Pm


def explicit_Ninv(psd_rfft, n):
    """N^-1 of a stationary chunk as F^H diag(1 / N_k) F / n with the n x n DFT matrix F
    and N_k on all n frequencies (N_k = N_{n-k})."""
    k = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(k, k) / n)
    full = psd_rfft[np.minimum(k, n - k)]
    return (F.conj().T @ (F / full[:, None])).real / n


def pin_jacobi(prob):
    """The comparison PCG's preconditioner (the paper's "diagonal preconditioner", read as
    pixel blocks): jacobi_blocks holds, on every kept pixel, the inverse of that pixel's
    ncomp x ncomp block of P^T diag(N^-1) P, where diag(N^-1) is the diagonal of the
    explicit N^-1 = F^H diag(1/N_k) F / n of each chunk; cut and unobserved pixels hold 0.
    With white noise N^-1 is itself diagonal, and the blocks are then exactly the diagonal
    pixel blocks of A = P^T N^-1 P (checked on a white-noise copy of the problem)."""
    nc = prob.ncomp
    for white in (False, True):
        if white:
            psd = [np.full_like(p, 2.5) for p in prob.psd]
            q = O.Problem(prob.pix, prob.cos, prob.sin, prob.tod, prob.offsets, prob.npix, nc,
                          psd, prob.tau, prob.rcond_min)
        else:
            q = prob
        Minv = O.jacobi_blocks(q)
        D = np.zeros((q.npix * nc, q.npix * nc))
        A = np.zeros_like(D)
        for c, (a, b) in enumerate(q.chunks()):
            Pc = explicit_pointing(q, a, b)
            Ni = explicit_Ninv(q.psd[c], b - a)
            D += Pc.T @ (np.diag(Ni)[:, None] * Pc)
            A += Pc.T @ Ni @ Pc
        for p in range(q.npix):
            sl = slice(p * nc, (p + 1) * nc)
            if not q.valid[p]:
                assert np.all(Minv[p] == 0)
                continue
            assert np.allclose(Minv[p] @ D[sl, sl], np.eye(nc), rtol=0, atol=1e-10), p
            if white:
                assert np.allclose(Minv[p] @ A[sl, sl], np.eye(nc), rtol=0, atol=1e-10), p


ALL_PINS = ["fourier_chi2", "white_noise", "noiseless", "gls", "fixed_lambda", "pcg", "jacobi"]


def run_pin(name):
    s = tiny()
    if name == "fourier_chi2":
        pin_fourier_chi2(O.problem_from_synth(s), np.random.default_rng(5))
    elif name == "white_noise":
        pin_white_noise(s)
    elif name == "noiseless":
        pin_noiseless(tiny(noiseless=True))
    elif name == "gls":
        pin_gls_convergence(O.problem_from_synth(s))
    elif name == "fixed_lambda":
        pin_fixed_lambda(O.problem_from_synth(s))
    elif name == "pcg":
        pin_pcg(O.problem_from_synth(s))
    elif name == "jacobi":
        pin_jacobi(O.problem_from_synth(tiny(width=4, n=256)))


@pytest.mark.parametrize("name", ALL_PINS)
def test_pin(name):
    run_pin(name)


# ----------------------------------------------------------------- further pins
def test_hits_closed_form_temperature_raster():
    """64 horizontal + 64 vertical sweeps at 4 samples/pixel: exactly 8 hits per pixel."""
    s = synth.config_temperature_64()
    prob = O.problem_from_synth(s)
    assert prob.hits.dtype.kind == "i"
    assert np.all(prob.hits == 8)
    assert np.all(prob.valid)


def test_temperature_binned_map_noiseless():
    """T-only, noiseless: the binned map is the per-pixel mean of the samples = m_true."""
    s = synth.config_temperature_64(noiseless=True)
    prob = O.problem_from_synth(s)
    prob.tod = exact_signal(s)
    prob.dtilde = [np.fft.rfft(prob.tod[a:b]) for a, b in prob.chunks()]
    mb, _ = O.messenger_step(prob, np.zeros((prob.npix, 1)), np.inf)
    assert np.max(np.abs(mb - s["m_true"])) < 1e-12


def test_large_lambda_forgets_start():
    """For very large lambda, F = 0: the next map does not depend on m_i (Sec. 2.1)."""
    prob = O.problem_from_synth(tiny())
    rng = np.random.default_rng(1)
    a, _ = O.messenger_step(prob, rng.standard_normal((prob.npix, 3)), 1e14)
    b, _ = O.messenger_step(prob, rng.standard_normal((prob.npix, 3)), 1e14)
    c, _ = O.messenger_step(prob, np.zeros((prob.npix, 3)), np.inf)
    assert rel(a, c) < 1e-9 and rel(b, c) < 1e-9


def test_spectral_radius_below_one():
    """The error propagator F(lambda) has spectral radius < 1 on the observed pixels
    (Sec. 2.1), and one messenger step equals m_d + F m_i."""
    prob = O.problem_from_synth(tiny())
    for lam in (1.0, 10.0):
        F = O.dense_F(prob, lam)
        rho = np.max(np.abs(np.linalg.eigvals(F)))
        assert rho < 1.0
        idx = np.flatnonzero(prob.valid)
        m = np.zeros((prob.npix, 3))
        m[idx] = np.random.default_rng(2).standard_normal((idx.size, 3))
        md, _ = O.messenger_step(prob, np.zeros_like(m), lam)
        m1, _ = O.messenger_step(prob, m, lam)
        assert rel(m1[idx].ravel(), md[idx].ravel() + F @ m[idx].ravel()) < 1e-10


def test_heterogeneous_tau_same_solution():
    """Any admissible T (here tau_c = 0.5 sigma_c^2 per chunk, Sec. 4.2) leaves the fixed
    point unchanged: lambda = 1 iterations still reach the GLS solution."""
    s = tiny()
    prob = O.problem_from_synth(s, tau=np.array([0.5, 0.8]))
    ref = O.dense_solve(prob)
    m, _ = O.run_messenger(prob, np.r_[np.inf, np.ones(400)])
    assert rel(m, ref) < 1e-7


def test_unbiased_over_noise_seeds():
    """<m_i> = m_true for every iterate (Sec. 2.1): the mean over 256 noise draws is within
    5 standard errors of m_true on every kept map component.  5 rather than 4: the maximum
    is taken over all components (768 here), and at 4 a correct solver would still fail
    about one draw set in twenty; 256 draws resolve a bias of sigma/16 per component."""
    base = tiny(seed=100)
    v = O.problem_from_synth(base).valid
    mt = base["m_true"] * v[:, None]        # no signal on cut pixels (their rows are zero)
    maps = []
    for k in range(256):
        s = tiny(seed=100 + k)
        s["tod"] = (exact_signal(base, mt) + (s["tod"] - exact_signal(s))).astype(np.float32)
        prob = O.problem_from_synth(s)
        m, _ = O.run_messenger(prob, O.cooling_schedule(O.lambda_max(prob), 3, 3))
        maps.append(m)
    maps = np.array(maps)
    mean = maps.mean(0)[v]
    err = maps.std(0)[v] / np.sqrt(len(maps))
    z = np.abs(mean - base["m_true"][v]) / err
    assert np.max(z) < 5.0


@pytest.mark.parametrize("n", [1000, 999, 1875, 2])
def test_rfft_convention_round_trip(n):
    """The oracle's spectrum convention: Parseval with multiplicity weights (no Nyquist bin
    for odd n), and round trip."""
    x = np.random.default_rng(n).standard_normal(n)
    X = np.fft.rfft(x)
    assert abs(np.sum(O.rfft_weights(n) * np.abs(X) ** 2) / n - x @ x) < 1e-9 * (x @ x)
    assert np.allclose(np.fft.irfft(X, n), x)


def test_noise_model_values():
    """The model PSD at hand-evaluated points: n = 8 samples at fs = 8 Hz puts bin k at k Hz;
    sigma = 2, f_knee = 1 Hz, alpha = 2 gives N(1) = 4 (1 + 1) = 8, N(2) = 4 (1 + 1/4) = 5,
    N(3) = 4 (1 + 1/9), N(4) = 4 (1 + 1/16) = 4.25, and the DC bin takes bin 1's 8."""
    N = O.psd_from_params(8, 8.0, 2.0, 1.0, 2.0)
    assert np.allclose(N, [8.0, 8.0, 5.0, 4.0 + 4.0 / 9.0, 4.25], rtol=1e-15, atol=0)
    # odd length: bins k = 0..3 of n = 7 at fs = 7 Hz, f_knee = 2 Hz, alpha = 1
    N = O.psd_from_params(7, 7.0, 1.0, 2.0, 1.0)
    assert np.allclose(N, [3.0, 3.0, 2.0, 1.0 + 2.0 / 3.0], rtol=1e-15, atol=0)


def test_schedule_shape():
    lam = O.cooling_schedule(1e4, 10, 10)
    assert lam.size == 101 and np.isinf(lam[0])
    assert lam[1] == pytest.approx(1e4) and lam[-1] == 1.0
    assert np.all(np.diff(lam[1:]) <= 0)


# ------------------------------------------------------------- planted mistakes
def _plant(monkeypatch, which):
    if which == "drop_lambda":
        orig = O.messenger_step

        def bad(prob, m, lam):
            return orig(prob, m, 1.0 if np.isfinite(lam) else lam)
        monkeypatch.setattr(O, "messenger_step", bad)
    elif which == "swap_qu":
        orig = O.Problem.weights

        def bad(self, a, b):
            w = orig(self, a, b)
            return w[:, [0, 2, 1]] if w.shape[1] == 3 else w
        monkeypatch.setattr(O.Problem, "weights", bad)
    elif which == "filter_sign":
        def bad(prob, m, lam):
            acc = np.zeros((prob.npix, prob.ncomp))
            for c, (a, b) in enumerate(prob.chunks()):
                n = b - a
                r = np.fft.rfft(prob.P(m, a, b))
                lt = lam * prob.tau[c] if np.isfinite(lam) else np.inf
                tt = prob.dtilde[c] if np.isinf(lt) else (lt * prob.dtilde[c] - prob.nbar(c) * r) / (lt + prob.nbar(c))
                acc += prob.PT(np.fft.irfft(tt, n), a, b) / prob.tau[c]
            return prob.bin(acc), 0.0
        monkeypatch.setattr(O, "messenger_step", bad)
    elif which == "chi2_no_mult":
        monkeypatch.setattr(O, "rfft_weights", lambda n: np.ones(n // 2 + 1))
    elif which == "nbar_is_n":
        monkeypatch.setattr(O.Problem, "nbar", lambda self, c: self.psd[c])
    elif which == "pcg_no_precond_update":
        orig = O.jacobi_blocks
        monkeypatch.setattr(O, "jacobi_blocks", lambda prob: 2.0 * orig(prob) + 1e-3)
    elif which == "jacobi_no_multiplicity":
        # c0 without the rfft multiplicities (the mean of 1/N over the rfft bins only)
        def bad(prob):
            nc = prob.ncomp
            M = np.zeros((prob.npix, nc, nc))
            for c, (a, b) in enumerate(prob.chunks()):
                c0 = np.mean(1.0 / prob.psd[c])
                pix = prob.pix[a:b]
                good = pix >= 0
                w = prob.weights(a, b)[good]
                np.add.at(M, pix[good], c0 * w[:, :, None] * w[:, None, :])
            Minv = np.zeros_like(M)
            Minv[prob.valid] = np.linalg.inv(M[prob.valid])
            return Minv
        monkeypatch.setattr(O, "jacobi_blocks", bad)
    elif which == "transposed_block":
        orig = O.Problem.bin

        def bad(self, acc):
            return np.einsum("pji,pj->pi", self.W + np.triu(np.ones(3), 1)[None] * 1e-2, acc) \
                if self.ncomp == 3 else orig(self, acc)
        monkeypatch.setattr(O.Problem, "bin", bad)


@pytest.mark.parametrize("which", ["drop_lambda", "swap_qu", "filter_sign", "chi2_no_mult",
                                   "nbar_is_n", "transposed_block", "pcg_no_precond_update",
                                   "jacobi_no_multiplicity"])
def test_planted_mistakes(monkeypatch, which):
    """Each planted slip in the oracle must break at least one pin."""
    _plant(monkeypatch, which)
    failures = 0
    for name in ALL_PINS:
        try:
            run_pin(name)
        except (AssertionError, np.linalg.LinAlgError, FloatingPointError):
            failures += 1
    assert failures >= 1, which


def test_chi2_modes_sum_and_unit_mean():
    """Per-mode chi^2 (Sec. 3.1): its multiplicity-weighted sum is chi^2, and for data that
    are pure noise around the true map each mode has unit mean (a chi^2 of 2 degrees of
    freedom rescaled to unit mean)."""
    s = synth.config_iqu(16, 2, 1 << 14, 41)
    prob = O.problem_from_synth(s)
    m = s["m_true"] * prob.valid[:, None]
    modes = O.chi2_modes(prob, m)
    tot = sum(np.sum(O.rfft_weights(len(md) * 2 - 2) * md) for md in modes)
    assert abs(tot - O.chi2(prob, m)) <= 1e-10 * tot
    allm = np.concatenate([md[1:-1] for md in modes])
    assert abs(allm.mean() - 1.0) < 0.05


def test_synth_uneven_and_angled_rasters():
    """Inputs of the uneven-chunk workload: lengths 2-3-5-smooth in range, pixel indices in
    range or -1, an axis-aligned raster reproduces the horizontal sweep pixel by pixel."""
    n = synth.smooth235_lengths(2 ** 16, 2 ** 20)
    assert len(n) == 228 and n[0] == 2 ** 16 and n[-1] == 2 ** 20
    for v in n[:40]:
        x = int(v)
        for f in (2, 3, 5):
            while x % f == 0:
                x //= f
        assert x == 1
    s = synth.config_uneven(32, 5, 2000, 12000, seed=3)
    lens = np.diff(s["offsets"])
    assert np.all((lens >= 2000) & (lens <= 12000))
    assert s["pix"].min() >= -1 and s["pix"].max() < 32 * 32
    p = synth.raster_angled(8, 2, 32, 0.0, 4)
    assert np.array_equal(p[:16], 8 * 4 + np.arange(16) // 2)        # row 4, left to right
    assert np.array_equal(p[16:32], 8 * 4 + 7 - np.arange(16) // 2)  # back, right to left


def test_adaptive_cooling_bookkeeping_and_target():
    """Plateau-driven cooling (Sec. 3.1).  With no plateau ever detected it is exactly the
    fixed schedule (one lambda = inf step, max_per_level iterations per level, the last level
    until max_iter); with every test a plateau each level runs min_per_level = 2 iterations;
    with a small tolerance it ends within 1e-6 of the brute-force GLS chi^2 (Eq. 2)."""
    prob = O.problem_from_synth(tiny(seed=31))
    lm = O.lambda_max(prob)
    L, k = 5, 3
    levels = [lm ** ((L - 1 - j) / (L - 1)) for j in range(L)]
    fixed = O.cooling_schedule(lm, L, k)
    m_a, chi_a, lam_a = O.run_messenger_adaptive(prob, levels, -np.inf, 2, k, len(fixed))
    m_f, chi_f = O.run_messenger(prob, fixed)
    assert np.array_equal(lam_a, fixed)
    assert np.array_equal(m_a, m_f) and np.array_equal(chi_a, chi_f)
    _, _, lam_b = O.run_messenger_adaptive(prob, levels, np.inf, 2, 50, 1000)
    assert np.array_equal(lam_b, [np.inf] + [l for l in levels for _ in range(2)])
    m_c, chi_c, lam_c = O.run_messenger_adaptive(prob, levels, 1e-9, 2, 200, 4000)
    assert lam_c[-1] == 1.0 and len(lam_c) < 4000
    ref = O.dense_solve(prob)
    c_ref = O.dense_chi2(prob, ref)
    assert (O.chi2(prob, m_c) - c_ref) / c_ref < 1e-6
    # every level change follows a measured decrease below the tolerance or the cap
    starts = [i for i in range(2, len(lam_c)) if lam_c[i] != lam_c[i - 1]]
    for s in starts:
        run = s - max(j for j in range(1, s) if lam_c[j] != lam_c[j - 1] or j == 1)
        rel = (chi_c[s - 2] - chi_c[s - 1]) / chi_c[s - 1]
        assert rel < 1e-9 or run >= 200
