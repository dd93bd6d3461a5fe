"""Pins of the FP64 adjoint oracle: central finite differences and a dense adjoint."""
import numpy as np
import pytest

import oracle.adjoint as A
import oracle.messenger as O
from paper_1705_01893_gb300 import synth


def setup(seed=3, width=8, ndet=2, n=1024):
    s = synth.config_iqu(width, ndet, n, seed)
    theta = np.array([[p[0], p[1], p[2]] for p in s["params"]])
    prob = A.build_problem(s, theta)
    lam = O.cooling_schedule(O.lambda_max(prob), 3, 2)
    m_true = s["m_true"] * prob.valid[:, None]
    return s, theta, lam, m_true


def test_adjoint_matches_dense_adjoint_in_d():
    """dL/dd by the transposed steps equals M^T (m_K - m_true) from explicit matrices."""
    s, theta, lam, m_true = setup()
    dd, _, _ = A.adjoint(s, theta, lam, m_true)
    ref = A.dense_d_gradient(s, theta, lam, m_true)
    assert np.linalg.norm(dd - ref) <= 1e-10 * np.linalg.norm(ref)


def test_adjoint_d_central_differences():
    """L is exactly quadratic in d, so a central difference along any direction is exact up
    to rounding."""
    s, theta, lam, m_true = setup(seed=4)
    dd, _, _ = A.adjoint(s, theta, lam, m_true)
    rng = np.random.default_rng(0)
    for _ in range(3):
        e = rng.standard_normal(dd.size)
        h = 1e-3
        Lp = A.loss(A.build_problem(s, theta, s["tod"].astype(np.float64) + h * e), lam, m_true)
        Lm = A.loss(A.build_problem(s, theta, s["tod"].astype(np.float64) - h * e), lam, m_true)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - dd @ e) <= 1e-8 * abs(fd)


@pytest.mark.parametrize("j", [0, 1, 2])
def test_adjoint_theta_central_differences(j):
    """dL/d(sigma, f_knee, alpha) of each chunk against central differences, step 1e-6
    relative (the lambda schedule held fixed)."""
    s, theta, lam, m_true = setup(seed=5)
    _, dth, _ = A.adjoint(s, theta, lam, m_true)
    for c in range(theta.shape[0]):
        h = 1e-6 * abs(theta[c, j])
        tp, tm = theta.copy(), theta.copy()
        tp[c, j] += h
        tm[c, j] -= h
        fd = (A.loss(A.build_problem(s, tp), lam, m_true) -
              A.loss(A.build_problem(s, tm), lam, m_true)) / (2 * h)
        assert abs(fd - dth[c, j]) <= 1e-4 * max(abs(fd), 1e-12), (c, j, fd, dth[c, j])


def test_adjoint_planted_mistake_is_caught():
    """Dropping the dW/dtau term changes dL/dsigma beyond the finite-difference tolerance."""
    s, theta, lam, m_true = setup(seed=5)
    _, dth, _ = A.adjoint(s, theta, lam, m_true)
    c, j = 0, 0
    h = 1e-6 * theta[c, j]
    tp, tm = theta.copy(), theta.copy()
    tp[c, j] += h
    tm[c, j] -= h
    fd = (A.loss(A.build_problem(s, tp), lam, m_true) -
          A.loss(A.build_problem(s, tm), lam, m_true)) / (2 * h)
    # recompute the gradient with the W-path term removed by hand
    prob = A.build_problem(s, theta)
    maps = A.forward(prob, lam)
    g = maps[-1] - m_true
    w_term = 0.0
    for i in reversed(range(len(lam))):
        u = prob.bin(g)
        g_next = np.zeros_like(g)
        for cc, (a, b) in enumerate(prob.chunks()):
            n = b - a
            N, nbar, tau, dnbar, dtau = A.psd_parts(n, s["params"][cc][3], *theta[cc])
            V = np.fft.rfft(prob.P(u, a, b))
            R = np.fft.rfft(prob.P(maps[i], a, b))
            Rp = np.fft.rfft(prob.P(maps[i + 1], a, b))
            if np.isinf(lam[i]):
                av, bv = np.ones_like(nbar), np.zeros_like(nbar)
            else:
                av = lam[i] * tau / (lam[i] * tau + nbar)
                bv = 1 - av
            T = av * prob.dtilde[cc] + bv * R
            if cc == c:
                w_term += np.sum(O.rfft_weights(n) * np.real(np.conj(V) * (Rp - T))) / n * dtau[j] / tau ** 2
            g_next += prob.PT(np.fft.irfft(bv * V, n), a, b) / tau
        g = g_next
    assert abs(fd - (dth[c, j] - w_term)) > 1e-3 * abs(fd)


@pytest.mark.parametrize("n", [1024, 999, 8])
def test_psd_parts_is_the_model_psd(n):
    """psd_parts (the adjoint's noise model with its derivatives) restates N(f); its N must
    be the messenger oracle's psd_from_params to rounding, with tau = sigma^2 and
    Nbar + tau = N, for even and odd lengths (DC floored to bin 1 in both)."""
    for sigma, fknee, alpha in ((1.0, 0.5, 2.0), (1.7, 3.0, 1.3)):
        N, nbar, tau, dnbar, dtau = A.psd_parts(n, 200.0, sigma, fknee, alpha)
        ref = O.psd_from_params(n, 200.0, sigma, fknee, alpha)
        assert np.allclose(N, ref, rtol=1e-14, atol=0)
        # Nbar + tau = N (comparing Nbar with N - tau would measure the cancellation)
        assert tau == sigma * sigma and np.allclose(nbar + tau, ref, rtol=1e-14, atol=0)
        assert np.all(nbar > 0)
        assert dnbar.shape == (3, n // 2 + 1) and dtau.shape == (3,)
