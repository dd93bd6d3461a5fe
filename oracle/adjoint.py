"""FP64 CPU oracle of the messenger iteration's adjoint: TEST INFRASTRUCTURE ONLY.

Loss L = 1/2 || m_K - m_true ||^2 after K messenger iterations (Sec. 2.1) with a fixed
cooling sequence lambda_1..K (the lambdas are constants: no gradient flows into the
schedule).  Parameters per chunk c: the data d_c and the noise model theta_c =
(sigma_c, f_knee_c, alpha_c) with N_c(f) = sigma^2 (1 + (f_knee / f)^alpha), DC floored to
bin 1, and tau_c = sigma_c^2, so Nbar_c = sigma^2 (f_knee / f)^alpha.

One step, per chunk (a = lambda tau / (lambda tau + Nbar), b = 1 - a, per Fourier mode):
    t_c   = irfft(a d~_c + b (P_c m)~)
    m'    = W sum_c P_c^T t_c / tau_c,        W = (sum_c P_c^T P_c / tau_c)^-1.
Its transpose, given gbar = dL/dm':  u = W gbar,  v_c = P_c u,
    dL/dd_c += irfft(a v~_c) / tau_c,         dL/dm  = sum_c P_c^T irfft(b v~_c) / tau_c,
    dL/dtheta_c += <v_c / tau_c, dt_c/dtheta_c>  +  (1/tau_c^2) <v_c, P_c m' - t_c> dtau/dtheta,
the last term from dW/dtau_c.  Inner products of real timestreams are evaluated mode by
mode, <x, y> = (1/n) sum_k w_k Re(conj(x~_k) y~_k).  Only tests/ may import this module.
"""
from __future__ import annotations

import numpy as np

from . import messenger as O


def psd_parts(n, fs, sigma, fknee, alpha):
    """N, Nbar, tau and the derivatives dNbar/dtheta, dtau/dtheta on the rfft bins."""
    k = np.arange(n // 2 + 1, dtype=np.float64)
    f = k * fs / n
    f[0] = f[1]                                   # DC bin takes bin 1's value (and slope)
    x = (fknee / f) ** alpha
    tau = sigma * sigma
    nbar = tau * x
    dnbar = np.stack([2.0 * sigma * x,            # d/dsigma
                      tau * alpha * x / fknee,    # d/dfknee
                      tau * x * np.log(fknee / f)])  # d/dalpha
    dtau = np.array([2.0 * sigma, 0.0, 0.0])
    return nbar + tau, nbar, tau, dnbar, dtau


def build_problem(s, theta, tod=None, rcond_min=1e-3):
    """Problem for data `tod` (default s['tod']) and theta [n_chunks, 3]."""
    off = s["offsets"]
    psd, tau = [], []
    for c in range(len(off) - 1):
        n = int(off[c + 1] - off[c])
        N, _, t, _, _ = psd_parts(n, s["params"][c][3], *theta[c])
        psd.append(N)
        tau.append(t)
    return O.Problem(s["pix"], s["cos"], s["sin"], s["tod"] if tod is None else tod, off,
                     s["npix"], s["ncomp"], psd, np.array(tau), rcond_min)


def forward(prob, lambdas, m0=None):
    """All iterates m_0..m_K (m_0 = m0 or zeros)."""
    m = np.zeros((prob.npix, prob.ncomp)) if m0 is None else np.array(m0, dtype=np.float64)
    maps = [m]
    for lam in lambdas:
        m, _ = O.messenger_step(prob, m, lam)
        maps.append(m)
    return maps


def loss(prob, lambdas, m_true):
    m = forward(prob, lambdas)[-1]
    return 0.5 * float(np.sum((m - m_true) ** 2))


def adjoint(s, theta, lambdas, m_true, tod=None):
    """(dL/dd [n], dL/dtheta [n_chunks, 3], L) by the transposed step sequence."""
    prob = build_problem(s, theta, tod)
    maps = forward(prob, lambdas)
    g = maps[-1] - m_true
    L = 0.5 * float(np.sum(g ** 2))
    dd = np.zeros(int(prob.offsets[-1]))
    dth = np.zeros((prob.nchunk, 3))
    parts = []
    for c, (a, b) in enumerate(prob.chunks()):
        parts.append(psd_parts(b - a, s["params"][c][3], *theta[c]))
    for i in reversed(range(len(lambdas))):
        lam = lambdas[i]
        u = prob.bin(g)                                # W gbar
        g_next = np.zeros_like(g)
        for c, (a, b) in enumerate(prob.chunks()):
            n = b - a
            _, nbar, tau, dnbar, dtau = parts[c]
            wk = O.rfft_weights(n)
            v = prob.P(u, a, b)
            V = np.fft.rfft(v)
            D = prob.dtilde[c]
            R = np.fft.rfft(prob.P(maps[i], a, b))
            Rp = np.fft.rfft(prob.P(maps[i + 1], a, b))
            if np.isinf(lam):
                av, bv = np.ones_like(nbar), np.zeros_like(nbar)
                dT_dnbar = np.zeros_like(V)
                dT_dtau = np.zeros_like(V)
            else:
                lt = lam * tau
                den = lt + nbar
                av, bv = lt / den, nbar / den
                dT_dnbar = lt * (R - D) / den ** 2
                dT_dtau = lam * nbar * (D - R) / den ** 2
            That = av * D + bv * R
            pair = lambda X: float(np.sum(wk * np.real(np.conj(V) * X))) / n  # noqa: E731
            dd[a:b] += np.fft.irfft(av * V, n) / tau
            g_next += prob.PT(np.fft.irfft(bv * V, n), a, b) / tau
            for j in range(3):
                dth[c, j] += pair(dT_dnbar * dnbar[j]) / tau
                dth[c, j] += pair(dT_dtau) * dtau[j] / tau
                dth[c, j] += pair(Rp - That) * dtau[j] / tau ** 2
        g = g_next
    return dd, dth, L


def dense_d_gradient(s, theta, lambdas, m_true):
    """dL/dd from the explicit linear map m_K = M d (m_0 = 0), built by composing dense
    operators: M_{i+1} = W P^T T^-1 A(lambda_i) + G(lambda_i) M_i."""
    prob = build_problem(s, theta)
    idx = np.flatnonzero(prob.valid)
    nc = prob.ncomp
    nu = idx.size * nc
    nt = int(prob.offsets[-1])
    Wd = np.zeros((nu, nu))
    for i, p in enumerate(idx):
        Wd[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc] = prob.W[p]
    Pd = np.zeros((nt, nu))
    for c, (a, b) in enumerate(prob.chunks()):
        Pd[a:b], _ = O.dense_P(prob, a, b)
    M = np.zeros((nu, nt))
    for lam in lambdas:
        Ab = np.zeros((nt, nt))
        Bb = np.zeros((nt, nt))
        for c, (a, b) in enumerate(prob.chunks()):
            n = b - a
            nbar = prob.nbar(c)
            tau = prob.tau[c]
            if np.isinf(lam):
                av, bv = np.ones_like(nbar), np.zeros_like(nbar)
            else:
                av = lam * tau / (lam * tau + nbar)
                bv = 1.0 - av
            Ab[a:b, a:b] = O.dense_circulant(np.fft.irfft(av, n)) / tau
            Bb[a:b, a:b] = O.dense_circulant(np.fft.irfft(bv, n)) / tau
        M = Wd @ Pd.T @ (Ab + Bb @ Pd @ M)
    mK = np.zeros((prob.npix, nc))
    mK[idx] = (M @ prob.tod).reshape(-1, nc)
    g = (mK - m_true)[idx].ravel()
    return M.T @ g
