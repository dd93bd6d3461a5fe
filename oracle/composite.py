"""FP64 CPU oracle of messenger mapmaking with a composite pointing matrix: TEST
INFRASTRUCTURE ONLY (only tests/ may import it; the CUDA path shares no code with it).

App. B: the pointing is a sum of two single-entry components, P = P_A + P_B (a differencing
instrument has entries +1 and -1 per sample, or gains g_A, g_B times the IQU weights), and
the messenger covariance is split as T = T_A + T_B.  Reading of the split (the paper's own
choice in its differential test): T_A = T_B = T/2 = tau_c/2 on chunk c.  The step in the
compact form of App. B is

    m' = m + D^-1 P^T (lambda^-1 Nbar + T)^-1 (d - P m),
    D  = P_A^T T_A^-1 P_A + P_B^T T_B^-1 P_B       (block diagonal: 3x3 per pixel),

with (lambda^-1 Nbar + T)^-1 applied per chunk as 1 / (Nbar_k / lambda + tau) on the rfft
bins (lambda = inf: 1 / tau).  Pixel cut as for one component: a pixel is kept iff either
component hits it and the reciprocal condition number of its block of D is >= rcond_min;
an entry that lands on a cut pixel is dropped from P.
"""
from __future__ import annotations

import numpy as np

from . import messenger as O


class CompositeProblem:
    """Chunks of data d with two pointing components (pix_a, w_a) and (pix_b, w_b)."""

    def __init__(self, comp_a, comp_b, tod, offsets, npix, ncomp, psd, tau, rcond_min=1e-3):
        # comp = (pix [n], cos [n] or None, sin [n] or None, gain)
        self.ncomp = int(ncomp)
        self.npix = int(npix)
        self.tod = np.asarray(tod, dtype=np.float64)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.nchunk = len(self.offsets) - 1
        self.psd = [np.asarray(p, dtype=np.float64) for p in psd]
        self.tau = np.asarray(tau, dtype=np.float64)
        self.rcond_min = float(rcond_min)
        self.comps = []
        for pix, cos, sin, gain in (comp_a, comp_b):
            pix = np.asarray(pix, dtype=np.int64)
            n = pix.shape[0]
            if self.ncomp == 1:
                w = np.full((n, 1), float(gain))
            else:
                w = float(gain) * np.stack([np.ones(n), np.asarray(cos, dtype=np.float64),
                                            np.asarray(sin, dtype=np.float64)], axis=1)
            self.comps.append((pix, w))
        self._plan()
        self.dtilde = [np.fft.rfft(self.tod[a:b]) for a, b in self.chunks()]

    def chunks(self):
        for c in range(self.nchunk):
            yield int(self.offsets[c]), int(self.offsets[c + 1])

    def nbar(self, c):
        """Nbar = N - T (T = T_A + T_B = tau_c) on the rfft bins of chunk c."""
        return self.psd[c] - self.tau[c]

    def _plan(self):
        """Hit counts of both components and the blocks of D (T_A = T_B = tau/2)."""
        nc = self.ncomp
        self.hits = np.zeros(self.npix, dtype=np.int64)
        self.D = np.zeros((self.npix, nc, nc))
        for c, (a, b) in enumerate(self.chunks()):
            for pix, w in self.comps:
                p = pix[a:b]
                good = p >= 0
                np.add.at(self.hits, p[good], 1)
                wg = w[a:b][good]
                np.add.at(self.D, p[good], wg[:, :, None] * wg[:, None, :] / (0.5 * self.tau[c]))
        self.rcond = np.zeros(self.npix)
        hit = self.hits > 0
        if nc == 1:
            self.rcond[hit] = 1.0
        else:
            ev = np.linalg.eigvalsh(self.D[hit])
            self.rcond[hit] = ev[:, 0] / ev[:, -1]
        self.valid = hit & (self.rcond >= self.rcond_min if nc == 3 else hit)
        self.W = np.zeros_like(self.D)
        self.W[self.valid] = np.linalg.inv(self.D[self.valid])

    def P(self, m, a, b):
        """(P_A + P_B) m for samples a..b; entries on unhit / cut pixels dropped."""
        out = np.zeros(b - a)
        for pix, w in self.comps:
            p = pix[a:b]
            good = (p >= 0) & self.valid[np.where(p >= 0, p, 0)]
            out[good] += np.sum(w[a:b][good] * m[p[good]], axis=1)
        return out

    def PT(self, t, a, b):
        """(P_A + P_B)^T t for samples a..b as an [npix, ncomp] map."""
        out = np.zeros((self.npix, self.ncomp))
        for pix, w in self.comps:
            p = pix[a:b]
            good = (p >= 0) & self.valid[np.where(p >= 0, p, 0)]
            np.add.at(out, p[good], w[a:b][good] * t[good][:, None])
        return out


def chi2(prob, m, lam=1.0):
    """(d - P m)^T N'(lambda)^-1 (d - P m), N' = N + (lambda - 1) T, per Fourier mode (Eq. 3)."""
    tot = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        r = prob.dtilde[c] - np.fft.rfft(prob.P(m, a, b))
        Np = prob.psd[c] + (lam - 1.0) * prob.tau[c]
        tot += np.sum(O.rfft_weights(n) * np.abs(r) ** 2 / Np) / n
    return tot


def step(prob, m, lam):
    """One step of the compact form; returns (m', chi^2 of the input map at lambda = 1)."""
    acc = np.zeros((prob.npix, prob.ncomp))
    x2 = chi2(prob, m)
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        r = np.fft.rfft(prob.tod[a:b] - prob.P(m, a, b))
        nbar = prob.psd[c] - prob.tau[c]
        den = prob.tau[c] if np.isinf(lam) else nbar / lam + prob.tau[c]
        acc += prob.PT(np.fft.irfft(r / den, n), a, b)
    return m + np.einsum("pij,pj->pi", prob.W, acc), x2


def run(prob, lambdas, m0=None):
    m = np.zeros((prob.npix, prob.ncomp)) if m0 is None else np.array(m0, dtype=np.float64)
    chis = []
    for lam in lambdas:
        m, x2 = step(prob, m, lam)
        chis.append(x2)
    return m, np.array(chis)


def dense_P(prob, a, b):
    """Explicit [n, npix*ncomp] pointing of samples a..b (both components, cut applied)."""
    nc = prob.ncomp
    M = np.zeros((b - a, prob.npix * nc))
    for pix, w in prob.comps:
        for s in range(a, b):
            p = pix[s]
            if p >= 0 and prob.valid[p]:
                M[s - a, p * nc:(p + 1) * nc] += w[s]
    return M


def dense_solution(prob, lam=1.0):
    """Minimum-norm least-squares solution of (P^T N'^-1 P) m = P^T N'^-1 d (Eq. 2 at
    lambda = 1) with N' = N + (lambda - 1) T, by explicit circulant N'^-1 (a differencing
    instrument leaves some modes, e.g. the mean, unconstrained; chi^2 at the solution is
    unique all the same)."""
    A = 0.0
    bv = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        Pc = dense_P(prob, a, b)
        n = b - a
        k = np.fft.irfft(1.0 / (prob.psd[c] + (lam - 1.0) * prob.tau[c]), n)
        Ninv = np.array([np.roll(k, j) for j in range(n)])
        A = A + Pc.T @ Ninv @ Pc
        bv = bv + Pc.T @ Ninv @ prob.tod[a:b]
    x = np.linalg.lstsq(A, bv, rcond=1e-10)[0]
    return x.reshape(prob.npix, prob.ncomp)
