"""Plain FP64 CPU oracle for messenger-field mapmaking (Huffenberger & Naess, 1705.01893).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
The CUDA product path never calls it and shares no code with it.

Everything is float64 NumPy, written for legibility, following the paper's order:

* data model d = P m + n (Sec. 2, Eq. 1); pointing P has one IQU pixel block per
  sample with weights (1, cos 2psi, sin 2psi), the single pencil beam case (Sec. 2.1);
* chi^2(m) = (d - Pm)^T N^-1 (d - Pm) (Eq. 3), evaluated mode by mode in the Fourier
  domain (Sec. 3.1);
* the two-step messenger iteration (Sec. 2.1) with N = Nbar + T and T = diag(tau_c)
  piecewise per chunk (Sec. 4.2), so the map step is the 1/tau_c weighted binning
  (P^T T^-1 P)^-1 P^T T^-1 t (App. A);
* the cooling parameter lambda (Sec. 2.1, Eq. for N'(lambda)) and its schedule (Sec. 3.1);
* preconditioned conjugate gradients, the paper's comparison solver (Sec. 1, Sec. 3.1);
* the brute-force dense GLS solve (Eq. 2) used as the convergence target (Sec. 3.2 uses
  the same device on a 50x50 map).

Readings where the paper is silent:
* noise is exactly circulant per chunk, independent between chunks; N_k is given on the
  rfft bins k = 0..n//2 with F unnormalised and F^-1 carrying 1/n;
* the model PSD is N(f) = sigma^2 (1 + (fknee/f)^alpha), DC bin floored to bin 1;
  tau_c = sigma_c^2 (the infimum of the model PSD, keeping Nbar positive definite);
* lambda = inf means t = d (Sec. 2.1: large lambda gives F = 0 and the binned map);
* pixel cut: a pixel is kept iff hits >= 1 and, for IQU, the reciprocal condition number
  (eigmin/eigmax) of its 3x3 block of P^T T^-1 P is >= rcond_min.  Samples on cut pixels
  keep their data but get zero pointing rows;
* the "diagonal preconditioner" of the comparison PCG is the 3x3 pixel-block Jacobi
  matrix sum_c c0_c P_c^T P_c, c0_c = (1/n_c) sum_k 1/N_c(f_k) over all n_c frequencies,
  the diagonal of the circulant N_c^-1: the pixel blocks of P^T diag(N^-1) P (for white
  noise exactly the diagonal pixel blocks of A = P^T N^-1 P);
* cooling schedule: levels lambda_j = lambda_max^((L-1-j)/(L-1)), j = 0..L-1, each run
  for a fixed number of iterations, lambda_max = max_c max_k Nbar_c(f_k)/tau_c, after one
  lambda = inf step.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------- problem
class Problem:
    """Concatenated chunks: pix int [n], cos/sin [n] (None for T-only), tod [n], offsets.

    ``psd`` is a list of per-chunk arrays N_c(f_k), k = 0..n_c//2; ``tau`` per chunk.
    All arithmetic in float64 (inputs are converted)."""

    def __init__(self, pix, cos, sin, tod, offsets, npix, ncomp, psd, tau, rcond_min=1e-3):
        self.pix = np.asarray(pix, dtype=np.int64)
        self.ncomp = int(ncomp)
        self.cos = None if cos is None else np.asarray(cos, dtype=np.float64)
        self.sin = None if sin is None else np.asarray(sin, dtype=np.float64)
        self.tod = np.asarray(tod, dtype=np.float64)
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.npix = int(npix)
        self.psd = [np.asarray(p, dtype=np.float64) for p in psd]
        self.tau = np.asarray(tau, dtype=np.float64)
        self.rcond_min = float(rcond_min)
        self.nchunk = len(self.offsets) - 1
        self._plan()
        self.dtilde = [np.fft.rfft(self.tod[a:b]) for a, b in self.chunks()]

    def chunks(self):
        for c in range(self.nchunk):
            yield int(self.offsets[c]), int(self.offsets[c + 1])

    def nbar(self, c):
        """Nbar = N - T (Sec. 2.1) on the rfft bins of chunk c."""
        return self.psd[c] - self.tau[c]

    # ------------------------------------------------------------------ pointing (Eq. 1)
    def weights(self, a, b):
        """Per-sample pointing weights [n, ncomp]: 1 (T) or (1, cos 2psi, sin 2psi)."""
        n = b - a
        if self.ncomp == 1:
            return np.ones((n, 1))
        return np.stack([np.ones(n), self.cos[a:b], self.sin[a:b]], axis=1)

    def P(self, m, a, b, use_cut=True):
        """(P m) for samples a..b; pix = -1 (and cut pixels when use_cut) give 0."""
        pix = self.pix[a:b]
        good = pix >= 0
        if use_cut:
            good &= self.valid[np.where(pix >= 0, pix, 0)]
        w = self.weights(a, b)
        out = np.zeros(b - a)
        out[good] = np.sum(w[good] * m[pix[good]], axis=1)
        return out

    def PT(self, t, a, b, use_cut=True):
        """(P^T t) for samples a..b as a [npix, ncomp] map (np.add.at accumulation)."""
        pix = self.pix[a:b]
        good = pix >= 0
        if use_cut:
            good &= self.valid[np.where(pix >= 0, pix, 0)]
        w = self.weights(a, b)
        out = np.zeros((self.npix, self.ncomp))
        np.add.at(out, pix[good], w[good] * t[good][:, None])
        return out

    # -------------------------------------------------------------------- weight maps
    def _plan(self):
        """Hit counts and the 3x3 (or 1x1) blocks of P^T T^-1 P (Sec. 2.1, Sec. 4.2)."""
        nc = self.ncomp
        self.hits = np.zeros(self.npix, dtype=np.int64)
        self.ptp = np.zeros((self.npix, nc, nc))
        for c, (a, b) in enumerate(self.chunks()):
            pix = self.pix[a:b]
            good = pix >= 0
            np.add.at(self.hits, pix[good], 1)
            w = self.weights(a, b)[good]
            np.add.at(self.ptp, pix[good], w[:, :, None] * w[:, None, :] / self.tau[c])
        self.rcond = np.zeros(self.npix)
        hit = self.hits > 0
        if nc == 1:
            self.rcond[hit] = 1.0
        else:
            ev = np.linalg.eigvalsh(self.ptp[hit])
            self.rcond[hit] = ev[:, 0] / ev[:, -1]
        self.valid = hit & (self.rcond >= self.rcond_min if nc == 3 else hit)
        self.W = np.zeros_like(self.ptp)
        self.W[self.valid] = np.linalg.inv(self.ptp[self.valid])

    def bin(self, acc):
        """m = (P^T T^-1 P)^-1 acc per pixel block; cut pixels -> 0."""
        return np.einsum("pij,pj->pi", self.W, acc)


# ------------------------------------------------------------------------ noise model
def psd_from_params(n, fs, sigma, fknee, alpha):
    """N(f_k) = sigma^2 (1 + (fknee / f_k)^alpha) for k >= 1 (Sec. 2.3 noise model with a
    free slope), f_k = k fs / n; the DC bin takes the value of bin 1."""
    k = np.arange(n // 2 + 1, dtype=np.float64)
    f = k * fs / n
    N = np.empty(n // 2 + 1)
    N[1:] = sigma ** 2 * (1.0 + (fknee / f[1:]) ** alpha)
    N[0] = N[1]
    return N


def problem_from_synth(s, rcond_min=1e-3, tau=None, psd=None):
    """Build a Problem from a synthetic-data dict (params rows = sigma, fknee, alpha, fs)."""
    off = s["offsets"]
    if psd is None:
        psd = [psd_from_params(int(off[c + 1] - off[c]), *s["params"][c][[3, 0, 1, 2]])
               for c in range(len(off) - 1)]
    if tau is None:
        tau = s["params"][:, 0] ** 2
    return Problem(s["pix"], s["cos"], s["sin"], s["tod"], off, s["npix"], s["ncomp"],
                   psd, tau, rcond_min)


def rfft_weights(n):
    """Multiplicity of rfft bin k in the full DFT: 1 for DC (and Nyquist if n even), else 2."""
    w = np.full(n // 2 + 1, 2.0)
    w[0] = 1.0
    if n % 2 == 0:
        w[-1] = 1.0
    return w


# ---------------------------------------------------------------------------- chi^2
def chi2(prob, m, lam=1.0):
    """chi^2(m, lambda) = (d - Pm)^T N'(lambda)^-1 (d - Pm), N' = N + (lambda - 1) T
    (Eq. 3 at lambda = 1; Sec. 2.1), summed over every Fourier mode of every chunk."""
    total = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        r = prob.dtilde[c] - np.fft.rfft(prob.P(m, a, b))
        Np = prob.psd[c] + (lam - 1.0) * prob.tau[c]
        total += np.sum(rfft_weights(n) * np.abs(r) ** 2 / Np) / n
    return total


def chi2_modes(prob, m, lam=1.0):
    """chi^2 per Fourier mode of each chunk (Sec. 3.1 examines it per mode): for bin k,
    |d~_k - (Pm)~_k|^2 / (n N'_k), which has unit mean when m is the true map."""
    out = []
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        r = prob.dtilde[c] - np.fft.rfft(prob.P(m, a, b))
        out.append(np.abs(r) ** 2 / (n * (prob.psd[c] + (lam - 1.0) * prob.tau[c])))
    return out


# ---------------------------------------------------------------- messenger iteration
def messenger_step(prob, m, lam):
    """One messenger iteration (Sec. 2.1):
       t   = (Nbar^-1 + (lam T)^-1)^-1 (Nbar^-1 d + (lam T)^-1 P m)
           -> per Fourier mode: t~ = (lam tau d~ + Nbar (Pm)~) / (lam tau + Nbar);
       m'  = (P^T T^-1 P)^-1 P^T T^-1 t.
    lam = inf gives t = d (the binned map).  Returns (m', chi^2(m))."""
    acc = np.zeros((prob.npix, prob.ncomp))
    x2 = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        r = np.fft.rfft(prob.P(m, a, b))
        dt = prob.dtilde[c]
        x2 += np.sum(rfft_weights(n) * np.abs(dt - r) ** 2 / prob.psd[c]) / n
        if np.isinf(lam):
            tt = dt
        else:
            lt = lam * prob.tau[c]
            nb = prob.nbar(c)
            tt = (lt * dt + nb * r) / (lt + nb)
        t = np.fft.irfft(tt, n)
        acc += prob.PT(t, a, b) / prob.tau[c]
    return prob.bin(acc), x2


def lambda_max(prob):
    """Largest Nbar_c(f_k) / tau_c over all chunks and bins (top of the cooling range)."""
    return max(float(np.max(prob.nbar(c) / prob.tau[c])) for c in range(prob.nchunk))


def cooling_schedule(lam_max, levels, iters_per_level):
    """One lambda = inf step, then `levels` geometric levels from lam_max down to 1, each
    repeated `iters_per_level` times (Sec. 3.1)."""
    if levels == 1:
        lv = [1.0]
    else:
        lv = [lam_max ** ((levels - 1 - j) / (levels - 1)) for j in range(levels)]
    return np.array([np.inf] + [l for l in lv for _ in range(iters_per_level)])


def run_messenger(prob, lambdas, m0=None):
    """Iterate messenger_step over a lambda sequence; returns (final map, chi^2 of each
    iteration's input map)."""
    m = np.zeros((prob.npix, prob.ncomp)) if m0 is None else np.array(m0, dtype=np.float64)
    chis = []
    for lam in lambdas:
        m, x2 = messenger_step(prob, m, lam)
        chis.append(x2)
    return m, np.array(chis)


def run_messenger_adaptive(prob, levels, rel_tol, min_per_level, max_per_level, max_iter,
                           m0=None):
    """Cooling driven by the chi^2 plateaus of Sec. 3.1: one lambda = inf step, then the
    levels in order, moving on once chi^2 has stopped falling at the current level.

    Reading of "plateau" (the paper describes it without a rule): chi^2 of the map entering
    iteration j is known once iteration j runs, so after iteration i the newest measured
    decrease is that of iteration i - 2, (chi2_{i-2} - chi2_{i-1}) / chi2_{i-1}.  The level
    advances when at least min_per_level of its iterations have run, iteration i - 2 ran at
    this level and that relative decrease is below rel_tol, or when max_per_level of its
    iterations have run (not applied to the last level, lambda = 1).  The run ends when the
    last level would advance, or after max_iter iterations.  Returns (final map, chi^2 of
    each iteration's input map, lambda of each iteration)."""
    m = np.zeros((prob.npix, prob.ncomp)) if m0 is None else np.array(m0, dtype=np.float64)
    chis, lams = [], []
    lam = np.inf
    level, start = -1, 0
    while True:
        m, x2 = messenger_step(prob, m, lam)
        chis.append(x2)
        lams.append(lam)
        it = len(chis)                         # iterations done
        if it >= max_iter:
            break
        if level < 0:
            level, start = 0, it
        else:
            count = it - start
            plateau = False
            if it - 2 >= start:
                rel = (chis[it - 2] - chis[it - 1]) / chis[it - 1]
                plateau = rel < rel_tol
            last = level == len(levels) - 1
            if count >= min_per_level and plateau or (not last and count >= max_per_level):
                if last:
                    break
                level, start = level + 1, it
        lam = levels[level]
    return m, np.array(chis), np.array(lams)


# ------------------------------------------------------------------------------- PCG
def apply_A(prob, m):
    """A m = P^T N^-1 P m with N^-1 applied per chunk as 1/N(f_k) on the Fourier modes."""
    out = np.zeros((prob.npix, prob.ncomp))
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        y = np.fft.irfft(np.fft.rfft(prob.P(m, a, b)) / prob.psd[c], n)
        out += prob.PT(y, a, b)
    return out


def rhs_b(prob):
    """b = P^T N^-1 d."""
    out = np.zeros((prob.npix, prob.ncomp))
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        out += prob.PT(np.fft.irfft(prob.dtilde[c] / prob.psd[c], n), a, b)
    return out


def jacobi_blocks(prob):
    """Inverse of the pixel-block preconditioner sum_c c0_c P_c^T P_c (cut pixels -> 0),
    c0_c = (N_c^-1)_jj = (1/n) sum over all n frequencies of 1/N_c(f_k) (rfft multiplicities)."""
    nc = prob.ncomp
    M = np.zeros((prob.npix, nc, nc))
    for c, (a, b) in enumerate(prob.chunks()):
        n = b - a
        c0 = np.sum(rfft_weights(n) / prob.psd[c]) / n
        pix = prob.pix[a:b]
        good = pix >= 0
        w = prob.weights(a, b)[good]
        np.add.at(M, pix[good], c0 * w[:, :, None] * w[:, None, :])
    Minv = np.zeros_like(M)
    Minv[prob.valid] = np.linalg.inv(M[prob.valid])
    return Minv


def pcg(prob, n_iter, x0=None):
    """Preconditioned conjugate gradients on A m = b, starting at 0 (Sec. 3.1).
    Returns (x_final, chi^2(x_i) for i = 0..n_iter-1: the iterate entering step i)."""
    Minv = jacobi_blocks(prob)
    b = rhs_b(prob)
    x = np.zeros((prob.npix, prob.ncomp)) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - apply_A(prob, x)
    z = np.einsum("pij,pj->pi", Minv, r)
    p = z.copy()
    rz = np.sum(r * z)
    chis = []
    for _ in range(n_iter):
        chis.append(chi2(prob, x))
        q = apply_A(prob, p)
        alpha = rz / np.sum(p * q)
        x = x + alpha * p
        r = r - alpha * q
        z = np.einsum("pij,pj->pi", Minv, r)
        rz_new = np.sum(r * z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, np.array(chis)


# ---------------------------------------------------------------- dense brute force
def dense_P(prob, a, b):
    """Explicit pointing matrix rows for samples a..b over the valid unknowns."""
    idx = np.flatnonzero(prob.valid)
    col = -np.ones(prob.npix, dtype=np.int64)
    col[idx] = np.arange(idx.size)
    nc = prob.ncomp
    Pm = np.zeros((b - a, idx.size * nc))
    w = prob.weights(a, b)
    for s in range(b - a):
        p = prob.pix[a + s]
        if p >= 0 and col[p] >= 0:
            Pm[s, col[p] * nc:(col[p] + 1) * nc] = w[s]
    return Pm, idx


def dense_circulant(first_col):
    n = first_col.size
    i = np.arange(n)
    return first_col[(i[:, None] - i[None, :]) % n]


def dense_Ninv(prob, c, lam=1.0):
    """Explicit N'(lambda)^-1 of chunk c: circulant with first column irfft(1 / N'_k)."""
    a, b = prob.offsets[c], prob.offsets[c + 1]
    n = int(b - a)
    return dense_circulant(np.fft.irfft(1.0 / (prob.psd[c] + (lam - 1.0) * prob.tau[c]), n))


def dense_solve(prob, lam=1.0):
    """m(lambda) = (P^T N'^-1 P)^-1 P^T N'^-1 d (Eq. 2 at lambda = 1; Sec. 2.1 otherwise),
    by explicit matrices; returns a [npix, ncomp] map with cut pixels at 0."""
    A = 0.0
    bv = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        Pc, idx = dense_P(prob, a, b)
        Ni = dense_Ninv(prob, c, lam)
        A = A + Pc.T @ Ni @ Pc
        bv = bv + Pc.T @ (Ni @ prob.tod[a:b])
    x = np.linalg.solve(A, bv)
    m = np.zeros((prob.npix, prob.ncomp))
    m[idx] = x.reshape(-1, prob.ncomp)
    return m


def dense_chi2(prob, m, lam=1.0):
    """(d - Pm)^T N'^-1 (d - Pm) with explicit circulant matrices."""
    tot = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        r = prob.tod[a:b] - prob.P(m, a, b)
        tot += r @ dense_Ninv(prob, c, lam) @ r
    return tot


def dense_F(prob, lam):
    """Explicit F(lambda) = I - (P^T T^-1 P)^-1 P^T (lambda^-1 Nbar + T)^-1 P (Sec. 2.1)."""
    K = 0.0
    for c, (a, b) in enumerate(prob.chunks()):
        Pc, idx = dense_P(prob, a, b)
        n = int(b - a)
        k = np.fft.irfft(1.0 / (prob.nbar(c) / lam + prob.tau[c]), n)
        K = K + Pc.T @ dense_circulant(k) @ Pc
    Wd = np.zeros((idx.size * prob.ncomp,) * 2)
    nc = prob.ncomp
    for i, p in enumerate(idx):
        Wd[i * nc:(i + 1) * nc, i * nc:(i + 1) * nc] = prob.W[p]
    return np.eye(Wd.shape[0]) - Wd @ K
