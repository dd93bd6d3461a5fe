"""Pins of the composite-pointing oracle (App. B, P = P_A + P_B, T_A = T_B = T/2) against
facts the paper and the algebra fix, independent of the oracle's own arithmetic."""
import math

import numpy as np

import oracle.composite as C
import oracle.messenger as O
from paper_1705_01893_gb300 import synth


def comp_problem(s, rcond_min=1e-3):
    off = s["offsets"]
    psd = [O.psd_from_params(int(off[c + 1] - off[c]), *s["params"][c][[3, 0, 1, 2]])
           for c in range(len(off) - 1)]
    tau = s["params"][:, 0] ** 2
    a = (s["pix"], s["cos"], s["sin"], s.get("gain_a", 1.0))
    b = (s["pix_b"], s.get("cos_b"), s.get("sin_b"), s.get("gain_b", -1.0))
    return C.CompositeProblem(a, b, s["tod"], off, s["npix"], s["ncomp"], psd, tau, rcond_min)


def tiny_diff(noiseless=False, seed=17050511):
    return synth.config_differential(width=8, n_chunks=3, n_per=512, sep=2.0, seed=seed,
                                     noiseless=noiseless)


def test_no_second_component_is_the_single_beam_step():
    """App. B's check: with P_B = 0 the composite step at lambda = 1 is the single-beam
    messenger step (Sec. 2.1) with messenger covariance T_A = tau/2."""
    s = synth.config_iqu(8, 2, 512, 11)
    s = dict(s)
    s["pix_b"] = np.full_like(s["pix"], -1)
    s["cos_b"], s["sin_b"] = s["cos"], s["sin"]
    s["gain_a"], s["gain_b"] = 1.0, 1.0
    cp = comp_problem(s)
    sp = O.problem_from_synth(s, tau=0.5 * s["params"][:, 0] ** 2)
    assert np.array_equal(cp.valid, sp.valid)
    m0 = np.random.default_rng(3).standard_normal((s["npix"], 3)) * sp.valid[:, None]
    mc, xc = C.step(cp, m0, 1.0)
    ms, xs = O.messenger_step(sp, m0, 1.0)
    assert np.linalg.norm(mc - ms) <= 1e-10 * np.linalg.norm(ms)
    assert abs(xc - xs) <= 1e-10 * xs


def test_gls_solution_is_a_fixed_point_and_noiseless_sky_too():
    """At lambda = 1 the update is D^-1 P^T N^-1 (d - P m), zero at any solution of the
    normal equations (Eq. 2); for noiseless data d = P m_true the residual vanishes at
    m_true for every lambda."""
    s = tiny_diff()
    prob = comp_problem(s)
    ms = C.dense_solution(prob)
    m1, _ = C.step(prob, ms, 1.0)
    assert np.linalg.norm(m1 - ms) <= 1e-8 * np.linalg.norm(ms)
    s0 = tiny_diff(noiseless=True)
    p0 = comp_problem(s0)
    mt = s0["m_true"] * p0.valid[:, None]
    p0.tod[:] = np.concatenate([p0.P(mt, a, b) for a, b in p0.chunks()])
    p0.dtilde = [np.fft.rfft(p0.tod[a:b]) for a, b in p0.chunks()]
    for lam in (1.0, 7.0, math.inf):
        m1, _ = C.step(p0, mt, lam)
        assert np.linalg.norm(m1 - mt) <= 1e-12 * np.linalg.norm(mt)


def test_iterations_reach_the_gls_chi2():
    """lambda = 1 iterations from zero (weighted Jacobi on the normal equations) bring chi^2
    (Eq. 3) to its minimum, which is unique although a differencing instrument leaves the
    map's mean unconstrained; the constrained part of the map converges too."""
    s = tiny_diff(seed=17050512)
    prob = comp_problem(s)
    ms = C.dense_solution(prob)
    c_ref = C.chi2(prob, ms)
    lam = np.concatenate([O.cooling_schedule(30.0, 6, 20), np.ones(1500)])
    m, chis = C.run(prob, lam)
    assert (C.chi2(prob, m) - c_ref) / c_ref < 1e-6
    v = prob.valid
    d = (m - ms)[v, 0]
    d -= d.mean()                                   # the unconstrained mean
    ref = ms[v, 0] - ms[v, 0].mean()
    assert np.linalg.norm(d) <= 1e-3 * np.linalg.norm(ref)


def test_fixed_lambda_reaches_the_lambda_solution():
    """At fixed lambda the update vanishes where P^T (Nbar / lambda + T)^-1 (d - P m) = 0,
    i.e. at the GLS solution for N' = Nbar + lambda T (Sec. 2.1's m(lambda)); iterating
    reaches its chi^2(., lambda) minimum."""
    s = tiny_diff(seed=17050513)
    prob = comp_problem(s)
    lam = 5.0
    ms = C.dense_solution(prob, lam)
    c_ref = C.chi2(prob, ms, lam)
    m, _ = C.run(prob, np.full(2000, lam))
    assert (C.chi2(prob, m, lam) - c_ref) / c_ref < 1e-6
    # and not the lambda = 1 solution
    c1 = C.chi2(prob, C.dense_solution(prob, 1.0), lam)
    assert (c1 - c_ref) / c_ref > 1e-4


# --------------------------------------------------------------- planted mistakes
def _step_variant(sign=1.0, lam_times=False):
    """C.step retyped with one slip: the residual's sign, or lambda multiplying Nbar."""
    def step(prob, m, lam):
        acc = np.zeros((prob.npix, prob.ncomp))
        x2 = C.chi2(prob, m)
        for c, (a, b) in enumerate(prob.chunks()):
            n = b - a
            r = np.fft.rfft(sign * (prob.tod[a:b] - prob.P(m, a, b)))
            nbar = prob.psd[c] - prob.tau[c]
            if np.isinf(lam):
                den = prob.tau[c]
            else:
                den = (nbar * lam if lam_times else nbar / lam) + prob.tau[c]
            acc += prob.PT(np.fft.irfft(r / den, n), a, b)
        return m + np.einsum("pij,pj->pi", prob.W, acc), x2
    return step


PINS = [test_no_second_component_is_the_single_beam_step,
        test_gls_solution_is_a_fixed_point_and_noiseless_sky_too,
        test_fixed_lambda_reaches_the_lambda_solution,
        test_iterations_reach_the_gls_chi2]


def test_planted_mistakes_break_a_pin(monkeypatch):
    """Each plausible slip in the composite oracle (the T split, the residual's sign, lambda
    on the wrong side of Nbar, the second beam missing from P^T) fails at least one pin."""
    orig_plan = C.CompositeProblem._plan

    def plan_full_t(self):             # T_A = T_B = tau instead of tau / 2
        orig_plan(self)
        self.D = 0.5 * self.D
        self.W = np.zeros_like(self.D)
        self.W[self.valid] = np.linalg.inv(self.D[self.valid])

    def pt_first_only(self, t, a, b):  # P_A^T t only
        out = np.zeros((self.npix, self.ncomp))
        pix, w = self.comps[0]
        p = pix[a:b]
        good = (p >= 0) & self.valid[np.where(p >= 0, p, 0)]
        np.add.at(out, p[good], w[a:b][good] * t[good][:, None])
        return out

    slips = {
        "T split": lambda mp: mp.setattr(C.CompositeProblem, "_plan", plan_full_t),
        "sign": lambda mp: mp.setattr(C, "step", _step_variant(sign=-1.0)),
        "lambda": lambda mp: mp.setattr(C, "step", _step_variant(lam_times=True)),
        "second beam": lambda mp: mp.setattr(C.CompositeProblem, "PT", pt_first_only),
    }
    for name, plant in slips.items():
        with monkeypatch.context() as mp:
            plant(mp)
            caught = False
            for pin in PINS:
                try:
                    with np.errstate(all="ignore"):
                        pin()
                except (AssertionError, np.linalg.LinAlgError):
                    caught = True
                    break
            assert caught, f"no pin caught the planted mistake: {name}"
