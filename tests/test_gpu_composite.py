"""GPU parity of composite pointing (App. B: P = g_a P_a + g_b P_b, T_A = T_B = T/2) against
the FP64 composite oracle: hit counts bit-exact, the pixel cut and D^-1 to 1e-10, single
steps <= 1e-5 relative L2, a cooled run <= 1e-4 map rms (over the kept pixels; a
differencing instrument leaves the mean unconstrained, which the update never moves
differently on the two sides) and chi^2 <= 1e-5."""
import math

import numpy as np
import pytest

import oracle.composite as C
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
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def comp_problem(s):
    off = s["offsets"]
    psd = [O.psd_from_params(int(off[c + 1] - off[c]), *s["params"][c][[3, 0, 1, 2]])
           for c in range(len(off) - 1)]
    a = (s["pix"], s["cos"], s["sin"], s["gain_a"])
    b = (s["pix_b"], s.get("cos_b"), s.get("sin_b"), s["gain_b"])
    return C.CompositeProblem(a, b, s["tod"], off, s["npix"], s["ncomp"], psd,
                              s["params"][:, 0] ** 2)


def differential():
    return synth.config_differential(width=16, n_chunks=6, n_per=3000, sep=2.0, seed=17050521)


def iqu_pair():
    """IQU detector pairs seen through two components: the second component is another
    detector's pointing (rolled by 7 samples) at gain 0.5."""
    s = dict(synth.config_iqu(16, 3, 3000, 17050522))
    s["pix_b"] = np.roll(s["pix"], 7)
    s["cos_b"] = np.roll(s["cos"], 7)
    s["sin_b"] = np.roll(s["sin"], 7)
    s["gain_a"], s["gain_b"] = 1.0, 0.5
    return s


@pytest.mark.parametrize("cfg", ["differential", "iqu_pair"])
def test_composite_plan_and_single_steps(cfg):
    s = differential() if cfg == "differential" else iqu_pair()
    prob = comp_problem(s)
    plan = binding.plan_from_synth(s, DEV)
    nc = s["ncomp"]
    hits = torch.empty(s["npix"], dtype=torch.int32, device=DEV)
    valid = torch.empty(s["npix"], dtype=torch.uint8, device=DEV)
    w = torch.empty(s["npix"], nc * nc, dtype=torch.float64, device=DEV)
    plan.maps(hits, valid, w)
    torch.cuda.synchronize()
    assert np.array_equal(hits.cpu().numpy(), prob.hits)
    v = valid.cpu().numpy().astype(bool)
    near = np.abs(prob.rcond - 1e-3) <= 1e-9
    assert np.array_equal(v[~near], prob.valid[~near])
    W = w.cpu().numpy().reshape(-1, nc, nc)
    assert rel(W[prob.valid], prob.W[prob.valid]) <= 1e-10
    lm = O.lambda_max(prob)
    assert abs(plan.lambda_max() - lm) <= 1e-12 * lm
    m0 = np.random.default_rng(8).standard_normal((s["npix"], nc)) * prob.valid[:, None]
    for lam in (math.inf, lm, 3.0, 1.0):
        m_ref, x_ref = C.step(prob, m0, lam)
        m = torch.as_tensor(m0).to(DEV)
        chi = torch.zeros(1, dtype=torch.float64, device=DEV)
        plan.messenger(m, [lam], chi)
        torch.cuda.synchronize()
        assert rel(m.cpu().numpy(), m_ref) <= 1e-5, lam
        assert abs(chi.item() - x_ref) <= 1e-5 * x_ref


@pytest.mark.parametrize("cfg", ["differential", "iqu_pair"])
def test_composite_cooled_run(cfg):
    s = differential() if cfg == "differential" else iqu_pair()
    prob = comp_problem(s)
    lam = np.concatenate([O.cooling_schedule(O.lambda_max(prob), 6, 6), np.ones(20)])
    m_ref, chi_ref = C.run(prob, lam)
    plan = binding.plan_from_synth(s, DEV)
    m = torch.zeros(s["npix"], s["ncomp"], dtype=torch.float64, device=DEV)
    chi = torch.zeros(len(lam), dtype=torch.float64, device=DEV)
    plan.messenger(m, lam, chi)
    torch.cuda.synchronize()
    g = m.cpu().numpy()[prob.valid]
    r = m_ref[prob.valid]
    rms = np.sqrt(np.mean((g - r) ** 2)) / np.sqrt(np.mean(r ** 2))
    assert rms <= 1e-4, rms
    assert np.max(np.abs(chi.cpu().numpy() - chi_ref) / chi_ref) <= 1e-5
    # chi^2 of the maps, per Fourier mode, on the composite pointing
    tot, modes = plan.chi2_modes(m, 1.0)
    c_ref = C.chi2(prob, m.cpu().numpy())
    assert abs(tot.item() - c_ref) <= 1e-5 * c_ref


def test_composite_refuses_single_component_forms():
    s = differential()
    plan = binding.plan_from_synth(s, DEV)
    m = torch.zeros(s["npix"], 1, dtype=torch.float64, device=DEV)
    for call in (lambda: plan.messenger_graph(m, [2.0]),
                 lambda: plan.pcg(m, 2),
                 lambda: plan.messenger_md(m, [2.0]),
                 lambda: plan.messenger_adaptive(m, [2.0, 1.0], 1e-3)):
        with pytest.raises(binding.MMError) as e:
            call()
        assert e.value.code == binding.MM_ERR_UNSUPPORTED
