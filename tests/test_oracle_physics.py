"""Pins for the oracle's physics and transport: the attenuation law (Eqs. 1-3),
the free-path distribution in a piecewise-constant medium (Eqs. 5-8), Kahn's
sampling against the Klein-Nishina law, table interpolation, energy
conservation and replay invariants."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle
import synth
from synth.materials import constant_material, toy_materials, ME_C2_MEV, E_GRID_MEV
from synth.scenes import Source


def test_mu_table_interpolation(oracle_lib):
    sc = synth.scenes.tiny_scene()
    g = oracle.Geometry(sc)
    lead = sc.materials[1]
    for k in range(32):
        mt, mp = g.mu(1, lead.energies[k])
        assert mt == lead.mu_compton[k] + lead.mu_photo[k] and mp == lead.mu_photo[k]
    e = math.sqrt(lead.energies[7] * lead.energies[8])
    f = (e - lead.energies[7]) / (lead.energies[8] - lead.energies[7])
    mt, mp = g.mu(1, e)
    ref_c = lead.mu_compton[7] + f * (lead.mu_compton[8] - lead.mu_compton[7])
    ref_p = lead.mu_photo[7] + f * (lead.mu_photo[8] - lead.mu_photo[7])
    assert abs(mt - (ref_c + ref_p)) < 1e-15 * mt and abs(mp - ref_p) < 1e-15 * mp
    assert g.mu(1, 1e-4) == g.mu(1, lead.energies[0])           # clamped below
    assert g.mu(1, 1e3) == g.mu(1, lead.energies[-1])           # clamped above
    assert g.mu(4, 1.0) == (0.0, 0.0)                           # vacuum


@pytest.mark.parametrize("mu,x", [(0.02, 30.0), (0.1, 10.0), (0.5, 3.0)])
def test_slab_transmission_exp(oracle_lib, mu, x):
    """Eqs. 2-3: a pure absorber slab transmits exp(-mu x) of a normal beam (binomial 3.5 sigma)."""
    sc = synth.scenes.slab_scene(x, constant_material("abs", 1.0, mu))
    g = oracle.Geometry(sc)
    src = Source(pos=(0.0, 0.0, -1.0), isotropic=False, direction=(0.0, 0.0, 1.0), e_kind="mono", e0=1.0, e1=1.0)
    n = 200000
    r = g.transport(src, 42, n, want_hash=False, want_len=False)
    c = dict(zip(oracle.COUNTER_NAMES, r["counters"].tolist()))
    p = math.exp(-mu * x)
    assert abs(c["escaped"] / n - p) < 3.5 * math.sqrt(p * (1 - p) / n)
    assert c["photo"] + c["escaped"] == n and c["compton"] == 0


def test_free_path_cdf_two_layers(oracle_lib):
    """Eq. 5 with Eqs. 6-8: P(T < t) = 1 - exp(-G(t)), G piecewise linear (KS test on Y ~ Exp(1))."""
    mu1, mu2, a, b = 0.05, 0.3, 10.0, 5.0
    sc = synth.scenes.layered_scene([a, b], [constant_material("m1", 1.0, mu1), constant_material("m2", 1.0, mu2)])
    g = oracle.Geometry(sc)
    rng = np.random.default_rng(0)
    Y = rng.exponential(size=6000)
    T = np.array([g.free_path([0, 0, 0], [0, 0, 1], 1.0, y)[0] for y in Y])
    fin = np.isfinite(T)
    p_escape = math.exp(-(mu1 * a + mu2 * b))
    assert abs((~fin).mean() - p_escape) < 4 * math.sqrt(p_escape * (1 - p_escape) / Y.size)

    def G(t):
        return np.where(t <= a, mu1 * t, mu1 * a + mu2 * (np.minimum(t, a + b) - a))

    def cdf_cond(t):
        return (1 - np.exp(-G(t))) / (1 - p_escape)

    assert stats.kstest(T[fin], cdf_cond).pvalue > 1e-3


def kn_density_eps(eps, alpha):
    """Klein-Nishina dsigma/deps (unnormalised) for eps = E'/E in [1/(1+2 alpha), 1]."""
    cost = 1.0 - (1.0 / eps - 1.0) / alpha
    return 1.0 / eps + eps - (1.0 - cost * cost)


@pytest.mark.parametrize("E", [0.05, 0.3, 1.0, 5.0, 20.0])
def test_kahn_matches_klein_nishina(oracle_lib, E):
    n = 200000
    eta, cost = oracle.kahn_sample(E, 1234, n)
    alpha = E / ME_C2_MEV
    eps = 1.0 / eta
    lo = 1.0 / (1.0 + 2.0 * alpha)
    assert eps.min() >= lo * (1 - 1e-12) and eps.max() <= 1.0 + 1e-12
    assert np.allclose(cost, 1.0 - (eta - 1.0) / alpha)
    edges = np.linspace(lo, 1.0, 51)
    counts, _ = np.histogram(eps, edges)
    w = np.array([integrate.quad(kn_density_eps, edges[i], edges[i + 1], args=(alpha,))[0] for i in range(50)])
    expected = n * w / w.sum()
    chi2 = float(((counts - expected) ** 2 / expected).sum())
    assert stats.chi2.sf(chi2, 49) > 1e-4, chi2


def test_transport_energy_conservation(oracle_lib):
    for sc, src in [(synth.scenes.tiny_scene(), synth.scenes.tiny_source()),
                    (synth.scenes.calorimeter_scene(), synth.scenes.calorimeter_source())]:
        g = oracle.Geometry(sc)
        r = g.transport(src, 3, 2000 if sc.name == "tiny" else 300)
        tally = r["tally"]
        nv = sc.n_volumes
        dep = tally[:, :nv].sum() + tally[:, nv].sum()
        assert abs(dep - tally[:, nv + 1].sum()) < 1e-10 * tally[:, nv + 1].sum()
        c = dict(zip(oracle.COUNTER_NAMES, r["counters"].tolist()))
        assert c["tracks"] == c["photo"] + c["escaped"] + c["cutoff"] + c["step_limit"]
        assert c["steps"] == c["geom_steps"] + c["phys_steps"]
        assert c["phys_steps"] == c["photo"] + c["compton"]


def test_transport_replay_and_threads(oracle_lib):
    """Histories are keyed by track id: subsets and thread counts do not change them."""
    sc = synth.scenes.tiny_scene()
    g = oracle.Geometry(sc)
    src = synth.scenes.tiny_source()
    a = g.transport(src, 77, 1000, threads=1)
    b = g.transport(src, 77, 200, tid0=300, threads=4)
    assert np.array_equal(a["hashes"][300:500], b["hashes"]) and np.array_equal(a["lengths"][300:500], b["lengths"])
    c = g.transport(src, 77, 1000, threads=3)
    assert np.array_equal(a["hashes"], c["hashes"]) and np.array_equal(a["counters"], c["counters"])
    assert np.allclose(a["tally"], c["tally"], rtol=1e-12, atol=1e-12)
    d = g.transport(src, 78, 1000, threads=1)
    assert not np.array_equal(a["hashes"], d["hashes"])


def test_uncollided_fraction_compton_slab(oracle_lib):
    """Eqs. 2-3 with the toy Compton+photo table: the fraction of tracks whose first event is
    leaving the slab equals exp(-mu_tot(E) x) at fixed energy."""
    m = toy_materials()["al"]
    x = 40.0
    sc = synth.scenes.slab_scene(x, m)
    g = oracle.Geometry(sc)
    src = Source(pos=(0.0, 0.0, -1.0), isotropic=False, direction=(0.0, 0.0, 1.0), e_kind="mono", e0=1.0, e1=1.0)
    n = 100000
    r = g.transport(src, 9, n, want_len=True)
    # an uncollided history is a straight line from z=-1 through the slab to the world boundary
    world_hz = sc.solids[0].params[2]
    straight = np.isclose(r["lengths"], world_hz + 1.0, rtol=0, atol=1e-9)
    mu, _ = g.mu(1, 1.0)
    p = math.exp(-mu * x)
    assert abs(straight.mean() - p) < 3.5 * math.sqrt(p * (1 - p) / n)
