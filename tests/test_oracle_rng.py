"""Pins for the oracle's counter-based generator, hash and source sampling.

Philox4x32-10 against the published known-answer vectors; FNV-1a against its
reference test vectors; the uniform mapping and the source distributions
against their closed-form laws (KS tests).
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _kat_rows():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expected", _kat_rows())
def test_philox_known_answers(oracle_lib, ctr, key, expected):
    assert oracle.philox4x32_10(ctr, key).tolist() == expected


def test_fnv1a_vectors(oracle_lib):
    with open(os.path.join(GOLDEN, "fnv1a64_vectors.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                s, h = line.rsplit(" ", 1)
                assert oracle.fnv1a(s.strip('"').encode()) == int(h, 16)


def test_uniform_range_and_law(oracle_lib):
    u = np.array([oracle.uniform(12345, tid, 1, d) for tid in range(200) for d in range(100)])
    assert u.min() > 0.0 and u.max() <= 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # distinct counters give distinct words: no repeats in 20000 draws of 53 bits
    assert len(np.unique(u)) == u.size


def test_uniform_is_top_53_bits_plus_one(oracle_lib):
    """A block gives two uniforms: the top 53 bits of (x1:x0) and of (x3:x2), each plus one, times 2^-53."""
    seed, tid, stream, draw = 0x0123456789ABCDEF, (7 << 32) + 5, 1, 3
    x = oracle.philox4x32_10([draw, tid & 0xffffffff, tid >> 32, stream], [seed & 0xffffffff, seed >> 32])
    wa = (int(x[1]) << 32) | int(x[0])
    wb = (int(x[3]) << 32) | int(x[2])
    assert oracle.uniform(seed, tid, stream, draw) == ((wa >> 11) + 1) * 2.0 ** -53
    assert oracle.uniform_pair(seed, tid, stream, draw) == (((wa >> 11) + 1) * 2.0 ** -53, ((wb >> 11) + 1) * 2.0 ** -53)


def test_isotropic_source_law(oracle_lib):
    src = synth.scenes.tiny_source()
    pos, d, E = oracle.source_sample(src, 99, 20000)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
    assert np.all(E == 1.0) and np.all(pos == 0.0)
    assert stats.kstest(d[:, 2], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    phi = np.arctan2(d[:, 1], d[:, 0])
    assert stats.kstest(phi, stats.uniform(-np.pi, 2 * np.pi).cdf).pvalue > 1e-3


def test_beam_spot_and_energy_laws(oracle_lib):
    src = synth.scenes.calorimeter_source()
    pos, d, E = oracle.source_sample(src, 7, 20000)
    assert np.all(d == np.array([0.0, 0.0, 1.0])) and np.all(pos[:, 2] == -10.0)
    assert stats.kstest(pos[:, 0] / 10.0, "norm").pvalue > 1e-3
    assert stats.kstest(pos[:, 1] / 10.0, "norm").pvalue > 1e-3
    assert abs(np.corrcoef(pos[:, 0], pos[:, 1])[0, 1]) < 0.03
    assert stats.kstest(E, stats.uniform(0.1, 9.9).cdf).pvalue > 1e-3


def test_axis_loguniform_source_law(oracle_lib):
    src = synth.scenes.barrel_source()
    pos, d, E = oracle.source_sample(src, 11, 20000)
    assert np.all(pos[:, :2] == 0.0)
    assert stats.kstest(pos[:, 2], stats.uniform(-1500, 3000).cdf).pvalue > 1e-3
    assert stats.kstest(np.log(E), stats.uniform(np.log(0.02), np.log(1000.0)).cdf).pvalue > 1e-3
    assert E.min() >= 0.02 * (1 - 1e-15) and E.max() <= 20.0 * (1 + 1e-15)


def test_subset_replay_of_sources(oracle_lib):
    """Keying by track id: a subset generated alone equals the same ids in a full batch."""
    src = synth.scenes.barrel_source()
    pa, da, ea = oracle.source_sample(src, 5, 1000)
    pb, db, eb = oracle.source_sample(src, 5, 100, tid0=450)
    assert np.array_equal(pa[450:550], pb) and np.array_equal(da[450:550], db) and np.array_equal(ea[450:550], eb)
