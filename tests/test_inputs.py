"""The seeded synthetic input generators: shapes, determinism, statistics."""
import numpy as np

from paper_1803_02481_gb300 import inputs


def test_block_field_layout_and_ragged_last_block():
    rng = np.random.default_rng(1)
    k = inputs.block_field(rng, 4095, 130, 64, -4, 4)
    assert k.shape == (130, 4095)
    # 64 blocks across, the last one 63 cells wide
    assert np.all(k[:64, 4032:] == k[0, 4032]) and k[0, 4031] != k[0, 4032]
    assert np.all(k[:64, :64] == k[0, 0]) and k[64, 0] != k[0, 0]
    assert 1e-4 <= k.min() and k.max() <= 1e4


def test_generators_are_deterministic():
    a = inputs.block_problem(127, seed=1)
    b = inputs.block_problem(127, seed=1)
    assert np.array_equal(a["k"], b["k"]) and np.array_equal(a["b"], b["b"])
    c = inputs.constant_problem(63, seed=0)
    assert np.all(c["k"] == 1.0) and np.abs(c["b"]).max() <= 1.0


def test_gaussian_random_field_statistics():
    rng = np.random.default_rng(2)
    g = inputs.gaussian_random_field(rng, 511, 383, ell=32.0)
    assert g.shape == (383, 511)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    # correlation at lag d ~ exp(-d^2 / (2 ell^2)): smooth at 1 cell, weak at 96
    c1 = np.corrcoef(g[:, :-1].ravel(), g[:, 1:].ravel())[0, 1]
    assert c1 > 0.99
    c96 = np.corrcoef(g[:, :-96].ravel(), g[:, 96:].ravel())[0, 1]
    assert abs(c96) < 0.25


def test_batch_problem_sides():
    probs = inputs.batch_problems(count=64, seed=4)
    sides = {p["n"] for p in probs}
    assert sides <= set(inputs.SIDES_BATCH)
    for p in probs[:5]:
        assert p["k"].shape == (p["n"], p["n"]) and p["b"].shape == (p["n"], p["n"])
        assert 1e-3 <= p["k"].min() and p["k"].max() <= 1e3


def test_adjoint_inputs_draw_order():
    a = inputs.adjoint_problem(63, seed=3)
    assert a["theta"].shape == (63, 63)
    assert np.abs(a["theta_obs"] - a["theta"]).max() > 0
    assert abs(np.std(a["theta"]) - 2.0) < 1e-12
