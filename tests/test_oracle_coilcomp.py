"""Pins for the oracle's coil compression (Sec. 2.2.1 / 2.2.2; principal components)."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth


@pytest.fixture(scope="module")
def setup(oracle_lib):
    import oracle
    p = synth.make_problem(16, 14, nt=600, nc=6, order=2, dwell=4e-6, turns=3.0, seed=41)
    rng = np.random.default_rng(42)
    y = oracle.forward(p, p["x_gt"]) + 0.1 * synth.random_kspace(rng, 6, 600)
    return p, y


def test_full_compression_is_a_unitary_coil_mixing(setup):
    import oracle
    from oracle import coilcomp
    p, y = setup
    q, yv, e = coilcomp.compress(p, y, p["nc"])
    rng = np.random.default_rng(43)
    x = synth.random_image(rng, 16 * 14)
    assert np.isclose(np.linalg.norm(oracle.forward(q, x)), np.linalg.norm(oracle.forward(p, x)), rtol=1e-12)
    assert np.allclose(oracle.adjoint(q, yv), oracle.adjoint(p, y), rtol=1e-10, atol=1e-10 * np.abs(y).max())


def test_energy_and_ordering(setup):
    from oracle import coilcomp
    p, y = setup
    e, U = coilcomp.compression_matrix(y)
    assert np.all(np.diff(e) <= 1e-9 * e[0])
    assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-12)
    for nv in (1, 3, 6):
        q, yv, _ = coilcomp.compress(p, y, nv)
        assert np.isclose(np.sum(np.abs(yv) ** 2), e[:nv].sum(), rtol=1e-12)
    # against the singular value decomposition of the data (a different factorisation): the
    # eigenvalues are the squared singular values, the columns the left singular vectors up to phase
    W, sv, _ = np.linalg.svd(y, full_matrices=False)
    assert np.allclose(e, sv ** 2, rtol=1e-10)
    assert np.allclose(np.abs(np.sum(W.conj() * U, axis=0)), 1.0, atol=1e-9)
    a = np.argmax(np.abs(U), axis=0)
    lead = U[a, np.arange(U.shape[1])]
    assert np.allclose(lead.imag, 0, atol=1e-14) and np.all(lead.real > 0)


def test_exactly_low_rank_data_loses_nothing(oracle_lib):
    """Data of rank 2 (two independent signal sources mixed into 6 channels): two virtual
    coils keep A^H y exactly."""
    import oracle
    from oracle import coilcomp
    p = synth.make_problem(12, 12, nt=400, nc=6, order=1, dwell=4e-6, turns=3.0, seed=44)
    rng = np.random.default_rng(45)
    M = rng.standard_normal((6, 2)) + 1j * rng.standard_normal((6, 2))
    y = M @ synth.random_kspace(rng, 2, 400)
    q, yv, e = coilcomp.compress(p, y, 2)
    assert e[2] < 1e-9 * e[0]
    assert np.allclose(oracle.adjoint(q, yv), oracle.adjoint(p, y), atol=1e-9 * np.abs(oracle.adjoint(p, y)).max())
