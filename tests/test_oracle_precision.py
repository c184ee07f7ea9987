"""Pins of the BF16 rounding emulation (``oracle.precision``): the rounding itself against
PyTorch's float32 -> bfloat16 conversion (round to nearest even), the dense operator pair
without rounding against the oracle's double sums, and the emulated error against the
first-order expectation from the rounding errors of its two factors."""

import numpy as np

from paper_2211_07532_gb300 import synth


def test_bf16_round_matches_library_conversion():
    import torch
    from oracle import precision
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000),
                        # exact ties: 8 significant bits plus a half ulp, odd and even last bits
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 3.0 + 2.0 ** -7,
                                  0.0, -0.0, 1e-40, 3.4e38])]).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    got = precision.bf16_round(v)
    assert np.array_equal(got, ref)
    assert precision.bf16_round(np.float32(1.0 + 2.0 ** -8))[()] == 1.0          # tie -> even
    assert precision.bf16_round(np.float32(1.0 + 3 * 2.0 ** -8))[()] == 1.0 + 2.0 ** -6


def test_dense_pair_without_rounding_is_the_oracle_operator(oracle_lib):
    import oracle
    from oracle import precision
    p = synth.make_problem(12, 10, nt=150, nc=3, order=2, dwell=4e-6, turns=2.0, seed=3)
    rng = np.random.default_rng(1)
    x = synth.random_image(rng, 120)
    y = synth.random_kspace(rng, 3, 150)
    fwd, adj = precision.bf16_operators(p, rounding=False)
    a, b = fwd(x), oracle.forward(p, x)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)
    a, b = adj(y), oracle.adjoint(p, y)
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(b)


def test_emulated_error_is_the_sum_of_both_roundings(oracle_lib):
    """E|dy_c(t)|^2 = sum_r |dE(t, r)|^2 |b_c(r)|^2 + |E(t, r)|^2 |db_c(r)|^2 to first order for
    independent zero-mean roundings; over all outputs of a white image the measured error energy
    must match that sum within 10 %.  Dropping either rounding fails (each carries about half)."""
    import oracle
    from oracle import precision
    p = synth.make_problem(24, 20, nt=700, nc=4, order=2, dwell=4e-6, turns=4.0, seed=11)
    rng = np.random.default_rng(2)
    x = synth.random_image(rng, 480).astype(np.complex128)
    fwd, _ = precision.bf16_operators(p)
    err = fwd(x) - oracle.forward(p, x)
    E = precision.encoding_matrix(p)
    dE = precision.bf16_complex(E.astype(np.complex64)) - E
    b = np.asarray(p["S"], np.complex128) * x[None, :]
    db = precision.bf16_complex(b.astype(np.complex64)) - b
    expect = np.sum(np.abs(dE) ** 2 @ (np.abs(b) ** 2).T) + np.sum(np.abs(E) ** 2 @ (np.abs(db) ** 2).T)
    ratio = float(np.sum(np.abs(err) ** 2) / expect)
    rel = float(np.linalg.norm(err) / np.linalg.norm(oracle.forward(p, x)))
    print(f"error energy / first-order expectation {ratio:.3f}; relative error {rel:.2e}")
    assert 0.9 < ratio < 1.1
    assert 1.5e-3 < rel < 3.5e-3          # ~sqrt(2) x 1.6e-3 (two roundings of 8 significant bits)
