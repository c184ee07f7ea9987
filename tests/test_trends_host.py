"""Host-side pieces of the simulation study (Sec. 2.2.2): the input recipe and the SNR reading."""

import numpy as np

from paper_2211_07532_gb300 import synth, trends


def test_object_sigma_reading():
    """sigma = mean |x| over the object (|x| > 0.1 max |x|) / SNR."""
    x = np.zeros(100, np.complex64)
    x[:10] = 2.0
    x[10:20] = 1j * 4.0
    x[20:30] = 0.3          # below 0.1 * max = 0.4: background, not counted
    assert np.isclose(trends.object_sigma(x, 10.0), 3.0 / 10.0)


def test_trend_problems_share_the_slice_across_accelerations():
    """One slice, several protocols: phantom, coils and B0 are the same for every R; the
    spiral has N / (2R) turns and the protocol's sample count."""
    a = trends.trend_problem(32, 2.0, nc=4)
    b = trends.trend_problem(32, 6.0, nc=4)
    for key in ("x_gt", "S", "omega", "h"):
        assert np.array_equal(a[key], b[key]), key
    assert a["nt"] == synth.ragged_protocol_nt(32, 2.0) and b["nt"] == synth.ragged_protocol_nt(32, 6.0)
    assert a["nl"] == 9 and a["nc"] == 4
    assert not np.array_equal(a["k"][:, :100], b["k"][:, :100])


def test_eddy_scale_scales_only_the_eddy_terms():
    p0 = synth.make_problem(16, nt=300, nc=2, order=2, eddy=False, seed=9)
    p1 = synth.make_problem(16, nt=300, nc=2, order=2, eddy_scale=1.0, seed=9)
    p2 = synth.make_problem(16, nt=300, nc=2, order=2, eddy_scale=0.1, seed=9)
    d1 = p1["k"].astype(np.float64) - p0["k"]
    d2 = p2["k"].astype(np.float64) - p0["k"]
    assert np.allclose(d2, 0.1 * d1, rtol=1e-4, atol=1e-3 * np.abs(d1).max())
