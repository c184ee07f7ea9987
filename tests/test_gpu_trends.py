"""The simulation study of Sec. 2.2.2 on synthetic inputs, reduced grid (R 2 and 6, 8 and 16
virtual coils, SNR 20 and 5): the trends of Figs. 4 and 5 that the paper reports and that
follow from the model, checked on the GPU reconstructions.

* the full model beats the model without 2nd-order terms at the long readout (R = 2);
* CS (undecimated wavelet, lambda = sigma / 2) beats LS (CGLS, 20 iterations) with the full model;
* fewer virtual coils and lower SNR raise the error."""

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def table():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    from paper_2211_07532_gb300 import trends
    ax.lib()
    return trends.run(ax, rs=(2.0, 6.0), coils=(8, 16), snrs=(20.0, 5.0), models=("Expanded", "Partial"),
                      r_for_snr=6.0)


def test_second_order_terms_matter_at_long_readouts(table):
    f4 = table["fig4"]
    print(f4)
    assert f4["Expanded"]["CS"][0] < 0.95 * f4["Partial"]["CS"][0]
    assert f4["Expanded"]["LS"][0] < f4["Partial"]["LS"][0]


def test_cs_beats_ls(table):
    f4 = table["fig4"]["Expanded"]
    assert all(c < l for c, l in zip(f4["CS"], f4["LS"]))


def test_error_grows_with_acceleration_fewer_coils_and_noise(table):
    a, b = table["fig5a"], table["fig5b"]
    print(a, b)
    for m in ("LS", "CS"):
        assert a[16][m][0] < a[16][m][1]            # R 2 < R 6
        assert a[8][m][1] > a[16][m][1]             # 8 coils worse than 16 at R 6
        assert b[16][m][1] > b[16][m][0]            # SNR 5 worse than SNR 20
