"""Pins for the error metrics of tests/metrics.py, on hand-computed cases."""
import numpy as np
import pytest

from tests.metrics import complex_err, paper_style_error, phase_err, power_err


def test_paper_style_error_hand_computed():
    """Table 1's report on a row whose interior SD is known exactly.

    n = 10: the interior is samples [2, 8).  There the reference's real part
    alternates +1, -1 (mean 0, population SD 1) and its imaginary part +2, -2
    (SD 2).  The test row adds 3e-5 and 2e-6 to two interior real samples
    and 4e-5 to one interior imaginary sample; samples outside the interior
    carry large errors that must not count."""
    ref = np.zeros(10, np.complex128)
    sign = np.array([1, -1, 1, -1, 1, -1], np.float64)
    ref[2:8] = sign + 2j * sign
    ref[0], ref[9] = 50 + 7j, -3 - 9j
    test = ref.copy()
    test[4] += 3e-5
    test[7] += 2e-6
    test[5] += 4e-5j
    test[0] += 1.0 + 1.0j   # outside the interior
    test[9] -= 5.0j
    rep = paper_style_error(test, ref)
    mx, mean, cnt = rep["real"]
    assert cnt == 1
    assert mx == pytest.approx(3e-5, rel=1e-9)
    assert mean == pytest.approx((3e-5 + 2e-6) / 6, rel=1e-9)
    mx, mean, cnt = rep["imag"]
    assert cnt == 1  # 4e-5 / SD 2 = 2e-5 > 1e-5
    assert mx == pytest.approx(2e-5, rel=1e-9)
    assert mean == pytest.approx(2e-5 / 6, rel=1e-9)
    # the threshold is in SD units: at 3e-5 SD the imaginary 2e-5 no longer counts
    assert paper_style_error(test, ref, threshold_sd=3e-5)["imag"][2] == 0


def test_row_errors_hand_computed():
    """Per-row power, complex and magnitude-weighted phase errors."""
    ref = np.array([[3 + 4j, 1 + 0j, 0 + 2j]])          # |c| = 5, 1, 2; P = 25, 1, 4
    got_c = ref + np.array([[0.5, 0, 0]])               # |dc| = 0.5 at the peak
    assert complex_err(got_c, ref)[0] == pytest.approx(0.5 / 5)
    got_p = np.array([[25.0, 1.5, 4.0]])                 # |dP| = 0.5 against max P 25
    assert power_err(got_p, ref)[0] == pytest.approx(0.5 / 25)
    ph = np.angle(ref).copy()
    ph[0, 2] += 0.1                                      # phase off by 0.1 rad where |c| = 2
    expected = abs(np.exp(1j * 0.1) - 1) * 2 / 5
    assert phase_err(ph, ref)[0] == pytest.approx(expected)
    # a phase of +pi and -pi are the same angle
    ref2 = np.array([[-1 + 0j]])
    assert phase_err(np.array([[-np.pi]]), ref2)[0] == pytest.approx(0.0, abs=1e-15)
