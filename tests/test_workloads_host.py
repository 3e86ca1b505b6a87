"""Host-side logic of the workloads (CPU only): the sigmoid fit of the
rigidity sweep, whose transition point p* is the sweep's reported number."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def wl():
    from paper_2604_06896_gb300 import workloads
    return workloads


@pytest.mark.parametrize("x0,w", [(3.81, 0.02), (3.95, 0.05), (4.05, 0.1)])
def test_fit_sigmoid_recovers_its_parameters(wl, x0, w):
    x = np.linspace(3.6, 4.2, 13)
    y = 1.0 / (1.0 + np.exp(-(x - x0) / w))
    fx0, fw = wl.fit_sigmoid(x, y)
    assert abs(fx0 - x0) < 1e-6 and abs(fw - w) < 1e-6 * max(1.0, w)


def test_fit_sigmoid_on_noisy_fractions(wl):
    """Fractions of a finite number of tissues (steps of 1/40) still place
    p* within a grid step."""
    x = np.linspace(3.6, 4.2, 13)
    y = np.round(40.0 / (1.0 + np.exp(-(x - 3.98) / 0.04))) / 40.0
    fx0, fw = wl.fit_sigmoid(x, y)
    assert abs(fx0 - 3.98) < 0.05 and 0 < fw < 0.1
