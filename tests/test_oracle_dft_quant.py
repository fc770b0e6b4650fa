"""Pins of the int32-quantised DFT oracle (oracle/dft_quant.py) against the
library FFT, the quantisation bound, exact cases and saturation."""
import numpy as np
import pytest

from oracle.dft_quant import INT32_MAX, SCALE, dft_quantized, pppm_quantized, quantize
from oracle.pppm import OraclePPPM
from workloads.water import make_workload


def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


@pytest.mark.parametrize("L,g", [(8, 4), (12, 4), (15, 5), (18, 6), (12, 12)])
@pytest.mark.parametrize("sign", [-1, 1])
def test_within_the_quantisation_bound_of_the_fft(L, g, sign):
    """Each output is off by at most half a quantum per node and per part."""
    x = _rand((5, L, 3), seed=L * g)
    out, sat = dft_quantized(x, axis=1, group=g, sign=sign)
    ref = np.fft.fft(x, axis=1) if sign < 0 else np.fft.ifft(x, axis=1) * L
    bound = (L // g) * 0.5 / SCALE + 1e-13
    assert not sat
    assert np.max(np.abs(out.real - ref.real)) <= bound
    assert np.max(np.abs(out.imag - ref.imag)) <= bound
    # and it is not the plain DFT: the rounding is there
    assert np.max(np.abs(out - ref)) > 0


def test_one_node_at_a_finer_scale_is_the_dft():
    """A single node and a scale of 10^8: the DFT rounded to the 10^-8 grid."""
    x = _rand((7, 10), seed=3) / 10
    out, sat = dft_quantized(x, axis=1, group=10, scale=1e8)
    ref = np.fft.fft(x, axis=1)
    assert not sat
    assert np.max(np.abs(out.real - ref.real)) <= 0.5e-8 + 1e-15
    assert np.max(np.abs(out.imag - ref.imag)) <= 0.5e-8 + 1e-15


def test_exact_when_every_partial_is_on_the_grid():
    """L = 4, one point a node: every partial x_t e^{-2 pi i k t/4} is x_t times
    +-1 or +-i, so inputs that are integers over the scale come out exactly."""
    rng = np.random.default_rng(7)
    xi = rng.integers(-10_000, 10_000, size=(4, 4)) + 1j * rng.integers(-10_000, 10_000, size=(4, 4))
    x = xi / SCALE
    out, _ = dft_quantized(x, axis=0, group=1)
    exact = np.zeros_like(xi, dtype=np.complex128)
    for k in range(4):
        for t in range(4):
            exact[k] += xi[t] * (1j ** (-(k * t) % 4))
    assert np.array_equal(np.rint(out * SCALE), exact)


def test_saturation_is_reported_and_clamped():
    q, sat = quantize(np.array([1e3, -1e3, 0.5]), SCALE)
    assert sat and q[0] == INT32_MAX and q[1] == -INT32_MAX - 1 and q[2] == 5_000_000
    _, sat2 = dft_quantized(np.full(8, 400.0 + 0j), axis=0, group=4)
    assert sat2
    _, sat3 = dft_quantized(np.full(8, 4.0 + 0j), axis=0, group=4)
    assert not sat3


def test_linear_axis_order_and_roundtrip():
    """Forward then inverse (divided by L) returns the input within the bound
    of both passes."""
    x = _rand((12,), seed=9)
    f, _ = dft_quantized(x, 0, 4, -1)
    b, _ = dft_quantized(f, 0, 4, +1)
    assert np.max(np.abs(b / 12 - x)) <= 2 * 3 * 0.5 / SCALE + 1e-12


@pytest.mark.parametrize("mesh,g", [((8, 12, 8), 4), ((10, 15, 10), 5), ((12, 18, 12), 6)])
def test_quantised_pppm_keeps_the_accuracy(mesh, g):
    """The paper's int32 runs on 128 waters: quantising every transform at
    10^7 changes the forces by far less than the discretisation error, and
    nothing saturates."""
    wb, w = make_workload("water128")
    o = OraclePPPM(wb.box, mesh, w["order"], w["beta"])
    ref = o.compute(wb.pos, wb.q)
    r = pppm_quantized(o, wb.pos, wb.q, g)
    assert not r["saturated"]
    d = np.linalg.norm(r["forces"] - ref["forces"]) / np.linalg.norm(ref["forces"])
    assert d < 1e-5, d
    assert abs(r["energy"] - ref["energy"]) / abs(ref["energy"]) < 1e-6
