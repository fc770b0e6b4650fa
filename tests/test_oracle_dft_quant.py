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


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("spectrum", ["half", "full"])
@pytest.mark.parametrize("mesh,g", [((8, 12, 8), 4), ((10, 15, 10), 5), ((12, 18, 12), 6)])
def test_quantised_pppm_keeps_the_accuracy(mesh, g, spectrum):
    """The paper's int32 runs on 128 waters: quantising every transform at
    10^7 changes the forces by far less than the discretisation error, and
    nothing saturates."""
    wb, w = make_workload("water128")
    o = OraclePPPM(wb.box, mesh, w["order"], w["beta"])
    ref = o.compute(wb.pos, wb.q)
    r = pppm_quantized(o, wb.pos, wb.q, g, spectrum=spectrum)
    assert not r["saturated"]
    d = _rel(r["forces"], ref["forces"])
    assert d < 1e-5, d
    assert abs(r["energy"] - ref["energy"]) / abs(ref["energy"]) < 1e-6
    assert _rel(r["virial"], ref["virial"]) < 1e-5


@pytest.mark.parametrize("spectrum", ["half", "full"])
@pytest.mark.parametrize("mesh", [(12, 18, 12), (10, 15, 9), (9, 12, 16)])
def test_with_no_axis_quantised_it_is_the_pppm(mesh, spectrum):
    """Exact transforms everywhere: both readings reproduce oracle.pppm, which
    pins the half-spectrum bookkeeping (the Hermitian extension along z, the
    mirrored spectrum for the energy and virial, odd and even meshes)."""
    wb, w = make_workload("water128")
    o = OraclePPPM(wb.box, mesh, w["order"], w["beta"])
    ref = o.compute(wb.pos, wb.q)
    r = pppm_quantized(o, wb.pos, wb.q, 3, axes=(), spectrum=spectrum)
    assert _rel(r["forces"], ref["forces"]) < 1e-13
    assert abs(r["energy"] - ref["energy"]) <= 1e-13 * abs(ref["energy"])
    assert _rel(r["virial"], ref["virial"]) < 1e-13


@pytest.mark.parametrize("mesh,g,axes", [((10, 15, 9), 3, (1, 2)), ((12, 15, 9), 3, (0, 1, 2))])
def test_odd_z_length_keeps_the_accuracy(mesh, g, axes):
    """An odd z length has no Nyquist plane: the half spectrum then holds
    (Nz + 1) / 2 planes, every one but kz = 0 doubled.  At 10^7 the quantised
    PPPM stays within 1e-5 (force) and 1e-6 (energy) of the plain one; at 10^3
    the effect is visible and grows with the number of quantised axes."""
    wb, w = make_workload("water128")
    o = OraclePPPM(wb.box, mesh, w["order"], w["beta"])
    ref = o.compute(wb.pos, wb.q)
    r = pppm_quantized(o, wb.pos, wb.q, g, axes=axes)
    assert not r["saturated"]
    assert _rel(r["forces"], ref["forces"]) < 1e-5
    assert abs(r["energy"] - ref["energy"]) / abs(ref["energy"]) < 1e-6
    coarse = _rel(pppm_quantized(o, wb.pos, wb.q, g, scale=1e3, axes=axes)["forces"], ref["forces"])
    assert 1e-3 < coarse < 0.1


def test_quantised_backward_passes_break_the_mirror_symmetry():
    """Why the real/complex reading matters: a backward pass splits the
    frequency index into nodes, and k -> -k maps that split onto another, so
    the quantised backward DFT of a spectrum with X(-ky, -kz) = conj X(ky, kz)
    no longer has B(y, -kz) = conj B(y, kz); the exact one does."""
    rng = np.random.default_rng(11)
    Ny, Nz = 12, 8
    X = rng.uniform(-1, 1, (Ny, Nz)) + 1j * rng.uniform(-1, 1, (Ny, Nz))
    X = 0.5 * (X + np.conj(np.roll(np.flip(X, axis=(0, 1)), 1, axis=(0, 1))))   # Hermitian in both indices
    def asym(B):
        return np.max(np.abs(np.roll(np.flip(B, axis=1), 1, axis=1) - np.conj(B)))
    exact = np.fft.ifft(X, axis=0) * Ny
    quant, _ = dft_quantized(X, 0, 4, +1, scale=1e4)
    assert asym(exact) < 1e-13
    assert asym(quant) > 0.5e-4


def test_the_two_readings_differ_at_a_coarse_scale():
    """At 10^2 the quantisation error is large and the two readings give
    different forces; at 10^7 both are within the FP32-level bar of the PPPM."""
    wb, w = make_workload("water128")
    o = OraclePPPM(wb.box, (12, 18, 12), w["order"], w["beta"])
    ref = o.compute(wb.pos, wb.q)
    half = pppm_quantized(o, wb.pos, wb.q, 6, scale=1e2)
    full = pppm_quantized(o, wb.pos, wb.q, 6, scale=1e2, spectrum="full")
    effect = _rel(half["forces"], ref["forces"])
    assert effect > 0.05 and _rel(full["forces"], half["forces"]) > 0.2 * effect
    # energy: the forward passes preserve the mirror symmetry (they split the
    # position index), so both readings have the same spectrum up to ties
    assert abs(full["energy"] - half["energy"]) < 0.2 * abs(half["energy"] - ref["energy"])


def test_only_the_chosen_axes_are_quantised():
    """axes=(1,): the y transforms alone are quantised; the error is then
    bounded by that axis' passes alone (smaller than all three)."""
    wb, w = make_workload("water128")
    o = OraclePPPM(wb.box, (12, 18, 12), w["order"], w["beta"])
    ref = o.compute(wb.pos, wb.q)
    y_only = _rel(pppm_quantized(o, wb.pos, wb.q, 9, scale=1e3, axes=(1,))["forces"], ref["forces"])
    all3 = _rel(pppm_quantized(o, wb.pos, wb.q, 6, scale=1e3)["forces"], ref["forces"])
    assert 0 < y_only < all3
    with pytest.raises(ValueError):
        pppm_quantized(o, wb.pos, wb.q, 9)          # 9 does not divide 12
    with pytest.raises(ValueError):
        pppm_quantized(o, wb.pos, wb.q, 6, spectrum="other")
