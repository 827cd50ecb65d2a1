"""Bandpass files (salt_band_load): parsing and resampling on the host, checked
against numpy's linear interpolation of the same samples and against closed
forms; no GPU needed."""
import numpy as np
import pytest

from paper_2504_08081_b300 import _abi


@pytest.fixture(scope="module")
def lib():
    from paper_2504_08081_b300 import build
    build.build()
    return _abi.lib()


def _write(path, wave, trans, sep=" ", header=True):
    with open(path, "w") as f:
        if header:
            f.write("# test bandpass\n\n")
        for w, t in zip(wave, trans):
            f.write("%.17g%s%.17g   # sample\n" % (w, sep, t))


def test_resampling_matches_linear_interpolation(lib, tmp_path):
    wave = np.linspace(4001.3, 5998.7, 700)
    trans = np.exp(-0.5 * ((wave - 5000.0) / 300.0) ** 2)
    p = tmp_path / "g.dat"
    _write(p, wave, trans, sep=", ")
    w, t = _abi.load_band(p, step=5.0)
    grid = np.arange(np.ceil(wave[0] / 5.0), np.floor(wave[-1] / 5.0) + 1) * 5.0
    np.testing.assert_array_equal(w, grid)
    np.testing.assert_allclose(t, np.interp(grid, wave, trans), rtol=0, atol=1e-15)


def test_step_zero_keeps_the_samples_and_scale_converts_units(lib, tmp_path):
    wave_nm = np.array([400.0, 450.5, 500.25, 610.0])
    trans = np.array([0.0, 0.5, 1.0, 0.0])
    p = tmp_path / "nm.txt"
    _write(p, wave_nm, trans, sep="\t", header=False)
    w, t = _abi.load_band(p, step=0.0, wave_scale=10.0)
    np.testing.assert_array_equal(w, wave_nm * 10.0)
    np.testing.assert_array_equal(t, trans)


def test_tophat_area_is_exact(lib, tmp_path):
    # a trapezoid-shaped curve with knots on the grid: the resampled trapezoid
    # integral equals the exact area (the curve is piecewise linear)
    wave = np.array([5000.0, 5100.0, 5900.0, 6000.0])
    trans = np.array([0.0, 1.0, 1.0, 0.0])
    p = tmp_path / "th.dat"
    _write(p, wave, trans)
    w, t = _abi.load_band(p, step=5.0)
    area = np.sum(0.5 * (t[1:] + t[:-1]) * np.diff(w))
    assert area == pytest.approx(900.0, abs=1e-9)


@pytest.mark.parametrize("content,why", [
    ("5000 1\n", "one sample"),
    ("5000 1\n4000 1\n", "descending"),
    ("5000 1\nabc 2\n", "garbage"),
    ("5000 1\n5100\n", "missing column"),
    ("5000 1\n-5100 1\n", "negative wavelength"),
    ("5000 nan\n5100 1\n", "non-finite"),
])
def test_malformed_files_are_refused(lib, tmp_path, content, why):
    p = tmp_path / "bad.dat"
    p.write_text(content)
    with pytest.raises(_abi.SaltError):
        _abi.load_band(p, step=5.0)


def test_missing_file_and_capacity(lib, tmp_path):
    import ctypes as C
    with pytest.raises(_abi.SaltError):
        _abi.load_band(tmp_path / "none.dat")
    p = tmp_path / "g.dat"
    _write(p, np.array([5000.0, 5010.0, 5020.0]), np.array([0.1, 0.2, 0.3]))
    n = C.c_int32()
    buf = np.empty(1)
    rc = lib.salt_band_load(None, str(p).encode(), 1.0, 0.0, buf.ctypes.data, buf.ctypes.data, 1, C.byref(n))
    assert rc == _abi.SALT_ERR_INVALID and n.value == 3
